"""Host-side pieces of the study drivers that need no GPU: the series solution the Couette
convergence study measures against (Sec. 3.2) and the wall law of the pipe start (Sec. 4)."""
import math

import numpy as np

from paper_2509_19171_gb300.couette_convergence import series


def test_couette_series_solves_the_diffusion_problem():
    U, nu = 0.03, 1e-3
    y = np.linspace(0.05, 0.95, 19)
    t, h, k = 20.0, 1e-3, 1e-2
    # boundary values, the steady limit and the start from rest
    assert np.allclose(series(np.array([0.0, 1.0]), t, U, nu), [0.0, U], atol=1e-15)
    assert np.allclose(series(y, 1e7, U, nu), U * y, atol=1e-15)
    assert np.abs(series(y, 1e-3, U, nu)).max() < 0.02 * U
    # u_t = nu u_yy by central differences
    ut = (series(y, t + k, U, nu) - series(y, t - k, U, nu)) / (2 * k)
    uyy = (series(y + h, t, U, nu) - 2 * series(y, t, U, nu) + series(y - h, t, U, nu)) / h ** 2
    assert np.abs(ut - nu * uyy).max() < 1e-6 * U
