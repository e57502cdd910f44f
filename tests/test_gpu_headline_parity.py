"""GPU parity of the headline form -- FP32 deviations with the learned per-element filter
control, population-split step -- against the FP64 oracle's learned step, through the C ABI.

The instantiations checked are the ones the throughput benchmark runs: the learned
prologue at D3Q27 N = 7 on affine hexahedra (features, BF16-weight network, per-element
filter, collision) followed by the assembly + collision of the shared nodes, then the
three split advection stages; and the same prologue on the curved D3Q19 N = 7 pipe.

Tolerance: 1e-6 of max |f| after every step (the FP32-deviation bound of the plain split
path).  The control's decisions are taken in FP32 on the GPU and in FP64 in the oracle:
the features that decide a fallback sit at least 5e-3 (log10 units) away from the range
limit in every step (asserted from the oracle), against an FP32 feature error below 1e-4
for these energies, so both sides take the same decisions.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import learned as Lr
from oracle.selbm import OracleSELBM

pytestmark = pytest.mark.gpu
TOL32 = 1e-6


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_19171_gb300 import build
    build.build()
    import paper_2509_19171_gb300 as pkg
    return pkg


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def smooth_state(o, seed):
    """Continuous state with modal spectra over every shell (smooth field + node noise)."""
    rng = np.random.default_rng(seed)
    X = o.Xg
    k = rng.integers(1, 3, (3, o.dim))
    u = np.stack([0.03 * np.sin(X @ k[c] + c) for c in range(o.dim)], 1) + 1e-4 * rng.standard_normal((o.G, o.dim))
    rho = 1 + 1e-3 * np.cos(X @ k[0]) + 1e-5 * rng.standard_normal(o.G)
    return o.initial_state(rho, u)


def tgv_box():
    return W.box_mesh((2, 2, 2), (0, 0, 0), (2 * math.pi,) * 3, (True, True, True))


def network(nin):
    """Random-initialised network (weights x 1.5, FP32-exact) that gives every element its
    own transfer function."""
    return np.float64(np.float32(Lr.init_params(nin, seed=11) * 1.5))


def oracle_learned_run(o, f, params, lo, hi, nsteps):
    """nsteps learned oracle steps; returns the states after each step and, per step, the
    features, in-range flags and transfer functions of the control."""
    states, feats, inr, sigs = [], [], [], []
    for _ in range(nsteps):
        f0, Fs = o.collide(f)
        f3 = o.stream(f0, Fs)
        sig, x, ok = o.learned_sigma(f3, params, lo, hi)
        o.time += o.dt
        f = o.apply_filter_elements(f3, sig)
        states.append(f)
        feats.append(x)
        inr.append(ok)
        sigs.append(sig)
    return states, feats, inr, sigs


def run_compare(P, o, s, f, params, lo, hi, nsteps, tol):
    s.set_state(np.ascontiguousarray(o.to_local(f)))
    states, feats, inr, sigs = oracle_learned_run(o, f, params, lo, hi, nsteps)
    for k, fo in enumerate(states):
        s.step(1)
        err = rel(s.get_state(), o.to_local(fo))
        assert err <= tol, (k, err)
    return feats, inr, sigs


@pytest.mark.parametrize("seed", [6, 7])
def test_headline_learned_fp32_d3q27_n7(P, seed):
    """D3Q27 N = 7 periodic box, FP32 deviations, learned control in range on every element:
    three steps, each within 1e-6 of the oracle's learned step; the network differentiates
    the elements, and no element falls back."""
    mesh, N = tgv_box(), 7
    filt = {"shape": 0, "gamma": 0.1, "kc": 5.0}
    o = OracleSELBM(mesh, "D3Q27", N, 1e-3, filt=filt)
    s = P.SELBM(mesh, "D3Q27", N, 1e-3, precision=P.FP32DEV, filt=filt)
    assert s.split
    nin = 2 * (N + 1)
    params, lo, hi = network(nin), np.full(nin, -35.0), np.full(nin, 5.0)
    s.set_learned_filter(params, lo, hi, mass_bound=1.0, ke_bound=1.0)
    f = smooth_state(o, seed)
    feats, inr, sigs = run_compare(P, o, s, f, params, lo, hi, 3, TOL32)
    assert all(ok.all() for ok in inr)
    st = s.learned_status()
    assert st["fixed_element_steps"] == 0 and st["fallback_flag"] == 0
    # the transfer functions of the last step match the oracle's and differ between elements
    sig_g = s.element_sigma()
    assert np.abs(sig_g - sigs[-1]).max() < 1e-5
    assert len(np.unique(np.round(sigs[-1][:, -1], 5))) > 1


def test_headline_learned_fp32_subset_out_of_range(P):
    """One feature's training range is cut so that about half of the elements leave it in
    every step: those keep the fixed filter, the rest take the network's.  GPU and oracle
    agree per step within 1e-6, and the library's fallback count equals the oracle's."""
    mesh, N = tgv_box(), 7
    filt = {"shape": 0, "gamma": 0.1, "kc": 5.0}
    o = OracleSELBM(mesh, "D3Q27", N, 1e-3, filt=filt)
    s = P.SELBM(mesh, "D3Q27", N, 1e-3, precision=P.FP32DEV, filt=filt)
    nin = 2 * (N + 1)
    params, lo, hi = network(nin), np.full(nin, -35.0), np.full(nin, 5.0)
    k_cut, limit = N + 1 + 4, -3.184        # |u| shell energy of degree 4
    hi[k_cut] = limit
    s.set_learned_filter(params, lo, hi, mass_bound=1.0, ke_bound=1.0)
    f = smooth_state(o, 6)
    feats, inr, _ = run_compare(P, o, s, f, params, lo, hi, 3, TOL32)
    nfix = []
    for x, ok in zip(feats, inr):
        assert np.abs(x[:, k_cut] - limit).min() > 5e-3          # decisions are not marginal
        assert 0 < (~ok).sum() < o.E                               # a real subset falls back
        nfix.append(int((~ok).sum()))
    # a step's filter runs at the start of the next step (a read-back applies it to the
    # copy it returns without counting): three steps have counted the filters of two
    st = s.learned_status()
    assert st["fixed_element_steps"] == nfix[0] + nfix[1] and st["fallback_flag"] == 0
    assert s.sync() == 0                                 # per-element fallbacks are routine: plain OK


def test_headline_learned_fp32_drift_fallback(P):
    """A negative mass bound trips the drift check at its first comparison: the filters of
    steps 1 and 2 are the network's, from step 3 on the fixed filter is used (FP32 form)."""
    mesh, N = tgv_box(), 7
    filt = {"shape": 0, "gamma": 0.1, "kc": 5.0}
    o = OracleSELBM(mesh, "D3Q27", N, 1e-3, filt=filt)
    s = P.SELBM(mesh, "D3Q27", N, 1e-3, precision=P.FP32DEV, filt=filt)
    nin = 2 * (N + 1)
    params, lo, hi = network(nin), np.full(nin, -35.0), np.full(nin, 5.0)
    s.set_learned_filter(params, lo, hi, mass_bound=-1.0, ke_bound=1.0)
    f = smooth_state(o, 6)
    s.set_state(np.ascontiguousarray(o.to_local(f)))
    f = o.step_learned(f, params, lo, hi)
    f = o.step_learned(f, params, lo, hi)
    f = o.step(o.step(f))
    s.step(4)
    assert s.sync() == P.OK_FALLBACK                    # the synchronising calls report it
    s.diagnostics()
    assert s.fallback_engaged
    assert rel(s.get_state(), o.to_local(f)) <= TOL32
    assert s.learned_status()["fallback_flag"] == 1


def test_headline_learned_fp32_curved_pipe_d3q19_n7(P):
    """Curved D3Q19 N = 7 pipe elements (per-node metrics and masses in the learned
    prologue), flux bounce-back walls and body force, FP32 deviations with the learned
    control: three steps within 1e-6 of the oracle."""
    N = 7
    mesh = W.pipe_mesh(n_core=2, n_radial=2, n_axial=1, length=1.0)
    filt = {"shape": 0, "gamma": 0.1, "kc": 5.0}
    g = (0.0, 0.0, 2e-4)
    o = OracleSELBM(mesh, "D3Q19", N, 2e-3, filt=filt, body_accel=g)
    s = P.SELBM(mesh, "D3Q19", N, 2e-3, precision=P.FP32DEV, filt=filt, body_accel=g)
    assert s.split
    nin = 2 * (N + 1)
    params, lo, hi = network(nin), np.full(nin, -35.0), np.full(nin, 5.0)
    s.set_learned_filter(params, lo, hi, mass_bound=1.0, ke_bound=1.0)
    f = smooth_state(o, 9)
    feats, inr, _ = run_compare(P, o, s, f, params, lo, hi, 3, TOL32)
    assert all(ok.all() for ok in inr)
    assert s.learned_status()["fixed_element_steps"] == 0


def test_learned_fp64_split_d3q27_n7(P, monkeypatch):
    """The same learned prologue in FP64 (population-split form forced on), D3Q27 N = 7:
    three steps within 1e-10 of the oracle (the learned-step bound of the FP64 form)."""
    monkeypatch.setenv("SELBM_SPLIT", "1")
    mesh, N = tgv_box(), 7
    filt = {"shape": 0, "gamma": 0.1, "kc": 5.0}
    o = OracleSELBM(mesh, "D3Q27", N, 1e-3, filt=filt)
    s = P.SELBM(mesh, "D3Q27", N, 1e-3, filt=filt)
    assert s.split
    nin = 2 * (N + 1)
    params, lo, hi = network(nin), np.full(nin, -35.0), np.full(nin, 5.0)
    s.set_learned_filter(params, lo, hi, mass_bound=1.0, ke_bound=1.0)
    f = smooth_state(o, 6)
    run_compare(P, o, s, f, params, lo, hi, 3, 1e-10)
    assert s.learned_status()["fixed_element_steps"] == 0
