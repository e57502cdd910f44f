"""CPU FP64 oracle for the filtered spectral-element lattice Boltzmann method
with flux bounce-back walls (Zhao, Patel, Lin, Min, Lee; arXiv 2509.19171).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
restatement of the paper's method in numpy float64.  It exists to check the
CUDA library.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline / reference arm may import it; the product path never does, and it
shares no code, tables or helpers with ``paper_2509_19171_gb300``.

Layout of the oracle:

* ``lattice``  - discrete velocity sets (Sec. 2.1, Eq. for f^eq)
* ``gll``      - GLL nodes/weights, derivative matrix, modal filter (Sec. 2.2, 2.4)
* ``geometry`` - isoparametric map, metrics, mass, global numbering, wall faces
* ``selbm``    - collision, SSPRK3 streaming with FBB, filter, moments (Sec. 2)
* ``learned``  - per-element modal features and the FP64 reference MLP

Parity status: every function is pinned by a ``-m "not gpu"`` test except
those marked "parity unpinned" in their docstring.
"""
