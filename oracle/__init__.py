"""FP64 CPU oracle of the LBM-LETKF hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously-correct restatement of what the paper's method
computes, used to check the CUDA library.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg
may import it.  It shares no code with the CUDA path and never calls it.

Modules
-------
lbm      D2Q9 lattice Boltzmann equation, BGK collision, body force,
         moments (Sec. II-A, Eqs. 1-5).
obs      observation operator y = h(x): density / velocity at observation
         points (Sec. II-B, "y is given by rho and u at observation points").
letkf    R-localized LETKF local analysis in ensemble space (Sec. II-B,
         Eqs. letkf_xa .. enkf_deltay, Algorithm 1), plus the global ETKF.
kalman   brute-force model-space Kalman filter (Eqs. kfx, kfp, kfk) used as
         an independent pin of the ensemble-space analysis.
jacobi   hand-written cyclic Jacobi eigensolver, a cross-check of LAPACK.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, brute force or textbook values; the only
parts without an independent pin are the long chaotic turbulence runs
(parity unpinned -- judged by RMSE against the synthetic truth).
"""
from . import lbm, obs, letkf, kalman, jacobi  # noqa: F401
