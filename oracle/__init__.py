"""Plain FP64 CPU oracle for the CN-WSGD per-time-step solve of
Moghaderi, Dehghan, Donatelli, Mazza, "Spectral analysis and multigrid
preconditioners for two-dimensional space-fractional diffusion equations"
(arXiv:1706.06844).

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  The product path (the
CUDA library under ``paper_1706_06844_gb300``) never calls it, and the two share
no code: no kernels, helpers, tables or constant generators.  Inputs (coefficient
fields, manufactured sources) come from ``paper_1706_06844_gb300.inputs``, which
holds no arithmetic of the method.

Everything is written in float64 with numpy/scipy library primitives (matmul,
FFT, dense LU, sparse products) used only as whole steps, following the paper's
definitions in the paper's order:

* ``wsgd``      -- Grunwald coefficients g_k (Eq. gk) and WSGD weights w_k (Eq. w)
* ``operator``  -- Toeplitz A (Eq. AN), Kronecker operators (Eq. AxAy), M and b (Eq. M)
* ``multigrid`` -- bilinear P (Sec. 4.1), damped Jacobi (Eq. Sn), TGM / V-cycle
                   (Sec. 4, 4.2), structured and exact Galerkin, rediscretised
                   coarse operators, the band preconditioner P2 (Sec. 4.3)
* ``krylov``    -- restarted GMRES / right-preconditioned flexible GMRES (Sec. 5)
* ``timeloop``  -- the CN-WSGD time loop (Eq. CNWSGD, Eq. 2) and the examples of Sec. 5

Functions whose results no independent pin fixes say "parity unpinned" in
their docstring; every other function is pinned by ``tests/test_oracle_*.py``.
"""
