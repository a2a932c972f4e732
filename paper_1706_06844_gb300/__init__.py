"""GB300 (sm_103a) solver for the per-time-step CN-WSGD system of the 2-D
two-sided space-fractional diffusion equation (arXiv:1706.06844): restarted
flexible GMRES preconditioned by a multigrid V-cycle, behind the C ABI of
``include/fde.h`` (``libfde.so``).

``paper_1706_06844_gb300.fde`` is the ctypes binding (same names as the C
functions); ``paper_1706_06844_gb300.inputs`` generates seeded synthetic inputs.
Importing the package does not load the CUDA library; ``fde.lib()`` does and
raises if it is missing.
"""
