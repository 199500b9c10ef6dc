"""FP64 CPU oracle for the CISOR hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously correct restatement of what the CUDA path computes,
written from the paper (Ma, Mansour, Liu, Boufounos, Kamilov, "Accelerated
Image Reconstruction for Nonlinear Diffractive Imaging", arXiv:1708.01663).
numpy/scipy in float64/complex128, one transmitter at a time, no blocking or
fusion.  Library primitives used as single steps: numpy FFT, dense LU solve,
scipy Bessel/Hankel functions.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA path (``paper_1708_01663_gb300``); the only common
module is ``paper_1708_01663_gb300.synth`` (seeded inputs, no method
arithmetic).

Modules
  model   grid, Green's function (Eq. 1), G / H / A / A^H (Eqs. 2-4), FFT convolution
  solve   BiCGSTAB / GMRES / dense LU for A u = u_in and A^H v = b (Eq. 13)
  grad    data term D (Eq. 7) and its adjoint-state gradient (Prop. 1, Eq. 12)
  prox    constrained isotropic TV prox by FGP (Eq. 8, Sec. III-A)
  fista   relaxed FISTA (Eqs. 9-11), step-size estimate
  mie     analytic Mie series for a dielectric cylinder (2D) -- pins the discretisation

Parity status of each function is stated in its module docstring.
"""
