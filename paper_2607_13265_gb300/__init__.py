"""GB300-native differentiable polarized path tracing (cached suffix replay).

Submodules:
  scenegen -- seeded synthetic scenes and jobs (input data only)
  build    -- nvcc build of the CUDA library (libdppt.so, sm_103a)
  api      -- ctypes binding of include/dppt.h, render_primal / render_adjoint,
              and the torch.autograd.Function PolarizedRender
Importing the package loads nothing; the CUDA library is loaded by ``api``.
"""
