"""GB300 (sm_103a) leapfrog of the spline geometric method for Maxwell's equations (arXiv 2302.04979, scheme 2).

``smx``     thin binding of the C ABI (include/smx.h) implemented in csrc/ (CUDA kernels + host setup)
``adjoint`` receiver-misfit gradients through the leapfrog (torch.autograd, sqrt(N) checkpoints)
``synth``   seeded synthetic inputs
``build``   compiles csrc/ into _build/libsmx.so
"""
