"""GB300-native differentiable freeform-lens ray tracer.

Forward: rays from a collimated beam, a point source or a grid of point
sources are traced through a lens with a bicubic B-spline freeform exit face
(and a flat or freeform entry face), and deposited with a smooth reconstruction
filter into an irradiance grid. Adjoint: the gradient of an irradiance loss is
carried back to the control-point heights. Both run as hand-written CUDA kernels
for sm_103a behind the C ABI declared in include/freeray.h; this package is the
thin Python binding over it (ctypes marshalling, torch tensors for device memory
and streams), the autograd functions, the graph-captured optimisation step and
the schedule autotuner.
"""
