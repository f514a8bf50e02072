"""GB300 (sm_103a) pose-differentiable Gaussian-splatting renderer.

Hot path of "Look Gauss, No Pose" (arXiv 2410.08743): tile-based 3D Gaussian
splatting forward and backward with the analytic se(3) camera-pose gradient,
as hand-written CUDA kernels behind the C ABI in include/gsplat.h.

Submodules (imported lazily so that `synth` needs no GPU library):
  _lib     ctypes binding of libgsplat (same names as the C entry points)
  render   Renderer object and the torch.autograd.Function
  synth    seeded synthetic scenes, cameras and requests
  build    nvcc build of libgsplat.so
"""

__all__ = ["build", "synth", "render", "_lib"]
