"""GB300-native 3DGUT hot path: UT projection, tile binning / radix sort and 3D-response
compositing (forward and backward) as sm_103a CUDA kernels behind the C ABI of
include/ut3d.h.

Submodules (imported lazily so that the input generators load without CUDA):
  abi     ctypes binding of libut3d.so (marshalling only)
  render  PyTorch wrapper: device buffers, streams, torch.autograd.Function
  synth   seeded synthetic inputs (scenes, cameras, options)
  build   compiles libut3d.so in-tree for sm_103a
"""
