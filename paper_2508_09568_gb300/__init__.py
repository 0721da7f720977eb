"""GB300-native (sm_103a) MHD bunch update: a C-ABI CUDA library plus a thin Python binding.

Submodules:
  workloads  seeded synthetic inputs (patch geometry, initial states); no method arithmetic
  build      in-tree nvcc build of libmhdbunch.so
  capi       ctypes binding of include/mhd_bunch.h (same names)
  bunch      MHDBunch: device-resident bunch handle (torch memory and stream)
  autograd   MHDStep: torch.autograd.Function over the step and its hand-written adjoint

Importing the package does not load the CUDA library; the first MHDBunch does, and it
fails loudly when the library or a GPU is missing.
"""
