"""GB300 (sm_103a) ideal-MHD + glm block update of the MPI-AMRVAC 3.0 method.

``amrvac``     ctypes binding of the C ABI in include/amrvac.h (CUDA library)
``workloads``  seeded synthetic inputs (block lists and initial states)
``build``      in-tree nvcc build of the CUDA library
"""
