"""GB300 (sm_103a) library for the primal-dual symmetric-cone MWU framework of
arXiv 2405.09157: SES and hard-margin SVM through one-pass-per-iteration CUDA
kernels behind the C ABI of include/pdscp.h.

Modules: ``api`` (torch-facing binding), ``_ffi`` (ctypes declarations),
``build`` (nvcc build of libpdscp.so), ``datagen`` (seeded synthetic inputs).
"""

__version__ = "0.1.0"
