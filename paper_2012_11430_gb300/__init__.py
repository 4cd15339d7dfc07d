"""GB300 (sm_103a) implementation of the data-parallel hot path of the multivariate
matrix-pencil Prony method (Bosner, arXiv 2012.11430).

The computation lives in the CUDA library libprony.so (C ABI, include/prony.h);
`binding` marshals numpy arrays / torch tensors to it, `refine` wraps the
exponential-sum kernels in a torch.autograd.Function for least-squares refinement.
"""
from .binding import (Context, PronyError, PronyInfo, PronyOpts, default_opts, load,  # noqa: F401
                      PRONY_OK, PRONY_EINVAL, PRONY_ERANK, PRONY_ENOCONV, PRONY_ENAN, PRONY_ECUDA, PRONY_ENOMEM,
                      PRONY_FP32, PRONY_BF16X3, PRONY_TF32X3, PRONY_BF16X2, PRONY_FFT32, PRECISIONS)
