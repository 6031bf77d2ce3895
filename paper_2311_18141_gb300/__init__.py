"""GB300-native CSR sparse-times-dense product (SpMM) library.

The compute path is the sm_103a CUDA library ``_lib/libspmm_gb300.so`` behind
the C ABI in ``include/spmm_gb300.h``; ``binding`` wraps it with ctypes and
``autograd`` adds a torch.autograd.Function.  ``inputs`` draws the seeded
synthetic workloads.  Submodules load lazily so that the input generators can
be used without a GPU.
"""

__all__ = ["binding", "inputs", "build"]
