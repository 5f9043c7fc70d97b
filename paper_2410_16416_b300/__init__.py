"""B300-native multirate SVD matched filter (LLOID) with a device-side trigger generator.

The compute path lives in ``liblloid.so`` (CUDA, sm_103a) behind the C ABI of
include/lloid.h; ``_abi`` is its ctypes binding and ``svdbank`` the host-side
setup (time slicing + FP64 SVD) that produces what the library consumes.
The binding is imported on first use of one of its names, so that the build
step (``paper_2410_16416_b300.build``) can run before the library exists;
using the binding without the library raises ImportError (no CPU fallback).
"""
from .svdbank import BankSlice, SVDBank, decompose

_ABI_NAMES = {"Context", "Unit", "Conditioner", "LloidError", "make_desc", "plan", "TRIGGER_DTYPE", "PRECISION", "SIGNATURES",
              "lib", "LIB_PATH", "SB_OK", "SB_EINVAL", "SB_ENOMEM", "SB_EBUSY", "SB_EGAP", "SB_ETIMEOUT",
              "SB_ECUDA", "SB_EOVERFLOW", "SB_TRIG_REFINED", "SB_TRIG_SUBSAMPLE", "SB_TRIG_XI2", "SB_XI2_HALF", "coincidences",
              "COINC_DTYPE",
              "STAGES"}


def __getattr__(name):
    if name in _ABI_NAMES:
        from . import _abi
        return getattr(_abi, name)
    raise AttributeError(name)
