"""GB300-native aura exchange of the TeraAgent distributed engine (arXiv 2509.24063).

Python binding over ``libtera.so`` (see ``include/tera.h``).  PyTorch supplies
device memory and streams only; every step runs in the library's CUDA kernels.
There is no CPU path: every entry point raises when the library or a CUDA
device is missing.
"""
from ._lib import (EBOUNDS, ECAPACITY, ECORRUPT, EDOMAIN, EINVAL, ENOMEM, EREFMISMATCH, ETIMEOUT, ECUDA,
                   MODE_RAW, MODE_XOR, OK, TeraError)
from .api import Context, PartitionBuffers, soa_from_state
from .exchange import AuraExchange
from .migrate import Migration

__all__ = ["Context", "PartitionBuffers", "AuraExchange", "Migration", "soa_from_state",
           "TeraError", "OK",
           "EINVAL", "ENOMEM", "ECAPACITY", "ECORRUPT", "EDOMAIN", "EREFMISMATCH", "ETIMEOUT",
           "ECUDA", "EBOUNDS", "MODE_RAW", "MODE_XOR"]
