"""GB300-native Kerdock fast sparsifying transform (arXiv 2105.05879).

The compute path is the C-ABI library ``libkerdock.so`` (CUDA for sm_103a, see
``include/kerdock.h``); ``kerdock`` is its Python binding.
"""
from .kerdock import (  # noqa: F401
    KERDOCK_BF16, KERDOCK_F32, KERDOCK_FLAG_FULL_OUTPUT, KerdockBatch, KerdockError, KerdockMLP,
    KerdockPlan,
    load_library, results_to_lists,
)
