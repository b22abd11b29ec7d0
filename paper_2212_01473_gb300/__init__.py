"""GB300-native exact maximal clique enumeration (arXiv 2212.01473's method).

The compute path is the CUDA library libmce.so (C ABI in include/mce.h);
this package is its Python binding. Importing the package does not load the
library; the first call does, and raises if it has not been built.
"""
from .engine import (mce_predict_priority, mce_autotune, mce_prepare, mce_run_prepared, MCE_EINVAL, MCE_ENOMEM, MCE_ECUDA, MCE_ERANGE, MCE_ETIMEOUT, MCE_EUNSUPPORTED, MCE_EBUDGET,
                     MCE_FLAG_DEVICE_PTRS, MCE_OK, MCE_ORDER_PLAIN, MCE_ORDER_PRIORITY, MCE_PIVOT_AUTO,
                     MCE_PIVOT_IP, MCE_PIVOT_IPX, MCEError, Result, enumerate_maximal_cliques, library,
                     mce_batch_create, mce_create, mce_default_opts, mce_destroy, mce_get_order,
                     mce_get_stats, mce_graph_info, mce_peel_noalloc, mce_selftest_waits, mce_microbench, mce_root_features, mce_run, mce_run_batch,
                     mce_run_list, decode_clique_records, list_maximal_cliques,
                     Model, MCE_MODEL_PARAMS, MCE_NUM_FEATURES)

__all__ = [name for name in dir() if name.startswith(("mce_", "MCE"))] + [
    "Model", "Result", "enumerate_maximal_cliques", "library", "decode_clique_records", "list_maximal_cliques"]
