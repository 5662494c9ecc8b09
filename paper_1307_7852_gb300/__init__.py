"""GB300-native k-NN graph construction (Wang et al., arXiv:1307.7852).

The computation lives in the CUDA library ``libknng.so`` (sources in
``csrc/``, C ABI in ``include/knng.h``); ``binding`` marshals tensors to it.
``synthetic`` generates seeded inputs shaped like the paper's workloads.
The library is loaded on first use, not at import.
"""
from .binding import (  # noqa: F401
    DTYPE_F16, DTYPE_F32, DTYPE_U8, METRIC_COSINE, METRIC_L2, PROP_BEST_FIRST, PROP_FIRST_ORDER, PROP_PAIRWISE,
    PART_FEATURES, PART_FEATURES_PCA, PART_PCA, PART_RANDOM, PREC_BF16, PREC_FP8E4M3, PREC_FP32, Handle,
    KnngError, Mlp, handle, knng_autotune, knng_build, knng_build_batched, knng_build_host, knng_build_learned, knng_divisions_used,
    knng_exact_knn, knng_launch_counter, knng_leaf_count, knng_leaf_knn, knng_leaf_offsets, knng_merge,
    knng_mlp_forward, knng_normalize_rows, knng_partition, knng_partition_learned, knng_partition_pca, knng_split_levels, knng_propagate, knng_propagate_best_first, knng_propagate_noalloc,
    knng_propagate_pairwise,
    knng_set_propagation_counters, knng_set_stage_events, knng_set_wait_limit, knng_sync, knng_tune_load, knng_tune_save, lib)
