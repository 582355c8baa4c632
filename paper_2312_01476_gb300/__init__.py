"""GB300 (sm_103a) tensor-join hot path of the context-enhanced E-join.

The operator R join_{E,mu,theta} S (Sec. III-C) over given embeddings:
row normalisation with selection pushdown, a blocked cosine-similarity
contraction (tcgen05/TMEM/TMA, or FP32 CUDA cores) fused with the threshold
predicate and pair compaction, and an exact re-score of the guard band.
The C ABI is declared in include/ejoin.h; ``ejoin`` is its Python binding.
"""
from .ejoin import (  # noqa: F401
    EJOIN_BF16, EJOIN_F32, EJOIN_FP8_E4M3, EJOIN_TF32, EJOIN_FLAG_COUNT_ONLY, EJOIN_FLAG_TIMING, EJOIN_FLAG_FUSED,
    EJOIN_FLAG_NO_SYMMETRY, EJOIN_FLAG_HOST_COPY, EJOIN_FLAG_GATHER_RESCORE, EJOIN_FLAG_SORT, EJOIN_FLAG_PANEL_RESCORE, PAIR_DTYPE,
    Ctx, EJoinError, Result, Sel, ejoin_create, ejoin_destroy, ejoin_last_stats, ejoin_normalize, ejoin_set_timeout,
    ejoin_padded_dim, ejoin_strerror, ejoin_threshold, ejoin_threshold_host, ejoin_top1, ejoin_topk, ejoin_eselect, ejoin_version, load_library,
    Batch, ejoin_batch,
)
