"""FP64 CPU oracle for IRCUR (test infrastructure; see ircur_oracle)."""

from .ircur_oracle import (  # noqa: F401
    IrcurResult,
    cur_product,
    cur_to_svd,
    dense_outputs,
    entries,
    hard_threshold,
    ircur,
    numerical_rank,
    pinv_from_svd,
    sample_indices,
    sample_size,
    splitmix64,
    stream_columns,
    truncated_svd,
)
