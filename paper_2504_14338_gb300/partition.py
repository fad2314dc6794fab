"""Host-side partitioning for running the hot path on several ranks (one GPU each).

The paper splits the spatial degrees of freedom into contiguous blocks, one per rank, each
rank holding the rows of every variable over its block (Section 3.2, `distribute_nx`), and
splits the regularisation pairs into contiguous ranges (Section 3.5, `distribute_reg_pairs`);
both give the remainder to the last rank.  The exchange steps are a MAX of the per-variable
scales (Step II), a SUM of the k x k Gram partials (Step III, eq. mos_partitioned) and a MIN
of (training error, candidate index) (Step IV).  On one GPU the same sums are formed with
``dopinf_gram(accumulate=1)`` over row blocks.
"""
import numpy as np


def block_range(count, rank, size):
    """[start, end) of rank's contiguous share of `count` items; the last rank takes the
    remainder of the floor division."""
    if size < 1 or not 0 <= rank < size:
        raise ValueError("bad rank/size")
    base = count // size
    start = rank * base
    end = count if rank == size - 1 else start + base
    return start, end


def rank_rows(n_per_var, n_vars, rank, size):
    """Global row indices (variable-major) held by a rank: its block of every variable."""
    a, b = block_range(n_per_var, rank, size)
    return np.concatenate([np.arange(a, b) + j * n_per_var for j in range(n_vars)])


def local_var_offsets(n_per_var, n_vars, rank, size):
    """Variable row offsets inside a rank's local (stacked) row block."""
    a, b = block_range(n_per_var, rank, size)
    return np.arange(n_vars + 1, dtype=np.int64) * (b - a)


def best_of(train_err, valid, first_index=0):
    """(error, global index) of the best valid local candidate; (inf, -1) if none."""
    best = (float("inf"), -1)
    for i, (e, v) in enumerate(zip(train_err, valid)):
        if v and (e < best[0] or best[1] < 0):
            best = (float(e), first_index + i)
    return best


def merge_best(pairs):
    """Global selection from per-rank (error, index): minimum error, lowest index on ties."""
    best = (float("inf"), -1)
    for e, i in pairs:
        if i < 0:
            continue
        if best[1] < 0 or e < best[0] or (e == best[0] and i < best[1]):
            best = (e, i)
    return best
