"""Oracle for the host-side blocking: diagonal block pointer, percentage
sampling, the structure-aware irregular blocking, regular blocking, and the
block task plan (levels of the block dependency structure).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Written independently
of the product's host code so that the two can be compared bit for bit.
"""
from __future__ import annotations

import numpy as np


def blockptr(n, colptr, rowidx):
    """Diagonal block pointer (Section 4.2, Algorithm 2), by its definition:
    blockptr[k] = number of stored entries (r, c) with r < k and c < k, i.e.
    the nonzeros of the leading k x k submatrix.  An entry (r, c) lies in
    every leading submatrix of order k > max(r, c).

    For a structurally symmetric pattern with a full diagonal this equals
    what Algorithm 2 computes from the strictly-lower counts per row.
    """
    cols = np.repeat(np.arange(n, dtype=np.int64), np.diff(colptr))
    m = np.maximum(cols, rowidx.astype(np.int64))
    h = np.bincount(m + 1, minlength=n + 1)[: n + 1]
    return np.cumsum(h).astype(np.int64)


def num_samples(N, sample_points=1000, b_min=32):
    """S = min(sample_points, floor(N / b_min)), at least 1.  The paper uses
    1000 samples (Section 4.1) on matrices with N >= 1.3e5; the cap keeps a
    basic block at least b_min rows on small matrices."""
    return max(1, min(int(sample_points), int(N) // max(1, int(b_min))))


def sample_rows(N, S):
    """Sample s (s = 0..S) sits at row idx(s) = floor(s N / S)."""
    s = np.arange(S + 1, dtype=np.int64)
    return (s * int(N)) // int(S)


def irregular_ptr(bp, N, sample_points=1000, step=2, max_num=3, stride=1,
                  b_min=32):
    """Structure-aware irregular blocking (Section 4.3, Algorithm 3).

    pct(s) = bp[idx(s)] / bp[N].  Walking the windows i = 0, stride, ...
    while i + step <= S:
      * if pct(i+step) - pct(i) >= step / S (the slope of a linear profile),
        the window is dense: mark a boundary at idx(i + step), reset l;
      * else if l >= max_num: mark a boundary at idx(i + step) anyway, reset
        l (bounds the size of blocks in sparse regions);
      * else skip: l += 1.
    The comparison is made exactly in integers:
    (bp[idx(i+step)] - bp[idx(i)]) * S >= step * bp[N].
    Boundaries start with 0; N is appended if the walk ends short of it, and
    repeated boundaries are dropped.
    """
    N = int(N)
    bp = np.asarray(bp, dtype=np.int64)
    S = num_samples(N, sample_points, b_min)
    idx = sample_rows(N, S)
    num = bp[idx]
    total = int(bp[N])
    ptr = [0]
    k = 0
    l = 0
    i = 0
    while i + step <= S:
        dense = (int(num[i + step]) - int(num[i])) * S >= step * total
        if dense:
            ptr.append(int(idx[i + step])); k += 1; l = 0
        elif l >= max_num:
            ptr.append(int(idx[i + step])); k += 1; l = 0
        else:
            l += 1
        i += stride
    if ptr[-1] < N:
        ptr.append(N)
    out = [ptr[0]]
    for p in ptr[1:]:
        if p > out[-1]:
            out.append(p)
    return np.asarray(out, dtype=np.int64)


def regular_ptr(N, b):
    """Regular 2-D blocking with fixed block size b (the last block takes
    the remainder)."""
    p = list(range(0, int(N), int(b))) + [int(N)]
    return np.asarray(sorted(set(p)), dtype=np.int64)


def block_plan(n, pcolptr, prowidx, ptr, dense_threshold=1.0):
    """Block structure and task lists of the right-looking blocked LU
    (Section 2.2, Algorithm 1) over blocks given by ``ptr``, restricted to
    non-empty blocks.

    ``pcolptr, prowidx`` is the filled, structurally symmetric L+U pattern.
    Returns a dict:
      blocks   int64[nb, 2] (I, J) of non-empty blocks, sorted by (J, I)
      bnnz     int64[nb] entries per block
      dense    bool[nb] nnz >= dense_threshold * bI * bJ (IEEE double)
      level    int64[p] level of each diagonal block: 0 if block row I has
               no non-empty block left of the diagonal, else
               1 + max level(I') over non-empty (I, I'), I' < I (the longest
               chain of the task graph in which Algorithm 1's step I' must
               finish before step I whenever block (I, I') is non-empty)
      getrf    per level: diagonal blocks I
      gessm    per level: (I, J), J > I, non-empty, level(I) = that level
      tstrf    per level: (J, I), J > I, non-empty, level(I) = that level
      ssssm    per level: list of ((K, J), [I, ...]) for targets K, J > I
               with (K, I), (I, J), (K, J) all non-empty, sources ascending
    """
    ptr = np.asarray(ptr, dtype=np.int64)
    p = ptr.size - 1
    cols = np.repeat(np.arange(n, dtype=np.int64), np.diff(pcolptr))
    rows = prowidx.astype(np.int64)
    bi = np.searchsorted(ptr, rows, side="right") - 1
    bj = np.searchsorted(ptr, cols, side="right") - 1
    key = bj * p + bi
    uk, cnt = np.unique(key, return_counts=True)
    BJ = uk // p
    BI = uk % p
    sizes = np.diff(ptr)
    dense = cnt.astype(np.float64) >= dense_threshold * (
        sizes[BI].astype(np.float64) * sizes[BJ].astype(np.float64))
    nonempty = set(zip(BI.tolist(), BJ.tolist()))
    lower = {}
    upper = {}
    for I, J in nonempty:
        if I > J:
            lower.setdefault(I, []).append(J)     # (I, J) below diagonal
        elif I < J:
            upper.setdefault(I, []).append(J)     # (I, J) above diagonal
    level = np.zeros(p, dtype=np.int64)
    for I in range(p):
        preds = lower.get(I, [])
        level[I] = 1 + max(level[J] for J in preds) if preds else 0
    nlev = int(level.max()) + 1 if p else 0
    getrf = [[] for _ in range(nlev)]
    gessm = [[] for _ in range(nlev)]
    tstrf = [[] for _ in range(nlev)]
    ssssm = [dict() for _ in range(nlev)]
    colblocks = {}                       # I -> rows K > I with (K, I) non-empty
    for I, J in nonempty:
        if I > J:
            colblocks.setdefault(J, []).append(I)
    for I in range(p):
        lv = int(level[I])
        getrf[lv].append(I)
        Us = sorted(upper.get(I, []))
        Ls = sorted(colblocks.get(I, []))
        for J in Us:
            gessm[lv].append((I, J))
        for K in Ls:
            tstrf[lv].append((K, I))
        for K in Ls:
            for J in Us:
                if (K, J) in nonempty:
                    ssssm[lv].setdefault((K, J), []).append(I)
    ss = []
    for lv in range(nlev):
        ss.append([(t, sorted(src)) for t, src in sorted(ssssm[lv].items())])
    order = np.lexsort((BI, BJ))
    return dict(p=p, ptr=ptr, blocks=np.stack([BI, BJ], 1)[order],
                bnnz=cnt[order].astype(np.int64), dense=dense[order],
                level=level, nlevels=nlev, getrf=getrf,
                gessm=[sorted(g) for g in gessm],
                tstrf=[sorted(t) for t in tstrf], ssssm=ss)
