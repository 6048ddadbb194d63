"""Seeded synthetic linear systems shaped like the paper's workloads.

This module is shared by the CPU oracle and the GPU path.  It holds no part of
the factorization method: it builds matrices (CSC, 0-based, rows sorted in each
column), orders them, and draws right-hand sides.  Every random number comes
from numpy's PCG64 generator seeded with the documented seed, drawn in the
order each function's docstring states, so both sides see identical inputs.

Workloads (sizes as named by the generators' callers):

* ``grid5``    2-D 5-point nonsymmetric operator on a k x k grid, geometric
  nested-dissection order (separators last).  Off-diagonals U(-1, 0) drawn
  independently for (i, j) and (j, i); diagonal 4 + U(0.5, 1.5).
* ``grid7_cd`` 3-D 7-point convection-diffusion operator on an m^3 grid, ND
  order.  Per axis the upwind neighbour gets -(1 + u), the downwind one
  -(1 - u), u ~ U(0, 0.3) per entry; diagonal = sum |off| + U(0.1, 1).
* ``grid7_theta`` 3-D 7-point operator with per-cell diffusion
  theta = exp(N(0, 0.5^2)), harmonic-mean face coefficients, central
  advection along (1, 1, 1) with cell Peclet 0.5, Dirichlet boundary faces.
* ``circuit_bbd`` bordered-block-diagonal circuit-like matrix: block-diagonal
  Chung-Lu subcircuits with Zipf(2.1) expected degrees (mean 6), plus a border
  whose nodes each link to 5% of all nodes, ordered border-last.
* ``batch_grid5`` many independent ``grid5`` systems with k ~ U{16..96}.

The paper measures on SuiteSparse matrices (Table 3), which are not available
here; these generators stand in for them, reproducing the structural traits the
paper describes (nonzeros concentrated bottom-right after ordering, Section 2.1;
a circuit matrix with 98% of its nonzeros in the border, Section 5.3; a
linear-profile grid, Section 5.3).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "SparseSystem", "nd_order", "grid5", "grid7_cd", "grid7_theta",
    "circuit_bbd", "batch_grid5", "coo_to_csc", "by_name",
]


@dataclass
class SparseSystem:
    """A square sparse system A x = B in CSC form (0-based, rows sorted).

    ``colptr`` int64[n+1], ``rowidx`` int32[nnz], ``values`` float64[nnz],
    ``rhs`` float64[n, nrhs] (Fortran order, column-major).
    """
    n: int
    colptr: np.ndarray
    rowidx: np.ndarray
    values: np.ndarray
    rhs: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.colptr[-1])

    @property
    def nrhs(self) -> int:
        return int(self.rhs.shape[1])

    def dense(self) -> np.ndarray:
        """Dense copy (small cases only)."""
        d = np.zeros((self.n, self.n))
        cols = np.repeat(np.arange(self.n), np.diff(self.colptr))
        d[self.rowidx, cols] = self.values
        return d


def coo_to_csc(n, rows, cols, vals, sum_duplicates=True):
    """COO -> CSC with rows sorted inside each column (duplicates summed)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    # one stable sort on the (column, row) key: the order of a two-key
    # lexicographic sort, with equal entries kept in input order
    order = np.argsort(cols * n + rows, kind="stable")
    rows, cols, vals = rows[order], cols[order], vals[order]
    if sum_duplicates and rows.size:
        key = cols * n + rows
        first = np.ones(key.size, dtype=bool)
        first[1:] = key[1:] != key[:-1]
        idx = np.cumsum(first) - 1
        v2 = np.bincount(idx, weights=vals, minlength=int(first.sum()))
        rows, cols, vals = rows[first], cols[first], v2
    colptr = np.zeros(n + 1, dtype=np.int64)
    colptr[1:] = np.cumsum(np.bincount(cols, minlength=n))
    return colptr, rows.astype(np.int32), vals


def nd_order(dims, leaf=8):
    """Geometric nested-dissection order of a 2-D or 3-D grid.

    Recursively split the longest axis (lowest axis index on ties) of the
    current box at mid = (lo + hi) // 2 with a one-cell separator plane;
    order left part, right part, then the separator.  Boxes of at most
    ``leaf`` cells, and separators, are listed in natural order (cell id
    x + nx*(y + ny*z), ascending).  Returns ``perm`` with perm[new] = old id.
    """
    dims = tuple(int(d) for d in dims)
    nd = len(dims)
    out = []

    def ids(lo, hi):
        rng_ = [np.arange(a, b) for a, b in zip(lo, hi)]
        g = np.meshgrid(*rng_, indexing="ij")
        cid = g[0].astype(np.int64)
        mul = dims[0]
        for a in range(1, nd):
            cid = cid + mul * g[a]
            mul *= dims[a]
        return np.sort(cid.ravel())

    stack = [("box", tuple([0] * nd), dims)]
    # iterative post-order: (left, right, separator)
    while stack:
        kind, lo, hi = stack.pop()
        if kind == "emit":
            out.append(ids(lo, hi))
            continue
        sizes = [b - a for a, b in zip(lo, hi)]
        if min(sizes) <= 0:
            continue
        if int(np.prod(sizes)) <= leaf:
            out.append(ids(lo, hi))
            continue
        ax = int(np.argmax(sizes))
        mid = (lo[ax] + hi[ax]) // 2
        lhi = list(hi); lhi[ax] = mid
        rlo = list(lo); rlo[ax] = mid + 1
        slo = list(lo); slo[ax] = mid
        shi = list(hi); shi[ax] = mid + 1
        # pushed in reverse so that left is processed first
        stack.append(("emit", tuple(slo), tuple(shi)))
        stack.append(("box", tuple(rlo), hi))
        stack.append(("box", lo, tuple(lhi)))
    perm = np.concatenate(out)
    assert perm.size == int(np.prod(dims))
    return perm


def _neighbours(dims):
    """Directed grid edges (i -> j) in natural ids, listed by axis then
    direction (-1, +1), then ascending i.  Returns (i, j, axis, dirn)."""
    nd = len(dims)
    n = int(np.prod(dims))
    cid = np.arange(n, dtype=np.int64)
    coord = []
    rem = cid.copy()
    for a in range(nd):
        coord.append(rem % dims[a])
        rem //= dims[a]
    stride = [int(np.prod(dims[:a])) for a in range(nd)]
    I, J, AX, DI = [], [], [], []
    for a in range(nd):
        for d in (-1, 1):
            ok = (coord[a] + d >= 0) & (coord[a] + d < dims[a])
            i = cid[ok]
            I.append(i); J.append(i + d * stride[a])
            AX.append(np.full(i.size, a)); DI.append(np.full(i.size, d))
    return (np.concatenate(I), np.concatenate(J), np.concatenate(AX),
            np.concatenate(DI))


def _permute(n, perm, rows, cols, vals):
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    return coo_to_csc(n, inv[rows], inv[cols], vals)


def _rhs(rng, n, nrhs):
    return np.asfortranarray(rng.standard_normal((nrhs, n)).T)


def grid5(k, seed=0, nrhs=1, order="nd"):
    """2-D 5-point operator on a k x k grid (n = k^2).

    Draw order: off-diagonal values U(-1, 0) for the directed edges in
    ``_neighbours`` order; then the diagonal 4 + U(0.5, 1.5) for cells in
    natural order; then the right-hand sides N(0, 1), one column at a time.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    dims = (k, k)
    n = k * k
    i, j, _, _ = _neighbours(dims)
    off = rng.uniform(-1.0, 0.0, size=i.size)
    diag = 4.0 + rng.uniform(0.5, 1.5, size=n)
    rows = np.concatenate([i, np.arange(n)])
    cols = np.concatenate([j, np.arange(n)])
    vals = np.concatenate([off, diag])
    perm = nd_order(dims) if order == "nd" else np.arange(n)
    colptr, rowidx, values = _permute(n, perm, rows, cols, vals)
    b = _rhs(rng, n, nrhs)
    return SparseSystem(n, colptr, rowidx, values, b, name=f"grid5_{k}x{k}",
                        meta={"dims": dims, "perm": perm, "seed": seed})


def grid7_cd(m, seed=0, nrhs=4, skew=0.3):
    """3-D 7-point convection-diffusion operator on an m^3 grid (n = m^3).

    Draw order: u ~ U(0, skew) for the directed edges in ``_neighbours`` order
    (the -1 neighbour along an axis is upwind and gets -(1 + u), the +1
    neighbour is downwind and gets -(1 - u)); then U(0.1, 1) per cell in
    natural order, added to the row sum of |off-diagonals| to give the
    diagonal; then the right-hand sides.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    dims = (m, m, m)
    n = m ** 3
    i, j, _, d = _neighbours(dims)
    u = rng.uniform(0.0, skew, size=i.size)
    off = np.where(d < 0, -(1.0 + u), -(1.0 - u))
    rowsum = np.zeros(n)
    np.add.at(rowsum, i, np.abs(off))
    diag = rowsum + rng.uniform(0.1, 1.0, size=n)
    rows = np.concatenate([i, np.arange(n)])
    cols = np.concatenate([j, np.arange(n)])
    vals = np.concatenate([off, diag])
    perm = nd_order(dims)
    colptr, rowidx, values = _permute(n, perm, rows, cols, vals)
    b = _rhs(rng, n, nrhs)
    return SparseSystem(n, colptr, rowidx, values, b, name=f"grid7cd_{m}^3",
                        meta={"dims": dims, "perm": perm, "seed": seed})


def grid7_theta(m, seed=0, nrhs=1, peclet=0.5, sigma=0.5):
    """3-D 7-point diffusion-advection operator A(theta) on an m^3 grid.

    Draw order: theta_c = exp(N(0, sigma^2)) per cell in natural order; then
    the right-hand sides.  Face coefficient = harmonic mean of the two cells'
    theta.  Central advection with constant velocity along (1, 1, 1) and cell
    Peclet ``peclet``: the upwind (-1) neighbour gets -theta_f (1 + Pe/2), the
    downwind (+1) neighbour -theta_f (1 - Pe/2).  The diagonal is the sum of
    the six face coefficients, a Dirichlet boundary face contributing the
    cell's own theta.

    ``meta['theta']`` holds theta (natural order) and ``meta['pattern']`` maps
    each stored value to how it depends on theta, for differentiation tests.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    dims = (m, m, m)
    n = m ** 3
    theta = np.exp(sigma * rng.standard_normal(n))
    i, j, _, d = _neighbours(dims)
    tf = 2.0 * theta[i] * theta[j] / (theta[i] + theta[j])
    off = np.where(d < 0, -tf * (1.0 + peclet / 2), -tf * (1.0 - peclet / 2))
    diag = np.zeros(n)
    np.add.at(diag, i, tf)
    # boundary faces: 2*nd faces per cell minus interior neighbours
    nface = np.zeros(n)
    np.add.at(nface, i, 1.0)
    diag += (2 * len(dims) - nface) * theta
    rows = np.concatenate([i, np.arange(n)])
    cols = np.concatenate([j, np.arange(n)])
    vals = np.concatenate([off, diag])
    perm = nd_order(dims)
    colptr, rowidx, values = _permute(n, perm, rows, cols, vals)
    b = _rhs(rng, n, nrhs)
    return SparseSystem(n, colptr, rowidx, values, b, name=f"grid7theta_{m}^3",
                        meta={"dims": dims, "perm": perm, "seed": seed,
                              "theta": theta, "peclet": peclet})


def circuit_bbd(n=200_000, border=4_000, seed=0, nrhs=8, block_lo=32,
                block_hi=256, mean_deg=6.0, zipf_a=2.1, border_frac=0.05):
    """Bordered-block-diagonal circuit-like matrix, ordered border-last.

    Body (n - border nodes): consecutive subcircuits with sizes drawn
    U{block_lo..block_hi} (the last one takes the remainder).  Per subcircuit,
    expected degrees w ~ Zipf(zipf_a) rescaled to mean ``mean_deg`` and capped
    at size-1; each unordered pair (a, b) is an edge with probability
    min(1, w_a w_b / sum w) (Chung-Lu); the subcircuit is ordered by ascending
    w (hubs last, stable).  Border: node t links to each of the n nodes
    independently with probability ``border_frac`` (about 5% of all nodes;
    self excluded), symmetric.  Off-diagonal magnitudes are
    log-uniform on [1e-3, 1] with a random sign; diagonal = row sum of
    |off-diagonals| x U(1.05, 2).

    Draw order: block sizes; per block: Zipf draws, pair coin flips; border
    coin flips, 64 border nodes at a time, each a 64 x n block of U(0, 1) in
    row-major order; magnitudes, signs (both for the stored off-diagonal
    entries in sorted (col, row) order); diagonal factors; RHS.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    nb = n - border
    sizes = []
    tot = 0
    while tot < nb:
        s = int(rng.integers(block_lo, block_hi + 1))
        s = min(s, nb - tot)
        sizes.append(s)
        tot += s
    E_i, E_j = [], []
    base = 0
    for s in sizes:
        w = rng.zipf(zipf_a, size=s).astype(np.float64)
        w *= mean_deg / w.mean()
        w = np.minimum(w, max(s - 1, 1))
        iu, ju = np.triu_indices(s, 1)
        p = np.minimum(1.0, w[iu] * w[ju] / w.sum())
        keep = rng.random(iu.size) < p
        order = np.argsort(w, kind="stable")      # old local -> new position
        pos = np.empty(s, dtype=np.int64)
        pos[order] = np.arange(s)
        E_i.append(base + pos[iu[keep]])
        E_j.append(base + pos[ju[keep]])
        base += s
    for t0 in range(0, border, 64):
        t1 = min(border, t0 + 64)
        hit = rng.random((t1 - t0, n)) < border_frac
        rr, cc = np.nonzero(hit)
        node = nb + t0 + rr
        keep = cc != node                           # no self links
        E_i.append(node[keep].astype(np.int64))
        E_j.append(cc[keep].astype(np.int64))
    ei = np.concatenate(E_i)
    ej = np.concatenate(E_j)
    # symmetric pattern, duplicates removed
    r = np.concatenate([ei, ej])
    c = np.concatenate([ej, ei])
    key = np.sort(c * n + r)                       # sort + dedupe
    key = key[np.r_[True, key[1:] != key[:-1]]] if key.size else key
    cols = key // n
    rows = key % n
    m = rows.size
    mag = 10.0 ** rng.uniform(-3.0, 0.0, size=m)
    sgn = np.where(rng.random(m) < 0.5, -1.0, 1.0)
    off = mag * sgn
    rowsum = np.bincount(rows, weights=np.abs(off), minlength=n)
    diag = rowsum * rng.uniform(1.05, 2.0, size=n)
    diag[diag == 0.0] = 1.0                      # isolated node
    colptr, rowidx, values = coo_to_csc(
        n, np.concatenate([rows, np.arange(n)]),
        np.concatenate([cols, np.arange(n)]), np.concatenate([off, diag]))
    b = _rhs(rng, n, nrhs)
    return SparseSystem(n, colptr, rowidx, values, b,
                        name=f"circuit_bbd_{n}_{border}",
                        meta={"border": border, "subcircuits": len(sizes),
                              "seed": seed})


def batch_grid5(count=256, seed=0, k_lo=16, k_hi=96):
    """``count`` independent grid5 systems; k_m ~ U{k_lo..k_hi} drawn from
    PCG64(seed), system m built by grid5(k_m, seed=seed + 1 + m)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ks = rng.integers(k_lo, k_hi + 1, size=count)
    return [grid5(int(k), seed=seed + 1 + m) for m, k in enumerate(ks)]


def by_name(name, **kw):
    """Named workloads: 'grid5_48' (n=2304), 'grid7cd_40' (n=64,000),
    'grid7theta_32' (n=32,768), 'grid7theta_6' (n=216),
    'circuit_200k' (n=200,000), 'circuit_20k' (n=20,000, 400 border)."""
    if name.startswith("grid5_"):
        return grid5(int(name.split("_")[1]), **kw)
    if name.startswith("grid7cd_"):
        return grid7_cd(int(name.split("_")[1]), **kw)
    if name.startswith("grid7theta_"):
        return grid7_theta(int(name.split("_")[1]), **kw)
    if name == "circuit_200k":
        return circuit_bbd(**kw)
    if name == "circuit_20k":
        return circuit_bbd(n=20_000, border=400, **kw)
    raise KeyError(name)
