"""Host analysis of the library (C ABI, no GPU needed) against the oracle's
independent plan code: filled pattern, diagonal block pointer (Algorithm 2),
block boundaries (Algorithm 3 / regular), block list, dense flags, levels and
every task list must be bit-exact."""
import re
import os

import numpy as np
import pytest

import workloads
from oracle import lu as OL, plan as OP

S = pytest.importorskip("paper_2512_04389_b300.slu")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "slu.h")).read()
    declared = set(re.findall(r"\b(slu_[a-z_]+)\s*\(", hdr))
    assert declared == set(S.EXPORTS)
    for name in declared:
        assert hasattr(S.lib, name), name


CASES = [
    ("grid5_48 irregular", lambda: workloads.grid5(48), {}),
    ("grid5_48 regular64", lambda: workloads.grid5(48),
     dict(blocking="regular", regular_block=64)),
    ("grid5_48 stride2", lambda: workloads.grid5(48), dict(stride=2)),
    ("grid7cd_12 bmin8", lambda: workloads.grid7_cd(12, nrhs=1), dict(b_min=8)),
    ("grid7theta_10", lambda: workloads.grid7_theta(10), dict(b_min=16)),
    ("circuit_3000", lambda: workloads.circuit_bbd(
        n=3000, border=60, block_lo=16, block_hi=64), dict(b_min=16)),
    ("grid5_7 tiny", lambda: workloads.grid5(7), dict(b_min=4)),
    ("dense threshold 0", lambda: workloads.grid5(20), dict(dense_threshold=0.0,
                                                             b_min=8)),
]


@pytest.mark.parametrize("name,mk,opts", CASES, ids=[c[0] for c in CASES])
def test_plan_bit_exact(name, mk, opts):
    s = mk()
    _check_plan(s, opts)


class _Sys:
    def __init__(self, n, colptr, rowidx, values):
        self.n, self.colptr, self.rowidx, self.values = n, colptr, rowidx, values


def _random_system(n, density, seed):
    """Random nonsymmetric pattern (each off-diagonal entry drawn on its
    own), rows listed in random order inside every column, diagonally
    dominant values."""
    rng = np.random.default_rng(seed)
    M = rng.random((n, n)) < density
    np.fill_diagonal(M, True)
    V = np.where(M, rng.uniform(-1, 1, (n, n)), 0.0)
    np.fill_diagonal(V, np.abs(V).sum(1) + 1.0)
    colptr = np.zeros(n + 1, np.int64)
    rows, vals = [], []
    for j in range(n):
        r = np.nonzero(M[:, j])[0]
        r = r[rng.permutation(r.size)]
        rows.append(r)
        vals.append(V[r, j])
        colptr[j + 1] = colptr[j] + r.size
    return _Sys(n, colptr, np.concatenate(rows).astype(np.int32),
                np.concatenate(vals))


@pytest.mark.parametrize("n,density,seed,opts", [
    (60, 0.05, 1, dict(b_min=4)),
    (150, 0.02, 2, dict(b_min=8, max_num=1)),
    (150, 0.02, 3, dict(blocking="regular", regular_block=17)),
    (300, 0.01, 4, dict(b_min=8, sample_points=100, step=1)),
    (300, 0.01, 5, dict(b_min=16, dense_threshold=0.0)),
])
def test_plan_bit_exact_random_unsorted(n, density, seed, opts):
    """Random nonsymmetric patterns with unsorted rows: the library's
    symmetrisation, symbolic factorization and plan match the oracle's."""
    _check_plan(_random_system(n, density, seed), opts)


def _check_plan(s, opts, oracle=None):
    P = S.Plan(s.n, s.colptr, s.rowidx, **opts)
    o = S.default_opts(**opts)
    if oracle is None:
        F = OL.lu(s.n, s.colptr, s.rowidx, s.values)
        pp, pr, _ = OL.lu_pattern(F)
    else:
        F, (pp, pr, _) = oracle
    e = P.export()
    assert np.array_equal(e["colptr"], pp)
    assert np.array_equal(e["rowidx"], pr)
    bp = OP.blockptr(s.n, pp, pr)
    assert np.array_equal(e["blockptr"], bp)
    if o.blocking == 0:
        ptr = OP.irregular_ptr(bp, s.n, o.sample_points, o.step, o.max_num,
                               o.stride, o.b_min)
        assert P.info["samples"] == OP.num_samples(s.n, o.sample_points,
                                                  o.b_min)
    else:
        ptr = OP.regular_ptr(s.n, o.regular_block)
    assert np.array_equal(e["ptr"], ptr)
    assert P.info["flops"] == OL.flops(F)
    pl = OP.block_plan(s.n, pp, pr, ptr, o.dense_threshold)
    b = P.export_blocks()
    assert np.array_equal(b["blocks"], pl["blocks"])
    assert np.array_equal(b["bnnz"], pl["bnnz"])
    assert np.array_equal(b["dense"], pl["dense"])
    assert np.array_equal(b["level"], pl["level"])
    t = P.export_tasks()
    assert P.info["nlevels"] == pl["nlevels"]
    for lv in range(pl["nlevels"]):
        g = t["getrf"][t["getrf_off"][lv]:t["getrf_off"][lv + 1]]
        assert g.tolist() == pl["getrf"][lv]
        ge = t["gessm"][2 * t["gessm_off"][lv]:2 * t["gessm_off"][lv + 1]]
        assert [tuple(x) for x in ge.reshape(-1, 2).tolist()] == pl["gessm"][lv]
        ts = t["tstrf"][2 * t["tstrf_off"][lv]:2 * t["tstrf_off"][lv + 1]]
        # tasks of one level are independent: compare as sorted lists
        assert sorted(tuple(x) for x in ts.reshape(-1, 2).tolist()) == \
            pl["tstrf"][lv]
        tg = t["tgt"].reshape(-1, 2)
        got = []
        for k in range(t["tgt_off"][lv], t["tgt_off"][lv + 1]):
            srcs = t["src"][t["srcoff"][k]:t["srcoff"][k + 1]].tolist()
            got.append((tuple(tg[k].tolist()), srcs))
        assert got == pl["ssssm"][lv]


@pytest.fixture(scope="module")
def grid7cd_40_oracle():
    s = workloads.grid7_cd(40)
    F = OL.lu(s.n, s.colptr, s.rowidx, s.values)
    return s, F, OL.lu_pattern(F)


# The autotuned options of the 40^3 convection-diffusion plans the benchmark
# times (FP64: max_num 1; FP32: S = 2000), and the paper's defaults.
TUNED_40 = [
    dict(dense_threshold=0.0, sample_points=1000, b_min=32, max_num=1),
    dict(dense_threshold=0.0, sample_points=2000, b_min=32, max_num=3,
         precision="fp32"),
    dict(blocking="regular", regular_block=128, dense_threshold=0.0),
]


@pytest.mark.parametrize("opts", TUNED_40,
                         ids=["fp64_S1000_m1", "fp32_S2000_m3", "regular128"])
def test_plan_bit_exact_grid7cd_40_tuned(grid7cd_40_oracle, opts):
    """Full size n = 64,000: the plans the benchmark factors are the
    oracle's plans bit for bit (pattern, Algorithm 2, Algorithm 3, blocks,
    dense flags, levels, every task list)."""
    s, F, pat = grid7cd_40_oracle
    _check_plan(s, opts, oracle=(F, pat))


@pytest.mark.parametrize("bad", ["dup", "range", "colptr"])
def test_analyze_rejects_bad_patterns(bad):
    cp = np.array([0, 2, 3], np.int64)
    ri = np.array([0, 1, 1], np.int32)
    if bad == "dup":
        ri = np.array([0, 0, 1], np.int32)
    elif bad == "range":
        ri = np.array([0, 2, 1], np.int32)
    else:
        cp = np.array([0, 3, 2], np.int64)
    with pytest.raises(S.SluError) as e:
        S.Plan(2, cp, ri)
    assert e.value.status == 1


def test_analyze_rejects_bad_options():
    s = workloads.grid5(4)
    with pytest.raises(S.SluError):
        S.Plan(s.n, s.colptr, s.rowidx, step=0)
    with pytest.raises(S.SluError):
        S.Plan(s.n, s.colptr, s.rowidx, blocking="regular", regular_block=0)


def test_empty_and_single():
    P = S.Plan(0, np.zeros(1, np.int64), np.zeros(0, np.int32))
    assert P.info["nblocks_1d"] == 0 and P.info["nlevels"] == 0
    P = S.Plan(1, np.array([0, 1]), np.array([0]))
    assert P.info["nnz_lu"] == 1 and P.info["nblocks_1d"] == 1
    # an entirely empty column still gets its diagonal
    P = S.Plan(3, np.array([0, 1, 1, 2]), np.array([0, 2]))
    assert P.info["nnz_sym"] == 3


@pytest.mark.parametrize("name,mk,opts", [
    ("grid7cd_16", lambda: workloads.grid7_cd(16), {}),
    ("circuit_4000", lambda: workloads.circuit_bbd(n=4000, border=80,
                                                   block_lo=16, block_hi=64),
     dict(dense_threshold=0.1, b_min=8)),
    ("random unsorted", lambda: _random_system(400, 0.01, 9), dict(b_min=8)),
])
def test_plan_independent_of_host_threads(name, mk, opts, monkeypatch):
    """The threaded analysis gives the same plan (every field, by digest)
    for 1, 2, 3, 7 and 16 host threads."""
    s = mk()
    digests = set()
    for t in (1, 2, 3, 7, 16):
        monkeypatch.setenv("SLU_HOST_THREADS", str(t))
        digests.add(S.Plan(s.n, s.colptr, s.rowidx, **opts).digest())
    assert len(digests) == 1


def test_size_limits():
    """Local row indices inside a block are 16-bit: a block of more than
    65535 rows is refused with NOT_SUPPORTED and one of exactly 65535 is
    planned; an order beyond 32-bit row indices is refused before any array
    is read."""
    import ctypes as C
    n = 70_000
    cp = np.arange(n + 1, dtype=np.int64)       # diagonal pattern
    ri = np.arange(n, dtype=np.int32)
    with pytest.raises(S.SluError) as e:
        S.Plan(n, cp, ri, blocking="regular", regular_block=n)
    assert e.value.status == 7
    P = S.Plan(n, cp, ri, blocking="regular", regular_block=65535)
    assert P.info["max_block"] == 65535 and P.info["nblocks_1d"] == 2
    out = C.c_void_p()
    st = S.lib.slu_analyze(2 ** 31, cp.ctypes.data, ri.ctypes.data,
                           C.byref(S.default_opts()), C.byref(out))
    assert st == 1 and not out.value


def _diag_system(n):
    return _Sys(n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32),
                np.full(n, 2.0))


def _dense_system(n, seed=3):
    rng = np.random.default_rng(seed)
    V = rng.uniform(-1, 1, (n, n)) + n * np.eye(n)
    return _Sys(n, np.arange(0, n * n + 1, n, dtype=np.int64),
                np.tile(np.arange(n, dtype=np.int32), n), V.T.reshape(-1).copy())


@pytest.mark.parametrize("name,mk,opts", [
    ("diagonal 300", lambda: _diag_system(300), dict(b_min=8)),
    ("diagonal 300 regular 7", lambda: _diag_system(300),
     dict(blocking="regular", regular_block=7)),
    ("dense 48", lambda: _dense_system(48), dict(b_min=4)),
    ("dense 48 regular 13", lambda: _dense_system(48),
     dict(blocking="regular", regular_block=13)),
])
def test_plan_bit_exact_degenerate(name, mk, opts):
    """The two ends of the density range: no off-diagonal entry (no fill, no
    flops, every block on level 0) and a fully dense pattern (Alg. 2's
    quadratic profile)."""
    s = mk()
    _check_plan(s, opts)
    P = S.Plan(s.n, s.colptr, s.rowidx, **opts)
    if name.startswith("diagonal"):
        assert P.info["flops"] == 0 and P.info["nlevels"] == 1
        assert P.info["nnz_lu"] == s.n
    else:
        assert P.info["nnz_lu"] == s.n * s.n
        assert np.array_equal(P.export()["blockptr"], np.arange(s.n + 1) ** 2)


@pytest.mark.parametrize("name,mk,opts", [
    ("grid5_48", lambda: workloads.grid5(48), {}),
    ("grid7cd_12 regular 37", lambda: workloads.grid7_cd(12),
     dict(blocking="regular", regular_block=37)),
    ("circuit_3000", lambda: workloads.circuit_bbd(n=3000, border=60,
                                                   block_lo=16, block_hi=64),
     dict(b_min=8)),
])
def test_flops_by_kernel_class(name, mk, opts):
    """The per-class flops behind the roofline fractions: column k of L has
    l_in entries in its own block row and l_out below it; GETRF does
    l_in + 2 l_in^2, the panels l_out + 4 l_in l_out, the Schur updates
    2 l_out^2 (u_k = l_k by symmetry), summing to Table 3's count.
    Recomputed from the oracle's fill pattern and the plan's boundaries."""
    s = mk()
    P = S.Plan(s.n, s.colptr, s.rowidx, **opts)
    cp, ri, _ = OL.lu_pattern(OL.lu(s.n, s.colptr, s.rowidx, s.values))
    blk = np.searchsorted(P.export()["ptr"], np.arange(s.n), side="right") - 1
    want = np.zeros(3)
    for k in range(s.n):
        r = ri[cp[k]:cp[k + 1]]
        r = r[r > k]
        lin = float(np.sum(blk[r] == blk[k]))
        lout = float(r.size) - lin
        want += [lin + 2 * lin * lin, lout + 4 * lin * lout, 2 * lout * lout]
    got = P.flops_by_class()
    assert [got["getrf"], got["panel"], got["ssssm"]] == want.tolist()
    assert sum(got.values()) == P.info["flops"] == OL.flops(
        OL.lu(s.n, s.colptr, s.rowidx, s.values))


@pytest.mark.parametrize("threads", ["1", "8"])
def test_first_bad_entry_is_reported(threads, monkeypatch):
    """With bad entries in several columns the analysis reports the one a
    sequential scan meets first, whichever thread scans it."""
    monkeypatch.setenv("SLU_HOST_THREADS", threads)
    n = 2000
    cp = np.arange(0, 2 * n + 1, 2, dtype=np.int64)      # two entries a column
    base = np.stack([np.arange(n), (np.arange(n) + 1) % n], 1).reshape(-1)
    for early, late, msg in ((("dup", 3), ("range", n - 5), "duplicate entry"),
                             (("range", 3), ("dup", n - 5), "out of range")):
        ri = base.astype(np.int32).copy()
        for what, col in (early, late):
            ri[2 * col + 1] = ri[2 * col] if what == "dup" else n + 7
        with pytest.raises(S.SluError) as e:
            S.Plan(n, cp, ri)
        assert e.value.status == 1 and msg in str(e.value)


@pytest.mark.parametrize("n,nnz_lu,expect", [
    (576, 14_858, 32),          # 25.8 filled entries per column
    (4_096, 174_226, 32),       # 42.5: last point of the first leaf
    (4_000, 170_998, 64),       # 42.7: first point of the second leaf
    (25_600, 1_569_316, 64),    # 61.3
    (1_000, 93_178, 64),        # 93.2
    (10_000, 965_846, 32),      # 96.6: third leaf
    (64_000, 42_558_222, 32),   # 665
    (20, 400, 20),              # capped by n
    (0, 0, 1),
])
def test_regular_size_selection_tree(n, nnz_lu, expect):
    """The selection tree's documented splits: filled entries per column
    <= 42.6 -> 32 rows, <= 95 -> 64, else 32; never more than n."""
    assert S.lib.slu_select_regular_block(n, nnz_lu) == expect


@pytest.mark.parametrize("mk", [lambda: workloads.grid5(48),
                                lambda: workloads.grid7_cd(12, nrhs=1),
                                lambda: workloads.circuit_bbd(
                                    n=3000, border=60, block_lo=16, block_hi=64)])
def test_regular_select_plan_is_the_regular_plan_of_the_selected_size(mk):
    """SLU_BLOCKING_REGULAR_SELECT blocks regularly with the tree's size for
    the filled pattern, and the plan is the oracle's regular plan of that
    size bit for bit."""
    s = mk()
    P = S.Plan(s.n, s.colptr, s.rowidx, blocking="regular_select")
    b = P.info["regular_block"]
    assert b == S.lib.slu_select_regular_block(s.n, P.info["nnz_lu"])
    _check_plan(s, dict(blocking="regular", regular_block=b))
    R = S.Plan(s.n, s.colptr, s.rowidx, blocking="regular", regular_block=b)
    assert np.array_equal(P.export()["ptr"], R.export()["ptr"])
    for k in ("blocks", "bnnz", "dense", "level"):
        assert np.array_equal(P.export_blocks()[k], R.export_blocks()[k])


def test_regular_select_per_batch_member():
    """In a batch, every member gets the size its own filled pattern
    selects: a sparse-filling 2-D grid and a dense-filling 3-D operator."""
    ms = [workloads.grid5(100), workloads.grid7_cd(14, nrhs=1)]
    PB = S.Plan([m.n for m in ms], [m.colptr for m in ms],
                [m.rowidx for m in ms], blocking="regular_select")
    ptr = PB.export()["ptr"]
    off = 0
    sizes = []
    for m in ms:
        Pm = S.Plan(m.n, m.colptr, m.rowidx, blocking="regular_select")
        b = Pm.info["regular_block"]
        sizes.append(b)
        mine = ptr[(ptr >= off) & (ptr <= off + m.n)] - off
        assert np.array_equal(mine, OP.regular_ptr(m.n, b))
        off += m.n
    assert sizes == [64, 32] and PB.info["regular_block"] == 64
