"""Batch analysis: a batch plan is the members' own plans laid out
block-diagonally (each member blocked by its own Algorithm 2/3 curve), with
levels merged by index."""
import numpy as np
import pytest

import workloads

S = pytest.importorskip("paper_2512_04389_b300.slu")


def _members():
    return [workloads.grid5(k, seed=3 + k) for k in (16, 23, 9, 31)]


@pytest.mark.parametrize("opts", [{}, dict(blocking="regular", regular_block=40),
                                  dict(b_min=8, stride=2)])
def test_batch_plan_is_concatenation_of_member_plans(opts):
    ms = _members()
    PB = S.Plan([m.n for m in ms], [m.colptr for m in ms],
                [m.rowidx for m in ms], **opts)
    eb = PB.export()
    bb = PB.export_blocks()
    off = 0
    ptrs, levels, blocks = [0], [], []
    nb_off = 0
    for m in ms:
        P = S.Plan(m.n, m.colptr, m.rowidx, **opts)
        e = P.export()
        b = P.export_blocks()
        ptrs += (e["ptr"][1:] + off).tolist()
        levels += b["level"].tolist()
        blocks.append(b["blocks"] + nb_off)
        off += m.n
        nb_off += P.info["nblocks_1d"]
    assert eb["ptr"].tolist() == ptrs
    assert bb["level"].tolist() == levels
    got = {tuple(x) for x in bb["blocks"].tolist()}
    exp = {tuple(x) for x in np.concatenate(blocks).tolist()}
    assert got == exp
    assert PB.info["nlevels"] == max(levels) + 1
    assert PB.info["flops"] == sum(S.Plan(m.n, m.colptr, m.rowidx, **opts).info["flops"]
                                   for m in ms)


@pytest.mark.parametrize("bad,msg", [("start", "colptr[0]"),
                                     ("monotone", "monotone"),
                                     ("negative_n", "bad batch member"),
                                     ("range", "out of range")])
def test_batch_rejects_malformed_member(bad, msg):
    """A malformed member is rejected before its row indices are read."""
    good = workloads.grid5(4)
    cp = np.array([0, 2, 3], np.int64)
    ri = np.array([0, 1, 1], np.int32)
    n = 2
    if bad == "start":
        cp = np.array([1, 2, 3], np.int64)
    elif bad == "monotone":
        cp = np.array([0, 5, 3], np.int64)
    elif bad == "negative_n":
        n = -1
    else:
        ri = np.array([0, 1, 2], np.int32)
    # straight through the C ABI, past the binding's own length checks
    import ctypes as C
    cps = [np.ascontiguousarray(good.colptr, np.int64), cp]
    ris = [np.ascontiguousarray(good.rowidx, np.int32), ri]
    na = np.array([good.n, n], np.int64)
    cpa = (C.c_void_p * 2)(*[c.ctypes.data for c in cps])
    ria = (C.c_void_p * 2)(*[r.ctypes.data for r in ris])
    o = S.default_opts()
    out = C.c_void_p()
    st = S.lib.slu_analyze_batch(2, na.ctypes.data, cpa, ria, C.byref(o),
                                 C.byref(out))
    assert st == 1 and not out.value
    assert msg in S.lib.slu_last_error().decode()
