"""Plan cache (slu_plan_serialize / slu_plan_deserialize / slu_plan_digest):
a loaded plan equals the analysed one field for field, and a buffer that is
truncated, corrupted or from another layout is refused, never half-read."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import workloads

S = pytest.importorskip("paper_2512_04389_b300.slu")
CSRC = os.path.join(os.path.dirname(S.__file__), "csrc")

CASES = [
    ("grid5_48", lambda: workloads.grid5(48), {}),
    ("grid5_48 fp32 all dense", lambda: workloads.grid5(48),
     dict(precision="fp32", dense_threshold=0.0)),
    ("grid7cd_12 regular 37", lambda: workloads.grid7_cd(12),
     dict(blocking="regular", regular_block=37)),
    ("circuit_3000", lambda: workloads.circuit_bbd(n=3000, border=60,
                                                   block_lo=16, block_hi=64),
     dict(dense_threshold=0.1, b_min=8)),
]


def _same_exports(P, Q):
    assert P.info == Q.info
    for f in ("export", "export_blocks", "export_tasks"):
        a, b = getattr(P, f)(), getattr(Q, f)()
        assert a.keys() == b.keys()
        for k in a:
            assert np.array_equal(a[k], b[k]), (f, k)
    assert P.flops_by_class() == Q.flops_by_class()


@pytest.mark.parametrize("name,mk,opts", CASES, ids=[c[0] for c in CASES])
def test_round_trip(name, mk, opts):
    s = mk()
    P = S.Plan(s.n, s.colptr, s.rowidx, **opts)
    b = P.to_bytes()
    Q = S.Plan.from_bytes(b)
    assert Q.digest() == P.digest()
    assert Q.to_bytes() == b
    _same_exports(P, Q)


def test_round_trip_batch_and_empty():
    ms = [workloads.grid5(k, seed=k) for k in (7, 12, 5)]
    PB = S.Plan([m.n for m in ms], [m.colptr for m in ms], [m.rowidx for m in ms])
    QB = S.Plan.from_bytes(PB.to_bytes())
    assert QB.digest() == PB.digest()
    _same_exports(PB, QB)
    P0 = S.Plan(0, np.zeros(1, np.int64), np.zeros(0, np.int32))
    Q0 = S.Plan.from_bytes(P0.to_bytes())
    assert Q0.info["n"] == 0 and Q0.digest() == P0.digest()


def test_digest_is_deterministic_and_sees_options():
    s = workloads.grid7_cd(10)
    d = [S.Plan(s.n, s.colptr, s.rowidx).digest() for _ in range(2)]
    assert d[0] == d[1]
    assert S.Plan(s.n, s.colptr, s.rowidx, dense_threshold=0.0).digest() != d[0]
    assert S.Plan(s.n, s.colptr, s.rowidx, precision="fp32").digest() != d[0]


def _raw(buf):
    out = C.c_void_p()
    a = np.frombuffer(buf, np.uint8)
    st = S.lib.slu_plan_deserialize(a.ctypes.data if a.size else None, a.size,
                                    C.byref(out))
    if out.value:
        S.lib.slu_plan_destroy(out)
    return st, S.lib.slu_last_error().decode()


def test_rejects_damaged_buffers():
    s = workloads.grid5(12)
    b = bytearray(S.Plan(s.n, s.colptr, s.rowidx).to_bytes())
    assert _raw(bytes(b))[0] == 0
    # every cut of the 96-byte header, and cuts through the payload
    for cut in list(range(0, 97)) + [128, 1000, len(b) // 2, len(b) - 1]:
        assert _raw(bytes(b[:cut]))[0] == 1, cut
    assert _raw(bytes(b) + b"\0")[0] == 1                      # trailing byte
    for pos in (100, len(b) // 3, len(b) - 3):                 # payload bit flips
        c = bytearray(b)
        c[pos] ^= 0x10
        st, msg = _raw(bytes(c))
        assert st == 1, pos
    c = bytearray(b)
    c[0] ^= 1                                                  # magic
    assert _raw(bytes(c))[0] == 1
    for pos in (8, 16):                                        # format, fingerprint
        c = bytearray(b)
        c[pos] ^= 1
        st, msg = _raw(bytes(c))
        assert st == 7 and "incompatible" in msg
    c = bytearray(b)
    c[12] ^= 1                                                 # byte-order mark
    assert _raw(bytes(c))[0] == 7


def test_serialize_into_short_buffer():
    s = workloads.grid5(8)
    P = S.Plan(s.n, s.colptr, s.rowidx)
    need = len(P.to_bytes())
    buf = np.zeros(need - 1, np.uint8)
    size = C.c_int64(need - 1)
    st = S.lib.slu_plan_serialize(P._h, buf.ctypes.data, C.byref(size))
    assert st == 1 and size.value == need
    assert not buf.any()                                        # nothing written


def test_serialization_lists_every_plan_field():
    """The serialized field list covers every member of slu_plan except the
    analysis times (in the header) and the device mirror."""
    hpp = open(os.path.join(CSRC, "slu_internal.hpp")).read()
    body = hpp[hpp.index("struct slu_plan {") + len("struct slu_plan {"):]
    body = body[:body.index("\n};")]
    body = re.sub(r"//[^\n]*", "", body)
    body = re.sub(r"=\s*\{[^}]*\}", "", body)       # brace initializers
    members = set()
    for decl in body.split(";"):
        decl = re.sub(r"=[^,;]*", "", decl.strip())
        decl = re.sub(r"\[\w+\]", "", decl)
        m = re.match(r"^(?:[\w:]+(?:<[^>]*>)?\s*\*?\s+)([\w\s,*]+)$", decl, re.S)
        if m:
            members |= {x.strip(" *") for x in m.group(1).split(",") if x.strip()}
    assert {"opts", "a2s", "f2s", "sp_off", "flops_cls", "dev"} <= members
    cpp = open(os.path.join(CSRC, "plan_io.cpp")).read()
    macro = cpp[cpp.index("#define SLU_PLAN_FIELDS(X)"):]
    macro = macro[:macro.index("\n\n")]
    listed = set(re.findall(r"X\((\w+)\)", macro))
    assert "phase_ms" in members
    assert listed == members - {"analyze_ms", "phase_ms", "dev"}


def test_save_and_load(tmp_path):
    s = workloads.grid7_cd(8)
    P = S.Plan(s.n, s.colptr, s.rowidx, b_min=8)
    f = tmp_path / "plan.bin"
    P.save(f)
    assert f.read_bytes() == P.to_bytes()
    Q = S.Plan.load(f)
    assert Q.digest() == P.digest()
    _same_exports(P, Q)
