"""Plan invariants (slu_plan_check): for many random and structured
patterns and every kind of option, each index the kernels take from the
plan is in range and every task relates the blocks its kernel expects.
This is the host-side evidence that no pattern leads a kernel outside its
arrays; a loaded plan that breaks an invariant is refused."""
import struct

import numpy as np
import pytest

import workloads

S = pytest.importorskip("paper_2512_04389_b300.slu")


def _pattern(n, rng, kind):
    if kind == "random":
        M = rng.random((n, n)) < rng.uniform(0.002, 0.08)
    elif kind == "banded":
        i, j = np.indices((n, n))
        M = np.abs(i - j) <= rng.integers(1, 6)
    elif kind == "arrowhead":
        M = np.zeros((n, n), bool)
        M[-rng.integers(1, 4):, :] = True
        M[:, -rng.integers(1, 4):] = True
    elif kind == "blockdiag":
        M = np.zeros((n, n), bool)
        at = 0
        while at < n:
            w = int(rng.integers(1, 40))
            M[at:at + w, at:at + w] = rng.random((min(w, n - at),) * 2) < 0.5
            at += w
    else:                                               # dense border
        M = rng.random((n, n)) < 0.01
        b = max(1, n // 10)
        M[-b:, :] = rng.random((b, n)) < 0.3
        M[:, -b:] |= M[-b:, :].T
    np.fill_diagonal(M, rng.random(n) < 0.9)            # some diagonals missing
    cp = np.zeros(n + 1, np.int64)
    rows = []
    for j in range(n):
        r = np.nonzero(M[:, j])[0]
        if rng.random() < 0.5:
            r = r[rng.permutation(r.size)]
        rows.append(r)
        cp[j + 1] = cp[j] + r.size
    ri = np.concatenate(rows).astype(np.int32) if n else np.zeros(0, np.int32)
    return cp, ri


def _options(rng, n):
    """Random plan options.  Blocks stay at least n / 64 rows wide: the
    Schur task count grows with the cube of the blocks per dimension, and
    one-row blocks of a filled 900-row pattern take a minute to plan."""
    prec = "fp32" if rng.random() < 0.5 else "fp64"
    thr = float(rng.choice([0.0, 0.05, 0.3, 0.6, 1.0, 2.0]))
    lo = max(1, n // 64)
    if rng.random() < 0.3:
        return dict(blocking="regular", regular_block=int(rng.integers(lo, lo + 200)),
                    precision=prec, dense_threshold=thr)
    return dict(precision=prec, dense_threshold=thr,
                b_min=int(lo * rng.choice([1, 2, 4, 8, 32])),
                sample_points=int(rng.choice([10, 100, 1000, 2000])),
                step=int(rng.integers(1, 4)), max_num=int(rng.integers(0, 5)),
                stride=int(rng.integers(1, 3)))


@pytest.mark.parametrize("seed", range(30))
def test_random_plans_satisfy_invariants(seed):
    rng = np.random.default_rng(1000 + seed)
    kinds = ["random", "banded", "arrowhead", "blockdiag", "border"]
    for trial in range(12):
        n = int(rng.choice([1, 2, 3, 7, 31, 64, 150, 400, 900]))
        cp, ri = _pattern(n, rng, kinds[trial % len(kinds)])
        opts = _options(rng, n)
        P = S.Plan(n, cp, ri, **opts)
        P.check()
        Q = S.Plan.from_bytes(P.to_bytes())         # the loader checks too
        assert Q.digest() == P.digest()


@pytest.mark.parametrize("seed", range(4))
def test_random_batches_satisfy_invariants(seed):
    rng = np.random.default_rng(2000 + seed)
    ns = [int(x) for x in rng.integers(1, 120, size=int(rng.integers(2, 9)))]
    pats = [_pattern(n, rng, "random") for n in ns]
    P = S.Plan(ns, [c for c, _ in pats], [r for _, r in pats],
               **_options(rng, max(ns)))
    P.check()


def test_workload_plans_satisfy_invariants():
    for s in (workloads.grid5(48), workloads.grid7_cd(16), workloads.grid7_theta(12),
              workloads.circuit_bbd(n=20_000, border=400)):
        for opts in ({}, dict(dense_threshold=0.0), dict(precision="fp32", b_min=8),
                     dict(blocking="regular", regular_block=64), dict(dense_threshold=0.1)):
            S.Plan(s.n, s.colptr, s.rowidx, **opts).check()


# the plan checksum, restated from its definition (64-bit multiply-xor over
# little-endian 8-byte words with FNV-1a's offset basis and prime, the byte
# count mixed in, splitmix64's finalizer) to forge a consistent header
def _checksum(payload):
    M = (1 << 64) - 1
    h, prime = 0xcbf29ce484222325, 0x100000001b3
    whole = len(payload) // 8 * 8
    for (w,) in struct.iter_unpack("<Q", payload[:whole]):
        h = ((h ^ w) * prime) & M
    tail = payload[whole:]
    if tail:
        h = ((h ^ int.from_bytes(tail, "little")) * prime) & M
    h = ((h ^ len(payload)) * prime) & M
    h ^= h >> 30
    h = (h * 0xbf58476d1ce4e5b9) & M
    h ^= h >> 27
    h = (h * 0x94d049bb133111eb) & M
    return h ^ (h >> 31)


HEADER = 96      # magic, format, byte order, fingerprint, digest, payload, timings


def test_checksum_definition():
    s = workloads.grid5(10)
    P = S.Plan(s.n, s.colptr, s.rowidx)
    b = P.to_bytes()
    assert struct.unpack_from("<Q", b, 24)[0] == _checksum(b[HEADER:]) == P.digest()


def test_loader_refuses_inconsistent_plan_with_valid_checksum():
    s = workloads.grid5(10)
    b = bytearray(S.Plan(s.n, s.colptr, s.rowidx).to_bytes())
    # payload: 72 bytes of options, n, nnz_a, nnz_sym, then A's column
    # pointers (count, then n + 1 values); break the second pointer
    at = HEADER + 72 + 24 + 8 + 8
    struct.pack_into("<q", b, at, 10 ** 9)
    struct.pack_into("<Q", b, 24, _checksum(bytes(b[HEADER:])))
    with pytest.raises(S.SluError) as e:
        S.Plan.from_bytes(bytes(b))
    assert e.value.status == 1 and "invariant" in str(e.value)
