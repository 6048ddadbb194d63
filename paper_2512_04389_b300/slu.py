"""Thin Python binding of the C ABI in ``include/slu.h`` (ctypes).

Argument marshalling only: every step of analysis runs in the library's host
code and every numerical step in its CUDA kernels.  torch supplies device
memory and the current CUDA stream.  If ``libslu_b300.so`` is missing or
cannot be loaded the import of this module raises; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libslu_b300.so")

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OUT_OF_MEMORY", 3: "CUDA_ERROR",
          4: "SINGULAR", 5: "NOT_CONVERGED", 6: "TIMEOUT", 7: "NOT_SUPPORTED"}
BLOCKING = {"irregular": 0, "regular": 1, "regular_select": 2}
PRECISION = {"fp64": 0, "fp32": 1}


class SluError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"slu {STATUS.get(status, status)}: {msg}")
        self.status = status


class Opts(C.Structure):
    _fields_ = [("blocking", C.c_int32), ("regular_block", C.c_int32),
                ("sample_points", C.c_int32), ("step", C.c_int32),
                ("max_num", C.c_int32), ("stride", C.c_int32),
                ("b_min", C.c_int32), ("precision", C.c_int32),
                ("dense_threshold", C.c_double), ("pivot_perturb", C.c_int32),
                ("pivot_tau_rel", C.c_double), ("refine_tol", C.c_double),
                ("refine_max_iter", C.c_int32), ("wait_budget_ms", C.c_int64),
                ("tc_passes", C.c_int32)]


class PlanInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz_a", C.c_int64), ("nnz_sym", C.c_int64),
                ("nnz_lu", C.c_int64), ("flops", C.c_int64),
                ("nblocks_1d", C.c_int32), ("nlevels", C.c_int32),
                ("nblocks", C.c_int64), ("ndense", C.c_int64),
                ("storage_elems", C.c_int64), ("n_getrf", C.c_int64),
                ("n_gessm", C.c_int64), ("n_tstrf", C.c_int64),
                ("n_ssssm_targets", C.c_int64), ("n_ssssm_pairs", C.c_int64),
                ("max_block", C.c_int32), ("samples", C.c_int32),
                ("analyze_ms", C.c_double), ("regular_block", C.c_int32),
                ("phase_ms", C.c_double * 6)]


PHASES = ("input", "symbolic", "blocking", "blocks", "tasks", "maps")


def _info_dict(i):
    d = {k: getattr(i, k) for k, _ in PlanInfo._fields_}
    d["phase_ms"] = dict(zip(PHASES, list(i.phase_ms)))
    return d


class FactorInfo(C.Structure):
    _fields_ = [("nperturb", C.c_int64), ("tau", C.c_double)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("backward_error", C.c_double)]


KERNEL_CLASSES = ["prep", "getrf", "panel", "ssssm", "solve_pull", "resid",
                  "inv", "solve_diag", "persistent"]


class Stats(C.Structure):
    _fields_ = [("launches", C.c_int64), ("calls", C.c_int64 * 9),
                ("ms", C.c_double * 9)]


# every entry point declared in include/slu.h
EXPORTS = ["slu_opts_default", "slu_analyze", "slu_analyze_batch",
           "slu_analyze_device", "slu_analyze_batch_device", "slu_plan_query",
           "slu_plan_export", "slu_plan_export_blocks", "slu_plan_export_tasks",
           "slu_factor", "slu_refactor", "slu_solve", "slu_solve_transpose",
           "slu_export_factors", "slu_grad_values", "slu_set_profiling", "slu_handle_stats",
           "slu_plan_flops", "slu_handle_trace", "slu_set_graph", "slu_solve_refine_noalloc",
           "slu_factor_batch", "slu_select_regular_block",
           "slu_set_persistent", "slu_persistent_tasks", "slu_set_persistent_tasks",
           "slu_set_persistent_solve",
           "slu_reorder", "slu_reorder_apply", "slu_permute_scale",
           "slu_plan_serialize", "slu_plan_deserialize", "slu_plan_digest", "slu_plan_check",
           "slu_plan_destroy",
           "slu_handle_destroy", "slu_last_error"]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with "
            "`python -m paper_2512_04389_b300.build` (there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    lib.slu_opts_default.argtypes = [C.POINTER(Opts)]
    lib.slu_opts_default.restype = None
    lib.slu_analyze.argtypes = [C.c_int64, P, P, C.POINTER(Opts), C.POINTER(P)]
    lib.slu_analyze_batch.argtypes = [C.c_int32, P, P, P, C.POINTER(Opts),
                                      C.POINTER(P)]
    lib.slu_analyze_device.argtypes = [C.c_int64, P, P, C.POINTER(Opts), P, C.POINTER(P)]
    lib.slu_analyze_batch_device.argtypes = [C.c_int32, P, P, P, C.POINTER(Opts), P,
                                             C.POINTER(P)]
    lib.slu_plan_query.argtypes = [P, C.POINTER(PlanInfo)]
    lib.slu_plan_export.argtypes = [P, P, P, P, P]
    lib.slu_plan_export_blocks.argtypes = [P, P, P, P, P, P]
    lib.slu_plan_export_tasks.argtypes = [P] + [P] * 10
    lib.slu_factor.argtypes = [P, P, P, C.POINTER(P), C.POINTER(FactorInfo)]
    lib.slu_refactor.argtypes = [P, P, P, C.POINTER(FactorInfo)]
    lib.slu_factor_batch.argtypes = [C.c_int32, P, P, P, P, C.POINTER(FactorInfo)]
    lib.slu_set_persistent.argtypes = [P, C.c_int32]
    lib.slu_set_persistent_solve.argtypes = [P, C.c_int32]
    lib.slu_persistent_tasks.argtypes = [P, P, C.c_int64, P]
    lib.slu_set_persistent_tasks.argtypes = [P, P, C.c_int64]
    lib.slu_reorder.argtypes = [C.c_int64, P, P, P, C.c_int32, C.c_int32, P, P, P, P]
    lib.slu_reorder_apply.argtypes = [C.c_int64, P, P, P, P, P, P, P, P, P, P]
    lib.slu_permute_scale.argtypes = [C.c_int64, C.c_int32, P, P, P, C.c_int64, P,
                                      C.c_int64, C.c_int32, P]
    lib.slu_select_regular_block.argtypes = [C.c_int64, C.c_int64]
    lib.slu_select_regular_block.restype = C.c_int32
    lib.slu_solve.argtypes = [P, P, C.c_int64, C.c_int32, P, C.c_int64, P,
                              C.POINTER(SolveInfo)]
    lib.slu_solve_transpose.argtypes = [P, P, C.c_int64, C.c_int32, P,
                                        C.c_int64, P]
    lib.slu_export_factors.argtypes = [P, P, P]
    lib.slu_grad_values.argtypes = [P, P, C.c_int64, P, C.c_int64, C.c_int32,
                                    P, P]
    lib.slu_set_profiling.argtypes = [P, C.c_int32]
    lib.slu_handle_stats.argtypes = [P, C.POINTER(Stats)]
    lib.slu_plan_flops.argtypes = [P, P]
    lib.slu_handle_trace.argtypes = [P, C.c_int64, P, P, P, P, P]
    lib.slu_set_graph.argtypes = [P, C.c_int32]
    lib.slu_solve_refine_noalloc.argtypes = [P, P, C.c_int64, C.c_int32, P,
                                             C.c_int64, P, C.POINTER(SolveInfo)]
    lib.slu_plan_serialize.argtypes = [P, P, C.POINTER(C.c_int64)]
    lib.slu_plan_deserialize.argtypes = [P, C.c_int64, C.POINTER(P)]
    lib.slu_plan_digest.argtypes = [P, C.POINTER(C.c_uint64)]
    lib.slu_plan_check.argtypes = [P]
    lib.slu_plan_destroy.argtypes = [P]
    lib.slu_plan_destroy.restype = None
    lib.slu_handle_destroy.argtypes = [P]
    lib.slu_handle_destroy.restype = None
    lib.slu_last_error.argtypes = []
    lib.slu_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("slu_opts_default", "slu_plan_destroy",
                        "slu_handle_destroy", "slu_last_error"):
            getattr(lib, name).restype = C.c_int
    return lib


lib = _load()


def _check(st, ok=(0,)):
    if st not in ok:
        raise SluError(st, lib.slu_last_error().decode())
    return st


def _np(a):
    return a.ctypes.data_as(C.c_void_p)


def default_opts(**kw):
    o = Opts()
    lib.slu_opts_default(C.byref(o))
    for k, v in kw.items():
        if k == "blocking" and isinstance(v, str):
            v = BLOCKING[v]
        if k == "precision" and isinstance(v, str):
            v = PRECISION[v]
        if k not in dict(Opts._fields_):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dev_ptr(t):
    import torch
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if t.dtype != torch.float64:
        raise ValueError(f"expected float64, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


def _values_ptr(t, nnz):
    """Device pointer of a value vector: float64, contiguous, exactly the
    plan's nnz(A) entries (the kernels read that many from the pointer)."""
    if t.dim() != 1 or t.shape[0] != nnz:
        raise ValueError(f"expected {nnz} values (the pattern's entries), "
                         f"got shape {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError("values must be contiguous")
    return _dev_ptr(t)


def _check_rows(t, n, what):
    if t.dim() not in (1, 2) or t.shape[0] != n:
        raise ValueError(f"{what} must have {n} rows, got shape {tuple(t.shape)}")


def _colmajor(B):
    """(tensor, leading dimension, columns, was_vector) in column-major."""
    if B.dim() == 1:
        Bc = B.contiguous()
        return Bc, max(1, Bc.shape[0]), 1, True
    n, k = B.shape
    if B.stride(0) == 1 and (k == 1 or B.stride(1) >= n):
        return B, (B.stride(1) if k > 1 else max(1, n)), k, False
    Bc = B.t().contiguous().t()
    return Bc, max(1, n), k, False


def _colmajor_empty(n, k, device):
    import torch
    X = torch.empty((k, n), dtype=torch.float64, device=device).t()
    return X, max(1, n)


def _pattern_arrays(n, colptr, rowidx):
    """Contiguous int64 colptr / int32 rowidx, long enough for what the
    library reads: colptr[0..n] and rowidx[0..colptr[n])."""
    cp = np.ascontiguousarray(colptr, dtype=np.int64)
    ri = np.ascontiguousarray(rowidx, dtype=np.int32)
    if n < 0:
        raise ValueError(f"n must be >= 0, got {n}")
    if cp.ndim != 1 or cp.shape[0] != n + 1:
        raise ValueError(f"colptr must have n + 1 = {n + 1} entries, "
                         f"got shape {cp.shape}")
    if ri.ndim != 1 or ri.shape[0] < max(int(cp[-1]), 0):
        raise ValueError(f"rowidx must have colptr[n] = {int(cp[-1])} entries, "
                         f"got shape {ri.shape}")
    return cp, ri


class Plan:
    """Result of the analysis (``slu_analyze``) of one sparsity pattern, or
    of a batch when ``n``, ``colptr`` and ``rowidx`` are lists.  With
    ``device=True`` the symbolic factorization and Algorithms 2 / 3 run on
    the current GPU (``slu_analyze_device``) on ``stream`` (the current
    torch stream when None); the plan is the same."""

    def __init__(self, n, colptr, rowidx, device=False, stream=None, **opts):
        self._h = C.c_void_p()
        self.device = bool(device)
        self._stream = stream
        if isinstance(n, (list, tuple)):          # batch of matrices
            return self._init_batch(n, colptr, rowidx, opts)
        self.n = int(n)
        self.colptr, self.rowidx = _pattern_arrays(self.n, colptr, rowidx)
        self.opts = default_opts(**opts)
        if self.device:
            _check(lib.slu_analyze_device(self.n, _np(self.colptr), _np(self.rowidx),
                                          C.byref(self.opts), _stream_ptr(stream),
                                          C.byref(self._h)))
        else:
            _check(lib.slu_analyze(self.n, _np(self.colptr), _np(self.rowidx),
                                   C.byref(self.opts), C.byref(self._h)))
        i = PlanInfo()
        _check(lib.slu_plan_query(self._h, C.byref(i)))
        self.info = _info_dict(i)

    @classmethod
    def from_bytes(cls, data):
        """A plan from ``to_bytes`` output (``slu_plan_deserialize``),
        without repeating the analysis."""
        self = cls.__new__(cls)
        self._h = C.c_void_p()
        self.device = False
        buf = np.frombuffer(memoryview(data).cast("B"), dtype=np.uint8)
        _check(lib.slu_plan_deserialize(_np(buf) if buf.size else None,
                                        buf.size, C.byref(self._h)))
        i = PlanInfo()
        _check(lib.slu_plan_query(self._h, C.byref(i)))
        self.info = _info_dict(i)
        self.n = int(self.info["n"])
        self.opts = None
        return self

    def _serialized(self):
        size = C.c_int64(0)
        _check(lib.slu_plan_serialize(self._h, None, C.byref(size)))
        buf = np.empty(size.value, np.uint8)
        _check(lib.slu_plan_serialize(self._h, _np(buf), C.byref(size)))
        return buf

    def to_bytes(self):
        """The plan as bytes (``slu_plan_serialize``), for a plan cache."""
        return self._serialized().tobytes()

    def save(self, path):
        """Write the serialized plan to a file (no intermediate copy)."""
        with open(path, "wb") as f:
            f.write(memoryview(self._serialized()))

    @classmethod
    def load(cls, path):
        """A plan from a file written by ``save``."""
        return cls.from_bytes(np.fromfile(path, dtype=np.uint8))

    def check(self):
        """Raise SluError unless every index the kernels take from the plan
        is in range (``slu_plan_check``)."""
        _check(lib.slu_plan_check(self._h))

    def digest(self):
        """64-bit checksum of the plan's contents (``slu_plan_digest``)."""
        d = C.c_uint64(0)
        _check(lib.slu_plan_digest(self._h, C.byref(d)))
        return d.value

    def _init_batch(self, ns, colptrs, rowidxs, opts):
        k = len(ns)
        if len(colptrs) != k or len(rowidxs) != k:
            raise ValueError(f"{k} orders but {len(colptrs)} colptr and "
                             f"{len(rowidxs)} rowidx arrays")
        self.members = [int(x) for x in ns]
        arrs = [_pattern_arrays(m, c, r)
                for m, c, r in zip(self.members, colptrs, rowidxs)]
        self._cps = [a[0] for a in arrs]
        self._ris = [a[1] for a in arrs]
        na = np.asarray(self.members, dtype=np.int64)
        cpa = (C.c_void_p * k)(*[c.ctypes.data for c in self._cps])
        ria = (C.c_void_p * k)(*[r.ctypes.data for r in self._ris])
        self.opts = default_opts(**opts)
        if self.device:
            _check(lib.slu_analyze_batch_device(k, _np(na), cpa, ria, C.byref(self.opts),
                                                _stream_ptr(self._stream), C.byref(self._h)))
        else:
            _check(lib.slu_analyze_batch(k, _np(na), cpa, ria, C.byref(self.opts),
                                         C.byref(self._h)))
        self.n = int(na.sum())
        i = PlanInfo()
        _check(lib.slu_plan_query(self._h, C.byref(i)))
        self.info = _info_dict(i)

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value:
            lib.slu_plan_destroy(self._h)
            self._h = C.c_void_p()

    def flops_by_class(self):
        """Algorithmic flops {getrf, panel, ssssm} of the factorization."""
        out = np.zeros(3)
        _check(lib.slu_plan_flops(self._h, _np(out)))
        return dict(zip(("getrf", "panel", "ssssm"), out.tolist()))

    def export(self):
        n, nnz, p = self.n, self.info["nnz_lu"], self.info["nblocks_1d"]
        bp = np.empty(n + 1, np.int64)
        ptr = np.empty(p + 1, np.int64)
        cp = np.empty(n + 1, np.int64)
        ri = np.empty(nnz, np.int32)
        _check(lib.slu_plan_export(self._h, _np(bp), _np(ptr), _np(cp), _np(ri)))
        return dict(blockptr=bp, ptr=ptr, colptr=cp, rowidx=ri)

    def export_blocks(self):
        nb, p = self.info["nblocks"], self.info["nblocks_1d"]
        bi = np.empty(nb, np.int32)
        bj = np.empty(nb, np.int32)
        bn = np.empty(nb, np.int64)
        de = np.empty(nb, np.uint8)
        lv = np.empty(p, np.int32)
        _check(lib.slu_plan_export_blocks(self._h, _np(bi), _np(bj), _np(bn),
                                          _np(de), _np(lv)))
        return dict(blocks=np.stack([bi, bj], 1), bnnz=bn,
                    dense=de.astype(bool), level=lv)

    def export_tasks(self):
        I = self.info
        L = I["nlevels"]
        out = {k: np.empty(L + 1, np.int64) for k in
               ("getrf_off", "gessm_off", "tstrf_off", "tgt_off")}
        out["getrf"] = np.empty(I["n_getrf"], np.int32)
        out["gessm"] = np.empty(2 * I["n_gessm"], np.int32)
        out["tstrf"] = np.empty(2 * I["n_tstrf"], np.int32)
        out["tgt"] = np.empty(2 * I["n_ssssm_targets"], np.int32)
        out["srcoff"] = np.empty(I["n_ssssm_targets"] + 1, np.int64)
        out["src"] = np.empty(I["n_ssssm_pairs"], np.int32)
        _check(lib.slu_plan_export_tasks(
            self._h, _np(out["getrf_off"]), _np(out["getrf"]),
            _np(out["gessm_off"]), _np(out["gessm"]), _np(out["tstrf_off"]),
            _np(out["tstrf"]), _np(out["tgt_off"]), _np(out["tgt"]),
            _np(out["srcoff"]), _np(out["src"])))
        return out


class Reordering:
    """``slu_reorder``: static-pivot matching and scaling (``scale``) and a
    nested-dissection ordering (``order``) of a general matrix (host CSC).
    ``matrix()`` gives the reordered CSC; ``rhs(b)`` / ``solution(y)`` map a
    CUDA right-hand side to the reordered system and its solution back
    (``slu_permute_scale``)."""

    def __init__(self, n, colptr, rowidx, values=None, scale=True, order=True,
                 leaf=64):
        self.n = int(n)
        self.colptr, self.rowidx = _pattern_arrays(self.n, colptr, rowidx)
        self.values = None if values is None else np.ascontiguousarray(values, np.float64)
        if self.values is not None and self.values.size != self.rowidx.size:
            raise ValueError("values must have one entry per pattern entry")
        flags = (1 if scale else 0) | (2 if order else 0)
        self.rowperm = np.zeros(self.n, np.int32)
        self.colperm = np.zeros(self.n, np.int32)
        self.rowscale = np.ones(self.n)
        self.colscale = np.ones(self.n)
        _check(lib.slu_reorder(self.n, _np(self.colptr), _np(self.rowidx),
                               None if self.values is None else _np(self.values),
                               flags, int(leaf), _np(self.rowperm), _np(self.colperm),
                               _np(self.rowscale), _np(self.colscale)))
        self._dev = None

    def matrix(self):
        """(colptr, rowidx, values) of the reordered, scaled matrix."""
        cp = np.zeros(self.n + 1, np.int64)
        ri = np.zeros(self.rowidx.size, np.int32)
        va = None if self.values is None else np.zeros(self.rowidx.size)
        _check(lib.slu_reorder_apply(
            self.n, _np(self.colptr), _np(self.rowidx),
            None if self.values is None else _np(self.values),
            _np(self.rowperm), _np(self.colperm), _np(self.rowscale),
            _np(self.colscale), _np(cp), _np(ri), None if va is None else _np(va)))
        return cp, ri, va

    def _device(self, device):
        import torch
        if self._dev is None:
            self._dev = tuple(torch.as_tensor(a, device=device) for a in
                              (self.rowperm, self.colperm, self.rowscale, self.colscale))
        return self._dev

    def _map(self, X, inverse, stream):
        import torch
        _check_rows(X, self.n, "X")
        Xc, ldx, k, vec = _colmajor(X)
        Y, ldy = _colmajor_empty(Xc.shape[0], k, Xc.device)
        rp, cpm, rs, cs = self._device(Xc.device)
        perm, sc = (cpm, cs) if inverse else (rp, rs)
        _check(lib.slu_permute_scale(self.n, k, C.c_void_p(perm.data_ptr()),
                                     C.c_void_p(sc.data_ptr()), _dev_ptr(Xc), ldx,
                                     _dev_ptr(Y), ldy, 1 if inverse else 0,
                                     _stream_ptr(stream)))
        return Y.reshape(-1) if vec else Y

    def rhs(self, B, stream=None):
        return self._map(B, False, stream)

    def solution(self, Y, stream=None):
        return self._map(Y, True, stream)


def factor_batch(plans, values, stream=None, allow_singular=False):
    """``slu_factor_batch``: independent plans factored in the same level
    walk; one Factor per plan (their factors equal ``Factor(plan, v)``'s)."""
    count = len(plans)
    if count != len(values):
        raise ValueError(f"{count} plans but {len(values)} value vectors")
    hp = (C.c_void_p * count)(*[p._h for p in plans])
    vp = (C.c_void_p * count)(*[_values_ptr(v, p.info["nnz_a"])
                                for p, v in zip(plans, values)])
    out = (C.c_void_p * count)()
    info = FactorInfo()
    st = lib.slu_factor_batch(count, hp, vp, _stream_ptr(stream), out,
                              C.byref(info))
    _check(st, (0, 4) if allow_singular else (0,))
    return [Factor._member(p, C.c_void_p(out[q]), values[q], st, info)
            for q, p in enumerate(plans)]


class Factor:
    """Factors of one matrix on the GPU (``slu_factor``)."""

    def __init__(self, plan, values, stream=None, allow_singular=False):
        self.plan = plan
        self._h = C.c_void_p()
        info = FactorInfo()
        st = lib.slu_factor(plan._h, _values_ptr(values, plan.info["nnz_a"]),
                            _stream_ptr(stream),
                            C.byref(self._h), C.byref(info))
        _check(st, (0, 4) if allow_singular else (0,))
        self.singular = st == 4
        self.values = values
        self.nperturb = info.nperturb
        self.tau = info.tau

    @classmethod
    def _member(cls, plan, handle, values, st, info):
        self = cls.__new__(cls)
        self.plan = plan
        self._h = handle
        self.singular = st == 4
        self.values = values
        self.nperturb = info.nperturb
        self.tau = info.tau
        return self

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value:
            lib.slu_handle_destroy(self._h)
            self._h = C.c_void_p()

    def refactor(self, values, stream=None, sync_info=False):
        info = FactorInfo() if sync_info else None
        _check(lib.slu_refactor(self._h,
                                _values_ptr(values, self.plan.info["nnz_a"]),
                                _stream_ptr(stream),
                                C.byref(info) if info is not None else None))
        self.values = values
        if info is not None:
            self.nperturb = info.nperturb

    def solve(self, B, stream=None, info=False, allow_not_converged=False):
        """X = A^{-1} B for a CUDA float64 tensor B of shape (n,) or (n, k)."""
        _check_rows(B, self.plan.n, "B")
        Bc, ldb, k, vec = _colmajor(B)
        X, ldx = _colmajor_empty(Bc.shape[0], k, Bc.device)
        si = SolveInfo()
        st = lib.slu_solve(self._h, _dev_ptr(Bc), ldb, k, _dev_ptr(X), ldx,
                           _stream_ptr(stream), C.byref(si) if info else None)
        _check(st, (0, 5) if allow_not_converged else (0,))
        out = X.reshape(-1) if vec else X
        if info:
            return out, {"iterations": si.iterations,
                         "backward_error": si.backward_error,
                         "converged": st == 0}
        return out

    def solve_transpose(self, G, stream=None):
        """Lam = A^{-T} G through the stored factors."""
        _check_rows(G, self.plan.n, "G")
        Gc, ldg, k, vec = _colmajor(G)
        L, ldl = _colmajor_empty(Gc.shape[0], k, Gc.device)
        _check(lib.slu_solve_transpose(self._h, _dev_ptr(Gc), ldg, k,
                                       _dev_ptr(L), ldl, _stream_ptr(stream)))
        return L.reshape(-1) if vec else L

    def grad_values(self, Lam, X, stream=None):
        """-sum_c Lam(row_p, c) X(col_p, c) over A's pattern (CSC order)."""
        import torch
        _check_rows(Lam, self.plan.n, "Lam")
        _check_rows(X, self.plan.n, "X")
        Lc, ldl, k, _ = _colmajor(Lam)
        Xc, ldx, k2, _ = _colmajor(X)
        if k != k2:
            raise ValueError(f"Lam has {k} columns, X has {k2}")
        out = torch.empty(self.plan.info["nnz_a"], dtype=torch.float64,
                          device=Lc.device)
        _check(lib.slu_grad_values(self._h, _dev_ptr(Lc), ldl, _dev_ptr(Xc),
                                   ldx, k, _dev_ptr(out), _stream_ptr(stream)))
        return out

    def set_graph(self, enable=True):
        """Replay refactor() from a recorded CUDA graph (needs a created
        stream, e.g. inside ``torch.cuda.stream(torch.cuda.Stream())``)."""
        _check(lib.slu_set_graph(self._h, 1 if enable else 0))

    def set_persistent(self, enable=True):
        """Run refactor()'s level walk as one persistent launch."""
        _check(lib.slu_set_persistent(self._h, 1 if enable else 0))

    def set_persistent_solve(self, enable=True):
        """Run every solve sweep as one persistent launch (per 4 RHS)."""
        _check(lib.slu_set_persistent_solve(self._h, 1 if enable else 0))

    def persistent_tasks(self):
        """The persistent launch's work list, int32 array (tasks, 7)."""
        n = np.zeros(1, np.int64)
        _check(lib.slu_persistent_tasks(self._h, None, 0, _np(n)))
        out = np.zeros((int(n[0]), 7), np.int32)
        _check(lib.slu_persistent_tasks(self._h, _np(out), int(n[0]), _np(n)))
        return out

    def set_persistent_tasks(self, tasks):
        t = np.ascontiguousarray(tasks, dtype=np.int32)
        if t.ndim != 2 or t.shape[1] != 7:
            raise ValueError("expected an int32 array of shape (tasks, 7)")
        _check(lib.slu_set_persistent_tasks(self._h, _np(t), t.shape[0]))

    def set_profiling(self, enable=True):
        _check(lib.slu_set_profiling(self._h, 1 if enable else 0))

    def stats(self):
        """Launch count and, while profiling, per-class event times (ms)."""
        st = Stats()
        _check(lib.slu_handle_stats(self._h, C.byref(st)))
        return {"launches": st.launches,
                "calls": dict(zip(KERNEL_CLASSES, list(st.calls))),
                "ms": dict(zip(KERNEL_CLASSES, list(st.ms)))}

    def trace(self, detail=False):
        """(classes, ms) of every launch profiled so far, in launch order;
        with ``detail`` also (levels, ctas): the factorization level of each
        launch (-1 outside the level loop) and its grid size (negative for
        the generic sparse kernels)."""
        n = np.zeros(1, np.int64)
        _check(lib.slu_handle_trace(self._h, 0, None, None, None, None, _np(n)))
        cls = np.empty(n[0], np.int32)
        ms = np.empty(n[0], np.float32)
        lv = np.empty(n[0], np.int32)
        ct = np.empty(n[0], np.int32)
        _check(lib.slu_handle_trace(self._h, n[0], _np(cls), _np(ms), _np(lv),
                                    _np(ct), _np(n)))
        return (cls, ms, lv, ct) if detail else (cls, ms)

    def export_factors(self, stream=None):
        """Factor values (FP64) in the order of ``plan.export()``'s pattern."""
        import torch
        out = torch.empty(self.plan.info["nnz_lu"], dtype=torch.float64,
                          device="cuda")
        _check(lib.slu_export_factors(self._h, _dev_ptr(out),
                                      _stream_ptr(stream)))
        return out
