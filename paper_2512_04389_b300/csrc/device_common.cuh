// Device-side helpers shared by the factorization and solve kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "slu_internal.hpp"

namespace slu {

// Device mirror of a plan's flat arrays (uploaded once per plan and device).
struct DevPlan {
    int device = -1;
    BlockDesc *bd = nullptr;
    int32_t *lcolptr = nullptr;
    uint16_t *lrow = nullptr;
    int32_t *dpos = nullptr, *sched = nullptr, *sgrp = nullptr;
    int32_t *lr_ptr = nullptr, *lr_pos = nullptr, *ps_task = nullptr, *pv_task = nullptr;
    uint16_t *lr_col = nullptr, *ne_col = nullptr, *ur_col = nullptr;
    int32_t *ur_ptr = nullptr, *ur_pos = nullptr;
    int64_t *ne_off = nullptr;
    int32_t *getrf = nullptr, *gessm = nullptr, *tstrf = nullptr;
    int32_t *gd = nullptr, *gs = nullptr;
    int32_t *dv_pos = nullptr, *dn_pos = nullptr;
    int32_t *tgt = nullptr, *src = nullptr;
    int64_t *srcoff = nullptr;
    int32_t *gm_task = nullptr, *gm_src = nullptr, *gg_tgt = nullptr,
            *gg_src = nullptr;
    uint32_t *gm_mask = nullptr;        // slice masks (FP64 plans), or null
    int64_t *gm_moff = nullptr;
    int64_t *gg_srcoff = nullptr;
    int64_t *a2s = nullptr, *f2s = nullptr;
    int64_t *a_rowptr = nullptr, *a_vpos = nullptr;
    int32_t *a_colidx = nullptr;
    int32_t *a_ri = nullptr, *a_ci = nullptr;   // A's entries: row, column
    int32_t *row_seg = nullptr;                  // batch member of each row
    int64_t *woff = nullptr;
    int32_t *inv_task = nullptr, *pd_task = nullptr, *pg_gessm = nullptr,
            *pg_tstrf = nullptr;
    int32_t *sp_pairs[4] = {nullptr, nullptr, nullptr, nullptr};
    int64_t *sp_poff[4] = {nullptr, nullptr, nullptr, nullptr};
    int64_t *sd_pair0[4] = {nullptr, nullptr, nullptr, nullptr};
    int64_t *lrow_off = nullptr, *urow_off = nullptr, *ucol_off = nullptr,
            *lcol_off = nullptr;
    int32_t *lrow_blk = nullptr, *urow_blk = nullptr, *ucol_blk = nullptr,
            *lcol_blk = nullptr;
};

// Row lists of the sparse diagonal blocks' strict lower (l*) and upper (u*)
// parts: row r of diagonal block I spans [p[doff + I + r], p[doff + I + r + 1])
// of the column (c) and value-slot (q) arrays.
struct RowLists {
    const int32_t *__restrict__ lp;
    const uint16_t *__restrict__ lc;
    const int32_t *__restrict__ lq;
    const int32_t *__restrict__ up;
    const uint16_t *__restrict__ uc;
    const int32_t *__restrict__ uq;
};

// Everything a block kernel needs to address block storage.
struct BlockArgs {
    const BlockDesc *__restrict__ bd;
    const int32_t *__restrict__ lcolptr;
    const uint16_t *__restrict__ lrow;
    const int32_t *__restrict__ dpos;
    const int32_t *__restrict__ sched;
    const int32_t *__restrict__ sgrp;
};

// Column jj of a block: value slots [vb, vb + cnt), local rows rows[t]
// (rows == nullptr for a dense tile, where the row of slot t is t).
__device__ __forceinline__ void colview(const BlockDesc &d, int jj,
                                        const BlockArgs &a, int64_t &vb,
                                        int &cnt, const uint16_t *&rows) {
    if (d.dense) {
        vb = d.voff + (int64_t)jj * d.ld;
        cnt = d.rows;
        rows = nullptr;
    } else {
        const int s = a.lcolptr[d.coff + jj];
        vb = d.voff + s;
        cnt = a.lcolptr[d.coff + jj + 1] - s;
        rows = a.lrow + d.roff + s;
    }
}

__device__ __forceinline__ int rowat(const uint16_t *rows, int t) {
    return rows ? (int)rows[t] : t;
}

// v != 0 (NaN counts as nonzero, -0 as zero) on the integer pipe: a double
// comparison runs on the FP64 pipe, which on B300 issues about two
// operations per SM and clock, so the zero tests that build skip masks use
// the bit pattern instead.
__device__ __forceinline__ bool nz(double v) {
    return (__double_as_longlong(v) & 0x7fffffffffffffffll) != 0;
}
__device__ __forceinline__ bool nz(float v) {
    return (__float_as_uint(v) & 0x7fffffffu) != 0;
}

// One element copied global -> shared by cp.async (sizeof(T) bytes, 4 or 8);
// with in == false nothing is read and the element is zero-filled.  The
// copies of a thread land by cp_async_wait_all; other threads see them after
// a barrier that follows it.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst, const T *src, bool in = true) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;"
                 :: "r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src), "n"((int)sizeof(T)),
                    "r"(in ? (int)sizeof(T) : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// Dynamic shared memory given to the kernels that stage blocks (one CTA per
// SM; the B300 limit per CTA is 227 KB).
constexpr size_t kStageSmem = 220 * 1024;

__host__ __device__ __forceinline__ size_t align16(size_t x) {
    return (x + 15) & ~size_t(15);
}

// One block seen column by column, either in place in global memory or as
// a copy staged in shared memory.  Column jj holds slots [off, off + cnt)
// of v with local rows rows[t] (rows == nullptr: dense, row of slot t is t).
template <typename T>
struct BlockView {
    const int32_t *cp;     // local colptr (cols + 1); nullptr when dense
    const uint16_t *rw;    // local rows of a sparse block
    T *v;                  // values
    const int32_t *dp;     // diagonal blocks: diagonal slot of each column
    int rows, ld;
    __device__ __forceinline__ void col(int jj, int &off, int &cnt,
                                        const uint16_t *&r) const {
        if (cp) {
            off = cp[jj];
            cnt = cp[jj + 1] - off;
            r = rw + off;
        } else {
            off = jj * ld;
            cnt = rows;
            r = nullptr;
        }
    }
};

// Stage block d into buf (cap bytes): its values, its local pattern and,
// for a diagonal block, its diagonal slots.  If the values do not fit, only
// the index data is staged and the values stay in global memory; if that
// does not fit either, the view is entirely global.  Called by all threads
// of the CTA; ends with __syncthreads() when anything was staged.
// *staged tells whether the values were staged (they must then be written
// back with unstage_block); *used receives the bytes taken from buf.
template <typename T>
__device__ BlockView<T> stage_block(const BlockDesc &d, const BlockArgs &a,
                                    T *val, unsigned char *buf, size_t cap,
                                    bool diag, bool *staged, size_t *used) {
    const int64_t nnz = d.dense ? (int64_t)d.ld * d.cols
                                : (int64_t)a.lcolptr[d.coff + d.cols];
    const size_t vbytes = align16(nnz * sizeof(T));
    const size_t ibytes = (diag ? align16((size_t)d.cols * 4) : 0) +
                          (d.dense ? 0 : align16((size_t)(d.cols + 1) * 4) +
                                             align16(nnz * 2));
    BlockView<T> v;
    v.rows = d.rows;
    v.ld = d.ld;
    v.cp = d.dense ? nullptr : a.lcolptr + d.coff;
    v.rw = d.dense ? nullptr : a.lrow + d.roff;
    v.v = val + d.voff;
    v.dp = diag ? a.dpos + d.doff : nullptr;
    *staged = false;
    *used = 0;
    const bool with_vals = vbytes + ibytes <= cap;
    if (!with_vals && (ibytes == 0 || ibytes > cap)) return v;
    unsigned char *p = buf;
    if (with_vals) {
        T *vv = reinterpret_cast<T *>(p);
        p += vbytes;
        for (int64_t e = threadIdx.x; e < nnz; e += blockDim.x) vv[e] = val[d.voff + e];
        v.v = vv;
        *staged = true;
    }
    if (diag) {
        int32_t *dp = reinterpret_cast<int32_t *>(p);
        p += align16((size_t)d.cols * 4);
        for (int e = threadIdx.x; e < d.cols; e += blockDim.x) dp[e] = a.dpos[d.doff + e];
        v.dp = dp;
    }
    if (!d.dense) {
        int32_t *cp = reinterpret_cast<int32_t *>(p);
        p += align16((size_t)(d.cols + 1) * 4);
        uint16_t *rw = reinterpret_cast<uint16_t *>(p);
        p += align16(nnz * 2);
        for (int e = threadIdx.x; e <= d.cols; e += blockDim.x) cp[e] = a.lcolptr[d.coff + e];
        for (int64_t e = threadIdx.x; e < nnz; e += blockDim.x) rw[e] = a.lrow[d.roff + e];
        v.cp = cp;
        v.rw = rw;
    }
    __syncthreads();
    *used = (size_t)(p - buf);
    return v;
}

// Copy a staged block's values back to global memory (all threads).
template <typename T>
__device__ void unstage_block(const BlockDesc &d, const BlockArgs &a,
                              const BlockView<T> &v, T *val) {
    const int64_t nnz = d.dense ? (int64_t)d.ld * d.cols
                                : (int64_t)a.lcolptr[d.coff + d.cols];
    __syncthreads();
    for (int64_t e = threadIdx.x; e < nnz; e += blockDim.x) val[d.voff + e] = v.v[e];
}

__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One thread: *c >= need within budget_ns (and 2^26 polls)?  The load is
// an acquire at GPU scope: what the counter's writers stored before their
// release is visible after it.
__device__ __forceinline__ bool wait_count(const int *c, int need, long long budget_ns) {
    const long long t0 = global_ns();
    for (int it = 0; it < (1 << 26); ++it) {
        int v;
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(c) : "memory");
        if (v >= need) return true;
        if (global_ns() - t0 > budget_ns) return false;
        __nanosleep(128);
    }
    return false;
}

inline bool cuda_ok(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return true;
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return false;
}

slu_status ensure_dev_plan(const slu_plan *P);
BlockArgs block_args(const slu_plan *P);

}  // namespace slu

namespace slu {
// One merged factorization behind the member handles of slu_factor_batch:
// the batch plan and its handle, freed with the last member handle.
struct BatchShared {
    slu_plan *plan = nullptr;
    slu_handle *h = nullptr;
    int refs = 0;
};
}  // namespace slu

// Handle: factor storage on one device plus refinement state.
struct slu_handle {
    const slu_plan *plan = nullptr;
    int device = -1;
    int prec = SLU_PREC_FP64;
    void *storage = nullptr;             // T[plan->storage]
    double *a_vals = nullptr;            // copy of A (FP64) for the residual
    double *scal = nullptr;              // [0] max|A|, [1] ||A||_inf
    unsigned long long *cnt = nullptr;   // [0] perturbed pivots, [1] zero pivot
    double tau_rel = 0.0;
    // member of a slu_factor_batch: storage, winv and a_vals point into the
    // shared batch handle's arrays (not owned)
    slu::BatchShared *batch = nullptr;
    // solve workspace (grown on demand)
    double *work = nullptr;
    int64_t work_elems = 0;
    double *red = nullptr;               // reduction scratch for refinement
    double *part = nullptr;              // solve partial sums (factor time)
    double *anorm_seg = nullptr;         // batch: ||A_q||_inf per member
    void *winv = nullptr;                // T[plan->wsize]: diagonal inverses
    // second stream for the deferred Schur updates, fork / join events
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // the level walk runs on a stream of the greatest priority, forked from
    // and joined back to the caller's stream
    cudaStream_t hi = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // solve graphs: the level sweeps of one solve, recorded once per
    // (right-hand side count, transposed) on a private stream over the
    // handle's vector buffer and replayed on the caller's stream
    struct SolveGraph { int nrhs; bool tr; cudaGraphExec_t exec; int64_t launches; };
    std::vector<SolveGraph> sgraphs;
    double *xbuf = nullptr;
    int64_t xbuf_cols = 0;
    cudaStream_t cap = nullptr;
    // graph mode
    bool use_graph = false;
    cudaGraphExec_t graph_exec = nullptr;
    const double *graph_values = nullptr;
    int64_t graph_launches = 0;         // kernels recorded in graph_exec
    bool capturing = false;
    // launch accounting and optional per-launch event timing
    int64_t launches = 0;
    bool profiling = false;
    struct Rec { int cls; cudaEvent_t a, b; int level, ctas; };
    int cur_level = -1;                  // factor level being launched, else -1
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;       // profiling events, reused
    size_t pool_next = 0;
    int64_t calls[SLU_KC_COUNT] = {0};
    double ms[SLU_KC_COUNT] = {0};
    // persistent launch: work list (5 ints per task), its counters and the
    // ticket, on the handle's device
    bool persistent = false;
    int32_t *ptasks = nullptr;
    int *pdone = nullptr;               // pcounters counters, then the ticket
    int64_t pntasks = 0, pcap = 0, pcounters = 0;
    // persistent solve: one work list per sweep (kStInts ints per task),
    // the counters of a sweep (2 p) and its ticket, on the handle's device
    // (levels run concurrently, so each sweep's partial sums get offsets
    // of their own: spoff, into spart of spart_elems doubles)
    bool persistent_solve = false;
    int32_t *stasks[4] = {nullptr, nullptr, nullptr, nullptr};
    int64_t *spoff[4] = {nullptr, nullptr, nullptr, nullptr};
    int64_t sntasks[4] = {0, 0, 0, 0};
    int *sdone = nullptr;
    double *spart = nullptr;
    int64_t spart_elems = 0;
    int sgrid[4] = {0, 0, 0, 0};        // persistent CTAs and shared memory
    size_t ssmem[4] = {0, 0, 0, 0};     // per sweep (set up when enabled)
};

namespace slu {
// Brackets one kernel launch: counts it and, when profiling, records a
// pair of events around it on `st`.
struct LaunchScope {
    slu_handle *h;
    int cls;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    int ctas;
    LaunchScope(const slu_handle *hc, int c, cudaStream_t s, int nctas = 0)
        : h(const_cast<slu_handle *>(hc)), cls(c), st(s), ctas(nctas) {
        h->launches++;
        if (h->profiling && !h->capturing) {
            while (h->pool.size() < h->pool_next + 2) {
                cudaEvent_t e;
                cudaEventCreate(&e);
                h->pool.push_back(e);
            }
            a = h->pool[h->pool_next++];
            b = h->pool[h->pool_next++];
            cudaEventRecord(a, st);
        }
    }
    ~LaunchScope() {
        if (a) {
            cudaEventRecord(b, st);
            h->recs.push_back({cls, a, b, h->cur_level, ctas});
        }
    }
};
}  // namespace slu
