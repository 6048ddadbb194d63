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
    int32_t *getrf = nullptr, *gessm = nullptr, *tstrf = nullptr;
    int32_t *tgt = nullptr, *src = nullptr;
    int64_t *srcoff = nullptr;
    int64_t *a2s = nullptr, *f2s = nullptr;
    int64_t *a_rowptr = nullptr, *a_vpos = nullptr;
    int32_t *a_colidx = nullptr;
    int64_t *lrow_off = nullptr, *urow_off = nullptr, *ucol_off = nullptr,
            *lcol_off = nullptr;
    int32_t *lrow_blk = nullptr, *urow_blk = nullptr, *ucol_blk = nullptr,
            *lcol_blk = nullptr;
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

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

inline bool cuda_ok(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return true;
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return false;
}

slu_status ensure_dev_plan(const slu_plan *P);
BlockArgs block_args(const slu_plan *P);

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
    // solve workspace (grown on demand)
    double *work = nullptr;
    int64_t work_elems = 0;
    double *red = nullptr;               // reduction scratch for refinement
    // launch accounting and optional per-launch event timing
    int64_t launches = 0;
    bool profiling = false;
    struct Rec { int cls; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    int64_t calls[SLU_KC_COUNT] = {0};
    double ms[SLU_KC_COUNT] = {0};
};

namespace slu {
// Brackets one kernel launch: counts it and, when profiling, records a
// pair of events around it on `st`.
struct LaunchScope {
    slu_handle *h;
    int cls;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    LaunchScope(const slu_handle *hc, int c, cudaStream_t s)
        : h(const_cast<slu_handle *>(hc)), cls(c), st(s) {
        h->launches++;
        if (h->profiling) {
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            cudaEventRecord(a, st);
        }
    }
    ~LaunchScope() {
        if (a) {
            cudaEventRecord(b, st);
            h->recs.push_back({cls, a, b});
        }
    }
};
}  // namespace slu
