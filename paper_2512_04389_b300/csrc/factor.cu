// Numerical factorization on the GPU: the right-looking blocked LU of
// Section 2.2 (Algorithm 1) over the plan's non-empty blocks, one level of
// the block dependency DAG at a time.  Per level:
//   GETRF  one CTA per diagonal block B_II -> L_II U_II (no row exchange;
//          the pivot test in FP64; |pivot| < tau replaced by +-tau and
//          counted): k_getrf_dense (dense storage, zero-skipping or
//          one-barrier dense steps) or k_getrf (sparse storage);
//   inverses of the dense diagonal factors (k_inv), used by the panels and
//          by the solves;
//   panels GESSM U_IJ = L_II^{-1} B_IJ and TSTRF L_JI = B_JI U_II^{-1}:
//          products with the inverses (k_panel_inv), per-lane substitution
//          for dense panels (k_panel_vec), height-group kernels for sparse
//          panels of sparse diagonal blocks (k_panel_grp), a right-looking
//          fallback (k_panel);
//   SSSSM  B_KJ -= sum_I L_KI U_IJ over the level's sources in ascending I
//          (deterministic, no atomics): dense tiles on the FP64 pipe
//          (k_ssssm_gemm) or the tcgen05 tensor cores (k_ssssm_tc, FP32),
//          the rest column by column (k_ssssm).  The updates the next level
//          does not read run on a second stream, overlapping it.
// Closure of the pattern under fill guarantees that every update lands on a
// stored slot; entries outside the pattern of a dense block are exact zeros
// and stay zero.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "device_common.cuh"

namespace slu {

// ---------------------------------------------------------------- kernels

// out = max |v| (as the bit pattern of a non-negative double, which orders
// like the value); *bad = 1 when some value is NaN or infinite.
__global__ void k_maxabs(int64_t n, const double *__restrict__ v,
                         unsigned long long *__restrict__ out,
                         unsigned long long *__restrict__ bad) {
    double m = 0.0;
    bool nonfinite = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double a = fabs(v[i]);
        nonfinite |= !(a <= 1.7976931348623157e308);   // NaN or inf
        m = fmax(m, a);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(~0u, m, o));
    if (__any_sync(~0u, nonfinite) && (threadIdx.x & 31) == 0) atomicOr(bad, 1ull);
    if ((threadIdx.x & 31) == 0 && m > 0.0)
        atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// ||A||_inf = max_i sum_j |a_ij| over the CSR view of A.
__global__ void k_anorm(int64_t n, const int64_t *__restrict__ rp,
                        const int64_t *__restrict__ vpos,
                        const double *__restrict__ v,
                        unsigned long long *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double s = 0.0;
    if (i < n)
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) s += fabs(v[vpos[q]]);
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(~0u, s, o));
    if ((threadIdx.x & 31) == 0 && s > 0.0)
        atomicMax(out, (unsigned long long)__double_as_longlong(s));
}

// Batch: ||A_q||_inf per member q (row sums of the member's rows).
__global__ void k_anorm_seg(int64_t n, const int64_t *__restrict__ rp,
                            const int64_t *__restrict__ vpos,
                            const double *__restrict__ v,
                            const int32_t *__restrict__ row_seg,
                            unsigned long long *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q) s += fabs(v[vpos[q]]);
    if (s > 0.0) atomicMax(&out[row_seg[i]], (unsigned long long)__double_as_longlong(s));
}

template <typename T>
__global__ void k_scatter(int64_t n, const int64_t *__restrict__ a2s,
                          const double *__restrict__ v, T *__restrict__ val) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        val[a2s[i]] = (T)v[i];
}

template <typename T>
__global__ void k_export(int64_t n, const int64_t *__restrict__ f2s,
                         const T *__restrict__ val, double *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)val[f2s[i]];
}


// Slot of local row r in a column with sorted local rows (dense: r itself);
// -1 when absent.
__device__ __forceinline__ int find_row(const uint16_t *rows, int cnt, int r) {
    if (!rows) return r < cnt ? r : -1;
    int lo = 0, hi = cnt - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int v = rows[mid];
        if (v == r) return mid;
        if (v < r) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}


// Column update vj(slot of row rs[t]) -= ls[t] * u for t < n, lanes over t.
// The source column (rows rs, values ls) sits in shared memory; the target
// column (rows rj, cj slots, values vj) may be in shared or global memory.
// Each lane first finds and loads up to 4 target slots, then writes them,
// so several global round trips are in flight at once.
template <typename T>
__device__ __forceinline__ void axpy_rows(T *vj, const uint16_t *rj, int cj,
                                          const uint16_t *rs, const T *ls,
                                          int n, T u, int lane) {
    for (int t0 = 0; t0 < n; t0 += 128) {
        int pr[4];
        T bv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int t = t0 + q * 32 + lane;
            pr[q] = t < n ? find_row(rj, cj, rs[t]) : -1;
            bv[q] = pr[q] >= 0 ? vj[pr[q]] : T(0);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int t = t0 + q * 32 + lane;
            if (pr[q] >= 0) vj[pr[q]] = (T)(bv[q] - ls[t] * u);
        }
    }
}

// Dense diagonal block: right-looking LU with the whole CTA.  Step k fixes
// the pivot (FP64, perturbation as in the sparse path), scales L(k+1:, k)
// and applies the rank-1 update to the trailing block.  Entries outside the
// symbolic pattern are exact zeros and stay zero.
// Pivot of step k: the FP64 test |piv| < tau and the +-tau replacement
// (sign of zero taken as +), counted once; returns the value to store.
// The tests run on the bit patterns (integer pipe): |piv| and tau >= 0 order
// like their patterns, a NaN pivot is never below tau, and -0 counts as +0.
__device__ __forceinline__ double fix_pivot(double piv, double tau,
                                           unsigned long long *cnt) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(piv);
    const unsigned long long mag = bits & 0x7fffffffffffffffull;
    const unsigned long long t = (unsigned long long)__double_as_longlong(tau);
    if (t != 0 && mag < t) {
        atomicAdd(&cnt[0], 1ull);
        return (mag != 0 && (bits >> 63)) ? -tau : tau;
    }
    if (mag == 0) atomicOr(&cnt[1], 1ull);
    return piv;
}

// Dense-stored diagonal block, right-looking LU that skips exact zeros.
// Storage is split: entry (r, c) with r, c >= p0 lives in shared memory S
// (column-major, leading dimension ls), the rest in the block's global
// storage G (leading dimension ld, L2-resident).  Step k, two barriers:
//   1. warp 0 scales L(k+1:, k) by the published reciprocal pivot and
//      compacts its nonzeros by ballot into a (row, value) list; warp 1
//      compacts the nonzeros of U(k, k+1:) into a (column, value) list;
//   2. all threads apply B(r, c) -= L(r, k) U(k, c) over the list product
//      (lane groups per column, four updates in flight per thread); thread
//      0 owns the product's first entry, (k+1, k+1) when that is updated,
//      and then fixes pivot k+1 (FP64 test and perturbation) and publishes
//      its reciprocal.
// The terms left out are exact zeros, so the result is that of the dense
// right-looking LU; a blocked tile skip would keep most of them, because
// the fill of a coarse block is scattered along its elimination tree.
#ifdef SLU_SELFCHECK
// checked builds only: bit 0 entry index, bit 1 list index, bit 2 update
__device__ unsigned long long g_selfcheck;
__device__ double g_selfcheck_sink[4];
extern "C" unsigned long long slu_selfcheck_read() {
    unsigned long long v = 0;
    cudaMemcpyFromSymbol(&v, g_selfcheck, sizeof(v));
    return v;
}
#define SLU_CHECK(cond, bit) \
    do { if (!(cond)) atomicOr(&g_selfcheck, 1ull << (bit)); } while (0)
#else
#define SLU_CHECK(cond, bit) do { } while (0)
#endif

template <typename T>
struct SplitBlock {
    T *G;
    int64_t ld;
    T *S;
    int ls, p0, n;
    __device__ __forceinline__ T &at(int r, int c) const {
#ifdef SLU_SELFCHECK
        if (r < 0 || c < 0 || r >= n || c >= n) {
            atomicOr(&g_selfcheck, 1ull);
            return reinterpret_cast<T *>(g_selfcheck_sink)[0];
        }
#endif
        return (r >= p0 && c >= p0) ? S[(int64_t)(c - p0) * ls + (r - p0)]
                                    : G[(int64_t)c * ld + r];
    }
};

// Shared-memory bytes of the step lists for a b-row block.
__host__ __device__ constexpr size_t lu_list_bytes(int b, size_t esz) {
    return 2 * (size_t)b * (esz + 2) + 64;
}

// One warp: compact the nonzeros of entries k+1..b-1 of a column (col =
// true: (r, k)) or of a row ((k, c)) into a (index, value) list; a column's
// listed values are then scaled by rcp and stored back (L(:, k)), one FP64
// multiply per 32 listed entries rather than per 32 rows scanned.
template <typename T>
__device__ __forceinline__ int lu_compact(const SplitBlock<T> &B, int b, int k,
                                          bool col, T rcp, T *X, uint16_t *I) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    int n = 0;
    for (int i0 = k + 1; i0 < b; i0 += 128) {
        T v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + 32 * q + lane;
            v[q] = i < b ? (col ? B.at(i, k) : B.at(k, i)) : T(0);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + 32 * q + lane;
            // only entries inside the block are listed
            const bool live = i < b && nz(v[q]);
            const unsigned m = __ballot_sync(0xffffffffu, live);
            if (live) {
                const int p = n + __popc(m & lt);
                SLU_CHECK(p < b && i < b, 1);
                I[p] = (uint16_t)i;
                X[p] = v[q];
            }
            n += __popc(m);
        }
    }
    if (col) {
        __syncwarp();
        for (int p = lane; p < n; p += 32) {
            const T l = X[p] * rcp;
            X[p] = l;
            B.at(I[p], k) = l;
        }
    }
    return n;
}

template <typename T>
__device__ void lu_skip(const SplitBlock<T> &B, int b, unsigned char *lists,
                        double tau, unsigned long long *cnt) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    const int warp = tid >> 5, nw = nt >> 5;
    T *Lv = reinterpret_cast<T *>(lists), *Uv = Lv + b;
    uint16_t *R = reinterpret_cast<uint16_t *>(Uv + b), *C = R + b;
    __shared__ T s_pinv;
    __shared__ int s_nR, s_nC;
    if (tid == 0 && b > 0) {
        const T pv = (T)fix_pivot((double)B.at(0, 0), tau, cnt);
        B.at(0, 0) = pv;
        s_pinv = T(1) / pv;
    }
    __syncthreads();
    for (int k = 0; k + 1 < b; ++k) {
        if (warp == 0) {
            const int n = lu_compact<T>(B, b, k, true, s_pinv, Lv, R);
            if (lane == 0) s_nR = n;
        } else if (warp == 1) {
            const int n = lu_compact<T>(B, b, k, false, T(0), Uv, C);
            if (lane == 0) s_nC = n;
        }
        __syncthreads();
        const int nR = s_nR, nC = s_nC;
        if (nR > 0) {
            const int g = nR > 16 ? 32 : nR > 8 ? 16 : nR > 4 ? 8 : nR > 2 ? 4 : nR > 1 ? 2 : 1;
            const int cpw = 32 / g, sub = lane / g, li = lane & (g - 1);
            for (int ci = warp * cpw + sub; ci < nC; ci += nw * cpw) {
                const int c = C[ci];
                const T u = Uv[ci];
                const bool cs = c >= B.p0;
                T *colG = B.G + (int64_t)c * B.ld;
                T *colS = cs ? B.S + (int64_t)(c - B.p0) * B.ls - B.p0 : B.S;
                if (nR > 2 * g) {           // uniform: four updates in flight
                    for (int r0 = li; r0 < nR; r0 += 4 * g) {
                        T *q[4];
                        T x[4], l[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int ri = r0 + j * g;
                            if (ri < nR) {
                                const int r = R[ri];
                                SLU_CHECK(r > k && r < b && c > k && c < b && ri < b && ci < b, 2);
                                q[j] = (cs && r >= B.p0) ? colS + r : colG + r;
                                x[j] = *q[j];
                                l[j] = Lv[ri];
                            }
                        }
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            if (r0 + j * g < nR) *q[j] = x[j] - l[j] * u;
                    }
                } else {                    // one or two rows per lane: no idle FP64 issue
                    for (int ri = li; ri < nR; ri += g) {
                        const int r = R[ri];
                        SLU_CHECK(r > k && r < b && c > k && c < b && ri < b && ci < b, 2);
                        T *q = (cs && r >= B.p0) ? colS + r : colG + r;
                        *q = *q - Lv[ri] * u;
                    }
                }
            }
        }
        if (tid == 0) {
            T &p = B.at(k + 1, k + 1);
            const T pv = (T)fix_pivot((double)p, tau, cnt);
            p = pv;
            s_pinv = T(1) / pv;
        }
        __syncthreads();
    }
}

// Dense LU of a block held whole in shared memory, one CTA barrier per
// step (FP32 storage, where the step chain, not arithmetic, is the bound).
// Step k: every thread reads the pivot A(k, k) (final after step k-1),
// applies the small-pivot test itself (thread 0 counts it) and forms the
// reciprocal; warps over columns c > k with U(k, c) != 0, lanes over rows:
// A(r, c) -= A(r, k) (U(k, c) / pivot).  Column k is read unscaled in step
// k; its scaling by the reciprocal (L(:, k)) and the write of the fixed
// pivot are deferred to step k+1, when nothing reads column k.
// The test |p| < tau is the FP64 one, taken in FP32 without FP64
// instructions: for a float x, x < tau exactly when x < tau_up, the
// smallest float >= tau; the replacement is tau rounded to FP32.
template <typename T>
__device__ void lu_dense_smem(T *S, int b, int ls, double tau,
                              unsigned long long *cnt) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nw = blockDim.x >> 5;
    const float tau_up = __double2float_ru(tau), tau_rn = (float)tau;
    T prev_rcp = T(0), prev_piv = T(0);
    for (int k = 0; k < b; ++k) {
        const T p = S[(int64_t)k * ls + k];
        const bool small = tau_up > 0.0f && fabsf((float)p) < tau_up;
        const T piv = small ? (T)(p >= T(0) ? tau_rn : -tau_rn) : p;
        const T rcp = T(1) / piv;
        if (tid == 0) {
            if (small) atomicAdd(&cnt[0], 1ull);
            else if (p == T(0)) atomicOr(&cnt[1], 1ull);
        }
        if (k > 0 && warp == ((k - 1) % nw)) {      // deferred: column k-1
            T *c = S + (int64_t)(k - 1) * ls;
            for (int r = k + lane; r < b; r += 32) c[r] *= prev_rcp;
            if (lane == 0) c[k - 1] = prev_piv;
        }
        const T *ck = S + (int64_t)k * ls;
        for (int c = k + 1 + warp; c < b; c += nw) {
            T *cc = S + (int64_t)c * ls;
            const T u = cc[k] * rcp;
            if (u == T(0)) continue;                    // uniform across the warp
            for (int r = k + 1 + lane; r < b; r += 32) cc[r] -= ck[r] * u;
        }
        prev_rcp = rcp;
        prev_piv = piv;
        __syncthreads();
    }
    if (b > 0 && warp == ((b - 1) % nw) && lane == 0) S[(int64_t)(b - 1) * ls + b - 1] = prev_piv;
    __syncthreads();
}

// Dense LU of an FP64 block held whole in shared memory with no CTA barrier
// between steps.  Column c belongs to warp c % nw, which alone updates it.
// Step k needs the pivot's reciprocal and the list of the nonzeros below the
// pivot in column k (rows and unscaled values), published by the owner of
// column k: in step k - 1 that warp updates column k first, fixes the pivot
// (the FP64 test on the bit pattern), forms the reciprocal, lists the column,
// scales it in place (L(:, k)) and sets `ready` = k -- while the other warps
// still update their columns of step k - 1, so the reciprocal's latency is
// off their path.  Every warp waits (lane 0, bounded) for ready >= k, then
// updates its columns c > k over the listed rows: A(r, c) -= a(r, k) u with
// u = U(k, c) / pivot.  A warp can fall behind only until it reaches the next
// column it owns, at most nw steps ahead of it, so kLuRing >= nw + 2 list
// slots are never written while still read.  A wait that runs out sets bit
// 3 of cnt[2] and the warp stops.
constexpr int kLuRing = 32;
__host__ __device__ constexpr size_t lu_owner_bytes(int b) {
    return (size_t)b * (b | 1) * sizeof(double) + (size_t)kLuRing * b * (sizeof(double) + 2);
}

__device__ void lu_owner(double *S, int b, int ls, double tau, unsigned long long *cnt,
                         unsigned char *ring) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    double *Lv = reinterpret_cast<double *>(ring);                       // kLuRing x b
    uint16_t *R = reinterpret_cast<uint16_t *>(Lv + (size_t)kLuRing * b); // kLuRing x b
    __shared__ double s_rcp[kLuRing];
    __shared__ int s_n[kLuRing];
    __shared__ volatile int s_ready;
    if (threadIdx.x == 0) s_ready = -1;
    __syncthreads();
    // the owner of column k, whole warp: the pivot's division is issued
    // first and runs while the unscaled column is listed; the list and the
    // reciprocal are published, and the column is scaled (L(:, k)) after
    auto publish = [&](int k) {
        double rc = 0.0;
        if (lane == 0) {
            double &p = S[(int64_t)k * ls + k];
            const double pv = fix_pivot(p, tau, cnt);
            p = pv;
            rc = 1.0 / pv;
        }
        const int slot = k % kLuRing;
        double *lv = Lv + (size_t)slot * b;
        uint16_t *rr = R + (size_t)slot * b;
        double *col = S + (int64_t)k * ls;
        int n = 0;
        for (int i0 = k + 1; i0 < b; i0 += 32) {
            const int i = i0 + lane;
            const double v = i < b ? col[i] : 0.0;
            const bool live = i < b && nz(v);
            const unsigned m = __ballot_sync(0xffffffffu, live);
            if (live) {
                const int q = n + __popc(m & lt);
                rr[q] = (uint16_t)i;
                lv[q] = v;
            }
            n += __popc(m);
        }
        rc = __shfl_sync(0xffffffffu, rc, 0);
        if (lane == 0) {
            s_rcp[slot] = rc;
            s_n[slot] = n;
        }
        __syncwarp();
        __threadfence_block();
        if (lane == 0) s_ready = k;
        for (int q = lane; q < n; q += 32) col[rr[q]] = lv[q] * rc;
    };
    if (warp == 0 && b > 0) publish(0);
    for (int k = 0; k + 1 < b; ++k) {
        int ok = 1;
        if (lane == 0) {
            // the owner of column k + 1 is on the step chain and spins hot;
            // the other warps back off, leaving it the issue slots
            const bool next = warp == (k + 1) % nw;
            for (int it = 0; s_ready < k; ++it) {
                if (it >= (1 << 22)) {
                    atomicOr(&cnt[2], 8ull);
                    ok = 0;
                    break;
                }
                if (!next || it >= 4096) __nanosleep(next ? 64 : 200);
            }
        }
        if (!__shfl_sync(0xffffffffu, ok, 0)) break;
        __syncwarp();
        __threadfence_block();
        const int slot = k % kLuRing;
        const int nR = s_n[slot];
        const double rc = s_rcp[slot];
        const double *lv = Lv + (size_t)slot * b;
        const uint16_t *rr = R + (size_t)slot * b;
        // this warp's columns c > k, the first of them k + 1 when owned
        const int c0 = k + 1 + (((warp - (k + 1)) % nw) + nw) % nw;
        for (int c = c0; c < b; c += nw) {
            double *cc = S + (int64_t)c * ls;
            const double a = cc[k];                     // U(k, c), final
            if (nR > 0 && nz(a)) {                      // uniform across the warp
                const double u = a * rc;
                for (int ri = lane; ri < nR; ri += 32) {
                    const int r = rr[ri];
                    cc[r] -= lv[ri] * u;
                }
            }
            if (c == k + 1) {
                __syncwarp();
                publish(k + 1);
            }
        }
    }
    __syncthreads();
}

// Dense diagonal block b x b at g (leading dimension ld): stage the largest
// trailing square that fits next to the step lists, factor, write back.
template <typename T>
__device__ void getrf_dense(T *g, int b, int64_t ld, double tau,
                            unsigned long long *cnt, unsigned char *smem,
                            size_t cap) {
    const size_t lb = align16(lu_list_bytes(b, sizeof(T)));
    int ms = 0;
    if (cap > lb) {
        ms = (int)sqrt((double)((cap - lb) / sizeof(T)));
        while (ms > 0 && (size_t)ms * (ms | 1) * sizeof(T) > cap - lb) --ms;
        ms = min(ms, b);
    }
    if constexpr (sizeof(T) == 8) {
        if (b <= 128 && lu_owner_bytes(b) <= cap) {
            // FP64 block that fits whole with the list ring: owned columns,
            // no barrier between steps
            const int ls = b | 1;
            double *S = reinterpret_cast<double *>(smem);
            for (int e = threadIdx.x; e < b * b; e += blockDim.x)
                cp_async_elem(&S[(e / b) * ls + e % b], &g[(int64_t)(e / b) * ld + e % b]);
            cp_async_wait_all();
            __syncthreads();
            lu_owner(S, b, ls, tau, cnt, smem + (size_t)b * ls * sizeof(double));
            for (int e = threadIdx.x; e < b * b; e += blockDim.x)
                g[(int64_t)(e / b) * ld + e % b] = S[(e / b) * ls + e % b];
            return;
        }
    }
    if (sizeof(T) == 4 && (size_t)b * b * sizeof(T) <= cap) {
        // FP32 block that fits whole: dense steps with one barrier each
        T *S = reinterpret_cast<T *>(smem);
        for (int e = threadIdx.x; e < b * b; e += blockDim.x)
            cp_async_elem(&S[e], &g[(int64_t)(e / b) * ld + e % b]);
        cp_async_wait_all();
        __syncthreads();
        lu_dense_smem<T>(S, b, b, tau, cnt);
        for (int e = threadIdx.x; e < b * b; e += blockDim.x)
            g[(int64_t)(e / b) * ld + e % b] = S[e];
        return;
    }
    const int p0 = b - ms, ls = ms | 1;
    T *S = reinterpret_cast<T *>(smem + lb);
    for (int e = threadIdx.x; e < ms * ms; e += blockDim.x) {
        const int r = e % ms, c = e / ms;
        cp_async_elem(&S[c * ls + r], &g[(int64_t)(p0 + c) * ld + p0 + r]);
    }
    cp_async_wait_all();
    __syncthreads();
    const SplitBlock<T> B{g, ld, S, ls, p0, b};
    lu_skip<T>(B, b, smem, tau, cnt);
    for (int e = threadIdx.x; e < ms * ms; e += blockDim.x) {
        const int r = e % ms, c = e / ms;
        g[(int64_t)(p0 + c) * ld + p0 + r] = S[c * ls + r];
    }
}

// Sparse-stored diagonal block with few height groups: left-looking by
// columns, the columns of one height in parallel (one warp each), a CTA
// barrier between heights.  Column jj: x = B(:, jj) in a per-warp dense
// vector; for each m < jj with U(m, jj) stored, ascending, x(m) is final and
// x(rows of L(:, m)) -= L(:, m) x(m) (column m has a smaller height, so it
// is finished); then U(:, jj) = x(<= jj), pivot x(jj) fixed in FP64 and
// L(:, jj) = x(> jj) / pivot.
template <typename T>
__device__ void getrf_sparse_groups(const BlockDesc &d, const BlockArgs &a,
                                    T *val, unsigned char *smem, double tau,
                                    unsigned long long *cnt) {
    const int m = d.rows, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    T *x = reinterpret_cast<T *>(smem) + (size_t)warp * m;
    const size_t xbytes = align16((size_t)nw * m * sizeof(T));
    bool staged;
    size_t used;
    const BlockView<T> B = stage_block<T>(d, a, val, smem + xbytes,
                                          kStageSmem - xbytes, true, &staged, &used);
    for (int i = lane; i < m; i += 32) x[i] = T(0);
    __syncwarp();
    const int32_t *sched = a.sched + d.doff;
    const int32_t *grp = a.sgrp + d.goff;
    for (int g = 0; g < d.ngroups; ++g) {
        for (int t = grp[g] + warp; t < grp[g + 1]; t += nw) {
            const int jj = sched[t];
            int oj, cj;
            const uint16_t *rj;
            B.col(jj, oj, cj, rj);
            const int dj = B.dp[jj];
            for (int e = lane; e < cj; e += 32) x[rj[e]] = B.v[oj + e];
            __syncwarp();
            for (int e = 0; e < dj; ++e) {
                const int mm = rj[e];
                const T xm = x[mm];
                if (xm == T(0)) continue;
                int om, cm;
                const uint16_t *rm;
                B.col(mm, om, cm, rm);
                const int dm = B.dp[mm];
                for (int q = dm + 1 + lane; q < cm; q += 32) x[rm[q]] -= B.v[om + q] * xm;
                __syncwarp();
            }
            T piv = T(0);
            if (lane == 0) piv = (T)fix_pivot((double)x[jj], tau, cnt);
            piv = __shfl_sync(0xffffffffu, piv, 0);
            const T rcp = T(1) / piv;
            for (int e = lane; e < cj; e += 32) {
                const int r = rj[e];
                const T v = r < jj ? x[r] : r == jj ? piv : x[r] * rcp;
                B.v[oj + e] = v;
                x[r] = T(0);
            }
            __syncwarp();
        }
        __syncthreads();
    }
    if (staged) unstage_block<T>(d, a, B, val);
}

// GETRF on dense-stored diagonal blocks, one CTA of kDenseLuThreads per block.
constexpr int kDenseLuThreads = 512;
template <typename T>
__global__ void __launch_bounds__(kDenseLuThreads, 1)
k_getrf_dense(const int32_t *__restrict__ ids, const BlockDesc *__restrict__ bd,
              T *__restrict__ val, const double *__restrict__ scal,
              double tau_rel, unsigned long long *__restrict__ cnt, size_t cap) {
    extern __shared__ __align__(16) unsigned char smem[];
    const BlockDesc d = bd[ids[blockIdx.x]];
    getrf_dense<T>(val + d.voff, d.rows, d.ld, tau_rel * scal[0], cnt, smem, cap);
}

// GETRF on sparse-stored diagonal blocks, one CTA per block: by height
// groups (getrf_sparse_groups) when the block's column DAG has on average
// at least four columns per height, else right-looking step by step.
// Arithmetic in the storage type; the pivot test and perturbation in FP64.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_getrf(const int32_t *__restrict__ ids, BlockArgs a, T *__restrict__ val,
        const double *__restrict__ scal, double tau_rel,
        unsigned long long *__restrict__ cnt) {
    const BlockDesc d = a.bd[ids[blockIdx.x]];
    extern __shared__ __align__(16) unsigned char smem[];
    const double tau = tau_rel * scal[0];
    if (4 * d.ngroups <= d.rows) {
        getrf_sparse_groups<T>(d, a, val, smem, tau, cnt);
        return;
    }
    // Sparse diagonal block, right-looking with the whole CTA: step k fixes
    // the pivot, scales L(k+1:, k), and applies the rank-1 update
    // B(r, j) -= L(r, k) U(k, j) for r, j in the rows of L(:, k) below the
    // diagonal (the columns of U(k, :) by symmetry of the pattern); one
    // warp per column j, lanes over rows r, slots found by binary search.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ double s_piv;
    // source column buffer (values, rows), then the staged block
    T *sv = reinterpret_cast<T *>(smem);
    uint16_t *sr = reinterpret_cast<uint16_t *>(sv + d.rows);
    const size_t sbytes = align16((size_t)d.rows * (sizeof(T) + 2));
    bool staged;
    size_t used;
    const BlockView<T> B = stage_block<T>(d, a, val, smem + sbytes,
                                          kStageSmem - sbytes, true, &staged,
                                          &used);
    for (int k = 0; k < d.rows; ++k) {
        int ok, ck;
        const uint16_t *rk;
        B.col(k, ok, ck, rk);
        const int dk = B.dp[k];
        const int nL = ck - dk - 1;
        if (threadIdx.x == 0) {
            const double piv = fix_pivot((double)B.v[ok + dk], tau, cnt);
            B.v[ok + dk] = (T)piv;
            s_piv = 1.0 / piv;
        }
        __syncthreads();
        if (nL == 0) continue;
        const T pinv = (T)s_piv;
        for (int e = threadIdx.x; e < nL; e += blockDim.x) {
            const T l = B.v[ok + dk + 1 + e] * pinv;
            B.v[ok + dk + 1 + e] = l;
            sv[e] = l;
            sr[e] = (uint16_t)rowat(rk, dk + 1 + e);
        }
        __syncthreads();
        for (int c = warp; c < nL; c += kWarps) {
            const int j = sr[c];
            int oj, cj;
            const uint16_t *rj;
            B.col(j, oj, cj, rj);
            const int pu = find_row(rj, B.dp[j], k);
            const T u = pu >= 0 ? B.v[oj + pu] : T(0);
            if (u == T(0)) continue;
            axpy_rows<T>(B.v + oj, rj, cj, sr, sv, nL, u, lane);
        }
        __syncthreads();
    }
    if (staged) unstage_block<T>(d, a, B, val);
}


// Dense GESSM / TSTRF: independent vectors (the columns of B_IJ for GESSM,
// the rows of B_JI for TSTRF), one thread per vector, solved by substitution
// against the dense diagonal factor; a chunk of vectors is staged in shared
// memory as X[i * V + t] (thread t's element i), so accesses are
// conflict-free and the factor entries are uniform (broadcast) loads.
template <typename T, typename Acc>
__device__ void panel_dense(bool gessm, const BlockDesc &d,
                            const BlockDesc &dd, T *__restrict__ val, Acc *X,
                            size_t smem_elems) {
    const int m = dd.rows;
    const int nvec = gessm ? d.cols : d.rows;
    // the caller guarantees 32 * m <= smem_elems
    const int V = (int)min((size_t)blockDim.x, smem_elems / (size_t)m) & ~31;
    const T *__restrict__ F = val + dd.voff;  // diagonal block, ld = m
    T *B = val + d.voff;
    const int ldb = d.ld;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int v0 = 0; v0 < nvec; v0 += V) {
        const int nv = min(V, nvec - v0);
        for (int e = tid; e < m * nv; e += nt) {
            int i, t;
            if (gessm) { t = e / m; i = e % m; }
            else       { i = e / nv; t = e % nv; }
            X[i * V + t] = gessm ? (Acc)B[(int64_t)(v0 + t) * ldb + i]
                                 : (Acc)B[(int64_t)i * ldb + v0 + t];
        }
        __syncthreads();
        if (tid < nv) {
            Acc *x = X + tid;
            if (gessm) {                       // unit lower L_II from the left
                for (int mm = 0; mm < m; ++mm) {
                    const Acc xm = x[mm * V];
                    if (xm == Acc(0)) continue;
                    const T *Lc = F + (int64_t)mm * m;
                    for (int r = mm + 1; r < m; ++r) x[r * V] -= (Acc)Lc[r] * xm;
                }
            } else {                           // upper U_II from the right
                for (int mm = 0; mm < m; ++mm) {
                    const Acc xm = x[mm * V] / (Acc)F[(int64_t)mm * m + mm];
                    x[mm * V] = xm;
                    if (xm == Acc(0)) continue;
                    for (int i = mm + 1; i < m; ++i)
                        x[i * V] -= (Acc)F[(int64_t)i * m + mm] * xm;
                }
            }
        }
        __syncthreads();
        for (int e = tid; e < m * nv; e += nt) {
            int i, t;
            if (gessm) { t = e / m; i = e % m; }
            else       { i = e / nv; t = e % nv; }
            const T v = (T)X[i * V + t];
            if (gessm) B[(int64_t)(v0 + t) * ldb + i] = v;
            else       B[(int64_t)i * ldb + v0 + t] = v;
        }
        __syncthreads();
    }
}

// GESSM / TSTRF against a sparse-stored diagonal block I, using the height
// groups of its column DAG (columns of one height do not depend on each
// other; there are far fewer heights than columns in a sparse block):
//   TSTRF  L_JI = B_JI U_II^{-1}, left-looking per column k:
//          L(:, k) = (B(:, k) - sum_{m < k, U(m,k) != 0} L(:, m) U(m, k)) / U(k, k);
//          one warp per column of the current height group, a CTA barrier
//          between groups (the columns m read are of smaller height);
//   GESSM  U_IJ = L_II^{-1} B_IJ, columns independent: one warp per column
//          j, x = B(:, j) in shared memory, then group by group each lane
//          takes rows r of the group: x(r) -= sum_{m < r} L(r, m) x(m)
//          over row r of L (kept by rows in lr_*), all m of smaller height.
// Fixed summation orders: deterministic.  The panel block may be dense or
// sparse (then a per-warp dense accumulator maps its pattern).
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_panel_grp(const int32_t *__restrict__ task, BlockArgs a,
            const int32_t *__restrict__ lr_ptr, const uint16_t *__restrict__ lr_col,
            const int32_t *__restrict__ lr_pos, T *__restrict__ val) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int32_t *tk = task + 3 * (int64_t)blockIdx.x;
    const int type = tk[0];
    const BlockDesc d = a.bd[tk[1]];
    const BlockDesc dd = a.bd[tk[2]];
    const int m = dd.rows, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // per-warp vectors at the front, the diagonal block staged behind them
    const int vlen = type == 0 ? m : d.rows;
    T *vec = reinterpret_cast<T *>(smem) + (size_t)warp * vlen;
    const size_t vbytes = align16((size_t)kWarps * vlen * sizeof(T));
    bool staged;
    size_t used;
    const BlockView<T> F = stage_block<T>(dd, a, val, smem + vbytes,
                                          kStageSmem - vbytes, true, &staged, &used);
    const int32_t *sched = a.sched + dd.doff;
    const int32_t *grp = a.sgrp + dd.goff;
    const int ng = dd.ngroups;
    if (type == 1) {                                   // TSTRF
        if (!d.dense)
            for (int i = lane; i < d.rows; i += 32) vec[i] = T(0);
        __syncwarp();
        for (int g = 0; g < ng; ++g) {
            for (int t = grp[g] + warp; t < grp[g + 1]; t += kWarps) {
                const int k = sched[t];
                int fo, fc;
                const uint16_t *fr;
                F.col(k, fo, fc, fr);
                const int dp = F.dp[k];
                const T rcp = T(1) / F.v[fo + dp];
                if (d.dense) {
                    T *ck = val + d.voff + (int64_t)k * d.ld;
                    for (int r = lane; r < d.rows; r += 32) {
                        T acc = ck[r];
                        for (int e = 0; e < dp; ++e) {
                            const T u = F.v[fo + e];
                            if (u != T(0))
                                acc -= val[d.voff + (int64_t)rowat(fr, e) * d.ld + r] * u;
                        }
                        ck[r] = acc * rcp;
                    }
                } else {
                    int64_t kb;
                    int kc;
                    const uint16_t *kr;
                    colview(d, k, a, kb, kc, kr);
                    for (int e = lane; e < kc; e += 32) vec[kr[e]] = val[kb + e];
                    __syncwarp();
                    for (int e = 0; e < dp; ++e) {
                        const T u = F.v[fo + e];
                        if (u == T(0)) continue;
                        int64_t mb;
                        int mc;
                        const uint16_t *mr;
                        colview(d, rowat(fr, e), a, mb, mc, mr);
                        for (int q = lane; q < mc; q += 32) vec[mr[q]] -= val[mb + q] * u;
                        __syncwarp();
                    }
                    for (int e = lane; e < kc; e += 32) {
                        val[kb + e] = vec[kr[e]] * rcp;
                        vec[kr[e]] = T(0);
                    }
                    __syncwarp();
                }
            }
            __syncthreads();
        }
    } else {                                           // GESSM
        const int32_t *rp = lr_ptr + dd.doff + dd.I;
        if (!d.dense)
            for (int i = lane; i < m; i += 32) vec[i] = T(0);
        __syncwarp();
        for (int j = warp; j < d.cols; j += kWarps) {
            int64_t jb;
            int jc;
            const uint16_t *jr;
            colview(d, j, a, jb, jc, jr);
            if (jc == 0) continue;                     // empty column: stays empty
            for (int e = lane; e < jc; e += 32) vec[rowat(jr, e)] = val[jb + e];
            __syncwarp();
            if (!d.dense && jc <= 2 * ng) {
                // short column: push form over its own rows, ascending (its
                // pattern is closed under the solve)
                for (int e = 0; e < jc; ++e) {
                    const int k = jr[e];
                    const T xk = vec[k];
                    if (xk == T(0)) continue;
                    int fo, fc;
                    const uint16_t *fr;
                    F.col(k, fo, fc, fr);
                    for (int q = F.dp[k] + 1 + lane; q < fc; q += 32)
                        vec[fr[q]] -= F.v[fo + q] * xk;
                    __syncwarp();
                }
            } else {
                for (int g = 0; g < ng; ++g) {
                    for (int t = grp[g] + lane; t < grp[g + 1]; t += 32) {
                        const int r = sched[t];
                        T x = vec[r];
                        for (int q = rp[r]; q < rp[r + 1]; ++q) x -= F.v[lr_pos[q]] * vec[lr_col[q]];
                        vec[r] = x;
                    }
                    __syncwarp();
                }
            }
            for (int e = lane; e < jc; e += 32) {
                const int r = rowat(jr, e);
                val[jb + e] = vec[r];
                if (!d.dense) vec[r] = T(0);
            }
            __syncwarp();
        }
    }
}

// Dense panel block against a sparse-stored diagonal block: one warp per
// chunk of V vectors, lane v owning vector v (GESSM: column v0 + v of
// B_IJ; TSTRF: row v0 + v of B_JI), kept interleaved in shared memory with
// row stride V + 1 (lanes hit distinct banks).  Each lane runs the whole
// substitution on its own vector, so no synchronisation is needed:
//   GESSM  rows r ascending: x(r) -= sum_m L(r, m) x(m), over row r of L
//          (the lr_* row lists, values gathered into row order);
//   TSTRF  columns k ascending: y(k) = (y(k) - sum_{m<k} y(m) U(m, k)) / U(k, k)
//          over column k of U (the block's own CSC).
// Every lane walks the same rows / columns (uniform loops, broadcast
// loads); lanes past the last vector work on zeros and store nothing.
template <typename T>
__global__ void __launch_bounds__(32)
k_panel_vec(const int32_t *__restrict__ task, BlockArgs a,
            const int32_t *__restrict__ lr_ptr, const uint16_t *__restrict__ lr_col,
            const int32_t *__restrict__ lr_pos, T *__restrict__ val) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int32_t *tk = task + 4 * (int64_t)blockIdx.x;
    const int type = tk[0], v0 = tk[3], lane = threadIdx.x;
    const BlockDesc d = a.bd[tk[1]];
    const BlockDesc dd = a.bd[tk[2]];
    const int m = dd.rows;
    const int V = panel_vec_width(m, (int)sizeof(T)), VS = V + 1;
    const int nv = min(V, (type == 0 ? d.cols : d.rows) - v0);
    T *X = reinterpret_cast<T *>(smem);
    const size_t xbytes = align16((size_t)m * VS * sizeof(T));
    unsigned char *rest = smem + xbytes;
    const size_t cap = kStageSmem - xbytes;
    T *B = val + d.voff;
    // load: X(r, v) = vector v at position r (coalesced along the stored
    // columns: GESSM vectors are columns, TSTRF vectors are rows)
    if (type == 0) {
        for (int v = 0; v < V; ++v)
            for (int r = lane; r < m; r += 32)
                X[r * VS + v] = v < nv ? B[(int64_t)(v0 + v) * d.ld + r] : T(0);
    } else if (lane < V) {
        for (int r = 0; r < m; ++r)
            X[r * VS + lane] = lane < nv ? B[(int64_t)r * d.ld + v0 + lane] : T(0);
    }
    // lanes >= V own no vector (V < 32 for tall blocks) and stay idle below
    if (dd.dense) {
        // dense diagonal factor (no explicit inverse): read it in place,
        // rows of L / columns of U by index
        const T *Fv = val + dd.voff;
        __syncwarp();
        if (type == 0) {
            for (int r = 0; r < m && lane < V; ++r) {
                T x = X[r * VS + lane];
                for (int mm = 0; mm < r; ++mm) x -= Fv[(int64_t)mm * dd.ld + r] * X[mm * VS + lane];
                X[r * VS + lane] = x;
            }
        } else {
            for (int k = 0; k < m && lane < V; ++k) {
                const T *Uc = Fv + (int64_t)k * dd.ld;
                T y = X[k * VS + lane];
                for (int mm = 0; mm < k; ++mm) y -= Uc[mm] * X[mm * VS + lane];
                X[k * VS + lane] = y * (T(1) / Uc[k]);
            }
        }
    } else if (type == 0) {
        const int32_t *rp = lr_ptr + dd.doff + dd.I;
        const int32_t q0 = rp[0], nq = rp[m] - q0;
        const T *Lv;
        const uint16_t *Lc;
        const int32_t *Rp;
        const size_t need = align16((size_t)nq * sizeof(T)) + align16((size_t)nq * 2) +
                            align16((size_t)(m + 1) * 4);
        if (need <= cap) {                       // rows of L staged in order
            T *lv = reinterpret_cast<T *>(rest);
            uint16_t *lc = reinterpret_cast<uint16_t *>(rest + align16((size_t)nq * sizeof(T)));
            int32_t *rr = reinterpret_cast<int32_t *>(
                rest + align16((size_t)nq * sizeof(T)) + align16((size_t)nq * 2));
            for (int q = lane; q < nq; q += 32) {
                lv[q] = val[dd.voff + lr_pos[q0 + q]];
                lc[q] = lr_col[q0 + q];
            }
            for (int r = lane; r <= m; r += 32) rr[r] = rp[r] - q0;
            Lv = lv;
            Lc = lc;
            Rp = rr;
            __syncwarp();
            for (int r = 0; r < m && lane < V; ++r) {
                T x = X[r * VS + lane];
                int q = Rp[r];
                const int qe = Rp[r + 1];
                for (; q + 4 <= qe; q += 4) {         // loads first, then the chain
                    T lv[4], xv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        lv[u] = Lv[q + u];
                        xv[u] = X[Lc[q + u] * VS + lane];
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) x -= lv[u] * xv[u];
                }
                for (; q < qe; ++q) x -= Lv[q] * X[Lc[q] * VS + lane];
                X[r * VS + lane] = x;
            }
        } else {                                 // rows of L read in place
            __syncwarp();
            for (int r = 0; r < m && lane < V; ++r) {
                T x = X[r * VS + lane];
                for (int q = rp[r]; q < rp[r + 1]; ++q)
                    x -= val[dd.voff + lr_pos[q]] * X[lr_col[q] * VS + lane];
                X[r * VS + lane] = x;
            }
        }
    } else {
        bool staged;
        size_t used;
        const BlockView<T> F = stage_block<T>(dd, a, val, rest, cap, true, &staged, &used);
        __syncwarp();
        for (int k = 0; k < m && lane < V; ++k) {
            int fo, fc;
            const uint16_t *fr;
            F.col(k, fo, fc, fr);
            const int dp = F.dp[k];
            T y = X[k * VS + lane];
            int e = 0;
            for (; e + 4 <= dp; e += 4) {
                T uv[4], xv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    uv[u] = F.v[fo + e + u];
                    xv[u] = X[fr[e + u] * VS + lane];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) y -= uv[u] * xv[u];
            }
            for (; e < dp; ++e) y -= F.v[fo + e] * X[fr[e] * VS + lane];
            X[k * VS + lane] = y * (T(1) / F.v[fo + dp]);
        }
    }
    __syncwarp();
    if (type == 0) {
        for (int v = 0; v < nv; ++v)
            for (int r = lane; r < m; r += 32) B[(int64_t)(v0 + v) * d.ld + r] = X[r * VS + v];
    } else if (lane < nv) {
        for (int r = 0; r < m; ++r) B[(int64_t)r * d.ld + v0 + lane] = X[r * VS + lane];
    }
}

// GESSM (blockIdx.x < ngessm) and TSTRF tasks of one level.
template <typename T, typename Acc>
__global__ void __launch_bounds__(kThreads)
k_panel(const int32_t *__restrict__ gessm, int ngessm,
        const int32_t *__restrict__ tstrf, BlockArgs a, T *__restrict__ val) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool is_gessm = (int)blockIdx.x < ngessm;
    const int t0 = is_gessm ? blockIdx.x : blockIdx.x - ngessm;
    const int32_t *pr = is_gessm ? gessm : tstrf;
    const BlockDesc d = a.bd[pr[2 * t0]];
    const BlockDesc dd = a.bd[pr[2 * t0 + 1]];
    if (d.dense && dd.dense &&
        (size_t)dd.rows * 32 <= kStageSmem / sizeof(Acc)) {
        panel_dense<T, Acc>(is_gessm, d, dd, val, reinterpret_cast<Acc *>(smem),
                            kStageSmem / sizeof(Acc));
        return;
    }
    // Right-looking over the columns k of the diagonal block, the whole CTA
    // per step.  Shared memory: a source-column buffer, then the diagonal
    // factor (read at every step), then the panel block if it also fits.
    const int mb = max(d.rows, dd.rows);
    T *sv = reinterpret_cast<T *>(smem);
    uint16_t *sr = reinterpret_cast<uint16_t *>(sv + mb);
    const size_t sbytes = align16((size_t)mb * (sizeof(T) + 2));
    bool staged_f, staged_b;
    size_t used_f, used_b;
    const BlockView<T> F = stage_block<T>(dd, a, val, smem + sbytes,
                                          kStageSmem - sbytes, true,
                                          &staged_f, &used_f);
    const size_t o2 = sbytes + used_f;
    const BlockView<T> Bv = stage_block<T>(d, a, val, smem + o2,
                                           kStageSmem - o2, false, &staged_b,
                                           &used_b);
    for (int k = 0; k < dd.rows; ++k) {
        int fk, fck;
        const uint16_t *frk;
        F.col(k, fk, fck, frk);
        const int dk = F.dp[k];
        const int nL = fck - dk - 1;     // rows of L_II(:,k) = cols of U_II(k,:)
        if (is_gessm) {
            // U_IJ(r, j) -= L_II(r, k) U_IJ(k, j) for every column j holding
            // row k (U_IJ(k, :) is final at step k).  Each lane looks for
            // row k in one column; the warp then walks the hits.
            if (nL == 0) continue;
            for (int e = threadIdx.x; e < nL; e += blockDim.x) {
                sv[e] = F.v[fk + dk + 1 + e];
                sr[e] = (uint16_t)rowat(frk, dk + 1 + e);
            }
            __syncthreads();
            for (int cb = warp * 32; cb < d.cols; cb += kWarps * 32) {
                const int c = cb + lane;
                int oc = 0, cc = 0, pk = -1;
                const uint16_t *rc = nullptr;
                T x = T(0);
                if (c < d.cols) {
                    Bv.col(c, oc, cc, rc);
                    pk = find_row(rc, cc, k);
                    if (pk >= 0) x = Bv.v[oc + pk];
                }
                unsigned hits = __ballot_sync(~0u, pk >= 0 && x != T(0));
                while (hits) {
                    const int src = __ffs(hits) - 1;
                    hits &= hits - 1;
                    const int c2 = cb + src;
                    const T x2 = __shfl_sync(~0u, x, src);
                    int o2c, c2c;
                    const uint16_t *r2c;
                    Bv.col(c2, o2c, c2c, r2c);
                    axpy_rows<T>(Bv.v + o2c, r2c, c2c, sr, sv, nL, x2, lane);
                }
            }
            __syncthreads();
        } else {
            // L_JI(:, k) /= U_II(k, k); then L_JI(r, j) -= L_JI(r, k) U_II(k, j)
            // for the columns j of U_II(k, :).
            int ok, ck;
            const uint16_t *rk;
            Bv.col(k, ok, ck, rk);
            if (ck == 0) continue;
            const T uinv = T(1) / F.v[fk + dk];
            for (int e = threadIdx.x; e < ck; e += blockDim.x) {
                const T l = Bv.v[ok + e] * uinv;
                Bv.v[ok + e] = l;
                sv[e] = l;
                sr[e] = (uint16_t)rowat(rk, e);
            }
            __syncthreads();
            for (int c = warp; c < nL; c += kWarps) {
                const int j = rowat(frk, dk + 1 + c);
                int fj, fcj;
                const uint16_t *frj;
                F.col(j, fj, fcj, frj);
                const int pu = find_row(frj, F.dp[j], k);
                const T u = pu >= 0 ? F.v[fj + pu] : T(0);
                if (u == T(0)) continue;
                int oj, cj;
                const uint16_t *rj;
                Bv.col(j, oj, cj, rj);
                axpy_rows<T>(Bv.v + oj, rj, cj, sr, sv, ck, u, lane);
            }
            __syncthreads();
        }
    }
    if (staged_b) unstage_block<T>(d, a, Bv, val);
}


// Explicit inverses of a dense diagonal block's factors.  One warp per
// column j of L^{-1} (forward solve of L x = e_j) or U^{-1} (backward solve
// of U x = e_j), x kept in shared memory; lane l owns rows l, l + 32, ...
// (chunk q: rows 32q .. 32q + 31).  Step mm needs column mm of the factor
// below mm (L) or above mm (U): it is loaded one step ahead into the warp's
// second column buffer, and the load records which 32-row chunks of it
// hold a nonzero.  The update x -= col * x(mm) then runs as a loop over the
// set bits of that mask, so no FP64 instruction is issued for a chunk of
// zeros (the FP64 pipe and the step chain bound this kernel; a predicated
// FP64 instruction costs as much as an executed one).  Steps with x(mm) = 0
// do nothing.  U's diagonal is inverted once per CTA, so a U^{-1} step
// multiplies by the reciprocal.  Task (diag block, 0: L^{-1} / 1: U^{-1},
// first column j0); a CTA's 8 warps take columns j0 .. j0 + 7.
// Shared memory (T): the reciprocals (rounded up to 32), then per warp x
// and two column buffers of the block's row count rounded up to 32.
constexpr int kInvRows = 12;      // 32-row chunks: blocks up to 384
__host__ __device__ constexpr size_t inv_smem_elems(int b) {
    return (size_t)((b + 31) & ~31) * (1 + 3 * 8);
}
template <typename T>
__device__ __forceinline__ void inv_body(const int32_t *tk, const BlockDesc *bd,
                                         const T *val, T *winv, const int64_t *woff,
                                         unsigned char *smem, size_t cap = kStageSmem) {
    const BlockDesc d = bd[tk[0]];
    const int which = tk[1], b = d.rows, bs = (b + 31) & ~31;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = tk[2] + warp;
    const T *F = val + d.voff;                        // dense LU, ld = b
    T *s_rcp = reinterpret_cast<T *>(smem);
    // the whole factor block is staged behind the warps' vectors when it
    // fits: every warp of the CTA walks the same columns
    T *staged = s_rcp + inv_smem_elems(b);
    const bool fits = (inv_smem_elems(b) + (size_t)b * b) * sizeof(T) <= cap;
    if (fits) {
        for (int64_t e = threadIdx.x; e < (int64_t)b * b; e += blockDim.x)
            cp_async_elem(&staged[e], &F[e]);
        cp_async_wait_all();
        F = staged;
    }
    __syncthreads();
    if (which == 1)                                   // uniform across the CTA
        for (int e = threadIdx.x; e < b; e += blockDim.x)
            s_rcp[e] = T(1) / F[(int64_t)e * b + e];
    __syncthreads();
    if (j >= b) return;
    T *x = s_rcp + bs + (size_t)warp * 3 * bs;
    T *const cb0 = x + bs, *const cb1 = x + 2 * bs;
    for (int r = lane; r < bs; r += 32) x[r] = (r == j) ? T(1) : T(0);
    const int nq = bs >> 5;
    // column mm into c (rows the step uses, zeros elsewhere); returns the
    // mask of its nonzero chunks.  All loads are issued before any vote; the
    // unrolled loops leave at the block's chunk count (warp-uniform), so a
    // step issues no instruction for chunks beyond the block.
    auto fetch = [&](int mm, T *c) -> unsigned {
        const T *col = F + (int64_t)mm * b;
        T v[kInvRows];
#pragma unroll
        for (int q = 0; q < kInvRows; ++q) {
            if (q >= nq) break;
            const int r = q * 32 + lane;
            const bool in = which == 0 ? (r > mm && r < b) : (r < mm);
            v[q] = in ? col[r] : T(0);
        }
        unsigned m = 0;
#pragma unroll
        for (int q = 0; q < kInvRows; ++q) {
            if (q >= nq) break;
            c[q * 32 + lane] = v[q];
            if (__ballot_sync(~0u, nz(v[q]))) m |= 1u << q;
        }
        return m;
    };
    const int step = which == 0 ? 1 : -1, end = which == 0 ? b : -1;
    unsigned mcur = fetch(j, cb0);
    int cur = 0;
    for (int mm = j; mm != end; mm += step) {
        const unsigned mnext = (mm + step != end) ? fetch(mm + step, cur ? cb0 : cb1) : 0u;
        __syncwarp();
        T xm = x[mm];
        if (which == 1) {
            xm *= s_rcp[mm];
            if (lane == 0) x[mm] = xm;
        }
        if (nz(xm)) {                                 // uniform across the warp
            const T *c = cur ? cb1 : cb0;
            for (unsigned m = mcur; m; m &= m - 1) {  // nonzero chunks only
                const int r = (__ffs(m) - 1) * 32 + lane;
                x[r] -= c[r] * xm;
            }
        }
        __syncwarp();
        mcur = mnext;
        cur ^= 1;
    }
    T *out = winv + woff[d.I] + (which ? (int64_t)b * b : 0) + (int64_t)j * b;
    for (int r = lane; r < b; r += 32) out[r] = x[r];
}

// FP32 inverses: the same column solves with x held in registers and every
// 32-row chunk updated at every step.  FP32 FMAs are cheap on B300 (64x the
// FP64 rate), so the masks of the FP64 body would only lengthen the chain.
template <typename T>
__device__ __forceinline__ void inv_body_reg(const int32_t *tk, const BlockDesc *bd,
                                             const T *val, T *winv, const int64_t *woff) {
    const BlockDesc d = bd[tk[0]];
    const int which = tk[1], b = d.rows;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = tk[2] + warp;
    if (j >= b) return;
    const T *F = val + d.voff;           // dense LU, ld = b
    T x[kInvRows];
#pragma unroll
    for (int q = 0; q < kInvRows; ++q) x[q] = (q * 32 + lane == j) ? T(1) : T(0);
    if (which == 0) {
        for (int mm = j; mm < b; ++mm) {
            const T xm = __shfl_sync(~0u, x[(mm >> 5) % kInvRows], mm & 31);
            if (xm == T(0)) continue;
            const T *Lc = F + (int64_t)mm * b;
#pragma unroll
            for (int q = 0; q < kInvRows; ++q) {
                const int r = q * 32 + lane;
                if (r > mm && r < b) x[q] -= Lc[r] * xm;
            }
        }
    } else {
        for (int mm = j; mm >= 0; --mm) {
            const T *Uc = F + (int64_t)mm * b;
            const T own = __shfl_sync(~0u, x[(mm >> 5) % kInvRows], mm & 31);
            const T xm = own / Uc[mm];
#pragma unroll
            for (int q = 0; q < kInvRows; ++q)
                if (q * 32 + lane == mm) x[q] = xm;
            if (xm == T(0)) continue;
#pragma unroll
            for (int q = 0; q < kInvRows; ++q) {
                const int r = q * 32 + lane;
                if (r < mm) x[q] -= Uc[r] * xm;
            }
        }
    }
    T *out = winv + woff[d.I] + (which ? (int64_t)b * b : 0) + (int64_t)j * b;
#pragma unroll
    for (int q = 0; q < kInvRows; ++q) {
        const int r = q * 32 + lane;
        if (r < b) out[r] = x[q];
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_inv(const int32_t *__restrict__ task, const BlockDesc *__restrict__ bd,
      const T *__restrict__ val, T *__restrict__ winv,
      const int64_t *__restrict__ woff, size_t cap) {
    extern __shared__ __align__(16) unsigned char smem[];
    if constexpr (sizeof(T) == 4)
        inv_body_reg<T>(task + 3 * (int64_t)blockIdx.x, bd, val, winv, woff);
    else
        inv_body<T>(task + 3 * (int64_t)blockIdx.x, bd, val, winv, woff, smem, cap);
}

// Column-pair masks of a staged 16 x 64 slice S (S[kk * 64 + c]): bit kk of
// pm[p] is set when S[kk][2p] or S[kk][2p + 1] is nonzero.  Warp w takes
// pairs 4w .. 4w + 3, lane l row kk = l & 15 of pairs 4w + 2 (l >> 4) + {0,
// 1}; rows kk >= nk count as zero.  All 256 threads.
template <typename T>
__device__ __forceinline__ void slice_pair_masks(const T *S, int nk,
                                                 unsigned short *pm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int kk = lane & 15, c = 8 * warp + 4 * (lane >> 4);
    bool z0 = false, z1 = false;
    if (kk < nk) {
        const T *r = S + kk * 64 + c;
        z0 = nz(r[0]) || nz(r[1]);
        z1 = nz(r[2]) || nz(r[3]);
    }
    const unsigned m0 = __ballot_sync(~0u, z0), m1 = __ballot_sync(~0u, z1);
    if (lane == 0) {
        pm[4 * warp + 0] = (unsigned short)(m0 & 0xffffu);
        pm[4 * warp + 1] = (unsigned short)(m1 & 0xffffu);
        pm[4 * warp + 2] = (unsigned short)(m0 >> 16);
        pm[4 * warp + 3] = (unsigned short)(m1 >> 16);
    }
}

// Dense GESSM / TSTRF through the inverses, one CTA per 64-wide chunk:
//   GESSM: U_IJ(:, c0:c0+64) = L_II^{-1} B_IJ(:, c0:c0+64)
//   TSTRF: L_JI(r0:r0+64, :) = B_JI(r0:r0+64, :) U_II^{-1}
// The chunk of B is staged in shared memory as X[k * 64 + t] (so the result
// can be written in place), the triangular inverse is staged in 16-deep
// k-slices Ts[kk * 64 + i], and each 64 x 64 block of outputs is
// accumulated in registers.  Both products have the form out(row, col) =
// sum_k A_k[row] B_k[col] with the vectors A_k, B_k rows of the staged
// arrays (GESSM: A_k = Ts row, B_k = X row; TSTRF: A_k = X row, B_k = Ts
// row), so the work runs as in the dense Schur tiles: warp w owns output
// rows 8w .. 8w+7, lane l row 8w + (l & 7) and column 4g + (l >> 3) of the
// 16 column groups g, and per column group it loops over only the k where
// its row group of A_k and group g of B_k hold a nonzero (column-pair masks
// of each slice; no FP64 work is issued for zeros).  A slice of X that is
// all zero is skipped before its inverse slice is loaded.  The terms left
// out are exact zeros.
template <typename T>
__device__ __forceinline__ void panel_inv_body(const int32_t *tk, const BlockDesc *bd,
                                               T *val, const T *winv,
                                               const int64_t *woff, const BlockArgs &a,
                                               unsigned char *smem) {
    constexpr int KT = 16;
    const int type = tk[0];
    const BlockDesc d = bd[tk[1]];
    const BlockDesc dd = bd[tk[2]];
    const int c0 = tk[3], m = dd.rows, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    T *X = reinterpret_cast<T *>(smem);                 // m x 64 chunk, X[k * 64 + c]
    T *Ts = X + (size_t)m * 64;                          // 2 x 16 x 64 inverse slices
    const int nsl = (m + KT - 1) / KT;
    unsigned short *xpm = reinterpret_cast<unsigned short *>(Ts + 2 * KT * 64);  // [nsl][32]
    unsigned short *tpm = xpm + (size_t)nsl * 32;                               // [2][32]
    const int64_t ld = d.ld;
    T *Bg = val + d.voff;
    const T *Inv = winv + woff[dd.I] + (type == 0 ? 0 : (int64_t)m * m);
    const int nv = min(64, (type == 0 ? d.cols : d.rows) - c0);
    // stage the chunk: GESSM columns c0.. (X[k][c] = B(k, c0 + c));
    // TSTRF rows c0.. (X[k][r] = B(c0 + r, k))
    if (d.dense) {
        for (int e = tid; e < m * 64; e += 256) {
            const int k = e / 64, c = e % 64;
            const T *src = c < nv ? (type == 0 ? &Bg[(int64_t)(c0 + c) * ld + k]
                                               : &Bg[(int64_t)k * ld + c0 + c])
                                  : Bg;
            cp_async_elem(&X[e], src, c < nv);
        }
        cp_async_wait_all();
    } else {
        // sparse panel block: scatter its pattern into the zeroed chunk
        for (int e = tid; e < m * 64; e += 256) X[e] = T(0);
        __syncthreads();
        if (type == 0) {                 // columns c0 + c of B_IJ, rows k
            for (int c = warp; c < nv; c += 8) {
                int64_t vb;
                int cn;
                const uint16_t *rw;
                colview(d, c0 + c, a, vb, cn, rw);
                for (int e = lane; e < cn; e += 32) X[rw[e] * 64 + c] = val[vb + e];
            }
        } else {                         // rows c0 .. c0 + nv of B_JI, columns k
            for (int k = warp; k < m; k += 8) {
                int64_t vb;
                int cn;
                const uint16_t *rw;
                colview(d, k, a, vb, cn, rw);
                for (int e = lane; e < cn; e += 32) {
                    const int r = rw[e] - c0;
                    if (r >= 0 && r < nv) X[k * 64 + r] = val[vb + e];
                }
            }
        }
    }
    __syncthreads();
    for (int sl = 0; sl < nsl; ++sl)
        slice_pair_masks<T>(X + (size_t)sl * KT * 64, min(KT, m - sl * KT), xpm + sl * 32);
    __syncthreads();
    const int rr = 8 * warp + (lane & 7), cc = lane >> 3;
    // inverse slice (output chunk ob, rows k0 .. k0 + 15) into buffer bf by
    // cp.async, entries outside the inverse zero-filled:
    //   GESSM: Ts[kk][ii] = Linv(ob + ii, k0 + kk)
    //   TSTRF: Ts[kk][ii] = Uinv(k0 + kk, ob + ii)
    auto issue = [&](int ob, int k0, int bf) {
        T *D = Ts + (size_t)bf * KT * 64;
        for (int e = tid; e < KT * 64; e += 256) {
            int kk, ii;
            if (type == 0) { ii = e % 64; kk = e / 64; }
            else           { kk = e % KT; ii = e / KT; }
            const int gi = ob + ii, gk = k0 + kk;
            const bool in = gi < m && gk < m;
            const T *src = !in ? Inv : type == 0 ? &Inv[(int64_t)gk * m + gi]
                                                 : &Inv[(int64_t)gi * m + gk];
            cp_async_elem(&D[kk * 64 + ii], src, in);
        }
        cp_async_commit();
    };
    // first slice from k0 on, below kend, whose slice of X holds a nonzero
    // (kend: none); a slice of X without one adds nothing
    auto next_live = [&](int k0, int kend) {
        for (; k0 < kend; k0 += KT) {
            const unsigned short *xp = xpm + (k0 / KT) * 32;
            bool any = false;
#pragma unroll
            for (int p = 0; p < 32; ++p) any |= xp[p] != 0;
            if (any) break;
        }
        return min(k0, kend);
    };
    for (int ob = 0; ob < m; ob += 64) {       // output chunk along m
        T acc[16];
#pragma unroll
        for (int g = 0; g < 16; ++g) acc[g] = T(0);
        // GESSM: out(i, c) = sum_{k <= i} Linv(i, k) X(k, c), i in [ob, ob+64)
        // TSTRF: out(r, i) = sum_{k <= i} X(r, k) Uinv(k, i), i in [ob, ob+64)
        // The inverse slices are double-buffered: the next live slice's
        // copies are in flight while the current one is multiplied.
        const int kend = min(m, ob + 64);
        __syncthreads();                          // buffers of the previous chunk read
        int k0 = next_live(0, kend), buf = 0;
        if (k0 < kend) issue(ob, k0, 0);
        while (k0 < kend) {
            cp_async_wait_all();
            __syncthreads();                      // slice k0 in buffer buf for all
            const T *TsB = Ts + (size_t)buf * KT * 64;
            unsigned short *tpB = tpm + buf * 32;
            slice_pair_masks<T>(TsB, min(KT, m - k0), tpB);
            __syncthreads();
            // the other buffer was last read before the first barrier above
            const int k1 = next_live(k0 + KT, kend);
            if (k1 < kend) issue(ob, k1, buf ^ 1);
            const unsigned short *xp = xpm + (k0 / KT) * 32;
            const unsigned short *apm = type == 0 ? tpB : xp;
            const unsigned short *bpm = type == 0 ? xp : tpB;
            const T *A = type == 0 ? TsB : X + (size_t)k0 * 64;
            const T *B = type == 0 ? X + (size_t)k0 * 64 : TsB;
            const unsigned amk = apm[4 * warp] | apm[4 * warp + 1] | apm[4 * warp + 2] |
                                 apm[4 * warp + 3];
            if (amk) {
#pragma unroll
                for (int g = 0; g < 16; ++g) {
                    unsigned km = amk & (unsigned)(bpm[2 * g] | bpm[2 * g + 1]);
                    if (km) {                             // uniform across the warp
                        int kk = __ffs(km) - 1;
                        km &= km - 1;
                        T x = A[kk * 64 + rr], y = B[kk * 64 + 4 * g + cc];
                        while (km) {
                            kk = __ffs(km) - 1;
                            km &= km - 1;
                            const T xn = A[kk * 64 + rr], yn = B[kk * 64 + 4 * g + cc];
                            acc[g] += x * y;
                            x = xn;
                            y = yn;
                        }
                        acc[g] += x * y;
                    }
                }
            }
            k0 = k1;
            buf ^= 1;
        }
#pragma unroll
        for (int g = 0; g < 16; ++g) {
            // (row, column) of the panel block; a sparse block keeps only
            // its pattern (the result is zero elsewhere)
            int br, bc;
            if (type == 0) { br = ob + rr; bc = c0 + 4 * g + cc; }
            else           { br = c0 + rr; bc = ob + 4 * g + cc; }
            const bool in = type == 0 ? (br < m && bc - c0 < nv)
                                      : (br - c0 < nv && bc < m);
            if (!in) continue;
            if (d.dense) {
                Bg[(int64_t)bc * ld + br] = acc[g];
            } else {
                int64_t vb;
                int cn;
                const uint16_t *rw;
                colview(d, bc, a, vb, cn, rw);
                const int q = find_row(rw, cn, br);
                if (q >= 0) val[vb + q] = acc[g];
            }
        }
    }
}

// FP32 panels through the inverses: the dense 64 x 64 register tiles (4 x 4
// per thread) over the inverse's triangle, every product executed (FP32
// FMAs are cheap; the masked FP64 body's bookkeeping would dominate).
template <typename T>
__device__ __forceinline__ void panel_inv_dense_body(const int32_t *tk, const BlockDesc *bd,
                                                     T *val, const T *winv,
                                                     const int64_t *woff, const BlockArgs &a,
                                                     unsigned char *smem) {
    constexpr int KT = 16;
    const int type = tk[0];
    const BlockDesc d = bd[tk[1]];
    const BlockDesc dd = bd[tk[2]];
    const int c0 = tk[3], m = dd.rows, tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    T *X = reinterpret_cast<T *>(smem);                 // m x 64 chunk, X[k * 64 + c]
    T *Ts = X + (size_t)m * 64;                          // 16 x 64 inverse slice
    const int64_t ld = d.ld;
    T *Bg = val + d.voff;
    const T *Inv = winv + woff[dd.I] + (type == 0 ? 0 : (int64_t)m * m);
    const int nv = min(64, (type == 0 ? d.cols : d.rows) - c0);
    // stage the chunk: GESSM columns c0.. (X[k][c] = B(k, c0 + c));
    // TSTRF rows c0.. (X[k][r] = B(c0 + r, k)); flag the 16-deep k-slices
    // of the chunk that hold a nonzero (all-zero slices contribute nothing)
    // and, per k, whether row k of the chunk holds one (the warps staging a
    // row ballot; m * 64 is a whole number of warps)
    int *zrow = reinterpret_cast<int *>(Ts + KT * 64);
    int *zflag = zrow + m;
    const int lane = tid & 31, warp = tid >> 5;
    if (d.dense) {
        for (int e = tid; e < m + (m + KT - 1) / KT; e += 256) zrow[e] = 0;
        __syncthreads();
        for (int e = tid; e < m * 64; e += 256) {
            const int k = e / 64, c = e % 64;
            T v = T(0);
            if (c < nv)
                v = type == 0 ? Bg[(int64_t)(c0 + c) * ld + k] : Bg[(int64_t)k * ld + c0 + c];
            X[e] = v;
            if (sizeof(T) == 8 && __ballot_sync(0xffffffffu, v != T(0)) && lane == 0) {
                atomicOr(&zrow[k], 1);
                atomicOr(&zflag[k / KT], 1);
            }
        }
    } else {
        // sparse panel block: scatter its pattern into the zeroed chunk (no
        // zero-row skipping: every row is flagged)
        for (int e = tid; e < m + (m + KT - 1) / KT; e += 256) zrow[e] = 1;
        for (int e = tid; e < m * 64; e += 256) X[e] = T(0);
        __syncthreads();
        if (type == 0) {                 // columns c0 + c of B_IJ, rows k
            for (int c = warp; c < nv; c += 8) {
                int64_t vb;
                int cn;
                const uint16_t *rw;
                colview(d, c0 + c, a, vb, cn, rw);
                for (int e = lane; e < cn; e += 32) X[rw[e] * 64 + c] = val[vb + e];
            }
        } else {                         // rows c0 .. c0 + nv of B_JI, columns k
            for (int k = warp; k < m; k += 8) {
                int64_t vb;
                int cn;
                const uint16_t *rw;
                colview(d, k, a, vb, cn, rw);
                for (int e = lane; e < cn; e += 32) {
                    const int r = rw[e] - c0;
                    if (r >= 0 && r < nv) X[k * 64 + r] = val[vb + e];
                }
            }
        }
    }
    __syncthreads();
    for (int ob = 0; ob < m; ob += 64) {       // output chunk along m
        T acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int jx = 0; jx < 4; ++jx) acc[i][jx] = T(0);
        // GESSM: out(i, c) = sum_{k <= i} Linv(i, k) X(k, c), i in [ob, ob+64)
        // TSTRF: out(r, i) = sum_{k <= i} X(r, k) Uinv(k, i), i in [ob, ob+64)
        const int kend = min(m, ob + 64);
        for (int k0 = 0; k0 < kend; k0 += KT) {
            if (sizeof(T) == 8 && !zflag[k0 / KT]) continue;  // uniform across the CTA
            for (int e = tid; e < KT * 64; e += 256) {
                int kk, ii;
                T v = T(0);
                if (type == 0) {               // Ts[kk][ii] = Linv(ob + ii, k0 + kk)
                    ii = e % 64; kk = e / 64;
                    const int gi = ob + ii, gk = k0 + kk;
                    if (gi < m && gk < m) v = Inv[(int64_t)gk * m + gi];
                } else {                       // Ts[kk][ii] = Uinv(k0 + kk, ob + ii)
                    kk = e % KT; ii = e / KT;
                    const int gi = ob + ii, gk = k0 + kk;
                    if (gi < m && gk < m) v = Inv[(int64_t)gi * m + gk];
                }
                Ts[kk * 64 + ii] = v;
            }
            __syncthreads();
            const int kn = min(KT, m - k0);
            for (int kk = 0; kk < kn; ++kk) {
                if (sizeof(T) == 8 && !zrow[k0 + kk]) continue;
                T a[4], bv[4];
                if (type == 0) {               // rows of out = ob + ty*4+i, cols = tx*4+jx
#pragma unroll
                    for (int i = 0; i < 4; ++i) a[i] = Ts[kk * 64 + ty * 4 + i];
#pragma unroll
                    for (int jx = 0; jx < 4; ++jx) bv[jx] = X[(k0 + kk) * 64 + tx * 4 + jx];
                } else {                       // rows = chunk rows ty*4+i, cols = ob + tx*4+jx
#pragma unroll
                    for (int i = 0; i < 4; ++i) a[i] = X[(k0 + kk) * 64 + ty * 4 + i];
#pragma unroll
                    for (int jx = 0; jx < 4; ++jx) bv[jx] = Ts[kk * 64 + tx * 4 + jx];
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int jx = 0; jx < 4; ++jx) acc[i][jx] += a[i] * bv[jx];
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int jx = 0; jx < 4; ++jx) {
                // (row, column) of the panel block; a sparse block keeps only
                // its pattern (the result is zero elsewhere)
                int br, bc;
                if (type == 0) { br = ob + ty * 4 + i; bc = c0 + tx * 4 + jx; }
                else           { br = c0 + ty * 4 + i; bc = ob + tx * 4 + jx; }
                const bool in = type == 0 ? (br < m && bc - c0 < nv)
                                          : (br - c0 < nv && bc < m);
                if (!in) continue;
                if (d.dense) {
                    Bg[(int64_t)bc * ld + br] = acc[i][jx];
                } else {
                    int64_t vb;
                    int cn;
                    const uint16_t *rw;
                    colview(d, bc, a, vb, cn, rw);
                    const int q = find_row(rw, cn, br);
                    if (q >= 0) val[vb + q] = acc[i][jx];
                }
            }
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_panel_inv(const int32_t *__restrict__ task, const BlockDesc *__restrict__ bd,
            T *__restrict__ val, const T *__restrict__ winv,
            const int64_t *__restrict__ woff, BlockArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    if constexpr (sizeof(T) == 4)
        panel_inv_dense_body<T>(task + 4 * (int64_t)blockIdx.x, bd, val, winv, woff, a, smem);
    else
        panel_inv_body<T>(task + 4 * (int64_t)blockIdx.x, bd, val, winv, woff, a, smem);
}

// SSSSM: target B_KJ -= sum over the level's sources I of L_KI U_IJ.
// One warp per target column jj: for each source, for each stored U_IJ(i,jj)
// (fetched 32 at a time and broadcast by shuffles),
// acc += L_KI(:,i) U_IJ(i,jj); then B_KJ(:,jj) -= acc at the stored rows.
template <typename T, typename Acc>
__global__ void __launch_bounds__(kThreads)
k_ssssm(const int32_t *__restrict__ tgt, const int64_t *__restrict__ srcoff,
        const int32_t *__restrict__ src, BlockArgs a, T *__restrict__ val,
        const int64_t *__restrict__ ne_off, const uint16_t *__restrict__ ne_col,
        size_t stage_cap) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const BlockDesc d = a.bd[tgt[blockIdx.x]];
    const int64_t s0 = srcoff[blockIdx.x], s1 = srcoff[blockIdx.x + 1];
    Acc *acc = reinterpret_cast<Acc *>(smem) + warp * d.rows;
    // a target with a single sparse L source stages that block once (its
    // columns are then read from shared memory by every warp)
    BlockView<T> LV{};
    bool lview = false;
    if (s1 - s0 == 1 && !a.bd[src[2 * s0]].dense) {
        const size_t ab = align16((size_t)kWarps * d.rows * sizeof(Acc));
        bool st;
        size_t used;
        LV = stage_block<T>(a.bd[src[2 * s0]], a, val, smem + ab,
                            stage_cap > ab ? stage_cap - ab : 0, false, &st, &used);
        lview = true;
    }
    for (int t = lane; t < d.rows; t += 32) acc[t] = Acc(0);
    __syncwarp();
    for (int jj = warp; jj < d.cols; jj += kWarps) {
        bool any = false;                 // warp-uniform: column received an update
        for (int64_t s = s0; s < s1; ++s) {
            const int32_t lb = src[2 * s];
            const BlockDesc dl = a.bd[lb];
            const BlockDesc du = a.bd[src[2 * s + 1]];
            int64_t vu;
            int cu;
            const uint16_t *ru;
            colview(du, jj, a, vu, cu, ru);
            // walk U(:, jj)'s stored rows, or, when L_KI is sparse with fewer
            // non-empty columns, those columns (U looked up); both ascending
            const int64_t ne0 = dl.dense ? 0 : ne_off[lb];
            const int nne = dl.dense ? 0 : (int)(ne_off[lb + 1] - ne0);
            const bool by_l = !dl.dense && nne < cu;
            const int nit = by_l ? nne : cu;
            for (int c0 = 0; c0 < nit; c0 += 32) {
                const int t = c0 + lane;
                int il = 0;
                Acc ul = Acc(0);
                if (t < nit) {
                    if (by_l) {
                        il = ne_col[ne0 + t];
                        const int q = find_row(ru, cu, il);
                        ul = q >= 0 ? (Acc)val[vu + q] : Acc(0);
                    } else {
                        il = rowat(ru, t);
                        ul = (Acc)val[vu + t];
                    }
                }
                const int nn = min(32, nit - c0);
                for (int k = 0; k < nn; ++k) {
                    const Acc u = __shfl_sync(~0u, ul, k);
                    const int i = __shfl_sync(~0u, il, k);
                    if (u == Acc(0)) continue;
                    if (lview) {
                        int ol, cl;
                        const uint16_t *rl;
                        LV.col(i, ol, cl, rl);
                        any |= cl > 0;
                        for (int e = lane; e < cl; e += 32)
                            acc[rowat(rl, e)] += (Acc)LV.v[ol + e] * u;
                    } else {
                        int64_t vl;
                        int cl;
                        const uint16_t *rl;
                        colview(dl, i, a, vl, cl, rl);
                        any |= cl > 0;
                        for (int e = lane; e < cl; e += 32)
                            acc[rowat(rl, e)] += (Acc)val[vl + e] * u;
                    }
                    __syncwarp();
                }
            }
        }
        if (!any) continue;               // nothing accumulated: column unchanged
        int64_t vb;
        int cn;
        const uint16_t *rows;
        colview(d, jj, a, vb, cn, rows);
        for (int t = lane; t < cn; t += 32) {
            const int r = rowat(rows, t);
            val[vb + t] = (T)((Acc)val[vb + t] - acc[r]);
            acc[r] = Acc(0);
        }
        __syncwarp();
    }
}


// SSSSM on dense tiles, FP32 storage, on the 5th-generation tensor cores:
// a 128 x 64 tile of a dense target B_KJ minus the sum over the level's
// dense sources of L_KI U_IJ.  Split precision (3xTF32): each operand x is
// split into hi = x with the 13 low mantissa bits cleared (exact in TF32)
// and lo = x - hi, and the tile accumulates hi*hi + hi*lo + lo*hi in FP32 in
// tensor memory (the dropped lo*lo term and the TF32 reading of lo are
// below FP32 rounding of the products).  K runs over the sources' columns
// in 32-deep chunks staged in shared memory (K-major core-matrix layout, no
// swizzle), two stages: while the tensor core works on one chunk the CTA
// stages the next.  One thread issues the MMAs and commits them to the
// stage's mbarrier; every wait is bounded, and a wait that runs out sets
// err (reported as a timeout) instead of hanging.
namespace tc {
constexpr int TM = 128, TN = 64, KC = 32;
constexpr int LBO = 128;                         // next core matrix along K
constexpr int SBO = (KC / 4) * 128;              // next 8-row group
constexpr int A_BYTES = TM * KC * 4, B_BYTES = TN * KC * 4;
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;   // hi, lo of A and B
constexpr size_t SMEM = 2 * STAGE_BYTES + 1024;
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t kmaj(int row, int k) {
    return (row >> 3) * SBO + (k >> 2) * LBO + (row & 7) * 16 + (k & 3) * 4;
}
__device__ __forceinline__ uint64_t desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((LBO >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((SBO >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
__device__ __forceinline__ void split(float x, float &hi, float &lo) {
    hi = __uint_as_float(__float_as_uint(x) & 0xffffe000u);
    lo = x - hi;
}
__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t parity) {
    uint32_t done = 0;
    for (int it = 0; it < (1 << 24) && !done; ++it)
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
    return done != 0;
}
}  // namespace tc

// One tile's work: `smem` (1024-byte aligned, tc::SMEM - 1024 bytes) holds
// the two stages, `mbar` the two initialised stage barriers whose expected
// parities `phase` carries from tile to tile, `tmem` the tile's 64 TMEM
// columns (allocated by the caller).  Every MMA it commits is waited for
// before it returns (a wait that runs out sets err[0]).
__device__ __forceinline__ void tc_body(const int32_t *tk, const int32_t *src,
                                        const BlockDesc *bd, float *val,
                                        unsigned long long *err, unsigned char *smem,
                                        uint64_t *mbar, uint32_t tmem,
                                        uint32_t (&phase)[2], int passes) {
    using namespace tc;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const BlockDesc d = bd[tk[0]];
    const int s0 = tk[1], s1 = tk[2], r0 = tk[3], c0 = tk[4];
    if (s0 >= s1) return;
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) |
                           ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
    // Register image of one chunk, one core matrix (8 rows x 4 k, 128
    // contiguous bytes in shared memory) per warp instruction: lane l holds
    // row (l & 7) and k (l >> 3) of it, so each store fills 32 distinct
    // banks and each global load reads 32-byte runs.  Warp w takes the A
    // core matrices q = w + 8 j (j < 16: row group q % 16, k group q / 16)
    // and the B core matrices q = w + 8 j (j < 8: column group q % 8, k
    // group q / 8).
    float ra[16], rb[8];
    const int lr = lane & 7, lk = lane >> 3;
    auto load = [&](const BlockDesc &L, const BlockDesc &U, int kk0) {
        const float *A = val + L.voff, *Bm = val + U.voff;
        const int K = L.cols;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int q = warp + 8 * j;
            const int gr = r0 + 8 * (q & 15) + lr, gk = kk0 + 4 * (q >> 4) + lk;
            ra[j] = (gk < K && gr < d.rows) ? A[(int64_t)gk * L.ld + gr] : 0.f;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int q = warp + 8 * j;
            const int gc = c0 + 8 * (q & 7) + lr, gk = kk0 + 4 * (q >> 3) + lk;
            rb[j] = (gk < K && gc < d.cols) ? Bm[(int64_t)gc * U.ld + gk] : 0.f;
        }
    };
    // three passes: hi and lo parts; one pass: the FP32 values as they are
    // (the TF32 MMA reads their upper 19 bits)
    auto store = [&](unsigned char *base) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int q = warp + 8 * j;
            const uint32_t o = kmaj(8 * (q & 15) + lr, 4 * (q >> 4) + lk);
            if (passes == 3) {
                float hi, lo;
                split(ra[j], hi, lo);
                *reinterpret_cast<float *>(base + o) = hi;
                *reinterpret_cast<float *>(base + A_BYTES + o) = lo;
            } else {
                *reinterpret_cast<float *>(base + o) = ra[j];
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int q = warp + 8 * j;
            const uint32_t o = kmaj(8 * (q & 7) + lr, 4 * (q >> 3) + lk);
            if (passes == 3) {
                float hi, lo;
                split(rb[j], hi, lo);
                *reinterpret_cast<float *>(base + 2 * A_BYTES + o) = hi;
                *reinterpret_cast<float *>(base + 2 * A_BYTES + B_BYTES + o) = lo;
            } else {
                *reinterpret_cast<float *>(base + 2 * A_BYTES + o) = rb[j];
            }
        }
    };
    int s = s0, k0 = 0;
    BlockDesc dl = bd[src[2 * s]], du = bd[src[2 * s + 1]];
    load(dl, du, 0);
    int chunk = 0;
    bool ok = true;
    for (;;) {
        const int st = chunk & 1;
        unsigned char *base = smem + st * STAGE_BYTES;
        if (chunk >= 2) {               // the MMAs of chunk - 2 read this stage
            // CTA-uniform: if any thread's bounded wait ran out, nothing more
            // is staged or issued (the stage may still be read) and the
            // drain below waits for what was committed
            const bool done = wait_phase(smem_u32(&mbar[st]), phase[st]);
            if (!__syncthreads_and(done)) {
                ok = false;
                break;
            }
            phase[st] ^= 1;
        }
        store(base);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a_hi = smem_u32(base), a_lo = a_hi + A_BYTES;
            const uint32_t b_hi = a_hi + 2 * A_BYTES, b_lo = b_hi + B_BYTES;
#pragma unroll
            for (int kk = 0; kk < KC / 8; ++kk) {
                const uint32_t off = kk * 2 * LBO;
                const uint32_t pa[3] = {a_hi, a_hi, a_lo}, pb[3] = {b_hi, b_lo, b_hi};
                for (int t = 0; t < passes; ++t) {
                    const uint32_t acc = (chunk > 0 || kk > 0 || t > 0) ? 1u : 0u;
                    asm volatile("{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
                                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                                 :: "r"(tmem), "l"(desc(pa[t] + off)), "l"(desc(pb[t] + off)),
                                    "r"(idesc), "r"(acc));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(&mbar[st])) : "memory");
        }
        ++chunk;
        k0 += KC;
        if (k0 >= dl.cols) {
            ++s;
            k0 = 0;
            if (s >= s1) break;
            dl = bd[src[2 * s]];
            du = bd[src[2 * s + 1]];
        }
        load(dl, du, k0);               // in flight while the tensor core works
    }
    // drain: every committed chunk not yet waited for (chunk - 2 and
    // chunk - 1, also after an expired wait, whose phase was not advanced);
    // each wait is bounded and runs even when an earlier one expired, so
    // TMEM is released only after the MMAs were given a second bound
    for (int c = max(0, chunk - 2); c < chunk; ++c) {
        const int st = c & 1;
        const bool done = wait_phase(smem_u32(&mbar[st]), phase[st]);
        ok = __syncthreads_and(done) && ok;
        phase[st] ^= 1;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        // warp w reads TMEM lanes 32 (w % 4) .. (rows), columns 32 (w / 4) ..
        const int row = 32 * (warp & 3) + lane, gr = r0 + row;
        for (int cb = 32 * (warp >> 2); cb < 32 * (warp >> 2) + 32; cb += 16) {
            uint32_t v[16];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                         "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]),
                           "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]),
                           "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                           "=r"(v[15])
                         : "r"(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)cb));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (gr < d.rows)
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int gc = c0 + cb + j;
                    if (gc < d.cols) val[d.voff + (int64_t)gc * d.ld + gr] -= __uint_as_float(v[j]);
                }
        }
    } else if (tid == 0) {
        atomicOr(&err[0], 1ull);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
}

// TMEM columns and stage barriers of a CTA that runs tensor-core tiles.
__device__ __forceinline__ uint32_t tc_setup(uint64_t *mbar, uint32_t *tmem_holder) {
    using namespace tc;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tmem_holder)), "r"(TN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return *tmem_holder;
}

__device__ __forceinline__ void tc_teardown(uint32_t tmem) {
    using namespace tc;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TN));
}

__global__ void __launch_bounds__(256)
k_ssssm_tc(const int32_t *__restrict__ task, const int32_t *__restrict__ src,
           const BlockDesc *__restrict__ bd, float *__restrict__ val,
           unsigned long long *__restrict__ err, int passes) {
    using namespace tc;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_holder;
    const int32_t *tk = task + 5 * (int64_t)blockIdx.x;
    if (tk[1] >= tk[2]) return;
    const uint32_t tmem = tc_setup(mbar, &tmem_holder);
    uint32_t phase[2] = {0, 0};
    tc_body(tk, src, bd, val, err, smem, mbar, tmem, phase, passes);
    tc_teardown(tmem);
}

// SSSSM on dense tiles (FP64): a 64 x 64 tile of a dense target B_KJ minus
// the sum over the level's dense sources of L_KI U_IJ, accumulated in
// registers over all sources and 16-deep k-slices and written once.  The
// FP64 pipe bounds this kernel (about two FMAs per SM and clock on B300),
// so the tile executes only products whose operands can both be nonzero,
// at the granularity of 8 x 4 sub-tiles: warp w owns rows 8w .. 8w+7, lane
// l row 8w + (l & 7) and column 4g + (l >> 3) of each of the 16 column
// groups g (16 accumulators).  While staging a slice, the warps record
// which 8-row groups of every column k of the A slice and which column
// pairs of every row k of the B slice hold a nonzero; warp w then runs,
// for each column group g, a loop over the k at which both its row group
// of A(:, k) and group g of B(k, :) hold one (set bits of a 16-bit mask,
// warp-uniform, so no FP64 instruction is issued for a skipped product).
// The terms left out are exact zeros: the result is the dense one.  Slices
// are double-buffered (the next slice's cp.async copies are in flight while
// the current one is multiplied), sources run in ascending
// I and k ascending within them, so the result is deterministic.
// Shared memory of one dense Schur tile: the double-buffered slices and
// their masks.  sAg[buf][k][h] bit j: rows 32h + 8j .. +7 of A(:, k) hold a
// nonzero; sBc[buf][c][h] bit k - 32h: B(k, c) is nonzero (k in the h-th
// 32-deep half of the slice).  Slices are 16 deep (the body also takes 64:
// measured on B300, 64-deep FP32 slices were slower, 132 against 91 ms for
// the 40^3 FP32 + refinement step, with fewer resident CTAs).
template <typename T>
struct GemmSmem {
    static constexpr int TM = 64, TN = 64, KT = 16, PAD = 16 / sizeof(T);
    T As[2][KT][TM];
    T Bs[2][KT][TN + PAD];
    unsigned char sAg[2][KT][2];
    unsigned sBc[2][TN][2];
};

// rsub: rows of the task's tile to skip (0, or 64 for the lower half of
// a 128-row FP32 tile when it runs as two 64-row tiles on the FP32 pipe)
// mk: the task's slice masks (one per source pair; null: every slice live)
template <typename T>
__device__ __forceinline__ void gemm_body(const int32_t *tk, const int32_t *src,
                                          const BlockDesc *bd, T *val,
                                          GemmSmem<T> &sm, int rsub = 0,
                                          const uint32_t *mk = nullptr) {
    constexpr int TM = GemmSmem<T>::TM, TN = GemmSmem<T>::TN, KT = GemmSmem<T>::KT;
    constexpr int NQ = KT * TM / 256;              // staged elements per thread
    using Mask = typename std::conditional<KT == 64, unsigned long long, unsigned>::type;
    auto &As = sm.As;
    auto &Bs = sm.Bs;
    auto &sAg = sm.sAg;
    auto &sBc = sm.sBc;
    const BlockDesc d = bd[tk[0]];
    const int s0 = tk[1], s1 = tk[2], r0 = tk[3] + rsub, c0 = tk[4];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (r0 >= d.rows) return;                      // uniform: an empty half
    T acc[TN / 4];
#pragma unroll
    for (int g = 0; g < TN / 4; ++g) acc[g] = T(0);
    if (s0 >= s1) return;
    // slice (pair ss, first column kk0) can contribute (slices of 16 columns)
    auto live = [&](int ss, int kk0) -> bool {
        if (!mk) return true;
        const int sl = kk0 / 16;
        return sl >= 32 || ((mk[ss - s0] >> sl) & 1u);
    };
    int s = s0, k0 = 0;
    BlockDesc dl = bd[src[2 * s]], du = bd[src[2 * s + 1]];
    while (!live(s, k0)) {                         // uniform: the first live slice
        k0 += KT;
        if (k0 >= dl.cols) {
            if (++s >= s1) return;                 // nothing to add
            k0 = 0;
            dl = bd[src[2 * s]];
            du = bd[src[2 * s + 1]];
        }
    }
    // Slices are copied into shared memory by cp.async (no register round
    // trip, so the tile fits five CTAs per SM): element e = tid + 256 q of
    // the A slice is (row e % 64, k e / 64), of the B slice (k e % KT,
    // column e / KT); elements outside the blocks are zero-filled.
    auto issue = [&](const BlockDesc &L, const BlockDesc &U, int kk0, int b) {
        const T *A = val + L.voff;
        const T *B = val + U.voff;
        const int K = L.cols;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int e = tid + 256 * q;
            const int r = e % TM, k = e / TM;
            const int gr = r0 + r, gk = kk0 + k;
            const bool in = gr < d.rows && gk < K;
            cp_async_elem(&As[b][k][r], in ? A + (int64_t)gk * L.ld + gr : A, in);
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int e = tid + 256 * q;
            const int k = e % KT, c = e / KT;
            const int gk = kk0 + k, gc = c0 + c;
            const bool in = gk < K && gc < d.cols;
            cp_async_elem(&Bs[b][k][c], in ? B + (int64_t)gc * U.ld + gk : B, in);
        }
        cp_async_commit();
    };
    // After the thread's own copies landed: masks of the slice in buffer b.
    // Warp w's lanes hold rows 32 (w & 1) .. + 31 of A column k = (w + 8 q)
    // / 2, whose ballot gives four 8-row groups; for KT = 16 the warp holds
    // B columns 2 (w + 8 q) and + 1, lanes 0-15 and 16-31 over k = 0 .. 15;
    // for KT = 64 it holds column (w + 8 q) / 2 over k = 32 ((w + 8 q) & 1)
    // + lane.
    auto mark = [&](int b) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int e = tid + 256 * q;
            const unsigned m = __ballot_sync(0xffffffffu, nz(As[b][e / TM][e % TM]));
            if (lane == 0)
                sAg[b][(warp + 8 * q) >> 1][warp & 1] =
                    (unsigned char)(((m & 0xffu) ? 1u : 0u) | ((m & 0xff00u) ? 2u : 0u) |
                                    ((m & 0xff0000u) ? 4u : 0u) | ((m & 0xff000000u) ? 8u : 0u));
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int e = tid + 256 * q;
            const unsigned m = __ballot_sync(0xffffffffu, nz(Bs[b][e % KT][e / KT]));
            if (lane == 0) {
                const int wq = warp + 8 * q;
                if (KT == 64) {
                    sBc[b][wq >> 1][wq & 1] = m;
                } else {
                    sBc[b][2 * wq][0] = m & 0xffffu;
                    sBc[b][2 * wq + 1][0] = m >> 16;
                }
            }
        }
    };
    const int rr = 8 * warp + (lane & 7), cc = lane >> 3;
    issue(dl, du, k0, 0);
    mark(0);
    __syncthreads();
    int buf = 0;
    for (;;) {
        // advance to the next live slice
        int ns = s, nk0 = k0 + KT;
        BlockDesc nl = dl, nu = du;
        for (;;) {
            if (nk0 >= nl.cols) {
                ++ns;
                nk0 = 0;
                if (ns >= s1) break;
                nl = bd[src[2 * ns]];
                nu = bd[src[2 * ns + 1]];
            }
            if (live(ns, nk0)) break;
            nk0 += KT;
        }
        const bool more = ns < s1;
        // the other buffer was last read before the barrier that ended the
        // previous slice
        if (more) issue(nl, nu, nk0, buf ^ 1);
        // k mask of this warp's row group (lane k of the first KT reads it)
        Mask amk = __ballot_sync(
            0xffffffffu, lane < KT && ((sAg[buf][lane & (KT - 1)][warp >> 2] >> (warp & 3)) & 1u));
        if (KT == 64)
            amk |= (Mask)__ballot_sync(
                       0xffffffffu, ((sAg[buf][(lane + 32) & (KT - 1)][warp >> 2] >> (warp & 3)) & 1u))
                   << (KT == 64 ? 32 : 0);
        if (amk) {
#pragma unroll
            for (int g = 0; g < TN / 4; ++g) {
                Mask bm = (Mask)(sBc[buf][4 * g][0] | sBc[buf][4 * g + 1][0] |
                                 sBc[buf][4 * g + 2][0] | sBc[buf][4 * g + 3][0]);
                if (KT == 64)
                    bm |= (Mask)(sBc[buf][4 * g][1] | sBc[buf][4 * g + 1][1] |
                                 sBc[buf][4 * g + 2][1] | sBc[buf][4 * g + 3][1])
                          << (KT == 64 ? 32 : 0);
                Mask km = amk & bm;
                if (km) {                                   // uniform across the warp
                    // operands of the next live k load while this k's FMA issues
                    int k = (KT == 64 ? __ffsll((long long)km) : __ffs((int)km)) - 1;
                    km &= km - 1;
                    T a = As[buf][k][rr], b = Bs[buf][k][4 * g + cc];
                    while (km) {
                        k = (KT == 64 ? __ffsll((long long)km) : __ffs((int)km)) - 1;
                        km &= km - 1;
                        const T an = As[buf][k][rr], bn = Bs[buf][k][4 * g + cc];
                        acc[g] += a * b;
                        a = an;
                        b = bn;
                    }
                    acc[g] += a * b;
                }
            }
        }
        if (!more) break;
        mark(buf ^ 1);
        __syncthreads();
        buf ^= 1;
        s = ns;
        k0 = nk0;
        dl = nl;
        du = nu;
    }
    const int r = r0 + rr;
    if (r < d.rows) {
#pragma unroll
        for (int g = 0; g < TN / 4; ++g) {
            const int c = c0 + 4 * g + cc;
            if (c < d.cols && nz(acc[g])) val[d.voff + (int64_t)c * d.ld + r] -= acc[g];
        }
    }
}

// One CTA per tile; blockIdx.y picks the 64-row half of a 128-row tile.
// Five CTAs per SM: a CTA waiting for its next slice or at its barrier
// leaves the FP64 pipe to four others.
template <typename T>
__global__ void __launch_bounds__(256, 5)
k_ssssm_gemm(const int32_t *__restrict__ task, const int32_t *__restrict__ src,
             const BlockDesc *__restrict__ bd, T *__restrict__ val,
             const uint32_t *__restrict__ mask, const int64_t *__restrict__ moff) {
    extern __shared__ __align__(16) unsigned char gemm_raw[];   // sizeof(GemmSmem<T>)
    gemm_body<T>(task + 5 * (int64_t)blockIdx.x, src, bd, val,
                 *reinterpret_cast<GemmSmem<T> *>(gemm_raw), 64 * (int)blockIdx.y,
                 mask ? mask + moff[blockIdx.x] : nullptr);
}

// ------------------------------------------------------------ persistent
// The whole level walk in one launch (see slu_set_persistent): persistent
// CTAs (one per SM for FP64, two for FP32) take tickets in the order of a
// work list that lists, level by level, the GETRF, inverse, panel and
// Schur-tile tasks of every member of the plan, the Schur tiles split as in
// the per-level walk into those the next level reads and the deferred
// rest.  A task waits (thread 0, acquire at GPU scope, bounded) until two
// counters of its member reach their phases' task counts, runs the same
// body as the per-level kernel, and increments its own counter (barrier,
// fence, atomic).  Every ticket a CTA waits on was
// taken earlier by a CTA that is running, so the walk cannot deadlock; a
// wait that runs out sets bit 1 of cnt[2] and the CTA leaves (the others
// then run out too).  FP32 CTAs hold 64 TMEM columns for the tensor-core
// tiles from start to end.
enum : int32_t { kPtGetrf = 0, kPtInv = 1, kPtPanel = 2, kPtSchur = 3, kPtSchurLate = 4 };
constexpr int kPtInts = 7;   // kind, idx, wait1, need1, wait2, need2, done
// Dynamic shared memory of a persistent CTA (plus 1 KB for alignment).
template <typename T>
__host__ __device__ constexpr size_t persist_smem() { return sizeof(T) == 4 ? 108 * 1024 : kStageSmem; }

struct PersistArgs {
    const int32_t *tasks;               // kPtInts per task
    int ntasks;
    int *done;                          // counters
    int *ticket;
    const int32_t *gd, *inv_task, *pd_task, *gm_task, *gm_src;
    const uint32_t *gm_mask;            // slice masks, or null
    const int64_t *gm_moff;
    const BlockDesc *bd;
    BlockArgs a;
    const int64_t *woff;
    const double *scal;
    double tau_rel;
    unsigned long long *cnt;
    long long budget_ns;
    int tc_passes;
};

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1)
k_factor_persistent(PersistArgs p, T *val, T *winv) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_holder;
    __shared__ int s_t, s_stop;
    const int tid = threadIdx.x;
    uint32_t tmem = 0;
    uint32_t phase[2] = {0, 0};
    if (sizeof(T) == 4) tmem = tc_setup(mbar, &tmem_holder);
    const double tau = p.tau_rel * p.scal[0];
    for (;;) {
        if (tid == 0) {
            const int t = atomicAdd(p.ticket, 1);
            int stop = t >= p.ntasks;
            if (!stop) {
                const int32_t *pt = p.tasks + kPtInts * (int64_t)t;
                if ((pt[2] >= 0 && !wait_count(p.done + pt[2], pt[3], p.budget_ns)) ||
                    (pt[4] >= 0 && !wait_count(p.done + pt[4], pt[5], p.budget_ns))) {
                    atomicOr(&p.cnt[2], 2ull);
                    stop = 1;
                }
            }
            s_t = t;
            s_stop = stop;
        }
        __syncthreads();
        if (s_stop) break;                              // uniform
        const int32_t *pt = p.tasks + kPtInts * (int64_t)s_t;
        const int kind = pt[0], idx = pt[1];
        if (kind == kPtGetrf) {
            const BlockDesc d = p.bd[p.gd[idx]];
            getrf_dense<T>(val + d.voff, d.rows, d.ld, tau, p.cnt, smem, persist_smem<T>());
        } else if (kind == kPtInv) {
            if constexpr (sizeof(T) == 4)
                inv_body_reg<T>(p.inv_task + 3 * (int64_t)idx, p.bd, val, winv, p.woff);
            else
                inv_body<T>(p.inv_task + 3 * (int64_t)idx, p.bd, val, winv, p.woff, smem,
                            persist_smem<T>());
        } else if (kind == kPtPanel) {
            if constexpr (sizeof(T) == 4)
                panel_inv_dense_body<T>(p.pd_task + 4 * (int64_t)idx, p.bd, val, winv,
                                        p.woff, p.a, smem);
            else
                panel_inv_body<T>(p.pd_task + 4 * (int64_t)idx, p.bd, val, winv, p.woff,
                                  p.a, smem);
        } else {
            if constexpr (sizeof(T) == 4) {
                if (p.tc_passes > 0) {
                    tc_body(p.gm_task + 5 * (int64_t)idx, p.gm_src, p.bd,
                            reinterpret_cast<float *>(val), p.cnt + 2, smem, mbar, tmem,
                            phase, p.tc_passes);
                } else {
                    for (int half = 0; half < 2; ++half) {
                        gemm_body<T>(p.gm_task + 5 * (int64_t)idx, p.gm_src, p.bd, val,
                                     *reinterpret_cast<GemmSmem<T> *>(smem), 64 * half);
                        __syncthreads();         // the halves share the staging buffers
                    }
                }
            } else
                gemm_body<T>(p.gm_task + 5 * (int64_t)idx, p.gm_src, p.bd, val,
                             *reinterpret_cast<GemmSmem<T> *>(smem), 0,
                             p.gm_mask ? p.gm_mask + p.gm_moff[idx] : nullptr);
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicAdd(p.done + pt[6], 1);
        }
    }
    if (sizeof(T) == 4) tc_teardown(tmem);
}

// ---------------------------------------------------------------- host side

template <typename V, typename A>
static bool upload(const std::vector<V, A> &h, V **d) {
    *d = nullptr;
    if (h.empty()) return true;
    if (!cuda_ok(cudaMalloc(d, h.size() * sizeof(V)), "cudaMalloc(plan)"))
        return false;
    return cuda_ok(cudaMemcpy(*d, h.data(), h.size() * sizeof(V),
                              cudaMemcpyHostToDevice),
                   "cudaMemcpy(plan)");
}

void free_dev_plan(slu_plan *P) {
    DevPlan *D = P->dev;
    if (!D) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (D->device >= 0) cudaSetDevice(D->device);
    void *ptrs[] = {D->bd, D->lcolptr, D->lrow, D->dpos, D->sched, D->sgrp,
                    D->getrf, D->gessm, D->tstrf, D->tgt, D->src, D->srcoff,
                    D->gd, D->gs, D->dv_pos, D->dn_pos, D->lr_ptr, D->lr_pos,
                    D->ps_task, D->lr_col, D->ne_col, D->ne_off, D->pv_task,
                    D->ur_ptr, D->ur_pos, D->ur_col,
                    D->gm_task, D->gm_src, D->gm_mask, D->gm_moff, D->gg_tgt, D->gg_src,
                    D->gg_srcoff,
                    D->a2s, D->f2s, D->a_rowptr, D->a_vpos, D->a_colidx,
                    D->a_ri, D->a_ci, D->row_seg, D->woff, D->inv_task,
                    D->pd_task, D->pg_gessm, D->pg_tstrf,
                    D->lrow_off, D->urow_off, D->ucol_off, D->lcol_off,
                    D->lrow_blk, D->urow_blk, D->ucol_blk, D->lcol_blk};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (int sw = 0; sw < 4; ++sw) {
        if (D->sp_pairs[sw]) cudaFree(D->sp_pairs[sw]);
        if (D->sp_poff[sw]) cudaFree(D->sp_poff[sw]);
        if (D->sd_pair0[sw]) cudaFree(D->sd_pair0[sw]);
    }
    if (cur >= 0) cudaSetDevice(cur);
    delete D;
    P->dev = nullptr;
}

slu_status ensure_dev_plan(const slu_plan *cP) {
    slu_plan *P = const_cast<slu_plan *>(cP);
    int dev = -1;
    if (!cuda_ok(cudaGetDevice(&dev), "cudaGetDevice")) return SLU_ERR_CUDA;
    if (P->dev && P->dev->device == dev) return SLU_OK;
    if (P->dev) free_dev_plan(P);
    DevPlan *D = new DevPlan();
    D->device = dev;
    P->dev = D;
    bool ok =
        upload(P->blocks, &D->bd) && upload(P->lcolptr, &D->lcolptr) &&
        upload(P->lrow, &D->lrow) && upload(P->dpos, &D->dpos) &&
        upload(P->sched, &D->sched) && upload(P->sgrp, &D->sgrp) &&
        upload(P->getrf, &D->getrf) && upload(P->gessm, &D->gessm) &&
        upload(P->gd, &D->gd) && upload(P->gs, &D->gs) &&
        upload(P->dv_pos, &D->dv_pos) && upload(P->dn_pos, &D->dn_pos) &&
        upload(P->lr_ptr, &D->lr_ptr) && upload(P->lr_pos, &D->lr_pos) &&
        upload(P->lr_col, &D->lr_col) && upload(P->ps_task, &D->ps_task) &&
        upload(P->ne_col, &D->ne_col) && upload(P->ne_off, &D->ne_off) &&
        upload(P->pv_task, &D->pv_task) &&
        upload(P->ur_ptr, &D->ur_ptr) && upload(P->ur_pos, &D->ur_pos) &&
        upload(P->ur_col, &D->ur_col) &&
        upload(P->tstrf, &D->tstrf) && upload(P->tgt, &D->tgt) &&
        upload(P->src, &D->src) && upload(P->srcoff, &D->srcoff) &&
        upload(P->gm_task, &D->gm_task) && upload(P->gm_src, &D->gm_src) &&
        upload(P->gm_mask, &D->gm_mask) && upload(P->gm_moff, &D->gm_moff) &&
        upload(P->gg_tgt, &D->gg_tgt) && upload(P->gg_src, &D->gg_src) &&
        upload(P->gg_srcoff, &D->gg_srcoff) &&
        upload(P->a2s, &D->a2s) && upload(P->f2s, &D->f2s) &&
        upload(P->a_rowptr, &D->a_rowptr) && upload(P->a_vpos, &D->a_vpos) &&
        upload(P->a_colidx, &D->a_colidx) &&
        upload(P->a_rowidx, &D->a_ri) && upload(P->a_ci, &D->a_ci) &&
        upload(P->row_seg, &D->row_seg) && upload(P->woff, &D->woff) &&
        upload(P->inv_task, &D->inv_task) && upload(P->pd_task, &D->pd_task) &&
        upload(P->pg_gessm, &D->pg_gessm) && upload(P->pg_tstrf, &D->pg_tstrf) &&
        upload(P->lrow_off, &D->lrow_off) && upload(P->urow_off, &D->urow_off) &&
        upload(P->ucol_off, &D->ucol_off) && upload(P->lcol_off, &D->lcol_off) &&
        upload(P->lrow_blk, &D->lrow_blk) && upload(P->urow_blk, &D->urow_blk) &&
        upload(P->ucol_blk, &D->ucol_blk) && upload(P->lcol_blk, &D->lcol_blk);
    for (int sw = 0; ok && sw < 4; ++sw)
        ok = upload(P->sp_pairs[sw], &D->sp_pairs[sw]) &&
             upload(P->sp_poff[sw], &D->sp_poff[sw]) &&
             upload(P->sd_pair0[sw], &D->sd_pair0[sw]);
    if (!ok) {
        free_dev_plan(P);
        return SLU_ERR_CUDA;
    }
    return SLU_OK;
}

BlockArgs block_args(const slu_plan *P) {
    const DevPlan *D = P->dev;
    return BlockArgs{D->bd, D->lcolptr, D->lrow, D->dpos, D->sched, D->sgrp};
}

static int grid_for(int64_t n, int threads) {
    const int64_t g = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 148 * 32));
}

// Dynamic shared memory of the generic SSSSM kernel: per-warp accumulators
// of the largest block and up to 64 KB for a staged sparse source.
static size_t ssssm_smem(const slu_plan *P, size_t acc_size) {
    return std::min(kStageSmem,
                    align16((size_t)kWarps * P->maxb * acc_size) + 64 * 1024);
}

template <typename T, typename Acc>
static slu_status set_smem_limits(size_t generic) {
    const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    const int big = (int)std::max(generic, kStageSmem);
    bool ok = cuda_ok(cudaFuncSetAttribute(k_getrf<T>, attr, big), "smem") &&
              cuda_ok(cudaFuncSetAttribute(k_getrf_dense<T>, attr, (int)kStageSmem), "smem") &&
              cuda_ok(cudaFuncSetAttribute(k_panel<T, Acc>, attr, big), "smem") &&
              cuda_ok(cudaFuncSetAttribute(k_panel_inv<T>, attr, (int)kStageSmem), "smem") &&
              cuda_ok(cudaFuncSetAttribute(k_inv<T>, attr, (int)kStageSmem), "smem") &&
              cuda_ok(cudaFuncSetAttribute(k_ssssm_gemm<T>, attr, (int)sizeof(GemmSmem<T>)),
                      "smem") &&
              cuda_ok(cudaFuncSetAttribute(k_panel_grp<T>, attr, (int)kStageSmem), "smem") &&
              cuda_ok(cudaFuncSetAttribute(k_panel_vec<T>, attr, (int)kStageSmem), "smem") &&
              cuda_ok(cudaFuncSetAttribute(k_ssssm_tc, attr, (int)tc::SMEM), "smem") &&
              cuda_ok(cudaFuncSetAttribute(k_factor_persistent<T>, attr,
                                           (int)(persist_smem<T>() + 1024)), "smem");
    if (ok)
        ok = cuda_ok(cudaFuncSetAttribute(k_ssssm<T, Acc>, attr, (int)kStageSmem), "smem");
    return ok ? SLU_OK : SLU_ERR_CUDA;
}

template <typename T>
static slu_status run_factor(slu_handle *h, const double *values,
                             cudaStream_t st) {
    using Acc = T;     // FP64 path accumulates in FP64, FP32 path in FP32
    const slu_plan *P = h->plan;
    const DevPlan *D = P->dev;
    T *val = static_cast<T *>(h->storage);
    const BlockArgs a = block_args(P);
    if (!cuda_ok(cudaMemsetAsync(val, 0, P->storage * sizeof(T), st),
                 "cudaMemsetAsync(storage)") ||
        !cuda_ok(cudaMemsetAsync(h->scal, 0, 2 * sizeof(double), st),
                 "cudaMemsetAsync(scal)") ||
        !cuda_ok(cudaMemsetAsync(h->cnt, 0, 4 * sizeof(unsigned long long), st),
                 "cudaMemsetAsync(cnt)"))
        return SLU_ERR_CUDA;
    if (P->nnz_a > 0) {
        {
            LaunchScope ls_(h, SLU_KC_PREP, st);
            k_maxabs<<<grid_for(P->nnz_a, 256), 256, 0, st>>>(
                P->nnz_a, values, reinterpret_cast<unsigned long long *>(h->scal),
                h->cnt + 3);
        }
        {
            LaunchScope ls_(h, SLU_KC_PREP, st);
            k_anorm<<<(int)((P->n + 255) / 256), 256, 0, st>>>(
                P->n, D->a_rowptr, D->a_vpos, values,
                reinterpret_cast<unsigned long long *>(h->scal + 1));
        }
        if (h->anorm_seg) {
            const int nseg = (int)P->seg.size() - 1;
            if (!cuda_ok(cudaMemsetAsync(h->anorm_seg, 0, nseg * sizeof(double), st),
                         "cudaMemsetAsync"))
                return SLU_ERR_CUDA;
            LaunchScope ls_(h, SLU_KC_PREP, st);
            k_anorm_seg<<<(int)((P->n + 255) / 256), 256, 0, st>>>(
                P->n, D->a_rowptr, D->a_vpos, values, D->row_seg,
                reinterpret_cast<unsigned long long *>(h->anorm_seg));
        }
        if (!cuda_ok(cudaMemcpyAsync(h->a_vals, values, P->nnz_a * sizeof(double),
                                     cudaMemcpyDeviceToDevice, st),
                     "cudaMemcpyAsync(A)"))
            return SLU_ERR_CUDA;
        {
            LaunchScope ls_(h, SLU_KC_PREP, st);
            k_scatter<T><<<grid_for(P->nnz_a, 256), 256, 0, st>>>(P->nnz_a, D->a2s,
                                                                values, val);
        }
    }
    if (h->persistent) {                 // the whole level walk, one launch
        if (!cuda_ok(cudaMemsetAsync(h->pdone, 0, (h->pcounters + 1) * sizeof(int), st),
                     "cudaMemsetAsync(counters)"))
            return SLU_ERR_CUDA;
        int nsm = 148;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
        nsm *= sizeof(T) == 4 ? 2 : 1;       // resident CTAs per SM
        const int64_t budget_ms = P->opts.wait_budget_ms > 0 ? P->opts.wait_budget_ms : 2000;
        PersistArgs pa{h->ptasks, (int)h->pntasks, h->pdone, h->pdone + h->pcounters,
                       D->gd, D->inv_task, D->pd_task, D->gm_task, D->gm_src, D->gm_mask,
                       D->gm_moff, D->bd, a,
                       D->woff, h->scal, h->tau_rel, h->cnt, budget_ms * 1000000ll,
                       P->opts.tc_passes};
        {
            LaunchScope ls_(h, SLU_KC_PERSIST, st, nsm);
            k_factor_persistent<T><<<nsm, 256, persist_smem<T>() + 1024, st>>>(
                pa, val, static_cast<T *>(h->winv));
        }
        return cuda_ok(cudaGetLastError(), "persistent launch") ? SLU_OK : SLU_ERR_CUDA;
    }
    const size_t smem_f = (size_t)kWarps * P->maxb * sizeof(double);
    const size_t smem_a = (size_t)kWarps * P->maxb * sizeof(Acc);
    const size_t smem_big = std::max(kStageSmem, std::max(smem_f, smem_a));
    // generic SSSSM: per-warp accumulators plus room to stage a sparse source
    const size_t smem_g = ssssm_smem(P, sizeof(Acc));
    bool deferred = false;
    // the level walk on the handle's high-priority stream: when the deferred
    // Schur tiles of the side stream hold the SMs, the block scheduler takes
    // the chain's kernels first as resources free up
    const cudaStream_t caller = st;
    if (h->hi) {
        if (!cuda_ok(cudaEventRecord(h->ev_in, caller), "cudaEventRecord") ||
            !cuda_ok(cudaStreamWaitEvent(h->hi, h->ev_in, 0), "cudaStreamWaitEvent"))
            return SLU_ERR_CUDA;
        st = h->hi;
    }
    for (int lv = 0; lv < P->nlevels; ++lv) {
        h->cur_level = lv;
        const int64_t g0 = P->gd_off[lv], g1 = P->gd_off[lv + 1];
        if (g1 > g0) {
            // shared memory for the level's largest dense diagonal block
            int mb = 0;
            for (int64_t g = g0; g < g1; ++g) mb = std::max(mb, P->blocks[P->gd[g]].rows);
            size_t cap = kStageSmem;
            if (sizeof(T) == 8 && mb <= 128 && lu_owner_bytes(mb) <= kStageSmem)
                cap = lu_owner_bytes(mb);
            else if (sizeof(T) == 4 && (size_t)mb * mb * sizeof(T) <= kStageSmem)
                cap = (size_t)mb * mb * sizeof(T);
            LaunchScope ls_(h, SLU_KC_GETRF, st, (int)(g1 - g0));
            k_getrf_dense<T><<<(int)(g1 - g0), kDenseLuThreads, cap, st>>>(
                D->gd + g0, D->bd, val, h->scal, h->tau_rel, h->cnt, cap);
        }
        const int64_t q0 = P->gs_off[lv], q1 = P->gs_off[lv + 1];
        if (q1 > q0) {
            LaunchScope ls_(h, SLU_KC_GETRF, st, -(int)(q1 - q0));
            k_getrf<T><<<(int)(q1 - q0), kThreads, smem_big, st>>>(
                D->gs + q0, a, val, h->scal, h->tau_rel, h->cnt);
        }
        const int64_t i0 = P->inv_off[lv], i1 = P->inv_off[lv + 1];
        if (i1 > i0) {
            LaunchScope ls_(h, SLU_KC_INV, st, (int)(i1 - i0));
            // shared memory for the level's largest block: its vectors, plus
            // the block itself (staged once per CTA) when that fits
            int mb = 0;
            for (int64_t i = i0; i < i1; ++i) mb = std::max(mb, P->blocks[P->inv_task[3 * i]].rows);
            size_t sm = inv_smem_elems(mb) * sizeof(T);
            if (sizeof(T) == 8 && sm + (size_t)mb * mb * sizeof(T) <= kStageSmem)
                sm += (size_t)mb * mb * sizeof(T);
            if (sizeof(T) == 4) sm = 0;           // FP32: vectors in registers
            k_inv<T><<<(int)(i1 - i0), 256, sm, st>>>(
                D->inv_task + 3 * i0, D->bd, val, static_cast<T *>(h->winv), D->woff, sm);
        }
        const int64_t d0 = P->pd_off[lv], d1 = P->pd_off[lv + 1];
        if (d1 > d0) {
            LaunchScope ls_(h, SLU_KC_PANEL, st, (int)(d1 - d0));
            k_panel_inv<T><<<(int)(d1 - d0), 256,
                             ((size_t)P->inv_maxb * 64 + 2 * 16 * 64) * sizeof(T) +
                                 8 * (size_t)P->inv_maxb + 256, st>>>(
                D->pd_task + 4 * d0, D->bd, val, static_cast<const T *>(h->winv),
                D->woff, a);
        }
        const int64_t e0 = P->pg_goff[lv], e1 = P->pg_goff[lv + 1];
        const int64_t t0 = P->pg_toff[lv], t1 = P->pg_toff[lv + 1];
        if (e1 - e0 + t1 - t0 > 0) {
            LaunchScope ls_(h, SLU_KC_PANEL, st, -(int)(e1 - e0 + t1 - t0));
            k_panel<T, Acc><<<(int)(e1 - e0 + t1 - t0), kThreads, smem_big, st>>>(
                D->pg_gessm + 2 * e0, (int)(e1 - e0), D->pg_tstrf + 2 * t0, a, val);
        }
        // Schur updates: the part the next level reads runs on the main
        // stream; the deferred part runs on the side stream, overlapping
        // the next level's GETRF and panels, and is joined before the next
        // level's updates (a target gets its updates in level order)
        if (deferred) {
            if (!cuda_ok(cudaStreamWaitEvent(st, h->ev_join, 0), "cudaStreamWaitEvent"))
                return SLU_ERR_CUDA;
            deferred = false;
        }
        const int64_t w0 = P->pv_off[lv], w1 = P->pv_off[lv + 1];
        if (w1 > w0) {
            LaunchScope ls_(h, SLU_KC_PANEL, st, -(int)(w1 - w0));
            k_panel_vec<T><<<(int)(w1 - w0), 32, kStageSmem, st>>>(
                D->pv_task + 4 * w0, a, D->lr_ptr, D->lr_col, D->lr_pos, val);
        }
        const int64_t u0 = P->ps_off[lv], u1 = P->ps_off[lv + 1];
        if (u1 > u0) {
            LaunchScope ls_(h, SLU_KC_PANEL, st, -(int)(u1 - u0));
            k_panel_grp<T><<<(int)(u1 - u0), kThreads, kStageSmem, st>>>(
                D->ps_task + 3 * u0, a, D->lr_ptr, D->lr_col, D->lr_pos, val);
        }
        const int64_t m0 = P->gm_off[lv], mm = P->gm_mid[lv], m1 = P->gm_off[lv + 1];
        const int64_t s0 = P->gg_off[lv], sm = P->gg_mid[lv], s1 = P->gg_off[lv + 1];
        auto updates = [&](int64_t ma, int64_t mb, int64_t sa, int64_t sb,
                           cudaStream_t ss) {
            if (mb > ma) {
                LaunchScope ls_(h, SLU_KC_SSSSM, ss, (int)(mb - ma));
                if (sizeof(T) == 4 && P->opts.tc_passes > 0)
                    k_ssssm_tc<<<(int)(mb - ma), 256, tc::SMEM, ss>>>(
                        D->gm_task + 5 * ma, D->gm_src, D->bd,
                        reinterpret_cast<float *>(val), h->cnt + 2, P->opts.tc_passes);
                else if (sizeof(T) == 4)   // 128-row tiles as two 64-row halves
                    k_ssssm_gemm<T><<<dim3((unsigned)(mb - ma), 2), 256, sizeof(GemmSmem<T>), ss>>>(
                        D->gm_task + 5 * ma, D->gm_src, D->bd, val, D->gm_mask,
                        D->gm_moff ? D->gm_moff + ma : nullptr);
                else
                    k_ssssm_gemm<T><<<(int)(mb - ma), 256, sizeof(GemmSmem<T>), ss>>>(
                        D->gm_task + 5 * ma, D->gm_src, D->bd, val, D->gm_mask,
                        D->gm_moff ? D->gm_moff + ma : nullptr);
            }
            if (sb > sa) {
                LaunchScope ls_(h, SLU_KC_SSSSM, ss, -(int)(sb - sa));
                k_ssssm<T, Acc><<<(int)(sb - sa), kThreads, smem_g, ss>>>(
                    D->gg_tgt + sa, D->gg_srcoff + sa, D->gg_src, a, val,
                    D->ne_off, D->ne_col, smem_g);
            }
        };
        updates(m0, mm, s0, sm, st);
        if (m1 > mm || s1 > sm) {
            if (!cuda_ok(cudaEventRecord(h->ev_fork, st), "cudaEventRecord") ||
                !cuda_ok(cudaStreamWaitEvent(h->side, h->ev_fork, 0), "cudaStreamWaitEvent"))
                return SLU_ERR_CUDA;
            updates(mm, m1, sm, s1, h->side);
            if (!cuda_ok(cudaEventRecord(h->ev_join, h->side), "cudaEventRecord"))
                return SLU_ERR_CUDA;
            deferred = true;
        }
    }
    if (deferred &&
        !cuda_ok(cudaStreamWaitEvent(st, h->ev_join, 0), "cudaStreamWaitEvent"))
        return SLU_ERR_CUDA;
    if (st != caller &&
        (!cuda_ok(cudaEventRecord(h->ev_out, st), "cudaEventRecord") ||
         !cuda_ok(cudaStreamWaitEvent(caller, h->ev_out, 0), "cudaStreamWaitEvent")))
        return SLU_ERR_CUDA;
    h->cur_level = -1;
    if (!cuda_ok(cudaGetLastError(), "factor launch")) return SLU_ERR_CUDA;
    return SLU_OK;
}

// The handle's stream of the greatest priority and its fork / join events.
static bool create_hi_stream(slu_handle *h) {
    int least = 0, greatest = 0;
    return cuda_ok(cudaDeviceGetStreamPriorityRange(&least, &greatest), "priorities") &&
           cuda_ok(cudaStreamCreateWithPriority(&h->hi, cudaStreamNonBlocking, greatest),
                   "cudaStreamCreateWithPriority") &&
           cuda_ok(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming),
                   "cudaEventCreate") &&
           cuda_ok(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming),
                   "cudaEventCreate");
}

static slu_status finish_info(slu_handle *h, cudaStream_t st,
                              slu_factor_info *info) {
    unsigned long long c[4];
    double s[2];
    if (!cuda_ok(cudaMemcpyAsync(c, h->cnt, sizeof(c), cudaMemcpyDeviceToHost, st),
                 "cudaMemcpyAsync(info)") ||
        !cuda_ok(cudaMemcpyAsync(s, h->scal, sizeof(s), cudaMemcpyDeviceToHost, st),
                 "cudaMemcpyAsync(info)") ||
        !cuda_ok(cudaStreamSynchronize(st), "factor"))
        return SLU_ERR_CUDA;
    if (info) {
        info->nperturb = (int64_t)c[0];
        info->tau = h->tau_rel * s[0];
    }
    if (c[3]) return fail(SLU_ERR_INVALID_ARG, "A holds a NaN or infinite value");
    if (c[2] & 2)
        return fail(SLU_ERR_TIMEOUT,
                    "a dependency wait of the persistent launch exceeded wait_budget_ms");
    if (c[2] & 8)
        return fail(SLU_ERR_TIMEOUT, "a step wait of the dense diagonal LU exceeded its bound");
    if (c[2]) return fail(SLU_ERR_TIMEOUT, "a tensor-core wait exceeded its bound");
    if (c[1]) return fail(SLU_ERR_SINGULAR, "zero pivot (perturbation off)");
    return SLU_OK;
}

// Kernel attributes (dynamic shared memory limits), set once per handle
// before any launch so that graph recording captures stream work only.
slu_status init_solve_attrs(const slu_handle *h);
static slu_status init_factor_attrs(const slu_handle *h) {
    const slu_plan *P = h->plan;
    const size_t g = (size_t)kWarps * P->maxb * sizeof(double);
    return h->prec == SLU_PREC_FP64 ? set_smem_limits<double, double>(g)
                                    : set_smem_limits<float, float>(g);
}

slu_status factor_into(slu_handle *h, const double *values, cudaStream_t st) {
    return h->prec == SLU_PREC_FP64 ? run_factor<double>(h, values, st)
                                    : run_factor<float>(h, values, st);
}

}  // namespace slu

using namespace slu;

static std::mutex g_batch_mu;

extern "C" void slu_handle_destroy(slu_handle *h) {
    if (!h) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (h->device >= 0) cudaSetDevice(h->device);
    BatchShared *shared = nullptr;
    if (h->batch) {                  // member view: the arrays are the batch's
        h->storage = nullptr;
        h->winv = nullptr;
        h->a_vals = nullptr;
        std::lock_guard<std::mutex> lock(g_batch_mu);
        if (--h->batch->refs == 0) shared = h->batch;
    }
    for (cudaEvent_t e : h->pool) cudaEventDestroy(e);
    for (auto &g : h->sgraphs) cudaGraphExecDestroy(g.exec);
    if (h->xbuf) cudaFree(h->xbuf);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->hi) cudaStreamDestroy(h->hi);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    void *ptrs[] = {h->storage, h->a_vals, h->scal, h->cnt, h->work, h->red,
                    h->part, h->anorm_seg, h->winv, h->ptasks, h->pdone,
                    h->stasks[0], h->stasks[1], h->stasks[2], h->stasks[3], h->sdone,
                    h->spoff[0], h->spoff[1], h->spoff[2], h->spoff[3], h->spart};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (cur >= 0) cudaSetDevice(cur);
    delete h;
    if (shared) {
        slu_handle_destroy(shared->h);
        slu_plan_destroy(shared->plan);
        delete shared;
    }
}

extern "C" slu_status slu_factor(const slu_plan *P, const double *values,
                                 void *stream, slu_handle **out,
                                 slu_factor_info *info) {
    if (!P || !out) return fail(SLU_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (P->nnz_a > 0 && !values)
        return fail(SLU_ERR_INVALID_ARG, "values is NULL");
    slu_status st = ensure_dev_plan(P);
    if (st != SLU_OK) return st;
    slu_handle *h = new slu_handle();
    h->plan = P;
    cudaGetDevice(&h->device);
    h->prec = P->opts.precision;
    const bool fp64 = h->prec == SLU_PREC_FP64;
    // The pivot test and perturbation run in FP64 for both storage
    // precisions (an FP32 pivot is read from FP32 storage, compared in FP64
    // and stored back in FP32), with one threshold for both: sqrt(eps64) ~
    // 2^-26 of max|A| (2^-12, sqrt(eps32), exceeds genuine pivots of the
    // circuit matrices).
    if (P->opts.pivot_perturb)
        h->tau_rel = P->opts.pivot_tau_rel > 0 ? P->opts.pivot_tau_rel
                                               : std::ldexp(1.0, -26);
    const size_t esz = fp64 ? sizeof(double) : sizeof(float);
    const bool ok =
        cuda_ok(cudaMalloc(&h->storage, std::max<int64_t>(1, P->storage) * esz),
                "cudaMalloc(storage)") &&
        cuda_ok(cudaMalloc(&h->scal, 4 * sizeof(double)), "cudaMalloc") &&
        cuda_ok(cudaMalloc(&h->cnt, 4 * sizeof(unsigned long long)), "cudaMalloc") &&
        cuda_ok(cudaMalloc(&h->a_vals, std::max<int64_t>(1, P->nnz_a) * sizeof(double)),
                "cudaMalloc(A)") &&
        cuda_ok(cudaMalloc(&h->part, std::max<int64_t>(1, P->part_elems) * 4 *
                                         sizeof(double)),
                "cudaMalloc(solve partials)") &&
        cuda_ok(cudaMalloc(&h->winv, std::max<int64_t>(1, P->wsize) * esz),
                "cudaMalloc(inverses)") &&
        (P->seg.size() <= 2 ||
         cuda_ok(cudaMalloc(&h->anorm_seg, (P->seg.size() - 1) * sizeof(double)),
                 "cudaMalloc(anorm_seg)"));
    if (!ok) {
        slu_handle_destroy(h);
        return SLU_ERR_OUT_OF_MEMORY;
    }
    if (!cuda_ok(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking),
                 "cudaStreamCreate") ||
        !cuda_ok(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming),
                 "cudaEventCreate") ||
        !cuda_ok(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming),
                 "cudaEventCreate") ||
        !create_hi_stream(h)) {
        slu_handle_destroy(h);
        return SLU_ERR_CUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = init_factor_attrs(h);
    if (st == SLU_OK) st = init_solve_attrs(h);
    if (st == SLU_OK) st = factor_into(h, values, s);
    if (st == SLU_OK) st = finish_info(h, s, info);
    if (st != SLU_OK && st != SLU_ERR_SINGULAR) {
        slu_handle_destroy(h);
        return st;
    }
    *out = h;
    return st;
}

// Equal options, field by field (the struct has padding).
static bool same_opts(const slu_opts &a, const slu_opts &b) {
    return a.blocking == b.blocking && a.regular_block == b.regular_block &&
           a.sample_points == b.sample_points && a.step == b.step &&
           a.max_num == b.max_num && a.stride == b.stride && a.b_min == b.b_min &&
           a.precision == b.precision && a.dense_threshold == b.dense_threshold &&
           a.pivot_perturb == b.pivot_perturb && a.pivot_tau_rel == b.pivot_tau_rel &&
           a.refine_tol == b.refine_tol && a.refine_max_iter == b.refine_max_iter &&
           a.wait_budget_ms == b.wait_budget_ms && a.tc_passes == b.tc_passes;
}

// Where member q of batch plan M lives, checked against the member's own
// plan: its blocks are M's blocks [b0, b0 + nblocks) (block columns shifted
// by p0) with equal shapes, storage kinds and relative value offsets, and
// its dense diagonal blocks' inverses equally shifted.  The factorization of
// a block depends on that block's data and its own plan only, so the
// member's slice of M's storage is then exactly what slu_factor on the
// member's plan computes.
struct MemberSlice { int64_t voff, woff, aoff; };
static bool member_slice(const slu_plan *M, const slu_plan *Q, int32_t p0,
                         int64_t b0, int64_t aoff, MemberSlice *out) {
    const int64_t nb = (int64_t)Q->blocks.size();
    if (b0 + nb > (int64_t)M->blocks.size()) return false;
    const int64_t vbase = nb ? M->blocks[b0].voff - Q->blocks[0].voff : 0;
    for (int64_t b = 0; b < nb; ++b) {
        const BlockDesc &m = M->blocks[b0 + b], &q = Q->blocks[b];
        if (m.I != q.I + p0 || m.J != q.J + p0 || m.rows != q.rows ||
            m.cols != q.cols || m.dense != q.dense || m.ld != q.ld ||
            m.voff != q.voff + vbase)
            return false;
    }
    int64_t wbase = -1;
    for (int32_t I = 0; I < Q->p; ++I) {
        const int64_t wm = M->woff[p0 + I], wq = Q->woff[I];
        if ((wm < 0) != (wq < 0)) return false;
        if (wq < 0) continue;
        if (wbase < 0) wbase = wm - wq;
        if (wm != wq + wbase) return false;
    }
    out->voff = vbase;
    out->woff = wbase < 0 ? 0 : wbase;
    out->aoff = aoff;
    return true;
}

extern "C" slu_status slu_factor_batch(int32_t count, const slu_plan *const *plans,
                                       const double *const *values, void *stream,
                                       slu_handle **out, slu_factor_info *info) {
    if (count < 1 || !plans || !values || !out)
        return fail(SLU_ERR_INVALID_ARG, "bad batch arguments");
    for (int32_t q = 0; q < count; ++q) out[q] = nullptr;
    for (int32_t q = 0; q < count; ++q) {
        const slu_plan *Q = plans[q];
        if (!Q) return fail(SLU_ERR_INVALID_ARG, "NULL plan in the batch");
        if (Q->seg.size() > 2)
            return fail(SLU_ERR_NOT_SUPPORTED, "a batch member is itself a batch plan");
        if (!same_opts(Q->opts, plans[0]->opts))
            return fail(SLU_ERR_NOT_SUPPORTED, "batch members differ in their options");
        if (Q->nnz_a > 0 && !values[q])
            return fail(SLU_ERR_INVALID_ARG, "values is NULL for a batch member");
    }
    // the batch plan: the members' patterns block-diagonally, each blocked
    // on its own (the analysis of slu_analyze_batch)
    std::vector<int64_t> ns(count);
    std::vector<const int64_t *> cps(count);
    std::vector<const int32_t *> ris(count);
    for (int32_t q = 0; q < count; ++q) {
        ns[q] = plans[q]->n;
        cps[q] = plans[q]->a_colptr.data();
        ris[q] = plans[q]->a_rowidx.data();
    }
    slu_plan *M = nullptr;
    slu_status st = slu_analyze_batch(count, ns.data(), cps.data(), ris.data(),
                                      &plans[0]->opts, &M);
    if (st != SLU_OK) return st;
    std::vector<MemberSlice> sl(count);
    {
        int32_t p0 = 0;
        int64_t b0 = 0, aoff = 0;
        for (int32_t q = 0; q < count; ++q) {
            if (!member_slice(M, plans[q], p0, b0, aoff, &sl[q])) {
                slu_plan_destroy(M);
                return fail(SLU_ERR_NOT_SUPPORTED,
                            "batch member's blocks differ from its own plan's");
            }
            p0 += plans[q]->p;
            b0 += (int64_t)plans[q]->blocks.size();
            aoff += plans[q]->nnz_a;
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *vals = nullptr;
    if (!cuda_ok(cudaMalloc(&vals, std::max<int64_t>(1, M->nnz_a) * sizeof(double)),
                 "cudaMalloc(batch values)")) {
        slu_plan_destroy(M);
        return SLU_ERR_OUT_OF_MEMORY;
    }
    for (int32_t q = 0; q < count && st == SLU_OK; ++q)
        if (plans[q]->nnz_a > 0 &&
            !cuda_ok(cudaMemcpyAsync(vals + sl[q].aoff, values[q],
                                     plans[q]->nnz_a * sizeof(double),
                                     cudaMemcpyDeviceToDevice, s),
                     "cudaMemcpyAsync(batch values)"))
            st = SLU_ERR_CUDA;
    slu_handle *H = nullptr;
    if (st == SLU_OK) st = slu_factor(M, vals, stream, &H, info);  // synchronizes s
    if (st != SLU_OK && H == nullptr) cudaStreamSynchronize(s);
    cudaFree(vals);
    if (H == nullptr) {
        slu_plan_destroy(M);
        return st;
    }
    const slu_status fst = st;                  // SLU_OK or SLU_ERR_SINGULAR
    BatchShared *shared = new BatchShared();
    shared->plan = M;
    shared->h = H;
    const size_t esz = H->prec == SLU_PREC_FP64 ? sizeof(double) : sizeof(float);
    for (int32_t q = 0; q < count && st == fst; ++q) {
        const slu_plan *Q = plans[q];
        slu_status e = ensure_dev_plan(Q);
        if (e != SLU_OK) { st = e; break; }
        slu_handle *h = new slu_handle();
        h->plan = Q;
        h->device = H->device;
        h->prec = H->prec;
        h->tau_rel = H->tau_rel;
        h->storage = static_cast<char *>(H->storage) + sl[q].voff * esz;
        h->winv = static_cast<char *>(H->winv) + sl[q].woff * esz;
        h->a_vals = H->a_vals + sl[q].aoff;
        {
            std::lock_guard<std::mutex> lock(g_batch_mu);
            h->batch = shared;
            shared->refs++;
        }
        // the member's max|A| entry is the batch's (the threshold the
        // factorization used), its ||A||_inf its own
        const double *anorm = H->anorm_seg ? H->anorm_seg + q : H->scal + 1;
        const bool ok =
            cuda_ok(cudaMalloc(&h->scal, 4 * sizeof(double)), "cudaMalloc") &&
            cuda_ok(cudaMalloc(&h->cnt, 4 * sizeof(unsigned long long)), "cudaMalloc") &&
            cuda_ok(cudaMalloc(&h->part, std::max<int64_t>(1, Q->part_elems) * 4 *
                                             sizeof(double)),
                    "cudaMalloc(solve partials)") &&
            cuda_ok(cudaMemsetAsync(h->cnt, 0, 4 * sizeof(unsigned long long), s), "cudaMemsetAsync") &&
            cuda_ok(cudaMemcpyAsync(h->scal, H->scal, sizeof(double),
                                    cudaMemcpyDeviceToDevice, s), "cudaMemcpyAsync") &&
            cuda_ok(cudaMemcpyAsync(h->scal + 1, anorm, sizeof(double),
                                    cudaMemcpyDeviceToDevice, s), "cudaMemcpyAsync") &&
            cuda_ok(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking),
                    "cudaStreamCreate") &&
            cuda_ok(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming),
                    "cudaEventCreate") &&
            cuda_ok(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming),
                    "cudaEventCreate") &&
            create_hi_stream(h);
        out[q] = h;
        if (!ok) st = SLU_ERR_CUDA;
    }
    if (st == fst && !cuda_ok(cudaStreamSynchronize(s), "slu_factor_batch")) st = SLU_ERR_CUDA;
    if (st != fst) {
        const std::string msg = slu_last_error();
        {
            bool none = true;
            for (int32_t q = 0; q < count; ++q) none = none && !out[q];
            if (none) {                       // no member took a reference
                slu_handle_destroy(H);
                slu_plan_destroy(M);
                delete shared;
            }
        }
        for (int32_t q = 0; q < count; ++q) {
            slu_handle_destroy(out[q]);
            out[q] = nullptr;
        }
        return fail(st, msg);
    }
    return fst;
}

extern "C" slu_status slu_refactor(slu_handle *h, const double *values,
                                   void *stream, slu_factor_info *info) {
    if (!h) return fail(SLU_ERR_INVALID_ARG, "NULL handle");
    if (h->plan->nnz_a > 0 && !values)
        return fail(SLU_ERR_INVALID_ARG, "values is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    slu_status st = SLU_OK;
    if (h->use_graph) {
        if (s == nullptr)
            return fail(SLU_ERR_INVALID_ARG, "graph mode needs a created stream");
        if (!h->graph_exec || h->graph_values != values) {
            if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
            h->graph_exec = nullptr;
            cudaGraph_t g = nullptr;
            if (!cuda_ok(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal),
                         "cudaStreamBeginCapture"))
                return SLU_ERR_CUDA;
            const int64_t l0 = h->launches;
            h->capturing = true;
            st = factor_into(h, values, s);
            h->capturing = false;
            h->graph_launches = h->launches - l0;   // counted per replay below
            h->launches = l0;
            const cudaError_t e = cudaStreamEndCapture(s, &g);
            if (st != SLU_OK) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            if (!cuda_ok(e, "cudaStreamEndCapture")) return SLU_ERR_CUDA;
            // the nodes keep the priorities of the streams they were
            // recorded on (the level walk's high priority)
            const bool ok = cuda_ok(cudaGraphInstantiate(&h->graph_exec, g,
                                                         cudaGraphInstantiateFlagUseNodePriority),
                                    "cudaGraphInstantiate");
            cudaGraphDestroy(g);
            if (!ok) return SLU_ERR_CUDA;
            h->graph_values = values;
        }
        if (!cuda_ok(cudaGraphLaunch(h->graph_exec, s), "cudaGraphLaunch"))
            return SLU_ERR_CUDA;
        h->launches += h->graph_launches;
    } else {
        st = factor_into(h, values, s);
        if (st != SLU_OK) return st;
    }
    if (info) return finish_info(h, s, info);
    return SLU_OK;
}

extern "C" slu_status slu_set_graph(slu_handle *h, int32_t enable) {
    if (!h) return fail(SLU_ERR_INVALID_ARG, "NULL handle");
    h->use_graph = enable != 0;
    if (!h->use_graph && h->graph_exec) {
        cudaGraphExecDestroy(h->graph_exec);
        h->graph_exec = nullptr;
        h->graph_values = nullptr;
    }
    return SLU_OK;
}

// Work list of the persistent launch (kPtInts per task; see the header).
// Phases per level: 0 GETRF, 1 inverses, 2 panels, 3 Schur tiles the next
// level reads, 4 the deferred Schur tiles.  For member q, counter
// ((q L) + level) 5 + phase counts finished tasks.  The main chain 0 -> 1 ->
// 2 -> 3 -> next level's 0 is wait 1; wait 2 orders the deferred tiles: a
// level's GETRF, inverse and panel tasks wait for the deferred tiles of two
// levels back (which may target their blocks), its Schur tiles for those of
// the level before (every target receives its updates in level order).
static slu_status build_persistent(const slu_plan *P, std::vector<int32_t> &tasks,
                                   int64_t *ncounters) {
    if (!P->gs.empty() || !P->pg_gessm.empty() || !P->pg_tstrf.empty() ||
        !P->pv_task.empty() || !P->ps_task.empty() || !P->gg_tgt.empty())
        return fail(SLU_ERR_NOT_SUPPORTED,
                    "persistent launch: the plan has sparse-stored blocks or "
                    "diagonal blocks without explicit inverses");
    constexpr int NP = 5;
    const int64_t L = P->nlevels;
    const int64_t nseg = P->row_seg.empty() ? 1 : (int64_t)P->seg.size() - 1;
    const int64_t nc = nseg * L * NP;
    auto member = [&](int32_t blk) -> int64_t {
        return P->row_seg.empty() ? 0 : P->row_seg[P->blocks[blk].r0];
    };
    auto cid = [&](int64_t q, int64_t lv, int ph) { return (q * L + lv) * NP + ph; };
    std::vector<int32_t> count(nc, 0);
    struct Item { int32_t kind, idx; int64_t c; };
    std::vector<Item> items;
    for (int64_t lv = 0; lv < L; ++lv) {
        for (int64_t i = P->gd_off[lv]; i < P->gd_off[lv + 1]; ++i)
            items.push_back({kPtGetrf, (int32_t)i, cid(member(P->gd[i]), lv, 0)});
        for (int64_t i = P->inv_off[lv]; i < P->inv_off[lv + 1]; ++i)
            items.push_back({kPtInv, (int32_t)i, cid(member(P->inv_task[3 * i]), lv, 1)});
        for (int64_t i = P->pd_off[lv]; i < P->pd_off[lv + 1]; ++i)
            items.push_back({kPtPanel, (int32_t)i, cid(member(P->pd_task[4 * i + 2]), lv, 2)});
        for (int64_t i = P->gm_off[lv]; i < P->gm_mid[lv]; ++i)
            items.push_back({kPtSchur, (int32_t)i, cid(member(P->gm_task[5 * i]), lv, 3)});
        for (int64_t i = P->gm_mid[lv]; i < P->gm_off[lv + 1]; ++i)
            items.push_back({kPtSchurLate, (int32_t)i, cid(member(P->gm_task[5 * i]), lv, 4)});
    }
    for (const Item &it : items) count[it.c]++;
    // per counter its two waits
    std::vector<int64_t> w1(nc, -1), w2(nc, -1);
    std::vector<int64_t> late(L + 1, -1);   // late[l + 1]: last non-empty phase 4 at level <= l
    for (int64_t q = 0; q < nseg; ++q) {
        int64_t main = -1;
        for (int64_t lv = 0; lv < L; ++lv) {
            const int64_t c4 = cid(q, lv, 4);
            late[lv + 1] = count[c4] ? c4 : late[lv];
        }
        for (int64_t lv = 0; lv < L; ++lv) {
            for (int ph = 0; ph < 4; ++ph) {
                const int64_t c = cid(q, lv, ph);
                if (!count[c]) continue;
                w1[c] = main;
                w2[c] = ph < 3 ? (lv >= 1 ? late[lv - 1] : -1) : late[lv];
                main = c;
            }
            const int64_t c4 = cid(q, lv, 4);
            if (count[c4]) {
                // after the panels of its level (the last main phase before
                // the Schur tiles), and after the deferred tiles before it
                const int64_t c3 = cid(q, lv, 3);
                w1[c4] = count[c3] ? w1[c3] : main;
                w2[c4] = late[lv];
            }
        }
    }
    tasks.clear();
    tasks.reserve(items.size() * kPtInts);
    for (const Item &it : items) {
        const int64_t a = w1[it.c], b = w2[it.c];
        tasks.push_back(it.kind);
        tasks.push_back(it.idx);
        tasks.push_back((int32_t)a);
        tasks.push_back(a >= 0 ? count[a] : 0);
        tasks.push_back((int32_t)b);
        tasks.push_back(b >= 0 ? count[b] : 0);
        tasks.push_back((int32_t)it.c);
    }
    *ncounters = nc;
    return SLU_OK;
}

static slu_status upload_persistent(slu_handle *h, const std::vector<int32_t> &tasks,
                                    int64_t ncounters) {
    if (h->ptasks) cudaFree(h->ptasks);
    if (h->pdone) cudaFree(h->pdone);
    h->ptasks = nullptr;
    h->pdone = nullptr;
    h->pntasks = (int64_t)tasks.size() / kPtInts;
    h->pcap = h->pntasks;
    h->pcounters = ncounters;
    if (!cuda_ok(cudaMalloc(&h->ptasks, std::max<size_t>(1, tasks.size()) * sizeof(int32_t)),
                 "cudaMalloc(work list)") ||
        !cuda_ok(cudaMalloc(&h->pdone, (ncounters + 1) * sizeof(int)), "cudaMalloc(counters)"))
        return SLU_ERR_OUT_OF_MEMORY;
    if (!tasks.empty() &&
        !cuda_ok(cudaMemcpy(h->ptasks, tasks.data(), tasks.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice), "cudaMemcpy(work list)"))
        return SLU_ERR_CUDA;
    return SLU_OK;
}

extern "C" slu_status slu_set_persistent(slu_handle *h, int32_t enable) {
    if (!h) return fail(SLU_ERR_INVALID_ARG, "NULL handle");
    if (h->graph_exec) {                 // a recorded graph holds the old path
        cudaGraphExecDestroy(h->graph_exec);
        h->graph_exec = nullptr;
        h->graph_values = nullptr;
    }
    if (!enable) {
        h->persistent = false;
        return SLU_OK;
    }
    std::vector<int32_t> tasks;
    int64_t nc = 0;
    slu_status st = build_persistent(h->plan, tasks, &nc);
    if (st == SLU_OK) st = upload_persistent(h, tasks, nc);
    h->persistent = st == SLU_OK;
    return st;
}

extern "C" slu_status slu_persistent_tasks(const slu_handle *h, int32_t *tasks,
                                           int64_t cap, int64_t *count) {
    if (!h || !count) return fail(SLU_ERR_INVALID_ARG, "NULL argument");
    *count = h->persistent ? h->pntasks : 0;
    const int64_t k = std::min<int64_t>(std::max<int64_t>(cap, 0), *count);
    if (k > 0 && tasks &&
        !cuda_ok(cudaMemcpy(tasks, h->ptasks, k * kPtInts * sizeof(int32_t),
                            cudaMemcpyDeviceToHost), "cudaMemcpy(work list)"))
        return SLU_ERR_CUDA;
    return SLU_OK;
}

extern "C" slu_status slu_set_persistent_tasks(slu_handle *h, const int32_t *tasks,
                                               int64_t count) {
    if (!h || (count > 0 && !tasks) || count < 0)
        return fail(SLU_ERR_INVALID_ARG, "bad arguments");
    if (!h->persistent)
        return fail(SLU_ERR_INVALID_ARG, "persistent launch not enabled");
    const slu_plan *P = h->plan;
    const int64_t lim[5] = {(int64_t)P->gd.size(), (int64_t)P->inv_task.size() / 3,
                            (int64_t)P->pd_task.size() / 4, (int64_t)P->gm_task.size() / 5,
                            (int64_t)P->gm_task.size() / 5};
    if (count > h->pcap)
        return fail(SLU_ERR_INVALID_ARG, "work list longer than the built one");
    for (int64_t t = 0; t < count; ++t) {
        const int32_t *r = tasks + kPtInts * t;
        if (r[0] < 0 || r[0] > 4 || r[1] < 0 || r[1] >= lim[r[0]] || r[2] < -1 ||
            r[2] >= h->pcounters || r[4] < -1 || r[4] >= h->pcounters || r[6] < 0 ||
            r[6] >= h->pcounters)
            return fail(SLU_ERR_INVALID_ARG, "work list entry out of range");
    }
    if (count > 0 &&
        !cuda_ok(cudaMemcpy(h->ptasks, tasks, count * kPtInts * sizeof(int32_t),
                            cudaMemcpyHostToDevice), "cudaMemcpy(work list)"))
        return SLU_ERR_CUDA;
    h->pntasks = count;
    if (h->graph_exec) {
        cudaGraphExecDestroy(h->graph_exec);
        h->graph_exec = nullptr;
        h->graph_values = nullptr;
    }
    return SLU_OK;
}

extern "C" slu_status slu_set_profiling(slu_handle *h, int32_t enable) {
    if (!h) return fail(SLU_ERR_INVALID_ARG, "NULL handle");
    h->recs.clear();
    h->pool_next = 0;
    for (int c = 0; c < SLU_KC_COUNT; ++c) {
        h->calls[c] = 0;
        h->ms[c] = 0.0;
    }
    h->profiling = enable != 0;
    return SLU_OK;
}

extern "C" slu_status slu_handle_stats(slu_handle *h, slu_stats *out) {
    if (!h || !out) return fail(SLU_ERR_INVALID_ARG, "NULL argument");
    for (auto &r : h->recs)      // launches may sit on either stream
        if (!cuda_ok(cudaEventSynchronize(r.b), "cudaEventSynchronize"))
            return SLU_ERR_CUDA;
    for (auto &r : h->recs) {
        float t = 0.f;
        if (!cuda_ok(cudaEventElapsedTime(&t, r.a, r.b), "cudaEventElapsedTime"))
            return SLU_ERR_CUDA;
        h->calls[r.cls]++;
        h->ms[r.cls] += t;
    }
    h->recs.clear();
    h->pool_next = 0;
    out->launches = h->launches;
    for (int c = 0; c < SLU_KC_COUNT; ++c) {
        out->calls[c] = h->calls[c];
        out->ms[c] = h->ms[c];
    }
    return SLU_OK;
}

extern "C" slu_status slu_handle_trace(slu_handle *h, int64_t cap,
                                       int32_t *cls, float *ms, int32_t *level,
                                       int32_t *ctas, int64_t *count) {
    if (!h || !count) return fail(SLU_ERR_INVALID_ARG, "NULL argument");
    for (auto &r : h->recs)
        if (!cuda_ok(cudaEventSynchronize(r.b), "cudaEventSynchronize"))
            return SLU_ERR_CUDA;
    *count = (int64_t)h->recs.size();
    for (int64_t i = 0; i < std::min<int64_t>(cap, *count); ++i) {
        float t = 0.f;
        if (!cuda_ok(cudaEventElapsedTime(&t, h->recs[i].a, h->recs[i].b),
                     "cudaEventElapsedTime"))
            return SLU_ERR_CUDA;
        if (cls) cls[i] = h->recs[i].cls;
        if (ms) ms[i] = t;
        if (level) level[i] = h->recs[i].level;
        if (ctas) ctas[i] = h->recs[i].ctas;
    }
    return SLU_OK;
}

extern "C" slu_status slu_export_factors(const slu_handle *h, double *out,
                                         void *stream) {
    if (!h || !out) return fail(SLU_ERR_INVALID_ARG, "NULL argument");
    const slu_plan *P = h->plan;
    const int64_t nnz = P->f_colptr[P->n];
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (nnz == 0) return SLU_OK;
    LaunchScope ls_(h, SLU_KC_PREP, s);
    if (h->prec == SLU_PREC_FP64)
        k_export<double><<<grid_for(nnz, 256), 256, 0, s>>>(
            nnz, P->dev->f2s, static_cast<const double *>(h->storage), out);
    else
        k_export<float><<<grid_for(nnz, 256), 256, 0, s>>>(
            nnz, P->dev->f2s, static_cast<const float *>(h->storage), out);
    return cuda_ok(cudaGetLastError(), "export launch") ? SLU_OK : SLU_ERR_CUDA;
}
