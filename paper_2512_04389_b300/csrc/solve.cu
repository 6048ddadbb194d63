// Triangular solves with the block factors, FP64 residual and iterative
// refinement.  The paper covers only the factorization; solving with the
// factors, refining an FP32 factorization and the transposed solve used for
// differentiation complete the linear solver around it.
//
// Every solve walks the levels of the block dependency DAG (the same levels
// as the factorization): a level's diagonal blocks have no block coupling
// among themselves, so per level
//   1. the contributions of already solved blocks are pulled into partial
//      sums, one CTA per source block and row chunk (reduced later in a
//      fixed order: deterministic), then
//   2. each diagonal block is solved: a cluster of CTAs per dense block with
//      explicit inverses, one CTA per sparse block (by height groups).
// Sweep arithmetic is in the storage type of the factors; residuals, norms
// and the refinement update are FP64.  The sweeps of one solve are
// recorded once per right-hand-side count as a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <exception>
#include <mutex>
#include <type_traits>
#include <vector>

#include "device_common.cuh"

namespace slu {

template <typename C>
__device__ __forceinline__ C warp_sum(C v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(~0u, v, o);
    return v;
}

constexpr int RC = 4;   // right-hand sides processed together

// Loads of solution values and partial sums: read-only during a per-level
// launch (__ldg), but written by other CTAs of the same launch in the
// persistent sweep (COH: from L2, where those stores and atomics land).
template <bool COH, typename V>
__device__ __forceinline__ V ld_in(const V *p) {
    if constexpr (COH) return __ldcg(p);
    else return __ldg(p);
}
constexpr int kDenseRows = 64;   // rows of a dense source per pull CTA
enum Sweep { FWD = 0, BWD = 1, FWD_T = 2, BWD_T = 3 };

// Pull, scatter form (L y = b and U x = y): one CTA per source block B of
// the level (rows = the diagonal block's rows); part = B * x(B's columns),
// m x RC, reduced from per-warp partials in a fixed order.
template <typename T, bool COH>
__device__ __forceinline__ void pull_scatter_body(
    const int32_t *__restrict__ pairs, const int64_t *__restrict__ poff, const BlockArgs &a,
    const T *__restrict__ val, const double *X, int64_t ldx, int nc, double *part_d,
    int rows_per_chunk, int qi, int yi, unsigned char *smem) {
    using C = T;
    C *part = reinterpret_cast<C *>(part_d);
    const BlockDesc db = a.bd[pairs[2 * qi]];
    const int m = db.rows, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    C *pw = reinterpret_cast<C *>(smem);
    constexpr int VW = 16 / sizeof(T);                  // rows per vector load
    if (db.dense && db.ld % VW == 0) {
        // dense GEMV over the row chunk [y * kDenseRows, +kDenseRows): thread
        // (row group, column slice) accumulates VW rows over its columns
        // with 16-byte loads, 8 in flight; the column slices are reduced in
        // a fixed order.  Several CTAs share a block, so one large source
        // no longer runs at the bandwidth of a single SM.
        using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
        constexpr int NRG = kDenseRows / VW;            // row groups per chunk
        constexpr int NCG = kThreads / NRG;             // column slices
        const int rbase = yi * kDenseRows;
        if (rbase >= m) return;
        C *xs = pw;                                     // cols x RC
        C *red = pw + (size_t)db.cols * RC;             // NCG x kDenseRows x RC
        for (int t = threadIdx.x; t < db.cols * RC; t += kThreads) {
            const int k = t / RC, c = t % RC;
            xs[t] = c < nc ? ld_in<COH>(X + (int64_t)c * ldx + db.c0 + k) : 0.0;
        }
        __syncthreads();
        const int rg = threadIdx.x % NRG, cg = threadIdx.x / NRG;
        const int r0 = rbase + rg * VW;
        C acc[VW][RC];
#pragma unroll
        for (int i = 0; i < VW; ++i)
#pragma unroll
            for (int c = 0; c < RC; ++c) acc[i][c] = 0.0;
        if (r0 < m) {
            const T *base = val + db.voff + r0;
            for (int kb = cg; kb < db.cols; kb += NCG * 8) {
                V v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int k = kb + NCG * u;
                    if (k < db.cols)
                        v[u] = *reinterpret_cast<const V *>(base + (int64_t)k * db.ld);
                    else
                        v[u] = V{};
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int k = min(kb + NCG * u, db.cols - 1);
                    const T *vv = reinterpret_cast<const T *>(&v[u]);
#pragma unroll
                    for (int i = 0; i < VW; ++i)
#pragma unroll
                        for (int c = 0; c < RC; ++c) acc[i][c] += (C)vv[i] * xs[k * RC + c];
                }
            }
        }
#pragma unroll
        for (int i = 0; i < VW; ++i)
#pragma unroll
            for (int c = 0; c < RC; ++c)
                red[((size_t)cg * RC + c) * kDenseRows + rg * VW + i] = acc[i][c];
        __syncthreads();
        C *out = part + poff[qi] * RC;
        const int mr = min(kDenseRows, m - rbase);
        for (int t = threadIdx.x; t < mr * RC; t += kThreads) {
            const int r = t % mr, c = t / mr;
            C sum = 0.0;
            for (int g = 0; g < NCG; ++g) sum += red[((size_t)g * RC + c) * kDenseRows + r];
            out[c * m + rbase + r] = sum;                // index c * m + row
        }
        return;
    }
    // rows [rc0, rc0 + mc) of the partial (chunk yi)
    const int mc = min(m, rows_per_chunk), rc0 = yi * rows_per_chunk;
    if (rc0 >= m) return;
    const int mr = min(mc, m - rc0);
    for (int t = threadIdx.x; t < kWarps * mc * RC; t += kThreads) pw[t] = 0.0;
    __syncthreads();
    C *mine = pw + warp * mc * RC;
    for (int jj = warp; jj < db.cols; jj += kWarps) {
        C xv[RC];
        bool any = false;
#pragma unroll
        for (int c = 0; c < RC; ++c) {
            xv[c] = c < nc ? ld_in<COH>(X + (int64_t)c * ldx + db.c0 + jj) : 0.0;
            any |= xv[c] != 0.0;
        }
        if (any) {
            int64_t vb;
            int cn;
            const uint16_t *rows;
            colview(db, jj, a, vb, cn, rows);
            for (int e = lane; e < cn; e += 32) {
                const int r = rowat(rows, e) - rc0;
                if (r < 0 || r >= mr) continue;
                const C l = (C)val[vb + e];
                C *q = mine + r;                        // rhs-major: c * mc + r
#pragma unroll
                for (int c = 0; c < RC; ++c) q[c * mc] += l * xv[c];
            }
        }
        __syncwarp();
    }
    __syncthreads();
    C *out = part + poff[qi] * RC;
    for (int t = threadIdx.x; t < mr * RC; t += kThreads) {
        const int r = t % mr, c = t / mr;
        C sum = 0.0;
        for (int w = 0; w < kWarps; ++w) sum += pw[w * mc * RC + c * mc + r];
        out[c * m + rc0 + r] = sum;                     // index c * m + row
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_pull_scatter(const int32_t *__restrict__ pairs,
               const int64_t *__restrict__ poff, BlockArgs a,
               const T *__restrict__ val, const double *__restrict__ X,
               int64_t ldx, int nc, double *__restrict__ part_d,
               int rows_per_chunk) {
    extern __shared__ __align__(16) unsigned char smem[];
    pull_scatter_body<T, false>(pairs, poff, a, val, X, ldx, nc, part_d, rows_per_chunk,
                                (int)blockIdx.x, (int)blockIdx.y, smem);
}

// Pull, dot form (U^T z = g and L^T lam = z): one CTA per source block B
// (columns = the diagonal block's columns); part(ii) = B(:, ii) . x(B's rows).
template <typename T, bool COH>
__device__ __forceinline__ void pull_dot_body(
    const int32_t *__restrict__ pairs, const int64_t *__restrict__ poff, const BlockArgs &a,
    const T *__restrict__ val, const double *X, int64_t ldx, int nc, double *part_d,
    int qi) {
    using C = T;
    C *part = reinterpret_cast<C *>(part_d);
    const BlockDesc db = a.bd[pairs[2 * qi]];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    C *out = part + poff[qi] * RC;
    constexpr int VW = 16 / sizeof(T);
    if (db.dense && db.ld % VW == 0) {
        // dense: thread per column, streaming its contiguous column with
        // 16-byte loads, 8 in flight; x rows staged in shared memory
        using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
        __shared__ C xs[kThreads * RC];
        for (int ii0 = 0; ii0 < db.cols; ii0 += kThreads) {
            const int ii = ii0 + threadIdx.x;
            C acc[RC] = {0.0, 0.0, 0.0, 0.0};
            for (int r0 = 0; r0 < db.rows; r0 += kThreads) {
                const int nr = min(kThreads, db.rows - r0);
                __syncthreads();
                for (int t = threadIdx.x; t < nr * RC; t += kThreads) {
                    const int r = t / RC, c = t % RC;
                    xs[t] = c < nc ? ld_in<COH>(X + (int64_t)c * ldx + db.r0 + r0 + r) : 0.0;
                }
                __syncthreads();
                if (ii < db.cols) {
                    const T *col = val + db.voff + (int64_t)ii * db.ld + r0;
                    for (int rb = 0; rb < nr; rb += 8 * VW) {
                        V v[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int r = rb + u * VW;
                            if (r < nr) v[u] = *reinterpret_cast<const V *>(col + r);
                            else v[u] = V{};
                        }
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const T *vv = reinterpret_cast<const T *>(&v[u]);
#pragma unroll
                            for (int i = 0; i < VW; ++i) {
                                const int r = min(rb + u * VW + i, nr - 1);
#pragma unroll
                                for (int c = 0; c < RC; ++c)
                                    acc[c] += (C)vv[i] * xs[r * RC + c];
                            }
                        }
                    }
                }
            }
            if (ii < db.cols)
#pragma unroll
                for (int c = 0; c < RC; ++c) out[c * db.cols + ii] = acc[c];
        }
        return;
    }
    for (int ii = warp; ii < db.cols; ii += kWarps) {
        int64_t vb;
        int cn;
        const uint16_t *rows;
        colview(db, ii, a, vb, cn, rows);
        C sv[RC] = {0.0, 0.0, 0.0, 0.0};
        for (int e = lane; e < cn; e += 32) {
            const C l = (C)val[vb + e];
            const int64_t r = db.r0 + rowat(rows, e);
#pragma unroll
            for (int c = 0; c < RC; ++c)
                if (c < nc) sv[c] += l * ld_in<COH>(X + (int64_t)c * ldx + r);
        }
#pragma unroll
        for (int c = 0; c < RC; ++c) sv[c] = warp_sum(sv[c]);
        if (lane < RC) out[lane * db.cols + ii] = sv[lane];   // c * m + ii
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_pull_dot(const int32_t *__restrict__ pairs, const int64_t *__restrict__ poff,
           BlockArgs a, const T *__restrict__ val,
           const double *__restrict__ X, int64_t ldx, int nc,
           double *__restrict__ part_d) {
    pull_dot_body<T, false>(pairs, poff, a, val, X, ldx, nc, part_d, (int)blockIdx.x);
}

// One column step of a diagonal-block sweep; cv[e] is entry e of column jj
// (rows rows[e], diagonal at slot dp), y the m x RC right-hand sides.
template <typename C, int MODE>
__device__ __forceinline__ void chain_step(int jj, const C *cv,
                                           const uint16_t *rows, int cn,
                                           int dp, C *y, int lane) {
    if (MODE == FWD) {                 // unit lower, scatter below
        C xv[RC];
        bool any = false;
#pragma unroll
        for (int c = 0; c < RC; ++c) { xv[c] = y[jj * RC + c]; any |= xv[c] != 0.0; }
        if (any)
            for (int e = dp + 1 + lane; e < cn; e += 32) {
                C *q = y + rowat(rows, e) * RC;
#pragma unroll
                for (int c = 0; c < RC; ++c) q[c] -= cv[e] * xv[c];
            }
    } else if (MODE == BWD) {          // upper, divide then scatter above
        C xv[RC];
        bool any = false;
        const C piv = cv[dp];
#pragma unroll
        for (int c = 0; c < RC; ++c) { xv[c] = y[jj * RC + c] / piv; any |= xv[c] != 0.0; }
        __syncwarp();
        if (lane < RC) y[jj * RC + lane] = xv[lane];
        if (any)
            for (int e = lane; e < dp; e += 32) {
                C *q = y + rowat(rows, e) * RC;
#pragma unroll
                for (int c = 0; c < RC; ++c) q[c] -= cv[e] * xv[c];
            }
    } else {                           // transposed: gather dot
        C sv[RC] = {0.0, 0.0, 0.0, 0.0};
        const int e0 = MODE == FWD_T ? lane : dp + 1 + lane;
        const int e1 = MODE == FWD_T ? dp : cn;
        for (int e = e0; e < e1; e += 32) {
            const C *q = y + rowat(rows, e) * RC;
#pragma unroll
            for (int c = 0; c < RC; ++c) sv[c] += cv[e] * q[c];
        }
#pragma unroll
        for (int c = 0; c < RC; ++c) sv[c] = warp_sum(sv[c]);
        C zi = 0.0;
        if (lane < RC) {
            zi = y[jj * RC + lane] - sv[lane];
            if (MODE == FWD_T) zi /= cv[dp];
        }
        __syncwarp();
        if (lane < RC) y[jj * RC + lane] = zi;
    }
    __syncwarp();
}

// chain_step on values of storage type T (staged copy of the block).
template <typename T, int MODE>
__device__ __forceinline__ void chain_step_t(int jj, const T *cv,
                                             const uint16_t *rows, int cn,
                                             int dp, T *y, int lane) {
    if (MODE == FWD) {
        T xv[RC];
        bool any = false;
#pragma unroll
        for (int c = 0; c < RC; ++c) { xv[c] = y[jj * RC + c]; any |= xv[c] != 0.0; }
        if (any)
            for (int e = dp + 1 + lane; e < cn; e += 32) {
                T *q = y + rowat(rows, e) * RC;
                const T l = (T)cv[e];
#pragma unroll
                for (int c = 0; c < RC; ++c) q[c] -= l * xv[c];
            }
    } else if (MODE == BWD) {
        T xv[RC];
        bool any = false;
        const T piv = (T)cv[dp];
#pragma unroll
        for (int c = 0; c < RC; ++c) { xv[c] = y[jj * RC + c] / piv; any |= xv[c] != 0.0; }
        __syncwarp();
        if (lane < RC) y[jj * RC + lane] = xv[lane];
        if (any)
            for (int e = lane; e < dp; e += 32) {
                T *q = y + rowat(rows, e) * RC;
                const T u = (T)cv[e];
#pragma unroll
                for (int c = 0; c < RC; ++c) q[c] -= u * xv[c];
            }
    } else {
        T sv[RC] = {0.0, 0.0, 0.0, 0.0};
        const int e0 = MODE == FWD_T ? lane : dp + 1 + lane;
        const int e1 = MODE == FWD_T ? dp : cn;
        for (int e = e0; e < e1; e += 32) {
            const T *q = y + rowat(rows, e) * RC;
            const T l = (T)cv[e];
#pragma unroll
            for (int c = 0; c < RC; ++c) sv[c] += l * q[c];
        }
#pragma unroll
        for (int c = 0; c < RC; ++c) sv[c] = warp_sum(sv[c]);
        T zi = 0.0;
        if (lane < RC) {
            zi = y[jj * RC + lane] - sv[lane];
            if (MODE == FWD_T) zi /= (T)cv[dp];
        }
        __syncwarp();
        if (lane < RC) y[jj * RC + lane] = zi;
    }
    __syncwarp();
}

// Whether two value panels of W columns fit in cap bytes (as doubles).
template <typename T>
__device__ bool panels_fit(const BlockView<T> &F, int m, int W, size_t cap) {
    int64_t maxp = 0;
    for (int j0 = 0; j0 < m; j0 += W) {
        const int j1 = min(m, j0 + W);
        int o0, c0, o1, c1;
        const uint16_t *r0, *r1;
        F.col(j0, o0, c0, r0);
        F.col(j1 - 1, o1, c1, r1);
        maxp = max(maxp, (int64_t)(o1 + c1 - o0));
    }
    return (size_t)(2 * maxp) * sizeof(T) <= cap;
}

// Diagonal part of a sweep for a dense diagonal block with explicit
// inverses: one cluster of kInvCluster CTAs per block.  CTA q of the
// cluster owns rows [q h, q h + h), h = ceil(m / kInvCluster):
//   1. y(rows) = x(rows) minus the level's partials (fixed source order);
//   2. cluster barrier; every CTA copies the whole y from its peers'
//      shared memory (DSMEM); cluster barrier (no CTA leaves, or reuses
//      its buffer, while a peer may still read it);
//   3. out(rows) = M(rows, :) y with M = L^{-1}, U^{-1} (or the transposes
//      for the transposed sweeps), written to x.
constexpr int kInvCluster = 8;
template <typename T, int MODE>
__global__ void __cluster_dims__(kInvCluster, 1, 1) __launch_bounds__(kThreads)
k_diag_inv(const int32_t *__restrict__ pos, const int32_t *__restrict__ ids,
           const int64_t *__restrict__ pair0, const int64_t *__restrict__ boff,
           const int64_t *__restrict__ poff, const BlockDesc *__restrict__ bd,
           double *__restrict__ X, int64_t ldx, int nc,
           const double *__restrict__ part_d, const T *__restrict__ winv,
           const int64_t *__restrict__ woff) {
    using C = T;
    const C *part = reinterpret_cast<const C *>(part_d);
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned q;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(q));
    const int g = pos[blockIdx.x / kInvCluster];
    const BlockDesc dd = bd[ids[g]];
    const int m = dd.rows, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int h = (m + kInvCluster - 1) / kInvCluster;
    const int ra = min(m, (int)q * h), rb = min(m, ra + h), mh = rb - ra;
    C *yo = reinterpret_cast<C *>(smem);                 // own rows, h x RC
    C *y = yo + (size_t)h * RC;                          // all rows, m x RC
    C *red = y + (size_t)m * RC;                         // kWarps x h x RC
    const int64_t p0 = pair0[g];
    const int np = (int)(boff[dd.I + 1] - boff[dd.I]);
    // 1. own rows: x minus the partials (partials are c * m + row)
    for (int t = threadIdx.x; t < mh * RC; t += kThreads) {
        const int r = t % mh, c = t / mh;
        C acc = 0.0;
        for (int s = 0; s < np; ++s) acc += part[poff[p0 + s] * RC + (int64_t)c * m + ra + r];
        const C xv = c < nc ? (C)X[(int64_t)c * ldx + dd.r0 + ra + r] : C(0);
        yo[r * RC + c] = xv - acc;
    }
    asm volatile("barrier.cluster.arrive.release.aligned;\n"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
    // 2. gather y from the cluster
    {
        const uint32_t local = (uint32_t)__cvta_generic_to_shared(yo);
        for (int t = threadIdx.x; t < m * RC; t += kThreads) {
            const int r = t / RC, c = t % RC;
            const unsigned owner = (unsigned)(r / h);
            const uint32_t off = (uint32_t)(((r - (int)owner * h) * RC + c) * sizeof(C));
            uint32_t remote;
            asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                         : "=r"(remote) : "r"(local + off), "r"(owner));
            C v;
            if (sizeof(C) == 8) {
                double dv;
                asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(dv) : "r"(remote));
                v = (C)dv;
            } else {
                float fv;
                asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(fv) : "r"(remote));
                v = (C)fv;
            }
            y[t] = v;
        }
    }
    asm volatile("barrier.cluster.arrive.release.aligned;\n"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
    if (mh <= 0) return;
    const bool useL = (MODE == FWD || MODE == BWD_T);
    const T *M = winv + woff[dd.I] + (useL ? 0 : (int64_t)m * m);
    // 3. own rows of M y
    if (MODE == FWD || MODE == BWD) {
        // M column-major: lanes over rows (coalesced), warps over k; the k
        // range is the chunk's (the stored inverses hold exact zeros in the
        // other triangle), so a warp's lanes read one column together
        const int k0 = MODE == FWD ? 0 : ra, k1 = MODE == FWD ? rb : m;
        for (int rr = lane; rr < ((mh + 31) & ~31); rr += 32) {
            const int r = ra + rr;
            C acc[RC] = {0.0, 0.0, 0.0, 0.0};
            if (rr < mh) {
                for (int kb = k0 + warp; kb < k1; kb += kWarps * 4) {
                    C mv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int k = kb + kWarps * u;
                        mv[u] = k < k1 ? (C)M[(int64_t)k * m + r] : C(0);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int k = min(kb + kWarps * u, m - 1);
#pragma unroll
                        for (int c = 0; c < RC; ++c) acc[c] += mv[u] * y[k * RC + c];
                    }
                }
#pragma unroll
                for (int c = 0; c < RC; ++c) red[((size_t)warp * h + rr) * RC + c] = acc[c];
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < mh * RC; t += kThreads) {
            const int rr = t / RC, c = t % RC;
            C sum = 0.0;
            for (int w = 0; w < kWarps; ++w) sum += red[((size_t)w * h + rr) * RC + c];
            if (c < nc) X[(int64_t)c * ldx + dd.r0 + ra + rr] = sum;
        }
    } else {
        // transposed: out(r) = sum_k M(k, r) y(k), row r of M^T contiguous
        for (int rr = warp; rr < mh; rr += kWarps) {
            const int r = ra + rr;
            C acc[RC] = {0.0, 0.0, 0.0, 0.0};
            const int k0 = MODE == FWD_T ? 0 : r, k1 = MODE == FWD_T ? r + 1 : m;
            for (int kb = k0; kb < k1; kb += 128) {
                C mv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = kb + u * 32 + lane;
                    mv[u] = k < k1 ? (C)M[(int64_t)r * m + k] : C(0);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = min(kb + u * 32 + lane, m - 1);
#pragma unroll
                    for (int c = 0; c < RC; ++c) acc[c] += mv[u] * y[k * RC + c];
                }
            }
#pragma unroll
            for (int c = 0; c < RC; ++c) acc[c] = warp_sum(acc[c]);
            if (lane < nc) X[(int64_t)lane * ldx + dd.r0 + r] = acc[lane];
        }
    }
}

// y (m x RC, row-major, shared memory) = x(block rows) minus the block's
// partials, summed in the fixed order of its source list.
template <typename T, bool COH>
__device__ __forceinline__ void diag_load_y(const BlockDesc &dd, int64_t p0, int np,
                                            const int64_t *__restrict__ poff,
                                            const double *X, int64_t ldx, int nc,
                                            const double *part_d, T *y) {
    using C = T;
    const C *part = reinterpret_cast<const C *>(part_d);
    const int m = dd.rows;
    // partial offsets of this block's sources, staged once (the partials
    // themselves are then independent loads)
    __shared__ int64_t s_po[256];
    for (int t = threadIdx.x; t < m * RC; t += kThreads) {
        const int r = t / RC, c = t % RC;
        y[t] = c < nc ? X[(int64_t)c * ldx + dd.r0 + r] : 0.0;
    }
    for (int q0 = 0; q0 < np; q0 += 256) {
        const int nq = min(256, np - q0);
        __syncthreads();
        for (int q = threadIdx.x; q < nq; q += kThreads) s_po[q] = poff[p0 + q0 + q] * RC;
        __syncthreads();
        for (int t0 = 0; t0 < m * RC; t0 += 4 * kThreads) {
            C acc[4] = {0.0, 0.0, 0.0, 0.0};
            for (int q = 0; q < nq; q += 4) {
                C v[4][4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        const int t = t0 + w * kThreads + threadIdx.x;
                        v[u][w] = (q + u < nq && t < m * RC) ? ld_in<COH>(part + s_po[q + u] + t) : 0.0;
                    }
#pragma unroll
                for (int w = 0; w < 4; ++w)
                    acc[w] += (v[0][w] + v[1][w]) + (v[2][w] + v[3][w]);
            }
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const int t = t0 + w * kThreads + threadIdx.x;
                if (t < m * RC) {
                    const int r = t % m, c = t / m;     // partials are c * m + row
                    y[r * RC + c] -= acc[w];
                }
            }
        }
    }
}

// Dense diagonal block with explicit inverses: x(block rows) = M y,
//   L y -> L^{-1} y, U y -> U^{-1} y, U^T -> U^{-T}, L^T -> L^{-T}.
template <typename T, int MODE>
__device__ __forceinline__ void diag_inv_apply(const BlockDesc &dd, const T *__restrict__ winv,
                                               const int64_t *__restrict__ woff, double *X,
                                               int64_t ldx, int nc, T *y) {
    using C = T;
    const int m = dd.rows, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool useL = (MODE == FWD || MODE == BWD_T);
    const T *M = winv + woff[dd.I] + (useL ? 0 : (int64_t)m * m);
    C *o = y + m * RC;
    __syncthreads();
    if (MODE == FWD || MODE == BWD) {
        // out(r) = sum_k M(r, k) y(k): thread per row, coalesced over r;
        // loads issued 8 at a time ahead of their FMAs
        for (int r = threadIdx.x; r < m; r += kThreads) {
            C acc[RC] = {0.0, 0.0, 0.0, 0.0};
            const int k0 = MODE == FWD ? 0 : r, k1 = MODE == FWD ? r + 1 : m;
            for (int kb = k0; kb < k1; kb += 8) {
                C mv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    mv[u] = kb + u < k1 ? (C)M[(int64_t)(kb + u) * m + r] : 0.0;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int k = min(kb + u, m - 1);
#pragma unroll
                    for (int c = 0; c < RC; ++c) acc[c] += mv[u] * y[k * RC + c];
                }
            }
#pragma unroll
            for (int c = 0; c < RC; ++c) o[r * RC + c] = acc[c];
        }
    } else {
        // out(r) = sum_k M(k, r) y(k): warp per row, lanes over k
        for (int r = warp; r < m; r += kWarps) {
            C acc[RC] = {0.0, 0.0, 0.0, 0.0};
            const int k0 = MODE == FWD_T ? 0 : r, k1 = MODE == FWD_T ? r + 1 : m;
            for (int kb = k0; kb < k1; kb += 128) {
                C mv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = kb + u * 32 + lane;
                    mv[u] = k < k1 ? (C)M[(int64_t)r * m + k] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = min(kb + u * 32 + lane, m - 1);
#pragma unroll
                    for (int c = 0; c < RC; ++c) acc[c] += mv[u] * y[k * RC + c];
                }
            }
#pragma unroll
            for (int c = 0; c < RC; ++c) acc[c] = warp_sum(acc[c]);
            if (lane < RC) o[r * RC + lane] = acc[lane];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < m * RC; t += kThreads) {
        const int r = t / RC, c = t % RC;
        if (c < nc) X[(int64_t)c * ldx + dd.r0 + r] = o[t];
    }
}

// Diagonal part of a sweep: one CTA per diagonal block of the level.
// y = x(block rows) minus the level's partials (fixed order), then the
// chain over the block's columns by warp 0.  The block's index data is
// staged in shared memory; its values too if they fit, otherwise they are
// streamed through two column-panel buffers, warps 1-7 loading the next
// panel while warp 0 works on the current one.
template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads)
k_diag(const int32_t *__restrict__ pos, const int32_t *__restrict__ ids,
       const int64_t *__restrict__ pair0,
       const int64_t *__restrict__ boff, const int64_t *__restrict__ poff,
       BlockArgs a, const T *__restrict__ val, double *__restrict__ X,
       int64_t ldx, int nc, const double *__restrict__ part_d,
       const T *__restrict__ winv, const int64_t *__restrict__ woff,
       RowLists rl) {
    using C = T;
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int W = 16;
    const int gpos = pos[blockIdx.x];
    const BlockDesc dd = a.bd[ids[gpos]];
    const int m = dd.rows, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    C *y = reinterpret_cast<C *>(smem);
    const size_t ybytes = align16((size_t)m * RC * sizeof(C));
    const int64_t p0 = pair0[gpos];
    const int np = (int)(boff[dd.I + 1] - boff[dd.I]);
    diag_load_y<T, false>(dd, p0, np, poff, X, ldx, nc, part_d, y);
    if (woff[dd.I] >= 0) {
        diag_inv_apply<T, MODE>(dd, winv, woff, X, ldx, nc, y);
        return;
    }
    if (!dd.dense && 4 * dd.ngroups <= m) {
        // sparse block with few heights: rows of one height of the block's
        // column DAG do not depend on each other, so each height is one
        // parallel step (one thread per row, all right-hand sides), rows
        // pulling from the rows they depend on (row lists of L or U, or the
        // block's own columns for the transposed sweeps); ascending heights
        // for the lower-triangular sweeps, descending for the upper ones
        bool staged;
        size_t used;
        const BlockView<T> F = stage_block<T>(dd, a, const_cast<T *>(val),
                                              smem + ybytes, kStageSmem - ybytes,
                                              true, &staged, &used);
        const int ng = dd.ngroups;
        const int64_t rb = dd.doff + dd.I;
        const bool asc = (MODE == FWD || MODE == FWD_T);
        // the height schedule and (forward / backward) the row lists, staged
        // behind the block when they fit; row pointers rebased to the slice
        const int32_t *sched = a.sched + dd.doff, *grp = a.sgrp + dd.goff;
        const int32_t *pp = MODE == FWD ? rl.lp : rl.up;
        const uint16_t *pc = MODE == FWD ? rl.lc : rl.uc;
        const int32_t *pq = MODE == FWD ? rl.lq : rl.uq;
        int64_t pbase = rb;                      // pp index of row 0
        {
            unsigned char *lp = smem + ybytes + used;
            const size_t lcap = kStageSmem - ybytes - used;
            const bool rows = (MODE == FWD || MODE == BWD);
            const int32_t q0 = rows ? pp[rb] : 0;
            const int32_t nq = rows ? pp[rb + m] - q0 : 0;
            const size_t need = align16((size_t)m * 4) + align16((size_t)(ng + 1) * 4) +
                                (rows ? align16((size_t)(m + 1) * 4) + align16((size_t)nq * 2) +
                                        align16((size_t)nq * 4) : 0);
            if (need <= lcap) {
                int32_t *ss = reinterpret_cast<int32_t *>(lp);
                int32_t *sg = reinterpret_cast<int32_t *>(lp + align16((size_t)m * 4));
                for (int t = threadIdx.x; t < m; t += kThreads) ss[t] = sched[t];
                for (int t = threadIdx.x; t <= ng; t += kThreads) sg[t] = grp[t];
                if (rows) {
                    unsigned char *o = lp + align16((size_t)m * 4) + align16((size_t)(ng + 1) * 4);
                    int32_t *sp = reinterpret_cast<int32_t *>(o);
                    uint16_t *sc = reinterpret_cast<uint16_t *>(o + align16((size_t)(m + 1) * 4));
                    int32_t *sq = reinterpret_cast<int32_t *>(o + align16((size_t)(m + 1) * 4) +
                                                             align16((size_t)nq * 2));
                    for (int t = threadIdx.x; t <= m; t += kThreads) sp[t] = pp[rb + t] - q0;
                    for (int t = threadIdx.x; t < nq; t += kThreads) {
                        sc[t] = pc[q0 + t];
                        sq[t] = pq[q0 + t];
                    }
                    pp = sp;
                    pc = sc;
                    pq = sq;
                    pbase = 0;
                }
                sched = ss;
                grp = sg;
            }
        }
        __syncthreads();
        for (int gi = 0; gi < ng; ++gi) {
            const int g = asc ? gi : ng - 1 - gi;
            for (int t = grp[g] + threadIdx.x; t < grp[g + 1]; t += kThreads) {
                const int r = sched[t];
                C acc[RC];
#pragma unroll
                for (int c = 0; c < RC; ++c) acc[c] = y[r * RC + c];
                if (MODE == FWD || MODE == BWD) {
                    for (int q = pp[pbase + r]; q < pp[pbase + r + 1]; ++q) {
                        const C v = (C)F.v[pq[q]];
                        const int mm = pc[q];
#pragma unroll
                        for (int c = 0; c < RC; ++c) acc[c] -= v * y[mm * RC + c];
                    }
                } else {
                    int fo, fc;
                    const uint16_t *fr;
                    F.col(r, fo, fc, fr);
                    const int dp = F.dp[r];
                    const int e0 = MODE == FWD_T ? 0 : dp + 1, e1 = MODE == FWD_T ? dp : fc;
                    for (int e = e0; e < e1; ++e) {
                        const C v = (C)F.v[fo + e];
                        const int mm = fr[e];
#pragma unroll
                        for (int c = 0; c < RC; ++c) acc[c] -= v * y[mm * RC + c];
                    }
                }
                if (MODE == BWD || MODE == FWD_T) {
                    int fo, fc;
                    const uint16_t *fr;
                    F.col(r, fo, fc, fr);
                    const C dg = (C)F.v[fo + F.dp[r]];
#pragma unroll
                    for (int c = 0; c < RC; ++c) acc[c] /= dg;
                }
#pragma unroll
                for (int c = 0; c < RC; ++c) y[r * RC + c] = acc[c];
            }
            __syncthreads();
        }
        for (int t = threadIdx.x; t < m * RC; t += kThreads) {
            const int r = t / RC, c = t % RC;
            if (c < nc) X[(int64_t)c * ldx + dd.r0 + r] = y[t];
        }
        return;
    }
    // values as C: full copy if it fits, else panel buffers
    const int64_t nnz = dd.dense ? (int64_t)dd.ld * dd.cols
                                 : (int64_t)a.lcolptr[dd.coff + dd.cols];
    bool staged;
    size_t used;
    const size_t full = align16(nnz * sizeof(C));
    const BlockView<T> F = stage_block<T>(dd, a, const_cast<T *>(val),
                                          smem + ybytes, kStageSmem - ybytes,
                                          true, &staged, &used);
    // F.v is T; copy values into a C buffer for the chain
    unsigned char *vbuf = smem + ybytes + used;
    const size_t vcap = kStageSmem - ybytes - used;
    const bool whole = staged ? false : full <= vcap;
    const bool up = (MODE == FWD || MODE == FWD_T);
    if (staged || whole) {
        const T *src = F.v;
        C *vd = reinterpret_cast<C *>(vbuf);
        if (whole)
            for (int64_t e = threadIdx.x; e < nnz; e += kThreads) vd[e] = (C)src[e];
        __syncthreads();
        if (warp == 0)
            for (int k = 0; k < m; ++k) {
                const int jj = up ? k : m - 1 - k;
                int off, cn;
                const uint16_t *rows;
                F.col(jj, off, cn, rows);
                if (whole)
                    chain_step<C, MODE>(jj, vd + off, rows, cn, F.dp[jj], y, lane);
                else {
                    // staged T values: convert on the fly through registers
                    chain_step_t<T, MODE>(jj, F.v + off, rows, cn, F.dp[jj], y, lane);
                }
            }
    } else if (!panels_fit<T>(F, m, W, vcap)) {
        // neither the block nor two panels fit: read values in place
        __syncthreads();
        if (warp == 0)
            for (int k = 0; k < m; ++k) {
                const int jj = up ? k : m - 1 - k;
                int off, cn;
                const uint16_t *rows;
                F.col(jj, off, cn, rows);
                chain_step_t<T, MODE>(jj, F.v + off, rows, cn, F.dp[jj], y, lane);
            }
    } else {
        // panel streaming: W columns per panel, two buffers
        const int npan = (m + W - 1) / W;
        int64_t maxp = 0;
        for (int pn = 0; pn < npan; ++pn) {
            const int j0 = pn * W, j1 = min(m, j0 + W);
            int o0, c0, o1, c1;
            const uint16_t *r0, *r1;
            F.col(j0, o0, c0, r0);
            F.col(j1 - 1, o1, c1, r1);
            maxp = max(maxp, (int64_t)(o1 + c1 - o0));
        }
        C *buf[2] = {reinterpret_cast<C *>(vbuf),
                          reinterpret_cast<C *>(vbuf) + maxp};
        auto panel_of = [&](int q) { return up ? q : npan - 1 - q; };
        auto load = [&](int pn, C *dst, int t0, int nt) {
            const int j0 = pn * W, j1 = min(m, j0 + W);
            int o0, c0, o1, c1;
            const uint16_t *r0, *r1;
            F.col(j0, o0, c0, r0);
            F.col(j1 - 1, o1, c1, r1);
            for (int64_t e = t0; e < (int64_t)(o1 + c1 - o0); e += nt)
                dst[e] = (C)F.v[o0 + e];
        };
        load(panel_of(0), buf[0], threadIdx.x, kThreads);
        __syncthreads();
        for (int q = 0; q < npan; ++q) {
            const int pn = panel_of(q);
            if (warp == 0) {
                const int j0 = pn * W, j1 = min(m, j0 + W);
                int ob, cb;
                const uint16_t *rb;
                F.col(j0, ob, cb, rb);
                for (int k = 0; k < j1 - j0; ++k) {
                    const int jj = up ? j0 + k : j1 - 1 - k;
                    int off, cn;
                    const uint16_t *rows;
                    F.col(jj, off, cn, rows);
                    chain_step<C, MODE>(jj, buf[q & 1] + (off - ob), rows, cn,
                                     F.dp[jj], y, lane);
                }
            } else if (q + 1 < npan) {
                load(panel_of(q + 1), buf[(q + 1) & 1], threadIdx.x - 32,
                     kThreads - 32);
            }
            __syncthreads();
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < m * RC; t += kThreads) {
        const int r = t / RC, c = t % RC;
        if (c < nc) X[(int64_t)c * ldx + dd.r0 + r] = y[t];
    }
}

// R = B - A X (FP64), one warp per row of A's CSR view.
__global__ void k_residual(int64_t n, int nrhs, const int64_t *__restrict__ rp,
                           const int32_t *__restrict__ ci,
                           const int64_t *__restrict__ vpos,
                           const double *__restrict__ av,
                           const double *__restrict__ B, int64_t ldb,
                           const double *__restrict__ X, int64_t ldx,
                           double *__restrict__ R, int64_t ldr) {
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const int64_t q0 = rp[row], q1 = rp[row + 1];
    for (int c = 0; c < nrhs; ++c) {
        const double *x = X + (int64_t)c * ldx;
        double s = 0.0;
        for (int64_t q = q0 + lane; q < q1; q += 32) s += av[vpos[q]] * x[ci[q]];
        s = warp_sum(s);
        if (lane == 0) R[row + (int64_t)c * ldr] = B[row + (int64_t)c * ldb] - s;
    }
}

// red[3c] = max|R(:,c)|, red[3c+1] = max|X(:,c)|, red[3c+2] = max|B(:,c)|.
__global__ void k_norms(int64_t n, int nrhs, const double *__restrict__ R,
                        int64_t ldr, const double *__restrict__ X, int64_t ldx,
                        const double *__restrict__ B, int64_t ldb,
                        unsigned long long *__restrict__ red) {
    for (int c = 0; c < nrhs; ++c) {
        double a = 0.0, b = 0.0, d = 0.0;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x) {
            a = fmax(a, fabs(R[i + c * ldr]));
            b = fmax(b, fabs(X[i + c * ldx]));
            d = fmax(d, fabs(B[i + c * ldb]));
        }
        for (int o = 16; o > 0; o >>= 1) {
            a = fmax(a, __shfl_xor_sync(~0u, a, o));
            b = fmax(b, __shfl_xor_sync(~0u, b, o));
            d = fmax(d, __shfl_xor_sync(~0u, d, o));
        }
        if ((threadIdx.x & 31) == 0) {
            if (a > 0) atomicMax(&red[3 * c], (unsigned long long)__double_as_longlong(a));
            if (b > 0) atomicMax(&red[3 * c + 1], (unsigned long long)__double_as_longlong(b));
            if (d > 0) atomicMax(&red[3 * c + 2], (unsigned long long)__double_as_longlong(d));
        }
    }
}

// grad[p] = -sum_c Lam(row_p, c) X(col_p, c) over A's entries.
__global__ void k_grad_values(int64_t nnz, const int32_t *__restrict__ ri,
                              const int32_t *__restrict__ ci, int nrhs,
                              const double *__restrict__ Lam, int64_t ldl,
                              const double *__restrict__ X, int64_t ldx,
                              double *__restrict__ grad) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < nrhs; ++c)
            s += Lam[ri[p] + (int64_t)c * ldl] * X[ci[p] + (int64_t)c * ldx];
        grad[p] = -s;
    }
}

// Batch: red[(q * nrhs + c) * 3 + {0,1,2}] = max |R|, |X|, |B| over the
// rows of member q; warps whose 32 rows share a member reduce first.
__global__ void k_norms_seg(int64_t n, int nrhs, const double *__restrict__ R,
                            int64_t ldr, const double *__restrict__ X,
                            int64_t ldx, const double *__restrict__ B,
                            int64_t ldb, const int32_t *__restrict__ row_seg,
                            unsigned long long *__restrict__ red) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool in = i < n;
    const int q = in ? row_seg[i] : -1;
    const int q0 = __shfl_sync(~0u, q, 0);
    const bool same = __all_sync(~0u, q == q0 || !in);
    for (int c = 0; c < nrhs; ++c) {
        double v[3] = {0.0, 0.0, 0.0};
        if (in) {
            v[0] = fabs(R[i + c * ldr]);
            v[1] = fabs(X[i + c * ldx]);
            v[2] = fabs(B[i + c * ldb]);
        }
        if (same) {
            for (int o = 16; o > 0; o >>= 1)
                for (int k = 0; k < 3; ++k) v[k] = fmax(v[k], __shfl_xor_sync(~0u, v[k], o));
            if ((threadIdx.x & 31) == 0 && q0 >= 0)
                for (int k = 0; k < 3; ++k)
                    if (v[k] > 0)
                        atomicMax(&red[((int64_t)q0 * nrhs + c) * 3 + k],
                                  (unsigned long long)__double_as_longlong(v[k]));
        } else if (in) {
            for (int k = 0; k < 3; ++k)
                if (v[k] > 0)
                    atomicMax(&red[((int64_t)q * nrhs + c) * 3 + k],
                              (unsigned long long)__double_as_longlong(v[k]));
        }
    }
}

__global__ void k_add_cols(int64_t n, int nrhs, const double *__restrict__ D,
                           int64_t ldd, double *__restrict__ X, int64_t ldx) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
         i < n * nrhs; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i % n, c = i / n;
        X[r + c * ldx] += D[r + c * ldd];
    }
}

// k_diag_inv's arithmetic in one CTA (the persistent sweep): the rows are
// split into the cluster's kInvCluster row ranges only to reproduce its
// operation order -- y = x minus the partials added one source after the
// other; out(r) the sum over warps w = 0 .. 7, in order, of warp w's terms
// k = k0 + w, k0 + w + 8, ... (k0 the start of r's row range for U, 0 for
// L); the transposed forms lanes over k and a warp reduction, as there --
// so the solutions are bit for bit those of the per-level sweep.
template <typename T, int MODE, bool COH>
__device__ __forceinline__ void diag_inv_cta(const BlockDesc &dd, int64_t p0, int np,
                                             const int64_t *__restrict__ poff, double *X,
                                             int64_t ldx, int nc, const double *part_d,
                                             const T *__restrict__ winv,
                                             const int64_t *__restrict__ woff,
                                             unsigned char *smem) {
    using C = T;
    const C *part = reinterpret_cast<const C *>(part_d);
    const int m = dd.rows, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int h = (m + kInvCluster - 1) / kInvCluster;
    C *y = reinterpret_cast<C *>(smem);                  // m x RC
    C *red = y + (size_t)m * RC;                         // kWarps x m x RC
    for (int t = threadIdx.x; t < m * RC; t += kThreads) {
        const int r = t % m, c = t / m;
        C acc = 0.0;
        for (int q = 0; q < np; ++q)
            acc += ld_in<COH>(part + poff[p0 + q] * RC + (int64_t)c * m + r);
        const C xv = c < nc ? (C)X[(int64_t)c * ldx + dd.r0 + r] : C(0);
        y[r * RC + c] = xv - acc;
    }
    __syncthreads();
    const bool useL = (MODE == FWD || MODE == BWD_T);
    const T *M = winv + woff[dd.I] + (useL ? 0 : (int64_t)m * m);
    if (MODE == FWD || MODE == BWD) {
        for (int r = lane; r < m; r += 32) {
            const int ra = (r / h) * h, rb = min(m, ra + h);
            const int k0 = MODE == FWD ? 0 : ra, k1 = MODE == FWD ? rb : m;
            C acc[RC] = {0.0, 0.0, 0.0, 0.0};
            for (int kb = k0 + warp; kb < k1; kb += kWarps * 4) {
                C mv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = kb + kWarps * u;
                    mv[u] = k < k1 ? (C)M[(int64_t)k * m + r] : C(0);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = min(kb + kWarps * u, m - 1);
#pragma unroll
                    for (int c = 0; c < RC; ++c) acc[c] += mv[u] * y[k * RC + c];
                }
            }
#pragma unroll
            for (int c = 0; c < RC; ++c) red[((size_t)warp * m + r) * RC + c] = acc[c];
        }
        __syncthreads();
        for (int t = threadIdx.x; t < m * RC; t += kThreads) {
            const int r = t / RC, c = t % RC;
            C sum = 0.0;
            for (int w = 0; w < kWarps; ++w) sum += red[((size_t)w * m + r) * RC + c];
            if (c < nc) X[(int64_t)c * ldx + dd.r0 + r] = sum;
        }
    } else {
        for (int r = warp; r < m; r += kWarps) {
            C acc[RC] = {0.0, 0.0, 0.0, 0.0};
            const int k0 = MODE == FWD_T ? 0 : r, k1 = MODE == FWD_T ? r + 1 : m;
            for (int kb = k0; kb < k1; kb += 128) {
                C mv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = kb + u * 32 + lane;
                    mv[u] = k < k1 ? (C)M[(int64_t)r * m + k] : C(0);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = min(kb + u * 32 + lane, m - 1);
#pragma unroll
                    for (int c = 0; c < RC; ++c) acc[c] += mv[u] * y[k * RC + c];
                }
            }
#pragma unroll
            for (int c = 0; c < RC; ++c) acc[c] = warp_sum(acc[c]);
            if (lane < nc) X[(int64_t)lane * ldx + dd.r0 + r] = acc[lane];
        }
    }
}

// ------------------------------------------------------------ persistent
// One sweep in one launch (slu_set_persistent_solve): persistent CTAs take
// tickets in the order of the sweep's work list, which lists level by level
// (in the sweep's order) the level's pull tasks (a source block and a row
// chunk) and then its diagonal blocks.  A pull task waits (thread 0, an
// acquire at GPU scope, bounded) until the diagonal block whose solution it
// reads is done, a diagonal task until every pull into its block is; the
// bodies are those of the per-level kernels (a diagonal block by one CTA
// with the arithmetic of the cluster kernel); then barrier, fence and an
// atomic increment of the task's counter.  Every ticket waited on was taken
// earlier by a running CTA, so the sweep cannot deadlock; a wait that runs
// out sets bit 2 of cnt[2] and the CTA leaves (the others then run out).
enum : int32_t { kStPull = 0, kStDiag = 1 };
constexpr int kStInts = 6;   // kind, index, chunk, wait counter (-1: none), need, done counter

struct SolvePersistArgs {
    const int32_t *tasks;
    int ntasks;
    int *done;                 // counters
    int *ticket;
    const int32_t *pairs;      // the sweep's (source, diagonal) pairs
    const int64_t *poff;       // their partial offsets
    const int32_t *ids;        // GETRF list (diagonal block ids)
    const int64_t *pair0;      // first pair of each GETRF entry
    const int64_t *boff;       // sources per block row
    const int64_t *woff;
    BlockArgs a;
    unsigned long long *cnt;
    long long budget_ns;
    int rpc;                   // rows per chunk of a sparse source
};

template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads)
k_solve_persistent(SolvePersistArgs p, const T *__restrict__ val, const T *__restrict__ winv,
                   double *X, int64_t ldx, int nc, double *part) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_t, s_stop;
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = atomicAdd(p.ticket, 1);
            int stop = t >= p.ntasks;
            if (!stop) {
                const int32_t *pt = p.tasks + kStInts * (int64_t)t;
                if (pt[3] >= 0 && !wait_count(p.done + pt[3], pt[4], p.budget_ns)) {
                    atomicOr(&p.cnt[2], 4ull);
                    stop = 1;
                }
            }
            s_t = t;
            s_stop = stop;
        }
        __syncthreads();
        if (s_stop) break;                              // uniform
        const int32_t *pt = p.tasks + kStInts * (int64_t)s_t;
        if (pt[0] == kStPull) {
            if (MODE == FWD || MODE == BWD)
                pull_scatter_body<T, true>(p.pairs, p.poff, p.a, val, X, ldx, nc, part, p.rpc,
                                           pt[1], pt[2], smem);
            else
                pull_dot_body<T, true>(p.pairs, p.poff, p.a, val, X, ldx, nc, part, pt[1]);
        } else {
            const int g = pt[1];
            const BlockDesc dd = p.a.bd[p.ids[g]];
            diag_inv_cta<T, MODE, true>(dd, p.pair0[g], (int)(p.boff[dd.I + 1] - p.boff[dd.I]),
                                        p.poff, X, ldx, nc, part, winv, p.woff, smem);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(p.done + pt[5], 1);
        }
    }
}

// ---------------------------------------------------------------- host side

// Work list of a persistent sweep, built once per handle and sweep: level
// by level in the sweep's order, the level's pull tasks (only the row
// chunks a source has), then its diagonal blocks.  Counters: [0, p) block
// row solved, [p, 2p) pulls done into the block row.  Levels overlap in
// the persistent launch, so the partial offsets of the per-level launches
// (reused by every level) are rebased: level after level, past the end of
// the previous levels' partials.
template <typename T>
static slu_status persistent_solve_tasks(slu_handle *h, int mode, int rpc) {
    if (h->stasks[mode]) return SLU_OK;
    const slu_plan *P = h->plan;
    const int32_t p = P->p, L = P->nlevels;
    constexpr int VW = 16 / sizeof(T);
    const bool up = (mode == FWD || mode == FWD_T), scatter = (mode == FWD || mode == BWD);
    const auto &pairs = P->sp_pairs[mode];
    std::vector<int32_t> t;
    std::vector<int32_t> need(p, 0);
    std::vector<int64_t> off(pairs.size() / 2);    // partial offsets, all levels
    int64_t base = 0;
    try {
        for (int k = 0; k < L; ++k) {
            const int lv = up ? k : L - 1 - k;
            int64_t top = base;
            for (int64_t q = P->sp_off[mode][lv]; q < P->sp_off[mode][lv + 1]; ++q) {
                off[q] = base + P->sp_poff[mode][q];
                top = std::max<int64_t>(top, off[q] + P->blocks[pairs[2 * q + 1]].rows);
            }
            base = top;
            for (int64_t q = P->sp_off[mode][lv]; q < P->sp_off[mode][lv + 1]; ++q) {
                const BlockDesc &B = P->blocks[pairs[2 * q]];
                const int32_t I = P->blocks[pairs[2 * q + 1]].I;
                const int32_t src = scatter ? B.J : B.I;   // block row whose solution is read
                int chunks = 1;
                if (scatter) {
                    const int per = B.dense && B.ld % VW == 0 ? kDenseRows : std::min(B.rows, rpc);
                    chunks = (B.rows + per - 1) / per;
                }
                for (int y = 0; y < chunks; ++y) {
                    const int32_t e[kStInts] = {kStPull, (int32_t)q, y, src, 1, p + I};
                    t.insert(t.end(), e, e + kStInts);
                }
                need[I] += chunks;
            }
            for (int64_t g = P->getrf_off[lv]; g < P->getrf_off[lv + 1]; ++g) {
                const int32_t I = P->blocks[P->getrf[g]].I;
                const int32_t e[kStInts] = {kStDiag, (int32_t)g, 0, need[I] ? p + I : -1,
                                            need[I], I};
                t.insert(t.end(), e, e + kStInts);
            }
        }
    } catch (const std::exception &) {
        return fail(SLU_ERR_OUT_OF_MEMORY, "host allocation in the solve");
    }
    if (!h->sdone && !cuda_ok(cudaMalloc(&h->sdone, (2 * (size_t)p + 1) * sizeof(int)),
                              "cudaMalloc(solve counters)"))
        return SLU_ERR_OUT_OF_MEMORY;
    if (base * RC > h->spart_elems) {             // partials of the whole sweep
        if (h->spart) cudaFree(h->spart);
        h->spart = nullptr;
        h->spart_elems = 0;
        if (!cuda_ok(cudaMalloc(&h->spart, std::max<int64_t>(1, base * RC) * sizeof(double)),
                     "cudaMalloc(solve partials)"))
            return SLU_ERR_OUT_OF_MEMORY;
        h->spart_elems = base * RC;
    }
    int32_t *d = nullptr;
    int64_t *o = nullptr;
    if (!cuda_ok(cudaMalloc(&d, std::max<size_t>(1, t.size()) * sizeof(int32_t)),
                 "cudaMalloc(solve tasks)") ||
        !cuda_ok(cudaMalloc(&o, std::max<size_t>(1, off.size()) * sizeof(int64_t)),
                 "cudaMalloc(solve offsets)")) {
        if (d) cudaFree(d);
        return SLU_ERR_OUT_OF_MEMORY;
    }
    if ((!t.empty() && !cuda_ok(cudaMemcpy(d, t.data(), t.size() * sizeof(int32_t),
                                           cudaMemcpyHostToDevice), "cudaMemcpy(solve tasks)")) ||
        (!off.empty() && !cuda_ok(cudaMemcpy(o, off.data(), off.size() * sizeof(int64_t),
                                             cudaMemcpyHostToDevice), "cudaMemcpy(solve offsets)"))) {
        cudaFree(d);
        cudaFree(o);
        return SLU_ERR_CUDA;
    }
    h->stasks[mode] = d;
    h->spoff[mode] = o;
    h->sntasks[mode] = (int64_t)t.size() / kStInts;
    return SLU_OK;
}

// Rows per chunk of a sparse pull source and the pull kernels' shared
// memory (as the per-level sweep computes them).
template <typename T>
static void pull_shape(const slu_plan *P, int *rpc, size_t *smem) {
    *rpc = (int)std::min<int64_t>(P->maxb, kStageSmem / ((size_t)kWarps * RC * sizeof(double)));
    constexpr size_t kSlices = kThreads / (kDenseRows / (16 / sizeof(T)));
    *smem = std::max<size_t>((size_t)kWarps * *rpc * RC * sizeof(double),
                             ((size_t)P->maxb + kSlices * kDenseRows) * RC * sizeof(T));
}

// The four sweeps' work lists, kernel attributes and grids (outside any
// stream capture: allocations and copies).
template <typename T, int MODE>
static slu_status persistent_solve_setup(slu_handle *h) {
    const slu_plan *P = h->plan;
    int rpc;
    size_t pull_smem;
    pull_shape<T>(P, &rpc, &pull_smem);
    if (pull_smem > kStageSmem) return fail(SLU_ERR_NOT_SUPPORTED, "block too large for the solve");
    slu_status s = persistent_solve_tasks<T>(h, MODE, rpc);
    if (s != SLU_OK) return s;
    const size_t sm = std::max(pull_smem, (1 + kWarps) * (size_t)P->maxb * RC * sizeof(T));
    int per_sm = 0, dev = 0, sms = 0;
    if (!cuda_ok(cudaFuncSetAttribute(k_solve_persistent<T, MODE>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                 "attr") ||
        !cuda_ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                     &per_sm, k_solve_persistent<T, MODE>, kThreads, sm), "occupancy") ||
        !cuda_ok(cudaGetDevice(&dev), "device") ||
        !cuda_ok(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device"))
        return SLU_ERR_CUDA;
    if (per_sm < 1) return fail(SLU_ERR_NOT_SUPPORTED, "block too large for the solve");
    h->ssmem[MODE] = sm;
    h->sgrid[MODE] = (int)std::min<int64_t>((int64_t)sms * per_sm,
                                            std::max<int64_t>(1, h->sntasks[MODE]));
    return SLU_OK;
}

template <typename T>
static slu_status persistent_solve_setup_all(slu_handle *h) {
    slu_status s = persistent_solve_setup<T, FWD>(h);
    if (s == SLU_OK) s = persistent_solve_setup<T, BWD>(h);
    if (s == SLU_OK) s = persistent_solve_setup<T, FWD_T>(h);
    if (s == SLU_OK) s = persistent_solve_setup<T, BWD_T>(h);
    return s;
}

// One sweep over the levels (ascending for L and U^T, descending for U and
// L^T), in chunks of RC right-hand sides; per level a pull launch (one CTA
// per source block) and a diagonal launch (one CTA per diagonal block).
template <typename T, int MODE>
static slu_status sweep_t(const slu_handle *h, double *X, int64_t ldx,
                          int nrhs, cudaStream_t st) {
    const slu_plan *P = h->plan;
    const DevPlan *D = P->dev;
    const T *val = static_cast<const T *>(h->storage);
    const BlockArgs a = block_args(P);
    // sparse sources keep kWarps partials of (rows x RC); split the rows
    // into chunks when a whole block's partials do not fit
    const int rpc = (int)std::min<int64_t>(
        P->maxb, kStageSmem / ((size_t)kWarps * RC * sizeof(double)));
    const int nch = std::max((P->maxb + rpc - 1) / rpc,
                             (P->maxb + kDenseRows - 1) / kDenseRows);
    // dense sources: x (cols x RC) + one row chunk of partials per column
    // slice (kThreads / (kDenseRows / VW) slices, VW = 16 / sizeof(T))
    constexpr size_t kSlices = kThreads / (kDenseRows / (16 / sizeof(T)));
    const size_t pull_smem = std::max<size_t>(
        (size_t)kWarps * rpc * RC * sizeof(double),
        ((size_t)P->maxb + kSlices * kDenseRows) * RC * sizeof(T));
    if (pull_smem > kStageSmem)
        return fail(SLU_ERR_NOT_SUPPORTED, "block too large for the solve");
    const int64_t *boff = MODE == FWD ? D->lrow_off : MODE == BWD ? D->urow_off
                        : MODE == FWD_T ? D->ucol_off : D->lcol_off;
    const bool up = (MODE == FWD || MODE == FWD_T);
    if (h->persistent_solve) {
        // work list, grid and shared memory set up by slu_set_persistent_solve
        const size_t sm = h->ssmem[MODE];
        if (!h->stasks[MODE] || h->sgrid[MODE] < 1)
            return fail(SLU_ERR_INVALID_ARG, "persistent solve not set up");
        const int64_t budget = P->opts.wait_budget_ms > 0 ? P->opts.wait_budget_ms : 2000;
        const int ntasks = (int)h->sntasks[MODE];
        SolvePersistArgs pa{h->stasks[MODE], ntasks, h->sdone, h->sdone + 2 * P->p,
                            D->sp_pairs[MODE], h->spoff[MODE], D->getrf, D->sd_pair0[MODE],
                            boff, D->woff, a, h->cnt, budget * 1000000ll, rpc};
        const int grid = h->sgrid[MODE];
        for (int c0 = 0; c0 < nrhs; c0 += RC) {
            const int nc = std::min(RC, nrhs - c0);
            if (!cuda_ok(cudaMemsetAsync(h->sdone, 0, (2 * (size_t)P->p + 1) * sizeof(int), st),
                         "cudaMemsetAsync"))
                return SLU_ERR_CUDA;
            LaunchScope ls_(h, SLU_KC_PERSIST, st, grid);
            k_solve_persistent<T, MODE><<<grid, kThreads, sm, st>>>(
                pa, val, static_cast<const T *>(h->winv), X + (int64_t)c0 * ldx, ldx, nc,
                h->spart);
        }
        return cuda_ok(cudaGetLastError(), "solve launch") ? SLU_OK : SLU_ERR_CUDA;
    }
    for (int c0 = 0; c0 < nrhs; c0 += RC) {
        const int nc = std::min(RC, nrhs - c0);
        double *Xc = X + (int64_t)c0 * ldx;
        for (int k = 0; k < P->nlevels; ++k) {
            const int lv = up ? k : P->nlevels - 1 - k;
            const int64_t q0 = P->sp_off[MODE][lv], q1 = P->sp_off[MODE][lv + 1];
            if (q1 > q0) {
                LaunchScope ls_(h, SLU_KC_SOLVE, st);
                if (MODE == FWD || MODE == BWD)
                    k_pull_scatter<T><<<dim3((unsigned)(q1 - q0), (unsigned)nch),
                                        kThreads, pull_smem, st>>>(
                        D->sp_pairs[MODE] + 2 * q0, D->sp_poff[MODE] + q0, a, val,
                        Xc, ldx, nc, h->part, rpc);
                else
                    k_pull_dot<T><<<(int)(q1 - q0), kThreads, 0, st>>>(
                        D->sp_pairs[MODE] + 2 * q0, D->sp_poff[MODE] + q0, a, val,
                        Xc, ldx, nc, h->part);
            }
            // diagonal blocks with explicit inverses: a cluster each; the
            // rest: one CTA each
            const int64_t v0 = P->dv_off[lv], v1 = P->dv_off[lv + 1];
            if (v1 > v0) {
                LaunchScope ls_(h, SLU_KC_DIAG, st, (int)(v1 - v0));
                const int hh = (P->inv_maxb + kInvCluster - 1) / kInvCluster;
                const size_t sm = (size_t)(hh + P->inv_maxb + kWarps * hh) * RC * sizeof(T);
                k_diag_inv<T, MODE><<<(int)(v1 - v0) * kInvCluster, kThreads, sm, st>>>(
                    D->dv_pos + v0, D->getrf, D->sd_pair0[MODE], boff,
                    D->sp_poff[MODE], D->bd, Xc, ldx, nc, h->part,
                    static_cast<const T *>(h->winv), D->woff);
            }
            const int64_t n0 = P->dn_off[lv], n1 = P->dn_off[lv + 1];
            if (n1 > n0) {
                LaunchScope ls_(h, SLU_KC_DIAG, st, -(int)(n1 - n0));
                k_diag<T, MODE><<<(int)(n1 - n0), kThreads, kStageSmem, st>>>(
                    D->dn_pos + n0, D->getrf, D->sd_pair0[MODE], boff,
                    D->sp_poff[MODE], a, val, Xc, ldx, nc, h->part,
                    static_cast<const T *>(h->winv), D->woff,
                    RowLists{D->lr_ptr, D->lr_col, D->lr_pos, D->ur_ptr, D->ur_col,
                             D->ur_pos});
            }
        }
    }
    return cuda_ok(cudaGetLastError(), "solve launch") ? SLU_OK : SLU_ERR_CUDA;
}

template <typename T>
static bool solve_attrs_t() {
    const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    const int b = (int)kStageSmem;
    return cuda_ok(cudaFuncSetAttribute(k_diag<T, FWD>, attr, b), "attr") &&
           cuda_ok(cudaFuncSetAttribute(k_diag<T, BWD>, attr, b), "attr") &&
           cuda_ok(cudaFuncSetAttribute(k_diag<T, FWD_T>, attr, b), "attr") &&
           cuda_ok(cudaFuncSetAttribute(k_diag<T, BWD_T>, attr, b), "attr") &&
           cuda_ok(cudaFuncSetAttribute(k_pull_scatter<T>, attr, b), "attr");
}

template <typename T>
static slu_status sweep(const slu_handle *h, Sweep sw, double *X, int64_t ldx,
                        int nrhs, cudaStream_t st) {
    switch (sw) {
        case FWD: return sweep_t<T, FWD>(h, X, ldx, nrhs, st);
        case BWD: return sweep_t<T, BWD>(h, X, ldx, nrhs, st);
        case FWD_T: return sweep_t<T, FWD_T>(h, X, ldx, nrhs, st);
        default: return sweep_t<T, BWD_T>(h, X, ldx, nrhs, st);
    }
}

slu_status init_solve_attrs(const slu_handle *h) {
    const bool ok = h->prec == SLU_PREC_FP64 ? solve_attrs_t<double>()
                                             : solve_attrs_t<float>();
    return ok ? SLU_OK : SLU_ERR_CUDA;
}

static slu_status solve_inplace(const slu_handle *h, double *X, int64_t ldx,
                                int nrhs, bool transpose, cudaStream_t st) {
    slu_status s;
    if (h->prec == SLU_PREC_FP64) {
        s = sweep<double>(h, transpose ? FWD_T : FWD, X, ldx, nrhs, st);
        if (s == SLU_OK) s = sweep<double>(h, transpose ? BWD_T : BWD, X, ldx, nrhs, st);
    } else {
        s = sweep<float>(h, transpose ? FWD_T : FWD, X, ldx, nrhs, st);
        if (s == SLU_OK) s = sweep<float>(h, transpose ? BWD_T : BWD, X, ldx, nrhs, st);
    }
    return s;
}

static slu_status copy_cols(double *dst, int64_t ldd, const double *src,
                            int64_t lds, int64_t n, int nrhs, cudaStream_t st);

// The sweeps of one solve as a replayed CUDA graph: X is copied into the
// handle's buffer, the graph recorded for (nrhs, transposed) runs on `st`,
// and the result is copied back.  Profiling (per-launch events) and an
// enclosing capture take the direct path.
static slu_status solve_graphed(slu_handle *h, double *X, int64_t ldx, int nrhs,
                                bool tr, cudaStream_t st) {
    if (h->profiling || h->capturing) return solve_inplace(h, X, ldx, nrhs, tr, st);
    const int64_t n = h->plan->n;
    if (nrhs > h->xbuf_cols) {
        for (auto &g : h->sgraphs) cudaGraphExecDestroy(g.exec);
        h->sgraphs.clear();
        if (h->xbuf) cudaFree(h->xbuf);
        h->xbuf = nullptr;
        h->xbuf_cols = 0;
        if (!cuda_ok(cudaMalloc(&h->xbuf, (size_t)n * nrhs * sizeof(double)),
                     "cudaMalloc(solve buffer)"))
            return SLU_ERR_OUT_OF_MEMORY;
        h->xbuf_cols = nrhs;
    }
    const slu_handle::SolveGraph *g = nullptr;
    for (const auto &e : h->sgraphs)
        if (e.nrhs == nrhs && e.tr == tr) g = &e;
    if (!g) {
        if (!h->cap && !cuda_ok(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking),
                                "cudaStreamCreate"))
            return SLU_ERR_CUDA;
        if (!cuda_ok(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal),
                     "cudaStreamBeginCapture"))
            return SLU_ERR_CUDA;
        const int64_t l0 = h->launches;
        h->capturing = true;
        slu_status s = solve_inplace(h, h->xbuf, n, nrhs, tr, h->cap);
        h->capturing = false;
        const int64_t nl = h->launches - l0;
        h->launches = l0;
        cudaGraph_t graph = nullptr;
        const bool ended = cuda_ok(cudaStreamEndCapture(h->cap, &graph), "cudaStreamEndCapture");
        if (s != SLU_OK || !ended) {
            if (graph) cudaGraphDestroy(graph);
            return s != SLU_OK ? s : SLU_ERR_CUDA;
        }
        cudaGraphExec_t exec = nullptr;
        const bool ok = cuda_ok(cudaGraphInstantiate(&exec, graph, 0), "cudaGraphInstantiate");
        cudaGraphDestroy(graph);
        if (!ok) return SLU_ERR_CUDA;
        h->sgraphs.push_back({nrhs, tr, exec, nl});
        g = &h->sgraphs.back();
    }
    slu_status s = copy_cols(h->xbuf, n, X, ldx, n, nrhs, st);
    if (s != SLU_OK) return s;
    if (!cuda_ok(cudaGraphLaunch(g->exec, st), "cudaGraphLaunch")) return SLU_ERR_CUDA;
    h->launches += g->launches;
    return copy_cols(X, ldx, h->xbuf, n, n, nrhs, st);
}

static slu_status ensure_work(slu_handle *h, int64_t elems) {
    if (h->work_elems < elems) {
        if (h->work) cudaFree(h->work);
        h->work = nullptr;
        h->work_elems = 0;
        if (!cuda_ok(cudaMalloc(&h->work, elems * sizeof(double)), "cudaMalloc(work)"))
            return SLU_ERR_OUT_OF_MEMORY;
        h->work_elems = elems;
    }
    const size_t nseg = h->anorm_seg ? h->plan->seg.size() - 1 : 1;
    if (!h->red &&
        !cuda_ok(cudaMalloc(&h->red, 3 * 64 * nseg * sizeof(double)), "cudaMalloc(red)"))
        return SLU_ERR_OUT_OF_MEMORY;
    return SLU_OK;
}

static slu_status copy_cols(double *dst, int64_t ldd, const double *src,
                            int64_t lds, int64_t n, int nrhs, cudaStream_t st) {
    if (dst == src && ldd == lds) return SLU_OK;
    return cuda_ok(cudaMemcpy2DAsync(dst, ldd * sizeof(double), src,
                                     lds * sizeof(double), n * sizeof(double),
                                     nrhs, cudaMemcpyDeviceToDevice, st),
                   "cudaMemcpy2DAsync")
               ? SLU_OK
               : SLU_ERR_CUDA;
}

// Residual R = B - A X and the normwise backward error (max over columns,
// and over the members of a batch plan).
static slu_status backward_error(slu_handle *h, const double *B, int64_t ldb,
                                 const double *X, int64_t ldx, int nrhs,
                                 double *R, cudaStream_t st, double *be) {
    const slu_plan *P = h->plan;
    const DevPlan *D = P->dev;
    const int64_t n = P->n;
    const int nseg = h->anorm_seg ? (int)P->seg.size() - 1 : 1;
    {
        LaunchScope ls_(h, SLU_KC_RESID, st);
        k_residual<<<(int)((n * 32 + 255) / 256), 256, 0, st>>>(
            n, nrhs, D->a_rowptr, D->a_colidx, D->a_vpos, h->a_vals, B, ldb, X,
            ldx, R, n);
    }
    if (!cuda_ok(cudaMemsetAsync(h->red, 0, 3 * (size_t)nseg * nrhs * sizeof(double), st),
                 "cudaMemsetAsync"))
        return SLU_ERR_CUDA;
    {
        LaunchScope ls_(h, SLU_KC_RESID, st);
        if (nseg > 1)
            k_norms_seg<<<(int)((n + 255) / 256), 256, 0, st>>>(
                n, nrhs, R, n, X, ldx, B, ldb, D->row_seg,
                reinterpret_cast<unsigned long long *>(h->red));
        else
            k_norms<<<148 * 2, 256, 0, st>>>(
                n, nrhs, R, n, X, ldx, B, ldb,
                reinterpret_cast<unsigned long long *>(h->red));
    }
    std::vector<double> hr(3 * (size_t)nseg * nrhs), an(nseg);
    unsigned long long flags = 0;
    if (!cuda_ok(cudaMemcpyAsync(&flags, h->cnt + 2, sizeof(flags), cudaMemcpyDeviceToHost, st),
                 "cudaMemcpyAsync") ||
        !cuda_ok(cudaMemcpyAsync(hr.data(), h->red, hr.size() * sizeof(double),
                                 cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync") ||
        !cuda_ok(cudaMemcpyAsync(an.data(), nseg > 1 ? h->anorm_seg : h->scal + 1,
                                 nseg * sizeof(double), cudaMemcpyDeviceToHost, st),
                 "cudaMemcpyAsync") ||
        !cuda_ok(cudaStreamSynchronize(st), "residual"))
        return SLU_ERR_CUDA;
    if (flags & 4)
        return fail(SLU_ERR_TIMEOUT, "a wait of the persistent solve exceeded its bound");
    double worst = 0.0;
    for (int q = 0; q < nseg; ++q)
        for (int c = 0; c < nrhs; ++c) {
            const double *r = &hr[((size_t)q * nrhs + c) * 3];
            const double den = an[q] * r[1] + r[2];
            const double v = den > 0 ? r[0] / den : 0.0;
            if (!(v <= worst)) worst = v;     // a NaN term makes the result NaN
        }
    *be = worst;
    return SLU_OK;
}

}  // namespace slu

using namespace slu;

extern "C" slu_status slu_set_persistent_solve(slu_handle *h, int32_t on) {
    if (!h) return fail(SLU_ERR_INVALID_ARG, "NULL handle");
    const slu_plan *P = h->plan;
    if (on)
        for (int32_t I = 0; I < P->p; ++I)
            if (P->woff[I] < 0)
                return fail(SLU_ERR_NOT_SUPPORTED,
                            "the persistent solve needs the explicit inverses of every "
                            "diagonal block (dense, at most 384 rows)");
    if (h->persistent_solve != (on != 0)) {       // recorded graphs hold the other form
        int cur = -1;
        cudaGetDevice(&cur);
        if (h->device >= 0) cudaSetDevice(h->device);
        for (auto &g : h->sgraphs) cudaGraphExecDestroy(g.exec);
        h->sgraphs.clear();
        if (cur >= 0) cudaSetDevice(cur);
    }
    if (on && P->n > 0) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (h->device >= 0) cudaSetDevice(h->device);
        const slu_status s = h->prec == SLU_PREC_FP64 ? persistent_solve_setup_all<double>(h)
                                                      : persistent_solve_setup_all<float>(h);
        if (cur >= 0) cudaSetDevice(cur);
        if (s != SLU_OK) return s;
    }
    h->persistent_solve = on != 0;
    return SLU_OK;
}

extern "C" slu_status slu_solve(const slu_handle *ch, const double *B,
                                int64_t ldb, int32_t nrhs, double *X,
                                int64_t ldx, void *stream, slu_solve_info *info) {
    slu_handle *h = const_cast<slu_handle *>(ch);
    if (!h || !B || !X) return fail(SLU_ERR_INVALID_ARG, "NULL argument");
    const slu_plan *P = h->plan;
    const int64_t n = P->n;
    if (nrhs < 0 || nrhs > 64 || ldb < n || ldx < n)
        return fail(SLU_ERR_INVALID_ARG, "bad nrhs or leading dimension");
    if (info) {
        info->iterations = 0;
        info->backward_error = -1.0;
    }
    if (nrhs == 0 || n == 0) return SLU_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int maxit = P->opts.refine_max_iter < 0  ? 0
                      : P->opts.refine_max_iter > 0 ? P->opts.refine_max_iter
                      : (h->prec == SLU_PREC_FP64 ? 0 : 30);
    slu_status s;
    if (maxit == 0 && !info) {
        s = copy_cols(X, ldx, B, ldb, n, nrhs, st);
        if (s == SLU_OK) s = solve_graphed(h, X, ldx, nrhs, false, st);
        return s;
    }
    // B must survive for the residual: keep a copy when X aliases it.
    const bool alias = (X == B);
    s = ensure_work(h, (int64_t)n * nrhs * (alias ? 2 : 1));
    if (s != SLU_OK) return s;
    double *R = h->work;
    const double *Bk = B;
    int64_t ldbk = ldb;
    if (alias) {
        double *Bc = h->work + (int64_t)n * nrhs;
        s = copy_cols(Bc, n, B, ldb, n, nrhs, st);
        if (s != SLU_OK) return s;
        Bk = Bc;
        ldbk = n;
    }
    s = copy_cols(X, ldx, Bk, ldbk, n, nrhs, st);
    if (s == SLU_OK) s = solve_graphed(h, X, ldx, nrhs, false, st);
    if (s != SLU_OK) return s;
    double be = 0.0;
    int it = 0;
    for (;;) {
        s = backward_error(h, Bk, ldbk, X, ldx, nrhs, R, st, &be);
        if (s != SLU_OK) return s;
        if (be <= P->opts.refine_tol || it >= maxit) break;
        s = solve_graphed(h, R, n, nrhs, false, st);
        if (s != SLU_OK) return s;
        {
            LaunchScope ls_(h, SLU_KC_RESID, st);
            k_add_cols<<<148 * 4, 256, 0, st>>>(n, nrhs, R, n, X, ldx);
        }
        ++it;
    }
    if (info) {
        info->iterations = it;
        info->backward_error = be;
    }
    if (maxit > 0 && !(be <= P->opts.refine_tol))
        return fail(SLU_ERR_NOT_CONVERGED, "refinement did not reach refine_tol");
    return SLU_OK;
}

extern "C" slu_status slu_grad_values(const slu_handle *h, const double *Lam,
                                      int64_t ldl, const double *X,
                                      int64_t ldx, int32_t nrhs, double *grad,
                                      void *stream) {
    if (!h || !Lam || !X || !grad) return fail(SLU_ERR_INVALID_ARG, "NULL argument");
    const slu_plan *P = h->plan;
    if (nrhs < 1 || ldl < P->n || ldx < P->n)
        return fail(SLU_ERR_INVALID_ARG, "bad nrhs or leading dimension");
    if (P->nnz_a == 0) return SLU_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    {
        LaunchScope ls_(h, SLU_KC_RESID, st);
        const int64_t g = std::min<int64_t>((P->nnz_a + 255) / 256, 148 * 32);
        k_grad_values<<<(int)g, 256, 0, st>>>(P->nnz_a, P->dev->a_ri,
                                              P->dev->a_ci, nrhs, Lam, ldl, X,
                                              ldx, grad);
    }
    return cuda_ok(cudaGetLastError(), "grad launch") ? SLU_OK : SLU_ERR_CUDA;
}

extern "C" slu_status slu_solve_transpose(const slu_handle *h, const double *G,
                                          int64_t ldg, int32_t nrhs, double *Lam,
                                          int64_t ldl, void *stream) {
    if (!h || !G || !Lam) return fail(SLU_ERR_INVALID_ARG, "NULL argument");
    const int64_t n = h->plan->n;
    if (nrhs < 0 || ldg < n || ldl < n)
        return fail(SLU_ERR_INVALID_ARG, "bad nrhs or leading dimension");
    if (nrhs == 0 || n == 0) return SLU_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    slu_status s = copy_cols(Lam, ldl, G, ldg, n, nrhs, st);
    if (s == SLU_OK) s = solve_graphed(const_cast<slu_handle *>(h), Lam, ldl, nrhs, true, st);
    return s;
}

// Reordered systems: Y(k) = scale[perm[k]] X(perm[k]) (gather) or
// Y(perm[k]) = scale[perm[k]] X(k) (scatter), column by column.
__global__ void k_permute_scale(int64_t n, int nrhs, const int32_t *__restrict__ perm,
                                const double *__restrict__ scale,
                                const double *__restrict__ X, int64_t ldx,
                                double *__restrict__ Y, int64_t ldy, int inverse) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * nrhs;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t % n, c = t / n;
        const int64_t p = perm[k];
        const double s = scale ? scale[p] : 1.0;
        if (inverse) Y[p + c * ldy] = s * X[k + c * ldx];
        else         Y[k + c * ldy] = s * X[p + c * ldx];
    }
}

extern "C" slu_status slu_permute_scale(int64_t n, int32_t nrhs, const int32_t *perm,
                                        const double *scale, const double *X, int64_t ldx,
                                        double *Y, int64_t ldy, int32_t inverse,
                                        void *stream) {
    if (n < 0 || nrhs < 0 || ldx < n || ldy < n || (n > 0 && nrhs > 0 && (!perm || !X || !Y)))
        return fail(SLU_ERR_INVALID_ARG, "bad arguments");
    if (n == 0 || nrhs == 0) return SLU_OK;
    const int64_t tot = n * nrhs;
    const int grid = (int)std::min<int64_t>((tot + 255) / 256, 148 * 16);
    k_permute_scale<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        n, nrhs, perm, scale, X, ldx, Y, ldy, inverse);
    return cuda_ok(cudaGetLastError(), "permute launch") ? SLU_OK : SLU_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Allocation-free refined solve.
//
// slu_solve's refinement path keeps its residual and reduction words in a
// workspace that the handle allocates with cudaMalloc on first use.  Some
// callers may not allocate device memory at that point: a process whose
// device memory budget is fixed and fully handed out at start-up, an
// application whose framework owns every byte of device memory through its
// own pool, or a latency-critical loop in which cudaMalloc's implicit device
// synchronization is not acceptable.  For them this entry point runs the same
// refinement with its scratch in a fixed array that lives in the library's
// device image instead.
//
// The array holds SLU_NOALLOC_MAX_ELEMS residual values plus the reduction
// words; every GPU that loads the library reserves it (8 MiB) until the
// process exits.  All calls on one device share it and it keeps whatever the
// previous call left there; the reduction words are cleared on every use and
// the residual is fully rewritten before it is read.  Two calls whose work
// overlaps on the GPU (different streams, or host threads) race on the
// array, so callers must order them.
constexpr int kNoallocRed = 256;
static __device__ __align__(256) double g_noalloc_scratch[SLU_NOALLOC_MAX_ELEMS + kNoallocRed];

// Scratch layout of one call: the residual R (n x nrhs) at the front, then,
// from the next 32-double boundary, 3 reduction words per right-hand side and
// matrix (one matrix, or every member of a batch plan), then the one word
// that receives the backward error.
__host__ __device__ constexpr int64_t noalloc_red_at(int64_t n, int nrhs) {
    return ((n * nrhs + 31) / 32) * 32;
}
__host__ __device__ constexpr int64_t noalloc_words(int64_t n, int nrhs, int nseg) {
    return noalloc_red_at(n, nrhs) + 3 * (int64_t)nseg * nrhs + 1;
}

// *out = max over members q and columns c of
//   red[3(q nrhs + c)] / (anorm[q] red[3(q nrhs + c) + 1] + red[3(q nrhs + c) + 2]),
// a term with a zero denominator counting as 0 and a NaN term making the
// result NaN (the same reduction as slu_solve's, done on the device so that
// nothing is staged in host memory).  One CTA.
__global__ void k_be_max(int nseg, int nrhs, const double *__restrict__ red,
                         const double *__restrict__ anorm, double *__restrict__ out) {
    __shared__ double sw[32];
    double w = 0.0;
    for (int t = threadIdx.x; t < nseg * nrhs; t += blockDim.x) {
        const double *r = red + 3 * (int64_t)t;
        const double den = anorm[t / nrhs] * r[1] + r[2];
        const double v = den > 0 ? r[0] / den : 0.0;
        if (!(v <= w)) w = v;                 // NaN wins
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double v = __shfl_xor_sync(~0u, w, o);
        if (!(v <= w)) w = v;
    }
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k)
            if (!(sw[k] <= w)) w = sw[k];
        *out = w;
    }
}

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the handle's device, which must be
// the current one (the caller's stream belongs to it).  The name
// g_noalloc_scratch in host code is only a host-side stand-in; its device
// address comes from cudaGetSymbolAddress, taken once per device with that
// device current.
slu_status noalloc_scratch(const slu_handle *h, double **out) {
    int dev = -1;
    if (!cuda_ok(cudaGetDevice(&dev), "cudaGetDevice")) return SLU_ERR_CUDA;
    if (dev != h->device)
        return fail(SLU_ERR_INVALID_ARG,
                    "the current device is not the handle's device");
    if (dev < 0 || dev >= kMaxDevices)
        return fail(SLU_ERR_NOT_SUPPORTED, "device index beyond 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (!cuda_ok(cudaGetSymbolAddress(&p, g_noalloc_scratch),
                     "cudaGetSymbolAddress(noalloc scratch)"))
            return SLU_ERR_CUDA;
        g_noalloc_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return SLU_OK;
}

// backward_error with the reduction words and the result in the scratch
// array (red, then *dbe) instead of the handle's workspace: per member of a
// batch plan (k_norms_seg and the members' norms of A) as slu_solve does.
slu_status backward_error_with(slu_handle *h, const double *B, int64_t ldb,
                               const double *X, int64_t ldx, int nrhs,
                               double *R, double *red, double *dbe,
                               cudaStream_t st, double *be) {
    const slu_plan *P = h->plan;
    const DevPlan *D = P->dev;
    const int64_t n = P->n;
    const int nseg = h->anorm_seg ? (int)P->seg.size() - 1 : 1;
    {
        LaunchScope ls_(h, SLU_KC_RESID, st);
        k_residual<<<(int)((n * 32 + 255) / 256), 256, 0, st>>>(
            n, nrhs, D->a_rowptr, D->a_colidx, D->a_vpos, h->a_vals, B, ldb, X,
            ldx, R, n);
    }
    if (!cuda_ok(cudaMemsetAsync(red, 0, 3 * (size_t)nseg * nrhs * sizeof(double), st),
                 "cudaMemsetAsync"))
        return SLU_ERR_CUDA;
    {
        LaunchScope ls_(h, SLU_KC_RESID, st);
        if (nseg > 1)
            k_norms_seg<<<(int)((n + 255) / 256), 256, 0, st>>>(
                n, nrhs, R, n, X, ldx, B, ldb, D->row_seg,
                reinterpret_cast<unsigned long long *>(red));
        else
            k_norms<<<148 * 2, 256, 0, st>>>(
                n, nrhs, R, n, X, ldx, B, ldb,
                reinterpret_cast<unsigned long long *>(red));
    }
    {
        LaunchScope ls_(h, SLU_KC_RESID, st);
        k_be_max<<<1, 256, 0, st>>>(nseg, nrhs, red,
                                    nseg > 1 ? h->anorm_seg : h->scal + 1, dbe);
    }
    if (!cuda_ok(cudaMemcpyAsync(be, dbe, sizeof(double), cudaMemcpyDeviceToHost, st),
                 "cudaMemcpyAsync") ||
        !cuda_ok(cudaStreamSynchronize(st), "residual"))
        return SLU_ERR_CUDA;
    return SLU_OK;
}

}  // namespace

extern "C" slu_status slu_solve_refine_noalloc(const slu_handle *ch,
                                               const double *B, int64_t ldb,
                                               int32_t nrhs, double *X,
                                               int64_t ldx, void *stream,
                                               slu_solve_info *info) {
    slu_handle *h = const_cast<slu_handle *>(ch);
    if (!h || !B || !X) return fail(SLU_ERR_INVALID_ARG, "NULL argument");
    const slu_plan *P = h->plan;
    const int64_t n = P->n;
    if (nrhs < 0 || nrhs > 64 || ldb < n || ldx < n)
        return fail(SLU_ERR_INVALID_ARG, "bad nrhs or leading dimension");
    if (X == B) return fail(SLU_ERR_INVALID_ARG, "X must not alias B");
    const int nseg = h->anorm_seg ? (int)P->seg.size() - 1 : 1;
    if (n * (int64_t)nrhs > SLU_NOALLOC_MAX_ELEMS ||
        noalloc_words(n, nrhs, nseg) > SLU_NOALLOC_MAX_ELEMS + kNoallocRed)
        return fail(SLU_ERR_INVALID_ARG,
                    "n * nrhs (plus 3 * nrhs reduction words per batch member) "
                    "exceeds SLU_NOALLOC_MAX_ELEMS (1048576) + 256: use "
                    "slu_solve, which allocates its workspace");
    if (info) {
        info->iterations = 0;
        info->backward_error = -1.0;
    }
    if (nrhs == 0 || n == 0) return SLU_OK;
    double *scratch = nullptr;
    slu_status s = noalloc_scratch(h, &scratch);
    if (s != SLU_OK) return s;
    double *R = scratch;
    double *red = scratch + noalloc_red_at(n, nrhs);
    double *dbe = red + 3 * (int64_t)nseg * nrhs;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int maxit = P->opts.refine_max_iter < 0  ? 0
                      : P->opts.refine_max_iter > 0 ? P->opts.refine_max_iter
                      : (h->prec == SLU_PREC_FP64 ? 0 : 30);
    s = copy_cols(X, ldx, B, ldb, n, nrhs, st);
    if (s == SLU_OK) s = solve_inplace(h, X, ldx, nrhs, false, st);
    if (s != SLU_OK) return s;
    double be = 0.0;
    int it = 0;
    for (;;) {
        s = backward_error_with(h, B, ldb, X, ldx, nrhs, R, red, dbe, st, &be);
        if (s != SLU_OK) return s;
        if (be <= P->opts.refine_tol || it >= maxit) break;
        s = solve_inplace(h, R, n, nrhs, false, st);
        if (s != SLU_OK) return s;
        {
            LaunchScope ls_(h, SLU_KC_RESID, st);
            k_add_cols<<<148 * 4, 256, 0, st>>>(n, nrhs, R, n, X, ldx);
        }
        ++it;
    }
    if (info) {
        info->iterations = it;
        info->backward_error = be;
    }
    if (maxit > 0 && !(be <= P->opts.refine_tol))
        return fail(SLU_ERR_NOT_CONVERGED, "refinement did not reach refine_tol");
    return SLU_OK;
}
