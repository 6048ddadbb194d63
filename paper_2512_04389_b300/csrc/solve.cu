// Triangular solves with the block factors, FP64 residual and iterative
// refinement.  The paper covers only the factorization; solving with the
// factors, refining an FP32 factorization and the transposed solve used for
// differentiation complete the linear solver around it.
//
// Every solve walks the levels of the block dependency DAG (the same levels
// as the factorization): a level's diagonal blocks have no block coupling
// among themselves, so one CTA per diagonal block of the level
//   1. pulls the contributions of already solved blocks into its rows
//      (per-warp partial sums reduced in a fixed order: deterministic), then
//   2. solves with its diagonal block.
// Arithmetic is FP64 whatever the storage type of the factors.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "device_common.cuh"

namespace slu {

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(~0u, v, o);
    return v;
}

// Adds sum over the listed blocks of B(:, jj) * x(c0 + jj) into part (one
// partial vector per warp; warps split the columns of each block).
template <typename T>
__device__ __forceinline__ void pull_scatter(const BlockArgs &a,
                                             const T *__restrict__ val,
                                             const int32_t *__restrict__ blk,
                                             int64_t b0, int64_t b1,
                                             const double *__restrict__ x,
                                             double *pw) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t bi = b0; bi < b1; ++bi) {
        const BlockDesc db = a.bd[blk[bi]];
        for (int jj = warp; jj < db.cols; jj += kWarps) {
            const double xv = x[db.c0 + jj];
            if (xv != 0.0) {
                int64_t vb;
                int cn;
                const uint16_t *rows;
                colview(db, jj, a, vb, cn, rows);
                for (int e = lane; e < cn; e += 32)
                    pw[rowat(rows, e)] += (double)val[vb + e] * xv;
            }
            __syncwarp();
        }
    }
}

// L y = b on the rows of one level's diagonal blocks (levels ascending):
// pull from blocks (I, I'), I' < I, then unit lower L_II.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_fwd(const int32_t *__restrict__ ids, BlockArgs a, const T *__restrict__ val,
      const int64_t *__restrict__ boff, const int32_t *__restrict__ blk,
      double *__restrict__ X, int64_t ldx, int nrhs) {
    extern __shared__ __align__(16) unsigned char smem[];
    const BlockDesc dd = a.bd[ids[blockIdx.x]];
    const int m = dd.rows, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double *y = reinterpret_cast<double *>(smem);
    double *part = y + m;
    const int64_t b0 = boff[dd.I], b1 = boff[dd.I + 1];
    for (int c = 0; c < nrhs; ++c) {
        double *x = X + (int64_t)c * ldx;
        for (int t = threadIdx.x; t < m; t += kThreads) y[t] = x[dd.r0 + t];
        for (int t = threadIdx.x; t < kWarps * m; t += kThreads) part[t] = 0.0;
        __syncthreads();
        pull_scatter(a, val, blk, b0, b1, x, part + warp * m);
        __syncthreads();
        for (int t = threadIdx.x; t < m; t += kThreads) {
            double s = 0.0;
            for (int w = 0; w < kWarps; ++w) s += part[w * m + t];
            y[t] -= s;
        }
        __syncthreads();
        if (warp == 0) {
            for (int jj = 0; jj < m; ++jj) {
                const double xv = y[jj];
                if (xv != 0.0) {
                    int64_t vb;
                    int cn;
                    const uint16_t *rows;
                    colview(dd, jj, a, vb, cn, rows);
                    const int dp = a.dpos[dd.doff + jj];
                    for (int e = dp + 1 + lane; e < cn; e += 32)
                        y[rowat(rows, e)] -= (double)val[vb + e] * xv;
                }
                __syncwarp();
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < m; t += kThreads) x[dd.r0 + t] = y[t];
        __syncthreads();
    }
}

// U x = y (levels descending): pull from blocks (I, J), J > I, then U_II.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_bwd(const int32_t *__restrict__ ids, BlockArgs a, const T *__restrict__ val,
      const int64_t *__restrict__ boff, const int32_t *__restrict__ blk,
      double *__restrict__ X, int64_t ldx, int nrhs) {
    extern __shared__ __align__(16) unsigned char smem[];
    const BlockDesc dd = a.bd[ids[blockIdx.x]];
    const int m = dd.rows, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double *y = reinterpret_cast<double *>(smem);
    double *part = y + m;
    const int64_t b0 = boff[dd.I], b1 = boff[dd.I + 1];
    for (int c = 0; c < nrhs; ++c) {
        double *x = X + (int64_t)c * ldx;
        for (int t = threadIdx.x; t < m; t += kThreads) y[t] = x[dd.r0 + t];
        for (int t = threadIdx.x; t < kWarps * m; t += kThreads) part[t] = 0.0;
        __syncthreads();
        pull_scatter(a, val, blk, b0, b1, x, part + warp * m);
        __syncthreads();
        for (int t = threadIdx.x; t < m; t += kThreads) {
            double s = 0.0;
            for (int w = 0; w < kWarps; ++w) s += part[w * m + t];
            y[t] -= s;
        }
        __syncthreads();
        if (warp == 0) {
            for (int jj = m - 1; jj >= 0; --jj) {
                int64_t vb;
                int cn;
                const uint16_t *rows;
                colview(dd, jj, a, vb, cn, rows);
                const int dp = a.dpos[dd.doff + jj];
                const double xv = y[jj] / (double)val[vb + dp];
                __syncwarp();
                if (lane == 0) y[jj] = xv;
                if (xv != 0.0)
                    for (int e = lane; e < dp; e += 32)
                        y[rowat(rows, e)] -= (double)val[vb + e] * xv;
                __syncwarp();
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < m; t += kThreads) x[dd.r0 + t] = y[t];
        __syncthreads();
    }
}

// Dot of column ii of each listed block with x on the block's rows; one warp
// owns column ii across all blocks, so no partial sums are needed.
template <typename T>
__device__ __forceinline__ double pull_dot(const BlockArgs &a,
                                           const T *__restrict__ val,
                                           const int32_t *__restrict__ blk,
                                           int64_t b0, int64_t b1, int ii,
                                           const double *__restrict__ x) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int64_t bi = b0; bi < b1; ++bi) {
        const BlockDesc db = a.bd[blk[bi]];
        int64_t vb;
        int cn;
        const uint16_t *rows;
        colview(db, ii, a, vb, cn, rows);
        for (int e = lane; e < cn; e += 32)
            s += (double)val[vb + e] * x[db.r0 + rowat(rows, e)];
    }
    return warp_sum(s);
}

// U^T z = g (levels ascending): z(ii) -= dot of column ii of blocks
// (I', I), I' < I, with z(I'); then a forward sweep with U_II^T.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_fwd_t(const int32_t *__restrict__ ids, BlockArgs a, const T *__restrict__ val,
        const int64_t *__restrict__ boff, const int32_t *__restrict__ blk,
        double *__restrict__ X, int64_t ldx, int nrhs) {
    extern __shared__ __align__(16) unsigned char smem[];
    const BlockDesc dd = a.bd[ids[blockIdx.x]];
    const int m = dd.rows, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double *z = reinterpret_cast<double *>(smem);
    const int64_t b0 = boff[dd.I], b1 = boff[dd.I + 1];
    for (int c = 0; c < nrhs; ++c) {
        double *x = X + (int64_t)c * ldx;
        for (int t = threadIdx.x; t < m; t += kThreads) z[t] = x[dd.r0 + t];
        __syncthreads();
        for (int ii = warp; ii < m; ii += kWarps) {
            const double s = pull_dot(a, val, blk, b0, b1, ii, x);
            if (lane == 0) z[ii] -= s;
        }
        __syncthreads();
        if (warp == 0) {
            for (int ii = 0; ii < m; ++ii) {
                int64_t vb;
                int cn;
                const uint16_t *rows;
                colview(dd, ii, a, vb, cn, rows);
                const int dp = a.dpos[dd.doff + ii];
                double s = 0.0;
                for (int e = lane; e < dp; e += 32)
                    s += (double)val[vb + e] * z[rowat(rows, e)];
                s = warp_sum(s);
                const double zi = (z[ii] - s) / (double)val[vb + dp];
                __syncwarp();
                if (lane == 0) z[ii] = zi;
                __syncwarp();
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < m; t += kThreads) x[dd.r0 + t] = z[t];
        __syncthreads();
    }
}

// L^T lam = z (levels descending): pull from blocks (K, I), K > I, then a
// backward sweep with L_II^T (unit diagonal).
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_bwd_t(const int32_t *__restrict__ ids, BlockArgs a, const T *__restrict__ val,
        const int64_t *__restrict__ boff, const int32_t *__restrict__ blk,
        double *__restrict__ X, int64_t ldx, int nrhs) {
    extern __shared__ __align__(16) unsigned char smem[];
    const BlockDesc dd = a.bd[ids[blockIdx.x]];
    const int m = dd.rows, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double *z = reinterpret_cast<double *>(smem);
    const int64_t b0 = boff[dd.I], b1 = boff[dd.I + 1];
    for (int c = 0; c < nrhs; ++c) {
        double *x = X + (int64_t)c * ldx;
        for (int t = threadIdx.x; t < m; t += kThreads) z[t] = x[dd.r0 + t];
        __syncthreads();
        for (int ii = warp; ii < m; ii += kWarps) {
            const double s = pull_dot(a, val, blk, b0, b1, ii, x);
            if (lane == 0) z[ii] -= s;
        }
        __syncthreads();
        if (warp == 0) {
            for (int ii = m - 1; ii >= 0; --ii) {
                int64_t vb;
                int cn;
                const uint16_t *rows;
                colview(dd, ii, a, vb, cn, rows);
                const int dp = a.dpos[dd.doff + ii];
                double s = 0.0;
                for (int e = dp + 1 + lane; e < cn; e += 32)
                    s += (double)val[vb + e] * z[rowat(rows, e)];
                s = warp_sum(s);
                const double zi = z[ii] - s;
                __syncwarp();
                if (lane == 0) z[ii] = zi;
                __syncwarp();
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < m; t += kThreads) x[dd.r0 + t] = z[t];
        __syncthreads();
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

__global__ void k_add_cols(int64_t n, int nrhs, const double *__restrict__ D,
                           int64_t ldd, double *__restrict__ X, int64_t ldx) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
         i < n * nrhs; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i % n, c = i / n;
        X[r + c * ldx] += D[r + c * ldd];
    }
}

// ---------------------------------------------------------------- host side

enum Sweep { FWD, BWD, FWD_T, BWD_T };

template <typename T>
static slu_status sweep(const slu_handle *h, Sweep sw, double *X, int64_t ldx,
                        int nrhs, cudaStream_t st) {
    const slu_plan *P = h->plan;
    const DevPlan *D = P->dev;
    const T *val = static_cast<const T *>(h->storage);
    const BlockArgs a = block_args(P);
    const bool scatter = (sw == FWD || sw == BWD);
    const size_t smem =
        (size_t)P->maxb * sizeof(double) * (scatter ? 1 + kWarps : 1);
    auto *kern = sw == FWD ? k_fwd<T> : sw == BWD ? k_bwd<T>
               : sw == FWD_T ? k_fwd_t<T> : k_bwd_t<T>;
    const int64_t *off = sw == FWD ? D->lrow_off : sw == BWD ? D->urow_off
                       : sw == FWD_T ? D->ucol_off : D->lcol_off;
    const int32_t *blk = sw == FWD ? D->lrow_blk : sw == BWD ? D->urow_blk
                       : sw == FWD_T ? D->ucol_blk : D->lcol_blk;
    if (smem > 48 * 1024 &&
        !cuda_ok(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem), "cudaFuncSetAttribute"))
        return SLU_ERR_CUDA;
    const bool up = (sw == FWD || sw == FWD_T);
    for (int k = 0; k < P->nlevels; ++k) {
        const int lv = up ? k : P->nlevels - 1 - k;
        const int64_t g0 = P->getrf_off[lv], g1 = P->getrf_off[lv + 1];
        if (g1 > g0) {
            LaunchScope ls_(h, SLU_KC_SOLVE, st);
            kern<<<(int)(g1 - g0), kThreads, smem, st>>>(D->getrf + g0, a, val,
                                                       off, blk, X, ldx, nrhs);
        }
    }
    return cuda_ok(cudaGetLastError(), "solve launch") ? SLU_OK : SLU_ERR_CUDA;
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

static slu_status ensure_work(slu_handle *h, int64_t elems) {
    if (h->work_elems < elems) {
        if (h->work) cudaFree(h->work);
        h->work = nullptr;
        h->work_elems = 0;
        if (!cuda_ok(cudaMalloc(&h->work, elems * sizeof(double)), "cudaMalloc(work)"))
            return SLU_ERR_OUT_OF_MEMORY;
        h->work_elems = elems;
    }
    if (!h->red &&
        !cuda_ok(cudaMalloc(&h->red, 3 * 64 * sizeof(double)), "cudaMalloc(red)"))
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

// Residual R = B - A X and the normwise backward error (max over columns).
static slu_status backward_error(slu_handle *h, const double *B, int64_t ldb,
                                 const double *X, int64_t ldx, int nrhs,
                                 double *R, cudaStream_t st, double *be) {
    const slu_plan *P = h->plan;
    const DevPlan *D = P->dev;
    const int64_t n = P->n;
    {
        LaunchScope ls_(h, SLU_KC_RESID, st);
        k_residual<<<(int)((n * 32 + 255) / 256), 256, 0, st>>>(
        n, nrhs, D->a_rowptr, D->a_colidx, D->a_vpos, h->a_vals, B, ldb, X, ldx,
        R, n);
    }
    if (!cuda_ok(cudaMemsetAsync(h->red, 0, 3 * nrhs * sizeof(double), st),
                 "cudaMemsetAsync"))
        return SLU_ERR_CUDA;
    {
        LaunchScope ls_(h, SLU_KC_RESID, st);
        k_norms<<<148 * 2, 256, 0, st>>>(
            n, nrhs, R, n, X, ldx, B, ldb,
            reinterpret_cast<unsigned long long *>(h->red));
    }
    double hr[3 * 64 + 1];
    if (!cuda_ok(cudaMemcpyAsync(hr, h->red, 3 * nrhs * sizeof(double),
                                 cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync") ||
        !cuda_ok(cudaMemcpyAsync(hr + 3 * 64, h->scal + 1, sizeof(double),
                                 cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync") ||
        !cuda_ok(cudaStreamSynchronize(st), "residual"))
        return SLU_ERR_CUDA;
    const double anorm = hr[3 * 64];
    double worst = 0.0;
    for (int c = 0; c < nrhs; ++c) {
        const double den = anorm * hr[3 * c + 1] + hr[3 * c + 2];
        worst = std::max(worst, den > 0 ? hr[3 * c] / den : 0.0);
    }
    *be = worst;
    return SLU_OK;
}

}  // namespace slu

using namespace slu;

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
        if (s == SLU_OK) s = solve_inplace(h, X, ldx, nrhs, false, st);
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
    if (s == SLU_OK) s = solve_inplace(h, X, ldx, nrhs, false, st);
    if (s != SLU_OK) return s;
    double be = 0.0;
    int it = 0;
    for (;;) {
        s = backward_error(h, Bk, ldbk, X, ldx, nrhs, R, st, &be);
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
    if (s == SLU_OK) s = solve_inplace(h, Lam, ldl, nrhs, true, st);
    return s;
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
constexpr int kNoallocRed = 3 * 64;
static __device__ __align__(256) double g_noalloc_scratch[SLU_NOALLOC_MAX_ELEMS + kNoallocRed];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  The name
// g_noalloc_scratch in host code is only a host-side stand-in; its device
// address comes from cudaGetSymbolAddress, taken once per device with that
// device current.
slu_status noalloc_scratch(double **out) {
    int dev = -1;
    if (!cuda_ok(cudaGetDevice(&dev), "cudaGetDevice")) return SLU_ERR_CUDA;
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

// backward_error with caller-given reduction words instead of h->red.
slu_status backward_error_with(slu_handle *h, const double *B, int64_t ldb,
                               const double *X, int64_t ldx, int nrhs,
                               double *R, double *red, cudaStream_t st,
                               double *be) {
    const slu_plan *P = h->plan;
    const DevPlan *D = P->dev;
    const int64_t n = P->n;
    {
        LaunchScope ls_(h, SLU_KC_RESID, st);
        k_residual<<<(int)((n * 32 + 255) / 256), 256, 0, st>>>(
            n, nrhs, D->a_rowptr, D->a_colidx, D->a_vpos, h->a_vals, B, ldb, X,
            ldx, R, n);
    }
    if (!cuda_ok(cudaMemsetAsync(red, 0, 3 * nrhs * sizeof(double), st),
                 "cudaMemsetAsync"))
        return SLU_ERR_CUDA;
    {
        LaunchScope ls_(h, SLU_KC_RESID, st);
        k_norms<<<148 * 2, 256, 0, st>>>(
            n, nrhs, R, n, X, ldx, B, ldb,
            reinterpret_cast<unsigned long long *>(red));
    }
    double hr[3 * 64 + 1];
    if (!cuda_ok(cudaMemcpyAsync(hr, red, 3 * nrhs * sizeof(double),
                                 cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync") ||
        !cuda_ok(cudaMemcpyAsync(hr + 3 * 64, h->scal + 1, sizeof(double),
                                 cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync") ||
        !cuda_ok(cudaStreamSynchronize(st), "residual"))
        return SLU_ERR_CUDA;
    double worst = 0.0;
    for (int c = 0; c < nrhs; ++c) {
        const double den = hr[3 * 64] * hr[3 * c + 1] + hr[3 * c + 2];
        worst = std::max(worst, den > 0 ? hr[3 * c] / den : 0.0);
    }
    *be = worst;
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
    if (n * (int64_t)nrhs > SLU_NOALLOC_MAX_ELEMS)
        return fail(SLU_ERR_INVALID_ARG,
                    "n * nrhs exceeds SLU_NOALLOC_MAX_ELEMS (1048576): use "
                    "slu_solve, which allocates its workspace");
    if (info) {
        info->iterations = 0;
        info->backward_error = -1.0;
    }
    if (nrhs == 0 || n == 0) return SLU_OK;
    double *scratch = nullptr;
    slu_status s = noalloc_scratch(&scratch);
    if (s != SLU_OK) return s;
    double *R = scratch;
    double *red = scratch + SLU_NOALLOC_MAX_ELEMS;
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
        s = backward_error_with(h, B, ldb, X, ldx, nrhs, R, red, st, &be);
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
