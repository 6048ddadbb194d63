// Numerical factorization on the GPU: the right-looking blocked LU of
// Section 2.2 (Algorithm 1) over the plan's non-empty blocks, one level of
// the block dependency DAG at a time.
//
// Per level three launches:
//   GETRF  one CTA per diagonal block B_II -> L_II U_II (no row exchange;
//          pivots in FP64; |pivot| < tau replaced by +-tau and counted);
//   panel  one CTA per GESSM task  U_IJ = L_II^{-1} B_IJ
//          and per TSTRF task      L_JI = B_JI U_II^{-1};
//   SSSSM  one CTA per target block B_KJ, which gathers every source I of
//          the level, B_KJ -= sum_I L_KI U_IJ, sources in ascending I, so the
//          result is deterministic and needs no atomics.
//
// The kernels work column by column with one warp per column and a dense
// per-warp accumulator in shared memory; a dense block is read as a block
// whose every column holds all rows.  Closure of the pattern under fill
// guarantees that every update lands on a stored slot.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "device_common.cuh"

namespace slu {

// ---------------------------------------------------------------- kernels

// out = max |v| (as the bit pattern of a non-negative double, which orders
// like the value).
__global__ void k_maxabs(int64_t n, const double *__restrict__ v,
                         unsigned long long *__restrict__ out) {
    double m = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(v[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(~0u, m, o));
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

// GETRF on diagonal blocks.  Columns run in height groups of the block's
// own column DAG; inside a group one warp per column performs the
// left-looking update x = B(:,jj); for m in struct U(:,jj) ascending:
// x(rows of L(:,m)) -= L(:,m) x(m); then U(:,jj) = x(<= jj),
// L(:,jj) = x(> jj) / pivot.  Accumulation is FP64 for every storage type.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_getrf(const int32_t *__restrict__ ids, BlockArgs a, T *__restrict__ val,
        const double *__restrict__ scal, double tau_rel,
        unsigned long long *__restrict__ cnt) {
    const BlockDesc d = a.bd[ids[blockIdx.x]];
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double *acc = reinterpret_cast<double *>(smem) + warp * d.rows;
    for (int t = lane; t < d.rows; t += 32) acc[t] = 0.0;
    __syncwarp();
    const double tau = tau_rel * scal[0];
    for (int g = 0; g < d.ngroups; ++g) {
        const int gs = a.sgrp[d.goff + g], ge = a.sgrp[d.goff + g + 1];
        for (int q = gs + warp; q < ge; q += kWarps) {
            const int jj = a.sched[d.doff + q];
            int64_t vb;
            int cn;
            const uint16_t *rows;
            colview(d, jj, a, vb, cn, rows);
            for (int t = lane; t < cn; t += 32)
                acc[rowat(rows, t)] = (double)val[vb + t];
            __syncwarp();
            const int dp = a.dpos[d.doff + jj];
            for (int t = 0; t < dp; ++t) {
                const int m = rowat(rows, t);
                const double x = acc[m];
                if (x != 0.0) {
                    int64_t vm;
                    int cm;
                    const uint16_t *rm;
                    colview(d, m, a, vm, cm, rm);
                    const int dpm = a.dpos[d.doff + m];
                    for (int u = dpm + 1 + lane; u < cm; u += 32)
                        acc[rowat(rm, u)] -= (double)val[vm + u] * x;
                }
                __syncwarp();
            }
            double piv = acc[jj];
            if (tau > 0.0 && fabs(piv) < tau) {
                piv = (piv >= 0.0) ? tau : -tau;
                if (lane == 0) atomicAdd(&cnt[0], 1ull);
            } else if (piv == 0.0) {
                if (lane == 0) atomicOr(&cnt[1], 1ull);
            }
            for (int t = lane; t < cn; t += 32) {
                const int r = rowat(rows, t);
                double v = acc[r];
                if (r > jj) v = v / piv;
                else if (r == jj) v = piv;
                val[vb + t] = (T)v;
                acc[r] = 0.0;
            }
            __syncwarp();
        }
        __syncthreads();
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
    Acc *acc = reinterpret_cast<Acc *>(smem) + warp * d.rows;
    for (int t = lane; t < d.rows; t += 32) acc[t] = Acc(0);
    __syncwarp();
    if (is_gessm) {
        // U_IJ(:,jj) = L_II^{-1} B_IJ(:,jj); columns independent.
        for (int jj = warp; jj < d.cols; jj += kWarps) {
            int64_t vb;
            int cn;
            const uint16_t *rows;
            colview(d, jj, a, vb, cn, rows);
            for (int t = lane; t < cn; t += 32)
                acc[rowat(rows, t)] = (Acc)val[vb + t];
            __syncwarp();
            for (int t = 0; t < cn; ++t) {
                const int m = rowat(rows, t);
                const Acc x = acc[m];
                if (x != Acc(0)) {
                    int64_t vm;
                    int cm;
                    const uint16_t *rm;
                    colview(dd, m, a, vm, cm, rm);
                    const int dpm = a.dpos[dd.doff + m];
                    for (int u = dpm + 1 + lane; u < cm; u += 32)
                        acc[rowat(rm, u)] -= (Acc)val[vm + u] * x;
                }
                __syncwarp();
            }
            for (int t = lane; t < cn; t += 32) {
                const int r = rowat(rows, t);
                val[vb + t] = (T)acc[r];
                acc[r] = Acc(0);
            }
            __syncwarp();
        }
    } else {
        // L_JI(:,ii) = (B_JI(:,ii) - sum_{m<ii} L_JI(:,m) U_II(m,ii)) / U_II(ii,ii),
        // columns in the height groups of the diagonal block.
        for (int g = 0; g < dd.ngroups; ++g) {
            const int gs = a.sgrp[dd.goff + g], ge = a.sgrp[dd.goff + g + 1];
            for (int q = gs + warp; q < ge; q += kWarps) {
                const int ii = a.sched[dd.doff + q];
                int64_t vb;
                int cn;
                const uint16_t *rows;
                colview(d, ii, a, vb, cn, rows);
                for (int t = lane; t < cn; t += 32)
                    acc[rowat(rows, t)] = (Acc)val[vb + t];
                __syncwarp();
                int64_t vu;
                int cu;
                const uint16_t *ru;
                colview(dd, ii, a, vu, cu, ru);
                const int dp = a.dpos[dd.doff + ii];
                for (int t = 0; t < dp; ++t) {
                    const Acc u = (Acc)val[vu + t];
                    if (u != Acc(0)) {
                        const int m = rowat(ru, t);
                        int64_t vm;
                        int cm;
                        const uint16_t *rm;
                        colview(d, m, a, vm, cm, rm);
                        for (int e = lane; e < cm; e += 32)
                            acc[rowat(rm, e)] -= (Acc)val[vm + e] * u;
                    }
                    __syncwarp();
                }
                const Acc piv = (Acc)val[vu + dp];
                for (int t = lane; t < cn; t += 32) {
                    const int r = rowat(rows, t);
                    val[vb + t] = (T)(acc[r] / piv);
                    acc[r] = Acc(0);
                }
                __syncwarp();
            }
            __syncthreads();
        }
    }
}

// SSSSM: target B_KJ -= sum over the level's sources I of L_KI U_IJ.
// One warp per target column jj: for each source, for each stored U_IJ(i,jj)
// (fetched 32 at a time and broadcast by shuffles),
// acc += L_KI(:,i) U_IJ(i,jj); then B_KJ(:,jj) -= acc at the stored rows.
template <typename T, typename Acc>
__global__ void __launch_bounds__(kThreads)
k_ssssm(const int32_t *__restrict__ tgt, const int64_t *__restrict__ srcoff,
        const int32_t *__restrict__ src, BlockArgs a, T *__restrict__ val) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const BlockDesc d = a.bd[tgt[blockIdx.x]];
    const int64_t s0 = srcoff[blockIdx.x], s1 = srcoff[blockIdx.x + 1];
    Acc *acc = reinterpret_cast<Acc *>(smem) + warp * d.rows;
    for (int t = lane; t < d.rows; t += 32) acc[t] = Acc(0);
    __syncwarp();
    for (int jj = warp; jj < d.cols; jj += kWarps) {
        for (int64_t s = s0; s < s1; ++s) {
            const BlockDesc dl = a.bd[src[2 * s]];
            const BlockDesc du = a.bd[src[2 * s + 1]];
            int64_t vu;
            int cu;
            const uint16_t *ru;
            colview(du, jj, a, vu, cu, ru);
            for (int c0 = 0; c0 < cu; c0 += 32) {
                const int t = c0 + lane;
                int il = 0;
                Acc ul = Acc(0);
                if (t < cu) {
                    il = rowat(ru, t);
                    ul = (Acc)val[vu + t];
                }
                const int nn = min(32, cu - c0);
                for (int k = 0; k < nn; ++k) {
                    const Acc u = __shfl_sync(~0u, ul, k);
                    const int i = __shfl_sync(~0u, il, k);
                    if (u == Acc(0)) continue;
                    int64_t vl;
                    int cl;
                    const uint16_t *rl;
                    colview(dl, i, a, vl, cl, rl);
                    for (int e = lane; e < cl; e += 32)
                        acc[rowat(rl, e)] += (Acc)val[vl + e] * u;
                    __syncwarp();
                }
            }
        }
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

// ---------------------------------------------------------------- host side

template <typename V>
static bool upload(const std::vector<V> &h, V **d) {
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
                    D->a2s, D->f2s, D->a_rowptr, D->a_vpos, D->a_colidx,
                    D->lrow_off, D->urow_off, D->ucol_off, D->lcol_off,
                    D->lrow_blk, D->urow_blk, D->ucol_blk, D->lcol_blk};
    for (void *p : ptrs)
        if (p) cudaFree(p);
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
    const bool ok =
        upload(P->blocks, &D->bd) && upload(P->lcolptr, &D->lcolptr) &&
        upload(P->lrow, &D->lrow) && upload(P->dpos, &D->dpos) &&
        upload(P->sched, &D->sched) && upload(P->sgrp, &D->sgrp) &&
        upload(P->getrf, &D->getrf) && upload(P->gessm, &D->gessm) &&
        upload(P->tstrf, &D->tstrf) && upload(P->tgt, &D->tgt) &&
        upload(P->src, &D->src) && upload(P->srcoff, &D->srcoff) &&
        upload(P->a2s, &D->a2s) && upload(P->f2s, &D->f2s) &&
        upload(P->a_rowptr, &D->a_rowptr) && upload(P->a_vpos, &D->a_vpos) &&
        upload(P->a_colidx, &D->a_colidx) &&
        upload(P->lrow_off, &D->lrow_off) && upload(P->urow_off, &D->urow_off) &&
        upload(P->ucol_off, &D->ucol_off) && upload(P->lcol_off, &D->lcol_off) &&
        upload(P->lrow_blk, &D->lrow_blk) && upload(P->urow_blk, &D->urow_blk) &&
        upload(P->ucol_blk, &D->ucol_blk) && upload(P->lcol_blk, &D->lcol_blk);
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

template <typename T, typename Acc>
static slu_status set_smem_limits(size_t bytes) {
    if (bytes <= 48 * 1024) return SLU_OK;
    const int b = (int)bytes;
    const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    const bool ok = cuda_ok(cudaFuncSetAttribute(k_getrf<T>, attr, b), "smem") &&
                    cuda_ok(cudaFuncSetAttribute(k_panel<T, Acc>, attr, b), "smem") &&
                    cuda_ok(cudaFuncSetAttribute(k_ssssm<T, Acc>, attr, b), "smem");
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
        !cuda_ok(cudaMemsetAsync(h->cnt, 0, 2 * sizeof(unsigned long long), st),
                 "cudaMemsetAsync(cnt)"))
        return SLU_ERR_CUDA;
    if (P->nnz_a > 0) {
        {
            LaunchScope ls_(h, SLU_KC_PREP, st);
            k_maxabs<<<grid_for(P->nnz_a, 256), 256, 0, st>>>(
                P->nnz_a, values, reinterpret_cast<unsigned long long *>(h->scal));
        }
        {
            LaunchScope ls_(h, SLU_KC_PREP, st);
            k_anorm<<<(int)((P->n + 255) / 256), 256, 0, st>>>(
                P->n, D->a_rowptr, D->a_vpos, values,
                reinterpret_cast<unsigned long long *>(h->scal + 1));
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
    const size_t smem_f = (size_t)kWarps * P->maxb * sizeof(double);
    const size_t smem_a = (size_t)kWarps * P->maxb * sizeof(Acc);
    if (set_smem_limits<T, Acc>(std::max(smem_f, smem_a)) != SLU_OK)
        return SLU_ERR_CUDA;
    for (int lv = 0; lv < P->nlevels; ++lv) {
        const int64_t g0 = P->getrf_off[lv], g1 = P->getrf_off[lv + 1];
        if (g1 > g0) {
                LaunchScope ls_(h, SLU_KC_GETRF, st);
                k_getrf<T><<<(int)(g1 - g0), kThreads, smem_f, st>>>(
                    D->getrf + g0, a, val, h->scal, h->tau_rel, h->cnt);
            }
        const int64_t e0 = P->gessm_off[lv], e1 = P->gessm_off[lv + 1];
        const int64_t t0 = P->tstrf_off[lv], t1 = P->tstrf_off[lv + 1];
        if (e1 - e0 + t1 - t0 > 0) {
                LaunchScope ls_(h, SLU_KC_PANEL, st);
                k_panel<T, Acc><<<(int)(e1 - e0 + t1 - t0), kThreads, smem_a, st>>>(
                    D->gessm + 2 * e0, (int)(e1 - e0), D->tstrf + 2 * t0, a, val);
            }
        const int64_t s0 = P->tgt_off[lv], s1 = P->tgt_off[lv + 1];
        if (s1 > s0) {
                LaunchScope ls_(h, SLU_KC_SSSSM, st);
                k_ssssm<T, Acc><<<(int)(s1 - s0), kThreads, smem_a, st>>>(
                    D->tgt + s0, D->srcoff + s0, D->src, a, val);
            }
    }
    if (!cuda_ok(cudaGetLastError(), "factor launch")) return SLU_ERR_CUDA;
    return SLU_OK;
}

static slu_status finish_info(slu_handle *h, cudaStream_t st,
                              slu_factor_info *info) {
    unsigned long long c[2];
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
    if (c[1]) return fail(SLU_ERR_SINGULAR, "zero pivot (perturbation off)");
    return SLU_OK;
}

slu_status factor_into(slu_handle *h, const double *values, cudaStream_t st) {
    return h->prec == SLU_PREC_FP64 ? run_factor<double>(h, values, st)
                                    : run_factor<float>(h, values, st);
}

}  // namespace slu

using namespace slu;

extern "C" void slu_handle_destroy(slu_handle *h) {
    if (!h) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (h->device >= 0) cudaSetDevice(h->device);
    for (auto &r : h->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    void *ptrs[] = {h->storage, h->a_vals, h->scal, h->cnt, h->work, h->red};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (cur >= 0) cudaSetDevice(cur);
    delete h;
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
    // Diagonal-block pivots are formed in FP64 for both storage precisions,
    // so one threshold serves both: sqrt(eps64) ~ 2^-26 of max|A|.
    if (P->opts.pivot_perturb)
        h->tau_rel = P->opts.pivot_tau_rel > 0 ? P->opts.pivot_tau_rel
                                               : std::ldexp(1.0, -26);
    const size_t esz = fp64 ? sizeof(double) : sizeof(float);
    const bool ok =
        cuda_ok(cudaMalloc(&h->storage, std::max<int64_t>(1, P->storage) * esz),
                "cudaMalloc(storage)") &&
        cuda_ok(cudaMalloc(&h->scal, 4 * sizeof(double)), "cudaMalloc") &&
        cuda_ok(cudaMalloc(&h->cnt, 2 * sizeof(unsigned long long)), "cudaMalloc") &&
        cuda_ok(cudaMalloc(&h->a_vals, std::max<int64_t>(1, P->nnz_a) * sizeof(double)),
                "cudaMalloc(A)");
    if (!ok) {
        slu_handle_destroy(h);
        return SLU_ERR_OUT_OF_MEMORY;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = factor_into(h, values, s);
    if (st == SLU_OK) st = finish_info(h, s, info);
    if (st != SLU_OK && st != SLU_ERR_SINGULAR) {
        slu_handle_destroy(h);
        return st;
    }
    *out = h;
    return st;
}

extern "C" slu_status slu_refactor(slu_handle *h, const double *values,
                                   void *stream, slu_factor_info *info) {
    if (!h) return fail(SLU_ERR_INVALID_ARG, "NULL handle");
    if (h->plan->nnz_a > 0 && !values)
        return fail(SLU_ERR_INVALID_ARG, "values is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const slu_status st = factor_into(h, values, s);
    if (st != SLU_OK) return st;
    if (info) return finish_info(h, s, info);
    return SLU_OK;
}

extern "C" slu_status slu_set_profiling(slu_handle *h, int32_t enable) {
    if (!h) return fail(SLU_ERR_INVALID_ARG, "NULL handle");
    for (auto &r : h->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    h->recs.clear();
    for (int c = 0; c < SLU_KC_COUNT; ++c) {
        h->calls[c] = 0;
        h->ms[c] = 0.0;
    }
    h->profiling = enable != 0;
    return SLU_OK;
}

extern "C" slu_status slu_handle_stats(slu_handle *h, slu_stats *out) {
    if (!h || !out) return fail(SLU_ERR_INVALID_ARG, "NULL argument");
    if (!h->recs.empty() &&
        !cuda_ok(cudaEventSynchronize(h->recs.back().b), "cudaEventSynchronize"))
        return SLU_ERR_CUDA;
    for (auto &r : h->recs) {
        float t = 0.f;
        if (!cuda_ok(cudaEventElapsedTime(&t, r.a, r.b), "cudaEventElapsedTime"))
            return SLU_ERR_CUDA;
        h->calls[r.cls]++;
        h->ms[r.cls] += t;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    h->recs.clear();
    out->launches = h->launches;
    for (int c = 0; c < SLU_KC_COUNT; ++c) {
        out->calls[c] = h->calls[c];
        out->ms[c] = h->ms[c];
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
