// Device symbolic analysis (slu_analyze_device): the steps of the host
// analysis that walk the pattern entry by entry, on the GPU.
//
//   1. pattern(A + A^T) plus the full diagonal: every entry (j, r) of A
//      contributes the keys (column j, row r) and (column r, row j), every
//      column its diagonal (j, j); one stable LSD radix sort of the keys and
//      a pass that drops repeated keys leave S in CSC with rows ascending.
//   2. The elimination tree of S (Section 1's symbolic factorization) as
//      the fixpoint of a parallel relaxation.  parent(k) starts at the
//      smallest row > k of S(:, k).  A sweep takes every strictly lower
//      entry (i, k) of S, climbs from k while parent(x) < i and lowers
//      parent(x) to i with an atomic minimum; the climbs of one row i share
//      a visited bitmap (one warp per row), so a sweep costs at most the
//      entries of L.  Every value parent(x) ever
//      holds is an ancestor of x in the elimination tree (the start value
//      is, because A(i, k) != 0 makes i an ancestor of k; the climb ends at
//      an ancestor x of k below i, and i, also an ancestor of k, is then an
//      ancestor of x).  A sweep in which no climb changes anything and every
//      climb ends at x with parent(x) = i leaves a tree in which each entry
//      (i, k) has i above k, built from ancestors only; the elimination tree
//      is the only such tree, because for a column j with parent p there is
//      a descendant v of j with S(p, v) != 0 and j lies on the path from v
//      up to p.  Values only decrease, so the sweeps terminate.
//   3. struct L by row subtrees: row i of L holds exactly the nodes on the
//      tree paths from each k < i with S(i, k) != 0 up to (not including) i.
//      One warp per row climbs from those k in parallel, marking visited
//      nodes in a per-warp bitmap (shared memory when it fits), and emits
//      for every node x of the row the keys (column x, row i) of L and
//      (column i, row x) of U, plus the diagonal (i, i).  The settled sweep
//      of step 2 visits the same nodes and counts them, so the key buffer
//      is allocated exactly.
//   4. A second radix sort of those keys gives the filled L+U pattern with
//      rows ascending in every column, the column pointers read off at the
//      boundaries.
//   5. Algorithm 2 (Section 4.2) over the filled pattern: num[index] counts
//      the entries of column i with row index > i (one atomic increment per
//      entry), and blockptr[i + 1] = blockptr[i] + 2 num[i] + 1 by an
//      exclusive prefix sum of the terms.
//   6. Section 4.3: the S sampled points of the percentage curve and
//      Algorithm 3's walk, one CTA per matrix of a batch.  The dense test
//      of every step runs in parallel; the walk itself, whose counter l
//      carries from one step to the next, runs on one thread.
// The results are the host analysis's, entry for entry: the symmetric
// pattern, the elimination tree and the filled pattern are unique, and the
// integer prefix sums and the walk are exact.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "slu_internal.hpp"

namespace slu {

namespace {

constexpr int kThreads = 256;

// --------------------------------------------------------------- scan --

constexpr int kScanItems = 8;
constexpr int kScanTile = kThreads * kScanItems;

// exclusive prefix sum of one tile of 2048 values in place; the tile's
// total goes to sums[tile]
__global__ void __launch_bounds__(kThreads)
k_scan_tile(int64_t *a, int64_t n, int64_t *sums) {
    __shared__ int64_t wsum[kThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? a[base + k] : 0;
        s += v[k];
    }
    int64_t inc = s;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += t;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        int64_t x = lane < kThreads / 32 ? wsum[lane] : 0;
#pragma unroll
        for (int off = 1; off < kThreads / 32; off <<= 1) {
            const int64_t t = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += t;
        }
        if (lane < kThreads / 32) wsum[lane] = x;
    }
    __syncthreads();
    int64_t ex = inc - s + (w > 0 ? wsum[w - 1] : 0);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) a[base + k] = ex;
        ex += v[k];
    }
    if (threadIdx.x == kThreads - 1) sums[blockIdx.x] = wsum[kThreads / 32 - 1];
}

__global__ void k_scan_add(int64_t *a, int64_t n, const int64_t *sums) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] += sums[i / kScanTile];
}

// ------------------------------------------------------- radix sort --

constexpr int kRadixItems = 32;                 // keys per thread per tile
constexpr int kRadixTile = kThreads * kRadixItems;

// digit counts of one tile, stored digit-major: hist[d * ntiles + tile]
__global__ void __launch_bounds__(kThreads)
k_radix_hist(const uint64_t *keys, int64_t n, int shift, int64_t ntiles,
             int64_t *hist) {
    __shared__ int cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int c = 0; c < kRadixItems; ++c) {
        const int64_t i = base + (int64_t)c * kThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// stable scatter of one tile: the tile is walked in chunks of 256 keys in
// order; inside a chunk a key's rank among equal digits is its rank within
// its warp (lanes of equal digit found by match) plus the counts of that
// digit in the warps before it
__global__ void __launch_bounds__(kThreads)
k_radix_scatter(const uint64_t *in, uint64_t *out, int64_t n, int shift,
                int64_t ntiles, const int64_t *offs) {
    __shared__ int wcnt[kThreads / 32][256];
    __shared__ int64_t base[256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    base[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + blockIdx.x];
#pragma unroll
    for (int q = 0; q < kThreads / 32; ++q) wcnt[q][threadIdx.x] = 0;
    __syncthreads();
    const int64_t t0 = (int64_t)blockIdx.x * kRadixTile;
    const unsigned lt = (1u << lane) - 1u;
    for (int c = 0; c < kRadixItems; ++c) {
        const int64_t i = t0 + (int64_t)c * kThreads + threadIdx.x;
        const bool valid = i < n;
        const uint64_t key = valid ? in[i] : 0;
        const int d = valid ? (int)((key >> shift) & 255) : 256;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[w][d] = __popc(peers);
        __syncthreads();
        int run = 0;
#pragma unroll
        for (int q = 0; q < kThreads / 32; ++q) {
            const int t = wcnt[q][threadIdx.x];
            wcnt[q][threadIdx.x] = run;
            run += t;
        }
        __syncthreads();
        if (valid) out[base[d] + wcnt[w][d] + rank] = key;
        __syncthreads();
        base[threadIdx.x] += run;
#pragma unroll
        for (int q = 0; q < kThreads / 32; ++q) wcnt[q][threadIdx.x] = 0;
        __syncthreads();
    }
}

// ------------------------------------------------ symmetric pattern --

// keys of pattern(A + A^T) + diag, unsorted: entry e of A gives keys 2e and
// 2e + 1, column j's diagonal key 2 nnz + j (one warp per column)
__global__ void __launch_bounds__(kThreads)
k_sym_keys(int64_t n, const int64_t *colptr, const int32_t *rowidx, int b,
           uint64_t *keys) {
    const int lane = threadIdx.x & 31;
    const int64_t nnz = colptr[n];
    for (int64_t j = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5; j < n;
         j += ((int64_t)gridDim.x * kThreads) >> 5) {
        for (int64_t e = colptr[j] + lane; e < colptr[j + 1]; e += 32) {
            const uint64_t r = (uint32_t)rowidx[e];
            keys[2 * e] = ((uint64_t)j << b) | r;
            keys[2 * e + 1] = (r << b) | (uint64_t)j;
        }
        if (lane == 0) keys[2 * nnz + j] = ((uint64_t)j << b) | (uint64_t)j;
    }
}

// flag[p] = 1 for the first of every run of equal keys; flag[m] = 0
__global__ void k_first_flags(const uint64_t *keys, int64_t m, int64_t *flag) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p <= m;
         p += (int64_t)gridDim.x * blockDim.x)
        flag[p] = p < m && (p == 0 || keys[p] != keys[p - 1]);
}

// S in CSC: rows, columns, column pointers and diagonal positions
__global__ void k_sym_compact(const uint64_t *keys, int64_t m, const int64_t *pos,
                              int b, int64_t n, int32_t *srow, int64_t *sptr,
                              int64_t *sdiag) {
    const uint64_t mask = ((uint64_t)1 << b) - 1;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = keys[p];
        if (p > 0 && key == keys[p - 1]) continue;
        const int64_t q = pos[p];
        const int32_t c = (int32_t)(key >> b), r = (int32_t)(key & mask);
        srow[q] = r;
        if (q == 0 || (p > 0 && (int32_t)(keys[p - 1] >> b) != c)) sptr[c] = q;
        if (r == c) sdiag[c] = q;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) sptr[n] = pos[m];
}

// ------------------------------------------------- elimination tree --

constexpr int32_t kRoot = INT32_MAX;            // parent of a root

__global__ void k_parent_init(int64_t n, const int64_t *sptr, const int64_t *sdiag,
                              const int32_t *srow, int32_t *parent) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        parent[k] = sdiag[k] + 1 < sptr[k + 1] ? srow[sdiag[k] + 1] : kRoot;
}

// ------------------------------------------------------- row subtrees --

constexpr int kStage = 128;                     // staged keys per warp

// Climbs from every k < i with S(i, k) != 0 toward i, one warp per row i
// (lanes take the k's), with a visited bitmap per warp so that climbs of
// one row that meet stop where the first passed; rows are taken largest
// index first from *ticket (late rows have the longest climbs).
//   SWEEP: one relaxation sweep of the elimination tree.  A climb that ends
//     at x with parent(x) > i lowers parent(x) to i (atomic minimum, reads of
//     parent from L2) and marks the sweep unsettled, as does one that finds
//     parent(x) below i after its read (a concurrent change).  The keys a
//     row's climbs visit are counted into *cursor: in a settled sweep the
//     tree is final and row i visits exactly row i of L.
//   EMIT: with the final tree, row i of L: the keys (column x, row i) and
//     (column i, row x) for every node x visited and the diagonal (i, i),
//     staged per warp and written at positions reserved from *cursor.
// A climb of a settled sweep and of EMIT visits the same nodes, so EMIT
// writes exactly the settled sweep's count.
template <bool EMIT>
__global__ void __launch_bounds__(kThreads)
k_row_climb(int64_t n, const int64_t *sptr, const int64_t *sdiag,
            const int32_t *srow, int32_t *parent, uint32_t *gbits, int64_t words,
            int b, uint64_t *keys, unsigned long long cap,
            unsigned long long *cursor, unsigned long long *ticket, int *unsettled) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    uint64_t *stage = reinterpret_cast<uint64_t *>(smem) + w * kStage;
    uint32_t *bits = gbits
        ? gbits + ((int64_t)blockIdx.x * (kThreads / 32) + w) * words
        : reinterpret_cast<uint32_t *>(smem + sizeof(uint64_t) * kStage * (kThreads / 32)) +
              w * words;
    for (int64_t t = lane; t < words; t += 32) bits[t] = 0;
    __syncwarp();
    int cnt = 0;                                // staged keys (warp-uniform)
    unsigned long long total = 0;               // counted keys (lane 0)
    int any = 0;                                // this lane lowered a parent
    auto flush = [&]() {
        unsigned long long at = 0;
        if (lane == 0 && cnt) at = atomicAdd(cursor, (unsigned long long)cnt);
        at = __shfl_sync(0xffffffffu, at, 0);
        for (int t = lane; t < cnt; t += 32)
            if (at + t < cap) keys[at + t] = stage[t];
        __syncwarp();
        cnt = 0;
    };
    for (;;) {
        unsigned long long r = 0;
        if (lane == 0) r = atomicAdd(ticket, 1ull);
        r = __shfl_sync(0xffffffffu, r, 0);
        if (r >= (unsigned long long)n) break;
        const int32_t i = (int32_t)(n - 1 - (int64_t)r);
        const int64_t q0 = sptr[i], q1 = sdiag[i];
        if (EMIT) {
            // room for the diagonal and one climbing step (64 keys): a run
            // of rows with no lower entries adds diagonals only
            if (cnt + 65 > kStage) flush();
            if (lane == 0) stage[cnt] = ((uint64_t)i << b) | (uint64_t)i;
            ++cnt;
        } else if (lane == 0) {
            ++total;
        }
        const int32_t mink = q0 < q1 ? srow[q0] : i;
        int64_t q = q0 + lane;
        int32_t x = q < q1 ? srow[q] : i;
        while (__any_sync(0xffffffffu, q < q1)) {
            bool emit = false;
            int32_t ex = 0;
            if (q < q1) {
                if (x < i) {
                    const uint32_t m = 1u << (x & 31);
                    const uint32_t old = atomicOr(bits + (x >> 5), m);
                    if (!(old & m)) {
                        emit = true;
                        ex = x;
                        const int32_t nx = EMIT ? __ldg(parent + x) : __ldcg(parent + x);
                        if (!EMIT && nx > i) {  // the climb ends below i
                            const int32_t was = atomicMin(parent + x, i);
                            any |= was != i;
                        }
                        x = nx > x ? nx : i;    // parents increase: climbs end
                    } else {
                        x = i;                  // joined a path already taken
                    }
                }
                if (x >= i) {
                    q += 32;
                    x = q < q1 ? srow[q] : i;
                }
            }
            const unsigned em = __ballot_sync(0xffffffffu, emit);
            if (EMIT) {
                if (emit) {
                    const int at = cnt + 2 * __popc(em & lt);
                    stage[at] = ((uint64_t)ex << b) | (uint64_t)i;
                    stage[at + 1] = ((uint64_t)i << b) | (uint64_t)ex;
                }
                cnt += 2 * __popc(em);
                __syncwarp();
                if (cnt + 65 > kStage) flush();
            } else if (lane == 0) {
                total += 2 * __popc(em);
            }
        }
        __syncwarp();
        // every bit set for this row lies in [mink, i)
        if (mink < i)
            for (int64_t t = (mink >> 5) + lane; t <= ((int64_t)i - 1) >> 5; t += 32)
                bits[t] = 0;
        __syncwarp();
    }
    if (EMIT) flush();
    else if (lane == 0 && total) atomicAdd(cursor, total);
    if (!EMIT && __any_sync(0xffffffffu, any) && lane == 0) atomicExch(unsettled, 1);
}

// --------------------------------------------------- filled pattern --

__global__ void k_filled_split(const uint64_t *keys, int64_t m, int b, int64_t n,
                               int32_t *frow, int64_t *fptr) {
    const uint64_t mask = ((uint64_t)1 << b) - 1;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = keys[p];
        frow[p] = (int32_t)(key & mask);
        if (p == 0 || (keys[p - 1] >> b) != (key >> b)) fptr[key >> b] = p;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) fptr[n] = m;
}

// Algorithm 2, counting: for every column i and every entry of it whose row
// index exceeds i, num[index] += 1
__global__ void k_alg2_count(const uint64_t *keys, int64_t m, int b, int32_t *num) {
    const uint64_t mask = ((uint64_t)1 << b) - 1;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = keys[p];
        const int64_t i = (int64_t)(key >> b), index = (int64_t)(key & mask);
        if (index > i) atomicAdd(num + index, 1);
    }
}

// Algorithm 2, the terms 2 num[i] + 1 of blockptr (the prefix sum follows)
__global__ void k_alg2_terms(const int32_t *num, int64_t n, int64_t *bp) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n;
         i += (int64_t)gridDim.x * blockDim.x)
        bp[i] = i < n ? 2 * (int64_t)num[i] + 1 : 0;
}

// ------------------------------------------------- Algorithm 3 --

struct SegJob {
    int64_t s0, N;          // first row, order
    int64_t S;              // samples
    int64_t nsteps;         // steps i = 0, stride, ... with i + step <= S
    int64_t out;            // first output slot (nsteps + 2 of them)
    int64_t flags;          // first dense-test slot (nsteps of them)
};

__device__ __forceinline__ int64_t idx_at(int64_t s, int64_t N, int64_t S) {
    return (s * N) / S;
}

// One CTA per matrix.  The dense test pct(i + step) - pct(i) >= step / S,
// exact in integers as (bp[idx(i + step)] - bp[idx(i)]) S >= step bp[N],
// for every step i = 0, stride, ... with i + step <= S, in parallel; then
// one thread walks the steps with the block-size counter l.
__global__ void k_alg3(const SegJob *jobs, const int64_t *bp, int32_t step,
                       int32_t max_num, int32_t stride, unsigned char *dense,
                       int64_t *out, int64_t *count) {
    const SegJob jb = jobs[blockIdx.x];
    const int64_t *b = bp + jb.s0;
    const int64_t total = b[jb.N] - b[0];
    const int64_t nsteps = jb.nsteps;
    for (int64_t t = threadIdx.x; t < nsteps; t += blockDim.x) {
        const int64_t i = t * stride;
        const int64_t a = b[idx_at(i, jb.N, jb.S)] - b[0];
        const int64_t c = b[idx_at(i + step, jb.N, jb.S)] - b[0];
        dense[jb.flags + t] = (c - a) * jb.S >= (int64_t)step * total;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    int64_t *o = out + jb.out;
    int64_t k = 0, last = 0;
    o[k++] = 0;
    int32_t l = 0;
    for (int64_t t = 0; t < nsteps; ++t) {
        bool mark;
        if (dense[jb.flags + t]) {
            mark = true;                        // dense region
        } else if (l >= max_num) {
            mark = true;                        // bound the block size
        } else {
            mark = false;
            ++l;
        }
        if (mark) {
            const int64_t pos = idx_at(t * stride + step, jb.N, jb.S);
            if (pos > last) o[k++] = last = pos;
            l = 0;
        }
    }
    if (last < jb.N) o[k++] = jb.N;
    count[blockIdx.x] = k;
}

// ------------------------------------------------------------ host --

// Device buffers of one call, released on the call's stream at the end.
struct Arena {
    cudaStream_t st;
    std::vector<void *> held;
    explicit Arena(cudaStream_t s) : st(s) {}
    ~Arena() { release(); }
    void release() {
        for (void *p : held) cudaFreeAsync(p, st);
        held.clear();
    }
    template <class T>
    T *get(int64_t count) {
        void *p = nullptr;
        const size_t bytes = std::max<size_t>(sizeof(T), sizeof(T) * (size_t)count);
        if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        held.push_back(p);
        return static_cast<T *>(p);
    }
    void drop(void *p) {
        auto it = std::find(held.begin(), held.end(), p);
        if (it != held.end()) {
            cudaFreeAsync(p, st);
            held.erase(it);
        }
    }
};

struct Ctx {
    cudaStream_t st;
    Arena ar;
    int sms = 148;
    explicit Ctx(cudaStream_t s) : st(s), ar(s) {}
    int grid(int64_t items, int per_sm = 16) const {
        const int64_t g = (items + kThreads - 1) / kThreads;
        return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)sms * per_sm));
    }
};

slu_status cuda_err(const char *what) {
    const cudaError_t e = cudaGetLastError();
    return fail(SLU_ERR_CUDA, std::string("device analysis, ") + what + ": " +
                                  cudaGetErrorString(e));
}

#define SLU_DEV_CHECK(what)                                       \
    do {                                                          \
        if (cudaPeekAtLastError() != cudaSuccess) return cuda_err(what); \
    } while (0)

// exclusive prefix sum of a[0 .. n) in place
slu_status dev_scan(Ctx &cx, int64_t *a, int64_t n) {
    if (n <= 0) return SLU_OK;
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    int64_t *sums = cx.ar.get<int64_t>(nb);
    if (!sums) return fail(SLU_ERR_OUT_OF_MEMORY, "device allocation in analyze");
    k_scan_tile<<<(unsigned)nb, kThreads, 0, cx.st>>>(a, n, sums);
    SLU_DEV_CHECK("scan");
    if (nb > 1) {
        const slu_status s = dev_scan(cx, sums, nb);
        if (s != SLU_OK) return s;
        k_scan_add<<<cx.grid(n), kThreads, 0, cx.st>>>(a, n, sums);
        SLU_DEV_CHECK("scan");
    }
    cx.ar.drop(sums);
    return SLU_OK;
}

// stable LSD sort of keys[0 .. m) on their low `bits` bits; *keys and *alt
// may be swapped, *keys holds the result
slu_status dev_sort(Ctx &cx, uint64_t **keys, uint64_t **alt, int64_t m, int bits) {
    if (m <= 1) return SLU_OK;
    const int64_t ntiles = (m + kRadixTile - 1) / kRadixTile;
    int64_t *hist = cx.ar.get<int64_t>(256 * ntiles);
    if (!hist) return fail(SLU_ERR_OUT_OF_MEMORY, "device allocation in analyze");
    for (int shift = 0; shift < bits; shift += 8) {
        k_radix_hist<<<(unsigned)ntiles, kThreads, 0, cx.st>>>(*keys, m, shift, ntiles, hist);
        SLU_DEV_CHECK("radix sort");
        const slu_status s = dev_scan(cx, hist, 256 * ntiles);
        if (s != SLU_OK) return s;
        k_radix_scatter<<<(unsigned)ntiles, kThreads, 0, cx.st>>>(*keys, *alt, m, shift,
                                                                   ntiles, hist);
        SLU_DEV_CHECK("radix sort");
        std::swap(*keys, *alt);
    }
    cx.ar.drop(hist);
    return SLU_OK;
}

// Copies between pageable host memory and the device through two pinned
// staging buffers (kept for the process, grown on demand): the DMA of one
// chunk overlaps the threaded host copy of the previous one, and the host
// threads touch the pageable pages in parallel.
struct Staging {
    std::mutex mu;
    void *buf[2] = {nullptr, nullptr};
    cudaEvent_t ev[2] = {nullptr, nullptr};
    size_t bytes = 0;
};
Staging &staging() {
    static Staging *s = new Staging();          // outlives every caller
    return *s;
}
constexpr size_t kChunk = (size_t)32 << 20;

void par_copy(void *dst, const void *src, size_t bytes) {
    const int nt = (int)std::min<size_t>(
        std::min<size_t>(16, std::max(1u, std::thread::hardware_concurrency())),
        std::max<size_t>(1, bytes >> 21));
    const size_t per = (bytes / nt + 4095) & ~(size_t)4095;
    std::vector<std::thread> th;
    try {
        for (int t = 1; t < nt && per * t < bytes; ++t)
            th.emplace_back([=] {
                const size_t a = per * t, e = std::min(bytes, per * (t + 1));
                std::memcpy(static_cast<char *>(dst) + a, static_cast<const char *>(src) + a, e - a);
            });
    } catch (const std::exception &) {
    }
    const size_t done = per * (th.size() + 1);
    std::memcpy(dst, src, std::min(bytes, per));
    if (done < bytes)
        std::memcpy(static_cast<char *>(dst) + done, static_cast<const char *>(src) + done,
                    bytes - done);
    for (auto &x : th) x.join();
}

// host (pageable) <-> device through the staging buffers; returns after
// the copy has finished
slu_status staged_copy(Ctx &cx, void *dst, const void *src, size_t bytes, bool to_device) {
    if (bytes == 0) return SLU_OK;
    Staging &sg = staging();
    std::lock_guard<std::mutex> lock(sg.mu);
    if (!sg.buf[0]) {
        for (int k = 0; k < 2; ++k)
            if (cudaHostAlloc(&sg.buf[k], kChunk, cudaHostAllocDefault) != cudaSuccess ||
                cudaEventCreateWithFlags(&sg.ev[k], cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                for (int j = 0; j < 2; ++j) {
                    if (sg.buf[j]) cudaFreeHost(sg.buf[j]);
                    if (sg.ev[j]) cudaEventDestroy(sg.ev[j]);
                    sg.buf[j] = nullptr;
                    sg.ev[j] = nullptr;
                }
                return fail(SLU_ERR_OUT_OF_MEMORY, "pinned staging allocation in analyze");
            }
        sg.bytes = kChunk;
    }
    const size_t nchunk = (bytes + kChunk - 1) / kChunk;
    auto len = [&](size_t c) { return std::min(kChunk, bytes - c * kChunk); };
    char *d = static_cast<char *>(dst);
    const char *s = static_cast<const char *>(src);
    if (to_device) {
        // host copy of chunk c into buffer c % 2 (after the DMA of chunk
        // c - 2 out of it finished), then its DMA
        for (size_t c = 0; c < nchunk; ++c) {
            const int k = (int)(c & 1);
            if (c >= 2 && cudaEventSynchronize(sg.ev[k]) != cudaSuccess)
                return cuda_err("copy to device");
            par_copy(sg.buf[k], s + c * kChunk, len(c));
            if (cudaMemcpyAsync(d + c * kChunk, sg.buf[k], len(c), cudaMemcpyHostToDevice,
                                cx.st) != cudaSuccess ||
                cudaEventRecord(sg.ev[k], cx.st) != cudaSuccess)
                return cuda_err("copy to device");
        }
        if (cudaStreamSynchronize(cx.st) != cudaSuccess) return cuda_err("copy to device");
        return SLU_OK;
    }
    // DMA of chunk c into buffer c % 2, then the host copy of chunk c - 1
    for (size_t c = 0; c <= nchunk; ++c) {
        if (c < nchunk) {
            const int k = (int)(c & 1);
            if (cudaMemcpyAsync(sg.buf[k], s + c * kChunk, len(c), cudaMemcpyDeviceToHost,
                                cx.st) != cudaSuccess ||
                cudaEventRecord(sg.ev[k], cx.st) != cudaSuccess)
                return cuda_err("copy to host");
        }
        if (c > 0) {
            const int k = (int)((c - 1) & 1);
            if (cudaEventSynchronize(sg.ev[k]) != cudaSuccess) return cuda_err("copy to host");
            par_copy(d + (c - 1) * kChunk, sg.buf[k], len(c - 1));
        }
    }
    return SLU_OK;
}

template <class T, class A>
slu_status to_host(Ctx &cx, std::vector<T, A> &dst, const T *src, int64_t count) {
    try {
        dst.resize((size_t)count);
    } catch (const std::exception &) {
        return fail(SLU_ERR_OUT_OF_MEMORY, "host allocation in analyze");
    }
    return staged_copy(cx, dst.data(), src, sizeof(T) * (size_t)count, false);
}

template <class T>
slu_status read_scalar(Ctx &cx, T *dst, const T *src) {
    if (cudaMemcpyAsync(dst, src, sizeof(T), cudaMemcpyDeviceToHost, cx.st) != cudaSuccess ||
        cudaStreamSynchronize(cx.st) != cudaSuccess)
        return cuda_err("copy to host");
    return SLU_OK;
}

double ms_since(std::chrono::steady_clock::time_point t) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t)
        .count();
}

slu_status symbolic_on_device(Ctx &cx, int64_t n, const int64_t *colptr,
                              const int32_t *rowidx, const std::vector<int64_t> &seg,
                              const slu_opts &o, bool irregular, slu_plan &P,
                              std::vector<std::vector<int64_t>> &seg_ptr,
                              DeviceSymbolicTimes &tm) {
    const auto t0 = std::chrono::steady_clock::now();
    const int64_t nnz = colptr[n];
    int b = 1;
    while (((int64_t)1 << b) < n) ++b;          // rows and columns fit b bits
    const int bits = 2 * b;
    // 1. pattern(A + A^T) + diag
    int64_t *dcp = cx.ar.get<int64_t>(n + 1);
    int32_t *dri = cx.ar.get<int32_t>(nnz);
    const int64_t m = 2 * nnz + n;
    uint64_t *ka = cx.ar.get<uint64_t>(m), *kb = cx.ar.get<uint64_t>(m);
    if (!dcp || !dri || !ka || !kb) return fail(SLU_ERR_OUT_OF_MEMORY, "device allocation in analyze");
    slu_status s = staged_copy(cx, dcp, colptr, sizeof(int64_t) * (n + 1), true);
    if (s == SLU_OK) s = staged_copy(cx, dri, rowidx, sizeof(int32_t) * nnz, true);
    if (s != SLU_OK) return s;
    k_sym_keys<<<cx.grid(32 * n, 32), kThreads, 0, cx.st>>>(n, dcp, dri, b, ka);
    SLU_DEV_CHECK("symmetric pattern");
    s = dev_sort(cx, &ka, &kb, m, bits);
    if (s != SLU_OK) return s;
    cx.ar.drop(dcp);
    cx.ar.drop(dri);
    cx.ar.drop(kb);
    int64_t *pos = cx.ar.get<int64_t>(m + 1);
    if (!pos) return fail(SLU_ERR_OUT_OF_MEMORY, "device allocation in analyze");
    k_first_flags<<<cx.grid(m + 1), kThreads, 0, cx.st>>>(ka, m, pos);
    SLU_DEV_CHECK("symmetric pattern");
    if ((s = dev_scan(cx, pos, m + 1)) != SLU_OK) return s;
    int64_t ns = 0;
    if ((s = read_scalar(cx, &ns, pos + m)) != SLU_OK) return s;
    int32_t *srow = cx.ar.get<int32_t>(ns);
    int64_t *sptr = cx.ar.get<int64_t>(n + 1), *sdiag = cx.ar.get<int64_t>(n);
    int32_t *parent = cx.ar.get<int32_t>(n);
    int *unsettled = cx.ar.get<int>(1);
    if (!srow || !sptr || !sdiag || !parent || !unsettled)
        return fail(SLU_ERR_OUT_OF_MEMORY, "device allocation in analyze");
    k_sym_compact<<<cx.grid(m), kThreads, 0, cx.st>>>(ka, m, pos, b, n, srow, sptr, sdiag);
    SLU_DEV_CHECK("symmetric pattern");
    cx.ar.drop(ka);
    cx.ar.drop(pos);
    P.nnz_sym = ns;
    // 2. elimination tree, and the count of the filled keys
    k_parent_init<<<cx.grid(n), kThreads, 0, cx.st>>>(n, sptr, sdiag, srow, parent);
    SLU_DEV_CHECK("elimination tree");
    const int64_t words = (n + 31) / 32;
    const size_t stage_bytes = sizeof(uint64_t) * kStage * (kThreads / 32);
    const size_t bitmap_bytes = sizeof(uint32_t) * (size_t)words * (kThreads / 32);
    size_t smem = stage_bytes + bitmap_bytes;
    int per_sm = (int)std::min<size_t>(8, (size_t)(224 * 1024) / smem);
    uint32_t *gbits = nullptr;
    if (smem > 200 * 1024 || per_sm < 1) {      // bitmaps in global memory
        smem = stage_bytes;
        per_sm = 2;
    }
    const int rgrid = cx.sms * per_sm;
    if (smem == stage_bytes) {
        gbits = cx.ar.get<uint32_t>((int64_t)rgrid * (kThreads / 32) * words);
        if (!gbits) return fail(SLU_ERR_OUT_OF_MEMORY, "device allocation in analyze");
    }
    if (cudaFuncSetAttribute(k_row_climb<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_row_climb<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return cuda_err("row climbs");
    unsigned long long *ctr = cx.ar.get<unsigned long long>(2);   // cursor, ticket
    if (!ctr) return fail(SLU_ERR_OUT_OF_MEMORY, "device allocation in analyze");
    tm.sweeps = 0;
    unsigned long long mf = 0;
    for (;;) {
        int flag = 0;
        if (cudaMemsetAsync(unsettled, 0, sizeof(int), cx.st) != cudaSuccess ||
            cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned long long), cx.st) != cudaSuccess)
            return cuda_err("elimination tree");
        k_row_climb<false><<<rgrid, kThreads, smem, cx.st>>>(
            n, sptr, sdiag, srow, parent, gbits, words, b, nullptr, 0, ctr, ctr + 1, unsettled);
        SLU_DEV_CHECK("elimination tree");
        if ((s = read_scalar(cx, &flag, unsettled)) != SLU_OK) return s;
        ++tm.sweeps;
        if (!flag) break;
        // every unsettled sweep lowers some parent value, which only
        // decreases, so this bound is never met by a correct relaxation
        if (tm.sweeps > n + 64)
            return fail(SLU_ERR_CUDA, "device analysis: elimination tree did not settle");
    }
    if ((s = read_scalar(cx, &mf, ctr)) != SLU_OK) return s;
    // 3. struct L and U with the final tree
    const int64_t nf = (int64_t)mf;
    uint64_t *fa = cx.ar.get<uint64_t>(nf), *fb = cx.ar.get<uint64_t>(nf);
    if (!fa || !fb) return fail(SLU_ERR_OUT_OF_MEMORY, "device allocation in analyze");
    if (cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned long long), cx.st) != cudaSuccess)
        return cuda_err("row climbs");
    k_row_climb<true><<<rgrid, kThreads, smem, cx.st>>>(
        n, sptr, sdiag, srow, parent, gbits, words, b, fa, mf, ctr, ctr + 1, unsettled);
    SLU_DEV_CHECK("row climbs");
    {
        unsigned long long again = 0;           // the settled sweep's count
        if ((s = read_scalar(cx, &again, ctr)) != SLU_OK) return s;
        if (again != mf)
            return fail(SLU_ERR_CUDA, "device analysis: row climbs disagree");
    }
    if (gbits) cx.ar.drop(gbits);
    cx.ar.drop(srow);
    cx.ar.drop(sptr);
    cx.ar.drop(sdiag);
    cx.ar.drop(parent);
    // 4. filled pattern
    if ((s = dev_sort(cx, &fa, &fb, nf, bits)) != SLU_OK) return s;
    int32_t *frow = reinterpret_cast<int32_t *>(fb);   // fits in the spare buffer
    int64_t *fptr = cx.ar.get<int64_t>(n + 1);
    if (!fptr) return fail(SLU_ERR_OUT_OF_MEMORY, "device allocation in analyze");
    k_filled_split<<<cx.grid(nf), kThreads, 0, cx.st>>>(fa, nf, b, n, frow, fptr);
    SLU_DEV_CHECK("filled pattern");
    if ((s = to_host(cx, P.f_colptr, fptr, n + 1)) != SLU_OK) return s;
    if ((s = to_host(cx, P.f_rowidx, frow, nf)) != SLU_OK) return s;
    if (cudaStreamSynchronize(cx.st) != cudaSuccess) return cuda_err("filled pattern");
    tm.symbolic_ms = ms_since(t0);
    // 5. Algorithm 2
    const auto t1 = std::chrono::steady_clock::now();
    int32_t *num = cx.ar.get<int32_t>(n);
    int64_t *bp = cx.ar.get<int64_t>(n + 1);
    if (!num || !bp) return fail(SLU_ERR_OUT_OF_MEMORY, "device allocation in analyze");
    if (cudaMemsetAsync(num, 0, sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1), cx.st) !=
        cudaSuccess)
        return cuda_err("Algorithm 2");
    k_alg2_count<<<cx.grid(nf), kThreads, 0, cx.st>>>(fa, nf, b, num);
    SLU_DEV_CHECK("Algorithm 2");
    k_alg2_terms<<<cx.grid(n + 1), kThreads, 0, cx.st>>>(num, n, bp);
    SLU_DEV_CHECK("Algorithm 2");
    if ((s = dev_scan(cx, bp, n + 1)) != SLU_OK) return s;
    // 6. sampling and Algorithm 3 per matrix
    std::vector<SegJob> jobs;
    int64_t nout = 0, nflag = 0;
    for (size_t q = 0; q + 1 < seg.size() && irregular; ++q) {
        SegJob jb;
        jb.s0 = seg[q];
        jb.N = seg[q + 1] - seg[q];
        if (jb.N == 0) continue;
        jb.S = std::max<int64_t>(1, std::min<int64_t>(o.sample_points, jb.N / o.b_min));
        jb.nsteps = jb.S >= o.step ? (jb.S - o.step) / o.stride + 1 : 0;
        jb.out = nout;
        jb.flags = nflag;
        nout += jb.nsteps + 2;
        nflag += jb.nsteps;
        jobs.push_back(jb);
    }
    std::vector<int64_t> outs, counts;
    if (!jobs.empty()) {
        SegJob *djobs = cx.ar.get<SegJob>((int64_t)jobs.size());
        unsigned char *dflag = cx.ar.get<unsigned char>(nflag);
        int64_t *dout = cx.ar.get<int64_t>(nout), *dcnt = cx.ar.get<int64_t>((int64_t)jobs.size());
        if (!djobs || !dflag || !dout || !dcnt)
            return fail(SLU_ERR_OUT_OF_MEMORY, "device allocation in analyze");
        if (cudaMemcpyAsync(djobs, jobs.data(), sizeof(SegJob) * jobs.size(),
                            cudaMemcpyHostToDevice, cx.st) != cudaSuccess)
            return cuda_err("Algorithm 3");
        k_alg3<<<(unsigned)jobs.size(), kThreads, 0, cx.st>>>(djobs, bp, o.step, o.max_num,
                                                              o.stride, dflag, dout, dcnt);
        SLU_DEV_CHECK("Algorithm 3");
        if ((s = to_host(cx, outs, dout, nout)) != SLU_OK) return s;
        if ((s = to_host(cx, counts, dcnt, (int64_t)jobs.size())) != SLU_OK) return s;
    }
    if ((s = to_host(cx, P.blockptr, bp, n + 1)) != SLU_OK) return s;
    if (cudaStreamSynchronize(cx.st) != cudaSuccess) return cuda_err("Algorithm 3");
    seg_ptr.assign(seg.size() > 0 ? seg.size() - 1 : 0, {});
    {
        size_t k = 0;
        for (size_t q = 0; q + 1 < seg.size() && irregular; ++q) {
            if (seg[q + 1] == seg[q]) continue;
            const SegJob &jb = jobs[k];
            if (counts[k] < 1 || counts[k] > jb.nsteps + 2)
                return fail(SLU_ERR_CUDA, "device analysis: Algorithm 3 output out of range");
            seg_ptr[q].assign(outs.begin() + jb.out, outs.begin() + jb.out + counts[k]);
            tm.samples = std::max<int64_t>(tm.samples, jb.S);
            ++k;
        }
    }
    tm.blocking_ms = ms_since(t1);
    return SLU_OK;
}

}  // namespace

slu_status device_symbolic(int64_t n, const int64_t *colptr, const int32_t *rowidx,
                           const std::vector<int64_t> &seg, const slu_opts &o,
                           bool irregular, void *stream, slu_plan &P,
                           std::vector<std::vector<int64_t>> &seg_ptr,
                           DeviceSymbolicTimes &tm) {
    tm = DeviceSymbolicTimes{};
    if (n == 0) {                               // nothing to analyse
        P.nnz_sym = 0;
        P.f_colptr.assign(1, 0);
        P.f_rowidx.clear();
        P.blockptr.assign(1, 0);
        seg_ptr.assign(seg.size() > 0 ? seg.size() - 1 : 0, {});
        return SLU_OK;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cuda_err("no CUDA device");
    Ctx cx(static_cast<cudaStream_t>(stream));
    if (cudaDeviceGetAttribute(&cx.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return cuda_err("device query");
    slu_status s;
    try {
        s = symbolic_on_device(cx, n, colptr, rowidx, seg, o, irregular, P, seg_ptr, tm);
    } catch (const std::exception &) {
        s = fail(SLU_ERR_OUT_OF_MEMORY, "host allocation in analyze");
    }
    // results already copied out (or an error): wait for the copies before
    // the buffers are returned and the host vectors read
    cudaStreamSynchronize(cx.st);
    cx.ar.release();
    if (s == SLU_OK && cudaStreamSynchronize(cx.st) != cudaSuccess)
        return cuda_err("device analysis");
    return s;
}

}  // namespace slu
