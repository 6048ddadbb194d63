// Internal structures of the irregular-block sparse LU library.
//
// Host analysis (analyze.cpp) builds an `slu_plan`; the device code
// (factor.cu, solve.cu) uploads its flat arrays once per plan and walks them.
//
// Storage of the factors.  The filled L+U pattern is cut by the block
// boundaries `ptr` (Algorithm 3, or regular) into 2-D blocks; only non-empty
// blocks are stored (Section 2.2: empty blocks are skipped).  Each block owns
// a contiguous run of value slots starting at `voff`:
//   dense  : column-major b_I x b_J tile, leading dimension `ld`; slots that
//            are not in the symbolic pattern hold exact zeros, which stay
//            zero through the factorization because the pattern is closed
//            under fill;
//   sparse : block-local CSC; column jj occupies local positions
//            [lcolptr[coff+jj], lcolptr[coff+jj+1]) with 16-bit local row
//            indices lrow[roff + pos] sorted ascending.
// A diagonal block keeps L's strict lower part and U's upper part (with the
// diagonal) of its rows and columns.
#pragma once
#include <cstdint>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "../../include/slu.h"

namespace slu {

struct BlockDesc {         // 64 bytes, read by every kernel
    int32_t I, J;          // block row, block column
    int32_t rows, cols;    // b_I, b_J
    int64_t voff;          // first value slot
    int64_t roff;          // sparse: first local row index slot
    int32_t coff;          // sparse: first local colptr slot (cols+1 of them)
    int32_t ld;            // dense: leading dimension (== rows)
    int32_t dense;         // 1 = dense tile
    int32_t r0, c0;        // first global row / column of the block
    int32_t doff;          // diagonal block: first dpos / sched slot
    int32_t goff;          // diagonal block: first height-group slot
    int32_t ngroups;       // diagonal block: number of height groups
};
static_assert(sizeof(BlockDesc) == 64, "BlockDesc layout");

struct DevPlan;            // device mirror, defined in device_common.cuh

// Allocator of the plan's pattern-sized arrays: resize() leaves the new
// elements uninitialized, so that the (threaded) pass that writes every one
// of them is the first to touch their pages; explicit values (assign,
// resize(n, v)) are stored as usual.
template <class T>
struct UninitAlloc : std::allocator<T> {
    template <class U>
    struct rebind {
        using other = UninitAlloc<U>;
    };
    UninitAlloc() = default;
    template <class U>
    UninitAlloc(const UninitAlloc<U> &) noexcept {}
    template <class U>
    void construct(U *p) noexcept {
        ::new (static_cast<void *>(p)) U;
    }
    template <class U, class... A>
    void construct(U *p, A &&...a) {
        ::new (static_cast<void *>(p)) U(std::forward<A>(a)...);
    }
};
template <class T>
using big_vector = std::vector<T, UninitAlloc<T>>;

}  // namespace slu

// Vectors per warp of the dense-panel substitution kernel: lane v owns
// vector v, stored interleaved (m rows x V) in shared memory within 112 KB;
// 0 when even 8 vectors of m rows do not fit.
#ifdef __CUDACC__
__host__ __device__
#endif
inline int panel_vec_width(int m, int esz) {
    for (int V = 32; V >= 8; V >>= 1)
        if ((long long)m * V * esz <= 112 * 1024) return V;
    return 0;
}

struct slu_plan {
    slu_opts opts;
    int64_t n = 0, nnz_a = 0, nnz_sym = 0;
    double analyze_ms = 0;
    double phase_ms[SLU_PHASE_COUNT] = {};
    // input pattern (copied) and its CSR view for the FP64 residual
    std::vector<int64_t> a_colptr;
    slu::big_vector<int32_t> a_rowidx;
    std::vector<int64_t> a_rowptr;       // CSR of A
    slu::big_vector<int32_t> a_colidx;
    slu::big_vector<int64_t> a_vpos;     // CSR entry -> position in values
    slu::big_vector<int32_t> a_ci;       // column of each CSC entry of A
    // filled, structurally symmetric L+U pattern (rows sorted)
    std::vector<int64_t> f_colptr;
    slu::big_vector<int32_t> f_rowidx;
    int64_t flops = 0;
    double flops_cls[3] = {0, 0, 0};     // getrf, panel, ssssm
    // blocking
    std::vector<int64_t> blockptr;       // Algorithm 2, n+1
    std::vector<int64_t> ptr;            // boundaries, p+1
    int32_t p = 0, samples = 0, maxb = 0;
    int32_t regular_block = 0;           // regular blocking: size used (max over members)
    std::vector<int64_t> seg;            // batch: row offsets of the members
    std::vector<int32_t> row_seg;        // batch: member of each row
    std::vector<int32_t> rowblk;         // row -> block index
    // blocks, sorted by (J, I)
    std::vector<slu::BlockDesc> blocks;
    std::vector<int64_t> bnnz;
    std::vector<int32_t> diagblk;        // I -> block id of (I, I)
    std::vector<int32_t> lcolptr;
    slu::big_vector<uint16_t> lrow;
    std::vector<int32_t> dpos, sched, sgrp;
    // strict lower part of each sparse diagonal block by rows: row r of
    // diagonal block I spans [lr_ptr[doff + I + r], lr_ptr[doff + I + r + 1])
    // of lr_col (local column, ascending) and lr_pos (slot in the block's
    // values); dense diagonal blocks have empty rows
    std::vector<int32_t> lr_ptr, lr_pos;
    std::vector<uint16_t> lr_col;
    // the strict upper part likewise by rows (ur_*), same indexing
    std::vector<int32_t> ur_ptr, ur_pos;
    std::vector<uint16_t> ur_col;
    // non-empty columns of each sparse block b: ne_col[ne_off[b] .. ne_off[b+1])
    std::vector<int64_t> ne_off;
    std::vector<uint16_t> ne_col;
    int64_t storage = 0;
    int64_t ndense = 0;
    // levels and tasks (block ids; the export calls translate to (I, J))
    std::vector<int32_t> level;
    int32_t nlevels = 0;
    std::vector<int64_t> getrf_off, gessm_off, tstrf_off, tgt_off;
    std::vector<int32_t> getrf;          // diag block ids
    // execution split of each level's GETRF list: dense-stored diagonal
    // blocks [gd_off[lv], gd_off[lv+1]) of gd, sparse ones likewise in gs
    std::vector<int64_t> gd_off, gs_off;
    std::vector<int32_t> gd, gs;
    // solve split of each level's diagonal blocks, as positions in the
    // GETRF list: with explicit inverses (dv) and without (dn)
    std::vector<int64_t> dv_off, dn_off;
    std::vector<int32_t> dv_pos, dn_pos;
    slu::big_vector<int32_t> gessm;      // pairs (blk(I,J), blk(I,I))
    slu::big_vector<int32_t> tstrf;      // pairs (blk(J,I), blk(I,I))
    slu::big_vector<int32_t> tgt;        // target block ids
    slu::big_vector<int64_t> srcoff;     // per target, into src pairs
    slu::big_vector<int32_t> src;        // pairs (blk(K,I), blk(I,J))
    // execution split of SSSSM per level: dense tiles (dense target, dense
    // sources) and the generic remainder
    std::vector<int64_t> gm_off;         // per level, into gm_task
    slu::big_vector<int32_t> gm_task;    // 5 per tile: tgt, s0, s1, r0, c0
    slu::big_vector<int32_t> gm_src;     // pairs (blk(K,I), blk(I,J))
    // FP64 plans: per tile and source pair a mask of the live 16-deep
    // slices (bit s: columns 16 s .. 16 s + 15 of block I can contribute);
    // the masks of task t start at gm_moff[t] (empty for FP32 plans)
    slu::big_vector<uint32_t> gm_mask;
    std::vector<int64_t> gm_moff;
    std::vector<int64_t> gg_off;         // per level, into gg_tgt
    slu::big_vector<int32_t> gg_tgt;
    std::vector<int64_t> gg_srcoff;
    slu::big_vector<int32_t> gg_src;
    // per level, the first gm / gg entry of the deferred part: targets whose
    // block row and column both lie beyond the next level (they may run
    // while the next level factors its diagonal blocks and panels)
    std::vector<int64_t> gm_mid, gg_mid;
    // GESSM / TSTRF tasks whose diagonal block is stored sparse, per level:
    // 3 ints (0 GESSM / 1 TSTRF, panel block, diagonal block)
    std::vector<int64_t> ps_off;
    std::vector<int32_t> ps_task;
    // the dense-panel subset of those, split into chunks of vectors (one
    // warp each): 4 ints (0 GESSM / 1 TSTRF, panel block, diagonal block,
    // first vector)
    std::vector<int64_t> pv_off;
    std::vector<int32_t> pv_task;
    // dense diagonal blocks: explicit inverses of L_II and U_II live in a
    // per-handle workspace at woff[I] (L^-1 then U^-1, b x b column-major
    // each); -1 for sparse diagonal blocks
    std::vector<int64_t> woff;
    int64_t wsize = 0;
    int32_t inv_maxb = 0;                // largest block on the inverse path
    std::vector<int64_t> inv_off;        // per level, into inv_task
    std::vector<int32_t> inv_task;       // 3 per task: diag blk, L(0)/U(1), j0
    // panel split: dense pairs as 64-wide chunks of inverse GEMMs, the
    // rest for the generic kernel
    std::vector<int64_t> pd_off;         // per level, into pd_task
    std::vector<int32_t> pd_task;        // 4 per task: 0 GESSM / 1 TSTRF, blk, diag, c0
    std::vector<int64_t> pg_off;         // per level: GESSM count prefix
    std::vector<int32_t> pg_gessm, pg_tstrf;
    std::vector<int64_t> pg_goff, pg_toff;
    // solve pull pairs, per sweep (0 L fwd, 1 U bwd, 2 U^T fwd, 3 L^T bwd):
    // per level the (source block, diagonal block) pairs, each with the
    // offset (doubles, per right-hand side chunk) of its partial vector,
    // and for every entry of the getrf list its first pair
    std::vector<int64_t> sp_off[4];
    std::vector<int32_t> sp_pairs[4];
    std::vector<int64_t> sp_poff[4];
    std::vector<int64_t> sd_pair0[4];
    int64_t part_elems = 0;              // per right-hand side
    // per diagonal block I: neighbour block lists for the solves
    std::vector<int64_t> lrow_off, urow_off, ucol_off, lcol_off;
    std::vector<int32_t> lrow_blk;       // (I, I'), I' < I
    std::vector<int32_t> urow_blk;       // (I, J),  J > I
    std::vector<int32_t> ucol_blk;       // (I', I), I' < I
    std::vector<int32_t> lcol_blk;       // (K, I),  K > I
    // value maps
    slu::big_vector<int64_t> a2s;        // A entry -> storage slot
    slu::big_vector<int64_t> f2s;        // filled entry -> storage slot
    // device mirror (lazily uploaded)
    slu::DevPlan *dev = nullptr;
};

namespace slu {
void set_error(const std::string &msg);
slu_status fail(slu_status st, const std::string &msg);
void free_dev_plan(slu_plan *plan);

// Device analysis (symbolic.cu) of a checked pattern (CSC, host arrays,
// rows in any order; `seg` its diagonal segments): sets P.nnz_sym,
// P.f_colptr, P.f_rowidx and P.blockptr exactly as the host analysis does
// and, when `irregular`, seg_ptr[q] = Algorithm 3's boundaries of segment q
// (local rows, empty for an empty segment).  Work runs on the current
// device, enqueued on `stream` (a cudaStream_t); returns after it finished.
struct DeviceSymbolicTimes {
    double symbolic_ms = 0;     // pattern, tree, struct L, filled pattern
    double blocking_ms = 0;     // Algorithm 2, sampling, Algorithm 3
    int64_t sweeps = 0;         // relaxation sweeps of the elimination tree
    int64_t samples = 0;        // largest S over the segments
};
slu_status device_symbolic(int64_t n, const int64_t *colptr, const int32_t *rowidx,
                           const std::vector<int64_t> &seg, const slu_opts &o,
                           bool irregular, void *stream, slu_plan &P,
                           std::vector<std::vector<int64_t>> &seg_ptr,
                           DeviceSymbolicTimes &tm);
}  // namespace slu
