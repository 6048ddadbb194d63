// Plan invariants (slu_plan_check): indices in range and the execution
// splits complete.
#include <algorithm>
#include <array>
#include <cstdint>
#include <exception>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "slu_internal.hpp"

using namespace slu;

// Plan invariants: every index the factorization and the solves take from a
// plan addresses an element of the array or block it names, every offset
// array is nondecreasing and ends at its array's length, and every task pair
// relates the blocks its kernel expects (linear in the plan's size); then
// the execution splits are complete (coverage_violation, N log N).  The
// analysis establishes these by construction; the check guards plans loaded
// from bytes and the analysis itself in the tests.

namespace slu {
namespace {

template <class V, class A>
bool offsets(const std::vector<V, A> &v, size_t size, int64_t last) {
    if (v.size() != size || (size && (v.front() != 0 || (int64_t)v.back() != last)))
        return false;
    for (size_t i = 1; i < v.size(); ++i)
        if (v[i] < v[i - 1]) return false;
    return true;
}

std::string plan_violation(const slu_plan &P) {
#define REQ(c, what)                  \
    do {                              \
        if (!(c)) return (what);      \
    } while (0)
    const int64_t n = P.n, p = P.p, nb = (int64_t)P.blocks.size();
    const int64_t L = P.nlevels;
    const std::vector<BlockDesc> &B = P.blocks;
    auto blk = [&](int64_t b) { return b >= 0 && b < nb; };
    REQ(n >= 0 && p >= 0 && p <= n && (n == 0) == (p == 0), "block count");
    // input pattern, its column of every entry and its CSR view
    REQ(P.nnz_a >= 0 && offsets(P.a_colptr, (size_t)n + 1, P.nnz_a), "A column pointers");
    REQ((int64_t)P.a_rowidx.size() == P.nnz_a && (int64_t)P.a_ci.size() == P.nnz_a,
        "A index arrays");
    for (int64_t j = 0; j < n; ++j)
        for (int64_t q = P.a_colptr[j]; q < P.a_colptr[j + 1]; ++q)
            REQ(P.a_rowidx[q] >= 0 && P.a_rowidx[q] < n && P.a_ci[q] == j, "A entries");
    REQ(offsets(P.a_rowptr, (size_t)n + 1, P.nnz_a) &&
            (int64_t)P.a_colidx.size() == P.nnz_a && (int64_t)P.a_vpos.size() == P.nnz_a,
        "A row view arrays");
    for (int64_t r = 0; r < n; ++r)
        for (int64_t t = P.a_rowptr[r]; t < P.a_rowptr[r + 1]; ++t) {
            const int64_t q = P.a_vpos[t];
            REQ(q >= 0 && q < P.nnz_a && P.a_rowidx[q] == r && P.a_ci[q] == P.a_colidx[t],
                "A row view entries");
        }
    // filled pattern and Algorithm 2's pointer
    REQ(P.f_colptr.size() == (size_t)n + 1 && offsets(P.f_colptr, (size_t)n + 1, P.f_colptr.back()),
        "filled column pointers");
    const int64_t nnz_lu = P.f_colptr[n];
    REQ((int64_t)P.f_rowidx.size() == nnz_lu, "filled row indices");
    for (int32_t r : P.f_rowidx) REQ(r >= 0 && r < n, "filled row index");
    REQ(P.blockptr.size() == (size_t)n + 1, "diagonal block pointer");
    // boundaries, rows -> blocks, batch members
    REQ(P.ptr.size() == (size_t)p + 1 && P.ptr.front() == 0 && P.ptr.back() == n,
        "block boundaries");
    int64_t maxb = 0;
    for (int64_t I = 0; I < p; ++I) {
        const int64_t w = P.ptr[I + 1] - P.ptr[I];
        REQ(w >= 1 && w <= 65535, "block width");
        maxb = std::max(maxb, w);
    }
    REQ(maxb == P.maxb, "largest block");
    REQ(P.rowblk.size() == (size_t)n, "row to block map");
    for (int64_t I = 0; I < p; ++I)
        for (int64_t r = P.ptr[I]; r < P.ptr[I + 1]; ++r) REQ(P.rowblk[r] == I, "row to block map");
    REQ(P.seg.size() >= 2 && offsets(P.seg, P.seg.size(), n), "batch segments");
    if (P.seg.size() > 2) {
        REQ(P.row_seg.size() == (size_t)n, "batch member of each row");
        for (int32_t s : P.row_seg) REQ(s >= 0 && s < (int64_t)P.seg.size() - 1, "batch member");
    }
    // blocks and their storage
    REQ((int64_t)P.bnnz.size() == nb && P.storage >= 0, "block counts");
    int64_t ndense = 0;
    for (int64_t b = 0; b < nb; ++b) {
        const BlockDesc &d = B[b];
        REQ(d.I >= 0 && d.I < p && d.J >= 0 && d.J < p, "block coordinates");
        REQ(d.rows == P.ptr[d.I + 1] - P.ptr[d.I] && d.cols == P.ptr[d.J + 1] - P.ptr[d.J] &&
                d.r0 == P.ptr[d.I] && d.c0 == P.ptr[d.J],
            "block extent");
        if (b) REQ(B[b - 1].J < d.J || (B[b - 1].J == d.J && B[b - 1].I < d.I), "block order");
        REQ(d.voff >= 0 && d.voff % 4 == 0 && (d.dense == 0 || d.dense == 1), "block slot");
        const int64_t cnt = P.bnnz[b];
        REQ(cnt >= 1 && cnt <= (int64_t)d.rows * d.cols, "block entry count");
        if (d.dense) {
            ++ndense;
            REQ(d.ld == d.rows && d.voff + (int64_t)d.rows * d.cols <= P.storage, "dense block storage");
        } else {
            REQ(d.coff >= 0 && (size_t)d.coff + d.cols + 1 <= P.lcolptr.size() && d.roff >= 0 &&
                    (size_t)(d.roff + cnt) <= P.lrow.size() && d.voff + cnt <= P.storage,
                "sparse block storage");
            REQ(P.lcolptr[d.coff] == 0 && P.lcolptr[d.coff + d.cols] == cnt, "sparse block columns");
            for (int32_t jj = 0; jj < d.cols; ++jj) {
                const int32_t s = P.lcolptr[d.coff + jj], e = P.lcolptr[d.coff + jj + 1];
                REQ(s <= e, "sparse block column pointers");
                for (int32_t t = s; t < e; ++t) {
                    const int32_t r = P.lrow[d.roff + t];
                    REQ(r < d.rows && (t == s || P.lrow[d.roff + t - 1] < r), "sparse block rows");
                }
            }
        }
    }
    REQ(ndense == P.ndense, "dense block count");
    // diagonal blocks: slots, column schedule, height groups, row lists
    REQ(P.diagblk.size() == (size_t)p, "diagonal block ids");
    REQ(P.lr_ptr.size() == P.dpos.size() + (size_t)p + 1 && P.ur_ptr.size() == P.lr_ptr.size() &&
            P.sched.size() == P.dpos.size() && P.lr_col.size() == P.lr_pos.size() &&
            P.ur_col.size() == P.ur_pos.size(),
        "diagonal slot arrays");
    std::vector<char> seen;
    for (int64_t I = 0; I < p; ++I) {
        const int32_t db = P.diagblk[I];
        REQ(blk(db) && B[db].I == I && B[db].J == I, "diagonal block id");
        const BlockDesc &d = B[db];
        const int32_t m = d.rows;
        REQ(d.doff >= 0 && (size_t)d.doff + m <= P.dpos.size() && d.goff >= 0 &&
                d.ngroups >= 1 && (size_t)d.goff + d.ngroups + 1 <= P.sgrp.size(),
            "diagonal block slots");
        REQ(P.sgrp[d.goff] == 0 && P.sgrp[d.goff + d.ngroups] == m, "height groups");
        for (int32_t g = 0; g < d.ngroups; ++g)
            REQ(P.sgrp[d.goff + g] < P.sgrp[d.goff + g + 1], "height groups");
        seen.assign(m, 0);
        for (int32_t t = 0; t < m; ++t) {
            const int32_t c = P.sched[d.doff + t];
            REQ(c >= 0 && c < m && !seen[c], "column schedule");
            seen[c] = 1;
        }
        for (int32_t jj = 0; jj < m; ++jj) {
            const int32_t dp = P.dpos[d.doff + jj];
            if (d.dense) {
                REQ(dp == jj, "diagonal position");
            } else {
                const int32_t s = P.lcolptr[d.coff + jj], e = P.lcolptr[d.coff + jj + 1];
                REQ(dp >= 0 && s + dp < e && P.lrow[d.roff + s + dp] == jj, "diagonal position");
            }
        }
        for (int upper = 0; upper < 2; ++upper) {
            const std::vector<int32_t> &rp = upper ? P.ur_ptr : P.lr_ptr;
            const std::vector<uint16_t> &rc = upper ? P.ur_col : P.lr_col;
            const std::vector<int32_t> &rq = upper ? P.ur_pos : P.lr_pos;
            const int64_t base = d.doff + I;
            REQ(rp[base + m] <= (int64_t)rc.size(), "diagonal row lists");
            for (int32_t r = 0; r < m; ++r) {
                REQ(rp[base + r] <= rp[base + r + 1] && rp[base + r] >= 0, "diagonal row lists");
                for (int32_t q = rp[base + r]; q < rp[base + r + 1]; ++q)
                    REQ(!d.dense && rc[q] < m && rq[q] >= 0 && rq[q] < P.bnnz[db],
                        "diagonal row list entry");
            }
        }
    }
    // non-empty columns of the sparse blocks
    REQ(offsets(P.ne_off, (size_t)nb + 1, (int64_t)P.ne_col.size()), "non-empty column offsets");
    for (int64_t b = 0; b < nb; ++b)
        for (int64_t q = P.ne_off[b]; q < P.ne_off[b + 1]; ++q)
            REQ(!B[b].dense && P.ne_col[q] < B[b].cols, "non-empty column");
    // value maps
    REQ((int64_t)P.f2s.size() == nnz_lu && (int64_t)P.a2s.size() == P.nnz_a, "value maps");
    for (int64_t s : P.f2s) REQ(s >= 0 && s < P.storage, "filled entry slot");
    for (int64_t s : P.a2s) REQ(s >= 0 && s < P.storage, "A entry slot");
    // levels and the task lists of Algorithm 1
    REQ(P.level.size() == (size_t)p && L >= 0 && (L == 0) == (p == 0), "levels");
    for (int32_t lv : P.level) REQ(lv >= 0 && lv < L, "level");
    REQ(offsets(P.getrf_off, (size_t)L + 1, (int64_t)P.getrf.size()) &&
            offsets(P.gessm_off, (size_t)L + 1, (int64_t)P.gessm.size() / 2) &&
            offsets(P.tstrf_off, (size_t)L + 1, (int64_t)P.tstrf.size() / 2) &&
            offsets(P.tgt_off, (size_t)L + 1, (int64_t)P.tgt.size()) &&
            P.gessm.size() % 2 == 0 && P.tstrf.size() % 2 == 0 && P.src.size() % 2 == 0 &&
            offsets(P.srcoff, P.tgt.size() + 1, (int64_t)P.src.size() / 2),
        "task offsets");
    auto is_diag = [&](int64_t b) { return blk(b) && B[b].I == B[b].J; };
    // panel pair (tb, db): GESSM U_IJ (type 0) or TSTRF L_JI (type 1)
    auto panel = [&](int type, int64_t tb, int64_t db) {
        if (!blk(tb) || !is_diag(db)) return false;
        const int32_t I = B[db].I;
        return type == 0 ? (B[tb].I == I && B[tb].J > I) : (B[tb].J == I && B[tb].I > I);
    };
    // Schur source pair (lb, ub) for target tb: L_KI and U_IJ
    auto source = [&](int64_t tb, int64_t lb, int64_t ub) {
        return blk(lb) && blk(ub) && B[lb].I == B[tb].I && B[ub].J == B[tb].J &&
               B[lb].J == B[ub].I && B[lb].J < std::min(B[tb].I, B[tb].J);
    };
    for (int64_t lv = 0; lv < L; ++lv) {
        for (int64_t g = P.getrf_off[lv]; g < P.getrf_off[lv + 1]; ++g)
            REQ(is_diag(P.getrf[g]) && P.level[B[P.getrf[g]].I] == lv, "GETRF task");
        for (int64_t e = P.gessm_off[lv]; e < P.gessm_off[lv + 1]; ++e)
            REQ(panel(0, P.gessm[2 * e], P.gessm[2 * e + 1]), "GESSM task");
        for (int64_t e = P.tstrf_off[lv]; e < P.tstrf_off[lv + 1]; ++e)
            REQ(panel(1, P.tstrf[2 * e], P.tstrf[2 * e + 1]), "TSTRF task");
    }
    for (size_t k = 0; k < P.tgt.size(); ++k) {
        REQ(blk(P.tgt[k]), "SSSSM target");
        for (int64_t q = P.srcoff[k]; q < P.srcoff[k + 1]; ++q)
            REQ(source(P.tgt[k], P.src[2 * q], P.src[2 * q + 1]), "SSSSM source");
    }
    // execution splits
    REQ(offsets(P.gd_off, (size_t)L + 1, (int64_t)P.gd.size()) &&
            offsets(P.gs_off, (size_t)L + 1, (int64_t)P.gs.size()) &&
            offsets(P.dv_off, (size_t)L + 1, (int64_t)P.dv_pos.size()) &&
            offsets(P.dn_off, (size_t)L + 1, (int64_t)P.dn_pos.size()),
        "GETRF split offsets");
    for (int32_t b : P.gd) REQ(is_diag(b) && B[b].dense, "dense GETRF task");
    for (int32_t b : P.gs) REQ(is_diag(b) && !B[b].dense, "sparse GETRF task");
    for (int64_t lv = 0; lv < L; ++lv) {
        for (int64_t q = P.dv_off[lv]; q < P.dv_off[lv + 1]; ++q)
            REQ(P.dv_pos[q] >= P.getrf_off[lv] && P.dv_pos[q] < P.getrf_off[lv + 1], "solve split");
        for (int64_t q = P.dn_off[lv]; q < P.dn_off[lv + 1]; ++q)
            REQ(P.dn_pos[q] >= P.getrf_off[lv] && P.dn_pos[q] < P.getrf_off[lv + 1], "solve split");
    }
    REQ(P.gm_task.size() % 5 == 0 && P.gm_src.size() % 2 == 0 && P.gg_src.size() % 2 == 0 &&
            offsets(P.gm_off, (size_t)L + 1, (int64_t)P.gm_task.size() / 5) &&
            offsets(P.gg_off, (size_t)L + 1, (int64_t)P.gg_tgt.size()) &&
            offsets(P.gg_srcoff, P.gg_tgt.size() + 1, (int64_t)P.gg_src.size() / 2) &&
            P.gm_mid.size() == (size_t)L && P.gg_mid.size() == (size_t)L,
        "SSSSM split offsets");
    for (int64_t lv = 0; lv < L; ++lv)
        REQ(P.gm_mid[lv] >= P.gm_off[lv] && P.gm_mid[lv] <= P.gm_off[lv + 1] &&
                P.gg_mid[lv] >= P.gg_off[lv] && P.gg_mid[lv] <= P.gg_off[lv + 1],
            "deferred SSSSM split");
    for (size_t t = 0; t < P.gm_task.size(); t += 5) {
        const int32_t tb = P.gm_task[t], s0 = P.gm_task[t + 1], s1 = P.gm_task[t + 2];
        const int32_t r0 = P.gm_task[t + 3], c0 = P.gm_task[t + 4];
        REQ(blk(tb) && B[tb].dense && s0 >= 0 && s0 < s1 &&
                (size_t)s1 <= P.gm_src.size() / 2 && r0 >= 0 && r0 < B[tb].rows && c0 >= 0 &&
                c0 < B[tb].cols,
            "dense SSSSM tile");
        for (int32_t q = s0; q < s1; ++q) {
            const int32_t lb = P.gm_src[2 * q], ub = P.gm_src[2 * q + 1];
            REQ(source(tb, lb, ub) && B[lb].dense && B[ub].dense, "dense SSSSM source");
        }
    }
    // slice masks: none, or one per source pair of every dense tile
    if (!P.gm_moff.empty() || !P.gm_mask.empty()) {
        REQ(offsets(P.gm_moff, P.gm_task.size() / 5 + 1, (int64_t)P.gm_mask.size()),
            "slice mask offsets");
        for (size_t t = 0; t < P.gm_task.size(); t += 5)
            REQ(P.gm_moff[t / 5 + 1] - P.gm_moff[t / 5] == P.gm_task[t + 2] - P.gm_task[t + 1],
                "slice masks per tile");
    }
    for (size_t k = 0; k < P.gg_tgt.size(); ++k) {
        REQ(blk(P.gg_tgt[k]), "generic SSSSM target");
        for (int64_t q = P.gg_srcoff[k]; q < P.gg_srcoff[k + 1]; ++q)
            REQ(source(P.gg_tgt[k], P.gg_src[2 * q], P.gg_src[2 * q + 1]), "generic SSSSM source");
    }
    // inverses and the panel kernels
    REQ(P.woff.size() == (size_t)p && P.wsize >= 0, "inverse slots");
    for (int64_t I = 0; I < p; ++I)
        if (P.woff[I] >= 0) {
            const BlockDesc &d = B[P.diagblk[I]];
            REQ(d.dense && d.rows <= P.inv_maxb &&
                    P.woff[I] + 2 * (int64_t)d.rows * d.rows <= P.wsize,
                "inverse slot");
        }
    auto has_inv = [&](int64_t db) { return is_diag(db) && P.woff[B[db].I] >= 0; };
    const int esz = P.opts.precision == SLU_PREC_FP64 ? 8 : 4;
    REQ(P.inv_task.size() % 3 == 0 && P.pd_task.size() % 4 == 0 && P.pv_task.size() % 4 == 0 &&
            P.ps_task.size() % 3 == 0 && P.pg_gessm.size() % 2 == 0 && P.pg_tstrf.size() % 2 == 0 &&
            offsets(P.inv_off, (size_t)L + 1, (int64_t)P.inv_task.size() / 3) &&
            offsets(P.pd_off, (size_t)L + 1, (int64_t)P.pd_task.size() / 4) &&
            offsets(P.pv_off, (size_t)L + 1, (int64_t)P.pv_task.size() / 4) &&
            offsets(P.ps_off, (size_t)L + 1, (int64_t)P.ps_task.size() / 3) &&
            offsets(P.pg_goff, (size_t)L + 1, (int64_t)P.pg_gessm.size() / 2) &&
            offsets(P.pg_toff, (size_t)L + 1, (int64_t)P.pg_tstrf.size() / 2),
        "panel split offsets");
    for (size_t t = 0; t < P.inv_task.size(); t += 3) {
        const int32_t db = P.inv_task[t], which = P.inv_task[t + 1], j0 = P.inv_task[t + 2];
        REQ(has_inv(db) && (which == 0 || which == 1) && j0 >= 0 && j0 < B[db].rows,
            "inverse task");
    }
    for (size_t t = 0; t < P.pd_task.size(); t += 4) {
        const int32_t ty = P.pd_task[t], tb = P.pd_task[t + 1], db = P.pd_task[t + 2];
        const int32_t c0 = P.pd_task[t + 3];
        REQ((ty == 0 || ty == 1) && panel(ty, tb, db) && has_inv(db) && c0 >= 0 &&
                c0 < (ty == 0 ? B[tb].cols : B[tb].rows),
            "panel task with inverse");
    }
    for (size_t t = 0; t < P.pv_task.size(); t += 4) {
        const int32_t ty = P.pv_task[t], tb = P.pv_task[t + 1], db = P.pv_task[t + 2];
        const int32_t v0 = P.pv_task[t + 3];
        const bool pair_ok = (ty == 0 || ty == 1) && panel(ty, tb, db);
        const int V = pair_ok ? panel_vec_width(B[db].rows, esz) : 0;
        REQ(pair_ok && B[tb].dense && V > 0 && v0 >= 0 && v0 % V == 0 &&
                v0 < (ty == 0 ? B[tb].cols : B[tb].rows),
            "vector panel task");
    }
    for (size_t t = 0; t < P.ps_task.size(); t += 3) {
        const int32_t ty = P.ps_task[t], tb = P.ps_task[t + 1], db = P.ps_task[t + 2];
        REQ((ty == 0 || ty == 1) && panel(ty, tb, db) && !B[db].dense, "sparse panel task");
    }
    for (size_t t = 0; t < P.pg_gessm.size(); t += 2)
        REQ(panel(0, P.pg_gessm[t], P.pg_gessm[t + 1]), "generic GESSM task");
    for (size_t t = 0; t < P.pg_tstrf.size(); t += 2)
        REQ(panel(1, P.pg_tstrf[t], P.pg_tstrf[t + 1]), "generic TSTRF task");
    // block lists by row and column (the solves' sources)
    const std::vector<int64_t> *offs[4] = {&P.lrow_off, &P.urow_off, &P.ucol_off, &P.lcol_off};
    const std::vector<int32_t> *ids[4] = {&P.lrow_blk, &P.urow_blk, &P.ucol_blk, &P.lcol_blk};
    for (int k = 0; k < 4; ++k) {
        REQ(offsets(*offs[k], (size_t)p + 1, (int64_t)ids[k]->size()), "block list offsets");
        for (int64_t I = 0; I < p; ++I)
            for (int64_t q = (*offs[k])[I]; q < (*offs[k])[I + 1]; ++q) {
                const int32_t b = (*ids[k])[q];
                const bool ok = blk(b) && (k == 0   ? B[b].I == I && B[b].J < I
                                           : k == 1 ? B[b].I == I && B[b].J > I
                                           : k == 2 ? B[b].J == I && B[b].I < I
                                                    : B[b].J == I && B[b].I > I);
                REQ(ok, "block list entry");
            }
    }
    // solve pull pairs per sweep
    for (int sw = 0; sw < 4; ++sw) {
        const std::vector<int32_t> &pr = P.sp_pairs[sw];
        REQ(pr.size() % 2 == 0 && offsets(P.sp_off[sw], (size_t)L + 1, (int64_t)pr.size() / 2) &&
                P.sp_poff[sw].size() == pr.size() / 2 && P.sd_pair0[sw].size() == P.getrf.size(),
            "solve pair offsets");
        for (size_t q = 0; q < pr.size() / 2; ++q) {
            const int32_t b = pr[2 * q], db = pr[2 * q + 1];
            REQ(blk(b) && is_diag(db) && P.sp_poff[sw][q] >= 0 &&
                    P.sp_poff[sw][q] + B[db].rows <= P.part_elems,
                "solve pair");
        }
        for (size_t g = 0; g < P.getrf.size(); ++g)
            REQ(P.sd_pair0[sw][g] >= 0 && (size_t)P.sd_pair0[sw][g] <= pr.size() / 2,
                "solve pair start");
    }
#undef REQ
    return std::string();
}

// Completeness of the execution splits (runs once plan_violation has found
// every index in range): per level, the dense/sparse GETRF lists and the
// solve's inverse split partition the level's GETRF list; every GESSM and
// TSTRF task is carried by exactly one panel kernel, whose chunks cover its
// vectors exactly once; every Schur source pair of the level is carried
// exactly once, by the dense tiles (which cover their target exactly once)
// or by the generic kernel, in ascending source order per target; every
// inverse-eligible diagonal block gets both inverses in row chunks covering
// it exactly once; and each sweep's pull pairs of a diagonal block are its
// block list in order.
std::string coverage_violation(const slu_plan &P) {
#define REQ(c, what)                  \
    do {                              \
        if (!(c)) return (what);      \
    } while (0)
    const int64_t L = P.nlevels;
    const std::vector<BlockDesc> &B = P.blocks;
    const int esz = P.opts.precision == SLU_PREC_FP64 ? 8 : 4;
    const int32_t kTile = P.opts.precision == SLU_PREC_FP32 ? 128 : 64;
    auto key = [](int64_t type, int64_t a, int64_t b) {
        return ((uint64_t)type << 62) | ((uint64_t)a << 31) | (uint64_t)b;
    };
    // chunk starts 0, step, 2 step, ... below `extent`, each exactly once
    auto covers = [](std::vector<int32_t> &starts, int32_t step, int32_t extent) {
        std::sort(starts.begin(), starts.end());
        if ((int64_t)starts.size() != (extent + step - 1) / step) return false;
        for (size_t i = 0; i < starts.size(); ++i)
            if (starts[i] != (int32_t)i * step) return false;
        return true;
    };
    for (int64_t lv = 0; lv < L; ++lv) {
        const int64_t g0 = P.getrf_off[lv], g1 = P.getrf_off[lv + 1];
        // GETRF: dense + sparse lists, and the solve split by positions
        std::vector<int32_t> want(P.getrf.begin() + g0, P.getrf.begin() + g1), got;
        got.insert(got.end(), P.gd.begin() + P.gd_off[lv], P.gd.begin() + P.gd_off[lv + 1]);
        got.insert(got.end(), P.gs.begin() + P.gs_off[lv], P.gs.begin() + P.gs_off[lv + 1]);
        std::sort(want.begin(), want.end());
        std::sort(got.begin(), got.end());
        REQ(got == want, "GETRF split");
        std::vector<int32_t> pos(P.dv_pos.begin() + P.dv_off[lv], P.dv_pos.begin() + P.dv_off[lv + 1]);
        pos.insert(pos.end(), P.dn_pos.begin() + P.dn_off[lv], P.dn_pos.begin() + P.dn_off[lv + 1]);
        std::sort(pos.begin(), pos.end());
        REQ((int64_t)pos.size() == g1 - g0, "solve split");
        for (size_t i = 0; i < pos.size(); ++i) REQ(pos[i] == g0 + (int64_t)i, "solve split");
        for (int64_t q = P.dv_off[lv]; q < P.dv_off[lv + 1]; ++q)
            REQ(P.woff[B[P.getrf[P.dv_pos[q]]].I] >= 0, "solve split");
        for (int64_t q = P.dn_off[lv]; q < P.dn_off[lv + 1]; ++q)
            REQ(P.woff[B[P.getrf[P.dn_pos[q]]].I] < 0, "solve split");
        // inverses: both triangles of every eligible block, 8-row chunks
        std::map<uint64_t, std::vector<int32_t>> inv;
        for (int64_t t = P.inv_off[lv]; t < P.inv_off[lv + 1]; ++t)
            inv[key(P.inv_task[3 * t + 1], P.inv_task[3 * t], 0)].push_back(P.inv_task[3 * t + 2]);
        size_t ninv = 0;
        for (int64_t g = g0; g < g1; ++g) {
            const int32_t db = P.getrf[g];
            if (P.woff[B[db].I] < 0) continue;
            for (int which = 0; which < 2; ++which) {
                auto it = inv.find(key(which, db, 0));
                REQ(it != inv.end() && covers(it->second, 8, B[db].rows), "inverse chunks");
                ++ninv;
            }
        }
        REQ(ninv == inv.size(), "inverse task of another level");
        // panels: each task in exactly one kernel, its vectors covered once
        std::map<uint64_t, std::vector<int32_t>> pd, pv;
        std::map<uint64_t, int> ps, pg;
        for (int64_t t = P.pd_off[lv]; t < P.pd_off[lv + 1]; ++t)
            pd[key(P.pd_task[4 * t], P.pd_task[4 * t + 1], P.pd_task[4 * t + 2])]
                .push_back(P.pd_task[4 * t + 3]);
        for (int64_t t = P.pv_off[lv]; t < P.pv_off[lv + 1]; ++t)
            pv[key(P.pv_task[4 * t], P.pv_task[4 * t + 1], P.pv_task[4 * t + 2])]
                .push_back(P.pv_task[4 * t + 3]);
        for (int64_t t = P.ps_off[lv]; t < P.ps_off[lv + 1]; ++t)
            ++ps[key(P.ps_task[3 * t], P.ps_task[3 * t + 1], P.ps_task[3 * t + 2])];
        for (int64_t t = P.pg_goff[lv]; t < P.pg_goff[lv + 1]; ++t)
            ++pg[key(0, P.pg_gessm[2 * t], P.pg_gessm[2 * t + 1])];
        for (int64_t t = P.pg_toff[lv]; t < P.pg_toff[lv + 1]; ++t)
            ++pg[key(1, P.pg_tstrf[2 * t], P.pg_tstrf[2 * t + 1])];
        size_t npanel = 0;
        for (int type = 0; type < 2; ++type) {
            const auto &task = type == 0 ? P.gessm : P.tstrf;
            const std::vector<int64_t> &off = type == 0 ? P.gessm_off : P.tstrf_off;
            for (int64_t e = off[lv]; e < off[lv + 1]; ++e) {
                const int32_t tb = task[2 * e], db = task[2 * e + 1];
                const uint64_t k = key(type, tb, db);
                const int32_t nvec = type == 0 ? B[tb].cols : B[tb].rows;
                const auto a = pd.find(k), b = pv.find(k);
                const int kinds = (a != pd.end()) + (b != pv.end()) + (int)ps.count(k) +
                                  (int)pg.count(k);
                REQ(kinds == 1, "panel task carried by one kernel");
                if (a != pd.end()) REQ(covers(a->second, 64, nvec), "panel chunks");
                if (b != pv.end())
                    REQ(covers(b->second, panel_vec_width(B[db].rows, esz), nvec), "panel vectors");
                if (ps.count(k)) REQ(ps[k] == 1, "sparse panel task repeated");
                if (pg.count(k)) REQ(pg[k] == 1, "generic panel task repeated");
                ++npanel;
            }
        }
        REQ(npanel == pd.size() + pv.size() + ps.size() + pg.size(), "panel task of another level");
        // Schur updates: every source pair once, dense tiles covering targets
        std::vector<std::array<int32_t, 3>> wantp, gotp;
        for (int64_t k = P.tgt_off[lv]; k < P.tgt_off[lv + 1]; ++k)
            for (int64_t q = P.srcoff[k]; q < P.srcoff[k + 1]; ++q)
                wantp.push_back({P.tgt[k], P.src[2 * q], P.src[2 * q + 1]});
        auto ascending = [&](const auto &sr, int64_t q0, int64_t q1) {
            for (int64_t q = q0 + 1; q < q1; ++q)
                if (B[sr[2 * q]].J <= B[sr[2 * q - 2]].J) return false;
            return true;
        };
        std::map<std::array<int32_t, 3>, std::vector<std::pair<int32_t, int32_t>>> tiles;
        for (int64_t t = P.gm_off[lv]; t < P.gm_off[lv + 1]; ++t)
            tiles[{P.gm_task[5 * t], P.gm_task[5 * t + 1], P.gm_task[5 * t + 2]}].push_back(
                {P.gm_task[5 * t + 3], P.gm_task[5 * t + 4]});
        std::map<int32_t, int> dense_tgt;
        for (auto &e : tiles) {
            const int32_t tb = e.first[0], s0 = e.first[1], s1 = e.first[2];
            REQ(++dense_tgt[tb] == 1, "dense target split over source ranges");
            REQ(ascending(P.gm_src, s0, s1), "dense sources out of order");
            for (int32_t q = s0; q < s1; ++q) gotp.push_back({tb, P.gm_src[2 * q], P.gm_src[2 * q + 1]});
            std::vector<std::pair<int32_t, int32_t>> &rc = e.second;
            std::sort(rc.begin(), rc.end());
            const int32_t nr = (B[tb].rows + kTile - 1) / kTile, nc = (B[tb].cols + 63) / 64;
            REQ((int64_t)rc.size() == (int64_t)nr * nc, "dense tiles of a target");
            for (int32_t i = 0; i < nr; ++i)
                for (int32_t j = 0; j < nc; ++j)
                    REQ(rc[(size_t)i * nc + j] == std::make_pair(i * kTile, j * 64),
                        "dense tiles of a target");
        }
        std::map<int32_t, int> generic_tgt;
        for (int64_t k = P.gg_off[lv]; k < P.gg_off[lv + 1]; ++k) {
            REQ(++generic_tgt[P.gg_tgt[k]] == 1, "generic target repeated");
            REQ(ascending(P.gg_src, P.gg_srcoff[k], P.gg_srcoff[k + 1]), "generic sources out of order");
            for (int64_t q = P.gg_srcoff[k]; q < P.gg_srcoff[k + 1]; ++q)
                gotp.push_back({P.gg_tgt[k], P.gg_src[2 * q], P.gg_src[2 * q + 1]});
        }
        std::sort(wantp.begin(), wantp.end());
        std::sort(gotp.begin(), gotp.end());
        REQ(gotp == wantp, "Schur source pairs of the level");
        // solve pulls: a diagonal block's pairs are its block list, in order
        const std::vector<int64_t> *offs[4] = {&P.lrow_off, &P.urow_off, &P.ucol_off, &P.lcol_off};
        const std::vector<int32_t> *ids[4] = {&P.lrow_blk, &P.urow_blk, &P.ucol_blk, &P.lcol_blk};
        for (int sw = 0; sw < 4; ++sw) {
            int64_t at = P.sp_off[sw][lv];
            for (int64_t g = g0; g < g1; ++g) {
                const int32_t db = P.getrf[g], I = B[db].I;
                REQ(P.sd_pair0[sw][g] == at, "solve pairs of a block");
                for (int64_t q = (*offs[sw])[I]; q < (*offs[sw])[I + 1]; ++q, ++at)
                    REQ(at < P.sp_off[sw][lv + 1] && P.sp_pairs[sw][2 * at] == (*ids[sw])[q] &&
                            P.sp_pairs[sw][2 * at + 1] == db,
                        "solve pairs of a block");
            }
            REQ(at == P.sp_off[sw][lv + 1], "solve pairs of a level");
        }
    }
#undef REQ
    return std::string();
}

}  // namespace
}  // namespace slu

extern "C" slu_status slu_plan_check(const slu_plan *P) {
    if (!P) return fail(SLU_ERR_INVALID_ARG, "NULL plan");
    try {
        std::string v = plan_violation(*P);
        if (v.empty()) v = coverage_violation(*P);
        if (!v.empty()) return fail(SLU_ERR_INVALID_ARG, "plan invariant violated: " + v);
    } catch (const std::exception &e) {
        return fail(SLU_ERR_OUT_OF_MEMORY, std::string("plan check: ") + e.what());
    }
    return SLU_OK;
}
