// Host analysis: pattern -> plan.
//
//   1. pattern(A + A^T) plus the full diagonal (the diagonal block pointer of
//      Section 4.2 relies on a structurally symmetric pattern);
//   2. elimination tree and symbolic factorization (the second phase named
//      in Section 1): struct L(:,j) = struct S(j+1:, j) united with the
//      structures of j's children in the elimination tree, minus j;
//   3. Algorithm 2: diagonal block pointer of the filled L+U pattern;
//   4. Section 4.3: S samples of the percentage curve and Algorithm 3, or a
//      regular blocking;
//   5. the block plan of Algorithm 1 restricted to non-empty blocks:
//      storage layout, levels of the block dependency DAG, task lists,
//      intra-block column schedules, value maps.
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <exception>
#include <new>
#include <numeric>
#include <system_error>
#include <thread>
#include <vector>

#include "slu_internal.hpp"

namespace slu {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

slu_status fail(slu_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

namespace {

// Worker threads for the host passes over the pattern: the hardware
// concurrency, or SLU_HOST_THREADS from the environment when set to a
// positive number, 16 at most, and fewer when the per-thread count arrays
// of a transpose (threads x destinations) would get large.  The plan does
// not depend on the count.
int host_threads(int64_t ndst) {
    int64_t t = std::max(1u, std::thread::hardware_concurrency());
    if (const char *e = std::getenv("SLU_HOST_THREADS")) {
        const long v = std::strtol(e, nullptr, 10);
        if (v > 0) t = v;
    }
    t = std::min<int64_t>(t, 16);
    t = std::min<int64_t>(t, std::max<int64_t>(1, ((int64_t)1 << 26) / std::max<int64_t>(ndst, 1)));
    return (int)t;
}

// Runs f(t) for t in [0, nt) on nt threads (the calling thread takes t = 0
// and every t whose thread could not be started).  Each t works on its own
// slice, so the result does not depend on which thread ran it.  An exception
// thrown by f is rethrown here after every thread has joined.
template <class F>
void run_threads(int nt, F f) {
    if (nt <= 1) {
        f(0);
        return;
    }
    std::vector<std::exception_ptr> err(nt);
    auto body = [&](int t) {
        try {
            f(t);
        } catch (...) {
            err[t] = std::current_exception();
        }
    };
    std::vector<std::thread> th;
    th.reserve(nt - 1);
    int started = 1;
    for (; started < nt; ++started) {
        try {
            th.emplace_back(body, started);
        } catch (const std::system_error &) {
            break;
        }
    }
    for (int t = started; t < nt; ++t) body(t);
    body(0);
    for (auto &x : th) x.join();
    for (auto &e : err)
        if (e) std::rethrow_exception(e);
}

// Stable transpose of a compressed pattern: source columns c in [0, nsrc)
// with entries e in [sp[c], sp[c+1]), each sent to destination dst(e) in
// [0, ndst).  A destination receives its entries in source order (c
// ascending, then e), exactly as a sequential counting sort would.
// total(d) receives each destination's count; base(d), called afterwards,
// must return the destination's first output slot; emit(slot, c, e) stores
// an entry.  Threads take contiguous source ranges balanced by entries.
template <class Dst, class Total, class Base, class Emit>
void stable_transpose(int64_t nsrc, const int64_t *sp, int64_t ndst, Dst dst,
                      Total total, Base base, Emit emit) {
    const int nt = host_threads(ndst);
    std::vector<int64_t> cut(nt + 1, nsrc);
    cut[0] = 0;
    for (int t = 1; t < nt; ++t)
        cut[t] = std::upper_bound(sp, sp + nsrc + 1, sp[nsrc] * t / nt) - sp - 1;
    for (int t = 1; t <= nt; ++t) cut[t] = std::max(cut[t], cut[t - 1]);
    std::vector<std::vector<int64_t>> cnt(nt);
    run_threads(nt, [&](int t) {
        cnt[t].assign(ndst, 0);
        for (int64_t c = cut[t]; c < cut[t + 1]; ++c)
            for (int64_t e = sp[c]; e < sp[c + 1]; ++e) cnt[t][dst(e)]++;
    });
    for (int64_t d = 0; d < ndst; ++d) {
        int64_t sum = 0;
        for (int t = 0; t < nt; ++t) sum += cnt[t][d];
        total(d, sum);
    }
    for (int64_t d = 0; d < ndst; ++d) {       // counts become start slots
        int64_t at = base(d);
        for (int t = 0; t < nt; ++t) {
            const int64_t c = cnt[t][d];
            cnt[t][d] = at;
            at += c;
        }
    }
    run_threads(nt, [&](int t) {
        std::vector<int64_t> &f = cnt[t];
        for (int64_t c = cut[t]; c < cut[t + 1]; ++c)
            for (int64_t e = sp[c]; e < sp[c + 1]; ++e) emit(f[dst(e)]++, c, e);
    });
}

// Cuts 0 = c_0 <= c_1 <= ... <= c_nt = nsrc of a range of columns whose
// entry prefix is w(c) (nondecreasing, w(0) = 0): part t, columns
// [c_t, c_{t+1}), holds about w(nsrc) / nt entries.
template <class W>
std::vector<int64_t> balanced_cuts(int64_t nsrc, W w, int nt) {
    std::vector<int64_t> cut(nt + 1, nsrc);
    cut[0] = 0;
    const int64_t tot = w(nsrc);
    for (int t = 1; t < nt; ++t) {
        const int64_t goal = tot / nt * t + tot % nt * t / nt;
        int64_t lo = 0, hi = nsrc;                 // last c with w(c) <= goal
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo + 1) / 2;
            if (w(mid) <= goal) lo = mid;
            else hi = mid - 1;
        }
        cut[t] = std::max(lo, cut[t - 1]);
    }
    return cut;
}

struct Sym {                      // symmetric pattern with diagonal
    std::vector<int64_t> p;
    std::vector<int32_t> i;
};

// pattern(A + A^T) plus the full diagonal, every column sorted.  Inputs:
// A's columns with rows ascending (ap, ai) and A's rows with columns
// ascending (rp, rc, the CSR view); column j of the result is the union of
// A(:, j), A(j, :) and {j}, merged without sorting.
void symmetrize(int64_t n, const int64_t *ap, const int32_t *ai,
                const int64_t *rp, const int32_t *rc, Sym &S) {
    S.p.assign(n + 1, 0);
    S.i.clear();
    S.i.reserve((size_t)(2 * ap[n] + n));
    std::vector<int32_t> t;
    for (int64_t j = 0; j < n; ++j) {
        const int32_t *a0 = ai + ap[j], *a1 = ai + ap[j + 1];
        const int32_t *r0 = rc + rp[j], *r1 = rc + rp[j + 1];
        t.resize((size_t)((a1 - a0) + (r1 - r0)));
        auto e = std::set_union(a0, a1, r0, r1, t.begin());
        t.resize((size_t)(e - t.begin()));
        // insert the diagonal in order
        auto d = std::lower_bound(t.begin(), t.end(), (int32_t)j);
        S.i.insert(S.i.end(), t.begin(), d);
        if (d == t.end() || *d != (int32_t)j) S.i.push_back((int32_t)j);
        S.i.insert(S.i.end(), d, t.end());
        S.p[j + 1] = (int64_t)S.i.size();
    }
}

// Liu's elimination tree of a symmetric pattern (upper part used), with
// path compression through the `anc` array.
void etree(int64_t n, const Sym &S, std::vector<int32_t> &parent) {
    parent.assign(n, -1);
    std::vector<int32_t> anc(n, -1);
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t q = S.p[j]; q < S.p[j + 1]; ++q) {
            int32_t r = S.i[q];
            if (r >= j) break;                  // rows sorted
            while (anc[r] != -1 && anc[r] != j) {
                const int32_t nx = anc[r];
                anc[r] = (int32_t)j;
                r = nx;
            }
            if (anc[r] == -1) {
                anc[r] = (int32_t)j;
                parent[r] = (int32_t)j;
            }
        }
    }
}

// struct L(:,j) (strictly lower, sorted): the rows > j of S(:,j) united
// with struct L(:,c) minus {j} for every child c of j.  Every list involved
// is sorted, so the union is built by merging (linear in the sizes, no
// sort).  A column needs only its children's columns, so the elimination
// tree's subtrees are independent: the subtrees hanging below the nodes
// with more than n / (8 nt) descendants go to threads whole (largest
// first, to the least loaded thread) and are built in postorder, each
// thread in a buffer of its own; the nodes above them follow on one thread
// in increasing order (children always precede their parent), and the
// columns are finally copied into Lp / Li in column order.
void symbolic(int64_t n, const Sym &S, const std::vector<int32_t> &par,
              std::vector<int64_t> &Lp, big_vector<int32_t> &Li) {
    std::vector<int64_t> chp(n + 1, 0);
    for (int64_t j = 0; j < n; ++j)
        if (par[j] >= 0) chp[par[j] + 1]++;
    for (int64_t j = 0; j < n; ++j) chp[j + 1] += chp[j];
    std::vector<int32_t> ch(chp[n]);
    {
        std::vector<int64_t> f(chp.begin(), chp.end() - 1);
        for (int64_t j = 0; j < n; ++j)
            if (par[j] >= 0) ch[f[par[j]]++] = (int32_t)j;
    }
    const int nt = host_threads(0);
    // where each column's list lives: buffer, offset, length
    std::vector<int32_t> cbuf(n);
    std::vector<int64_t> coff(n), clen(n);
    std::vector<std::vector<int32_t>> buf(nt + 1);   // buf[nt]: upper nodes
    auto build = [&](int64_t j, int b, std::vector<int32_t> &col,
                     std::vector<int32_t> &tmp) {
        col.clear();
        {
            const int32_t *lo = S.i.data() + S.p[j], *hi = S.i.data() + S.p[j + 1];
            lo = std::upper_bound(lo, hi, (int32_t)j);  // rows sorted
            col.assign(lo, hi);
        }
        for (int64_t c = chp[j]; c < chp[j + 1]; ++c) {
            const int32_t k = ch[c];
            const int32_t *kb = buf[cbuf[k]].data() + coff[k];
            const int32_t *lo = std::upper_bound(kb, kb + clen[k], (int32_t)j);
            const int32_t *hi = kb + clen[k];            // drop j itself
            if (lo == hi) continue;
            tmp.resize(col.size() + (size_t)(hi - lo));
            auto end = std::set_union(col.begin(), col.end(), lo, hi, tmp.begin());
            tmp.resize((size_t)(end - tmp.begin()));
            col.swap(tmp);
        }
        cbuf[j] = b;
        coff[j] = (int64_t)buf[b].size();
        clen[j] = (int64_t)col.size();
        buf[b].insert(buf[b].end(), col.begin(), col.end());
    };
    // subtree sizes (children precede their parent)
    std::vector<int64_t> sz(n, 1);
    for (int64_t j = 0; j < n; ++j)
        if (par[j] >= 0) sz[par[j]] += sz[j];
    const int64_t grain = std::max<int64_t>(1, n / (8 * (int64_t)nt));
    std::vector<int32_t> roots;
    for (int64_t j = 0; j < n; ++j)
        if (sz[j] <= grain && (par[j] < 0 || sz[par[j]] > grain))
            roots.push_back((int32_t)j);
    std::stable_sort(roots.begin(), roots.end(),
                     [&](int32_t a, int32_t b) { return sz[a] > sz[b]; });
    std::vector<std::vector<int32_t>> mine(nt);
    {
        std::vector<int64_t> load(nt, 0);
        for (int32_t r : roots) {
            const int t = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            mine[t].push_back(r);
            load[t] += sz[r];
        }
    }
    run_threads(nt, [&](int t) {
        std::vector<int32_t> col, tmp;
        std::vector<std::pair<int32_t, int64_t>> st;   // (node, next child)
        for (int32_t r : mine[t]) {
            st.assign(1, {r, chp[r]});
            while (!st.empty()) {
                auto &top = st.back();
                if (top.second < chp[top.first + 1]) {
                    const int32_t c = ch[top.second++];
                    st.push_back({c, chp[c]});
                } else {
                    build(top.first, t, col, tmp);
                    st.pop_back();
                }
            }
        }
    });
    {
        std::vector<int32_t> col, tmp;
        for (int64_t j = 0; j < n; ++j)
            if (sz[j] > grain) build(j, nt, col, tmp);
    }
    Lp.assign(n + 1, 0);
    for (int64_t j = 0; j < n; ++j) Lp[j + 1] = Lp[j] + clen[j];
    Li.resize(Lp[n]);
    const std::vector<int64_t> cut = balanced_cuts(
        n, [&](int64_t j) { return Lp[j]; }, nt);
    run_threads(nt, [&](int t) {
        for (int64_t j = cut[t]; j < cut[t + 1]; ++j)
            std::copy(buf[cbuf[j]].data() + coff[j],
                      buf[cbuf[j]].data() + coff[j] + clen[j], Li.data() + Lp[j]);
    });
}

int64_t idx_of(int64_t s, int64_t N, int64_t S) { return (s * N) / S; }

}  // namespace

// Algorithm 2 (Section 4.2): count, for each row, the entries left of the
// diagonal; growing the leading submatrix from i x i to (i+1) x (i+1) adds
// row i's and (by symmetry) column i's off-diagonal entries plus the
// diagonal, so blockptr[i+1] = blockptr[i] + 2 num[i] + 1.
void diagonal_block_pointer(int64_t n, const int64_t *colptr,
                            const int32_t *rowidx, int64_t *blockptr) {
    std::vector<int64_t> num(n, 0);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = colptr[i]; j < colptr[i + 1]; ++j) {
            const int64_t index = rowidx[j];
            if (index > i) num[index] += 1;
        }
    blockptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        num[i] = 2 * num[i] + 1;
        blockptr[i + 1] = blockptr[i] + num[i];
    }
}

// Section 4.3, Algorithm 3 over S samples of the percentage curve
// pct(s) = bp[idx(s)] / bp[N], idx(s) = floor(s N / S).  The threshold is
// the linear-profile slope step / S; the test
// pct(i+step) - pct(i) >= step / S is evaluated exactly as
// (bp[idx(i+step)] - bp[idx(i)]) * S >= step * bp[N].
void irregular_blocking(int64_t N, const int64_t *bp, int32_t S, int32_t step,
                        int32_t max_num, int32_t stride,
                        std::vector<int64_t> &ptr) {
    ptr.clear();
    ptr.push_back(0);
    const int64_t total = bp[N];
    int32_t l = 0;
    for (int64_t i = 0; i + step <= S; i += stride) {
        const int64_t a = bp[idx_of(i, N, S)];
        const int64_t b = bp[idx_of(i + step, N, S)];
        bool mark;
        if ((b - a) * (int64_t)S >= (int64_t)step * total) {
            mark = true;                         // dense region
        } else if (l >= max_num) {
            mark = true;                         // bound the block size
        } else {
            mark = false;
            ++l;
        }
        if (mark) {
            const int64_t pos = idx_of(i + step, N, S);
            if (pos > ptr.back()) ptr.push_back(pos);
            l = 0;
        }
    }
    if (ptr.back() < N) ptr.push_back(N);
}

}  // namespace slu

using namespace slu;

extern "C" void slu_opts_default(slu_opts *o) {
    std::memset(o, 0, sizeof(*o));
    o->blocking = SLU_BLOCKING_IRREGULAR;
    o->regular_block = 128;
    o->sample_points = 1000;
    o->step = 2;
    o->max_num = 3;
    o->stride = 1;
    o->b_min = 32;
    o->precision = SLU_PREC_FP64;
    o->dense_threshold = 0.6;
    o->pivot_perturb = 1;
    o->pivot_tau_rel = 0.0;
    o->refine_tol = 1e-14;
    o->refine_max_iter = 0;
    o->wait_budget_ms = 2000;
    o->tc_passes = 3;
}

extern "C" const char *slu_last_error(void) { return g_err.c_str(); }

static slu_status build_blocks(slu_plan &P) {
    const int64_t n = P.n;
    const int32_t p = P.p;
    P.rowblk.assign(n, 0);
    for (int32_t b = 0; b < p; ++b)
        for (int64_t r = P.ptr[b]; r < P.ptr[b + 1]; ++r) P.rowblk[r] = b;
    P.maxb = 0;
    for (int32_t b = 0; b < p; ++b)
        P.maxb = std::max<int32_t>(P.maxb, (int32_t)(P.ptr[b + 1] - P.ptr[b]));
    if (P.maxb > 65535)
        return fail(SLU_ERR_NOT_SUPPORTED, "block larger than 65535 rows");
    // Both passes below walk the filled pattern block column by block
    // column; block columns are independent, so threads take contiguous
    // ranges of them balanced by entries, and pass 1's per-thread block
    // lists are concatenated in column order.
    const int nt = host_threads(p);
    const std::vector<int64_t> cutJ = balanced_cuts(
        p, [&](int64_t J) { return P.f_colptr[P.ptr[J]]; }, nt);
    // pass 1: non-empty blocks and their counts, block column by column
    std::vector<int64_t> bcol_first(p + 1, 0);   // first block id of col J
    std::vector<std::vector<BlockDesc>> tblk(nt);
    std::vector<std::vector<int64_t>> tnnz(nt);
    run_threads(nt, [&](int t) {
        std::vector<int64_t> cnt(p, 0);
        std::vector<int32_t> touched;
        for (int32_t J = (int32_t)cutJ[t]; J < cutJ[t + 1]; ++J) {
            touched.clear();
            for (int64_t j = P.ptr[J]; j < P.ptr[J + 1]; ++j)
                for (int64_t q = P.f_colptr[j]; q < P.f_colptr[j + 1]; ++q) {
                    const int32_t I = P.rowblk[P.f_rowidx[q]];
                    if (cnt[I]++ == 0) touched.push_back(I);
                }
            std::sort(touched.begin(), touched.end());
            bcol_first[J] = (int64_t)tblk[t].size();   // local, offset below
            for (int32_t I : touched) {
                BlockDesc d;
                std::memset(&d, 0, sizeof(d));
                d.I = I;
                d.J = J;
                d.rows = (int32_t)(P.ptr[I + 1] - P.ptr[I]);
                d.cols = (int32_t)(P.ptr[J + 1] - P.ptr[J]);
                d.r0 = (int32_t)P.ptr[I];
                d.c0 = (int32_t)P.ptr[J];
                d.dense = (double)cnt[I] >= P.opts.dense_threshold *
                                                ((double)d.rows * (double)d.cols);
                d.doff = d.goff = -1;
                tblk[t].push_back(d);
                tnnz[t].push_back(cnt[I]);
                cnt[I] = 0;
            }
        }
    });
    P.blocks.clear();
    P.bnnz.clear();
    for (int t = 0; t < nt; ++t) {
        const int64_t base = (int64_t)P.blocks.size();
        for (int64_t J = cutJ[t]; J < cutJ[t + 1]; ++J) bcol_first[J] += base;
        P.blocks.insert(P.blocks.end(), tblk[t].begin(), tblk[t].end());
        P.bnnz.insert(P.bnnz.end(), tnnz[t].begin(), tnnz[t].end());
        std::vector<BlockDesc>().swap(tblk[t]);
        std::vector<int64_t>().swap(tnnz[t]);
    }
    bcol_first[p] = (int64_t)P.blocks.size();
    const int64_t nb = (int64_t)P.blocks.size();
    {
        int64_t ncol = 0;
        for (int64_t b = 0; b < nb; ++b) {
            const BlockDesc &d = P.blocks[b];
            if (d.dense) continue;
            ncol += d.cols + 1;
            // local positions inside a sparse block are 32-bit
            if (P.bnnz[b] > INT32_MAX)
                return fail(SLU_ERR_NOT_SUPPORTED,
                            "sparse block with more than 2^31 entries");
        }
        if (ncol > INT32_MAX)
            return fail(SLU_ERR_NOT_SUPPORTED, "too many sparse block columns");
    }
    // storage layout
    int64_t voff = 0, roff = 0, coff = 0, ndiag_slots = 0;
    P.ndense = 0;
    P.diagblk.assign(p, -1);
    for (int64_t b = 0; b < nb; ++b) {
        BlockDesc &d = P.blocks[b];
        d.voff = voff;
        if (d.dense) {
            d.ld = d.rows;
            d.roff = -1;
            d.coff = -1;
            voff += (int64_t)d.rows * d.cols;
            P.ndense++;
        } else {
            d.ld = 0;
            d.roff = roff;
            d.coff = (int32_t)coff;
            voff += P.bnnz[b];
            roff += P.bnnz[b];
            coff += d.cols + 1;
        }
        voff = (voff + 3) & ~int64_t(3);        // 32-byte aligned blocks
        if (d.I == d.J) {
            P.diagblk[d.I] = (int32_t)b;
            d.doff = (int32_t)ndiag_slots;
            ndiag_slots += d.rows;
        }
    }
    P.storage = voff;
    P.lcolptr.assign(coff, 0);
    P.lrow.resize(roff);                  // every slot written by pass 2
    P.f2s.resize(P.f_colptr[n]);
    P.dpos.assign(ndiag_slots, 0);
    // pass 2: local CSC, filled -> storage map, diagonal positions (each
    // block column writes only its own blocks' slots and its own entries)
    run_threads(nt, [&](int tt) {
        std::vector<int64_t> run(p, 0);             // running local position
        std::vector<int32_t> bid(p, -1);
        for (int32_t J = (int32_t)cutJ[tt]; J < cutJ[tt + 1]; ++J) {
            for (int64_t b = bcol_first[J]; b < bcol_first[J + 1]; ++b) {
                bid[P.blocks[b].I] = (int32_t)b;
                run[P.blocks[b].I] = 0;
            }
            for (int64_t j = P.ptr[J]; j < P.ptr[J + 1]; ++j) {
                const int32_t jj = (int32_t)(j - P.ptr[J]);
                for (int64_t b = bcol_first[J]; b < bcol_first[J + 1]; ++b) {
                    const BlockDesc &d = P.blocks[b];
                    if (!d.dense) P.lcolptr[d.coff + jj] = (int32_t)run[d.I];
                }
                for (int64_t q = P.f_colptr[j]; q < P.f_colptr[j + 1]; ++q) {
                    const int32_t r = P.f_rowidx[q];
                    const int32_t I = P.rowblk[r];
                    const BlockDesc &d = P.blocks[bid[I]];
                    const int32_t rl = r - d.r0;
                    int64_t t;
                    if (d.dense) {
                        t = (int64_t)jj * d.ld + rl;
                    } else {
                        t = run[I]++;
                        P.lrow[d.roff + t] = (uint16_t)rl;
                    }
                    P.f2s[q] = d.voff + t;
                    if (I == J && rl == jj)
                        P.dpos[d.doff + jj] =
                            d.dense ? rl : (int32_t)(t - P.lcolptr[d.coff + jj]);
                }
            }
            for (int64_t b = bcol_first[J]; b < bcol_first[J + 1]; ++b) {
                const BlockDesc &d = P.blocks[b];
                if (!d.dense) P.lcolptr[d.coff + d.cols] = (int32_t)run[d.I];
                bid[d.I] = -1;
            }
        }
    });
    // intra-diagonal-block column schedule: height(jj) = 1 + max height of
    // the columns m < jj with U(m, jj) stored (0 if none); a column only
    // reads columns of smaller height, so each height is one parallel group.
    P.sched.assign(ndiag_slots, 0);
    P.sgrp.clear();
    std::vector<int32_t> h, order;
    for (int32_t I = 0; I < p; ++I) {
        BlockDesc &d = P.blocks[P.diagblk[I]];
        const int32_t m = d.rows;
        h.assign(m, 0);
        int32_t hmax = 0;
        for (int32_t jj = 0; jj < m; ++jj) {
            int32_t best = -1;
            if (d.dense) {
                best = jj - 1;                  // dense: a chain
            } else {
                const int32_t s = P.lcolptr[d.coff + jj];
                const int32_t dp = P.dpos[d.doff + jj];
                for (int32_t t = 0; t < dp; ++t)
                    best = std::max(best, h[P.lrow[d.roff + s + t]]);
            }
            h[jj] = best + 1;
            hmax = std::max(hmax, h[jj]);
        }
        order.resize(m);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(),
                         [&](int32_t a, int32_t b) { return h[a] < h[b]; });
        d.goff = (int32_t)P.sgrp.size();
        d.ngroups = m ? hmax + 1 : 0;
        int32_t g = 0;
        for (int32_t t = 0; t < m; ++t) {
            P.sched[d.doff + t] = order[t];
            while (g <= h[order[t]]) {
                P.sgrp.push_back(t);
                ++g;
            }
        }
        P.sgrp.push_back(m);
    }
    // non-empty columns of the sparse blocks
    P.ne_off.assign(nb + 1, 0);
    P.ne_col.clear();
    for (int64_t b = 0; b < nb; ++b) {
        const BlockDesc &d = P.blocks[b];
        if (!d.dense)
            for (int32_t jj = 0; jj < d.cols; ++jj)
                if (P.lcolptr[d.coff + jj + 1] > P.lcolptr[d.coff + jj])
                    P.ne_col.push_back((uint16_t)jj);
        P.ne_off[b + 1] = (int64_t)P.ne_col.size();
    }
    // rows of the strict lower part of the sparse diagonal blocks
    P.lr_ptr.assign(ndiag_slots + p + 1, 0);
    P.lr_col.clear();
    P.lr_pos.clear();
    P.ur_ptr.assign(ndiag_slots + p + 1, 0);
    P.ur_col.clear();
    P.ur_pos.clear();
    for (int upper = 0; upper < 2; ++upper) {
        std::vector<int32_t> &rptr = upper ? P.ur_ptr : P.lr_ptr;
        std::vector<uint16_t> &rcol = upper ? P.ur_col : P.lr_col;
        std::vector<int32_t> &rpos = upper ? P.ur_pos : P.lr_pos;
        std::vector<int32_t> cnt;
        std::vector<int64_t> at;
        for (int32_t I = 0; I < p; ++I) {
            const BlockDesc &d = P.blocks[P.diagblk[I]];
            const int64_t base = d.doff + I;
            const int32_t m = d.rows;
            cnt.assign(m, 0);
            auto keep = [&](int32_t r, int32_t jj) { return upper ? r < jj : r > jj; };
            if (!d.dense)
                for (int32_t jj = 0; jj < m; ++jj)
                    for (int32_t t = P.lcolptr[d.coff + jj]; t < P.lcolptr[d.coff + jj + 1]; ++t)
                        if (keep(P.lrow[d.roff + t], jj)) cnt[P.lrow[d.roff + t]]++;
            const int32_t start = (int32_t)rcol.size();
            at.assign(m + 1, 0);
            for (int32_t r = 0; r < m; ++r) at[r + 1] = at[r] + cnt[r];
            for (int32_t r = 0; r <= m; ++r) rptr[base + r] = start + (int32_t)at[r];
            rcol.resize(start + at[m]);
            rpos.resize(start + at[m]);
            if (!d.dense)
                for (int32_t jj = 0; jj < m; ++jj)
                    for (int32_t t = P.lcolptr[d.coff + jj]; t < P.lcolptr[d.coff + jj + 1]; ++t) {
                        const int32_t r = P.lrow[d.roff + t];
                        if (!keep(r, jj)) continue;
                        const int64_t q = start + at[r]++;
                        rcol[q] = (uint16_t)jj;
                        rpos[q] = t;
                    }
        }
        if (rcol.size() > (size_t)INT32_MAX)
            return fail(SLU_ERR_NOT_SUPPORTED, "sparse diagonal blocks too large");
    }
    return SLU_OK;
}

// Levels: level(I) = 0 if block row I has no non-empty block left of the
// diagonal, else 1 + max level(I') over non-empty (I, I'), I' < I: the
// longest chain of the task graph of Algorithm 1 restricted to non-empty
// blocks (step I' writes into block row/column I exactly when (I, I') is
// non-empty, the pattern being symmetric).  Tasks of a level:
//   GETRF(I), GESSM(I,J) for non-empty (I,J), TSTRF(J,I) for non-empty
//   (J,I), and SSSSM into every non-empty (K,J) with (K,I) and (I,J)
//   non-empty, the sources of one target gathered in ascending I.
static void build_levels_and_tasks(slu_plan &P) {
    const int32_t p = P.p;
    const int64_t nb = (int64_t)P.blocks.size();
    std::vector<std::vector<int32_t>> lower_row(p), upper_row(p),
        lower_col(p), upper_col(p);
    for (int64_t b = 0; b < nb; ++b) {
        const BlockDesc &d = P.blocks[b];
        if (d.I > d.J) {
            lower_row[d.I].push_back((int32_t)b);
            lower_col[d.J].push_back((int32_t)b);
        } else if (d.I < d.J) {
            upper_row[d.I].push_back((int32_t)b);
            upper_col[d.J].push_back((int32_t)b);
        }
    }
    // blocks are sorted by (J, I): lower_col[J] and upper_col[J] ascend in
    // I, lower_row[I] and upper_row[I] ascend in J.
    P.level.assign(p, 0);
    int32_t maxlev = -1;
    for (int32_t I = 0; I < p; ++I) {
        int32_t best = -1;
        for (int32_t b : lower_row[I])
            best = std::max(best, P.level[P.blocks[b].J]);
        P.level[I] = best + 1;
        maxlev = std::max(maxlev, P.level[I]);
    }
    P.nlevels = maxlev + 1;
    const int32_t L = P.nlevels;
    // (K, J) -> block id (-1 if empty): a p x p table when it is small, else
    // a binary search of column J's blocks (ascending in I)
    std::vector<int32_t> table;
    if ((int64_t)p * p <= ((int64_t)1 << 24)) {
        table.assign((size_t)p * p, -1);
        for (int64_t b = 0; b < nb; ++b)
            table[(size_t)P.blocks[b].I * p + P.blocks[b].J] = (int32_t)b;
    }
    auto find = [&](int32_t K, int32_t J) -> int32_t {
        if (!table.empty()) return table[(size_t)K * p + J];
        if (K == J) return P.diagblk[J];
        const auto &w = (K > J) ? lower_col[J] : upper_col[J];
        auto it = std::lower_bound(
            w.begin(), w.end(), K,
            [&](int32_t b, int32_t key) { return P.blocks[b].I < key; });
        if (it != w.end() && P.blocks[*it].I == K) return *it;
        return -1;
    };
    // block rows of each level, ascending
    std::vector<std::vector<int32_t>> rows_of(L);
    for (int32_t I = 0; I < p; ++I) rows_of[P.level[I]].push_back(I);
    // tile rows: 128 for FP32 (one tensor-core MMA tile), 64 for FP64;
    // tile columns: 64
    const int32_t kTile = P.opts.precision == SLU_PREC_FP32 ? 128 : 64;
    // The lists of one level depend on nothing built for another level, so
    // threads take whole levels; the lists are then concatenated in level
    // order.  Inside a level: Schur targets ordered by (K, J), the source
    // pairs of a target in the order found (block rows I ascending, then
    // lower_col[I], then upper_row[I]); the execution split takes first the
    // targets in a block row or column of the next level (needed by its
    // GETRF / GESSM / TSTRF), then the rest, and splits each target's pairs
    // into dense tiles (dense target, dense sources) and the generic rest.
    struct Tgt {
        int32_t K, J, tb;
        int64_t first, count;
    };
    struct Lvl {                      // indices relative to the level
        std::vector<int32_t> getrf, gessm, tstrf, gd, gs, tgt, src;
        std::vector<int64_t> srcend;  // per target, end of its pairs in src
        std::vector<int32_t> gm_task, gm_src, gg_tgt, gg_src;
        std::vector<int64_t> gg_srcend;
        std::vector<uint32_t> gm_mask;    // per dense tile and source pair
        int64_t gm_mid = 0, gg_mid = 0;
    };
    // Live slices of the FP64 dense tiles: for the tile of target (K, J)
    // with rows r0 .. r0 + 63 and columns c0 .. c0 + 63 and its source pair
    // (K, I), (I, J), bit s is set when some column k of slice s (columns
    // 16 s .. 16 s + 15 of block I) holds, in the filled pattern, a row in the
    // tile's rows and one in its columns (U(k, c) is nonzero exactly when
    // column k holds row c, the pattern being symmetric); slices from 32 on
    // always count as live.  A slice without its bit holds only exact zeros
    // in the product, so the tile skips it.  Tiles are indexed globally:
    // tile (X, t) = rows 64 t .. 64 t + 63 of block X.
    const bool masks = P.opts.precision == SLU_PREC_FP64;
    std::vector<int64_t> tile_base(p + 1, 0);
    int32_t max_sl = 1;
    for (int32_t X = 0; X < p; ++X) {
        const int32_t rows = (int32_t)(P.ptr[X + 1] - P.ptr[X]);
        tile_base[X + 1] = tile_base[X] + (rows + 63) / 64;
        max_sl = std::max(max_sl, std::min(32, (rows + 15) / 16));
    }
    // tile of every row (rows 64 t .. 64 t + 63 of a block form its tile t)
    std::vector<int32_t> row_tile(masks ? (size_t)P.n : 0);
    for (int32_t X = 0; masks && X < p; ++X)
        for (int64_t r = P.ptr[X]; r < P.ptr[X + 1]; ++r)
            row_tile[r] = (int32_t)(tile_base[X] + (r - P.ptr[X]) / 64);
    auto tile_of = [&](int32_t r) -> int64_t { return row_tile[r]; };
    std::vector<Lvl> lvl(L);
    std::atomic<int32_t> next_lv{0};
    run_threads(std::min<int>(host_threads(nb), std::max(1, L)), [&](int) {
        std::vector<int32_t> slot(nb, -1), trip, pairs, dense_pairs, other;
        std::vector<int64_t> at;
        std::vector<Tgt> vec;
        // mask entries to fill: (block row I, entry, tile of the rows, tile
        // of the columns); per-slice masks of the columns of one block I
        struct MaskReq { int32_t I; int64_t e, tk, tj; };
        std::vector<MaskReq> req, req2;
        std::vector<Tgt> vec2;
        std::vector<uint16_t> tab(masks ? (size_t)tile_base[p] * max_sl : 0, 0);
        std::vector<int64_t> touched;
        // stable counting sort of src into dst by key(x) in [0, p)
        std::vector<int64_t> cnt(p + 1);
        auto by_key = [&](const auto &src, auto &dst, auto key) {
            std::fill(cnt.begin(), cnt.end(), 0);
            for (const auto &x : src) cnt[key(x) + 1]++;
            for (int32_t i = 0; i < p; ++i) cnt[i + 1] += cnt[i];
            dst.resize(src.size());
            for (const auto &x : src) dst[cnt[key(x)]++] = x;
        };
        for (int32_t lv; (lv = next_lv.fetch_add(1)) < L;) {
            Lvl &o = lvl[lv];
            vec.clear();
            trip.clear();
            for (int32_t I : rows_of[lv]) {
                const int32_t db = P.diagblk[I];
                o.getrf.push_back(db);
                for (int32_t b : upper_row[I]) {
                    o.gessm.push_back(b);
                    o.gessm.push_back(db);
                }
                for (int32_t b : lower_col[I]) {
                    o.tstrf.push_back(b);
                    o.tstrf.push_back(db);
                }
                for (int32_t lb : lower_col[I]) {
                    const int32_t K = P.blocks[lb].I;
                    for (int32_t ub : upper_row[I]) {
                        const int32_t J = P.blocks[ub].J;
                        const int32_t tb = find(K, J);
                        if (tb < 0) continue;
                        if (slot[tb] < 0) {
                            slot[tb] = (int32_t)vec.size();
                            vec.push_back(Tgt{K, J, tb, 0, 0});
                        }
                        trip.push_back(slot[tb]);
                        trip.push_back(lb);
                        trip.push_back(ub);
                    }
                }
            }
            // group the pairs by target, keeping their order (counting sort)
            at.assign(vec.size() + 1, 0);
            for (size_t t = 0; t < trip.size(); t += 3) at[trip[t] + 1]++;
            for (size_t k = 0; k < vec.size(); ++k) {
                vec[k].first = at[k];
                vec[k].count = at[k + 1];
                at[k + 1] += at[k];
            }
            pairs.resize(trip.size() / 3 * 2);
            for (size_t t = 0; t < trip.size(); t += 3) {
                const int64_t q = at[trip[t]]++;
                pairs[2 * q] = trip[t + 1];
                pairs[2 * q + 1] = trip[t + 2];
            }
            for (const Tgt &t : vec) slot[t.tb] = -1;
            // targets by (K, J) (unique per level): a comparison sort for a
            // few, else counting sorts by J, then stably by K
            if ((int64_t)vec.size() <= 64) {
                std::sort(vec.begin(), vec.end(), [](const Tgt &x, const Tgt &y) {
                    return x.K != y.K ? x.K < y.K : x.J < y.J;
                });
            } else {
                by_key(vec, vec2, [](const Tgt &t) { return t.J; });
                by_key(vec2, vec, [](const Tgt &t) { return t.K; });
            }
            o.tgt.reserve(vec.size());
            o.srcend.reserve(vec.size());
            o.src.reserve(pairs.size());
            for (const Tgt &t : vec) {
                o.tgt.push_back(t.tb);
                o.src.insert(o.src.end(), pairs.begin() + 2 * t.first,
                             pairs.begin() + 2 * (t.first + t.count));
                o.srcend.push_back((int64_t)o.src.size() / 2);
            }
            for (int32_t db : o.getrf) (P.blocks[db].dense ? o.gd : o.gs).push_back(db);
            for (int pass = 0; pass < 2; ++pass) {
                if (pass == 1) {
                    o.gm_mid = (int64_t)o.gm_task.size() / 5;
                    o.gg_mid = (int64_t)o.gg_tgt.size();
                }
                for (size_t k = 0; k < o.tgt.size(); ++k) {
                    const int32_t tb = o.tgt[k];
                    const BlockDesc &td = P.blocks[tb];
                    const bool next = P.level[std::min(td.I, td.J)] == lv + 1;
                    if (next != (pass == 0)) continue;
                    dense_pairs.clear();
                    other.clear();
                    for (int64_t q = k ? o.srcend[k - 1] : 0; q < o.srcend[k]; ++q) {
                        const int32_t lb = o.src[2 * q], ub = o.src[2 * q + 1];
                        auto &to = td.dense && P.blocks[lb].dense && P.blocks[ub].dense
                                       ? dense_pairs : other;
                        to.push_back(lb);
                        to.push_back(ub);
                    }
                    if (!dense_pairs.empty()) {
                        const int32_t s0 = (int32_t)(o.gm_src.size() / 2);
                        o.gm_src.insert(o.gm_src.end(), dense_pairs.begin(), dense_pairs.end());
                        const int32_t s1 = (int32_t)(o.gm_src.size() / 2);
                        for (int32_t r0 = 0; r0 < td.rows; r0 += kTile)
                            for (int32_t c0 = 0; c0 < td.cols; c0 += 64) {
                                const int32_t t5[5] = {tb, s0, s1, r0, c0};
                                o.gm_task.insert(o.gm_task.end(), t5, t5 + 5);
                                if (!masks) continue;
                                const int64_t tk = tile_of(td.r0 + r0), tj = tile_of(td.c0 + c0);
                                for (size_t q = 0; q < dense_pairs.size(); q += 2) {
                                    req.push_back({P.blocks[dense_pairs[q]].J,
                                                   (int64_t)o.gm_mask.size(), tk, tj});
                                    o.gm_mask.push_back(0);
                                }
                            }
                    }
                    if (!other.empty()) {
                        o.gg_tgt.push_back(tb);
                        o.gg_src.insert(o.gg_src.end(), other.begin(), other.end());
                        o.gg_srcend.push_back((int64_t)o.gg_src.size() / 2);
                    }
                }
            }
            if (masks && !req.empty()) {
                by_key(req, req2, [](const MaskReq &x) { return x.I; });
                req.swap(req2);
                for (size_t a0 = 0; a0 < req.size();) {
                    const int32_t I = req[a0].I;
                    size_t a1 = a0;
                    while (a1 < req.size() && req[a1].I == I) ++a1;
                    // per tile and slice: the columns of block I (bit k mod
                    // 16) holding a row of the tile below block I
                    const int64_t k0 = P.ptr[I], k1 = P.ptr[I + 1];
                    for (int64_t k = k0; k < k1; ++k) {
                        const int32_t sl = (int32_t)((k - k0) / 16);
                        if (sl >= 32) break;
                        const uint16_t bit = (uint16_t)(1u << ((k - k0) % 16));
                        // rows below block I: the column's rows ascend
                        const int32_t *c0 = P.f_rowidx.data() + P.f_colptr[k];
                        const int32_t *c1 = P.f_rowidx.data() + P.f_colptr[k + 1];
                        for (const int32_t *f = std::lower_bound(c0, c1, (int32_t)k1); f < c1; ++f) {
                            const int64_t at = (int64_t)row_tile[*f] * max_sl + sl;
                            if (!tab[at]) touched.push_back(at);
                            tab[at] |= bit;
                        }
                    }
                    const int32_t nsl = std::min<int32_t>(32, (int32_t)((k1 - k0 + 15) / 16));
                    for (size_t a = a0; a < a1; ++a) {
                        uint32_t m = 0;
                        for (int32_t sl = 0; sl < nsl; ++sl)
                            if (tab[req[a].tk * max_sl + sl] & tab[req[a].tj * max_sl + sl])
                                m |= 1u << sl;
                        o.gm_mask[req[a].e] = m;
                    }
                    for (int64_t at : touched) tab[at] = 0;
                    touched.clear();
                    a0 = a1;
                }
                req.clear();
            }
            // Inside each of the level's two tile launches the tiles run
            // longest first (live slices x 8 x 4 sub-tiles of the tile), so a
            // launch does not end on a few long tiles started last (list
            // scheduling, longest processing time first).  Every tile writes
            // only its own rows and columns of its target, so the order
            // changes no result.
            const int64_t nt = (int64_t)o.gm_task.size() / 5;
            if (nt > 1) {
                std::vector<int64_t> mo(nt + 1, 0);
                for (int64_t t = 0; t < nt; ++t)
                    mo[t + 1] = mo[t] + (o.gm_task[5 * t + 2] - o.gm_task[5 * t + 1]);
                std::vector<uint64_t> cost(nt);
                for (int64_t t = 0; t < nt; ++t) {
                    const int32_t *tk = &o.gm_task[5 * t];
                    const BlockDesc &td = P.blocks[tk[0]];
                    int64_t live = 0;
                    for (int32_t q = tk[1]; q < tk[2]; ++q) {
                        const int32_t nsl = (P.blocks[o.gm_src[2 * q]].cols + 15) / 16;
                        live += masks ? __builtin_popcount(o.gm_mask[mo[t] + (q - tk[1])]) +
                                            std::max(0, nsl - 32)
                                      : nsl;
                    }
                    const int32_t rt = std::min(kTile, td.rows - tk[3]);
                    const int32_t ct = std::min(64, td.cols - tk[4]);
                    // key: cost descending, then task ascending (unique keys)
                    const uint64_t c = std::min<uint64_t>(
                        (uint64_t)live * ((rt + 7) / 8) * ((ct + 3) / 4), 0xffffffffull);
                    cost[t] = ((0xffffffffull - c) << 32) | (uint64_t)(t - (t < o.gm_mid ? 0 : o.gm_mid));
                }
                std::sort(cost.begin(), cost.begin() + o.gm_mid);
                std::sort(cost.begin() + o.gm_mid, cost.end());
                std::vector<int64_t> perm(nt);
                for (int64_t t = 0; t < nt; ++t)
                    perm[t] = (int64_t)(cost[t] & 0xffffffffull) + (t < o.gm_mid ? 0 : o.gm_mid);
                std::vector<int32_t> task2(o.gm_task.size());
                std::vector<uint32_t> mask2(o.gm_mask.size());
                int64_t m = 0;
                for (int64_t t = 0; t < nt; ++t) {
                    const int64_t u = perm[t];
                    std::copy(o.gm_task.begin() + 5 * u, o.gm_task.begin() + 5 * u + 5,
                              task2.begin() + 5 * t);
                    if (masks) {
                        std::copy(o.gm_mask.begin() + mo[u], o.gm_mask.begin() + mo[u + 1],
                                  mask2.begin() + m);
                        m += mo[u + 1] - mo[u];
                    }
                }
                o.gm_task.swap(task2);
                o.gm_mask.swap(mask2);
            }
        }
    });
    // concatenation in level order (each level's slice copied by a thread
    // of its own, first touching its pages); offsets per level
    const int ntc = std::min<int>(host_threads(0), std::max(1, L));
    auto concat = [&](std::vector<int32_t> Lvl::*f, auto &out, std::vector<int64_t> *off,
                      int64_t per) {
        std::vector<int64_t> at(L + 1, 0);
        for (int32_t lv = 0; lv < L; ++lv) at[lv + 1] = at[lv] + (int64_t)(lvl[lv].*f).size();
        out.resize((size_t)at[L]);
        if (off) {
            off->assign(L + 1, 0);
            for (int32_t lv = 0; lv <= L; ++lv) (*off)[lv] = at[lv] / per;
        }
        std::atomic<int32_t> nx{0};
        run_threads(ntc, [&](int) {
            for (int32_t lv; (lv = nx.fetch_add(1)) < L;) {
                const auto &v = lvl[lv].*f;
                std::copy(v.begin(), v.end(), out.begin() + at[lv]);
            }
        });
    };
    concat(&Lvl::getrf, P.getrf, &P.getrf_off, 1);
    concat(&Lvl::gessm, P.gessm, &P.gessm_off, 2);
    concat(&Lvl::tstrf, P.tstrf, &P.tstrf_off, 2);
    concat(&Lvl::gd, P.gd, &P.gd_off, 1);
    concat(&Lvl::gs, P.gs, &P.gs_off, 1);
    concat(&Lvl::tgt, P.tgt, &P.tgt_off, 1);
    concat(&Lvl::src, P.src, nullptr, 1);
    concat(&Lvl::gg_tgt, P.gg_tgt, &P.gg_off, 1);
    concat(&Lvl::gg_src, P.gg_src, nullptr, 1);
    P.srcoff.assign(1, 0);
    P.srcoff.reserve(P.tgt.size() + 1);
    P.gg_srcoff.assign(1, 0);
    P.gg_srcoff.reserve(P.gg_tgt.size() + 1);
    {
        int64_t sb = 0, gb = 0;
        for (const Lvl &o : lvl) {
            for (int64_t e : o.srcend) P.srcoff.push_back(sb + e);
            for (int64_t e : o.gg_srcend) P.gg_srcoff.push_back(gb + e);
            sb += (int64_t)o.src.size() / 2;
            gb += (int64_t)o.gg_src.size() / 2;
        }
    }
    // dense tiles: source pair indices become global; slice masks in task
    // order, gm_moff[t] = first mask of task t (one mask per source pair of
    // the task).  Offsets per level first, then each level's slices copied
    // by a thread of its own (first touching their pages).
    P.gm_off.assign(L + 1, 0);
    P.gm_mid.assign(L, 0);
    P.gg_mid.assign(L, 0);
    P.gm_mask.clear();
    P.gm_moff.clear();
    {
        std::vector<int64_t> tat(L + 1, 0), sat(L + 1, 0), mat(L + 1, 0);
        for (int32_t lv = 0; lv < L; ++lv) {
            const Lvl &o = lvl[lv];
            tat[lv + 1] = tat[lv] + (int64_t)o.gm_task.size();
            sat[lv + 1] = sat[lv] + (int64_t)o.gm_src.size();
            mat[lv + 1] = mat[lv] + (int64_t)o.gm_mask.size();
            P.gm_mid[lv] = tat[lv] / 5 + o.gm_mid;
            P.gg_mid[lv] = P.gg_off[lv] + o.gg_mid;
            P.gm_off[lv + 1] = tat[lv + 1] / 5;
        }
        P.gm_task.resize((size_t)tat[L]);
        P.gm_src.resize((size_t)sat[L]);
        if (masks) {
            P.gm_mask.resize((size_t)mat[L]);
            P.gm_moff.resize(P.gm_task.size() / 5 + 1);
            P.gm_moff[0] = 0;
        }
        std::atomic<int32_t> nx{0};
        run_threads(ntc, [&](int) {
            for (int32_t lv; (lv = nx.fetch_add(1)) < L;) {
                const Lvl &o = lvl[lv];
                const int32_t base = (int32_t)(sat[lv] / 2);
                for (size_t t = 0; t < o.gm_task.size(); t += 5) {
                    int32_t *d = P.gm_task.data() + tat[lv] + t;
                    d[0] = o.gm_task[t];
                    d[1] = o.gm_task[t + 1] + base;
                    d[2] = o.gm_task[t + 2] + base;
                    d[3] = o.gm_task[t + 3];
                    d[4] = o.gm_task[t + 4];
                }
                std::copy(o.gm_src.begin(), o.gm_src.end(), P.gm_src.begin() + sat[lv]);
                if (!masks) continue;
                std::copy(o.gm_mask.begin(), o.gm_mask.end(), P.gm_mask.begin() + mat[lv]);
                // gm_moff[t + 1] for the level's tasks: the level's first
                // mask is mat[lv], its tasks' masks follow in task order
                int64_t m = mat[lv], t = tat[lv] / 5;
                for (size_t q = 0; q < o.gm_task.size(); q += 5, ++t) {
                    m += o.gm_task[q + 2] - o.gm_task[q + 1];
                    P.gm_moff[t + 1] = m;
                }
            }
        });
    }
    std::vector<Lvl>().swap(lvl);
    auto flat = [&](std::vector<std::vector<int32_t>> &v,
                    std::vector<int64_t> &off, std::vector<int32_t> &ids) {
        off.assign(p + 1, 0);
        ids.clear();
        for (int32_t I = 0; I < p; ++I) {
            ids.insert(ids.end(), v[I].begin(), v[I].end());
            off[I + 1] = (int64_t)ids.size();
        }
    };
    flat(lower_row, P.lrow_off, P.lrow_blk);
    flat(upper_row, P.urow_off, P.urow_blk);
    flat(upper_col, P.ucol_off, P.ucol_blk);
    flat(lower_col, P.lcol_off, P.lcol_blk);
    // inverses of dense diagonal blocks and the panel split
    constexpr int32_t kChunk = 64;
    const int64_t esz = P.opts.precision == SLU_PREC_FP64 ? 8 : 4;
    // a 64-wide chunk of the largest block must fit the kernels' shared memory
    auto inv_ok = [&](const BlockDesc &d) {
        return d.dense && d.rows <= 384 &&
               ((int64_t)d.rows * 64 + 16 * 64) * esz + 8 * d.rows + 256 <= 220 * 1024;
    };
    P.woff.assign(p, -1);
    P.wsize = 0;
    P.inv_maxb = 0;
    for (int32_t I = 0; I < p; ++I) {
        const BlockDesc &d = P.blocks[P.diagblk[I]];
        if (inv_ok(d)) {
            P.inv_maxb = std::max(P.inv_maxb, d.rows);
            P.woff[I] = P.wsize;
            P.wsize += 2 * (int64_t)d.rows * d.rows;
        }
    }
    P.dv_off.assign(L + 1, 0);
    P.dn_off.assign(L + 1, 0);
    P.dv_pos.clear();
    P.dn_pos.clear();
    for (int32_t lv = 0; lv < L; ++lv) {
        for (int64_t g = P.getrf_off[lv]; g < P.getrf_off[lv + 1]; ++g)
            (P.woff[P.blocks[P.getrf[g]].I] >= 0 ? P.dv_pos : P.dn_pos)
                .push_back((int32_t)g);
        P.dv_off[lv + 1] = (int64_t)P.dv_pos.size();
        P.dn_off[lv + 1] = (int64_t)P.dn_pos.size();
    }
    P.inv_off.assign(L + 1, 0);
    P.pd_off.assign(L + 1, 0);
    P.pg_goff.assign(L + 1, 0);
    P.pg_toff.assign(L + 1, 0);
    P.inv_task.clear();
    P.pd_task.clear();
    P.pg_gessm.clear();
    P.pg_tstrf.clear();
    P.ps_off.assign(L + 1, 0);
    P.ps_task.clear();
    P.pv_off.assign(L + 1, 0);
    P.pv_task.clear();
    // dense panels against a sparse diagonal block: chunks of V vectors
    auto add_vec = [&](int32_t type, int32_t tb, int32_t db) {
        const int32_t m = P.blocks[db].rows;
        const int32_t nvec = type == 0 ? P.blocks[tb].cols : P.blocks[tb].rows;
        const int32_t V = panel_vec_width(m, (int)esz);
        for (int32_t v0 = 0; v0 < nvec; v0 += V) {
            const int32_t t4[4] = {type, tb, db, v0};
            P.pv_task.insert(P.pv_task.end(), t4, t4 + 4);
        }
    };
    for (int32_t lv = 0; lv < L; ++lv) {
        for (int64_t g = P.getrf_off[lv]; g < P.getrf_off[lv + 1]; ++g) {
            const BlockDesc &d = P.blocks[P.getrf[g]];
            if (!inv_ok(d)) continue;
            for (int32_t which = 0; which < 2; ++which)
                for (int32_t j0 = 0; j0 < d.rows; j0 += 8) {
                    const int32_t t3[3] = {P.getrf[g], which, j0};
                    P.inv_task.insert(P.inv_task.end(), t3, t3 + 3);
                }
        }
        for (int64_t e = P.gessm_off[lv]; e < P.gessm_off[lv + 1]; ++e) {
            const int32_t tb = P.gessm[2 * e], db = P.gessm[2 * e + 1];
            if (inv_ok(P.blocks[db])) {
                for (int32_t c0 = 0; c0 < P.blocks[tb].cols; c0 += kChunk) {
                    const int32_t t4[4] = {0, tb, db, c0};
                    P.pd_task.insert(P.pd_task.end(), t4, t4 + 4);
                }
            } else if (P.blocks[tb].dense &&
                       panel_vec_width(P.blocks[db].rows, (int)esz) > 0) {
                add_vec(0, tb, db);
            } else if (!P.blocks[db].dense) {
                const int32_t t3[3] = {0, tb, db};
                P.ps_task.insert(P.ps_task.end(), t3, t3 + 3);
            } else {
                P.pg_gessm.push_back(tb);
                P.pg_gessm.push_back(db);
            }
        }
        for (int64_t e = P.tstrf_off[lv]; e < P.tstrf_off[lv + 1]; ++e) {
            const int32_t tb = P.tstrf[2 * e], db = P.tstrf[2 * e + 1];
            if (inv_ok(P.blocks[db])) {
                for (int32_t r0 = 0; r0 < P.blocks[tb].rows; r0 += kChunk) {
                    const int32_t t4[4] = {1, tb, db, r0};
                    P.pd_task.insert(P.pd_task.end(), t4, t4 + 4);
                }
            } else if (P.blocks[tb].dense &&
                       panel_vec_width(P.blocks[db].rows, (int)esz) > 0) {
                add_vec(1, tb, db);
            } else if (!P.blocks[db].dense) {
                const int32_t t3[3] = {1, tb, db};
                P.ps_task.insert(P.ps_task.end(), t3, t3 + 3);
            } else {
                P.pg_tstrf.push_back(tb);
                P.pg_tstrf.push_back(db);
            }
        }
        P.inv_off[lv + 1] = (int64_t)P.inv_task.size() / 3;
        P.pd_off[lv + 1] = (int64_t)P.pd_task.size() / 4;
        P.pg_goff[lv + 1] = (int64_t)P.pg_gessm.size() / 2;
        P.pg_toff[lv + 1] = (int64_t)P.pg_tstrf.size() / 2;
        P.ps_off[lv + 1] = (int64_t)P.ps_task.size() / 3;
        P.pv_off[lv + 1] = (int64_t)P.pv_task.size() / 4;
    }
    // solve pull pairs per sweep and level (the four sweeps independently,
    // one thread each; each owns its arrays)
    int64_t part_sw[4] = {0, 0, 0, 0};
    run_threads(std::min(4, host_threads(0)), [&](int t) {
        for (int sw = t; sw < 4; sw += std::min(4, host_threads(0))) {
            const auto &off = sw == 0 ? P.lrow_off : sw == 1 ? P.urow_off
                            : sw == 2 ? P.ucol_off : P.lcol_off;
            const auto &ids = sw == 0 ? P.lrow_blk : sw == 1 ? P.urow_blk
                            : sw == 2 ? P.ucol_blk : P.lcol_blk;
            P.sp_off[sw].assign(L + 1, 0);
            P.sp_pairs[sw].clear();
            P.sp_poff[sw].clear();
            P.sp_pairs[sw].reserve(2 * ids.size());
            P.sp_poff[sw].reserve(ids.size());
            P.sd_pair0[sw].assign(P.getrf.size(), 0);
            for (int32_t lv = 0; lv < L; ++lv) {
                int64_t acc = 0;
                for (int64_t g = P.getrf_off[lv]; g < P.getrf_off[lv + 1]; ++g) {
                    const int32_t db = P.getrf[g];
                    const int32_t I = P.blocks[db].I;
                    P.sd_pair0[sw][g] = (int64_t)P.sp_pairs[sw].size() / 2;
                    for (int64_t q = off[I]; q < off[I + 1]; ++q) {
                        P.sp_pairs[sw].push_back(ids[q]);
                        P.sp_pairs[sw].push_back(db);
                        P.sp_poff[sw].push_back(acc);
                        acc += P.blocks[db].rows;
                    }
                }
                P.sp_off[sw][lv + 1] = (int64_t)P.sp_pairs[sw].size() / 2;
                part_sw[sw] = std::max(part_sw[sw], acc);
            }
        }
    });
    P.part_elems = std::max(std::max(part_sw[0], part_sw[1]), std::max(part_sw[2], part_sw[3]));
}

// Analysis of one pattern; `seg` (row offsets, size nseg + 1) splits it
// into independent diagonal segments (a batch of matrices laid out block-
// diagonally), each blocked on its own.  With `device` the symbolic
// factorization, Algorithm 2, the sampling and Algorithm 3 run on the
// current GPU, enqueued on `stream`.
static slu_status analyze_impl(int64_t n, const int64_t *colptr,
                               const int32_t *rowidx, const slu_opts *opts,
                               const std::vector<int64_t> &seg,
                               slu_plan **out, bool device = false,
                               void *stream = nullptr) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!out) return fail(SLU_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 0 || n > INT32_MAX - 1)
        return fail(SLU_ERR_INVALID_ARG, "n out of range");
    if (!colptr || (n > 0 && !rowidx))
        return fail(SLU_ERR_INVALID_ARG, "NULL pattern array");
    slu_opts o;
    if (opts) o = *opts;
    else slu_opts_default(&o);
    if (o.blocking != SLU_BLOCKING_IRREGULAR &&
        o.blocking != SLU_BLOCKING_REGULAR &&
        o.blocking != SLU_BLOCKING_REGULAR_SELECT)
        return fail(SLU_ERR_INVALID_ARG, "unknown blocking");
    if (o.blocking == SLU_BLOCKING_REGULAR && o.regular_block <= 0)
        return fail(SLU_ERR_INVALID_ARG, "regular_block must be positive");
    if (o.sample_points <= 0 || o.step <= 0 || o.max_num < 0 ||
        o.stride <= 0 || o.b_min <= 0)
        return fail(SLU_ERR_INVALID_ARG, "bad blocking parameters");
    if (o.precision != SLU_PREC_FP64 && o.precision != SLU_PREC_FP32)
        return fail(SLU_ERR_INVALID_ARG, "unknown precision");
    if (o.tc_passes != 0 && o.tc_passes != 1 && o.tc_passes != 3)
        return fail(SLU_ERR_INVALID_ARG, "tc_passes must be 0, 1 or 3");
    if (!(o.dense_threshold >= 0.0))
        return fail(SLU_ERR_INVALID_ARG, "dense_threshold must be >= 0");
    if (colptr[0] != 0) return fail(SLU_ERR_INVALID_ARG, "colptr[0] must be 0");
    for (int64_t j = 0; j < n; ++j)
        if (colptr[j + 1] < colptr[j])
            return fail(SLU_ERR_INVALID_ARG, "colptr not monotone");
    const int64_t nnz = colptr[n];
    // row indices in range and no repeated (row, column): threads take
    // column ranges, each stopping at its first bad entry; the entry
    // reported is the earliest one, the one a sequential scan would meet
    try {
        const int nt = host_threads(n);
        const std::vector<int64_t> cut =
            balanced_cuts(n, [&](int64_t j) { return colptr[j]; }, nt);
        std::vector<int64_t> bad(nt, INT64_MAX);
        std::vector<int> kind(nt, 0);
        run_threads(nt, [&](int t) {
            std::vector<int32_t> seen(n, -1);   // column that last held row r
            for (int64_t j = cut[t]; j < cut[t + 1]; ++j)
                for (int64_t q = colptr[j]; q < colptr[j + 1]; ++q) {
                    const int32_t r = rowidx[q];
                    if (r < 0 || r >= n || seen[r] == j) {
                        bad[t] = q;
                        kind[t] = (r < 0 || r >= n) ? 1 : 2;
                        return;
                    }
                    seen[r] = (int32_t)j;
                }
        });
        const int t = (int)(std::min_element(bad.begin(), bad.end()) - bad.begin());
        if (kind[t] == 1) return fail(SLU_ERR_INVALID_ARG, "row index out of range");
        if (kind[t] == 2) return fail(SLU_ERR_INVALID_ARG, "duplicate entry");
    } catch (const std::exception &) {
        return fail(SLU_ERR_OUT_OF_MEMORY, "host allocation in analyze");
    }
    slu_plan *P = new (std::nothrow) slu_plan();
    if (!P) return fail(SLU_ERR_OUT_OF_MEMORY, "plan allocation");
    // phase k's time runs from the previous mark (the start of the call
    // for the first) to mark(k)
    auto tm = t0;
    auto mark = [&](int k) {
        const auto now = std::chrono::steady_clock::now();
        P->phase_ms[k] = std::chrono::duration<double, std::milli>(now - tm).count();
        tm = now;
    };
    try {
        P->opts = o;
        P->n = n;
        P->nnz_a = nnz;
        P->a_colptr.assign(colptr, colptr + n + 1);
        // copies by column ranges on the threads (first touch of the pages)
        P->a_rowidx.resize(nnz);
        P->a_ci.resize(nnz);
        {
            const int nt = host_threads(0);
            const std::vector<int64_t> cut =
                balanced_cuts(n, [&](int64_t j) { return colptr[j]; }, nt);
            run_threads(nt, [&](int t) {
                for (int64_t j = cut[t]; j < cut[t + 1]; ++j)
                    for (int64_t q = colptr[j]; q < colptr[j + 1]; ++q) {
                        P->a_rowidx[q] = rowidx[q];
                        P->a_ci[q] = (int32_t)j;
                    }
            });
        }
        // CSR view of A for the residual (columns ascending in every row)
        P->a_rowptr.assign(n + 1, 0);
        P->a_colidx.resize(nnz);
        P->a_vpos.resize(nnz);
        stable_transpose(
            n, colptr, n, [&](int64_t q) { return rowidx[q]; },
            [&](int64_t r, int64_t c) { P->a_rowptr[r + 1] = c; },
            [&](int64_t r) {
                if (r == 0)
                    for (int64_t i = 0; i < n; ++i) P->a_rowptr[i + 1] += P->a_rowptr[i];
                return P->a_rowptr[r];
            },
            [&](int64_t at, int64_t j, int64_t q) {
                P->a_colidx[at] = (int32_t)j;
                P->a_vpos[at] = q;
            });
        // A's columns with rows ascending and their input positions: the
        // transpose of the CSR view, taken in row order
        std::vector<int64_t> sp(n + 1, 0);
        big_vector<int32_t> si(nnz);
        big_vector<int64_t> sq(nnz);
        stable_transpose(
            n, P->a_rowptr.data(), n, [&](int64_t t) { return P->a_colidx[t]; },
            [&](int64_t j, int64_t c) { sp[j + 1] = c; },
            [&](int64_t j) {
                if (j == 0)
                    for (int64_t i = 0; i < n; ++i) sp[i + 1] += sp[i];
                return sp[j];
            },
            [&](int64_t at, int64_t r, int64_t t) {
                si[at] = (int32_t)r;
                sq[at] = P->a_vpos[t];
            });
        mark(SLU_PHASE_INPUT);
        std::vector<std::vector<int64_t>> dev_ptr;   // device Algorithm 3
        DeviceSymbolicTimes dtm;
        if (device) {
            // symbolic factorization, Algorithm 2, sampling and Algorithm 3
            // on the GPU (same results as the host branch below)
            const slu_status ds = device_symbolic(
                n, colptr, rowidx, seg, o, o.blocking == SLU_BLOCKING_IRREGULAR,
                stream, *P, dev_ptr, dtm);
            if (ds != SLU_OK) {
                delete P;
                return ds;
            }
            // flops = sum_k (l_k + 2 l_k^2), l_k the entries of column k
            // below the diagonal; the column holds l_k + 1 + u_k entries,
            // u_k = (blockptr[k + 1] - blockptr[k] - 1) / 2 above it
            P->flops = 0;
            for (int64_t k = 0; k < n; ++k) {
                const int64_t u = (P->blockptr[k + 1] - P->blockptr[k] - 1) / 2;
                const int64_t l = P->f_colptr[k + 1] - P->f_colptr[k] - 1 - u;
                P->flops += l + 2 * l * l;
            }
            mark(SLU_PHASE_SYMBOLIC);
        } else {
            std::vector<int64_t> Lp;
            big_vector<int32_t> Li;
            {
                Sym S;
                symmetrize(n, sp.data(), si.data(), P->a_rowptr.data(),
                           P->a_colidx.data(), S);
                P->nnz_sym = S.p[n];
                std::vector<int32_t> parent;
                etree(n, S, parent);
                symbolic(n, S, parent, Lp, Li);
            }
            // filled L+U pattern: column j = U rows (k < j with j in L(:,k),
            // ascending), the diagonal j, then L rows (ascending)
            std::vector<int64_t> ucnt(n, 0);
            P->f_colptr.assign(n + 1, 0);
            stable_transpose(
                n, Lp.data(), n, [&](int64_t q) { return Li[q]; },
                [&](int64_t j, int64_t c) { ucnt[j] = c; },
                [&](int64_t j) {
                    if (j == 0) {
                        for (int64_t i = 0; i < n; ++i)
                            P->f_colptr[i + 1] = P->f_colptr[i] + ucnt[i] + 1 + (Lp[i + 1] - Lp[i]);
                        P->f_rowidx.resize(P->f_colptr[n]);
                    }
                    return P->f_colptr[j];
                },
                [&](int64_t at, int64_t k, int64_t) { P->f_rowidx[at] = (int32_t)k; });
            run_threads(host_threads(0), [&](int t) {
                const int nt = host_threads(0);
                for (int64_t j = t; j < n; j += nt) {
                    int64_t f = P->f_colptr[j] + ucnt[j];
                    P->f_rowidx[f++] = (int32_t)j;
                    for (int64_t q = Lp[j]; q < Lp[j + 1]; ++q) P->f_rowidx[f++] = Li[q];
                }
            });
            // flops = sum_k (l_k + 2 l_k u_k); by symmetry u_k = l_k
            P->flops = 0;
            for (int64_t k = 0; k < n; ++k) {
                const int64_t l = Lp[k + 1] - Lp[k];
                P->flops += l + 2 * l * l;
            }
            std::vector<int64_t>().swap(Lp);
            big_vector<int32_t>().swap(Li);
            mark(SLU_PHASE_SYMBOLIC);
            // Algorithm 2 on the filled pattern
            P->blockptr.assign(n + 1, 0);
            diagonal_block_pointer(n, P->f_colptr.data(), P->f_rowidx.data(),
                                   P->blockptr.data());
        }
        // blocking, segment by segment: for a block-diagonal pattern the
        // diagonal block pointer of segment [s0, s1) is bp[s0 + k] - bp[s0]
        P->seg = seg;
        P->ptr.assign(1, 0);
        P->samples = 0;
        std::vector<int64_t> bps, ps;
        for (size_t q = 0; q + 1 < seg.size(); ++q) {
            const int64_t s0 = seg[q], N = seg[q + 1] - seg[q];
            if (N == 0) continue;
            if (o.blocking == SLU_BLOCKING_IRREGULAR && device) {
                ps = dev_ptr[q];
                P->samples = std::max<int32_t>(
                    P->samples, (int32_t)std::max<int64_t>(
                                    1, std::min<int64_t>(o.sample_points, N / o.b_min)));
            } else if (o.blocking == SLU_BLOCKING_IRREGULAR) {
                bps.resize(N + 1);
                for (int64_t k = 0; k <= N; ++k)
                    bps[k] = P->blockptr[s0 + k] - P->blockptr[s0];
                int64_t S_ = std::min<int64_t>(o.sample_points, N / o.b_min);
                if (S_ < 1) S_ = 1;
                P->samples = std::max<int32_t>(P->samples, (int32_t)S_);
                irregular_blocking(N, bps.data(), (int32_t)S_, o.step,
                                   o.max_num, o.stride, ps);
            } else {
                // fixed size, or the selection tree's size for this
                // segment (its filled entries: bp over the segment)
                int64_t rb = o.regular_block;
                if (o.blocking == SLU_BLOCKING_REGULAR_SELECT)
                    rb = slu_select_regular_block(
                        N, P->blockptr[s0 + N] - P->blockptr[s0]);
                P->regular_block = std::max<int32_t>(P->regular_block, (int32_t)rb);
                ps.clear();
                for (int64_t r = 0; r < N; r += rb) ps.push_back(r);
                ps.push_back(N);
            }
            for (size_t t = 1; t < ps.size(); ++t) P->ptr.push_back(s0 + ps[t]);
        }
        P->p = (int32_t)P->ptr.size() - 1;
        P->row_seg.clear();
        if (seg.size() > 2) {
            P->row_seg.resize(n);
            for (size_t q = 0; q + 1 < seg.size(); ++q)
                for (int64_t r = seg[q]; r < seg[q + 1]; ++r) P->row_seg[r] = (int32_t)q;
        }
        mark(SLU_PHASE_BLOCKING);
        if (device) {           // the device's Algorithm 2 / 3 time
            P->phase_ms[SLU_PHASE_SYMBOLIC] -= dtm.blocking_ms;
            P->phase_ms[SLU_PHASE_BLOCKING] += dtm.blocking_ms;
        }
        const slu_status st = build_blocks(*P);
        if (st != SLU_OK) {
            delete P;
            return st;
        }
        mark(SLU_PHASE_BLOCKS);
        build_levels_and_tasks(*P);
        mark(SLU_PHASE_TASKS);
        // flops per kernel class from the block of each column's rows;
        // threads sum contiguous column ranges (every term is an integer,
        // so the sums are exact below 2^53 whatever their order)
        const int ntc = host_threads(0);
        const std::vector<int64_t> cutc = balanced_cuts(
            n, [&](int64_t k) { return P->f_colptr[k]; }, ntc);
        std::vector<std::array<double, 3>> fc(ntc, {0.0, 0.0, 0.0});
        run_threads(ntc, [&](int t) {
            for (int64_t k = cutc[t]; k < cutc[t + 1]; ++k) {
                const int32_t I = P->rowblk[k];
                double lin = 0, lout = 0;
                for (int64_t q = P->f_colptr[k]; q < P->f_colptr[k + 1]; ++q) {
                    const int32_t r = P->f_rowidx[q];
                    if (r <= k) continue;
                    if (P->rowblk[r] == I) lin += 1; else lout += 1;
                }
                fc[t][0] += lin + 2 * lin * lin;
                fc[t][1] += lout + 4 * lin * lout;
                fc[t][2] += 2 * lout * lout;
            }
        });
        for (int t = 0; t < ntc; ++t)
            for (int c = 0; c < 3; ++c) P->flops_cls[c] += fc[t][c];
        // A entry -> storage slot, through the filled pattern: both columns
        // are sorted by row, so one walk per column finds every position
        // (sq is a permutation, so the column ranges write disjoint slots)
        P->a2s.resize(nnz);
        run_threads(ntc, [&](int t) {
            for (int64_t j = cutc[t]; j < cutc[t + 1]; ++j) {
                int64_t f = P->f_colptr[j];
                for (int64_t q = sp[j]; q < sp[j + 1]; ++q) {
                    while (P->f_rowidx[f] < si[q]) ++f;
                    P->a2s[sq[q]] = P->f2s[f];
                }
            }
        });
    } catch (const std::exception &e) {
        delete P;
        return fail(SLU_ERR_OUT_OF_MEMORY,
                    std::string("host allocation in analyze: ") + e.what());
    }
    mark(SLU_PHASE_MAPS);
    P->analyze_ms = std::chrono::duration<double, std::milli>(
                        std::chrono::steady_clock::now() - t0).count();
    *out = P;
    return SLU_OK;
}

// Regular-size selection tree (SLU_BLOCKING_REGULAR_SELECT), on the filled
// entries per column.  Fitted (depth-2 search minimising the mean log of
// time / best time) to B300 timings of the FP64 factor + solve with regular
// blocks of 32, 64, 128 and 256 rows over 21 seeded matrices: 2-D 5-point
// grids (n 576 .. 25,600), 3-D convection-diffusion and theta operators (n
// 1,000 .. 64,000) and bordered circuits (n 4,000 .. 20,000).  Geometric-
// mean slowdown against the best size of each matrix: 1.022, against 1.041
// for always 32 and 1.25 for always 64.  The order n entered no split of
// the best tree; it caps the size.
extern "C" int32_t slu_select_regular_block(int64_t n, int64_t nnz_lu) {
    if (n <= 0) return 1;
    const double per_col = (double)std::max<int64_t>(nnz_lu, 0) / (double)n;
    const int32_t b = per_col <= 42.6 ? 32 : per_col <= 95.0 ? 64 : 32;
    return (int32_t)std::min<int64_t>(b, n);
}

extern "C" slu_status slu_analyze(int64_t n, const int64_t *colptr,
                                  const int32_t *rowidx, const slu_opts *opts,
                                  slu_plan **out) {
    return analyze_impl(n, colptr, rowidx, opts,
                        std::vector<int64_t>{0, std::max<int64_t>(n, 0)}, out);
}

extern "C" slu_status slu_analyze_device(int64_t n, const int64_t *colptr,
                                         const int32_t *rowidx, const slu_opts *opts,
                                         void *stream, slu_plan **out) {
    return analyze_impl(n, colptr, rowidx, opts,
                        std::vector<int64_t>{0, std::max<int64_t>(n, 0)}, out, true,
                        stream);
}

static slu_status batch_impl(int32_t count, const int64_t *n,
                             const int64_t *const *colptr,
                             const int32_t *const *rowidx, const slu_opts *opts,
                             slu_plan **out, bool device, void *stream) {
    if (!out) return fail(SLU_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (count < 1 || !n || !colptr || !rowidx)
        return fail(SLU_ERR_INVALID_ARG, "bad batch arguments");
    // every member's column pointers are checked before any of its row
    // indices is read, so a malformed member cannot send the reads below
    // outside the caller's arrays
    int64_t N = 0, nnz = 0;
    for (int32_t q = 0; q < count; ++q) {
        const int64_t m = n[q];
        const int64_t *cq = colptr[q];
        if (m < 0 || !cq || (m > 0 && !rowidx[q]))
            return fail(SLU_ERR_INVALID_ARG, "bad batch member");
        if (m > INT32_MAX - 1 - N)
            return fail(SLU_ERR_INVALID_ARG, "batch too large");
        if (cq[0] != 0)
            return fail(SLU_ERR_INVALID_ARG, "colptr[0] must be 0");
        for (int64_t j = 0; j < m; ++j)
            if (cq[j + 1] < cq[j])
                return fail(SLU_ERR_INVALID_ARG, "colptr not monotone");
        if (cq[m] > INT64_MAX - nnz)
            return fail(SLU_ERR_INVALID_ARG, "batch too large");
        N += m;
        nnz += cq[m];
    }
    std::vector<int64_t> seg, cp;
    std::vector<int32_t> ri;
    try {
        seg.assign(1, 0);
        for (int32_t q = 0; q < count; ++q) seg.push_back(seg.back() + n[q]);
        cp.assign(N + 1, 0);
        ri.reserve(nnz);
    } catch (const std::exception &) {
        return fail(SLU_ERR_OUT_OF_MEMORY, "host allocation in analyze");
    }
    for (int32_t q = 0; q < count; ++q) {
        for (int64_t j = 0; j < n[q]; ++j) {
            for (int64_t e = colptr[q][j]; e < colptr[q][j + 1]; ++e) {
                const int32_t r = rowidx[q][e];
                if (r < 0 || r >= n[q])
                    return fail(SLU_ERR_INVALID_ARG, "row index out of range");
                ri.push_back((int32_t)(seg[q] + r));
            }
            cp[seg[q] + j + 1] = (int64_t)ri.size();
        }
    }
    return analyze_impl(N, cp.data(), ri.data(), opts, seg, out, device, stream);
}

extern "C" slu_status slu_analyze_batch(int32_t count, const int64_t *n,
                                        const int64_t *const *colptr,
                                        const int32_t *const *rowidx,
                                        const slu_opts *opts, slu_plan **out) {
    return batch_impl(count, n, colptr, rowidx, opts, out, false, nullptr);
}

extern "C" slu_status slu_analyze_batch_device(int32_t count, const int64_t *n,
                                               const int64_t *const *colptr,
                                               const int32_t *const *rowidx,
                                               const slu_opts *opts, void *stream,
                                               slu_plan **out) {
    return batch_impl(count, n, colptr, rowidx, opts, out, true, stream);
}

extern "C" slu_status slu_plan_query(const slu_plan *P, slu_plan_info *info) {
    if (!P || !info) return fail(SLU_ERR_INVALID_ARG, "NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->n = P->n;
    info->nnz_a = P->nnz_a;
    info->nnz_sym = P->nnz_sym;
    info->nnz_lu = P->f_colptr.empty() ? 0 : P->f_colptr.back();
    info->flops = P->flops;
    info->nblocks_1d = P->p;
    info->nlevels = P->nlevels;
    info->nblocks = (int64_t)P->blocks.size();
    info->ndense = P->ndense;
    info->storage_elems = P->storage;
    info->n_getrf = (int64_t)P->getrf.size();
    info->n_gessm = (int64_t)P->gessm.size() / 2;
    info->n_tstrf = (int64_t)P->tstrf.size() / 2;
    info->n_ssssm_targets = (int64_t)P->tgt.size();
    info->n_ssssm_pairs = (int64_t)P->src.size() / 2;
    info->max_block = P->maxb;
    info->samples = P->samples;
    info->regular_block = P->regular_block;
    info->analyze_ms = P->analyze_ms;
    for (int k = 0; k < SLU_PHASE_COUNT; ++k) info->phase_ms[k] = P->phase_ms[k];
    return SLU_OK;
}

extern "C" slu_status slu_plan_export(const slu_plan *P, int64_t *blockptr,
                                      int64_t *ptr, int64_t *colptr,
                                      int32_t *rowidx) {
    if (!P) return fail(SLU_ERR_INVALID_ARG, "NULL plan");
    if (blockptr)
        std::memcpy(blockptr, P->blockptr.data(), P->blockptr.size() * 8);
    if (ptr) std::memcpy(ptr, P->ptr.data(), P->ptr.size() * 8);
    if (colptr) std::memcpy(colptr, P->f_colptr.data(), P->f_colptr.size() * 8);
    if (rowidx) std::memcpy(rowidx, P->f_rowidx.data(), P->f_rowidx.size() * 4);
    return SLU_OK;
}

extern "C" slu_status slu_plan_export_blocks(const slu_plan *P, int32_t *bi,
                                             int32_t *bj, int64_t *bnnz,
                                             uint8_t *dense, int32_t *level) {
    if (!P) return fail(SLU_ERR_INVALID_ARG, "NULL plan");
    for (size_t b = 0; b < P->blocks.size(); ++b) {
        if (bi) bi[b] = P->blocks[b].I;
        if (bj) bj[b] = P->blocks[b].J;
        if (bnnz) bnnz[b] = P->bnnz[b];
        if (dense) dense[b] = (uint8_t)P->blocks[b].dense;
    }
    if (level) std::memcpy(level, P->level.data(), P->level.size() * 4);
    return SLU_OK;
}

extern "C" slu_status slu_plan_export_tasks(
    const slu_plan *P, int64_t *getrf_off, int32_t *getrf, int64_t *gessm_off,
    int32_t *gessm, int64_t *tstrf_off, int32_t *tstrf, int64_t *tgt_off,
    int32_t *tgt, int64_t *srcoff, int32_t *src) {
    if (!P) return fail(SLU_ERR_INVALID_ARG, "NULL plan");
    const auto &B = P->blocks;
    auto cp = [](int64_t *dst, const auto &v) {
        if (dst) std::memcpy(dst, v.data(), v.size() * 8);
    };
    cp(getrf_off, P->getrf_off);
    cp(gessm_off, P->gessm_off);
    cp(tstrf_off, P->tstrf_off);
    cp(tgt_off, P->tgt_off);
    cp(srcoff, P->srcoff);
    if (getrf)
        for (size_t i = 0; i < P->getrf.size(); ++i) getrf[i] = B[P->getrf[i]].I;
    if (gessm)
        for (size_t i = 0; i < P->gessm.size() / 2; ++i) {
            gessm[2 * i] = B[P->gessm[2 * i]].I;
            gessm[2 * i + 1] = B[P->gessm[2 * i]].J;
        }
    if (tstrf)
        for (size_t i = 0; i < P->tstrf.size() / 2; ++i) {
            tstrf[2 * i] = B[P->tstrf[2 * i]].I;
            tstrf[2 * i + 1] = B[P->tstrf[2 * i]].J;
        }
    if (tgt)
        for (size_t i = 0; i < P->tgt.size(); ++i) {
            tgt[2 * i] = B[P->tgt[i]].I;
            tgt[2 * i + 1] = B[P->tgt[i]].J;
        }
    if (src)
        for (size_t i = 0; i < P->src.size() / 2; ++i)
            src[i] = B[P->src[2 * i]].J;
    return SLU_OK;
}

extern "C" slu_status slu_plan_flops(const slu_plan *P, double *out) {
    if (!P || !out) return fail(SLU_ERR_INVALID_ARG, "NULL argument");
    for (int c = 0; c < 3; ++c) out[c] = P->flops_cls[c];
    return SLU_OK;
}

extern "C" void slu_plan_destroy(slu_plan *P) {
    if (!P) return;
    free_dev_plan(P);
    delete P;
}
