// General-matrix front end (host): what a general nonsymmetric matrix needs
// before the paper's method applies to it.  The paper factors matrices
// that arrive reordered (Section 1: reordering reduces fill and makes the
// nonzeros gather at the bottom right; Section 2.1) and, like the solvers
// it compares against, pivots statically.  Two steps:
//
//   1. Static pivoting by a maximum-product transversal: a row permutation
//      sigma (row sigma(j) matched to column j) maximising prod_j
//      |a_{sigma(j) j}|, found as a minimum-cost perfect matching on the
//      costs c_ij = log(max_i |a_ij|) - log |a_ij| >= 0 by shortest
//      augmenting paths (Dijkstra on reduced costs c_ij - u_i - v_j, the
//      Hungarian method for sparse matrices).  Its optimal duals give row
//      scales exp(u_i) and column scales exp(v_j) / max_i |a_ij| under
//      which every matched entry has magnitude 1 and no entry exceeds 1 (the
//      objective and scaling of Duff and Koster's MC64, option 5).
//   2. A fill-reducing symmetric ordering: nested dissection of the graph
//      of B + B^T (B = A with the matched entries moved to the diagonal) by
//      recursive bisection at the middle level of a breadth-first level
//      structure rooted at a pseudo-peripheral node (George's automatic
//      nested dissection); each separator is ordered after the two parts
//      it splits, parts of at most `leaf` nodes in their own order.  This
//      puts the separators, where the fill concentrates, at the bottom
//      right, as the irregular blocking expects.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <queue>
#include <utility>
#include <vector>

#include "slu_internal.hpp"

using namespace slu;

namespace {

bool check_pattern(int64_t n, const int64_t *cp, const int32_t *ri) {
    if (n < 0 || n > INT32_MAX - 1 || !cp || (n > 0 && !ri) || cp[0] != 0) return false;
    for (int64_t j = 0; j < n; ++j)
        if (cp[j + 1] < cp[j]) return false;
    for (int64_t q = 0; q < cp[n]; ++q)
        if (ri[q] < 0 || ri[q] >= n) return false;
    return true;
}

// Minimum-cost perfect matching of columns to rows on c (entries of A);
// row_of_col, u (rows), v (columns) are the matching and optimal duals
// with c_ij - u_i - v_j >= 0 everywhere and = 0 on matched entries.
// False when no perfect matching exists (structurally singular).
bool min_cost_matching(int64_t n, const int64_t *cp, const int32_t *ri,
                       const std::vector<double> &c, std::vector<int32_t> &row_of_col,
                       std::vector<double> &u, std::vector<double> &v) {
    const double inf = std::numeric_limits<double>::infinity();
    row_of_col.assign(n, -1);
    std::vector<int32_t> col_of_row(n, -1);
    u.assign(n, inf);
    v.assign(n, 0.0);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t q = cp[j]; q < cp[j + 1]; ++q) u[ri[q]] = std::min(u[ri[q]], c[q]);
    for (int64_t i = 0; i < n; ++i)
        if (u[i] == inf) return false;                  // empty row
    // greedy matching on tight entries (c_ij == u_i, v_j = 0)
    for (int64_t j = 0; j < n; ++j)
        for (int64_t q = cp[j]; q < cp[j + 1]; ++q) {
            const int32_t i = ri[q];
            if (col_of_row[i] < 0 && c[q] - u[i] <= 0.0) {
                col_of_row[i] = (int32_t)j;
                row_of_col[j] = i;
                break;
            }
        }
    std::vector<double> d(n, inf);
    std::vector<int32_t> pred(n, -1);
    std::vector<char> done(n, 0);
    std::vector<int32_t> touched, fin;
    using Item = std::pair<double, int32_t>;
    for (int64_t j0 = 0; j0 < n; ++j0) {
        if (row_of_col[j0] >= 0) continue;
        std::priority_queue<Item, std::vector<Item>, std::greater<Item>> heap;
        auto relax = [&](int32_t col, double base) {
            for (int64_t q = cp[col]; q < cp[col + 1]; ++q) {
                const int32_t k = ri[q];
                if (done[k] || c[q] == inf) continue;
                const double nd = base + std::max(0.0, c[q] - u[k] - v[col]);
                if (nd < d[k]) {
                    if (d[k] == inf) touched.push_back(k);
                    d[k] = nd;
                    pred[k] = col;
                    heap.push({nd, k});
                }
            }
        };
        relax((int32_t)j0, 0.0);
        int32_t found = -1;
        double D = 0.0;
        while (!heap.empty()) {
            const auto [di, i] = heap.top();
            heap.pop();
            if (done[i] || di > d[i]) continue;
            done[i] = 1;
            fin.push_back(i);
            if (col_of_row[i] < 0) {
                found = i;
                D = di;
                break;
            }
            relax(col_of_row[i], di);
        }
        if (found < 0) return false;                    // no augmenting path
        // duals: rows settled before `found` and the columns they reach
        v[j0] += D;
        for (int32_t k : fin) {
            if (k == found) continue;
            u[k] += d[k] - D;
            v[col_of_row[k]] += D - d[k];
        }
        // augment along the predecessor chain
        for (int32_t i = found;;) {
            const int32_t j = pred[i];
            const int32_t prev = row_of_col[j];
            row_of_col[j] = i;
            col_of_row[i] = j;
            if (j == (int32_t)j0) break;
            i = prev;
        }
        for (int32_t k : touched) {
            d[k] = inf;
            done[k] = 0;
            pred[k] = -1;
        }
        touched.clear();
        fin.clear();
    }
    return true;
}

// Nested dissection of the symmetric graph (xadj, adj; no self loops).
struct Dissection {
    const std::vector<int64_t> &xadj;
    const std::vector<int32_t> &adj;
    int32_t leaf;
    std::vector<int32_t> part;     // part id of every node
    std::vector<int32_t> level;    // BFS level scratch
    std::vector<int32_t> order;    // the result, position -> node
    int32_t next_id = 1;

    // BFS from r over the nodes of part `id`; returns the nodes by level
    // (levels[l] .. levels[l+1] of `q`) and the last level's size
    void bfs(int32_t r, int32_t id, std::vector<int32_t> &q, std::vector<int64_t> &lv) {
        q.clear();
        lv.assign(1, 0);
        q.push_back(r);
        level[r] = 0;
        size_t head = 0;
        int32_t cur = 0;
        std::vector<int32_t> seen;
        seen.push_back(r);
        while (head < q.size()) {
            const int32_t x = q[head];
            if (level[x] != cur) {
                lv.push_back((int64_t)head);
                cur = level[x];
            }
            ++head;
            for (int64_t e = xadj[x]; e < xadj[x + 1]; ++e) {
                const int32_t y = adj[e];
                if (part[y] != id || level[y] >= 0) continue;
                level[y] = cur + 1;
                q.push_back(y);
            }
        }
        lv.push_back((int64_t)q.size());
        for (int32_t x : q) level[x] = -1;
    }

    void run(std::vector<int32_t> nodes, int32_t id) {
        if (nodes.empty()) return;
        if ((int64_t)nodes.size() <= leaf) {
            std::sort(nodes.begin(), nodes.end());
            order.insert(order.end(), nodes.begin(), nodes.end());
            return;
        }
        // pseudo-peripheral root of the component holding the smallest node
        std::sort(nodes.begin(), nodes.end());
        std::vector<int32_t> q;
        std::vector<int64_t> lv;
        int32_t r = nodes[0];
        bfs(r, id, q, lv);
        for (int it = 0; it < 4; ++it) {
            const int64_t depth = (int64_t)lv.size() - 2;
            int32_t best = q[lv[lv.size() - 2]];           // a node of the last level,
            for (int64_t t = lv[lv.size() - 2]; t < lv.back(); ++t)   // the least degree
                if (xadj[q[t] + 1] - xadj[q[t]] < xadj[best + 1] - xadj[best] ||
                    (xadj[q[t] + 1] - xadj[q[t]] == xadj[best + 1] - xadj[best] && q[t] < best))
                    best = q[t];
            std::vector<int32_t> q2;
            std::vector<int64_t> lv2;
            bfs(best, id, q2, lv2);
            if ((int64_t)lv2.size() - 2 <= depth) break;
            r = best;
            q.swap(q2);
            lv.swap(lv2);
        }
        if ((int64_t)q.size() < (int64_t)nodes.size()) {
            // more than one component: this one, then the rest, no separator
            const int32_t a = next_id++, b = next_id++;
            std::vector<int32_t> comp(q.begin(), q.end()), rest;
            for (int32_t x : comp) part[x] = a;
            for (int32_t x : nodes)
                if (part[x] == id) {
                    part[x] = b;
                    rest.push_back(x);
                }
            run(std::move(comp), a);
            run(std::move(rest), b);
            return;
        }
        const int64_t L = (int64_t)lv.size() - 1;        // number of levels
        if (L < 3) {                                       // no level splits it
            order.insert(order.end(), nodes.begin(), nodes.end());
            return;
        }
        // separator: the level at which the cumulative count passes half
        int64_t m = 1;
        while (m < L - 1 && lv[m + 1] <= (int64_t)q.size() / 2) ++m;
        const int32_t a = next_id++, b = next_id++, s = next_id++;
        std::vector<int32_t> A(q.begin(), q.begin() + lv[m]), B(q.begin() + lv[m + 1], q.end()),
            S(q.begin() + lv[m], q.begin() + lv[m + 1]);
        for (int32_t x : A) part[x] = a;
        for (int32_t x : B) part[x] = b;
        for (int32_t x : S) part[x] = s;
        run(std::move(A), a);
        run(std::move(B), b);
        std::sort(S.begin(), S.end());
        order.insert(order.end(), S.begin(), S.end());
    }
};

}  // namespace

extern "C" slu_status slu_reorder(int64_t n, const int64_t *colptr, const int32_t *rowidx,
                                  const double *values, int32_t flags, int32_t leaf,
                                  int32_t *rowperm, int32_t *colperm, double *rowscale,
                                  double *colscale) {
    if (!check_pattern(n, colptr, rowidx))
        return fail(SLU_ERR_INVALID_ARG, "bad pattern");
    if ((flags & ~(SLU_REORDER_SCALE | SLU_REORDER_ORDER)) != 0)
        return fail(SLU_ERR_INVALID_ARG, "unknown reorder flags");
    if ((flags & SLU_REORDER_SCALE) && !values)
        return fail(SLU_ERR_INVALID_ARG, "scaling needs the values");
    if (n > 0 && (!rowperm || !colperm))
        return fail(SLU_ERR_INVALID_ARG, "NULL permutation array");
    try {
        std::vector<int32_t> row_of_col(n);
        std::vector<double> rs(n, 1.0), cs(n, 1.0);
        for (int64_t j = 0; j < n; ++j) row_of_col[j] = (int32_t)j;
        if (flags & SLU_REORDER_SCALE) {
            const double inf = std::numeric_limits<double>::infinity();
            std::vector<double> cmax(n, 0.0), c(colptr[n]);
            for (int64_t j = 0; j < n; ++j)
                for (int64_t q = colptr[j]; q < colptr[j + 1]; ++q) {
                    if (!std::isfinite(values[q]))
                        return fail(SLU_ERR_INVALID_ARG, "A holds a NaN or infinite value");
                    cmax[j] = std::max(cmax[j], std::fabs(values[q]));
                }
            for (int64_t j = 0; j < n; ++j) {
                if (cmax[j] == 0.0)
                    return fail(SLU_ERR_SINGULAR, "a column of A holds no nonzero");
                for (int64_t q = colptr[j]; q < colptr[j + 1]; ++q) {
                    const double a = std::fabs(values[q]);
                    c[q] = a > 0.0 ? std::log(cmax[j]) - std::log(a) : inf;
                }
            }
            std::vector<double> u, v;
            if (!min_cost_matching(n, colptr, rowidx, c, row_of_col, u, v))
                return fail(SLU_ERR_SINGULAR, "A is structurally singular (no perfect matching)");
            for (int64_t i = 0; i < n; ++i) rs[i] = std::exp(u[i]);
            for (int64_t j = 0; j < n; ++j) cs[j] = std::exp(v[j]) / cmax[j];
        }
        std::vector<int32_t> pi(n);
        if (flags & SLU_REORDER_ORDER) {
            // graph of B + B^T, B(j, j') = A(row_of_col[j], j')
            std::vector<int32_t> col_of_row(n);
            for (int64_t j = 0; j < n; ++j) col_of_row[row_of_col[j]] = (int32_t)j;
            std::vector<std::vector<int32_t>> nb(n);
            for (int64_t jp = 0; jp < n; ++jp)
                for (int64_t q = colptr[jp]; q < colptr[jp + 1]; ++q) {
                    const int32_t j = col_of_row[rowidx[q]];
                    if (j == (int32_t)jp) continue;
                    nb[j].push_back((int32_t)jp);
                    nb[jp].push_back(j);
                }
            std::vector<int64_t> xadj(n + 1, 0);
            std::vector<int32_t> adj;
            for (int64_t j = 0; j < n; ++j) {
                std::sort(nb[j].begin(), nb[j].end());
                nb[j].erase(std::unique(nb[j].begin(), nb[j].end()), nb[j].end());
                adj.insert(adj.end(), nb[j].begin(), nb[j].end());
                xadj[j + 1] = (int64_t)adj.size();
                std::vector<int32_t>().swap(nb[j]);
            }
            Dissection nd{xadj, adj, std::max<int32_t>(leaf, 1), {}, {}, {}};
            nd.part.assign(n, 0);
            nd.level.assign(n, -1);
            std::vector<int32_t> all(n);
            for (int64_t j = 0; j < n; ++j) all[j] = (int32_t)j;
            nd.run(std::move(all), 0);
            pi.swap(nd.order);
        } else {
            for (int64_t j = 0; j < n; ++j) pi[j] = (int32_t)j;
        }
        for (int64_t k = 0; k < n; ++k) {
            colperm[k] = pi[k];
            rowperm[k] = row_of_col[pi[k]];
        }
        if (rowscale) std::copy(rs.begin(), rs.end(), rowscale);
        if (colscale) std::copy(cs.begin(), cs.end(), colscale);
    } catch (const std::bad_alloc &) {
        return fail(SLU_ERR_OUT_OF_MEMORY, "host allocation in slu_reorder");
    }
    return SLU_OK;
}

extern "C" slu_status slu_reorder_apply(int64_t n, const int64_t *colptr, const int32_t *rowidx,
                                        const double *values, const int32_t *rowperm,
                                        const int32_t *colperm, const double *rowscale,
                                        const double *colscale, int64_t *out_colptr,
                                        int32_t *out_rowidx, double *out_values) {
    if (!check_pattern(n, colptr, rowidx) || !out_colptr || (n > 0 && (!rowperm || !colperm)) ||
        (colptr[n] > 0 && !out_rowidx))
        return fail(SLU_ERR_INVALID_ARG, "bad arguments");
    if (out_values && !values) return fail(SLU_ERR_INVALID_ARG, "values needed for out_values");
    try {
        // inverse row permutation, checked to be a permutation
        std::vector<int32_t> pos(n, -1);
        std::vector<char> seen(n, 0);
        for (int64_t k = 0; k < n; ++k) {
            if (rowperm[k] < 0 || rowperm[k] >= n || pos[rowperm[k]] >= 0 ||
                colperm[k] < 0 || colperm[k] >= n || seen[colperm[k]])
                return fail(SLU_ERR_INVALID_ARG, "rowperm / colperm are not permutations");
            pos[rowperm[k]] = (int32_t)k;
            seen[colperm[k]] = 1;
        }
        out_colptr[0] = 0;
        std::vector<std::pair<int32_t, double>> col;
        for (int64_t k = 0; k < n; ++k) {
            const int32_t j = colperm[k];
            col.clear();
            for (int64_t q = colptr[j]; q < colptr[j + 1]; ++q) {
                const int32_t i = rowidx[q];
                double x = 0.0;
                if (values)
                    x = (rowscale ? rowscale[i] : 1.0) * values[q] * (colscale ? colscale[j] : 1.0);
                col.push_back({pos[i], x});
            }
            std::sort(col.begin(), col.end(),
                      [](const std::pair<int32_t, double> &a, const std::pair<int32_t, double> &b) {
                          return a.first < b.first;
                      });
            const int64_t o = out_colptr[k];
            for (size_t t = 0; t < col.size(); ++t) {
                out_rowidx[o + (int64_t)t] = col[t].first;
                if (out_values) out_values[o + (int64_t)t] = col[t].second;
            }
            out_colptr[k + 1] = o + (int64_t)col.size();
        }
    } catch (const std::bad_alloc &) {
        return fail(SLU_ERR_OUT_OF_MEMORY, "host allocation in slu_reorder_apply");
    }
    return SLU_OK;
}
