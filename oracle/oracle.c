/*
 * CPU FP64 oracle for sparse LU without row exchanges.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code with the GPU library.
 *
 * What it computes.  The paper's numerical factorization (Section 2.2,
 * Algorithm 1) reorders the work of a plain LU factorization A = L U into
 * 2-D blocks; it does not change the result, so the oracle is the plain
 * definition: a left-looking Gilbert-Peierls column LU (the algorithm behind
 * KLU, named in Section 1), L unit lower triangular, U upper triangular, no
 * row exchanges (static pivoting).  For column j:
 *   1. symbolic: the set of rows reachable from the rows of A(:,j) in the
 *      graph of L(:, 0:j-1) (edge k -> i for every stored L(i,k)); a depth
 *      first search yields them in topological order;
 *   2. x := A(:,j) scattered into a dense work vector;
 *   3. for k in topological order with k < j: x(i) -= L(i,k) x(k) for the
 *      stored rows i of L(:,k);
 *   4. U(0:j, j) := x at reached rows <= j; the pivot is x(j); a pivot with
 *      |pivot| < tau is replaced by copysign-like +-tau (sign of zero taken
 *      as +) and counted; L(i, j) := x(i) / pivot for reached rows i > j.
 * No entry is ever dropped, so the stored pattern is the symbolic one
 * (explicit zeros of A take part structurally).
 *
 * Also here: triangular solves with L, U, L^T and U^T on CSC factors.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct {
    int64_t n;
    int64_t *Lp; int32_t *Li; double *Lx;   /* strictly lower part, CSC   */
    int64_t *Up; int32_t *Ui; double *Ux;   /* upper part incl. diagonal  */
    int64_t nperturb;
    int64_t lcap, ucap;
} orc_lu;

enum { ORC_OK = 0, ORC_NOMEM = 1, ORC_SINGULAR = 2, ORC_BADARG = 3 };

static int grow(orc_lu *F, int lower, int64_t need)
{
    int64_t *cap = lower ? &F->lcap : &F->ucap;
    if (need <= *cap) return 0;
    int64_t nc = *cap ? *cap : 1024;
    while (nc < need) nc *= 2;
    if (lower) {
        int32_t *i2 = realloc(F->Li, (size_t)nc * sizeof(int32_t));
        if (!i2) return 1;
        F->Li = i2;
        double *x2 = realloc(F->Lx, (size_t)nc * sizeof(double));
        if (!x2) return 1;
        F->Lx = x2;
    } else {
        int32_t *i2 = realloc(F->Ui, (size_t)nc * sizeof(int32_t));
        if (!i2) return 1;
        F->Ui = i2;
        double *x2 = realloc(F->Ux, (size_t)nc * sizeof(double));
        if (!x2) return 1;
        F->Ux = x2;
    }
    *cap = nc;
    return 0;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

void orc_lu_free(orc_lu *F)
{
    if (!F) return;
    free(F->Lp); free(F->Li); free(F->Lx);
    free(F->Up); free(F->Ui); free(F->Ux);
    free(F);
}

/* Factor A (CSC, n x n).  tau = 0 disables perturbation; a zero pivot then
 * returns ORC_SINGULAR.  On success *out owns the factors. */
int orc_lu_factor(int64_t n, const int64_t *Ap, const int32_t *Ai,
                  const double *Ax, double tau, orc_lu **out)
{
    *out = NULL;
    if (n < 0) return ORC_BADARG;
    orc_lu *F = calloc(1, sizeof(orc_lu));
    if (!F) return ORC_NOMEM;
    F->n = n;
    F->Lp = calloc((size_t)n + 1, sizeof(int64_t));
    F->Up = calloc((size_t)n + 1, sizeof(int64_t));
    double *x = calloc((size_t)n + 1, sizeof(double));
    int64_t *mark = malloc(((size_t)n + 1) * sizeof(int64_t));
    int32_t *stack = malloc(((size_t)n + 1) * sizeof(int32_t));
    int64_t *pos = malloc(((size_t)n + 1) * sizeof(int64_t));
    int32_t *topo = malloc(((size_t)n + 1) * sizeof(int32_t));
    int32_t *rows = malloc(((size_t)n + 1) * sizeof(int32_t));
    int rc = ORC_OK;
    if (!F->Lp || !F->Up || !x || !mark || !stack || !pos || !topo || !rows) {
        rc = ORC_NOMEM; goto done;
    }
    for (int64_t i = 0; i < n; ++i) mark[i] = -1;

    for (int64_t j = 0; j < n; ++j) {
        /* 1. reach of struct(A(:,j)) in the graph of L(:,0:j-1) */
        int64_t top = n;                       /* topo[top..n) is the output */
        for (int64_t p = Ap[j]; p < Ap[j + 1]; ++p) {
            int32_t r = Ai[p];
            if (r < 0 || r >= n) { rc = ORC_BADARG; goto done; }
            if (mark[r] == j) continue;
            int64_t head = 0;
            stack[0] = r;
            mark[r] = j;
            pos[r] = (r < j) ? F->Lp[r] : 0;
            while (head >= 0) {
                int32_t v = stack[head];
                int pushed = 0;
                if (v < j) {
                    int64_t q = pos[v], end = F->Lp[v + 1];
                    while (q < end) {
                        int32_t w = F->Li[q++];
                        if (mark[w] != j) {
                            pos[v] = q;
                            mark[w] = j;
                            stack[++head] = w;
                            pos[w] = (w < j) ? F->Lp[w] : 0;
                            pushed = 1;
                            break;
                        }
                    }
                    if (!pushed) pos[v] = end;
                }
                if (!pushed) {                 /* finished: emit post-order */
                    --head;
                    topo[--top] = v;
                }
            }
        }
        /* 2. scatter A(:,j) */
        for (int64_t p = Ap[j]; p < Ap[j + 1]; ++p) x[Ai[p]] += Ax[p];
        /* 3. eliminate in topological order */
        for (int64_t t = top; t < n; ++t) {
            int32_t k = topo[t];
            if (k >= j) continue;
            double xk = x[k];
            for (int64_t q = F->Lp[k]; q < F->Lp[k + 1]; ++q)
                x[F->Li[q]] -= F->Lx[q] * xk;
        }
        /* 4. split into U(:,j) and L(:,j), rows sorted */
        int64_t cnt = n - top;
        memcpy(rows, topo + top, (size_t)cnt * sizeof(int32_t));
        qsort(rows, (size_t)cnt, sizeof(int32_t), cmp_i32);
        double piv = x[j];
        if (fabs(piv) < tau || (tau == 0.0 && piv == 0.0)) {
            if (tau == 0.0) { rc = ORC_SINGULAR; goto done; }
            piv = (piv >= 0.0) ? tau : -tau;
            F->nperturb++;
        }
        x[j] = piv;
        int64_t nu = 0, nl = 0;
        for (int64_t t = 0; t < cnt; ++t) (rows[t] <= j) ? ++nu : ++nl;
        if (grow(F, 0, F->Up[j] + nu) || grow(F, 1, F->Lp[j] + nl)) {
            rc = ORC_NOMEM; goto done;
        }
        int64_t pu = F->Up[j], pl = F->Lp[j];
        for (int64_t t = 0; t < cnt; ++t) {
            int32_t r = rows[t];
            if (r <= j) { F->Ui[pu] = r; F->Ux[pu++] = x[r]; }
            else        { F->Li[pl] = r; F->Lx[pl++] = x[r] / piv; }
            x[r] = 0.0;
        }
        F->Up[j + 1] = pu;
        F->Lp[j + 1] = pl;
    }
done:
    free(x); free(mark); free(stack); free(pos); free(topo); free(rows);
    if (rc != ORC_OK) { orc_lu_free(F); return rc; }
    *out = F;
    return ORC_OK;
}

int64_t orc_lu_n(const orc_lu *F) { return F->n; }
int64_t orc_lu_lnnz(const orc_lu *F) { return F->Lp[F->n]; }
int64_t orc_lu_unnz(const orc_lu *F) { return F->Up[F->n]; }
int64_t orc_lu_nperturb(const orc_lu *F) { return F->nperturb; }

void orc_lu_copy(const orc_lu *F, int64_t *Lp, int32_t *Li, double *Lx,
                 int64_t *Up, int32_t *Ui, double *Ux)
{
    int64_t n = F->n;
    memcpy(Lp, F->Lp, (size_t)(n + 1) * sizeof(int64_t));
    memcpy(Up, F->Up, (size_t)(n + 1) * sizeof(int64_t));
    memcpy(Li, F->Li, (size_t)F->Lp[n] * sizeof(int32_t));
    memcpy(Lx, F->Lx, (size_t)F->Lp[n] * sizeof(double));
    memcpy(Ui, F->Ui, (size_t)F->Up[n] * sizeof(int32_t));
    memcpy(Ux, F->Ux, (size_t)F->Up[n] * sizeof(double));
}

/* Solves on nrhs column-major right-hand sides X (leading dimension ld),
 * overwritten in place.  L is unit lower (strict part stored), U upper with
 * its diagonal stored as the last entry of each column (rows sorted). */
void orc_lsolve(int64_t n, const int64_t *Lp, const int32_t *Li,
                const double *Lx, double *X, int64_t ld, int32_t nrhs)
{
    for (int32_t c = 0; c < nrhs; ++c) {
        double *x = X + (int64_t)c * ld;
        for (int64_t k = 0; k < n; ++k) {
            double xk = x[k];
            for (int64_t q = Lp[k]; q < Lp[k + 1]; ++q) x[Li[q]] -= Lx[q] * xk;
        }
    }
}

void orc_usolve(int64_t n, const int64_t *Up, const int32_t *Ui,
                const double *Ux, double *X, int64_t ld, int32_t nrhs)
{
    for (int32_t c = 0; c < nrhs; ++c) {
        double *x = X + (int64_t)c * ld;
        for (int64_t k = n - 1; k >= 0; --k) {
            int64_t d = Up[k + 1] - 1;           /* diagonal entry */
            double xk = x[k] / Ux[d];
            x[k] = xk;
            for (int64_t q = Up[k]; q < d; ++q) x[Ui[q]] -= Ux[q] * xk;
        }
    }
}

/* L^T x = b: backward over columns of L (dot products). */
void orc_ltsolve(int64_t n, const int64_t *Lp, const int32_t *Li,
                 const double *Lx, double *X, int64_t ld, int32_t nrhs)
{
    for (int32_t c = 0; c < nrhs; ++c) {
        double *x = X + (int64_t)c * ld;
        for (int64_t k = n - 1; k >= 0; --k) {
            double s = x[k];
            for (int64_t q = Lp[k]; q < Lp[k + 1]; ++q) s -= Lx[q] * x[Li[q]];
            x[k] = s;
        }
    }
}

/* U^T x = b: forward over columns of U (dot products). */
void orc_utsolve(int64_t n, const int64_t *Up, const int32_t *Ui,
                 const double *Ux, double *X, int64_t ld, int32_t nrhs)
{
    for (int32_t c = 0; c < nrhs; ++c) {
        double *x = X + (int64_t)c * ld;
        for (int64_t k = 0; k < n; ++k) {
            int64_t d = Up[k + 1] - 1;
            double s = x[k];
            for (int64_t q = Up[k]; q < d; ++q) s -= Ux[q] * x[Ui[q]];
            x[k] = s / Ux[d];
        }
    }
}
