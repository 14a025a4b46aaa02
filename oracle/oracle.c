/*
 * oracle.c -- plain, slow, obviously correct CPU reference (TEST INFRASTRUCTURE).
 *
 * Only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg may load this file's library.  The product path never calls it, and it
 * shares no code with the CUDA library.
 *
 * Everything here is FP64 with sequential sums in index order, compiled with
 * -ffp-contract=off (no fused multiply-add), so that each result is the plain
 * definition evaluated left to right:
 *
 *   oracle_csr_spmv   y_i = sum_j A_ij x_j over the stored entries of row i, in
 *                     stored order: the product A x = y that every format of
 *                     Sec. 4 and Sec. 5 computes (CSR storage: Sec. 4, CSR).
 *   oracle_pcg        textbook Jacobi-preconditioned conjugate gradients
 *                     (Hestenes-Stiefel), the solver the paper uses for the
 *                     Newton update K dx = R (Sec. 2.1, Sec. 4), one sparse
 *                     product per iteration.
 *   oracle_refine     FP64 iterative refinement around a low-precision inner
 *                     CG on the symmetrically scaled matrix B = S A S,
 *                     S = diag(A)^(-1/2), with B stored in FP32 or BF16 and FP64
 *                     dot products.  The paper runs FP64 only (Sec. 2); this
 *                     is the mixed-precision layer built on top of it.
 *   oracle_refine_reliable  the same pieces without restarts: one low-precision
 *                     CG whose recurrence residual is replaced by the FP64 true
 *                     residual (and x updated in FP64) each time it has fallen
 *                     by a factor delta ("reliable updates", Sleijpen and van
 *                     der Vorst 1996); the search direction is kept.
 *
 *   oracle_assemble_matrix / oracle_assemble_vector
 *                     the global stiffness values and a global residual vector
 *                     from element quantities: every global entry is the sum of
 *                     the element contributions to it (Sec. 4 writes this as
 *                     the row sums K^elem 1 of a matrix with one row per global
 *                     non-zero), here summed in ascending element order, with
 *                     homogeneous Dirichlet rows eliminated symmetrically.
 *
 * The paper gives no code for CG; these routines follow the standard
 * algorithm step by step.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Host threads for the row loop of oracle_csr_spmv (1 unless the benchmark's
 * CPU baseline asks for more).  Each row is still one sequential sum in stored
 * order, so the product -- and every routine built on it -- gives bitwise the
 * same result for any thread count; the other loops stay sequential. */
static int g_threads = 1;

void oracle_set_threads(int threads) { g_threads = threads < 1 ? 1 : threads; }

int oracle_get_threads(void) { return g_threads; }

/* y = A x, CSR, FP64, row by row, entries in stored order. */
void oracle_csr_spmv(int64_t n, const int64_t* rowptr, const int32_t* colind,
                     const double* val, const double* x, double* y) {
#pragma omp parallel for schedule(static) num_threads(g_threads) if (g_threads > 1)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) s = s + val[p] * x[colind[p]];
        y[i] = s;
    }
}

static double dot(int64_t n, const double* a, const double* b) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s = s + a[i] * b[i];
    return s;
}

/* diag(A) entries; 0 where a row stores no diagonal */
static void diagonal(int64_t n, const int64_t* rowptr, const int32_t* colind,
                     const double* val, double* d) {
    for (int64_t i = 0; i < n; ++i) {
        d[i] = 0.0;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
            if (colind[p] == i) d[i] = d[i] + val[p];
    }
}

enum { OR_CONVERGED = 0, OR_NOT_CONVERGED = 1, OR_BREAKDOWN = 2, OR_BAD_INPUT = 3 };

/*
 * Jacobi-preconditioned CG (M = diag(A) when jacobi != 0, M = I otherwise).
 *   r = b - A x0;  z = M^-1 r;  p = z;  rho = r.z
 *   repeat: q = A p;  alpha = rho / (p.q);  x += alpha p;  r -= alpha q;
 *           stop when ||r|| / ||b|| <= tol;
 *           z = M^-1 r;  rho' = r.z;  beta = rho' / rho;  p = z + beta p
 * After the loop the true residual ||b - A x|| / ||b|| is checked; if it is
 * above tol the iteration restarts from the current x (at most max_restarts
 * times).  iters counts every CG step over all restarts.
 * Returns 0 converged, 1 not converged, 2 breakdown (p.q <= 0 or non-finite),
 * 3 bad input (zero/negative diagonal with jacobi).
 */
int oracle_pcg(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val,
               const double* b, double* x, double tol, int max_iter, int jacobi,
               int max_restarts, int* iters_out, double* relres_out, double* true_relres_out) {
    double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* z = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* p = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* q = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* dg = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int status = OR_NOT_CONVERGED;
    int iters = 0;
    double relres = 0.0, true_relres = 0.0;
    diagonal(n, rowptr, colind, val, dg);
    if (jacobi)
        for (int64_t i = 0; i < n; ++i)
            if (!(dg[i] > 0.0)) { status = OR_BAD_INPUT; goto done; }
    double bnorm = sqrt(dot(n, b, b));
    if (bnorm == 0.0) {
        for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
        status = OR_CONVERGED;
        goto done;
    }
    for (int restart = 0; restart <= max_restarts; ++restart) {
        oracle_csr_spmv(n, rowptr, colind, val, x, q);
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
        relres = sqrt(dot(n, r, r)) / bnorm;
        if (relres <= tol) { status = OR_CONVERGED; true_relres = relres; goto done; }
        for (int64_t i = 0; i < n; ++i) z[i] = jacobi ? r[i] / dg[i] : r[i];
        for (int64_t i = 0; i < n; ++i) p[i] = z[i];
        double rho = dot(n, r, z);
        int converged = 0;
        while (iters < max_iter) {
            oracle_csr_spmv(n, rowptr, colind, val, p, q);
            double pq = dot(n, p, q);
            if (!(pq > 0.0) || !isfinite(pq)) { status = OR_BREAKDOWN; goto final; }
            double alpha = rho / pq;
            for (int64_t i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];
            for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];
            ++iters;
            relres = sqrt(dot(n, r, r)) / bnorm;
            if (!isfinite(relres)) { status = OR_BREAKDOWN; goto final; }
            if (relres <= tol) { converged = 1; break; }
            for (int64_t i = 0; i < n; ++i) z[i] = jacobi ? r[i] / dg[i] : r[i];
            double rho_new = dot(n, r, z);
            double beta = rho_new / rho;
            rho = rho_new;
            for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        }
        if (!converged) { status = OR_NOT_CONVERGED; break; }
        /* verify on the true residual */
        oracle_csr_spmv(n, rowptr, colind, val, x, q);
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
        true_relres = sqrt(dot(n, r, r)) / bnorm;
        if (true_relres <= tol) { status = OR_CONVERGED; goto done; }
    }
final:
    oracle_csr_spmv(n, rowptr, colind, val, x, q);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    true_relres = sqrt(dot(n, r, r)) / bnorm;
done:
    if (iters_out) *iters_out = iters;
    if (relres_out) *relres_out = relres;
    if (true_relres_out) *true_relres_out = true_relres;
    free(r); free(z); free(p); free(q); free(dg);
    return status;
}

/*
 * Jacobi-PCG with one reduction per iteration (Chronopoulos and Gear's
 * rearrangement of the same recurrences): with u = M^-1 r and w = A u,
 *   gamma = r.u, delta = w.u;  first step: beta = 0, alpha = gamma / delta;
 *   later: beta = gamma / gamma_prev, alpha = gamma / (delta - beta gamma / alpha_prev);
 *   p = u + beta p, s = w + beta s (s = A p), x += alpha p, r -= alpha s.
 * In exact arithmetic it produces the iterates of oracle_pcg.  Stops when
 * ||r|| <= tol ||b|| (checked on the r that the next product starts from);
 * true-residual restarts and status codes as oracle_pcg.
 */
int oracle_pcg_single_reduction(int64_t n, const int64_t* rowptr, const int32_t* colind,
                                const double* val, const double* b, double* x, double tol,
                                int max_iter, int jacobi, int max_restarts, int* iters_out,
                                double* relres_out, double* true_relres_out) {
    size_t nb = sizeof(double) * (size_t)(n > 0 ? n : 1);
    double *r = (double*)malloc(nb), *u = (double*)malloc(nb), *w = (double*)malloc(nb);
    double *p = (double*)malloc(nb), *sv = (double*)malloc(nb), *dg = (double*)malloc(nb);
    int status = OR_NOT_CONVERGED, iters = 0;
    double relres = 0.0, true_relres = 0.0;
    diagonal(n, rowptr, colind, val, dg);
    if (jacobi)
        for (int64_t i = 0; i < n; ++i)
            if (!(dg[i] > 0.0)) { status = OR_BAD_INPUT; goto done1; }
    double bnorm = sqrt(dot(n, b, b));
    if (bnorm == 0.0) {
        for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
        status = OR_CONVERGED;
        goto done1;
    }
    for (int restart = 0; restart <= max_restarts; ++restart) {
        oracle_csr_spmv(n, rowptr, colind, val, x, w);
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - w[i];
        relres = sqrt(dot(n, r, r)) / bnorm;
        if (relres <= tol) { status = OR_CONVERGED; true_relres = relres; goto done1; }
        for (int64_t i = 0; i < n; ++i) {
            u[i] = jacobi ? r[i] / dg[i] : r[i];
            p[i] = 0.0;
            sv[i] = 0.0;
        }
        double gamma_prev = 0.0, alpha = 0.0;
        int first = 1, converged = 0;
        for (;;) {
            oracle_csr_spmv(n, rowptr, colind, val, u, w);
            double gamma = dot(n, r, u);
            double delta = dot(n, w, u);
            relres = sqrt(dot(n, r, r)) / bnorm;
            if (!first) ++iters;
            if (!isfinite(relres) || !isfinite(gamma) || !isfinite(delta)) { status = OR_BREAKDOWN; goto final1; }
            if (relres <= tol) { converged = 1; break; }
            if (iters >= max_iter) break;
            double beta, denom;
            if (first) {
                beta = 0.0;
                denom = delta;
            } else {
                beta = gamma / gamma_prev;
                denom = delta - beta * gamma / alpha;
            }
            if (!(denom > 0.0)) { status = OR_BREAKDOWN; goto final1; }
            alpha = gamma / denom;
            gamma_prev = gamma;
            first = 0;
            for (int64_t i = 0; i < n; ++i) {
                p[i] = u[i] + beta * p[i];
                sv[i] = w[i] + beta * sv[i];
                x[i] = x[i] + alpha * p[i];
                r[i] = r[i] - alpha * sv[i];
                u[i] = jacobi ? r[i] / dg[i] : r[i];
            }
        }
        if (!converged) { status = OR_NOT_CONVERGED; break; }
        oracle_csr_spmv(n, rowptr, colind, val, x, w);
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - w[i];
        true_relres = sqrt(dot(n, r, r)) / bnorm;
        if (true_relres <= tol) { status = OR_CONVERGED; goto done1; }
    }
final1:
    oracle_csr_spmv(n, rowptr, colind, val, x, w);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - w[i];
    true_relres = sqrt(dot(n, r, r)) / bnorm;
done1:
    if (iters_out) *iters_out = iters;
    if (relres_out) *relres_out = relres;
    if (true_relres_out) *true_relres_out = true_relres;
    free(r); free(u); free(w); free(p); free(sv); free(dg);
    return status;
}

/* Round a float to bfloat16 (round to nearest, ties to even), returned as float. */
static float round_bf16(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) {           /* inf / nan: truncate, keep nan */
        if (u & 0x007fffffu) u |= 0x00400000u;
        u &= 0xffff0000u;
    } else {
        uint32_t lsb = (u >> 16) & 1u;
        u = u + 0x7fffu + lsb;
        u &= 0xffff0000u;
    }
    float g;
    memcpy(&g, &u, 4);
    return g;
}

/* Exported for the pin test that checks the rounding against another bf16 converter. */
float oracle_round_bf16(float f) { return round_bf16(f); }

/* y = B w with B in float (values already rounded to the storage type), float sums. */
static void spmv_f32(int64_t n, const int64_t* rowptr, const int32_t* colind,
                     const float* bv, const float* w, float* y) {
    for (int64_t i = 0; i < n; ++i) {
        float s = 0.0f;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) s = s + bv[p] * w[colind[p]];
        y[i] = s;
    }
}

static double dot_f(int64_t n, const float* a, const float* b) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s = s + (double)a[i] * (double)b[i];
    return s;
}

/* B = S A S in the refinement's storage: bv[k] = round((s_i * a_ik) * s_k), with
 * s_i = 1/sqrt(a_ii) in FP64, rounded to float (storage 0) or bfloat16 (1).
 * Returns 0, or 2 if a diagonal entry is not positive. */
int oracle_scaled_values(int64_t n, const int64_t* rowptr, const int32_t* colind,
                         const double* val, int storage, float* bv) {
    double* d = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    diagonal(n, rowptr, colind, val, d);
    for (int64_t i = 0; i < n; ++i) {
        if (!(d[i] > 0.0)) { free(d); return 2; }
        d[i] = 1.0 / sqrt(d[i]);
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            float f = (float)(d[i] * val[k] * d[colind[k]]);
            bv[k] = storage == 1 ? round_bf16(f) : f;
        }
    free(d);
    return 0;
}

/* y = B x in float, rows summed left to right (the refinement's inner product). */
void oracle_csr_spmv_f32(int64_t n, const int64_t* rowptr, const int32_t* colind,
                         const float* bv, const float* x, float* y) {
    spmv_f32(n, rowptr, colind, bv, x, y);
}

/*
 * Mixed-precision iterative refinement.
 *   S = diag(A)^(-1/2);  B = S A S rounded to float (storage 0) or bfloat16 (storage 1)
 *   x = x0
 *   repeat: r = b - A x                                  (FP64)
 *           stop when ||r|| / ||b|| <= tol
 *           solve B w = S r by plain CG in float vectors with FP64 dot products
 *             until ||B w - S r|| <= inner_tol ||S r|| (recurrence) or max_inner
 *           x = x + S w                                   (FP64)
 * diag(B) = 1, so Jacobi on B is the identity and the inner CG is unpreconditioned.
 * Returns 0 converged, 1 not converged (max_outer), 2 breakdown/stagnation.
 * outer_out / inner_out: refinement steps and total inner CG steps.
 */
int oracle_refine(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val,
                  const double* b, double* x, double tol, double inner_tol, int max_outer,
                  int max_inner, int storage, int* outer_out, int* inner_out,
                  double* true_relres_out) {
    int64_t nnz = rowptr[n];
    double* s = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* t = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    float* bv = (float*)malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
    float* rs = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    float* w = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    float* ri = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    float* p = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    float* q = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    int status = 1, outer = 0, inner_total = 0;
    double relres = 0.0;
    diagonal(n, rowptr, colind, val, t);
    for (int64_t i = 0; i < n; ++i) {
        if (!(t[i] > 0.0)) { status = 2; goto done; }
        s[i] = 1.0 / sqrt(t[i]);
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            float f = (float)(s[i] * val[k] * s[colind[k]]);
            bv[k] = storage == 1 ? round_bf16(f) : f;
        }
    double bnorm = sqrt(dot(n, b, b));
    if (bnorm == 0.0) {
        for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
        status = 0;
        goto done;
    }
    double prev = INFINITY;
    for (outer = 0; outer <= max_outer; ++outer) {
        oracle_csr_spmv(n, rowptr, colind, val, x, t);
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - t[i];
        relres = sqrt(dot(n, r, r)) / bnorm;
        if (relres <= tol) { status = 0; break; }
        if (outer == max_outer) { status = 1; break; }
        if (!isfinite(relres) || relres > prev) { status = 2; break; }
        prev = relres;
        /* inner: B w = S r, w0 = 0 */
        for (int64_t i = 0; i < n; ++i) {
            rs[i] = (float)(s[i] * r[i]);
            w[i] = 0.0f;
            ri[i] = rs[i];
            p[i] = rs[i];
        }
        double rsn = sqrt(dot_f(n, rs, rs));
        double rho = dot_f(n, ri, ri);
        for (int k = 0; k < max_inner; ++k) {
            spmv_f32(n, rowptr, colind, bv, p, q);
            double pq = dot_f(n, p, q);
            if (!(pq > 0.0)) break;
            float alpha = (float)(rho / pq);
            for (int64_t i = 0; i < n; ++i) w[i] = w[i] + alpha * p[i];
            for (int64_t i = 0; i < n; ++i) ri[i] = ri[i] - alpha * q[i];
            ++inner_total;
            double rho_new = dot_f(n, ri, ri);
            if (sqrt(rho_new) <= inner_tol * rsn) break;
            float beta = (float)(rho_new / rho);
            rho = rho_new;
            for (int64_t i = 0; i < n; ++i) p[i] = ri[i] + beta * p[i];
        }
        for (int64_t i = 0; i < n; ++i) x[i] = x[i] + s[i] * (double)w[i];
    }
done:
    if (outer_out) *outer_out = outer;
    if (inner_out) *inner_out = inner_total;
    if (true_relres_out) *true_relres_out = relres;
    free(s); free(r); free(t); free(bv); free(rs); free(w); free(ri); free(p); free(q);
    return status;
}

/*
 * Mixed-precision CG with reliable updates (no restarts).
 *   S, B as in oracle_refine.  x = x0;  r = b - A x (FP64);  rs = float(S r)
 *   w = 0;  r_in = rs;  p = rs;  rho = r_in.r_in;  m = ||rs||;  c = ||r|| / ||rs||
 *   repeat (at most max_iter steps):
 *       q = B p;  alpha = rho / (p.q)            (p.q <= 0: breakdown)
 *       w += alpha p;  r_in -= alpha q;  rho' = r_in.r_in
 *       if sqrt(rho') <= delta m  or  c sqrt(rho') <= tol ||b||:      (reliable update)
 *           x += S w (FP64);  w = 0;  r = b - A x (FP64)
 *           stop when ||r|| <= tol ||b||;  stop (stagnation) when ||r|| did not
 *             decrease since the previous update
 *           r_in = float(S r);  rho' = r_in.r_in;  m = ||r_in||;  c = ||r|| / ||r_in||
 *       beta = rho' / rho;  rho = rho';  p = r_in + beta p
 * Vectors w, r_in, p, q are float, products float, dot products FP64 (as in
 * oracle_refine).  Returns 0 converged, 1 not converged (max_iter), 2 breakdown or
 * stagnation; updates_out counts reliable updates, iters_out CG steps.
 */
int oracle_refine_reliable(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val,
                           const double* b, double* x, double tol, double delta, int max_iter,
                           int storage, int* updates_out, int* iters_out, double* true_relres_out) {
    int64_t nnz = rowptr[n];
    double* s = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* t = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    float* bv = (float*)malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
    float* w = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    float* ri = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    float* p = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    float* q = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    int status = 1, updates = 0, iters = 0;
    double relres = 0.0, bnorm, rho, m, c, prev;
    diagonal(n, rowptr, colind, val, t);
    for (int64_t i = 0; i < n; ++i) {
        if (!(t[i] > 0.0)) { status = 2; goto done; }
        s[i] = 1.0 / sqrt(t[i]);
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            float f = (float)(s[i] * val[k] * s[colind[k]]);
            bv[k] = storage == 1 ? round_bf16(f) : f;
        }
    bnorm = sqrt(dot(n, b, b));
    if (bnorm == 0.0) {
        for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
        status = 0;
        goto done;
    }
    /* true residual, scaled and rounded: the start and every reliable update */
    oracle_csr_spmv(n, rowptr, colind, val, x, t);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - t[i];
    relres = sqrt(dot(n, r, r)) / bnorm;
    if (relres <= tol) { status = 0; goto done; }
    for (int64_t i = 0; i < n; ++i) {
        ri[i] = (float)(s[i] * r[i]);
        w[i] = 0.0f;
        p[i] = ri[i];
    }
    rho = dot_f(n, ri, ri);
    m = sqrt(rho);
    c = relres * bnorm / m;
    prev = relres;
    while (iters < max_iter) {
        spmv_f32(n, rowptr, colind, bv, p, q);
        double pq = dot_f(n, p, q);
        if (!(pq > 0.0) || !isfinite(pq)) { status = 2; goto done; }
        float alpha = (float)(rho / pq);
        for (int64_t i = 0; i < n; ++i) w[i] = w[i] + alpha * p[i];
        for (int64_t i = 0; i < n; ++i) ri[i] = ri[i] - alpha * q[i];
        ++iters;
        double rho_new = dot_f(n, ri, ri);
        if (!isfinite(rho_new)) { status = 2; goto done; }
        if (sqrt(rho_new) <= delta * m || c * sqrt(rho_new) <= tol * bnorm) {
            ++updates;
            for (int64_t i = 0; i < n; ++i) {
                x[i] = x[i] + s[i] * (double)w[i];
                w[i] = 0.0f;
            }
            oracle_csr_spmv(n, rowptr, colind, val, x, t);
            for (int64_t i = 0; i < n; ++i) r[i] = b[i] - t[i];
            relres = sqrt(dot(n, r, r)) / bnorm;
            if (relres <= tol) { status = 0; goto done; }
            if (!(relres < prev)) { status = 2; goto done; }
            prev = relres;
            for (int64_t i = 0; i < n; ++i) ri[i] = (float)(s[i] * r[i]);
            rho_new = dot_f(n, ri, ri);
            m = sqrt(rho_new);
            c = relres * bnorm / m;
        }
        float beta = (float)(rho_new / rho);
        rho = rho_new;
        for (int64_t i = 0; i < n; ++i) p[i] = ri[i] + beta * p[i];
    }
    /* iteration limit: fold in the last correction and report the true residual */
    for (int64_t i = 0; i < n; ++i) x[i] = x[i] + s[i] * (double)w[i];
    oracle_csr_spmv(n, rowptr, colind, val, x, t);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - t[i];
    relres = sqrt(dot(n, r, r)) / bnorm;
    status = relres <= tol ? 0 : 1;
done:
    if (updates_out) *updates_out = updates;
    if (iters_out) *iters_out = iters;
    if (true_relres_out) *true_relres_out = relres;
    free(s); free(r); free(t); free(bv); free(w); free(ri); free(p); free(q);
    return status;
}

/* Position of column j in row i of a CSR with ascending columns, or -1. */
static int64_t csr_find(const int64_t* rowptr, const int32_t* colind, int64_t i, int32_t j) {
    int64_t lo = rowptr[i], hi = rowptr[i + 1] - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (colind[mid] == j) return mid;
        if (colind[mid] < j) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

/*
 * Global values in CSR order from element matrices.  Element e has npe nodes
 * elem_nodes[e * npe + a] and dpn dofs per node (dof = dpn * node + c); its
 * matrix Ke[e] is m x m, m = npe * dpn, row/column dpn * a + c.  For every
 * stored entry (I, J):
 *   values = 0 + Ke[e1](.,.) + Ke[e2](.,.) + ...   over the elements holding both
 *   dofs, in ascending element order;
 * a row with mask[I] set is the identity row (its diagonal 1, nothing else
 * stored), and contributions to entries with a masked row or column are dropped
 * (symmetric elimination of homogeneous Dirichlet conditions; mask may be NULL).
 * Returns 0, or -1 when a contribution to an unmasked entry has no stored
 * position, or a masked row has no diagonal.
 */
int oracle_assemble_matrix(int64_t n, const int64_t* rowptr, const int32_t* colind, int64_t n_elems,
                           int npe, int dpn, const int32_t* elem_nodes, const double* Ke,
                           const uint8_t* mask, double* values) {
    const int m = npe * dpn;
    for (int64_t p = 0; p < rowptr[n]; ++p) values[p] = 0.0;
    for (int64_t e = 0; e < n_elems; ++e)
        for (int a = 0; a < npe; ++a)
            for (int ci = 0; ci < dpn; ++ci) {
                const int64_t I = (int64_t)dpn * elem_nodes[e * npe + a] + ci;
                if (mask && mask[I]) continue;
                for (int b = 0; b < npe; ++b)
                    for (int cj = 0; cj < dpn; ++cj) {
                        const int32_t J = dpn * elem_nodes[e * npe + b] + cj;
                        if (mask && mask[J]) continue;
                        const int64_t p = csr_find(rowptr, colind, I, J);
                        if (p < 0) return -1;
                        values[p] += Ke[e * m * m + (int64_t)(dpn * a + ci) * m + dpn * b + cj];
                    }
            }
    if (mask)
        for (int64_t i = 0; i < n; ++i)
            if (mask[i]) {
                const int64_t p = csr_find(rowptr, colind, i, (int32_t)i);
                if (p < 0) return -1;
                values[p] = 1.0;
            }
    return 0;
}

/*
 * A global vector from element vectors Re[e] (m entries, dpn * a + c):
 *   r_I = 0 + Re[e1](.) + Re[e2](.) + ...   over the elements holding dof I, in
 *   ascending element order; r_I = 0 on masked rows (mask may be NULL).
 */
void oracle_assemble_vector(int64_t n, int64_t n_elems, int npe, int dpn, const int32_t* elem_nodes,
                            const double* Re, const uint8_t* mask, double* r) {
    const int m = npe * dpn;
    for (int64_t i = 0; i < n; ++i) r[i] = 0.0;
    for (int64_t e = 0; e < n_elems; ++e)
        for (int a = 0; a < npe; ++a)
            for (int c = 0; c < dpn; ++c) {
                const int64_t I = (int64_t)dpn * elem_nodes[e * npe + a] + c;
                if (mask && mask[I]) continue;
                r[I] += Re[e * m + dpn * a + c];
            }
}

/*
 * Flexible CG with a low-precision inner CG as the preconditioner.
 *
 * Outer: the flexible conjugate gradient method of Y. Notay, "Flexible conjugate
 * gradients", SIAM J. Sci. Comput. 22 (2000), keeping one previous direction:
 *   x = 0;  r = b
 *   repeat:  z = M_k(r)
 *            p = z                                   (first step)
 *            p = z - (z.q / p.q) p                    (later: A-orthogonal to the last p)
 *            q = A p;  alpha = (p.r) / (p.q)          (p.q <= 0: breakdown)
 *            x += alpha p;  r -= alpha q               (FP64)
 *            stop when ||r|| / ||b|| <= tol, then check the true residual and
 *            restart from x (at most 3 times) as oracle_pcg does
 * Preconditioner M_k: `inner_steps` steps of plain CG on B w = S r from w = 0,
 * B = S A S, S = diag(A)^(-1/2) (fewer if the inner residual vanishes), then
 * z = S w.  storage 0 / 1: B rounded to float / bfloat16 with float vectors
 * and FP64 dot products, the inner arithmetic of oracle_refine; storage 2: B
 * and the inner vectors in FP64 (no rounding of B), for the pins.  The inner
 * CG is a different polynomial in B at every step, so the outer iteration must
 * be flexible.  Returns 0 converged, 1 not converged (max_iter outer steps),
 * 2 breakdown, 3 bad input (non-positive diagonal); iters_out counts outer
 * steps, inner_out inner steps.
 */
int oracle_fcg(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val,
               const double* b, double* x, double tol, int inner_steps, int max_iter, int storage,
               int* iters_out, int* inner_out, double* true_relres_out) {
    const int64_t nnz = rowptr[n];
    const size_t nd = (size_t)(n > 0 ? n : 1);
    double* s = (double*)malloc(sizeof(double) * nd);
    double* r = (double*)malloc(sizeof(double) * nd);
    double* z = (double*)malloc(sizeof(double) * nd);
    double* p = (double*)malloc(sizeof(double) * nd);
    double* q = (double*)malloc(sizeof(double) * nd);
    float* bv = (float*)malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
    double* bd = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    float* wf = (float*)malloc(sizeof(float) * nd);
    float* rf = (float*)malloc(sizeof(float) * nd);
    float* pf = (float*)malloc(sizeof(float) * nd);
    float* qf = (float*)malloc(sizeof(float) * nd);
    double* wd = (double*)malloc(sizeof(double) * nd);
    double* rd = (double*)malloc(sizeof(double) * nd);
    double* pd = (double*)malloc(sizeof(double) * nd);
    double* qd = (double*)malloc(sizeof(double) * nd);
    int status = 1, iters = 0, inner = 0;
    double relres = 0.0, pq_prev = 0.0;
    diagonal(n, rowptr, colind, val, z);
    for (int64_t i = 0; i < n; ++i) {
        if (!(z[i] > 0.0)) { status = 3; goto done; }
        s[i] = 1.0 / sqrt(z[i]);
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            bd[k] = s[i] * val[k] * s[colind[k]];
            float f = (float)bd[k];
            bv[k] = storage == 1 ? round_bf16(f) : f;
        }
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    double bnorm = sqrt(dot(n, b, b));
    if (bnorm == 0.0) { status = 0; goto done; }
    for (int restart = 0; restart <= 3; ++restart) {
        oracle_csr_spmv(n, rowptr, colind, val, x, q);
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
        relres = sqrt(dot(n, r, r)) / bnorm;
        if (relres <= tol) { status = 0; goto done; }
        int converged = 0;
        for (int k = 0; iters < max_iter; ++k) {
            /* z = S w, w = inner_steps CG steps on B w = S r */
            if (storage == 2) {
                for (int64_t i = 0; i < n; ++i) { wd[i] = 0.0; rd[i] = s[i] * r[i]; pd[i] = rd[i]; }
                double rho = dot(n, rd, rd);
                for (int j = 0; j < inner_steps && rho > 0.0; ++j) {
                    oracle_csr_spmv(n, rowptr, colind, bd, pd, qd);
                    double piq = dot(n, pd, qd);
                    if (!(piq > 0.0)) break;
                    double a = rho / piq;
                    for (int64_t i = 0; i < n; ++i) wd[i] = wd[i] + a * pd[i];
                    for (int64_t i = 0; i < n; ++i) rd[i] = rd[i] - a * qd[i];
                    ++inner;
                    double rn = dot(n, rd, rd);
                    double bt = rn / rho;
                    rho = rn;
                    for (int64_t i = 0; i < n; ++i) pd[i] = rd[i] + bt * pd[i];
                }
                for (int64_t i = 0; i < n; ++i) z[i] = s[i] * wd[i];
            } else {
                for (int64_t i = 0; i < n; ++i) { wf[i] = 0.0f; rf[i] = (float)(s[i] * r[i]); pf[i] = rf[i]; }
                double rho = dot_f(n, rf, rf);
                for (int j = 0; j < inner_steps && rho > 0.0; ++j) {
                    spmv_f32(n, rowptr, colind, bv, pf, qf);
                    double piq = dot_f(n, pf, qf);
                    if (!(piq > 0.0)) break;
                    float a = (float)(rho / piq);
                    for (int64_t i = 0; i < n; ++i) wf[i] = wf[i] + a * pf[i];
                    for (int64_t i = 0; i < n; ++i) rf[i] = rf[i] - a * qf[i];
                    ++inner;
                    double rn = dot_f(n, rf, rf);
                    float bt = (float)(rn / rho);
                    rho = rn;
                    for (int64_t i = 0; i < n; ++i) pf[i] = rf[i] + bt * pf[i];
                }
                for (int64_t i = 0; i < n; ++i) z[i] = s[i] * (double)wf[i];
            }
            /* the new direction, A-orthogonal to the previous one */
            if (k == 0) {
                for (int64_t i = 0; i < n; ++i) p[i] = z[i];
            } else {
                double beta = -dot(n, z, q) / pq_prev;
                for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
            }
            oracle_csr_spmv(n, rowptr, colind, val, p, q);
            double pq = dot(n, p, q);
            double pr = dot(n, p, r);
            if (!(pq > 0.0) || !isfinite(pq) || !isfinite(pr)) { status = 2; goto final; }
            double alpha = pr / pq;
            pq_prev = pq;
            for (int64_t i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];
            for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];
            ++iters;
            relres = sqrt(dot(n, r, r)) / bnorm;
            if (!isfinite(relres)) { status = 2; goto final; }
            if (relres <= tol) { converged = 1; break; }
        }
        if (!converged) { status = 1; break; }
        oracle_csr_spmv(n, rowptr, colind, val, x, q);
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
        relres = sqrt(dot(n, r, r)) / bnorm;
        if (relres <= tol) { status = 0; goto done; }
    }
final:
    oracle_csr_spmv(n, rowptr, colind, val, x, q);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    relres = bnorm > 0 ? sqrt(dot(n, r, r)) / bnorm : 0.0;
done:
    if (iters_out) *iters_out = iters;
    if (inner_out) *inner_out = inner;
    if (true_relres_out) *true_relres_out = relres;
    free(s); free(r); free(z); free(p); free(q); free(bv); free(bd);
    free(wf); free(rf); free(pf); free(qf); free(wd); free(rd); free(pd); free(qd);
    return status;
}
