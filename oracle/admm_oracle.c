/*
 * FP64 reference ("oracle") for ADMM LP decoding -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously-correct CPU code written from the paper
 * "Decomposition Methods for Large Scale LP Decoding" (Barman, Liu, Draper,
 * Recht).  Only the test suite, the package smoke check and the benchmark's
 * CPU-baseline leg may load this library; the product (liblpdec) never does,
 * and the two share no code, headers or tables.
 *
 *   oracle_project         Euclidean projection onto the parity polytope PP_d,
 *                          Algorithm 2 (Section 4.4) in the paper's order.
 *   oracle_project_bisect  The same projection by a second route: bisection on
 *                          f_r^T z(beta) = r (Lemma 4 and eq. (derivative)).
 *   oracle_decode          Algorithm 1 (Section 3.3) over a batch of frames, with
 *                          the over-relaxation of Section 5.2.
 *
 * All arithmetic is double precision.  Readings taken where the paper is
 * silent or garbled:
 *   - Algorithm 2's final else-branch is garbled.  Instead of it, the bracket
 *     [beta_i, beta_{i+1}] of consecutive breakpoints with g(beta_i) > r >=
 *     g(beta_{i+1}) is located on the FULL breakpoint set E1, L1, E2, L2, 0 and
 *     beta_max, and beta_opt is solved from eq. (find-beta) on that piece, where
 *     g(beta) = |C| - beta|A| + sum_{k in A} f_k v_k.
 *   - Over-relaxation (Section 5.2 cites Boyd et al. Sec. 3.4.3 without a
 *     formula): P_j x is replaced by q = rho P_j x + (1 - rho) z_j^old in both
 *     the z- and the lambda-update.  rho = 1 is Algorithm 1 exactly.
 *   - Stopping constant eps^2 M d is taken as eps^2 E (E = number of edges; the
 *     same for regular codes).  eps = 0 disables the test (fixed iterations).
 *   - iters = number of completed sweeps when the test first passes.
 *   - certificate = (residual test passes at the final iterate with
 *     eps_c = max(eps, 1e-5)) AND (max_i min(x_i, 1 - x_i) <= cert_tol) AND
 *     (the rounded word satisfies every check).
 *   - Hard decision b_i = [x_i > 1/2] (Section 5.1 rounds non-integer output).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_MAX_D 64

static double clip01(double a) { return a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a); }

/* Stable sort of indices so that u[idx[0]] >= u[idx[1]] >= ... (ties keep the
 * lower index first).  Insertion sort: d is small. */
static void sort_desc_idx(int d, const double *u, int *idx)
{
    for (int k = 0; k < d; ++k) idx[k] = k;
    for (int k = 1; k < d; ++k) {
        int t = idx[k];
        int p = k - 1;
        while (p >= 0 && u[idx[p]] < u[t]) { idx[p + 1] = idx[p]; --p; }
        idx[p + 1] = t;
    }
}

/* f_r(k) for the sorted vector: +1 on the first r+1 entries, -1 after, eq. (fr-def). */
static double f_r(int k, int r) { return k <= r ? 1.0 : -1.0; }

/* g(beta) = f_r^T Pi_[0,1](v - beta f_r), eq. (def.zProj), v sorted descending. */
static double g_of_beta(int d, const double *v, int r, double beta)
{
    double s = 0.0;
    for (int k = 0; k < d; ++k) s += f_r(k, r) * clip01(v[k] - beta * f_r(k, r));
    return s;
}

static void sort_asc(int n, double *a)
{
    for (int k = 1; k < n; ++k) {
        double t = a[k];
        int p = k - 1;
        while (p >= 0 && a[p] > t) { a[p + 1] = a[p]; --p; }
        a[p + 1] = t;
    }
}

/* Steps shared by both projection routes: Algorithm 2 up to the breakpoint search.
 * Returns 1 when the projection is zhat (written to z in the original order),
 * 0 when beta_opt must still be found; v, q, r and beta_max are filled. */
static int project_prefix(int d, const double *u, double *z, double *v, int *q,
                          int *r_out, double *beta_max_out)
{
    /* sort descending, v = Q u (q[k] = original index of v[k]) */
    sort_desc_idx(d, u, q);
    for (int k = 0; k < d; ++k) v[k] = u[q[k]];
    /* zhat = Pi_[0,1](v) */
    double zhat[ORACLE_MAX_D];
    double s = 0.0;
    for (int k = 0; k < d; ++k) { zhat[k] = clip01(v[k]); s += zhat[k]; }
    /* r = even floor of ||zhat||_1 (the constituent parity, Lemma 3) */
    int r = 2 * (int)floor(s / 2.0);
    if (r > d) r = d - (d & 1); /* guard against rounding; s <= d always */
    *r_out = r;
    /* r = d: zhat is the projection */
    if (r == d) {
        for (int k = 0; k < d; ++k) z[q[k]] = zhat[k];
        return 1;
    }
    /* beta_max (Lemma 4); the 1-based v_{r+1}, v_{r+2} are v[r], v[r+1] here */
    *beta_max_out = (r <= d - 2) ? 0.5 * (v[r] - v[r + 1]) : v[r];
    /* f_r^T zhat <= r  ->  zhat is the projection (eq. (fr-def), Lemma 4) */
    double g0 = 0.0;
    for (int k = 0; k < d; ++k) g0 += f_r(k, r) * zhat[k];
    if (g0 <= (double)r) {
        for (int k = 0; k < d; ++k) z[q[k]] = zhat[k];
        return 1;
    }
    return 0;
}

/* Algorithm 2.  Returns 0 on success, -1 if d is out of range. */
int oracle_project(int d, const double *u, double *z)
{
    if (d < 1 || d > ORACLE_MAX_D) return -1;
    double v[ORACLE_MAX_D];
    int q[ORACLE_MAX_D];
    int r;
    double beta_max = 0.0;
    if (project_prefix(d, u, z, v, q, &r, &beta_max)) return 0;

    /* Breakpoints where an entry of z(beta) enters or leaves (0,1): the sets
     * E1 = {v_i - 1}, L1 = {v_i} (i <= r+1) and E2 = {-v_i}, L2 = {1 - v_i}
     * (i >= r+2), restricted to [0, beta_max], plus 0 and beta_max. */
    double bp[4 * ORACLE_MAX_D + 2];
    int nb = 0;
    bp[nb++] = 0.0;
    bp[nb++] = beta_max;
    for (int k = 0; k < d; ++k) {
        double c1, c2;
        if (k <= r) { c1 = v[k] - 1.0; c2 = v[k]; }
        else        { c1 = -v[k];      c2 = 1.0 - v[k]; }
        if (c1 > 0.0 && c1 < beta_max) bp[nb++] = c1;
        if (c2 > 0.0 && c2 < beta_max) bp[nb++] = c2;
    }
    sort_asc(nb, bp);

    /* march: g is continuous and nonincreasing (eq. (derivative)); g(0) > r and
     * g(beta_max) <= r (Lemma 4).  Find the first breakpoint with g <= r. */
    int i = 1;
    while (i < nb - 1 && g_of_beta(d, v, r, bp[i]) > (double)r) ++i;
    double lo = bp[i - 1], hi = bp[i];

    /* eq. (find-beta) on the open piece (lo, hi): the active set A and clipped
     * set C are constant there; read them at the midpoint. */
    double mid = 0.5 * (lo + hi);
    int nA = 0, nC = 0;
    double sumA = 0.0;
    for (int k = 0; k < d; ++k) {
        double t = v[k] - mid * f_r(k, r);
        if (t >= 1.0) { if (f_r(k, r) > 0) ++nC; else --nC; }  /* clipped at 1 */
        else if (t > 0.0) { ++nA; sumA += f_r(k, r) * v[k]; }
    }
    double beta;
    if (nA == 0) beta = hi; /* g constant on the piece: only possible if g(hi) == r */
    else beta = ((double)nC + sumA - (double)r) / (double)nA;
    if (beta < lo) beta = lo;
    if (beta > hi) beta = hi;

    /* return z* = Q^T Pi_[0,1](v - beta_opt f_r) */
    for (int k = 0; k < d; ++k) z[q[k]] = clip01(v[k] - beta * f_r(k, r));
    return 0;
}

/* Second route: bisection for f_r^T z(beta) = r on [0, beta_max]. */
int oracle_project_bisect(int d, const double *u, double *z)
{
    if (d < 1 || d > ORACLE_MAX_D) return -1;
    double v[ORACLE_MAX_D];
    int q[ORACLE_MAX_D];
    int r;
    double beta_max = 0.0;
    if (project_prefix(d, u, z, v, q, &r, &beta_max)) return 0;
    double lo = 0.0, hi = beta_max;
    for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (g_of_beta(d, v, r, mid) > (double)r) lo = mid; else hi = mid;
    }
    double beta = 0.5 * (lo + hi);
    for (int k = 0; k < d; ++k) z[q[k]] = clip01(v[k] - beta * f_r(k, r));
    return 0;
}

/* Project many vectors of one degree: v and z are [count x d] row-major. */
int oracle_project_many(int d, int64_t count, const double *v, double *z, int use_bisect)
{
    for (int64_t t = 0; t < count; ++t) {
        int rc = use_bisect ? oracle_project_bisect(d, v + t * d, z + t * d)
                            : oracle_project(d, v + t * d, z + t * d);
        if (rc) return rc;
    }
    return 0;
}

/*
 * Algorithm 1 for frames [f_lo, f_hi) of a batch.
 *
 * H is given by rows (CSR): the edges of check j are e = row_ptr[j] ..
 * row_ptr[j+1]-1, variable col_idx[e]; the k-th of them is the k-th row of P_j.
 * gamma is [n_frames x n]; per-frame outputs are indexed by frame number.
 * resid_out (may be NULL) receives, per frame, the primal and dual residuals
 * of Section 3.3 after the last iteration run: sum_j ||P_j x - z_j||^2 and
 * sum_j ||z_j - z_j_old||^2.
 * Returns 0, or -1 on a bad argument / allocation failure.
 */
int oracle_decode(int n, int m, const int32_t *row_ptr, const int32_t *col_idx,
                  int f_lo, int f_hi, const double *gamma,
                  double mu, double rho, double eps, int max_iter, double cert_tol,
                  double *x_out, uint8_t *bits_out, int32_t *iters_out,
                  uint8_t *conv_out, uint8_t *cert_out, double *resid_out)
{
    if (n <= 0 || m <= 0 || mu <= 0.0 || max_iter < 1) return -1;
    const int E = row_ptr[m];
    double *z = (double *)malloc(sizeof(double) * (size_t)E);
    double *lam = (double *)malloc(sizeof(double) * (size_t)E);
    double *acc = (double *)malloc(sizeof(double) * (size_t)n);
    double *deg = (double *)malloc(sizeof(double) * (size_t)n);
    double *x = (double *)malloc(sizeof(double) * (size_t)n);
    if (!z || !lam || !acc || !deg || !x) {
        free(z); free(lam); free(acc); free(deg); free(x);
        return -1;
    }
    /* |N_v(i)|: the diagonal of P = sum_j P_j^T P_j (Section 3.2) */
    for (int i = 0; i < n; ++i) deg[i] = 0.0;
    for (int e = 0; e < E; ++e) deg[col_idx[e]] += 1.0;

    const double eps_c = eps > 1e-5 ? eps : 1e-5;
    for (int f = f_lo; f < f_hi; ++f) {
        const double *g = gamma + (size_t)f * (size_t)n;
        /* Algorithm 1 initialization: z_j = lambda_j = 0 */
        for (int e = 0; e < E; ++e) { z[e] = 0.0; lam[e] = 0.0; }
        int k = 0, converged = 0;
        double Rp = 0.0, Rd = 0.0;
        while (k < max_iter) {
            /* x-update (Section 3.2): x_i = Pi_[0,1]( (sum_{j in N_v(i)} (z_j^(i) - lambda_j^(i)/mu)
             *                            - gamma_i/mu) / |N_v(i)| ) */
            for (int i = 0; i < n; ++i) acc[i] = 0.0;
            for (int e = 0; e < E; ++e) acc[col_idx[e]] += z[e] - lam[e] / mu;
            for (int i = 0; i < n; ++i) x[i] = clip01((acc[i] - g[i] / mu) / deg[i]);
            /* z- and lambda-updates, over-relaxed (Section 5.2): for each check j */
            Rp = 0.0;
            Rd = 0.0;
            for (int j = 0; j < m; ++j) {
                const int e0 = row_ptr[j];
                const int d = row_ptr[j + 1] - e0;
                double vj[ORACLE_MAX_D], zj[ORACLE_MAX_D], qj[ORACLE_MAX_D], zold[ORACLE_MAX_D];
                for (int t = 0; t < d; ++t) {
                    zold[t] = z[e0 + t];
                    qj[t] = rho * x[col_idx[e0 + t]] + (1.0 - rho) * zold[t];
                    vj[t] = qj[t] + lam[e0 + t] / mu;      /* v_j = P_j x + lambda_j / mu */
                }
                oracle_project(d, vj, zj);                  /* z_j = Pi_PP(v_j) */
                for (int t = 0; t < d; ++t) {
                    z[e0 + t] = zj[t];
                    lam[e0 + t] += mu * (qj[t] - zj[t]);    /* lambda_j += mu (P_j x - z_j) */
                    const double dp = x[col_idx[e0 + t]] - zj[t];
                    const double dd = zj[t] - zold[t];
                    Rp += dp * dp;
                    Rd += dd * dd;
                }
            }
            ++k;
            /* stopping test (Section 3.3): both residuals below eps^2 E */
            if (eps > 0.0 && Rp < eps * eps * (double)E && Rd < eps * eps * (double)E) {
                converged = 1;
                break;
            }
        }
        /* outputs */
        double *xo = x_out + (size_t)f * (size_t)n;
        uint8_t *bo = bits_out + (size_t)f * (size_t)n;
        double frac = 0.0;
        for (int i = 0; i < n; ++i) {
            xo[i] = x[i];
            bo[i] = x[i] > 0.5 ? 1 : 0;
            double mi = x[i] < 1.0 - x[i] ? x[i] : 1.0 - x[i];
            if (mi > frac) frac = mi;
        }
        int syndrome_ok = 1;
        for (int j = 0; j < m && syndrome_ok; ++j) {
            int par = 0;
            for (int e = row_ptr[j]; e < row_ptr[j + 1]; ++e) par ^= bo[col_idx[e]];
            if (par) syndrome_ok = 0;
        }
        const int resid_ok = Rp < eps_c * eps_c * (double)E && Rd < eps_c * eps_c * (double)E;
        iters_out[f] = k;
        conv_out[f] = (uint8_t)converged;
        if (resid_out) {
            resid_out[2 * (size_t)f] = Rp;
            resid_out[2 * (size_t)f + 1] = Rd;
        }
        cert_out[f] = (uint8_t)(resid_ok && frac <= cert_tol && syndrome_ok);
    }
    free(z); free(lam); free(acc); free(deg); free(x);
    return 0;
}

/*
 * Appendix, Algorithm 3: maximize c^T z over the parity polytope PP_d.  The
 * optimum is an even-weight vertex.  Let r be the number of positive c_i.
 * r even: z = [c > 0].  r odd: either drop the smallest positive entry i_p or
 * add the largest non-positive entry i_n, whichever costs less; that is, add
 * i_n when c_{i_p} + c_{i_n} > 0, else drop i_p.  (The printed comparison of
 * c_{i_p} with c_{i_n} always holds; the appendix's text compares the values
 * of the two even neighbours, sum_pos + c_{i_n} against sum_pos - c_{i_p},
 * which is the test used here.)  Ties pick the lowest index.
 */
int oracle_lp_max(int d, const double *c, double *z)
{
    if (d < 1 || d > ORACLE_MAX_D) return -1;
    int r = 0, ip = -1, in = -1;
    for (int k = 0; k < d; ++k) {
        z[k] = c[k] > 0.0 ? 1.0 : 0.0;
        if (c[k] > 0.0) {
            ++r;
            if (ip < 0 || c[k] < c[ip]) ip = k;
        } else if (in < 0 || c[k] > c[in]) {
            in = k;
        }
    }
    if (r % 2 == 0) return 0;
    if (in >= 0 && c[ip] + c[in] > 0.0) z[in] = 1.0;
    else z[ip] = 0.0;
    return 0;
}

/*
 * Appendix: dual subgradient ascent on the un-augmented Lagrangian
 * L_0 = gamma^T x + sum_j lambda_j^T (P_j x - z_j), for frames [f_lo, f_hi):
 *   x_i = [ -gamma_i - sum_{j in N_v(i)} lambda_j^(i) > 0 ]   (Heaviside)
 *   z_j = argmax_{z in PP_d} lambda_j^T z                      (Algorithm 3)
 *   lambda_j += mu (P_j x - z_j)
 * both updates taken from the previous lambda.  The method stops when the
 * subgradient P_j x - z_j vanishes for every j (then lambda is dual optimal and
 * x an integral LP optimum: the output is certified), else after max_iter.
 */
int oracle_decode_dual(int n, int m, const int32_t *row_ptr, const int32_t *col_idx, int f_lo, int f_hi,
                       const double *gamma, double mu, int max_iter, double *x_out, uint8_t *bits_out,
                       int32_t *iters_out, uint8_t *cert_out)
{
    if (n <= 0 || m <= 0 || mu <= 0.0 || max_iter < 1) return -1;
    const int E = row_ptr[m];
    double *lam = (double *)malloc(sizeof(double) * (size_t)E);
    double *acc = (double *)malloc(sizeof(double) * (size_t)n);
    double *x = (double *)malloc(sizeof(double) * (size_t)n);
    if (!lam || !acc || !x) { free(lam); free(acc); free(x); return -1; }
    for (int f = f_lo; f < f_hi; ++f) {
        const double *g = gamma + (size_t)f * (size_t)n;
        for (int e = 0; e < E; ++e) lam[e] = 0.0;
        int k = 0, done = 0;
        while (k < max_iter && !done) {
            for (int i = 0; i < n; ++i) acc[i] = 0.0;
            for (int e = 0; e < E; ++e) acc[col_idx[e]] += lam[e];
            for (int i = 0; i < n; ++i) x[i] = (-g[i] - acc[i] > 0.0) ? 1.0 : 0.0;
            int mismatches = 0;
            for (int j = 0; j < m; ++j) {
                const int e0 = row_ptr[j], d = row_ptr[j + 1] - e0;
                double zj[ORACLE_MAX_D];
                oracle_lp_max(d, lam + e0, zj);
                for (int t = 0; t < d; ++t) {
                    const double s = x[col_idx[e0 + t]] - zj[t];
                    if (s != 0.0) ++mismatches;
                    lam[e0 + t] += mu * s;
                }
            }
            ++k;
            done = mismatches == 0;
        }
        for (int i = 0; i < n; ++i) {
            x_out[(size_t)f * n + i] = x[i];
            bits_out[(size_t)f * n + i] = x[i] > 0.5 ? 1 : 0;
        }
        iters_out[f] = k;
        cert_out[f] = (uint8_t)done;
    }
    free(lam); free(acc); free(x);
    return 0;
}
