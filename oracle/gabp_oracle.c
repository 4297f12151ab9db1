/*
 * CPU FP64 oracle for Gaussian belief propagation on rank-1 factor graphs.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference the CUDA path is
 * checked against.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * may load it.  It shares no code, header or constant with the CUDA library.
 *
 * A factor f is exp(-(s_f / 2) (a_f . x_f - r_f)^2) over the k_f variables x_f: a
 * rank-1 Gaussian with precision s a a^T and information s r a.  The prior of the paper
 * (Sec. 3.1, "Derivation of the Factor Graph": P = gamma L^T L) is the sum over cells of
 * such factors with a = row i of L; an observation y with noise variance sigma^2 and
 * observation row h is the factor with a = h, s = 1/sigma^2, r = y (Sec. 3.2,
 * "Including Observations", generalised from the nodewise form to a row of H).
 *
 * Message passing follows the paper's loopy belief propagation (App. A, Eqs. for the
 * variable-to-factor and factor-to-variable messages and the state update), in
 * information form: each factor-to-variable message is a pair (eta, Lambda) meaning
 * exp(-Lambda x^2 / 2 + eta x).  One synchronous ("flooding") iteration (Alg. 2,
 * "Iterate MP Until Convergence") computes every new message from the previous
 * iteration's messages only, then damps it (Sec. 3.2 "Update Damping"; here beta is the
 * weight on the OLD message, so the paper's learning rate eta corresponds to 1 - beta).
 *
 * Every function is written for clarity, not speed: loops in the paper's order, leave-one-
 * out sums computed directly, no blocking or fusion.  The factor loop carries an OpenMP
 * pragma because every factor of a synchronous iteration is independent (Alg. 1 note that
 * the inner loops are independent); the result does not depend on the thread count.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_NOTPD 2
#define ORC_ERR_OOM 3

int orc_version(void) { return 1; }

/*
 * Factor-to-variable messages of one rank-1 factor (App. A, factor-to-variable message,
 * generalised from the pairwise Eq. for a_ij, b_ij to k variables).
 *
 * Inputs, per slot u = 0..k-1: the coefficient a[u], and the cavity (variable-to-factor)
 * message of variable u, given as precision lam_c[u] and information eta_c[u]
 * (App. A, variable-to-factor update: the product of all other incoming messages).
 *
 * For target slot v, integrating the factor against the cavities of the other slots
 * gives a Gaussian in x_v with
 *     V_v = 1/s + sum_{u != v} a_u^2 / lam_c[u]          (variance of a_v x_v - r given the rest)
 *     m_v = r - sum_{u != v} a_u * eta_c[u] / lam_c[u]  (its mean)
 *     Lambda_out[v] = a_v^2 / V_v,   eta_out[v] = a_v * m_v / V_v.
 * Slots with a_u = 0 are skipped.
 *
 * A cavity of (near) zero precision.  Away from the observations the precision recursion
 * drives some cavity precisions geometrically towards zero while their information stays
 * finite: the cavity tends to the linear potential exp(eta_u x_u).  Integrating the factor
 * against it over x_u (substitute z = a_u x_u + sum_{w != u} a_w x_w - r) leaves
 * exp(-(eta_u / a_u) sum_{w != u} a_w x_w) up to a constant, so the message to every other
 * slot v tends to (eta, Lambda) = (-a_v eta_u / a_u, 0), and the formulas above converge to
 * it as lam_c[u] -> 0 (the difference is of relative order lam_c[u] V / a_u^2).  A cavity
 * precision below 1e-20 a_u^2 (zero and negative included) is raised to 1e-20 a_u^2: the
 * messages are then that limit to a relative 1e-20 V, and no term overflows.  With several
 * such slots in one factor the messages to the others are the limit along the path where
 * their precisions shrink in proportion to a_u^2.
 */
#define ORC_LAM_FLOOR 1e-20

void orc_factor_update(int k, const double *a, double s, double r, const double *lam_c,
                       const double *eta_c, double *lam_out, double *eta_out) {
    for (int v = 0; v < k; ++v) {
        double V = 1.0 / s;
        double mv = r;
        for (int u = 0; u < k; ++u) {
            if (u == v || a[u] == 0.0) continue;
            const double floor_u = ORC_LAM_FLOOR * (a[u] * a[u]);
            const double lam = lam_c[u] >= floor_u ? lam_c[u] : floor_u;
            V += a[u] * a[u] / lam;
            mv -= a[u] * (eta_c[u] / lam);
        }
        lam_out[v] = a[v] * a[v] / V;
        eta_out[v] = a[v] * mv / V;
    }
}

/* Beliefs (App. A, state update): Lambda_v = sum of incoming Lambda, eta_v = sum of incoming
 * eta, summed slot by slot in the factor list order. */
void orc_beliefs(int64_t n, int64_t nf, const int64_t *ptr, const int64_t *var,
                 const double *msg_eta, const double *msg_lam, double *bel_eta, double *bel_lam) {
    for (int64_t i = 0; i < n; ++i) { bel_eta[i] = 0.0; bel_lam[i] = 0.0; }
    for (int64_t f = 0; f < nf; ++f)
        for (int64_t j = ptr[f]; j < ptr[f + 1]; ++j) {
            bel_eta[var[j]] += msg_eta[j];
            bel_lam[var[j]] += msg_lam[j];
        }
}

/* Number of factor slots touching each variable. */
void orc_degrees(int64_t n, int64_t nf, const int64_t *ptr, const int64_t *var, int64_t *deg) {
    for (int64_t i = 0; i < n; ++i) deg[i] = 0;
    for (int64_t f = 0; f < nf; ++f)
        for (int64_t j = ptr[f]; j < ptr[f + 1]; ++j) deg[var[j]] += 1;
}

/*
 * Initial messages.
 *   mode 0 (cold):  Lambda = s a_v^2 (the factor's own diagonal entry), eta = 0
 *   mode 1 (paper): Lambda = 1e-8, eta = 0 (Alg. 1 / Alg. 2 initialisation read as a small
 *                   precision with zero information)
 *   mode 2 (warm):  given beliefs (mu0, lam0) per variable: Lambda = lam0_v / deg(v),
 *                   eta = mu0_v * Lambda, so that the initial beliefs equal (mu0, lam0).
 */
int orc_init_messages(int mode, int64_t n, int64_t nf, const int64_t *ptr, const int64_t *var,
                      const double *coef, const double *s, const double *mu0, const double *lam0,
                      double *msg_eta, double *msg_lam) {
    int64_t *deg = NULL;
    if (mode == 2) {
        deg = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        if (!deg) return ORC_ERR_OOM;
        orc_degrees(n, nf, ptr, var, deg);
    }
    for (int64_t f = 0; f < nf; ++f)
        for (int64_t j = ptr[f]; j < ptr[f + 1]; ++j) {
            if (mode == 0) {
                msg_lam[j] = s[f] * coef[j] * coef[j];
                msg_eta[j] = 0.0;
            } else if (mode == 1) {
                msg_lam[j] = 1e-8;
                msg_eta[j] = 0.0;
            } else if (mode == 2) {
                msg_lam[j] = lam0[var[j]] / (double)deg[var[j]];
                msg_eta[j] = mu0[var[j]] * msg_lam[j];
            } else {
                free(deg);
                return ORC_ERR_ARG;
            }
        }
    free(deg);
    return ORC_OK;
}

/* Variable -> slot lists (CSR): for variable i, the slots j with var[j] == i, in slot order. */
static int build_node_slots(int64_t n, int64_t nf, const int64_t *ptr, const int64_t *var,
                            int64_t **nptr_out, int64_t **nslot_out) {
    int64_t ne = ptr[nf];
    int64_t *nptr = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
    int64_t *nslot = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ne > 0 ? ne : 1));
    int64_t *fill = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    if (!nptr || !nslot || !fill) { free(nptr); free(nslot); free(fill); return ORC_ERR_OOM; }
    for (int64_t j = 0; j < ne; ++j) nptr[var[j] + 1] += 1;
    for (int64_t i = 0; i < n; ++i) nptr[i + 1] += nptr[i];
    for (int64_t j = 0; j < ne; ++j) {
        int64_t i = var[j];
        nslot[nptr[i] + fill[i]] = j;
        fill[i] += 1;
    }
    free(fill);
    *nptr_out = nptr;
    *nslot_out = nslot;
    return ORC_OK;
}

/*
 * New damped messages of factor f from the old messages: the cavity of each slot j = (f, x_u)
 * is the product of every message into x_u except the one from f (App. A, variable-to-factor
 * message), summed directly over the other slots in slot order; then the factor-to-variable
 * messages and damping.  msg_* are read, out_* written (distinct buffers); beta = weight on
 * the old message.
 */
static void factor_step(int64_t f, const int64_t *ptr, const int64_t *var, const double *coef,
                        const double *s, const double *r, double beta, const int64_t *nptr,
                        const int64_t *nslot, const double *msg_eta, const double *msg_lam,
                        double *out_eta, double *out_lam) {
    double lam_c[64], eta_c[64], lam_h[64], eta_h[64];
    int k = (int)(ptr[f + 1] - ptr[f]);
    const int64_t j0 = ptr[f];
    for (int u = 0; u < k; ++u) {
        const int64_t j = j0 + u, i = var[j];
        double lc = 0.0, ec = 0.0;
        for (int64_t q = nptr[i]; q < nptr[i + 1]; ++q) {
            if (nslot[q] == j) continue;
            lc += msg_lam[nslot[q]];
            ec += msg_eta[nslot[q]];
        }
        lam_c[u] = lc;
        eta_c[u] = ec;
    }
    orc_factor_update(k, coef + j0, s[f], r[f], lam_c, eta_c, lam_h, eta_h);
    for (int u = 0; u < k; ++u) {
        out_lam[j0 + u] = beta * msg_lam[j0 + u] + (1.0 - beta) * lam_h[u];
        out_eta[j0 + u] = beta * msg_eta[j0 + u] + (1.0 - beta) * eta_h[u];
    }
}

/* One synchronous damped iteration: new messages of every factor from the old ones only. */
static void one_iteration(int64_t nf, const int64_t *ptr, const int64_t *var,
                          const double *coef, const double *s, const double *r, double beta,
                          const int64_t *nptr, const int64_t *nslot,
                          const double *msg_eta, const double *msg_lam, double *out_eta,
                          double *out_lam) {
#pragma omp parallel for schedule(static)
    for (int64_t f = 0; f < nf; ++f)
        factor_step(f, ptr, var, coef, s, r, beta, nptr, nslot, msg_eta, msg_lam, out_eta, out_lam);
}

/*
 * One synchronous damped iteration of the factors fids[0..nsub) only (a subdomain's factors,
 * Sec. 3.2.1 domain decomposition): the arithmetic of one_iteration, reading msg_* at the slots
 * of the variables those factors touch and writing out_* at their own slots.
 */
int orc_iterate_factors(int64_t n, int64_t nf, const int64_t *ptr, const int64_t *var,
                        const double *coef, const double *s, const double *r, double beta,
                        int64_t nsub, const int64_t *fids, const double *msg_eta,
                        const double *msg_lam, double *out_eta, double *out_lam) {
    if (n < 0 || nf < 0 || nsub < 0) return ORC_ERR_ARG;
    for (int64_t q = 0; q < nsub; ++q) {
        const int64_t f = fids[q];
        if (f < 0 || f >= nf || ptr[f + 1] - ptr[f] > 64 || ptr[f + 1] < ptr[f] || !(s[f] > 0.0))
            return ORC_ERR_ARG;
    }
    int64_t *nptr = NULL, *nslot = NULL;
    if (build_node_slots(n, nf, ptr, var, &nptr, &nslot) != ORC_OK) return ORC_ERR_OOM;
    for (int64_t q = 0; q < nsub; ++q)
        factor_step(fids[q], ptr, var, coef, s, r, beta, nptr, nslot, msg_eta, msg_lam, out_eta, out_lam);
    free(nptr);
    free(nslot);
    return ORC_OK;
}

/*
 * Run `iters` synchronous iterations in place on (msg_eta, msg_lam) and return the final
 * beliefs.  Factors may have at most 64 slots.
 */
int orc_gabp_run(int64_t n, int64_t nf, const int64_t *ptr, const int64_t *var,
                 const double *coef, const double *s, const double *r, double beta, int iters,
                 double *msg_eta, double *msg_lam, double *bel_eta, double *bel_lam) {
    if (n < 0 || nf < 0 || iters < 0) return ORC_ERR_ARG;
    for (int64_t f = 0; f < nf; ++f)
        if (ptr[f + 1] - ptr[f] > 64 || ptr[f + 1] < ptr[f] || !(s[f] > 0.0)) return ORC_ERR_ARG;
    int64_t ne = ptr[nf];
    for (int64_t j = 0; j < ne; ++j)
        if (var[j] < 0 || var[j] >= n) return ORC_ERR_ARG;
    int64_t *nptr = NULL, *nslot = NULL;
    if (build_node_slots(n, nf, ptr, var, &nptr, &nslot) != ORC_OK) return ORC_ERR_OOM;
    double *te = (double *)malloc(sizeof(double) * (size_t)(ne > 0 ? ne : 1));
    double *tl = (double *)malloc(sizeof(double) * (size_t)(ne > 0 ? ne : 1));
    if (!te || !tl) { free(te); free(tl); free(nptr); free(nslot); return ORC_ERR_OOM; }
    for (int t = 0; t < iters; ++t) {
        one_iteration(nf, ptr, var, coef, s, r, beta, nptr, nslot, msg_eta, msg_lam, te, tl);
        memcpy(msg_eta, te, sizeof(double) * (size_t)ne);
        memcpy(msg_lam, tl, sizeof(double) * (size_t)ne);
    }
    orc_beliefs(n, nf, ptr, var, msg_eta, msg_lam, bel_eta, bel_lam);
    free(te);
    free(tl);
    free(nptr);
    free(nslot);
    return ORC_OK;
}

/* out = A x with A = sum_f s_f a_f a_f^T (the posterior precision: prior plus H^T R^-1 H). */
void orc_apply_A(int64_t n, int64_t nf, const int64_t *ptr, const int64_t *var,
                 const double *coef, const double *s, const double *x, double *out) {
    for (int64_t i = 0; i < n; ++i) out[i] = 0.0;
    for (int64_t f = 0; f < nf; ++f) {
        double dot = 0.0;
        for (int64_t j = ptr[f]; j < ptr[f + 1]; ++j) dot += coef[j] * x[var[j]];
        for (int64_t j = ptr[f]; j < ptr[f + 1]; ++j) out[var[j]] += s[f] * coef[j] * dot;
    }
}

/* out = b with b = sum_f s_f r_f a_f (the posterior information vector H^T R^-1 y). */
void orc_rhs(int64_t n, int64_t nf, const int64_t *ptr, const int64_t *var, const double *coef,
             const double *s, const double *r, double *out) {
    for (int64_t i = 0; i < n; ++i) out[i] = 0.0;
    for (int64_t f = 0; f < nf; ++f)
        for (int64_t j = ptr[f]; j < ptr[f + 1]; ++j) out[var[j]] += s[f] * r[f] * coef[j];
}

/*
 * Banded Cholesky of A = sum_f s_f a_f a_f^T in the natural (row-major) ordering.  `bw` is the
 * half bandwidth; every pair of variables sharing a factor must be within bw of each other
 * (checked).  Band storage: B[i*(bw+1) + d] holds A[i][i-d] for d = 0..bw (lower band); on
 * success it holds the lower Cholesky factor G (A = G G^T) in the same places.
 */
static int band_assemble(int64_t n, int64_t nf, const int64_t *ptr, const int64_t *var,
                         const double *coef, const double *s, int64_t bw, double *B) {
    const int64_t w = bw + 1;
    for (int64_t f = 0; f < nf; ++f)
        for (int64_t p = ptr[f]; p < ptr[f + 1]; ++p)
            for (int64_t q = ptr[f]; q < ptr[f + 1]; ++q) {
                int64_t i = var[p], j = var[q];
                if (j > i) continue;
                if (i - j > bw) return ORC_ERR_ARG;
                B[i * w + (i - j)] += s[f] * coef[p] * coef[q];
            }
    return ORC_OK;
}

static int band_cholesky(int64_t n, int64_t bw, double *B) {
    const int64_t w = bw + 1;
    for (int64_t i = 0; i < n; ++i) {
        int64_t jlo = i - bw > 0 ? i - bw : 0;
        for (int64_t j = jlo; j <= i; ++j) {
            double sum = B[i * w + (i - j)];
            int64_t klo = (i - bw > j - bw ? i - bw : j - bw);
            if (klo < 0) klo = 0;
            for (int64_t k = klo; k < j; ++k) sum -= B[i * w + (i - k)] * B[j * w + (j - k)];
            if (j == i) {
                if (!(sum > 0.0)) return ORC_ERR_NOTPD;
                B[i * w] = sqrt(sum);
            } else {
                B[i * w + (i - j)] = sum / B[j * w];
            }
        }
    }
    return ORC_OK;
}

/* Exact posterior mean: solve A x = b by the banded Cholesky above, then the two triangular
 * solves.  The solution overwrites b. */
int orc_band_solve(int64_t n, int64_t nf, const int64_t *ptr, const int64_t *var,
                   const double *coef, const double *s, int64_t bw, double *b) {
    if (bw < 0 || n <= 0) return ORC_ERR_ARG;
    const int64_t w = bw + 1;
    double *B = (double *)calloc((size_t)(n * w), sizeof(double));
    if (!B) return ORC_ERR_OOM;
    int rc = band_assemble(n, nf, ptr, var, coef, s, bw, B);
    if (rc == ORC_OK) rc = band_cholesky(n, bw, B);
    if (rc != ORC_OK) { free(B); return rc; }
    /* forward: G z = b */
    for (int64_t i = 0; i < n; ++i) {
        double sum = b[i];
        int64_t klo = i - bw > 0 ? i - bw : 0;
        for (int64_t k = klo; k < i; ++k) sum -= B[i * w + (i - k)] * b[k];
        b[i] = sum / B[i * w];
    }
    /* backward: G^T x = z */
    for (int64_t i = n - 1; i >= 0; --i) {
        double sum = b[i];
        int64_t khi = i + bw < n - 1 ? i + bw : n - 1;
        for (int64_t k = i + 1; k <= khi; ++k) sum -= B[k * w + (k - i)] * b[k];
        b[i] = sum / B[i * w];
    }
    free(B);
    return ORC_OK;
}

/*
 * Exact marginal variances diag(A^-1) by selected inversion on the band (Takahashi, Fagan and
 * Chen's recurrences, in the Cholesky form used for GMRFs).  With A = G G^T (G lower, band bw),
 * S = A^-1 satisfies S G = G^-T; reading off the entries on and above the diagonal gives, for
 * j >= i,
 *     S_ij = delta_ij / G_ii^2 - (1 / G_ii) sum_{k = i+1..i+bw} G_ki S_kj,
 * and every S_kj it needs has |k - j| <= bw, so the band of S is closed under the recurrence:
 * rows are taken from the last to the first, and in each row j from the band's edge down to i.
 * var_out[i] = S_ii.  Costs n bw^2 multiply-adds and two n x (bw+1) arrays.
 */
int orc_band_selinv(int64_t n, int64_t nf, const int64_t *ptr, const int64_t *var,
                    const double *coef, const double *s, int64_t bw, double *var_out) {
    if (bw < 0 || n <= 0) return ORC_ERR_ARG;
    const int64_t w = bw + 1;
    double *B = (double *)calloc((size_t)(n * w), sizeof(double));
    double *S = (double *)calloc((size_t)(n * w), sizeof(double));   /* S[a*w + (a-b)] = S_ab, a >= b */
    if (!B || !S) { free(B); free(S); return ORC_ERR_OOM; }
    int rc = band_assemble(n, nf, ptr, var, coef, s, bw, B);
    if (rc == ORC_OK) rc = band_cholesky(n, bw, B);
    if (rc != ORC_OK) { free(B); free(S); return rc; }
    for (int64_t i = n - 1; i >= 0; --i) {
        const int64_t khi = i + bw < n - 1 ? i + bw : n - 1;
        const double gii = B[i * w];
        for (int64_t j = khi; j >= i; --j) {
            double sum = 0.0;
            for (int64_t k = i + 1; k <= khi; ++k) {
                const double gki = B[k * w + (k - i)];
                const double skj = k >= j ? S[k * w + (k - j)] : S[j * w + (j - k)];
                sum += gki * skj;
            }
            const double sij = ((j == i ? 1.0 / gii : 0.0) - sum) / gii;
            S[j * w + (j - i)] = sij;
        }
        var_out[i] = S[i * w];
    }
    free(B);
    free(S);
    return ORC_OK;
}

/*
 * The posterior precision A = sum_f s_f a_f a_f^T as a CSR matrix with sorted column indices
 * (the fine level of the iterative exact solve).  Pass rp = NULL to get only the row lengths:
 * then row_len[i] = number of distinct columns of row i.  With rp given (rp[i+1] - rp[i] =
 * row_len[i]), the columns and values of each row are written.  Rows are independent; entries
 * are summed factor by factor in factor-list order.
 */
int orc_assemble_csr(int64_t n, int64_t nf, const int64_t *ptr, const int64_t *var,
                     const double *coef, const double *s, int64_t *row_len, const int64_t *rp,
                     int64_t *ci, double *val) {
    int64_t *nptr = NULL, *nslot = NULL, *fac = NULL;
    if (n < 0 || nf < 0) return ORC_ERR_ARG;
    if (build_node_slots(n, nf, ptr, var, &nptr, &nslot) != ORC_OK) return ORC_ERR_OOM;
    /* factor of each slot */
    const int64_t ne = ptr[nf];
    fac = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ne > 0 ? ne : 1));
    if (!fac) { free(nptr); free(nslot); return ORC_ERR_OOM; }
    for (int64_t f = 0; f < nf; ++f)
        for (int64_t j = ptr[f]; j < ptr[f + 1]; ++j) fac[j] = f;
    int err = 0;
#pragma omp parallel reduction(| : err)
    {
        int64_t cols[512];
        double vals[512];
#pragma omp for schedule(dynamic, 4096)
        for (int64_t i = 0; i < n; ++i) {
            int nc = 0;
            for (int64_t q = nptr[i]; q < nptr[i + 1] && !err; ++q) {
                const int64_t jslot = nslot[q], f = fac[jslot];
                for (int64_t p = ptr[f]; p < ptr[f + 1]; ++p) {
                    const int64_t c = var[p];
                    const double a = s[f] * coef[jslot] * coef[p];
                    int t = 0;
                    while (t < nc && cols[t] != c) ++t;
                    if (t == nc) {
                        if (nc == 512) { err = 1; break; }
                        cols[nc] = c;
                        vals[nc] = 0.0;
                        ++nc;
                    }
                    vals[t] += a;
                }
            }
            if (!rp) {
                row_len[i] = nc;
                continue;
            }
            /* insertion sort by column */
            for (int a = 1; a < nc; ++a) {
                int64_t c = cols[a];
                double v = vals[a];
                int b = a - 1;
                while (b >= 0 && cols[b] > c) { cols[b + 1] = cols[b]; vals[b + 1] = vals[b]; --b; }
                cols[b + 1] = c;
                vals[b + 1] = v;
            }
            if (rp[i + 1] - rp[i] != nc) { err = 1; continue; }
            for (int a = 0; a < nc; ++a) { ci[rp[i] + a] = cols[a]; val[rp[i] + a] = vals[a]; }
        }
    }
    free(fac);
    free(nptr);
    free(nslot);
    return err ? ORC_ERR_ARG : ORC_OK;
}

/*
 * `sweeps` Gauss-Seidel sweeps on M x = b for a CSR matrix M (the smoother of the multigrid
 * preconditioner): row by row, x_i = (b_i - sum_{j != i} M_ij x_j) / M_ii with the newest x_j,
 * rows in increasing order (backward = 0) or decreasing order (backward = 1).  A forward sweep
 * before the coarse correction and a backward sweep after it make the V-cycle symmetric.
 */
int orc_gs_sweep(int64_t n, const int64_t *rp, const int64_t *ci, const double *val,
                 const double *b, double *x, int backward, int sweeps) {
    for (int t = 0; t < sweeps; ++t)
        for (int64_t ii = 0; ii < n; ++ii) {
            const int64_t i = backward ? n - 1 - ii : ii;
            double d = 0.0, sum = b[i];
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
                if (ci[p] == i) d = val[p];
                else sum -= val[p] * x[ci[p]];
            }
            if (!(d > 0.0)) return ORC_ERR_NOTPD;
            x[i] = sum / d;
        }
    return ORC_OK;
}
