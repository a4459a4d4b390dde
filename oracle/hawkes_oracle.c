/*
 * FP64 CPU oracle for the exact log-likelihood of a multivariate linear
 * exponential Hawkes process and its gradient.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, sequential, obviously
 * correct statement of what the GPU library computes.  It shares no code,
 * header, table or constant with the CUDA library, and the library never
 * calls it.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg load it.
 *
 * Model (paper, Section 2, Eq. hawkes_excitation with one decay kernel per
 * source mark):
 *     lambda_p(t) = mu_p + sum_{l : l before t} alpha[p][c_l] beta_{c_l} exp(-beta_{c_l} (t - t_l))
 * Row p of alpha is the TARGET, column q the SOURCE (the formula of Eq.
 * hawkes_excitation indexes alpha by (target, source mark)).  Marks are
 * 0-based.  A shared decay is the special case beta_j = beta for all j.
 *
 * Log-likelihood (paper, Section 2, Eq. general_hawkes_likelihood):
 *     L = sum_k log lambda_{c_k}(t_k) - sum_m int_0^T lambda_m(t) dt
 * with the closed-form compensator (paper, Section 2, text after the NLL
 * objective, and the second term of Eq. grad_alpha):
 *     int_0^T sum_m lambda_m = T sum_i mu_i
 *                              + sum_l colsum_{c_l} (1 - exp(-beta_{c_l} (T - t_l))),
 *     colsum_j = sum_i alpha[i][j].
 *
 * Source-indexed state (paper, Appendix B, the K recurrence of Eq.
 * alpha_grad_recurrence, here with a per-source decay):
 *     S_1 = 0,  S_k = D_k (S_{k-1} + e_{c_{k-1}}),  D_k = diag(exp(-beta_j (t_k - t_{k-1}))),
 *     lambda_k = mu_{c_k} + sum_j alpha[c_k][j] beta_j S_{k,j}.
 * Ties (t_k == t_{k-1}) follow the recurrence: an earlier-indexed event
 * counts with weight exp(0) = 1.
 *
 * Gradients (paper, Appendix B, Eqs. grad_mu, grad_alpha, grad_gamma):
 *   dL/dmu_i       = sum_{k : c_k = i} w_k - T,                 w_k = 1 / lambda_k
 *   dL/dalpha_ij   = beta_j sum_{k : c_k = i} w_k S_{k,j} - E_j,
 *                    E_j = sum_{l : c_l = j} (1 - exp(-beta_j (T - t_l)))
 *   dL/dbeta_j     = sum_k w_k alpha[c_k][j] (S_{k,j} - beta_j G_{k,j}) - colsum_j F_j,
 *                    F_j = sum_{l : c_l = j} (T - t_l) exp(-beta_j (T - t_l))
 * where G_{k,j} = sum_{l<k, c_l=j} (t_k - t_l) exp(-beta_j (t_k - t_l)) = -dS_{k,j}/dbeta_j
 * obeys G_1 = 0, G_k = D_k (G_{k-1} + dt_k (S_{k-1} + e_{c_{k-1}})).
 * This is Eq. grad_gamma rewritten with a source-indexed state: the paper's
 * (1 - gamma t) R + gamma L equals R - gamma (alpha G); the G form avoids the
 * cancellation of t R against L when t is large.  The paper's own R/L form is
 * also given below (oracle_paper_grad_shared) as a cross-check for small T.
 *
 * Return codes: 0 ok, 1 invalid argument, 2 unsorted times, 3 mark out of
 * range, 4 time outside [0, T], 5 parameter outside its domain, 6 an
 * intensity <= 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_OK = 0, OR_INVALID = 1, OR_UNSORTED = 2, OR_MARK = 3, OR_TIME = 4,
       OR_PARAM = 5, OR_NONPOS = 6 };

static int check_inputs(int64_t N, const double* t, const int32_t* c, double T,
                        int32_t M, const double* mu, const double* alpha,
                        const double* beta)
{
    if (M <= 0 || N < 0 || !(T >= 0.0) || !isfinite(T)) return OR_INVALID;
    if (N > 0 && (!t || !c)) return OR_INVALID;
    if (!mu || !alpha || !beta) return OR_INVALID;
    for (int32_t i = 0; i < M; ++i) {
        if (!(mu[i] > 0.0) || !isfinite(mu[i])) return OR_PARAM;
        if (!(beta[i] > 0.0) || !isfinite(beta[i])) return OR_PARAM;
    }
    for (int64_t e = 0; e < (int64_t)M * M; ++e)
        if (!(alpha[e] >= 0.0) || !isfinite(alpha[e])) return OR_PARAM;
    for (int64_t k = 0; k < N; ++k) {
        if (c[k] < 0 || c[k] >= M) return OR_MARK;
        if (!(t[k] >= 0.0) || !(t[k] <= T)) return OR_TIME;
        if (k > 0 && t[k] < t[k - 1]) return OR_UNSORTED;
    }
    return OR_OK;
}

/* Log-likelihood and gradient in one forward pass (forward-mode G state).
 * Any of lam, dmu, dalpha, dbeta may be NULL.  dbeta is per source (length M);
 * for a shared decay the caller sums it.  Memory O(M^2 + M); time O(N M). */
/* The same for a slice of a longer sequence: its first event sees the state S0, G0
 * (the paper, Section 3.3: a batch depends on the events before it only through one
 * carried state; NULL = zero state).  base_term = 0 leaves out -T sum(mu) from L and -T
 * from dL/dmu, so that the slices of a sequence add up to the whole. */
int oracle_loglik_grad_carry(int64_t N, const double* t, const int32_t* c, double T,
                             int32_t M, const double* mu, const double* alpha,
                             const double* beta, const double* S0, const double* G0,
                             int base_term, double* out_ll, double* lam,
                             double* dmu, double* dalpha, double* dbeta)
{
    int rc = check_inputs(N, t, c, T, M, mu, alpha, beta);
    if (rc) return rc;
    double* S = calloc((size_t)M, sizeof(double));
    double* G = calloc((size_t)M, sizeof(double));
    double* E = calloc((size_t)M, sizeof(double));
    double* F = calloc((size_t)M, sizeof(double));
    if (!S || !G || !E || !F) { free(S); free(G); free(E); free(F); return OR_INVALID; }
    if (S0) memcpy(S, S0, sizeof(double) * (size_t)M);
    if (G0) memcpy(G, G0, sizeof(double) * (size_t)M);
    if (dmu) memset(dmu, 0, sizeof(double) * (size_t)M);
    if (dalpha) memset(dalpha, 0, sizeof(double) * (size_t)M * (size_t)M);
    if (dbeta) memset(dbeta, 0, sizeof(double) * (size_t)M);

    double logsum = 0.0;
    for (int64_t k = 0; k < N; ++k) {
        if (k > 0) {
            /* S_k = D_k (S_{k-1} + e_{c_{k-1}}), G_k = D_k (G_{k-1} + dt (S_{k-1} + e_{c_{k-1}})) */
            double dt = t[k] - t[k - 1];
            int32_t prev = c[k - 1];
            for (int32_t j = 0; j < M; ++j) {
                double d = exp(-beta[j] * dt);
                double P = S[j] + (j == prev ? 1.0 : 0.0);
                G[j] = d * (G[j] + dt * P);
                S[j] = d * P;
            }
        }
        int32_t i = c[k];
        const double* arow = alpha + (size_t)i * (size_t)M;
        double exc = 0.0;
        for (int32_t j = 0; j < M; ++j) exc += arow[j] * beta[j] * S[j];
        double lk = mu[i] + exc;
        if (!(lk > 0.0)) { rc = OR_NONPOS; break; }
        if (lam) lam[k] = lk;
        logsum += log(lk);
        double w = 1.0 / lk;
        if (dmu) dmu[i] += w;
        if (dalpha) {
            double* drow = dalpha + (size_t)i * (size_t)M;
            for (int32_t j = 0; j < M; ++j) drow[j] += w * beta[j] * S[j];
        }
        if (dbeta)
            for (int32_t j = 0; j < M; ++j) dbeta[j] += w * arow[j] * (S[j] - beta[j] * G[j]);
        /* compensator pieces of event k as a source */
        double x = beta[i] * (T - t[k]);
        E[i] += -expm1(-x);
        F[i] += (T - t[k]) * exp(-x);
    }
    if (rc == OR_OK) {
        double summu = 0.0, comp = 0.0;
        for (int32_t i = 0; i < M; ++i) summu += mu[i];
        for (int32_t j = 0; j < M; ++j) {
            double cs = 0.0;
            for (int32_t i = 0; i < M; ++i) cs += alpha[(size_t)i * M + j];
            comp += cs * E[j];
            if (dbeta) dbeta[j] -= cs * F[j];
        }
        if (out_ll) *out_ll = logsum - (base_term ? T * summu : 0.0) - comp;
        if (dmu && base_term) for (int32_t i = 0; i < M; ++i) dmu[i] -= T;
        if (dalpha)
            for (int32_t i = 0; i < M; ++i)
                for (int32_t j = 0; j < M; ++j) dalpha[(size_t)i * M + j] -= E[j];
    }
    free(S); free(G); free(E); free(F);
    return rc;
}

int oracle_loglik_grad(int64_t N, const double* t, const int32_t* c, double T,
                       int32_t M, const double* mu, const double* alpha,
                       const double* beta, double* out_ll, double* lam,
                       double* dmu, double* dalpha, double* dbeta)
{
    return oracle_loglik_grad_carry(N, t, c, T, M, mu, alpha, beta, NULL, NULL, 1, out_ll,
                                    lam, dmu, dalpha, dbeta);
}

/* State contributions of a slice's events at time t_next (for the carry exchange):
 * aggS[j] = sum_{l: c_l = j} exp(-beta_j (t_next - t_l)), aggG the same times (t_next - t_l). */
int oracle_slice_aggregate(int64_t N, const double* t, const int32_t* c, int32_t M,
                           const double* beta, double t_next, double* aggS, double* aggG)
{
    memset(aggS, 0, sizeof(double) * (size_t)M);
    memset(aggG, 0, sizeof(double) * (size_t)M);
    for (int64_t k = 0; k < N; ++k) {
        if (c[k] < 0 || c[k] >= M) return OR_MARK;
        if (t[k] > t_next) return OR_TIME;
        double x = t_next - t[k];
        double e = exp(-beta[c[k]] * x);
        aggS[c[k]] += e;
        aggG[c[k]] += x * e;
    }
    return OR_OK;
}

/* Gradient by the reverse-time adjoint of the same transitions (small N:
 * stores every state, O(N M) memory).  psi_k = dL_log/dS_k obeys
 *     psi_N = w_N beta (.) alpha[c_N,:],   psi_k = w_k beta (.) alpha[c_k,:] + D_{k+1} psi_{k+1},
 * and dL/dbeta_j = sum_k w_k alpha[c_k][j] S_{k,j} - sum_{k>=2} dt_k psi_{k,j} S_{k,j}
 *                  - colsum_j F_j  (chain rule through D_k, dS_{k,j}/dbeta_j|local = -dt_k S_{k,j}).
 * dmu and dalpha are as in oracle_loglik_grad. */
int oracle_grad_adjoint(int64_t N, const double* t, const int32_t* c, double T,
                        int32_t M, const double* mu, const double* alpha,
                        const double* beta, double* out_ll, double* dmu,
                        double* dalpha, double* dbeta)
{
    int rc = check_inputs(N, t, c, T, M, mu, alpha, beta);
    if (rc) return rc;
    size_t NM = (size_t)(N > 0 ? N : 1) * (size_t)M;
    double* S = calloc(NM, sizeof(double));        /* S[k*M + j] */
    double* w = calloc((size_t)(N > 0 ? N : 1), sizeof(double));
    double* psi = calloc((size_t)M, sizeof(double));
    double* E = calloc((size_t)M, sizeof(double));
    double* F = calloc((size_t)M, sizeof(double));
    if (!S || !w || !psi || !E || !F) { rc = OR_INVALID; goto done; }
    memset(dmu, 0, sizeof(double) * (size_t)M);
    memset(dalpha, 0, sizeof(double) * (size_t)M * (size_t)M);
    memset(dbeta, 0, sizeof(double) * (size_t)M);

    double logsum = 0.0;
    for (int64_t k = 0; k < N; ++k) {
        double* Sk = S + (size_t)k * M;
        if (k > 0) {
            const double* Sp = S + (size_t)(k - 1) * M;
            double dt = t[k] - t[k - 1];
            for (int32_t j = 0; j < M; ++j)
                Sk[j] = exp(-beta[j] * dt) * (Sp[j] + (j == c[k - 1] ? 1.0 : 0.0));
        }
        int32_t i = c[k];
        double lk = mu[i];
        for (int32_t j = 0; j < M; ++j) lk += alpha[(size_t)i * M + j] * beta[j] * Sk[j];
        if (!(lk > 0.0)) { rc = OR_NONPOS; goto done; }
        logsum += log(lk);
        w[k] = 1.0 / lk;
        dmu[i] += w[k];
        for (int32_t j = 0; j < M; ++j) {
            dalpha[(size_t)i * M + j] += w[k] * beta[j] * Sk[j];
            dbeta[j] += w[k] * alpha[(size_t)i * M + j] * Sk[j];
        }
        double x = beta[i] * (T - t[k]);
        E[i] += -expm1(-x);
        F[i] += (T - t[k]) * exp(-x);
    }
    /* reverse sweep */
    for (int64_t k = N - 1; k >= 0; --k) {
        if (k < N - 1) {
            double dt1 = t[k + 1] - t[k];
            for (int32_t j = 0; j < M; ++j) psi[j] *= exp(-beta[j] * dt1);
        }
        int32_t i = c[k];
        for (int32_t j = 0; j < M; ++j) psi[j] += w[k] * beta[j] * alpha[(size_t)i * M + j];
        if (k > 0) {
            double dt = t[k] - t[k - 1];
            const double* Sk = S + (size_t)k * M;
            for (int32_t j = 0; j < M; ++j) dbeta[j] -= dt * psi[j] * Sk[j];
        }
    }
    {
        double summu = 0.0, comp = 0.0;
        for (int32_t i = 0; i < M; ++i) summu += mu[i];
        for (int32_t j = 0; j < M; ++j) {
            double cs = 0.0;
            for (int32_t i = 0; i < M; ++i) cs += alpha[(size_t)i * M + j];
            comp += cs * E[j];
            dbeta[j] -= cs * F[j];
        }
        *out_ll = logsum - T * summu - comp;
        for (int32_t i = 0; i < M; ++i) dmu[i] -= T;
        for (int32_t i = 0; i < M; ++i)
            for (int32_t j = 0; j < M; ++j) dalpha[(size_t)i * M + j] -= E[j];
    }
done:
    free(S); free(w); free(psi); free(E); free(F);
    return rc;
}

/* The paper's own gradient formulas for one shared decay gamma (Appendix B,
 * Eqs. grad_mu, grad_alpha, grad_gamma), driven by the paper's three state
 * recurrences: R (Eq. intensity_state_recurrence, target-indexed, alpha
 * folded in), K (Eq. alpha_grad_recurrence) and L (Eq.
 * gamma_grad_recurrence):
 *   R_i = e^{-g dt}(R_{i-1} + alpha[:, m_{i-1}]),  K_i = e^{-g dt}(K_{i-1} + e_{m_{i-1}}),
 *   L_i = e^{-g dt}(L_{i-1} + t_{i-1} alpha[:, m_{i-1}]),
 *   dL/dgamma = sum_i [(1 - g t_i) R_{m_i} + g L_{m_i}] / lambda_i
 *               - sum_m sum_i alpha[m][m_i] (T - t_i) e^{-g (T - t_i)}.
 * The (1 - g t) R + g L combination loses about log10(g t) digits; use it
 * only with small T.  Outputs dL/dmu[M], dL/dalpha[M*M], dL/dgamma (scalar). */
int oracle_paper_grad_shared(int64_t N, const double* t, const int32_t* c, double T,
                             int32_t M, const double* mu, const double* alpha,
                             double gamma, double* out_ll, double* dmu,
                             double* dalpha, double* dgamma)
{
    if (!(gamma > 0.0)) return OR_PARAM;
    double* bvec = malloc(sizeof(double) * (size_t)M);
    if (!bvec) return OR_INVALID;
    for (int32_t j = 0; j < M; ++j) bvec[j] = gamma;
    int rc = check_inputs(N, t, c, T, M, mu, alpha, bvec);
    free(bvec);
    if (rc) return rc;
    double* R = calloc((size_t)M, sizeof(double));
    double* K = calloc((size_t)M, sizeof(double));
    double* L = calloc((size_t)M, sizeof(double));
    if (!R || !K || !L) { free(R); free(K); free(L); return OR_INVALID; }
    memset(dmu, 0, sizeof(double) * (size_t)M);
    memset(dalpha, 0, sizeof(double) * (size_t)M * (size_t)M);
    double g_acc = 0.0, logsum = 0.0;
    for (int64_t k = 0; k < N; ++k) {
        if (k > 0) {
            double d = exp(-gamma * (t[k] - t[k - 1]));
            int32_t q = c[k - 1];
            for (int32_t p = 0; p < M; ++p) {
                double a = alpha[(size_t)p * M + q];
                R[p] = d * (R[p] + a);
                L[p] = d * (L[p] + t[k - 1] * a);
                K[p] = d * (K[p] + (p == q ? 1.0 : 0.0));
            }
        }
        int32_t p = c[k];
        double lk = mu[p] + gamma * R[p];
        if (!(lk > 0.0)) { rc = OR_NONPOS; break; }
        logsum += log(lk);
        dmu[p] += 1.0 / lk;
        for (int32_t q = 0; q < M; ++q) dalpha[(size_t)p * M + q] += gamma * K[q] / lk;
        g_acc += ((1.0 - gamma * t[k]) * R[p] + gamma * L[p]) / lk;
    }
    if (rc == OR_OK) {
        double summu = 0.0, comp = 0.0;
        for (int32_t i = 0; i < M; ++i) summu += mu[i];
        for (int64_t k = 0; k < N; ++k) {
            int32_t q = c[k];
            double cs = 0.0;
            for (int32_t m = 0; m < M; ++m) cs += alpha[(size_t)m * M + q];
            double x = gamma * (T - t[k]);
            comp += cs * (-expm1(-x));
            g_acc -= cs * (T - t[k]) * exp(-x);
            for (int32_t pp = 0; pp < M; ++pp) dalpha[(size_t)pp * M + q] -= -expm1(-x);
        }
        for (int32_t i = 0; i < M; ++i) dmu[i] -= T;
        *out_ll = logsum - T * summu - comp;
        *dgamma = g_acc;
    }
    free(R); free(K); free(L);
    return rc;
}

/* Batched form: B independent sequences, events of sequence s are
 * [offsets[s], offsets[s+1]) of t and c, each with its own T[s], mu[s*M..],
 * alpha[s*M*M..], beta[s*M..].  Outputs are per sequence; grads may be NULL. */
int oracle_loglik_grad_varlen(const double* t, const int32_t* c, const int64_t* offsets,
                              int32_t B, const double* T, int32_t M,
                              const double* mu, const double* alpha, const double* beta,
                              double* out_ll, double* dmu, double* dalpha, double* dbeta)
{
    if (B < 0 || !offsets) return OR_INVALID;
    if (offsets[0] != 0) return OR_INVALID;
    for (int32_t s = 0; s < B; ++s)
        if (offsets[s + 1] < offsets[s]) return OR_INVALID;
    for (int32_t s = 0; s < B; ++s) {
        int64_t o = offsets[s], n = offsets[s + 1] - offsets[s];
        size_t pm = (size_t)s * M, pa = (size_t)s * M * M;
        int rc = oracle_loglik_grad(n, t ? t + o : NULL, c ? c + o : NULL, T[s], M,
                                    mu + pm, alpha + pa, beta + pm, out_ll + s, NULL,
                                    dmu ? dmu + pm : NULL, dalpha ? dalpha + pa : NULL,
                                    dbeta ? dbeta + pm : NULL);
        if (rc) return rc;
    }
    return OR_OK;
}

/* Integer pass: per-mark event counts, bit-exact reference for the library's
 * validate-and-count step.  Returns the same codes as check of the inputs. */
int oracle_mark_counts(int64_t N, const int32_t* c, int32_t M, int64_t* counts)
{
    if (M <= 0 || N < 0) return OR_INVALID;
    memset(counts, 0, sizeof(int64_t) * (size_t)M);
    for (int64_t k = 0; k < N; ++k) {
        if (c[k] < 0 || c[k] >= M) return OR_MARK;
        counts[c[k]] += 1;
    }
    return OR_OK;
}

/* Lazy per-component form for a sparse alpha, with the gradient on alpha's support.
 *
 * The same model and results as oracle_loglik_grad (paper, Section 2, Eq.
 * hawkes_excitation with one decay per source; Eq. general_hawkes_likelihood; Appendix B,
 * Eqs. grad_mu, grad_alpha, grad_gamma), computed so that an event costs O(nonzeros of its
 * row of alpha) instead of O(M): component j of the source-indexed state is kept only as
 * its value S_j, G_j just after the last event of mark j (at time last_j), and decayed to
 * the time t it is read at:
 *     S_j(t) = S_j e^{-beta_j (t - last_j)},  G_j(t) = e^{-beta_j (t - last_j)} (G_j + (t - last_j) S_j),
 * the closed form of the recurrence S_k = D_k (S_{k-1} + e_{c_{k-1}}) between two events of
 * mark j.  An event of mark i reads the components j with alpha[i][j] != 0 only (the others
 * add nothing to its intensity or to dL/dbeta_j), and then adds its own jump to S_i.
 *   ll, dmu [M], dbeta [M]: as oracle_loglik_grad (exact for any alpha).
 *   dalpha [M*M]: dL/dalpha_ij for the entries with alpha[i][j] != 0 (the support: the
 *                 interactions the model has), 0 for the entries outside it.
 * Ties follow index order, as in oracle_loglik_grad (dt = 0 gives weight 1). */
int oracle_loglik_grad_support(int64_t N, const double* t, const int32_t* c, double T,
                               int32_t M, const double* mu, const double* alpha,
                               const double* beta, double* ll, double* dmu, double* dalpha,
                               double* dbeta)
{
    int rc = check_inputs(N, t, c, T, M, mu, alpha, beta);
    if (rc) return rc;
    int64_t* rowp = calloc((size_t)M + 1, sizeof(int64_t));
    double *S = calloc((size_t)M, sizeof(double)), *G = calloc((size_t)M, sizeof(double));
    double *last = calloc((size_t)M, sizeof(double)), *E = calloc((size_t)M, sizeof(double));
    double *F = calloc((size_t)M, sizeof(double)), *xs = calloc((size_t)M, sizeof(double));
    double *xg = calloc((size_t)M, sizeof(double));
    if (!rowp || !S || !G || !last || !E || !F || !xs || !xg) { rc = OR_INVALID; goto done; }
    int64_t nnz = 0;
    for (int32_t i = 0; i < M; ++i) {
        rowp[i] = nnz;
        for (int32_t j = 0; j < M; ++j) nnz += alpha[(size_t)i * M + j] != 0.0;
    }
    rowp[M] = nnz;
    int32_t* col = malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    if (!col) { rc = OR_INVALID; goto done; }
    for (int32_t i = 0, e = 0; i < M; ++i)
        for (int32_t j = 0; j < M; ++j)
            if (alpha[(size_t)i * M + j] != 0.0) col[e++] = j;
    memset(dmu, 0, sizeof(double) * (size_t)M);
    memset(dalpha, 0, sizeof(double) * (size_t)M * M);
    memset(dbeta, 0, sizeof(double) * (size_t)M);
    double logsum = 0.0;
    for (int64_t k = 0; k < N; ++k) {
        const int32_t i = c[k];
        const double* arow = alpha + (size_t)i * M;
        double lk = mu[i];
        for (int64_t e = rowp[i]; e < rowp[i + 1]; ++e) {       /* read the row's components */
            const int32_t j = col[e];
            const double dt = t[k] - last[j];
            const double d = exp(-beta[j] * dt);
            xs[e - rowp[i]] = S[j] * d;
            xg[e - rowp[i]] = d * (G[j] + dt * S[j]);
            lk += arow[j] * beta[j] * xs[e - rowp[i]];
        }
        if (!(lk > 0.0)) { rc = OR_NONPOS; break; }
        logsum += log(lk);
        const double w = 1.0 / lk;
        dmu[i] += w;
        for (int64_t e = rowp[i]; e < rowp[i + 1]; ++e) {
            const int32_t j = col[e];
            dalpha[(size_t)i * M + j] += w * xs[e - rowp[i]];
            dbeta[j] += w * arow[j] * (xs[e - rowp[i]] - beta[j] * xg[e - rowp[i]]);
        }
        {                                                        /* the event's own jump */
            const double dt = t[k] - last[i];
            const double d = exp(-beta[i] * dt);
            G[i] = d * (G[i] + dt * S[i]);
            S[i] = d * S[i] + 1.0;
            last[i] = t[k];
        }
        const double x = T - t[k];
        E[i] += -expm1(-beta[i] * x);
        F[i] += x * exp(-beta[i] * x);
    }
    if (rc == OR_OK) {
        double summu = 0.0, comp = 0.0;
        for (int32_t r = 0; r < M; ++r) summu += mu[r];
        for (int32_t j = 0; j < M; ++j) {
            double cs = 0.0;
            for (int32_t r = 0; r < M; ++r) cs += alpha[(size_t)r * M + j];
            comp += cs * E[j];
            dbeta[j] -= cs * F[j];
        }
        *ll = logsum - T * summu - comp;
        for (int32_t r = 0; r < M; ++r) dmu[r] -= T;
        for (int32_t r = 0; r < M; ++r)
            for (int64_t e = rowp[r]; e < rowp[r + 1]; ++e) {
                const int32_t j = col[e];
                dalpha[(size_t)r * M + j] = beta[j] * dalpha[(size_t)r * M + j] - E[j];
            }
    }
    free(col);
done:
    free(rowp); free(S); free(G); free(last); free(E); free(F); free(xs); free(xg);
    return rc;
}

/* Integer pass: the chunk table of B sequences cut into chunks of C consecutive
 * events (paper, Section 3.3: the stream is processed in contiguous batches, each
 * depending on the earlier ones only through one carried state).  Sequence s owns
 * events [offsets[s], offsets[s+1]) and ceil(len_s / C) chunks; chunk_base[s] is the
 * number of chunks of the sequences before s (chunk_base[B] = all chunks) and
 * chunk_seq[b] the sequence that owns chunk b (chunk_seq holds chunk_base[B] entries;
 * the caller sizes it from the same formula).  A sequence's chunk q covers its events
 * [q C, min((q + 1) C, len)). */
int oracle_chunk_table(int32_t B, const int64_t* offsets, int32_t C, int64_t* chunk_base,
                       int32_t* chunk_seq)
{
    if (B <= 0 || C <= 0 || offsets[0] != 0) return OR_INVALID;
    int64_t nb = 0;
    for (int32_t s = 0; s < B; ++s) {
        int64_t len = offsets[s + 1] - offsets[s];
        if (len < 0) return OR_INVALID;
        chunk_base[s] = nb;
        int64_t n = len / C + (len % C != 0 ? 1 : 0);
        for (int64_t q = 0; q < n; ++q) chunk_seq[nb + q] = s;
        nb += n;
    }
    chunk_base[B] = nb;
    return OR_OK;
}

/* Integer pass of the pair kernels of one sequence: the marks are dealt into P blocks
 * (block of mark c = c mod P, position c / P), and the events of every chunk of C events
 * are ordered by (block, position, index in the chunk).  Outputs, per chunk b:
 *   bucket_start[b (P + 1) + q] = number of the chunk's events whose block is below q
 *                                 (q = 0..P; the last entry is the chunk's length),
 *   order[b C + r]              = the index in the chunk of its r-th event in that order.
 * This is a stable counting sort, written as plain nested loops over the blocks, the
 * positions in a block and the chunk's events. */
int oracle_bucket_order(int64_t N, const int32_t* c, int32_t M, int32_t C, int32_t P,
                        int32_t* bucket_start, int32_t* order)
{
    if (N < 0 || M <= 0 || C <= 0 || P <= 0) return OR_INVALID;
    int64_t nb = N / C + (N % C != 0 ? 1 : 0);
    for (int64_t b = 0; b < nb; ++b) {
        int64_t s0 = b * C, s1 = s0 + C < N ? s0 + C : N;
        int32_t* bs = bucket_start + b * (P + 1);
        int32_t r = 0;
        for (int32_t q = 0; q < P; ++q) {
            bs[q] = r;
            for (int32_t pos = 0; pos * P + q < M; ++pos)          /* marks of block q, by position */
                for (int64_t k = s0; k < s1; ++k)                  /* their events, by index */
                    if (c[k] == pos * P + q) order[s0 + r++] = (int32_t)(k - s0);
        }
        bs[P] = r;
        if (r != (int32_t)(s1 - s0)) return OR_MARK;
    }
    return OR_OK;
}

/* Integer pass: the support of alpha row by row, in column order: the entries with
 * alpha[i][j] != 0, or every entry when `all` is set.  row_ptr [M+1]; col holds row_ptr[M]
 * entries (at most M*M). */
int oracle_support_rows(int32_t M, const double* alpha, int32_t all, int32_t* row_ptr,
                        int32_t* col)
{
    if (M <= 0) return OR_INVALID;
    int32_t e = 0;
    for (int32_t i = 0; i < M; ++i) {
        row_ptr[i] = e;
        for (int32_t j = 0; j < M; ++j)
            if (all || alpha[(size_t)i * M + j] != 0.0) col[e++] = j;
    }
    row_ptr[M] = e;
    return OR_OK;
}

/* Integer pass: the events cut into segments of L consecutive events and ordered by
 * (segment, mark, index).  start [nseg*M + 1]: the first position of each (segment, mark)
 * in that order (start[nseg*M] = N); order [N]: the index of the event at each position. */
int oracle_mark_sort(int64_t N, const int32_t* c, int32_t M, int64_t L, int32_t* start,
                     int32_t* order)
{
    if (N < 0 || M <= 0 || L <= 0) return OR_INVALID;
    int64_t nseg = N / L + (N % L != 0 ? 1 : 0);
    int64_t r = 0;
    for (int64_t s = 0; s < nseg; ++s) {
        int64_t s0 = s * L, s1 = s0 + L < N ? s0 + L : N;
        for (int32_t m = 0; m < M; ++m) {
            start[s * M + m] = (int32_t)r;
            for (int64_t k = s0; k < s1; ++k)
                if (c[k] == m) order[r++] = (int32_t)k;
        }
    }
    start[nseg * M] = (int32_t)r;
    return r == N ? OR_OK : OR_MARK;
}

/* Conditioning scales of the results (for stating errors of near-zero results):
 *   scale_ll       = sum_k |log lambda_k| + Lambda(T)
 *   scale_dbeta[j] = sum_k |w_k alpha[c_k][j] (S_{k,j} - beta_j G_{k,j})| + colsum_j F_j
 * i.e. the sums of magnitudes of the terms whose difference is L or dL/dbeta_j.  A result
 * that is much smaller than its scale is ill-conditioned: rounding of its terms, relative
 * to the scale, is amplified by scale / |result|. */
int oracle_condition(int64_t N, const double* t, const int32_t* c, double T, int32_t M,
                     const double* mu, const double* alpha, const double* beta,
                     double* scale_ll, double* scale_dbeta)
{
    int rc = check_inputs(N, t, c, T, M, mu, alpha, beta);
    if (rc) return rc;
    double* S = calloc((size_t)M, sizeof(double));
    double* G = calloc((size_t)M, sizeof(double));
    double* F = calloc((size_t)M, sizeof(double));
    if (!S || !G || !F) { free(S); free(G); free(F); return OR_INVALID; }
    memset(scale_dbeta, 0, sizeof(double) * (size_t)M);
    double sabs = 0.0, logsum = 0.0, comp = 0.0;
    for (int64_t k = 0; k < N; ++k) {
        if (k > 0) {
            double dt = t[k] - t[k - 1];
            int32_t prev = c[k - 1];
            for (int32_t j = 0; j < M; ++j) {
                double d = exp(-beta[j] * dt);
                double P = S[j] + (j == prev ? 1.0 : 0.0);
                G[j] = d * (G[j] + dt * P);
                S[j] = d * P;
            }
        }
        int32_t i = c[k];
        const double* arow = alpha + (size_t)i * (size_t)M;
        double lk = mu[i];
        for (int32_t j = 0; j < M; ++j) lk += arow[j] * beta[j] * S[j];
        if (!(lk > 0.0)) { rc = OR_NONPOS; break; }
        sabs += fabs(log(lk));
        logsum += log(lk);
        double w = 1.0 / lk;
        for (int32_t j = 0; j < M; ++j) scale_dbeta[j] += fabs(w * arow[j] * (S[j] - beta[j] * G[j]));
        double x = beta[i] * (T - t[k]);
        F[i] += (T - t[k]) * exp(-x);
        double cs = 0.0;
        for (int32_t r = 0; r < M; ++r) cs += alpha[(size_t)r * M + i];
        comp += cs * (-expm1(-x));
    }
    if (rc == OR_OK) {
        double summu = 0.0;
        for (int32_t r = 0; r < M; ++r) summu += mu[r];
        *scale_ll = sabs + T * summu + comp;
        for (int32_t j = 0; j < M; ++j) {
            double cs = 0.0;
            for (int32_t r = 0; r < M; ++r) cs += alpha[(size_t)r * M + j];
            scale_dbeta[j] += cs * F[j];
        }
    }
    free(S); free(G); free(F);
    return rc;
}

/* Several decay kernels (paper, Section 2, Eq. hawkes_excitation with its sum over
 * kernels k = 1..K): kernel q has its own interaction matrix alpha^(q) and decays
 * beta^(q)_j (one per source; the paper's model has them equal within a kernel),
 *     lambda_p(t) = mu_p + sum_q sum_{l before t} alpha^(q)[p][c_l] beta^(q)_{c_l}
 *                          exp(-beta^(q)_{c_l} (t - t_l)).
 * Each kernel keeps its own source-indexed state S^(q) (and G^(q)); lambda sums the
 * kernels, and the gradients with respect to alpha^(q) and beta^(q) are the single-kernel
 * formulas above with S^(q), G^(q), E^(q), F^(q), colsum^(q).
 * alpha: [K][M][M], beta: [K][M]; dalpha: [K][M][M], dbeta: [K][M]; lam (optional): [N]. */
int oracle_loglik_grad_multi(int64_t N, const double* t, const int32_t* c, double T,
                             int32_t M, int32_t K, const double* mu, const double* alpha,
                             const double* beta, double* out_ll, double* lam,
                             double* dmu, double* dalpha, double* dbeta)
{
    if (K < 1) return OR_INVALID;
    for (int32_t q = 0; q < K; ++q) {
        int rc = check_inputs(N, t, c, T, M, mu, alpha + (size_t)q * M * M, beta + (size_t)q * M);
        if (rc) return rc;
    }
    const size_t KM = (size_t)K * (size_t)M;
    double* S = calloc(KM, sizeof(double));
    double* G = calloc(KM, sizeof(double));
    double* E = calloc(KM, sizeof(double));
    double* F = calloc(KM, sizeof(double));
    if (!S || !G || !E || !F) { free(S); free(G); free(E); free(F); return OR_INVALID; }
    if (dmu) memset(dmu, 0, sizeof(double) * (size_t)M);
    if (dalpha) memset(dalpha, 0, sizeof(double) * KM * (size_t)M);
    if (dbeta) memset(dbeta, 0, sizeof(double) * KM);

    int rc = OR_OK;
    double logsum = 0.0;
    for (int64_t k = 0; k < N; ++k) {
        if (k > 0) {
            double dt = t[k] - t[k - 1];
            int32_t prev = c[k - 1];
            for (int32_t q = 0; q < K; ++q)
                for (int32_t j = 0; j < M; ++j) {
                    size_t v = (size_t)q * M + j;
                    double d = exp(-beta[v] * dt);
                    double P = S[v] + (j == prev ? 1.0 : 0.0);
                    G[v] = d * (G[v] + dt * P);
                    S[v] = d * P;
                }
        }
        int32_t i = c[k];
        double exc = 0.0;
        for (int32_t q = 0; q < K; ++q) {
            const double* arow = alpha + ((size_t)q * M + i) * M;
            for (int32_t j = 0; j < M; ++j) {
                size_t v = (size_t)q * M + j;
                exc += arow[j] * beta[v] * S[v];
            }
        }
        double lk = mu[i] + exc;
        if (!(lk > 0.0)) { rc = OR_NONPOS; break; }
        if (lam) lam[k] = lk;
        logsum += log(lk);
        double w = 1.0 / lk;
        if (dmu) dmu[i] += w;
        for (int32_t q = 0; q < K; ++q) {
            const double* arow = alpha + ((size_t)q * M + i) * M;
            for (int32_t j = 0; j < M; ++j) {
                size_t v = (size_t)q * M + j;
                if (dalpha) dalpha[((size_t)q * M + i) * M + j] += w * beta[v] * S[v];
                if (dbeta) dbeta[v] += w * arow[j] * (S[v] - beta[v] * G[v]);
            }
            /* compensator pieces of event k as a source of kernel q */
            size_t vi = (size_t)q * M + i;
            double x = beta[vi] * (T - t[k]);
            E[vi] += -expm1(-x);
            F[vi] += (T - t[k]) * exp(-x);
        }
    }
    if (rc == OR_OK) {
        double summu = 0.0, comp = 0.0;
        for (int32_t i = 0; i < M; ++i) summu += mu[i];
        for (int32_t q = 0; q < K; ++q)
            for (int32_t j = 0; j < M; ++j) {
                size_t v = (size_t)q * M + j;
                double cs = 0.0;
                for (int32_t i = 0; i < M; ++i) cs += alpha[((size_t)q * M + i) * M + j];
                comp += cs * E[v];
                if (dbeta) dbeta[v] -= cs * F[v];
            }
        if (out_ll) *out_ll = logsum - T * summu - comp;
        if (dmu) for (int32_t i = 0; i < M; ++i) dmu[i] -= T;
        if (dalpha)
            for (int32_t q = 0; q < K; ++q)
                for (int32_t i = 0; i < M; ++i)
                    for (int32_t j = 0; j < M; ++j)
                        dalpha[((size_t)q * M + i) * M + j] -= E[(size_t)q * M + j];
    }
    free(S); free(G); free(E); free(F);
    return rc;
}

/* Conditioning scales of L and of each dL/dbeta^(q)_j with several decay kernels: the
 * sums of magnitudes of their terms, as oracle_condition does for one kernel, with the
 * intensity (and w = 1 / lambda) summed over the kernels:
 *   scale_ll = sum_k |log lambda_k| + T sum_i mu_i + sum_q sum_j colsum^(q)_j E^(q)_j,
 *   scale_dbeta[q][j] = sum_k |w_k alpha^(q)[c_k][j] (S^(q)_j - beta^(q)_j G^(q)_j)|
 *                       + colsum^(q)_j F^(q)_j.
 * alpha: [K][M][M], beta: [K][M]; scale_dbeta: [K][M]. */
int oracle_condition_multi(int64_t N, const double* t, const int32_t* c, double T,
                           int32_t M, int32_t K, const double* mu, const double* alpha,
                           const double* beta, double* scale_ll, double* scale_dbeta)
{
    if (K < 1) return OR_INVALID;
    for (int32_t q = 0; q < K; ++q) {
        int rc = check_inputs(N, t, c, T, M, mu, alpha + (size_t)q * M * M, beta + (size_t)q * M);
        if (rc) return rc;
    }
    const size_t KM = (size_t)K * (size_t)M;
    double* S = calloc(KM, sizeof(double));
    double* G = calloc(KM, sizeof(double));
    double* E = calloc(KM, sizeof(double));
    double* F = calloc(KM, sizeof(double));
    if (!S || !G || !E || !F) { free(S); free(G); free(E); free(F); return OR_INVALID; }
    memset(scale_dbeta, 0, sizeof(double) * KM);
    int rc = OR_OK;
    double sabs = 0.0;
    for (int64_t k = 0; k < N; ++k) {
        if (k > 0) {
            double dt = t[k] - t[k - 1];
            int32_t prev = c[k - 1];
            for (size_t v = 0; v < KM; ++v) {
                double d = exp(-beta[v] * dt);
                double P = S[v] + ((int32_t)(v % (size_t)M) == prev ? 1.0 : 0.0);
                G[v] = d * (G[v] + dt * P);
                S[v] = d * P;
            }
        }
        int32_t i = c[k];
        double lk = mu[i];
        for (int32_t q = 0; q < K; ++q) {
            const double* arow = alpha + ((size_t)q * M + i) * M;
            for (int32_t j = 0; j < M; ++j) lk += arow[j] * beta[(size_t)q * M + j] * S[(size_t)q * M + j];
        }
        if (!(lk > 0.0)) { rc = OR_NONPOS; break; }
        sabs += fabs(log(lk));
        double w = 1.0 / lk;
        for (int32_t q = 0; q < K; ++q) {
            const double* arow = alpha + ((size_t)q * M + i) * M;
            for (int32_t j = 0; j < M; ++j) {
                size_t v = (size_t)q * M + j;
                scale_dbeta[v] += fabs(w * arow[j] * (S[v] - beta[v] * G[v]));
            }
            size_t vi = (size_t)q * M + i;
            double x = beta[vi] * (T - t[k]);
            E[vi] += -expm1(-x);
            F[vi] += (T - t[k]) * exp(-x);
        }
    }
    if (rc == OR_OK) {
        double summu = 0.0, comp = 0.0;
        for (int32_t i = 0; i < M; ++i) summu += mu[i];
        for (int32_t q = 0; q < K; ++q)
            for (int32_t j = 0; j < M; ++j) {
                size_t v = (size_t)q * M + j;
                double cs = 0.0;
                for (int32_t r = 0; r < M; ++r) cs += alpha[((size_t)q * M + r) * M + j];
                comp += cs * E[v];
                scale_dbeta[v] += cs * F[v];
            }
        *scale_ll = sabs + T * summu + comp;
    }
    free(S); free(G); free(E); free(F);
    return rc;
}
