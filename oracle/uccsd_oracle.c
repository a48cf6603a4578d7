/*
 * UCCSD state-vector oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of what the VQE-UCCSD hot path
 * computes (Sugisaki, Nakano, Mochizuki, arXiv:2402.17993).  It exists to
 * check the CUDA library; only the test suite, the smoke entry point and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header or
 * table with the CUDA path: it never forms Pauli strings, it applies
 * fermionic ladder operators to occupation-number basis states directly.
 *
 * Conventions (readings of the paper, Section 2.3):
 *   - spin orbital P = 2p + s (s = 0 alpha, 1 beta); bit P of a basis index
 *     is the occupation of P (Jordan-Wigner ordering);
 *   - a_P |x> = (-1)^{#occupied below P} |x ^ 2^P> if P occupied, else 0;
 *     a^dag_P likewise with P empty;
 *   - Eq. 2: H = sum h_PQ a^dag_P a_Q + 1/2 sum g_PQRS a^dag_P a^dag_Q a_S a_R
 *     with g_PQRS = <PQ|RS> = (pr|qs) delta(s_P,s_R) delta(s_Q,s_S) built
 *     from chemist-notation spatial integrals (pq|rs), h_PQ = h_pq delta;
 *   - Eq. 4 generators: singles tau = a^dag_a a_i, doubles
 *     tau = a^dag_a a^dag_b a_j a_i (i<j occupied, a<b virtual),
 *     G = tau - tau^dag, one amplitude per tuple;
 *   - Eq. 5: the ordered product of exp(theta_k G_k / M), excitation 1
 *     acting first on |HF>, repeated M times; Eq. 6: the forward list then
 *     the reversed list, each with theta_k / (2M), repeated M times.  A
 *     schedule (k, scale) lists the factors in the order they act.
 *
 * The state is a dense array of 2^n complex amplitudes stored as
 * interleaved (re, im) doubles.  All work loops either over every basis
 * index ("full" mode) or over the basis states with n_alpha alpha and
 * n_beta beta electrons ("sector" mode).  In sector mode every produced
 * index is checked to lie in the sector; a violation is reported as error.
 *
 * Parity pins for every function live in the CPU test suite (dense
 * Kronecker-product Jordan-Wigner matrices, scipy expm, numpy eigh, the
 * Hartree-Fock closed form, finite differences, exact Fourier derivatives).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_ERR_ARG 1
#define ORACLE_ERR_SECTOR 2
#define ORACLE_ERR_NOMEM 3

static int popc64(uint64_t v) { return __builtin_popcountll(v); }

/* a_p |x>: returns the sign (+1 or -1) and *y, or 0 if orbital p is empty. */
static int ladder_ann(int p, uint64_t x, uint64_t *y) {
    if (!((x >> p) & 1u)) return 0;
    *y = x ^ (1ull << p);
    return (popc64(x & ((1ull << p) - 1ull)) & 1) ? -1 : 1;
}

/* a^dag_p |x>: returns the sign and *y, or 0 if orbital p is occupied. */
static int ladder_cre(int p, uint64_t x, uint64_t *y) {
    if ((x >> p) & 1u) return 0;
    *y = x ^ (1ull << p);
    return (popc64(x & ((1ull << p) - 1ull)) & 1) ? -1 : 1;
}

/* Apply a product of ladder operators written left to right as
 * ops[0] ops[1] ... ops[len-1]; the rightmost acts first.  dag[t] != 0 marks
 * a creation operator.  Returns the total sign or 0 if annihilated. */
static int apply_ladder_string(int len, const int *idx, const int *dag,
                               uint64_t x, uint64_t *y) {
    int sign = 1;
    uint64_t cur = x;
    for (int t = len - 1; t >= 0; --t) {
        uint64_t nxt;
        int s = dag[t] ? ladder_cre(idx[t], cur, &nxt) : ladder_ann(idx[t], cur, &nxt);
        if (s == 0) return 0;
        sign *= s;
        cur = nxt;
    }
    *y = cur;
    return sign;
}

/* Spin-orbital integrals from spatial ones (Eq. 2). */
static double h_so(int n_orb, const double *h, int P, int Q) {
    if ((P & 1) != (Q & 1)) return 0.0;
    return h[(P >> 1) * n_orb + (Q >> 1)];
}
/* <PQ|RS> = (pr|qs) with spin deltas. */
static double g_so(int n_orb, const double *eri, int P, int Q, int R, int S) {
    if ((P & 1) != (R & 1) || (Q & 1) != (S & 1)) return 0.0;
    int p = P >> 1, q = Q >> 1, r = R >> 1, s = S >> 1;
    return eri[(((size_t)p * n_orb + r) * n_orb + q) * n_orb + s];
}

/* Basis states of the (n_alpha, n_beta) sector, ascending. */
static int64_t sector_list(int n_qubits, int n_alpha, int n_beta, uint64_t **out) {
    uint64_t amask = 0;
    for (int q = 0; q < n_qubits; q += 2) amask |= 1ull << q;
    uint64_t bmask = ((n_qubits >= 64) ? ~0ull : ((1ull << n_qubits) - 1ull)) & ~amask;
    uint64_t N = 1ull << n_qubits;
    int64_t cnt = 0;
    for (uint64_t x = 0; x < N; ++x)
        if (popc64(x & amask) == n_alpha && popc64(x & bmask) == n_beta) ++cnt;
    uint64_t *lst = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(cnt > 0 ? cnt : 1));
    if (!lst) return -1;
    int64_t i = 0;
    for (uint64_t x = 0; x < N; ++x)
        if (popc64(x & amask) == n_alpha && popc64(x & bmask) == n_beta) lst[i++] = x;
    *out = lst;
    return cnt;
}

static int in_sector(uint64_t x, int n_qubits, int n_alpha, int n_beta) {
    uint64_t amask = 0;
    for (int q = 0; q < n_qubits; q += 2) amask |= 1ull << q;
    return popc64(x & amask) == n_alpha && popc64(x & ~amask) == n_beta;
}

/* Iteration domain: either all 2^n indices or an explicit sector list. */
typedef struct {
    int n_qubits, n_alpha, n_beta;
    const uint64_t *list; /* NULL: all 2^n */
    int64_t count;
} domain_t;

static inline uint64_t dom_at(const domain_t *d, int64_t i) {
    return d->list ? d->list[i] : (uint64_t)i;
}

int oracle_sector_size(int n_qubits, int n_alpha, int n_beta, int64_t *count) {
    uint64_t *lst = NULL;
    int64_t c = sector_list(n_qubits, n_alpha, n_beta, &lst);
    if (c < 0) return ORACLE_ERR_NOMEM;
    free(lst);
    *count = c;
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------
 * Neumaier's improved Kahan summation (A. Neumaier, 1974).
 * ---------------------------------------------------------------------- */
typedef struct { double s, c; } nsum_t;
static inline void nsum_add(nsum_t *a, double v) {
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}
static inline double nsum_get(const nsum_t *a) { return a->s + a->c; }

/* Re <u|v> over the domain, compensated, reduced in a fixed order. */
static double re_dot(const domain_t *d, const double *u, const double *v) {
    nsum_t acc = {0.0, 0.0};
    for (int64_t i = 0; i < d->count; ++i) {
        uint64_t x = dom_at(d, i);
        nsum_add(&acc, u[2 * x] * v[2 * x]);
        nsum_add(&acc, u[2 * x + 1] * v[2 * x + 1]);
    }
    return nsum_get(&acc);
}

/* ------------------------------------------------------------------------
 * H |psi> by Eq. 2 applied literally: every (P,Q) and (P,Q,R,S) term with a
 * nonzero integral acts on every basis state with a nonzero amplitude.
 * Single-threaded scatter.  sigma gets H psi + e_core psi.
 * ---------------------------------------------------------------------- */
int oracle_h_apply_eq2(int n_orb, const double *h, const double *eri, double e_core,
                       const double *psi, double *sigma) {
    int n = 2 * n_orb;
    if (n_orb < 1 || n > 30) return ORACLE_ERR_ARG;
    uint64_t N = 1ull << n;
    memset(sigma, 0, sizeof(double) * 2 * N);
    for (uint64_t x = 0; x < N; ++x) {
        double pr = psi[2 * x], pi = psi[2 * x + 1];
        if (pr == 0.0 && pi == 0.0) continue;
        sigma[2 * x] += e_core * pr;
        sigma[2 * x + 1] += e_core * pi;
        for (int P = 0; P < n; ++P)
            for (int Q = 0; Q < n; ++Q) {
                double c = h_so(n_orb, h, P, Q);
                if (c == 0.0) continue;
                int idx[2] = {P, Q}, dag[2] = {1, 0};
                uint64_t y;
                int s = apply_ladder_string(2, idx, dag, x, &y);
                if (!s) continue;
                sigma[2 * y] += c * s * pr;
                sigma[2 * y + 1] += c * s * pi;
            }
        for (int P = 0; P < n; ++P)
            for (int Q = 0; Q < n; ++Q)
                for (int R = 0; R < n; ++R)
                    for (int S = 0; S < n; ++S) {
                        double g = g_so(n_orb, eri, P, Q, R, S);
                        if (g == 0.0) continue;
                        /* a^dag_P a^dag_Q a_S a_R */
                        int idx[4] = {P, Q, S, R}, dag[4] = {1, 1, 0, 0};
                        uint64_t y;
                        int s = apply_ladder_string(4, idx, dag, x, &y);
                        if (!s) continue;
                        sigma[2 * y] += 0.5 * g * s * pr;
                        sigma[2 * y + 1] += 0.5 * g * s * pi;
                    }
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------
 * H |psi> by the Slater-Condon rules, determinant driven, gather form:
 *   sigma_x = sum_{x'} <x|H|x'> psi_{x'}, with <x|H|x'> = <x'|H|x> for the
 * real symmetric H of real integrals, evaluated with x as the ket:
 *   diagonal  sum_I h_II + 1/2 sum_{I,J} (<IJ|IJ> - <IJ|JI>) + e_core
 *   single    I->A: sgn (h_AI + sum_{J occ, J != I} (<AJ|IJ> - <AJ|JI>))
 *   double    IJ->AB: sgn (<AB|IJ> - <AB|JI>)
 * where sgn is the ladder sign of a^dag_A a_I |x> or a^dag_A a^dag_B a_J a_I |x>.
 * Only spin-conserving replacements are enumerated (the others vanish).
 * ---------------------------------------------------------------------- */
static int h_apply_sc_dom(int n_orb, const double *h, const double *eri, double e_core,
                          const domain_t *d, const double *psi, double *sigma) {
    int n = 2 * n_orb;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
    for (int64_t ii = 0; ii < d->count; ++ii) {
        uint64_t x = dom_at(d, ii);
        int occ[64], vir[64], no = 0, nv = 0;
        for (int P = 0; P < n; ++P) {
            if ((x >> P) & 1u) occ[no++] = P;
            else vir[nv++] = P;
        }
        double diag = e_core;
        for (int a = 0; a < no; ++a) {
            int I = occ[a];
            diag += h_so(n_orb, h, I, I);
            for (int b = 0; b < no; ++b) {
                int J = occ[b];
                diag += 0.5 * (g_so(n_orb, eri, I, J, I, J) - g_so(n_orb, eri, I, J, J, I));
            }
        }
        double sr = diag * psi[2 * x], si = diag * psi[2 * x + 1];
        /* singles */
        for (int a = 0; a < no; ++a)
            for (int b = 0; b < nv; ++b) {
                int I = occ[a], A = vir[b];
                if ((I & 1) != (A & 1)) continue;
                int idx[2] = {A, I}, dag[2] = {1, 0};
                uint64_t y;
                int s = apply_ladder_string(2, idx, dag, x, &y);
                if (!s) continue;
                if (d->list && !in_sector(y, d->n_qubits, d->n_alpha, d->n_beta)) { bad = 1; continue; }
                double m = h_so(n_orb, h, A, I);
                for (int c = 0; c < no; ++c) {
                    int J = occ[c];
                    if (J == I) continue;
                    m += g_so(n_orb, eri, A, J, I, J) - g_so(n_orb, eri, A, J, J, I);
                }
                m *= s;
                sr += m * psi[2 * y];
                si += m * psi[2 * y + 1];
            }
        /* doubles */
        for (int a = 0; a < no; ++a)
            for (int a2 = a + 1; a2 < no; ++a2)
                for (int b = 0; b < nv; ++b)
                    for (int b2 = b + 1; b2 < nv; ++b2) {
                        int I = occ[a], J = occ[a2], A = vir[b], B = vir[b2];
                        double m = g_so(n_orb, eri, A, B, I, J) - g_so(n_orb, eri, A, B, J, I);
                        if (m == 0.0) continue;
                        int idx[4] = {A, B, J, I}, dag[4] = {1, 1, 0, 0};
                        uint64_t y;
                        int s = apply_ladder_string(4, idx, dag, x, &y);
                        if (!s) continue;
                        if (d->list && !in_sector(y, d->n_qubits, d->n_alpha, d->n_beta)) { bad = 1; continue; }
                        m *= s;
                        sr += m * psi[2 * y];
                        si += m * psi[2 * y + 1];
                    }
        sigma[2 * x] = sr;
        sigma[2 * x + 1] = si;
    }
    return bad ? ORACLE_ERR_SECTOR : ORACLE_OK;
}

int oracle_h_apply_sc(int n_orb, const double *h, const double *eri, double e_core,
                      const double *psi, double *sigma) {
    int n = 2 * n_orb;
    if (n_orb < 1 || n > 30) return ORACLE_ERR_ARG;
    domain_t d = {n, 0, 0, NULL, (int64_t)(1ull << n)};
    return h_apply_sc_dom(n_orb, h, eri, e_core, &d, psi, sigma);
}

/* ------------------------------------------------------------------------
 * Excitation generator G = tau - tau^dag (Eq. 4).  ex = (i, j, a, b) with
 * j = b = -1 for a single.  out = G psi over the domain (out zeroed on the
 * domain first; each output index is written by one input index at most,
 * since tau and tau^dag are injective and have disjoint ranges).
 * ---------------------------------------------------------------------- */
static int apply_generator_dom(const int32_t *ex, const domain_t *d,
                               const double *psi, double *out) {
    int i = ex[0], j = ex[1], a = ex[2], b = ex[3];
    int single = (j < 0);
    int t_idx[4], t_dag[4], td_idx[4], td_dag[4], len;
    if (single) {
        /* tau = a^dag_a a_i ; tau^dag = a^dag_i a_a */
        len = 2;
        t_idx[0] = a; t_dag[0] = 1; t_idx[1] = i; t_dag[1] = 0;
        td_idx[0] = i; td_dag[0] = 1; td_idx[1] = a; td_dag[1] = 0;
    } else {
        /* tau = a^dag_a a^dag_b a_j a_i ; tau^dag = a^dag_i a^dag_j a_b a_a */
        len = 4;
        t_idx[0] = a; t_dag[0] = 1; t_idx[1] = b; t_dag[1] = 1;
        t_idx[2] = j; t_dag[2] = 0; t_idx[3] = i; t_dag[3] = 0;
        td_idx[0] = i; td_dag[0] = 1; td_idx[1] = j; td_dag[1] = 1;
        td_idx[2] = b; td_dag[2] = 0; td_idx[3] = a; td_dag[3] = 0;
    }
#pragma omp parallel for schedule(static)
    for (int64_t ii = 0; ii < d->count; ++ii) {
        uint64_t x = dom_at(d, ii);
        out[2 * x] = 0.0;
        out[2 * x + 1] = 0.0;
    }
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t ii = 0; ii < d->count; ++ii) {
        uint64_t x = dom_at(d, ii);
        double pr = psi[2 * x], pi = psi[2 * x + 1];
        if (pr == 0.0 && pi == 0.0) continue;
        uint64_t y;
        int s = apply_ladder_string(len, t_idx, t_dag, x, &y);
        if (s) {
            if (d->list && !in_sector(y, d->n_qubits, d->n_alpha, d->n_beta)) bad = 1;
            else { out[2 * y] += s * pr; out[2 * y + 1] += s * pi; }
        }
        s = apply_ladder_string(len, td_idx, td_dag, x, &y);
        if (s) {
            if (d->list && !in_sector(y, d->n_qubits, d->n_alpha, d->n_beta)) bad = 1;
            else { out[2 * y] -= s * pr; out[2 * y + 1] -= s * pi; }
        }
    }
    return bad ? ORACLE_ERR_SECTOR : ORACLE_OK;
}

int oracle_apply_generator(int n_qubits, const int32_t *ex, const double *psi, double *out) {
    if (n_qubits < 1 || n_qubits > 30) return ORACLE_ERR_ARG;
    domain_t d = {n_qubits, 0, 0, NULL, (int64_t)(1ull << n_qubits)};
    return apply_generator_dom(ex, &d, psi, out);
}

/* U(phi) psi = psi + sin(phi) G psi + (1 - cos(phi)) G^2 psi, in place.
 * Exact because G^3 = -G (the spectrum of G is {0, +i, -i}). */
static int rotate_dom(const int32_t *ex, double phi, const domain_t *d,
                      double *psi, double *t1, double *t2) {
    int rc = apply_generator_dom(ex, d, psi, t1);
    if (rc) return rc;
    rc = apply_generator_dom(ex, d, t1, t2);
    if (rc) return rc;
    double sn = sin(phi), cm = 1.0 - cos(phi);
#pragma omp parallel for schedule(static)
    for (int64_t ii = 0; ii < d->count; ++ii) {
        uint64_t x = dom_at(d, ii);
        psi[2 * x] += sn * t1[2 * x] + cm * t2[2 * x];
        psi[2 * x + 1] += sn * t1[2 * x + 1] + cm * t2[2 * x + 1];
    }
    return ORACLE_OK;
}

int oracle_rotate(int n_qubits, const int32_t *ex, double phi, double *psi) {
    if (n_qubits < 1 || n_qubits > 30) return ORACLE_ERR_ARG;
    uint64_t N = 1ull << n_qubits;
    double *t1 = (double *)malloc(sizeof(double) * 2 * N);
    double *t2 = (double *)malloc(sizeof(double) * 2 * N);
    if (!t1 || !t2) { free(t1); free(t2); return ORACLE_ERR_NOMEM; }
    domain_t d = {n_qubits, 0, 0, NULL, (int64_t)N};
    int rc = rotate_dom(ex, phi, &d, psi, t1, t2);
    free(t1); free(t2);
    return rc;
}

/* Reference determinant: the n_alpha lowest alpha and n_beta lowest beta
 * spin orbitals occupied. */
static uint64_t hf_index(int n_alpha, int n_beta) {
    uint64_t x = 0;
    for (int p = 0; p < n_alpha; ++p) x |= 1ull << (2 * p);
    for (int p = 0; p < n_beta; ++p) x |= 1ull << (2 * p + 1);
    return x;
}

static int check_excitations(int n_qubits, int K, const int32_t *ijab) {
    for (int k = 0; k < K; ++k) {
        const int32_t *e = ijab + 4 * k;
        int single = e[1] < 0;
        if (single && e[3] >= 0) return 1;
        for (int t = 0; t < 4; ++t) {
            if (single && (t == 1 || t == 3)) continue;
            if (e[t] < 0 || e[t] >= n_qubits) return 1;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * Energy (and optionally the adjoint gradient) of the Trotterised ansatz.
 *   psi = prod over the schedule of exp(theta_k scale G_k) |HF>
 *   E   = <psi|H|psi>  (H includes e_core)
 *   dE/dtheta_k = sum over schedule entries of k of
 *                 scale * 2 Re <lambda|G_k|phi>
 * with phi the state right after that factor and lambda = U_after^dag H psi,
 * swept backwards from phi = psi, lambda = H psi.
 * h_method: 0 = Eq. 2 literal (full domain only), 1 = Slater-Condon.
 * use_sector: 1 = loop over the (n_alpha, n_beta) sector only.
 * psi_out (2 * 2^n doubles) and sigma_out may be NULL.
 * ---------------------------------------------------------------------- */
int oracle_energy_grad(int n_orb, const double *h, const double *eri, double e_core,
                       int n_alpha, int n_beta, int K, const int32_t *ijab,
                       int n_ops, const int32_t *op_k, const double *op_scale,
                       const double *theta, int use_sector, int h_method,
                       double *E, double *grad, double *psi_out, double *sigma_out) {
    int n = 2 * n_orb;
    if (n_orb < 1 || n > 30 || n_alpha < 0 || n_beta < 0 || n_alpha > n_orb || n_beta > n_orb)
        return ORACLE_ERR_ARG;
    if (check_excitations(n, K, ijab)) return ORACLE_ERR_ARG;
    for (int o = 0; o < n_ops; ++o)
        if (op_k[o] < 0 || op_k[o] >= K) return ORACLE_ERR_ARG;
    if (use_sector && h_method == 0) return ORACLE_ERR_ARG;
    uint64_t N = 1ull << n;
    domain_t d = {n, n_alpha, n_beta, NULL, (int64_t)N};
    uint64_t *lst = NULL;
    if (use_sector) {
        int64_t c = sector_list(n, n_alpha, n_beta, &lst);
        if (c < 0) return ORACLE_ERR_NOMEM;
        d.list = lst;
        d.count = c;
    }
    double *psi = (double *)calloc(2 * N, sizeof(double));
    double *sig = (double *)calloc(2 * N, sizeof(double));
    double *t1 = (double *)calloc(2 * N, sizeof(double));
    double *t2 = (double *)calloc(2 * N, sizeof(double));
    int rc = ORACLE_OK;
    if (!psi || !sig || !t1 || !t2) { rc = ORACLE_ERR_NOMEM; goto done; }

    psi[2 * hf_index(n_alpha, n_beta)] = 1.0;
    for (int o = 0; o < n_ops && !rc; ++o) {
        int k = op_k[o];
        rc = rotate_dom(ijab + 4 * k, theta[k] * op_scale[o], &d, psi, t1, t2);
    }
    if (rc) goto done;
    if (h_method == 0) rc = oracle_h_apply_eq2(n_orb, h, eri, e_core, psi, sig);
    else rc = h_apply_sc_dom(n_orb, h, eri, e_core, &d, psi, sig);
    if (rc) goto done;
    *E = re_dot(&d, psi, sig);
    if (psi_out) memcpy(psi_out, psi, sizeof(double) * 2 * N);
    if (sigma_out) memcpy(sigma_out, sig, sizeof(double) * 2 * N);

    if (grad) {
        /* psi becomes phi and sig becomes lambda; both swept backwards. */
        double *t3 = (double *)calloc(2 * N, sizeof(double));
        if (!t3) { rc = ORACLE_ERR_NOMEM; goto done; }
        for (int k = 0; k < K; ++k) grad[k] = 0.0;
        for (int o = n_ops - 1; o >= 0 && !rc; --o) {
            int k = op_k[o];
            const int32_t *ex = ijab + 4 * k;
            double phi = theta[k] * op_scale[o];
            rc = apply_generator_dom(ex, &d, psi, t3);
            if (rc) break;
            grad[k] += op_scale[o] * 2.0 * re_dot(&d, sig, t3);
            rc = rotate_dom(ex, -phi, &d, psi, t1, t2);
            if (rc) break;
            rc = rotate_dom(ex, -phi, &d, sig, t1, t2);
        }
        free(t3);
    }
done:
    free(psi); free(sig); free(t1); free(t2); free(lst);
    return rc;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------
 * Sum of generators A = sum_k theta_k G_k (Eq. 4, G = tau - tau^dag) as a
 * sparse matrix on the (n_alpha, n_beta) sector basis (ascending basis
 * states), one column per basis state, each entry taken from the ladder
 * operators acting on that single state.  This is the exponent of the
 * Trotter-free ansatz exp(T - T^dag)|HF> of Eq. 3.
 * Outputs: col_ptr[dim + 1]; row[nnz] (row positions in the sector list);
 * val[nnz].  With cap < required nnz nothing but *nnz_out is written.
 * ---------------------------------------------------------------------- */
static int64_t sector_pos(const uint64_t *lst, int64_t cnt, uint64_t y) {
    int64_t lo = 0, hi = cnt - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (lst[mid] == y) return mid;
        if (lst[mid] < y) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

int oracle_generator_sum_sector(int n_qubits, int n_alpha, int n_beta, int K, const int32_t *ijab,
                                const double *theta, int64_t cap, int64_t *col_ptr, int64_t *row,
                                double *val, int64_t *nnz_out) {
    if (n_qubits < 1 || n_qubits > 30 || K < 0 || check_excitations(n_qubits, K, ijab))
        return ORACLE_ERR_ARG;
    uint64_t *lst = NULL;
    int64_t cnt = sector_list(n_qubits, n_alpha, n_beta, &lst);
    if (cnt < 0) return ORACLE_ERR_NOMEM;
    int64_t nnz = 0;
    int bad = 0;
    for (int pass = 0; pass < 2 && !bad; ++pass) {
        if (pass == 1 && nnz > cap) break;
        int64_t w = 0;
        for (int64_t c = 0; c < cnt; ++c) {
            if (pass == 1) col_ptr[c] = w;
            for (int k = 0; k < K; ++k) {
                const int32_t *e = ijab + 4 * k;
                int tl[4], tdg[4], ul[4], udg[4], len;
                if (e[1] < 0) {
                    len = 2;
                    tl[0] = e[2]; tdg[0] = 1; tl[1] = e[0]; tdg[1] = 0;
                    ul[0] = e[0]; udg[0] = 1; ul[1] = e[2]; udg[1] = 0;
                } else {
                    len = 4;
                    tl[0] = e[2]; tdg[0] = 1; tl[1] = e[3]; tdg[1] = 1;
                    tl[2] = e[1]; tdg[2] = 0; tl[3] = e[0]; tdg[3] = 0;
                    ul[0] = e[0]; udg[0] = 1; ul[1] = e[1]; udg[1] = 1;
                    ul[2] = e[3]; udg[2] = 0; ul[3] = e[2]; udg[3] = 0;
                }
                uint64_t y;
                int s = apply_ladder_string(len, tl, tdg, lst[c], &y);
                double coef = theta[k];
                if (!s) {
                    s = apply_ladder_string(len, ul, udg, lst[c], &y);
                    coef = -theta[k];
                }
                if (!s) continue;
                if (pass == 1) {
                    int64_t r = sector_pos(lst, cnt, y);
                    if (r < 0) { bad = 1; break; }
                    row[w] = r;
                    val[w] = s * coef;
                }
                ++w;
            }
            if (bad) break;
        }
        if (pass == 0) nnz = w;
        else col_ptr[cnt] = w;
    }
    free(lst);
    if (bad) return ORACLE_ERR_SECTOR;
    *nnz_out = nnz;
    return ORACLE_OK;
}
