/*
 * uccsd.h -- C ABI of the GB300 (sm_103a) VQE-UCCSD state-vector library.
 *
 * The library evaluates the energy and gradient of the Trotterised unitary
 * coupled-cluster singles and doubles ansatz used for the correlation step
 * of the FMO scheme in Sugisaki, Nakano and Mochizuki, "Size-consistency and
 * orbital-invariance issues revealed by VQE-UCCSD calculations with the FMO
 * scheme" (arXiv:2402.17993):
 *
 *   H      = sum_pq h_pq a+_p a_q + 1/2 sum_pqrs g_pqrs a+_p a+_q a_s a_r   (Eq. 2)
 *   |Psi>  = exp(T - T+) |Psi_HF>                                           (Eq. 3)
 *   T      = sum t_i^a a+_a a_i + 1/2 sum t_ij^ab a+_a a+_b a_j a_i        (Eq. 4)
 *   exp(T - T+) ~ [ prod_k exp(theta_k G_k / M) ]^M   (first order, Eq. 5)
 *   second order: [ prod_{1..K} exp(theta G/2M) prod_{K..1} exp(theta G/2M) ]^M (Eq. 6)
 *   E      = <Psi|H|Psi>   (Section 2.3; evaluated exactly, no shot noise)
 *
 * Conventions (this library's readings of the paper, stated once here):
 *   - Jordan-Wigner mapping; spin orbital P = 2p + s (s = 0 alpha, 1 beta) is
 *     qubit P, and bit P of a basis index is its occupation.
 *   - g_pqrs of Eq. 2 = <pq|rs> = (pr|qs) from chemist-notation spatial
 *     integrals eri[p][q][r][s] = (pq|rs), with spin deltas.
 *   - |Psi_HF> occupies the n_alpha lowest alpha and n_beta lowest beta
 *     spin orbitals.
 *   - One amplitude per excitation row (i, j, a, b) over spin orbitals;
 *     singles use j = b = -1.  Generator G = tau - tau+ with
 *     tau = a+_a a_i (single) or a+_a a+_b a_j a_i (double).
 *   - The excitation list is the circuit order: row 0 acts first on |HF>.
 *   - The gradient is dE/dtheta_k of the same Trotterised energy, from one
 *     adjoint (reverse) sweep.
 *
 * Ownership: the caller owns every array passed in; the library copies what
 * it keeps before returning.  A context owns all device memory it allocates
 * and frees it in uccsd_destroy.  Device outputs are written on `stream`
 * (a cudaStream_t passed as void*; NULL = legacy default stream) and are
 * ready when that stream reaches the point of the call.  Host outputs are
 * valid when the call returns (the call synchronises `stream`).
 *
 * Errors: every call returns a uccsd_status; nothing is thrown across the
 * ABI and nothing exits.  uccsd_last_error() describes the last failure of a
 * context.  A CUDA error marks the context as failed; later compute calls
 * return UCCSD_ERR_STATE.
 *
 * Threading: a context is not thread-safe; use one context per host thread
 * and stream.  Distinct contexts are independent.
 */
#ifndef UCCSD_GB300_H
#define UCCSD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct uccsd_ctx uccsd_ctx;

typedef enum {
    UCCSD_OK = 0,
    UCCSD_ERR_ARG = 1,     /* invalid argument (value, range, symmetry, finiteness) */
    UCCSD_ERR_OOM = 2,     /* device allocation failed */
    UCCSD_ERR_CUDA = 3,    /* a CUDA runtime call or kernel failed */
    UCCSD_ERR_STATE = 4,   /* call order violated or context failed earlier */
    UCCSD_ERR_TIMEOUT = 5, /* a bounded device wait gave up */
    UCCSD_ERR_BUDGET = 6   /* requested footprint exceeds the context's HBM budget */
} uccsd_status;

typedef enum {
    UCCSD_FP64 = 0,       /* complex128 state, FP64 arithmetic throughout */
    UCCSD_FP32_STATE = 1  /* 8-byte FP32 state slots and FP32 rotations; FP64 energy and
                             gradient reductions.  The method's amplitudes are real (real
                             integrals, real generators, real reference), so a slot holds
                             one real amplitude as the unevaluated sum hi + lo of two FP32
                             words, lo the rounding error of hi kept by error-free
                             transformations (TwoSum, FMA) */
} uccsd_prec;

typedef enum {
    UCCSD_LAYOUT_FULL = 0,   /* each slot is the full 2^n amplitude vector (index = occupation bits) */
    UCCSD_LAYOUT_SECTOR = 1, /* each slot holds only the (n_alpha, n_beta) sector: C(n_orb, n_alpha) x
                                C(n_orb, n_beta) amplitudes, alpha-string rank major, strings ascending */
    UCCSD_LAYOUT_SCBK = 2    /* each slot is the 2^(n-2) vector of the symmetry-conserving
                                Bravyi-Kitaev encoding with its two parity qubits tapered off
                                (the paper's qubit counts, Section 2.3), in the qubit order of
                                uccsd_pauli_terms_scbk: the determinant (alpha string sa, beta
                                string sb) sits at the tapered Bravyi-Kitaev image of its
                                up-then-down occupation vector, which splits as f(sa) + g(sb) */
} uccsd_layout;

typedef struct {
    int n_qubits;         /* 2 * n_orb */
    int n_orb, n_alpha, n_beta;
    int K;                /* excitations (amplitudes) */
    int n_ops;            /* factors in the Trotter schedule (K * M or 2 * K * M) */
    int n_groups;         /* X-mask groups of the Jordan-Wigner Hamiltonian */
    int n_terms;          /* Pauli terms of the Jordan-Wigner Hamiltonian */
    int n_fwd_runs;       /* shared-memory passes of the forward sweep */
    int n_adj_runs;       /* shared-memory passes of the adjoint sweep */
    int batch;            /* state slots reserved */
    int precision;        /* uccsd_prec */
    int layout;           /* uccsd_layout */
    size_t device_bytes;  /* device memory held by the context alone (the
                             precomputed pair lists of a plan are one copy
                             per device, shared by all contexts of the plan,
                             and not counted here) */
    uint64_t launches;    /* kernels launched by this context so far */
} uccsd_info_t;

/* Create a context on CUDA device `device`.  hbm_budget_bytes = 0 means no
 * budget; otherwise allocations that would exceed it fail with
 * UCCSD_ERR_BUDGET before touching the device.  *out = NULL on failure. */
uccsd_status uccsd_create(uccsd_ctx **out, int device, uccsd_prec prec,
                          size_t hbm_budget_bytes);

/* Free all device memory of the context.  NULL is accepted. */
void uccsd_destroy(uccsd_ctx *ctx);

/* Stream of the context's set-up transfers: the uploads, clears and
 * reallocations made by uccsd_set_hamiltonian, uccsd_set_reference,
 * uccsd_set_excitations, uccsd_set_batch and uccsd_opt_init.
 *   stream NULL (the default): the context's own non-blocking stream; each
 *          set-up call waits for its transfers before it returns.
 *   stream a cudaStream_t: the transfers are enqueued on it (host arrays are
 *          first copied to pinned staging owned by the context) and the calls
 *          return without waiting.  Work launched later on the same stream
 *          sees the data; the caller orders work on other streams after it,
 *          and must not change the context's problem while earlier work that
 *          reads it is still running.
 * A host that sets up many contexts while others compute uses this form:
 * a host wait on any stream can be held up by unrelated work that shares its
 * hardware queue.  Switching streams first waits for the copies staged on the
 * previous one.  Errors: UCCSD_ERR_STATE on a failed context, UCCSD_ERR_CUDA
 * if that wait fails. */
uccsd_status uccsd_set_setup_stream(uccsd_ctx *ctx, void *stream);

/* Context-owned message of the last failure; valid until the next call on
 * the context.  Never NULL. */
const char *uccsd_last_error(const uccsd_ctx *ctx);

/* Static name of a status code. */
const char *uccsd_status_string(uccsd_status st);

/* Hamiltonian of Eq. 2 (Section 2.2) from spatial integrals.
 *   h    n_orb*n_orb row-major, symmetric to 1e-12 (host pointer)
 *   eri  n_orb^4 row-major chemist (pq|rs) with 8-fold symmetry to 1e-12
 *   e_core constant energy added to H.
 * 1 <= n_orb <= 15.  The Jordan-Wigner compile (X-mask/Z-mask grouping)
 * runs on the host; its tables are copied to the device.  Non-finite or
 * asymmetric input -> UCCSD_ERR_ARG.  Invalidates excitations and state. */
uccsd_status uccsd_set_hamiltonian(uccsd_ctx *ctx, int n_orb, const double *h,
                                   const double *eri, double e_core);

/* State layout in device memory (default UCCSD_LAYOUT_FULL).  The
 * Hamiltonian and the ansatz conserve the alpha and beta electron counts, so
 * only the amplitudes of the (n_alpha, n_beta) sector are ever nonzero; every
 * kernel touches only those.  UCCSD_LAYOUT_FULL keeps them at their place in
 * the 2^n vector (the rest stays zero); UCCSD_LAYOUT_SECTOR stores them as a
 * dense C(n_orb, n_alpha) x C(n_orb, n_beta) array (4.4% of 2^n at 26
 * qubits); UCCSD_LAYOUT_SCBK keeps them at their place in the 2^(n-2)
 * vector of the tapered symmetry-conserving Bravyi-Kitaev encoding (the
 * paper's qubit counts: 16 qubits for an 18-qubit Jordan-Wigner fragment).
 * The arithmetic and its order are identical, so energies and gradients are
 * bitwise the same in all three layouts.  uccsd_get_state returns the 2^n
 * vector in the first two and the tapered vector in the third.  Must come
 * before uccsd_set_reference (after
 * uccsd_set_hamiltonian, which clears the reference, it may be called again);
 * otherwise UCCSD_ERR_STATE.  Unknown layout: UCCSD_ERR_ARG. */
uccsd_status uccsd_set_layout(uccsd_ctx *ctx, int layout);

/* Reference determinant |Psi_HF> (Eq. 3): n_alpha, n_beta electrons in the
 * lowest spin orbitals of each spin.  Needs the Hamiltonian first. */
uccsd_status uccsd_set_reference(uccsd_ctx *ctx, int n_alpha, int n_beta);

/* Stateless builder of the spin-conserving UCCSD list of Eq. 4: singles
 * (i, -1, a, -1) with i occupied, a virtual, same spin; then doubles
 * (i, j, a, b), i < j occupied, a < b virtual, spin multiset conserved;
 * each block in lexicographic order.  Writes min(count, cap) rows of 4
 * int32 to `out` (host; may be NULL when cap = 0) and the full count to
 * *n_out. */
uccsd_status uccsd_build_uccsd_list(int n_orb, int n_alpha, int n_beta,
                                    int32_t *out, int cap, int *n_out);

/* Ordered excitation list (host, K rows of (i, j, a, b); j = b = -1 for
 * singles) and the Trotter schedule of Eq. 5 (trotter_order = 1) or Eq. 6
 * (trotter_order = 2) with n_slices = M >= 1.  Every row must map occupied
 * to virtual orbitals of |Psi_HF> and conserve spin.  Needs the reference. */
uccsd_status uccsd_set_excitations(uccsd_ctx *ctx, int K, const int32_t *ijab,
                                   int trotter_order, int n_slices);

/* Reserve B >= 1 state slots for the batched call (default 1). */
uccsd_status uccsd_set_batch(uccsd_ctx *ctx, int B);

/* Energy of slot 0 for amplitudes theta[K].  theta_on_device != 0: theta
 * and E are device pointers (E: one double), written on `stream`;
 * otherwise host pointers and the call synchronises. */
uccsd_status uccsd_energy(uccsd_ctx *ctx, const double *theta, int theta_on_device,
                          double *E, void *stream);

/* Energy and the gradient dE/dtheta[K] (adjoint sweep) of slot 0.
 * grad has the residency of theta. */
uccsd_status uccsd_energy_grad(uccsd_ctx *ctx, const double *theta, int theta_on_device,
                               double *E, double *grad, void *stream);

/* B independent evaluations of the same fragment: theta is B*K row-major,
 * E is B, grad is B*K (or NULL for energies only).  1 <= B <= reserved
 * batch.  Same residency rules as uccsd_energy_grad. */
uccsd_status uccsd_energy_grad_batch(uccsd_ctx *ctx, int B, const double *theta,
                                     int theta_on_device, double *E, double *grad,
                                     void *stream);

/* One call over B contexts, for example the monomer and dimer fragments of
 * an FMO job (Eq. 1), each with its own Hamiltonian, reference and list:
 * thetas[i] (K_i doubles), grads[i] (K_i doubles, or grads = NULL for
 * energies only) and E (B doubles) are device pointers.  Each evaluation
 * runs on its context's own stream, forked from `stream` and joined back
 * into it, so the fragments overlap on the device; outputs are ready when
 * `stream` reaches the point of the call (also inside a stream capture).
 * A context may appear more than once (its evaluations run in order).
 * Errors: UCCSD_ERR_ARG for a null pointer or contexts on different
 * devices, UCCSD_ERR_STATE for a failed context or one without
 * excitations; every context is checked before anything is enqueued. */
uccsd_status uccsd_energy_grad_batched(uccsd_ctx *const *ctxs, int B, const double *const *thetas,
                                       double *E, double *const *grads, void *stream);

/* Capture one B-slot evaluation (as uccsd_energy_grad_batch with device
 * pointers: theta B*K, E B, grad B*K or NULL) into a CUDA graph owned by the
 * context, replacing any earlier capture.  The graph keeps the pointers:
 * each uccsd_replay re-reads theta from the same buffer and rewrites E and
 * grad.  Nothing runs during the capture itself.  Profiling must be off.
 * Used by serving loops to replace an evaluation's kernel launches by one
 * graph launch (the paper's per-evaluation cost, Section 3.1, is dominated
 * by overheads the GPU cannot hide). */
uccsd_status uccsd_capture(uccsd_ctx *ctx, int B, const double *theta_dev, double *E_dev,
                           double *grad_dev, void *stream);

/* Launch the captured graph on `stream`. */
uccsd_status uccsd_replay(uccsd_ctx *ctx, void *stream);

/* Copy the state vector of slot `slot` after the last uccsd_energy or
 * energies-only batch call to host memory as 2*2^n interleaved (re, im)
 * doubles (UCCSD_FP32_STATE: re = hi + lo, im = 0); in UCCSD_LAYOUT_SCBK
 * the 2*2^(n-2) doubles of the tapered encoding, in the phase convention of
 * its up-then-down orbital order (the amplitudes that
 * uccsd_pauli_terms_scbk's Hamiltonian acts on).  len must be >= 2*2^n.  Synchronises the context's last stream.
 * After a gradient call the slot's content is unspecified (the adjoint
 * sweep may leave it partly swept back). */
uccsd_status uccsd_get_state(uccsd_ctx *ctx, int slot, double *out_re_im, size_t len);

/* Sizes and counters of the context. */
uccsd_status uccsd_info(const uccsd_ctx *ctx, uccsd_info_t *info);

/* Kernel families of the evaluation, for uccsd_get_profile. */
enum {
    UCCSD_K_CS = 0,       /* cos/sin of the schedule factors */
    UCCSD_K_FORWARD = 1,  /* forward sweep passes (Eq. 5 / Eq. 6) */
    UCCSD_K_HAPPLY = 2,   /* H psi and energy partials (Eq. 2, Section 2.3) */
    UCCSD_K_ADJOINT = 3,  /* adjoint sweep passes (gradient) */
    UCCSD_K_REDUCE = 4,   /* final energy/gradient reductions */
    UCCSD_K_FAMILIES = 5
};

typedef struct {
    double ms[UCCSD_K_FAMILIES];        /* accumulated device time per family */
    uint64_t launches[UCCSD_K_FAMILIES];
    uint64_t calls;                     /* evaluations profiled */
} uccsd_profile_t;

/* Profiling (off by default): with on != 0 every evaluation records CUDA
 * events around each kernel family on the evaluation stream and
 * synchronises at its end to accumulate the device times; on = 0 stops it.
 * Either call resets the accumulators. */
uccsd_status uccsd_set_profiling(uccsd_ctx *ctx, int on);
uccsd_status uccsd_get_profile(const uccsd_ctx *ctx, uccsd_profile_t *out);

/* Energy of a state vector that the caller already holds on the device,
 * computed without allocating any device memory.  The paper has no
 * counterpart; it exists for callers that cannot call cudaMalloc when they
 * need an energy: serving or real-time loops held to a memory budget
 * reserved up front (an allocation there may fail, or stall the device
 * while other work is in flight), and plugins inside programs whose device
 * allocator belongs to another framework (memory taken behind that
 * allocator's back is memory it cannot account for).
 *
 *   ctx    context with set_hamiltonian and set_reference done (its tables
 *          were uploaded then; set_excitations is not needed)
 *   psi    device pointer to 2^n amplitudes in the context's precision
 *          (complex128 for UCCSD_FP64, complex64 for UCCSD_FP32_STATE),
 *          interleaved (re, im); only entries with n_alpha alpha and n_beta
 *          beta electrons are read (the others must be zero)
 *   E      device pointer to one double, written on `stream`:
 *          <psi|H|psi> (UCCSD_FP64) or <psi|H|psi>/<psi|psi> (FP32 state),
 *          the same quantity the context's evaluations report
 *
 * Scratch: a fixed device array of 2 * UCCSD_NOALLOC_MAX_TILES doubles
 * (64 KiB) inside the library, held by every GPU that loads the library
 * until the process exits: two partials per H-apply tile, and a state has
 * C(n_orb, n_alpha) * ceil(C(n_orb, n_beta) / 2048) tiles.  That covers
 * every closed-shell state up to 26 qubits (1716 tiles at 13 orbitals and
 * 6 + 6 electrons); a state with more tiles (28 qubits at 7 + 7 electrons:
 * 6864) is rejected with UCCSD_ERR_ARG.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture.  All calls in the process share the array and
 * it keeps the last call's partials; each call overwrites what it reads, so
 * nothing has to be cleared, but calls that overlap on the GPU (different
 * streams or contexts without ordering between them) race on it. */
#define UCCSD_NOALLOC_MAX_TILES 4096
uccsd_status uccsd_expectation_noalloc(uccsd_ctx *ctx, const void *psi, double *E,
                                       void *stream);

/* Host-only: Jordan-Wigner compile statistics of the Hamiltonian of Eq. 2
 * without creating a context (no device use).  Any output may be NULL. */
uccsd_status uccsd_hamiltonian_stats(int n_orb, const double *h, const double *eri,
                                     double e_core, int *n_groups, int *n_terms);

/* Host-only check hook (no device use): the precomputed pair lists that the
 * excitation sweeps apply for an excitation list (Eq. 5, first order, one
 * slice), expanded to determinants.  The forward sweep's plan for nvec = 1,
 * the adjoint's for nvec = 2, with amplitudes of amp_bytes bytes (8 for the
 * FP32 state, 16 for FP64).  Row i of out (cap rows of 7 int32, row-major):
 *   factor  schedule index of the factor (the excitation row here)
 *   first, second  the determinants (bit q = occupation of spin orbital q)
 *           whose amplitudes the sweep rotates as
 *           first' = c first - sign s second, second' = c second + sign s first
 *           with c, s the cosine and sine of the factor's angle; both -1 for
 *           the padding pairs that complete a bank-conflict-free group
 *   sign    +1 or -1
 *   entry, partner entry  the two tile entries (shared-memory slots)
 *   index   position of the pair in its factor's list for its tile.
 * Writes min(count, cap) rows and *n_out = count.  UCCSD_ERR_ARG for an
 * invalid list or arguments, or a plan too large for precomputed lists. */
uccsd_status uccsd_plan_pairs(int n_orb, int n_alpha, int n_beta, const int32_t *ijab, int K,
                              int amp_bytes, int nvec, int32_t *out, int cap, int *n_out);

/* Host-only check hook (no device use): the order in which the FP32
 * H-apply (Eq. 2, one column of beta strings per thread) takes each
 * column's beta single excitations in its mixed alpha-beta groups.  The
 * C(n_orb, n_beta) columns are the beta strings in ascending order; a
 * column's ns = n_beta (n_orb - n_beta) singles j -> b in natural order are
 * j occupied ascending, then b empty ascending.  out[t * C(n_orb, n_beta) +
 * column] = the natural index of the single taken at slot t.  Every order
 * gives the same contributions; this one is chosen per group of eight
 * columns against shared-memory bank conflicts.  Writes min(count, cap)
 * entries and *n_out = count; UCCSD_ERR_ARG for sizes outside
 * 1 <= n_orb <= 15, 0 <= n_beta <= n_orb. */
uccsd_status uccsd_happly_mixed_order(int n_orb, int n_beta, int32_t *out, int cap, int *n_out);

/* Host-only check hook (no device use): the entry maps of the sweep plan
 * (Eq. 5, first order, one slice; the forward's plan for nvec = 1, the
 * adjoint's for nvec = 2, amplitudes of amp_bytes bytes), by which the
 * sweeps read and write their tiles in the sector order.  One row of 5
 * int32 per entry of every tile of every run that holds sector entries:
 *   run, tile, entry  the run, its tile (CTA) and the tile entry
 *   index             the map's sector index of the entry: rank of its alpha
 *                     string x C(n_orb, n_beta) + rank of its beta string,
 *                     strings ranked in ascending order within a popcount
 *   det               the entry's determinant (bit q = occupation of spin
 *                     orbital q), decoded independently of the map
 * Writes min(count, cap) rows and *n_out = count.  UCCSD_ERR_ARG for an
 * invalid list or arguments, or a plan of more than 2^26 map entries. */
uccsd_status uccsd_plan_entry_map(int n_orb, int n_alpha, int n_beta, const int32_t *ijab, int K,
                                  int amp_bytes, int nvec, int32_t *out, int cap, int *n_out);

/* Host-only: the compiled Jordan-Wigner Pauli terms of Eq. 2 in the
 * X^x Z^z form: H = sum_t coef[t] X^{xmask[t]} Z^{zmask[t]}, where
 * X^x Z^z |y> = (-1)^{popcount(y & z)} |y ^ x>.  Writes min(count, cap)
 * terms and *n_out = count.  Any array may be NULL when cap = 0. */
uccsd_status uccsd_pauli_terms(int n_orb, const double *h, const double *eri, double e_core,
                               uint32_t *xmask, uint32_t *zmask, double *coef, int cap,
                               int *n_out);

/* Energy of the Trotter-free ansatz (Eq. 3), the reference of Section 3.2
 * (the paper computes it with SciPy's expm_multiply):
 *   |Psi> = exp(sum_k theta_k G_k) |HF>,   E = <Psi|H|Psi>,
 * for the context's excitation list (its order, trotter_order and n_slices
 * do not enter).  exp is a truncated Taylor series on the device in s steps
 * of m terms, chosen from the bound ||sum theta_k G_k|| <= sum |theta_k| so
 * that the truncation error of the state stays below the state precision's
 * unit roundoff (2^-53 FP64, 2^-24 FP32 state); cost s*m generator-sum
 * passes, about sum |theta_k| * 20.  theta: K doubles on the host
 * (theta_on_device = 0) or the device (1; read back to the host for the
 * step choice); E: one double, same residency.  Synchronises `stream`.
 * Afterwards uccsd_get_state(ctx, 0, ...) returns |Psi>.  Errors:
 * UCCSD_ERR_STATE before set_excitations, UCCSD_ERR_ARG for null or non-
 * finite theta; uses two extra state vectors of device memory (allocated on
 * first use, counted against the HBM budget: UCCSD_ERR_BUDGET). */
uccsd_status uccsd_energy_trotter_free(uccsd_ctx *ctx, const double *theta, int theta_on_device,
                                       double *E, void *stream);

/* Energy and gradient of the Trotter-free ansatz (see uccsd_energy_trotter_free).
 * The gradient is the Duhamel integral
 *   dE/dtheta_k = 2 int_0^1 Re <lambda(tau)|G_k|phi(tau)> dtau,
 *   phi(tau) = exp(tau A)|HF>,  lambda(tau) = exp(tau A) exp(-A) (H - s)|Psi>,
 * A = sum_k theta_k G_k, by Gauss-Legendre quadrature with the node count
 * chosen from a derivative bound of the integrand; cost about four times
 * the energy's.  grad: K doubles, same residency as theta.  Afterwards the
 * device state is not |Psi> (uccsd_get_state returns UCCSD_ERR_STATE). */
uccsd_status uccsd_energy_grad_trotter_free(uccsd_ctx *ctx, const double *theta, int theta_on_device,
                                            double *E, double *grad, void *stream);

/* ---- Device optimiser for the serving loop (no counterpart in the paper, which
 *      used COBYLA and Powell; Section 2.3) ---- */

/* Fixed-step L-BFGS on the device (two-loop recursion, Nocedal and Wright
 * Algorithm 7.4): memory m in [1, 32] pairs, steps capped at max_step in the
 * max-norm, the first step -first_scale * grad; pairs with s.y <= 1e-16
 * max(1, y.y) are not stored.  Allocates (2 m + 3) K + m doubles of state and
 * max_steps doubles of energy history and resets them.  Requires
 * uccsd_set_excitations (which discards the optimiser).  Errors:
 * UCCSD_ERR_STATE, UCCSD_ERR_ARG for parameters out of range,
 * UCCSD_ERR_BUDGET / UCCSD_ERR_OOM. */
uccsd_status uccsd_opt_init(uccsd_ctx *ctx, int memory, double max_step, double first_scale,
                            int max_steps);

/* One optimiser step on `stream`, asynchronous: theta (K doubles, device) is
 * the point at which E (one double, device) and grad (K doubles, device)
 * were evaluated; it is replaced by the next point, and E is appended to the
 * history (the first max_steps steps).  One single-CTA kernel. */
uccsd_status uccsd_opt_step(uccsd_ctx *ctx, double *theta, const double *E, const double *grad,
                            void *stream);

/* Capture one VQE iteration of a single-slot solve into the context's graph
 * (replacing any earlier capture): the energy and adjoint gradient at
 * theta_dev (K doubles on the device) into E_dev (1) and grad_dev (K),
 * followed by one uccsd_opt_step that updates theta_dev in place.  Each
 * uccsd_replay then runs one iteration of the Section 2.3 loop (ansatz
 * state, energy, gradient, classical update) as one graph launch.  Needs
 * uccsd_opt_init first; the optimiser history advances on every replay.
 * The graph holds the optimiser buffers' addresses, which a later
 * uccsd_opt_init may change (histories of more than 1022 steps live in
 * device buffers, shorter ones in a record of a process-wide pinned block):
 * capture again after calling uccsd_opt_init.
 * Errors as uccsd_capture; UCCSD_ERR_STATE without uccsd_opt_init. */
uccsd_status uccsd_capture_vqe_step(uccsd_ctx *ctx, double *theta_dev, double *E_dev,
                                    double *grad_dev, void *stream);

/* Energies recorded by uccsd_opt_step, in step order, to host E (min(steps,
 * cap) doubles); *n_out = steps recorded.  Synchronises the last stream the
 * optimiser ran on. */
uccsd_status uccsd_opt_history(uccsd_ctx *ctx, double *E, int cap, int *n_out);

/* ---- Bounded device wait of the serving loop (no counterpart in the paper,
 *      whose fragment jobs ran one after another; Section 3.1) ---- */

/* Enqueue on `stream` (not the default stream) a gate: a one-thread kernel
 * that waits until *flag >= target and then lets the work enqueued behind
 * it on the stream run.  A server prepares a fragment and enqueues its solve
 * behind a gate before the request is due, then releases the flag at the
 * request's arrival; no host launch is on that path.
 *   flag        device-readable uint32 written by the host: pinned host
 *               memory (readable by the device at the same address under
 *               unified addressing) or device memory that a copy on another
 *               stream writes.  It must not be written by a kernel that is
 *               itself waiting.
 *   timeout_ns  the gate's time limit, in (0, 10 s].  The gate polls about
 *               every microsecond; when the limit passes (or an iteration
 *               cap derived from it, should the GPU's timer stall) it gives
 *               up, records that, and returns.  The work behind it then runs
 *               anyway; uccsd_gate_status tells the caller to discard it.
 * While gates wait, the thread that releases them must not make a call
 * that waits for the device (cudaDeviceSynchronize, cudaFree, cudaFreeHost,
 * a pinned allocation, a synchronous copy): it would wait for the gates it
 * is to release, until their time limit.  The flag must stay allocated
 * until the gate has finished.
 * One gate per context at a time: UCCSD_ERR_STATE while the previous one is
 * still waiting.  Errors: UCCSD_ERR_ARG for a null flag or stream or a
 * limit out of range, UCCSD_ERR_CUDA if the launch fails. */
uccsd_status uccsd_gate_enqueue(uccsd_ctx *ctx, const uint32_t *flag, uint32_t target,
                                uint64_t timeout_ns, void *stream);

/* State of the context's last gate.  wait != 0 blocks until the gate kernel
 * has finished (never longer than its time limit); wait = 0 only looks.
 * *released = 1 once the flag released it (UCCSD_OK); *released = 0 with
 * UCCSD_OK while it is still waiting; UCCSD_ERR_TIMEOUT if it gave up.
 * UCCSD_ERR_STATE without a gate. */
uccsd_status uccsd_gate_status(uccsd_ctx *ctx, int wait, int *released);

/* Stream bookkeeping for callers that enqueue work while gates hold the
 * device (the serving loop's preparing threads).  A launch can wait in the
 * driver while a hardware queue is full of work held by a gate; these calls
 * are plain C calls, so a caller's language runtime may let the thread that
 * releases the gates run meanwhile.
 * uccsd_stream_mark records the context's completion marker (an event) on
 * `stream`: it completes when the work enqueued on `stream` before it has.
 * uccsd_mark_done sets *done to 1 once the last recorded marker has
 * completed, else 0 (no wait); UCCSD_ERR_STATE before any mark.
 * uccsd_zero_async enqueues the zeroing of `bytes` bytes of device memory
 * at `ptr` on `stream`.  Errors: UCCSD_ERR_ARG for null arguments,
 * UCCSD_ERR_CUDA if CUDA refuses the call. */
uccsd_status uccsd_stream_mark(uccsd_ctx *ctx, void *stream);
uccsd_status uccsd_mark_done(uccsd_ctx *ctx, int *done);
uccsd_status uccsd_zero_async(uccsd_ctx *ctx, void *ptr, size_t bytes, void *stream);

/* ---- Trotter-schedule helpers (Section 2.3 ordering; Section 3.2 extrapolation) ---- */

/* First-order (Moller-Plesset) amplitude of every excitation of the context's
 * list, the magnitudes by which Section 2.3 orders the cluster operators
 * (magnitude ordering after Tranter et al.):
 *   t_k = <HF|H tau_k|HF> / (eps_i + eps_j - eps_a - eps_b)   (singles: eps_i - eps_a)
 * with eps the Fock diagonal of the reference determinant.  The numerator is
 * half the adjoint gradient at theta = 0, computed on the device by one
 * energy-and-gradient evaluation on `stream` (the call synchronises it); the
 * denominators come from the diagonal of H on the host.  t: host array of K
 * doubles, in list order.  Requires uccsd_set_excitations.  Errors:
 * UCCSD_ERR_STATE before set_excitations, UCCSD_ERR_ARG for a null t or a
 * denominator of magnitude <= 1e-12.  In UCCSD_FP32_STATE contexts the
 * numerators carry FP32 state rounding (relative error about 1e-6). */
uccsd_status uccsd_mp1_amplitudes(uccsd_ctx *ctx, double *t, void *stream);

/* Host-only: magnitude ordering (Section 2.3).  Writes the K rows of ijab
 * (K x 4 int32, the layout of uccsd_set_excitations) to ijab_out in order of
 * decreasing |t[k]|, rows of equal |t| in their input order (a stable sort),
 * and perm[k] = the input index of output row k (perm may be NULL).  ijab_out
 * may alias ijab.  The gradient of a context built from ijab_out is in the
 * output order: grad_in[perm[k]] = grad_out[k].  Errors: UCCSD_ERR_ARG for
 * K < 0, null arrays with K > 0, or a non-finite t. */
uccsd_status uccsd_magnitude_order(int K, const int32_t *ijab, const double *t, int32_t *ijab_out,
                                   int32_t *perm);

/* Host-only: Trotter-error extrapolation (Section 3.2, Fig. 3).  Least-
 * squares fit of E(M) = alpha (1/M)^beta + gamma to n energies E[m] at slice
 * counts M[m] (>= 1, at least 3 distinct values); out[0..2] = alpha, beta,
 * gamma, where gamma estimates the Trotter-free energy.  beta is searched in
 * [1e-3, 64] (variable projection: alpha and gamma solved exactly for each
 * beta).  Errors: UCCSD_ERR_ARG for n < 3, M < 1, fewer than 3 distinct M,
 * non-finite E or null arrays. */
uccsd_status uccsd_trotter_extrapolate(int n, const int *M, const double *E, double *out);

/* Host-only: the Hamiltonian of Eq. 2 under the symmetry-conserving
 * Bravyi-Kitaev encoding with two qubits tapered off (the SCBKT encoding of
 * Section 2.3, giving n - 2 qubits).  Spin orbitals in up-then-down order
 * (alpha p -> p, beta p -> n/2 + p); Bravyi-Kitaev tree by recursive halving,
 * whose node n/2 - 1 holds the alpha-electron parity and root n - 1 the total
 * parity; those two qubits are replaced by the eigenvalues (-1)^n_alpha and
 * (-1)^(n_alpha + n_beta) and removed.  Output terms, in the convention of
 * uccsd_pauli_terms: H = sum coef[t] X^{xmask[t]} Z^{zmask[t]} on
 * *n_qubits_out = 2 n_orb - 2 qubits, merged and sorted; writes min(count,
 * cap) terms, *n_out = count.  The spectrum of the result equals that of H on
 * the states whose alpha and total electron numbers have the parities of
 * n_alpha and n_alpha + n_beta.  Errors: UCCSD_ERR_ARG for n_orb outside
 * [2, 15], electron counts outside [0, n_orb], non-finite integrals or null
 * outputs with cap > 0.  The state-vector path does not use this encoding:
 * its electron-sector layout removes the N_alpha and N_beta symmetries
 * entirely. */
uccsd_status uccsd_pauli_terms_scbk(int n_orb, const double *h, const double *eri, double e_core,
                                    int n_alpha, int n_beta, uint32_t *xmask, uint32_t *zmask,
                                    double *coef, int cap, int *n_out, int *n_qubits_out);

#ifdef __cplusplus
}
#endif
#endif /* UCCSD_GB300_H */
