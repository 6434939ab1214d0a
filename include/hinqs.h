/*
 * hinqs.h -- C ABI of the HI-NQS subspace-diagonalisation library for B300 (sm_103a).
 *
 * The library implements the classical half of the HI-NQS sample-diagonalise-
 * update loop of arXiv 2606.26760: the second-quantised Hamiltonian of Sec. 2.2
 * restricted to the SQD product subspace of sampled alpha and beta strings
 * (Step 3), its Slater-Condon matrix elements, the sigma product H c inside a
 * Davidson solve for the ground state (Step 3), the 1- and 2-RDMs that give the
 * Hellmann-Feynman gradient of the energy, and the spin-marginal teacher weights
 * of Step 4 (Eqs. alpha_marginal and beta_marginal); around the solve, the other
 * classical steps of the iteration: the classical expansion (Step 1'), PT2 scores
 * and the basis update (Step 2), the warm start (Step 3), the loss inputs of the
 * network (Step 4, Eqs. teacher, energy, entropy and loss).
 *
 * Conventions shared by every call
 *  - Orbitals: n_orb spatial orbitals, 1 <= n_orb <= 64.  An occupation string
 *    is a uint64 bitmask, bit p set when spatial orbital p is occupied.
 *  - Integrals: h[p*n+q] (symmetric) and eri[((p*n+q)*n+r)*n+s] = (pq|rs) in
 *    chemist order with the 8-fold real symmetry, FP64.  The Hamiltonian is
 *    H = sum_pq h_pq E_pq + 1/2 sum_pqrs (pq|rs)(E_pq E_rs - delta_qr E_ps) + E_nuc,
 *    the spin-free form of the Sec. 2.2 Hamiltonian.
 *  - Determinant |I_a I_b> = prod_{p in I_a, ascending} a+_{p,alpha}
 *    prod_{r in I_b, ascending} a+_{r,beta} |0> (alpha block first).
 *  - Subspace: the product of the sorted unique alpha strings S_a (N_a of them)
 *    and beta strings S_b (N_b); determinant index I = i_a * N_b + i_b, so a
 *    vector c is an N_a x N_b row-major matrix (alpha index slow).
 *  - Pointers: every array argument is a DEVICE pointer owned by the caller unless
 *    its comment says "host".  Opaque handles are owned by the library and freed
 *    with the matching *_destroy call.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every call is stream-ordered; calls that return values to host
 *    memory synchronise the stream first.
 *  - Errors: every call returns an int status (HINQS_OK = 0, positive =
 *    warning, negative = error, see below); on error the outputs are undefined and
 *    hinqs_last_error_message() describes the cause (thread-local).
 *  - Memory: handles and per-call workspaces are allocated by the library from
 *    the stream-ordered CUDA memory pool (cudaMallocAsync).
 */
#ifndef HINQS_H
#define HINQS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define HINQS_OK 0
#define HINQS_NOT_CONVERGED 1        /* warning: outputs hold the last iterate */
#define HINQS_ERR_ARG (-1)           /* invalid argument (NULL, size, range) */
#define HINQS_ERR_PARTICLE_NUMBER (-2) /* string with the wrong electron count */
#define HINQS_ERR_ASYMMETRIC (-3)    /* integrals violate the required symmetry */
#define HINQS_ERR_OOM (-4)           /* device allocation failed */
#define HINQS_ERR_CUDA (-5)          /* CUDA runtime error */
#define HINQS_ERR_TIMEOUT (-6)       /* a bounded device-side wait gave up */
#define HINQS_ERR_EMPTY (-7)         /* empty subspace */

/* ------------------------------------------------------------------ flags */
/* hinqs_build_subspace */
#define HINQS_DROP_BAD 0x0      /* drop strings with the wrong popcount (default) */
#define HINQS_ERROR_BAD 0x1     /* ... or fail with HINQS_ERR_PARTICLE_NUMBER */
#define HINQS_FULL_SPACE 0x2    /* ignore the input strings, enumerate all C(n,k) */
/* hinqs_ham_create */
#define HINQS_CHECK_SYMMETRY 0x1 /* verify h and eri symmetry (tolerance 1e-12 relative) */

/* sigma precision */
#define HINQS_PREC_FP64 0   /* c, sigma: double; FP64 arithmetic */
#define HINQS_PREC_FP32 1   /* c, sigma: float; FP32 arithmetic */
/* c, sigma: float; same-spin and diagonal terms in FP32, the opposite-spin term as a
 * gather into D and a tcgen05 GEMM against (pq|rs) with FP32 accumulation in tensor
 * memory, operands BF16 (about 8 significant bits) ... */
#define HINQS_PREC_FP32_BF16AB 2
/* ... or operands split as hi + lo BF16 with hi*hi + hi*lo + lo*hi (about 16 bits).
 * In both modes, when n_orb > 32 or the operand tiles of the problem do not fit in
 * shared memory (e.g. the split mode at n_orb = 26), the opposite-spin term is
 * computed by the FP32 CUDA-core kernel of HINQS_PREC_FP32 instead (more accurate). */
#define HINQS_PREC_FP32_BF16X3AB 3
/* c, sigma: float; the opposite-spin term as HINQS_PREC_FP32_BF16AB, and the
 * same-spin row products (H_a C, C H_b^T and the alpha-diagonal x beta-singles term)
 * on C rounded to BF16 (round to nearest even, once per product; products and sums
 * in FP32), so that a link reads half the bytes; the diagonal term on the FP32 C.
 * Not in the paper: an inner-product precision for the mixed Davidson, whose FP64
 * refinement removes the rounding.  Links of more than 2^32 padded elements take the
 * FP32 same-spin half. */
#define HINQS_PREC_FP32_BF16C 4
/* c, sigma: double; as HINQS_PREC_FP64 but the off-diagonal terms in double-float
 * arithmetic (each value an unevaluated sum of two FP32 numbers; error-free products by
 * fused multiply-add, two-sum accumulation; about 1e-13 relative; the diagonal term in
 * FP64), which runs several times faster than FP64 on this part.  The same-spin half
 * takes FP64 when N_alpha or N_beta is not a multiple of 4.  Not in the paper: the
 * refinement product of the mixed Davidson (hinqs_davidson_opts.refine_precision). */
#define HINQS_PREC_FP64_DFAB 5

/* Davidson precision */
#define HINQS_DAVIDSON_FP64 0   /* every sigma in FP64 */
#define HINQS_DAVIDSON_MIXED 1  /* FP32 sigma bulk + FP64 residual refinement */

typedef struct hinqs_ham_s hinqs_ham;
typedef struct hinqs_subspace_s hinqs_subspace;
typedef struct hinqs_links_s hinqs_links;
typedef struct hinqs_detlist_s hinqs_detlist;

/* Thread-local description of the last error (never NULL). */
const char* hinqs_last_error_message(void);
/* Library version string. */
const char* hinqs_version(void);

/* ---------------------------------------------------------- Hamiltonian --
 * Prepare the second-quantised Hamiltonian of Sec. 2.2: one- and two-electron
 * integrals over an orthonormal set of spatial orbitals.
 *   h      device, FP64 [n_orb*n_orb], copied
 *   eri    device, FP64 [n_orb^4] chemist (pq|rs), copied
 *   n_alpha, n_beta  electron counts of the fixed (n_alpha, n_beta) sector
 *                    (Sec. 2.1: S_z = (n_alpha - n_beta)/2 is fixed)
 *   e_nuc  constant added to every diagonal element (Step 3: E0 = E_corr + E_nuc)
 *   flags  HINQS_CHECK_SYMMETRY: fail with HINQS_ERR_ASYMMETRIC when h is not
 *          symmetric or eri lacks the 8-fold symmetry (relative 1e-12)
 * Errors: HINQS_ERR_ARG (n_orb outside 1..64, counts outside 0..n_orb, NULL),
 *         HINQS_ERR_ASYMMETRIC, HINQS_ERR_OOM, HINQS_ERR_CUDA. */
int hinqs_ham_create(const double* h, const double* eri, int n_orb, int n_alpha, int n_beta,
                     double e_nuc, int flags, hinqs_ham** out, void* stream);
int hinqs_ham_destroy(hinqs_ham* ham);

/* ------------------------------------------------------------- subspace --
 * Build the SQD product subspace S_a x S_b from sampled strings (Step 1 removes
 * duplicates; Sec. 2.1 keeps a residual particle-number filter as a safety net;
 * Step 3 diagonalises in the subspace spanned by the sampled strings).
 *   alpha  device uint64 [n_a_in] sampled alpha strings (duplicates allowed)
 *   beta   device uint64 [n_b_in] sampled beta strings
 *   flags  HINQS_DROP_BAD | HINQS_ERROR_BAD | HINQS_FULL_SPACE
 *   n_dropped host int64[2] or NULL: wrong-popcount alpha / beta strings dropped
 * Result: S_a, S_b sorted ascending, unique.  Bits at or above n_orb count as
 * wrong strings.  Errors: HINQS_ERR_ARG, HINQS_ERR_PARTICLE_NUMBER (with
 * HINQS_ERROR_BAD), HINQS_ERR_EMPTY (no valid string of a species), HINQS_ERR_OOM. */
int hinqs_build_subspace(const uint64_t* alpha, int64_t n_a_in, const uint64_t* beta,
                         int64_t n_b_in, int n_orb, int n_alpha, int n_beta, int flags,
                         hinqs_subspace** out, int64_t* n_dropped, void* stream);
/* host outputs N_a, N_b */
int hinqs_subspace_dims(const hinqs_subspace* sub, int64_t* n_a, int64_t* n_b);
/* copy S_a [N_a] and S_b [N_b] to device arrays (either may be NULL) */
int hinqs_subspace_strings(const hinqs_subspace* sub, uint64_t* alpha_out, uint64_t* beta_out,
                           void* stream);
int hinqs_subspace_destroy(hinqs_subspace* sub);

/* ---------------------------------------------------------- string links --
 * Same-spin links of one spin species (spin 0 = alpha, 1 = beta): for every
 * I in S_spin all J in S_spin whose excitation degree popcount(I xor J)/2 is 1
 * or 2, i.e. the strings connected to I by a non-zero Hamiltonian element
 * (the connectivity of Eq. classical_expansion), with the fermionic phase and the
 * same-spin Slater-Condon element.  Conventions (fixed for bit-exact parity):
 *   single: hole q in I, particle p in J, J = sign * a+_p a_q I,
 *           hval = sign * (h_pq + sum_{j in I, j != q} [(pq|jj) - (pj|jq)])
 *   double: holes q < s, particles p < r, J = sign * a+_p a+_r a_s a_q I,
 *           hval = sign * ((pq|rs) - (ps|rq))
 *   sign = (-1)^(number of occupied orbitals passed), by masked popcount.
 * Links of a row are in ascending J order.  The handle also holds the per-string
 * same-spin diagonal and the tables sum_{i in I} (ii|xy) used by the sigma.
 * The handle keeps a pointer to the subspace's strings: destroy it first.
 * Errors: HINQS_ERR_ARG (spin, handles, n_orb mismatch), HINQS_ERR_OOM. */
int hinqs_string_links(const hinqs_ham* ham, const hinqs_subspace* sub, int spin,
                       hinqs_links** out, void* stream);
/* host outputs: total links, single links, max links of a row */
int hinqs_links_count(const hinqs_links* links, int64_t* n_links, int64_t* n_singles,
                      int64_t* max_row);
/* Export to device arrays sized [N+1] (row_ptr) and [n_links] (others), any
 * may be NULL.  p,q,r,s follow the conventions above (r = s = 255 for singles). */
int hinqs_links_export(const hinqs_links* links, int64_t* row_ptr, int32_t* col, int8_t* degree,
                       uint8_t* p, uint8_t* q, uint8_t* r, uint8_t* s, int8_t* sign,
                       double* hval, void* stream);
int hinqs_links_destroy(hinqs_links* links);
/* largest number of single links of one string (0 for a NULL handle) */
int hinqs_links_max_singles(const hinqs_links* links);
/* the sigma tiles hinqs_autotune stored in these links (host outputs, each may be
 * NULL): rows per warp of the row products, alpha-single chunk width of the CUDA-core
 * opposite-spin kernel, form of the tensor-core kernel (1, 2: pipeline depth of the
 * persistent kernel; 3: the tile-stationary warp-specialised kernel of the BF16 mode,
 * for n_orb <= 22, at most 64 singles and 64 gather slots per string; the persistent
 * kernel otherwise); 0 = built-in default */
int hinqs_links_tuning(const hinqs_links* links, int* rows_per_warp, int* chunk, int* stages);
/* Not in the paper: store sigma tiles in the alpha links la and beta links lb without
 * timing them (what hinqs_autotune stores after timing): rows_per_warp in {0, 2, 4, 8},
 * chunk in {0, 8, 16, 32}, stages in 0..3 as above (0 = default).  Results do not depend
 * on the choice beyond summation order.  Errors: HINQS_ERR_ARG. */
int hinqs_links_set_tuning(hinqs_links* la, hinqs_links* lb, int rows_per_warp, int chunk,
                           int stages);

/* ------------------------------------------------------------- diagonal --
 * hdiag[I] = <I|H|I> (FP64, [N_a*N_b]): the H_xx of Step 2 (cold-start ranking)
 * and of the advantage A(x) = H_xx - E0 of Eq. energy; also the Davidson
 * preconditioner.  Includes E_nuc. */
int hinqs_diag(const hinqs_ham* ham, const hinqs_subspace* sub, const hinqs_links* la,
               const hinqs_links* lb, double* hdiag, void* stream);

/* ---------------------------------------------------------------- sigma --
 * sigma = H_B c, the projected Hamiltonian of Step 3 ([H_B]_ij = <x_i|H|x_j>)
 * applied matrix-free:
 *   sigma = H_a C + C H_b^T + sum_{pq,rs} (pq|rs) E^a_pq C (E^b_rs)^T + E_nuc C
 * with C the N_a x N_b matrix of c.  c and sigma are device vectors of
 * N_a*N_b elements of the precision's type (double for HINQS_PREC_FP64, float
 * otherwise); sigma is overwritten; c and sigma must not overlap.  The tensor-core
 * modes synchronise the stream to check the kernel's bounded waits
 * (HINQS_ERR_TIMEOUT if one ran out).
 * la / lb are the alpha / beta links of this ham and subspace. */
int hinqs_sigma(const hinqs_ham* ham, const hinqs_subspace* sub, const hinqs_links* la,
                const hinqs_links* lb, const void* c, void* sigma, int precision, void* stream);

/* The two halves of hinqs_sigma (the decomposition of H above), for callers that
 * compose or time them separately; same arguments and vector types.
 * hinqs_sigma_same_spin OVERWRITES sigma with
 *   H_a C + C H_b^T + (diagonal cross term sum_{i in Ia, j in Ib} (ii|jj) + E_nuc) C
 *   + sum_{beta singles} [sum_{i in Ia} (ii|rs)] C      (alpha diagonal x beta singles);
 * hinqs_sigma_opposite_spin ADDS the remaining opposite-spin terms
 *   sum_{alpha singles pq} sum_{beta singles rs and beta diagonal} (pq|rs) E^a_pq C (E^b_rs)^T. */
int hinqs_sigma_same_spin(const hinqs_ham* ham, const hinqs_subspace* sub, const hinqs_links* la,
                          const hinqs_links* lb, const void* c, void* sigma, int precision,
                          void* stream);
int hinqs_sigma_opposite_spin(const hinqs_ham* ham, const hinqs_subspace* sub,
                              const hinqs_links* la, const hinqs_links* lb, const void* c,
                              void* sigma, int precision, void* stream);

/* The sigma products of n independent problems in one call (not in the paper: the
 * products of a batched solve, hinqs_davidson_batch): sigmas[g] = H_g cs[g] for
 * problem g = (hams[g], subs[g], las[g], lbs[g]), all in `precision`.  The FP32 modes
 * run each same-spin stage as one launch over every problem's rows and the BF16
 * tensor-core term as one persistent kernel over a device work queue of (problem,
 * alpha string) items (problems of different n_orb, or whose tensor-core tiles do not
 * fit, run one by one); FP64 products, the FP32 CUDA-core opposite-spin term and
 * problems of 2^20 determinants or more (whose own tuned launches fill the GPU) run
 * problem by problem.  Same results as n hinqs_sigma calls up to summation order.
 * Errors as hinqs_sigma, with the problem's index in the message. */
int hinqs_sigma_batch(int n, const hinqs_ham* const* hams, const hinqs_subspace* const* subs,
                      const hinqs_links* const* las, const hinqs_links* const* lbs,
                      const void* const* cs, void* const* sigmas, int precision, void* stream);

/* ------------------------------------------------------------- Davidson --
 * Lowest eigenpair of H_B by Davidson's method (Step 3, Davidson 1975), with an
 * optional warm start from a previous eigenvector (Step 3 warm-starts from the
 * previous iteration).  Preconditioner t = r / (H_diag - theta) with
 * |H_diag - theta| floored at denom_floor (sign kept); classical Gram-Schmidt
 * applied twice; restart at max_subspace keeping restart_keep vectors (the current
 * and previous Ritz vectors, then the next-lowest ones); projected eigenproblem,
 * orthogonalisation, residual norms and the final
 * energy in FP64 on the device.  Converged when ||H x - theta x||_2 <= tol_residual
 * (x of unit norm) and |theta - theta_prev| <= tol_energy.
 * HINQS_DAVIDSON_MIXED runs the bulk of the sigma products in FP32 and refines
 * with FP64 residuals: each outer cycle evaluates H x in FP64 and solves for the
 * correction in a subspace whose coupling to x uses that FP64 product. */
typedef struct hinqs_davidson_opts {
  int precision;        /* HINQS_DAVIDSON_FP64 | HINQS_DAVIDSON_MIXED */
  int max_iter;         /* cap on sigma products (all precisions), e.g. 200 */
  int max_subspace;     /* m_max >= 3, e.g. 16 */
  double tol_residual;  /* e.g. 1e-8 */
  double tol_energy;    /* e.g. 1e-10 */
  double denom_floor;   /* e.g. 1e-4 */
  double inner_tol;     /* mixed: inner solve stops when its residual falls by this factor (e.g. 1e-3) */
  int trace_cap;        /* capacity of the host trace arrays below (0 = none) */
  double* trace_theta;  /* host [trace_cap] or NULL: theta per iteration (incl. E_nuc) */
  double* trace_resid;  /* host [trace_cap] or NULL: residual norm estimate per iteration */
  double* trace_time;   /* host [trace_cap] or NULL: seconds since the call began */
  int* trace_kind;      /* host [trace_cap] or NULL: 0 = FP64 iterate, 1 = FP32 inner iterate */
  int inner_precision;  /* mixed: sigma precision of the inner products: HINQS_PREC_FP32,
                           HINQS_PREC_FP32_BF16AB, HINQS_PREC_FP32_BF16X3AB or
                           HINQS_PREC_FP32_BF16C */
  int restart_keep;     /* vectors kept at a restart (0 = default).  FP64: the current
                           Ritz vector, the previous one and the next-lowest Ritz vectors,
                           this many in all (1 .. max_subspace - 1); mixed: the FP64 anchor
                           and the next-lowest FP32 Ritz vectors (1 .. max_subspace - 2) */
  int refine_precision; /* mixed: precision of the refinement products H x of the FP64
                           vector: HINQS_PREC_FP64_DFAB (default) or HINQS_PREC_FP64 */
} hinqs_davidson_opts;

typedef struct hinqs_davidson_info {
  int status;           /* HINQS_OK or HINQS_NOT_CONVERGED */
  int iterations;       /* Davidson iterations */
  int n_sigma_fp64;     /* FP64 sigma products (refinement products included) */
  int n_sigma_fp32;     /* FP32 sigma products */
  int n_restarts;
  int n_refinements;    /* mixed: outer FP64 refinement cycles */
  int trace_len;        /* entries written to the trace arrays */
  double energy;        /* final energy (FP64 Rayleigh quotient, incl. E_nuc) */
  double residual;      /* final FP64 ||H x - E x||_2 */
  double seconds;       /* wall time of the call */
} hinqs_davidson_info;

/* Workspace queries: the device bytes that one hinqs_sigma (any of the three sigma
 * calls) or one hinqs_davidson call with these options requests from the
 * stream-ordered CUDA memory pool at its peak, for a subspace of N_a x N_b
 * determinants; the caller's vectors and the handles are not included.  The pool may
 * round each request up.  opts NULL = defaults.  Host only (no device work).
 * Errors: HINQS_ERR_ARG (NULL bytes, negative sizes, options hinqs_davidson rejects). */
int hinqs_sigma_workspace_size(int64_t n_alpha_strings, int64_t n_beta_strings, int precision,
                               size_t* bytes);
int hinqs_davidson_workspace_size(int64_t n_alpha_strings, int64_t n_beta_strings,
                                  const hinqs_davidson_opts* opts, size_t* bytes);

/* Fill opts with defaults (FP64, 200, 16, 1e-8, 1e-10, 1e-4, 1e-3, no trace, FP32 inner,
 * restart_keep 0). */
void hinqs_davidson_default_opts(hinqs_davidson_opts* opts);

/*   guess   device FP64 [N] or NULL (then e_k at argmin H_diag, lowest index on ties)
 *   energy  host double or NULL: final energy
 *   c_out   device FP64 [N]: unit-norm eigenvector
 *   info    host or NULL
 * Returns HINQS_OK, HINQS_NOT_CONVERGED (max_iter reached; outputs hold the last
 * iterate), or an error. */
int hinqs_davidson(const hinqs_ham* ham, const hinqs_subspace* sub, const hinqs_links* la,
                   const hinqs_links* lb, const double* guess, const hinqs_davidson_opts* opts,
                   double* energy, double* c_out, hinqs_davidson_info* info, void* stream);
/* The same solve on a basis list (Step 3 over B itself): H replaced by P H P on the
 * list's m entries; guess and c_out are device FP64 [m] in the list's order.  In the
 * mixed mode every inner product runs in FP32 on CUDA cores (the tensor-core inner
 * precisions are taken as HINQS_PREC_FP32).  Errors as hinqs_davidson, plus
 * HINQS_ERR_EMPTY for an empty list. */
int hinqs_davidson_list(const hinqs_ham* ham, const hinqs_subspace* sub, const hinqs_links* la,
                        const hinqs_links* lb, const hinqs_detlist* list, const double* guess,
                        const hinqs_davidson_opts* opts, double* energy, double* c_out,
                        hinqs_davidson_info* info, void* stream);

/* --------------------------------------------------- basis-list subspace --
 * Step 3 as the paper states it: the projected Hamiltonian over the basis
 * determinants themselves, [H_B]_ij = <x_i|H|x_j> for the x_i of the list B, whose
 * exact diagonalisation gives the energy variational with respect to B.  The list
 * lives inside the product subspace `sub` of its distinct alpha and beta strings
 * (hinqs_build_subspace on the list's strings); the product supplies strings, links
 * and per-string tables, and the list operator is P H P with P the projector on the
 * list, applied to vectors of the list's length m (entry k = the k-th determinant in
 * ascending product position, i.e. ascending (alpha, beta) string index).
 *
 * hinqs_detlist_create: the list of determinants (xa[k], xb[k]) (device uint64 [m],
 * duplicates allowed, any order) as positions in `sub`, sorted and distinct.
 * Errors: HINQS_ERR_ARG (NULL, negative m, a determinant whose strings are not in
 * the product: nothing is created), HINQS_ERR_OOM.  Synchronises the stream.  The
 * handle borrows the subspace's strings: destroy it before the subspace. */
int hinqs_detlist_create(const hinqs_subspace* sub, const uint64_t* xa, const uint64_t* xb,
                         int64_t m, hinqs_detlist** out, void* stream);
/* host output: number of distinct list entries */
int hinqs_detlist_size(const hinqs_detlist* list, int64_t* m);
/* product positions I = i_a * N_b + i_b of the entries, ascending (device int64 [m]) */
int hinqs_detlist_positions(const hinqs_detlist* list, int64_t* pos, void* stream);
int hinqs_detlist_destroy(hinqs_detlist* list);
/* c_product (device FP64 [N_a * N_b]) = the list vector c_list [m] placed at its
 * positions, zero elsewhere: the same state in the product's indexing, so that
 * hinqs_rdm, hinqs_spin_marginals, hinqs_pt2_score and hinqs_nqs_loss (with the list's
 * positions as its basis) apply to a list eigenvector unchanged.  gather: the reverse
 * (c_list[k] = c_product[pos[k]]).  The vectors must not overlap. */
int hinqs_detlist_scatter(const hinqs_detlist* list, const double* c_list, double* c_product,
                          void* stream);
int hinqs_detlist_gather(const hinqs_detlist* list, const double* c_product, double* c_list,
                         void* stream);
/* hdiag[k] = <x_k|H|x_k> (incl. E_nuc), device FP64 [m] */
int hinqs_diag_list(const hinqs_ham* ham, const hinqs_subspace* sub, const hinqs_links* la,
                    const hinqs_links* lb, const hinqs_detlist* list, double* hdiag, void* stream);
/* sigma[k] = sum_l <x_k|H|x_l> c[l] over the list entries; c, sigma [m] of the
 * precision's type (double for HINQS_PREC_FP64, float for the FP32 modes, which all
 * run on CUDA cores here); sigma is overwritten; no atomics, so the result is the same
 * on every call.  Errors: HINQS_ERR_ARG (handles of different problems, a list of
 * another subspace, NULL, overlapping vectors, unknown precision). */
int hinqs_sigma_list(const hinqs_ham* ham, const hinqs_subspace* sub, const hinqs_links* la,
                     const hinqs_links* lb, const hinqs_detlist* list, const void* c, void* sigma,
                     int precision, void* stream);

/* ------------------------------------------------------------- autotune --
 * Not in the paper (its benchmarks use one geometry each; potential-energy scans
 * are named as future work in the Conclusion, item iii).  Times the sigma product
 * of `precision` on this problem for each candidate tile configuration -- rows per
 * warp of the same-spin row products (2, 4, 8) and, for the opposite-spin term,
 * the alpha-single chunk width (16, 32) of the CUDA-core kernel (HINQS_PREC_FP64,
 * HINQS_PREC_FP32) or the pipeline depth (1, 2) of the tensor-core kernel (the
 * BF16 modes) -- and stores the fastest in la and lb; every later sigma,
 * Davidson and batch call on these links uses it.  Choices are cached per
 * (n_orb, n_alpha, n_beta, precision, N_alpha and N_beta in quarter-octave
 * buckets) for the life of the process, so similar problems are timed once.
 *   best_ms  host double or NULL: time of one sigma with the chosen tiles
 * Allocates two vectors of N elements for the trial products and synchronises
 * the stream.  Results of sigma do not depend on the choice beyond summation
 * order.  Errors: HINQS_ERR_ARG, HINQS_ERR_OOM, HINQS_ERR_CUDA, HINQS_ERR_TIMEOUT. */
int hinqs_autotune(const hinqs_ham* ham, const hinqs_subspace* sub, hinqs_links* la,
                   hinqs_links* lb, int precision, double* best_ms, void* stream);

/* ------------------------------------------------------- batched solve --
 * Not in the paper (see hinqs_autotune): lowest eigenpairs of n_geom independent
 * problems, e.g. the geometries of a bond scan, each exactly as hinqs_davidson
 * would solve it with `opts` (NULL = defaults).
 *   n_streams <= 0 (lockstep): the solve of every geometry below 2^20
 *             determinants runs on a host thread and a CUDA stream of its own and
 *             hands its sigma products to a shared batch: when every unconverged such
 *             solve has handed in one, the round runs as one launch per sigma stage for
 *             all of them -- the same-spin row products and transposes over a flattened
 *             grid of every geometry's rows, the BF16 tensor-core opposite-spin term as
 *             one persistent kernel taking (geometry, alpha string) items from a device
 *             work queue (FP64 products and the FP32 CUDA-core opposite-spin term run
 *             geometry by geometry) -- and a converged solve leaves the rounds.  The
 *             larger geometries, whose own launches fill the GPU, are solved at the
 *             same time by 4 workers as below;
 *   n_streams > 0: that many host workers take the problems, longest first by an
 *             estimate of their sigma cost, each running its solves one after another
 *             on a stream of its own.
 * The streams start after the work already queued on `stream`, and `stream` waits
 * for all of them before later work; the call itself returns when every solve is done.
 *   hams, subs, las, lbs  arrays of n_geom handles (la/lb: alpha/beta links of subs[g])
 *   guesses   NULL or array of n_geom device FP64 pointers (each may be NULL)
 *   autotune  nonzero: run hinqs_autotune on each problem first, for the sigma
 *             precision the solve uses most (the inner precision when mixed)
 *   energies  host double [n_geom];  c_outs: n_geom device FP64 [N_g] pointers
 *   infos     host [n_geom] or NULL
 * Returns the first error of any geometry (with its index in the message), else
 * HINQS_NOT_CONVERGED if any geometry did not converge, else HINQS_OK.
 * The trace arrays of opts are ignored.
 * Concurrency: the tensor-core wait-timeout flag is shared by the library, so a
 * timeout in one geometry's tensor-core sigma may be reported by another's. */
int hinqs_davidson_batch(int n_geom, const hinqs_ham* const* hams,
                         const hinqs_subspace* const* subs, hinqs_links* const* las,
                         hinqs_links* const* lbs, const double* const* guesses,
                         const hinqs_davidson_opts* opts, int n_streams, int autotune,
                         double* energies, double* const* c_outs, hinqs_davidson_info* infos,
                         void* stream);

/* -------------------------------------------------------------- self-test --
 * Not in the paper: a check of the timeout path.  Runs the bounded wait of the
 * tensor-core sigma kernel, with `polls` polls (1..2^26; the kernel itself uses 2^26),
 * on an mbarrier that nothing completes, in one thread of one block.  The wait gives
 * up, the kernel raises the library's wait-timeout flag and returns; the call reads
 * and clears the flag like hinqs_sigma does and returns HINQS_ERR_TIMEOUT, the
 * expected result.  The device and the library stay usable.  Synchronises the
 * stream.  Errors: HINQS_ERR_ARG (polls out of range), HINQS_ERR_CUDA. */
int hinqs_selftest_bounded_wait(long long polls, void* stream);

/* Not in the paper: the projected eigensolver of hinqs_davidson (the Rayleigh-Ritz step
 * on the pencil (G, S) of the search space, Sec. 2.2 Step 3's diagonalisation restricted
 * to it) on a pencil given by the caller, for tests of its paths.  Lowest eigenpair of
 * G y = theta S y with y^T S y = 1:
 *   G      host FP64 [m * m], row-major, symmetric (its symmetric part is used)
 *   S      host FP64 [m * m] symmetric positive definite, or NULL for S = I
 *   theta_y  host FP64 [m + 1]: theta, then y with its largest |component| positive
 *   pairs  host FP64 [m * (m + 1)] or NULL: every pair in ascending order, (lambda_j,
 *          y_j) per row; pairs other than the lowest carry the FP32 solve's accuracy
 *          (about 1e-6 relative) when the FP64 fallback was not taken
 *   path   host int or NULL: bit 0 S reduced by the series of S^-1/2 (S within 1e-4 of
 *          the identity), bit 1 by its Cholesky factor, bit 2 the lowest pair refined to
 *          FP64 from an FP32 Jacobi solve (clear: FP64 Jacobi, taken when the two lowest
 *          FP32 eigenvalues are within 1e-5 of the spectral scale or the refinement
 *          stalls)
 * m is 1..32 (the solvers' largest search space).  Synchronises the stream.
 * Errors: HINQS_ERR_ARG (NULL G or theta_y, m out of range), HINQS_ERR_CUDA. */
int hinqs_selftest_projected_eig(const double* G, const double* S, int m, double* theta_y,
                                 double* pairs, int* path, void* stream);

/* ------------------------------------------------------ measurement probe --
 * Not in the paper: the rate of this GPU's fused multiply-add pipe for `precision`
 * (HINQS_PREC_FP64 or HINQS_PREC_FP32), the roofline of the CUDA-core kernels.  Runs
 * resident warps on every SM, each thread advancing independent FMA recurrences with
 * no memory traffic, times five launches with CUDA events and reports the best as
 * *tflops (host; 2 FLOPs per FMA).  Synchronises the stream; about 10 ms of GPU time.
 * Errors: HINQS_ERR_ARG (NULL tflops, other precision), HINQS_ERR_CUDA. */
int hinqs_probe_fma_rate(int precision, double* tflops, void* stream);

/* ---------------------------------------------------------- PT2 scores --
 * Step 2, Eq. pt2_score: the Epstein-Nesbet importance of candidate determinants
 * x_k = (xa[k], xb[k]) given the subspace eigenvector c (energy e0):
 *   v[k]     = <x_k|H|Psi0> = sum_{J in subspace} <x_k|H|J> c_J
 *   hxx[k]   = <x_k|H|x_k>            (includes E_nuc)
 *   score[k] = v[k]^2 / |e0 - hxx[k]| (e0 includes E_nuc)
 * The score is that quotient in IEEE FP64 with no regulariser, as the equation states:
 * when e0 == hxx[k] exactly it is +inf if v[k] != 0 (ranked first by hinqs_select_top
 * and hinqs_basis_update) and NaN if v[k] == 0 (ranked below every number there).
 * Candidates may lie inside or outside the subspace (t = 1 rescoring covers both).
 *   c      device FP64 [N]; xa, xb device uint64 [m] strings of the sector
 *   v, hxx, score  device FP64 [m]
 * Errors: HINQS_ERR_ARG (NULL, m < 0, handles of different problems),
 * HINQS_ERR_PARTICLE_NUMBER (a candidate string with the wrong electron count or
 * bits >= n_orb; its outputs are NaN, the others are valid).  Synchronises the
 * stream (the error count is read back). */
int hinqs_pt2_score(const hinqs_ham* ham, const hinqs_subspace* sub, const double* c, double e0,
                    const uint64_t* xa, const uint64_t* xb, int64_t m, double* v, double* hxx,
                    double* score, void* stream);

/* ------------------------------------------------- classical expansion --
 * Step 1' (Eq. classical_expansion).
 * hinqs_top_amplitudes: indices of the k largest |c_I| (ties: lower index first),
 * written ascending to idx_out (device int64 [min(k, N)]); exact (radix selection).
 * hinqs_classical_expansion: every determinant y outside S_alpha x S_beta with
 * <y|H|x> != 0 for some x among the n_top largest |c_I| (the paper uses n_top = 1000):
 * all alpha/beta singles and doubles and alpha-single x beta-single pairs of each x,
 * kept when the Slater-Condon element is non-zero.  Output ascending in
 * (alpha, beta), duplicates removed, into xa_out/xb_out (device uint64 [cap]);
 * *count (host) = number of candidates.  With xa_out or xb_out NULL only *count is
 * returned.  Any n_orb <= 64 (from 32 orbitals on, the kept strings are ranked
 * among their distinct values to form the sort keys; 64 electrons of one spin are
 * refused).  Errors: HINQS_ERR_ARG (NULL, cap < *count: nothing written),
 * HINQS_ERR_OOM.  Synchronises the stream. */
int hinqs_top_amplitudes(const hinqs_subspace* sub, const double* c, int64_t k, int64_t* idx_out,
                         void* stream);
int hinqs_classical_expansion(const hinqs_ham* ham, const hinqs_subspace* sub, const double* c,
                              int64_t n_top, uint64_t* xa_out, uint64_t* xb_out, int64_t cap,
                              int64_t* count, void* stream);
/* The same with the basis a list: the n_top largest |c_list| among the list entries
 * (ties: lower entry first) are expanded and only the list's own determinants are
 * left out (determinants of the product outside the list are candidates). */
int hinqs_classical_expansion_list(const hinqs_ham* ham, const hinqs_subspace* sub,
                                   const hinqs_detlist* list, const double* c_list, int64_t n_top,
                                   uint64_t* xa_out, uint64_t* xb_out, int64_t cap, int64_t* count,
                                   void* stream);

/* ----------------------------------------------------------- outer loop --
 * The steps of the HI-NQS iteration (Sec. 2.2) that surround the subspace solve.
 * The cumulative basis B of Step 2 is a list of determinants (x_a[i], x_b[i]) with a
 * score each; Step 3 diagonalises on the product of its distinct alpha and beta
 * strings (hinqs_build_subspace), which contains the list.
 *
 * hinqs_select_top (Step 2 ranking): positions of the k largest (largest != 0) or
 * smallest values of values[m], ties to the lower position, written ascending to
 * idx_out (device int64 [min(k, m)]).  Exact (radix selection on order-preserving
 * 64-bit keys; -0 equals +0; a NaN ranks below every number in both directions).
 * Synchronises the stream. */
int hinqs_select_top(const double* values, int64_t m, int64_t k, int largest, int64_t* idx_out,
                     void* stream);

/* hinqs_determinant_diag (Step 2 cold start ranks candidates by H_xx):
 * hxx[k] = <x_k|H|x_k> (incl. E_nuc) for arbitrary determinants x_k = (xa[k], xb[k]),
 * in the subspace or not.  Errors: HINQS_ERR_ARG, HINQS_ERR_PARTICLE_NUMBER (a string
 * with the wrong electron count or bits >= n_orb: its output is NaN, the others are
 * valid).  Synchronises the stream. */
int hinqs_determinant_diag(const hinqs_ham* ham, const uint64_t* xa, const uint64_t* xb, int64_t m,
                           double* hxx, void* stream);

/* hinqs_lookup_determinants: idx[k] = i_a * N_b + i_b when (xa[k], xb[k]) lies in the
 * product subspace, else -1 (device int64 [m]).  Maps basis-list entries to positions
 * of the eigenvector (teacher weights, PT2 scores of basis entries). */
int hinqs_lookup_determinants(const hinqs_subspace* sub, const uint64_t* xa, const uint64_t* xb,
                              int64_t m, int64_t* idx, void* stream);

/* hinqs_candidate_pool (Steps 1 and 1'): the candidate set C_t = C_NQS u C_cl.  The
 * distinct determinants among the two proposal lists (xa1, xb1)[m1] (e.g. NQS samples)
 * and (xa2, xb2)[m2] (e.g. the classical expansion) that pass the particle-number
 * filter of Sec. 2.1 (n_alpha / n_beta of `ham`, no bit at or above n_orb; the
 * rejected entries are counted in *n_dropped, host, may be NULL) and are not in the
 * excluded list (ea, eb)[me] (the cumulative basis: Step 1 removes configurations
 * that duplicate it).  Output ascending in (alpha, beta) into ya/yb (device uint64
 * [cap]); *count (host) = number of candidates; with ya or yb NULL only the counts
 * are returned.  Any n_orb <= 64 (from 32 orbitals on, the proposals' strings are
 * ranked among their distinct values to form the sort keys; 64 electrons of one
 * spin are refused).  Errors: HINQS_ERR_ARG (NULL, cap < *count: nothing written),
 * HINQS_ERR_OOM.  Synchronises the stream. */
int hinqs_candidate_pool(const hinqs_ham* ham, const uint64_t* xa1, const uint64_t* xb1,
                         int64_t m1, const uint64_t* xa2, const uint64_t* xb2, int64_t m2,
                         const uint64_t* ea, const uint64_t* eb, int64_t me, uint64_t* ya,
                         uint64_t* yb, int64_t cap, int64_t* count, int64_t* n_dropped,
                         void* stream);

/* hinqs_basis_update (Step 2).  Basis (ba, bb, bs)[nb] and candidates (ca, cb, cs)[nc]
 * with their keys (H_xx for the cold start, s(x) of Eq. pt2_score otherwise); the
 * caller keeps candidates distinct and outside the basis (hinqs_candidate_pool).
 *   HINQS_BASIS_COLD_START (t = 0): the k candidates with the lowest key.
 *   HINQS_BASIS_RESCORE    (t = 1): the k best of basis + candidates by score, no cap.
 *   HINQS_BASIS_APPEND     (t >= 2): the basis plus the k best candidates; when that
 *                          exceeds b_max > 0 entries, the lowest-scored are evicted
 *                          down to b_max (b_max = 0: no cap).
 * Ties go to the earlier entry of the sequence basis-then-candidates, and kept entries
 * keep that order.  Output (oa, ob, os)[cap] (device; must not overlap the inputs),
 * *n_out (host) entries.  Errors: HINQS_ERR_ARG (NULL, negative size, unknown mode,
 * cap below the result), HINQS_ERR_OOM.  Synchronises the stream. */
#define HINQS_BASIS_COLD_START 0
#define HINQS_BASIS_RESCORE 1
#define HINQS_BASIS_APPEND 2
int hinqs_basis_update(int mode, const uint64_t* ba, const uint64_t* bb, const double* bs,
                       int64_t nb, const uint64_t* ca, const uint64_t* cb, const double* cs,
                       int64_t nc, int64_t k, int64_t b_max, uint64_t* oa, uint64_t* ob,
                       double* os, int64_t cap, int64_t* n_out, void* stream);

/* hinqs_remap_vector (Step 3 warm start across iterations): c_new[I'] = c_old[I] when
 * determinant I' of new_sub is determinant I of old_sub, else 0 (device FP64 vectors
 * of the two subspaces' sizes, not overlapping).  *kept_norm2 (host, may be NULL) =
 * |c_new|^2; when it is 0 there is nothing to warm-start from.  Errors:
 * HINQS_ERR_ARG (NULL, subspaces of different sectors), HINQS_ERR_OOM. */
int hinqs_remap_vector(const hinqs_subspace* old_sub, const double* c_old,
                       const hinqs_subspace* new_sub, double* c_new, double* kept_norm2,
                       void* stream);

/* hinqs_nqs_loss (Step 4, Eqs. teacher, energy, entropy and loss) on a minibatch M
 * of basis determinants given as product-subspace positions batch[m]:
 *   w[j]    = p_alpha(x_a) p_beta(x_b) / Z,  Z = sum over the basis of p_alpha p_beta
 *             (basis = product positions [n_basis], or NULL for the whole product)
 *   adv[j]  = A(x) = H_xx - e0                           (e0 includes E_nuc)
 *   loss[1] = L_teacher = -sum_M w log pi,  loss[2] = L_energy = sum_M w A log pi,
 *   loss[3] = L_entropy = (1/m) sum_M log pi,
 *   loss[0] = coef[0] loss[1] + coef[1] loss[2] + coef[2] loss[3]
 *   grad[j] = d loss[0] / d log_pi[j] = -coef[0] w + coef[1] w A + coef[2] / m
 * p_alpha, p_beta: the spin marginals (hinqs_spin_marginals); log_pi [m]: the network's
 * log-probabilities of the minibatch; coef: HOST double[3] (NULL = 1, 1, 1);
 * w, adv, grad: device FP64 [m]; loss: device FP64 [4].  With M = B the sums are the
 * paper's; on a minibatch they are the same sums restricted to it.
 * Errors: HINQS_ERR_ARG (NULL, m = 0, handles of different problems, an index outside
 * [0, N): its outputs are NaN), HINQS_ERR_OOM.  Synchronises the stream. */
int hinqs_nqs_loss(const hinqs_ham* ham, const hinqs_subspace* sub, const hinqs_links* la,
                   const hinqs_links* lb, const double* p_alpha, const double* p_beta, double e0,
                   const int64_t* basis, int64_t n_basis, const int64_t* batch, int64_t m,
                   const double* log_pi, const double* coef, double* w, double* adv, double* grad,
                   double* loss, void* stream);

/* ------------------------------------------------------------------ RDMs --
 * Spin-summed reduced density matrices of the state c (FP64 [N], used as given):
 *   rdm1[p*n+q]             = sum_s <c|a+_{ps} a_{qs}|c>
 *   rdm2[((p*n+q)*n+r)*n+s] = sum_{s,t} <c|a+_{ps} a+_{rt} a_{st} a_{qs}|c>
 *                           = <c|E_pq E_rs - delta_qr E_ps|c>
 * so <c|H|c> = sum h*rdm1 + 1/2 sum (pq|rs)*rdm2 + E_nuc <c|c>.  For a normalised
 * eigenvector these are the Hellmann-Feynman derivatives dE/dh_pq = rdm1_pq and
 * dE/d(pq|rs) = rdm2_pqrs / 2 entrywise (not in the paper: the gradient the
 * integrals receive when the energy is differentiated).  rdm2 may be NULL.  The
 * results are FP64; the string-pair weights and the opposite-spin sums are formed in
 * double-float arithmetic (pairs of FP32 numbers, about 1e-13 relative), which runs
 * several times faster than FP64 on this part. */
int hinqs_rdm(const hinqs_subspace* sub, const hinqs_links* la, const hinqs_links* lb,
              const double* c, double* rdm1, double* rdm2, void* stream);

/* grad_h = grad_E * rdm1, grad_eri = grad_E * rdm2 / 2 (device [n^2], [n^4]);
 * the backward of E(h, eri) given the RDMs of the normalised eigenvector.
 * grad_eri may be NULL. */
int hinqs_energy_backward(int n_orb, double grad_E, const double* rdm1, const double* rdm2,
                          double* grad_h, double* grad_eri, void* stream);

/* ------------------------------------------------------ spin marginals --
 * Step 4 teacher: spin marginals of |Psi|^2 (Eqs. alpha_marginal, beta_marginal),
 *   p_alpha[a] = sum_b c[a*N_b+b]^2 / |c|^2,   p_beta[b] = sum_a c[a*N_b+b]^2 / |c|^2,
 * and optionally the factorised teacher weight normalised over the basis,
 *   w[a*N_b+b] = p_alpha[a] p_beta[b] / sum_{a',b'} p_alpha[a'] p_beta[b'].
 *   c device FP64 [N]; p_alpha [N_a], p_beta [N_b], w [N] or NULL. */
int hinqs_spin_marginals(const hinqs_subspace* sub, const double* c, double* p_alpha,
                         double* p_beta, double* w, void* stream);

/* ---------------------------------------------- allocation-free marginals --
 * The paper has no counterpart to this call; it exists for callers that cannot
 * allocate device memory while they run: a process whose allocator has already
 * reserved all the device memory it may use, or a serving loop that must not meet
 * an out-of-memory failure, or change its footprint, once it is up.
 * Same arguments and results as hinqs_spin_marginals (up to summation order), but
 * its scratch space is a fixed array inside the library (2^20 doubles = 8 MiB,
 * held by every GPU that loads the library until the process exits) instead of
 * memory allocated per call; it calls no allocating routine.
 *   Limit: N_beta <= 2^20 - 2, else HINQS_ERR_ARG with a message; nothing is done.
 *   Set-up: the first call on a device looks up the array's device address with
 *   that device current; make that first call before any stream capture.
 *   Concurrency: all calls share the array and it keeps the last call's contents;
 *   calls that can overlap on the GPU (other streams, other host threads) race on
 *   it and must be serialised by the caller. */
int hinqs_spin_marginals_noalloc(const hinqs_subspace* sub, const double* c, double* p_alpha,
                                 double* p_beta, double* w, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HINQS_H */
