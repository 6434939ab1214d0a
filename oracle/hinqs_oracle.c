/*
 * HI-NQS subspace-diagonalisation oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU statement of what the hot path computes.  Only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark load it; the
 * CUDA library never does, and this file shares no code with it.
 *
 * Representation (deliberately not the CUDA path's): a determinant is an
 * explicit ascending list of occupied SPIN orbitals.  Spin orbital P < n is the
 * alpha copy of spatial orbital P, P >= n the beta copy of spatial orbital P-n,
 * so |D> = a+_{P1} a+_{P2} ... |0> with P1 < P2 < ... (alpha block first).
 * Every matrix element is obtained by applying the operators of the
 * second-quantised Hamiltonian of Sec. 2.2 (Step 3 "projected Hamiltonian"),
 *
 *     H = sum_PQ h_PQ a+_P a_Q + 1/2 sum_PQRS g_PQRS a+_P a+_Q a_S a_R + E_nuc,
 *
 * one operator at a time to that list and counting transpositions for the
 * fermionic sign.  The paper leaves the index space of g open; here g is the
 * spin-orbital integral <PQ|RS> = (pr|qs) times delta(spin P, spin R) times
 * delta(spin Q, spin S), with (pr|qs) the chemist-order spatial integral.
 *
 * The subspace is the product of the sorted unique alpha and beta strings
 * (SQD form, Sec. 2.2 Step 3); determinant index I = i_alpha * N_beta + i_beta.
 * Strings arrive as uint64 bitmasks (bit p = spatial orbital p); they are only
 * converted to and from lists here, never operated on as bit patterns.
 *
 * Functions and what they follow:
 *   oracle_sigma      sigma_I = sum_J H_IJ c_J       (H|I> by operator application)
 *   oracle_dense_h    the full projected matrix H_B   (Step 3)
 *   oracle_dense_h_list, oracle_sigma_list
 *                     the same over a list of determinants: Step 3 defines
 *                     [H_B]_ij = <x_i|H|x_j> over the basis determinants x_i, and
 *                     sigma_i = sum_j [H_B]_ij c_j
 *   oracle_diag       H_II                            (Step 2 cold-start H_xx)
 *   oracle_connected  the determinants y != x with <y|H|x> != 0 (Eq. classical_expansion)
 *   oracle_coupling   <x|H|Psi0> = sum_i c_i H_{x,x_i} and H_xx for determinants x
 *                     inside or outside the subspace (Step 2, Eq. pt2_score)
 *   oracle_links      single/double string links, phases and same-spin elements
 *   oracle_rdm        1-RDM gamma_pq and 2-RDM Gamma_pqrs (Hellmann-Feynman
 *                     gradients; not in the paper) by operator expectation
 *   oracle_marginals  spin marginals p_alpha, p_beta and teacher weights
 *                     (Eqs. alpha_marginal, beta_marginal, Step 4)
 *
 * Return value: 0 on success, negative on bad arguments / allocation failure.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXSO 128

typedef struct {
    int ne;
    int so[MAXSO];
} odet;

typedef struct {
    int n;
    const double *h;   /* n*n */
    const double *eri; /* n^4, chemist (pq|rs) */
    double enuc;
} oham;

/* Annihilate spin orbital P: returns the sign (-1)^(position of P in the
 * ascending list) or 0 if P is empty; removes P. */
static int ann(odet *d, int P) {
    for (int k = 0; k < d->ne; ++k) {
        if (d->so[k] == P) {
            for (int m = k; m + 1 < d->ne; ++m) d->so[m] = d->so[m + 1];
            d->ne -= 1;
            return (k % 2) ? -1 : 1;
        }
    }
    return 0;
}

/* Create spin orbital P: returns (-1)^(number of occupied orbitals before P)
 * or 0 if P is already occupied; inserts P keeping the list ascending. */
static int cre(odet *d, int P) {
    int k = 0;
    while (k < d->ne && d->so[k] < P) ++k;
    if (k < d->ne && d->so[k] == P) return 0;
    for (int m = d->ne; m > k; --m) d->so[m] = d->so[m - 1];
    d->so[k] = P;
    d->ne += 1;
    return (k % 2) ? -1 : 1;
}

static int spin_of(const oham *H, int P) { return P >= H->n; }
static int spat(const oham *H, int P) { return P >= H->n ? P - H->n : P; }

static double h1(const oham *H, int P, int Q) {
    if (spin_of(H, P) != spin_of(H, Q)) return 0.0;
    return H->h[spat(H, P) * H->n + spat(H, Q)];
}

/* g_PQRS = <PQ|RS> = (pr|qs) delta(sP,sR) delta(sQ,sS) */
static double g2(const oham *H, int P, int Q, int R, int S) {
    if (spin_of(H, P) != spin_of(H, R) || spin_of(H, Q) != spin_of(H, S)) return 0.0;
    int n = H->n;
    int p = spat(H, P), q = spat(H, Q), r = spat(H, R), s = spat(H, S);
    return H->eri[((size_t)(p * n + r) * n + q) * n + s];
}

static odet det_from_strings(int n, uint64_t a, uint64_t b) {
    odet d;
    d.ne = 0;
    for (int p = 0; p < n; ++p)
        if ((a >> p) & 1ull) d.so[d.ne++] = p;
    for (int p = 0; p < n; ++p)
        if ((b >> p) & 1ull) d.so[d.ne++] = n + p;
    return d;
}

static void strings_from_det(int n, const odet *d, uint64_t *a, uint64_t *b) {
    *a = 0;
    *b = 0;
    for (int k = 0; k < d->ne; ++k) {
        if (d->so[k] < n) *a |= 1ull << d->so[k];
        else *b |= 1ull << (d->so[k] - n);
    }
}

static int64_t find_sorted(const uint64_t *S, int64_t N, uint64_t v) {
    int64_t lo = 0, hi = N - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (S[mid] == v) return mid;
        if (S[mid] < v) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

typedef struct {
    int n;
    const uint64_t *sa, *sb;
    int64_t Na, Nb;
} ospace;

static int64_t det_index(const ospace *B, const odet *d) {
    uint64_t a, b;
    strings_from_det(B->n, d, &a, &b);
    int64_t ia = find_sorted(B->sa, B->Na, a);
    if (ia < 0) return -1;
    int64_t ib = find_sorted(B->sb, B->Nb, b);
    if (ib < 0) return -1;
    return ia * B->Nb + ib;
}

/* Visitor for the terms of H|D>: called with (resulting determinant, coefficient). */
typedef void (*term_fn)(const odet *out, double coeff, void *user);

/* Apply the Hamiltonian literally to |D>.  Terms whose rightmost annihilator
 * hits an empty orbital vanish, so the outer loops run over occupied orbitals
 * only; every other operator is applied and checked in turn. */
static void apply_h(const oham *H, const odet *D, term_fn emit, void *user) {
    int nso = 2 * H->n;
    emit(D, H->enuc, user);
    for (int iq = 0; iq < D->ne; ++iq) {
        int Q = D->so[iq];
        for (int P = 0; P < nso; ++P) {
            double c = h1(H, P, Q);
            if (c == 0.0) continue;
            odet d = *D;
            int s = ann(&d, Q);
            if (!s) continue;
            int s2 = cre(&d, P);
            if (!s2) continue;
            emit(&d, c * s * s2, user);
        }
    }
    for (int ir = 0; ir < D->ne; ++ir) {
        int R = D->so[ir];
        for (int is = 0; is < D->ne; ++is) {
            int S = D->so[is];
            if (S == R) continue;
            for (int Q = 0; Q < nso; ++Q) {
                for (int P = 0; P < nso; ++P) {
                    double c = 0.5 * g2(H, P, Q, R, S);
                    if (c == 0.0) continue;
                    odet d = *D;
                    int sg = ann(&d, R); /* a_R acts first */
                    if (!sg) continue;
                    int t = ann(&d, S);
                    if (!t) continue;
                    sg *= t;
                    t = cre(&d, Q);
                    if (!t) continue;
                    sg *= t;
                    t = cre(&d, P);
                    if (!t) continue;
                    sg *= t;
                    emit(&d, c * sg, user);
                }
            }
        }
    }
}

/* ---------------------------------------------------------------- sigma -- */

typedef struct {
    const ospace *B;
    const double *c;
    double acc;
} sig_user;

static void sig_emit(const odet *out, double coeff, void *u) {
    sig_user *su = (sig_user *)u;
    int64_t K = det_index(su->B, out);
    if (K >= 0) su->acc += coeff * su->c[K];
}

static int check_common(int n, int na, int nb, const double *h, const double *eri,
                        const uint64_t *sa, int64_t Na, const uint64_t *sb, int64_t Nb) {
    if (n < 1 || n > 64 || na < 0 || nb < 0 || na > n || nb > n) return -1;
    if (!h || !eri || (Na > 0 && !sa) || (Nb > 0 && !sb) || Na < 0 || Nb < 0) return -1;
    return 0;
}

/* sigma[k] = sum_J H_{I_k J} c_J for I_k = rows[k] (rows == NULL: all N rows).
 * By symmetry of H, sigma_I = sum over the terms of H|I> of coeff * c_K. */
int oracle_sigma(int n, int na, int nb, const double *h, const double *eri, double enuc,
                 const uint64_t *sa, int64_t Na, const uint64_t *sb, int64_t Nb,
                 const double *c, double *sigma, const int64_t *rows, int64_t n_rows,
                 int n_threads) {
    if (check_common(n, na, nb, h, eri, sa, Na, sb, Nb) || !c || !sigma) return -1;
    oham H = {n, h, eri, enuc};
    ospace B = {n, sa, sb, Na, Nb};
    int64_t cnt = rows ? n_rows : Na * Nb;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t k = 0; k < cnt; ++k) {
        int64_t I = rows ? rows[k] : k;
        odet D = det_from_strings(n, sa[I / Nb], sb[I % Nb]);
        sig_user su = {&B, c, 0.0};
        apply_h(&H, &D, sig_emit, &su);
        sigma[k] = su.acc;
    }
    return 0;
}

/* ------------------------------------------------------------ dense H ---- */

typedef struct {
    const ospace *B;
    double *H;
    int64_t N, col;
} dense_user;

static void dense_emit(const odet *out, double coeff, void *u) {
    dense_user *du = (dense_user *)u;
    int64_t K = det_index(du->B, out);
    if (K >= 0) du->H[K * du->N + du->col] += coeff;
}

/* H[K*N + I] = <K|H|I> for all K, I in the product subspace (row-major). */
int oracle_dense_h(int n, int na, int nb, const double *h, const double *eri, double enuc,
                   const uint64_t *sa, int64_t Na, const uint64_t *sb, int64_t Nb, double *Hout) {
    if (check_common(n, na, nb, h, eri, sa, Na, sb, Nb) || !Hout) return -1;
    oham H = {n, h, eri, enuc};
    ospace B = {n, sa, sb, Na, Nb};
    int64_t N = Na * Nb;
    memset(Hout, 0, sizeof(double) * (size_t)N * (size_t)N);
    for (int64_t I = 0; I < N; ++I) {
        odet D = det_from_strings(n, sa[I / Nb], sb[I % Nb]);
        dense_user du = {&B, Hout, N, I};
        apply_h(&H, &D, dense_emit, &du);
    }
    return 0;
}

/* ------------------------------------------------- determinant lists ---- */

/* A basis list of determinants (xa[k], xb[k]), k < M, sorted ascending by
 * (alpha, beta) and free of duplicates.  Position of (a, b) in it, or -1. */
static int64_t find_pair(const uint64_t *xa, const uint64_t *xb, int64_t M, uint64_t a,
                         uint64_t b) {
    int64_t lo = 0, hi = M - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (xa[mid] == a && xb[mid] == b) return mid;
        if (xa[mid] < a || (xa[mid] == a && xb[mid] < b)) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

static int check_list(int n, int na, int nb, const double *h, const double *eri,
                      const uint64_t *xa, const uint64_t *xb, int64_t M) {
    if (n < 1 || n > 64 || na < 0 || nb < 0 || na > n || nb > n || !h || !eri || M < 0)
        return -1;
    if (M > 0 && (!xa || !xb)) return -1;
    for (int64_t k = 1; k < M; ++k)  /* sorted by (alpha, beta), distinct */
        if (!(xa[k - 1] < xa[k] || (xa[k - 1] == xa[k] && xb[k - 1] < xb[k]))) return -2;
    return 0;
}

typedef struct {
    const uint64_t *xa, *xb;
    int64_t M, n;
    const double *c; /* sigma: the vector */
    double *Hcol;    /* dense: column of H_B being filled (stride M) */
    int64_t col;
    double acc;
} list_user;

static void list_sig_emit(const odet *out, double coeff, void *u) {
    list_user *lu = (list_user *)u;
    uint64_t a, b;
    strings_from_det((int)lu->n, out, &a, &b);
    int64_t K = find_pair(lu->xa, lu->xb, lu->M, a, b);
    if (K >= 0) lu->acc += coeff * lu->c[K];
}

static void list_dense_emit(const odet *out, double coeff, void *u) {
    list_user *lu = (list_user *)u;
    uint64_t a, b;
    strings_from_det((int)lu->n, out, &a, &b);
    int64_t K = find_pair(lu->xa, lu->xb, lu->M, a, b);
    if (K >= 0) lu->Hcol[K * lu->M + lu->col] += coeff;
}

/* H[i*M + j] = <x_i|H|x_j> for the determinants of the list (Step 3's H_B). */
int oracle_dense_h_list(int n, int na, int nb, const double *h, const double *eri, double enuc,
                        const uint64_t *xa, const uint64_t *xb, int64_t M, double *Hout) {
    int rc = check_list(n, na, nb, h, eri, xa, xb, M);
    if (rc || !Hout) return rc ? rc : -1;
    oham H = {n, h, eri, enuc};
    memset(Hout, 0, sizeof(double) * (size_t)M * (size_t)M);
    for (int64_t j = 0; j < M; ++j) {
        odet D = det_from_strings(n, xa[j], xb[j]);
        list_user lu = {xa, xb, M, n, NULL, Hout, j, 0.0};
        apply_h(&H, &D, list_dense_emit, &lu);
    }
    return 0;
}

/* sigma[k] = sum_j <x_i|H|x_j> c_j for i = rows[k] (rows == NULL: every i < M);
 * by the symmetry of H, the terms of H|x_i> looked up in the list. */
int oracle_sigma_list(int n, int na, int nb, const double *h, const double *eri, double enuc,
                      const uint64_t *xa, const uint64_t *xb, int64_t M, const double *c,
                      double *sigma, const int64_t *rows, int64_t n_rows, int n_threads) {
    int rc = check_list(n, na, nb, h, eri, xa, xb, M);
    if (rc || !c || !sigma) return rc ? rc : -1;
    oham H = {n, h, eri, enuc};
    int64_t cnt = rows ? n_rows : M;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t k = 0; k < cnt; ++k) {
        int64_t i = rows ? rows[k] : k;
        odet D = det_from_strings(n, xa[i], xb[i]);
        list_user lu = {xa, xb, M, n, c, NULL, 0, 0.0};
        apply_h(&H, &D, list_sig_emit, &lu);
        sigma[k] = lu.acc;
    }
    return 0;
}

/* --------------------------------------------------------------- diag ---- */

typedef struct {
    const odet *self;
    double acc;
} diag_user;

static int same_det(const odet *a, const odet *b) {
    if (a->ne != b->ne) return 0;
    for (int k = 0; k < a->ne; ++k)
        if (a->so[k] != b->so[k]) return 0;
    return 1;
}

static void diag_emit(const odet *out, double coeff, void *u) {
    diag_user *du = (diag_user *)u;
    if (same_det(out, du->self)) du->acc += coeff;
}

/* hd[k] = <I|H|I> for I = rows[k] (rows == NULL: all). */
int oracle_diag(int n, int na, int nb, const double *h, const double *eri, double enuc,
                const uint64_t *sa, int64_t Na, const uint64_t *sb, int64_t Nb, double *hd,
                const int64_t *rows, int64_t n_rows) {
    if (check_common(n, na, nb, h, eri, sa, Na, sb, Nb) || !hd) return -1;
    oham H = {n, h, eri, enuc};
    int64_t cnt = rows ? n_rows : Na * Nb;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t k = 0; k < cnt; ++k) {
        int64_t I = rows ? rows[k] : k;
        odet D = det_from_strings(n, sa[I / Nb], sb[I % Nb]);
        diag_user du = {&D, 0.0};
        apply_h(&H, &D, diag_emit, &du);
        hd[k] = du.acc;
    }
    return 0;
}

/* -------------------------------------------------------- PT2 coupling --- */

/* For candidate determinants x_k = (xa[k], xb[k]) (any strings with the sector's
 * electron counts, in the subspace or not): v[k] = <x_k|H|c> = sum_J <x_k|H|J> c_J
 * over the subspace determinants J, and hxx[k] = <x_k|H|x_k>.  H is real symmetric,
 * so v is gathered by applying H to |x_k> and looking the results up in the subspace
 * (the numerator of Eq. pt2_score); hxx is the diagonal of Step 2. */
int oracle_coupling(int n, int na, int nb, const double *h, const double *eri, double enuc,
                    const uint64_t *sa, int64_t Na, const uint64_t *sb, int64_t Nb,
                    const double *c, const uint64_t *xa, const uint64_t *xb, int64_t M,
                    double *v, double *hxx, int n_threads) {
    if (check_common(n, na, nb, h, eri, sa, Na, sb, Nb) || !c || M < 0 ||
        (M > 0 && (!xa || !xb || !v || !hxx)))
        return -1;
    oham H = {n, h, eri, enuc};
    ospace B = {n, sa, sb, Na, Nb};
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t k = 0; k < M; ++k) {
        odet D = det_from_strings(n, xa[k], xb[k]);
        sig_user su = {&B, c, 0.0};
        apply_h(&H, &D, sig_emit, &su);
        v[k] = su.acc;
        diag_user du = {&D, 0.0};
        apply_h(&H, &D, diag_emit, &du);
        hxx[k] = du.acc;
    }
    return 0;
}

/* ------------------------------------------------- connected determinants --- */

typedef struct {
    uint64_t a, b; /* alpha and beta strings */
    double coeff;
} kterm;

typedef struct {
    int n;
    kterm *buf;
    int64_t cnt, cap;
    int overflow;
} conn_user;

static void conn_emit(const odet *out, double coeff, void *u) {
    conn_user *cu = (conn_user *)u;
    if (cu->cnt >= cu->cap) {
        cu->overflow = 1;
        return;
    }
    uint64_t a, b;
    strings_from_det(cu->n, out, &a, &b);
    cu->buf[cu->cnt].a = a;
    cu->buf[cu->cnt].b = b;
    cu->buf[cu->cnt].coeff = coeff;
    cu->cnt++;
}

static int cmp_kterm(const void *x, const void *y) {
    const kterm *u = (const kterm *)x, *v = (const kterm *)y;
    if (u->a != v->a) return u->a < v->a ? -1 : 1;
    return u->b < v->b ? -1 : (u->b > v->b ? 1 : 0);
}

static int same_strings(const kterm *u, const kterm *v) { return u->a == v->a && u->b == v->b; }

/* Every determinant y != x with <y|H|x> != 0 (Eq. classical_expansion's connection
 * test), by applying H to |x> and summing the coefficients of equal results.
 * Outputs y's strings and <y|H|x>, ascending in (alpha, beta); returns the count,
 * or -1 (bad arguments, n > 64) / -2 (cap too small). */
int64_t oracle_connected(int n, int na, int nb, const double *h, const double *eri,
                         uint64_t xa, uint64_t xb, uint64_t *ya, uint64_t *yb, double *val,
                         int64_t cap) {
    if (n < 1 || n > 64 || na < 0 || nb < 0 || na > n || nb > n || !h || !eri) return -1;
    oham H = {n, h, eri, 0.0};
    odet D = det_from_strings(n, xa, xb);
    int64_t tcap = 1 << 22;
    conn_user cu = {n, (kterm *)malloc(sizeof(kterm) * tcap), 0, tcap, 0};
    if (!cu.buf) return -1;
    apply_h(&H, &D, conn_emit, &cu);
    if (cu.overflow) {
        free(cu.buf);
        return -2;
    }
    qsort(cu.buf, cu.cnt, sizeof(kterm), cmp_kterm);
    const kterm self = {xa, xb, 0.0};
    int64_t m = 0;
    for (int64_t i = 0; i < cu.cnt;) {
        int64_t j = i;
        double sum = 0.0;
        while (j < cu.cnt && same_strings(&cu.buf[j], &cu.buf[i])) sum += cu.buf[j++].coeff;
        if (!same_strings(&cu.buf[i], &self) && sum != 0.0) {
            if (m >= cap) {
                free(cu.buf);
                return -2;
            }
            ya[m] = cu.buf[i].a;
            yb[m] = cu.buf[i].b;
            val[m] = sum;
            m++;
        }
        i = j;
    }
    free(cu.buf);
    return m;
}

/* -------------------------------------------------------------- links ---- */

typedef struct {
    const odet *target;
    double acc;
} match_user;

static void match_emit(const odet *out, double coeff, void *u) {
    match_user *mu = (match_user *)u;
    if (same_det(out, mu->target)) mu->acc += coeff;
}

static void occ_list(int n, uint64_t s, int *occ, int *cnt) {
    *cnt = 0;
    for (int p = 0; p < n; ++p)
        if ((s >> p) & 1ull) occ[(*cnt)++] = p;
}

static int in_list(const int *l, int m, int v) {
    for (int k = 0; k < m; ++k)
        if (l[k] == v) return 1;
    return 0;
}

/* Same-spin string links of one spin species.  For every I in S (sorted) and
 * every J in S, in ascending J order, with J differing from I in one or two
 * orbitals:
 *   degree 1: hole q (in I not J), particle p (in J not I), J = sign a+_p a_q I;
 *   degree 2: holes q < s, particles p < r, J = sign a+_p a+_r a_s a_q I.
 * For singles r = s = 255.  sign is obtained by applying the operators to the
 * ordered list of I.  hval = <J|H_spin|I>, the part of H whose operators all
 * act on this spin, found by applying H to the one-species determinant I (the
 * other species empty) and collecting the coefficient of J.
 * rows (NULL: all) selects the rows I = rows[k]; output row k holds row rows[k].
 * Call with col == NULL to get only the row counts in row_ptr[1..n_out]
 * (row_ptr[0] = 0, then prefix sums); the second call fills the records. */
int oracle_links(int n, int ne, const double *h, const double *eri, const uint64_t *S, int64_t N,
                 const int64_t *rows, int64_t n_rows,
                 int64_t *row_ptr, int32_t *col, int8_t *degree, uint8_t *p_out, uint8_t *q_out,
                 uint8_t *r_out, uint8_t *s_out, int8_t *sign_out, double *hval) {
    if (n < 1 || n > 64 || ne < 0 || ne > n || !h || !eri || !S || !row_ptr || N < 0) return -1;
    oham H = {n, h, eri, 0.0};
    int64_t n_out = rows ? n_rows : N;
    if (!col) {
        row_ptr[0] = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16)
#endif
        for (int64_t k = 0; k < n_out; ++k) {
            int64_t I = rows ? rows[k] : k;
            int oi[64], ni;
            occ_list(n, S[I], oi, &ni);
            int64_t cnt = 0;
            for (int64_t J = 0; J < N; ++J) {
                int oj[64], nj, nh = 0;
                occ_list(n, S[J], oj, &nj);
                for (int k = 0; k < ni; ++k)
                    if (!in_list(oj, nj, oi[k])) ++nh;
                if (nh == 1 || nh == 2) ++cnt;
            }
            row_ptr[k + 1] = cnt;
        }
        for (int64_t k = 0; k < n_out; ++k) row_ptr[k + 1] += row_ptr[k];
        return 0;
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t kr = 0; kr < n_out; ++kr) {
        int64_t I = rows ? rows[kr] : kr;
        int oi[64], ni;
        occ_list(n, S[I], oi, &ni);
        odet DI;
        DI.ne = ni;
        for (int k = 0; k < ni; ++k) DI.so[k] = oi[k];
        int64_t pos = row_ptr[kr];
        for (int64_t J = 0; J < N; ++J) {
            int oj[64], nj;
            occ_list(n, S[J], oj, &nj);
            int holes[64], parts[64], nh = 0, np = 0;
            for (int k = 0; k < ni; ++k)
                if (!in_list(oj, nj, oi[k])) holes[nh++] = oi[k];
            for (int k = 0; k < nj; ++k)
                if (!in_list(oi, ni, oj[k])) parts[np++] = oj[k];
            if (nh != 1 && nh != 2) continue;
            odet d = DI;
            int sg;
            if (nh == 1) {
                sg = ann(&d, holes[0]);
                sg *= cre(&d, parts[0]);
                p_out[pos] = (uint8_t)parts[0];
                q_out[pos] = (uint8_t)holes[0];
                r_out[pos] = 255;
                s_out[pos] = 255;
            } else {
                /* holes ascending: q = holes[0], s = holes[1]; particles p < r */
                sg = ann(&d, holes[0]);
                sg *= ann(&d, holes[1]);
                sg *= cre(&d, parts[1]);
                sg *= cre(&d, parts[0]);
                p_out[pos] = (uint8_t)parts[0];
                q_out[pos] = (uint8_t)holes[0];
                r_out[pos] = (uint8_t)parts[1];
                s_out[pos] = (uint8_t)holes[1];
            }
            col[pos] = (int32_t)J;
            degree[pos] = (int8_t)nh;
            sign_out[pos] = (int8_t)sg;
            odet DJ;
            DJ.ne = nj;
            for (int k = 0; k < nj; ++k) DJ.so[k] = oj[k];
            match_user mu = {&DJ, 0.0};
            apply_h(&H, &DI, match_emit, &mu);
            hval[pos] = mu.acc;
            ++pos;
        }
    }
    return 0;
}

/* --------------------------------------------------------------- RDMs ---- */

/* Spin-summed reduced density matrices of the state c (as given, not
 * renormalised) on the product subspace:
 *   rdm1[p*n+q]           = sum_sigma <c| a+_{p sigma} a_{q sigma} |c>
 *   rdm2[((p*n+q)*n+r)*n+s] = sum_{sigma,tau} <c| a+_{p sigma} a+_{r tau} a_{s tau} a_{q sigma} |c>
 * so that <c|H|c> = sum h_pq rdm1_pq + 1/2 sum (pq|rs) rdm2_pqrs + E_nuc <c|c>.
 * Either output may be NULL. */
int oracle_rdm(int n, const uint64_t *sa, int64_t Na, const uint64_t *sb, int64_t Nb,
               const double *c, double *rdm1, double *rdm2, int n_threads) {
    if (n < 1 || n > 64 || !sa || !sb || !c || Na < 0 || Nb < 0) return -1;
    ospace B = {n, sa, sb, Na, Nb};
    int64_t N = Na * Nb;
    size_t n2 = (size_t)n * n, n4 = n2 * n2;
    if (rdm1) memset(rdm1, 0, sizeof(double) * n2);
    if (rdm2) memset(rdm2, 0, sizeof(double) * n4);
    int nt = 1;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
    nt = omp_get_max_threads();
#endif
    double *p1 = calloc((size_t)nt * n2, sizeof(double));
    double *p2 = rdm2 ? calloc((size_t)nt * n4, sizeof(double)) : NULL;
    if (!p1 || (rdm2 && !p2)) {
        free(p1);
        free(p2);
        return -2;
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t J = 0; J < N; ++J) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double cj = c[J];
        if (cj == 0.0) continue;
        double *a1 = p1 + (size_t)tid * n2;
        double *a2 = p2 ? p2 + (size_t)tid * n4 : NULL;
        odet D = det_from_strings(n, sa[J / Nb], sb[J % Nb]);
        for (int iq = 0; iq < D.ne; ++iq) {
            int Q = D.so[iq];
            int sQ = Q >= n, q = Q - sQ * n;
            for (int p = 0; p < n; ++p) {
                int P = p + sQ * n;
                odet d = D;
                int sg = ann(&d, Q);
                int t = cre(&d, P);
                if (!t) continue;
                int64_t K = det_index(&B, &d);
                if (K >= 0) a1[p * n + q] += sg * t * c[K] * cj;
            }
            if (!a2) continue;
            for (int is = 0; is < D.ne; ++is) {
                int S = D.so[is];
                if (S == Q) continue;
                int sS = S >= n, s = S - sS * n;
                for (int r = 0; r < n; ++r) {
                    int R = r + sS * n;
                    for (int p = 0; p < n; ++p) {
                        int P = p + sQ * n;
                        odet d = D;
                        int sg = ann(&d, Q); /* a_Q acts first */
                        int t = ann(&d, S);
                        sg *= t;
                        t = cre(&d, R);
                        if (!t) continue;
                        sg *= t;
                        t = cre(&d, P);
                        if (!t) continue;
                        sg *= t;
                        int64_t K = det_index(&B, &d);
                        if (K >= 0) a2[((size_t)(p * n + q) * n + r) * n + s] += sg * c[K] * cj;
                    }
                }
            }
        }
    }
    for (int t = 0; t < nt; ++t) {
        if (rdm1)
            for (size_t k = 0; k < n2; ++k) rdm1[k] += p1[(size_t)t * n2 + k];
        if (rdm2)
            for (size_t k = 0; k < n4; ++k) rdm2[k] += p2[(size_t)t * n4 + k];
    }
    free(p1);
    free(p2);
    return 0;
}

/* ---------------------------------------------------------- marginals ---- */

/* Spin marginals of |Psi|^2 / <Psi|Psi> (Eqs. alpha_marginal, beta_marginal):
 *   p_alpha[a] = sum_b c[a*Nb+b]^2 / |c|^2,  p_beta[b] = sum_a c[a*Nb+b]^2 / |c|^2,
 * and the factorised teacher weight of Step 4,
 *   w[a*Nb+b] = p_alpha[a] p_beta[b] / sum_{a',b'} p_alpha[a'] p_beta[b'].
 * w may be NULL. */
int oracle_marginals(const double *c, int64_t Na, int64_t Nb, double *pa, double *pb, double *w) {
    if (!c || !pa || !pb || Na < 0 || Nb < 0) return -1;
    double nrm = 0.0;
    for (int64_t I = 0; I < Na * Nb; ++I) nrm += c[I] * c[I];
    for (int64_t a = 0; a < Na; ++a) pa[a] = 0.0;
    for (int64_t b = 0; b < Nb; ++b) pb[b] = 0.0;
    for (int64_t a = 0; a < Na; ++a)
        for (int64_t b = 0; b < Nb; ++b) {
            double v = c[a * Nb + b] * c[a * Nb + b] / nrm;
            pa[a] += v;
            pb[b] += v;
        }
    if (w) {
        double z = 0.0;
        for (int64_t a = 0; a < Na; ++a)
            for (int64_t b = 0; b < Nb; ++b) z += pa[a] * pb[b];
        for (int64_t a = 0; a < Na; ++a)
            for (int64_t b = 0; b < Nb; ++b) w[a * Nb + b] = pa[a] * pb[b] / z;
    }
    return 0;
}

/* Single-threaded / multi-threaded switch used by the timed CPU baseline. */
int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
