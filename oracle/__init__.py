"""HI-NQS CPU oracle (FP64) -- TEST INFRASTRUCTURE ONLY.

Plain, slow and independent of the CUDA path: the arithmetic lives in
`hinqs_oracle.c` (explicit occupied-spin-orbital lists, literal operator
application, see that file's header); this module compiles it with gcc, loads
it with ctypes and adds the numpy-level steps:

* build_subspace   -- particle-number filter (Sec. 2.1 "residual particle-number
                      filter") and set semantics (Step 1 dedupe) by np.unique,
                      giving the SQD product subspace of Step 3.
* ground_state_dense -- Step 3 exact diagonalisation of the projected H by
                      numpy.linalg.eigh (a library primitive) on the dense matrix.
* lanczos          -- Step 3 for subspaces too large for a dense matrix: Lanczos
                      with full reorthogonalisation on the matrix-free sigma.
* basis lists      -- Step 3 as the paper states it: [H_B]_ij = <x_i|H|x_j> over a
                      list of basis determinants (sort_list, dense_h_list,
                      sigma_list, ground_state_dense_list), and the classical
                      expansion that leaves out only that list.
* outer loop       -- candidate pools (Steps 1, 1'), the Step 2 basis update
                      (select_top, basis_update), H_xx of arbitrary determinants,
                      the Step 3 warm start (remap_vector), the Step 4 loss inputs
                      (nqs_loss: Eqs. teacher, energy, entropy, loss) and the Step 5
                      stopping rule, by sorts, sets and dictionaries.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  The CUDA library never loads it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hinqs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-Wall", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, dbl = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        lib.oracle_sigma.argtypes = [i32, i32, i32, P, P, dbl, P, i64, P, i64, P, P, P, i64, i32]
        lib.oracle_dense_h.argtypes = [i32, i32, i32, P, P, dbl, P, i64, P, i64, P]
        lib.oracle_diag.argtypes = [i32, i32, i32, P, P, dbl, P, i64, P, i64, P, P, i64]
        lib.oracle_links.argtypes = [i32, i32, P, P, P, i64, P, i64, P, P, P, P, P, P, P, P, P]
        lib.oracle_rdm.argtypes = [i32, P, i64, P, i64, P, P, P, i32]
        lib.oracle_marginals.argtypes = [P, i64, i64, P, P, P]
        lib.oracle_connected.argtypes = [i32, i32, i32, P, P, ctypes.c_uint64, ctypes.c_uint64,
                                         P, P, P, i64]
        lib.oracle_connected.restype = i64
        lib.oracle_coupling.argtypes = [i32, i32, i32, P, P, dbl, P, i64, P, i64, P, P, P, i64,
                                        P, P, i32]
        lib.oracle_dense_h_list.argtypes = [i32, i32, i32, P, P, dbl, P, P, i64, P]
        lib.oracle_sigma_list.argtypes = [i32, i32, i32, P, P, dbl, P, P, i64, P, P, P, i64, i32]
        lib.oracle_max_threads.argtypes = []
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def popcount(v: int) -> int:
    return bin(int(v)).count("1")


def build_subspace(alpha, beta, n_alpha: int, n_beta: int, drop_bad: bool = True):
    """Sorted unique alpha and beta strings; strings with the wrong electron
    count are dropped (drop_bad) or raise ValueError."""
    out = []
    for strings, ne in ((alpha, n_alpha), (beta, n_beta)):
        s = [int(x) for x in np.asarray(strings, dtype=np.uint64).ravel()]
        good = [x for x in s if popcount(x) == ne]
        if len(good) != len(s) and not drop_bad:
            raise ValueError("string with the wrong particle number")
        out.append(np.unique(np.array(good, dtype=np.uint64)))
    return out[0], out[1]


class Ham:
    """Integrals in an orthonormal spatial-orbital basis: h[n,n], chemist eri[n,n,n,n]."""

    def __init__(self, h, eri, e_nuc, n_alpha, n_beta):
        self.h = _f64(h)
        self.eri = _f64(eri)
        self.n = self.h.shape[0]
        self.e_nuc = float(e_nuc)
        self.n_alpha = int(n_alpha)
        self.n_beta = int(n_beta)


def sigma(H: Ham, sa, sb, c, rows=None, n_threads: int = 0):
    """sigma = H c on the product subspace (rows: only those outputs)."""
    lib = _load()
    sa, sb, c = _u64(sa), _u64(sb), _f64(c)
    rows_a = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    m = len(sa) * len(sb) if rows_a is None else len(rows_a)
    out = np.zeros(m)
    rc = lib.oracle_sigma(H.n, H.n_alpha, H.n_beta, _p(H.h), _p(H.eri), H.e_nuc,
                          _p(sa), len(sa), _p(sb), len(sb), _p(c), _p(out),
                          _p(rows_a), 0 if rows_a is None else len(rows_a), n_threads)
    if rc:
        raise ValueError(f"oracle_sigma failed ({rc})")
    return out


def pt2_scores(H: Ham, sa, sb, c, E0: float, xa, xb, n_threads: int = 0):
    """Step 2, Eq. pt2_score: for candidates x = (xa[k], xb[k]) return
    (v, hxx, s) with v = <x|H|c> (sum over the subspace), hxx = <x|H|x> and
    s = v^2 / |E0 - hxx|.  E0 and hxx both include E_nuc."""
    lib = _load()
    sa, sb, c = _u64(sa), _u64(sb), _f64(c)
    xa, xb = _u64(xa), _u64(xb)
    M = len(xa)
    v, hxx = np.zeros(M), np.zeros(M)
    rc = lib.oracle_coupling(H.n, H.n_alpha, H.n_beta, _p(H.h), _p(H.eri), H.e_nuc, _p(sa), len(sa),
                             _p(sb), len(sb), _p(c), _p(xa), _p(xb), M, _p(v), _p(hxx), n_threads)
    if rc:
        raise ValueError(f"oracle_coupling failed ({rc})")
    return v, hxx, v * v / np.abs(E0 - hxx)


def connected(H: Ham, xa: int, xb: int, cap: int = 1 << 20):
    """Determinants y != x with <y|H|x> != 0: (ya, yb, <y|H|x>), ascending (n <= 64)."""
    lib = _load()
    ya, yb, val = np.zeros(cap, np.uint64), np.zeros(cap, np.uint64), np.zeros(cap)
    m = lib.oracle_connected(H.n, H.n_alpha, H.n_beta, _p(H.h), _p(H.eri), int(xa), int(xb),
                             _p(ya), _p(yb), _p(val), cap)
    if m < 0:
        raise ValueError(f"oracle_connected failed ({m})")
    return ya[:m], yb[:m], val[:m]


def top_amplitudes(c, k: int):
    """Indices of the k largest |c_i| (ties: lower index first), ascending."""
    c = np.asarray(c)
    order = np.lexsort((np.arange(len(c)), -np.abs(c)))
    return np.sort(order[:k])


def classical_expansion(H: Ham, sa, sb, c, n_top: int):
    """Eq. classical_expansion: every y outside the product subspace S_a x S_b with
    <y|H|x> != 0 for some x among the n_top largest |c| (Step 1'); returned as
    (ya, yb) ascending in (alpha, beta)."""
    sa, sb = _u64(sa), _u64(sb)
    keys = set()
    for I in top_amplitudes(c, n_top):
        ya, yb, _ = connected(H, sa[I // len(sb)], sb[I % len(sb)])
        for a, b in zip(ya.tolist(), yb.tolist()):
            ia = np.searchsorted(sa, a)
            ib = np.searchsorted(sb, b)
            inside = ia < len(sa) and sa[ia] == a and ib < len(sb) and sb[ib] == b
            if not inside:
                keys.add((a, b))
    out = sorted(keys)
    return (np.array([k[0] for k in out], dtype=np.uint64),
            np.array([k[1] for k in out], dtype=np.uint64))


def dense_h(H: Ham, sa, sb):
    lib = _load()
    sa, sb = _u64(sa), _u64(sb)
    N = len(sa) * len(sb)
    out = np.zeros((N, N))
    rc = lib.oracle_dense_h(H.n, H.n_alpha, H.n_beta, _p(H.h), _p(H.eri), H.e_nuc,
                            _p(sa), len(sa), _p(sb), len(sb), _p(out))
    if rc:
        raise ValueError(f"oracle_dense_h failed ({rc})")
    return out


def diag(H: Ham, sa, sb, rows=None):
    lib = _load()
    sa, sb = _u64(sa), _u64(sb)
    rows_a = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    m = len(sa) * len(sb) if rows_a is None else len(rows_a)
    out = np.zeros(m)
    rc = lib.oracle_diag(H.n, H.n_alpha, H.n_beta, _p(H.h), _p(H.eri), H.e_nuc,
                         _p(sa), len(sa), _p(sb), len(sb), _p(out),
                         _p(rows_a), 0 if rows_a is None else len(rows_a))
    if rc:
        raise ValueError(f"oracle_diag failed ({rc})")
    return out


def links(H: Ham, S, n_e: int, rows=None):
    """Same-spin single/double links of the sorted string set S (see oracle_links);
    rows: only those rows (output row k is row rows[k])."""
    lib = _load()
    S = _u64(S)
    N = len(S)
    rows_a = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    n_out = N if rows_a is None else len(rows_a)
    nr = 0 if rows_a is None else len(rows_a)
    row_ptr = np.zeros(n_out + 1, dtype=np.int64)
    rc = lib.oracle_links(H.n, n_e, _p(H.h), _p(H.eri), _p(S), N, _p(rows_a), nr, _p(row_ptr),
                          None, None, None, None, None, None, None, None)
    if rc:
        raise ValueError(f"oracle_links failed ({rc})")
    nnz = int(row_ptr[-1])
    out = dict(row_ptr=row_ptr, col=np.zeros(nnz, np.int32), degree=np.zeros(nnz, np.int8),
               p=np.zeros(nnz, np.uint8), q=np.zeros(nnz, np.uint8), r=np.zeros(nnz, np.uint8),
               s=np.zeros(nnz, np.uint8), sign=np.zeros(nnz, np.int8), hval=np.zeros(nnz))
    rc = lib.oracle_links(H.n, n_e, _p(H.h), _p(H.eri), _p(S), N, _p(rows_a), nr, _p(row_ptr),
                          _p(out["col"]),
                          _p(out["degree"]), _p(out["p"]), _p(out["q"]), _p(out["r"]),
                          _p(out["s"]), _p(out["sign"]), _p(out["hval"]))
    if rc:
        raise ValueError(f"oracle_links failed ({rc})")
    return out


def rdm(n: int, sa, sb, c, want2: bool = True, n_threads: int = 0):
    """Spin-summed 1-RDM (n,n) and 2-RDM (n,n,n,n) of the state c as given."""
    lib = _load()
    sa, sb, c = _u64(sa), _u64(sb), _f64(c)
    g1 = np.zeros((n, n))
    g2 = np.zeros((n, n, n, n)) if want2 else None
    rc = lib.oracle_rdm(n, _p(sa), len(sa), _p(sb), len(sb), _p(c), _p(g1), _p(g2), n_threads)
    if rc:
        raise ValueError(f"oracle_rdm failed ({rc})")
    return g1, g2


def marginals(c, Na: int, Nb: int, want_w: bool = False):
    lib = _load()
    c = _f64(c)
    pa, pb = np.zeros(Na), np.zeros(Nb)
    w = np.zeros(Na * Nb) if want_w else None
    rc = lib.oracle_marginals(_p(c), Na, Nb, _p(pa), _p(pb), _p(w))
    if rc:
        raise ValueError(f"oracle_marginals failed ({rc})")
    return (pa, pb, w) if want_w else (pa, pb)


def ground_state_dense(H: Ham, sa, sb):
    """(E0, c0) of the projected Hamiltonian by dense numpy.linalg.eigh."""
    Hm = dense_h(H, sa, sb)
    evals, evecs = np.linalg.eigh(Hm)
    return float(evals[0]), evecs[:, 0]


def lanczos(H: Ham, sa, sb, tol: float = 1e-10, max_iter: int = 400, seed: int = 7,
            n_threads: int = 0, trace=None):
    """Lowest eigenpair by Lanczos with full reorthogonalisation (Golub & Van Loan,
    Sec. 10.1), on the matrix-free oracle sigma.  Returns (E0, c0, residual norm).
    trace: optional list that receives (lowest Ritz value, time.perf_counter()) after
    every iteration."""
    N = len(sa) * len(sb)
    rng = np.random.default_rng(seed)
    q = rng.standard_normal(N)
    q /= np.linalg.norm(q)
    Q = [q]
    alphas, betas = [], []
    theta, y = None, None
    for j in range(min(max_iter, N)):
        w = sigma(H, sa, sb, Q[j], n_threads=n_threads)
        a = float(Q[j] @ w)
        alphas.append(a)
        w = w - a * Q[j] - (betas[-1] * Q[j - 1] if j > 0 else 0.0)
        Qm = np.array(Q)
        for _ in range(2):
            w = w - Qm.T @ (Qm @ w)
        b = float(np.linalg.norm(w))
        T = np.diag(alphas) + np.diag(betas, 1) + np.diag(betas, -1)
        ev, evec = np.linalg.eigh(T)
        theta, y = ev[0], evec[:, 0]
        if trace is not None:
            trace.append((float(theta), time.perf_counter()))
        # residual of the Ritz pair = |b * last component of y|
        if abs(b * y[-1]) < tol or b < 1e-14 or j + 1 == N:
            break
        betas.append(b)
        Q.append(w / b)
    x = np.array(Q[:len(y)]).T @ y
    x /= np.linalg.norm(x)
    r = sigma(H, sa, sb, x, n_threads=n_threads) - theta * x
    return float(theta), x, float(np.linalg.norm(r))


# ------------------------------------------------------------- basis lists --
# Step 3 defines the projected Hamiltonian over the basis determinants themselves,
# [H_B]_ij = <x_i|H|x_j>, and its exact diagonalisation gives the variational E_0
# of that list.  A list here is held sorted by (alpha, beta) without duplicates.

def sort_list(xa, xb):
    """The determinants (xa[k], xb[k]) as a basis list: distinct, sorted by (alpha, beta)."""
    pairs = sorted(set(zip(_u64(xa).tolist(), _u64(xb).tolist())))
    return (np.array([p[0] for p in pairs], dtype=np.uint64),
            np.array([p[1] for p in pairs], dtype=np.uint64))


def dense_h_list(H: Ham, xa, xb):
    """[H_B]_ij = <x_i|H|x_j> over a sorted basis list (Step 3)."""
    lib = _load()
    xa, xb = _u64(xa), _u64(xb)
    M = len(xa)
    out = np.zeros((M, M))
    rc = lib.oracle_dense_h_list(H.n, H.n_alpha, H.n_beta, _p(H.h), _p(H.eri), H.e_nuc,
                                 _p(xa), _p(xb), M, _p(out))
    if rc:
        raise ValueError(f"oracle_dense_h_list failed ({rc})")
    return out


def sigma_list(H: Ham, xa, xb, c, rows=None, n_threads: int = 0):
    """sigma_i = sum_j <x_i|H|x_j> c_j over a sorted basis list (rows: only those i)."""
    lib = _load()
    xa, xb, c = _u64(xa), _u64(xb), _f64(c)
    rows_a = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    m = len(xa) if rows_a is None else len(rows_a)
    out = np.zeros(m)
    rc = lib.oracle_sigma_list(H.n, H.n_alpha, H.n_beta, _p(H.h), _p(H.eri), H.e_nuc,
                               _p(xa), _p(xb), len(xa), _p(c), _p(out), _p(rows_a),
                               0 if rows_a is None else len(rows_a), n_threads)
    if rc:
        raise ValueError(f"oracle_sigma_list failed ({rc})")
    return out


def ground_state_dense_list(H: Ham, xa, xb):
    """(E0, c0) of Step 3 on a sorted basis list, by numpy.linalg.eigh of H_B."""
    evals, evecs = np.linalg.eigh(dense_h_list(H, xa, xb))
    return float(evals[0]), evecs[:, 0]


def classical_expansion_list(H: Ham, xa, xb, c, n_top: int):
    """Eq. classical_expansion with the basis a list: every determinant y not in the
    list with <y|H|x> != 0 for some x among the n_top list entries of largest |c|
    (ties to the lower position); (ya, yb) ascending in (alpha, beta)."""
    xa, xb = _u64(xa), _u64(xb)
    members = set(zip(xa.tolist(), xb.tolist()))
    keys = set()
    for i in top_amplitudes(c, n_top):
        ya, yb, _ = connected(H, xa[i], xb[i])
        keys |= set(zip(ya.tolist(), yb.tolist()))
    out = sorted(keys - members)
    return (np.array([k[0] for k in out], dtype=np.uint64),
            np.array([k[1] for k in out], dtype=np.uint64))


def energy_from_rdm(H: Ham, g1, g2, norm2: float = 1.0):
    """<c|H|c> = sum h g1 + 1/2 sum (pq|rs) g2 + E_nuc <c|c>."""
    return float(np.sum(H.h * g1) + 0.5 * np.sum(H.eri * g2) + H.e_nuc * norm2)


# ------------------------------------------------------------------------------------
# Outer loop of Sec. 2.2 around the subspace solve: candidate pools (Steps 1 and 1'),
# the basis update of Step 2, the warm start of Step 3, the inputs of the NQS losses
# of Step 4 (Eqs. teacher, energy, entropy, loss) and the stopping rule of Step 5.
# Plain set / sort / dictionary definitions; the matrix elements come from the C
# oracle above.

BASIS_COLD_START, BASIS_RESCORE, BASIS_APPEND = 0, 1, 2


def select_top(values, k: int, largest: bool = True):
    """Positions of the k largest (largest=True) or smallest values, ties to the lower
    position, returned ascending.  Step 2 keeps the top K candidates by s(x) and the
    cold start the K_0 lowest H_xx.  Finite values and +-inf only."""
    v = np.asarray(values, dtype=np.float64)
    k = max(0, min(int(k), len(v)))
    order = np.lexsort((np.arange(len(v)), -v if largest else v))
    return np.sort(order[:k])


def determinant_diag(H: Ham, xa, xb):
    """H_xx = <x|H|x> (incl. E_nuc) of arbitrary determinants x = (xa[k], xb[k]):
    the cold-start ranking of Step 2, computed by the operator application of
    oracle_coupling (a one-determinant subspace with a zero vector is passed, so only
    the diagonal is used)."""
    xa, xb = _u64(xa), _u64(xb)
    if len(xa) == 0:
        return np.zeros(0)
    _, hxx, _ = pt2_scores(H, xa[:1], xb[:1], np.zeros(1), 0.0, xa, xb)
    return hxx


def lookup(sa, sb, xa, xb):
    """Index I = i_a * N_b + i_b of each determinant (xa[k], xb[k]) in the product
    subspace S_a x S_b, or -1 when it is not there."""
    pos_a = {int(s): i for i, s in enumerate(np.asarray(sa, dtype=np.uint64).tolist())}
    pos_b = {int(s): i for i, s in enumerate(np.asarray(sb, dtype=np.uint64).tolist())}
    Nb = len(pos_b)
    out = np.full(len(xa), -1, dtype=np.int64)
    for k, (a, b) in enumerate(zip(np.asarray(xa, dtype=np.uint64).tolist(),
                                   np.asarray(xb, dtype=np.uint64).tolist())):
        if a in pos_a and b in pos_b:
            out[k] = pos_a[a] * Nb + pos_b[b]
    return out


def candidate_pool(pools, exclude, n_alpha: int, n_beta: int):
    """Candidate set C_t of Steps 1 and 1': the distinct determinants of the union of
    `pools` (a list of (xa, xb) pairs of arrays: NQS samples, classical expansion)
    that have the sector's electron counts (the particle-number safety filter of
    Sec. 2.1) and are not in `exclude` = (ea, eb), the cumulative basis (Step 1
    removes configurations duplicating entries of B).  Returns (ya, yb, n_dropped)
    ascending in (alpha, beta); n_dropped counts pool entries with a wrong count."""
    ex = set(zip(np.asarray(exclude[0], dtype=np.uint64).tolist(),
                 np.asarray(exclude[1], dtype=np.uint64).tolist()))
    keep, dropped = set(), 0
    for xa, xb in pools:
        for a, b in zip(np.asarray(xa, dtype=np.uint64).tolist(),
                        np.asarray(xb, dtype=np.uint64).tolist()):
            if popcount(a) != n_alpha or popcount(b) != n_beta:
                dropped += 1
            elif (a, b) not in ex:
                keep.add((a, b))
    out = sorted(keep)
    return (np.array([t[0] for t in out], dtype=np.uint64),
            np.array([t[1] for t in out], dtype=np.uint64), dropped)


def basis_update(mode: int, basis, cand, k: int, b_max: int = 0):
    """Step 2 basis update.  basis = (ba, bb, bs) and cand = (ca, cb, cs): determinants
    with their keys (H_xx for the cold start, s(x) of Eq. pt2_score otherwise).
      BASIS_COLD_START (t = 0): B = the k candidates with the lowest H_xx.
      BASIS_RESCORE    (t = 1): B = the k best of B u C by s(x), no cap.
      BASIS_APPEND     (t >= 2): the k best candidates are appended to B; while
                       |B| > b_max (b_max > 0) the lowest-scored entries are evicted.
    Ties go to the earlier entry of the sequence (basis first, then candidates), and
    the kept entries stay in that order.  Returns (ba, bb, bs)."""
    ba, bb, bs = (np.asarray(x) for x in basis)
    ca, cb, cs = (np.asarray(x) for x in cand)
    ba, bb, ca, cb = (x.astype(np.uint64) for x in (ba, bb, ca, cb))
    bs, cs = bs.astype(np.float64), cs.astype(np.float64)
    if mode == BASIS_COLD_START:
        sel = select_top(cs, k, largest=False)
        return ca[sel], cb[sel], cs[sel]
    if mode == BASIS_RESCORE:
        pa, pb, ps = (np.concatenate(x) for x in ((ba, ca), (bb, cb), (bs, cs)))
        sel = select_top(ps, k)
        return pa[sel], pb[sel], ps[sel]
    if mode == BASIS_APPEND:
        sel = select_top(cs, k)
        pa, pb, ps = (np.concatenate(x) for x in ((ba, ca[sel]), (bb, cb[sel]), (bs, cs[sel])))
        if b_max > 0 and len(ps) > b_max:
            keep = select_top(ps, b_max)
            pa, pb, ps = pa[keep], pb[keep], ps[keep]
        return pa, pb, ps
    raise ValueError(f"unknown basis update mode {mode}")


def remap_vector(sa_old, sb_old, c_old, sa_new, sb_new):
    """Warm start of Step 3 after a basis change: the previous eigenvector carried to
    the new product subspace, c_new[I'] = c_old[I] where determinant I' of the new
    subspace is determinant I of the old one, else 0."""
    na_new, nb_new = len(sa_new), len(sb_new)
    xa = np.repeat(np.asarray(sa_new, dtype=np.uint64), nb_new)
    xb = np.tile(np.asarray(sb_new, dtype=np.uint64), na_new)
    old = lookup(sa_old, sb_old, xa, xb)
    c_old = np.asarray(c_old, dtype=np.float64)
    return np.where(old >= 0, c_old[np.maximum(old, 0)], 0.0)


def nqs_loss(H: Ham, sa, sb, c, E0: float, batch, log_pi, coef=(1.0, 1.0, 1.0), basis=None):
    """Inputs and values of the NQS losses of Step 4 on a minibatch.
      p_alpha, p_beta  spin marginals of |Psi0|^2 (Eqs. alpha_marginal, beta_marginal)
      w(x)   = p_alpha(x_a) p_beta(x_b) / sum_{x' in B} p_alpha(x'_a) p_beta(x'_b)
               (B = `basis`, product-subspace indices, or the whole product if None)
      A(x)   = H_xx - E0                              (advantage, Eq. energy)
      L_teacher = - sum_{x in M} w(x) log pi(x)       (Eq. teacher)
      L_energy  =   sum_{x in M} w(x) A(x) log pi(x)  (Eq. energy)
      L_entropy =   (1/|M|) sum_{x in M} log pi(x)    (Eq. entropy)
      L_total   = coef . (L_teacher, L_energy, L_entropy)   (Eq. loss)
      grad[x]   = d L_total / d log pi(x)
    over the minibatch M = `batch` (product-subspace indices).  Returns a dict."""
    sa, sb = _u64(sa), _u64(sb)
    Na, Nb = len(sa), len(sb)
    batch = np.asarray(batch, dtype=np.int64)
    log_pi = _f64(log_pi)
    pa, pb = marginals(c, Na, Nb)
    members = np.arange(Na * Nb) if basis is None else np.asarray(basis, dtype=np.int64)
    Z = 0.0
    for I in members.tolist():
        Z += pa[I // Nb] * pb[I % Nb]
    w = pa[batch // Nb] * pb[batch % Nb] / Z
    hxx = diag(H, sa, sb, rows=batch)
    A = hxx - E0
    M = len(batch)
    lt = -float(np.sum(w * log_pi))
    le = float(np.sum(w * A * log_pi))
    ls = float(np.sum(log_pi)) / M if M else 0.0
    ct, ce, cs = (float(x) for x in coef)
    grad = -ct * w + ce * w * A + (cs / M if M else 0.0)
    return dict(w=w, A=A, hxx=hxx, teacher=lt, energy=le, entropy=ls,
                total=ct * lt + ce * le + cs * ls, grad=grad)


def converged(energies, delta: float = 1e-9, patience: int = 5, max_iter: int = 50) -> bool:
    """Step 5: stop when |E(t) - E(t-1)| < delta for `patience` consecutive iterations,
    or after max_iter iterations."""
    if len(energies) >= max_iter:
        return True
    if len(energies) <= patience:
        return False
    d = np.abs(np.diff(np.asarray(energies, dtype=np.float64)))
    return bool(np.all(d[-patience:] < delta))
