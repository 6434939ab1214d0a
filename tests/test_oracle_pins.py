"""Pins of the CPU oracle against facts fixed by the paper and by the mathematics.

Each test checks the oracle against something other than itself: textbook closed
forms (two-site Hubbard, minimal-basis H2), a Jordan-Wigner Fock-space
construction of the same Hamiltonian (an independent sign convention built from
matrix products), library eigen-solvers on limits with known spectra, the
full-space Hilbert dimensions of Table 1, the variational bound of Step 3,
central finite differences of the energy, and the normalisation of the teacher
weights of Step 4.
"""
import itertools
import os
from math import comb

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def full_space(n, na, nb):
    return synth.all_strings(n, na), synth.all_strings(n, nb)


def fci_dense(h, eri, e_nuc, na, nb, sa=None, sb=None):
    n = h.shape[0]
    H = oracle.Ham(h, eri, e_nuc, na, nb)
    if sa is None:
        sa, sb = oracle.build_subspace(*full_space(n, na, nb), na, nb)
    return oracle.ground_state_dense(H, sa, sb)


# ------------------------------------------------------------------ closed forms


@pytest.mark.parametrize("t,U", [(1.0, 4.0), (0.7, 0.0), (1.3, 9.5), (0.2, -1.0)])
def test_two_site_hubbard(t, U):
    """Half-filled two-site Hubbard model: E0 = (U - sqrt(U^2 + 16 t^2)) / 2."""
    h = np.array([[0.0, -t], [-t, 0.0]])
    eri = np.zeros((2, 2, 2, 2))
    eri[0, 0, 0, 0] = U
    eri[1, 1, 1, 1] = U
    E, _ = fci_dense(h, eri, 0.0, 1, 1)
    assert abs(E - (U - np.sqrt(U * U + 16 * t * t)) / 2) < 1e-12


def _h2_integrals(hgg, huu, Jgg, Juu, Jgu, K):
    h = np.diag([hgg, huu])
    eri = np.zeros((2, 2, 2, 2))
    eri[0, 0, 0, 0] = Jgg
    eri[1, 1, 1, 1] = Juu
    eri[0, 0, 1, 1] = eri[1, 1, 0, 0] = Jgu
    for idx in [(0, 1, 0, 1), (0, 1, 1, 0), (1, 0, 0, 1), (1, 0, 1, 0)]:
        eri[idx] = K
    return h, eri


@pytest.mark.parametrize("vals", [
    (-1.2528, -0.4756, 0.6746, 0.6975, 0.6636, 0.1813),   # H2 / STO-3G near R = 1.4 bohr
    (-1.1, -0.3, 0.7, 0.55, 0.6, 0.25),
    (-0.9, -0.5, 0.5, 0.5, 0.45, 0.3),
])
def test_h2_minimal_basis(vals):
    """Minimal-basis H2 (orbitals g, u; symmetry kills h_gu, (gg|gu), (uu|gu)):
    E0 = (E1+E2)/2 - sqrt((E2-E1)^2/4 + K^2), E1 = 2h_gg + (gg|gg),
    E2 = 2h_uu + (uu|uu), K = (gu|gu).  Distinguishes (gg|uu) from (gu|gu), so a
    transposed integral index fails it."""
    hgg, huu, Jgg, Juu, Jgu, K = vals
    h, eri = _h2_integrals(*vals)
    E, c = fci_dense(h, eri, 0.0, 1, 1)
    E1, E2 = 2 * hgg + Jgg, 2 * huu + Juu
    ref = 0.5 * (E1 + E2) - np.sqrt(0.25 * (E2 - E1) ** 2 + K * K)
    assert ref < hgg + huu + Jgu - K  # the closed-shell pair holds the ground state
    assert abs(E - ref) < 1e-12


def test_one_body_limit():
    """ERI = 0: E0 = sum of the lowest n_alpha plus lowest n_beta eigenvalues of h."""
    h, _, _ = synth.integrals(6, 11)
    eri = np.zeros((6,) * 4)
    for na, nb in [(2, 3), (1, 0), (3, 3), (0, 2)]:
        E, _ = fci_dense(h, eri, 0.25, na, nb)
        ev = np.linalg.eigvalsh(h)
        assert abs(E - (ev[:na].sum() + ev[:nb].sum() + 0.25)) < 1e-12


def test_orbital_rotation_invariance():
    """The full-space energy is invariant under h -> U^T h U, (pq|rs) -> rotated."""
    h, eri, _ = synth.integrals(5, 12)
    E0, _ = fci_dense(h, eri, 0.0, 2, 2)
    rng = np.random.default_rng(3)
    U, _ = np.linalg.qr(rng.standard_normal((5, 5)))
    h2 = U.T @ h @ U
    eri2 = np.einsum("pqrs,pi,qj,rk,sl->ijkl", eri, U, U, U, U)
    E1, _ = fci_dense(h2, eri2, 0.0, 2, 2)
    assert abs(E0 - E1) < 1e-11


# ------------------------------------------------------- Jordan-Wigner pin


def _jw_ops(m):
    """Annihilators a_j on m modes, Fock index bit j = occupation of mode j,
    a_j = (prod_{k<j} Z_k) sigma^-_j."""
    dim = 1 << m
    ops = []
    for j in range(m):
        rows, cols, vals = [], [], []
        for x in range(dim):
            if (x >> j) & 1:
                y = x ^ (1 << j)
                parity = bin(x & ((1 << j) - 1)).count("1")
                rows.append(y)
                cols.append(x)
                vals.append(-1.0 if parity % 2 else 1.0)
        ops.append(sp.csr_matrix((vals, (rows, cols)), shape=(dim, dim)))
    return ops


def _jw_hamiltonian(h, eri, e_nuc):
    """H in the 2n-mode Fock space; mode P < n = alpha P, mode n+p = beta p.
    Coefficients follow the spin-free chemistry convention
    1/2 sum (pq|rs) a+_{p s} a+_{r t} a_{s' t} a_{q s} -- written independently."""
    n = h.shape[0]
    a = _jw_ops(2 * n)
    ad = [x.T.tocsr() for x in a]
    H = sp.identity(1 << (2 * n), format="csr") * e_nuc
    for s in range(2):
        for p in range(n):
            for q in range(n):
                if h[p, q] != 0:
                    H = H + h[p, q] * (ad[s * n + p] @ a[s * n + q])
    for s1 in range(2):
        for s2 in range(2):
            for p, q, r, s in itertools.product(range(n), repeat=4):
                v = eri[p, q, r, s]
                if v == 0:
                    continue
                H = H + 0.5 * v * (ad[s1 * n + p] @ ad[s2 * n + r] @ a[s2 * n + s] @ a[s1 * n + q])
    return H


def _fock_index(n, sa, sb):
    return np.array([int(x) | (int(y) << n) for x in sa for y in sb], dtype=np.int64)


@pytest.mark.parametrize("n,na,nb,seed", [(4, 2, 2, 21), (4, 1, 3, 22), (3, 2, 1, 23)])
def test_dense_h_matches_jordan_wigner(n, na, nb, seed):
    h, eri, _ = synth.integrals(n, seed)
    Hjw = _jw_hamiltonian(h, eri, 0.3).toarray()
    sa, sb = full_space(n, na, nb)
    sa, sb = oracle.build_subspace(sa, sb, na, nb)
    idx = _fock_index(n, sa, sb)
    ref = Hjw[np.ix_(idx, idx)]
    Ho = oracle.dense_h(oracle.Ham(h, eri, 0.3, na, nb), sa, sb)
    assert np.max(np.abs(Ho - ref)) < 1e-12
    # the sector is closed: H maps it to itself (N and S_z conservation)
    rest = np.setdiff1d(np.arange(Hjw.shape[0]), idx)
    assert np.max(np.abs(Hjw[np.ix_(rest, idx)])) == 0.0


def test_links_match_jordan_wigner():
    """Link phases and same-spin elements against one-species JW operators."""
    n, ne = 5, 2
    h, eri, _ = synth.integrals(n, 31)
    S = np.sort(synth.all_strings(n, ne))
    L = oracle.links(oracle.Ham(h, eri, 0.0, ne, 0), S, ne)
    a = _jw_ops(n)
    ad = [x.T.tocsr() for x in a]
    Hjw = _jw_hamiltonian(h, eri, 0.0).toarray()  # 2n modes, beta empty -> alpha block
    for I in range(len(S)):
        for k in range(L["row_ptr"][I], L["row_ptr"][I + 1]):
            J = L["col"][k]
            x, y = int(S[I]), int(S[J])
            p, q, r, s = (int(L[c][k]) for c in "pqrs")
            if L["degree"][k] == 1:
                op = ad[p] @ a[q]
                assert bin(x ^ y).count("1") == 2
            else:
                op = ad[p] @ ad[r] @ a[s] @ a[q]
                assert bin(x ^ y).count("1") == 4 and q < s and p < r
            assert op[y, x] == L["sign"][k]
            assert abs(Hjw[y, x] - L["hval"][k]) < 1e-12
    # every pair at distance 1 or 2 is present exactly once, in ascending J order
    for I in range(len(S)):
        cols = L["col"][L["row_ptr"][I]:L["row_ptr"][I + 1]]
        want = [J for J in range(len(S)) if bin(int(S[I]) ^ int(S[J])).count("1") in (2, 4)]
        assert list(cols) == want


def test_rdm_matches_jordan_wigner():
    """Every 1- and 2-RDM element against expectation values of JW operator
    products on the Fock-space vector (any vector, not only an eigenvector)."""
    n, na, nb = 4, 2, 1
    sa, sb = oracle.build_subspace(*full_space(n, na, nb), na, nb)
    c = synth.random_vector(len(sa) * len(sb), 77)
    g1, g2 = oracle.rdm(n, sa, sb, c)
    psi = np.zeros(1 << (2 * n))
    psi[_fock_index(n, sa, sb)] = c
    a = _jw_ops(2 * n)
    ad = [x.T.tocsr() for x in a]
    for p, q in itertools.product(range(n), repeat=2):
        ref = sum(psi @ (ad[s * n + p] @ (a[s * n + q] @ psi)) for s in range(2))
        assert abs(g1[p, q] - ref) < 1e-12
    for p, q, r, s in itertools.product(range(n), repeat=4):
        ref = 0.0
        for s1 in range(2):
            for s2 in range(2):
                v = a[s1 * n + q] @ psi
                v = a[s2 * n + s] @ v
                v = ad[s2 * n + r] @ v
                v = ad[s1 * n + p] @ v
                ref += psi @ v
        assert abs(g2[p, q, r, s] - ref) < 1e-12


# --------------------------------------------------------- brute force / solvers


def test_small_workload_lanczos_vs_eigh():
    w = synth.workload("fp64_small")
    H = oracle.Ham(w["h"], w["eri"], w["e_nuc"], 3, 3)
    sa, sb = oracle.build_subspace(w["alpha"], w["beta"], 3, 3)
    assert len(sa) * len(sb) == comb(8, 3) ** 2 == 3136
    Hm = oracle.dense_h(H, sa, sb)
    assert np.max(np.abs(Hm - Hm.T)) < 1e-13
    E, c = oracle.ground_state_dense(H, sa, sb)
    El, cl, r = oracle.lanczos(H, sa, sb, tol=1e-11)
    assert abs(E - El) < 1e-10 and r < 1e-8
    assert abs(abs(c @ cl) - 1) < 1e-8
    # matrix-free sigma equals the dense product; diagonal equals diag(H)
    x = synth.random_vector(len(c), 5)
    assert np.max(np.abs(oracle.sigma(H, sa, sb, x) - Hm @ x)) < 1e-11
    assert np.max(np.abs(oracle.diag(H, sa, sb) - np.diag(Hm))) < 1e-13


def test_variational_interlacing():
    """Step 3 is variational: removing strings never lowers the energy."""
    h, eri, _ = synth.integrals(7, 41)
    sa, sb = full_space(7, 3, 2)
    E_full, _ = fci_dense(h, eri, 0.0, 3, 2)
    rng = np.random.default_rng(0)
    prev = E_full
    keep_a, keep_b = list(sa), list(sb)
    for _ in range(4):
        keep_a = list(rng.choice(keep_a, size=int(len(keep_a) * 0.8), replace=False))
        keep_b = list(rng.choice(keep_b, size=int(len(keep_b) * 0.8), replace=False))
        a2, b2 = oracle.build_subspace(keep_a, keep_b, 3, 2)
        E, _ = fci_dense(h, eri, 0.0, 3, 2, a2, b2)
        assert E >= prev - 1e-12
        prev = E


# ------------------------------------------------------------------------ RDMs


def test_rdm_traces_and_energy_identity():
    h, eri, _ = synth.integrals(6, 51)
    sa, sb = oracle.build_subspace(*full_space(6, 3, 2), 3, 2)
    H = oracle.Ham(h, eri, 0.7, 3, 2)
    E, c = oracle.ground_state_dense(H, sa, sb)
    g1, g2 = oracle.rdm(6, sa, sb, c)
    N = 5
    assert abs(np.trace(g1) - N) < 1e-12
    assert abs(np.einsum("pprr->", g2) - N * (N - 1)) < 1e-11
    assert np.max(np.abs(g1 - g1.T)) < 1e-13
    assert np.max(np.abs(g2 - g2.transpose(2, 3, 0, 1))) < 1e-13
    assert abs(oracle.energy_from_rdm(H, g1, g2) - E) < 1e-11
    # partial trace: sum_r Gamma_pqrr = (N-1) gamma_pq
    assert np.max(np.abs(np.einsum("pqrr->pq", g2) - (N - 1) * g1)) < 1e-12


def test_rdm_hellmann_feynman_finite_difference():
    """dE/dh_pq = gamma_pq and dE/d(pq|rs) = Gamma_pqrs / 2, entrywise; a
    symmetric perturbation moves a whole symmetry orbit, so the central FD is
    compared with the sum of the entrywise derivatives over the orbit."""
    n = 5
    h, eri, _ = synth.integrals(n, 61)
    sa, sb = oracle.build_subspace(*full_space(n, 2, 2), 2, 2)
    E, c = fci_dense(h, eri, 0.0, 2, 2, sa, sb)
    g1, g2 = oracle.rdm(n, sa, sb, c)
    d = 1e-5
    for (p, q) in [(0, 1), (2, 2), (1, 4)]:
        dh = np.zeros_like(h)
        dh[p, q] = dh[q, p] = 1.0
        Ep, _ = fci_dense(h + d * dh, eri, 0.0, 2, 2, sa, sb)
        Em, _ = fci_dense(h - d * dh, eri, 0.0, 2, 2, sa, sb)
        assert abs((Ep - Em) / (2 * d) - np.sum(dh * g1)) < 1e-7
    for (p, q, r, s) in [(0, 1, 2, 3), (1, 1, 0, 0), (0, 2, 0, 2), (4, 3, 3, 1)]:
        de = np.zeros_like(eri)
        for idx in {(p, q, r, s), (q, p, r, s), (p, q, s, r), (q, p, s, r),
                    (r, s, p, q), (s, r, p, q), (r, s, q, p), (s, r, q, p)}:
            de[idx] = 1.0
        Ep, _ = fci_dense(h, eri + d * de, 0.0, 2, 2, sa, sb)
        Em, _ = fci_dense(h, eri - d * de, 0.0, 2, 2, sa, sb)
        assert abs((Ep - Em) / (2 * d) - 0.5 * np.sum(de * g2)) < 1e-7


# -------------------------------------------------------------- marginals


def test_marginals_product_state_and_normalisation():
    rng = np.random.default_rng(4)
    u, v = rng.standard_normal(7), rng.standard_normal(5)
    c = 3.0 * np.outer(u, v).ravel()
    pa, pb, w = oracle.marginals(c, 7, 5, want_w=True)
    assert np.allclose(pa, u * u / (u @ u), atol=1e-15, rtol=1e-13)
    assert np.allclose(pb, v * v / (v @ v), atol=1e-15, rtol=1e-13)
    assert abs(pa.sum() - 1) < 1e-14 and abs(pb.sum() - 1) < 1e-14
    assert abs(w.sum() - 1) < 1e-14
    # generic state: both marginals sum to one; w is the normalised outer product
    c = rng.standard_normal(35)
    pa, pb, w = oracle.marginals(c, 7, 5, want_w=True)
    assert abs(pa.sum() - 1) < 1e-14 and abs(pb.sum() - 1) < 1e-14
    assert np.allclose(w, np.outer(pa, pb).ravel() / np.outer(pa, pb).sum(), rtol=1e-13)
    # brute force definition with explicit loops
    c2 = (c * c / (c @ c)).reshape(7, 5)
    assert np.allclose(pa, [sum(c2[a, b] for b in range(5)) for a in range(7)], rtol=1e-13)


# --------------------------------------------------------------- subspace


def test_particle_number_filter():
    a = np.array([0b111, 0b1011, 0b11, 0b111, 0b1110], dtype=np.uint64)
    sa, sb = oracle.build_subspace(a, a, 3, 2)
    assert list(sa) == [0b111, 0b1011, 0b1110]
    assert list(sb) == [0b11]
    with pytest.raises(ValueError):
        oracle.build_subspace(a, a, 3, 2, drop_bad=False)


def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_dimensions.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, n, na, nb, ndet, digits = line.split()
            rows.append((name, int(n), int(na), int(nb), float(ndet), digits))
    return rows


@pytest.mark.parametrize("row", _table1(), ids=lambda r: r[0])
def test_table1_full_space_dimensions(row):
    """Full-space product dimension C(M,n_a) C(M,n_b) against Table 1's N_det^Ref."""
    name, n, na, nb, ndet, digits = row
    dim = comb(n, na) * comb(n, nb)
    if digits == "exact":
        assert dim == int(ndet)
    else:
        assert float(f"{dim:.{int(digits) - 1}e}") == ndet
    if comb(n, na) <= 5000:
        sa, sb = oracle.build_subspace(synth.all_strings(n, na), synth.all_strings(n, nb), na, nb)
        assert len(sa) * len(sb) == dim


# ------------------------------------------------------ PT2 coupling pins


@pytest.mark.parametrize("n,na,nb,seed", [(4, 2, 2, 31), (5, 2, 1, 32)])
def test_pt2_coupling_matches_jordan_wigner(n, na, nb, seed):
    """Eq. pt2_score numerator and H_xx for every determinant of the sector, with a
    random c on a sampled subspace: <x|H|c> = (H_JW c_embedded)_x, H_xx = H_JW[x, x]."""
    h, eri, _ = synth.integrals(n, seed)
    Hjw = _jw_hamiltonian(h, eri, 0.7).toarray()
    fa, fb = full_space(n, na, nb)
    rng = np.random.default_rng(seed)
    sa = np.sort(rng.choice(fa, size=max(1, len(fa) // 2), replace=False))
    sb = np.sort(rng.choice(fb, size=max(1, (len(fb) + 1) // 2), replace=False))
    H = oracle.Ham(h, eri, 0.7, na, nb)
    c = synth.random_vector(len(sa) * len(sb), seed)
    full = np.zeros(Hjw.shape[0])
    full[_fock_index(n, sa, sb)] = c
    xa = np.repeat(fa, len(fb))
    xb = np.tile(fb, len(fa))
    v, hxx, s = oracle.pt2_scores(H, sa, sb, c, -3.0, xa, xb)
    fidx = np.array([int(a) | (int(b) << n) for a, b in zip(xa, xb)])
    assert np.max(np.abs(v - (Hjw @ full)[fidx])) < 1e-12
    assert np.max(np.abs(hxx - np.diag(Hjw)[fidx])) < 1e-12
    assert np.allclose(s, v * v / np.abs(-3.0 - hxx), rtol=1e-14, atol=0)


def test_pt2_coupling_inside_subspace_is_eigen_equation():
    """For x in the subspace and c its ground state, <x|H|Psi0> = E0 c_x, so the
    score of a basis member is E0^2 c_x^2 / |E0 - H_xx|."""
    w = synth.workload("fp64_small")
    H = oracle.Ham(w["h"], w["eri"], 0.4, 3, 3)
    sa, sb = oracle.build_subspace(w["alpha"][:40], w["beta"][:30], 3, 3)
    E, c = oracle.ground_state_dense(H, sa, sb)
    xa, xb = np.repeat(sa, len(sb)), np.tile(sb, len(sa))
    v, hxx, s = oracle.pt2_scores(H, sa, sb, c, E, xa, xb)
    assert np.max(np.abs(v - E * c)) < 1e-11
    hd = oracle.diag(H, sa, sb)
    assert np.max(np.abs(hxx - hd)) < 1e-12


# ------------------------------------------------- classical expansion pins


@pytest.mark.parametrize("n,na,nb,seed", [(4, 2, 2, 51), (5, 2, 1, 52), (4, 1, 0, 53)])
def test_connected_matches_jordan_wigner(n, na, nb, seed):
    """Eq. classical_expansion's connection test: y != x with <y|H|x> != 0, and the
    element, against the Fock-space matrix."""
    h, eri, _ = synth.integrals(n, seed)
    Hjw = _jw_hamiltonian(h, eri, 0.0).toarray()
    H = oracle.Ham(h, eri, 0.0, na, nb)
    fa, fb = full_space(n, na, nb)
    for xa in fa:
        for xb in fb:
            x = int(xa) | (int(xb) << n)
            ya, yb, val = oracle.connected(H, xa, xb)
            col = Hjw[:, x].copy()
            col[x] = 0.0
            ref = np.nonzero(np.abs(col) > 0)[0]
            got = np.array([int(a) | (int(b) << n) for a, b in zip(ya, yb)], dtype=np.int64)
            assert sorted(got.tolist()) == sorted(ref.tolist())
            assert np.max(np.abs(col[got] - val), initial=0.0) < 1e-12


def test_connected_counts_generic_integrals():
    """With generic integrals every single and double is connected:
    2 x n_e(n - n_e) singles, 2 x C(n_e,2) C(n - n_e,2) doubles, (n_e(n - n_e))^2 mixed."""
    from math import comb
    n, ne = 8, 3
    h, eri, _ = synth.integrals(n, 61)
    H = oracle.Ham(h, eri, 0.0, ne, ne)
    ya, yb, _ = oracle.connected(H, 0b10101, 0b1011)
    s1 = ne * (n - ne)
    assert len(ya) == 2 * s1 + 2 * comb(ne, 2) * comb(n - ne, 2) + s1 * s1


def test_connected_wide_orbitals_embeds_small_problem():
    """Strings above bit 32: an 8-orbital problem placed, order-preserving, on eight of
    40 orbitals (integrals zero elsewhere) has the same connected set and elements,
    relabelled, since the phases count occupied orbitals between two positions and the
    embedding keeps that order.  With generic 40-orbital integrals the count of
    singles and doubles holds as on small n."""
    from math import comb
    n, N, na, nb = 8, 40, 3, 2
    pos = np.array([1, 6, 17, 31, 32, 33, 38, 39])
    h, eri, _ = synth.integrals(n, 62)
    hw, eriw = np.zeros((N, N)), np.zeros((N, N, N, N))
    hw[np.ix_(pos, pos)] = h
    eriw[np.ix_(pos, pos, pos, pos)] = eri

    def up(s):
        return sum(1 << int(pos[p]) for p in range(n) if (int(s) >> p) & 1)

    Hs, Hw = oracle.Ham(h, eri, 0.0, na, nb), oracle.Ham(hw, eriw, 0.0, na, nb)
    for xa, xb in [(0b10101, 0b11), (0b11100000, 0b10000001), (0b1011, 0b1100000)]:
        ya, yb, val = oracle.connected(Hs, xa, xb)
        wa, wb, wval = oracle.connected(Hw, up(xa), up(xb))
        ref = {(up(a), up(b)): v for a, b, v in zip(ya, yb, val)}
        got = dict(zip(zip(wa.tolist(), wb.tolist()), wval.tolist()))
        assert set(got) == set(ref) and len(ref) > 10
        assert max(abs(got[k] - ref[k]) for k in ref) < 1e-12
        assert list(zip(wa.tolist(), wb.tolist())) == sorted(got)
    hg, erig, _ = synth.integrals(N, 63)
    ya, _, _ = oracle.connected(oracle.Ham(hg, erig, 0.0, na, nb), (1 << 35) | 0b110, (1 << 39) | 1)
    s = [na * (N - na), nb * (N - nb)]
    assert len(ya) == sum(s) + comb(na, 2) * comb(N - na, 2) + comb(nb, 2) * comb(N - nb, 2) + s[0] * s[1]


def test_classical_expansion_excludes_subspace_and_is_union():
    w = synth.workload("fp64_small")
    H = oracle.Ham(w["h"], w["eri"], 0.0, 3, 3)
    sa, sb = oracle.build_subspace(w["alpha"][:12], w["beta"][:9], 3, 3)
    c = synth.random_vector(len(sa) * len(sb), 3)
    top = oracle.top_amplitudes(c, 6)
    assert len(top) == 6 and set(top) == set(np.argsort(-np.abs(c))[:6])
    xa, xb = oracle.classical_expansion(H, sa, sb, c, 6)
    inside = set((int(a), int(b)) for a in sa for b in sb)
    got = set(zip(xa.tolist(), xb.tolist()))
    assert not (got & inside)
    union = set()
    for I in top:
        ya, yb, _ = oracle.connected(H, sa[I // len(sb)], sb[I % len(sb)])
        union |= set(zip(ya.tolist(), yb.tolist()))
    assert got == union - inside


# ------------------------------------------------------------ basis-list pins
# Step 3 over the basis list itself: [H_B]_ij = <x_i|H|x_j> for the listed
# determinants.  Pinned against the Jordan-Wigner matrix restricted to the list (the
# list need not be a product of strings), the variational bound of Step 3 and its
# special cases, and a brute-force classical expansion.


def _random_list(n, na, nb, m, seed):
    fa, fb = full_space(n, na, nb)
    rng = np.random.default_rng(seed)
    pairs = {(int(fa[rng.integers(len(fa))]), int(fb[rng.integers(len(fb))])) for _ in range(4 * m)}
    pairs = sorted(pairs)[:m] if len(pairs) > m else sorted(pairs)
    pairs = [pairs[i] for i in sorted(rng.choice(len(pairs), min(m, len(pairs)), replace=False))]
    return (np.array([p[0] for p in pairs], dtype=np.uint64),
            np.array([p[1] for p in pairs], dtype=np.uint64))


def _list_fock(n, xa, xb):
    return np.array([int(a) | (int(b) << n) for a, b in zip(xa, xb)], dtype=np.int64)


@pytest.mark.parametrize("n,na,nb,m,seed", [(4, 2, 2, 20, 71), (5, 2, 2, 37, 72), (4, 1, 3, 9, 73)])
def test_dense_h_list_matches_jordan_wigner(n, na, nb, m, seed):
    h, eri, _ = synth.integrals(n, seed)
    Hjw = _jw_hamiltonian(h, eri, 0.4).toarray()
    xa, xb = oracle.sort_list(*_random_list(n, na, nb, m, seed))
    H = oracle.Ham(h, eri, 0.4, na, nb)
    idx = _list_fock(n, xa, xb)
    ref = Hjw[np.ix_(idx, idx)]
    assert np.max(np.abs(oracle.dense_h_list(H, xa, xb) - ref)) < 1e-12
    c = synth.random_vector(len(xa), seed)
    assert np.max(np.abs(oracle.sigma_list(H, xa, xb, c) - ref @ c)) < 1e-12
    rows = np.array([len(xa) - 1, 0, len(xa) // 2])
    assert np.max(np.abs(oracle.sigma_list(H, xa, xb, c, rows=rows) - (ref @ c)[rows])) < 1e-12


def test_list_ground_state_bounds_and_limits():
    """One determinant gives H_xx; the whole product gives the product's ground state;
    a list lies above the product of its strings, which lies above the full space, and
    a longer list (containing the shorter) never lies higher (Step 3 is variational)."""
    n, na, nb = 6, 2, 2
    h, eri, e_nuc = synth.integrals(n, 74)
    H = oracle.Ham(h, eri, e_nuc, na, nb)
    Hjw = _jw_hamiltonian(h, eri, e_nuc)
    xa, xb = oracle.sort_list(*_random_list(n, na, nb, 60, 74))
    E1, c1 = oracle.ground_state_dense_list(H, xa[:1], xb[:1])
    x0 = int(xa[0]) | (int(xb[0]) << n)
    assert abs(E1 - Hjw[x0, x0]) < 1e-12 and abs(abs(c1[0]) - 1.0) < 1e-15
    sa, sb = oracle.build_subspace(xa, xb, na, nb)
    pa, pb = np.repeat(sa, len(sb)), np.tile(sb, len(sa))
    E_prod, _ = oracle.ground_state_dense(H, sa, sb)
    E_prod_list, _ = oracle.ground_state_dense_list(H, pa, pb)
    assert abs(E_prod - E_prod_list) < 1e-11
    E_list, c_list = oracle.ground_state_dense_list(H, xa, xb)
    E_fci, _ = fci_dense(h, eri, e_nuc, na, nb)
    assert E_list >= E_prod - 1e-12 and E_prod >= E_fci - 1e-12
    assert E_list > E_prod + 1e-6  # a strict sub-list of a generic product lies higher
    half = np.sort(np.random.default_rng(1).choice(len(xa), len(xa) // 2, replace=False))
    E_half, _ = oracle.ground_state_dense_list(H, xa[half], xb[half])
    assert E_half >= E_list - 1e-12
    # the eigen-equation through the JW matrix restricted to the list
    idx = _list_fock(n, xa, xb)
    Hl = Hjw.toarray()[np.ix_(idx, idx)]
    assert np.max(np.abs(Hl @ c_list - E_list * c_list)) < 1e-10


def test_sort_list_and_unsorted_lists_rejected():
    xa = np.array([5, 3, 5, 3], dtype=np.uint64)
    xb = np.array([6, 9, 6, 3], dtype=np.uint64)
    sa, sb = oracle.sort_list(xa, xb)
    assert sa.tolist() == [3, 3, 5] and sb.tolist() == [3, 9, 6]
    h, eri, _ = synth.integrals(4, 75)
    H = oracle.Ham(h, eri, 0.0, 2, 2)
    with pytest.raises(ValueError):
        oracle.dense_h_list(H, xa, xb)


def test_classical_expansion_list_against_jordan_wigner():
    """Determinants outside the list connected (non-zero JW element) to one of the n_top
    largest |c| of the list; members of the product that are not in the list are
    candidates too."""
    n, na, nb = 5, 2, 1
    h, eri, _ = synth.integrals(n, 76)
    Hjw = _jw_hamiltonian(h, eri, 0.0).toarray()
    H = oracle.Ham(h, eri, 0.0, na, nb)
    xa, xb = oracle.sort_list(*_random_list(n, na, nb, 12, 76))
    c = synth.random_vector(len(xa), 76)
    ya, yb = oracle.classical_expansion_list(H, xa, xb, c, 4)
    fock = _list_fock(n, xa, xb)
    top = np.argsort(-np.abs(c), kind="stable")[:4]
    ref = set()
    for i in top:
        col = Hjw[:, fock[i]]
        ref |= set(np.nonzero(np.abs(col) > 0)[0].tolist())
    ref -= set(fock.tolist())
    got = set(_list_fock(n, ya, yb).tolist())
    assert got == ref
    sa, sb = oracle.build_subspace(xa, xb, na, nb)
    prod = set(int(a) | (int(b) << n) for a in sa for b in sb)
    assert got & (prod - set(fock.tolist()))  # product members outside the list appear
    assert list(zip(ya.tolist(), yb.tolist())) == sorted(zip(ya.tolist(), yb.tolist()))
