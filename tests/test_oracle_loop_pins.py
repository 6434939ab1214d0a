"""Pins of the oracle's outer-loop functions (Sec. 2.2 Steps 1-5 around the subspace
solve) against facts other than themselves: Python's own sort and set semantics on
small inputs, a hand-worked basis update (tests/golden/basis_update_example.txt),
the diagonal of a Jordan-Wigner Fock-space Hamiltonian, the invariance of the
Rayleigh quotient when an eigenvector is carried to a larger subspace, closed forms
of the teacher weights and advantages for a single-determinant ground state and for
a uniform state, and central differences of the total loss."""
import os

import numpy as np
import pytest

import oracle
import synth
from test_oracle_pins import _fock_index, _jw_hamiltonian, full_space

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ selection


@pytest.mark.parametrize("seed", range(6))
def test_select_top_matches_python_sort(seed):
    """Top-k with ties to the lower position: against Python's stable sort."""
    rng = np.random.default_rng(seed)
    m = int(rng.integers(1, 40))
    v = rng.integers(-4, 5, size=m).astype(np.float64) * 0.25     # many ties
    v[rng.random(m) < 0.1] = np.inf
    v[rng.random(m) < 0.1] = -np.inf
    v[rng.random(m) < 0.1] = -0.0
    for k in (0, 1, m // 2, m, m + 3):
        big = sorted(range(m), key=lambda i: (-v[i], i))[:k]
        small = sorted(range(m), key=lambda i: (v[i], i))[:k]
        assert list(oracle.select_top(v, k)) == sorted(big)
        assert list(oracle.select_top(v, k, largest=False)) == sorted(small)


# ------------------------------------------------------------- basis update


def _golden_basis_cases():
    entries, cases = {"basis": [], "cand": []}, []
    with open(os.path.join(GOLDEN, "basis_update_example.txt")) as f:
        for line in f:
            t = line.split("#")[0].split()
            if not t:
                continue
            if t[0] in entries:
                entries[t[0]].append((t[1], float(t[2])))
            elif t[0] == "case":
                arrow = t.index("->")
                cases.append((t[1], int(t[2]), int(t[3]), t[arrow + 1:]))
    return entries, cases


def test_basis_update_hand_worked_example():
    entries, cases = _golden_basis_cases()
    labels = [e[0] for e in entries["basis"]] + [e[0] for e in entries["cand"]]
    code = {lab: i for i, lab in enumerate(labels)}     # label -> a fake determinant id
    def arr(kind):
        a = np.array([code[e[0]] for e in entries[kind]], dtype=np.uint64)
        return a, a + np.uint64(100), np.array([e[1] for e in entries[kind]])
    modes = dict(cold=oracle.BASIS_COLD_START, rescore=oracle.BASIS_RESCORE,
                 append=oracle.BASIS_APPEND)
    assert len(cases) == 6
    for mode, K, bmax, expect in cases:
        ba, bb, bs = oracle.basis_update(modes[mode], arr("basis"), arr("cand"), K, bmax)
        assert [labels[int(x)] for x in ba] == expect, (mode, K, bmax)
        assert np.all(bb == ba + np.uint64(100))


def test_basis_update_invariants():
    rng = np.random.default_rng(3)
    ba = np.arange(50, dtype=np.uint64)
    ca = np.arange(50, 130, dtype=np.uint64)
    bs, cs = rng.random(50), rng.random(80)
    for K, bmax in ((10, 55), (40, 60), (0, 50), (80, 200)):
        na, nb_, ns = oracle.basis_update(oracle.BASIS_APPEND, (ba, ba, bs), (ca, ca, cs), K, bmax)
        assert len(na) == min(50 + K, bmax)
        kept = set(na.tolist())
        dropped = [s for a, s in zip(np.concatenate([ba, ca]).tolist(), np.concatenate([bs, cs]))
                   if a not in kept]
        # every evicted or unselected entry scores no higher than every kept one,
        # except candidates that were never among the top K
        top_c = set(ca[oracle.select_top(cs, K)].tolist())
        evicted = [s for a, s in zip(np.concatenate([ba, ca]).tolist(), np.concatenate([bs, cs]))
                   if a not in kept and (a < 50 or a in top_c)]
        if evicted:
            assert max(evicted) <= ns.min()
        assert len(dropped) == 130 - len(na)


# ------------------------------------------------------- pools and lookups


def test_candidate_pool_matches_set_semantics():
    rng = np.random.default_rng(8)
    n, na, nb = 6, 2, 3
    Sa, Sb = synth.all_strings(n, na), synth.all_strings(n, nb)
    bad = np.array([0b111, 0b1], dtype=np.uint64)             # wrong electron counts
    pools = []
    for m in (40, 25):
        xa = rng.choice(np.concatenate([Sa, bad]), m)
        xb = rng.choice(Sb, m)
        pools.append((xa, xb))
    ea, eb = rng.choice(Sa, 12), rng.choice(Sb, 12)
    ya, yb, dropped = oracle.candidate_pool(pools, (ea, eb), na, nb)
    # independent statement: numpy unique of the keys of the good entries, minus
    # np.isin against the excluded keys
    allx = np.concatenate([p[0] for p in pools]).astype(np.int64)
    ally = np.concatenate([p[1] for p in pools]).astype(np.int64)
    good = np.array([bin(a).count("1") == na for a in allx.tolist()])
    keys = np.unique(allx[good] * 4096 + ally[good])
    keys = keys[~np.isin(keys, ea.astype(np.int64) * 4096 + eb.astype(np.int64))]
    assert dropped == int((~good).sum())
    assert np.array_equal(ya.astype(np.int64) * 4096 + yb.astype(np.int64), keys)


def test_lookup_brute_force():
    sa = np.array([3, 5, 6, 9, 10], dtype=np.uint64)
    sb = np.array([3, 12], dtype=np.uint64)
    xa = np.array([5, 6, 7, 10, 3], dtype=np.uint64)
    xb = np.array([12, 3, 3, 5, 3], dtype=np.uint64)
    got = oracle.lookup(sa, sb, xa, xb)
    ref = [list(sa).index(a) * len(sb) + list(sb).index(b) if a in list(sa) and b in list(sb)
           else -1 for a, b in zip(xa, xb)]
    assert list(got) == ref == [3, 4, -1, -1, 0]


# ------------------------------------------------------------------ H_xx


@pytest.mark.parametrize("n,na,nb,seed", [(4, 2, 2, 41), (4, 1, 3, 42)])
def test_determinant_diag_matches_jordan_wigner(n, na, nb, seed):
    h, eri, _ = synth.integrals(n, seed)
    Hjw = _jw_hamiltonian(h, eri, -0.7)
    sa, sb = full_space(n, na, nb)
    xa = np.repeat(sa, len(sb))
    xb = np.tile(sb, len(sa))
    idx = np.array([int(a) | (int(b) << n) for a, b in zip(xa, xb)])
    ref = np.asarray(Hjw.diagonal())[idx]
    got = oracle.determinant_diag(oracle.Ham(h, eri, -0.7, na, nb), xa, xb)
    assert np.max(np.abs(got - ref)) < 1e-12


# ------------------------------------------------------------- warm start


def test_remap_vector_preserves_rayleigh_quotient():
    """Carrying the ground state of S_a x S_b into a larger product subspace keeps
    its norm and its Rayleigh quotient; carrying it back recovers it."""
    w = synth.workload("fp64_small")
    n, na, nb = w["n_orb"], w["n_alpha"], w["n_beta"]
    H = oracle.Ham(w["h"], w["eri"], w["e_nuc"], na, nb)
    A, B = synth.all_strings(n, na), synth.all_strings(n, nb)
    sa, sb = np.sort(A[::3]), np.sort(B[::2])
    E, c = oracle.ground_state_dense(H, sa, sb)
    sa2, sb2 = np.sort(A[::1]), np.sort(B[::1])
    c2 = oracle.remap_vector(sa, sb, c, sa2, sb2)
    assert abs(c2 @ c2 - 1.0) < 1e-14
    H2 = oracle.dense_h(H, sa2, sb2)
    assert abs(c2 @ H2 @ c2 - E) < 1e-12
    assert np.array_equal(oracle.remap_vector(sa2, sb2, c2, sa, sb), c)
    # identity on the same subspace; zeros where nothing overlaps
    assert np.array_equal(oracle.remap_vector(sa, sb, c, sa, sb), c)
    other = np.setdiff1d(A, sa)
    assert not np.any(oracle.remap_vector(sa, sb, c, other, sb))


# ---------------------------------------------------------- NQS loss inputs


def test_nqs_loss_single_determinant_ground_state():
    """With (pq|rs) = 0 and a diagonal h the determinants are eigenstates and the
    ground state is the determinant of the lowest orbitals: the teacher weight is
    one there and zero elsewhere, and A(x) = sum over x's occupied orbitals of
    h_pp minus the same sum for the ground determinant (both spins)."""
    n, na, nb = 6, 2, 3
    h = np.diag(np.sort(np.random.default_rng(1).uniform(-2, 0, n)))
    eri = np.zeros((n,) * 4)
    H = oracle.Ham(h, eri, 0.4, na, nb)
    sa, sb = full_space(n, na, nb)
    sa, sb = np.sort(sa), np.sort(sb)
    E0, c = oracle.ground_state_dense(H, sa, sb)
    eps = np.diag(h)
    assert abs(E0 - (eps[:na].sum() + eps[:nb].sum() + 0.4)) < 1e-12
    batch = np.arange(len(sa) * len(sb))
    logpi = np.random.default_rng(2).uniform(-9, -1, len(batch))
    r = oracle.nqs_loss(H, sa, sb, c, E0, batch, logpi, coef=(0.7, 0.2, 0.1))
    occ = lambda s: [p for p in range(n) if (int(s) >> p) & 1]
    A_ref = np.array([sum(eps[occ(a)]) + sum(eps[occ(b)]) for a in sa for b in sb]) \
        - eps[:na].sum() - eps[:nb].sum()
    assert np.max(np.abs(r["A"] - A_ref)) < 1e-12
    hf = list(sa).index((1 << na) - 1) * len(sb) + list(sb).index((1 << nb) - 1)
    w_ref = np.zeros(len(batch))
    w_ref[hf] = 1.0
    assert np.max(np.abs(r["w"] - w_ref)) < 1e-12
    assert abs(r["teacher"] + logpi[hf]) < 1e-10
    assert abs(r["energy"]) < 1e-10      # w A vanishes: A = 0 where w = 1
    assert abs(r["entropy"] - logpi.mean()) < 1e-12


def test_nqs_loss_uniform_state_and_list_basis():
    """A uniform state gives w = 1/|B| on the product subspace; with log pi = log w
    over all of B the teacher loss is the entropy log|B| and the entropy loss -log|B|.
    On a listed basis the weights are renormalised over the list."""
    w = synth.workload("fp64_small")
    H = oracle.Ham(w["h"], w["eri"], w["e_nuc"], 3, 3)
    sa, sb = np.sort(w["alpha"])[:7], np.sort(w["beta"])[:5]
    N = 35
    c = np.full(N, 0.3)
    batch = np.arange(N)
    r = oracle.nqs_loss(H, sa, sb, c, -1.0, batch, np.full(N, -np.log(N)))
    assert np.allclose(r["w"], 1.0 / N, rtol=1e-14)
    assert abs(r["teacher"] - np.log(N)) < 1e-13
    assert abs(r["entropy"] + np.log(N)) < 1e-13
    # a minibatch keeps the basis normalisation: still 1/|B| each, not 1/|M|
    r = oracle.nqs_loss(H, sa, sb, c, -1.0, batch[3:13], np.full(10, -2.0))
    assert np.allclose(r["w"], 1.0 / N, rtol=1e-14)
    assert abs(r["entropy"] + 2.0) < 1e-14
    basis = np.array([0, 3, 4, 11, 20, 34])
    c = np.random.default_rng(5).standard_normal(N)
    r = oracle.nqs_loss(H, sa, sb, c, -1.0, basis, np.zeros(6), basis=basis)
    assert abs(r["w"].sum() - 1.0) < 1e-14


def test_nqs_loss_gradient_central_differences():
    w = synth.workload("fp64_small")
    H = oracle.Ham(w["h"], w["eri"], w["e_nuc"], 3, 3)
    sa, sb = np.sort(w["alpha"])[:6], np.sort(w["beta"])[:6]
    rng = np.random.default_rng(9)
    c = rng.standard_normal(36)
    batch = rng.choice(36, 10, replace=False)
    logpi = rng.uniform(-6, -1, 10)
    coef = (0.5, 1.5, -0.3)
    E0 = -3.0
    g = oracle.nqs_loss(H, sa, sb, c, E0, batch, logpi, coef)["grad"]
    for k in range(10):
        d = np.zeros(10)
        d[k] = 1e-4
        up = oracle.nqs_loss(H, sa, sb, c, E0, batch, logpi + d, coef)["total"]
        dn = oracle.nqs_loss(H, sa, sb, c, E0, batch, logpi - d, coef)["total"]
        assert abs((up - dn) / 2e-4 - g[k]) < 1e-9


# --------------------------------------------------------------- stopping rule


def test_convergence_rule():
    """Step 5: five consecutive changes below 1e-9 Ha, or 50 iterations."""
    e = [-1.0, -1.1, -1.2] + [-1.2 - 1e-10 * k for k in range(1, 5)]
    assert not oracle.converged(e)                  # only four small changes so far
    assert oracle.converged(e + [-1.2 - 5e-10])     # the fifth
    assert not oracle.converged(e + [-1.3])
    assert oracle.converged(list(np.linspace(0, -1, 50)))
