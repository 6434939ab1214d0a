"""The outer-loop calls (Sec. 2.2 Steps 1-5 around the subspace solve) against the
oracle, through the C ABI.

Integer work (selections, candidate sets, lookups, basis lists) is compared bit for
bit; where a selection is decided by floating-point keys, both sides are given the
same keys (the library's), as the decision must be taken in one precision.  FP64
values: H_xx to 1e-12 relative, PT2 scores to 1e-9 relative where |E0 - H_xx| is not
tiny, loss inputs and values to 1e-12 relative (sums of at most a few thousand terms
in another order), energies to 1e-9 Ha (Davidson to a 1e-8 residual against dense
eigh)."""
import os

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

hq = pytest.importorskip("paper_2606_26760_b300")
from paper_2606_26760_b300.loop import HiNqsLoop  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _np_u64(t):
    return t.cpu().numpy().astype(np.uint64)


# ------------------------------------------------------------------ selection


@pytest.mark.parametrize("m", [0, 1, 7, 1000, 70001])
def test_select_top_matches_oracle(m):
    rng = np.random.default_rng(m)
    v = rng.integers(-50, 50, size=m).astype(np.float64) * 0.125   # many ties
    if m:
        v[rng.random(m) < 0.02] = np.inf
        v[rng.random(m) < 0.02] = -np.inf
        v[rng.random(m) < 0.05] = -0.0
        v[rng.random(m) < 0.05] = 0.0
    for k in sorted({0, 1, m // 3, m, m + 5}):
        for largest in (True, False):
            got = hq.select_top(v, k, largest).cpu().numpy()
            ref = oracle.select_top(v, k, largest)
            assert np.array_equal(got, ref), (m, k, largest)


def test_select_top_distinct_values_large():
    """1e6 distinct values: the selection must be exactly the sorted prefix."""
    v = synth.random_vector(1_000_000, 5)
    for k in (1, 4096, 999_999):
        assert np.array_equal(hq.select_top(v, k).cpu().numpy(), oracle.select_top(v, k))
        assert np.array_equal(hq.select_top(v, k, False).cpu().numpy(),
                              oracle.select_top(v, k, False))


# ------------------------------------------------------ H_xx and lookups


@pytest.mark.parametrize("n,na,nb,seed", [(10, 3, 4, 61), (16, 5, 5, 62), (7, 0, 2, 63)])
def test_determinant_diag_matches_oracle(n, na, nb, seed):
    h, eri, _ = synth.integrals(n, seed)
    ham = hq.Hamiltonian(h, eri, na, nb, 0.37)
    xa = synth.hf_weighted_samples(n, na, 500, seed)
    xb = synth.hf_weighted_samples(n, nb, 500, seed + 100)
    got = hq.determinant_diag(ham, xa, xb).cpu().numpy()
    ref = oracle.determinant_diag(oracle.Ham(h, eri, 0.37, na, nb), xa, xb)
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_determinant_diag_rejects_wrong_electron_count():
    h, eri, _ = synth.integrals(6, 3)
    ham = hq.Hamiltonian(h, eri, 2, 2, 0.0)
    xa = np.array([0b11, 0b111, 0b101], dtype=np.uint64)
    xb = np.array([0b11, 0b11, 0b1000001], dtype=np.uint64)   # bit 6 >= n_orb
    with pytest.raises(hq.HinqsError) as e:
        hq.determinant_diag(ham, xa, xb)
    assert e.value.code == hq.ERR_PARTICLE_NUMBER


def test_lookup_matches_oracle():
    w = synth.workload("precision")
    n, na, nb = w["n_orb"], w["n_alpha"], w["n_beta"]
    sub = hq.build_subspace(w["alpha"], w["beta"], n, na, nb)
    sa, sb = oracle.build_subspace(w["alpha"], w["beta"], na, nb)
    xa = synth.hf_weighted_samples(n, na, 20000, 71)
    xb = synth.hf_weighted_samples(n, nb, 20000, 72)
    got = hq.lookup_determinants(sub, xa, xb).cpu().numpy()
    ref = oracle.lookup(sa, sb, xa, xb)
    assert np.array_equal(got, ref)
    assert (ref >= 0).sum() > 100 and (ref < 0).sum() > 100   # both cases present


# ------------------------------------------------------------- candidate pool


@pytest.mark.parametrize("m1,m2,me", [(0, 0, 0), (1, 0, 0), (5000, 3000, 700), (300, 0, 5000),
                                      (0, 2500, 0)])
def test_candidate_pool_matches_oracle(m1, m2, me):
    n, na, nb = 12, 4, 3
    h, eri, _ = synth.integrals(n, 7)
    ham = hq.Hamiltonian(h, eri, na, nb, 0.0)
    rng = np.random.default_rng(m1 + 7 * m2 + me)

    def dets(m, seed):
        xa = synth.hf_weighted_samples(n, na, m, seed)
        xb = synth.hf_weighted_samples(n, nb, m, seed + 1)
        bad = rng.random(m) < 0.03
        xa[bad] ^= np.uint64(1)                            # wrong electron count
        far = rng.random(m) < 0.01
        xb[far] |= np.uint64(1 << 40)                      # bit above n_orb
        return xa, xb
    p1, p2 = dets(m1, 1), dets(m2, 3)
    ex = dets(me, 5)
    got_a, got_b, dropped = hq.candidate_pool(ham, p1, p2 if m2 else None, ex if me else None)
    ra, rb, rd = oracle.candidate_pool([p1, p2], ex, na, nb)
    assert np.array_equal(_np_u64(got_a), ra) and np.array_equal(_np_u64(got_b), rb)
    assert dropped == rd


@pytest.mark.parametrize("n,na,nb", [(33, 4, 3), (40, 3, 5), (64, 2, 2), (32, 4, 4)])
def test_candidate_pool_wide_orbitals_matches_oracle(n, na, nb):
    """From 32 orbitals on the pool sorts ranks of the proposals' distinct strings
    instead of packed strings: the same set and order as the oracle's, wrong electron
    counts and bits above n_orb dropped, the basis excluded."""
    h, eri, _ = synth.integrals(n, 8)
    ham = hq.Hamiltonian(h, eri, na, nb, 0.0)
    rng = np.random.default_rng(n)

    def dets(m, seed):
        xa = synth.hf_weighted_samples(n, na, m, seed)
        xb = synth.hf_weighted_samples(n, nb, m, seed + 1)
        bad = rng.random(m) < 0.03
        xa[bad] ^= np.uint64(1)
        if n < 64:
            far = rng.random(m) < 0.02
            xb[far] |= np.uint64(1 << (n + (63 - n) // 2))   # a bit at or above n_orb
        return xa, xb
    p1, p2, ex = dets(3000, 11), dets(800, 13), dets(500, 15)
    ex = (np.concatenate([ex[0], p1[0][:40]]), np.concatenate([ex[1], p1[1][:40]]))
    got_a, got_b, dropped = hq.candidate_pool(ham, p1, p2, ex)
    ra, rb, rd = oracle.candidate_pool([p1, p2], ex, na, nb)
    assert len(ra) > 0
    assert np.array_equal(_np_u64(got_a), ra) and np.array_equal(_np_u64(got_b), rb)
    assert dropped == rd


def test_candidate_pool_everything_excluded():
    n, na, nb = 8, 3, 3
    h, eri, _ = synth.integrals(n, 1)
    ham = hq.Hamiltonian(h, eri, na, nb, 0.0)
    xa = synth.hf_weighted_samples(n, na, 400, 9)
    xb = synth.hf_weighted_samples(n, nb, 400, 10)
    ya, yb, d = hq.candidate_pool(ham, (xa, xb), None, (xa[::-1].copy(), xb[::-1].copy()))
    assert ya.numel() == 0 and yb.numel() == 0 and d == 0


# --------------------------------------------------------------- basis update


def _golden_cases():
    entries, cases = {"basis": [], "cand": []}, []
    with open(os.path.join(GOLDEN, "basis_update_example.txt")) as f:
        for line in f:
            t = line.split("#")[0].split()
            if not t:
                continue
            if t[0] in entries:
                entries[t[0]].append((t[1], float(t[2])))
            elif t[0] == "case":
                cases.append((t[1], int(t[2]), int(t[3]), t[t.index("->") + 1:]))
    return entries, cases


def test_basis_update_hand_worked_example():
    entries, cases = _golden_cases()
    labels = [e[0] for e in entries["basis"]] + [e[0] for e in entries["cand"]]
    code = {lab: i + 1 for i, lab in enumerate(labels)}
    def arr(kind):
        a = np.array([code[e[0]] for e in entries[kind]], dtype=np.uint64)
        return a, a * np.uint64(3), np.array([e[1] for e in entries[kind]])
    modes = dict(cold=hq.BASIS_COLD_START, rescore=hq.BASIS_RESCORE, append=hq.BASIS_APPEND)
    for mode, K, bmax, expect in cases:
        oa, ob, os_ = hq.basis_update(modes[mode], arr("basis"), arr("cand"), K, bmax)
        assert [labels[int(x) - 1] for x in _np_u64(oa)] == expect, (mode, K, bmax)
        assert np.array_equal(_np_u64(ob), _np_u64(oa) * np.uint64(3))


@pytest.mark.parametrize("mode,nb,nc,k,bmax", [
    (0, 0, 3000, 700, 0), (1, 900, 2500, 1000, 0), (1, 0, 10, 20, 0), (2, 1200, 3000, 500, 1500),
    (2, 1200, 3000, 500, 0), (2, 0, 100, 40, 30), (2, 800, 0, 10, 500), (2, 800, 50, 0, 900)])
def test_basis_update_matches_oracle(mode, nb, nc, k, bmax):
    rng = np.random.default_rng(nb + nc + k)
    keys = np.arange(nb + nc, dtype=np.uint64) * np.uint64(7) + np.uint64(1)
    ba, ca = keys[:nb], keys[nb:]
    bs = np.round(rng.standard_normal(nb), 2)          # ties on purpose
    cs = np.round(rng.standard_normal(nc), 2)
    basis = (ba, ba + np.uint64(1), bs) if nb else None
    oa, ob, os_ = hq.basis_update(mode, basis, (ca, ca + np.uint64(1), cs), k, bmax)
    ra, rb, rs = oracle.basis_update(mode, (ba, ba + np.uint64(1), bs),
                                     (ca, ca + np.uint64(1), cs), k, bmax)
    assert np.array_equal(_np_u64(oa), ra) and np.array_equal(_np_u64(ob), rb)
    assert np.array_equal(os_.cpu().numpy(), rs)


# ------------------------------------------------------------------ warm start


def test_remap_vector_matches_oracle():
    w = synth.workload("precision")
    n, na, nb = w["n_orb"], w["n_alpha"], w["n_beta"]
    a2 = synth.hf_weighted_strings(n, na, 2600, 81)     # overlaps the workload's strings
    b2 = synth.hf_weighted_strings(n, nb, 1500, 82)
    old = hq.build_subspace(w["alpha"], w["beta"], n, na, nb)
    new = hq.build_subspace(a2, b2, n, na, nb)
    sa, sb = oracle.build_subspace(w["alpha"], w["beta"], na, nb)
    sa2, sb2 = oracle.build_subspace(a2, b2, na, nb)
    c = synth.random_vector(old.N, 83)
    got, kept = hq.remap_vector(old, torch.tensor(c, device="cuda"), new)
    ref = oracle.remap_vector(sa, sb, c, sa2, sb2)
    assert np.array_equal(got.cpu().numpy(), ref)
    assert abs(kept - ref @ ref) <= 1e-12 * (ref @ ref)
    back, _ = hq.remap_vector(new, got, old)
    mask = oracle.remap_vector(sa2, sb2, np.ones(len(sa2) * len(sb2)), sa, sb) > 0
    assert np.array_equal(back.cpu().numpy(), np.where(mask, c, 0.0))


# ------------------------------------------------------------- NQS loss inputs


def _loss_case(seed=12):
    w = synth.workload("fp64_small")
    n, na, nb = w["n_orb"], w["n_alpha"], w["n_beta"]
    rng = np.random.default_rng(seed)
    a = rng.choice(w["alpha"], 40, replace=False)
    b = rng.choice(w["beta"], 33, replace=False)
    ham = hq.Hamiltonian(w["h"], w["eri"], na, nb, w["e_nuc"] + 0.5)
    sub = hq.build_subspace(a, b, n, na, nb)
    la, lb = hq.string_links(ham, sub, 0), hq.string_links(ham, sub, 1)
    H = oracle.Ham(w["h"], w["eri"], w["e_nuc"] + 0.5, na, nb)
    sa, sb = oracle.build_subspace(a, b, na, nb)
    c = rng.standard_normal(sub.N)
    return ham, sub, la, lb, H, sa, sb, c, rng


@pytest.mark.parametrize("use_list", [False, True])
def test_nqs_loss_matches_oracle(use_list):
    ham, sub, la, lb, H, sa, sb, c, rng = _loss_case()
    ct = torch.tensor(c, device="cuda")
    pa, pb = hq.spin_marginals(sub, ct)
    basis = np.sort(rng.choice(sub.N, 700, replace=False)) if use_list else None
    for m in (1, 257, 700):
        batch = (rng.choice(basis, m, replace=False) if use_list
                 else rng.choice(sub.N, m, replace=False))
        logpi = rng.uniform(-12, -0.5, m)
        coef = (0.9, 0.35, -0.2)
        E0 = -4.2
        r = hq.nqs_loss(ham, sub, la, lb, pa, pb, E0, batch, logpi, coef, basis)
        ref = oracle.nqs_loss(H, sa, sb, c, E0, batch, logpi, coef, basis)
        for key in ("w", "grad"):
            got = r[key].cpu().numpy()
            assert np.max(np.abs(got - ref[key])) <= 1e-12 * max(1e-300, np.max(np.abs(ref[key])))
        assert np.max(np.abs(r["adv"].cpu().numpy() - ref["A"])) <= 1e-12 * np.max(np.abs(ref["A"]))
        loss = r["loss"].cpu().numpy()
        for i, key in enumerate(("total", "teacher", "energy", "entropy")):
            assert abs(loss[i] - ref[key]) <= 1e-12 * max(1.0, abs(ref[key])), key


def test_nqs_loss_autograd_and_bad_index():
    ham, sub, la, lb, H, sa, sb, c, rng = _loss_case(13)
    ct = torch.tensor(c, device="cuda")
    pa, pb = hq.spin_marginals(sub, ct)
    batch = torch.tensor(rng.choice(sub.N, 64, replace=False), device="cuda")
    logpi = torch.tensor(rng.uniform(-8, -1, 64), device="cuda", requires_grad=True)
    L = hq.NqsLoss.apply(logpi, ham, sub, la, lb, pa, pb, -3.0, batch, (1.0, 0.5, 0.1), None)
    L.backward()
    r = hq.nqs_loss(ham, sub, la, lb, pa, pb, -3.0, batch, logpi.detach(), (1.0, 0.5, 0.1))
    assert torch.equal(logpi.grad, r["grad"])
    assert float(L.detach()) == float(r["loss"][0])
    bad = batch.clone()
    bad[5] = sub.N
    with pytest.raises(hq.HinqsError) as e:
        hq.nqs_loss(ham, sub, la, lb, pa, pb, -3.0, bad, logpi.detach())
    assert e.value.code == hq.ERR_ARG


# ------------------------------------------------------------- the whole loop


def _embed(sa, sb, xa, xb, c_list):
    """A vector over the sorted list (xa, xb) placed in the product's indexing."""
    c = np.zeros(len(sa) * len(sb))
    c[oracle.lookup(sa, sb, xa, xb)] = c_list
    return c


def _oracle_chain_step(H, chain, t, samples, na, nb, k0, k, b_max, n_top, mode):
    """One outer iteration done by the oracle alone (Steps 1, 1', 2 and 3 on the basis
    list or on the product of its strings), updating `chain` in place."""
    samples = tuple(np.asarray(x, dtype=np.uint64) for x in samples)
    if t == 0:
        ya, yb, _ = oracle.candidate_pool([samples], (np.zeros(0), np.zeros(0)), na, nb)
        keys = oracle.determinant_diag(H, ya, yb)
        basis = oracle.basis_update(oracle.BASIS_COLD_START, ([], [], []), (ya, yb, keys), k0)
    else:
        if mode == "list":
            ea, eb = oracle.classical_expansion_list(H, chain["la"], chain["lb"], chain["c_list"],
                                                     n_top)
        else:
            ea, eb = oracle.classical_expansion(H, chain["sa"], chain["sb"], chain["c"], n_top)
        b = chain["basis"]
        ya, yb, _ = oracle.candidate_pool([samples, (ea, eb)], (b[0], b[1]), na, nb)
        _, _, keys = oracle.pt2_scores(H, chain["sa"], chain["sb"], chain["c"], chain["E"], ya, yb)
        if t == 1:
            _, _, bk = oracle.pt2_scores(H, chain["sa"], chain["sb"], chain["c"], chain["E"],
                                         b[0], b[1])
            basis = oracle.basis_update(oracle.BASIS_RESCORE, (b[0], b[1], bk), (ya, yb, keys), k)
        else:
            basis = oracle.basis_update(oracle.BASIS_APPEND, b, (ya, yb, keys), k, b_max)
    sa, sb = oracle.build_subspace(basis[0], basis[1], na, nb)
    if mode == "list":
        la_, lb_ = oracle.sort_list(basis[0], basis[1])
        E, c_list = oracle.ground_state_dense_list(H, la_, lb_)
        c = _embed(sa, sb, la_, lb_, c_list)
        chain.update(la=la_, lb=lb_, c_list=c_list)
    else:
        E, c = oracle.ground_state_dense(H, sa, sb)
    chain.update(basis=tuple(np.asarray(x) for x in basis), sa=sa, sb=sb, c=c, E=E)


@pytest.mark.parametrize("mode", ["list", "product"])
def test_outer_loop_stepwise_parity(mode):
    """Five iterations of Steps 1-3 on n = 10, 2/2 (full product 45 x 45): each step
    of the library's loop is re-done by the oracle from the same inputs (the samples,
    the previous basis, eigenvector and energy) and must give the same candidate set,
    the same basis list, scores within tolerance and the dense-eigh energy."""
    n, na, nb = 10, 2, 2
    h, eri, e_nuc = synth.integrals(n, 6)
    ham = hq.Hamiltonian(h, eri, na, nb, e_nuc)
    H = oracle.Ham(h, eri, e_nuc, na, nb)
    loop = HiNqsLoop(ham, k0=30, k=25, b_max=70, n_top=20, mode=mode)

    def sampler(t):
        return (synth.hf_weighted_samples(n, na, 150, 500 + 2 * t),
                synth.hf_weighted_samples(n, nb, 150, 501 + 2 * t))

    # an independent chain run by the oracle alone: its own keys, basis updates and
    # dense-eigh eigenvectors carried across iterations, compared with the library's
    chain = dict(basis=None, sa=None, sb=None, c=None, E=None)
    for t in range(5):
        rec = loop.step(sampler(t))
        _oracle_chain_step(H, chain, t, sampler(t), na, nb, k0=30, k=25, b_max=70, n_top=20,
                           mode=mode)
        assert np.array_equal(chain["basis"][0], _np_u64(loop.basis[0]))
        assert np.array_equal(chain["basis"][1], _np_u64(loop.basis[1]))
        # the chain's PT2 keys come from its own dense-eigh eigenvector, the library's from
        # a Davidson eigenvector at a 1e-8 residual: they differ by about residual / gap
        assert np.allclose(chain["basis"][2], loop.basis[2].cpu().numpy(), rtol=1e-6, atol=1e-14)
        assert abs(chain["E"] - rec.energy) < 1e-9
        L = loop.last
        samples = tuple(np.asarray(x, dtype=np.uint64) for x in L["samples"])
        pool = tuple(_np_u64(x) for x in L["pool"])
        keys = L["keys"].cpu().numpy()
        basis = tuple(_np_u64(x) for x in loop.basis[:2])
        if t == 0:
            ra, rb, _ = oracle.candidate_pool([samples], (np.zeros(0), np.zeros(0)), na, nb)
            assert np.array_equal(pool[0], ra) and np.array_equal(pool[1], rb)
            ref_keys = oracle.determinant_diag(H, *pool)
            assert np.max(np.abs(keys - ref_keys)) <= 1e-12 * np.max(np.abs(ref_keys))
            ref_basis = oracle.basis_update(oracle.BASIS_COLD_START, ([], [], []),
                                            (pool[0], pool[1], keys), 30)
            assert not rec.warm_start
        else:
            sa_p, sb_p = (_np_u64(x) for x in L["sub_before"].strings())
            c_p = L["c_before"].cpu().numpy()
            E_p = L["energy_before"]
            xa_cl, xb_cl = (_np_u64(x) for x in L["expansion"])
            if mode == "list":
                lxa, lxb = oracle.sort_list(*(_np_u64(x) for x in L["basis_before"][:2]))
                ea, eb = oracle.classical_expansion_list(H, lxa, lxb,
                                                         L["c_list_before"].cpu().numpy(), 20)
            else:
                ea, eb = oracle.classical_expansion(H, sa_p, sb_p, c_p, 20)
            assert np.array_equal(xa_cl, ea) and np.array_equal(xb_cl, eb)
            bb = tuple(_np_u64(x) for x in L["basis_before"][:2])
            ra, rb, _ = oracle.candidate_pool([samples, (ea, eb)], bb, na, nb)
            assert np.array_equal(pool[0], ra) and np.array_equal(pool[1], rb)
            _, rh, rs = oracle.pt2_scores(H, sa_p, sb_p, c_p, E_p, ra, rb)
            ok = np.abs(E_p - rh) > 1e-3
            assert np.allclose(keys[ok], rs[ok], rtol=1e-9, atol=1e-10 * np.max(rs[ok]))
            if t == 1:
                bk = L["basis_keys"].cpu().numpy()
                ref_basis = oracle.basis_update(oracle.BASIS_RESCORE, (bb[0], bb[1], bk),
                                                (pool[0], pool[1], keys), 25)
            else:
                bs = L["basis_before"][2].cpu().numpy()
                ref_basis = oracle.basis_update(oracle.BASIS_APPEND, (bb[0], bb[1], bs),
                                                (pool[0], pool[1], keys), 25, 70)
            assert rec.warm_start
        assert np.array_equal(basis[0], ref_basis[0]) and np.array_equal(basis[1], ref_basis[1])
        assert np.array_equal(loop.basis[2].cpu().numpy(), ref_basis[2])
        sa, sb = oracle.build_subspace(basis[0], basis[1], na, nb)
        if mode == "list":
            E_ref, _ = oracle.ground_state_dense_list(H, *oracle.sort_list(basis[0], basis[1]))
            E_prod, _ = oracle.ground_state_dense(H, sa, sb)
            assert rec.energy >= E_prod - 1e-9  # the list is a subset of the product
        else:
            E_ref, _ = oracle.ground_state_dense(H, sa, sb)
        assert abs(rec.energy - E_ref) < 1e-9, (t, rec.energy, E_ref)
        assert rec.n_basis <= (30 if t == 0 else 70 if t >= 2 else 25)
    # Step 4 on the final basis list, one minibatch of its positions
    pos = loop.basis_positions().cpu().numpy()
    assert np.all(pos >= 0)
    rng = np.random.default_rng(3)
    batch = rng.choice(pos, min(50, len(pos)), replace=False)
    logpi = rng.uniform(-9, -1, len(batch))
    r = loop.teacher(batch, logpi, (1.0, 0.2, 0.05))
    sa, sb = (_np_u64(x) for x in loop.sub.strings())
    ref = oracle.nqs_loss(H, sa, sb, loop.c.cpu().numpy(), loop.energy, batch, logpi,
                          (1.0, 0.2, 0.05), basis=pos)
    assert np.allclose(r["w"].cpu().numpy(), ref["w"], rtol=1e-12, atol=0)
    assert abs(float(r["loss"][0]) - ref["total"]) <= 1e-12 * max(1.0, abs(ref["total"]))
