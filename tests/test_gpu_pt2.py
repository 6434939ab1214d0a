"""PT2 scores of candidate determinants (Step 2, Eq. pt2_score) against the oracle.

FP64 on both sides; the coupling sums at most a few thousand products in another
order than the oracle, so |v - v_oracle| <= 1e-11 max|v| and H_xx agrees to 1e-12
relative.  Scores are compared where |E0 - H_xx| is not tiny (relative 1e-9)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

hq = pytest.importorskip("paper_2606_26760_b300")


def _case(n, na, nb, seed, fa_frac=0.5, fb_frac=0.5):
    h, eri, _ = synth.integrals(n, seed)
    rng = np.random.default_rng(seed)
    fa, fb = synth.all_strings(n, na), synth.all_strings(n, nb)
    sa = rng.choice(fa, size=max(1, int(len(fa) * fa_frac)), replace=False)
    sb = rng.choice(fb, size=max(1, int(len(fb) * fb_frac)), replace=False)
    return h, eri, 0.25, sa, sb, fa, fb


def _check(got, ref, tol):
    scale = max(1.0, float(np.max(np.abs(ref))))
    assert np.max(np.abs(got - ref)) <= tol * scale


@pytest.mark.parametrize("n,na,nb,seed", [(8, 3, 3, 41), (10, 3, 4, 42), (6, 2, 0, 43), (12, 4, 4, 44)])
def test_pt2_matches_oracle_full_sector(n, na, nb, seed):
    h, eri, e_nuc, sa, sb, fa, fb = _case(n, na, nb, seed, 0.5, 0.6)
    if n == 12:  # keep the candidate list small: sampled strings
        rng = np.random.default_rng(seed + 1)
        fa = rng.choice(fa, 40, replace=False)
        fb = rng.choice(fb, 30, replace=False)
    ham = hq.Hamiltonian(h, eri, na, nb, e_nuc)
    sub = hq.build_subspace(sa, sb, n, na, nb)
    H = oracle.Ham(h, eri, e_nuc, na, nb)
    osa, osb = oracle.build_subspace(sa, sb, na, nb)
    c = synth.random_vector(len(osa) * len(osb), seed)
    xa = np.repeat(fa, len(fb))
    xb = np.tile(fb, len(fa))
    E0 = -7.5
    v, hxx, s = hq.pt2_score(ham, sub, torch.tensor(c, device="cuda"), E0, xa, xb)
    rv, rh, rs = oracle.pt2_scores(H, osa, osb, c, E0, xa, xb)
    _check(v.cpu().numpy(), rv, 1e-11)
    _check(hxx.cpu().numpy(), rh, 1e-12)
    ok = np.abs(E0 - rh) > 1e-3
    assert np.allclose(s.cpu().numpy()[ok], rs[ok], rtol=1e-9, atol=1e-14)


def test_pt2_external_candidates_precision_workload():
    """2000 x 2000 subspace; 300 candidates built from strings outside it (and some
    mixed inside/outside pairs)."""
    w = synth.workload("precision")
    n, na, nb = w["n_orb"], w["n_alpha"], w["n_beta"]
    ham = hq.Hamiltonian(w["h"], w["eri"], na, nb, w["e_nuc"])
    sub = hq.build_subspace(w["alpha"], w["beta"], n, na, nb)
    H = oracle.Ham(w["h"], w["eri"], w["e_nuc"], na, nb)
    sa, sb = oracle.build_subspace(w["alpha"], w["beta"], na, nb)
    more = synth.hf_weighted_strings(n, na, 2400, 1234)
    out_a = np.array([x for x in more if x not in set(sa.tolist())], dtype=np.uint64)
    out_b = np.array([x for x in synth.hf_weighted_strings(n, nb, 2400, 4321)
                      if x not in set(sb.tolist())], dtype=np.uint64)
    rng = np.random.default_rng(9)
    xa = np.concatenate([rng.choice(out_a, 200), rng.choice(sa, 50), rng.choice(out_a, 50)])
    xb = np.concatenate([rng.choice(out_b, 200), rng.choice(out_b, 50), rng.choice(sb, 50)])
    c = synth.random_vector(len(sa) * len(sb), 5)
    c /= np.linalg.norm(c)
    E0 = -26.8
    v, hxx, s = hq.pt2_score(ham, sub, torch.tensor(c, device="cuda"), E0, xa, xb)
    rv, rh, rs = oracle.pt2_scores(H, sa, sb, c, E0, xa, xb)
    _check(v.cpu().numpy(), rv, 1e-11)
    _check(hxx.cpu().numpy(), rh, 1e-12)
    assert np.allclose(s.cpu().numpy(), rs, rtol=1e-9, atol=1e-16)


def test_pt2_inside_subspace_is_eigen_equation():
    """For x in the subspace and the FP64 Davidson eigenvector, <x|H|Psi0> = E0 c_x
    up to the residual (1e-9)."""
    w = synth.workload("fp64_small")
    ham = hq.Hamiltonian(w["h"], w["eri"], 3, 3, w["e_nuc"])
    sub = hq.build_subspace(w["alpha"], w["beta"], 8, 3, 3)
    la, lb = hq.string_links(ham, sub, 0), hq.string_links(ham, sub, 1)
    r = hq.davidson(ham, sub, la, lb, tol_residual=1e-10)
    ga, gb = sub.strings()
    xa = np.repeat(ga.cpu().numpy().view(np.uint64), sub.Nb)
    xb = np.tile(gb.cpu().numpy().view(np.uint64), sub.Na)
    v, hxx, s = hq.pt2_score(ham, sub, r.c, r.energy, xa, xb)
    assert float((v - r.energy * r.c).abs().max()) < 1e-9
    hd = hq.diag(ham, sub, la, lb)
    assert float((hxx - hd).abs().max()) < 1e-12


def test_pt2_errors():
    w = synth.workload("fp64_small")
    ham = hq.Hamiltonian(w["h"], w["eri"], 3, 3, w["e_nuc"])
    sub = hq.build_subspace(w["alpha"], w["beta"], 8, 3, 3)
    c = torch.ones(sub.N, dtype=torch.float64, device="cuda")
    xa = np.array([0b111, 0b1011, 0b11], dtype=np.uint64)   # last has 2 electrons
    xb = np.array([0b111, 0b111, 0b111], dtype=np.uint64)
    with pytest.raises(hq.HinqsError) as e:
        hq.pt2_score(ham, sub, c, -1.0, xa, xb)
    assert e.value.code == hq.ERR_PARTICLE_NUMBER
    v, hxx, s = hq.pt2_score(ham, sub, c, -1.0, np.zeros(0, np.uint64), np.zeros(0, np.uint64))
    assert v.numel() == 0


def test_pt2_score_at_a_zero_denominator():
    """Eq. pt2_score has no regulariser: with E0 equal to a candidate's H_xx the score is
    v^2 / 0, +inf when v != 0 and NaN when v = 0 (c = 0), on both sides, each side
    taking E0 from its own H_xx so that the denominator is exactly zero."""
    h, eri, e_nuc, sa, sb, fa, fb = _case(8, 3, 3, 51, 0.5, 0.5)
    ham = hq.Hamiltonian(h, eri, 3, 3, e_nuc)
    sub = hq.build_subspace(sa, sb, 8, 3, 3)
    H = oracle.Ham(h, eri, e_nuc, 3, 3)
    osa, osb = oracle.build_subspace(sa, sb, 3, 3)
    c = synth.random_vector(len(osa) * len(osb), 51)
    xa = np.repeat(fa[:6], 6)
    xb = np.tile(fb[:6], 6)
    v, hxx, _ = hq.pt2_score(ham, sub, torch.tensor(c, device="cuda"), -5.0, xa, xb)
    rv, rh, _ = oracle.pt2_scores(H, osa, osb, c, -5.0, xa, xb)
    k = int(np.argmax(np.abs(rv)))
    assert abs(rv[k]) > 1e-6 and abs(v.cpu().numpy()[k]) > 1e-6
    e0_gpu = float(hxx.cpu().numpy()[k])
    _, _, s = hq.pt2_score(ham, sub, torch.tensor(c, device="cuda"), e0_gpu, xa, xb)
    with np.errstate(divide="ignore", invalid="ignore"):
        _, _, rs = oracle.pt2_scores(H, osa, osb, c, float(rh[k]), xa, xb)
    assert np.isposinf(s.cpu().numpy()[k]) and np.isposinf(rs[k])
    zero = np.zeros_like(c)
    _, _, s0 = hq.pt2_score(ham, sub, torch.tensor(zero, device="cuda"), e0_gpu, xa, xb)
    with np.errstate(divide="ignore", invalid="ignore"):
        _, _, rs0 = oracle.pt2_scores(H, osa, osb, zero, float(rh[k]), xa, xb)
    assert np.isnan(s0.cpu().numpy()[k]) and np.isnan(rs0[k])
    # every other candidate: the finite quotient, equal on both sides
    ok = np.abs(float(rh[k]) - rh) > 1e-3
    assert np.all(s0.cpu().numpy()[ok] == 0.0) and np.all(rs0[ok] == 0.0)
