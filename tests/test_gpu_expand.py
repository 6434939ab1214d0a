"""Classical expansion (Step 1', Eq. classical_expansion) and the selection of the
largest amplitudes, against the oracle.  Both are integer/set results: the chosen
indices and the candidate determinants must agree exactly (same order)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

hq = pytest.importorskip("paper_2606_26760_b300")


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("k", [1, 7, 64, 1000, 3136, 5000])
def test_top_amplitudes_exact_with_ties(k):
    w = synth.workload("fp64_small")
    sub = hq.build_subspace(w["alpha"], w["beta"], 8, 3, 3)
    rng = np.random.default_rng(k)
    c = rng.standard_normal(sub.N)
    c[rng.choice(sub.N, 300, replace=False)] = 0.0          # ties at zero
    c[rng.choice(sub.N, 50, replace=False)] = 0.125         # ties at a value
    c[rng.choice(sub.N, 50, replace=False)] = -0.125        # equal magnitude, other sign
    got = hq.top_amplitudes(sub, torch.tensor(c, device="cuda"), k).cpu().numpy()
    assert np.array_equal(got, oracle.top_amplitudes(c, min(k, sub.N)))


def test_top_amplitudes_full_size():
    w = synth.workload("precision")
    sub = hq.build_subspace(w["alpha"], w["beta"], 16, 5, 5)
    c = synth.random_vector(sub.N, 17)
    got = hq.top_amplitudes(sub, torch.tensor(c, device="cuda"), 1000).cpu().numpy()
    assert np.array_equal(got, oracle.top_amplitudes(c, 1000))


def _expansion_case(n, na, nb, seed, frac_a, frac_b):
    h, eri, _ = synth.integrals(n, seed)
    rng = np.random.default_rng(seed)
    fa, fb = synth.all_strings(n, na), synth.all_strings(n, nb)
    sa = rng.choice(fa, max(1, int(len(fa) * frac_a)), replace=False)
    sb = rng.choice(fb, max(1, int(len(fb) * frac_b)), replace=False)
    return h, eri, sa, sb


@pytest.mark.parametrize("n,na,nb,seed,n_top", [(8, 3, 3, 71, 10), (10, 3, 4, 72, 6),
                                                (6, 2, 0, 73, 4), (12, 4, 4, 74, 3),
                                                (8, 3, 3, 75, 100000)])
def test_classical_expansion_matches_oracle(n, na, nb, seed, n_top):
    h, eri, sa, sb = _expansion_case(n, na, nb, seed, 0.3, 0.4)
    ham = hq.Hamiltonian(h, eri, na, nb, 0.0)
    sub = hq.build_subspace(sa, sb, n, na, nb)
    H = oracle.Ham(h, eri, 0.0, na, nb)
    osa, osb = oracle.build_subspace(sa, sb, na, nb)
    c = synth.random_vector(len(osa) * len(osb), seed)
    xa, xb = hq.classical_expansion(ham, sub, torch.tensor(c, device="cuda"), n_top)
    ra, rb = oracle.classical_expansion(H, osa, osb, c, min(n_top, len(c)))
    assert np.array_equal(_u64(xa), ra) and np.array_equal(_u64(xb), rb)


def test_classical_expansion_precision_workload():
    """2000 x 2000 subspace, the 200 largest amplitudes of a random vector."""
    w = synth.workload("precision")
    ham = hq.Hamiltonian(w["h"], w["eri"], 5, 5, 0.0)
    sub = hq.build_subspace(w["alpha"], w["beta"], 16, 5, 5)
    H = oracle.Ham(w["h"], w["eri"], 0.0, 5, 5)
    sa, sb = oracle.build_subspace(w["alpha"], w["beta"], 5, 5)
    c = synth.random_vector(sub.N, 19)
    xa, xb = hq.classical_expansion(ham, sub, torch.tensor(c, device="cuda"), 200)
    ra, rb = oracle.classical_expansion(H, sa, sb, c, 200)
    assert len(ra) > 0
    assert np.array_equal(_u64(xa), ra) and np.array_equal(_u64(xb), rb)


def test_classical_expansion_degenerate_and_errors():
    w = synth.workload("fp64_small")
    ham = hq.Hamiltonian(w["h"], w["eri"], 3, 3, 0.0)
    sub = hq.build_subspace(w["alpha"], w["beta"], 8, 3, 3)
    c = torch.ones(sub.N, dtype=torch.float64, device="cuda")
    # the full sector is the subspace: nothing lies outside it
    xa, xb = hq.classical_expansion(ham, sub, c, 50)
    assert xa.numel() == 0 and xb.numel() == 0
    xa, xb = hq.classical_expansion(ham, sub, c, 0)
    assert xa.numel() == 0
    with pytest.raises(hq.HinqsError) as e:
        hq.classical_expansion(ham, sub, c, -1)
    assert e.value.code == hq.ERR_ARG


@pytest.mark.parametrize("n,na,nb,seed,n_top", [(33, 1, 1, 81, 4), (40, 2, 2, 82, 6),
                                                (36, 3, 2, 83, 3), (64, 1, 2, 84, 5),
                                                (32, 2, 2, 85, 5)])
def test_classical_expansion_wide_orbitals_matches_oracle(n, na, nb, seed, n_top):
    """From 32 orbitals on the candidates are keyed by the ranks of their distinct
    strings: the same set and order as the oracle's (orbitals up to 64 use the upper
    half of the 64-bit word)."""
    h, eri, _ = synth.integrals(n, seed)
    rng = np.random.default_rng(seed)
    fa, fb = synth.hf_weighted_samples(n, na, 60, seed), synth.hf_weighted_samples(n, nb, 50, seed + 1)
    sa, sb = np.unique(fa), np.unique(fb)
    ham = hq.Hamiltonian(h, eri, na, nb, 0.0)
    sub = hq.build_subspace(sa, sb, n, na, nb)
    H = oracle.Ham(h, eri, 0.0, na, nb)
    osa, osb = oracle.build_subspace(sa, sb, na, nb)
    c = rng.standard_normal(len(osa) * len(osb))
    xa, xb = hq.classical_expansion(ham, sub, torch.tensor(c, device="cuda"), n_top)
    ra, rb = oracle.classical_expansion(H, osa, osb, c, n_top)
    assert len(ra) > 0
    assert np.array_equal(_u64(xa), ra) and np.array_equal(_u64(xb), rb)
