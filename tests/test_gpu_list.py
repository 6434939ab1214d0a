"""Step 3 over the basis list itself ([H_B]_ij = <x_i|H|x_j> for the listed
determinants) on the GPU against the oracle's statement of it.

Lists are random subsets of a product (so they are not products themselves), drawn
from small sectors, ragged sizes, orbitals above bit 32, an empty beta sector, and
the 4.0e6-determinant precision workload.  Tolerances: FP64 products and energies as
the product-mode parity tests (1e-11 relative per element, 1e-9 Ha), FP32 products
2e-5 relative, the mixed solver 1e-6 Ha; positions, sets and orders bit-exact."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

hq = pytest.importorskip("paper_2606_26760_b300")


def _np_u64(t):
    return t.cpu().numpy().view(np.uint64) if isinstance(t, torch.Tensor) else np.asarray(t, np.uint64)


def _case(n, na, nb, n_sa, n_sb, frac, seed):
    """A product of sampled strings and a random fraction of its determinants."""
    h, eri, _ = synth.integrals(n, seed)
    rng = np.random.default_rng(seed)
    fa, fb = synth.all_strings(n, na), synth.all_strings(n, nb)
    sa = np.sort(rng.choice(fa, min(n_sa, len(fa)), replace=False))
    sb = np.sort(rng.choice(fb, min(n_sb, len(fb)), replace=False))
    xa = np.repeat(sa, len(sb))
    xb = np.tile(sb, len(sa))
    keep = rng.random(len(xa)) < frac
    keep[rng.integers(len(xa))] = True
    xa, xb = xa[keep], xb[keep]
    # the product is that of the list's own strings (as Step 3 builds it)
    perm = rng.permutation(len(xa))
    return h, eri, 0.35, xa[perm], xb[perm]


CASES = [  # n, na, nb, alpha strings, beta strings, fraction, seed
    (8, 3, 3, 56, 56, 0.3, 81),
    (10, 3, 4, 41, 73, 0.15, 82),
    (12, 4, 4, 60, 50, 0.2, 83),
    (6, 2, 0, 15, 1, 0.6, 84),
    (40, 2, 2, 30, 25, 0.4, 85),
    (7, 1, 3, 7, 35, 0.5, 86),
]


def _setup(n, na, nb, xa, xb, h, eri, e_nuc):
    ham = hq.Hamiltonian(h, eri, na, nb, e_nuc)
    sub = hq.build_subspace(xa, xb, n, na, nb)
    la, lb = hq.string_links(ham, sub, 0), hq.string_links(ham, sub, 1)
    lst = hq.detlist(sub, xa, xb)
    H = oracle.Ham(h, eri, e_nuc, na, nb)
    oxa, oxb = oracle.sort_list(xa, xb)
    return ham, sub, la, lb, lst, H, oxa, oxb


@pytest.mark.parametrize("n,na,nb,n_sa,n_sb,frac,seed", CASES)
def test_list_positions_and_sigma_match_oracle(n, na, nb, n_sa, n_sb, frac, seed):
    h, eri, e_nuc, xa, xb = _case(n, na, nb, n_sa, n_sb, frac, seed)
    ham, sub, la, lb, lst, H, oxa, oxb = _setup(n, na, nb, xa, xb, h, eri, e_nuc)
    assert lst.m == len(oxa)
    sa, sb = (_np_u64(x) for x in sub.strings())
    ref_pos = oracle.lookup(sa, sb, oxa, oxb)
    assert np.array_equal(lst.positions().cpu().numpy(), ref_pos)
    c = synth.random_vector(lst.m, seed)
    got = hq.sigma_list(ham, sub, la, lb, lst, torch.tensor(c, device="cuda")).cpu().numpy()
    ref = oracle.sigma_list(H, oxa, oxb, c)
    assert np.max(np.abs(got - ref)) <= 1e-11 * max(1.0, np.max(np.abs(ref)))
    got32 = hq.sigma_list(ham, sub, la, lb, lst,
                          torch.tensor(c, device="cuda", dtype=torch.float32)).cpu().numpy()
    assert np.max(np.abs(got32 - ref)) <= 2e-5 * max(1.0, np.max(np.abs(ref)))
    hd = hq.diag_list(ham, sub, la, lb, lst).cpu().numpy()
    ref_hd = oracle.determinant_diag(H, oxa, oxb)
    assert np.max(np.abs(hd - ref_hd)) <= 1e-12 * max(1.0, np.max(np.abs(ref_hd)))
    # no atomics: the same product bit for bit on a second call
    again = hq.sigma_list(ham, sub, la, lb, lst, torch.tensor(c, device="cuda")).cpu().numpy()
    assert np.array_equal(got, again)


def test_list_of_the_whole_product_is_the_product_sigma():
    w = synth.workload("fp64_small")
    n, na, nb = w["n_orb"], w["n_alpha"], w["n_beta"]
    ham = hq.Hamiltonian(w["h"], w["eri"], na, nb, w["e_nuc"])
    sub = hq.build_subspace(w["alpha"], w["beta"], n, na, nb)
    la, lb = hq.string_links(ham, sub, 0), hq.string_links(ham, sub, 1)
    sa, sb = (_np_u64(x) for x in sub.strings())
    lst = hq.detlist(sub, np.repeat(sa, len(sb))[::-1].copy(), np.tile(sb, len(sa))[::-1].copy())
    assert lst.m == sub.N and np.array_equal(lst.positions().cpu().numpy(), np.arange(sub.N))
    c = torch.tensor(synth.random_vector(sub.N, 4), device="cuda")
    a = hq.sigma_list(ham, sub, la, lb, lst, c)
    b = hq.sigma(ham, sub, la, lb, c)
    assert torch.max(torch.abs(a - b)).item() <= 1e-12 * torch.max(torch.abs(b)).item()


def test_list_create_errors_and_duplicates():
    n, na, nb = 8, 3, 3
    fa, fb = synth.all_strings(n, na), synth.all_strings(n, nb)
    sub = hq.build_subspace(fa[:10], fb[:10], n, na, nb)
    xa = np.array([fa[3], fa[1], fa[3], fa[1]], dtype=np.uint64)
    xb = np.array([fb[2], fb[0], fb[2], fb[9]], dtype=np.uint64)
    lst = hq.detlist(sub, xa, xb)
    sa, sb = (_np_u64(x) for x in sub.strings())
    ref = sorted(set(oracle.lookup(sa, sb, xa, xb).tolist()))
    assert lst.m == 3 and min(ref) >= 0 and lst.positions().cpu().tolist() == ref
    with pytest.raises(hq.HinqsError) as e:
        hq.detlist(sub, np.array([fa[20]], dtype=np.uint64), np.array([fb[0]], dtype=np.uint64))
    assert e.value.code == hq.ERR_ARG
    empty = hq.detlist(sub, np.zeros(0, np.uint64), np.zeros(0, np.uint64))
    assert empty.m == 0
    ham = hq.Hamiltonian(*synth.integrals(n, 1)[:2], na, nb, 0.0)
    la, lb = hq.string_links(ham, sub, 0), hq.string_links(ham, sub, 1)
    with pytest.raises(hq.HinqsError) as e:
        hq.davidson_list(ham, sub, la, lb, empty)
    assert e.value.code == hq.ERR_EMPTY


@pytest.mark.parametrize("n,na,nb,n_sa,n_sb,frac,seed", [CASES[0], CASES[1], CASES[4], CASES[5]])
def test_davidson_list_vs_dense(n, na, nb, n_sa, n_sb, frac, seed):
    h, eri, e_nuc, xa, xb = _case(n, na, nb, n_sa, n_sb, frac, seed)
    ham, sub, la, lb, lst, H, oxa, oxb = _setup(n, na, nb, xa, xb, h, eri, e_nuc)
    E_ref, c_ref = oracle.ground_state_dense_list(H, oxa, oxb)
    for prec, tol in ((hq.DAVIDSON_FP64, 1e-9), (hq.DAVIDSON_MIXED, 1e-6)):
        r = hq.davidson_list(ham, sub, la, lb, lst, precision=prec, tol_residual=1e-8,
                             inner_precision=hq.PREC_FP32_BF16AB)
        assert r.status == hq.OK
        assert abs(r.energy - E_ref) < tol, (prec, r.energy, E_ref)
    c = r.c.cpu().numpy()
    assert abs(abs(c @ c_ref) - 1.0) < 1e-8
    # the list energy lies above the energy of the product of its strings (Step 3 is
    # variational in B), and the list state's RDMs reproduce it through the product
    E_prod, _ = oracle.ground_state_dense(H, *oracle.build_subspace(oxa, oxb, na, nb))
    assert r.energy >= E_prod - 1e-9
    c_prod = hq.detlist_scatter(lst, r.c)
    assert torch.equal(hq.detlist_gather(lst, c_prod), r.c)
    g1, g2 = hq.rdm(sub, la, lb, c_prod)
    e_id = float((ham.h * g1).sum() + 0.5 * (ham.eri * g2).sum()) + e_nuc
    assert abs(e_id - E_ref) < 1e-8
    sa, sb = (_np_u64(x) for x in sub.strings())
    r1, r2 = oracle.rdm(n, sa, sb, c_prod.cpu().numpy())
    assert np.max(np.abs(g1.cpu().numpy() - r1)) < 1e-11
    assert np.max(np.abs(g2.cpu().numpy() - r2)) < 1e-11


def test_list_on_the_precision_workload_sampled_rows():
    """30,000 random determinants of the 2000 x 2000 product: every list position, and
    256 sampled rows of the FP64 list product against the oracle's list sigma."""
    w = synth.workload("precision")
    n, na, nb = w["n_orb"], w["n_alpha"], w["n_beta"]
    rng = np.random.default_rng(90)
    sa, sb = oracle.build_subspace(w["alpha"], w["beta"], na, nb)
    I = np.sort(rng.choice(len(sa) * len(sb), 30000, replace=False))
    xa, xb = sa[I // len(sb)], sb[I % len(sb)]
    ham = hq.Hamiltonian(w["h"], w["eri"], na, nb, w["e_nuc"])
    sub = hq.build_subspace(xa, xb, n, na, nb)
    la, lb = hq.string_links(ham, sub, 0), hq.string_links(ham, sub, 1)
    lst = hq.detlist(sub, xa, xb)
    H = oracle.Ham(w["h"], w["eri"], w["e_nuc"], na, nb)
    assert lst.m == 30000
    c = synth.random_vector(lst.m, 91)
    got = hq.sigma_list(ham, sub, la, lb, lst, torch.tensor(c, device="cuda")).cpu().numpy()
    rows = np.sort(rng.choice(lst.m, 256, replace=False))
    ref = oracle.sigma_list(H, xa, xb, c, rows=rows)
    assert np.max(np.abs(got[rows] - ref)) <= 1e-11 * max(1.0, np.max(np.abs(ref)))
    r64 = hq.davidson_list(ham, sub, la, lb, lst, tol_residual=1e-9, max_iter=400)
    rmx = hq.davidson_list(ham, sub, la, lb, lst, precision=hq.DAVIDSON_MIXED, tol_residual=1e-7,
                           max_iter=600)
    assert r64.status == hq.OK and rmx.status == hq.OK
    assert abs(r64.energy - rmx.energy) < 1e-6
    # residual certificate through the oracle on sampled rows: (H c - E c)_i
    cc = r64.c.cpu().numpy()
    res = oracle.sigma_list(H, xa, xb, cc, rows=rows) - r64.energy * cc[rows]
    assert np.max(np.abs(res)) < 1e-8


def test_classical_expansion_list_matches_oracle():
    h, eri, e_nuc, xa, xb = _case(8, 3, 3, 30, 30, 0.2, 87)
    ham, sub, la, lb, lst, H, oxa, oxb = _setup(8, 3, 3, xa, xb, h, eri, e_nuc)
    c = synth.random_vector(lst.m, 87)
    ya, yb = hq.classical_expansion_list(ham, sub, lst, torch.tensor(c, device="cuda"), 12)
    ra, rb = oracle.classical_expansion_list(H, oxa, oxb, c, 12)
    assert np.array_equal(_np_u64(ya), ra) and np.array_equal(_np_u64(yb), rb)
    # members of the product outside the list are candidates in list mode
    sa, sb = (_np_u64(x) for x in sub.strings())
    inside = oracle.lookup(sa, sb, ra, rb) >= 0
    assert inside.any()
