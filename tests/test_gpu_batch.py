"""Batched multi-geometry solve and the sigma tile autotuner, against the oracle.

A bond scan is a set of independent ground-state problems (one per geometry), so
the batched solve must give, geometry by geometry, what the single solve gives:
energies within 1e-9 Ha of the oracle's dense ground state for the FP64 solver,
1e-6 Ha for the mixed one, eigenvectors equal up to sign.  The autotuner changes
only the tiling of the sigma product, so sigma stays within the single-call
tolerances of the parity tests (FP64 1e-11, FP32 2e-5, BF16 tensor-core 2e-2,
BF16x3 2e-4, relative to the largest |sigma|)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

hq = pytest.importorskip("paper_2606_26760_b300")


def _problem(w):
    ham = hq.Hamiltonian(w["h"], w["eri"], w["n_alpha"], w["n_beta"], w["e_nuc"])
    sub = hq.build_subspace(w["alpha"], w["beta"], w["n_orb"], w["n_alpha"], w["n_beta"])
    return ham, sub, hq.string_links(ham, sub, 0), hq.string_links(ham, sub, 1)


def _oracle_gs(w):
    H = oracle.Ham(w["h"], w["eri"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    sa, sb = oracle.build_subspace(w["alpha"], w["beta"], w["n_alpha"], w["n_beta"])
    E, c = oracle.ground_state_dense(H, sa, sb)
    return H, sa, sb, E, c


@pytest.fixture(scope="module")
def small_scan():
    """Six geometries of a 10-orbital, (3,3) scan with uneven subspaces (<= 55 x 55)."""
    ws = synth.bond_scan_workload(n_geom=6, n_orb=10, n_e=3, lo=12, hi=55)
    return ws, [_oracle_gs(w) for w in ws], [_problem(w) for w in ws]


def test_batch_fp64_matches_oracle(small_scan):
    ws, gs, probs = small_scan
    res = hq.davidson_batch(probs, n_streams=3, tol_residual=1e-9)
    assert len(res) == len(ws)
    for r, (_, _, _, E, c) in zip(res, gs):
        assert r.status == hq.OK
        assert abs(r.energy - E) < 1e-9
        x = r.c.cpu().numpy()
        assert abs(abs(np.dot(x, c)) - 1.0) < 1e-8
        assert r.residual < 1e-8


def test_batch_mixed_autotuned_matches_oracle(small_scan):
    ws, gs, probs = small_scan
    for inner in (hq.PREC_FP32, hq.PREC_FP32_BF16AB, hq.PREC_FP32_BF16X3AB):
        res = hq.davidson_batch(probs, precision=hq.DAVIDSON_MIXED, inner_precision=inner,
                                tol_residual=1e-7, tol_energy=1e-9, max_iter=600, n_streams=4,
                                autotune=True)
        for r, (_, _, _, E, _) in zip(res, gs):
            assert r.status == hq.OK
            assert abs(r.energy - E) < 1e-6


def test_batch_equals_single_solves(small_scan):
    """Same options, same answers: the queue and the streams change nothing."""
    ws, gs, probs = small_scan
    guesses = [None] * len(probs)
    guesses[2] = torch.tensor(gs[2][4], dtype=torch.float64, device="cuda")
    batch = hq.davidson_batch(probs, guesses=guesses, n_streams=2)
    for p, g, b in zip(probs, guesses, batch):
        s = hq.davidson(*p, guess=g)
        assert abs(s.energy - b.energy) < 1e-10
        assert abs(abs(torch.dot(s.c, b.c).item()) - 1.0) < 1e-9
    # the warm-started geometry is already converged at its first check
    assert batch[2].iterations <= 2


def test_batch_one_stream_and_more_streams_than_problems(small_scan):
    ws, gs, probs = small_scan
    for ns in (1, 16):
        res = hq.davidson_batch(probs[:3], n_streams=ns)
        for r, (_, _, _, E, _) in zip(res, gs[:3]):
            assert abs(r.energy - E) < 1e-9


def test_batch_not_converged_and_empty(small_scan):
    ws, gs, probs = small_scan
    assert hq.davidson_batch([]) == []
    res = hq.davidson_batch(probs, max_iter=2)
    assert any(r.status == hq.NOT_CONVERGED for r in res)
    with pytest.raises(ValueError):
        hq.davidson_batch(probs[:1], guesses=[torch.zeros(3, dtype=torch.float64, device="cuda")])


def test_batch_follows_caller_stream(small_scan):
    """Work queued on the caller's stream before the call (the guess) is seen by
    the worker streams, and the caller's stream sees the eigenvectors after it."""
    ws, gs, probs = small_scan
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = torch.zeros(probs[0][1].N, dtype=torch.float64, device="cuda")
        torch.cuda._sleep(20_000_000)
        g.copy_(torch.tensor(gs[0][4], dtype=torch.float64).to("cuda", non_blocking=True))
        res = hq.davidson_batch(probs[:1], guesses=[g])
        norm = torch.linalg.norm(res[0].c)
    s.synchronize()
    assert abs(res[0].energy - gs[0][3]) < 1e-9
    assert res[0].iterations <= 2
    assert abs(norm.item() - 1.0) < 1e-12


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-5), (2, 2e-2), (3, 2e-4)])
def test_autotune_keeps_sigma_parity(prec, tol):
    h, eri, _ = synth.integrals(10, 101)
    rng = np.random.default_rng(5)
    a = rng.choice(synth.all_strings(10, 3), size=41, replace=False)
    b = rng.choice(synth.all_strings(10, 4), size=73, replace=False)
    w = dict(h=h, eri=eri, e_nuc=0.37, alpha=a, beta=b, n_orb=10, n_alpha=3, n_beta=4)
    ham, sub, la, lb = _problem(w)
    ms = hq.autotune(ham, sub, la, lb, prec)
    assert ms > 0.0
    H = oracle.Ham(h, eri, 0.37, 3, 4)
    sa, sb = oracle.build_subspace(a, b, 3, 4)
    c = synth.random_vector(len(sa) * len(sb), 9)
    ref = oracle.sigma(H, sa, sb, c)
    dt = torch.float64 if prec == 0 else torch.float32
    cd = torch.tensor(c, dtype=dt, device="cuda")
    got = hq.sigma(ham, sub, la, lb, cd, precision=prec).double().cpu().numpy()
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
    # a second call on the same problem class returns the cached choice
    assert hq.autotune(ham, sub, la, lb, prec) == ms


def test_autotune_argument_errors():
    w = synth.workload("fp64_small")
    ham, sub, la, lb = _problem(w)
    with pytest.raises(hq.HinqsError) as e:
        hq.autotune(ham, sub, la, lb, 7)
    assert e.value.code == hq.ERR_ARG
    with pytest.raises(hq.HinqsError) as e:
        hq.autotune(ham, sub, lb, la, 0)
    assert e.value.code == hq.ERR_ARG


@pytest.mark.slow
def test_bond_scan_mixed_batch_vs_fp64_batch():
    """24 geometries of the 16-orbital (5,5) scan at a reduced string count
    (50..400 per species): the mixed BF16 batch agrees with the FP64 batch."""
    ws = synth.bond_scan_workload(n_geom=24, lo=50, hi=400)
    probs = [_problem(w) for w in ws]
    ref = hq.davidson_batch(probs, tol_residual=1e-8, max_iter=400)
    mix = hq.davidson_batch(probs, precision=hq.DAVIDSON_MIXED, inner_precision=hq.PREC_FP32_BF16AB,
                            tol_residual=1e-6, tol_energy=1e-8, max_iter=600, autotune=True)
    for r, m in zip(ref, mix):
        assert r.status == hq.OK and m.status == hq.OK
        assert abs(r.energy - m.energy) < 1e-6
        assert abs(abs(torch.dot(r.c, m.c).item()) - 1.0) < 1e-5


# ------------------------------------------------ lockstep batch (one launch per stage)


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-6), (2, 1e-5), (3, 1e-6), (4, 1e-5),
                                      (5, 1e-12)])
def test_sigma_batch_equals_single_products(small_scan, prec, tol):
    """The batched kernels (flattened row products and transposes over every geometry,
    the tensor-core term over a device work queue) against one product per geometry:
    the same arithmetic up to the order of the reductions; the scan's string counts
    are mostly not multiples of 4 (the unaligned row-product path)."""
    ws, gs, probs = small_scan
    dt = torch.float64 if prec in (0, 5) else torch.float32
    cs = [torch.tensor(synth.random_vector(p[1].N, 30 + i), dtype=dt, device="cuda")
          for i, p in enumerate(probs)]
    assert any(p[1].Nb % 4 for p in probs) and any(p[1].Na % 4 for p in probs)
    got = hq.sigma_batch(probs, cs, precision=prec)
    for p, c, g in zip(probs, cs, got):
        ref = hq.sigma(*p, c, precision=prec)
        assert float(torch.max(torch.abs(g - ref))) <= tol * float(torch.max(torch.abs(ref)))


def test_batch_lockstep_matches_oracle(small_scan):
    ws, gs, probs = small_scan
    res = hq.davidson_batch(probs, n_streams=0, tol_residual=1e-9)
    for r, (_, _, _, E, c) in zip(res, gs):
        assert r.status == hq.OK and abs(r.energy - E) < 1e-9
        assert abs(abs(np.dot(r.c.cpu().numpy(), c)) - 1.0) < 1e-8
    for inner in (hq.PREC_FP32, hq.PREC_FP32_BF16AB, hq.PREC_FP32_BF16X3AB, hq.PREC_FP32_BF16C):
        res = hq.davidson_batch(probs, precision=hq.DAVIDSON_MIXED, inner_precision=inner,
                                tol_residual=1e-7, tol_energy=1e-9, max_iter=600, n_streams=0)
        for r, (_, _, _, E, _) in zip(res, gs):
            assert r.status == hq.OK and abs(r.energy - E) < 1e-6


def test_batch_lockstep_equals_worker_form(small_scan):
    """Lockstep rounds change the launches, not the solves: the same FP64 answers as the
    worker form, including a warm-started geometry that leaves the rounds at once and a
    geometry that hits max_iter."""
    ws, gs, probs = small_scan
    guesses = [None] * len(probs)
    guesses[1] = torch.tensor(gs[1][4], dtype=torch.float64, device="cuda")
    a = hq.davidson_batch(probs, guesses=guesses, n_streams=0)
    b = hq.davidson_batch(probs, guesses=guesses, n_streams=3)
    for x, y in zip(a, b):
        assert abs(x.energy - y.energy) < 1e-10 and x.status == y.status
    assert a[1].iterations <= 2
    short = hq.davidson_batch(probs, max_iter=3, n_streams=0)
    assert any(r.status == hq.NOT_CONVERGED for r in short)


def test_batch_lockstep_with_large_geometry(small_scan):
    """A geometry of 2^20 determinants or more runs on a worker stream beside the
    lockstep rounds of the small ones: the energies equal those of single solves."""
    ws, gs, probs = small_scan
    big = synth.bond_scan_workload(n_geom=1)[0]
    pb = _problem(big)
    assert pb[1].N >= 1 << 20
    opts = dict(precision=hq.DAVIDSON_MIXED, inner_precision=hq.PREC_FP32_BF16AB,
                tol_residual=1e-6, tol_energy=1e-9, max_iter=600)
    res = hq.davidson_batch(probs[:3] + [pb], n_streams=0, **opts)
    single = [hq.davidson(*p, **opts) for p in probs[:3] + [pb]]
    for r, s1 in zip(res, single):
        assert r.status == hq.OK and s1.status == hq.OK
        assert abs(r.energy - s1.energy) < 1e-8
    for r, (_, _, _, E, _) in zip(res[:3], gs[:3]):
        assert abs(r.energy - E) < 1e-6
