"""Checkpoint and resume of the outer loop on the device: a loop saved after two
iterations and loaded again (subspace and links rebuilt, eigenvector restored) takes
its third step exactly like the loop that never stopped: the same candidate set, the
same basis list and the same energy to 1e-10 Ha."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

hq = pytest.importorskip("paper_2606_26760_b300")
from paper_2606_26760_b300.loop import HiNqsLoop  # noqa: E402


def test_resume_continues_like_the_uninterrupted_loop(tmp_path):
    n, na, nb = 10, 2, 2
    h, eri, e_nuc = synth.integrals(n, 6)
    ham = hq.Hamiltonian(h, eri, na, nb, e_nuc)

    def sampler(t):
        return (synth.hf_weighted_samples(n, na, 150, 700 + 2 * t),
                synth.hf_weighted_samples(n, nb, 150, 701 + 2 * t))

    live = HiNqsLoop(ham, k0=30, k=25, b_max=70, n_top=20)
    for t in range(2):
        live.step(sampler(t))
    path = str(tmp_path / "loop.npz")
    live.save(path)
    resumed = HiNqsLoop.load(path, ham)
    assert resumed.t == 2 and resumed.energies == live.energies
    r_live = live.step(sampler(2))
    r_back = resumed.step(sampler(2))
    for key in ("pool",):
        for a, b in zip(live.last[key], resumed.last[key]):
            assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
    for a, b in zip(live.basis[:2], resumed.basis[:2]):
        assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
    assert r_back.warm_start and r_back.n_basis == r_live.n_basis
    assert abs(r_back.energy - r_live.energy) < 1e-10
