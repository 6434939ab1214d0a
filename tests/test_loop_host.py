"""Host logic of the outer loop (no GPU): the Step 5 stopping rule of HiNqsLoop agrees
with the oracle's statement of it on hand-made energy sequences."""
import numpy as np

import oracle
from paper_2606_26760_b300.loop import HiNqsLoop


def test_stopping_rule_matches_oracle():
    rng = np.random.default_rng(0)
    seqs = [[], [-1.0], [-1.0] * 5, [-1.0] * 6, [-1.0, -1.1] + [-1.2] * 5,
            [-1.0, -1.1] + [-1.2] * 6, list(np.linspace(0.0, -1.0, 50)),
            list(np.linspace(0.0, -1.0, 49)),
            [-2.0 - 1e-10 * k for k in range(8)], [-2.0 - 2e-9 * k for k in range(8)]]
    seqs += [list(np.cumsum(rng.choice([0.0, 1e-10, 1e-8], 20))) for _ in range(20)]
    for seq in seqs:
        loop = HiNqsLoop(ham=None, k0=1, k=1, b_max=0)
        loop.energies = list(seq)
        assert loop.converged() == oracle.converged(seq), seq


def test_checkpoint_round_trip_host_state(tmp_path):
    """save() then load(rebuild=False) restores the basis list, its keys, the energies,
    the iteration count, the budgets and the eigenvector exactly (host arrays only;
    the device rebuild is a composition of build_subspace and string_links)."""
    import torch
    from paper_2606_26760_b300.loop import IterationRecord

    class FakeSub:
        def strings(self):
            return torch.tensor([3, 5, 6]), torch.tensor([3, 9])

    loop = HiNqsLoop(ham=None, k0=30, k=25, b_max=70, n_top=20, patience=4)
    loop.t = 3
    loop.basis = (torch.tensor([3, 5, 6]), torch.tensor([3, 3, 9]),
                  torch.tensor([0.5, 0.25, 0.125], dtype=torch.float64))
    loop.sub = FakeSub()
    loop.c = torch.tensor(np.linspace(-1, 1, 6))
    loop.energy = -1.25
    loop.energies = [-1.0, -1.2, -1.25]
    loop.history = [IterationRecord(t, 10 + t, 0, 3, 3, 2, e, 1e-9, 0, t > 0)
                    for t, e in enumerate(loop.energies)]
    p = str(tmp_path / "ckpt.npz")
    loop.save(p)
    back = HiNqsLoop.load(p, ham=None, rebuild=False)
    assert back.t == 3 and (back.k0, back.k, back.b_max, back.n_top, back.patience) == (30, 25, 70, 20, 4)
    assert back.energies == loop.energies and back.energy == -1.25
    for a, b in zip(back.basis, loop.basis):
        assert torch.equal(a, b)
    assert torch.equal(back.c, loop.c)
    assert back.history == loop.history
    jl = tmp_path / "hist.jsonl"
    back.write_history_jsonl(str(jl))
    lines = jl.read_text().splitlines()
    assert len(lines) == 3 and '"energy": -1.2' in lines[1]
