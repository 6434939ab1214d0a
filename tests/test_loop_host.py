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
