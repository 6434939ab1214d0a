"""Geometry sharding across ranks: the assignment logic, and a world-size-2 gloo run
on CPU where each rank solves its share with the oracle (tiny geometries) and the
gathered energies equal a serial solve of every geometry."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import synth
from paper_2606_26760_b300 import sharding


def test_lpt_assign_covers_every_geometry_once_and_balances():
    rng = np.random.default_rng(3)
    costs = rng.integers(500, 4000, 24) * rng.integers(500, 4000, 24)
    for world in (1, 2, 3, 4, 8, 30):
        parts = sharding.lpt_assign(costs, world)
        flat = sorted(g for p in parts for g in p)
        assert flat == list(range(24))
        loads = [sum(costs[g] for g in p) for p in parts]
        # greedy list-scheduling bound: no rank exceeds the mean load plus one geometry
        assert max(loads) <= sum(costs) / world + max(costs)
        for p in parts:  # each rank solves its largest geometry first
            assert all(costs[p[i]] >= costs[p[i + 1]] for i in range(len(p) - 1))


def test_lpt_assign_deterministic_ties_and_errors():
    assert sharding.lpt_assign([1, 1, 1, 1], 2) == [[0, 2], [1, 3]]
    assert sharding.lpt_assign([], 3) == [[], [], []]
    with pytest.raises(ValueError):
        sharding.lpt_assign([1.0], 0)


def _scan():
    return synth.bond_scan_workload(n_geom=5, n_orb=8, n_e=2, lo=6, hi=20)


def _oracle_energy(w):
    H = oracle.Ham(w["h"], w["eri"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    sa, sb = oracle.build_subspace(w["alpha"], w["beta"], w["n_alpha"], w["n_beta"])
    E, _ = oracle.ground_state_dense(H, sa, sb)
    return E


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws = _scan()
    costs = [sharding.geometry_cost(len(w["alpha"]), len(w["beta"])) for w in ws]
    solved = []

    def solve_one(g):
        solved.append(g)
        return _oracle_energy(ws[g]), 0

    energies, statuses = sharding.solve_sharded(costs, solve_one, rank, world)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"),
            np.array([energies, [float(len(solved))] * len(energies)]))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_scan_gloo_two_ranks(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    serial = [_oracle_energy(w) for w in _scan()]
    got = [np.load(tmp_path / f"rank{r}.npy") for r in range(world)]
    for g in got:  # every rank holds every geometry's energy
        assert np.allclose(g[0], serial, rtol=0, atol=1e-12)
    # each geometry was solved by exactly one rank
    assert int(got[0][1][0] + got[1][1][0]) == len(serial)
