"""The timeout path, exercised without faulting or hanging the GPU: the tensor-core
kernel's bounded mbarrier wait runs out on a barrier that nothing completes, the
library reports HINQS_ERR_TIMEOUT, and the device and the library stay usable (the
flag is cleared and the next tensor-core sigma gives the same result as before)."""
import time

import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

hq = pytest.importorskip("paper_2606_26760_b300")


def test_bounded_wait_runs_out_and_library_stays_usable():
    w = synth.workload("fp64_small")
    ham = hq.Hamiltonian(w["h"], w["eri"], w["n_alpha"], w["n_beta"], w["e_nuc"])
    sub = hq.build_subspace(w["alpha"], w["beta"], w["n_orb"], w["n_alpha"], w["n_beta"])
    la, lb = hq.string_links(ham, sub, 0), hq.string_links(ham, sub, 1)
    c = torch.tensor(synth.random_vector(sub.N, 5), dtype=torch.float32, device="cuda")
    before = hq.sigma(ham, sub, la, lb, c, precision=hq.PREC_FP32_BF16X3AB)
    t0 = time.perf_counter()
    rc = hq.selftest_bounded_wait(4096)
    elapsed = time.perf_counter() - t0
    assert rc == hq.ERR_TIMEOUT
    assert elapsed < 30.0
    after = hq.sigma(ham, sub, la, lb, c, precision=hq.PREC_FP32_BF16X3AB)  # raises if flagged
    scale = float(before.abs().max())
    assert float((after - before).abs().max()) <= 1e-5 * scale
    assert hq.selftest_bounded_wait(1) == hq.ERR_TIMEOUT
