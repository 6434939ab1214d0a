"""The allocation-free spin-marginal call (collected last: a failure here leaves
every other test already run).

hinqs_spin_marginals_noalloc serves callers that cannot allocate device memory
while they run; its scratch is a fixed device array inside the library.  It must
give the same marginals and teacher weights as hinqs_spin_marginals, on two calls
in a row (the array keeps the previous call's contents), and refuse sizes beyond
its fixed capacity with an argument error.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

hq = pytest.importorskip("paper_2606_26760_b300")


def _call_noalloc(sub, c):
    dev = c.device
    pa = torch.empty(sub.Na, dtype=torch.float64, device=dev)
    pb = torch.empty(sub.Nb, dtype=torch.float64, device=dev)
    w = torch.empty(sub.N, dtype=torch.float64, device=dev)
    hq.spin_marginals_noalloc(sub, c, pa, pb, w)
    return pa, pb, w


def test_noalloc_marginals_match_allocating_call():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    torch.cuda.set_device(0)
    w_ = synth.workload("precision")
    sub = hq.build_subspace(w_["alpha"], w_["beta"], w_["n_orb"], w_["n_alpha"], w_["n_beta"])
    small = hq.build_subspace(synth.all_strings(8, 3), synth.all_strings(8, 2), 8, 3, 2)
    for S, seeds in ((sub, (3, 4)), (small, (5, 6))):
        for seed in seeds:  # two calls in a row on the shared scratch
            c = torch.tensor(synth.random_vector(S.N, seed), dtype=torch.float64, device="cuda")
            ra, rb, rw = hq.spin_marginals(S, c, want_w=True)
            pa, pb, w = _call_noalloc(S, c)
            torch.cuda.synchronize()
            for x, y in ((pa, ra), (pb, rb), (w, rw)):
                assert torch.max(torch.abs(x - y)).item() <= 1e-14 * max(1.0, torch.max(y).item())
            assert abs(pa.sum().item() - 1.0) < 1e-13 and abs(pb.sum().item() - 1.0) < 1e-13


def test_noalloc_rejects_sizes_beyond_capacity():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    # one alpha string (no alpha electrons), many beta strings:
    # C(40, 5) = 658008 beta strings fit the 2^20 - 2 doubles of fixed scratch ...
    fit = hq.build_subspace(None, None, 40, 0, 5, flags=hq.FULL_SPACE)
    assert fit.Na == 1 and fit.Nb == 658008
    c = torch.tensor(synth.random_vector(fit.N, 8), dtype=torch.float64, device="cuda")
    pa, pb, w = _call_noalloc(fit, c)
    ra, rb, rw = hq.spin_marginals(fit, c, want_w=True)
    assert torch.max(torch.abs(pb - rb)).item() <= 1e-14
    # ... C(24, 10) = 1961256 do not: the call refuses with an argument error
    huge = hq.build_subspace(None, None, 24, 0, 10, flags=hq.FULL_SPACE)
    assert huge.Nb > 2**20 - 2
    c = torch.zeros(huge.N, dtype=torch.float64, device="cuda")
    c[0] = 1.0
    with pytest.raises(hq.HinqsError) as e:
        _call_noalloc(huge, c)
    assert e.value.code == hq.ERR_ARG and "scratch" in str(e.value)
