"""The workspace queries against what the calls really take from the stream-ordered
pool: the high-water mark of the device's default memory pool, read through the CUDA
runtime, rises during one call by no more than the reported size (plus the pool's
rounding of each request, at most 64 MiB over the call's few dozen requests) and by
at least 90% of it."""
import ctypes
import gc

import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

hq = pytest.importorskip("paper_2606_26760_b300")

USED_CURRENT, USED_HIGH = 7, 8   # cudaMemPoolAttrUsedMemCurrent / cudaMemPoolAttrUsedMemHigh
SLACK = 64 << 20


def _pool():
    rt = ctypes.CDLL("libcudart.so.13")
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0
    return rt, pool


def _peak_of(fn):
    rt, pool = _pool()
    gc.collect()   # release unreferenced handles of earlier tests before the baseline
    torch.cuda.synchronize()
    cur = ctypes.c_uint64()
    assert rt.cudaMemPoolGetAttribute(pool, USED_CURRENT, ctypes.byref(cur)) == 0
    zero = ctypes.c_uint64(0)
    assert rt.cudaMemPoolSetAttribute(pool, USED_HIGH, ctypes.byref(zero)) == 0
    fn()
    torch.cuda.synchronize()
    high = ctypes.c_uint64()
    assert rt.cudaMemPoolGetAttribute(pool, USED_HIGH, ctypes.byref(high)) == 0
    return high.value - cur.value


@pytest.fixture(scope="module")
def problem():
    w = synth.workload("precision")
    n, na, nb = w["n_orb"], w["n_alpha"], w["n_beta"]
    ham = hq.Hamiltonian(w["h"], w["eri"], na, nb, w["e_nuc"])
    sub = hq.build_subspace(w["alpha"], w["beta"], n, na, nb)
    la, lb = hq.string_links(ham, sub, 0), hq.string_links(ham, sub, 1)
    return ham, sub, la, lb


@pytest.mark.parametrize("prec", [hq.DAVIDSON_FP64, hq.DAVIDSON_MIXED])
def test_davidson_workspace_matches_pool_usage(problem, prec):
    ham, sub, la, lb = problem
    out = torch.empty(sub.N, dtype=torch.float64, device="cuda")
    bound = hq.davidson_workspace_size(sub.Na, sub.Nb, prec, 12)
    peak = _peak_of(lambda: hq.davidson(ham, sub, la, lb, precision=prec, max_subspace=12,
                                        max_iter=4, inner_precision=hq.PREC_FP32_BF16AB,
                                        out=out))
    assert 0.9 * bound <= peak <= bound + SLACK, (peak, bound)


@pytest.mark.parametrize("prec", [hq.PREC_FP64, hq.PREC_FP32, hq.PREC_FP32_BF16C, hq.PREC_FP64_DFAB])
def test_sigma_workspace_matches_pool_usage(problem, prec):
    ham, sub, la, lb = problem
    dt = torch.float64 if prec in (hq.PREC_FP64, hq.PREC_FP64_DFAB) else torch.float32
    c = torch.ones(sub.N, dtype=dt, device="cuda")
    y = torch.empty_like(c)
    bound = hq.sigma_workspace_size(sub.Na, sub.Nb, prec)
    peak = _peak_of(lambda: hq.sigma(ham, sub, la, lb, c, out=y, precision=prec))
    assert 0.9 * bound <= peak <= bound + SLACK, (peak, bound)
