"""The allocation-free spin-marginal call (collected last: a failure here leaves
every other test already run).

hinqs_spin_marginals_noalloc serves callers that cannot allocate device memory
while they run; its scratch is a fixed device array inside the library.  It must
give the same marginals and teacher weights as hinqs_spin_marginals, on two calls
in a row (the array keeps the previous call's contents), take nothing from the
stream-ordered pool once its first call has looked up the array, and refuse sizes
beyond its fixed capacity with an argument error.
"""
import ctypes

import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

hq = pytest.importorskip("paper_2606_26760_b300")

# cudaMemPoolAttr values of the CUDA runtime
RESERVED_CURRENT, RESERVED_HIGH, USED_CURRENT, USED_HIGH = 5, 6, 7, 8


def _call_noalloc(sub, c):
    dev = c.device
    pa = torch.empty(sub.Na, dtype=torch.float64, device=dev)
    pb = torch.empty(sub.Nb, dtype=torch.float64, device=dev)
    w = torch.empty(sub.N, dtype=torch.float64, device=dev)
    hq.spin_marginals_noalloc(sub, c, pa, pb, w)
    return pa, pb, w


def _compare(sub, c):
    ra, rb, rw = hq.spin_marginals(sub, c, want_w=True)
    pa, pb, w = _call_noalloc(sub, c)
    torch.cuda.synchronize()
    for x, y in ((pa, ra), (pb, rb), (w, rw)):
        assert torch.max(torch.abs(x - y)).item() <= 1e-14 * max(1.0, torch.max(y).item())
    assert abs(pa.sum().item() - 1.0) < 1e-13 and abs(pb.sum().item() - 1.0) < 1e-13


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
            _compare(S, c)


def test_noalloc_many_alpha_rows_and_long_beta_rows():
    """Shapes that change how the fixed scratch is cut: 40 alpha strings with 658,008
    beta strings (one chunk of 64 rows), and 780 alpha strings with 91,390 beta strings
    (only 11 column-partial rows fit the scratch, so each chunk takes 71 alpha rows)."""
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    for n, na, nb, seed in ((40, 1, 5, 21), (40, 2, 4, 22)):
        sub = hq.build_subspace(None, None, n, na, nb, flags=hq.FULL_SPACE)
        assert sub.Na > 1
        for k in range(2):
            c = torch.tensor(synth.random_vector(sub.N, seed + 10 * k), dtype=torch.float64,
                             device="cuda")
            _compare(sub, c)
            del c
        torch.cuda.empty_cache()


def test_noalloc_takes_nothing_from_the_pool():
    """After the first call (which looks up the array's device address), a further call
    leaves the stream-ordered pool's used and reserved high-water marks unchanged."""
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    rt = ctypes.CDLL("libcudart.so.13")
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0

    def attr(a):
        v = ctypes.c_uint64()
        assert rt.cudaMemPoolGetAttribute(pool, a, ctypes.byref(v)) == 0
        return v.value

    sub = hq.build_subspace(synth.all_strings(10, 3), synth.all_strings(10, 4), 10, 3, 4)
    c = torch.tensor(synth.random_vector(sub.N, 9), dtype=torch.float64, device="cuda")
    pa = torch.empty(sub.Na, dtype=torch.float64, device="cuda")
    pb = torch.empty(sub.Nb, dtype=torch.float64, device="cuda")
    w = torch.empty(sub.N, dtype=torch.float64, device="cuda")
    hq.spin_marginals_noalloc(sub, c, pa, pb, w)  # set-up call
    torch.cuda.synchronize()
    zero = ctypes.c_uint64(0)
    for a in (USED_HIGH, RESERVED_HIGH):
        assert rt.cudaMemPoolSetAttribute(pool, a, ctypes.byref(zero)) == 0
    before = (attr(USED_CURRENT), attr(RESERVED_CURRENT))
    torch_before = torch.cuda.memory_allocated()
    hq.spin_marginals_noalloc(sub, c, pa, pb, w)
    torch.cuda.synchronize()
    assert attr(USED_HIGH) <= before[0] and attr(USED_CURRENT) == before[0]
    assert attr(RESERVED_HIGH) <= before[1] and attr(RESERVED_CURRENT) == before[1]
    assert torch.cuda.memory_allocated() == torch_before


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


def test_noalloc_binding_rejects_bad_buffers():
    """The binding checks caller-owned buffers before the call (a short or float32
    output would be written past its end on the device)."""
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    sub = hq.build_subspace(synth.all_strings(8, 3), synth.all_strings(8, 2), 8, 3, 2)
    c = torch.tensor(synth.random_vector(sub.N, 2), dtype=torch.float64, device="cuda")
    pa = torch.empty(sub.Na, dtype=torch.float64, device="cuda")
    pb = torch.empty(sub.Nb, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        hq.spin_marginals_noalloc(sub, c, pa[:-1], pb)
    with pytest.raises(ValueError):
        hq.spin_marginals_noalloc(sub, c, pa.float(), pb)
    with pytest.raises(ValueError):
        hq.spin_marginals_noalloc(sub, c.float(), pa, pb)
    with pytest.raises(ValueError):
        hq.spin_marginals_noalloc(sub, c, pa, pb, torch.empty(sub.N - 1, dtype=torch.float64,
                                                              device="cuda"))
