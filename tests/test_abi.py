"""CPU-side checks of the C-ABI library: it loads and exports every entry point
that include/hinqs.h declares (no compute call is made without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hinqs.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hinqs_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import paper_2606_26760_b300 as hq
    from paper_2606_26760_b300 import build as hb
    hb.build()
    return hq.load_library()


def test_header_declares_the_hot_path_calls():
    names = declared_functions()
    for required in ["hinqs_build_subspace", "hinqs_string_links", "hinqs_sigma",
                     "hinqs_davidson", "hinqs_rdm", "hinqs_spin_marginals"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    import paper_2606_26760_b300 as hq
    assert sorted(hq.EXPORTED) == declared_functions()


def test_argument_errors_without_gpu(lib):
    """Host-side validation returns HINQS_ERR_ARG before touching the device."""
    out = ctypes.c_void_p()
    lib.hinqs_ham_create.restype = ctypes.c_int
    rc = lib.hinqs_ham_create(None, None, 8, 3, 3, 0.0, 0, ctypes.byref(out), None)
    assert rc == -1
    assert b"NULL" in lib.hinqs_last_error_message()
    dummy = ctypes.c_void_p(16)
    rc = lib.hinqs_ham_create(dummy, dummy, 65, 3, 3, 0.0, 0, ctypes.byref(out), None)
    assert rc == -1 and b"n_orb" in lib.hinqs_last_error_message()
    rc = lib.hinqs_build_subspace(None, 4, None, 4, 8, 3, 3, 0, ctypes.byref(out), None, None)
    assert rc == -1
    rc = lib.hinqs_string_links(None, None, 0, ctypes.byref(out), None)
    assert rc == -1
    rc = lib.hinqs_energy_backward(0, 1.0, None, None, None, None, None)
    assert rc == -1
    lib.hinqs_selftest_bounded_wait.argtypes = [ctypes.c_longlong, ctypes.c_void_p]
    assert lib.hinqs_selftest_bounded_wait(0, None) == -1
    assert lib.hinqs_selftest_bounded_wait((1 << 26) + 1, None) == -1
    P = ctypes.c_void_p
    lib.hinqs_selftest_projected_eig.argtypes = [P, P, ctypes.c_int, P, P, P, P]
    buf = (ctypes.c_double * 4)()
    assert lib.hinqs_selftest_projected_eig(None, None, 1, buf, None, None, None) == -1
    assert lib.hinqs_selftest_projected_eig(buf, None, 0, buf, None, None, None) == -1
    assert lib.hinqs_selftest_projected_eig(buf, None, 33, buf, None, None, None) == -1


def test_product_path_has_no_cpu_fallback():
    """Without a CUDA device every compute entry of the binding raises."""
    import torch
    import paper_2606_26760_b300 as hq
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        hq.build_subspace([7, 11], [7, 11], 4, 3, 3)
    src = open(os.path.join(ROOT, "paper_2606_26760_b300", "__init__.py")).read()
    assert "import oracle" not in src and "from oracle" not in src


def test_workspace_queries_without_gpu(lib):
    """Host-only size queries: linear in the number of determinants, the mixed solver
    below the FP64 one at the same subspace size (FP32 correction basis), argument
    errors for bad options."""
    import paper_2606_26760_b300 as hq
    s64 = hq.sigma_workspace_size(2000, 2000, hq.PREC_FP64)
    assert s64 == 2 * 4_000_000 * 8
    assert hq.sigma_workspace_size(2000, 2000, hq.PREC_FP32_BF16AB) == s64 // 2
    small = hq.davidson_workspace_size(100, 100)
    big = hq.davidson_workspace_size(1000, 1000)
    const = small - (big - small) // 99           # bytes that do not grow with N
    assert big - const == 100 * (small - const)
    assert hq.davidson_workspace_size(2000, 2000, hq.DAVIDSON_MIXED) < \
        hq.davidson_workspace_size(2000, 2000, hq.DAVIDSON_FP64)
    assert hq.davidson_workspace_size(2000, 2000, max_subspace=24) > \
        hq.davidson_workspace_size(2000, 2000, max_subspace=8)
    with pytest.raises(hq.HinqsError):
        hq.davidson_workspace_size(10, 10, max_subspace=2)
    with pytest.raises(hq.HinqsError):
        hq.sigma_workspace_size(10, 10, 7)
