"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Integer/index work (subspace, links, degrees, phases) must be bit-exact.
Floating point tolerances, derived from the arithmetic:
  * FP64 sigma: each element sums at most a few thousand products in a different
    order than the oracle; |err| <= 1e-11 * (|H_II c_I| + max|sigma|).
  * FP32 sigma: inputs and matrix elements rounded to FP32 (u = 6e-8) and FP32
    accumulation of <= ~10^3 terms; |err| <= 2e-5 * (|H_II c_I| + max|sigma|).
  * energies: 1e-9 Ha for the FP64 Davidson, 1e-6 Ha for the mixed one.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

hq = pytest.importorskip("paper_2606_26760_b300")


def _u64_np(t):
    return t.cpu().numpy().view(np.uint64)


def make_case(name):
    """Small cases the oracle finishes in seconds; several tiles and ragged sizes."""
    if name == "full_8_3_3":
        w = synth.workload("fp64_small")
        return w["h"], w["eri"], 0.0, 8, 3, 3, w["alpha"], w["beta"]
    if name == "ragged_10_3_4":
        h, eri, _ = synth.integrals(10, 101)
        rng = np.random.default_rng(5)
        a = synth.all_strings(10, 3)
        b = synth.all_strings(10, 4)
        a = rng.choice(a, size=41, replace=False)
        b = rng.choice(b, size=73, replace=False)
        return h, eri, 0.37, 10, 3, 4, a, b
    if name == "no_beta_6_2_0":
        h, eri, _ = synth.integrals(6, 102)
        return h, eri, 0.0, 6, 2, 0, synth.all_strings(6, 2), np.array([0], dtype=np.uint64)
    if name == "hf_12_4_4":
        h, eri, _ = synth.integrals(12, 103)
        a = synth.hf_weighted_strings(12, 4, 60, 7)
        b = synth.hf_weighted_strings(12, 4, 50, 8)
        return h, eri, -1.5, 12, 4, 4, a, b
    if name == "wide_40_2_2":   # n_orb above 32: strings use the upper half of the word
        h, eri, _ = synth.integrals(40, 104)
        rng = np.random.default_rng(9)
        A = synth.all_strings(40, 2)
        return (h, eri, 0.2, 40, 2, 2, rng.choice(A, 30, replace=False),
                rng.choice(A, 25, replace=False))
    if name == "single_alpha_9_3_2":   # one alpha string: no alpha links at all
        h, eri, _ = synth.integrals(9, 105)
        return h, eri, 0.0, 9, 3, 2, np.array([0b111], dtype=np.uint64), synth.all_strings(9, 2)
    if name == "filled_5_5_1":   # every alpha orbital occupied
        h, eri, _ = synth.integrals(5, 106)
        return (h, eri, 0.1, 5, 5, 1, np.array([0b11111], dtype=np.uint64),
                synth.all_strings(5, 1))
    raise KeyError(name)


SMALL = ["full_8_3_3", "ragged_10_3_4", "no_beta_6_2_0", "hf_12_4_4", "wide_40_2_2",
         "single_alpha_9_3_2", "filled_5_5_1"]


class Built:
    def __init__(self, h, eri, e_nuc, n, na, nb, a, b):
        self.H = oracle.Ham(h, eri, e_nuc, na, nb)
        self.sa, self.sb = oracle.build_subspace(a, b, na, nb)
        self.ham = hq.Hamiltonian(h, eri, na, nb, e_nuc)
        self.sub = hq.build_subspace(a, b, n, na, nb)
        self.la = hq.string_links(self.ham, self.sub, 0)
        self.lb = hq.string_links(self.ham, self.sub, 1)
        self.n, self.na, self.nb = n, na, nb


_cache = {}
_gs = {}


def ground_state(B):
    """Oracle ground state: dense eigh up to 3500 determinants, else Lanczos."""
    if id(B) not in _gs:
        if len(B.sa) * len(B.sb) <= 3500:
            _gs[id(B)] = oracle.ground_state_dense(B.H, B.sa, B.sb)
        else:
            E, c, r = oracle.lanczos(B.H, B.sa, B.sb, tol=1e-12)
            assert r < 1e-9
            _gs[id(B)] = (E, c)
    return _gs[id(B)]


def built(name):
    if name not in _cache:
        _cache[name] = Built(*make_case(name))
    return _cache[name]


@pytest.fixture(scope="module")
def precision_workload():
    w = synth.workload("precision")
    return Built(w["h"], w["eri"], w["e_nuc"], w["n_orb"], w["n_alpha"], w["n_beta"],
                 w["alpha"], w["beta"])


# ----------------------------------------------------------------- subspace --


def test_build_subspace_filters_sorts_dedupes():
    n, na, nb = 10, 3, 2
    rng = np.random.default_rng(11)
    a = synth.hf_weighted_samples(n, na, 5000, 3)
    b = synth.hf_weighted_samples(n, nb, 3000, 4)
    bad = np.array([0b1111, 0b1, 1 << 40 | 0b11, 0], dtype=np.uint64)
    a = np.concatenate([a, bad, a[:100]])
    rng.shuffle(a)
    b = np.concatenate([b, bad[:2]])
    sub = hq.build_subspace(a, b, n, na, nb)
    sa, sb = oracle.build_subspace(
        [x for x in a if (int(x) >> n) == 0], [x for x in b if (int(x) >> n) == 0], na, nb)
    ga, gb = sub.strings()
    assert np.array_equal(_u64_np(ga), sa) and np.array_equal(_u64_np(gb), sb)
    n_bad_a = sum(1 for x in a if bin(int(x)).count("1") != na or (int(x) >> n))
    n_bad_b = sum(1 for x in b if bin(int(x)).count("1") != nb or (int(x) >> n))
    assert sub.dropped == (n_bad_a, n_bad_b)


def test_build_subspace_error_mode_and_empty():
    with pytest.raises(hq.HinqsError) as e:
        hq.build_subspace(np.array([7, 15], np.uint64), np.array([3], np.uint64), 6, 3, 2,
                          flags=hq.ERROR_BAD)
    assert e.value.code == hq.ERR_PARTICLE_NUMBER
    with pytest.raises(hq.HinqsError) as e:
        hq.build_subspace(np.array([15], np.uint64), np.array([3], np.uint64), 6, 3, 2)
    assert e.value.code == hq.ERR_EMPTY


def test_full_space_matches_enumeration_and_table1():
    for n, k in [(8, 3), (10, 5), (16, 7), (20, 7), (26, 7)]:
        sub = hq.build_subspace(None, None, n, k, k, flags=hq.FULL_SPACE)
        ga, _ = sub.strings()
        ref = np.sort(synth.all_strings(n, k)) if n <= 20 else None
        if ref is not None:
            assert np.array_equal(_u64_np(ga), ref)
        assert sub.Na == sub.Nb
    # Table 1 dimensions C(M, n_a) C(M, n_b), up to the 77520-string CAS(14,20)
    import os
    rows = []
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "table1_dimensions.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, n, na, nb, ndet, digits = line.split()
        rows.append((int(n), int(na), int(nb), float(ndet), digits))
    for n, na, nb, ndet, digits in rows:
        sub = hq.build_subspace(None, None, n, na, nb, flags=hq.FULL_SPACE)
        dim = sub.Na * sub.Nb
        if digits == "exact":
            assert dim == int(ndet)
        else:
            assert float(f"{dim:.{int(digits) - 1}e}") == ndet


# -------------------------------------------------------------------- links --


def _compare_links(gpu, ref, rows=None):
    rp = gpu["row_ptr"].cpu().numpy()
    keys = ["col", "degree", "p", "q", "r", "s", "sign"]
    g = {k: gpu[k].cpu().numpy() for k in keys + ["hval"]}
    rows = range(len(rp) - 1) if rows is None else rows
    for k_out, I in enumerate(rows):
        a0, a1 = rp[I], rp[I + 1]
        b0, b1 = ref["row_ptr"][k_out], ref["row_ptr"][k_out + 1]
        assert a1 - a0 == b1 - b0, f"row {I}: {a1 - a0} vs {b1 - b0} links"
        for k in keys:
            assert np.array_equal(g[k][a0:a1].astype(np.int64), ref[k][b0:b1].astype(np.int64)), (I, k)
        assert np.max(np.abs(g["hval"][a0:a1] - ref["hval"][b0:b1]), initial=0.0) < 1e-12


@pytest.mark.parametrize("name", SMALL)
def test_links_bit_exact(name):
    B = built(name)
    for spin, S, ne, L in ((0, B.sa, B.na, B.la), (1, B.sb, B.nb, B.lb)):
        ref = oracle.links(B.H, S, ne)
        _compare_links(L.export(), ref)
        assert L.n_links == len(ref["col"])
        assert L.n_singles == int(np.sum(ref["degree"] == 1))


def test_links_sampled_rows_full_size(precision_workload):
    B = precision_workload
    rng = np.random.default_rng(9)
    for S, ne, L in ((B.sa, B.na, B.la), (B.sb, B.nb, B.lb)):
        rows = np.sort(rng.choice(len(S), size=64, replace=False))
        ref = oracle.links(B.H, S, ne, rows=rows)
        _compare_links(L.export(), ref, rows=rows)


# ------------------------------------------------------------ diag / sigma --


@pytest.mark.parametrize("name", SMALL)
def test_diag(name):
    B = built(name)
    d = hq.diag(B.ham, B.sub, B.la, B.lb).cpu().numpy()
    ref = oracle.diag(B.H, B.sa, B.sb)
    assert np.max(np.abs(d - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def _sigma_tol(rel, hd, c, ref):
    return rel * (np.abs(hd * c) + np.max(np.abs(ref)))


@pytest.mark.parametrize("name", SMALL)
def test_sigma_fp64_and_fp32(name):
    B = built(name)
    N = len(B.sa) * len(B.sb)
    for seed in (1, 2):
        c = synth.random_vector(N, seed)
        ref = oracle.sigma(B.H, B.sa, B.sb, c)
        hd = oracle.diag(B.H, B.sa, B.sb)
        ct = torch.tensor(c, dtype=torch.float64, device="cuda")
        s64 = hq.sigma(B.ham, B.sub, B.la, B.lb, ct).cpu().numpy()
        assert np.all(np.abs(s64 - ref) <= _sigma_tol(1e-11, hd, c, ref))
        s32 = hq.sigma(B.ham, B.sub, B.la, B.lb, ct.float()).double().cpu().numpy()
        assert np.all(np.abs(s32 - ref) <= _sigma_tol(2e-5, hd, c, ref))


@pytest.mark.parametrize("name", SMALL)
def test_sigma_tensor_core_modes(name):
    """Opposite-spin term on the tensor cores: operands rounded to BF16 (u = 2^-9)
    bound the error by ~1e-2 of the term scale; the hi+lo split by ~1e-4."""
    B = built(name)
    N = len(B.sa) * len(B.sb)
    c = synth.random_vector(N, 1)
    ref = oracle.sigma(B.H, B.sa, B.sb, c)
    hd = oracle.diag(B.H, B.sa, B.sb)
    ct = torch.tensor(c, dtype=torch.float32, device="cuda")
    for prec, rel in ((hq.PREC_FP32_BF16AB, 2e-2), (hq.PREC_FP32_BF16X3AB, 2e-4)):
        s = hq.sigma(B.ham, B.sub, B.la, B.lb, ct, precision=prec).double().cpu().numpy()
        assert np.all(np.abs(s - ref) <= _sigma_tol(rel, hd, c, ref)), prec


def test_sigma_tensor_core_full_size(precision_workload):
    B = precision_workload
    c = synth.random_vector(B.sub.N, 3)
    ct = torch.tensor(c, dtype=torch.float32, device="cuda")
    rows = np.sort(np.random.default_rng(4).choice(B.sub.N, size=256, replace=False))
    ref = oracle.sigma(B.H, B.sa, B.sb, c, rows=rows)
    hd = oracle.diag(B.H, B.sa, B.sb, rows=rows)
    s32 = hq.sigma(B.ham, B.sub, B.la, B.lb, ct).double()
    for prec, rel in ((hq.PREC_FP32_BF16AB, 2e-2), (hq.PREC_FP32_BF16X3AB, 2e-4)):
        s = hq.sigma(B.ham, B.sub, B.la, B.lb, ct, precision=prec).double()
        sr = s.cpu().numpy()[rows]
        assert np.all(np.abs(sr - ref) <= _sigma_tol(rel, hd, c[rows], ref)), prec
        # and against the FP32 CUDA-core product everywhere (a property at full size)
        assert float(torch.max(torch.abs(s - s32))) <= rel * float(torch.max(torch.abs(s32)))


def test_sigma_tensor_core_wide_beta_space():
    """More than 2^17 beta strings (n = 24, 6 beta electrons: the whole space of 134,596
    strings, three alpha strings): the tensor-core gather takes its 8-byte slots and
    reads the C row from global memory.  BF16 and split-BF16 products against the
    oracle on sampled rows, and against the FP32 CUDA-core product everywhere."""
    n, na, nb = 24, 1, 6
    h, eri, _ = synth.integrals(n, 107)
    a = np.array([1, 1 << 5, 1 << 23], dtype=np.uint64)
    b = synth.all_strings(n, nb)
    B = Built(h, eri, 0.3, n, na, nb, a, b)
    assert B.sub.Nb > (1 << 17)
    c = synth.random_vector(B.sub.N, 11)
    ct = torch.tensor(c, dtype=torch.float32, device="cuda")
    rows = np.sort(np.random.default_rng(12).choice(B.sub.N, size=48, replace=False))
    ref = oracle.sigma(B.H, B.sa, B.sb, c, rows=rows)
    hd = oracle.diag(B.H, B.sa, B.sb, rows=rows)
    s32 = hq.sigma(B.ham, B.sub, B.la, B.lb, ct).double()
    for prec, rel in ((hq.PREC_FP32_BF16AB, 2e-2), (hq.PREC_FP32_BF16X3AB, 2e-4)):
        s = hq.sigma(B.ham, B.sub, B.la, B.lb, ct, precision=prec).double()
        sr = s.cpu().numpy()[rows]
        assert np.all(np.abs(sr - ref) <= _sigma_tol(rel, hd, c[rows], ref)), prec
        assert float(torch.max(torch.abs(s - s32))) <= rel * float(torch.max(torch.abs(s32)))


def _bf16(x):
    """Round to BF16 (round to nearest, ties to even), returned as float64."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("name", SMALL)
def test_sigma_bf16c_mode(name):
    """HINQS_PREC_FP32_BF16C against the oracle: C rounded to BF16 (u = 2^-9) in every
    off-diagonal product bounds the error by ~1e-2 of the sigma scale; the diagonal
    term stays on the FP32 C, so the error of hdiag * c is FP32-sized.  The small
    cases have row lengths that are not multiples of 4 or of the 64-element padding
    of the BF16 copies (the guarded loads and the padded tails)."""
    B = built(name)
    N = len(B.sa) * len(B.sb)
    c = synth.random_vector(N, 1)
    ref = oracle.sigma(B.H, B.sa, B.sb, c)
    hd = oracle.diag(B.H, B.sa, B.sb)
    ct = torch.tensor(c, dtype=torch.float32, device="cuda")
    s = hq.sigma(B.ham, B.sub, B.la, B.lb, ct, precision=hq.PREC_FP32_BF16C).double().cpu().numpy()
    assert np.all(np.abs(s - ref) <= 2e-2 * np.max(np.abs(ref - hd * c)) + 2e-5 * np.abs(ref) +
                  1e-5 * np.max(np.abs(ref)))


@pytest.mark.parametrize("name", SMALL)
def test_sigma_bf16c_exact_parts(name):
    """What the BF16 operand changes and nothing else.  (1) For a vector whose entries
    are BF16 numbers the rounding is the identity, so the mode equals the FP32
    same-spin half plus the BF16 tensor-core term (HINQS_PREC_FP32_BF16AB) up to FP32
    summation order.  (2) The same-spin half is linear and rounds only the operand of
    the off-diagonal products: same(c) - same(bf16(c)) = hdiag * (c - bf16(c)), with
    hdiag from the oracle."""
    B = built(name)
    N = len(B.sa) * len(B.sb)
    c = synth.random_vector(N, 2)
    cb = _bf16(c)
    cbt = torch.tensor(cb, dtype=torch.float32, device="cuda")
    a = hq.sigma(B.ham, B.sub, B.la, B.lb, cbt, precision=hq.PREC_FP32_BF16C)
    b = hq.sigma(B.ham, B.sub, B.la, B.lb, cbt, precision=hq.PREC_FP32_BF16AB)
    assert float(torch.max(torch.abs(a - b))) <= 2e-6 * float(torch.max(torch.abs(b)))
    ct = torch.tensor(c, dtype=torch.float32, device="cuda")
    s1, s2 = torch.empty_like(ct), torch.empty_like(ct)
    hq.sigma_part(B.ham, B.sub, B.la, B.lb, ct, s1, "same", precision=hq.PREC_FP32_BF16C)
    hq.sigma_part(B.ham, B.sub, B.la, B.lb, cbt, s2, "same", precision=hq.PREC_FP32_BF16C)
    hd = oracle.diag(B.H, B.sa, B.sb)
    d = (s1 - s2).double().cpu().numpy()
    want = hd * (ct.double().cpu().numpy() - cb)
    scale = float(torch.max(torch.abs(s1)))
    assert np.all(np.abs(d - want) <= 1e-6 * scale + 1e-5 * np.abs(want))


def test_sigma_bf16c_full_size(precision_workload):
    """The bench configuration: 256 sampled rows against the oracle, and the whole
    vector against the FP32 CUDA-core product (the rows are 2000 floats: 16-byte
    aligned, BF16 copies padded from 2000 to 2048)."""
    B = precision_workload
    c = synth.random_vector(B.sub.N, 3)
    ct = torch.tensor(c, dtype=torch.float32, device="cuda")
    rows = np.sort(np.random.default_rng(4).choice(B.sub.N, size=256, replace=False))
    ref = oracle.sigma(B.H, B.sa, B.sb, c, rows=rows)
    hd = oracle.diag(B.H, B.sa, B.sb, rows=rows)
    s = hq.sigma(B.ham, B.sub, B.la, B.lb, ct, precision=hq.PREC_FP32_BF16C).double()
    sr = s.cpu().numpy()[rows]
    off = ref - hd * c[rows]
    assert np.all(np.abs(sr - ref) <= 2e-2 * np.max(np.abs(off)) + 2e-5 * np.abs(ref))
    s32 = hq.sigma(B.ham, B.sub, B.la, B.lb, ct).double()
    assert float(torch.max(torch.abs(s - s32))) <= 2e-2 * float(torch.max(torch.abs(s32)))


@pytest.mark.parametrize("name", SMALL)
def test_sigma_fp64_double_float_opposite_spin(name):
    """HINQS_PREC_FP64_DFAB: the opposite-spin term in double-float arithmetic (FP32
    pairs, error-free products, two-sum accumulation, ~2^-44 per term) is held to the
    FP64 bound against the oracle."""
    B = built(name)
    N = len(B.sa) * len(B.sb)
    for seed in (1, 2):
        c = synth.random_vector(N, seed)
        ref = oracle.sigma(B.H, B.sa, B.sb, c)
        hd = oracle.diag(B.H, B.sa, B.sb)
        ct = torch.tensor(c, dtype=torch.float64, device="cuda")
        s = hq.sigma(B.ham, B.sub, B.la, B.lb, ct, precision=hq.PREC_FP64_DFAB).cpu().numpy()
        assert np.all(np.abs(s - ref) <= _sigma_tol(1e-11, hd, c, ref))


def test_sigma_double_float_full_size(precision_workload):
    """Sampled rows against the oracle and the whole vector against the FP64 product."""
    B = precision_workload
    c = synth.random_vector(B.sub.N, 5)
    ct = torch.tensor(c, dtype=torch.float64, device="cuda")
    s = hq.sigma(B.ham, B.sub, B.la, B.lb, ct, precision=hq.PREC_FP64_DFAB)
    s64 = hq.sigma(B.ham, B.sub, B.la, B.lb, ct)
    assert float(torch.max(torch.abs(s - s64))) <= 1e-12 * float(torch.max(torch.abs(s64)))
    rows = np.sort(np.random.default_rng(6).choice(B.sub.N, size=128, replace=False))
    ref = oracle.sigma(B.H, B.sa, B.sb, c, rows=rows)
    hd = oracle.diag(B.H, B.sa, B.sb, rows=rows)
    assert np.all(np.abs(s.cpu().numpy()[rows] - ref) <= _sigma_tol(1e-11, hd, c[rows], ref))


def test_davidson_mixed_refinement_precisions():
    """The mixed solver's refinement products in double-float (the default) and in FP64
    reach the same eigenpair."""
    B = built("hf_12_4_4")
    E, _ = ground_state(B)
    kw = dict(precision=hq.DAVIDSON_MIXED, inner_precision=hq.PREC_FP32_BF16C,
              tol_residual=1e-9, tol_energy=1e-12, max_iter=600)
    a = hq.davidson(B.ham, B.sub, B.la, B.lb, refine_precision=hq.PREC_FP64_DFAB, **kw)
    b = hq.davidson(B.ham, B.sub, B.la, B.lb, refine_precision=hq.PREC_FP64, **kw)
    assert a.status == hq.OK and b.status == hq.OK
    assert abs(a.energy - E) <= 1e-9 and abs(b.energy - E) <= 1e-9
    assert abs(abs(torch.dot(a.c, b.c).item()) - 1.0) <= 1e-12


def test_sigma_halves_sum_to_sigma(precision_workload):
    """hinqs_sigma_same_spin + hinqs_sigma_opposite_spin == hinqs_sigma in every mode."""
    B = precision_workload
    c = torch.tensor(synth.random_vector(B.sub.N, 7), device="cuda")
    for prec, x in ((hq.PREC_FP64, c), (hq.PREC_FP32, c.float()),
                    (hq.PREC_FP32_BF16AB, c.float()), (hq.PREC_FP32_BF16X3AB, c.float()),
                    (hq.PREC_FP32_BF16C, c.float()), (hq.PREC_FP64_DFAB, c)):
        full = hq.sigma(B.ham, B.sub, B.la, B.lb, x, precision=prec)
        part = torch.empty_like(x)
        hq.sigma_part(B.ham, B.sub, B.la, B.lb, x, part, "same", precision=prec)
        hq.sigma_part(B.ham, B.sub, B.la, B.lb, x, part, "opposite", precision=prec)
        tol = (1e-12 if prec in (hq.PREC_FP64, hq.PREC_FP64_DFAB) else 1e-5) * float(
            torch.max(torch.abs(full)))
        assert float(torch.max(torch.abs(full - part))) <= tol


def test_sigma_full_size_sampled_rows(precision_workload):
    """The bench configuration (n=16, 5/5, 2000 x 2000): 512 sampled rows."""
    B = precision_workload
    N = B.sub.N
    assert N == 4_000_000
    c = synth.random_vector(N, 3)
    ct = torch.tensor(c, dtype=torch.float64, device="cuda")
    rows = np.sort(np.random.default_rng(4).choice(N, size=512, replace=False))
    ref = oracle.sigma(B.H, B.sa, B.sb, c, rows=rows)
    hd = oracle.diag(B.H, B.sa, B.sb, rows=rows)
    s64 = hq.sigma(B.ham, B.sub, B.la, B.lb, ct).cpu().numpy()[rows]
    assert np.all(np.abs(s64 - ref) <= _sigma_tol(1e-11, hd, c[rows], ref))
    s32 = hq.sigma(B.ham, B.sub, B.la, B.lb, ct.float()).double().cpu().numpy()[rows]
    assert np.all(np.abs(s32 - ref) <= _sigma_tol(2e-5, hd, c[rows], ref))
    d = hq.diag(B.ham, B.sub, B.la, B.lb).cpu().numpy()[rows]
    assert np.max(np.abs(d - hd)) < 1e-11


def test_sigma_hermitian_full_size(precision_workload):
    """<x, H y> = <H x, y> at full size (a property at any size)."""
    B = precision_workload
    x = torch.tensor(synth.random_vector(B.sub.N, 5), dtype=torch.float64, device="cuda")
    y = torch.tensor(synth.random_vector(B.sub.N, 6), dtype=torch.float64, device="cuda")
    hx = hq.sigma(B.ham, B.sub, B.la, B.lb, x)
    hy = hq.sigma(B.ham, B.sub, B.la, B.lb, y)
    a, b = float(x @ hy), float(hx @ y)
    assert abs(a - b) <= 1e-12 * (float(x.norm() * hy.norm()) + 1.0)


# ----------------------------------------------------------------- davidson --


@pytest.mark.parametrize("name", ["full_8_3_3", "ragged_10_3_4", "hf_12_4_4", "wide_40_2_2",
                                  "single_alpha_9_3_2", "filled_5_5_1"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_davidson_vs_dense(name, prec):
    B = built(name)
    E, c0 = ground_state(B)
    p = hq.DAVIDSON_FP64 if prec == "fp64" else hq.DAVIDSON_MIXED
    res = hq.davidson(B.ham, B.sub, B.la, B.lb, precision=p, tol_residual=1e-8,
                      max_subspace=12, max_iter=300)
    assert res.status == hq.OK
    tol = 1e-9 if prec == "fp64" else 1e-6
    assert abs(res.energy - E) <= tol
    c = res.c.cpu().numpy()
    assert abs(abs(c @ c0) - 1.0) < 1e-8
    assert res.residual <= 1e-8
    # the reported residual is the FP64 one
    Hc = oracle.sigma(B.H, B.sa, B.sb, c)
    assert np.linalg.norm(Hc - res.energy * c) <= 2e-8


def test_davidson_full_size_properties(precision_workload):
    """The bench configuration (4.0e6 determinants): FP64 and mixed solvers agree,
    and the oracle's sampled rows confirm the residual of both eigenvectors."""
    B = precision_workload
    r64 = hq.davidson(B.ham, B.sub, B.la, B.lb, precision=hq.DAVIDSON_FP64, tol_residual=1e-8,
                      max_iter=400, max_subspace=16)
    rmx = hq.davidson(B.ham, B.sub, B.la, B.lb, precision=hq.DAVIDSON_MIXED, tol_residual=1e-8,
                      max_iter=400, max_subspace=16)
    assert r64.status == hq.OK and rmx.status == hq.OK
    assert abs(r64.energy - rmx.energy) <= 1e-8
    assert rmx.n_sigma_fp64 < r64.n_sigma_fp64
    rows = np.sort(np.random.default_rng(17).choice(B.sub.N, size=256, replace=False))
    for res in (r64, rmx):
        c = res.c.cpu().numpy()
        assert abs(np.linalg.norm(c) - 1.0) < 1e-12
        Hc = oracle.sigma(B.H, B.sa, B.sb, c, rows=rows)
        assert np.max(np.abs(Hc - res.energy * c[rows])) <= 1e-8


@pytest.mark.parametrize("inner", ["bf16", "bf16x3", "bf16c"])
def test_davidson_mixed_tensor_core_inner(inner):
    """Mixed Davidson whose inner products use the tensor-core term (and, bf16c, BF16
    operands in the same-spin products too): the FP64 refinement still reaches the
    FP64 energy."""
    B = built("hf_12_4_4")
    E, c0 = ground_state(B)
    p = {"bf16": hq.PREC_FP32_BF16AB, "bf16x3": hq.PREC_FP32_BF16X3AB,
         "bf16c": hq.PREC_FP32_BF16C}[inner]
    res = hq.davidson(B.ham, B.sub, B.la, B.lb, precision=hq.DAVIDSON_MIXED, inner_precision=p,
                      tol_residual=1e-8, max_subspace=12, max_iter=400)
    assert res.status == hq.OK
    assert abs(res.energy - E) <= 1e-6
    assert res.residual <= 1e-8


def test_davidson_warm_start_and_not_converged():
    B = built("hf_12_4_4")
    E, c0 = ground_state(B)
    g = torch.tensor(c0, dtype=torch.float64, device="cuda")
    res = hq.davidson(B.ham, B.sub, B.la, B.lb, guess=g, tol_residual=1e-8)
    assert res.status == hq.OK and res.iterations <= 3 and abs(res.energy - E) < 1e-9
    res = hq.davidson(B.ham, B.sub, B.la, B.lb, max_iter=2, tol_residual=1e-12)
    assert res.status == hq.NOT_CONVERGED and res.iterations == 2


# ---------------------------------------------------------- RDM / backward --


@pytest.mark.parametrize("name", SMALL)
def test_rdm_matches_oracle(name):
    B = built(name)
    c = synth.random_vector(B.sub.N, 12)
    g1, g2 = hq.rdm(B.sub, B.la, B.lb, torch.tensor(c, dtype=torch.float64, device="cuda"))
    r1, r2 = oracle.rdm(B.n, B.sa, B.sb, c)
    scale = float(c @ c)
    assert np.max(np.abs(g1.cpu().numpy() - r1)) < 1e-11 * scale
    assert np.max(np.abs(g2.cpu().numpy() - r2)) < 1e-11 * scale


def test_rdm_long_beta_rows_matches_oracle():
    """Beta rows too long for the staged opposite-spin kernel (n = 20, 5 beta electrons:
    the whole space of 15,504 strings, three alpha strings), so the unstaged form runs;
    every element against the oracle."""
    n, na, nb = 20, 1, 5
    h, eri, _ = synth.integrals(n, 108)
    a = np.array([1, 1 << 7, 1 << 19], dtype=np.uint64)
    B = Built(h, eri, 0.0, n, na, nb, a, synth.all_strings(n, nb))
    assert B.sub.Nb == 15504
    c = synth.random_vector(B.sub.N, 31)
    g1, g2 = hq.rdm(B.sub, B.la, B.lb, torch.tensor(c, dtype=torch.float64, device="cuda"))
    r1, r2 = oracle.rdm(B.n, B.sa, B.sb, c)
    scale = float(c @ c)
    assert np.max(np.abs(g1.cpu().numpy() - r1)) < 1e-11 * scale
    assert np.max(np.abs(g2.cpu().numpy() - r2)) < 1e-11 * scale


def test_energy_autograd_hellmann_feynman():
    h, eri, e_nuc, n, na, nb, a, b = make_case("hf_12_4_4")
    sub = hq.build_subspace(a, b, n, na, nb)
    ht = torch.tensor(h, device="cuda", requires_grad=True)
    et = torch.tensor(eri, device="cuda", requires_grad=True)
    E = hq.energy(ht, et, sub, na, nb, e_nuc, tol_residual=1e-10)
    E.backward()
    H = oracle.Ham(h, eri, e_nuc, na, nb)
    sa, sb = oracle.build_subspace(a, b, na, nb)
    Eo, c0 = ground_state(built("hf_12_4_4"))
    assert abs(float(E) - Eo) < 1e-9
    r1, r2 = oracle.rdm(n, sa, sb, c0)
    assert np.max(np.abs(ht.grad.cpu().numpy() - r1)) < 1e-8
    assert np.max(np.abs(et.grad.cpu().numpy() - 0.5 * r2)) < 1e-8


# ---------------------------------------------------------------- marginals --


@pytest.mark.parametrize("name", SMALL)
def test_spin_marginals(name):
    B = built(name)
    c = synth.random_vector(B.sub.N, 13)
    pa, pb, w = hq.spin_marginals(B.sub, torch.tensor(c, dtype=torch.float64, device="cuda"),
                                  want_w=True)
    ra, rb, rw = oracle.marginals(c, B.sub.Na, B.sub.Nb, want_w=True)
    assert np.max(np.abs(pa.cpu().numpy() - ra)) < 1e-14
    assert np.max(np.abs(pb.cpu().numpy() - rb)) < 1e-14
    assert np.max(np.abs(w.cpu().numpy() - rw)) < 1e-14
