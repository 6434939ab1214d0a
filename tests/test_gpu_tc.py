"""The opposite-spin term on the tensor cores against an emulation of exactly what it
computes: D(J_a, I_b; rs) and (pq|rs) rounded to BF16 by round-to-nearest-even, the
products accumulated wide (the kernel accumulates in FP32 in tensor memory), then
scattered over the alpha singles.  The links and phases come from the oracle; the
only approximation left between the two sides is the FP32 accumulation order, so the
bound is a few FP32 roundings of the term scale (2e-5 relative), far tighter than the
BF16 parity bound of the sigma tests (2e-2).  The cases span several 128-string beta
tiles with a ragged tail, beta counts with and without 16-byte aligned rows of C (the
two ways the kernel copies a row), and more alpha strings than one CTA takes."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

hq = pytest.importorskip("paper_2606_26760_b300")


def _bf16(x):
    """Round float32 values to BF16 (round to nearest, ties to even), returned as float64."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _singles(H, S, ne):
    """Per string: [(J, p, q, sign)] of its single links (J = sign a+_p a_q I)."""
    L = oracle.links(H, S, ne)
    out = []
    for I in range(len(S)):
        row = []
        for k in range(L["row_ptr"][I], L["row_ptr"][I + 1]):
            if L["degree"][k] == 1:
                row.append((int(L["col"][k]), int(L["p"][k]), int(L["q"][k]), int(L["sign"][k])))
        out.append(row)
    return out


def _fold(p, q):
    p, q = max(p, q), min(p, q)
    return p * (p + 1) // 2 + q


def _emulated_opposite(H, sa, sb, na, nb, c32):
    n = H.n
    K = n * (n + 1) // 2
    Na, Nb = len(sa), len(sb)
    C = np.asarray(c32, dtype=np.float32).reshape(Na, Nb)
    Bf = np.zeros((K, K))
    for p in range(n):
        for q in range(p + 1):
            for r in range(n):
                for s in range(r + 1):
                    Bf[_fold(p, q), _fold(r, s)] = H.eri[p, q, r, s]
    Bf = _bf16(Bf.astype(np.float32))
    A_s, B_s = _singles(H, sa, na), _singles(H, sb, nb)
    out = np.zeros((Na, Nb))
    for Ja in range(Na):
        if not A_s[Ja]:
            continue
        Cb = _bf16(C[Ja])
        D = np.zeros((Nb, K))
        for Ib in range(Nb):
            for (Jb, r, s, sg) in B_s[Ib]:
                D[Ib, _fold(r, s)] += sg * Cb[Jb]
            for j in range(n):
                if (int(sb[Ib]) >> j) & 1:
                    D[Ib, _fold(j, j)] += Cb[Ib]
        E = D @ Bf.T  # [Nb, folded pq]
        for (Ia, p, q, sg) in A_s[Ja]:
            out[Ia] += sg * E[:, _fold(p, q)]
    return out


@pytest.mark.parametrize("stages", [0, 1, 2, 3])
@pytest.mark.parametrize("n_sa,n_sb,seed", [(90, 300, 1), (70, 301, 2), (200, 130, 3)])
def test_opposite_spin_bf16_matches_emulation(n_sa, n_sb, seed, stages):
    """Each form of the tensor-core kernel (0: default, 1 and 2: pipeline depth of the
    persistent kernel, 3: the tile-stationary warp-specialised kernel)."""
    n, na, nb = 12, 4, 4
    h, eri, e_nuc = synth.integrals(n, 40 + seed)
    rng = np.random.default_rng(seed)
    fa, fb = synth.all_strings(n, na), synth.all_strings(n, nb)
    a = rng.choice(fa, n_sa, replace=False)
    b = rng.choice(fb, n_sb, replace=False)
    H = oracle.Ham(h, eri, e_nuc, na, nb)
    sa, sb = oracle.build_subspace(a, b, na, nb)
    ham = hq.Hamiltonian(h, eri, na, nb, e_nuc)
    sub = hq.build_subspace(a, b, n, na, nb)
    la, lb = hq.string_links(ham, sub, 0), hq.string_links(ham, sub, 1)
    hq.set_tuning(la, lb, stages=stages)
    c = synth.random_vector(sub.N, seed).astype(np.float32)
    ref = _emulated_opposite(H, sa, sb, na, nb, c)
    ct = torch.tensor(c, device="cuda")
    got = torch.zeros_like(ct)
    hq.sigma_part(ham, sub, la, lb, ct, got, "opposite", precision=hq.PREC_FP32_BF16AB)
    g = got.double().cpu().numpy().reshape(ref.shape)
    assert np.max(np.abs(g - ref)) <= 2e-5 * np.max(np.abs(ref))
    # the same operands at the full FP32 product differ only by the BF16 rounding
    f32 = torch.zeros_like(ct)
    hq.sigma_part(ham, sub, la, lb, ct, f32, "opposite", precision=hq.PREC_FP32)
    assert float(torch.max(torch.abs(f32 - got))) <= 2e-2 * float(torch.max(torch.abs(f32)))
