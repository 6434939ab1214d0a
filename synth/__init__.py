"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and bench.py.

This module generates *inputs only*: one-electron integrals h_pq, chemist-order
two-electron integrals (pq|rs) and occupation strings (uint64 bitmasks, bit p =
spatial orbital p).  It holds none of the method's arithmetic (no excitation
degrees, phases, matrix elements, eigen-solves, RDMs or marginals).

Recipes (the paper's molecular integrals, computed with PySCF for the systems of
Table 1, are not published, so seeded synthetics with the same shapes stand in):

* integrals(n, seed): h symmetric, diagonal U(-2, 0) sorted ascending (so the
  lowest orbitals form a meaningful Hartree-Fock reference), off-diagonal
  N(0, 0.1); (pq|rs) = sum_{L<24} B^L_pq B^L_rs with B^L symmetric,
  B^L_pq ~ N(0, 0.3) / (1 + |p-q|).  The ERI tensor is 8-fold symmetric and
  positive semidefinite as a (pq)x(rs) matrix by construction.  E_nuc = 0.
* hf_weighted_strings(n, n_e, count, seed): excitation rank k relative to the
  string of the lowest n_e orbitals is drawn with probability proportional to
  0.3^k, k in [0, min(n_e, n-n_e)]; k holes are drawn uniformly among the
  lowest n_e orbitals and k particles uniformly among the rest; duplicates are
  rejected until `count` unique strings are collected (draw order is kept).
* bond_scan(k): integrals interpolated between two seeded endpoint sets with
  s = smoothstep((R - 0.9) / 2.1), R in [0.9, 3.0]; B^L is interpolated (not
  the ERI) so every geometry's ERI stays PSD.
"""
from __future__ import annotations

import itertools
from math import comb

import numpy as np

N_CHOLESKY = 24


def integrals(n_orb: int, seed: int, n_chol: int = N_CHOLESKY):
    """Return (h[n,n], eri[n,n,n,n], e_nuc) as float64 arrays (chemist order)."""
    h, B = _endpoint(n_orb, seed, n_chol)
    return h, _eri_from_factors(B), 0.0


def _endpoint(n_orb: int, seed: int, n_chol: int):
    rng = np.random.default_rng(seed)
    diag = np.sort(rng.uniform(-2.0, 0.0, size=n_orb))
    off = rng.normal(0.0, 0.1, size=(n_orb, n_orb))
    h = np.triu(off, 1)
    h = h + h.T + np.diag(diag)
    p = np.arange(n_orb)
    decay = 1.0 / (1.0 + np.abs(p[:, None] - p[None, :]))
    B = np.empty((n_chol, n_orb, n_orb))
    for L in range(n_chol):
        g = rng.normal(0.0, 0.3, size=(n_orb, n_orb))
        g = np.triu(g) + np.triu(g, 1).T
        B[L] = g * decay
    return h, B


def _eri_from_factors(B):
    n = B.shape[1]
    Bf = B.reshape(B.shape[0], n * n)
    return (Bf.T @ Bf).reshape(n, n, n, n)


def smoothstep(x):
    x = np.clip(x, 0.0, 1.0)
    return x * x * (3.0 - 2.0 * x)


def bond_scan_R(n_geom: int = 24):
    return 0.9 + 2.1 * np.arange(n_geom) / max(n_geom - 1, 1)


def bond_scan(n_orb: int, R: float, seed: int = 4, n_chol: int = N_CHOLESKY):
    """Integrals of one synthetic bond-scan geometry at scan parameter R."""
    h0, B0 = _endpoint(n_orb, 1000 * seed + 1, n_chol)
    h1, B1 = _endpoint(n_orb, 1000 * seed + 2, n_chol)
    s = float(smoothstep((R - 0.9) / 2.1))
    h = (1.0 - s) * h0 + s * h1
    B = (1.0 - s) * B0 + s * B1
    return h, _eri_from_factors(B), 0.0


def _bits(orbs):
    v = 0
    for o in orbs:
        v |= 1 << int(o)
    return v


def _draw_batch(rng, n_orb, n_e, pk, size):
    """`size` HF-weighted strings (with repeats) as uint64, vectorised."""
    kmax = len(pk) - 1
    ks = rng.choice(kmax + 1, size=size, p=pk)
    # a uniformly random k-subset = the k smallest of iid uniform keys
    occ_rank = np.argsort(np.argsort(rng.random((size, n_e)), axis=1), axis=1)
    vir_rank = np.argsort(np.argsort(rng.random((size, n_orb - n_e)), axis=1), axis=1)
    keep_occ = occ_rank >= ks[:, None]          # orbitals that stay occupied
    add_vir = vir_rank < ks[:, None]            # particles
    occ_w = (np.uint64(1) << np.arange(n_e, dtype=np.uint64))
    vir_w = (np.uint64(1) << np.arange(n_e, n_orb, dtype=np.uint64))
    v = (keep_occ.astype(np.uint64) * occ_w).sum(axis=1, dtype=np.uint64)
    v = v | (add_vir.astype(np.uint64) * vir_w).sum(axis=1, dtype=np.uint64)
    return v


def _pk(n_orb, n_e, ratio):
    kmax = min(n_e, n_orb - n_e)
    pk = ratio ** np.arange(kmax + 1)
    return pk / pk.sum()


def hf_weighted_strings(n_orb: int, n_e: int, count: int, seed: int, ratio: float = 0.3):
    """`count` unique strings, HF-weighted, in first-draw order, as uint64."""
    total = comb(n_orb, n_e)
    if count > total:
        raise ValueError(f"only {total} strings exist for n_orb={n_orb}, n_e={n_e}")
    rng = np.random.default_rng(seed)
    pk = _pk(n_orb, n_e, ratio)
    seen: set[int] = set()
    out: list[int] = []
    # Higher ranks can hold most of the strings; keep drawing until done.
    while len(out) < count:
        for v in _draw_batch(rng, n_orb, n_e, pk, 65536).tolist():
            if v not in seen:
                seen.add(v)
                out.append(v)
                if len(out) == count:
                    break
    return np.array(out, dtype=np.uint64)


def hf_weighted_samples(n_orb: int, n_e: int, n_samples: int, seed: int, ratio: float = 0.3):
    """`n_samples` HF-weighted strings WITH duplicates (raw sampler output)."""
    rng = np.random.default_rng(seed)
    return _draw_batch(rng, n_orb, n_e, _pk(n_orb, n_e, ratio), n_samples)


def all_strings(n_orb: int, n_e: int):
    """Every string with n_e of n_orb bits set, as uint64 (combinatorial order)."""
    return np.array([_bits(c) for c in itertools.combinations(range(n_orb), n_e)],
                    dtype=np.uint64)


def random_vector(n: int, seed: int):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n)


# Named workloads (sizes and seeds of the five synthetic configurations).
WORKLOADS = {
    "fp64_small": dict(n_orb=8, n_alpha=3, n_beta=3, n_str_alpha=56, n_str_beta=56,
                       int_seed=1, str_seed_alpha=None, str_seed_beta=None),
    "precision": dict(n_orb=16, n_alpha=5, n_beta=5, n_str_alpha=2000, n_str_beta=2000,
                      int_seed=2, str_seed_alpha=20, str_seed_beta=21),
    "differentiation": dict(n_orb=20, n_alpha=7, n_beta=7, n_str_alpha=5000, n_str_beta=5000,
                            int_seed=3, str_seed_alpha=31, str_seed_beta=32),
    "large": dict(n_orb=26, n_alpha=7, n_beta=7, n_str_alpha=20000, n_str_beta=20000,
                  int_seed=5, str_seed_alpha=51, str_seed_beta=52),
}


def workload(name: str):
    """Return dict(h, eri, e_nuc, alpha, beta, n_orb, n_alpha, n_beta) for a named workload."""
    w = WORKLOADS[name]
    h, eri, e_nuc = integrals(w["n_orb"], w["int_seed"])
    if w["str_seed_alpha"] is None:
        a = all_strings(w["n_orb"], w["n_alpha"])
        b = all_strings(w["n_orb"], w["n_beta"])
    else:
        a = hf_weighted_strings(w["n_orb"], w["n_alpha"], w["n_str_alpha"], w["str_seed_alpha"])
        b = hf_weighted_strings(w["n_orb"], w["n_beta"], w["n_str_beta"], w["str_seed_beta"])
    return dict(h=h, eri=eri, e_nuc=e_nuc, alpha=a, beta=b, n_orb=w["n_orb"],
                n_alpha=w["n_alpha"], n_beta=w["n_beta"])


def bond_scan_workload(n_geom: int = 24, n_orb: int = 16, n_e: int = 5, lo: int = 500, hi: int = 4000,
                       seed: int = 4, size_seed0: int = 40):
    """The 24-geometry bond scan: list of dicts like `workload`, uneven subspaces."""
    out = []
    for k, R in enumerate(bond_scan_R(n_geom)):
        rng = np.random.default_rng(size_seed0 + k)
        na, nb = (int(x) for x in rng.integers(lo, hi + 1, size=2))
        h, eri, e_nuc = bond_scan(n_orb, float(R), seed)
        a = hf_weighted_strings(n_orb, n_e, na, 1000 + 2 * k)
        b = hf_weighted_strings(n_orb, n_e, nb, 1001 + 2 * k)
        out.append(dict(h=h, eri=eri, e_nuc=e_nuc, alpha=a, beta=b, n_orb=n_orb,
                        n_alpha=n_e, n_beta=n_e, R=float(R)))
    return out
