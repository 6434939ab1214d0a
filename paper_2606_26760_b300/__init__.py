"""HI-NQS subspace diagonalisation on B300: thin Python binding of libhinqs.so.

Every step of the hot path runs in the library's CUDA kernels; this module only
marshals arguments (torch tensors provide device memory and the current CUDA
stream).  There is no CPU fallback: if the library is not built, or no CUDA
device is present, the calls raise.

Names follow the C ABI in include/hinqs.h:
    Hamiltonian            hinqs_ham_create      (Sec. 2.2 Hamiltonian)
    build_subspace         hinqs_build_subspace  (Step 1 dedupe, Sec. 2.1 filter, Step 3 SQD product)
    string_links           hinqs_string_links    (Slater-Condon connectivity, Eq. classical_expansion)
    diag                   hinqs_diag            (H_xx of Step 2)
    sigma                  hinqs_sigma           (projected H applied, Step 3)
    davidson               hinqs_davidson        (Step 3 Davidson)
    rdm / energy_backward  hinqs_rdm / hinqs_energy_backward (Hellmann-Feynman gradient)
    spin_marginals         hinqs_spin_marginals  (Step 4, Eqs. alpha_marginal / beta_marginal)
    HinqsEnergy            torch.autograd.Function: E(h, eri) with the RDM backward
    pt2_score, top_amplitudes, classical_expansion   (Step 2 Eq. pt2_score, Step 1')
    candidate_pool, determinant_diag, select_top, basis_update, lookup_determinants,
    remap_vector           the outer loop's Steps 1, 2 and the Step 3 warm start
    nqs_loss / NqsLoss     Step 4 loss inputs (Eqs. teacher, energy, entropy, loss)
The outer iteration itself (Steps 1-5) is loop.HiNqsLoop.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field
from math import comb

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhinqs.so")

OK, NOT_CONVERGED = 0, 1
ERR_ARG, ERR_PARTICLE_NUMBER, ERR_ASYMMETRIC, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_EMPTY = (
    -1, -2, -3, -4, -5, -6, -7)
DROP_BAD, ERROR_BAD, FULL_SPACE = 0x0, 0x1, 0x2
CHECK_SYMMETRY = 0x1
PREC_FP64, PREC_FP32, PREC_FP32_BF16AB, PREC_FP32_BF16X3AB, PREC_FP32_BF16C, PREC_FP64_DFAB = (
    0, 1, 2, 3, 4, 5)
DAVIDSON_FP64, DAVIDSON_MIXED = 0, 1
BASIS_COLD_START, BASIS_RESCORE, BASIS_APPEND = 0, 1, 2


class HinqsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"hinqs error {code}: {msg}")
        self.code = code


_lib = None
# outputs up to this many entries are sized by their upper bound and filled in one
# call; above it a counting call sizes them first (the work is then done twice)
_ONE_PASS_CAP = 1 << 26


class _Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("max_subspace", ctypes.c_int), ("tol_residual", ctypes.c_double),
                ("tol_energy", ctypes.c_double), ("denom_floor", ctypes.c_double),
                ("inner_tol", ctypes.c_double), ("trace_cap", ctypes.c_int),
                ("trace_theta", ctypes.POINTER(ctypes.c_double)),
                ("trace_resid", ctypes.POINTER(ctypes.c_double)),
                ("trace_time", ctypes.POINTER(ctypes.c_double)),
                ("trace_kind", ctypes.POINTER(ctypes.c_int)),
                ("inner_precision", ctypes.c_int), ("restart_keep", ctypes.c_int),
                ("refine_precision", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int),
                ("n_sigma_fp64", ctypes.c_int), ("n_sigma_fp32", ctypes.c_int),
                ("n_restarts", ctypes.c_int), ("n_refinements", ctypes.c_int),
                ("trace_len", ctypes.c_int), ("energy", ctypes.c_double),
                ("residual", ctypes.c_double), ("seconds", ctypes.c_double)]


EXPORTED = [
    "hinqs_last_error_message", "hinqs_version", "hinqs_ham_create", "hinqs_ham_destroy",
    "hinqs_build_subspace", "hinqs_subspace_dims", "hinqs_subspace_strings",
    "hinqs_subspace_destroy", "hinqs_string_links", "hinqs_links_count", "hinqs_links_export",
    "hinqs_links_destroy", "hinqs_diag", "hinqs_sigma", "hinqs_davidson_default_opts",
    "hinqs_davidson", "hinqs_rdm", "hinqs_energy_backward", "hinqs_spin_marginals",
    "hinqs_spin_marginals_noalloc", "hinqs_sigma_same_spin", "hinqs_sigma_opposite_spin",
    "hinqs_links_max_singles", "hinqs_autotune", "hinqs_davidson_batch", "hinqs_links_tuning",
    "hinqs_pt2_score", "hinqs_top_amplitudes", "hinqs_classical_expansion",
    "hinqs_select_top", "hinqs_determinant_diag", "hinqs_lookup_determinants",
    "hinqs_candidate_pool", "hinqs_basis_update", "hinqs_remap_vector", "hinqs_nqs_loss",
    "hinqs_sigma_workspace_size", "hinqs_davidson_workspace_size", "hinqs_selftest_bounded_wait",
    "hinqs_selftest_projected_eig",
    "hinqs_probe_fma_rate", "hinqs_detlist_create", "hinqs_detlist_size",
    "hinqs_detlist_positions", "hinqs_detlist_destroy", "hinqs_detlist_scatter",
    "hinqs_detlist_gather", "hinqs_diag_list", "hinqs_sigma_list", "hinqs_davidson_list",
    "hinqs_classical_expansion_list", "hinqs_links_set_tuning", "hinqs_sigma_batch",
]


def load_library(path: str = LIB_PATH):
    """Load libhinqs.so (no compute; works without a GPU)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is not built: run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    PP = ctypes.POINTER(ctypes.c_void_p)
    PI64 = ctypes.POINTER(ctypes.c_int64)
    lib.hinqs_last_error_message.restype = ctypes.c_char_p
    lib.hinqs_version.restype = ctypes.c_char_p
    lib.hinqs_ham_create.argtypes = [P, P, I, I, I, D, I, PP, P]
    lib.hinqs_ham_destroy.argtypes = [P]
    lib.hinqs_build_subspace.argtypes = [P, I64, P, I64, I, I, I, I, PP, PI64, P]
    lib.hinqs_subspace_dims.argtypes = [P, PI64, PI64]
    lib.hinqs_subspace_strings.argtypes = [P, P, P, P]
    lib.hinqs_subspace_destroy.argtypes = [P]
    lib.hinqs_string_links.argtypes = [P, P, I, PP, P]
    lib.hinqs_links_count.argtypes = [P, PI64, PI64, PI64]
    lib.hinqs_links_export.argtypes = [P, P, P, P, P, P, P, P, P, P, P]
    lib.hinqs_links_destroy.argtypes = [P]
    lib.hinqs_links_max_singles.argtypes = [P]
    lib.hinqs_links_tuning.argtypes = [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int)]
    lib.hinqs_diag.argtypes = [P, P, P, P, P, P]
    lib.hinqs_sigma.argtypes = [P, P, P, P, P, P, I, P]
    lib.hinqs_sigma_same_spin.argtypes = [P, P, P, P, P, P, I, P]
    lib.hinqs_sigma_opposite_spin.argtypes = [P, P, P, P, P, P, I, P]
    lib.hinqs_davidson_default_opts.argtypes = [ctypes.POINTER(_Opts)]
    lib.hinqs_davidson_default_opts.restype = None
    lib.hinqs_davidson.argtypes = [P, P, P, P, P, ctypes.POINTER(_Opts),
                                   ctypes.POINTER(ctypes.c_double), P, ctypes.POINTER(_Info), P]
    lib.hinqs_autotune.argtypes = [P, P, P, P, I, ctypes.POINTER(ctypes.c_double), P]
    lib.hinqs_davidson_batch.argtypes = [I, P, P, P, P, P, ctypes.POINTER(_Opts), I, I, P, P,
                                         P, P]
    lib.hinqs_rdm.argtypes = [P, P, P, P, P, P, P]
    lib.hinqs_pt2_score.argtypes = [P, P, P, D, P, P, I64, P, P, P, P]
    lib.hinqs_top_amplitudes.argtypes = [P, P, I64, P, P]
    lib.hinqs_classical_expansion.argtypes = [P, P, P, I64, P, P, I64, PI64, P]
    lib.hinqs_select_top.argtypes = [P, I64, I64, I, P, P]
    lib.hinqs_determinant_diag.argtypes = [P, P, P, I64, P, P]
    lib.hinqs_lookup_determinants.argtypes = [P, P, P, I64, P, P]
    lib.hinqs_candidate_pool.argtypes = [P, P, P, I64, P, P, I64, P, P, I64, P, P, I64, PI64,
                                         PI64, P]
    lib.hinqs_basis_update.argtypes = [I, P, P, P, I64, P, P, P, I64, I64, I64, P, P, P, I64,
                                       PI64, P]
    lib.hinqs_remap_vector.argtypes = [P, P, P, P, ctypes.POINTER(ctypes.c_double), P]
    lib.hinqs_nqs_loss.argtypes = [P, P, P, P, P, P, D, P, I64, P, I64, P,
                                   ctypes.POINTER(ctypes.c_double), P, P, P, P, P]
    lib.hinqs_sigma_workspace_size.argtypes = [I64, I64, I, ctypes.POINTER(ctypes.c_size_t)]
    lib.hinqs_davidson_workspace_size.argtypes = [I64, I64, ctypes.POINTER(_Opts),
                                                  ctypes.POINTER(ctypes.c_size_t)]
    lib.hinqs_selftest_bounded_wait.argtypes = [ctypes.c_longlong, P]
    lib.hinqs_selftest_projected_eig.argtypes = [P, P, I, P, P, P, P]
    lib.hinqs_probe_fma_rate.argtypes = [I, ctypes.POINTER(ctypes.c_double), P]
    lib.hinqs_detlist_create.argtypes = [P, P, P, I64, PP, P]
    lib.hinqs_detlist_size.argtypes = [P, PI64]
    lib.hinqs_detlist_positions.argtypes = [P, P, P]
    lib.hinqs_detlist_destroy.argtypes = [P]
    lib.hinqs_detlist_scatter.argtypes = [P, P, P, P]
    lib.hinqs_detlist_gather.argtypes = [P, P, P, P]
    lib.hinqs_diag_list.argtypes = [P, P, P, P, P, P, P]
    lib.hinqs_sigma_list.argtypes = [P, P, P, P, P, P, P, I, P]
    lib.hinqs_davidson_list.argtypes = [P, P, P, P, P, P, ctypes.POINTER(_Opts),
                                        ctypes.POINTER(ctypes.c_double), P, ctypes.POINTER(_Info),
                                        P]
    lib.hinqs_classical_expansion_list.argtypes = [P, P, P, P, I64, P, P, I64, PI64, P]
    lib.hinqs_links_set_tuning.argtypes = [P, P, I, I, I]
    lib.hinqs_sigma_batch.argtypes = [I, P, P, P, P, P, P, I, P]
    lib.hinqs_energy_backward.argtypes = [I, D, P, P, P, P, P]
    lib.hinqs_spin_marginals.argtypes = [P, P, P, P, P, P]
    lib.hinqs_spin_marginals_noalloc.argtypes = [P, P, P, P, P, P]
    _lib = lib
    return lib


def _check(rc, allow_warning=False):
    if rc == OK or (allow_warning and rc > 0):
        return rc
    raise HinqsError(rc, _lib.hinqs_last_error_message().decode())


def _dev():
    if not torch.cuda.is_available():
        raise RuntimeError("hinqs needs a CUDA device; there is no CPU fallback")
    return torch.device("cuda", torch.cuda.current_device())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _on_dev(x, dtype):
    dev = _dev()
    if isinstance(x, torch.Tensor):
        return x.to(device=dev, dtype=dtype).contiguous()
    import numpy as np
    return torch.from_numpy(np.ascontiguousarray(x)).to(device=dev, dtype=dtype)


def _u64(x):
    import numpy as np
    if isinstance(x, torch.Tensor):
        return x.to(device=_dev()).contiguous()
    a = np.ascontiguousarray(np.asarray(x, dtype=np.uint64)).view(np.int64)
    return torch.from_numpy(a).to(_dev())


class Hamiltonian:
    """Prepared integrals (device copies): h[n,n], eri[n,n,n,n] chemist order."""

    def __init__(self, h, eri, n_alpha: int, n_beta: int, e_nuc: float = 0.0,
                 check_symmetry: bool = False):
        lib = load_library()
        self.h = _on_dev(h, torch.float64)
        self.eri = _on_dev(eri, torch.float64)
        self.n = int(self.h.shape[0])
        self.n_alpha, self.n_beta, self.e_nuc = int(n_alpha), int(n_beta), float(e_nuc)
        out = ctypes.c_void_p()
        _check(lib.hinqs_ham_create(_ptr(self.h), _ptr(self.eri), self.n, self.n_alpha,
                                    self.n_beta, self.e_nuc, CHECK_SYMMETRY if check_symmetry else 0,
                                    ctypes.byref(out), _stream()))
        self.handle = out

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.hinqs_ham_destroy(self.handle)
            self.handle = None


class Subspace:
    def __init__(self, handle, n, n_alpha, n_beta, dropped):
        self.handle = handle
        self.n, self.n_alpha, self.n_beta = n, n_alpha, n_beta
        na, nb = ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.hinqs_subspace_dims(handle, ctypes.byref(na), ctypes.byref(nb)))
        self.Na, self.Nb = na.value, nb.value
        self.N = self.Na * self.Nb
        self.dropped = dropped

    def strings(self):
        a = torch.empty(self.Na, dtype=torch.int64, device=_dev())
        b = torch.empty(self.Nb, dtype=torch.int64, device=_dev())
        _check(_lib.hinqs_subspace_strings(self.handle, _ptr(a), _ptr(b), _stream()))
        return a, b

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.hinqs_subspace_destroy(self.handle)
            self.handle = None


def build_subspace(alpha, beta, n_orb: int, n_alpha: int, n_beta: int, flags: int = DROP_BAD):
    """SQD product subspace from sampled strings (uint64 bitmasks)."""
    lib = load_library()
    _dev()
    a = _u64(alpha) if alpha is not None else None
    b = _u64(beta) if beta is not None else None
    out = ctypes.c_void_p()
    dropped = (ctypes.c_int64 * 2)()
    _check(lib.hinqs_build_subspace(_ptr(a), 0 if a is None else a.numel(), _ptr(b),
                                    0 if b is None else b.numel(), n_orb, n_alpha, n_beta, flags,
                                    ctypes.byref(out), dropped, _stream()))
    return Subspace(out, n_orb, n_alpha, n_beta, (dropped[0], dropped[1]))


class Links:
    def __init__(self, handle, spin, sub):
        self.handle, self.spin, self._sub = handle, spin, sub
        nl, ns, mr = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.hinqs_links_count(handle, ctypes.byref(nl), ctypes.byref(ns), ctypes.byref(mr)))
        self.n_links, self.n_singles, self.max_row = nl.value, ns.value, mr.value
        self.max_srow = _lib.hinqs_links_max_singles(handle)

    def tuning(self):
        """(rows per warp, CUDA-core chunk, tensor-core stages) chosen by autotune (0 = default)."""
        r, c, st = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(_lib.hinqs_links_tuning(self.handle, ctypes.byref(r), ctypes.byref(c), ctypes.byref(st)))
        return r.value, c.value, st.value

    def export(self):
        dev = _dev()
        N = self._sub.Nb if self.spin else self._sub.Na
        m = self.n_links
        out = dict(row_ptr=torch.empty(N + 1, dtype=torch.int64, device=dev),
                   col=torch.empty(m, dtype=torch.int32, device=dev),
                   degree=torch.empty(m, dtype=torch.int8, device=dev),
                   p=torch.empty(m, dtype=torch.uint8, device=dev),
                   q=torch.empty(m, dtype=torch.uint8, device=dev),
                   r=torch.empty(m, dtype=torch.uint8, device=dev),
                   s=torch.empty(m, dtype=torch.uint8, device=dev),
                   sign=torch.empty(m, dtype=torch.int8, device=dev),
                   hval=torch.empty(m, dtype=torch.float64, device=dev))
        _check(_lib.hinqs_links_export(self.handle, *(_ptr(out[k]) for k in (
            "row_ptr", "col", "degree", "p", "q", "r", "s", "sign", "hval")), _stream()))
        return out

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.hinqs_links_destroy(self.handle)
            self.handle = None


def string_links(ham: Hamiltonian, sub: Subspace, spin: int) -> Links:
    out = ctypes.c_void_p()
    _check(_lib.hinqs_string_links(ham.handle, sub.handle, spin, ctypes.byref(out), _stream()))
    return Links(out, spin, sub)


def set_tuning(la, lb, rows_per_warp: int = 0, chunk: int = 0, stages: int = 0):
    """hinqs_links_set_tuning: pin the sigma tiles of (la, lb) without timing them."""
    _check(_lib.hinqs_links_set_tuning(la.handle, lb.handle, int(rows_per_warp), int(chunk),
                                       int(stages)))


def diag(ham, sub, la, lb, out=None):
    out = torch.empty(sub.N, dtype=torch.float64, device=_dev()) if out is None else out
    _check(_lib.hinqs_diag(ham.handle, sub.handle, la.handle, lb.handle, _ptr(out), _stream()))
    return out


def sigma(ham, sub, la, lb, c, out=None, precision: int | None = None):
    """sigma = H_B c; precision from c's dtype (float64 -> FP64, float32 -> FP32) unless
    given (the tensor-core modes take float32 vectors)."""
    if precision is None:
        precision = PREC_FP64 if c.dtype == torch.float64 else PREC_FP32
    dt = _vec_dtype(precision)
    if c.dtype != dt or not c.is_cuda or not c.is_contiguous():
        raise ValueError(f"c must be a contiguous CUDA {dt} tensor")
    if c.numel() != sub.N:
        raise ValueError(f"c has {c.numel()} elements, subspace has {sub.N}")
    out = torch.empty_like(c) if out is None else out
    _check(_lib.hinqs_sigma(ham.handle, sub.handle, la.handle, lb.handle, _ptr(c), _ptr(out),
                            precision, _stream()))
    return out


def sigma_batch(problems, cs, precision: int | None = None, outs=None):
    """hinqs_sigma_batch: [H_g c_g] for problems [(ham, sub, la, lb), ...] in one call."""
    G = len(problems)
    if G == 0:
        return []
    if precision is None:
        precision = PREC_FP64 if cs[0].dtype == torch.float64 else PREC_FP32
    dt = _vec_dtype(precision)
    for c, p in zip(cs, problems):
        if c.dtype != dt or not c.is_cuda or not c.is_contiguous() or c.numel() != p[1].N:
            raise ValueError(f"each c must be a contiguous CUDA {dt} tensor of its subspace size")
    outs = [torch.empty_like(c) for c in cs] if outs is None else outs
    VP = ctypes.c_void_p * G
    _check(_lib.hinqs_sigma_batch(G, VP(*[p[0].handle for p in problems]),
                                  VP(*[p[1].handle for p in problems]),
                                  VP(*[p[2].handle for p in problems]),
                                  VP(*[p[3].handle for p in problems]),
                                  VP(*[c.data_ptr() for c in cs]), VP(*[o.data_ptr() for o in outs]),
                                  precision, _stream()))
    return outs


def sigma_part(ham, sub, la, lb, c, out, part: str, precision: int | None = None):
    """part = "same" (overwrites out) or "opposite" (adds into out); see hinqs.h."""
    if precision is None:
        precision = PREC_FP64 if c.dtype == torch.float64 else PREC_FP32
    fn = _lib.hinqs_sigma_same_spin if part == "same" else _lib.hinqs_sigma_opposite_spin
    _check(fn(ham.handle, sub.handle, la.handle, lb.handle, _ptr(c), _ptr(out), precision, _stream()))
    return out


@dataclass
class DavidsonResult:
    energy: float
    c: torch.Tensor
    status: int
    iterations: int
    n_sigma_fp64: int
    n_sigma_fp32: int
    n_restarts: int
    n_refinements: int
    residual: float
    seconds: float
    trace: dict = field(default_factory=dict)


def _vec_dtype(precision):
    """Vector dtype of a sigma precision: float64 for the FP64 modes, else float32."""
    return torch.float64 if precision in (PREC_FP64, PREC_FP64_DFAB) else torch.float32


def _make_opts(precision, max_iter, max_subspace, tol_residual, tol_energy, denom_floor, inner_tol,
               inner_precision, restart_keep=0, refine_precision=None):
    opts = _Opts()
    _lib.hinqs_davidson_default_opts(ctypes.byref(opts))
    opts.precision, opts.max_iter, opts.max_subspace = precision, max_iter, max_subspace
    opts.tol_residual, opts.tol_energy, opts.denom_floor = tol_residual, tol_energy, denom_floor
    opts.inner_tol = inner_tol
    opts.inner_precision = inner_precision
    opts.restart_keep = restart_keep
    if refine_precision is not None:
        opts.refine_precision = refine_precision
    return opts


def _davidson_call(fn, args, n, guess, precision, max_iter, max_subspace, tol_residual,
                   tol_energy, denom_floor, inner_tol, trace_cap, inner_precision, out,
                   restart_keep=0, refine_precision=None):
    opts = _make_opts(precision, max_iter, max_subspace, tol_residual, tol_energy, denom_floor,
                      inner_tol, inner_precision, restart_keep, refine_precision)
    bufs = None
    if trace_cap > 0:
        bufs = ((ctypes.c_double * trace_cap)(), (ctypes.c_double * trace_cap)(),
                (ctypes.c_double * trace_cap)(), (ctypes.c_int * trace_cap)())
        opts.trace_cap = trace_cap
        opts.trace_theta = ctypes.cast(bufs[0], ctypes.POINTER(ctypes.c_double))
        opts.trace_resid = ctypes.cast(bufs[1], ctypes.POINTER(ctypes.c_double))
        opts.trace_time = ctypes.cast(bufs[2], ctypes.POINTER(ctypes.c_double))
        opts.trace_kind = ctypes.cast(bufs[3], ctypes.POINTER(ctypes.c_int))
    c = torch.empty(n, dtype=torch.float64, device=_dev()) if out is None else out
    if out is not None:
        _check_vec(out, n, "out")
    if guess is not None and (guess.dtype != torch.float64 or guess.numel() != n):
        raise ValueError("guess must be a float64 tensor of the subspace size")
    e = ctypes.c_double()
    info = _Info()
    rc = fn(*args, _ptr(guess), ctypes.byref(opts), ctypes.byref(e), _ptr(c), ctypes.byref(info),
            _stream())
    _check(rc, allow_warning=True)
    tr = {}
    if bufs is not None:
        k = info.trace_len
        tr = dict(theta=list(bufs[0][:k]), resid=list(bufs[1][:k]), time=list(bufs[2][:k]),
                  kind=list(bufs[3][:k]))
    return DavidsonResult(e.value, c, rc, info.iterations, info.n_sigma_fp64, info.n_sigma_fp32,
                          info.n_restarts, info.n_refinements, info.residual, info.seconds, tr)


def davidson(ham, sub, la, lb, guess=None, precision: int = DAVIDSON_FP64, max_iter: int = 200,
             max_subspace: int = 16, tol_residual: float = 1e-8, tol_energy: float = 1e-10,
             denom_floor: float = 1e-4, inner_tol: float = 1e-3, trace_cap: int = 0,
             inner_precision: int = PREC_FP32, out=None, restart_keep: int = 0,
             refine_precision: int | None = None) -> DavidsonResult:
    """hinqs_davidson: lowest eigenpair of H on the product subspace (Step 3)."""
    return _davidson_call(_lib.hinqs_davidson, (ham.handle, sub.handle, la.handle, lb.handle),
                          sub.N, guess, precision, max_iter, max_subspace, tol_residual,
                          tol_energy, denom_floor, inner_tol, trace_cap, inner_precision, out,
                          restart_keep, refine_precision)


def davidson_list(ham, sub, la, lb, lst, guess=None, precision: int = DAVIDSON_FP64,
                  max_iter: int = 200, max_subspace: int = 16, tol_residual: float = 1e-8,
                  tol_energy: float = 1e-10, denom_floor: float = 1e-4, inner_tol: float = 1e-3,
                  trace_cap: int = 0, inner_precision: int = PREC_FP32,
                  out=None, restart_keep: int = 0,
                  refine_precision: int | None = None) -> DavidsonResult:
    """hinqs_davidson_list: lowest eigenpair of H_B over the basis list `lst` (Step 3);
    the eigenvector is indexed by the list's entries."""
    return _davidson_call(_lib.hinqs_davidson_list,
                          (ham.handle, sub.handle, la.handle, lb.handle, lst.handle), lst.m,
                          guess, precision, max_iter, max_subspace, tol_residual, tol_energy,
                          denom_floor, inner_tol, trace_cap, inner_precision, out, restart_keep,
                          refine_precision)


class DetList:
    """A basis list of determinants inside a product subspace (Step 3's H_B over B)."""

    def __init__(self, handle, sub):
        self.handle, self._sub = handle, sub   # the list borrows the subspace's strings
        m = ctypes.c_int64()
        _check(_lib.hinqs_detlist_size(handle, ctypes.byref(m)))
        self.m = m.value

    def positions(self):
        """Product positions (int64, ascending) of the list entries."""
        out = torch.empty(self.m, dtype=torch.int64, device=_dev())
        _check(_lib.hinqs_detlist_positions(self.handle, _ptr(out), _stream()))
        return out

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.hinqs_detlist_destroy(self.handle)
            self.handle = None


def detlist(sub, xa, xb) -> DetList:
    """hinqs_detlist_create: the determinants (xa[k], xb[k]) of `sub` as a basis list."""
    xa, xb = _u64(xa), _u64(xb)
    if xa.numel() != xb.numel():
        raise ValueError("xa and xb must have the same length")
    out = ctypes.c_void_p()
    _check(_lib.hinqs_detlist_create(sub.handle, _ptr(xa), _ptr(xb), xa.numel(), ctypes.byref(out),
                                     _stream()))
    return DetList(out, sub)


def detlist_scatter(lst, c_list):
    """hinqs_detlist_scatter: the list vector placed in the product's indexing."""
    _check_vec(c_list, lst.m, "c_list")
    out = torch.empty(lst._sub.N, dtype=torch.float64, device=_dev())
    _check(_lib.hinqs_detlist_scatter(lst.handle, _ptr(c_list), _ptr(out), _stream()))
    return out


def detlist_gather(lst, c_product):
    """hinqs_detlist_gather: the product vector's entries at the list's positions."""
    _check_vec(c_product, lst._sub.N, "c_product")
    out = torch.empty(lst.m, dtype=torch.float64, device=_dev())
    _check(_lib.hinqs_detlist_gather(lst.handle, _ptr(c_product), _ptr(out), _stream()))
    return out


def diag_list(ham, sub, la, lb, lst):
    """hinqs_diag_list: <x_k|H|x_k> of the list entries."""
    out = torch.empty(lst.m, dtype=torch.float64, device=_dev())
    _check(_lib.hinqs_diag_list(ham.handle, sub.handle, la.handle, lb.handle, lst.handle, _ptr(out),
                                _stream()))
    return out


def sigma_list(ham, sub, la, lb, lst, c, out=None, precision: int | None = None):
    """hinqs_sigma_list: sigma = P H P c over the basis list (float64 or float32 c)."""
    if precision is None:
        precision = PREC_FP64 if c.dtype == torch.float64 else PREC_FP32
    dt = _vec_dtype(precision)
    if c.dtype != dt or not c.is_cuda or not c.is_contiguous() or c.numel() != lst.m:
        raise ValueError(f"c must be a contiguous CUDA {dt} tensor of the list's length")
    out = torch.empty_like(c) if out is None else out
    if out.dtype != dt or out.numel() != lst.m or not out.is_contiguous():
        raise ValueError("out must match c")
    _check(_lib.hinqs_sigma_list(ham.handle, sub.handle, la.handle, lb.handle, lst.handle, _ptr(c),
                                 _ptr(out), precision, _stream()))
    return out


def sigma_workspace_size(n_alpha_strings: int, n_beta_strings: int,
                         precision: int = PREC_FP64) -> int:
    """hinqs_sigma_workspace_size: device bytes one sigma product requests at its peak."""
    lib = load_library()
    b = ctypes.c_size_t()
    _check(lib.hinqs_sigma_workspace_size(int(n_alpha_strings), int(n_beta_strings), precision,
                                          ctypes.byref(b)))
    return b.value


def davidson_workspace_size(n_alpha_strings: int, n_beta_strings: int,
                            precision: int = DAVIDSON_FP64, max_subspace: int = 16,
                            restart_keep: int = 0) -> int:
    """hinqs_davidson_workspace_size: device bytes one davidson() call with these
    options requests at its peak (besides the caller's vectors and the handles)."""
    lib = load_library()
    opts = _Opts()
    lib.hinqs_davidson_default_opts(ctypes.byref(opts))
    opts.precision, opts.max_subspace, opts.restart_keep = precision, max_subspace, restart_keep
    b = ctypes.c_size_t()
    _check(lib.hinqs_davidson_workspace_size(int(n_alpha_strings), int(n_beta_strings),
                                             ctypes.byref(opts), ctypes.byref(b)))
    return b.value


def selftest_bounded_wait(polls: int = 4096) -> int:
    """hinqs_selftest_bounded_wait: run the tensor-core kernel's bounded wait on a
    barrier nothing completes; returns the status code (ERR_TIMEOUT is expected)."""
    lib = load_library()
    _dev()
    return lib.hinqs_selftest_bounded_wait(int(polls), _stream())


def selftest_projected_eig(G, S=None, want_pairs: bool = False):
    """hinqs_selftest_projected_eig: the Davidson solvers' projected eigensolver on the
    pencil (G, S) (host arrays, m x m, m <= 32).  Returns (theta, y, pairs, path); pairs
    is an m x (m + 1) array of (lambda_j, y_j) rows when asked for, else None."""
    lib = load_library()
    import numpy as np
    G = np.ascontiguousarray(G, dtype=np.float64)
    m = G.shape[0]
    Sa = None if S is None else np.ascontiguousarray(S, dtype=np.float64)
    ty = np.zeros(m + 1)
    pairs = np.zeros((m, m + 1)) if want_pairs else None
    path = ctypes.c_int(0)
    _check(lib.hinqs_selftest_projected_eig(
        G.ctypes.data, None if Sa is None else Sa.ctypes.data, m, ty.ctypes.data,
        None if pairs is None else pairs.ctypes.data, ctypes.byref(path), _stream()))
    return ty[0], ty[1:], pairs, path.value


def probe_fma_rate(precision: int = PREC_FP64) -> float:
    """hinqs_probe_fma_rate: measured FMA rate (TFLOP/s) of the FP64 or FP32 pipe."""
    lib = load_library()
    _dev()
    r = ctypes.c_double()
    _check(lib.hinqs_probe_fma_rate(int(precision), ctypes.byref(r), _stream()))
    return r.value


def write_trace_jsonl(result: "DavidsonResult", path: str, label: str = "") -> None:
    """Write a Davidson trace (davidson(..., trace_cap > 0)) as JSON lines: iteration,
    theta (incl. E_nuc), residual norm estimate, seconds since the call began, and
    whether the iterate is an FP64 one (kind 0) or an FP32 inner one (kind 1)."""
    import json
    tr = result.trace or {}
    with open(path, "w") as f:
        for i, (th, r, t, k) in enumerate(zip(tr.get("theta", []), tr.get("resid", []),
                                              tr.get("time", []), tr.get("kind", []))):
            f.write(json.dumps({"label": label, "iter": i, "theta": th, "residual": r,
                                "seconds": t, "kind": "fp64" if k == 0 else "fp32_inner"})
                    + "\n")


def autotune(ham, sub, la, lb, precision: int = PREC_FP32) -> float:
    """hinqs_autotune: time the sigma tile candidates on this problem, keep the
    fastest in la/lb; returns the milliseconds of one sigma with the choice."""
    ms = ctypes.c_double()
    _check(_lib.hinqs_autotune(ham.handle, sub.handle, la.handle, lb.handle, precision,
                               ctypes.byref(ms), _stream()))
    return ms.value


def davidson_batch(problems, guesses=None, precision: int = DAVIDSON_FP64, max_iter: int = 200,
                   max_subspace: int = 16, tol_residual: float = 1e-8, tol_energy: float = 1e-10,
                   denom_floor: float = 1e-4, inner_tol: float = 1e-3,
                   inner_precision: int = PREC_FP32, n_streams: int = 0, autotune: bool = False,
                   outs=None, refine_precision: int | None = None):
    """hinqs_davidson_batch over `problems` = [(ham, sub, la, lb), ...]: every
    geometry solved as davidson() would; n_streams <= 0 runs them in lockstep with one
    batched launch per sigma stage per round, n_streams > 0 on that many worker streams.
    Returns a list of DavidsonResult (no trace), in the order of `problems`."""
    G = len(problems)
    if G == 0:
        return []
    opts = _make_opts(precision, max_iter, max_subspace, tol_residual, tol_energy, denom_floor,
                      inner_tol, inner_precision, refine_precision=refine_precision)
    dev = _dev()
    cs = outs if outs is not None else [torch.empty(p[1].N, dtype=torch.float64, device=dev)
                                        for p in problems]
    if guesses is not None:
        for g, p in zip(guesses, problems):
            if g is not None and (g.dtype != torch.float64 or g.numel() != p[1].N):
                raise ValueError("each guess must be a float64 tensor of its subspace size")
    VP = ctypes.c_void_p * G
    hams = VP(*[p[0].handle for p in problems])
    subs = VP(*[p[1].handle for p in problems])
    las = VP(*[p[2].handle for p in problems])
    lbs = VP(*[p[3].handle for p in problems])
    gp = VP(*[(g.data_ptr() if g is not None else None) for g in guesses]) if guesses else None
    cp = VP(*[c.data_ptr() for c in cs])
    energies = (ctypes.c_double * G)()
    infos = (_Info * G)()
    rc = _lib.hinqs_davidson_batch(G, hams, subs, las, lbs, gp, ctypes.byref(opts), n_streams,
                                   1 if autotune else 0, energies, cp, infos, _stream())
    _check(rc, allow_warning=True)
    return [DavidsonResult(energies[g], cs[g], infos[g].status, infos[g].iterations,
                           infos[g].n_sigma_fp64, infos[g].n_sigma_fp32, infos[g].n_restarts,
                           infos[g].n_refinements, infos[g].residual, infos[g].seconds, {})
            for g in range(G)]


def pt2_score(ham, sub, c, e0: float, xa, xb):
    """hinqs_pt2_score (Step 2, Eq. pt2_score): (v, hxx, score) per candidate
    x = (xa[k], xb[k]); xa, xb int64/uint64 tensors or numpy uint64 arrays."""
    dev = _dev()
    xa = _u64(xa)
    xb = _u64(xb)
    if xa.numel() != xb.numel():
        raise ValueError("xa and xb must have the same length")
    if c.dtype != torch.float64 or c.numel() != sub.N:
        raise ValueError("c must be a float64 tensor of the subspace size")
    m = xa.numel()
    v = torch.empty(m, dtype=torch.float64, device=dev)
    hxx = torch.empty_like(v)
    sc = torch.empty_like(v)
    _check(_lib.hinqs_pt2_score(ham.handle, sub.handle, _ptr(c), float(e0), _ptr(xa), _ptr(xb), m,
                                _ptr(v), _ptr(hxx), _ptr(sc), _stream()))
    return v, hxx, sc


def top_amplitudes(sub, c, k: int):
    """hinqs_top_amplitudes: indices (int64, ascending) of the k largest |c|."""
    k = max(0, min(int(k), sub.N))
    out = torch.empty(k, dtype=torch.int64, device=_dev())
    _check(_lib.hinqs_top_amplitudes(sub.handle, _ptr(c), k, _ptr(out), _stream()))
    return out


def classical_expansion(ham, sub, c, n_top: int = 1000):
    """hinqs_classical_expansion (Step 1', Eq. classical_expansion): (xa, xb) int64
    tensors of the candidate strings, ascending in (alpha, beta)."""
    if c.dtype != torch.float64 or c.numel() != sub.N:
        raise ValueError("c must be a float64 tensor of the subspace size")
    cnt = ctypes.c_int64()
    # excitations enumerated per selected determinant: an upper bound on the output
    n, na, nb = sub.n, sub.n_alpha, sub.n_beta
    s1a, s1b = na * (n - na), nb * (n - nb)
    per = (s1a + s1b + comb(na, 2) * comb(n - na, 2) + comb(nb, 2) * comb(n - nb, 2)
           + s1a * s1b)
    bound = min(max(0, int(n_top)), sub.N) * per
    if bound <= _ONE_PASS_CAP:  # one call writes straight into buffers of the bound
        xa = torch.empty(bound, dtype=torch.int64, device=_dev())
        xb = torch.empty(bound, dtype=torch.int64, device=_dev())
        _check(_lib.hinqs_classical_expansion(ham.handle, sub.handle, _ptr(c), n_top, _ptr(xa),
                                              _ptr(xb), bound, ctypes.byref(cnt), _stream()))
        return xa[:cnt.value], xb[:cnt.value]
    _check(_lib.hinqs_classical_expansion(ham.handle, sub.handle, _ptr(c), n_top, None, None, 0,
                                          ctypes.byref(cnt), _stream()))
    m = cnt.value
    xa = torch.empty(m, dtype=torch.int64, device=_dev())
    xb = torch.empty(m, dtype=torch.int64, device=_dev())
    _check(_lib.hinqs_classical_expansion(ham.handle, sub.handle, _ptr(c), n_top, _ptr(xa),
                                          _ptr(xb), m, ctypes.byref(cnt), _stream()))
    return xa, xb


def classical_expansion_list(ham, sub, lst, c_list, n_top: int = 1000):
    """hinqs_classical_expansion_list (Step 1' with the basis a list): (xa, xb) of the
    determinants outside the list connected to its n_top largest |c_list| entries."""
    _check_vec(c_list, lst.m, "c_list")
    cnt = ctypes.c_int64()
    n, na, nb = sub.n, sub.n_alpha, sub.n_beta
    s1a, s1b = na * (n - na), nb * (n - nb)
    per = (s1a + s1b + comb(na, 2) * comb(n - na, 2) + comb(nb, 2) * comb(n - nb, 2)
           + s1a * s1b)
    bound = min(max(0, int(n_top)), lst.m) * per
    args = (ham.handle, sub.handle, lst.handle, _ptr(c_list), n_top)
    if bound > _ONE_PASS_CAP:
        _check(_lib.hinqs_classical_expansion_list(*args, None, None, 0, ctypes.byref(cnt),
                                                   _stream()))
        bound = cnt.value
    xa = torch.empty(bound, dtype=torch.int64, device=_dev())
    xb = torch.empty(bound, dtype=torch.int64, device=_dev())
    _check(_lib.hinqs_classical_expansion_list(*args, _ptr(xa), _ptr(xb), bound, ctypes.byref(cnt),
                                               _stream()))
    return xa[:cnt.value], xb[:cnt.value]


def _f64_dev(x, n=None, what="values"):
    t = _on_dev(x, torch.float64)
    if n is not None and t.numel() != n:
        raise ValueError(f"{what} must have {n} elements")
    return t


def select_top(values, k: int, largest: bool = True):
    """hinqs_select_top (Step 2 ranking): ascending positions (int64) of the k largest
    (or smallest) values, ties to the lower position."""
    lib = load_library()
    v = _f64_dev(values)
    k = max(0, min(int(k), v.numel()))
    out = torch.empty(k, dtype=torch.int64, device=_dev())
    _check(lib.hinqs_select_top(_ptr(v), v.numel(), k, 1 if largest else 0, _ptr(out), _stream()))
    return out


def determinant_diag(ham, xa, xb):
    """hinqs_determinant_diag: H_xx (incl. E_nuc) of arbitrary determinants."""
    xa, xb = _u64(xa), _u64(xb)
    if xa.numel() != xb.numel():
        raise ValueError("xa and xb must have the same length")
    out = torch.empty(xa.numel(), dtype=torch.float64, device=_dev())
    _check(_lib.hinqs_determinant_diag(ham.handle, _ptr(xa), _ptr(xb), xa.numel(), _ptr(out),
                                       _stream()))
    return out


def lookup_determinants(sub, xa, xb):
    """hinqs_lookup_determinants: product-subspace position of each determinant, or -1."""
    xa, xb = _u64(xa), _u64(xb)
    if xa.numel() != xb.numel():
        raise ValueError("xa and xb must have the same length")
    out = torch.empty(xa.numel(), dtype=torch.int64, device=_dev())
    _check(_lib.hinqs_lookup_determinants(sub.handle, _ptr(xa), _ptr(xb), xa.numel(), _ptr(out),
                                          _stream()))
    return out


def candidate_pool(ham, first, second=None, exclude=None):
    """hinqs_candidate_pool (Steps 1, 1'): distinct determinants of the proposal lists
    `first` and `second` ((xa, xb) pairs) with the sector's electron counts, minus the
    `exclude` list; returns (ya, yb, n_dropped), ascending in (alpha, beta)."""
    def pair(p):
        if p is None:
            return None, None, 0
        a, b = _u64(p[0]), _u64(p[1])
        if a.numel() != b.numel():
            raise ValueError("alpha and beta lists must have the same length")
        return a, b, a.numel()
    a1, b1, m1 = pair(first)
    a2, b2, m2 = pair(second)
    ea, eb, me = pair(exclude)
    cnt, drop = ctypes.c_int64(), ctypes.c_int64()
    args = (ham.handle, _ptr(a1), _ptr(b1), m1, _ptr(a2), _ptr(b2), m2, _ptr(ea), _ptr(eb), me)
    if m1 + m2 <= _ONE_PASS_CAP:  # the pool holds at most m1 + m2 candidates: one call
        ya = torch.empty(m1 + m2, dtype=torch.int64, device=_dev())
        yb = torch.empty(m1 + m2, dtype=torch.int64, device=_dev())
        _check(_lib.hinqs_candidate_pool(*args, _ptr(ya), _ptr(yb), m1 + m2, ctypes.byref(cnt),
                                         ctypes.byref(drop), _stream()))
        return ya[:cnt.value], yb[:cnt.value], drop.value
    _check(_lib.hinqs_candidate_pool(*args, None, None, 0, ctypes.byref(cnt), ctypes.byref(drop),
                                     _stream()))
    m = cnt.value
    ya = torch.empty(m, dtype=torch.int64, device=_dev())
    yb = torch.empty(m, dtype=torch.int64, device=_dev())
    _check(_lib.hinqs_candidate_pool(*args, _ptr(ya), _ptr(yb), m, ctypes.byref(cnt),
                                     ctypes.byref(drop), _stream()))
    return ya, yb, drop.value


def basis_update(mode: int, basis, cand, k: int, b_max: int = 0):
    """hinqs_basis_update (Step 2): basis and cand are (xa, xb, key) triples (basis may
    be None); returns the new basis (xa, xb, key)."""
    lib = load_library()

    def triple(t):
        if t is None:
            return None, None, None, 0
        a, b, v = _u64(t[0]), _u64(t[1]), _f64_dev(t[2])
        if not (a.numel() == b.numel() == v.numel()):
            raise ValueError("determinant lists and keys must have the same length")
        return a, b, v, a.numel()
    ba, bb, bs, nb = triple(basis)
    ca, cb, cs, nc = triple(cand)
    k = max(0, int(k))
    if mode == BASIS_COLD_START:
        cap = min(k, nc)
    elif mode == BASIS_RESCORE:
        cap = min(k, nb + nc)
    else:
        cap = nb + min(k, nc)
        if b_max > 0:
            cap = min(cap, int(b_max))
    dev = _dev()
    oa = torch.empty(cap, dtype=torch.int64, device=dev)
    ob = torch.empty(cap, dtype=torch.int64, device=dev)
    os_ = torch.empty(cap, dtype=torch.float64, device=dev)
    n_out = ctypes.c_int64()
    _check(lib.hinqs_basis_update(int(mode), _ptr(ba), _ptr(bb), _ptr(bs), nb, _ptr(ca), _ptr(cb),
                                   _ptr(cs), nc, k, int(b_max), _ptr(oa), _ptr(ob), _ptr(os_), cap,
                                   ctypes.byref(n_out), _stream()))
    n = n_out.value
    return oa[:n], ob[:n], os_[:n]


def remap_vector(old_sub, c_old, new_sub):
    """hinqs_remap_vector (Step 3 warm start): (c_new, |c_new|^2)."""
    if c_old.dtype != torch.float64 or c_old.numel() != old_sub.N:
        raise ValueError("c_old must be a float64 tensor of the old subspace size")
    c_new = torch.empty(new_sub.N, dtype=torch.float64, device=_dev())
    kept = ctypes.c_double()
    _check(_lib.hinqs_remap_vector(old_sub.handle, _ptr(c_old), new_sub.handle, _ptr(c_new),
                                   ctypes.byref(kept), _stream()))
    return c_new, kept.value


def nqs_loss(ham, sub, la, lb, p_alpha, p_beta, e0: float, batch, log_pi, coef=(1.0, 1.0, 1.0),
             basis=None):
    """hinqs_nqs_loss (Step 4): dict(w, adv, grad, loss) for the minibatch `batch`
    (product-subspace positions); loss = [total, teacher, energy, entropy]."""
    dev = _dev()
    batch = _on_dev(batch, torch.int64)
    lp = _f64_dev(log_pi, batch.numel(), "log_pi")
    bas = None if basis is None else _on_dev(basis, torch.int64)
    m = batch.numel()
    w = torch.empty(m, dtype=torch.float64, device=dev)
    adv, grad = torch.empty_like(w), torch.empty_like(w)
    loss = torch.empty(4, dtype=torch.float64, device=dev)
    cf = (ctypes.c_double * 3)(*[float(x) for x in coef])
    _check(_lib.hinqs_nqs_loss(ham.handle, sub.handle, la.handle, lb.handle, _ptr(p_alpha),
                               _ptr(p_beta), float(e0), _ptr(bas), 0 if bas is None else bas.numel(),
                               _ptr(batch), m, _ptr(lp), cf, _ptr(w), _ptr(adv), _ptr(grad),
                               _ptr(loss), _stream()))
    return dict(w=w, adv=adv, grad=grad, loss=loss)


class NqsLoss(torch.autograd.Function):
    """L_total of Step 4 (Eq. loss) as a function of the network's log-probabilities
    on a minibatch; the backward multiplies the library's d L_total / d log pi."""

    @staticmethod
    def forward(ctx, log_pi, ham, sub, la, lb, p_alpha, p_beta, e0, batch, coef, basis):
        r = nqs_loss(ham, sub, la, lb, p_alpha, p_beta, e0, batch, log_pi.detach(), coef, basis)
        ctx.save_for_backward(r["grad"])
        return r["loss"][0].to(log_pi.dtype)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return (g * grad).to(g.dtype), None, None, None, None, None, None, None, None, None, None


def rdm(sub, la, lb, c, want2: bool = True):
    n = sub.n
    g1 = torch.empty((n, n), dtype=torch.float64, device=_dev())
    g2 = torch.empty((n, n, n, n), dtype=torch.float64, device=_dev()) if want2 else None
    _check(_lib.hinqs_rdm(sub.handle, la.handle, lb.handle, _ptr(c), _ptr(g1), _ptr(g2), _stream()))
    return g1, g2


def energy_backward(n_orb, grad_E, rdm1, rdm2):
    gh = torch.empty_like(rdm1)
    ge = torch.empty_like(rdm2) if rdm2 is not None else None
    _check(_lib.hinqs_energy_backward(n_orb, float(grad_E), _ptr(rdm1), _ptr(rdm2), _ptr(gh),
                                      _ptr(ge), _stream()))
    return gh, ge


def _check_vec(t, n, what):
    """A caller-owned FP64 buffer the kernels read or write n elements of: float64,
    contiguous, on the current device and at least n long (a short or mistyped
    buffer would be written past its end on the device)."""
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{what} must be a torch tensor")
    if t.dtype != torch.float64:
        raise ValueError(f"{what} must be float64, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if t.device != _dev():
        raise ValueError(f"{what} must be on {_dev()}, got {t.device}")
    if t.numel() < n:
        raise ValueError(f"{what} holds {t.numel()} elements, needs {n}")


def spin_marginals(sub, c, want_w: bool = False):
    _check_vec(c, sub.N, "c")
    pa = torch.empty(sub.Na, dtype=torch.float64, device=_dev())
    pb = torch.empty(sub.Nb, dtype=torch.float64, device=_dev())
    w = torch.empty(sub.N, dtype=torch.float64, device=_dev()) if want_w else None
    _check(_lib.hinqs_spin_marginals(sub.handle, _ptr(c), _ptr(pa), _ptr(pb), _ptr(w), _stream()))
    return (pa, pb, w) if want_w else (pa, pb)


def spin_marginals_noalloc(sub, c, p_alpha, p_beta, w=None):
    """hinqs_spin_marginals_noalloc: the library allocates nothing (its scratch is a
    fixed 8 MiB device array); the caller provides every output buffer."""
    _check_vec(c, sub.N, "c")
    _check_vec(p_alpha, sub.Na, "p_alpha")
    _check_vec(p_beta, sub.Nb, "p_beta")
    if w is not None:
        _check_vec(w, sub.N, "w")
    _check(_lib.hinqs_spin_marginals_noalloc(sub.handle, _ptr(c), _ptr(p_alpha), _ptr(p_beta),
                                             _ptr(w), _stream()))
    return p_alpha, p_beta, w


class HinqsEnergy(torch.autograd.Function):
    """E0(h, eri) of the projected Hamiltonian (Step 3) with the Hellmann-Feynman
    backward dE/dh = gamma, dE/d(pq|rs) = Gamma/2 (entrywise)."""

    @staticmethod
    def forward(ctx, h, eri, sub, n_alpha, n_beta, e_nuc, opts):
        ham = Hamiltonian(h.detach(), eri.detach(), n_alpha, n_beta, e_nuc)
        la, lb = string_links(ham, sub, 0), string_links(ham, sub, 1)
        res = davidson(ham, sub, la, lb, **(opts or {}))
        ctx.sub, ctx.la, ctx.lb, ctx.c, ctx.n = sub, la, lb, res.c, ham.n
        ctx.ham = ham
        return torch.tensor(res.energy, dtype=torch.float64, device=h.device)

    @staticmethod
    def backward(ctx, grad_E):
        g1, g2 = rdm(ctx.sub, ctx.la, ctx.lb, ctx.c, want2=ctx.needs_input_grad[1])
        gh, ge = energy_backward(ctx.n, float(grad_E), g1, g2)
        return gh, ge, None, None, None, None, None


def energy(h, eri, sub, n_alpha, n_beta, e_nuc=0.0, **opts):
    return HinqsEnergy.apply(h, eri, sub, n_alpha, n_beta, e_nuc, opts)
