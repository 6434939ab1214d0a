"""The HI-NQS outer iteration (Sec. 2.2, Steps 1-5) around the subspace solve.

Orchestration only: every step below is one call of the CUDA library (the binding in
this package); this module decides which call comes next.

    Step 1   the NQS samples of iteration t arrive as (x_alpha, x_beta) device arrays
             (the Transformer sampler itself is not part of this library)
    Step 1'  t >= 1: classical singles/doubles expansion of the n_top largest |c_i|
             (Eq. classical_expansion)                       hinqs_classical_expansion
             candidate set C_t: distinct, particle-number filtered, minus the basis
                                                             hinqs_candidate_pool
    Step 2   t = 0: the K_0 candidates with the lowest H_xx  hinqs_determinant_diag
             t = 1: PT2 rescoring of basis and candidates, the top K, no cap
             t >= 2: PT2 scores of the candidates, the top K appended, eviction
             above B_max (Eq. pt2_score)                     hinqs_pt2_score,
                                                             hinqs_basis_update
    Step 3   Davidson on H_B over the basis list itself (mode "list", as Step 3
             states: [H_B]_ij = <x_i|H|x_j>), or on the product of the basis strings
             (mode "product", the SQD form); warm-started from the previous
             eigenvector carried over                        hinqs_build_subspace,
                                                             hinqs_detlist_create,
                                                             hinqs_remap_vector,
                                                             hinqs_davidson_list /
                                                             hinqs_davidson
    Step 4   teacher marginals and the loss inputs for the network
                                                             hinqs_spin_marginals,
                                                             hinqs_nqs_loss
    Step 5   stop after `patience` consecutive |E(t) - E(t-1)| < delta, or max_iter
"""
from __future__ import annotations

import dataclasses
import json
from dataclasses import dataclass, field

import numpy as np
import torch

from . import (BASIS_APPEND, BASIS_COLD_START, BASIS_RESCORE, DAVIDSON_FP64, Hamiltonian,
               basis_update, build_subspace, candidate_pool, classical_expansion,
               classical_expansion_list, davidson, davidson_list, detlist, detlist_gather,
               detlist_scatter, determinant_diag, lookup_determinants, nqs_loss, pt2_score,
               remap_vector, spin_marginals, string_links)


@dataclass
class IterationRecord:
    t: int
    n_candidates: int        # |C_t|
    n_dropped: int           # proposals rejected by the particle-number filter
    n_basis: int             # |B| after the update
    n_alpha_strings: int
    n_beta_strings: int
    energy: float
    residual: float
    davidson_status: int
    warm_start: bool


@dataclass
class HiNqsLoop:
    """State of the outer iteration.  `ham` is a prepared Hamiltonian; k0, k and b_max
    are the cold-start budget K_0, the per-iteration budget K and the cap B_max of
    Step 2; n_top is N_e of Step 1' (the paper uses 1000).  mode "list" diagonalises
    H_B over the basis list (Step 3; B_max then bounds the solve), "product" over the
    product of the list's distinct strings (which contains the list).  `c` is always
    the eigenvector in the product's indexing (zero outside the list in list mode);
    `c_list` is the list eigenvector in list mode."""

    ham: Hamiltonian
    k0: int
    k: int
    b_max: int
    n_top: int = 1000
    delta: float = 1e-9
    patience: int = 5
    max_iter: int = 50
    davidson_opts: dict = field(default_factory=lambda: dict(precision=DAVIDSON_FP64,
                                                             tol_residual=1e-8,
                                                             tol_energy=1e-11, max_iter=400))
    mode: str = "list"
    t: int = 0
    basis: tuple | None = None          # (x_alpha, x_beta, key) of the cumulative basis
    lst: object = None                  # the basis list inside `sub` (list mode)
    c_list: torch.Tensor | None = None  # eigenvector over the list entries (list mode)
    sub: object = None
    la: object = None
    lb: object = None
    c: torch.Tensor | None = None
    energy: float | None = None
    energies: list = field(default_factory=list)
    history: list = field(default_factory=list)
    # inputs of the last step (for inspection and checking)
    last: dict = field(default_factory=dict)

    def step(self, samples):
        """One iteration: candidates from `samples` (and the classical expansion),
        basis update, subspace solve.  Returns the IterationRecord."""
        ham = self.ham
        last = dict(t=self.t, samples=samples, basis_before=self.basis, sub_before=self.sub,
                    c_before=self.c, c_list_before=self.c_list, energy_before=self.energy)
        if self.t == 0:
            ya, yb, dropped = candidate_pool(ham, samples)
            hxx = determinant_diag(ham, ya, yb)
            last.update(pool=(ya, yb), expansion=None, keys=hxx)
            self.basis = basis_update(BASIS_COLD_START, None, (ya, yb, hxx), self.k0)
        else:
            if self.mode == "list":
                xa_cl, xb_cl = classical_expansion_list(ham, self.sub, self.lst, self.c_list,
                                                        self.n_top)
            else:
                xa_cl, xb_cl = classical_expansion(ham, self.sub, self.c, self.n_top)
            ya, yb, dropped = candidate_pool(ham, samples, (xa_cl, xb_cl),
                                             exclude=self.basis[:2])
            _, _, sc = pt2_score(ham, self.sub, self.c, self.energy, ya, yb)
            last.update(pool=(ya, yb), expansion=(xa_cl, xb_cl), keys=sc)
            if self.t == 1:
                # every cold-start entry gets one PT2 evaluation before any eviction
                _, _, sb = pt2_score(ham, self.sub, self.c, self.energy, self.basis[0],
                                     self.basis[1])
                last.update(basis_keys=sb)
                self.basis = basis_update(BASIS_RESCORE, (self.basis[0], self.basis[1], sb),
                                          (ya, yb, sc), self.k)
            else:
                self.basis = basis_update(BASIS_APPEND, self.basis, (ya, yb, sc), self.k,
                                          self.b_max)
        sub = build_subspace(self.basis[0], self.basis[1], ham.n, ham.n_alpha, ham.n_beta)
        la, lb = string_links(ham, sub, 0), string_links(ham, sub, 1)
        guess, warm = None, False
        if self.c is not None:
            g, kept = remap_vector(self.sub, self.c, sub)
            if kept > 0.0:
                guess, warm = g, True
        if self.mode == "list":
            lst = detlist(sub, self.basis[0], self.basis[1])
            if guess is not None:
                guess = detlist_gather(lst, guess)
                if float(torch.dot(guess, guess)) == 0.0:
                    guess, warm = None, False
            res = davidson_list(ham, sub, la, lb, lst, guess=guess, **self.davidson_opts)
            self.lst, self.c_list = lst, res.c
            c_prod = detlist_scatter(lst, res.c)
        else:
            res = davidson(ham, sub, la, lb, guess=guess, **self.davidson_opts)
            c_prod = res.c
        self.sub, self.la, self.lb, self.c, self.energy = sub, la, lb, c_prod, res.energy
        self.energies.append(res.energy)
        rec = IterationRecord(self.t, int(ya.numel()), int(dropped), int(self.basis[0].numel()),
                              sub.Na, sub.Nb, res.energy, res.residual, res.status, warm)
        self.history.append(rec)
        self.last = last
        self.t += 1
        return rec

    def converged(self) -> bool:
        """Step 5: `patience` consecutive energy changes below delta, or max_iter."""
        e = self.energies
        if len(e) >= self.max_iter:
            return True
        if len(e) <= self.patience:
            return False
        return all(abs(e[-i] - e[-i - 1]) < self.delta for i in range(1, self.patience + 1))

    def run(self, sampler):
        """Iterate until converged(); sampler(t) gives the Step 1 samples of iteration t."""
        while not self.converged():
            self.step(sampler(self.t))
        return self.history

    # ------------------------------------------------------ checkpoint / resume
    # The only state the paper carries across iterations is the basis and the
    # eigenvector that warm-starts the next solve (Step 3); a checkpoint holds those,
    # the energies (for the Step 5 rule) and the budgets, as host arrays in one .npz.

    def save(self, path: str) -> None:
        """Write the loop state (basis list with keys, subspace strings, eigenvector,
        energies, iteration count, budgets) to `path` (numpy .npz)."""
        st = dict(mode=np.array(self.mode), t=np.int64(self.t), k0=np.int64(self.k0), k=np.int64(self.k),
                  b_max=np.int64(self.b_max), n_top=np.int64(self.n_top),
                  delta=np.float64(self.delta), patience=np.int64(self.patience),
                  max_iter=np.int64(self.max_iter),
                  energies=np.asarray(self.energies, dtype=np.float64),
                  history=np.array(json.dumps([dataclasses.asdict(r) for r in self.history])))
        if self.basis is not None:
            st["basis_alpha"] = self.basis[0].cpu().numpy()
            st["basis_beta"] = self.basis[1].cpu().numpy()
            st["basis_key"] = self.basis[2].cpu().numpy()
        if self.sub is not None:
            sa, sb = self.sub.strings()
            st["sub_alpha"], st["sub_beta"] = sa.cpu().numpy(), sb.cpu().numpy()
            st["c"] = self.c.cpu().numpy()
            st["energy"] = np.float64(self.energy)
        with open(path, "wb") as f:
            np.savez(f, **st)

    @classmethod
    def load(cls, path: str, ham, davidson_opts: dict | None = None, rebuild: bool = True):
        """Resume from a checkpoint written by save().  With rebuild the product
        subspace and its links are built again on the device and the eigenvector is
        put back, so the next step warm-starts from it; without rebuild only the host
        state is restored (the basis, energies and counters, as device-free tensors)."""
        z = np.load(path)
        kw = dict(k0=int(z["k0"]), k=int(z["k"]), b_max=int(z["b_max"]), n_top=int(z["n_top"]),
                  delta=float(z["delta"]), patience=int(z["patience"]),
                  max_iter=int(z["max_iter"]))
        if davidson_opts is not None:
            kw["davidson_opts"] = davidson_opts
        if "mode" in z:
            kw["mode"] = str(z["mode"])
        loop = cls(ham, **kw)
        loop.t = int(z["t"])
        loop.energies = [float(x) for x in z["energies"]]
        loop.history = [IterationRecord(**r) for r in json.loads(str(z["history"]))]
        dev = torch.device("cuda", torch.cuda.current_device()) if rebuild else torch.device("cpu")
        if "basis_alpha" in z:
            loop.basis = (torch.from_numpy(z["basis_alpha"]).to(dev),
                          torch.from_numpy(z["basis_beta"]).to(dev),
                          torch.from_numpy(z["basis_key"]).to(dev))
        if "sub_alpha" in z:
            loop.energy = float(z["energy"])
            if rebuild:
                loop.sub = build_subspace(torch.from_numpy(z["sub_alpha"]).to(dev),
                                          torch.from_numpy(z["sub_beta"]).to(dev),
                                          ham.n, ham.n_alpha, ham.n_beta)
                loop.la, loop.lb = string_links(ham, loop.sub, 0), string_links(ham, loop.sub, 1)
                loop.c = torch.from_numpy(z["c"]).to(dev)
                if loop.mode == "list":
                    loop.lst = detlist(loop.sub, loop.basis[0], loop.basis[1])
                    loop.c_list = detlist_gather(loop.lst, loop.c)
            else:
                loop.c = torch.from_numpy(z["c"])
        return loop

    def write_history_jsonl(self, path: str) -> None:
        """One JSON line per iteration (IterationRecord fields): the per-iteration
        energy and basis size that Step 5 and the paper's convergence plots use."""
        with open(path, "w") as f:
            for r in self.history:
                f.write(json.dumps(dataclasses.asdict(r)) + "\n")

    def basis_positions(self):
        """Positions of the basis-list determinants in the current product subspace."""
        return lookup_determinants(self.sub, self.basis[0], self.basis[1])

    def teacher(self, batch, log_pi, coef=(1.0, 1.0, 1.0), over_list: bool = True):
        """Step 4 on a minibatch of basis positions: dict(w, adv, grad, loss) from
        hinqs_nqs_loss, with the teacher weights normalised over the basis list
        (over_list) or over the whole product subspace."""
        pa, pb = spin_marginals(self.sub, self.c)
        basis = self.basis_positions() if over_list else None
        return nqs_loss(self.ham, self.sub, self.la, self.lb, pa, pb, self.energy, batch, log_pi,
                        coef, basis)
