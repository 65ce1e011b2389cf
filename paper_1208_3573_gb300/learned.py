"""Learned proposal of the W pattern J_j: training and inference driver.

Not in the paper: Sec. 4 builds J_j by fixed rules (powers of A, the
Neumann-series sparsified powers with dropping by count); those stay the
fallback.  Here a network scores every candidate row of a candidate pattern
CAND(:,j) -- pattern(A^2) for the 7-point operators -- and the diagonal plus
the best-scored candidates form J_j.  Every computation runs in libdiaf.so:
features (diaf_propose_features), scores (diaf_mlp_forward), the kept
pattern (diaf_propose_select), the training targets (diaf_scaled_residuals,
diaf_toggle_targets) and the training step (diaf_mlp_grad, diaf_mlp_adam).
This module only arranges the calls and builds the toggled patterns.

Training targets come from the exact columnwise solve itself.  Around a base
pattern J0 (by default the fixed rule at the same size), candidate c of
column j is toggled -- dropped when in J0, added otherwise -- for all columns
at once, one candidate slot at a time, and the change of the per-column
residual res = ||A w_j - v_j|| / |v_jj| of the FP64 solve is recorded as
  target = log(res(J0 \\ {c})^2 / res(J0)^2)      (c in J0)
  target = log(res(J0)^2 / res(J0 + {c})^2)       (c not in J0)
i.e. how much the residual of column j depends on c: larger is more useful.
The network is fitted to these values (mean squared error, Adam).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import diaf

NPARAM = diaf.PROP_NPARAM
NFEAT, HIDDEN = diaf.PROP_NFEAT, diaf.PROP_HIDDEN


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights for the ReLU layers, zero biases (float32, packed as
    W1[32][8], b1[32], W2[32][32], b2[32], w3[32], b3)."""
    g = np.random.default_rng(seed)
    W1 = g.normal(0.0, np.sqrt(2.0 / NFEAT), (HIDDEN, NFEAT))
    W2 = g.normal(0.0, np.sqrt(2.0 / HIDDEN), (HIDDEN, HIDDEN))
    w3 = g.normal(0.0, np.sqrt(1.0 / HIDDEN), HIDDEN)
    theta = np.concatenate([W1.ravel(), np.zeros(HIDDEN), W2.ravel(), np.zeros(HIDDEN), w3, [0.0]])
    assert theta.size == NPARAM
    return theta.astype(np.float32)


def _entry_keys(n: int, colptr: np.ndarray, rowidx: np.ndarray) -> np.ndarray:
    col = np.repeat(np.arange(n, dtype=np.int64), np.diff(colptr))
    return col * n + rowidx.astype(np.int64)


def _subpattern(CAND, mask: np.ndarray, device) -> diaf.DeviceCSC:
    col = np.repeat(np.arange(CAND.n), np.diff(CAND.colptr))
    cnt = np.bincount(col[mask], minlength=CAND.n)
    colptr = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int32)
    rowidx = CAND.rowidx[mask].astype(np.int32)
    return diaf.DeviceCSC(CAND.n, torch.from_numpy(colptr).to(device), torch.from_numpy(rowidx).to(device))


def host_pattern(P: diaf.DeviceCSC):
    """A device pattern as a host workloads.Pattern (numpy arrays)."""
    from workloads.csc import Pattern
    return Pattern(P.n, P.colptr.cpu().numpy().astype(np.int32), P.rowidx.cpu().numpy().astype(np.int32))


def fixed_rule(A_dev: diaf.DeviceCSC, keep: int, k: int = 2) -> diaf.DeviceCSC:
    """The fixed rule the proposal is compared with: sparsified powers of
    order k (Sec. 4.1) dropped by count to `keep` entries per column."""
    return diaf.sparsified_powers(A_dev, k, 0, keep)


@dataclass
class Targets:
    """Per-candidate training targets of one instance (CAND's entry order)."""

    value: torch.Tensor   # float64 [CAND.nnz] on the device; NaN on the diagonal (always kept, not trained)
    in_base: np.ndarray   # bool [CAND.nnz]
    res_base: torch.Tensor  # per-column scaled residual of J0 (device)


def scaled_residuals(F: diaf.Factors) -> np.ndarray:
    """Per column ||A w_j - v_j|| / |v_jj| (diaf_scaled_residuals; host copy,
    inf where v_jj = 0).  With a diagonal V this is the norm of column j of
    A W V^-1 - I."""
    return diaf.scaled_residuals(F).cpu().numpy()


def toggle_targets(A_dev: diaf.DeviceCSC, CAND, base, budget: torch.Tensor, vrule: int = diaf.RULE_UPPER,
                   tie_tol: float = 1e-9, clip: float = 8.0, alg: str = "S") -> Targets:
    """Targets by toggling one candidate slot of every column at a time around
    `base` (host Patterns CAND, base with base within CAND).  One FP64
    factorisation per slot, all columns at once; the per-column measure is
    ||A w_j - v_j|| / |v_jj| (scale-free: the column of A W V^-1 - I when V is
    diagonal).  The measure, the log-ratio and the clip run on the device
    (diaf_scaled_residuals, diaf_toggle_targets); the host only builds the
    toggled patterns."""
    dev = A_dev.colptr.device
    n = CAND.n
    ck = _entry_keys(n, CAND.colptr, CAND.rowidx)
    bk = _entry_keys(n, base.colptr, base.rowidx)
    in_base = np.isin(ck, bk)
    if int(in_base.sum()) != base.nnz:
        raise ValueError("the base pattern must lie within the candidate pattern")
    col = np.repeat(np.arange(n), np.diff(CAND.colptr))
    slot = np.arange(CAND.nnz) - CAND.colptr[col]
    diag = CAND.rowidx == col
    CAND_dev = diaf.DeviceCSC.from_host(CAND, dev)
    in_base_dev = torch.from_numpy(in_base.astype(np.uint8)).to(dev)

    def residual(mask):
        F = diaf.factor(A_dev, _subpattern(CAND, mask, dev), vrule, budget, alg=alg, prec="fp64", tie_tol=tie_tol)
        r = diaf.scaled_residuals(F)
        F.close()
        return r

    r0 = residual(in_base)
    value = torch.full((CAND.nnz,), float("nan"), dtype=torch.float64, device=dev)
    for t in range(int(slot.max()) + 1 if CAND.nnz else 0):
        tog = (slot == t) & ~diag
        if not tog.any():
            continue
        diaf.toggle_targets(CAND_dev, in_base_dev, r0, residual(in_base ^ tog), t, clip, value)
    return Targets(value, in_base, r0)


class Proposer:
    """The proposal network on the GPU: float32 parameters and Adam moments."""

    def __init__(self, params: np.ndarray | None = None, seed: int = 0, device="cuda"):
        p = init_params(seed) if params is None else np.asarray(params, dtype=np.float32)
        assert p.size == NPARAM
        self.device = device
        self.params = torch.from_numpy(p.copy()).to(device)
        self.m = torch.zeros(NPARAM, dtype=torch.float32, device=device)
        self.v = torch.zeros(NPARAM, dtype=torch.float32, device=device)
        self.step = 0
        self.target_scale = 1.0

    # -- inference
    def scores(self, A_dev: diaf.DeviceCSC, CAND_dev: diaf.DeviceCSC) -> torch.Tensor:
        return diaf.mlp_forward(self.params, diaf.propose_features(A_dev, CAND_dev))

    def propose(self, A_dev: diaf.DeviceCSC, CAND_dev: diaf.DeviceCSC, keep: int) -> diaf.DeviceCSC:
        """J_j for every column: the diagonal plus the keep-1 best candidates."""
        return diaf.propose_select(CAND_dev, self.scores(A_dev, CAND_dev), keep)

    # -- training
    def fit(self, feats: list[torch.Tensor], targets: list, epochs: int = 30, batch: int = 8192,
            lr: float = 3e-3, seed: int = 0) -> list[float]:
        """Adam on the mean squared error over the rows with a finite target
        (targets -- device tensors or arrays -- are rescaled to unit standard
        deviation; the ranking is unchanged).  Returns the mean training loss
        of every epoch."""
        ts = [torch.as_tensor(t, dtype=torch.float64).to(f.device) for f, t in zip(feats, targets)]
        X = torch.cat([f[torch.isfinite(t)] for f, t in zip(feats, ts)])
        y = torch.cat([t[torch.isfinite(t)] for t in ts])
        self.target_scale = float(y.std(correction=0).item()) or 1.0
        Y = (y / self.target_scale).to(torch.float32)
        N = X.shape[0]
        g = np.random.default_rng(seed)
        grad = torch.empty(NPARAM, dtype=torch.float32, device=X.device)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        hist = []
        for _ in range(epochs):
            perm = torch.from_numpy(g.permutation(N)).to(X.device)
            Xs, Ys = X[perm].contiguous(), Y[perm].contiguous()
            acc = torch.zeros(1, dtype=torch.float32, device=X.device)
            nb = 0
            for s in range(0, N, batch):
                xb, yb = Xs[s:s + batch], Ys[s:s + batch]
                diaf.mlp_grad(self.params, xb, yb, grad, loss)
                self.step += 1
                diaf.mlp_adam(self.params, grad, self.m, self.v, self.step, lr)
                acc += loss
                nb += 1
            hist.append(float(acc.item()) / max(nb, 1))
        return hist

    def save(self, path: str) -> None:
        np.savez(path, params=self.params.cpu().numpy(), target_scale=self.target_scale)

    @staticmethod
    def load(path: str, device="cuda") -> "Proposer":
        z = np.load(path)
        p = Proposer(z["params"], device=device)
        p.target_scale = float(z["target_scale"])
        return p
