"""CPU oracle of the learned W-pattern proposal -- TEST INFRASTRUCTURE ONLY.

Not part of the paper (its W-pattern rules are the heuristics of Sec. 4);
this is the plain definition of what the proposal kernels compute, in
float64 numpy, for the tests: the eight candidate features, the network
8 -> 32 -> 32 -> 1 with ReLU, the gradient of the mean squared error by
backpropagation written out per layer, one Adam step (Kingma & Ba,
"Adam: a method for stochastic optimization", 2015, Algorithm 1) and the
per-column top-k selection, and the training targets (the scaled
per-column residual and the clipped log-ratio of one toggled candidate
slot).  Shares no code with the CUDA library.

Pins (tests/test_oracle_learned.py): features of a hand-worked 1D stencil;
gradients against central finite differences; Adam's first step against
its closed form lr * g / (|g| + eps); selection against brute force; toggle
targets of a hand-worked three-column example and their invariance under a
common scaling of the residuals.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

NFEAT, HIDDEN = 8, 32
# parameter layout: W1[H][F], b1[H], W2[H][H], b2[H], w3[H], b3
_SIZES = [("W1", (HIDDEN, NFEAT)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
          ("w3", (HIDDEN,)), ("b3", ())]
NPARAM = sum(int(np.prod(s)) for _, s in _SIZES)


def unpack(theta: np.ndarray) -> dict:
    out, off = {}, 0
    for name, shape in _SIZES:
        size = int(np.prod(shape))
        out[name] = theta[off:off + size].reshape(shape)
        off += size
    return out


def pack(parts: dict) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).reshape(-1) for name, _ in _SIZES])


def features(A, CAND) -> np.ndarray:
    """[CAND.nnz, 8] features of every candidate c of every column j, in
    CAND's entry order:
      0  1 if c == j
      1  1 if A_cj != 0 (c is a row of the column)
      2  |A_cj| / max_i |A_ij|
      3  |(A^2)_cj| / max over the column's candidates |(A^2)_c'j|
      4  log(|a_cc| / |a_jj|), clamped to [-10, 10], 0 if either is zero
      5  |A_jc| / |a_jj| (0 if a_jj = 0)
      6  nnz(A(:,c)) / nnz(A(:,j))
      7  +1 if c < j, -1 if c > j, 0 if c == j"""
    M = sp.csc_matrix((A.vals, A.rowidx, A.colptr), shape=(A.n, A.n))
    M2 = (M @ M).tocsc()
    Md = M.todok() if A.n <= 4096 else None
    cnt = np.diff(A.colptr)
    diag = np.abs(M.diagonal())
    F = np.zeros((CAND.nnz, NFEAT))

    def entry(r, c):
        return abs(Md[r, c]) if Md is not None else abs(M[r, c])

    for j in range(A.n):
        rows = A.rowidx[A.colptr[j]:A.colptr[j + 1]]
        absj = np.abs(A.vals[A.colptr[j]:A.colptr[j + 1]])
        colmax = absj.max() if absj.size else 0.0
        ajj = diag[j]
        cand = CAND.rowidx[CAND.colptr[j]:CAND.colptr[j + 1]]
        a2 = np.array([abs(M2[c, j]) for c in cand])
        a2max = a2.max() if a2.size else 0.0
        for t, c in enumerate(cand):
            f = F[CAND.colptr[j] + t]
            hit = np.nonzero(rows == c)[0]
            acj = absj[hit[0]] if hit.size else 0.0
            f[0] = 1.0 if c == j else 0.0
            f[1] = 1.0 if acj > 0 else 0.0
            f[2] = acj / colmax if colmax > 0 else 0.0
            f[3] = a2[t] / a2max if a2max > 0 else 0.0
            f[4] = np.clip(np.log(diag[c] / ajj), -10, 10) if (diag[c] > 0 and ajj > 0) else 0.0
            f[5] = entry(j, c) / ajj if ajj > 0 else 0.0
            f[6] = cnt[c] / cnt[j] if cnt[j] > 0 else 0.0
            f[7] = 1.0 if c < j else (-1.0 if c > j else 0.0)
    return F


def relu(x):
    return np.maximum(x, 0.0)


def forward(theta: np.ndarray, X: np.ndarray):
    """y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3 for every row x of X;
    returns y and the layer activations (pre and post) for the backward pass."""
    p = unpack(theta)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = relu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = relu(z2)
    y = h2 @ p["w3"] + p["b3"]
    return y, (z1, h1, z2, h2)


def loss(theta, X, t) -> float:
    y, _ = forward(theta, X)
    return float(np.mean((y - t) ** 2))


def grad(theta, X, t):
    """(loss, d loss / d theta) for loss = mean_s (y_s - t_s)^2, by the chain rule
    layer by layer (the ReLU derivative is taken as 0 at 0)."""
    p = unpack(theta)
    y, (z1, h1, z2, h2) = forward(theta, X)
    N = X.shape[0]
    dy = 2.0 * (y - t) / N                       # dL/dy_s
    g = {"w3": h2.T @ dy, "b3": np.sum(dy)}
    dz2 = np.outer(dy, p["w3"]) * (z2 > 0)       # dL/dz2
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"]) * (z1 > 0)             # dL/dz1
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return float(np.mean((y - t) ** 2)), pack(g)


def adam_step(theta, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One step of Adam: biased moments, bias correction by 1 - beta^step,
    update lr * mhat / (sqrt(vhat) + eps).  Returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def select(CAND, score: np.ndarray, keep: int):
    """Per column: the diagonal (if a candidate), then the candidates by
    decreasing score, ties to the lower row, NaN last; min(keep, count) rows,
    returned sorted, as (colptr, rowidx)."""
    colptr = [0]
    rows_out = []
    for j in range(CAND.n):
        lo, hi = CAND.colptr[j], CAND.colptr[j + 1]
        cand = CAND.rowidx[lo:hi]
        sc = np.where(np.isnan(score[lo:hi]), -np.inf, score[lo:hi]).astype(np.float64)
        sc = np.where(cand == j, np.inf, sc)
        order = sorted(range(cand.size), key=lambda t: (-sc[t], cand[t]))
        kept = sorted(int(cand[t]) for t in order[:min(keep, cand.size)])
        rows_out.extend(kept)
        colptr.append(len(rows_out))
    return np.array(colptr, dtype=np.int32), np.array(rows_out, dtype=np.int32)


def scaled_residuals(res: np.ndarray, Vcp: np.ndarray, Vri: np.ndarray, Vv: np.ndarray) -> np.ndarray:
    """res_j / |V(j,j)| per column (inf when V(j,j) is zero or absent)."""
    n = res.size
    out = np.full(n, np.inf)
    for j in range(n):
        for p in range(Vcp[j], Vcp[j + 1]):
            if Vri[p] == j and abs(Vv[p]) > 0:
                out[j] = res[j] / abs(Vv[p])
    return out


def toggle_targets_slot(CAND, in_base: np.ndarray, r0: np.ndarray, rt: np.ndarray, slot: int, clip: float,
                        value: np.ndarray) -> np.ndarray:
    """Targets of candidate slot `slot`: for every column j whose candidate
    list has an entry e at position `slot` other than j itself,
      value[e] = +(L(rt_j) - L(r0_j))   if the candidate is in the base pattern
      value[e] = -(L(rt_j) - L(r0_j))   otherwise,
    clipped to [-clip, clip], with L(r) = log(min(max(r^2, lo), hi)) (hi for a
    non-finite r^2), lo = 1e-30 max(M, 1e-300), hi = 1e30 M, M the largest
    finite r0_j^2 (1 when none is positive).  Other entries are unchanged."""
    sq = r0.astype(np.float64) ** 2
    ok = np.isfinite(sq) & (sq > 0)
    M = float(sq[ok].max()) if ok.any() else 1.0
    lo, hi = max(M, 1e-300) * 1e-30, 1e30 * M

    def L(r):
        v = float(r) ** 2
        return np.log(min(max(v, lo), hi)) if np.isfinite(v) else np.log(hi)

    for j in range(CAND.n):
        e = CAND.colptr[j] + slot
        if e >= CAND.colptr[j + 1] or CAND.rowidx[e] == j:
            continue
        d = L(rt[j]) - L(r0[j])
        value[e] = min(max(d if in_base[e] else -d, -clip), clip)
    return value
