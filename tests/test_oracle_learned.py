"""Pins of the learned-proposal oracle and of the sparsified-powers W rule it
is compared with (CPU only).

The proposal network is not in the paper; its oracle is pinned against
hand-worked features, finite differences, Adam's closed-form first steps and
brute-force selection.  The fixed rule (sparsified powers of Sec. 4.1) is
pinned against hand-expanded Neumann terms on 1D stencils.
"""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import learned as L
from oracle.sparsified import sparsified_powers
from workloads.csc import CSC, Pattern
from workloads import patterns as pats


def _csc(M) -> CSC:
    return CSC.from_scipy(sp.csc_matrix(M))


def _tridiag(n, sub, diag, sup):
    return sp.diags([np.full(n - 1, sub), diag, np.full(n - 1, sup)], [-1, 0, 1]).tocsc()


def test_features_hand_worked():
    # A[i,i] = 2 + i, A[i+1,i] = -1, A[i,i+1] = -0.5; column 2, candidates pattern(A^2)(:,2) = rows 0..4.
    A = _csc(_tridiag(5, -1.0, 2.0 + np.arange(5.0), -0.5))
    CAND = pats.pattern_power(A, 2)
    F = L.features(A, CAND)
    lo, hi = CAND.colptr[2], CAND.colptr[3]
    assert list(CAND.rowidx[lo:hi]) == [0, 1, 2, 3, 4]
    # (A^2)(:,2) = [0.25, -3.5, 17, -9, 1]; |A(:,2)| = [0.5, 4, 1] on rows 1..3
    want = np.array([
        [0, 0, 0.0, 0.25 / 17, np.log(2 / 4), 0.0, 2 / 3, 1],
        [0, 1, 0.125, 3.5 / 17, np.log(3 / 4), 0.25, 1.0, 1],
        [1, 1, 1.0, 1.0, 0.0, 1.0, 1.0, 0],
        [0, 1, 0.25, 9 / 17, np.log(5 / 4), 0.125, 1.0, -1],
        [0, 0, 0.0, 1 / 17, np.log(6 / 4), 0.0, 2 / 3, -1],
    ])
    np.testing.assert_allclose(F[lo:hi], want, rtol=1e-14, atol=1e-15)


def test_features_log_clamp_and_complex():
    # |a_cc| / |a_jj| = e^12 clamps at 10; complex entries enter through their modulus
    M = sp.csc_matrix(np.array([[np.exp(12.0), 1j], [3 + 4j, 1.0]]))
    A = _csc(M)
    CAND = pats.pattern_of(A)
    F = L.features(A, CAND)
    # column 1: candidates 0, 1; a_00 / a_11 = e^12 -> clamp 10
    assert F[CAND.colptr[1]][4] == 10.0
    # column 0: candidate 1 has |A_10| = 5, column max e^12; |A_01| / |a_00| = 1 / e^12
    f = F[CAND.colptr[0] + 1]
    np.testing.assert_allclose(f[2], 5 / np.exp(12.0), rtol=1e-14)
    np.testing.assert_allclose(f[5], 1 / np.exp(12.0), rtol=1e-14)


def test_grad_matches_central_differences():
    g = np.random.default_rng(3)
    theta = g.normal(0, 0.5, L.NPARAM)
    X = g.normal(0, 1, (64, L.NFEAT))
    t = g.normal(0, 1, 64)
    f0, gr = L.grad(theta, X, t)
    assert abs(f0 - L.loss(theta, X, t)) < 1e-14
    h = 1e-6
    idx = g.choice(L.NPARAM, 120, replace=False)
    for i in idx:
        e = np.zeros(L.NPARAM)
        e[i] = h
        fd = (L.loss(theta + e, X, t) - L.loss(theta - e, X, t)) / (2 * h)
        assert abs(fd - gr[i]) <= 1e-6 * max(1.0, abs(gr[i])), (i, fd, gr[i])


def test_grad_zero_at_exact_fit():
    # a target equal to the network's own output gives zero loss and gradient
    g = np.random.default_rng(4)
    theta = g.normal(0, 0.5, L.NPARAM)
    X = g.normal(0, 1, (16, L.NFEAT))
    y, _ = L.forward(theta, X)
    f, gr = L.grad(theta, X, y)
    assert f == 0.0 and np.all(gr == 0.0)


def test_adam_constant_gradient_steps():
    # with a constant gradient g, mhat = g and vhat = g^2 at every step, so
    # each step moves by exactly lr * g / (|g| + eps)
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    theta = np.zeros(4)
    m = np.zeros(4)
    v = np.zeros(4)
    lr = 0.01
    for step in range(1, 6):
        new, m, v = L.adam_step(theta, g, m, v, step, lr)
        np.testing.assert_allclose(new - theta, -lr * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-18)
        theta = new


def test_adam_minimises_quadratic():
    theta = np.array([2.0, -3.0])
    m = np.zeros(2)
    v = np.zeros(2)
    for step in range(1, 3001):
        theta, m, v = L.adam_step(theta, 2 * theta, m, v, step, 0.05)
    assert np.all(np.abs(theta) < 1e-2)


def test_select_matches_brute_force():
    g = np.random.default_rng(5)
    n = 9
    M = (g.random((n, n)) < 0.5) | np.eye(n, dtype=bool)
    P = Pattern(n, *(lambda S: (S.indptr.astype(np.int32), S.indices.astype(np.int32)))(
        sp.csc_matrix(M.astype(float))))
    score = g.normal(0, 1, P.nnz)
    for keep in (1, 2, 4, 9):
        cp, ri = L.select(P, score, keep)
        for j in range(n):
            cand = list(P.rowidx[P.colptr[j]:P.colptr[j + 1]])
            sc = dict(zip(cand, score[P.colptr[j]:P.colptr[j + 1]]))
            k = min(keep, len(cand))
            best = max((s for s in itertools.combinations(cand, k) if j in s),
                       key=lambda s: sum(sc[c] for c in s if c != j))
            assert list(ri[cp[j]:cp[j + 1]]) == sorted(best)


def test_select_ties_and_nan():
    # one 4x4 column block: column 0 candidates 0..3, scores tie on rows 2, 3; NaN on row 1
    P = Pattern(4, np.array([0, 4, 5, 6, 7], np.int32), np.array([0, 1, 2, 3, 1, 2, 3], np.int32))
    score = np.array([-5.0, np.nan, 1.0, 1.0, 0, 0, 0])
    cp, ri = L.select(P, score, 2)
    assert list(ri[cp[0]:cp[1]]) == [0, 2]      # diagonal, then the lower row of the tie
    cp, ri = L.select(P, score, 4)
    assert list(ri[cp[0]:cp[1]]) == [0, 1, 2, 3]  # NaN ranks last but is kept when everything is


def test_neumann_pattern_1d_expansion():
    # A = tridiag(-1.5, 2, -0.5): S e_j = 0.25 e_{j-1} + 0.75 e_{j+1},
    # S^2 e_j = 0.0625 e_{j-2} + 0.375 e_j + 0.5625 e_{j+2};
    # s_j = 1.375 e_j + 0.25 e_{j-1} + 0.75 e_{j+1} + 0.0625 e_{j-2} + 0.5625 e_{j+2}
    A = _csc(_tridiag(9, -1.5, np.full(9, 2.0), -0.5))
    full = sparsified_powers(A, k=2)
    np.testing.assert_array_equal(full.colptr, pats.pattern_power(A, 2).colptr)
    np.testing.assert_array_equal(full.rowidx, pats.pattern_power(A, 2).rowidx)
    j = 4
    P3 = sparsified_powers(A, k=2, keep=3)
    assert list(P3.col(j)) == [4, 5, 6]
    P4 = sparsified_powers(A, k=2, keep=4)
    assert list(P4.col(j)) == [3, 4, 5, 6]
    # dropping by count inside the expansion: t_1 keeps only e_{j+1}, so
    # t_2 = S e_{j+1} = 0.25 e_j + 0.75 e_{j+2}; e_{j-1}, e_{j-2} never appear
    Pd = sparsified_powers(A, k=2, p_l=1)
    assert list(Pd.col(j)) == [4, 5, 6]


def test_neumann_pattern_keeps_diagonal():
    A = _csc(_tridiag(6, -3.0, np.full(6, 0.1), -3.0))  # tiny diagonal: off-diagonal terms dominate
    P = sparsified_powers(A, k=2, keep=1)
    for j in range(6):
        assert list(P.col(j)) == [j]


def test_sparsified_powers_matches_dense_series():
    # without dropping, the structure is that of I + S + S^2 (dense, no cancellation on random values)
    g = np.random.default_rng(21)
    M = sp.random(30, 30, density=0.08, random_state=21, format="csc")
    M.data = g.normal(size=M.data.size)
    M = (M + sp.identity(30) * 3.0).tocsc()
    A = _csc(M)
    P = sparsified_powers(A, k=2)
    D = np.diag(M.diagonal())
    S = -np.linalg.solve(D, M.toarray() - D)
    Wd = np.eye(30) + S + S @ S
    for j in range(30):
        want = np.nonzero(np.abs(Wd[:, j]) > 1e-14)[0]
        assert list(P.col(j)) == list(want)


def test_toggle_targets_hand_worked():
    # three columns, candidates {0,1}, {0,1,2}, {1,2}; slot 1 toggles (0,1)->row 1,
    # (1,1)->row 1 is the diagonal (skipped), (2,1)->row 2 is the diagonal (skipped);
    # slot 0 toggles row 0 of column 1 and row 1 of column 2
    CAND = Pattern(3, np.array([0, 2, 5, 7], dtype=np.int32), np.array([0, 1, 0, 1, 2, 1, 2], dtype=np.int32))
    in_base = np.array([1, 1, 0, 1, 1, 1, 1], dtype=bool)
    r0 = np.array([1.0, 2.0, np.inf])  # M = 4: lo = 4e-30, hi = 4e30
    rt = np.array([2.0, 1.0, 3.0])
    v = np.full(7, np.nan)
    L.toggle_targets_slot(CAND, in_base, r0, rt, 1, 8.0, v)
    # column 0, row 1 (in the base): dropping it doubled the residual: +log 4
    assert v[1] == pytest.approx(np.log(4.0), rel=1e-15)
    assert np.isnan(v[[0, 2, 3, 4, 5, 6]]).all()
    L.toggle_targets_slot(CAND, in_base, r0, rt, 0, 8.0, v)
    # column 1, row 0 (not in the base): adding it halved the residual: +log 4
    assert v[2] == pytest.approx(np.log(4.0), rel=1e-15)
    # column 2, row 1 (in the base): r0 = inf counts as hi = 4e30, rt = 3:
    # log 9 - log 4e30 = -67.9..., clipped to -8
    assert v[5] == -8.0
    assert np.isnan(v[[0, 3, 4, 6]]).all()
    # column 0 slot 0 is the diagonal: untouched
    assert np.isnan(v[0])


def test_toggle_targets_scale_invariant():
    from workloads import operators as ops
    A = ops.lognormal3d(5, seed=2)
    CAND = pats.pattern_power(A, 2)
    g = np.random.default_rng(4)
    in_base = g.random(CAND.nnz) < 0.5
    r0 = g.lognormal(0, 1, A.n)
    rt = r0 * g.lognormal(0, 0.5, A.n)
    for slot in range(6):
        v1 = L.toggle_targets_slot(CAND, in_base, r0, rt, slot, 8.0, np.full(CAND.nnz, np.nan))
        v2 = L.toggle_targets_slot(CAND, in_base, 1e3 * r0, 1e3 * rt, slot, 8.0, np.full(CAND.nnz, np.nan))
        np.testing.assert_allclose(v1, v2, rtol=1e-12, atol=1e-12)
        e = CAND.colptr[:-1] + slot
        ok = (e < CAND.colptr[1:])
        ok[ok] &= CAND.rowidx[e[ok]] != np.arange(A.n)[ok]
        assert np.isfinite(v1[e[ok]]).all() and (np.abs(v1[e[ok]]) <= 8.0).all()


def test_scaled_residuals_definition():
    res = np.array([1.0, 2.0, 3.0])
    Vcp = np.array([0, 1, 3, 4])
    Vri = np.array([0, 0, 1, 0])
    Vv = np.array([-2.0, 5.0, 4.0, 7.0])
    out = L.scaled_residuals(res, Vcp, Vri, Vv)
    assert out[0] == 0.5 and out[1] == 0.5 and out[2] == np.inf  # column 2 has no diagonal entry
