"""Pins of the stabilised DIAF-Q (Sec. 3.2) in the oracle, CPU only.

Independent restatement with LAPACK (numpy QR / SVD / lstsq) of the paper's
construction: impose v_jj = r, take v_hat = e^{i theta} z with z the top
right singular vector of M_hat (the columns of M_j = Q(I_j,:)^* other than
j) and theta the argument of the first component of U_hat^* p; then w_j
from eq. condwj.  The result does not depend on the phases of Q's columns or
of the singular vectors, so the comparison is direct.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from workloads.csc import CSC, Pattern


def _random_problem(n, density, seed, cplx):
    g = np.random.default_rng(seed)
    M = sp.random(n, n, density=density, random_state=seed, format="csc")
    M.data = g.normal(size=M.data.size) + (1j * g.normal(size=M.data.size) if cplx else 0)
    M = M + sp.identity(n) * (0.3 + 0j if cplx else 0.3)
    A = CSC.from_scipy(M)
    PW = Pattern(n, A.colptr.copy(), A.rowidx.copy())
    # fixed V pattern: diagonal plus up to three other rows of the tile, so I_j is known
    rows, cols = [], []
    for j in range(n):
        tile_rows = np.unique(np.concatenate([A.col(c) for c in PW.col(j)]))
        others = tile_rows[tile_rows != j]
        pick = g.choice(others, size=min(3, others.size), replace=False) if others.size else []
        for i in sorted(set([j, *pick])):
            rows.append(i)
            cols.append(j)
    Vf = sp.csc_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    Vf.sort_indices()
    V = Pattern(n, Vf.indptr.astype(np.int32), Vf.indices.astype(np.int32))
    return A, PW, V


def _lapack_stabilised(A, PW, V, j, r):
    """(w, v) of the stabilised DIAF-Q for column j from numpy's LAPACK."""
    Ad = A.to_scipy().toarray()
    J = PW.col(j)
    T_full = Ad[:, J]
    Rj = np.nonzero(np.any(T_full != 0, axis=1))[0]
    T = T_full[Rj]
    Q, _ = np.linalg.qr(T)
    I = V.col(j)
    QI = np.array([Q[np.searchsorted(Rj, i)] if i in Rj else np.zeros(len(J)) for i in I])
    M = QI.conj().T                                   # k x l
    jp = int(np.nonzero(I == j)[0][0])
    Mh = np.delete(M, jp, axis=1)
    U, s, Vh = np.linalg.svd(Mh, full_matrices=False)
    z = Vh[0].conj()                                  # top right singular vector of M_hat
    pt = U[:, 0].conj() @ M[:, jp]                    # first component of U_hat^* p
    eth = pt / abs(pt) if abs(pt) > 0 else 1.0
    v = np.zeros(len(I), dtype=complex)
    v[jp] = r
    v[np.arange(len(I)) != jp] = eth * z
    v /= np.linalg.norm(v)
    b = np.zeros(T_full.shape[0], dtype=complex)
    b[I] = v
    w = np.linalg.lstsq(T_full, b, rcond=None)[0]     # eq. condwj: least squares over W's column
    return w, v, s


@pytest.mark.parametrize("cplx", [False, True])
def test_stabilised_matches_lapack_restatement(cplx):
    A, PW, V = _random_problem(40, 0.08, 7 if cplx else 3, cplx)
    o = O.factor(A, PW, O.RULE_FIXED, None, V, alg="Q", stab_tol=2.0, stab_r=2.0)  # every column stabilised
    checked = 0
    for j in range(A.n):
        I = V.col(j)
        if I.size < 2:
            continue
        assert o.flags[j] & O.F_STABILISED
        w, v, s = _lapack_stabilised(A, PW, V, j, 2.0)
        np.testing.assert_array_equal(o.I(j), I)
        # the residual is unique even where z or theta is not
        r = A.to_scipy()[:, PW.col(j)] @ w
        r[I] -= v
        assert abs(np.linalg.norm(r) - o.res[j]) <= 1e-10 * max(1.0, o.res[j])
        if o.flags[j] & O.F_DEGENERATE:
            continue  # z or theta not unique (p orthogonal to U_hat(:,1): any theta will do)
        np.testing.assert_allclose(o.v(j), v, atol=1e-12)
        np.testing.assert_allclose(o.w(j), w, atol=1e-10 * max(1, np.abs(w).max()))
        checked += 1
    assert checked > 15


def test_stabilised_vjj_and_norm_and_residual_bound():
    A, PW, V = _random_problem(60, 0.06, 11, False)
    plain = O.factor(A, PW, O.RULE_FIXED, None, V, alg="Q")
    r = 2.0
    stab = O.factor(A, PW, O.RULE_FIXED, None, V, alg="Q", stab_tol=2.0, stab_r=r)
    for j in range(A.n):
        v = stab.v(j)
        if v.size < 2:
            assert not stab.flags[j] & O.F_STABILISED
            continue
        jp = int(np.nonzero(stab.I(j) == j)[0][0])
        assert abs(v[jp] - r / np.sqrt(r * r + 1)) < 1e-14      # v_jj imposed (then unit norm)
        assert abs(np.linalg.norm(v) - 1) < 1e-13
        # the unconstrained v of eq. nocond minimises the residual, so imposing v_jj cannot lower it
        assert stab.res[j] >= plain.res[j] * (1 - 1e-12) - 1e-14


def test_trigger_threshold():
    A, PW, V = _random_problem(60, 0.06, 5, True)
    plain = O.factor(A, PW, O.RULE_FIXED, None, V, alg="Q")
    vjj = np.array([abs(plain.v(j)[plain.I(j) == j][0]) for j in range(A.n)])
    tol = float(np.median(vjj))
    stab = O.factor(A, PW, O.RULE_FIXED, None, V, alg="Q", stab_tol=tol)
    lcount = np.diff(plain.voff)
    want = (vjj < tol) & (lcount > 1)
    got = (stab.flags & O.F_STABILISED) != 0
    np.testing.assert_array_equal(got, want)
    # untouched columns are the plain solution
    for j in np.nonzero(~want)[0]:
        np.testing.assert_array_equal(stab.v(j), plain.v(j))
    off = O.factor(A, PW, O.RULE_FIXED, None, V, alg="Q", stab_tol=0.0)
    assert not np.any(off.flags & O.F_STABILISED)


def test_theta_maximises_over_the_phase():
    # ||M (r e_j + e^{i phi} z)|| is largest at the chosen phase (paper: the maximiser in the SVD basis)
    A, PW, V = _random_problem(30, 0.1, 13, True)
    r = 2.0
    for j in range(A.n):
        if V.col(j).size < 3:
            continue
        w, v, s = _lapack_stabilised(A, PW, V, j, r)
        Ad = A.to_scipy().toarray()
        Jc = PW.col(j)
        T_full = Ad[:, Jc]
        Rj = np.nonzero(np.any(T_full != 0, axis=1))[0]
        Q, _ = np.linalg.qr(T_full[Rj])
        I = V.col(j)
        QI = np.array([Q[np.searchsorted(Rj, i)] if i in Rj else np.zeros(len(Jc)) for i in I])
        jp = int(np.nonzero(I == j)[0][0])
        base = v * np.sqrt(r * r + 1)
        zhat = np.delete(base, jp)
        best = np.linalg.norm(QI.conj().T @ base)
        for phi in np.linspace(0, 2 * np.pi, 73):
            u = base.copy()
            u[np.arange(len(I)) != jp] = np.exp(1j * phi) * zhat
            assert np.linalg.norm(QI.conj().T @ u) <= best * (1 + 1e-12)
        break
