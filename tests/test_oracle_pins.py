"""Pins the CPU oracle to what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms (single-index W columns), textbook special cases (sparse approximate
inverse = diagonal V, Sec. 2.1 Example and Sec. 3.2 Example exai), exact
factoring of scaled permutations (Sec. 4.2 Example teje), brute-force
optimisation over the unit sphere, LAPACK, exact rational arithmetic,
invariants (leverage sums, monotonicity in the patterns, the Frobenius
identity and the two-sided bound eqn:minbound of Sec. 3.2).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from tests._problems import dense, pattern_from_matrix, pattern_from_sets, random_sparse
from workloads import diagonal_pattern, make_workload, pattern_of, pattern_power, upper_budget

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _phase_align(a, b):
    """b scaled by the unit scalar that best aligns it with a."""
    z = np.vdot(b, a)
    return b * (z / abs(z)) if abs(z) > 0 else b


# --------------------------------------------------------------- building blocks
@pytest.mark.parametrize("shape", [(7, 3), (25, 13), (5, 5), (40, 1), (3, 6)])
@pytest.mark.parametrize("cplx", [False, True])
def test_householder_qr_vs_lapack(shape, cplx, rng):
    m, k = shape
    T = rng.standard_normal(shape) + (1j * rng.standard_normal(shape) if cplx else 0)
    Q, R = O.householder_qr(T)
    p = min(m, k)
    assert np.allclose(Q.conj().T @ Q, np.eye(p), atol=1e-13)
    assert np.allclose(np.triu(R), R)
    assert np.allclose(Q @ R[:p, :], T, atol=1e-12)
    Rl = np.linalg.qr(T, mode="r")
    assert np.allclose(np.abs(np.diag(R[:p, :p])), np.abs(np.diag(Rl[:p, :p])), rtol=1e-12)


@pytest.mark.parametrize("shape", [(13, 13), (25, 13), (4, 9), (1, 3), (60, 60)])
@pytest.mark.parametrize("cplx", [False, True])
def test_jacobi_svd_vs_lapack(shape, cplx, rng):
    G = rng.standard_normal(shape) + (1j * rng.standard_normal(shape) if cplx else 0)
    s, V, GV, sweeps = O.jacobi_svd(G)
    assert sweeps > 0
    sl = np.linalg.svd(G, compute_uv=False)
    s_sorted = np.sort(s)[::-1]
    ref = np.zeros_like(s_sorted); ref[:sl.size] = sl
    assert np.allclose(s_sorted, ref, rtol=1e-12, atol=1e-13 * sl[0])
    assert np.allclose(V.conj().T @ V, np.eye(shape[1]), atol=1e-13)
    assert np.allclose(G @ V, GV, atol=1e-12 * sl[0])
    Gram = GV.conj().T @ GV
    off = Gram - np.diag(np.diag(Gram))
    assert np.abs(off).max() <= 1e-12 * sl[0] ** 2


def test_jacobi_graded_matrix_small_singular_value():
    # one-sided Jacobi keeps relative accuracy of a tiny singular value
    D = np.diag([1.0, 1e-3, 1e-6, 1e-9])
    rng = np.random.default_rng(5)
    U, _ = np.linalg.qr(rng.standard_normal((4, 4)))
    G = U @ D
    s, *_ = O.jacobi_svd(G)
    assert np.allclose(np.sort(s), [1e-9, 1e-6, 1e-3, 1.0], rtol=1e-9)


# --------------------------------------------------------------- closed forms (k_j = 1)
@pytest.mark.parametrize("cplx", [False, True])
def test_single_index_closed_form(cplx):
    A = random_sparse(40, 0.12, 7, cplx)
    Ad = dense(A)
    PW = diagonal_pattern(A.n)
    bud = upper_budget(A)
    rS = O.factor(A, PW, O.RULE_UPPER, bud, alg="S")
    rQ = O.factor(A, PW, O.RULE_UPPER, bud, alg="Q")
    for j in range(A.n):
        a = Ad[:, j]
        rows = np.nonzero(a)[0]
        # rule: diagonal plus the (budget-1) upper rows of largest |a_ij| (leverage |a_ij|^2/||a||^2)
        cand = [i for i in rows if i < j]
        s = min(bud[j] - 1, len(cand))
        key = np.abs(a[cand]) ** 2 / np.linalg.norm(a) ** 2
        order = sorted(range(len(cand)), key=lambda t: (-key[t], cand[t]))
        I = np.sort(np.array([j] + [cand[t] for t in order[:s]], dtype=np.int32))
        assert np.array_equal(rS.I(j), I) and np.array_equal(rQ.I(j), I)
        aI = a[I]
        out = np.delete(a, I)
        ph = np.conj(a[j]) / abs(a[j])
        # DIAF-S: w = unit scalar, v = a(I) w, res = ||a outside I||
        assert np.allclose(rS.w(j), [ph], atol=1e-14)
        assert np.allclose(rS.v(j), aI * ph, rtol=1e-13)
        assert rS.res[j] == pytest.approx(np.linalg.norm(out), rel=1e-12, abs=1e-14)
        # DIAF-Q: v = a(I)/||a(I)||, w = ||a(I)|| / ||a||^2, res^2 = 1 - ||a(I)||^2/||a||^2
        nI, na = np.linalg.norm(aI), np.linalg.norm(a)
        assert np.allclose(rQ.v(j), aI / nI * ph, rtol=1e-12, atol=1e-15)
        assert np.allclose(rQ.w(j), [nI / na**2 * ph], rtol=1e-12)
        assert rQ.res[j] == pytest.approx(np.sqrt(max(0.0, 1 - nI**2 / na**2)), rel=1e-10, abs=1e-12)


def test_selection_rule_hand_example():
    """Tile with known leverage: for column 5 with J = {5} the tile is A(:,5)
    whose leverage is |a_i5|^2 / ||a_5||^2.  Rows 1 and 3 tie exactly; the
    lower row must win, and the budget caps the count."""
    n = 6
    M = np.eye(n) * 4.0
    M[0, 5], M[1, 5], M[3, 5], M[4, 5] = 1.0, 3.0, 3.0, 2.0
    A = random_sparse(n, 0.0, 0)
    A = type(A).from_scipy(sp.csc_matrix(M))
    PW = diagonal_pattern(n)
    bud = np.array([1, 1, 1, 1, 1, 3], np.int32)  # diagonal + 2 extra for column 5
    r = O.factor(A, PW, O.RULE_UPPER, bud, alg="S")
    assert list(r.I(5)) == [1, 3, 5]
    bud[5] = 2
    r = O.factor(A, PW, O.RULE_UPPER, bud, alg="S")
    assert list(r.I(5)) == [1, 5]  # tie 1 vs 3 resolved to the lower row
    bud[5] = 5
    r = O.factor(A, PW, O.RULE_UPPER, bud, alg="S")
    assert list(r.I(5)) == [0, 1, 3, 4, 5]
    r = O.factor(A, PW, O.RULE_UPPER, None, alg="S")  # no budget: all admissible
    assert list(r.I(5)) == [0, 1, 3, 4, 5]
    r = O.factor(A, PW, O.RULE_LOWER, None, alg="S")
    assert list(r.I(5)) == [5]


# --------------------------------------------------------------- special cases
@pytest.mark.parametrize("cplx", [False, True])
def test_spai_reduction(cplx):
    """V diagonal (I_j = {j}): DIAF-Q is the sparse approximate inverse column
    argmin ||A(:,J_j) w - e_j||; DIAF-S takes the smallest right singular vector
    of A(:,J_j) without row j (Sec. 2.1 Example; Sec. 3.2 Example exai)."""
    A = random_sparse(50, 0.08, 3, cplx)
    Ad = dense(A)
    PW = pattern_power(A, 2)
    D = diagonal_pattern(A.n)
    rQ = O.factor(A, PW, O.RULE_FIXED, None, D, alg="Q")
    rS = O.factor(A, PW, O.RULE_FIXED, None, D, alg="S")
    for j in range(A.n):
        J = PW.col(j)
        Aj = Ad[:, J]
        e = np.zeros(A.n, Ad.dtype); e[j] = 1
        wl, *_ = np.linalg.lstsq(Aj, e, rcond=None)
        # v_j = unit with v_jj > 0 => v_j = 1 exactly, so w_j is the SPAI column
        assert np.allclose(rQ.v(j), [1.0], atol=1e-14)
        assert np.allclose(rQ.w(j), wl, rtol=1e-9, atol=1e-12 * np.abs(wl).max())
        Ah = np.delete(Aj, j, axis=0)
        _, s, Vh = np.linalg.svd(Ah)
        assert rS.res[j] == pytest.approx(s[-1], rel=1e-10, abs=1e-13)
        wr = Vh[-1].conj()
        wo = rS.w(j)
        assert abs(abs(np.vdot(wr, wo)) - 1) < 1e-10


def test_scaled_permutation_exact():
    """A = D P with W pattern = pattern(A^*) and V diagonal gives A W V^-1 = I
    (Sec. 4.2 Example teje: A with orthogonal columns)."""
    n = 40
    rng = np.random.default_rng(11)
    perm = rng.permutation(n)
    d = rng.uniform(0.5, 3.0, n) * rng.choice([-1, 1], n)
    Ad = np.zeros((n, n)); Ad[np.arange(n), perm] = d
    A = type(random_sparse(2, 0.0, 0)).from_scipy(sp.csc_matrix(Ad))
    PW = pattern_from_matrix(sp.csc_matrix(Ad.T))
    D = diagonal_pattern(n)
    for alg in ("S", "Q"):
        r = O.factor(A, PW, O.RULE_FIXED, None, D, alg=alg)
        W = r.W_csc().toarray(); V = r.V_csc().toarray()
        assert np.allclose(Ad @ W @ np.linalg.inv(V), np.eye(n), atol=1e-13)
        assert np.all(r.res < 1e-14)


@pytest.mark.parametrize("alg", ["S", "Q"])
def test_full_I_gives_zero_residual(alg):
    """I_j containing every row of A(:,J_j) gives res_j = 0."""
    A = random_sparse(30, 0.1, 5)
    PW = pattern_of(A)
    full = pattern_from_matrix((sp.csc_matrix(np.abs(dense(A))) @ sp.csc_matrix(np.abs(dense(A)))) != 0)
    r = O.factor(A, PW, O.RULE_FIXED, None, full, alg=alg)
    assert np.all(r.res <= 1e-12 * np.abs(dense(A)).max())
    if alg == "Q":  # all singular values of M_j equal 1: degenerate exactly when k_j >= 2
        k = PW.counts()
        assert np.all((r.flags[k >= 2] & O.F_DEGENERATE) != 0)
        assert np.all((r.flags[k == 1] & O.F_DEGENERATE) == 0)


# --------------------------------------------------------------- brute force / random bounds
def _tiny_problem(cplx, seed, n=9):
    rng = np.random.default_rng(seed)
    Ad = rng.standard_normal((n, n)) * (rng.random((n, n)) < 0.45)
    if cplx:
        Ad = Ad + 1j * rng.standard_normal((n, n)) * (Ad != 0)
    Ad += 4 * np.eye(n)
    A = type(random_sparse(2, 0.0, 0)).from_scipy(sp.csc_matrix(Ad))
    sets = []
    for j in range(n):
        k = rng.integers(1, 4)
        others = rng.choice([i for i in range(n) if i != j], size=k - 1, replace=False)
        sets.append([j, *others])
    return A, Ad, pattern_from_sets(n, sets)


def _sphere_min(f, k, cplx, rng, starts=40):
    from scipy.optimize import minimize
    dim = 2 * k if cplx else k
    best = np.inf
    for _ in range(starts):
        x0 = rng.standard_normal(dim)
        r = minimize(lambda x: f(x), x0, method="BFGS", options={"gtol": 1e-12, "maxiter": 2000})
        r = minimize(lambda x: f(x), r.x, method="Nelder-Mead",
                     options={"xatol": 1e-13, "fatol": 1e-15, "maxiter": 20000})
        best = min(best, r.fun)
    return best


@pytest.mark.parametrize("cplx", [False, True])
def test_bruteforce_tiny(cplx):
    """On tiles with k_j <= 3 the oracle's objective agrees with direct
    minimisation over the unit sphere: DIAF-S min ||(I-P_I) A w||, ||w||=1;
    DIAF-Q max ||M_j v||, ||v|| = 1 (eq. nocond), residual of eq. condwj."""
    A, Ad, PW = _tiny_problem(cplx, 3)
    bud = upper_budget(A)
    rS = O.factor(A, PW, O.RULE_UPPER, bud, alg="S")
    rQ = O.factor(A, PW, O.RULE_UPPER, bud, alg="Q")
    rng = np.random.default_rng(0)
    for j in range(A.n):
        J = PW.col(j); k = J.size
        I = rS.I(j)
        assert np.array_equal(I, rQ.I(j))
        Aj = Ad[:, J]
        Ah = np.delete(Aj, I, axis=0)

        def unpack(x, k=k):
            return x[:k] + 1j * x[k:] if cplx else x

        def fS(x):
            w = unpack(x)
            return np.linalg.norm(Ah @ w) / np.linalg.norm(w)

        best = _sphere_min(fS, k, cplx, rng)
        assert rS.res[j] == pytest.approx(best, rel=1e-7, abs=1e-10)
        # DIAF-Q: residual = min_w ||A_j w - v|| maximised over unit v on I (= sqrt(1 - ||M v||^2))
        Q, _ = np.linalg.qr(Aj)
        l = I.size

        def fQ(x, l=l):
            v = x[:l] + 1j * x[l:] if cplx else x
            v = v / np.linalg.norm(v)
            return -np.linalg.norm(Q[I, :].conj().T @ v)

        sig = -_sphere_min(fQ, l, cplx, rng, starts=20)
        assert rQ.res[j] == pytest.approx(np.sqrt(max(0.0, 1 - sig**2)), rel=1e-6, abs=1e-9)


@pytest.mark.parametrize("cplx", [False, True])
def test_objective_below_random_unit_vectors(cplx):
    w_ = make_workload("convdiff32") if not cplx else make_workload("helmholtz40")
    A, PW = w_.A, w_.PW
    Ad = A.to_scipy().tocsc()
    cols = np.arange(0, A.n, 97)
    rS = O.factor(A, PW, O.RULE_UPPER, w_.budget, alg="S", cols=cols)
    rQ = O.factor(A, PW, O.RULE_UPPER, w_.budget, alg="Q", cols=cols)
    rng = np.random.default_rng(1)
    for t, j in enumerate(cols):
        J = PW.col(j)
        Aj = Ad[:, J].toarray()
        I = rS.I(t)
        Ah = np.delete(Aj, I, axis=0)
        Wr = rng.standard_normal((J.size, 1000)) + (1j * rng.standard_normal((J.size, 1000)) if cplx else 0)
        Wr /= np.linalg.norm(Wr, axis=0)
        assert rS.res[t] <= np.linalg.norm(Ah @ Wr, axis=0).min() * (1 + 1e-12)
        # DIAF-Q: for random unit v on I, min_w ||A_j w - v|| >= res_Q
        Vr = rng.standard_normal((I.size, 200)) + (1j * rng.standard_normal((I.size, 200)) if cplx else 0)
        Vr /= np.linalg.norm(Vr, axis=0)
        full = np.zeros((A.n, 200), Vr.dtype); full[I, :] = Vr
        X, *_ = np.linalg.lstsq(Aj, full, rcond=None)
        assert rQ.res[t] <= np.linalg.norm(Aj @ X - full, axis=0).min() * (1 + 1e-12)


# --------------------------------------------------------------- invariants
@pytest.mark.parametrize("alg", ["S", "Q"])
def test_monotone_in_patterns(alg):
    """Residual is non-increasing when J_j grows (I fixed) and when I_j grows
    (J fixed): a minimum over a larger set (cf. Sec. 5 Example 5.3, monotone nrm)."""
    A = random_sparse(60, 0.06, 9)
    P1 = pattern_of(A)
    P2 = pattern_power(A, 2)
    P3 = pattern_power(A, 3)
    Vd = diagonal_pattern(A.n)
    Vg = pattern_from_matrix(sp.triu(A.to_scipy()) != 0)
    Vg2 = pattern_from_matrix(sp.triu(abs(A.to_scipy()) @ abs(A.to_scipy())) != 0)
    res = {}
    for pn, P in (("1", P1), ("2", P2), ("3", P3)):
        for vn, V in (("d", Vd), ("g", Vg), ("g2", Vg2)):
            res[pn + vn] = O.factor(A, P, O.RULE_FIXED, None, V, alg=alg).res
    tol = 1e-10
    for vn in ("d", "g", "g2"):
        assert np.all(res["2" + vn] <= res["1" + vn] * (1 + tol) + 1e-9)
        assert np.all(res["3" + vn] <= res["2" + vn] * (1 + tol) + 1e-9)
    for pn in "123":
        assert np.all(res[pn + "g"] <= res[pn + "d"] * (1 + tol) + 1e-9)
        assert np.all(res[pn + "g2"] <= res[pn + "g"] * (1 + tol) + 1e-9)


@pytest.mark.parametrize("name", ["convdiff32", "helmholtz40", "powerlaw6k"])
def test_leverage_invariants(name):
    """h_i = ||Q(i,:)||^2 are the diagonal of the hat matrix T (T^* T)^-1 T^*:
    0 <= h_i <= 1 and sum_i h_i = k_j."""
    w_ = make_workload(name)
    Ad = w_.A.to_scipy().tocsc()
    for j in np.linspace(0, w_.n - 1, 25).astype(int):
        c = O.column(w_.A, w_.PW, int(j), w_.vrule, w_.budget)
        J = w_.PW.col(j)
        T = Ad[c.rows, :][:, J].toarray()
        hat = np.real(np.einsum("ij,ji->i", T, np.linalg.solve(T.conj().T @ T, T.conj().T)))
        assert np.allclose(c.h, hat, atol=1e-12)
        assert c.h.sum() == pytest.approx(J.size, rel=1e-12)
        assert c.h.min() >= -1e-15 and c.h.max() <= 1 + 1e-12


@pytest.mark.parametrize("alg", ["S", "Q"])
def test_frobenius_identity_and_minbound(alg):
    """||AW - V||_F^2 = sum_j res_j^2, and the two-sided bound eqn:minbound:
    ||AWV^-1 - I||_F / ||V^-1||_2 <= ||AW - V||_F <= ||AWV^-1 - I||_F ||V||_2."""
    w_ = make_workload("convdiff32")
    r = O.factor(w_.A, w_.PW, w_.vrule, w_.budget, alg=alg)
    A = w_.A.to_scipy().toarray(); W = r.W_csc().toarray(); V = r.V_csc().toarray()
    nrm = np.linalg.norm(A @ W - V)
    assert nrm**2 == pytest.approx((r.res**2).sum(), rel=1e-10)
    E = np.linalg.norm(A @ W @ np.linalg.inv(V) - np.eye(A.shape[0]))
    s = np.linalg.svd(V, compute_uv=False)
    assert E * s[-1] <= nrm * (1 + 1e-9)
    assert nrm <= E * s[0] * (1 + 1e-9)


@pytest.mark.parametrize("alg", ["S", "Q"])
def test_residual_matches_singular_value(alg):
    """DIAF-S: res_j = sigma_min(A_hat_j); DIAF-Q: res_j^2 = 1 - ||M_j||_2^2."""
    w_ = make_workload("powerlaw6k")
    r = O.factor(w_.A, w_.PW, w_.vrule, w_.budget, alg=alg)
    ok = (r.flags & (O.F_RANK_DEFICIENT | O.F_EMPTY)) == 0
    if alg == "S":
        assert np.allclose(r.res[ok], r.sig[ok, 0], rtol=1e-9, atol=1e-12)
    else:
        assert np.allclose(r.res[ok] ** 2, 1 - r.sig[ok, 0] ** 2, atol=1e-12)


def test_phase_and_norms():
    w_ = make_workload("helmholtz40")
    for alg in ("S", "Q"):
        r = O.factor(w_.A, w_.PW, w_.vrule, w_.budget, alg=alg)
        for t in range(0, w_.n, 37):
            I = r.I(t); v = r.v(t); w = r.w(t)
            vjj = v[np.searchsorted(I, t)]
            assert abs(vjj.imag) <= 1e-15 * abs(vjj) and vjj.real >= 0
            if alg == "S":
                assert np.linalg.norm(w) == pytest.approx(1.0, rel=1e-13)
            else:
                assert np.linalg.norm(v) == pytest.approx(1.0, rel=1e-13)


def test_exact_rational_pin():
    """A 3x3 rational example solved in exact arithmetic (sympy): DIAF-S with
    J_2 = {1, 2} and I_2 = {2}: res^2 = smallest eigenvalue of A_hat^T A_hat."""
    sympy = pytest.importorskip("sympy")
    M = sympy.Matrix([[2, 1, 0], [1, 3, 1], [0, 1, 4]])
    Ah = M[[0, 1], [1, 2]]  # rows {0,1} (row 2 removed), columns J = {1,2}
    ev = min((Ah.T * Ah).eigenvals().keys(), key=lambda e: float(e))
    A = type(random_sparse(2, 0.0, 0)).from_scipy(sp.csc_matrix(np.array(M.tolist(), dtype=float)))
    PW = pattern_from_sets(3, [[0], [1], [1, 2]])
    r = O.factor(A, PW, O.RULE_FIXED, None, diagonal_pattern(3), alg="S")
    assert r.res[2] ** 2 == pytest.approx(float(ev), rel=1e-13)


# --------------------------------------------------------------- edge cases
def test_empty_w_column_and_degenerate_tile():
    A = random_sparse(12, 0.2, 2)
    sets = [A.col(j) for j in range(A.n)]
    sets[4] = []
    PW = pattern_from_sets(A.n, sets)
    for alg in ("S", "Q"):
        r = O.factor(A, PW, O.RULE_UPPER, upper_budget(A), alg=alg)
        assert r.flags[4] & O.F_EMPTY
        assert r.w(4).size == 0
        assert np.all(np.isfinite(r.res))


def test_vcount_and_budget_caps():
    w_ = make_workload("powerlaw6k")
    lc = O.vcount(w_.A, w_.PW, w_.vrule, w_.budget)
    assert np.all(lc >= 1) and np.all(lc <= w_.budget)
    lc_all = O.vcount(w_.A, w_.PW, w_.vrule, None)
    assert np.all(lc_all >= lc)


# --------------------------------------------------------------- Krylov references
def test_bicgstab_reference_against_scipy():
    w_ = make_workload("convdiff32")
    A = w_.A.to_scipy()
    x, its, rr, st = O.bicgstab(A, w_.b, None, tol=1e-8)
    assert st == "ok" and rr <= 1e-8
    assert np.allclose(x, 1.0, atol=1e-5)
    from scipy.sparse.linalg import bicgstab as sbicg
    cnt = [0]
    xs, info = sbicg(A, w_.b, rtol=1e-8, atol=0.0, callback=lambda _: cnt.__setitem__(0, cnt[0] + 1))
    assert info == 0 and abs(cnt[0] - its) <= 1


def test_preconditioned_solves_converge():
    w_ = make_workload("convdiff32")
    A = w_.A.to_scipy()
    _, its0, _, _ = O.bicgstab(A, w_.b)
    for alg in ("S", "Q"):
        r = O.factor(w_.A, w_.PW, w_.vrule, w_.budget, alg=alg)
        M = O.Preconditioner(r.W_csc(), r.V_csc())
        x, its, rr, st = O.bicgstab(A, w_.b, M)
        assert st == "ok" and its < its0
        assert np.allclose(x, 1.0, atol=1e-5)


def test_gmres_reference():
    w_ = make_workload("helmholtz40")
    A = w_.A.to_scipy()
    r = O.factor(w_.A, w_.PW, w_.vrule, w_.budget, alg="S")
    M = O.Preconditioner(r.W_csc(), r.V_csc())
    x, its, rr, st = O.gmres(A, w_.b, M, restart=50, tol=1e-6)
    assert st == "ok" and np.linalg.norm(w_.b - A @ x) <= 1e-6 * np.linalg.norm(w_.b) * 1.0001


def test_block_rule_reductions():
    """Block-diagonal V (RULE_BLOCK): blocks of one row reduce to the diagonal
    V; one block holding every row reduces to RULE_ALL; every entry of V lies
    in its column's block."""
    from tests._problems import random_sparse
    from workloads import diagonal_pattern, pattern_of
    A = random_sparse(120, 0.04, 31, False)
    PW = pattern_of(A)
    n = A.n
    for alg in ("S", "Q"):
        one = O.factor(A, PW, O.RULE_BLOCK, np.full(n, 3, np.int32), None, alg=alg, blocks=np.arange(n))
        diag = O.factor(A, PW, O.RULE_FIXED, None, diagonal_pattern(n), alg=alg)
        np.testing.assert_array_equal(one.Vrowidx, diag.Vrowidx)
        np.testing.assert_allclose(one.res, diag.res, rtol=0, atol=0)
        allb = O.factor(A, PW, O.RULE_BLOCK, np.full(n, 4, np.int32), None, alg=alg, blocks=np.zeros(n))
        ref = O.factor(A, PW, O.RULE_ALL, np.full(n, 4, np.int32), None, alg=alg)
        np.testing.assert_array_equal(allb.Vrowidx, ref.Vrowidx)
        np.testing.assert_allclose(allb.res, ref.res, rtol=0, atol=0)
        blocks = np.arange(n) // 16
        b16 = O.factor(A, PW, O.RULE_BLOCK, np.full(n, 5, np.int32), None, alg=alg, blocks=blocks)
        for j in range(n):
            assert np.all(blocks[b16.I(j)] == blocks[j])
            assert j in b16.I(j)
