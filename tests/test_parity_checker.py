"""The parity checker itself, on the CPU: the oracle's own result passes it,
and mistakes planted on the host into a copy of that result fail it.

The planted mistakes are the ones the GPU could make on columns with several
optimal vectors, where no vector comparison is possible: a unit w_j that is
feasible but not optimal (with its residual reported honestly), a v_j that
is not T(I,:) w_j (DIAF-S, Sec. 2.2), a w_j that is not the least-squares
solution of eq. condwj for its v_j (DIAF-Q, Sec. 2.1), and a reported
residual that is not the returned pair's."""
import numpy as np
import pytest

import oracle as O
from tests._parity import (F_DEG, F_EMPTY, F_RANK, _tile, assert_parity, compare, oracle_as_factors, recompute)
from workloads import make_workload


@pytest.fixture(scope="module")
def powerlaw():
    return make_workload("powerlaw6k")


def _one(w, alg, j):
    """The oracle's result for column j alone (compare() indexes it by list position)."""
    return O.factor(w.A, w.PW, w.vrule, w.budget, alg=alg, tie_tol=w.tie_tol, cols=[j])


def _honest_res(g, w, j):
    g["res"][j] = recompute(g, w.A, w.PW, [j])["res"][0]


def _tile_times(w, j, x):
    """A(:,J_j) x as a dense n-vector."""
    J = w.PW.col(j)
    return w.A.to_scipy()[:, J] @ x


def _degenerate_cols(o, w):
    """Columns with several optimal vectors where not every unit w is optimal
    (Ahat = T(R_j minus I_j, :) is not zero)."""
    k = w.PW.counts()
    out = []
    for j in np.nonzero((o.flags & (F_DEG | F_RANK)) != 0)[0]:
        if k[j] < 2 or o.flags[j] & F_EMPTY:
            continue
        T = _tile(w.A, w.PW, j)
        R = np.unique(np.concatenate([w.A.col(c) for c in w.PW.col(j)]))
        Ahat = T[~np.isin(R, o.I(j))]
        if Ahat.size and np.linalg.norm(Ahat, 2) > 1e-3 * np.linalg.norm(T, 2):
            out.append(int(j))
    return out


@pytest.mark.parametrize("alg", ["S", "Q"])
def test_oracle_passes_its_own_check(powerlaw, alg):
    w = powerlaw
    o = O.factor(w.A, w.PW, w.vrule, w.budget, alg=alg, tie_tol=w.tie_tol)
    rep = compare(oracle_as_factors(o), o, w.A, w.PW, alg)
    assert_parity(rep)
    assert rep["degenerate"] > 100 or alg == "Q"  # the power-law operator has many non-unique optima under DIAF-S


def test_wrong_unit_w_on_degenerate_column_fails(powerlaw):
    """DIAF-S: a feasible unit w_j that is not a minimiser, with v_j = T(I,:) w_j
    and its true residual reported, must fail on optimality."""
    w = powerlaw
    o = O.factor(w.A, w.PW, w.vrule, w.budget, alg="S", tie_tol=w.tie_tol)
    cols = _degenerate_cols(o, w)
    assert cols
    rng = np.random.default_rng(3)
    failed = 0
    for j in cols[:20]:
        g = oracle_as_factors(o)
        sl = slice(g["Wcp"][j], g["Wcp"][j + 1])
        x = g["Wv"][sl] + 0.3 * rng.standard_normal(sl.stop - sl.start)
        x /= np.linalg.norm(x)
        g["Wv"][sl] = x
        I = g["Vri"][g["Vcp"][j]:g["Vcp"][j + 1]]
        g["Vv"][g["Vcp"][j]:g["Vcp"][j + 1]] = _tile_times(w, j, x)[I]
        _honest_res(g, w, j)
        rep = compare(g, _one(w, "S", j), w.A, w.PW, "S", cols=[j])
        assert not rep["I_mismatch"] and not rep["self_bad"] and not rep["vec_bad"]
        failed += bool(rep["res_bad"])
    assert failed == min(20, len(cols))


def test_v_not_projection_fails(powerlaw):
    """DIAF-S: v_j must be (A w_j) on I_j; a perturbed v_j (reported
    residual honest) fails the first-order check."""
    w = powerlaw
    o = O.factor(w.A, w.PW, w.vrule, w.budget, alg="S", tie_tol=w.tie_tol)
    j = _degenerate_cols(o, w)[0]
    g = oracle_as_factors(o)
    sl = slice(g["Vcp"][j], g["Vcp"][j + 1])
    g["Vv"][sl] += 1e-5 * np.linalg.norm(g["Vv"][sl])
    _honest_res(g, w, j)
    rep = compare(g, _one(w, "S", j), w.A, w.PW, "S", cols=[j])
    assert rep["valid_bad"] and rep["valid_bad"][0][1][0][0] == "v != T(I,:) w"


def test_w_not_least_squares_fails():
    """DIAF-Q: w_j off the least-squares solution of eq. condwj by 1e-6
    relative moves the residual only to second order; the normal equations
    catch it."""
    w = make_workload("convdiff32")
    o = O.factor(w.A, w.PW, w.vrule, w.budget, alg="Q", tie_tol=w.tie_tol)
    j = 500
    g = oracle_as_factors(o)
    sl = slice(g["Wcp"][j], g["Wcp"][j + 1])
    g["Wv"][sl] *= 1 + 1e-6
    _honest_res(g, w, j)
    rep = compare(g, _one(w, "Q", j), w.A, w.PW, "Q", cols=[j], vec_tol=1e-8)
    assert not rep["res_bad"]                       # second order: invisible to the residual
    assert rep["valid_bad"] and rep["valid_bad"][0][1][0][0] == "w not the least-squares solution"


def test_non_singular_vector_fails():
    """DIAF-S on a column with a unique optimum: w_j rotated by 1e-5 towards
    the next singular vector is caught by the eigen-residual (and by the
    vector comparison)."""
    w = make_workload("convdiff32")
    o = O.factor(w.A, w.PW, w.vrule, w.budget, alg="S", tie_tol=w.tie_tol)
    j = 500
    g = oracle_as_factors(o)
    sl = slice(g["Wcp"][j], g["Wcp"][j + 1])
    x = g["Wv"][sl].copy()
    d = np.zeros_like(x); d[0] = 1.0
    d -= np.vdot(x, d) * x
    x = x + 1e-5 * d / np.linalg.norm(d)
    x /= np.linalg.norm(x)
    g["Wv"][sl] = x
    I = g["Vri"][g["Vcp"][j]:g["Vcp"][j + 1]]
    g["Vv"][g["Vcp"][j]:g["Vcp"][j + 1]] = _tile_times(w, j, x)[I]
    _honest_res(g, w, j)
    rep = compare(g, _one(w, "S", j), w.A, w.PW, "S", cols=[j])
    assert rep["valid_bad"] and rep["valid_bad"][0][1][0][0] == "w not a singular vector"
    assert rep["vec_bad"]


def test_dishonest_residual_fails(powerlaw):
    w = powerlaw
    o = O.factor(w.A, w.PW, w.vrule, w.budget, alg="S", tie_tol=w.tie_tol)
    j = int(np.argmax(o.res))
    g = oracle_as_factors(o)
    g["res"][j] *= 1 + 1e-6
    rep = compare(g, _one(w, "S", j), w.A, w.PW, "S", cols=[j])
    assert rep["self_bad"] and not rep["res_bad"]
