"""Pins for the oracle's dual subgradient decoder (appendix) and its linear
maximization over the parity polytope (Algorithm 3), against brute force,
closed forms of the first iterations, the Feldman LP (HiGHS) and maximum-
likelihood decoding by enumeration."""
from __future__ import annotations

import numpy as np
import pytest

import _pins as P
from paper_1204_0556_gb300 import inputs as I


@pytest.mark.parametrize("d", range(1, 9))
def test_lp_max_against_even_vertices(oracle_mod, d):
    """Algorithm 3 returns an even-weight binary vertex attaining
    max_{z in PP_d} c^T z (the maximum of a linear function over a polytope is
    attained at a vertex, and PP_d's vertices are the even-weight words)."""
    V = P.even_vertices(d).astype(np.float64)
    rng = np.random.default_rng(100 + d)
    cases = [rng.normal(size=d) for _ in range(300)]
    cases += [rng.integers(-2, 3, size=d).astype(np.float64) for _ in range(300)]  # ties and zeros
    for c in cases:
        z = oracle_mod.lp_max(c)
        assert set(np.unique(z)) <= {0.0, 1.0}
        assert int(z.sum()) % 2 == 0
        assert c @ z == pytest.approx((V @ c).max(), abs=1e-12), (c, z)


def test_lp_max_odd_repairs(oracle_mod):
    """The two repairs of an odd positive set, worked by hand: adding the
    largest non-positive entry wins when c_ip + c_in > 0, else dropping the
    smallest positive entry wins (on a tie the drop is taken)."""
    assert oracle_mod.lp_max([3.0, 0.5, -0.2]).tolist() == [1.0, 1.0, 0.0]  # r = 2: even
    assert oracle_mod.lp_max([3.0, 0.5, 2.0, -0.2]).tolist() == [1.0, 1.0, 1.0, 1.0]  # add 5.3 > drop 5.0
    assert oracle_mod.lp_max([3.0, 0.1, 2.0, -0.2]).tolist() == [1.0, 0.0, 1.0, 0.0]  # add 4.9 < drop 5.0
    assert oracle_mod.lp_max([3.0, 0.5, 2.0, -0.5]).tolist() == [1.0, 0.0, 1.0, 0.0]  # tie 5.0: drop
    assert oracle_mod.lp_max([3.0, 0.5, 2.0, -0.6]).tolist() == [1.0, 0.0, 1.0, 0.0]
    assert oracle_mod.lp_max([0.5, -0.1, 2.0, 1.0]).tolist() == [1.0, 1.0, 1.0, 1.0]  # add 3.4 > drop 3.0
    assert oracle_mod.lp_max([0.5, -0.3, -0.1, 2.0, 1.0]).tolist() == [1.0, 0.0, 1.0, 1.0, 1.0]  # largest non-positive
    assert oracle_mod.lp_max([0.7, 0.5, 0.5, -0.1]).tolist() == [1.0, 1.0, 1.0, 1.0]  # add 1.6 > drop 1.2
    assert oracle_mod.lp_max([0.7, 0.5, 0.5, -0.6]).tolist() == [1.0, 0.0, 1.0, 0.0]  # drop the first 0.5
    assert oracle_mod.lp_max([1.0]).tolist() == [0.0]  # PP_1 = {0}


def _dual(oracle_mod, code, gamma, **kw):
    return oracle_mod.decode_dual(code.row_ptr, code.col_idx, code.n, gamma, **kw)


def test_first_two_iterations_closed_form(oracle_mod):
    """From lambda = 0: x^1 = [gamma < 0] and z^1 = 0, so lambda_e^1 = mu x^1_i
    on every edge of variable i; then x^2_i = [gamma_i < -mu d_v(i) x^1_i]."""
    code = I.benchmark_code("C96", 0)
    gamma = I.awgn_llr(code, 1.0, 8, 3).astype(np.float64)
    mu = 0.75
    r1 = _dual(oracle_mod, code, gamma, mu=mu, max_iter=1)
    np.testing.assert_array_equal(r1["x"], (gamma < 0).astype(np.float64))
    np.testing.assert_array_equal(r1["iters"], 1)
    np.testing.assert_array_equal(r1["cert"], (gamma >= 0).all(axis=1))
    dv = np.diff(code.col_ptr)
    r2 = _dual(oracle_mod, code, gamma, mu=mu, max_iter=2)
    want = (gamma < -mu * dv[None, :] * (gamma < 0)).astype(np.float64)
    np.testing.assert_array_equal(r2["x"], want)


def test_noiseless_certified_in_one_iteration(oracle_mod):
    code = I.benchmark_code("C96", 0)
    r = _dual(oracle_mod, code, np.full((3, code.n), 2.0), mu=0.25, max_iter=50)
    assert (r["iters"] == 1).all() and r["cert"].all() and not r["bits"].any()


def test_certified_output_is_lp_optimum(oracle_mod):
    """A vanishing subgradient certifies optimality: the certified x is an
    integral point of the fundamental polytope whose cost equals the Feldman
    LP optimum (solved independently by HiGHS)."""
    code = I.benchmark_code("C96", 0)
    gamma = I.awgn_llr(code, 3.0, 24, 11).astype(np.float32).astype(np.float64)
    r = _dual(oracle_mod, code, gamma, mu=0.25, max_iter=5000)
    H = code.dense()
    certified = np.flatnonzero(r["cert"])
    assert len(certified) >= 18
    for f in certified:
        assert np.all(H @ r["bits"][f] % 2 == 0)
        _, obj = P.feldman_lp(code.rows(), code.n, gamma[f])
        assert float(gamma[f] @ r["x"][f]) == pytest.approx(obj, abs=1e-7 * (1 + abs(obj)))


def test_certified_output_is_ml_codeword(oracle_mod):
    """On a code small enough to enumerate, a certified output is a
    maximum-likelihood codeword (an integral LP optimum is ML)."""
    code = I.gallager_code(18, 3, 6, 5)
    H = code.dense().astype(np.int64)
    allw = ((np.arange(2 ** code.n)[:, None] >> np.arange(code.n)[None, :]) & 1).astype(np.int64)
    words = allw[~((allw @ H.T) % 2).any(axis=1)].astype(np.float64)
    assert len(words) >= 2 ** (code.n - code.m)
    gamma = I.awgn_llr(code, 1.5, 40, 21).astype(np.float32).astype(np.float64)
    r = _dual(oracle_mod, code, gamma, mu=0.25, max_iter=5000)
    assert r["cert"].sum() >= 25
    for f in np.flatnonzero(r["cert"]):
        assert float(gamma[f] @ r["x"][f]) == pytest.approx((words @ gamma[f]).min(), abs=1e-9)


def test_step_scaling_invariance(oracle_mod):
    """Scaling gamma and mu together scales every lambda^k and leaves every
    Heaviside and parity-polytope decision unchanged."""
    code = I.benchmark_code("C96", 0)
    gamma = I.awgn_llr(code, 2.5, 16, 8).astype(np.float32).astype(np.float64)
    a = _dual(oracle_mod, code, gamma, mu=0.25, max_iter=400)
    b = _dual(oracle_mod, code, 4.0 * gamma, mu=1.0, max_iter=400)
    np.testing.assert_array_equal(a["x"], b["x"])
    np.testing.assert_array_equal(a["iters"], b["iters"])
    c = _dual(oracle_mod, code, gamma, mu=1.0, max_iter=400)
    assert not np.array_equal(a["iters"], c["iters"])  # mu does matter


def test_threads_do_not_change_dual_results(oracle_mod):
    code = I.benchmark_code("C96", 0)
    gamma = I.awgn_llr(code, 3.0, 20, 4).astype(np.float64)
    a = _dual(oracle_mod, code, gamma, mu=0.25, max_iter=300, threads=1)
    b = _dual(oracle_mod, code, gamma, mu=0.25, max_iter=300, threads=5)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])
