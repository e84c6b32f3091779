"""Pins for the oracle's ADMM decoder (Algorithm 1 with over-relaxation).

The decoder is an iteration whose limit is the Feldman LP optimum
(eq. (feldmanLP); the convergence proposition of Section 3.3), so it is pinned
against an exact LP solve by SciPy's HiGHS on tiny codes, and against the
special cases the paper fixes (noiseless input, certificate semantics).
"""
import numpy as np
import pytest

import _pins as P
from paper_1204_0556_gb300 import inputs as I


def _decode(oracle_mod, code, gamma, **kw):
    return oracle_mod.decode(code.row_ptr, code.col_idx, code.n, gamma, **kw)


@pytest.mark.parametrize("n,seed,ebn0", [(12, 0, 1.0), (12, 3, 2.0), (24, 2, 1.5), (24, 5, 3.0)])
@pytest.mark.parametrize("rho", [1.0, 1.9])
def test_reaches_feldman_lp_optimum(oracle_mod, n, seed, ebn0, rho):
    code = I.gallager_code(n, 3, 6, seed)
    gamma = I.awgn_llr(code, ebn0, 12, seed + 10).astype(np.float64)
    r = _decode(oracle_mod, code, gamma, mu=3.0, rho=rho, eps=1e-12, max_iter=40000)
    assert r["converged"].all()
    for f in range(len(gamma)):
        xs, obj = P.feldman_lp(code.rows(), code.n, gamma[f])
        got = float(gamma[f] @ r["x"][f])
        assert abs(got - obj) <= 1e-8 * (1 + abs(obj)), (f, got, obj)
        # feasibility of the ADMM output for the LP (fundamental polytope)
        for row in code.rows():
            assert P.in_parity_polytope(r["x"][f][row], tol=1e-7)


def test_unique_optimum_matches_point(oracle_mod):
    """Where the LP optimum is unique (checked by re-solving under small random
    cost perturbations), ADMM's x matches the LP's x."""
    code = I.gallager_code(24, 3, 6, 7)
    gamma = I.awgn_llr(code, 1.5, 16, 77).astype(np.float64)
    r = _decode(oracle_mod, code, gamma, mu=3.0, rho=1.9, eps=1e-12, max_iter=40000)
    rng = np.random.default_rng(0)
    checked = 0
    for f in range(len(gamma)):
        xs, _ = P.feldman_lp(code.rows(), code.n, gamma[f])
        unique = True
        for _ in range(3):
            xp, _ = P.feldman_lp(code.rows(), code.n, gamma[f] + 1e-6 * rng.normal(size=code.n))
            if np.abs(xp - xs).max() > 1e-6:
                unique = False
        if unique:
            np.testing.assert_allclose(r["x"][f], xs, atol=1e-5)
            checked += 1
    assert checked >= 8


def test_noiseless_all_zeros(oracle_mod):
    """Noiseless all-zeros input (gamma > 0): x = 0 after one sweep, certified."""
    code = I.benchmark_code("C96", 0)
    gamma = np.full((3, code.n), 4.0)
    r = _decode(oracle_mod, code, gamma, mu=3.0, rho=1.9, eps=1e-5, max_iter=200)
    assert np.all(r["x"] == 0.0)
    assert np.all(r["iters"] == 1)
    assert np.all(r["converged"] == 1)
    assert np.all(r["cert"] == 1)
    assert np.all(r["bits"] == 0)


def test_fixed_iterations_when_eps_zero(oracle_mod):
    code = I.benchmark_code("C96", 0)
    gamma = I.awgn_llr(code, 2.0, 8, 1).astype(np.float64)
    r = _decode(oracle_mod, code, gamma, mu=3.0, rho=1.9, eps=0.0, max_iter=37)
    assert np.all(r["iters"] == 37)
    assert np.all(r["converged"] == 0)


def test_certificate_only_on_integral_codewords(oracle_mod):
    """Search seeded low-SNR frames for fractional LP optima (pseudocodewords):
    there the certificate must be 0; wherever it is 1, x is integral and a codeword."""
    code = I.gallager_code(12, 3, 6, 0)
    H = code.dense()
    gamma = I.awgn_llr(code, 0.0, 200, 11).astype(np.float64)
    r = _decode(oracle_mod, code, gamma, mu=3.0, rho=1.9, eps=1e-10, max_iter=20000)
    fractional = 0
    for f in range(len(gamma)):
        xs, _ = P.feldman_lp(code.rows(), code.n, gamma[f])
        if np.min(np.abs(xs - 0.5)) < 0.4:  # clearly fractional LP optimum
            fractional += 1
            assert r["cert"][f] == 0
        if r["cert"][f]:
            assert np.all(np.minimum(r["x"][f], 1 - r["x"][f]) <= 1e-2)
            assert np.all(H @ r["bits"][f] % 2 == 0)
    assert fractional >= 3
    assert r["cert"].sum() >= 50


def test_converges_faster_with_overrelaxation(oracle_mod):
    """Section 5.2: rho = 1.9 needs markedly fewer iterations than rho = 1 (frames that
    converge under both; frames stuck at the iteration cap say nothing about speed)."""
    code = I.benchmark_code("C96", 0)
    gamma = I.awgn_llr(code, 3.0, 60, 5).astype(np.float64)
    a = _decode(oracle_mod, code, gamma, mu=3.0, rho=1.0, eps=1e-5, max_iter=1000)
    b = _decode(oracle_mod, code, gamma, mu=3.0, rho=1.9, eps=1e-5, max_iter=1000)
    both = (a["converged"] == 1) & (b["converged"] == 1)
    assert both.sum() >= 40
    assert b["iters"][both].mean() < 0.8 * a["iters"][both].mean()


def test_objective_gap_shrinks_with_iterations(oracle_mod):
    """Convergence proposition of Section 3.3: gamma^T x_hat - gamma^T x* -> 0 as T grows."""
    code = I.gallager_code(24, 3, 6, 2)
    gamma = I.awgn_llr(code, 1.0, 6, 21).astype(np.float64)
    gaps = []
    for T in (3, 30, 3000):
        r = _decode(oracle_mod, code, gamma, mu=3.0, rho=1.0, eps=0.0, max_iter=T)
        g = 0.0
        for f in range(len(gamma)):
            _, obj = P.feldman_lp(code.rows(), code.n, gamma[f])
            g += abs(float(gamma[f] @ r["x"][f]) - obj)
        gaps.append(g)
    assert gaps[2] < gaps[0]
    assert gaps[2] < 1e-6


def test_threads_do_not_change_results(oracle_mod):
    code = I.benchmark_code("C96", 0)
    gamma = I.awgn_llr(code, 2.0, 20, 3).astype(np.float64)
    a = _decode(oracle_mod, code, gamma, mu=3.0, rho=1.9, eps=1e-5, max_iter=200, threads=1)
    b = _decode(oracle_mod, code, gamma, mu=3.0, rho=1.9, eps=1e-5, max_iter=200, threads=4)
    for k in a:
        assert np.array_equal(a[k], b[k])
