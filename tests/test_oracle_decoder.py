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


# ---------------------------------------------------------------------------
# Hand-derived iterates on codes with irregular variable degrees.
#
# Code A: n = 5, checks c0 = {0, 1, 2}, c1 = {0, 3}, c2 = {0, 1, 4}, so the
# variable degrees are |N_v| = (3, 2, 1, 1, 1) and E = 8.  mu = 2, rho = 3/2 and
# gamma_i = -mu |N_v(i)| a_i with a = (1/2, 1/8, 1/8, 1/8, 1/8):
# gamma = (-3, -1/2, -1/4, -1/4, -1/4).
_ROWS_A = [[0, 1, 2], [0, 3], [0, 1, 4]]
_GAMMA_A = [-3.0, -0.5, -0.25, -0.25, -0.25]


def test_first_two_iterations_closed_form(oracle_mod):
    """Algorithm 1 from z = lambda = 0, worked by hand (Section 3.2 x-update,
    Section 5.2 over-relaxation with q = rho P_j x + (1 - rho) z_old).

    Sweep 1.  x_i = Pi_[0,1](-gamma_i / (mu |N_v(i)|)) = a = (1/2, 1/8, 1/8, 1/8, 1/8).
      (Putting gamma_i/mu outside the 1/|N_v(i)| average, the garbled form of
      Section 3.4, would give x_0 = Pi(3/2) = 1 instead.)
      z_old = lambda = 0, so v_j = q_j = rho P_j x:
      c0 and c2: v = (3/4, 3/16, 3/16).  In the cube, but the odd-set facet
        z_0 - z_1 - z_2 <= 0 is violated by 3/8; moving along f = (1, -1, -1),
        (3/4 - b) - 2 (3/16 + b) = 0 gives b = 1/8, z = (5/8, 5/16, 5/16)
        = 3/8 (000) + 5/16 (110) + 5/16 (101), a point of PP_3 with v - z = b f
        in the facet's normal cone.  lambda/mu = q - z = (1/8, -1/8, -1/8).
      c1: v = (3/4, 3/16); PP_2 is the diagonal, so z = mean = (15/32, 15/32),
        lambda/mu = (9/32, -9/32).
    Sweep 2.  w = z - lambda/mu per edge: c0, c2: (1/2, 7/16, 7/16);
      c1: (3/16, 3/4).  x_i = Pi((sum_e w_e - gamma_i/mu) / |N_v(i)|):
      x_0 = (1/2 + 3/16 + 1/2 + 3/2)/3 = 43/48, x_1 = (7/16 + 7/16 + 1/4)/2 = 9/16,
      x_2 = 7/16 + 1/8 = 9/16, x_3 = 3/4 + 1/8 = 7/8, x_4 = 7/16 + 1/8 = 9/16.
    The projections above are also checked by brute force (Wolfe's algorithm)."""
    code = I.code_from_rows(5, _ROWS_A)
    assert list(code.var_degrees) == [3, 2, 1, 1, 1]
    for v, z in (([0.75, 0.1875, 0.1875], [0.625, 0.3125, 0.3125]), ([0.75, 0.1875], [15 / 32, 15 / 32])):
        np.testing.assert_allclose(P.brute_project(np.array(v)), z, atol=1e-12)
    gamma = np.array([_GAMMA_A])
    r1 = _decode(oracle_mod, code, gamma, mu=2.0, rho=1.5, eps=0.0, max_iter=1)
    np.testing.assert_allclose(r1["x"][0], [1 / 2, 1 / 8, 1 / 8, 1 / 8, 1 / 8], rtol=0, atol=1e-14)
    r2 = _decode(oracle_mod, code, gamma, mu=2.0, rho=1.5, eps=0.0, max_iter=2)
    np.testing.assert_allclose(r2["x"][0], [43 / 48, 9 / 16, 9 / 16, 7 / 8, 9 / 16], rtol=0, atol=1e-14)
    assert r1["iters"][0] == 1 and r2["iters"][0] == 2


def test_stopping_threshold_is_eps2_times_edges(oracle_mod):
    """Section 3.3 stops when both residuals fall below eps^2 E (E = 8 edges
    for code A; the paper writes eps^2 M d for regular codes).

    After sweep 1 of code A (iterates in the test above):
      R_p = sum_e (x_i(e) - z_e)^2 = 11/128 + 61/512 + 11/128 = 149/512,
      R_d = sum_e (z_e - 0)^2 = 150/256 + 450/1024 + 150/256 = 825/512 = 1.611.
    eps = 0.46: eps^2 E = 1.6928 > R_d, so the decoder stops after one sweep.
    eps = 0.44: eps^2 E = 1.5488 < R_d, so it does not.  The bracket rules out
    the other constants a reading could take: eps^2 M = 3 eps^2, eps^2 n and
    eps^2 alone stop at neither, and eps^2 M max_d = 9 eps^2 stops at both."""
    code = I.code_from_rows(5, _ROWS_A)
    gamma = np.array([_GAMMA_A])
    a = _decode(oracle_mod, code, gamma, mu=2.0, rho=1.5, eps=0.46, max_iter=50)
    b = _decode(oracle_mod, code, gamma, mu=2.0, rho=1.5, eps=0.44, max_iter=50)
    assert a["iters"][0] == 1 and a["converged"][0] == 1
    assert b["iters"][0] >= 2
    # the residuals the oracle reports after its last sweep are those above
    np.testing.assert_allclose([a["rp"][0], a["rd"][0]], [149 / 512, 825 / 512], rtol=1e-13, atol=0)


def test_stopping_uses_primal_residual_of_unrelaxed_x(oracle_mod):
    """Code B: checks {0, 1, 2} and {3} (a degree-1 check: PP_1 = {0}, so its z
    is 0 at every sweep), E = 4, mu = 2, rho = 3/2, gamma = (-1/4, -1/4, -1/4, -4).
    Sweep 1: x = (1/8, 1/8, 1/8, Pi(2) = 1).  The first check's v = (3/16)^3 lies
    in PP_3 (each entry at most the sum of the others, total below 2), so z = v.
      R_p = 3 (1/8 - 3/16)^2 + (1 - 0)^2 = 259/256 = 1.0117,
      R_d = 3 (3/16)^2 + 0 = 27/256.
    Here the primal residual decides: eps = 0.51 (eps^2 E = 1.0404) stops after
    one sweep and eps = 0.50 (eps^2 E = 1) does not.  A test on R_d alone would
    stop at both; a primal residual taken with the relaxed q = rho x instead of
    x would give (3/2)^2 = 2.25 on the degree-1 check and stop at neither."""
    code = I.code_from_rows(4, [[0, 1, 2], [3]])
    gamma = np.array([[-0.25, -0.25, -0.25, -4.0]])
    a = _decode(oracle_mod, code, gamma, mu=2.0, rho=1.5, eps=0.51, max_iter=50)
    b = _decode(oracle_mod, code, gamma, mu=2.0, rho=1.5, eps=0.50, max_iter=50)
    assert a["iters"][0] == 1 and a["converged"][0] == 1
    np.testing.assert_allclose(a["x"][0], [1 / 8, 1 / 8, 1 / 8, 1.0], rtol=0, atol=1e-15)
    assert b["iters"][0] >= 2
    np.testing.assert_allclose([a["rp"][0], a["rd"][0]], [259 / 256, 27 / 256], rtol=1e-13, atol=0)


@pytest.mark.parametrize("n,m,seed", [(12, 6, 1), (14, 7, 4), (16, 8, 9)])
@pytest.mark.parametrize("rho", [1.0, 1.9])
def test_irregular_code_reaches_feldman_lp_optimum(oracle_mod, n, m, seed, rho):
    """On a code with irregular variable degrees, weighting gamma_i by anything
    but 1/|N_v(i)| inside the x-update (Section 3.2) moves the fixed point to
    the LP with cost |N_v(i)| gamma_i, whose argmin differs here: the decoder
    must reach the Feldman LP optimum of gamma itself."""
    code = I.random_code(n, m, 3, 5, seed)
    assert len(set(code.var_degrees.tolist())) >= 3
    gamma = I.awgn_llr(code, 1.5, 12, seed + 30).astype(np.float64)
    r = _decode(oracle_mod, code, gamma, mu=3.0, rho=rho, eps=1e-12, max_iter=40000)
    assert r["converged"].all()
    for f in range(len(gamma)):
        _, obj = P.feldman_lp(code.rows(), code.n, gamma[f])
        got = float(gamma[f] @ r["x"][f])
        assert abs(got - obj) <= 1e-8 * (1 + abs(obj)), (f, got, obj)


def test_threads_do_not_change_results(oracle_mod):
    code = I.benchmark_code("C96", 0)
    gamma = I.awgn_llr(code, 2.0, 20, 3).astype(np.float64)
    a = _decode(oracle_mod, code, gamma, mu=3.0, rho=1.9, eps=1e-5, max_iter=200, threads=1)
    b = _decode(oracle_mod, code, gamma, mu=3.0, rho=1.9, eps=1e-5, max_iter=200, threads=4)
    for k in a:
        assert np.array_equal(a[k], b[k])


def test_reported_residuals_decide_the_stop(oracle_mod):
    """The residuals the oracle reports are the ones its stopping test reads
    (Section 3.3): a frame that stops at iteration K has max(R_p, R_d) below
    eps^2 E after K fixed iterations and not after K - 1."""
    code = I.benchmark_code("C96", 0)
    gamma = I.awgn_llr(code, 2.5, 12, 3).astype(np.float64)
    eps = 1e-5
    thr = eps * eps * int(code.row_ptr[-1])
    r = _decode(oracle_mod, code, gamma, mu=3.0, rho=1.9, eps=eps, max_iter=300)
    checked = 0
    for f in range(len(gamma)):
        K = int(r["iters"][f])
        if not r["converged"][f] or K < 2:
            continue
        at = _decode(oracle_mod, code, gamma[f:f + 1], mu=3.0, rho=1.9, eps=0.0, max_iter=K)
        before = _decode(oracle_mod, code, gamma[f:f + 1], mu=3.0, rho=1.9, eps=0.0, max_iter=K - 1)
        assert max(at["rp"][0], at["rd"][0]) < thr
        assert max(before["rp"][0], before["rd"][0]) >= thr
        np.testing.assert_array_equal(at["x"][0], r["x"][f])
        checked += 1
    assert checked >= 8
