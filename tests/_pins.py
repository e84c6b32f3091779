"""Independent checks used to pin the oracle (no code shared with it or the CUDA path).

* ``even_vertices(d)``: the vertex set P_d of the parity polytope (Section 2,
  eq. (spcConst)), enumerated.
* ``min_norm_point``: Wolfe's (1976) minimum-norm-point algorithm over a finite
  point set; projecting v onto conv(P_d) is the min-norm point of {e - v}.
* ``in_parity_polytope``: Jeroslow's facet description of PP_d (cited in
  Section 2): the unit cube plus, for every odd-size subset S,
  sum_S z - sum_{S^c} z <= |S| - 1.
* ``vi_gap``: max over even vertices e of (v - z)^T (e - z); together with
  membership, a value <= 0 certifies z = Pi_PP(v) exactly (first-order
  optimality of a convex projection).
* ``feldman_lp``: the LP relaxation (eq. (feldmanLP)) written with the odd-set
  facets and solved by SciPy's HiGHS.
"""
from __future__ import annotations

import itertools

import numpy as np


def even_vertices(d: int) -> np.ndarray:
    pts = np.array(list(itertools.product([0, 1], repeat=d)), dtype=np.float64)
    return pts[pts.sum(axis=1) % 2 == 0]


def odd_sets(d: int) -> np.ndarray:
    """Sign matrix: row per odd subset S, +1 on S and -1 elsewhere."""
    pts = np.array(list(itertools.product([0, 1], repeat=d)), dtype=np.float64)
    pts = pts[pts.sum(axis=1) % 2 == 1]
    return 2.0 * pts - 1.0


def min_norm_point(P: np.ndarray, tol: float = 1e-15, max_major: int = 1000) -> np.ndarray:
    """Point of minimum Euclidean norm in conv(rows of P) (Wolfe's algorithm)."""
    P = np.asarray(P, dtype=np.float64)
    norms = np.einsum("ij,ij->i", P, P)
    scale = max(1.0, float(norms.max()))
    S = [int(np.argmin(norms))]
    lam = np.array([1.0])
    x = P[S[0]].copy()
    for _ in range(max_major):
        dots = P @ x
        j = int(np.argmin(dots))
        if x @ x - dots[j] <= tol * scale or j in S:
            break
        S.append(j)
        lam = np.append(lam, 0.0)
        for _minor in range(10 * len(P)):
            Q = P[S]
            s = len(S)
            A = np.zeros((s + 1, s + 1))
            A[:s, :s] = Q @ Q.T
            A[:s, s] = 1.0
            A[s, :s] = 1.0
            rhs = np.zeros(s + 1)
            rhs[s] = 1.0
            a = np.linalg.lstsq(A, rhs, rcond=None)[0][:s]
            if np.all(a > 1e-14):
                lam = a
                x = Q.T @ a
                break
            neg = a <= 1e-14
            theta = float(np.min(lam[neg] / (lam[neg] - a[neg])))
            lam = theta * a + (1.0 - theta) * lam
            keep = lam > 1e-14
            S = [S[i] for i in range(s) if keep[i]]
            lam = lam[keep]
            lam = lam / lam.sum()
            x = P[S].T @ lam
    return x


def brute_project(v: np.ndarray) -> np.ndarray:
    """Pi_PP(v) as the nearest point of conv(P_d), by Wolfe's algorithm."""
    v = np.asarray(v, dtype=np.float64)
    V = even_vertices(len(v))
    return v + min_norm_point(V - v)


def in_parity_polytope(z: np.ndarray, tol: float = 1e-9) -> bool:
    z = np.asarray(z, dtype=np.float64)
    if np.any(z < -tol) or np.any(z > 1 + tol):
        return False
    F = odd_sets(len(z))
    rhs = (F > 0).sum(axis=1) - 1.0
    return bool(np.all(F @ z <= rhs + tol))


def vi_gap(v: np.ndarray, z: np.ndarray) -> float:
    V = even_vertices(len(v))
    return float(np.max((V - z) @ (np.asarray(v) - z)))


def two_slice_member(z: np.ndarray, tol: float = 1e-9) -> bool:
    """Lemma 2 (two-slice): z in conv(PP_d^r u PP_d^{r+2}), r = even floor of ||z||_1,
    checked through the majorization bounds of eq. (simple_majorize_bnd)."""
    z = np.sort(np.asarray(z, dtype=np.float64))[::-1]
    d = len(z)
    s = z.sum()
    r = 2 * int(np.floor(s / 2 + 1e-12))
    if r >= d:
        return bool(abs(s - d) < tol and np.all(z > 1 - tol))
    alpha = (2 + r - s) / 2
    pref = np.cumsum(z)
    for q in range(1, d):
        bound = alpha * min(q, r) + (1 - alpha) * min(q, r + 2)
        if pref[q - 1] > bound + tol:
            return False
    return bool(np.all(z >= -tol) and np.all(z <= 1 + tol))


def feldman_lp(rows, n: int, gamma: np.ndarray):
    """min gamma^T x s.t. x in the fundamental polytope (odd-set facets of every check).

    Returns (x*, objective)."""
    from scipy.optimize import linprog

    A, b = [], []
    for r in rows:
        r = [int(c) for c in r]
        F = odd_sets(len(r))
        for row in F:
            a = np.zeros(n)
            a[r] = row
            A.append(a)
            b.append((row > 0).sum() - 1.0)
    res = linprog(np.asarray(gamma, dtype=np.float64), A_ub=np.array(A), b_ub=np.array(b),
                  bounds=[(0.0, 1.0)] * n, method="highs",
                  options={"primal_feasibility_tolerance": 1e-10,
                           "dual_feasibility_tolerance": 1e-10})
    if res.status != 0:
        raise RuntimeError(res.message)
    return res.x, float(res.fun)
