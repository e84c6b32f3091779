"""Pins for the oracle's projection onto the parity polytope (Algorithm 2).

Nothing here re-types the oracle: every expected value comes from the paper's
statements (golden file), from an independent brute-force solver over the
enumerated vertices (Wolfe's min-norm point), from the exact optimality
certificate of a convex projection, or from invariants the paper proves.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import _pins as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "projection_pins.txt")


def _parse_vec(s):
    return np.array([float(Fraction(t.strip())) for t in s.split(",")], dtype=np.float64)


def _golden():
    out = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            a, b, why = [t.strip() for t in line.split(";", 2)]
            out.append((_parse_vec(a), _parse_vec(b), why))
    return out


@pytest.mark.parametrize("bisect", [False, True])
def test_golden_pins(oracle_mod, bisect):
    cases = _golden()
    assert len(cases) >= 15
    for u, want, why in cases:
        got = oracle_mod.project(u, bisect=bisect)
        np.testing.assert_allclose(got, want, atol=1e-12, err_msg=why)


def _random_vectors(rng, d, count):
    """Mix of the regimes the decoder produces: near-vertex, interior, far, ties."""
    out = []
    for t in range(count):
        kind = t % 6
        if kind == 0:
            v = rng.normal(0.5, 0.6, d)
        elif kind == 1:
            v = rng.integers(0, 2, d) + rng.normal(0, 0.05, d)
        elif kind == 2:
            v = rng.normal(0.5, 3.0, d)
        elif kind == 3:
            v = np.round(rng.normal(0.5, 0.7, d) * 4) / 4  # many ties
        elif kind == 4:
            v = rng.uniform(0, 1, d)
        else:
            v = np.full(d, rng.normal(0.5, 0.5))  # all equal
        out.append(v)
    return out


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 6])
def test_against_brute_force(oracle_mod, d):
    rng = np.random.default_rng(100 + d)
    for v in _random_vectors(rng, d, 240):
        z = oracle_mod.project(v)
        zb = P.brute_project(v)
        np.testing.assert_allclose(z, zb, atol=1e-9, err_msg=str(v))


@pytest.mark.parametrize("d", [7, 8, 10, 12])
def test_variational_inequality(oracle_mod, d):
    """z in PP_d and (v - z)^T (e - z) <= 0 for every even vertex e certify z = Pi_PP(v)."""
    rng = np.random.default_rng(200 + d)
    for v in _random_vectors(rng, d, 60):
        z = oracle_mod.project(v)
        assert P.in_parity_polytope(z), (v, z)
        assert P.vi_gap(v, z) <= 1e-12 * max(1.0, np.abs(v).max()), (v, z)


@pytest.mark.parametrize("d", [3, 6, 9, 16, 30])
def test_two_routes_agree(oracle_mod, d):
    rng = np.random.default_rng(300 + d)
    V = np.array(_random_vectors(rng, d, 600))
    a = oracle_mod.project_many(V)
    b = oracle_mod.project_many(V, bisect=True)
    assert np.abs(a - b).max() <= 1e-12


@pytest.mark.parametrize("d", [4, 6, 8, 13, 20, 32])
def test_two_slice_and_lemma3(oracle_mod, d):
    """Lemma 2 membership of the output and the Lemma 3 l1 bracket."""
    rng = np.random.default_rng(400 + d)
    for v in _random_vectors(rng, d, 300):
        z = oracle_mod.project(v)
        assert P.two_slice_member(z), (v, z)
        s = np.clip(v, 0, 1).sum()
        lo = 2 * np.floor(s / 2)
        hi = 2 * np.ceil(s / 2)
        assert lo - 1e-9 <= z.sum() <= hi + 1e-9


@pytest.mark.parametrize("d", [5, 6, 11, 24])
def test_invariants(oracle_mod, d):
    rng = np.random.default_rng(500 + d)
    vecs = _random_vectors(rng, d, 200)
    for a, b in zip(vecs[:-1], vecs[1:]):
        za = oracle_mod.project(a)
        zb = oracle_mod.project(b)
        # Proposition 1/2: permutation equivariance
        p = rng.permutation(d)
        np.testing.assert_allclose(oracle_mod.project(a[p]), za[p], atol=1e-12)
        # Proposition 2: the projection keeps the order of v
        order = np.argsort(-a, kind="stable")
        assert np.all(np.diff(za[order]) <= 1e-12)
        # even-flip symmetry: complementing an even set T maps P_d (hence PP_d) to itself
        T = rng.permutation(d)[: 2 * rng.integers(0, d // 2 + 1)]
        fa = a.copy()
        fa[T] = 1.0 - fa[T]
        want = za.copy()
        want[T] = 1.0 - want[T]
        np.testing.assert_allclose(oracle_mod.project(fa), want, atol=1e-12)
        # firm nonexpansiveness of a convex projection
        lhs = np.sum((za - zb) ** 2)
        rhs = np.dot(a - b, za - zb)
        assert lhs <= rhs + 1e-12


@pytest.mark.parametrize("d", [3, 6, 15])
def test_padding_with_very_negative_entries(oracle_mod, d):
    """PP_D restricted to z_k = 0 (k >= d) is PP_d x {0}: padding with very negative
    entries must give the lower-dimensional projection."""
    rng = np.random.default_rng(600 + d)
    for v in _random_vectors(rng, d, 100):
        z = oracle_mod.project(v)
        zp = oracle_mod.project(np.concatenate([v, np.full(32 - d, -1e6)]))
        np.testing.assert_allclose(zp[:d], z, atol=1e-12)
        assert np.all(zp[d:] == 0.0)


def test_degree_out_of_range(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.project(np.zeros(65))
