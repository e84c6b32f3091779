"""Seeded input generators: code shapes, index-layout consistency, LLR statistics."""
import numpy as np
import pytest

from paper_1204_0556_gb300 import inputs as I


def _check_layouts(c: I.Code):
    E = c.E
    assert c.col_ptr[-1] == E and len(c.col_idx) == E and len(c.row_idx) == E
    assert sorted(c.edge_perm.tolist()) == list(range(E))
    rows_of_edge = np.repeat(np.arange(c.m), np.diff(c.row_ptr))
    for i in range(c.n):
        sl = slice(c.col_ptr[i], c.col_ptr[i + 1])
        assert np.all(c.col_idx[c.edge_perm[sl]] == i)
        assert np.all(rows_of_edge[c.edge_perm[sl]] == c.row_idx[sl])
        assert np.all(np.diff(c.row_idx[sl]) > 0)
    for j in range(c.m):
        assert np.all(np.diff(c.col_idx[c.row_ptr[j]:c.row_ptr[j + 1]]) > 0)


@pytest.mark.parametrize("name,n,m,E,dc,dv", [
    ("C96", 96, 48, 288, {6}, {3}),
    ("C1056", 1056, 528, 3168, {6}, {3}),
    ("C2640", 2640, 1320, 10560, {8}, {4}),
    ("C4000", 4000, 400, 12000, {30}, {3}),
])
def test_benchmark_shapes(name, n, m, E, dc, dv):
    c = I.benchmark_code(name, 0)
    assert (c.n, c.m, c.E) == (n, m, E)
    assert set(c.check_degrees.tolist()) == dc
    assert set(c.var_degrees.tolist()) == dv
    _check_layouts(c)


def test_irregular_shape():
    c = I.benchmark_code("C8000", 0)
    assert (c.n, c.m, c.E) == (8000, 1600, 24000)
    d = c.check_degrees
    assert d.min() >= 6 and d.max() <= 20 and d.sum() == 24000
    assert set(c.var_degrees.tolist()) == {3}
    _check_layouts(c)


def test_four_cycle_removal():
    c = I.benchmark_code("C1056", 0)
    assert I.count_4cycles(c.rows()) == 0
    raw = I.gallager_code(1056, 3, 6, 0, remove_4cycles=False)
    assert I.count_4cycles(raw.rows()) > 0


def test_determinism():
    a = I.benchmark_code("C1056", 0)
    b = I.benchmark_code("C1056", 0)
    assert np.array_equal(a.col_idx, b.col_idx)
    la = I.awgn_llr(a, 2.0, 4, 1)
    lb = I.awgn_llr(a, 2.0, 4, 1)
    assert np.array_equal(la, lb)
    assert not np.array_equal(la, I.awgn_llr(a, 2.0, 4, 2))


def test_awgn_llr_statistics():
    c = I.benchmark_code("C1056", 0)
    g = I.awgn_llr(c, 2.0, 200, 5).astype(np.float64)
    s2 = I.sigma2_for(2.0, 0.5)
    # gamma = 2 y / sigma^2 with y ~ N(1, sigma^2): mean 2/s2, variance 4/s2
    assert abs(g.mean() - 2 / s2) < 0.02 * (2 / s2)
    assert abs(g.var() - 4 / s2) < 0.03 * (4 / s2)


def test_per_frame_snr():
    c = I.benchmark_code("C96", 0)
    snr = np.array([1.0, 4.0] * 500)
    g = I.awgn_llr(c, snr, 1000, 9).astype(np.float64)
    lo, hi = g[0::2], g[1::2]
    assert lo.mean() < hi.mean()


def test_bsc_llr():
    c = I.benchmark_code("C96", 0)
    g = I.bsc_llr(c, 0.05, 100, 3)
    mag = np.log(0.95 / 0.05)
    assert np.allclose(np.abs(g), mag, rtol=1e-6)
    assert 0.03 < (g < 0).mean() < 0.07


def test_random_code_covers_every_variable():
    c = I.random_code(600, 60, 10, 20, 8)
    dc = np.diff(c.row_ptr)
    dv = np.diff(c.col_ptr)
    assert dc.min() >= 10 and dc.max() <= 20
    assert dv.min() >= 1 and dv.max() > dv.min()  # irregular variable degrees, none empty
    assert c.E == int(dc.sum()) == int(dv.sum())
    d = I.random_code(600, 60, 10, 20, 8)
    assert np.array_equal(c.col_idx, d.col_idx) and np.array_equal(c.edge_perm, d.edge_perm)
