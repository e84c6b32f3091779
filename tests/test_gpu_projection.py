"""GPU projection onto PP_d (the decoder's check update, run alone) vs the FP64 oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _vectors(rng, d, count):
    """Regimes seen inside the decoder, plus ties, vertices and wide values."""
    parts = [
        rng.normal(0.5, 0.6, (count, d)),
        rng.integers(0, 2, (count, d)) + rng.normal(0, 0.05, (count, d)),
        rng.normal(0.5, 3.0, (count, d)),
        np.round(rng.normal(0.5, 0.7, (count, d)) * 4) / 4,
        rng.uniform(0, 1, (count, d)),
        np.repeat(rng.normal(0.5, 0.5, (count, 1)), d, axis=1),
        rng.integers(0, 2, (count, d)).astype(np.float64),
    ]
    return np.concatenate(parts).astype(np.float32)


def _run(gpu, V):
    import torch

    z = gpu.project(torch.from_numpy(V).cuda())
    torch.cuda.synchronize()
    return z.cpu().numpy()


@pytest.mark.parametrize("d", list(range(1, 33)))
def test_projection_matches_oracle(gpu, oracle_mod, d):
    rng = np.random.default_rng(1000 + d)
    V = _vectors(rng, d, 3000)
    zg = _run(gpu, V)
    zo = oracle_mod.project_many(V.astype(np.float64))
    scale = np.maximum(1.0, np.abs(V).max(axis=1, keepdims=True))
    err = np.abs(zg - zo) / scale
    assert err.max() <= 2e-5, (d, err.max(), V[np.argmax(err.max(axis=1))])


@pytest.mark.parametrize("d", [6, 8, 30])
def test_projection_million_vectors(gpu, oracle_mod, d):
    rng = np.random.default_rng(2000 + d)
    V = rng.normal(0.5, 0.8, (1_000_000, d)).astype(np.float32)
    zg = _run(gpu, V)
    idx = rng.choice(len(V), 50_000, replace=False)
    zo = oracle_mod.project_many(V[idx].astype(np.float64))
    assert np.abs(zg[idx] - zo).max() <= 2e-5 * max(1.0, float(np.abs(V[idx]).max()))
    # every output lies in the unit cube
    assert zg.min() >= 0.0 and zg.max() <= 1.0


def test_projection_pins(gpu):
    """The hand-derived pins of tests/golden also hold on the GPU."""
    from test_oracle_projection import _golden

    for u, want, why in _golden():
        z = _run(gpu, u.astype(np.float32)[None, :])[0]
        np.testing.assert_allclose(z, want, atol=2e-6, err_msg=why)
