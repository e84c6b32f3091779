"""Mixed-code persistent launch (lpdec_decode_mixed) vs per-code decodes and the oracle."""
import numpy as np
import pytest

from _stopping import assert_stop_near_threshold
from paper_1204_0556_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _mixed_batch(names, counts, seed, snr_lo=1.5, snr_hi=4.0):
    codes = [I.benchmark_code(nm, k) for k, nm in enumerate(names)]
    fc = np.concatenate([np.full(n, c, dtype=np.int32) for c, n in enumerate(counts)])
    rng = np.random.default_rng(seed)
    fc = fc[rng.permutation(len(fc))]
    snr = rng.uniform(snr_lo, snr_hi, len(fc))
    frames = []
    for f, c in enumerate(fc):
        frames.append(I.awgn_llr(codes[c], snr[f], 1, seed * 100000 + f)[0])
    return codes, fc, frames


def _run_mixed(gpu, codes, fc, frames, **kw):
    import torch

    Cs = [gpu.Code(c) for c in codes]
    try:
        llr = torch.from_numpy(np.concatenate(frames).astype(np.float32)).cuda()
        out = gpu.decode_mixed(Cs, fc, llr, gpu.make_params(**kw))
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in out.items()}
    finally:
        for C in Cs:
            C.close()


def _split(codes, fc, packed):
    """Unpack the mixed outputs per frame."""
    xs, bs = [], []
    off = 0
    for c in fc:
        n = codes[c].n
        xs.append(packed["x"][off:off + n])
        bs.append(packed["bits"][off:off + n])
        off += n
    return xs, bs


def test_mixed_equals_per_code_decodes(gpu):
    from test_gpu_decode import gpu_decode

    codes, fc, frames = _mixed_batch(["C1056", "C2640", "C4000", "C96", "C8000"], [14, 10, 6, 9, 4], seed=3)
    kw = dict(mu=3.0, rho=1.9, eps=1e-5, max_iter=300)
    got = _run_mixed(gpu, codes, fc, frames, **kw)
    xs, bs = _split(codes, fc, got)
    for c, code in enumerate(codes):
        idx = np.nonzero(fc == c)[0]
        ref = gpu_decode(gpu, code, np.stack([frames[f] for f in idx]), **kw)
        for r, f in enumerate(idx):
            assert np.array_equal(xs[f], ref["x"][r]), (code.name, f)
            assert np.array_equal(bs[f], ref["bits"][r])
            assert got["iters"][f] == ref["iters"][r] and got["cert"][f] == ref["cert"][r]


def test_mixed_matches_oracle(gpu, oracle_mod):
    codes, fc, frames = _mixed_batch(["C1056", "C2640", "C4000"], [12, 12, 6], seed=5)
    kw = dict(mu=3.0, rho=1.9, eps=1e-5, max_iter=400)
    got = _run_mixed(gpu, codes, fc, frames, **kw)
    xs, bs = _split(codes, fc, got)
    same = 0
    for f, c in enumerate(fc):
        code = codes[c]
        ref = oracle_mod.decode(code.row_ptr, code.col_idx, code.n, frames[f][None, :].astype(np.float64), **kw)
        err = np.abs(xs[f] - ref["x"][0]).max()
        if got["iters"][f] == ref["iters"][0]:
            same += 1
            assert err <= 1e-4, (code.name, f, err)
        else:
            assert abs(int(got["iters"][f]) - int(ref["iters"][0])) <= 10
            assert err <= 1e-3
            # the two stops straddle eps^2 E by a rounding margin (tests/_stopping.py)
            assert_stop_near_threshold(oracle_mod, code, frames[f], got["iters"][f], ref["iters"][0], mu=3.0,
                                       rho=1.9, eps=1e-5)
        if np.abs(ref["x"][0] - 0.5).min() > 1e-3:
            assert np.array_equal(bs[f], ref["bits"][0])
    assert same >= 0.9 * len(fc)


def test_mixed_with_idle_codes_and_one_frame(gpu):
    codes, fc, frames = _mixed_batch(["C96", "C1056", "C4000"], [0, 1, 0], seed=7)
    got = _run_mixed(gpu, codes, fc, frames, eps=1e-5, max_iter=100)
    assert got["iters"][0] >= 1


def test_mixed_rejects_bad_arguments(gpu):
    import torch

    code = I.benchmark_code("C96", 0)
    C = gpu.Code(code)
    try:
        llr = torch.zeros(code.n, dtype=torch.float32, device="cuda")
        x = torch.empty_like(llr)
        s = int(torch.cuda.current_stream().cuda_stream)
        with pytest.raises(gpu.LpdecError) as ei:  # frame_code out of range
            gpu.lpdec_decode_mixed([C.handle], 1, [1], llr.data_ptr(), gpu.make_params(), x.data_ptr(), 0, 0, 0, s)
        assert ei.value.status == gpu.LPDEC_EINVAL
        with pytest.raises(gpu.LpdecError):
            gpu.decode_mixed([C], [0], llr, gpu.make_params(schedule="streamed"))
    finally:
        C.close()
