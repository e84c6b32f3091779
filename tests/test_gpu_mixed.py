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


def test_mixed_full_bench_size(gpu, oracle_mod):
    """`bench.py --workload mixed` at full size, in the bench's launch
    configuration: 3 x 10^4 frames of C1056 / C2640 / C4000 (12000 / 12000 /
    6000, shuffled by Philox key 3), Eb/N0 ~ U[1.5, 4.0] dB per frame (key 4),
    LLR seeds 40 + code, eps = 1e-5, at most 1000 iterations, every code's tile
    autotuned as the bench does.  Every frame of the one launch equals the
    per-code decode of the same frame bit for bit, and sampled frames of each
    code match the oracle (x within 1e-4 where the iteration counts agree, and
    any other count explained by the stopping threshold)."""
    import torch

    codes = [I.benchmark_code("C1056", 0), I.benchmark_code("C2640", 1), I.benchmark_code("C4000", 2)]
    F = 30_000
    counts = [int(0.4 * F), int(0.4 * F), F - 2 * int(0.4 * F)]
    order = np.random.Generator(np.random.Philox(key=3)).permutation(F)
    fc = np.concatenate([np.full(n, c, dtype=np.int32) for c, n in enumerate(counts)])[order]
    snr = np.random.Generator(np.random.Philox(key=4)).uniform(1.5, 4.0, F)
    per = {}
    for c, code in enumerate(codes):
        idx = np.nonzero(fc == c)[0]
        per[c] = (idx, I.awgn_llr(code, snr[idx], len(idx), 40 + c))
    offsets = np.concatenate([[0], np.cumsum([codes[c].n for c in fc])])
    packed = np.empty(offsets[-1], dtype=np.float32)
    for c, (idx, llr) in per.items():
        for r, f in enumerate(idx):
            packed[offsets[f]:offsets[f + 1]] = llr[r]
    kw = dict(mu=3.0, rho=1.9, eps=1e-5, max_iter=1000)
    p = gpu.make_params(state="f32", schedule="resident", **kw)
    Cs = [gpu.Code(cd) for cd in codes]
    try:
        stream = int(torch.cuda.current_stream().cuda_stream)
        for c, C in enumerate(Cs):  # the bench's autotuning: up to 16384 frames, 60 fixed iterations
            sample = torch.from_numpy(np.ascontiguousarray(per[c][1][:16384])).cuda()
            gpu.lpdec_autotune(C.handle, gpu.make_params(mu=3.0, rho=1.9, eps=0.0, max_iter=60, state="f32",
                                                         schedule="resident"),
                               sample.shape[0], sample.data_ptr(), stream)
        out = gpu.decode_mixed(Cs, fc, torch.from_numpy(packed).cuda(), p)
        got = {k: v.cpu().numpy() for k, v in out.items()}
        alone = {c: {k: v.cpu().numpy() for k, v in gpu.decode(Cs[c], torch.from_numpy(llr).cuda(), p).items()}
                 for c, (idx, llr) in per.items()}
    finally:
        for C in Cs:
            C.close()
    for c, (idx, llr) in per.items():
        n = codes[c].n
        x = np.stack([got["x"][offsets[f]:offsets[f + 1]] for f in idx])
        b = np.stack([got["bits"][offsets[f]:offsets[f + 1]] for f in idx])
        assert np.array_equal(x, alone[c]["x"].reshape(len(idx), n)), codes[c].name
        assert np.array_equal(b, alone[c]["bits"].reshape(len(idx), n)), codes[c].name
        assert np.array_equal(got["iters"][idx], alone[c]["iters"]), codes[c].name
        assert np.array_equal(got["cert"][idx], alone[c]["cert"]), codes[c].name
    rng = np.random.default_rng(31)
    for c, (idx, llr) in per.items():
        code = codes[c]
        rows = rng.choice(len(idx), 6, replace=False)
        ref = oracle_mod.decode(code.row_ptr, code.col_idx, code.n, llr[rows].astype(np.float64), **kw)
        for k, r in enumerate(rows):
            f = idx[r]
            xg = got["x"][offsets[f]:offsets[f + 1]]
            if got["iters"][f] == ref["iters"][k]:
                assert np.abs(xg - ref["x"][k]).max() <= 1e-4, (code.name, f)
            else:
                assert_stop_near_threshold(oracle_mod, code, llr[r], got["iters"][f], ref["iters"][k], mu=3.0,
                                           rho=1.9, eps=1e-5)
