"""CUDA-graph capture: the mixed-code plan launch and the single-code decode,
captured once and replayed on new LLRs, match direct decodes."""
import numpy as np
import pytest

from paper_1204_0556_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _buffers(torch, total, F):
    return {"x": torch.empty(total, dtype=torch.float32, device="cuda"),
            "bits": torch.empty(total, dtype=torch.uint8, device="cuda"),
            "iters": torch.empty(F, dtype=torch.int32, device="cuda"),
            "cert": torch.empty(F, dtype=torch.uint8, device="cuda")}


def test_mixed_plan_captured_in_a_graph(gpu):
    import torch

    from test_gpu_mixed import _mixed_batch

    codes, fc, frames = _mixed_batch(["C1056", "C2640", "C4000"], [8, 6, 4], seed=13)
    _, _, frames2 = _mixed_batch(["C1056", "C2640", "C4000"], [8, 6, 4], seed=14)
    Cs = [gpu.Code(c) for c in codes]
    p = gpu.make_params(mu=3.0, rho=1.9, eps=1e-5, max_iter=300)
    plan = gpu.lpdec_mixed_plan_create([C.handle for C in Cs], fc, p)
    try:
        total = sum(len(f) for f in frames)
        llr = torch.from_numpy(np.concatenate(frames).astype(np.float32)).cuda()
        out = _buffers(torch, total, len(fc))
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                gpu.lpdec_mixed_plan_decode(plan, llr.data_ptr(), out["x"].data_ptr(), out["bits"].data_ptr(),
                                            out["iters"].data_ptr(), out["cert"].data_ptr(), int(s.cuda_stream))
        for batch in (frames, frames2):  # replay twice, on two different batches
            llr.copy_(torch.from_numpy(np.concatenate(batch).astype(np.float32)))
            g.replay()
            torch.cuda.synchronize()
            ref = gpu.decode_mixed(Cs, fc, torch.from_numpy(np.concatenate(batch).astype(np.float32)).cuda(), p)
            torch.cuda.synchronize()
            for k in out:
                assert torch.equal(out[k], ref[k]), k
    finally:
        gpu.lpdec_mixed_plan_destroy(plan)
        for C in Cs:
            C.close()


@pytest.mark.parametrize("schedule", ["resident", "streamed"])
def test_single_code_decode_captured_in_a_graph(gpu, schedule):
    import torch

    code = I.benchmark_code("C96", 0)
    C = gpu.Code(code)
    try:
        p = gpu.make_params(eps=0.0, max_iter=50, schedule=schedule)
        llr = torch.from_numpy(I.awgn_llr(code, 2.0, 32, 5)).cuda()
        out = _buffers(torch, 32 * code.n, 32)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                gpu.lpdec_decode(C.handle, 32, llr.data_ptr(), p, out["x"].data_ptr(), out["bits"].data_ptr(),
                                 out["iters"].data_ptr(), out["cert"].data_ptr(), int(s.cuda_stream))
        llr.copy_(torch.from_numpy(I.awgn_llr(code, 2.0, 32, 6)))
        g.replay()
        torch.cuda.synchronize()
        ref = gpu.decode(C, llr.clone(), p)
        torch.cuda.synchronize()
        assert torch.equal(out["x"].view(32, -1), ref["x"]) and torch.equal(out["iters"], ref["iters"])
    finally:
        C.close()
