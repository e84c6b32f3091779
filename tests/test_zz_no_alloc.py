"""lpdec_decode_noalloc: decoding for callers that cannot allocate device memory
while they run (fixed-footprint receive loops, hosts whose allocator owns all
device memory).  Its output must equal lpdec_decode's on the same inputs, call
after call, although every call reuses the same fixed scratch array."""
import numpy as np
import pytest

from paper_1204_0556_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _outputs(torch, F, n):
    return {
        "x": torch.empty((F, n), dtype=torch.float32, device="cuda"),
        "bits": torch.empty((F, n), dtype=torch.uint8, device="cuda"),
        "iters": torch.empty((F,), dtype=torch.int32, device="cuda"),
        "cert": torch.empty((F,), dtype=torch.uint8, device="cuda"),
    }


def _call(fn, C, llr, p, out, stream):
    fn(C.handle, llr.shape[0], llr.data_ptr(), p, out["x"].data_ptr(), out["bits"].data_ptr(),
       out["iters"].data_ptr(), out["cert"].data_ptr(), stream)


@pytest.mark.parametrize("schedule,eps", [("resident", 1e-5), ("streamed", 0.0)])
def test_noalloc_matches_decode_twice(gpu, schedule, eps):
    import torch

    code = I.benchmark_code("C1056", 0)
    C = gpu.Code(code)
    try:
        s = int(torch.cuda.current_stream().cuda_stream)
        p = gpu.make_params(mu=3.0, rho=1.9, eps=eps, max_iter=120, schedule=schedule)
        for call, seed in enumerate((31, 32)):  # two calls in a row share the fixed scratch
            llr = torch.from_numpy(I.awgn_llr(code, 2.0, 96, seed)).cuda()
            ref = _outputs(torch, 96, code.n)
            got = _outputs(torch, 96, code.n)
            _call(gpu.lpdec_decode, C, llr, p, ref, s)
            _call(gpu.lpdec_decode_noalloc, C, llr, p, got, s)
            torch.cuda.synchronize()
            err = (got["x"] - ref["x"]).abs().max().item()
            assert err <= 1e-4, (call, err)
            for k in ("bits", "iters", "cert"):
                assert torch.equal(got[k], ref[k]), (call, k)
    finally:
        C.close()


def test_noalloc_rejects_oversized_scratch(gpu):
    import torch

    code = I.benchmark_code("C1056", 0)
    C = gpu.Code(code)
    try:
        F = 2000  # STREAMED FP32 state: 2 x 2000 x 3168 x 4 B = 50.7 MB > 32 MiB
        llr = torch.zeros((F, code.n), dtype=torch.float32, device="cuda")
        out = _outputs(torch, F, code.n)
        p = gpu.make_params(eps=0.0, max_iter=10, schedule="streamed")
        with pytest.raises(gpu.LpdecError) as ei:
            _call(gpu.lpdec_decode_noalloc, C, llr, p, out, int(torch.cuda.current_stream().cuda_stream))
        assert ei.value.status == gpu.LPDEC_ENOMEM
        assert "scratch" in str(ei.value)
    finally:
        C.close()
