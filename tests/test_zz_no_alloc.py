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


@pytest.mark.parametrize("schedule,eps,ring", [("resident", 1e-5, 0), ("streamed", 0.0, 0), ("streamed", 0.0, 6)])
def test_noalloc_matches_decode_twice(gpu, schedule, eps, ring):
    """Both entry points run the same kernels with the same tile, so the outputs
    are identical bit for bit.  ring = 6: the STREAMED tile is set to the ring
    kernel (5 groups of 192 threads, 6 slots), whose bulk copies read the
    parked state out of the fixed array."""
    import torch

    code = I.benchmark_code("C1056", 0)
    C = gpu.Code(code)
    try:
        if ring:
            gpu.lpdec_set_streamed_tile(C.handle, 0, 192, 5, ring)
            assert gpu.lpdec_get_tile(C.handle, 0, gpu.SCHED_STREAMED)["ring_slots"] == ring
        s = int(torch.cuda.current_stream().cuda_stream)
        p = gpu.make_params(mu=3.0, rho=1.9, eps=eps, max_iter=120, schedule=schedule)
        for call, seed in enumerate((31, 32)):  # two calls in a row share the fixed scratch
            llr = torch.from_numpy(I.awgn_llr(code, 2.0, 96, seed)).cuda()
            ref = _outputs(torch, 96, code.n)
            got = _outputs(torch, 96, code.n)
            _call(gpu.lpdec_decode, C, llr, p, ref, s)
            _call(gpu.lpdec_decode_noalloc, C, llr, p, got, s)
            torch.cuda.synchronize()
            for k in ("x", "bits", "iters", "cert"):
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
