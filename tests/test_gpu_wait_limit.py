"""Failure handling of the STREAMED kernels without a GPU fault: the first
waits on a frame's parked-state copies (plain kernel) or on a ring slot's tag
and copies (ring kernel) are given a limit of one SM clock, so they run out.
The launch must still end (the copies in flight are waited for with the
default limit), every frame must be either finished with its normal result or
marked LPDEC_FRAME_ABANDONED, and the context must stay usable."""
import numpy as np
import pytest

from paper_1204_0556_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("ring", [0, 6])
def test_wait_limit_abandons_frames_and_the_gpu_stays_usable(gpu, ring):
    import torch

    code = I.benchmark_code("C1056", 0)
    F, iters = 600, 20
    llr = torch.from_numpy(I.awgn_llr(code, 2.0, F, 808)).cuda()
    C = gpu.Code(code)

    def run(schedule):
        out = {"x": torch.full((F, code.n), float("nan"), device="cuda"),
               "bits": torch.full((F, code.n), 7, dtype=torch.uint8, device="cuda"),
               "iters": torch.full((F,), -7, dtype=torch.int32, device="cuda"),
               "cert": torch.full((F,), 7, dtype=torch.uint8, device="cuda")}
        gpu.decode(C, llr, gpu.make_params(mu=3.0, rho=1.9, eps=0.0, max_iter=iters, schedule=schedule), out=out)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in out.items()}

    try:
        gpu.lpdec_set_tile(C.handle, 0, 192, 5)
        if ring:
            gpu.lpdec_set_streamed_tile(C.handle, 0, 192, 5, ring)
        ref = run("resident")
        gpu.lpdec_set_wait_limit(1)
        try:
            got = run("streamed")
        finally:
            gpu.lpdec_set_wait_limit(0)
        done = got["iters"] == iters
        abandoned = got["iters"] == gpu.LPDEC_FRAME_ABANDONED
        assert np.all(done | abandoned)
        assert np.all(got["cert"][abandoned] == 0)
        for k in ("x", "bits", "cert"):
            assert np.array_equal(got[k][done], ref[k][done]), k
        if ring:  # groups claim slots before the producer fills them: some tag waits run out
            assert abandoned.any()
        print(f"ring={ring}: {int(abandoned.sum())} of {F} frames abandoned, {int(done.sum())} finished")
        # the default limit again: the same decode gives every frame's normal result
        again = run("streamed")
        for k in ref:
            assert np.array_equal(again[k], ref[k]), k
    finally:
        C.close()
