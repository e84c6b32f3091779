"""Parity of the CUDA dual subgradient decoder (appendix, Algorithm 3) with the
FP64 oracle.  Every decision of the method is exact on both sides (lambda is
an integer multiple of mu; the steps used here are dyadic, so the oracle's
lambda sums are exact too), so x, bits, iteration counts and certificates must
be identical, frame by frame."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1204_0556_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _gpu_dual(L, code_obj, llr32, mu, max_iter):
    import torch

    c = L.Code(code_obj)
    try:
        out = L.decode_dual(c, torch.from_numpy(llr32).cuda(), mu=mu, max_iter=max_iter)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in out.items()}
    finally:
        c.close()


def _assert_identical(got, want):
    np.testing.assert_array_equal(got["iters"], want["iters"])
    np.testing.assert_array_equal(got["cert"], want["cert"])
    np.testing.assert_array_equal(got["bits"], want["bits"])
    np.testing.assert_array_equal(got["x"].astype(np.float64), want["x"])


def _run_both(gpu, oracle_mod, code, llr32, mu, max_iter):
    got = _gpu_dual(gpu, code, llr32, mu, max_iter)
    want = oracle_mod.decode_dual(code.row_ptr, code.col_idx, code.n, llr32.astype(np.float64), mu=mu,
                                  max_iter=max_iter)
    _assert_identical(got, want)
    return got


@pytest.mark.parametrize("mu", [0.25, 0.5, 1.0])
@pytest.mark.parametrize("ebn0", [2.0, 4.0])
def test_c96_identical(gpu, oracle_mod, mu, ebn0):
    code = I.benchmark_code("C96", 0)
    llr = I.awgn_llr(code, ebn0, 300, 40 + int(ebn0))
    _run_both(gpu, oracle_mod, code, llr, mu, 1500)


def test_c1056_identical(gpu, oracle_mod):
    """Regular (3,6) form (check degree 6, variable degree 3) on the headline code."""
    code = I.benchmark_code("C1056", 1)
    llr = I.awgn_llr(code, 3.5, 400, 5)
    got = _run_both(gpu, oracle_mod, code, llr, 0.25, 3000)
    assert got["cert"].mean() > 0.8


@pytest.mark.parametrize("name,ebn0,frames", [("C2640", 3.5, 96), ("C4000", 4.5, 48), ("C8000", 4.0, 24)])
def test_other_forms_identical(gpu, oracle_mod, name, ebn0, frames):
    """(4,8) regular form, the generic form with 30-wide checks, and an
    irregular code (check degrees 6..20)."""
    code = I.benchmark_code(name, 1)
    llr = I.awgn_llr(code, ebn0, frames, 9)
    _run_both(gpu, oracle_mod, code, llr, 0.25, 2000)


def test_global_index_form_identical(gpu, oracle_mod):
    """A code whose 16-bit index copy does not fit in shared memory beside a
    frame's state: the kernel reads the int32 index arrays from global memory."""
    code = I.gallager_code(12000, 3, 6, 3)
    llr = I.awgn_llr(code, 4.0, 12, 2)
    _run_both(gpu, oracle_mod, code, llr, 0.25, 600)


def test_ties_at_the_heaviside_step(gpu, oracle_mod):
    """LLRs on a grid of mu/2 make -gamma_i - mu S_i hit exactly zero (x = 0
    there) and give equal entries within checks (Algorithm 3's ties)."""
    code = I.benchmark_code("C1056", 1)
    rng = np.random.default_rng(3)
    mu = 0.5
    llr = (rng.integers(-3, 9, size=(64, code.n)) * (mu / 2)).astype(np.float32)
    _run_both(gpu, oracle_mod, code, llr, mu, 800)


def test_first_iteration_and_ragged_batch(gpu, oracle_mod):
    code = I.benchmark_code("C1056", 1)
    llr = I.awgn_llr(code, 1.0, 37, 8)
    got = _run_both(gpu, oracle_mod, code, llr, 0.25, 1)
    np.testing.assert_array_equal(got["bits"], (llr < 0).astype(np.uint8))


def test_bad_llr_frame(gpu, oracle_mod):
    code = I.benchmark_code("C96", 0)
    llr = I.awgn_llr(code, 4.0, 10, 1)
    llr[3, 7] = np.nan
    llr[6, 0] = np.inf
    got = _gpu_dual(gpu, code, llr, 0.25, 500)
    assert got["iters"][3] == -1 and got["iters"][6] == -1
    assert not got["x"][3].any() and not got["cert"][3]
    ok = [f for f in range(10) if f not in (3, 6)]
    want = oracle_mod.decode_dual(code.row_ptr, code.col_idx, code.n, llr[ok].astype(np.float64), mu=0.25,
                                  max_iter=500)
    np.testing.assert_array_equal(got["iters"][ok], want["iters"])
    np.testing.assert_array_equal(got["bits"][ok], want["bits"])


def test_tiles_agree(gpu, oracle_mod):
    """Any valid tile gives the same outputs; invalid tiles are rejected."""
    import torch

    code = I.benchmark_code("C1056", 1)
    llr = torch.from_numpy(I.awgn_llr(code, 3.0, 100, 12)).cuda()
    c = gpu.Code(code)
    try:
        ref = {k: v.cpu() for k, v in gpu.decode_dual(c, llr, mu=0.25, max_iter=2000).items()}
        for gt, g in ((32, 1), (64, 7), (128, 5), (256, 4), (96, 10)):
            gpu.lpdec_dual_set_tile(c.handle, gt, g)
            out = gpu.decode_dual(c, llr, mu=0.25, max_iter=2000)
            for k in ref:
                assert torch.equal(out[k].cpu(), ref[k]), (gt, g, k)
        for gt, g in ((48, 2), (32, 16), (512, 4)):
            with pytest.raises(gpu.LpdecError):
                gpu.lpdec_dual_set_tile(c.handle, gt, g)
        gpu.lpdec_dual_set_tile(c.handle, 0, 0)
    finally:
        c.close()


def test_argument_errors_and_empty_batch(gpu):
    import torch

    code = I.benchmark_code("C96", 0)
    c = gpu.Code(code)
    try:
        empty = torch.empty((0, code.n), dtype=torch.float32, device="cuda")
        out = gpu.decode_dual(c, empty, mu=0.25, max_iter=10)
        assert out["x"].shape == (0, code.n)
        llr = torch.zeros((2, code.n), dtype=torch.float32, device="cuda")
        for mu, it in ((0.0, 10), (-1.0, 10), (float("nan"), 10), (0.25, 0), (0.25, 40000)):
            with pytest.raises(gpu.LpdecError):
                gpu.decode_dual(c, llr, mu=mu, max_iter=it)
    finally:
        c.close()
