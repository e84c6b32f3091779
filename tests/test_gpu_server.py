"""Continuous-batching server: results equal lone decodes, error codes, drain on destroy."""
import time

import numpy as np
import pytest

from paper_1204_0556_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def server_codes(gpu):
    names = ["C96", "C1056", "C2640", "C8000"]
    codes = [I.benchmark_code(nm, k) for k, nm in enumerate(names)]
    handles = [gpu.Code(c) for c in codes]
    yield codes, handles
    for h in handles:
        h.close()


def test_results_identical_alone_and_in_the_mix(gpu, server_codes):
    """Requests of four codes arrive while others are in flight; every frame's
    result equals lpdec_decode of that frame on its own."""
    from test_gpu_decode import gpu_decode

    codes, handles = server_codes
    p = gpu.make_params(mu=3.0, rho=1.9, eps=1e-5, max_iter=600, iters_per_launch=8)
    srv = gpu.Server(budget_bytes=2 << 30)
    try:
        ids = [srv.add_code(h) for h in handles]
        rng = np.random.default_rng(9)
        plan = []
        for r in range(60):
            c = int(rng.integers(0, 4))
            nf = int(rng.integers(1, 4))
            llr = I.awgn_llr(codes[c], float(rng.uniform(1.5, 4.5)), nf, 5000 + r)
            plan.append((c, llr, srv.submit(ids[c], llr, p)))
            if r % 7 == 0:
                time.sleep(0.002)  # let rounds start while more requests arrive
        results = [srv.poll(rid, ids[c], len(llr), timeout_ms=60_000) for c, llr, rid in plan]
        st = srv.stats()
    finally:
        srv.close()
    assert st["frames"] == sum(len(llr) for _, llr, _ in plan)
    assert st["p99_ms"] >= st["p50_ms"] > 0
    for (c, llr, _), got in zip(plan, results):
        assert got is not None
        ref = gpu_decode(gpu, codes[c], llr, mu=3.0, rho=1.9, eps=1e-5, max_iter=600)
        for k in ("x", "bits", "iters", "cert"):
            assert np.array_equal(got[k], ref[k]), (codes[c].name, k)


def test_poll_timeout_and_errors(gpu, server_codes):
    codes, handles = server_codes
    p = gpu.make_params(eps=0.0, max_iter=1000, iters_per_launch=4)
    srv = gpu.Server(budget_bytes=1 << 30)
    try:
        cid = srv.add_code(handles[3])  # C8000: 1000 iterations of 512 frames take far longer than 0 ms
        rid = srv.submit(cid, I.awgn_llr(codes[3], 1.0, 512, 77), p)
        assert srv.poll(rid, cid, 512, timeout_ms=0) is None  # LPDEC_ETIMEOUT: not done yet
        with pytest.raises(gpu.LpdecError) as ei:  # a code's requests share one parameter set
            srv.submit(cid, I.awgn_llr(codes[3], 1.0, 1, 78), gpu.make_params(eps=0.0, max_iter=999))
        assert ei.value.status == gpu.LPDEC_EINVAL
        with pytest.raises(gpu.LpdecError):
            srv.submit(cid + 5, I.awgn_llr(codes[3], 1.0, 1, 79), p)
        assert srv.poll(rid, cid, 512, timeout_ms=120_000) is not None
        with pytest.raises(gpu.LpdecError):  # already released
            srv.poll(rid, cid, 512, timeout_ms=0)
    finally:
        srv.close()


def test_budget_exhaustion(gpu, server_codes):
    codes, handles = server_codes
    srv = gpu.Server(budget_bytes=4096)
    try:
        cid = srv.add_code(handles[1])
        with pytest.raises(gpu.LpdecError) as ei:
            srv.submit(cid, I.awgn_llr(codes[1], 2.0, 1, 1), gpu.make_params())
        assert ei.value.status == gpu.LPDEC_ENOMEM
    finally:
        srv.close()


def test_destroy_drains_submitted_frames(gpu, server_codes):
    codes, handles = server_codes
    srv = gpu.Server(budget_bytes=1 << 30)
    cid = srv.add_code(handles[1])
    for r in range(10):
        srv.submit(cid, I.awgn_llr(codes[1], 2.0, 4, 600 + r), gpu.make_params(eps=1e-5, max_iter=200,
                                                                                iters_per_launch=8))
    srv.close()  # returns after the worker finished every submitted frame
