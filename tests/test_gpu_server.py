"""Continuous-batching server: results equal lone decodes, error codes, drain on destroy."""
import time

import numpy as np
import pytest

from _stopping import assert_stop_near_threshold
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
    t0 = time.perf_counter()
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
        ctr = srv.counters()
        wall_ms = (time.perf_counter() - t0) * 1000.0
    finally:
        srv.close()
    assert st["frames"] == sum(len(llr) for _, llr, _ in plan)
    assert st["p99_ms"] >= st["p50_ms"] > 0
    # every code ran rounds of its own; the device-busy time is the union of
    # the rounds' spans, so it lies within the wall time
    assert ctr["rounds"] >= 4
    assert 0 < ctr["round_gpu_ms"] <= wall_ms
    for (c, llr, _), got in zip(plan, results):
        assert got is not None
        ref = gpu_decode(gpu, codes[c], llr, mu=3.0, rho=1.9, eps=1e-5, max_iter=600)
        for k in ("x", "bits", "iters", "cert"):
            assert np.array_equal(got[k], ref[k]), (codes[c].name, k)


def test_served_frames_match_the_oracle(gpu, oracle_mod, server_codes):
    """Served frames against the FP64 oracle directly (Algorithm 1 per frame):
    fixed-iteration requests of three codes arrive while others are in flight;
    every frame's x is within 1e-4 of the oracle's decode of that frame, and
    bits, certificates and syndromes agree on frames with no oracle entry near
    1/2 or the certificate bound."""
    from test_gpu_decode import assert_parity, oracle_decode

    codes, handles = server_codes
    kw = dict(mu=3.0, rho=1.9, eps=0.0, max_iter=120)
    p = gpu.make_params(iters_per_launch=8, **kw)
    srv = gpu.Server(budget_bytes=2 << 30)
    try:
        ids = [srv.add_code(h) for h in handles[:3]]
        rng = np.random.default_rng(21)
        plan = []
        for r in range(24):
            c = int(rng.integers(0, 3))
            llr = I.awgn_llr(codes[c], float(rng.uniform(1.5, 4.0)), 2, 7000 + r)
            plan.append((c, llr, srv.submit(ids[c], llr, p)))
            if r % 5 == 0:
                time.sleep(0.002)
        results = [srv.poll(rid, ids[c], len(llr), timeout_ms=60_000) for c, llr, rid in plan]
    finally:
        srv.close()
    for c in range(3):
        got_parts = [g for (cc, _, _), g in zip(plan, results) if cc == c]
        if not got_parts:
            continue
        llr = np.concatenate([l for cc, l, _ in plan if cc == c])
        got = {k: np.concatenate([g[k] for g in got_parts]) for k in ("x", "bits", "iters", "cert")}
        ref = oracle_decode(oracle_mod, codes[c], llr, **kw)
        assert_parity(codes[c], got, ref, 1e-4, min_clean=0.3)


def test_add_code_while_frames_in_flight(gpu, server_codes):
    """Codes may be added while the scheduler runs rounds for others: the
    round works on its own copy of the pool list, so the list growing (and
    reallocating) under it is harmless, and the new codes join later rounds.
    Every result still equals lpdec_decode of the frame alone."""
    from test_gpu_decode import gpu_decode

    codes, handles = server_codes
    p = gpu.make_params(mu=3.0, rho=1.9, eps=1e-5, max_iter=300, iters_per_launch=4)
    srv = gpu.Server(budget_bytes=6 << 30)
    try:
        first = srv.add_code(handles[1])
        plan = []
        for r in range(16):
            llr = I.awgn_llr(codes[1], 1.5, 8, 8100 + r)
            plan.append((first, 1, llr, srv.submit(first, llr, p)))
        # twelve more pools, added one by one between submits while C1056 frames run
        for k in range(12):
            c = (0, 2, 1)[k % 3]
            cid = srv.add_code(handles[c])
            llr = I.awgn_llr(codes[c], 2.5, 2, 8200 + k)
            plan.append((cid, c, llr, srv.submit(cid, llr, p)))
        results = [srv.poll(rid, cid, len(llr), timeout_ms=120_000) for cid, _, llr, rid in plan]
    finally:
        srv.close()
    for (cid, c, llr, _), got in zip(plan, results):
        assert got is not None
        ref = gpu_decode(gpu, codes[c], llr, mu=3.0, rho=1.9, eps=1e-5, max_iter=300)
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


def test_served_stream_of_the_bench(gpu, oracle_mod, server_codes):
    """The served workload of `bench.py --workload served` in its configuration
    (C96 / C1056 / C2640 / C8000 with the bench's seeds, codes drawn per request
    by Philox key 6, the bench's pools of 2048 frames per code, eps = 1e-5, at
    most 1000 iterations, rounds of 8 iterations, 8 GB budget), 20,000 one-frame
    requests queued as fast as they can be submitted: every result equals
    lpdec_decode of the same frame, and two frames per code match the oracle."""
    import torch

    codes, handles = server_codes
    POOL, R = 2048, 20_000
    snr_rng = np.random.Generator(np.random.Philox(key=7))
    pools = [I.awgn_llr(c, snr_rng.uniform(1.5, 4.5, POOL), POOL, 8 + 10 * k) for k, c in enumerate(codes)]
    which = np.random.Generator(np.random.Philox(key=6)).integers(0, 4, R).astype(np.int32)
    cursor = [0, 0, 0, 0]
    frame_of = np.zeros(R, dtype=np.int64)
    for i, c in enumerate(which):
        frame_of[i] = cursor[c]
        cursor[c] = (cursor[c] + 1) % POOL
    kw = dict(mu=3.0, rho=1.9, eps=1e-5, max_iter=1000)
    p = gpu.make_params(state="f32", iters_per_launch=8, **kw)
    srv = gpu.Server(budget_bytes=8 << 30)
    try:
        ids = [srv.add_code(h) for h in handles]
        rids = [srv.submit(ids[c], pools[c][frame_of[i]], p) for i, c in enumerate(which)]
        got = [srv.poll(rid, ids[c], 1, timeout_ms=300_000) for rid, c in zip(rids, which)]
    finally:
        srv.close()
    pr = gpu.make_params(state="f32", schedule="resident", **kw)
    for c in range(4):
        ref = {k: v.cpu().numpy() for k, v in gpu.decode(handles[c], torch.from_numpy(pools[c]).cuda(), pr).items()}
        for i in np.nonzero(which == c)[0]:
            g, f = got[i], frame_of[i]
            assert g is not None
            assert np.array_equal(g["x"][0], ref["x"][f]), (codes[c].name, i)
            assert np.array_equal(g["bits"][0], ref["bits"][f]), (codes[c].name, i)
            assert g["iters"][0] == ref["iters"][f] and g["cert"][0] == ref["cert"][f], (codes[c].name, i)
        rows = np.nonzero(which == c)[0][:2]
        llr = np.stack([pools[c][frame_of[i]] for i in rows])
        oref = oracle_mod.decode(codes[c].row_ptr, codes[c].col_idx, codes[c].n, llr.astype(np.float64), **kw)
        for k, i in enumerate(rows):
            if got[i]["iters"][0] == oref["iters"][k]:
                assert np.abs(got[i]["x"][0] - oref["x"][k]).max() <= 1e-4, (codes[c].name, i)
            else:
                assert_stop_near_threshold(oracle_mod, codes[c], llr[k], got[i]["iters"][0], oref["iters"][k],
                                           mu=3.0, rho=1.9, eps=1e-5)
