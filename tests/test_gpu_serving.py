"""Continuous batching (lse_serve_*): requests that arrive while others run
are admitted as slots and memory free up, their work overlaps on the device,
and every result equals the same request fitted alone.  The requests here are
small (N <= 512, groups of at most 5), so every group and every lone fit runs
in the same mode (two-block clusters on the double-float path) and the
results must agree bit for bit."""
import time

import numpy as np
import pytest

from paper_1705_06073_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lse_mod():
    from paper_1705_06073_gb300 import build, lse
    build.build()
    return lse


def requests(n=24, seed=5500):
    rs = synth.Stream(seed)
    out = []
    for i in range(n):
        u = rs.uniform(3)
        N = int(round(2.0 ** (6.0 + 3.0 * float(u[0]))))  # 64 .. 512, log-uniform
        K = 2 + int(u[1] * max(1, N // 32 - 2))
        out.append(synth.make_instance(N, K, 5.0 + 20.0 * float(u[2]), seed + i))
    return out


def test_results_are_the_same_alone_and_in_the_mix(lse_mod):
    lse = lse_mod
    cfg = lse.lse_config_default(precision=lse.LSE_PREC_MIXED_DF)
    reqs = requests()
    srv = lse.Server(cfg, streams=4, max_group=5, K_cap=1024)
    got = {}
    try:
        # staggered arrivals: submit in bursts while earlier groups are running
        for i, inst in enumerate(reqs):
            assert srv.submit(inst.y, i) == lse.LSE_OK
            if i % 6 == 5:
                for r in srv.poll():
                    got[r["request_id"]] = r
        t0 = time.time()
        while srv.in_flight() and time.time() - t0 < 120:
            for r in srv.poll():
                got[r["request_id"]] = r
            time.sleep(0.001)
        assert srv.in_flight() == 0
    finally:
        srv.close()
    assert sorted(got) == list(range(len(reqs)))
    ctx = lse.lse_create(cfg)
    try:
        for i, inst in enumerate(reqs):
            alone = lse.lse_fit(ctx, inst.y)
            r = got[i]
            assert r["status"] == lse.LSE_OK
            assert r["K"] == alone["K"]
            assert np.array_equal(r["theta"], alone["theta"])
            assert np.array_equal(r["gamma"], alone["gamma"])
            assert r["beta"] == alone["beta"] and r["n_evals"] == alone["n_evals"]
    finally:
        lse.lse_destroy(ctx)


def test_admission_by_device_memory_budget(lse_mod):
    lse = lse_mod
    budget = 64 << 20  # 64 MiB: a few small groups at a time
    cfg = lse.lse_config_default(precision=lse.LSE_PREC_MIXED_DF, hbm_budget_bytes=budget)
    srv = lse.Server(cfg, streams=8, max_group=8, K_cap=1024)
    try:
        # a request whose workspace alone exceeds the budget is refused
        big = np.ones(65536, np.complex64)
        assert srv.submit(big, 999) == lse.LSE_EBUDGET
        reqs = requests(16, seed=7700)
        for i, inst in enumerate(reqs):
            assert srv.submit(inst.y, i) == lse.LSE_OK
        peak = 0
        got = {}
        t0 = time.time()
        while srv.in_flight() and time.time() - t0 < 120:
            peak = max(peak, srv.device_bytes())
            for r in srv.poll():
                got[r["request_id"]] = r
        assert sorted(got) == list(range(16))
        assert all(r["status"] == lse.LSE_OK for r in got.values())
        assert 0 < peak <= budget
    finally:
        srv.close()
