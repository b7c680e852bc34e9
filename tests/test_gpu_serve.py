"""Serving on the GPU through the native request server (lrs_server_*):
requests of different shapes and operators solved one at a time and
concurrently with continuous batching give identical results (the kernels'
arithmetic depends neither on what else runs nor on the number of CTAs a
request's sweep gets)."""
import numpy as np
import pytest

from tests.gpu_helpers import gpu_available

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_2311_03824_gb300 import build
    build.build()


def small_mix():
    from paper_2311_03824_gb300 import lrs as L
    from paper_2311_03824_gb300.serve import Request
    return [Request(0, "gaussian", 256, 64, 3, 80, 3, 11, T=20),
            Request(1, "gaussian", 320, 48, 5, 96, 4, 12, T=20),
            Request(2, "dft", 4096, 32, 4, 900, 41, 13, T=20, nx=64, ny=64, a_dtype=L.LRS_A_FP32),
            Request(3, "gaussian", 512, 80, 2, 128, 6, 14, T=20, a_dtype=L.LRS_A_FP8_HI),
            Request(4, "gaussian", 192, 64, 8, 64, 2, 15, T=20),
            Request(5, "dft", 4096, 48, 3, 1200, 60, 16, T=20, nx=64, ny=64, a_dtype=L.LRS_A_FP32)]


def test_alone_equals_mix():
    import torch
    import bench
    from paper_2311_03824_gb300 import serve as S
    reqs = small_mix()
    budget = int(0.5 * torch.cuda.mem_get_info()[0])
    gen_a = bench.C4Inputs()
    inputs_a = {rq.rid: gen_a(rq) for rq in reqs}
    alone = S.Server(budget, slots=1, keep_outputs=True).run(reqs, lambda rq: inputs_a[rq.rid])
    gen_a.score(alone, reqs)
    gen_m = bench.C4Inputs()
    # made before: the submissions take no time, so the requests queue together
    inputs_m = {rq.rid: gen_m(rq) for rq in reqs}
    srv = S.Server(budget, slots=4, keep_outputs=True)
    mix = srv.run(reqs, lambda rq: inputs_m[rq.rid])
    assert srv.peak_running >= 2          # the requests did run concurrently
    for a, r in zip(alone, mix):
        assert a.error is None and r.error is None, (a.error, r.error)
    # outputs compared before scoring consumes them
    gen_m.score(mix, reqs)
    for a, r in zip(alone, mix):
        assert r.rel_err == a.rel_err, r.rid
        assert r.rel_err < 0.5
    summ = S.summarize(mix, srv.makespan, reqs)
    assert summ["failed"] == 0 and summ["p99_latency_s"] >= summ["p50_latency_s"] > 0


def test_alone_equals_mix_bitwise():
    import torch
    import bench
    from paper_2311_03824_gb300 import serve as S
    reqs = small_mix()
    budget = int(0.5 * torch.cuda.mem_get_info()[0])
    alone = S.Server(budget, slots=1, keep_outputs=True).run(reqs, bench.C4Inputs())
    mix = S.Server(budget, slots=4, keep_outputs=True).run(reqs, bench.C4Inputs())
    for a, r in zip(alone, mix):
        assert a.error is None and r.error is None
        for x, y in zip(a.outputs, r.outputs):
            assert np.array_equal(x, y), r.rid


def test_batched_requests_equal_alone_bitwise():
    """batch = 4: the Gaussian requests of one rank and A_k form queued
    together share one persistent launch per sweep; every output equals the
    request solved alone."""
    import torch
    import bench
    from paper_2311_03824_gb300 import serve as S
    from paper_2311_03824_gb300.serve import Request
    # request 0 (another rank) runs alone long enough for 1-4 to queue behind it
    reqs = [Request(0, "gaussian", 2048, 512, 8, 400, 20, 20, T=20),
            Request(1, "gaussian", 320, 48, 3, 96, 4, 22, T=20),
            Request(2, "gaussian", 200, 100, 3, 70, 2, 23, T=20),
            Request(3, "gaussian", 448, 32, 3, 120, 6, 24, T=20),
            Request(4, "gaussian", 256, 64, 5, 80, 3, 25, T=20)]
    budget = int(0.5 * torch.cuda.mem_get_info()[0])
    gen = bench.C4Inputs()
    inputs = {rq.rid: gen(rq) for rq in reqs}     # made before: submissions take no time
    alone = S.Server(budget, slots=1, keep_outputs=True).run(reqs, lambda rq: inputs[rq.rid])
    srv = S.Server(budget, slots=1, keep_outputs=True, batch=4)   # the queue forms
    batched = srv.run(reqs, lambda rq: inputs[rq.rid])
    # 1-4 are queued while request 0 runs: 1-3 (rank 3) form one batch
    assert [r.group_size for r in batched] == [1, 3, 3, 3, 1], [(r.group, r.group_size) for r in batched]
    for a, r in zip(alone, batched):
        assert a.error is None and r.error is None, (a.error, r.error)
        for x, y in zip(a.outputs, r.outputs):
            assert np.array_equal(x, y), r.rid
