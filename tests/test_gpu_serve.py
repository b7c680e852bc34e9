"""Serving on the GPU: requests of different shapes and operators solved
alone and concurrently in the continuous-batching loop give identical
results (the kernels' arithmetic depends neither on what else runs nor on
the number of CTAs a request's sweep gets)."""
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
    from paper_2311_03824_gb300 import serve as S
    reqs = small_mix()
    stream = torch.cuda.Stream()
    alone = {rq.rid: S.solve_on_device(rq, stream, grid=0, keep_outputs=True) for rq in reqs}
    free = torch.cuda.mem_get_info()[0]
    srv = S.Server(int(0.5 * free), slots=4, keep_outputs=True)
    res = srv.run(reqs)
    assert srv.peak_running >= 2          # the requests did run concurrently
    for r in res:
        assert r.error is None, r.error
        out_a, err_a = alone[r.rid]
        for a, b in zip(out_a, r.outputs):
            assert np.array_equal(a, b), r.rid
        assert r.rel_err == err_a
    summ = S.summarize(res, srv.makespan, reqs)
    assert summ["failed"] == 0 and summ["p99_latency_s"] >= summ["p50_latency_s"] > 0
