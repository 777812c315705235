"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own
timing, agree on the slowest rank's time and on the whole-job rate (weak
scaling: every rank steps its own box, no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = [120.0, 150.0][rank]
    ms_max = bench.max_over_ranks(ms_local, world, dist, "cpu")
    rate = bench.whole_job_rate(256 ** 3, 100, ms_max, world)
    q.put((rank, ms_max, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, ms_max, rate in out:
        assert ms_max == 150.0
        assert rate == pytest.approx(2 * 256 ** 3 * 100 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(10, 2, 1000.0, 1) == pytest.approx(20.0)


def test_committed_profile_matches_the_headline_kernel_sources():
    """The ncu summary the bench reads its DRAM traffic from was taken on the
    sources the headline kernel is compiled from now (their fingerprint: the
    FP32 tiled translation unit, the tile table and every header they
    include); a kernel change without a new capture fails here, as the
    bench's traffic would otherwise silently turn null."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    kv = bench.profile_summary("substep55_fp32_lag_tmem_256")
    assert kv is not None, "no committed profile for the current kernel sources"
    traffic = bench.profile_traffic("substep55_fp32_lag_tmem_256")
    gbs = bench.profile_dram_gbs("substep55_fp32_lag_tmem_256")
    # DRAM bytes per launch at least the algorithmic bytes (10 F w / 3 per
    # point at 256^3, F = 5, FP32), and an achieved rate below a few TB/s
    alg = 256 ** 3 * 10 * 5 * 4 / 3.0
    assert alg <= traffic < 1.5 * alg
    assert 1000.0 < gbs < 8000.0
