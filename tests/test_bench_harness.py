"""bench.py's multi-process harness on CPU: world-size-2 gloo ranks agree on the
max-over-ranks time and pass the barriers (the path `--gpus N` takes with one
replica of the solve per GPU; no data-path collective exists)."""

import multiprocessing as mp
import os
import socket

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_env()
    bench.barrier(w)
    v = bench.reduce_max(1.5 * (r + 1), w)
    bench.barrier(w)
    q.put((r, w, v))
    dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 2, 3.0), (1, 2, 3.0)]


def test_single_process_harness_is_identity():
    assert bench.reduce_max(2.5, 1) == 2.5
    bench.barrier(1)


def test_dslash_algorithmic_bytes():
    # 16 links x 18 reals x 4 B + 2 vectors x 24 B = 1200 B; two-row Naik storage 1008 B
    assert bench.dslash_bytes_per_site("fp32", 18) == 1200
    assert bench.dslash_bytes_per_site("fp32", 12) == 1008
    assert bench.dslash_bytes_per_site("fp64", 12) == 2400
    assert bench.dslash_bytes_per_site("fx16", 12) == 512


def test_clock_summary_flags_throttling():
    c = bench.ClockSampler()
    c.samples = [(1900.0, 2070.0, 0x0, 99.0), (1800.0, 2070.0, 0x4, 99.0), (300.0, 2070.0, 0x1, 0.0)]
    s = c.summary()
    assert s["sm_mhz"] == 1850.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_oracle_cpu_baseline_runs_one_process_per_source():
    """The CPU baseline's process pool (spawned workers, links in shared
    memory) on a small lattice: four sources, four workers, a positive
    per-source time scaled to the requested iteration count, and the same
    number of iterations timed on every source."""
    import synth

    dims = (4, 4, 4, 6)
    fat, lng = synth.gauge_field(dims, 0.3, 1000)
    srcs = [synth.gaussian_source(dims, 5000 + k) for k in range(4)]
    old = bench.DIMS
    bench.DIMS = dims  # the workers receive the parent's lattice with each task
    try:
        pool = bench.OraclePool(fat, lng, 4)
        try:
            wall, per = pool.sample(srcs, 2)
        finally:
            pool.close()
    finally:
        bench.DIMS = old
    assert pool.workers == 4 and len(per) == 4 and all(t > 0 for t in per) and wall > 0
