"""Benchmark: 32^4 improved-staggered even-odd CG to 1e-10, mixed vs plain FP64.

Workload (the paper's staggered CG, Sec. 4.1, on a synthetic stand-in for its
equilibrated ensembles): 32^4 lattice, thin links exp(0.3 i H) reunitarised,
fat = U + 1/8 staples, Naik = -1/24 UUU, periodic, m = 0.01, 4 seeded
Gaussian even-site sources, FP64 true relative residual 1e-10.

A step solves all 4 sources with the chosen solver: mixed-precision CG
(FP32 sloppy operator and vectors, FP64 reliable updates) on the 4 sources
at once, one stag_batch_solve call through the C ABI (every system its own
CG and stopping point, one multi-right-hand-side Dslash per operator
application), inputs resident in HBM.  `value` is seconds per source solve.
The same JSON line carries the plain FP64 CG time (stag_cg per source), the
Dslash roofline (device time of the dominant kernel per launch, measured
with CUDA events on its launch stream during the timed region), the
end-to-end time with host buffers, the oracle's CPU time on a bounded
sample, and the SM clocks seen.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Dslash HBM GB/s (% peak); 32^4 CG secs to 1e-10 rel. residual, plain vs chosen"
DIMS = (32, 32, 32, 32)
EPS = 0.3
MASS = 0.01
NSRC = 4
TOL = 1e-10
GAUGE_SEED = 1000
SOURCE_SEEDS = [5000 + k for k in range(NSRC)]
CHOSEN = "mixed32"
BATCHED = True  # the 4 sources in one batched call (multi-right-hand-side operator)
RECON = 12
FLOP_PER_SITE = 1146
# algorithmic bytes per output site of one Dslash: 16 link matrices (8 fat x
# 9 complex + 8 Naik x NL complex) read once, the input vector read once,
# the output written once
ELEM_BYTES = {"fp64": 16, "fp32": 8, "fp16": 4, "fx16": 4, "df64": 16, "fx16l": 4}
VEC_BYTES = {"fp64": 48, "fp32": 24, "fp16": 16, "fx16": 16, "df64": 48, "fx16l": 24}
MODE_PREC = {"plain64": "fp64", "mixed32": "fp32", "mixed16": "fp16", "mixedfx16": "fx16", "mixed16l": "fx16l"}
# arithmetic type of the Krylov loop of each solver mode (FP32 arithmetic on
# 16-bit storage for the 16-bit modes)
DTYPE = {"plain64": "f64", "mixed32": "f32", "mixed16": "f32", "mixedfx16": "f32", "mixed16l": "f32"}


# the library's kernel families (stag.h, instrumentation)
FAMILIES = ("dslash", "dslash_epi", "dslash64", "dslash64_epi", "dslash_mrhs", "dslash_mrhs_epi", "dslash_mrhs64",
            "dslash_mrhs64_epi", "dslash_df", "dslash_df_epi", "blas", "reduce", "convert")


def dslash_bytes_per_site(prec, recon):
    nl = 6 if (recon == 12 and prec != "fp64") else 9
    return (8 * 9 + 8 * nl) * ELEM_BYTES[prec] + 2 * VEC_BYTES[prec]


def kernel_source_hash(kernel_id="k_dslash"):
    h = hashlib.sha256()
    files = ("dslash_impl.cuh", "common.cuh", "links.cu")
    if kernel_id.startswith("k_dslash_m"):
        files = files + ("mrhs_kernels.cuh", "dslash_mrhs.cuh")
    for f in files:
        with open(os.path.join(ROOT, "paper_1712_00143_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def ncu_traffic(kernel_id):
    """dram bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "dslash_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    ent = d.get(kernel_id)
    if not ent or ent.get("source_hash") != kernel_source_hash(kernel_id):
        return None
    return ent.get("bytes_per_launch")


# ------------------------------------------------------------------ clocks
REASON_BITS = {
    0x1: "gpu_idle",
    0x2: "applications_clocks_setting",
    0x4: "sw_power_cap",
    0x8: "hw_slowdown",
    0x20: "sw_thermal_slowdown",
    0x40: "hw_thermal_slowdown",
    0x80: "hw_power_brake_slowdown",
    0x100: "display_clock_setting",
}


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def __enter__(self):
        cmd = [
            "nvidia-smi",
            f"--id={self.index}",
            "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active,utilization.gpu",
            "--format=csv,noheader,nounits",
            "-lms",
            "200",
        ]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return self
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 4:
                continue
            try:
                sm, smax = float(parts[0]), float(parts[1])
                reasons = int(parts[2], 16) if parts[2].startswith("0x") else int(parts[2])
                util = float(parts[3])
            except ValueError:
                continue
            self.samples.append((sm, smax, reasons, util))

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        loaded = [s for s in self.samples if s[3] >= 50] or self.samples
        reasons = 0
        for s in loaded:
            reasons |= s[2]
        names = [n for b, n in REASON_BITS.items() if reasons & b and n != "gpu_idle"]
        return {
            "sm_mhz": statistics.median(s[0] for s in loaded),
            "sm_max_mhz": max(s[1] for s in self.samples),
            "reasons": names,
            "samples": len(loaded),
        }


# ------------------------------------------------------------------ distributed harness
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def reduce_max(value, world):
    """Max over ranks of a float (identity for a single process)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


# ------------------------------------------------------------------ inputs
def make_inputs():
    import synth

    fat, lng = synth.gauge_field(DIMS, EPS, GAUGE_SEED)
    srcs = [synth.gaussian_source(DIMS, s) for s in SOURCE_SEEDS]
    return fat, lng, srcs


# ------------------------------------------------------------------ CPU baseline (oracle)
# The oracle as it stands, one process per source (spawned, so no GPU state
# is inherited), the four sources solved side by side on four host cores;
# the links reach the processes through shared memory, not by copy.
_SHARED = {}


def _oracle_worker_init(names, shape, dtype):
    from multiprocessing import shared_memory

    import numpy as np

    for key, name in names.items():
        shm = shared_memory.SharedMemory(name=name)
        _SHARED[key] = (shm, np.ndarray(shape, dtype=dtype, buffer=shm.buf))


def _oracle_worker_sample(args):
    import oracle

    b, sample_iters, dims, mass, tol = args
    t = time.perf_counter()
    oracle.cg(_SHARED["fat"][1], _SHARED["lng"][1], b, mass, dims, tol=tol, max_iter=sample_iters)
    return time.perf_counter() - t


class OraclePool:
    """Spawned worker processes holding the links (shared memory)."""

    def __init__(self, fat, lng, workers):
        import multiprocessing as mp
        from multiprocessing import shared_memory

        import numpy as np

        self.shms = []
        names = {}
        for key, a in (("fat", fat), ("lng", lng)):
            shm = shared_memory.SharedMemory(create=True, size=a.nbytes)
            np.ndarray(a.shape, dtype=a.dtype, buffer=shm.buf)[...] = a
            self.shms.append(shm)
            names[key] = shm.name
        # one BLAS thread per worker: the workers are the parallelism
        env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in env:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(workers, initializer=_oracle_worker_init,
                                                     initargs=(names, fat.shape, fat.dtype))
        finally:
            for k, v in env.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.workers = workers

    def sample(self, srcs, sample_iters):
        """Wall time of `sample_iters` oracle CG iterations on every source at once."""
        t = time.perf_counter()
        per = self.pool.map(_oracle_worker_sample, [(b, sample_iters, DIMS, MASS, TOL) for b in srcs])
        return time.perf_counter() - t, per

    def close(self):
        self.pool.close()
        self.pool.join()
        for shm in self.shms:
            shm.close()
            shm.unlink()


def cpu_baseline(fat, lng, srcs, iters_full, sample_iters=3, pool=None):
    """The FP64 numpy oracle, timed on a bounded sample and scaled to a solve.

    Runs `sample_iters` oracle CG iterations (each one operator application
    plus vector updates, and one true-residual application) on each source,
    the sources in parallel processes, and scales the wall time per source to
    the `iters_full` iterations of a full solve."""
    own = pool is None
    if own:
        pool = OraclePool(fat, lng, min(len(srcs), os.cpu_count() or 1))
    try:
        pool.sample(srcs[:1], 1)  # workers started and the links attached before timing
        wall, per = pool.sample(srcs, sample_iters)
    finally:
        if own:
            pool.close()
    per_source = wall / len(srcs)
    return {
        "value": per_source / (sample_iters + 1) * (iters_full + 1),
        "unit": "s",
        "cores": pool.workers,
        "kind": "oracle",
        "sample": f"{sample_iters} FP64 CG iterations of the numpy oracle on each of the {len(srcs)} 32^4 sources, "
        f"one process per source on {pool.workers} host cores ({wall:.1f} s wall), per-source time scaled to "
        f"the {iters_full} iterations of a full FP64 solve",
    }


# ------------------------------------------------------------------ GPU arm
def run_gpu(args, rank, world, local_rank):
    global CHOSEN
    CHOSEN = args.chosen
    import numpy as np
    import torch

    import paper_1712_00143_gb300 as stag

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    fat, lng, srcs = make_inputs()
    h = stag.stag_load_links(DIMS, torch.from_numpy(fat).to(dev), torch.from_numpy(lng).to(dev), recon_long=RECON)
    bs = [torch.from_numpy(b).to(dev) for b in srcs]
    xs = [torch.zeros_like(b) for b in bs]
    stream = torch.cuda.current_stream()
    Vh = h.Vh

    B = torch.stack(bs).contiguous()
    X = torch.zeros_like(B)

    def step(mode):
        if BATCHED and mode == CHOSEN:
            return stag.stag_batch_solve([(h, X, B, NSRC, MASS)], mode=mode, tol=TOL)
        infos = []
        for x, b in zip(xs, bs):
            infos.append(stag.stag_cg(h, x, b, MASS, mode=mode, tol=TOL))
        return infos

    fam_plain, fam_epi = ("dslash_mrhs", "dslash_mrhs_epi") if BATCHED else ("dslash", "dslash_epi")

    # plain FP64 reference solve (one pass over the sources, after one warm-up)
    step("plain64")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain_infos = step("plain64")
    torch.cuda.synchronize()
    plain_s = (time.perf_counter() - t0) / NSRC

    for _ in range(args.warmup):
        step(CHOSEN)
    torch.cuda.synchronize()

    stag.stag_profile_reset()
    # event pairs around the two Dslash kernels only, one launch in 8 of each,
    # so that the timed steps carry little instrumentation
    stag.stag_profile_select(f"{fam_plain},{fam_epi}", 8)
    stag.stag_profile_enable(True)
    launches0 = stag.stag_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    infos_all = []
    with ClockSampler(local_rank) as clk:
        barrier(world)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed launches
        e0.record(stream)
        for _ in range(args.steps):
            infos_all += step(CHOSEN)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        barrier(world)
    launches = stag.stag_launch_count() - launches0
    shapes = {k: stag.stag_tuned_shape(h, MODE_PREC[CHOSEN], i) for i, k in enumerate(("plain", "epilogue"))}
    mrhs_shape = stag.stag_tuned_mrhs(h, MODE_PREC[CHOSEN], NSRC) if BATCHED else None
    mrhs_shape_epi = stag.stag_tuned_mrhs(h, MODE_PREC[CHOSEN], NSRC, epilogue=True) if BATCHED else None
    mrhs_var = stag.stag_tuned_mrhs_variant(h, MODE_PREC[CHOSEN], NSRC) if BATCHED else None
    mrhs_var_epi = stag.stag_tuned_mrhs_variant(h, MODE_PREC[CHOSEN], NSRC, epilogue=True) if BATCHED else None
    df_shape = stag.stag_tuned_shape(h, "df64", 0)
    n_d, ms_d = stag.stag_profile_read(fam_plain)
    n_e, ms_e = stag.stag_profile_read(fam_epi)
    # one more (untimed) step with every launch of every family timed: where
    # the device time of a step goes
    stag.stag_profile_reset()
    stag.stag_profile_select("", 1)
    step(CHOSEN)
    torch.cuda.synchronize()
    breakdown = {}
    for fam in FAMILIES:
        n, ms = stag.stag_profile_read(fam)
        if n:
            breakdown[fam] = {"launches": n, "ms": round(ms, 3)}
    stag.stag_profile_enable(False)
    ms_total = reduce_max(e0.elapsed_time(e1), world)
    ms_per_step = ms_total / args.steps
    value = ms_per_step / 1e3 / NSRC

    # end to end through the C ABI with host buffers: H2D of the sources and
    # D2H of the solutions inside the timed region
    hb = [torch.from_numpy(b).pin_memory() for b in srcs]
    hx = [torch.empty_like(b) for b in hb]
    hx = [t.pin_memory() for t in hx]
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(max(1, min(args.steps, 3))):
        if BATCHED:
            bd = torch.stack([t.to(dev, non_blocking=True) for t in hb]).contiguous()
            xd = torch.zeros_like(bd)
            stag.stag_batch_solve([(h, xd, bd, NSRC, MASS)], mode=CHOSEN, tol=TOL)
            for k in range(NSRC):
                hx[k].copy_(xd[k], non_blocking=True)
        else:
            for k in range(NSRC):
                bd = hb[k].to(dev, non_blocking=True)
                xd = torch.zeros_like(bd)
                stag.stag_cg(h, xd, bd, MASS, mode=CHOSEN, tol=TOL)
                hx[k].copy_(xd, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = reduce_max((time.perf_counter() - t0) / max(1, min(args.steps, 3)) / NSRC, world)
    vec_bytes = Vh * 3 * 16

    # verify every timed solve
    ok = all(i["converged"] and i["true_rel_resid"] <= TOL for i in infos_all + plain_infos)
    prec = MODE_PREC[CHOSEN]
    per_launch_ms = ms_d / max(n_d, 1)
    pbits = {"fp32": 32, "fp16": 16, "fx16": 15, "fp64": 64, "fx16l": 31}[prec]
    nl = 6 if RECON == 12 else 9
    if BATCHED:
        # one launch: the links once and NSRC input and output vectors
        bytes_launch = ((8 * 9 + 8 * nl) * ELEM_BYTES[prec] + 2 * NSRC * VEC_BYTES[prec]) * Vh
        # template arguments of the launched kernel: format, Naik entries, N,
        # threads per site, register cap
        kernel_id = f"k_dslash_mv<{pbits},{nl},{NSRC},{mrhs_shape[0]},{mrhs_shape[1]}>"
        sites_launch = NSRC * Vh
    else:
        bytes_launch = dslash_bytes_per_site(prec, RECON) * Vh
        kernel_id = f"k_dslash<{pbits},{nl}>"
        sites_launch = Vh
    achieved = bytes_launch / (per_launch_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    traffic = ncu_traffic(kernel_id)
    iters = [i["iters"] for i in infos_all[:NSRC]]
    iters_plain = [i["iters"] for i in plain_infos]

    result = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(fat, lng, srcs, iters_plain[0])
        clocks = clk.summary()
        result = {
            "metric": METRIC,
            "value": value,
            "unit": "s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms_per_step,
            "higher_is_better": False,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": DTYPE[CHOSEN],
            "data": "synthetic",
            "config": {
                "workload": "32^4 even-odd improved-staggered CG, m=0.01, eps=0.3, 4 Gaussian sources, "
                "1e-10 FP64 true residual",
                "solver": f"{CHOSEN}, {NSRC} sources batched (stag_batch_solve)" if BATCHED else CHOSEN,
                "link_storage": f"{prec}, Naik recon {RECON}",
                "sources_per_step": NSRC,
                "l2": "inputs larger than L2 (links 0.5-1.2 GB per precision)",
                "parallelism": "replicas" if world > 1 else "single GPU",
            },
            "plain_fp64": {"value": plain_s, "unit": "s", "iters": iters_plain},
            "speedup_vs_plain": plain_s / value,
            "iters": iters,
            "all_converged": ok,
            "roofline": {
                "bound": "hbm",
                "kernel": kernel_id,
                "achieved": achieved,
                "peak": peak,
                "peak_kind": peak_kind,
                "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": traffic,
                "algorithmic_bytes_per_launch": bytes_launch,
                "launches_timed": n_d,
                "launches_sampled_every": 8,
                "launches_excluded": "chunks of queued iterations cut short by a stop flag (reliable-update "
                "trigger, convergence): their launches after the flag return at once",
                "avg_launch_us": per_launch_ms * 1e3,
                "gflops": FLOP_PER_SITE * sites_launch / (per_launch_ms * 1e-3) / 1e9,
                "epilogue_variant_avg_us": ms_e / max(n_e, 1) * 1e3,
                "launch_shape": ({"multi_rhs": {"variant": mrhs_var, "block": 128, "threads_per_site": mrhs_shape[0],
                                                "rhs_per_thread": NSRC // mrhs_shape[0],
                                                "min_blocks_per_sm": mrhs_shape[1],
                                                "tuned_us_per_launch": mrhs_shape[2],
                                                "chosen_by": "autotuner (stag_tuned_mrhs)"},
                                  "multi_rhs_epilogue": {"variant": mrhs_var_epi, "block": 128,
                                                         "threads_per_site": mrhs_shape_epi[0],
                                                         "rhs_per_thread": NSRC // mrhs_shape_epi[0],
                                                         "min_blocks_per_sm": mrhs_shape_epi[1],
                                                         "tuned_us_per_launch": mrhs_shape_epi[2],
                                                         "chosen_by": "autotuner (stag_tuned_mrhs_epi)"}}
                                 if BATCHED else
                                 {k: {"block": v[0], "min_blocks_per_sm": v[1], "tuned_us": v[2]}
                                  for k, v in shapes.items()}),
            },
            "e2e": {
                "value": e2e_s,
                "unit": "s",
                "h2d_bytes_per_step": NSRC * vec_bytes,
                "d2h_bytes_per_step": NSRC * vec_bytes,
            },
            "step_breakdown_ms": breakdown,
            "reliable_update_operator": dict(df_summary(breakdown, Vh, NSRC) or {},
                                             launch_shape={"block": 128, "threads_per_site": df_shape[1],
                                                           "tuned_us": df_shape[2]}),
            "gpu_launches": launches,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
    h.free()
    return result


def df_summary(breakdown, Vh, nrhs):
    """The reliable updates' FP64-class operator (double-float, links read
    once for up to four right-hand sides): device time per launch and its
    algorithmic bytes (links 2304 B per site, nrhs input and output vectors
    of 48 B; the epilogue form also reads y and b)."""
    out = {}
    for fam, extra in (("dslash_df", 0), ("dslash_df_epi", 2)):
        ent = breakdown.get(fam)
        if not ent:
            continue
        us = ent["ms"] / ent["launches"] * 1e3
        byt = (2304 + (2 + extra) * 48 * nrhs) * Vh
        out[fam] = {"launches": ent["launches"], "avg_launch_us": us, "algorithmic_bytes_per_launch": byt,
                    "GB/s": byt / (us * 1e-6) / 1e9, "arithmetic": "double-float on the FP32 pipes"}
    return out or None


# ------------------------------------------------------------------ reference arm (oracle)
def run_reference(args, rank, world):
    if rank != 0:
        return None
    import oracle  # noqa: F401

    fat, lng, srcs = make_inputs()
    iters_full = ORACLE_FULL_ITERS
    times = []
    pool = OraclePool(fat, lng, min(len(srcs), os.cpu_count() or 1))
    try:
        for k in range(args.warmup + args.steps):
            c = cpu_baseline(fat, lng, srcs, iters_full, sample_iters=2, pool=pool)
            if k >= args.warmup:
                times.append(c["value"])
    finally:
        pool.close()
    v = statistics.mean(times)
    return {
        "impl": "reference",
        "metric": METRIC,
        "value": v,
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": v * NSRC * 1e3,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {
            "workload": "32^4 even-odd improved-staggered CG, m=0.01, eps=0.3, 4 Gaussian sources, "
            "1e-10 FP64 true residual",
            "solver": "FP64 numpy oracle",
        },
        "cpu_baseline": dict(c, value=v),
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# Iterations the FP64 oracle's own CG needs to reach 1e-10 on the bench
# workload (source 0), measured by running the oracle to convergence once.
ORACLE_FULL_ITERS = 487


def run_dslash_sweep(args):
    """Dslash bandwidth sweep over lattice sizes, storage formats and Naik
    storage (the paper's single-GPU L^4 sweep, Sec. 4.1, Fig. 9): one JSON
    line per case with the kernel's device time per launch (CUDA events on
    its launch stream), algorithmic GB/s, GFLOP/s at 1146 flop/site and the
    fraction of the measured HBM bandwidth."""
    import torch

    import paper_1712_00143_gb300 as stag
    import synth

    peak, peak_kind = measured_peaks()
    for L in args.sweep_dims:
        dims = tuple(int(v) for v in L.split("x")) if "x" in L else (int(L),) * 4
        fat, lng = synth.gauge_field(dims, EPS, GAUGE_SEED)
        fd, ld = torch.from_numpy(fat).cuda(), torch.from_numpy(lng).cuda()
        del fat, lng
        for recon in args.sweep_recons:
            for prec in args.sweep_precs:
                if prec in ("fp64", "df64") and recon == 12:
                    continue
                copy = "fx16" if prec == "fx16l" else prec  # the hybrid reads the fixed-point link copy
                h = stag.stag_load_links(dims, fd, ld, recon_long=recon, prec_mask=1 << stag.PREC[copy])
                for nrhs in args.sweep_nrhs:
                    psi = torch.from_numpy(synth.random_spinor(dims, 3)).cuda()
                    if nrhs > 1:
                        psi = psi.unsqueeze(0).repeat(nrhs, 1, 1).contiguous()
                    out = torch.empty_like(psi)
                    fam = ("dslash" if nrhs == 1 else "dslash_mrhs") + ("64" if prec == "fp64" else "")
                    if prec == "df64":
                        fam = "dslash_df"
                    for _ in range(3):
                        stag.stag_dslash(h, out, psi, 1, prec, nrhs=nrhs)
                    torch.cuda.synchronize()
                    stag.stag_profile_reset()
                    stag.stag_profile_select(fam, 1)
                    stag.stag_profile_enable(True)
                    for _ in range(args.sweep_reps):
                        stag.stag_dslash(h, out, psi, 1, prec, nrhs=nrhs)
                    n, ms = stag.stag_profile_read(fam)
                    stag.stag_profile_enable(False)
                    stag.stag_profile_select("", 1)
                    per = ms / max(n, 1)  # one launch covers min(nrhs, 8) (double-float: 4) right-hand sides
                    k = min(nrhs, 4 if prec == "df64" else 8)
                    nl = 6 if (recon == 12 and prec != "fp64") else 9
                    byt = ((8 * 9 + 8 * nl) * ELEM_BYTES[prec] + 2 * k * VEC_BYTES[prec]) * h.Vh
                    gbs = byt / (per * 1e-3) / 1e9
                    print(json.dumps({"dslash": "x".join(map(str, dims)), "prec": prec, "recon": recon, "nrhs": k,
                                      "us": per * 1e3, "GB/s": gbs, "frac": gbs / peak, "peak_kind": peak_kind,
                                      "GFLOP/s": FLOP_PER_SITE * k * h.Vh / (per * 1e-3) / 1e9,
                                      "us_per_rhs": per * 1e3 / k, "bytes_per_launch": byt,
                                      "tuned_shape": stag.stag_tuned_shape(h, prec, 0)}), flush=True)
                    del psi, out
                h.free()
        del fd, ld
        torch.cuda.empty_cache()


def _timed(fn, reps=1):
    import torch

    torch.cuda.synchronize()
    t = time.perf_counter()
    out = None
    for _ in range(reps):
        out = fn()
    torch.cuda.synchronize()
    return (time.perf_counter() - t) / reps, out


def run_config(args):
    """Secondary workloads of the paper's CG path, one JSON line each (not the
    headline): `small` 8^4 FP64 CG; `multishift` 48^3x96 nine-shift CG;
    `batch` 12 lattices x 8 right-hand sides in one batched call vs one
    stag_cg per system; `learned` training and evaluating the network
    preconditioner on 32^4; `netpass` one network forward and one
    loss-and-gradient pass on 32^4; `links` fat and Naik links built from
    thin links on the GPU; `gaugeforce` the Symanzik one-loop gauge force;
    `fermionforce` the fermion force through the link construction."""
    import torch

    import paper_1712_00143_gb300 as stag
    import synth

    dev = torch.device("cuda")
    if args.config == "small":
        dims, mass = (8, 8, 8, 8), 0.1
        fat, lng = synth.gauge_field(dims, EPS, GAUGE_SEED)
        h = stag.stag_load_links(dims, torch.from_numpy(fat).to(dev), torch.from_numpy(lng).to(dev))
        b = torch.from_numpy(synth.gaussian_source(dims, 5000)).to(dev)
        res = {}
        for mode in ("plain64", "mixed32", "mixedfx16"):
            x = torch.zeros_like(b)
            for _ in range(3):
                x.zero_()
                stag.stag_cg(h, x, b, mass, mode=mode)
            sec, info = _timed(lambda: (x.zero_(), stag.stag_cg(h, x, b, mass, mode=mode))[1], reps=5)
            res[mode] = {"s": sec, "iters": info["iters"], "true_rel_resid": info["true_rel_resid"]}
        print(json.dumps({"config": "8^4 single-mass CG, m=0.1, 1e-10", "unit": "s", "results": res}), flush=True)
        h.free()
    elif args.config == "multishift":
        dims, mass = (48, 48, 48, 96), 0.005
        shifts = [10 ** (-4 + k / 2) for k in range(9)]
        fat, lng = synth.gauge_field(dims, EPS, GAUGE_SEED)
        h = stag.stag_load_links(dims, torch.from_numpy(fat).to(dev), torch.from_numpy(lng).to(dev), recon_long=12,
                                 prec_mask=0b11011)
        del fat, lng
        b = torch.from_numpy(synth.gaussian_source(dims, 5000)).to(dev)
        xs = [torch.zeros_like(b) for _ in shifts]
        res = {}
        for mode in ("mixed32", "mixedfx16"):
            stag.stag_multishift_cg(h, xs, b, mass, shifts, mode=mode)
            sec, infos = _timed(lambda: stag.stag_multishift_cg(h, xs, b, mass, shifts, mode=mode), reps=2)
            res[mode] = {"s": sec, "iters": [i["iters"] for i in infos],
                         "max_true_rel_resid": max(i["true_rel_resid"] for i in infos)}
        print(json.dumps({"config": "48^3x96 multi-shift CG, 9 shifts 1e-4..1, m=0.005, 1e-10 every shift",
                          "unit": "s", "results": res}), flush=True)
        h.free()
    elif args.config == "batch":
        dims_list = [(16, 16, 16, 16)] * 4 + [(24, 24, 24, 48)] * 4 + [(32, 32, 32, 32)] * 4
        masses = [0.01, 0.02, 0.05]
        items = []
        for j, dims in enumerate(dims_list):
            fat, lng = synth.gauge_field(dims, EPS, GAUGE_SEED + j)
            h = stag.stag_load_links(dims, torch.from_numpy(fat).to(dev), torch.from_numpy(lng).to(dev), recon_long=12,
                                     prec_mask=0b11011)
            bd = torch.from_numpy(synth.gaussian_source(dims, 5000 + 100 * j, nrhs=8)).to(dev)
            items.append((h, torch.zeros_like(bd), bd, 8, masses[j % 3]))
        res = {}
        for mode in ("mixed32", "mixedfx16", "mixed16l"):
            def batched():
                for it in items:
                    it[1].zero_()
                return stag.stag_batch_solve(items, mode=mode)

            def sequential():
                out = []
                for h, x, bd, n, m in items:
                    x.zero_()
                    for i in range(n):
                        out.append(stag.stag_cg(h, x[i], bd[i], m, mode=mode))
                return out

            batched()
            tb, ib = _timed(batched, reps=2)
            sequential()
            ts, isq = _timed(sequential, reps=1)
            res[mode] = {"batched_s": tb, "sequential_s": ts, "speedup": ts / tb,
                         "all_converged": all(i["converged"] for i in ib + isq),
                         "max_true_rel_resid": max(i["true_rel_resid"] for i in ib)}
        print(json.dumps({"config": "12 lattices (4x16^4, 4x24^3x48, 4x32^4) x 8 RHS, m in {0.01,0.02,0.05}, 1e-10",
                          "unit": "s", "results": res}), flush=True)
        for it in items:
            it[0].free()
    elif args.config == "netpass":
        # one network forward (z = N(r)) and one loss-and-gradient pass (32^4 by default)
        dims = (args.net_dims,) * 4
        fat, lng = synth.gauge_field(dims, EPS, GAUGE_SEED)
        h = stag.stag_load_links(dims, torch.from_numpy(fat).to(dev), torch.from_numpy(lng).to(dev), recon_long=12,
                                 prec_mask=0b0010)
        del fat, lng
        net = stag.stag_net_create((1, 16, 16, 16, 1), seed=1)
        r = torch.from_numpy(synth.random_spinor(dims, 1)).to(dev)
        e = torch.from_numpy(synth.random_spinor(dims, 2)).to(dev)
        z = torch.empty_like(r)
        lg = lambda: stag.stag_net_loss_grad(net, h, r, e, loss="residual", mass=0.01)  # noqa: E731
        stag.stag_net_apply(net, h, z, r)
        lg()
        t_f, _ = _timed(lambda: stag.stag_net_apply(net, h, z, r), reps=5)
        t_b, _ = _timed(lg, reps=3)
        stag.stag_profile_reset()
        stag.stag_profile_enable(True)
        lg()
        fam = {f: stag.stag_profile_read(f) for f in ("net", "net_tc", "net_bwd")}
        stag.stag_profile_enable(False)
        # the 16 -> 16 tensor-core layer against the HBM roofline: per site
        # 8 fat hops of 72 B, the input record (384 B) and pre + output (768 B)
        n_tc, ms_tc = fam["net_tc"]
        tc_us = ms_tc / max(n_tc, 1) * 1e3
        tc_bytes = 1728 * 2 * h.Vh
        tc_roof = {"kernel": "k_net_layer_tc", "avg_launch_us": tc_us, "bytes_per_launch": tc_bytes,
                   "achieved_gbs": tc_bytes / (tc_us * 1e-6) / 1e9 if tc_us > 0 else None}
        if tc_roof["achieved_gbs"]:
            peak, peak_kind = measured_peaks()
            tc_roof.update(peak_gbs=peak, peak_kind=peak_kind, frac=tc_roof["achieved_gbs"] / peak)
        flops_fw = 0
        ch = (1, 16, 16, 16, 1)
        for l in range(4):
            # per site: 8 transports (66 flop) per input channel + 9 x Cin x Cout real-by-complex-3 mixes (12 flop)
            flops_fw += 2 * h.Vh * (8 * ch[l] * 66 + 9 * ch[l] * ch[l + 1] * 12)
        print(json.dumps({"config": f"network 1-16-16-16-1 on {args.net_dims}^4", "forward_s": t_f, "loss_grad_s": t_b,
                          "forward_gflops": flops_fw / t_f / 1e9, "tc_layer": tc_roof,
                          "families_ms": {k: {"launches": v[0], "ms": v[1]} for k, v in fam.items()}}), flush=True)
        net.free()
        h.free()
    elif args.config == "links":
        # fat and Naik links from thin links on the GPU (FP64), 32^4 and 48^3 x 96
        import oracle.links as olk

        from synth.gauge import Lattice, thin_links

        # per (site, direction): 6 staples x 2 complex 3x3 products + 2 Naik products,
        # 216 flop each (27 complex FMA), plus the combination: about 3080 flop
        flop_per_link = 14 * 216 + 36 + 18
        rows = {}
        for dims in ((32, 32, 32, 32), (48, 48, 48, 96)):
            lat = Lattice(dims)
            thin = thin_links(lat, EPS, GAUGE_SEED).reshape(lat.V, 4, 3, 3).to(dev)
            fat, lng = stag.stag_build_links(dims, thin)
            torch.cuda.synchronize()
            stag.stag_profile_reset()
            stag.stag_profile_select("links", 1)
            stag.stag_profile_enable(True)
            wall, _ = _timed(lambda: stag.stag_build_links(dims, thin, fat, lng), reps=5)
            n, ms = stag.stag_profile_read("links")
            stag.stag_profile_enable(False)
            stag.stag_profile_select("", 1)
            per = ms / max(n, 1) * 1e-3
            tf = 4 * lat.V * flop_per_link / per / 1e12
            rows["x".join(map(str, dims))] = {"device_s": per, "wall_s": wall, "fp64_tflops": tf}
            del thin, fat, lng
            torch.cuda.empty_cache()
        # the oracle on a 16^4 sample (numpy, one core), scaled per site
        d16 = (16, 16, 16, 16)
        lat = Lattice(d16)
        t16 = thin_links(lat, EPS, GAUGE_SEED).reshape(lat.V, 4, 3, 3).numpy()
        t0 = time.perf_counter()
        olk.fat_links(t16, d16)
        olk.naik_links(t16, d16)
        per_site = (time.perf_counter() - t0) / lat.V
        print(json.dumps({"config": "link construction (3-staple fat + Naik) from thin links, FP64",
                          "unit": "s", "results": rows,
                          "roofline": {"bound": "fp64_alu", "flop_per_link": flop_per_link,
                                       "note": "FP64 peak about 1.2 TFLOP/s on GB300 (measured DGEMM 1.10)"},
                          "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": "16^4, scaled per site",
                                           "s_per_site": per_site,
                                           "value_32_4": per_site * 32 ** 4}}), flush=True)
    elif args.config == "gaugeforce":
        # Symanzik one-loop gauge force (FP64) on 24^4 (the paper's per-node weak-scaling
        # volume, Fig. 7) and 32^4
        import oracle.gauge_force as ogf

        from synth.gauge import Lattice, thin_links

        beta = 6.0
        coef = ogf.luscher_weisz_coefficients(0.87)
        # executed flop per link of the staple-reuse algorithm: the staple table
        # (24 staples per site x 2 complex 3x3 products of 216 flop, a quarter per
        # link) and, per (nu, s), rectangles 1-2 (4 products), rectangle 3 and the
        # four parallelograms (5 products + the shared left factor), coefficient
        # updates; then U Sigma and TA.  Walking every staple link by link instead
        # (MILC's baseline, Sec. 4.2) costs 40884 flop per link.
        flop_per_link = 24 * 2 * 216 // 4 + 6 * (10 * 216 + 7 * 36 + 18) + 216 + 40
        flop_walk = (6 * 2 + 42 * 4 + 1) * 216 + 48 * 36 + 60
        rows = {}
        for dims in ((24, 24, 24, 24), (32, 32, 32, 32)):
            lat = Lattice(dims)
            thin = thin_links(lat, EPS, GAUGE_SEED).reshape(lat.V, 4, 3, 3).to(dev)
            F = stag.stag_gauge_force(dims, thin, beta, *coef)
            torch.cuda.synchronize()
            stag.stag_profile_reset()
            stag.stag_profile_select("gauge_force", 1)
            stag.stag_profile_enable(True)
            reps = 3
            wall, _ = _timed(lambda: stag.stag_gauge_force(dims, thin, beta, *coef, force=F), reps=reps)
            n, ms = stag.stag_profile_read("gauge_force")  # two kernels per call
            stag.stag_profile_enable(False)
            stag.stag_profile_select("", 1)
            per = ms / reps * 1e-3
            rows["x".join(map(str, dims))] = {"device_s": per, "wall_s": wall, "launches_per_call": n / reps,
                                              "fp64_tflops": 4 * lat.V * flop_per_link / per / 1e12,
                                              "gflop_per_site": 4 * flop_per_link / 1e9}
            del thin, F
            torch.cuda.empty_cache()
        # the oracle on a 4^4 x 6 sample (numpy, one core), scaled per link
        d = (4, 4, 4, 6)
        lat = Lattice(d)
        ts = thin_links(lat, EPS, GAUGE_SEED).reshape(lat.V, 4, 3, 3).numpy()
        t0 = time.perf_counter()
        ogf.force(ts, d, beta, *coef)
        per_link = (time.perf_counter() - t0) / (4 * lat.V)
        print(json.dumps({"config": "Symanzik one-loop gauge force (plaquette, rectangle, parallelogram), FP64",
                          "coefficients": {"beta": beta, "u0": 0.87, "c_pl": coef[0], "c_rt": coef[1], "c_pg": coef[2]},
                          "unit": "s", "results": rows,
                          "algorithm": "three-link staples stored once, reused by every loop",
                          "roofline": {"bound": "fp64_alu", "flop_per_link": flop_per_link,
                                       "flop_per_link_walking_each_staple": flop_walk,
                                       "note": "FP64 peak about 1.2 TFLOP/s on GB300 (measured DGEMM 1.10)"},
                          "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": "4^4 x 6, scaled per link",
                                           "s_per_link": per_link, "value_24_4": per_link * 4 * 24 ** 4}}),
              flush=True)
    elif args.config == "fermionforce":
        # fermion force of an 8-term rational pseudofermion action (FP64) on 24^4
        # and 32^4: outer products of the 8 solution pairs, then the chain rule
        # through the fat and Naik links
        import numpy as np

        import oracle.fermion_force as off

        from synth.gauge import Lattice, thin_links

        nt = 8
        alphas = tuple(np.linspace(0.05, 0.4, nt))
        # executed flop per link: the chain pass, 36 products of 3x3 complex
        # matrices (216 flop each), 15 scalings (18 flop), TA (40); the outer
        # pass, two 3x3 outer products accumulated per term (144 flop)
        flop_per_link = 36 * 216 + 15 * 18 + 40 + 144 * nt
        rows = {}
        for dims in ((24, 24, 24, 24), (32, 32, 32, 32)):
            lat = Lattice(dims)
            thin = thin_links(lat, EPS, GAUGE_SEED).reshape(lat.V, 4, 3, 3).to(dev)
            xs = torch.from_numpy(np.stack([synth.random_spinor(dims, 10 + i) for i in range(nt)])).to(dev)
            ys = torch.from_numpy(np.stack([synth.random_spinor(dims, 50 + i) for i in range(nt)])).to(dev)
            F = stag.stag_fermion_force(dims, thin, xs, ys, alphas)
            torch.cuda.synchronize()
            stag.stag_profile_reset()
            stag.stag_profile_select("fermion_force", 1)
            stag.stag_profile_enable(True)
            reps = 3
            wall, _ = _timed(lambda: stag.stag_fermion_force(dims, thin, xs, ys, alphas, force=F), reps=reps)
            n, ms = stag.stag_profile_read("fermion_force")  # two kernels per call
            stag.stag_profile_enable(False)
            stag.stag_profile_select("", 1)
            per = ms / reps * 1e-3
            rows["x".join(map(str, dims))] = {"device_s": per, "wall_s": wall, "launches_per_call": n / reps,
                                              "fp64_tflops": 4 * lat.V * flop_per_link / per / 1e12}
            del thin, xs, ys, F
            torch.cuda.empty_cache()
        # the oracle on a 6^4 sample (numpy, one core), scaled per link
        d = (6, 6, 6, 6)
        lat = Lattice(d)
        ts = thin_links(lat, EPS, GAUGE_SEED).reshape(lat.V, 4, 3, 3).numpy()
        ox = [synth.random_spinor(d, 10 + i) for i in range(nt)]
        oy = [synth.random_spinor(d, 50 + i) for i in range(nt)]
        t0 = time.perf_counter()
        off.fermion_force(ts, ox, oy, alphas, d)
        per_link = (time.perf_counter() - t0) / (4 * lat.V)
        print(json.dumps({"config": f"fermion force through the 3-staple fat + Naik links, {nt} terms, FP64",
                          "unit": "s", "results": rows,
                          "roofline": {"bound": "fp64_alu", "flop_per_link": flop_per_link,
                                       "note": "FP64 peak about 1.2 TFLOP/s on GB300 (measured DGEMM 1.10)"},
                          "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": "6^4, scaled per link",
                                           "s_per_link": per_link, "value_32_4": per_link * 4 * 32 ** 4}}),
              flush=True)
    elif args.config == "learned":
        # 32^4, m = 0.01: 2000 (residual, error) pairs from the unpreconditioned
        # mixed CG on 24 training fields, network 1-16-16-16-1 trained on the
        # GPU, flexible CG with it on 8 held-out fields vs mixed CG
        import numpy as np

        from paper_1712_00143_gb300.learned import make_pairs

        dims, mass = (32, 32, 32, 32), 0.01
        ntrain, nheld, npairs = args.learned_fields, 8, args.learned_pairs
        per = -(-npairs // ntrain)
        t0 = time.perf_counter()
        handles, pairs = [], []
        for j in range(ntrain):
            fat, lng = synth.gauge_field(dims, EPS, 1000 + j)
            h = stag.stag_load_links(dims, torch.from_numpy(fat).to(dev), torch.from_numpy(lng).to(dev), recon_long=12,
                                     prec_mask=0b10011)
            del fat, lng
            handles.append(h)
            b = torch.from_numpy(synth.gaussian_source(dims, 5000 + 100 * j)).to(dev)
            ks = np.unique(np.linspace(1, 470, per).astype(int))
            pairs += make_pairs(h, [b], mass, ks)
        pairs = pairs[:npairs]
        t_pairs = time.perf_counter() - t0
        net = stag.stag_net_create((1, 16, 16, 16, 1), seed=1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        losses = stag.stag_net_train(net, pairs, epochs=args.learned_epochs, batch=8, lr=1e-3, seed=1,
                                     loss="residual", mass=mass)
        t_train = time.perf_counter() - t0
        del pairs
        for h in handles:
            h.free()
        torch.cuda.empty_cache()
        raw = stag.stag_net_create((1, 16, 16, 16, 1), seed=1)
        held = []
        for j in range(nheld):
            fat, lng = synth.gauge_field(dims, EPS, 2000 + j)
            h = stag.stag_load_links(dims, torch.from_numpy(fat).to(dev), torch.from_numpy(lng).to(dev), recon_long=12)
            del fat, lng
            b = torch.from_numpy(synth.gaussian_source(dims, 5000 + 100 * (2000 + j))).to(dev)
            row = {}
            for name, kw in (("mixedfx16", {"mode": "mixedfx16"}), ("plain64", {"mode": "plain64"}),
                             ("learned_fcg", {"mode": "learned", "precond": net}),
                             ("untrained_fcg", {"mode": "learned", "precond": raw})):
                x = torch.zeros_like(b)
                stag.stag_cg(h, x, b, mass, tol=TOL, **kw)  # warm
                x.zero_()
                sec, info = _timed(lambda: stag.stag_cg(h, x, b, mass, tol=TOL, **kw))
                row[name] = {"s": sec, "iters": info["iters"], "true_rel_resid": info["true_rel_resid"],
                             "fallback": info["precond_fallback"]}
            held.append(row)
            h.free()
        summ = {k: {"mean_s": float(np.mean([r[k]["s"] for r in held])),
                    "mean_iters": float(np.mean([r[k]["iters"] for r in held])),
                    "all_converged": all(r[k]["true_rel_resid"] <= TOL for r in held),
                    "fallbacks": int(sum(r[k]["fallback"] for r in held))} for k in held[0]}
        nl = len(losses) // args.learned_epochs
        print(json.dumps({"config": f"32^4 m=0.01 learned preconditioner: {len(losses)//args.learned_epochs} pairs from "
                                    f"{ntrain} training fields, {args.learned_epochs} epochs, {nheld} held-out fields",
                          "loss": "residual ||M N(r) - r||^2 / ||r||^2",
                          "pair_generation_s": t_pairs, "training_s": t_train,
                          "loss_first_epoch": float(np.mean(losses[:nl])), "loss_last_epoch": float(np.mean(losses[-nl:])),
                          "held_out": summ,
                          "iteration_gain_vs_untrained": summ["untrained_fcg"]["mean_iters"] / summ["learned_fcg"]["mean_iters"],
                          "iteration_gain_vs_mixed_cg": summ["mixedfx16"]["mean_iters"] / summ["learned_fcg"]["mean_iters"],
                          "time_learned_over_plain64": summ["learned_fcg"]["mean_s"] / summ["plain64"]["mean_s"]}),
              flush=True)
        net.free()
        raw.free()


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--chosen", default=CHOSEN, choices=sorted(MODE_PREC),
                    help="solver mode of the timed step (the 4 sources batched)")
    ap.add_argument("--dslash-sweep", action="store_true", help="Dslash bandwidth sweep instead of the solve")
    ap.add_argument("--sweep-dims", nargs="+", default=["8", "16", "24", "32", "40", "48", "48x48x48x96"])
    ap.add_argument("--sweep-precs", nargs="+", default=["fp64", "fp32", "fp16", "fx16"])
    ap.add_argument("--sweep-recons", nargs="+", type=int, default=[18, 12])
    ap.add_argument("--sweep-reps", type=int, default=20)
    ap.add_argument("--sweep-nrhs", nargs="+", type=int, default=[1])
    ap.add_argument("--net-dims", type=int, default=32, help="lattice extent of the netpass config")
    ap.add_argument("--config", default="headline",
                    choices=["headline", "small", "multishift", "batch", "learned", "netpass", "links",
                             "gaugeforce", "fermionforce"])
    ap.add_argument("--learned-pairs", type=int, default=2000)
    ap.add_argument("--learned-fields", type=int, default=24)
    ap.add_argument("--learned-epochs", type=int, default=2)
    args = ap.parse_args(argv)
    if args.dslash_sweep:
        run_dslash_sweep(args)
        return
    if args.config != "headline":
        run_config(args)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        # the oracle runs on rank 0's host cores only; other ranks do no work
        res = run_reference(args, rank, world) if rank == 0 else None
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group(backend="nccl")
    res = run_gpu(args, rank, world, local_rank)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
