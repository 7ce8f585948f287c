#!/usr/bin/env python
"""Benchmark of the GB300 estimator (one JSON line on stdout, rank 0).

Default workload: the 3D 25-point star (radius 4) sweep, fp64, 640x512x512 with
x = 640 contiguous, 151 block shapes x 5 folding variants = 755 candidates.  One
step estimates every candidate (block and wave enumeration, bitmap counting, model,
ranking) with the batched form: one persistent enumeration launch per scratch pass,
replayed as a CUDA graph, descriptors already resident on the device.  Reported:
  value      candidates/s of that step (device time, CUDA events, L2 flushed between
             steps), summed over ranks (weak scaling: every rank runs the full sweep)
  e2e        the same metric through ws_estimate_batch with host buffers (descriptor
             compile, host->device copies, kernels, device->host results) per step
  plain      candidates/s of the plain form (one synchronous launch sequence per candidate)
  served     the Poisson request stream through the continuous-batching server (p50/p99)
  roofline   the kernel with the largest share of the step, against the rate that bounds
             it (all three under roofline.kernels): the representative-block kernel
             (exact per-address path) against the measured int32-add rate, the row walk
             against the measured L2 red.or rate, the counting kernel against the
             measured HBM copy bandwidth (MEASURED_PEAKS.json); traffic = the DRAM bytes
             per launch ncu measured for that kernel on this workload, read from
             profiles/dram_traffic_<workload>.txt while the kernel source is unchanged
  cpu_baseline  the CPU oracle on a bounded sample of the same sweep, all host cores

--impl reference times the CPU oracle itself on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "configs/sec and unique sectors/sec (exact vs oracle), batched+served vs plain; p50/p99"
UNIT = "configs/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # default: 1000 timed steps on the GPU (about 0.7 s, so the clock sampler sees the timed
    # region several times); 3 for the reference arm, whose steps take seconds each
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="stencil_25pt", choices=["stencil_25pt", "lbm", "mixed", "stencil_7pt"])
    ap.add_argument("--serve-seconds", type=float, default=8.0)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--arena-gb", type=float, default=48.0)
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the default tuning instead of autotuning the plan before timing")
    ap.add_argument("--subset", type=int, default=1,
                    help="keep every K-th candidate (small cases for profiling); 1 = the whole workload")
    return ap.parse_args()


def workload(name):
    from paper_2204_14242_gb300 import workloads as W
    if name == "stencil_25pt":
        return W.stencil_25pt_sweep(), {"workload": "3D 25-point star r=4 sweep, fp64, 640x512x512 (x=640 contiguous), "
                                                   "151 block shapes x {none,2y,4y,2z,4z} folding = 755 candidates",
                                        "candidates": 755, "modelled_gpu": "A100-SXM4-40G (Table 1)"}
    if name == "lbm":
        return W.lbm_sweep(), {"workload": "LBM-shaped: 27 D3Q27 + 15 D3Q15 fp64 arrays, 256^3, 755 candidates",
                               "candidates": 755, "modelled_gpu": "A100-SXM4-40G (Table 1)"}
    if name == "mixed":
        return W.mixed_set(), {"workload": "20000 seeded mixed stencils (seed 20221)", "candidates": 20000,
                               "modelled_gpu": "A100-SXM4-40G (Table 1)"}
    return [W.stencil_7pt_128()], {"workload": "3D 7-point star 128^3 block 32x4x1 wave 8", "candidates": 1}


def cores():
    return len(os.sched_getaffinity(0))


def step_time_over_ranks(ms_step: float, dist=None, device=None) -> float:
    """Slowest rank's step time (the job finishes when the last replica does)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms_step
    import torch
    t = torch.tensor([ms_step], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(candidates_per_rank: int, world: int, ms_step: float) -> float:
    """Whole-job candidates per second: every rank runs its own full workload (weak scaling)."""
    return world * candidates_per_rank / (ms_step * 1e-3)


# ---- clocks during the timed region ---------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.reader.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---- reference arm: the CPU oracle --------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2204_14242_gb300 import workloads as W
    cfgs, cfg_meta = workload(args.workload)
    hw = W.a100()
    ncore = cores()
    per_step = max(1, min(len(cfgs), ncore))
    stride = max(1, len(cfgs) // (per_step * max(1, args.steps + args.warmup)))
    pool = cfgs[::stride]
    k = 0
    def step():
        nonlocal k
        batch = [pool[(k + i) % len(pool)] for i in range(per_step)]
        k += per_step
        t = time.perf_counter()
        oracle.estimate(batch, hw, threads=ncore)
        return time.perf_counter() - t
    for _ in range(args.warmup):
        step()
    times = [step() for _ in range(args.steps)]
    sec = sum(times) / len(times)
    value = per_step / sec
    sample = f"{per_step} candidates per step, every {stride}-th of the {len(cfgs)}-candidate sweep, rotating"
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "int64+f64", "data": "synthetic",
           "config": dict(cfg_meta, parallelism="host threads", l2="n/a (CPU)"),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncore, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def cpu_baseline(cfgs, hw, seconds):
    import oracle
    ncore = cores()
    # calibrate on a few candidates, then size the sample for about `seconds` of work
    probe = cfgs[:: max(1, len(cfgs) // ncore)][:ncore]
    t = time.perf_counter()
    oracle.estimate(probe, hw, threads=ncore)
    dt = max(time.perf_counter() - t, 1e-3)
    n = max(ncore, min(len(cfgs), int(len(probe) * seconds / dt)))
    stride = max(1, len(cfgs) // n)
    sample = cfgs[::stride][:n]
    t = time.perf_counter()
    oracle.estimate(sample, hw, threads=ncore)
    dt = time.perf_counter() - t
    # one core: an evenly spread part of the sample, sized for about a third of the time
    # above (per-candidate single-core time estimated as dt x cores / sample size)
    n1 = max(1, min(len(sample), int(seconds / 3 / max(dt * ncore / len(sample), 1e-6))))
    one = sample[::max(1, len(sample) // n1)][:n1]
    t = time.perf_counter()
    oracle.estimate(one, hw, threads=1)
    dt1 = time.perf_counter() - t
    return {"value": len(sample) / dt, "unit": UNIT, "cores": ncore, "kind": "oracle",
            "value_1core": len(one) / dt1,
            "sample": f"{len(sample)} candidates (every {stride}-th of {len(cfgs)}), std::set enumerator, "
                      f"one candidate per thread, {dt:.1f} s; 1 core: {len(one)} of them in {dt1:.1f} s"}


def measured_hbm_gbs():
    """Copy bandwidth measured on the GB300s (driver-written), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def kernel_source_digest():
    """sha256 of the kernels' source: DRAM traffic taken by ncu holds only for this source."""
    import hashlib
    with open(os.path.join(ROOT, "paper_2204_14242_gb300", "csrc", "ws_kernels.cu"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def recorded_traffic(workload_key):
    """DRAM bytes per launch of each kernel (dram__bytes_read.sum + dram__bytes_write.sum,
    one ncu capture of this workload), from profiles/dram_traffic_<workload>.txt when it
    was taken from the current kernel source; else {}."""
    path = os.path.join(ROOT, "profiles", f"dram_traffic_{workload_key}.txt")
    try:
        lines = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    except OSError:
        return {}
    kv = {ln[0]: ln[1] for ln in lines if len(ln) >= 2}
    if kv.get("kernel_source_sha256") != kernel_source_digest():
        return {}
    return {k: int(v) for k, v in kv.items() if k.endswith("_kernel")}


def kernel_rooflines(profs, peaks, workload_key=None):
    """Each kernel's achieved rate against the device rate that bounds it; the one with
    the largest share of the step is reported at the top level.

    enum_kernel  representative block, exact per-address path: addresses evaluated
                 (valid threads x issued accesses of the block) / s vs int32 adds / s
    rows_kernel  row walk: 64-bit red.or inserts (one per bitmap unit a sector range
                 covers) / s vs the measured L2 red.or rate on distinct words
    count_kernel bitmap bytes read / s vs the measured HBM copy bandwidth
    """
    med = lambda k: statistics.median(p[k] for p in profs)
    last = profs[-1]
    block_addresses = int(last["block_addresses"])
    ms = {"enum_kernel": med("ms_enum"), "rows_kernel": med("ms_rows"), "count_kernel": med("ms_count")}
    hbm, hbm_src = measured_hbm_gbs()
    k = {}
    a = block_addresses / (ms["enum_kernel"] * 1e-3) if ms["enum_kernel"] > 0 else 0.0
    k["enum_kernel"] = {"bound": "alu", "achieved": a / 1e9, "peak": peaks["int_ops_per_s"] / 1e9,
                        "unit": "G addresses/s vs G int32-add/s (measured)", "frac": a / peaks["int_ops_per_s"],
                        "per_launch": block_addresses, "ms": ms["enum_kernel"]}
    r = last["row_reds"] / (ms["rows_kernel"] * 1e-3) if ms["rows_kernel"] > 0 else 0.0
    k["rows_kernel"] = {"bound": "l2_atomic", "achieved": r / 1e9, "peak": peaks["l2_red_per_s"] / 1e9,
                        "unit": "G red.or/s (measured)", "frac": r / peaks["l2_red_per_s"],
                        "per_launch": int(last["row_reds"]), "ms": ms["rows_kernel"]}
    b = last["bitmap_bytes"] / (ms["count_kernel"] * 1e-3) if ms["count_kernel"] > 0 else 0.0
    k["count_kernel"] = {"bound": "hbm", "achieved": b / 1e9, "peak": hbm, "unit": f"GB/s ({hbm_src})",
                         "frac": b / 1e9 / hbm, "per_launch": int(last["bitmap_bytes"]), "ms": ms["count_kernel"]}
    top = max(ms, key=ms.get)
    traffic = recorded_traffic(workload_key) if workload_key else {}
    for name in k:
        k[name]["traffic"] = traffic.get(name)
    out = dict(k[top])
    out.update({"kernel": top, "share": ms[top] / last["ms_total"], "kernels": k,
                "ms_model": med("ms_model"), "ms_rank": med("ms_rank"), "ms_step_profiled": med("ms_total")})
    return out


def serve(B, W, ctx, hw, seconds, seed=20222, rate_hz=200.0):
    """Poisson request stream through the server; latency from arrival to completed poll."""
    n_req = max(1, int(seconds * rate_hz))
    reqs = W.request_stream(n_requests=n_req, seed=seed, rate_hz=rate_hz)
    arrays = [B.marshal(r.configs) for r in reqs]
    srv = B.Server(ctx, hw, mem_budget=int(24 << 30), max_inflight=4, max_step_cfgs=4096)
    try:
        return _serve(B, srv, reqs, arrays, rate_hz)
    finally:
        srv.close()


def _serve(B, srv, reqs, arrays, rate_hz):
    lat = {}
    done = threading.Event()
    submitted = {}
    lock = threading.Lock()

    def poller():
        while not done.is_set() or submitted:
            with lock:
                items = list(submitted.items())
            if not items:
                time.sleep(0.0002)
                continue
            for rid, t_arr in items:
                rc, res, order = srv.poll(rid, timeout_us=200)
                if rc == B.WS_EAGAIN:
                    continue
                now = time.perf_counter()
                with lock:
                    del submitted[rid]
                lat[rid] = (now - t_arr, rc, len(res) if res is not None else 0)

    th = threading.Thread(target=poller, daemon=True)
    th.start()
    t0 = time.perf_counter()
    for r, arr in zip(reqs, arrays):
        target = t0 + r.arrival_s
        while True:
            d = target - time.perf_counter()
            if d <= 0:
                break
            time.sleep(min(d, 0.001))
        rid = srv.submit(arrays=arr)
        with lock:
            submitted[rid] = target
    done.set()
    th.join()
    t1 = time.perf_counter()
    stats = srv.stats()
    ls = sorted(v[0] for v in lat.values())
    ok = sum(1 for v in lat.values() if v[1] == 0)
    cfg_done = sum(v[2] for v in lat.values())
    q = lambda p: ls[min(len(ls) - 1, int(math.ceil(p * len(ls))) - 1)] * 1e3
    offered = sum(len(r.configs) for r in reqs) / max(reqs[-1].arrival_s, 1e-9)
    return {"requests": len(reqs), "ok": ok, "p50_ms": q(0.50), "p99_ms": q(0.99), "configs_per_s": cfg_done / (t1 - t0),
            "offered_configs_per_s": offered, "steps": stats["steps"], "peak_scratch_bytes": stats["peak_bytes"],
            "rate_hz": rate_hz, "seconds": t1 - t0}


def main():
    args = parse()
    if args.steps is None:
        args.steps = 3 if args.impl == "reference" else 1000
    if args.impl == "reference":
        run_reference(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    from paper_2204_14242_gb300 import _build
    _build.build()
    from paper_2204_14242_gb300 import binding as B
    from paper_2204_14242_gb300 import workloads as W

    cfgs, cfg_meta = workload(args.workload)
    if args.subset > 1:
        cfgs = cfgs[::args.subset]
        cfg_meta = dict(cfg_meta, candidates=len(cfgs), subset=f"every {args.subset}-th candidate")
    hw = W.a100()
    ctx = B.Context(local, int(args.arena_gb * (1 << 30)))
    peaks = B.ws_measure_peaks(ctx)    # before the plan takes the arena
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")
    arrays = B.marshal(cfgs)
    plan = B.Plan(ctx, arrays=arrays, hw=hw)
    prof0 = plan.profile(stream)   # first direct step: also warms up the kernels
    tuning = plan.autotune(stream) if args.autotune else None

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(max(args.warmup, 3)):
        with torch.cuda.stream(stream):
            flush.random_(0, 255)
        plan.execute(B.WS_MODE_BATCHED, stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for s, e in evs:
        with torch.cuda.stream(stream):
            flush.random_(0, 255)          # L2 flush outside the timed events
        s.record(stream)
        plan.execute(B.WS_MODE_BATCHED, stream)
        e.record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = [s.elapsed_time(e) for s, e in evs]
    ms_step = step_time_over_ranks(sum(ms) / len(ms), dist, f"cuda:{local}")
    res, order = plan.results(stream)
    value = job_throughput(len(cfgs), world, ms_step)
    unique_sectors = int(res["blk_load_sectors"].sum() + res["blk_store_sectors"].sum() + res["wave_load_sectors"].sum()
                         + res["wave_store_sectors"].sum())
    sectors_per_s = world * unique_sectors / (ms_step * 1e-3)

    # per-kernel rooflines: CUDA events around each kernel on its own launch stream
    profs = [plan.profile(stream) for _ in range(3)]
    roofline = kernel_rooflines(profs, peaks, args.workload if args.subset == 1 else None)
    launches_per_step = profs[-1]["launches"]

    extra = {}
    if not args.no_plain and rank == 0 and len(cfgs) <= 4096:
        t = time.perf_counter()
        plan.execute(B.WS_MODE_PLAIN, stream)
        torch.cuda.synchronize()
        plain_s = time.perf_counter() - t
        rp, op = plan.results(stream)
        extra["plain"] = {"value": len(cfgs) / plain_s, "unit": UNIT, "ms_per_step": plain_s * 1e3,
                          "identical_to_batched": rp.tobytes() == res.tobytes()}
        extra["batched_over_plain"] = value / world / extra["plain"]["value"]
    # the resident plan is released first: the server and each one-shot call then have
    # the arena to themselves
    plan.close()
    if args.serve_seconds > 0 and rank == 0:
        extra["served"] = serve(B, W, ctx, hw, args.serve_seconds)
        sv = extra["served"]
        if sv["offered_configs_per_s"] > sv["configs_per_s"]:
            # over capacity at the specified rate: also serve at ~70 % of the measured capacity
            mean_k = sv["offered_configs_per_s"] / 200.0
            rate = max(1.0, 0.7 * sv["configs_per_s"] / mean_k)
            extra["served_at_70pct_capacity"] = serve(B, W, ctx, hw, args.serve_seconds, rate_hz=rate)

    # e2e: host buffers in, host results out, every step
    e2e_steps = max(2, min(args.steps, 5))
    h2d = profs[-1]["upload_bytes"]
    d2h = len(cfgs) * (B.RESULT.itemsize + 4)
    B.ws_estimate_batch(ctx, hw=hw, mode=B.WS_MODE_BATCHED, stream=stream, arrays=arrays)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(e2e_steps):
        r2, o2 = B.ws_estimate_batch(ctx, hw=hw, mode=B.WS_MODE_BATCHED, stream=stream, arrays=arrays)
    e2e_s = (time.perf_counter() - t) / e2e_steps
    if r2.tobytes() != res.tobytes() or o2.tobytes() != order.tobytes():
        raise SystemExit("e2e results differ from the resident plan's")

    out = None
    if rank == 0:
        base = cpu_baseline(cfgs, hw, args.cpu_seconds) if world == 1 and args.cpu_seconds > 0 else None
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "int64+f64", "data": "synthetic",
               "config": dict(cfg_meta, parallelism=f"replicas x{world} (independent candidates, no collective)",
                              l2="flushed between steps (256 MiB write)", mode="batched: persistent + CUDA graph",
                              tuning=tuning),
               "unique_sectors_per_s": sectors_per_s,
               "e2e": {"value": len(cfgs) / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                       "d2h_bytes_per_step": int(d2h)},
               "roofline": roofline,
               "gpu_launches": launches_per_step * args.steps,
               "clocks": clk, "cpu_baseline": base}
        out.update(extra)
        print(json.dumps(out))
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
