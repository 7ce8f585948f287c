"""Writes the stored oracle results that the full-size GPU parity tests compare against.

Run on the CPU (no GPU, no CUDA library involved):

    python tests/make_oracle_golden.py [--only NAME ...] [--threads N]

Every expected value is computed by the CPU oracle (``oracle/``, a plain std::set
enumerator of Sec. 4.2-4.5 of the paper) from the seeded generators of
``paper_2204_14242_gb300.workloads`` (which describe inputs and hold none of the
method's arithmetic).  Nothing here loads or calls the CUDA path.

Sets written to ``tests/golden/oracle_<name>.npz``:
  * stencil_25pt_sweep   all 755 candidates (25-point star, 640x512x512, Sec. 5.2)
  * lbm_sweep            all 755 candidates (27 D3Q27 + 15 D3Q15 arrays, 256^3, Sec. 5.3)
  * mixed_set_sample     a stratified seeded sample of the 20,000-candidate mixed set:
                         the 12 smallest and 12 largest by enumeration work, the 8 with the
                         largest address range, and one seeded pick from each of 180 equal
                         strata of the work order (>= 200 candidates)
  * request_stream_small every candidate of the 24-request stream (seed 77, 4..40
                         candidates per request) that the server test submits

Each file holds the candidate indices, the oracle's integer and fp64 outputs
(``oracle.INT_KEYS`` / ``oracle.DBL_KEYS`` columns) and a SHA-256 fingerprint of the
oracle's flattened inputs, so a test can tell when the generators have drifted.
"""
from __future__ import annotations

import argparse
import hashlib
import math
import os
import sys
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

import oracle  # noqa: E402
from paper_2204_14242_gb300 import workloads as W  # noqa: E402

GOLDEN = os.path.join(HERE, "golden")
SERVER_STREAM = dict(n_requests=24, seed=77, kmin=4, kmax=40)


def fingerprint(configs, hw) -> str:
    """SHA-256 of the oracle's flattened inputs for these candidates."""
    h = hashlib.sha256()
    for a in oracle.flatten(configs, hw):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def work_proxy(c: W.Config, hw: W.Hardware) -> int:
    """Threads of one modelled wave x accesses per thread: a cost estimate used only to
    stratify the sample (the oracle's run time grows with it)."""
    T = c.B[0] * c.B[1] * c.B[2]
    warps = -(-T // 32)
    bpsm = max(1, min(hw.max_blocks_sm, hw.max_threads_sm // (32 * warps)))
    fy = c.fold if c.fold_axis == 1 else 1
    fz = c.fold if c.fold_axis == 2 else 1
    g = (-(-c.N[0] // c.B[0]), -(-c.N[1] // (c.B[1] * fy)), -(-c.N[2] // (c.B[2] * fz)))
    waves = min(hw.sms * bpsm, g[0] * g[1] * g[2])
    acc = sum(len(f.accesses) for f in c.fields) * c.fold
    return waves * T * acc


def range_proxy(c: W.Config) -> int:
    """Bytes of address space one wave-level field spans, roughly: planes of the domain
    the wave and its stencil reach, times the number of fields."""
    fz = c.fold if c.fold_axis == 2 else 1
    es = max(f.elem_bytes for f in c.fields)
    r = max(max(abs(a.dz) for a in f.accesses) for f in c.fields)
    return es * c.N[0] * c.N[1] * (c.B[2] * fz + 2 * r + 1) * len(c.fields)


def mixed_sample(cfgs, hw, seed: int = 20231):
    n = len(cfgs)
    work = np.array([work_proxy(c, hw) for c in cfgs], np.int64)
    order = np.argsort(work, kind="stable")
    chosen = set(order[:12].tolist()) | set(order[-12:].tolist())
    rng = np.array([range_proxy(c) for c in cfgs], np.int64)
    chosen |= set(np.argsort(rng, kind="stable")[-8:].tolist())
    strata = 180
    r = W.SplitMix64(seed)
    for s in range(strata):
        lo, hi = (s * n) // strata, ((s + 1) * n) // strata
        chosen.add(int(order[r.randint(lo, hi - 1)]))
    return sorted(chosen)


def run_oracle(configs, hw, threads: int):
    """One oracle call per candidate on a pool of host threads (each call single-threaded),
    largest first, so that the biggest candidates do not end up last on one thread."""
    n = len(configs)
    out_i = np.zeros((n, len(oracle.INT_KEYS)), np.int64)
    out_d = np.zeros((n, len(oracle.DBL_KEYS)), np.float64)
    cost = [work_proxy(c, hw) for c in configs]
    todo = sorted(range(n), key=lambda i: -cost[i])
    done = [0]
    t0 = time.time()

    def one(i):
        oi, od = oracle.estimate_arrays([configs[i]], hw, threads=1)
        out_i[i], out_d[i] = oi[0], od[0]
        done[0] += 1
        if done[0] % 50 == 0:
            print(f"    {done[0]}/{n} after {time.time() - t0:.0f} s", flush=True)

    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(one, todo))
    return out_i, out_d


def write(name, configs, idx, hw, threads, extra=None):
    sel = [configs[i] for i in idx]
    t0 = time.time()
    out_i, out_d = run_oracle(sel, hw, threads)
    path = os.path.join(GOLDEN, f"oracle_{name}.npz")
    arrays = dict(idx=np.asarray(idx, np.int64), out_i=out_i, out_d=out_d,
                  int_keys=np.array(oracle.INT_KEYS), dbl_keys=np.array(oracle.DBL_KEYS),
                  fingerprint=np.array(fingerprint(sel, hw)))
    if extra:
        arrays.update(extra)
    np.savez_compressed(path, **arrays)
    print(f"{name}: {len(idx)} candidates in {time.time() - t0:.0f} s -> {path}", flush=True)


def sets():
    hw = W.a100()
    c1 = W.stencil_25pt_sweep()
    c2 = W.lbm_sweep()
    yield "stencil_25pt_sweep", lambda: (c1, list(range(len(c1))), hw, None)
    yield "lbm_sweep", lambda: (c2, list(range(len(c2))), hw, None)

    def mixed():
        c3 = W.mixed_set()
        return c3, mixed_sample(c3, hw), hw, None
    yield "mixed_set_sample", mixed

    def stream():
        reqs = W.request_stream(**SERVER_STREAM)
        flat = [c for r in reqs for c in r.configs]
        starts = np.cumsum([0] + [len(r.configs) for r in reqs]).astype(np.int64)
        return flat, list(range(len(flat))), hw, dict(request_starts=starts)
    yield "request_stream_small", stream


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", nargs="*", default=None)
    ap.add_argument("--threads", type=int, default=max(1, len(os.sched_getaffinity(0))))
    a = ap.parse_args()
    oracle.build()
    for name, make in sets():
        if a.only and name not in a.only:
            continue
        configs, idx, hw, extra = make()
        write(name, configs, idx, hw, a.threads, extra)


if __name__ == "__main__":
    main()
