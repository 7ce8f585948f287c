"""GB300 validation and calibration of the estimator.

Two things the paper does on its own hardware, done here on GB300:

* calibration (Sec. 3): the LOAD and SCALE streaming kernels on repeated data sets of
  growing size give the effective L2 size (where the transfer rate falls from the L2
  level) and the L2 and DRAM bandwidths; an fp64 FMA loop gives the fp64 rate.  Together
  with the device's SM count they form a GB300 hardware descriptor.
* validation (Sec. 5): the 3D 25-point star stencil and a pull lattice-Boltzmann step run
  for a set of launch configurations; the estimator predicts, from the same address
  expressions and the calibrated descriptor, the L2 <- L1 load volume, the DRAM load and
  store volumes and the time; the measured volumes come from the counters the paper uses
  (lts__t_sectors_srcunit_tex_op_read, dram__bytes_read / _write) in an ncu run of the
  same command, and `report` compares them and refits the hit-rate coefficients of the
  capacity model (Sec. 4.5) to the measurements.

Commands (one GPU):
  python -m paper_2204_14242_gb300.validation calibrate > calib.json
  python -m paper_2204_14242_gb300.validation run --set stencil --calib calib.json > pred.json
  ncu --metrics <METRICS> --clock-control none -k regex:star_kernel -c 3 --csv --log-file m.csv \\
      python -m paper_2204_14242_gb300.validation run --set stencil --calib calib.json --once --only 0,1,2
  python -m paper_2204_14242_gb300.validation report pred.json m.csv ... > report.md
"""
from __future__ import annotations

import argparse
import csv
import ctypes
import json
import math
import os
import sys

import numpy as np

from . import binding as B
from . import workloads as W

METRICS = ("lts__t_sectors_srcunit_tex_op_read.sum,lts__t_sectors_srcunit_tex_op_write.sum,"
           "dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum")


def _lib():
    lib = B.load()
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.ws_val_stream.argtypes = [I, P, P, P, I64, I, I, I, P]
    lib.ws_val_fma.argtypes = [P, I, I, I, P]
    lib.ws_val_star.argtypes = [P, P, P, I, P, I, I, I, P]
    lib.ws_val_lbm.argtypes = [P, P, I, P, P, P, I, I, I, D, P]
    lib.ws_val_regs.argtypes = [I, I, I, I]
    for f in ("ws_val_stream", "ws_val_fma", "ws_val_star", "ws_val_lbm", "ws_val_regs"):
        getattr(lib, f).restype = I
    return lib


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"{what} failed with status {rc}")


# ---- calibration ----------------------------------------------------------------------------
def _time(torch, fn, reps=3):
    best = float("inf")
    for _ in range(reps + 1):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        fn()
        e.record()
        torch.cuda.synchronize()
        best = min(best, s.elapsed_time(e) * 1e-3)
    return best


def calibrate(device: int = 0) -> dict:
    """LOAD / SCALE rates over data-set sizes, the fp64 FMA rate, and the descriptor."""
    import torch
    torch.cuda.set_device(device)
    lib = _lib()
    props = torch.cuda.get_device_properties(device)
    sms = props.multi_processor_count
    blocks, threads = sms * 16, 256
    big = 1 << 28                               # 2 GiB of doubles
    a = torch.rand(big, dtype=torch.float64, device="cuda")
    b = torch.empty(big, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    sizes = [int(2 ** (k / 2)) for k in range(40, 62)]   # 1 MiB .. 2 GiB in sqrt(2) steps
    rows = []
    for nbytes in sizes:
        elems = max(1, nbytes // 8)
        per_pass = blocks * threads * 8
        iters = max(4, int(8e9 / per_pass))      # about 8 GB of LOAD traffic per launch
        t_load = _time(torch, lambda: _check(lib.ws_val_stream(0, a.data_ptr(), None, out.data_ptr(), elems, blocks,
                                                                threads, iters, None), "LOAD"))
        iters_s = max(2, iters // 2)
        t_scale = _time(torch, lambda: _check(lib.ws_val_stream(1, a.data_ptr(), b.data_ptr(), None, elems, blocks,
                                                                 threads, iters_s, None), "SCALE"))
        rows.append({"bytes": nbytes, "load_gbs": per_pass * iters / t_load / 1e9,
                     "scale_gbs": 2 * per_pass * iters_s / t_scale / 1e9})
    fiters = 4000
    t_fma = _time(torch, lambda: _check(lib.ws_val_fma(out.data_ptr(), sms * 8, 256, fiters, None), "FMA"))
    fp64 = sms * 8 * 256 * fiters * 64 * 8 * 2 / t_fma   # FMA counted as two flops
    # the model's fp peak is for the stencils' add-dominated mix: one flop per instruction,
    # half the FMA flop rate (as for the descriptors of Table 1)
    load = np.array([r["load_gbs"] for r in rows])
    sz = np.array([r["bytes"] for r in rows], float)
    l2_level = float(np.median(load[sz <= 16 << 20]))
    dram_level = float(np.median(load[sz >= 1 << 30]))
    # effective L2 (Sec. 3: the data-set size up to which L2 hits can be relied on): where
    # the LOAD rate falls below 90 % of its small-data-set level, interpolated in log size
    thr = 0.9 * l2_level
    eff = float(sz[-1])
    for i in range(1, len(sz)):
        if load[i - 1] >= thr > load[i]:
            f = (math.log(load[i - 1]) - math.log(thr)) / (math.log(load[i - 1]) - math.log(load[i]))
            eff = float(math.exp(math.log(sz[i - 1]) + f * (math.log(sz[i]) - math.log(sz[i - 1]))))
            break
    scale_dram = float(np.median([r["scale_gbs"] for r in rows if r["bytes"] >= 1 << 30]))
    hw = W.gb300(l2_bytes=eff, bw_l2=l2_level * 1e9, bw_dram=scale_dram * 1e9, fp_peak=fp64 / 2, sms=sms)
    return {"device": props.name, "sms": sms, "scan": rows, "l2_level_gbs": l2_level, "dram_level_gbs": dram_level,
            "scale_dram_gbs": scale_dram, "effective_l2_bytes": eff, "fp64_flops": fp64,
            "hw": {k: getattr(hw, k) for k in ("sms", "clock_hz", "l1_bytes", "l2_bytes", "bw_l2", "bw_dram",
                                                "fp_peak")}}


def hardware(calib: dict | None) -> W.Hardware:
    if not calib:
        return W.gb300()
    return W.gb300(**{k: calib["hw"][k] for k in ("l2_bytes", "bw_l2", "bw_dram", "fp_peak", "clock_hz", "sms")})


# ---- validation kernels and their estimator descriptions --------------------------------------
PAD = 4


def _layout(N):
    sx = N[0] + 2 * PAD
    sy = sx * (N[1] + 2 * PAD)
    strides = (1, sx, sy)
    return strides, PAD * (1 + sx + sy), sy * (N[2] + 2 * PAD)


def stencil_set():
    """25-point star (r = 4), fp64, 640 x 512 x 512: shapes and foldings of Sec. 5."""
    N = (640, 512, 512)
    shapes = [(32, 4, 1), (64, 2, 2), (128, 1, 1), (256, 2, 1), (512, 2, 1), (32, 8, 4), (16, 4, 8), (8, 8, 8),
              (64, 1, 8), (16, 2, 32), (8, 1, 64), (1024, 1, 1)]
    folds = [(0, 1), (2, 2), (1, 2)]
    out = []
    for i, Bs in enumerate(shapes):
        axis, f = folds[i % 3]
        out.append({"kind": "star", "N": N, "B": Bs, "fold_axis": axis, "fold": f, "r": 4})
    return out


def lbm_set():
    """Pull D3Q19 step, fp64, 256 x 256 x 128 (19 source + 19 destination arrays)."""
    N = (256, 256, 128)
    shapes = [(32, 4, 1), (64, 2, 2), (128, 1, 1), (256, 1, 1), (32, 8, 2), (16, 8, 4), (64, 1, 4), (8, 8, 8)]
    out = []
    for i, Bs in enumerate(shapes):
        axis, f = [(0, 1), (2, 2), (1, 2), (0, 1)][i % 4]
        out.append({"kind": "lbm", "N": N, "B": Bs, "fold_axis": axis, "fold": f, "q": 19})
    return out


SCAN_SHAPES = [(512, 2, 1), (256, 2, 2), (128, 2, 4), (64, 2, 8), (32, 2, 16), (16, 2, 32)]
SCAN_XY = [128, 192, 256, 320, 384, 448, 512, 576, 640, 768, 896, 1024]


def sizescan_set():
    """Layer-condition size scan (Sec. 5.7): the 25-point star on domains with square XY
    planes of growing size and a constant total of 2^27 points (z = 2^27 / XY^2), for block
    shapes of increasing z extent (waves of 1 .. 32 layers)."""
    out = []
    for Bs in SCAN_SHAPES:
        for xy in SCAN_XY:
            z = max(16, (1 << 27) // (xy * xy))
            out.append({"kind": "star", "N": (xy, xy, z), "B": Bs, "fold_axis": 0, "fold": 1, "r": 4})
    return out


D3Q19 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1), (1, 1, 0), (-1, -1, 0),
         (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1),
         (0, -1, 1)]


def model_config(v, regs: int = 0) -> W.Config:
    """The estimator's description of a validation kernel: the same address expressions
    (padded row-major arrays, base pointers aligned to 512 B by the allocator) and the
    kernel's registers per thread (which bound its resident blocks per SM)."""
    strides, c0, _ = _layout(v["N"])
    if v["kind"] == "star":
        src = W.Field(8, [W.Access(*o) for o in W.star_offsets(v["r"])], strides=strides, const_off=c0)
        dst = W.Field(8, [W.Access(0, 0, 0, 1)], strides=strides, const_off=c0)
        fields, flops = [src, dst], 6 * v["r"] + 3
    else:
        fields = [W.Field(8, [W.Access(-c[0], -c[1], -c[2])], strides=strides, const_off=c0) for c in D3Q19]
        fields += [W.Field(8, [W.Access(0, 0, 0, 1)], strides=strides, const_off=c0) for _ in D3Q19]
        flops = 3 * len(D3Q19) + 1
    return W.Config(N=tuple(v["N"]), B=tuple(v["B"]), fields=fields, fold_axis=v["fold_axis"], fold=v["fold"],
                    flops_per_lup=float(flops), regs_per_thread=max(0, regs))


def run(which: str, calib: dict | None, once: bool, only=None, reps: int = 5, predict_only: bool = False):
    """Runs the validation kernels (timed by CUDA events, or once each for an ncu
    capture) and prints one JSON line per configuration with the estimator's
    predictions for it."""
    import torch
    lib = _lib()
    hw = hardware(calib)
    ctx = B.Context(0, 8 << 30)
    sets = {"stencil": stencil_set, "lbm": lbm_set, "sizescan": sizescan_set}[which]()
    idx = range(len(sets)) if only is None else only
    for i in idx:
        v = sets[i]
        N = v["N"]
        _, _, elems = _layout(N)
        Nc = (ctypes.c_int32 * 3)(*N)
        Bc = (ctypes.c_int32 * 3)(*v["B"])
        if predict_only:
            launch = None
        elif v["kind"] == "star":
            src = torch.rand(elems, dtype=torch.float64, device="cuda")
            dst = torch.zeros(elems, dtype=torch.float64, device="cuda")
            launch = lambda: _check(lib.ws_val_star(src.data_ptr(), dst.data_ptr(), Nc, v["r"], Bc, v["fold_axis"],
                                                    v["fold"], PAD, None), "ws_val_star")
        else:
            q = len(D3Q19)
            srcs = [torch.rand(elems, dtype=torch.float64, device="cuda") for _ in range(q)]
            dsts = [torch.zeros(elems, dtype=torch.float64, device="cuda") for _ in range(q)]
            sp = torch.tensor([t.data_ptr() for t in srcs], dtype=torch.int64, device="cuda")
            dp = torch.tensor([t.data_ptr() for t in dsts], dtype=torch.int64, device="cuda")
            cc = (ctypes.c_int32 * (3 * q))(*[x for c in D3Q19 for x in c])
            launch = lambda: _check(lib.ws_val_lbm(sp.data_ptr(), dp.data_ptr(), q, cc, Nc, Bc, v["fold_axis"],
                                                   v["fold"], PAD, 0.6, None), "ws_val_lbm")
        torch.cuda.synchronize()
        if predict_only:
            t = None
        elif once:
            launch()
            torch.cuda.synchronize()
            t = None
        else:
            t = _time(torch, launch, reps)
        regs = lib.ws_val_regs(0 if v["kind"] == "star" else 1, v["r"] if v["kind"] == "star" else v["q"],
                               v["fold_axis"], v["fold"])
        res, _ = B.ws_estimate_batch(ctx, [model_config(v, regs)], hw)
        r = B.results_to_dicts(res)[0]
        a100, _ = B.ws_estimate_batch(ctx, [model_config(v, regs)], W.a100())
        a100 = B.results_to_dicts(a100)[0]
        lups = N[0] * N[1] * N[2]
        print(json.dumps({"i": i, **{k: v[k] for k in v}, "regs": regs, "lups": lups, "seconds": t,
                          "glups": lups / t / 1e9 if t else None,
                          "pred": {k: r[k] for k in ("v_l1", "v_l2_load", "v_l2_store", "v_dram_load", "v_dram_store",
                                                     "t_pred", "glups", "limiter", "o_l1", "o_y", "o_z",
                                                     "l1_req_sectors", "blk_load_sectors", "lups_block",
                                                     "wave_load_sectors", "lups_wave", "ov_y", "ov_z",
                                                     "wave_store_req_sectors", "wave_store_sectors")},
                          "a100_v_dram_load": a100["v_dram_load"],
                          "hw": {k: getattr(hw, k) for k in ("l2_bytes", "bw_l2", "bw_dram", "fp_peak")}}),
              flush=True)
        del launch
        torch.cuda.empty_cache()
    ctx.close()


# ---- report ----------------------------------------------------------------------------------
def _ncu_rows(paths):
    """Per captured launch (in order): metric -> value, from ncu --csv logs."""
    out = []
    for p in paths:
        rows = list(csv.reader(open(p)))
        hi = [i for i, r in enumerate(rows) if "Metric Name" in r][0]
        h = rows[hi]
        ki, ii, mi, ui, vi = (h.index("Kernel Name"), h.index("ID"), h.index("Metric Name"), h.index("Metric Unit"),
                              h.index("Metric Value"))
        launches = {}
        for r in rows[hi + 1:]:
            if len(r) <= vi:
                continue
            val = float(r[vi].replace(",", ""))
            unit = r[ui]
            scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "ns": 1e-9, "us": 1e-6, "usecond": 1e-6,
                     "ms": 1e-3, "msecond": 1e-3, "nsecond": 1e-9, "sector": 1, "": 1}.get(unit, 1)
            launches.setdefault((p, int(r[ii])), {})[r[mi]] = val * scale
        out += [launches[k] for k in sorted(launches)]
    return out


def _rhat(p, O):
    a, b, c = p
    return a * np.exp(-b * np.exp(-c * O))


def report(pred_path: str, ncu_paths, only=None) -> str:
    preds = [json.loads(l) for l in open(pred_path) if l.strip().startswith("{")]
    meas = _ncu_rows(ncu_paths)
    ids = only if only is not None else [p["i"] for p in preds][:len(meas)]
    byi = {p["i"]: p for p in preds}
    lines = ["| # | kernel | block | fold | L2<-L1 load B/LUP pred / meas | DRAM load B/LUP pred / meas | "
             "DRAM store B/LUP pred / meas | GLup/s pred / meas | limiter |", "|" + "---|" * 9]
    pts = []
    for k, i in enumerate(ids):
        if k >= len(meas) or i not in byi:
            continue
        p, m = byi[i], meas[k]
        lups = p["lups"]
        l2 = 32.0 * m.get("lts__t_sectors_srcunit_tex_op_read.sum", float("nan")) / lups
        dl = m.get("dram__bytes_read.sum", float("nan")) / lups
        ds = m.get("dram__bytes_write.sum", float("nan")) / lups
        gl = lups / m.get("gpu__time_duration.sum", float("nan")) / 1e9
        pr = p["pred"]
        fold = "-" if p["fold_axis"] == 0 else f"{p['fold']}{'yz'[p['fold_axis'] - 1]}"
        lines.append(f"| {i} | {p['kind']} | {tuple(p['B'])} | {fold} | {pr['v_l2_load']:.1f} / {l2:.1f} | "
                     f"{pr['v_dram_load']:.1f} / {dl:.1f} | {pr['v_dram_store']:.1f} / {ds:.1f} | "
                     f"{pr['glups']:.1f} / {p['glups'] if p['glups'] else gl:.1f} | {'L1 L2 DRAM FP'.split()[pr['limiter']]} |")
        pts.append((p, l2, dl, ds, p["glups"] if p["glups"] else gl))
    if not pts:
        return "\n".join(lines)
    err = lambda a, b: abs(a - b) / max(b, 1e-12)
    e_l2 = [err(p["pred"]["v_l2_load"], l2) for p, l2, _, _, _ in pts]
    e_dl = [err(p["pred"]["v_dram_load"], dl) for p, _, dl, _, _ in pts]
    e_ds = [err(p["pred"]["v_dram_store"], ds) for p, _, _, ds, _ in pts]
    lines.append("")
    lines.append(f"Median relative error: L2<-L1 load {np.median(e_l2):.2f}, DRAM load {np.median(e_dl):.2f}, "
                 f"DRAM store {np.median(e_ds):.2f}.")
    tp = np.array([p["pred"]["t_pred"] for p, *_ in pts])
    tm = np.array([1.0 / (g * 1e9) for *_, g in pts])
    if len(pts) > 2:
        rp, rm = np.argsort(np.argsort(tp)), np.argsort(np.argsort(tm))
        rho = 1 - 6 * np.sum((rp - rm) ** 2) / (len(pts) * (len(pts) ** 2 - 1))
        lines.append(f"Rank correlation (Spearman) of predicted and measured time: {rho:.2f}.")
    # refit of the L1 hit-rate curve: measured V_L2L1 = V_comp + (1 - R)(V_up - V_comp)
    O, R = [], []
    for p, l2, *_ in pts:
        pr = p["pred"]
        v_up = pr["v_l1"]
        v_comp = 32.0 * pr["blk_load_sectors"] / pr["lups_block"]
        if v_up - v_comp > 1e-9 and math.isfinite(l2):
            O.append(pr["o_l1"])
            R.append(min(1.0, max(0.0, 1.0 - (l2 - v_comp) / (v_up - v_comp))))
    if len(O) >= 3:
        try:
            from scipy.optimize import least_squares
            f = least_squares(lambda q: _rhat(q, np.array(O)) - np.array(R), x0=[1.0, 0.01, -3.07],
                              bounds=([0.0, 1e-6, -50.0], [1.0, 50.0, 0.0]))
            lines.append(f"Refitted L1 hit-rate coefficients (a, b, c) of R(O) = a exp(-b exp(-c O)) from "
                         f"{len(O)} configurations: ({f.x[0]:.3f}, {f.x[1]:.4f}, {f.x[2]:.3f}); residual rms "
                         f"{math.sqrt(np.mean(f.fun ** 2)):.3f}.")
        except ImportError:
            pass
    return "\n".join(lines)


def scan_report(pred_path: str, ncu_paths, only=None) -> str:
    """DRAM load volume (B/LUP) over the XY plane size, per block shape: predicted with
    the calibrated GB300 descriptor and with the A100 one, and measured where counters
    were captured (in the order of `only`)."""
    preds = [json.loads(l) for l in open(pred_path) if l.strip().startswith("{")]
    meas = _ncu_rows(ncu_paths) if ncu_paths else []
    measured = {}
    for k, i in enumerate(only or []):
        if k < len(meas):
            measured[i] = meas[k].get("dram__bytes_read.sum", float("nan"))
    shapes = sorted({tuple(p["B"]) for p in preds}, key=lambda b: b[2])
    xys = sorted({p["N"][0] for p in preds})
    head = "| XY | " + " | ".join(f"{b} GB300 / A100 / meas" for b in shapes) + " |"
    lines = [head, "|" + "---|" * (len(shapes) + 1)]
    for xy in xys:
        cells = []
        for b in shapes:
            p = next((q for q in preds if tuple(q["B"]) == b and q["N"][0] == xy), None)
            if p is None:
                cells.append("")
                continue
            m = measured.get(p["i"])
            ms = f"{m / p['lups']:.1f}" if m is not None else "-"
            cells.append(f"{p['pred']['v_dram_load']:.1f} / {p['a100_v_dram_load']:.1f} / {ms}")
        lines.append(f"| {xy} | " + " | ".join(cells) + " |")
    return "\n".join(lines)


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2204_14242_gb300.validation")
    sub = ap.add_subparsers(dest="cmd", required=True)
    c = sub.add_parser("calibrate")
    c.add_argument("--device", type=int, default=0)
    r = sub.add_parser("run")
    r.add_argument("--set", choices=["stencil", "lbm", "sizescan"], default="stencil")
    r.add_argument("--predict-only", action="store_true", help="estimator predictions only (no kernel runs)")
    r.add_argument("--calib")
    r.add_argument("--once", action="store_true", help="one launch per configuration (for an ncu capture)")
    r.add_argument("--only", help="comma-separated configuration indices")
    p = sub.add_parser("report")
    p.add_argument("pred")
    p.add_argument("ncu", nargs="+")
    p.add_argument("--only")
    p.add_argument("--scan", action="store_true", help="size-scan table (DRAM load over the XY plane size)")
    a = ap.parse_args(argv)
    if a.cmd == "calibrate":
        print(json.dumps(calibrate(a.device)))
    elif a.cmd == "run":
        calib = json.load(open(a.calib)) if a.calib else None
        only = [int(x) for x in a.only.split(",")] if a.only else None
        run(a.set, calib, a.once, only, predict_only=a.predict_only)
    else:
        only = [int(x) for x in a.only.split(",")] if a.only else None
        print(scan_report(a.pred, a.ncu, only) if a.scan else report(a.pred, a.ncu, only))


if __name__ == "__main__":
    main()
