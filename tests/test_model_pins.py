"""Pins of the oracle's floating-point half: the capacity-miss model (Sec. 4.5) and the
limiters (Sec. 2), against closed forms derived by hand (CPU only).

The 7-point case (``workloads.stencil_7pt_128``: fp64, 128^3, block 32x4x1, a wave of 8
blocks, A100 column of Table 1) has every integer input of the model pinned already
(``test_oracle_pins.test_7pt_block_and_wave_closed_form``): 128 / 1024 LUPs, 232 request
and 120 compulsory sectors, 36 block lines, 16 resident blocks per SM (2048 threads /
128), 832 wave sectors in 208 lines, 256 store sectors in 64 lines, ov_y 64, ov_z 480,
and the y / z sets starting 4 and 128 blocks before the wave.  From these:

  O_L1 = 128 B x 36 lines x 16 blocks / 192 KiB              = 3/8
  O_y  = 4 blocks x (128 B x 208 lines / 8 blocks) / 20 MiB    = 13/20480
  O_z  = 128 blocks x (128 B x 208 lines / 8 blocks) / 20 MiB  = 13/640
  O_st = 128 B x 64 store lines / 20 MiB                       = 1/2560
  T_L1 = (64 cycles / 128 LUP) / (1.41 GHz x 108 SMs)
  T_FP = 7 flop / 4.9 TFlop/s

With hit curves R(O) = a exp(-b exp(-c O)) chosen so that exp(-c O) is 2, 3 or 4 at this
O and b times it is ln 2, every R is a / 2, and each volume becomes a rational number:
  V_L2<-L1 = 30 + (1 - 1/2)(58 - 30) = 44 B/LUP           (compulsory 30, request 58)
  V_DRAM   = 26 - (64/2 + 480/4) x 32 B / 1024 = 21.25 B/LUP (R_y = 1/2, R_z = 1/4)
  T_L2     = (44 + 8) / 5000 GB/s,  T_DRAM = (21.25 + 8) / 1400 GB/s = T_pred (DRAM bound).
With b = 1, c = 0 every R is a / e whatever O is.

A second case pins the store terms: a streaming copy whose destination starts 8 bytes
past a sector boundary.  Each warp stores 256 bytes over 9 sectors (288 requests in the
wave), the wave's 8 contiguous rows store 8192 bytes over 257 sectors and 65 lines, so
V_red,st = 32 x (288 - 257) / 1024 B/LUP and O_st = 128 x 65 / 20 MiB = 13/32768; a hit
curve with R_st(13/32768) = 1/2 charges half of it as DRAM load.

The last test plants plausible mistakes in a copy of the oracle (a sign flip on c, lines
and sectors swapped, a missing SM or blocks-per-SM factor, the y / z hit rates swapped)
and checks that these pins catch each one.
"""
import ctypes
import json
import math
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import brute_force
import oracle
from paper_2204_14242_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "model_7pt.json")
RTOL = 1e-12


def ev(x):
    """Evaluates a hand-derived closed form (numbers, + - * /, exp and log only)."""
    if isinstance(x, (int, float)):
        return float(x)
    return float(eval(x, {"__builtins__": {}}, {"exp": math.exp, "log": math.log}))


def gold():
    with open(GOLDEN) as f:
        return json.load(f)


def table1(g, hit):
    h = g["hardware"]
    hw = W.a100()
    assert (hw.sms, hw.clock_hz, hw.l1_bytes, hw.l2_bytes) == (h["sms"], h["clock_hz"], h["l1_bytes"], h["l2_bytes"])
    assert (hw.bw_l2, hw.bw_dram, hw.fp_peak) == (h["bw_l2"], h["bw_dram"], h["fp_peak"])
    hw.hit = tuple(tuple(ev(v) for v in row) for row in hit)
    return hw


def misaligned_store_copy():
    N = (128, 128, 128)
    st = W.dense_strides(N)
    src = W.Field(8, [W.Access(0, 0, 0, 0)], align=0, strides=st)
    dst = W.Field(8, [W.Access(0, 0, 0, 1)], align=8, strides=st)
    return W.Config(N=N, B=(32, 4, 1), fields=[src, dst], wave_blocks_override=8, name="copy_dst_plus_8")


def pin_failures(estimate):
    """Every pin of this file, checked against `estimate(configs, hw) -> list of dicts`;
    returns the failures (an empty list when all hold)."""
    g = gold()
    bad = []

    def close(what, got, want):
        if not (got == want or math.isclose(got, want, rel_tol=RTOL, abs_tol=0.0)):
            bad.append((what, got, want))

    s7 = g["stencil_7pt"]
    for name, case in s7["cases"].items():
        r = estimate([W.stencil_7pt_128()], table1(g, case["hit"]))[0]
        for k, v in s7["integers"].items():
            if r[k] != v:
                bad.append((name, k, r[k], v))
        for k, v in s7["oversubscription"].items():
            close((name, k), r[k], ev(v))
        for k, v in case["expect"].items():
            close((name, k), r[k], ev(v))
        if r["limiter"] != case["limiter"]:
            bad.append((name, "limiter", r["limiter"], case["limiter"]))
        # the L1 hit rate is recovered from the L2 <- L1 volume: R = (req - V) / (req - comp)
        close((name, "R_l1"), (58.0 - r["v_l2_load"]) / 28.0, ev(case["R"]["l1"]))
    m = g["misaligned_store_copy"]
    r = estimate([misaligned_store_copy()], table1(g, m["hit"]))[0]
    for k, v in m["integers"].items():
        if r[k] != v:
            bad.append(("misaligned", k, r[k], v))
    for k, v in m["oversubscription"].items():
        close(("misaligned", k), r[k], ev(v))
    for k, v in m["expect"].items():
        close(("misaligned", k), r[k], ev(v))
    if r["limiter"] != m["limiter"]:
        bad.append(("misaligned", "limiter", r["limiter"], m["limiter"]))
    return bad


def test_hand_reductions_agree():
    """The reduced fractions in the golden file are the products written out."""
    g = gold()
    for part in (g["stencil_7pt"], g["misaligned_store_copy"]):
        for k, v in part["oversubscription"].items():
            assert ev(v) == pytest.approx(ev(part["oversubscription_reduced"][k]), rel=1e-15)
    crafted = g["stencil_7pt"]["cases"]["crafted_halves"]
    # the crafted curves land on their stated hit rates at this case's oversubscription
    o = {k: ev(v) for k, v in g["stencil_7pt"]["oversubscription_reduced"].items()}
    for row, key, lev in ((0, "o_l1", "l1"), (1, "o_y", "y"), (2, "o_z", "z")):
        a, b, c = (ev(x) for x in crafted["hit"][row])
        assert a * math.exp(-b * math.exp(-c * o[key])) == pytest.approx(ev(crafted["R"][lev]), rel=1e-14)


def test_misaligned_store_copy_integers_by_brute_force():
    """The new integer inputs of the store terms, by the numpy brute force as well."""
    g = gold()["misaligned_store_copy"]["integers"]
    want = brute_force.count(misaligned_store_copy(), W.a100())
    for k, v in g.items():
        if k in want:
            assert want[k] == v, (k, want[k], v)


def test_model_terms_match_hand_derivations():
    assert pin_failures(oracle.estimate) == []


# ---- planted mistakes (in a copy of the oracle, compiled on the CPU) ---------------------

MUTANTS = {
    "sign of c": ("std::exp(-h[2] * O)", "std::exp(h[2] * O)"),
    "sectors for lines in the wave allocation": ("128.0 * (double)wll / (double)Weff",
                                                 "128.0 * (double)wls / (double)Weff"),
    "no SM factor in T_L1": ("(hw.clock * (double)hw.sms)", "(hw.clock)"),
    "store sectors for store lines in O_st": ("128.0 * (double)wsl / hw.l2", "128.0 * (double)wss / hw.l2"),
    "no blocks-per-SM factor in O_L1": ("(double)bll * (double)bpsm / hw.l1", "(double)bll / hw.l1"),
    "y and z hit rates swapped": ("r_y * (32.0 * (double)ovy) + r_z * (32.0 * (double)ovz)",
                                  "r_z * (32.0 * (double)ovy) + r_y * (32.0 * (double)ovz)"),
    "O_z from the y distance": ("(double)zdist * alloc_per_block", "(double)ydist * alloc_per_block"),
    "redundant stores not charged": ("(1.0 - r_st) * v_red_st", "(1.0 - r_st) * 0.0"),
}


def _variant_estimator(lib_path):
    lib = ctypes.CDLL(lib_path)
    P = ctypes.c_void_p
    lib.orc_estimate.argtypes = [ctypes.c_int, P, P, P, P, P, P, P, ctypes.c_int]
    lib.orc_estimate.restype = ctypes.c_int

    def estimate(configs, hw):
        cfg_i, cfg_d, fld_i, acc_i, hw_d = oracle.flatten(configs, hw)
        n = len(configs)
        oi = np.zeros((n, len(oracle.INT_KEYS)), np.int64)
        od = np.zeros((n, len(oracle.DBL_KEYS)), np.float64)
        fld_i, acc_i = np.ascontiguousarray(fld_i), np.ascontiguousarray(acc_i)
        assert lib.orc_estimate(n, cfg_i.ctypes.data, cfg_d.ctypes.data, fld_i.ctypes.data, acc_i.ctypes.data,
                                hw_d.ctypes.data, oi.ctypes.data, od.ctypes.data, 1) == 0
        out = []
        for i in range(n):
            d = {k: int(oi[i, j]) for j, k in enumerate(oracle.INT_KEYS)}
            d.update({k: float(od[i, j]) for j, k in enumerate(oracle.DBL_KEYS)})
            out.append(d)
        return out
    return estimate


def test_planted_mistakes_are_caught():
    src_dir = os.path.dirname(oracle.__file__)
    with open(os.path.join(src_dir, "oracle.cpp")) as f:
        src = f.read()
    tmp = tempfile.mkdtemp(prefix="oracle_mut_")
    try:
        shutil.copy(os.path.join(src_dir, "oracle.h"), tmp)
        procs = {}
        for i, (name, (old, new)) in enumerate(MUTANTS.items()):
            assert src.count(old) == 1, f"planting '{name}': the oracle text changed"
            cpp = os.path.join(tmp, f"m{i}.cpp")
            with open(cpp, "w") as f:
                f.write(src.replace(old, new))
            so = os.path.join(tmp, f"m{i}.so")
            procs[name] = (so, subprocess.Popen(["g++", "-std=c++17", "-O1", "-ffp-contract=off", "-fPIC", "-shared",
                                                 "-pthread", cpp, "-o", so]))
        for name, (so, p) in procs.items():
            assert p.wait() == 0, name
            assert pin_failures(_variant_estimator(so)), f"planted mistake not caught: {name}"
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
