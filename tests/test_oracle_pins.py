"""Pins of the CPU oracle against things other than itself (all CPU, no GPU).

* brute force: the numpy meshgrid + unique evaluation of Sec. 4.2 on tiny grids;
* closed forms: 7-point block and wave (derived from the geometry below), the
  wave-depth law of Sec. 5.7, the bank-conflict examples of Sec. 4.2, a streaming
  copy, the D3Q15 240 B/LUP of Sec. 5.3;
* invariants: inclusion between levels, sector/line bounds, monotonicity in the
  stencil radius, invariance under a one-line shift of the alignment;
* model special cases fixed by the paper (Sec. 4.5, Sec. 5.5, Sec. 2).
"""
import json
import math
import os

import numpy as np
import pytest

import brute_force
import oracle
from paper_2204_14242_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
INT_KEYS = [k for k in oracle.INT_KEYS if k not in ("status", "limiter")]


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def tiny_hw(sms=3):
    return W.Hardware(sms=sms, max_blocks_sm=2)


def random_tiny(rng: W.SplitMix64):
    """Tiny random candidate: N <= 14^3, <= 64 threads, any alignment, odd layouts."""
    N = (rng.randint(1, 14), rng.randint(1, 12), rng.randint(1, 10))
    shapes = [(bx, by, bz) for bx in (1, 2, 3, 4, 8, 16, 32) for by in (1, 2, 3, 4) for bz in (1, 2, 4)
              if bx * by * bz <= 64]
    B = rng.choice(shapes)
    axis, f = rng.choice([(0, 1), (1, 2), (1, 3), (2, 2), (2, 4), (1, 4)])
    fields = []
    for _ in range(rng.randint(1, 3)):
        esize = rng.choice((1, 2, 4, 8, 16))
        kind = rng.randint(0, 3)
        if kind == 0:
            st = (1, N[0], N[0] * N[1])
        elif kind == 1:                      # padded rows
            px = N[0] + rng.randint(1, 9)
            st = (1, px, px * (N[1] + rng.randint(0, 3)))
        elif kind == 2:                      # x not contiguous (AoS-like / transposed)
            st = (rng.randint(2, 5), rng.randint(1, 3) * 100, 977)
        else:                                # negative y stride
            st = (1, -N[0], N[0] * N[1] * 3)
        accs = set()
        r = rng.randint(0, 2)
        for _ in range(rng.randint(1, 7)):
            accs.add(W.Access(rng.randint(-r, r), rng.randint(-r, r), rng.randint(-r, r),
                              0, rng.randint(0, 2) if kind == 2 else 0))
        if rng.randint(0, 2):
            accs.add(W.Access(0, 0, 0, 1, 0))
            if rng.randint(0, 3) == 0:
                accs.add(W.Access(1, 0, 0, 1, 0))
        fields.append(W.Field(esize, sorted(accs, key=lambda a: (a.dx, a.dy, a.dz, a.is_store, a.dc)),
                              align=rng.randint(-70, 70), strides=st, const_off=rng.randint(-5, 5)))
    return W.Config(N=N, B=B, fields=fields, fold_axis=axis, fold=f,
                    wave_blocks_override=rng.choice((0, 1, 2, 3, 5)), flops_per_lup=3.0)


def test_oracle_matches_brute_force_on_tiny_grids():
    rng = W.SplitMix64(7)
    for i in range(120):
        c = random_tiny(rng)
        hw = tiny_hw(rng.randint(1, 4))
        want = brute_force.count(c, hw)
        got = oracle.estimate([c], hw)[0]
        assert got["status"] == 0
        for k, v in want.items():
            assert got[k] == v, (i, k, got[k], v, c)


def test_oracle_matches_brute_force_on_paper_like_shapes():
    """Real block shapes and the 25-point star on a domain small enough to brute-force."""
    hw = W.Hardware(sms=4)
    N = (48, 24, 40)
    cfgs = W.stencil_25pt_sweep(N=N)
    rng = W.SplitMix64(11)
    for _ in range(12):
        c = rng.choice(cfgs)
        want = brute_force.count(c, hw)
        got = oracle.estimate([c], hw)[0]
        for k, v in want.items():
            assert got[k] == v, (c.name, k, got[k], v)


def test_7pt_block_and_wave_closed_form():
    """3D 7-point star, fp64, 128^3, block 32x4x1, wave of 8 blocks.

    Geometry: a row is 128 doubles = 1024 B = 32 sectors; the middle block covers
    x 64..95, y 64..67, z 64 (bytes 512..767 of each row = sectors 16..23).
      block loads: rows 64..67 of plane 64 need sectors 15..24 (x-1 / x+1 spill one
      sector each way) = 4 x 10; rows 63 and 68 (y-+1) 8 each; planes 63 and 65 (z-+1)
      4 rows x 8 each: 40 + 16 + 64 = 120 sectors; lines: 4 x 4 + 2 x 2 + 2 x 4 x 2 = 36.
      requests per warp (one row): 8 + 9 + 9 + 4 x 8 = 58, four warps = 232.
      every half warp instruction touches 16 consecutive doubles: 1 cycle, 8 instructions,
      8 half warps: 64 cycles.
    The wave holds blocks 8256..8263 = x 0..127, y 64..71, z 64 (whole rows): plane 64
    rows 63..72 (10 x 32) + planes 63, 65 rows 64..71 (2 x 8 x 32) = 832 sectors, 208 lines.
    y set = the previous block row (y 60..63): its footprint shares rows 63 and 64 of
    plane 64 with the wave: ov_y = 64.  z set = the wave one plane back: it shares plane 63
    rows 64..71 and plane 64 rows 64..71 (512 sectors), of which row 64 of plane 64 is
    already in the y footprint: ov_z = 480.
    """
    r = oracle.estimate([W.stencil_7pt_128()], W.a100())[0]
    want = dict(lups_block=128, lups_wave=1024, l1_req_sectors=232, l1_bank_cycles=64,
                l1_store_sectors=32, blk_load_sectors=120, blk_load_lines=36, blk_store_sectors=32,
                blk_store_lines=8, wave_load_sectors=832, wave_load_lines=208,
                wave_store_sectors=256, wave_store_lines=64, wave_store_req_sectors=256,
                ov_y=64, ov_z=480, wave_blocks=8, wave_first_block=8256, y_dist_blocks=4,
                z_dist_blocks=128)
    for k, v in want.items():
        assert r[k] == v, (k, r[k], v)
    assert r["v_l1"] == 58.0
    # capacity model off: compulsory volumes only, every overlap hits
    hw = W.a100()
    hw.capacity_model = 0
    r0 = oracle.estimate([W.stencil_7pt_128()], hw)[0]
    assert r0["v_l2_load"] == 30.0
    assert r0["v_dram_load"] == 32.0 * (832 - 64 - 480) / 1024   # 9 B/LUP
    assert r0["v_dram_store"] == 8.0


@pytest.mark.parametrize("depth,B,fold", [(1, (32, 1, 1), 1), (2, (32, 1, 2), 1), (4, (32, 1, 4), 1),
                                          (8, (32, 1, 8), 1), (32, (32, 1, 32), 1),
                                          (8, (32, 1, 4), 2), (32, (32, 1, 8), 4),
                                          (16, (32, 1, 16), 1)])
def test_wave_depth_law(depth, B, fold):
    """Sec. 5.7: a wave of d whole xy layers loads (d+8)/d values per LUP for the
    range-4 star (no z reuse): 72/40/24/16/10 B/LUP for d = 1/2/4/8/32."""
    g = golden("wave_depth_law.json")
    N = (32, 32, 256)
    fields = W.copy_fields(N, W.star_offsets(4))
    # one slab of blocks = one wave (32 blocks of 32 x 1 x bz threads)
    c = W.Config(N=N, B=B, fields=fields, fold_axis=2 if fold > 1 else 0, fold=fold,
                 wave_blocks_override=32)
    r = oracle.estimate([c], W.a100())[0]
    assert r["lups_wave"] == depth * 32 * 32
    v = 32.0 * r["wave_load_sectors"] / r["lups_wave"]
    assert r["wave_load_sectors"] == (depth + 8) * 32 * 32 * 8 // 32
    if str(depth) in g["dram_load_bytes_per_lup"]:
        assert v == g["dram_load_bytes_per_lup"][str(depth)]
        num, den = g["values_loaded_per_layer"][str(depth)]
        assert v == 8.0 * num / den
    else:
        assert v == 8.0 * (depth + 8) / depth


@pytest.mark.parametrize("stride", [1, 2, 16])
def test_bank_conflict_examples(stride):
    """Sec. 4.2: doubles at A[tid], B[2 tid], D[16 tid] take 1 / 2 / 16 cycles per half warp."""
    g = golden("bank_conflicts.json")
    N = (64, 4, 4)
    f = W.Field(8, [W.Access(0, 0, 0, 0)], strides=(stride, 64 * stride, 256 * stride))
    c = W.Config(N=N, B=(32, 1, 1), fields=[f])
    r = oracle.estimate([c], W.a100())[0]
    half_warps = 2
    assert r["l1_bank_cycles"] == g["cycles_per_half_warp_by_stride"][str(stride)] * half_warps


@pytest.mark.parametrize("B", [(16, 2, 1), (16, 4, 8), (32, 2, 2), (64, 1, 4), (256, 4, 1)])
def test_contiguous_half_warps_take_one_wavefront(B):
    """Sec. 5.4: a block at least 16 wide loads one contiguous block per half warp."""
    g = golden("bank_conflicts.json")
    N = (256, 64, 64)
    c = W.Config(N=N, B=B, fields=W.copy_fields(N, W.star_offsets(2)))
    r = oracle.estimate([c], W.a100())[0]
    T = B[0] * B[1] * B[2]
    instr = 13 + 1
    assert r["l1_bank_cycles"] == g["contiguous_width_16_or_more"]["cycles_per_half_warp"] * (T // 16) * instr


def test_narrow_blocks_increase_bank_cycles():
    """Sec. 5.4: each halving of the block width below 16 adds bank conflicts."""
    N = (256, 256, 64)
    prev = None
    for B in [(16, 8, 1), (8, 16, 1), (4, 32, 1), (2, 64, 1), (1, 128, 1)]:
        c = W.Config(N=N, B=B, fields=W.copy_fields(N, W.star_offsets(1)))
        r = oracle.estimate([c], W.a100())[0]
        if prev is not None:
            assert r["l1_bank_cycles"] > prev
        prev = r["l1_bank_cycles"]


@pytest.mark.parametrize("esize,B", [(8, (32, 4, 2)), (8, (4, 8, 8)), (4, (8, 8, 2)), (4, (64, 2, 1)),
                                     (8, (128, 1, 8))])
def test_streaming_copy_moves_esize_bytes_everywhere(esize, B):
    """dst[0] = src[0], aligned, block width a whole number of sectors: every level moves
    exactly elem_bytes per LUP for the load and for the store."""
    N = (256, 64, 64)
    c = W.Config(N=N, B=B, fields=W.copy_fields(N, [(0, 0, 0)], esize=esize))
    r = oracle.estimate([c], W.a100())[0]
    lb, lw = r["lups_block"], r["lups_wave"]
    assert 32 * r["l1_req_sectors"] == esize * lb
    assert 32 * r["blk_load_sectors"] == esize * lb
    assert 32 * r["l1_store_sectors"] == esize * lb
    assert 32 * r["wave_load_sectors"] == esize * lw
    assert 32 * r["wave_store_sectors"] == esize * lw
    assert r["wave_store_req_sectors"] == r["wave_store_sectors"]


def contiguous_sectors(first_byte, nbytes):
    return (first_byte + nbytes - 1) // 32 - first_byte // 32 + 1


def test_d3q15_streaming_volume():
    """Sec. 5.3: the D3Q15 pull kernel streams 2 x 15 x 8 = 240 B/LUP.

    The wave below covers four whole planes, so each array's footprint is one contiguous
    run of 4096 doubles shifted by -c_i: its sectors follow in closed form."""
    gold = golden("streaming_volumes.json")["lbm_d3q15"]["bytes_per_lup"]
    N = (32, 32, 64)
    st = W.dense_strides(N)
    fields = [W.Field(8, [W.Access(-c[0], -c[1], -c[2], 0), W.Access(0, 0, 0, 1)], strides=st)
              for c in W.D3Q15]
    c = W.Config(N=N, B=(32, 1, 4), fields=fields, wave_blocks_override=32)
    r = oracle.estimate([c], W.a100())[0]
    n = 4 * 32 * 32
    z0 = r["wave_first_block"] // 32 * 4
    want = 0
    for cc in W.D3Q15:
        lin = z0 * 1024 - (cc[0] + 32 * cc[1] + 1024 * cc[2])
        want += contiguous_sectors(8 * lin, 8 * n)
    assert r["wave_load_sectors"] == want
    assert r["wave_store_sectors"] == 15 * n // 4
    v = 32.0 * (r["wave_load_sectors"] + r["wave_store_sectors"]) / r["lups_wave"]
    assert gold <= v <= gold * 1.01


def test_invariants_random_and_radius_monotone():
    rng = W.SplitMix64(3)
    hw = W.Hardware(sms=6)
    for _ in range(25):
        N = (rng.randint(40, 90), rng.randint(20, 60), rng.randint(20, 50))
        B = rng.choice(W.block_shapes())
        axis, f = rng.choice(W.FOLD_VARIANTS)
        esize = rng.choice((4, 8))
        prev = None
        for r_ in (1, 2, 3):
            c = W.Config(N=N, B=B, fields=W.copy_fields(N, W.star_offsets(r_), esize=esize),
                         fold_axis=axis, fold=f)
            o = oracle.estimate([c], hw)[0]
            for lv in ("blk_load", "wave_load", "wave_store", "blk_store"):
                s, l = o[lv + "_sectors"], o[lv + "_lines"]
                assert l <= s <= 4 * l
            assert o["l1_req_sectors"] >= o["blk_load_sectors"]
            assert o["wave_load_sectors"] >= o["blk_load_sectors"]
            assert o["ov_y"] + o["ov_z"] <= o["wave_load_sectors"]
            assert o["wave_store_req_sectors"] >= o["wave_store_sectors"]
            assert 32 * o["wave_store_sectors"] >= esize * o["lups_wave"]
            if prev is not None:
                for k in ("l1_req_sectors", "l1_bank_cycles", "blk_load_sectors", "blk_load_lines",
                          "wave_load_sectors", "wave_load_lines", "ov_y", "y_lines", "z_lines"):
                    assert o[k] >= prev[k], k
                for k in ("lups_block", "lups_wave", "wave_store_sectors", "l1_store_sectors"):
                    assert o[k] == prev[k], k
            prev = o


def test_one_line_alignment_shift_changes_nothing():
    rng = W.SplitMix64(5)
    hw = W.Hardware(sms=5)
    for _ in range(10):
        c = random_tiny(rng)
        base = oracle.estimate([c], hw)[0]
        for f in c.fields:
            f.align += 128 * rng.randint(-3, 3)
        moved = oracle.estimate([c], hw)[0]
        for k in INT_KEYS:
            assert moved[k] == base[k], k


def test_model_special_cases_fixed_by_the_paper():
    """Sec. 4.5 / 5.5: with R_hit = 1 the L2->L1 volume is the compulsory one; with
    R_hit = 0 it is the whole L1 request volume (upper bound); in between it is linear
    in R_hit.  Sec. 2: the prediction is the slowest limiter."""
    c = W.stencil_25pt_sweep(variants=[(0, 1)])[40]
    base = W.a100()
    r = {}
    for name, hit in (("one", (1.0, 0.0, 0.0)), ("zero", (0.0, 0.0, 0.0)), ("half", (0.5, 0.0, 0.0))):
        hw = W.a100()
        hw.hit = (hit,) * 4
        r[name] = oracle.estimate([c], hw)[0]
    off = W.a100()
    off.capacity_model = 0
    r["off"] = oracle.estimate([c], off)[0]
    o = r["one"]
    comp = 32.0 * o["blk_load_sectors"] / o["lups_block"]
    req = 32.0 * o["l1_req_sectors"] / o["lups_block"]
    assert o["v_l2_load"] == comp
    assert r["off"]["v_l2_load"] == comp
    assert r["zero"]["v_l2_load"] == req
    assert math.isclose(r["half"]["v_l2_load"], 0.5 * (comp + req), rel_tol=1e-15)
    # overlaps: all hit (R = 1) vs none (R = 0); redundant stores: none miss vs all miss
    lw = o["lups_wave"]
    assert math.isclose(o["v_dram_load"], 32.0 * (o["wave_load_sectors"] - o["ov_y"] - o["ov_z"]) / lw,
                        rel_tol=1e-15)
    z = r["zero"]
    red = 32.0 * (z["wave_store_req_sectors"] - z["wave_store_sectors"]) / lw
    assert math.isclose(z["v_dram_load"], 32.0 * z["wave_load_sectors"] / lw + red, rel_tol=1e-15)
    for x in r.values():
        ts = [x["t_l1"], x["t_l2"], x["t_dram"], x["t_fp"]]
        assert x["t_pred"] == max(ts) and ts[x["limiter"]] == max(ts)
        assert x["glups"] == 1e-9 / x["t_pred"]
    # a DRAM-bound candidate stops being DRAM-bound when DRAM gets very fast
    fast = W.a100()
    fast.bw_dram = 1e18
    assert oracle.estimate([c], fast)[0]["limiter"] != 2


def test_fp_is_never_the_limiter_of_the_25pt_stencil():
    """Sec. 4.1 / 5.2: 25 flops per LUP against >= 16 B/LUP stays below the machine balance."""
    gold = golden("streaming_volumes.json")["arithmetic_intensity"]
    hw = W.a100()
    assert math.isclose(hw.fp_peak / hw.bw_dram, gold["machine_balance"], rel_tol=1e-12)
    cfgs = W.stencil_25pt_sweep(N=(160, 128, 128))
    rng = W.SplitMix64(1)
    sample = [rng.choice(cfgs) for _ in range(12)]
    for o in oracle.estimate(sample, hw, threads=4):
        assert o["limiter"] != 3
        assert o["t_fp"] < o["t_dram"]


def test_rank_is_stable_and_quantised():
    t = [3e-12, 1e-12, 2e-12, 1e-12, float("inf"), 2e-12 * (1 + 2.0 ** -45), float("nan")]
    order = oracle.rank(t)
    assert list(order) == [1, 3, 2, 5, 0, 4, 6]
    assert oracle.rank_key(1.0 + 2.0 ** -45) == 1.0
    assert oracle.rank_key(1.0 + 2.0 ** -39) == 1.0 + 2.0 ** -39


def test_malformed_candidates_get_an_error_status():
    N = (64, 64, 64)
    bad = [W.Config(N=N, B=(64, 32, 1), fields=W.copy_fields(N, [(0, 0, 0)])),      # 2048 threads
           W.Config(N=N, B=(1, 1, 128), fields=W.copy_fields(N, [(0, 0, 0)])),      # bz > 64
           W.Config(N=(0, 4, 4), B=(32, 1, 1), fields=W.copy_fields(N, [(0, 0, 0)])),
           W.Config(N=N, B=(32, 1, 1), fields=W.copy_fields(N, [(0, 0, 0)]), fold_axis=0, fold=2),
           W.Config(N=N, B=(1024, 1, 1), fields=W.copy_fields(N, [(0, 0, 0)]), regs_per_thread=255)]
    for o in oracle.estimate(bad, W.a100()):
        assert o["status"] == -1 and o["t_pred"] == float("inf")
