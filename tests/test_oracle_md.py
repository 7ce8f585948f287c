"""Pins of the oracle's multi-dimensional address space (Sec. 4.4.1).

In that space a wave-level sector is the tuple (innermost coordinate in bytes // 32,
y, z): two tuples differ when any coordinate differs, the base alignment is not part
of it, and a cache line that wraps around to the next row is counted at both row
ends.  The representative block keeps linear addresses.  The pins: a numpy brute
force written from that definition, the 7-point case derived by hand, invariance under
any alignment shift, and the paper's remark that the difference to linear addresses is
small on large grids.
"""
import dataclasses

import pytest

import brute_force
import oracle
from paper_2204_14242_gb300 import workloads as W
from test_oracle_pins import random_tiny, tiny_hw

INT = ["lups_block", "lups_wave", "l1_req_sectors", "l1_bank_cycles", "l1_store_sectors",
       "blk_load_sectors", "blk_load_lines", "blk_store_sectors", "blk_store_lines",
       "wave_load_sectors", "wave_load_lines", "wave_store_sectors", "wave_store_lines",
       "wave_store_req_sectors", "ov_y", "ov_z", "y_lines", "z_lines"]


def md(c):
    return dataclasses.replace(c, address_mode=1)


def test_md_oracle_matches_brute_force_on_tiny_grids():
    rng = W.SplitMix64(31)
    for i in range(120):
        c = md(random_tiny(rng))
        hw = tiny_hw(rng.randint(1, 4))
        want = brute_force.count(c, hw)
        got = oracle.estimate([c], hw)[0]
        assert got["status"] == 0
        for k in INT:
            assert got[k] == want[k], (i, k, got[k], want[k], c)


def test_md_7pt_wave_closed_form():
    """7-point star, fp64, 128^3, block 32x4x1, wave of 8 blocks = x 0..127, y 64..71, z 64.
    Linear addresses give 832 wave sectors because the x-1 / x+1 neighbours of a row end
    fall into the adjacent rows, which the wave reads anyway.  In the multi-dimensional
    space those neighbours are their own sectors at x = -1 and x = 128 (innermost byte
    -8 -> sector -1, byte 1024 -> sector 32): one extra sector and one extra line at both
    ends of each of the 8 rows that carry the x accesses (z = 64, y = 64..71): 848 sectors
    and 208 + 16 = 224 lines.  Stores (offset 0) and the overlaps with the y / z sets
    (whose rows are interior) do not change: 256 / 64, ov_y 64, ov_z 480.  The block
    keeps linear addresses (120 sectors, 36 lines)."""
    lin = oracle.estimate([W.stencil_7pt_128()], W.a100())[0]
    got = oracle.estimate([md(W.stencil_7pt_128())], W.a100())[0]
    assert lin["wave_load_sectors"] == 832 and lin["wave_load_lines"] == 208
    assert got["wave_load_sectors"] == 848 and got["wave_load_lines"] == 224
    assert got["wave_store_sectors"] == 256 and got["wave_store_lines"] == 64
    assert got["ov_y"] == 64 and got["ov_z"] == 480
    assert got["blk_load_sectors"] == 120 and got["blk_load_lines"] == 36
    for k in ("lups_block", "lups_wave", "l1_req_sectors", "l1_bank_cycles", "blk_store_sectors"):
        assert got[k] == lin[k], k


def test_md_counts_ignore_the_alignment():
    rng = W.SplitMix64(32)
    hw = tiny_hw(2)
    wave_keys = ["wave_load_sectors", "wave_load_lines", "wave_store_sectors", "wave_store_lines",
                 "wave_store_req_sectors", "ov_y", "ov_z", "y_lines", "z_lines"]
    for i in range(40):
        c = md(random_tiny(rng))
        shifted = dataclasses.replace(
            c, fields=[dataclasses.replace(f, align=f.align + 1 + 37 * j) for j, f in enumerate(c.fields)])
        a, b = oracle.estimate([c, shifted], hw)
        for k in wave_keys:
            assert a[k] == b[k], (i, k)


def test_md_differs_little_from_linear_on_a_wide_grid():
    """25-point star on 640-wide fp64 rows: the only difference is one sector at each
    end of a row that carries the x halo, about 2 of 160 sectors per row."""
    N = (640, 48, 40)
    c = W.Config(N=N, B=(64, 2, 1), fields=W.copy_fields(N, W.star_offsets(4)), flops_per_lup=25.0)
    hw = W.Hardware(sms=8)
    lin, got = oracle.estimate([c, md(c)], hw)
    d = (got["wave_load_sectors"] - lin["wave_load_sectors"]) / lin["wave_load_sectors"]
    assert 0 <= d < 2.0 / 160 + 1e-9, d
    assert got["wave_store_sectors"] == lin["wave_store_sectors"]
