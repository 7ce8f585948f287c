"""Host descriptor compiler (CPU): thread groups agree with the oracle, every address
the kernels can produce lies inside the bitmap the compiler sized for it, and the
validation rules reject what they should."""
import numpy as np
import pytest

import brute_force
import oracle
from paper_2204_14242_gb300 import binding as B
from paper_2204_14242_gb300 import workloads as W
from test_oracle_pins import random_tiny


def sample_configs():
    rng = W.SplitMix64(21)
    out = [(random_tiny(rng), W.Hardware(sms=rng.randint(1, 4), max_blocks_sm=2)) for _ in range(150)]
    out += [(c, W.a100()) for c in W.stencil_25pt_sweep(N=(96, 64, 48))[::37]]
    out += [(W.stencil_7pt_128(), W.a100())]
    return out


def test_thread_groups_match_the_oracle():
    for c, hw in sample_configs():
        info = B.ws_describe([c], hw)[0]
        o = oracle.estimate([c], hw)[0]
        assert info["status"] == o["status"] == 0
        assert info["wave_first"] == o["wave_first_block"]
        assert info["wave_blocks"] == o["wave_blocks"]
        assert info["y_dist"] == o["y_dist_blocks"]
        assert info["z_dist"] == o["z_dist_blocks"]
        assert info["blocks_per_sm"] == o["blocks_per_sm"]
        # y / z candidate ranges + predicates reproduce the brute-force block sets
        grp = brute_force.thread_groups(c, hw)
        g = info["grid"]
        ys = [b for b in range(info["y_lo"], info["y_hi"]) if (b // g[0]) % g[1] != g[1] - 1]
        assert ys == list(grp["y"])
        zs = [b for b in range(info["z_lo"], info["z_hi"]) if b not in set(ys)]
        assert zs == list(grp["z"])


def test_z_set_ends_before_the_y_set_ends():
    """The row walk gives the z set one slot per thread row: outside the last block row the
    y set removes [y_lo, y_hi) from the z blocks of a row, and z_hi <= y_hi (both sets are
    the wave shifted back, the z set by a whole slab), so only the z blocks before y_lo can
    remain.  Checked on random candidates, the sweeps and wave-size overrides: the single
    slot per row, read off the compiler's ranges, must give the y and z block sets that
    tests/brute_force.py enumerates on its own (wave shifted back by a block row / slab,
    blocks outside the grid dropped, minus the wave and, for z, minus the y set)."""
    rng = W.SplitMix64(23)
    cases = [(random_tiny(rng), W.Hardware(sms=rng.randint(1, 6), max_blocks_sm=rng.randint(1, 4)))
             for _ in range(300)]
    cases += [(c, W.a100()) for c in W.stencil_25pt_sweep(N=(96, 64, 48))[::5]]
    for c, hw in cases:
        info = B.ws_describe([c], hw)[0]
        assert info["status"] == 0
        if info["y_hi"] > info["y_lo"] and info["z_hi"] > info["z_lo"]:
            assert info["z_hi"] <= info["y_hi"]
        g = info["grid"]
        grp = brute_force.thread_groups(c, hw)          # independent enumeration of the sets
        last_row = lambda b: (b // g[0]) % g[1] == g[1] - 1
        ys = [b for b in range(info["y_lo"], info["y_hi"]) if not last_row(b)]
        assert ys == [int(b) for b in grp["y"]]
        # the single-slot reading: z blocks of other rows lie before y_lo (or the y set is empty)
        single = [b for b in range(info["z_lo"], info["z_hi"])
                  if last_row(b) or info["y_hi"] <= info["y_lo"] or b < info["y_lo"]]
        assert single == [int(b) for b in grp["z"]]


def test_bitmaps_contain_every_sector():
    for c, hw in sample_configs():
        finfo = B.ws_describe_fields(c, hw)
        grp = brute_force.thread_groups(c, hw)
        g = grp["grid"]
        for fi, f in enumerate(c.fields):
            loads = {(a.dx, a.dy, a.dz, a.dc) for a in f.accesses if not a.is_store}
            stores = {(a.dx, a.dy, a.dz, a.dc) for a in f.accesses if a.is_store}
            for lv, groups in ((0, ("rep",)), (1, ("wave", "y", "z"))):
                lo = finfo[fi]["lo_sector"][lv]
                hi = lo + 32 * finfo[fi]["words"][lv]
                assert lo % 32 == 0 and finfo[fi]["words"][lv] % 4 == 0
                for name in groups:
                    p, kv, warp, lane = brute_force.threads(c, g, grp[name])
                    for offs in (loads, stores):
                        for o in brute_force.folded(c, offs):
                            m = brute_force.needed(c, offs, o, kv)
                            sec = np.floor_divide(brute_force.addresses(f, p, o)[m], 32)
                            if sec.size:
                                assert sec.min() >= lo and sec.max() < hi, (c, fi, lv, name)


def test_validation_rules():
    N = (64, 64, 64)
    ok = W.Config(N=N, B=(32, 4, 1), fields=W.copy_fields(N, W.star_offsets(1)))
    bad = [
        W.Config(N=N, B=(64, 32, 1), fields=ok.fields),                            # 2048 threads
        W.Config(N=N, B=(1, 1, 128), fields=ok.fields),                            # bz > 64
        W.Config(N=(0, 4, 4), B=(32, 1, 1), fields=ok.fields),                     # empty domain
        W.Config(N=(1 << 21, 4, 4), B=(32, 1, 1), fields=ok.fields),               # N > 2^20
        W.Config(N=N, B=(32, 1, 1), fields=ok.fields, fold_axis=0, fold=2),        # fold without axis
        W.Config(N=N, B=(32, 1, 1), fields=ok.fields, fold_axis=1, fold=17),       # fold > 16
        W.Config(N=N, B=(1024, 1, 1), fields=ok.fields, regs_per_thread=255),      # no block fits
        W.Config(N=N, B=(32, 1, 1), fields=[W.Field(8, [W.Access(0, 0, 0)], strides=(1 << 41, 1, 1))]),
        W.Config(N=N, B=(32, 1, 1), fields=[W.Field(0, [W.Access(0, 0, 0)], strides=(1, 64, 4096))]),
    ]
    info = B.ws_describe([ok] + bad, W.a100())
    assert info[0]["status"] == 0
    assert all(s == B.WS_EINVAL for s in info["status"][1:]), list(info["status"])
    # the oracle rejects the first five (its own, looser, rules) as well
    for o in oracle.estimate(bad[:3] + bad[4:5] + bad[6:7], W.a100()):
        assert o["status"] == -1


def test_folded_instruction_counts():
    N = (64, 64, 64)
    for r in (1, 2, 4):
        for axis, f in W.FOLD_VARIANTS:
            c = W.Config(N=N, B=(32, 2, 2), fields=W.copy_fields(N, W.star_offsets(r)), fold_axis=axis, fold=f)
            info = B.ws_describe([c], W.a100())[0]
            # a star of radius r folded f times along y or z: the fold-axis line grows to
            # 2r + f points, the 4r points off that axis are repeated f times
            assert info["folded_loads"] == 2 * r + f + 4 * r * f
            assert info["folded_stores"] == f


@pytest.mark.timeout(120)
def test_plan_dry_run_host_pipeline():
    """The host half of plan creation (compile, list sharing, groups, passes, items) on
    linear and multi-dimensional batches, without a device."""
    import dataclasses
    from test_gpu_parity import random_uniform_tiny, edge_configs
    B.load()
    hw = W.a100()
    sweep = W.stencil_25pt_sweep(N=(160, 128, 96))
    one = B.ws_plan_dry_run(sweep, hw)
    two = B.ws_plan_dry_run(sweep + sweep, hw)
    assert one["candidates_ok"] == len(sweep) and one["fields"] == 2 * len(sweep) and one["passes"] == 1
    # candidates sharing a field and a folding share its lists on the device
    assert two["access_entries"] == one["access_entries"] and two["fields"] == 2 * one["fields"]
    assert one["scratch_bytes"] == one["bitmap_bytes"]
    small = B.ws_plan_dry_run(sweep, hw, scratch_bytes=one["bitmap_bytes"] // 7)
    assert small["passes"] > 1 and small["count_items"] == one["count_items"]
    seg = B.ws_plan_dry_run(sweep, hw, tuning={"walk": B.WS_WALK_SEGMENT})
    adr = B.ws_plan_dry_run(sweep, hw, tuning={"walk": B.WS_WALK_ADDRESS})
    assert one["row_items"] > 0 and seg["row_items"] == 0 and adr["row_items"] == 0
    assert seg["enum_items"] == adr["enum_items"] > one["enum_items"]
    # multi-dimensional candidates: a block and a wave descriptor per field; the wave
    # lists (virtual strides of the candidate) are never shared
    md = lambda c: dataclasses.replace(c, address_mode=B.WS_ADDR_MULTIDIM)
    rng = W.SplitMix64(808)
    batch = [random_tiny(rng) for _ in range(150)] + [random_uniform_tiny(rng) for _ in range(150)] + edge_configs()
    lin = B.ws_plan_dry_run(batch, W.Hardware(sms=3, max_blocks_sm=2))
    mdr = B.ws_plan_dry_run([md(c) for c in batch], W.Hardware(sms=3, max_blocks_sm=2))
    assert mdr["candidates_ok"] == lin["candidates_ok"] and mdr["fields"] == 2 * lin["fields"]
    m1 = B.ws_plan_dry_run([md(c) for c in sweep[:40]], hw)
    m2 = B.ws_plan_dry_run([md(c) for c in sweep[:40]] * 2, hw)
    assert m2["access_entries"] > m1["access_entries"]
