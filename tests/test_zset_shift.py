"""The z set as the wave moved back one block slab (Sec. 4.5 layer sets), on the oracle.

The z set is the wave's blocks shifted back by one slab of blocks (the reading of the layer
sets used throughout), minus the wave and the y set.  When it is the whole shifted wave (the
wave lies beyond the first slab, spans at most one slab, ends before the y set begins, and
all its points lie inside the domain in z), every thread of the z set has the same valid
points as its wave twin moved by B_z * f_z rows in z and issues the same accesses, so each
field's z-set addresses are its wave addresses less esize * stride_z * B_z * f_z bytes.  A
move by a multiple of 128 bytes maps lines to lines: the z set then has exactly the wave's
line count, which the GPU path uses instead of enumerating the whole z set.  These tests
check that consequence on the CPU oracle, which enumerates the z set point by point, and that
a move off the 128-byte grid does change the count (so the condition is not vacuous).
"""
import pytest

import oracle
from paper_2204_14242_gb300 import workloads as W


def ceil_div(a, b):
    return -(-a // b)


def shifted_wave(c: W.Config, hw: W.Hardware) -> bool:
    """True when the z set is the whole wave moved back one block slab (block ranges as the
    representative wave and the layer sets define them)."""
    fy = c.fold if c.fold_axis == 1 else 1
    fz = c.fold if c.fold_axis == 2 else 1
    g = (ceil_div(c.N[0], c.B[0]), ceil_div(c.N[1], c.B[1] * fy), ceil_div(c.N[2], c.B[2] * fz))
    total = g[0] * g[1] * g[2]
    T = c.B[0] * c.B[1] * c.B[2]
    bpsm = min(hw.max_blocks_sm, hw.max_threads_sm // (32 * ceil_div(T, 32)))
    wave = c.wave_blocks_override or hw.sms * bpsm
    weff = min(wave, total)
    rep = g[0] // 2 + g[0] * (g[1] // 2 + g[1] * (g[2] // 2))
    s = min(wave * (rep // wave), total - weff)
    slab = g[0] * g[1]
    y_lo, y_hi = max(0, s - g[0]), min(s, s + weff - g[0])
    if y_hi <= y_lo or g[1] == 1:
        y_lo = y_hi = 0
    z_lo, z_hi = max(0, s - slab), min(s, s + weff - slab)
    if z_hi <= z_lo:
        return False
    inside = ((s + weff - 1) // slab + 1) * c.B[2] * fz <= c.N[2]
    return (s >= slab and weff <= slab and z_lo == s - slab and z_hi == s + weff - slab
            and (y_hi <= y_lo or z_hi <= y_lo) and inside)


def move_bytes(c: W.Config, f: W.Field) -> int:
    fz = c.fold if c.fold_axis == 2 else 1
    st = f.strides if f.strides is not None else (1, c.N[0], c.N[0] * c.N[1])
    return f.elem_bytes * st[2] * c.B[2] * fz


def candidates(seed, n, on_grid):
    """Small stencils whose z set is the shifted wave; fields moved by a multiple of 128 bytes
    (on_grid) or by a multiple of 8 bytes that is not one of 128."""
    rng = W.SplitMix64(seed)
    out = []
    while len(out) < n:
        B = rng.choice([(4, 2, 1), (8, 1, 2), (2, 2, 2), (4, 4, 1), (8, 2, 1), (4, 1, 4)])
        axis, f = rng.choice([(0, 1), (1, 2), (2, 2), (1, 4)])
        N = (rng.randint(5, 16), rng.randint(4, 12), rng.randint(6, 24))
        fields = []
        for _ in range(rng.randint(1, 3)):
            esize = rng.choice((4, 8))
            r = rng.randint(1, 2)
            accs = {W.Access(rng.randint(-r, r), rng.randint(-r, r), rng.randint(-r, r), 0, 0)
                    for _ in range(rng.randint(1, 6))}
            accs.add(W.Access(0, 0, 0, 1, 0))
            pitch = N[0] + rng.randint(0, 5)
            plane = pitch * (N[1] + rng.randint(0, 3))
            fz = f if axis == 2 else 1
            step = esize * B[2] * fz
            # round the plane up so that esize * plane * B2 * fz is (or is not) a multiple of 128
            while (step * plane) % 128 != 0 if on_grid else (step * plane) % 128 == 0:
                plane += 1
            fields.append(W.Field(esize, sorted(accs, key=lambda a: (a.dx, a.dy, a.dz, a.is_store)),
                                  align=rng.randint(-40, 40), strides=(1, pitch, plane)))
        c = W.Config(N=N, B=B, fields=fields, fold_axis=axis, fold=f,
                     wave_blocks_override=rng.choice((1, 2, 3, 4)), flops_per_lup=1.0)
        if shifted_wave(c, W.Hardware(sms=3, max_blocks_sm=2)):
            out.append(c)
    return out


def test_shifted_z_set_has_the_wave_line_count():
    hw = W.Hardware(sms=3, max_blocks_sm=2)
    cfgs = candidates(2027, 150, on_grid=True)
    assert all(move_bytes(c, f) % 128 == 0 for c in cfgs for f in c.fields)
    for c, r in zip(cfgs, oracle.estimate(cfgs, hw)):
        assert r["status"] == 0
        assert r["z_lines"] == r["wave_load_lines"], (c, r["z_lines"], r["wave_load_lines"])


def test_a_move_off_the_line_grid_changes_the_count():
    hw = W.Hardware(sms=3, max_blocks_sm=2)
    cfgs = candidates(2028, 150, on_grid=False)
    res = oracle.estimate(cfgs, hw)
    assert all(r["status"] == 0 for r in res)
    assert sum(r["z_lines"] != r["wave_load_lines"] for r in res) > 0


@pytest.mark.gpu
def test_gpu_matches_the_oracle_on_shifted_z_sets():
    """The GPU path takes the line count of a shifted z set from the wave and clips its
    ranges to the wave's address range; both kinds of candidates, through the C ABI, must give
    the oracle's results exactly (fp64 values within 1e-12)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import numpy as np
    from paper_2204_14242_gb300 import binding as B
    hw = W.Hardware(sms=3, max_blocks_sm=2)
    cfgs = candidates(2027, 150, on_grid=True) + candidates(2028, 150, on_grid=False)
    want = oracle.estimate(cfgs, hw)
    with B.Context(0, 1 << 30) as ctx:
        for mode in (B.WS_MODE_BATCHED, B.WS_MODE_PLAIN):
            res, order = B.ws_estimate_batch(ctx, cfgs, hw, mode=mode)
            got = B.results_to_dicts(res)
            for i, (g, w) in enumerate(zip(got, want)):
                assert g["status"] == w["status"] == 0, (i, g["status"], w["status"])
                for k in B.RESULT_INT:
                    assert g[k] == w[k], (mode, i, k, g[k], w[k])
                for k in B.RESULT_DBL:
                    assert np.isclose(g[k], w[k], rtol=1e-12, atol=0.0), (mode, i, k, g[k], w[k])
