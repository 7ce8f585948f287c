"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer counts must match bit for bit; fp64 volumes and times within 1e-12 relative
(the only differences allowed are exp() rounding between CUDA and the host libm);
rankings must be identical.  Small cases are checked in full against the oracle run
here; the full-size workloads run exactly as the benchmark launches them and are
checked, candidate by candidate and ranking by ranking, against the oracle results
stored under tests/golden/ by tests/make_oracle_golden.py (every candidate of the
25-point and LBM sweeps, a stratified sample of 212 mixed candidates, every candidate
of the served stream).
"""
import os

import numpy as np
import pytest

import oracle
from make_oracle_golden import SERVER_STREAM, fingerprint
from paper_2204_14242_gb300 import binding as B
from paper_2204_14242_gb300 import workloads as W
from test_oracle_pins import random_tiny

pytestmark = pytest.mark.gpu
RTOL = 1e-12
THREADS = max(1, len(os.sched_getaffinity(0)))


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    B.load()
    c = B.Context(0, 24 << 30)
    yield c
    c.close()


def assert_match(res, want, idx=None, what=""):
    got = B.results_to_dicts(res)
    idx = range(len(want)) if idx is None else idx
    for j, i in enumerate(idx):
        g, w = got[i], want[j]
        assert g["status"] == w["status"], (what, i, g["status"], w["status"])
        if w["status"] != 0:
            continue
        for k in B.RESULT_INT:
            assert g[k] == w[k], (what, i, k, g[k], w[k])
        assert g["limiter"] == w["limiter"], (what, i)
        for k in B.RESULT_DBL:
            assert np.isclose(g[k], w[k], rtol=RTOL, atol=0.0), (what, i, k, g[k], w[k])


GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def stored_oracle(name, configs, hw):
    """Oracle results stored for `name`: (indices, list of result dicts).  The stored
    fingerprint of the oracle's inputs must match these candidates."""
    z = np.load(os.path.join(GOLDEN, f"oracle_{name}.npz"))
    idx = [int(i) for i in z["idx"]]
    assert str(z["fingerprint"]) == fingerprint([configs[i] for i in idx], hw), f"{name}: generator drifted"
    ik, dk = [str(k) for k in z["int_keys"]], [str(k) for k in z["dbl_keys"]]
    out = []
    for r_i, r_d in zip(z["out_i"], z["out_d"]):
        d = {k: int(v) for k, v in zip(ik, r_i)}
        d.update({k: float(v) for k, v in zip(dk, r_d)})
        out.append(d)
    return idx, out, z


def assert_ranking(order, t_gpu, t_oracle, what=""):
    """The GPU's order equals the oracle's rank of the oracle's times.  The rank key
    quantises t_pred to 40 bits; GPU and host exp() may differ by an ulp, which can move a
    time across a quantisation boundary.  Only then may the orders differ, and the GPU order
    must still be the same rule applied to its own times."""
    want = [int(i) for i in oracle.rank(t_oracle)]
    if [int(i) for i in order] == want:
        return
    kg = [oracle.rank_key(float(t)) for t in t_gpu]
    ko = [oracle.rank_key(float(t)) for t in t_oracle]
    moved = [i for i in range(len(kg)) if kg[i] != ko[i]]
    assert moved, (what, "orders differ although every rank key agrees")
    assert len(moved) <= max(1, len(kg) // 1000), (what, moved)
    assert [int(i) for i in order] == [int(i) for i in oracle.rank(t_gpu)], what


def test_7pt_all_modes(ctx):
    c = [W.stencil_7pt_128()]
    want = oracle.estimate(c, W.a100())
    for mode in (B.WS_MODE_PLAIN, B.WS_MODE_BATCHED, B.WS_MODE_DIRECT):
        res, order = B.ws_estimate_batch(ctx, c, W.a100(), mode=mode)
        assert_match(res, want, what=f"mode {mode}")
    assert res[0]["wave_load_sectors"] == 832 and res[0]["ov_z"] == 480


@pytest.mark.parametrize("seed", [1, 2])
def test_random_tiny_candidates(ctx, seed):
    rng = W.SplitMix64(100 + seed)
    hw = W.Hardware(sms=3, max_blocks_sm=2)
    cfgs = [random_tiny(rng) for _ in range(300)]
    want = oracle.estimate(cfgs, hw, threads=THREADS)
    res, order = B.ws_estimate_batch(ctx, cfgs, hw, mode=B.WS_MODE_BATCHED)
    assert_match(res, want, what="tiny")
    assert list(order) == list(oracle.rank([w["t_pred"] for w in want]))


@pytest.mark.parametrize("banks,bank_bytes,pair", [(12, 8, 1024), (32, 4, 512), (16, 8, 96)])
def test_bank_layouts(ctx, banks, bank_bytes, pair):
    """Bank-conflict cycles for other bank layouts (the power-of-two fast path and the
    general one) against the oracle."""
    rng = W.SplitMix64(900 + banks + pair)
    hw = W.Hardware(sms=3, max_blocks_sm=2, banks=banks, bank_bytes=bank_bytes, pair_dist_bytes=pair)
    cfgs = [random_tiny(rng) for _ in range(120)] + [random_uniform_tiny(rng) for _ in range(80)]
    want = oracle.estimate(cfgs, hw, threads=THREADS)
    res, order = B.ws_estimate_batch(ctx, cfgs, hw)
    assert_match(res, want, what=f"banks {banks}x{bank_bytes}/{pair}")


def test_modes_are_bit_identical(ctx):
    rng = W.SplitMix64(55)
    hw = W.Hardware(sms=5)
    cfgs = [random_tiny(rng) for _ in range(60)] + W.stencil_25pt_sweep(N=(128, 96, 80))[::29]
    outs = []
    for mode in (B.WS_MODE_PLAIN, B.WS_MODE_BATCHED, B.WS_MODE_DIRECT):
        res, order = B.ws_estimate_batch(ctx, cfgs, hw, mode=mode)
        outs.append((res.tobytes(), order.tobytes()))
    assert outs[0] == outs[1] == outs[2]


def test_graph_replay_is_repeatable(ctx):
    cfgs = W.stencil_25pt_sweep(N=(160, 128, 96))[::7]
    with B.Plan(ctx, cfgs, W.a100()) as p:
        p.execute(B.WS_MODE_BATCHED)
        r1, o1 = p.results()
        for _ in range(3):
            p.execute(B.WS_MODE_BATCHED)
        r2, o2 = p.results()
    assert r1.tobytes() == r2.tobytes() and o1.tobytes() == o2.tobytes()


def sample(n_total, k, seed):
    rng = W.SplitMix64(seed)
    idx = {0, n_total - 1}
    while len(idx) < k:
        idx.add(rng.randint(0, n_total - 1))
    return sorted(idx)


def test_25pt_sweep_full_size(ctx):
    """640x512x512 (x = 640), 755 candidates in one batched launch: every candidate and the
    whole ranking against the stored oracle results."""
    cfgs = W.stencil_25pt_sweep()
    hw = W.a100()
    idx, want, _ = stored_oracle("stencil_25pt_sweep", cfgs, hw)
    assert idx == list(range(len(cfgs)))
    with B.Plan(ctx, cfgs, hw) as p:
        p.execute(B.WS_MODE_BATCHED)
        res, order = p.results()
    assert (res["status"] == 0).all()
    assert_match(res, want, idx, "25pt")
    assert_ranking(order, res["t_pred"], [w["t_pred"] for w in want], "25pt")


def test_lbm_sweep_full_size(ctx):
    """256^3, 42 arrays, 755 candidates: every candidate and the ranking against the stored
    oracle results."""
    cfgs = W.lbm_sweep()
    hw = W.a100()
    idx, want, _ = stored_oracle("lbm_sweep", cfgs, hw)
    assert idx == list(range(len(cfgs)))
    with B.Plan(ctx, cfgs, hw) as p:
        p.execute(B.WS_MODE_BATCHED)
        res, order = p.results()
    assert (res["status"] == 0).all()
    assert_match(res, want, idx, "lbm")
    assert_ranking(order, res["t_pred"], [w["t_pred"] for w in want], "lbm")


def test_mixed_set_full_size(ctx):
    """20,000 seeded mixed candidates in one plan, as the benchmark runs them; a stratified
    sample of 212 (the 12 smallest and 12 largest by enumeration work, the 8 with the widest
    address range, one from each of 180 strata of the work order) against the stored oracle
    results, and the ranking of the sample by the oracle's rule."""
    cfgs = W.mixed_set()
    hw = W.a100()
    idx, want, _ = stored_oracle("mixed_set_sample", cfgs, hw)
    assert len(idx) >= 200
    with B.Plan(ctx, cfgs, hw) as p:
        p.execute(B.WS_MODE_BATCHED)
        res, order = p.results()
    assert (res["status"] == 0).all()
    assert_match(res, want, idx, "mixed")
    # the global order restricted to the sample is the oracle's order of the sample
    pos = np.empty(len(cfgs), np.int64)
    pos[order] = np.arange(len(cfgs))
    got = [idx[j] for j in sorted(range(len(idx)), key=lambda j: pos[idx[j]])]
    want_order = [idx[j] for j in oracle.rank([w["t_pred"] for w in want])]
    if got != want_order:
        assert_ranking([idx.index(i) for i in got], res["t_pred"][idx], [w["t_pred"] for w in want], "mixed")


def random_uniform_tiny(rng: W.SplitMix64):
    """Tiny candidate whose fields share element size and strides (one uniform field
    group), with row lengths that do not divide a warp, x strides on both sides of the
    32-byte interval limit, negative x or y strides and ragged folds."""
    N = (rng.randint(1, 40), rng.randint(1, 12), rng.randint(1, 9))
    B = rng.choice([(3, 2, 2), (5, 3, 1), (6, 1, 4), (12, 2, 1), (32, 1, 1), (40, 1, 1), (7, 4, 2), (64, 1, 1),
                    (4, 4, 4), (1, 8, 2)])
    axis, f = rng.choice([(0, 1), (1, 2), (1, 3), (2, 2), (2, 4), (1, 4)])
    esize = rng.choice((1, 2, 4, 8, 16))
    kind = rng.randint(0, 3)
    px = N[0] + rng.randint(0, 5)
    if kind == 0:
        st = (1, px, px * N[1])
    elif kind == 1:                          # x stride: 2 or 3 elements (AoS)
        sx = rng.choice((2, 3))
        st = (sx, sx * px, sx * px * N[1])
    elif kind == 2:                          # descending x
        st = (-1, px, px * N[1])
    else:                                    # descending y
        st = (1, -px, px * N[1] * 2)
    fields = []
    for _ in range(rng.randint(1, 4)):
        accs = set()
        r = rng.randint(0, 3)
        for _ in range(rng.randint(1, 9)):
            accs.add(W.Access(rng.randint(-r, r), rng.randint(-r, r), rng.randint(-r, r), 0, 0))
        if rng.randint(0, 2):
            accs.add(W.Access(0, 0, 0, 1, 0))
            if rng.randint(0, 3) == 0:
                accs.add(W.Access(-1, 1, 0, 1, 0))
        fields.append(W.Field(esize, sorted(accs, key=lambda a: (a.dx, a.dy, a.dz, a.is_store, a.dc)),
                              align=rng.randint(-70, 70), strides=st, const_off=rng.randint(-5, 5)))
    return W.Config(N=N, B=B, fields=fields, fold_axis=axis, fold=f,
                    wave_blocks_override=rng.choice((0, 1, 2, 3, 5)), flops_per_lup=3.0)


def edge_configs():
    N = (70, 33, 19)
    st = W.dense_strides(N)
    return [
        W.Config(N=(5, 3, 2), B=(32, 4, 2), fields=W.copy_fields((5, 3, 2), W.star_offsets(1))),   # domain < block
        W.Config(N=N, B=(32, 4, 2), fields=W.copy_fields(N, W.box_offsets(2))),                   # ragged
        W.Config(N=N, B=(8, 4, 1), fields=W.copy_fields(N, W.star_offsets(3)), fold_axis=1, fold=16),
        W.Config(N=N, B=(1024, 1, 1), fields=W.copy_fields(N, W.star_offsets(1))),
        W.Config(N=N, B=(1, 1, 64), fields=W.copy_fields(N, W.star_offsets(1)), fold_axis=2, fold=4),
        W.Config(N=N, B=(16, 2, 2), fields=[W.Field(4, [W.Access(0, 0, 0, 0, k) for k in range(3)] +
                                                    [W.Access(0, 0, 0, 1, 1)], align=-20, strides=(3, 3 * 70, 3 * 70 * 33))]),
        W.Config(N=N, B=(32, 2, 1), fields=[W.Field(2, [W.Access(1, -1, 0), W.Access(0, 0, 0, 1)], align=6,
                                                    strides=st, const_off=-7)]),
        W.Config(N=((1 << 20), 3, 2), B=(256, 1, 1), fields=W.copy_fields(((1 << 20), 3, 2), W.star_offsets(2))),
        W.Config(N=N, B=(64, 32, 1), fields=W.copy_fields(N, [(0, 0, 0)])),                         # invalid
        W.Config(N=N, B=(32, 1, 1), fields=[W.Field(8, [W.Access(0, 0, 0)], strides=(-1, -70, -70 * 33))]),
    ]


def test_edge_cases(ctx):
    hw = W.a100()
    cfgs = edge_configs()
    want = oracle.estimate(cfgs, hw, threads=THREADS)
    res, order = B.ws_estimate_batch(ctx, cfgs, hw)
    assert res[8]["status"] == B.WS_EINVAL
    want[8]["status"] = B.WS_EINVAL
    assert_match(res, want, what="edge")
    assert list(order) == list(oracle.rank([w["t_pred"] for w in want]))
    # empty batch
    r0, o0 = B.ws_estimate_batch(ctx, [], hw)
    assert len(r0) == 0


def test_one_shot_estimate_in_parts(ctx):
    """ws_estimate_batch cuts batches of 4096 or more candidates into parts that compile while
    earlier parts run, in one scratch the context keeps zeroed between calls: results and the
    global ranking of two calls in a row are bit-identical to one resident plan's, and
    sampled candidates match the oracle."""
    hw = W.a100()
    cfgs = W.stencil_25pt_sweep(N=(160, 128, 96)) + W.mixed_set(3600, seed=31)
    with B.Plan(ctx, cfgs, hw) as p:
        p.execute(B.WS_MODE_BATCHED)
        res, order = p.results()
    for _ in range(2):
        r2, o2 = B.ws_estimate_batch(ctx, cfgs, hw)
        assert r2.tobytes() == res.tobytes()
        assert list(o2) == list(order)
    idx = sample(755, 8, 41)   # the 25-point candidates (the mixed ones match the plan above)
    want = oracle.estimate([cfgs[i] for i in idx], hw, threads=THREADS)
    assert_match(r2, want, idx, "parts")


@pytest.mark.parametrize("seed", [11, 12])
def test_interval_walk_uniform_groups(ctx, seed):
    """Uniform field groups take the interval walk: both walks against the oracle."""
    rng = W.SplitMix64(300 + seed)
    hw = W.Hardware(sms=3, max_blocks_sm=2)
    cfgs = [random_uniform_tiny(rng) for _ in range(250)]
    want = oracle.estimate(cfgs, hw, threads=THREADS)
    ranks = list(oracle.rank([w["t_pred"] for w in want]))
    for walk in (B.WS_WALK_INTERVAL, B.WS_WALK_SEGMENT, B.WS_WALK_ADDRESS):
        with B.Plan(ctx, cfgs, hw, tuning={"walk": walk}) as p:
            p.execute(B.WS_MODE_BATCHED)
            res, order = p.results()
        assert_match(res, want, what=f"walk {walk}")
        assert list(order) == ranks


def test_interval_and_address_walks_identical(ctx):
    """The row walk, the per-warp interval walk and the per-address walk give
    bit-identical results on the workload families and the edge cases."""
    hw = W.a100()
    rng = W.SplitMix64(77)
    cfgs = (W.stencil_25pt_sweep(N=(160, 128, 96))[::9] + W.lbm_sweep(N=(96, 64, 48))[::37] +
            W.mixed_set(2000)[::50] + edge_configs() + [random_tiny(rng) for _ in range(100)])
    outs, stats = [], []
    for walk in (B.WS_WALK_INTERVAL, B.WS_WALK_SEGMENT, B.WS_WALK_ADDRESS):
        with B.Plan(ctx, cfgs, hw, tuning={"walk": walk}) as p:
            p.execute(B.WS_MODE_BATCHED)
            res, order = p.results()
            outs.append((res.tobytes(), order.tobytes()))
            p.execute(B.WS_MODE_PLAIN)
            res2, order2 = p.results()
            assert res2.tobytes() == res.tobytes() and order2.tobytes() == order.tobytes()
            prof = p.profile()
            # address evaluations and modelled (warp, instruction) pairs are properties of
            # the candidates, however they are walked
            stats.append((prof["addresses"], prof["warp_instr"], prof["block_addresses"]))
    assert outs[0] == outs[1] == outs[2]
    assert stats[0] == stats[1] == stats[2], stats
    assert stats[0][0] > stats[0][2] > 0


def test_multidim_address_space(ctx):
    """The multi-dimensional address space of Sec. 4.4.1 for the wave-level sets, under
    each walk, against the oracle; the 7-point case against its closed form."""
    import dataclasses
    rng = W.SplitMix64(808)
    hw = W.Hardware(sms=3, max_blocks_sm=2)
    md = lambda c: dataclasses.replace(c, address_mode=B.WS_ADDR_MULTIDIM)
    cfgs = ([md(random_tiny(rng)) for _ in range(150)] + [md(random_uniform_tiny(rng)) for _ in range(150)] +
            [md(c) for c in edge_configs()])
    want = oracle.estimate(cfgs, hw, threads=THREADS)
    for w in want:
        if w["status"] != 0:
            w["status"] = B.WS_EINVAL
    for walk in (B.WS_WALK_INTERVAL, B.WS_WALK_SEGMENT, B.WS_WALK_ADDRESS):
        with B.Plan(ctx, cfgs, hw, tuning={"walk": walk}) as p:
            p.execute(B.WS_MODE_BATCHED)
            res, order = p.results()
        assert_match(res, want, what=f"md walk {walk}")
    res, order = B.ws_estimate_batch(ctx, [md(W.stencil_7pt_128())], W.a100())
    assert res[0]["wave_load_sectors"] == 848 and res[0]["wave_load_lines"] == 224
    assert res[0]["ov_y"] == 64 and res[0]["ov_z"] == 480 and res[0]["blk_load_sectors"] == 120
    sweep = [md(c) for c in W.stencil_25pt_sweep(N=(160, 128, 96))[::29]]
    want = oracle.estimate(sweep, W.a100(), threads=THREADS)
    res, order = B.ws_estimate_batch(ctx, sweep, W.a100())
    assert_match(res, want, what="md 25pt")


def test_multi_pass_equals_single_pass(ctx):
    cfgs = W.lbm_sweep(N=(128, 96, 64))[::5]
    hw = W.a100()
    with B.Plan(ctx, cfgs, hw, tuning={"pass_mb": -1}) as p:
        p.execute(B.WS_MODE_BATCHED)
        ref, ref_o = p.results()
        assert p.profile()["passes"] == 1
    with B.Plan(ctx, cfgs, hw, tuning={"pass_mb": 16}) as p:
        assert p.profile()["passes"] > 4
        p.execute(B.WS_MODE_BATCHED)
        r16, o16 = p.results()
    assert r16.tobytes() == ref.tobytes() and o16.tobytes() == ref_o.tobytes()
    small = B.Context(0, 96 << 20)
    try:
        with B.Plan(small, cfgs, hw, tuning={"pass_mb": -1}) as p:
            prof = p.profile()
            assert prof["passes"] > 1
            p.execute(B.WS_MODE_BATCHED)
            res, order = p.results()
    finally:
        small.close()
    assert res.tobytes() == ref.tobytes() and order.tobytes() == ref_o.tobytes()


def test_retuning_to_more_passes_keeps_results(ctx):
    """Re-layout after creation (as the autotuner does) to many more passes than the plan
    was created with; counters of every pass must stay separate from the results."""
    cfgs = W.lbm_sweep(N=(128, 96, 64))[::9]
    hw = W.a100()
    with B.Plan(ctx, cfgs, hw, tuning={"pass_mb": -1}) as p:
        p.execute(B.WS_MODE_BATCHED)
        ref, ref_o = p.results()
    with B.Plan(ctx, cfgs, hw, tuning={"pass_mb": 200}) as p:
        assert p.profile()["passes"] >= 1
        p.autotune()        # tries 96 MiB passes: more passes than at creation
        for mode in (B.WS_MODE_BATCHED, B.WS_MODE_DIRECT):
            p.execute(mode)
            res, order = p.results()
            assert res.tobytes() == ref.tobytes() and order.tobytes() == ref_o.tobytes()


def test_segmented_and_standalone_ranking(ctx):
    cfgs = W.stencil_25pt_sweep(N=(96, 64, 64))[::3]
    hw = W.a100()
    seg = [0, 40, 41, 120, len(cfgs)]
    with B.Plan(ctx, cfgs, hw, segments=seg) as p:
        p.execute(B.WS_MODE_BATCHED)
        res, order = p.results()
    for a, b in zip(seg[:-1], seg[1:]):
        want = a + oracle.rank(res["t_pred"][a:b])
        assert list(order[a:b]) == list(want)
    o2 = B.ws_rank(ctx, res)
    assert list(o2) == list(oracle.rank(res["t_pred"]))


def test_autotune_keeps_results(ctx):
    cfgs = W.stencil_25pt_sweep(N=(160, 128, 96))[::11]
    hw = W.a100()
    with B.Plan(ctx, cfgs, hw) as p:
        p.execute(B.WS_MODE_BATCHED)
        r1, o1 = p.results()
        best = p.autotune()
        assert best["chunk_warps"] in (64, 256, 1024, 4096) and best["pass_mb"] in (96, 1024, 8192, -1)
        assert best["enum_threads"] in (128, 256, 512)
        p.execute(B.WS_MODE_BATCHED)
        r2, o2 = p.results()
        prof = p.profile()
    assert r1.tobytes() == r2.tobytes() and o1.tobytes() == o2.tobytes()
    # per pass enumeration, row walk and counting; then model, counting rank and scatter
    assert prof["launches"] == 3 * prof["passes"] + 3 and prof["addresses"] > 0 and prof["ms_enum"] > 0
    # creation times: the host part (compile, grouping, layout) and the device part
    assert prof["ms_create_host"] > 0 and prof["ms_create_device"] > 0
    assert prof["upload_bytes"] > 0
    # the counting reads only the bitmap pages the row walk wrote into
    assert 0 < prof["count_bytes"] < prof["bitmap_bytes"]


def test_server_results_same_alone_and_in_the_mix(ctx):
    hw = W.a100()
    reqs = W.request_stream(**SERVER_STREAM)
    alone = []
    for r in reqs:
        res, order = B.ws_estimate_batch(ctx, r.configs, hw)
        alone.append((res, order))
    with B.Server(ctx, hw, mem_budget=8 << 30, max_inflight=3) as srv:
        ids = [srv.submit(r.configs) for r in reqs]
        got = {}
        pending = set(ids)
        for _ in range(2000):
            for rid in list(pending):
                rc, res, order = srv.poll(rid, timeout_us=10000)
                if rc == B.WS_OK:
                    got[rid] = (res, order)
                    pending.discard(rid)
                else:
                    assert rc == B.WS_EAGAIN
            if not pending:
                break
        assert not pending
        stats = srv.stats()
    assert stats["completed"] == len(reqs) and stats["steps"] >= 1
    for rid, (res_a, ord_a) in zip(ids, alone):
        res, order = got[rid]
        assert res.tobytes() == res_a.tobytes()
        assert order.tobytes() == ord_a.tobytes()
    # every served result and every request's ranking against the stored oracle results
    flat = [c for r in reqs for c in r.configs]
    idx, want, z = stored_oracle("request_stream_small", flat, hw)
    starts = [int(x) for x in z["request_starts"]]
    assert len(starts) == len(reqs) + 1 and starts[-1] == len(flat)
    for k, rid in enumerate(ids):
        res, order = got[rid]
        w = want[starts[k]:starts[k + 1]]
        assert_match(res, w, what=f"served request {k}")
        assert_ranking(order, res["t_pred"], [x["t_pred"] for x in w], f"served request {k}")


def big_field_candidate(fold):
    """One field read by the 25-point star and written in place, 1024^3 fp64, blocks of
    4x1x64 threads folded along z: its bitmaps take tens of MiB (41 MiB folded twice,
    161 MiB eight times)."""
    N = (1024, 1024, 1024)
    f = W.Field(8, [W.Access(*o) for o in W.star_offsets(4)] + [W.Access(0, 0, 0, 1)], strides=W.dense_strides(N))
    return W.Config(N=N, B=(4, 1, 64), fields=[f], fold_axis=2, fold=fold, flops_per_lup=25.0)


def test_pipelined_estimate_falls_back_to_one_plan(ctx):
    """ws_estimate_batch cuts 4096 or more candidates into parts that share one scratch.  A
    field that fits the whole arena but not that scratch makes the call run the batch as
    one plan: results and order byte-identical to a resident plan's.  A field too large for
    the whole arena gets WS_ENOMEM in its own result while the others are estimated."""
    hw = W.a100()
    rng = W.SplitMix64(515)
    small = [random_tiny(rng) for _ in range(4200)]
    big = big_field_candidate(2)
    need = B.ws_plan_dry_run([big], hw)["bitmap_bytes"]
    cfgs = small[:2000] + [big] + small[2000:]
    with B.Plan(ctx, cfgs, hw) as p:
        p.execute(B.WS_MODE_BATCHED)
        ref, ref_order = p.results()
    assert (ref["status"] == 0).all()
    # the parts share a scratch of three fifths of the free arena: less than the big field
    # needs, while one plan (its descriptors, the whole batch's bitmaps, 8 MiB of headroom)
    # still fits the arena
    arena = int(need * 1.25) + (12 << 20)
    tight = B.Context(0, arena)
    try:
        res, order = B.ws_estimate_batch(tight, cfgs, hw)
        assert res.tobytes() == ref.tobytes() and order.tobytes() == ref_order.tobytes()
        # a field larger than this whole arena: its own WS_ENOMEM, the rest as one plan gives
        huge = big_field_candidate(8)
        assert B.ws_plan_dry_run([huge], hw)["bitmap_bytes"] > arena
        cfgs2 = small[:2000] + [huge] + small[2000:]
        res2, order2 = B.ws_estimate_batch(tight, cfgs2, hw)
    finally:
        tight.close()
    assert res2[2000]["status"] == B.WS_ENOMEM
    keep = np.ones(len(cfgs2), bool)
    keep[2000] = False
    assert res2[keep].tobytes() == ref[keep].tobytes()
    assert int(order2[-1]) == 2000          # an unestimated candidate ranks last
