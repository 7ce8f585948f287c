"""GB300 validation (paper Sec. 5.5-5.7) and calibration (Sec. 3) on the GPU.

* The validation kernels compute what they claim: the 3D star stencil and the pull
  lattice-Boltzmann step against fp64 references on small padded grids (so the traffic
  the counters measure belongs to a real stencil of the modelled shape).
* The estimator's descriptions of those kernels (`validation.model_config`, with the
  kernels' own registers per thread) give, through the C ABI, exactly the oracle's
  results, under the calibrated GB300 descriptor and under Table 1's A100.
* The streaming kernels of Sec. 3 finish, run at a positive rate no higher than the
  memory system allows (1.2x the measured HBM copy rate on a 1 GiB data set), and run
  faster on an L2-resident data set than on a 1 GiB one; the whole calibration yields a
  usable descriptor.
No profiler runs inside these tests.
"""
import ctypes
import json
import os

import numpy as np
import pytest

import oracle
from paper_2204_14242_gb300 import binding as B
from paper_2204_14242_gb300 import validation as V
from paper_2204_14242_gb300 import workloads as W
from test_gpu_parity import THREADS, assert_match

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("needs a GPU")
    return t


def hbm_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


def padded(N, pad):
    sx, sy = N[0] + 2 * pad, (N[0] + 2 * pad) * (N[1] + 2 * pad)
    return sx, sy, sy * (N[2] + 2 * pad)


@pytest.mark.parametrize("r,Bs,axis,fold", [(1, (32, 4, 1), 0, 1), (4, (16, 2, 2), 1, 2), (4, (8, 4, 4), 2, 4),
                                           (2, (64, 1, 1), 2, 2)])
def test_star_kernel_is_the_stencil_it_models(torch, r, Bs, axis, fold):
    lib = V._lib()
    N, pad = (37, 21, 19), 4
    sx, sy, n = padded(N, pad)
    g = torch.Generator().manual_seed(7)
    src = torch.rand(n, dtype=torch.float64, generator=g)
    dst = torch.zeros(n, dtype=torch.float64, device="cuda")
    Nc, Bc = (ctypes.c_int32 * 3)(*N), (ctypes.c_int32 * 3)(*Bs)
    s_dev = src.cuda()
    assert lib.ws_val_star(s_dev.data_ptr(), dst.data_ptr(), Nc, r, Bc, axis, fold, pad, None) == 0
    torch.cuda.synchronize()
    got = dst.cpu().numpy().reshape(N[2] + 2 * pad, N[1] + 2 * pad, N[0] + 2 * pad)
    a = src.numpy().reshape(got.shape)
    z, y, x = (slice(pad, pad + N[2]), slice(pad, pad + N[1]), slice(pad, pad + N[0]))
    s = np.zeros((N[2], N[1], N[0]))
    for d in range(1, r + 1):   # the kernel's order of summation
        s = s + (a[z, y, slice(pad - d, pad - d + N[0])] + a[z, y, slice(pad + d, pad + d + N[0])]
                 + a[z, slice(pad - d, pad - d + N[1]), x] + a[z, slice(pad + d, pad + d + N[1]), x]
                 + a[slice(pad - d, pad - d + N[2]), y, x] + a[slice(pad + d, pad + d + N[2]), y, x])
    want = 0.5 * a[z, y, x] + (0.5 / (6.0 * r)) * s
    np.testing.assert_allclose(got[z, y, x], want, rtol=1e-13, atol=0)
    inner = np.zeros(got.shape, bool)
    inner[z, y, x] = True
    assert not got[~inner].any()          # ghost layers are never written


@pytest.mark.parametrize("Bs,axis,fold", [((32, 4, 1), 0, 1), ((16, 2, 2), 1, 2), ((8, 4, 4), 2, 4)])
def test_lbm_kernel_is_the_pull_step_it_models(torch, Bs, axis, fold):
    lib = V._lib()
    N, pad, q, omega = (20, 12, 10), 1, len(V.D3Q19), 0.6
    sx, sy, n = padded(N, pad)
    g = torch.Generator().manual_seed(11)
    srcs = [torch.rand(n, dtype=torch.float64, generator=g) for _ in range(q)]
    s_dev = [t.cuda() for t in srcs]
    d_dev = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(q)]
    sp = torch.tensor([t.data_ptr() for t in s_dev], dtype=torch.int64, device="cuda")
    dp = torch.tensor([t.data_ptr() for t in d_dev], dtype=torch.int64, device="cuda")
    cc = (ctypes.c_int32 * (3 * q))(*[x for c in V.D3Q19 for x in c])
    Nc, Bc = (ctypes.c_int32 * 3)(*N), (ctypes.c_int32 * 3)(*Bs)
    assert lib.ws_val_lbm(sp.data_ptr(), dp.data_ptr(), q, cc, Nc, Bc, axis, fold, pad, omega, None) == 0
    torch.cuda.synchronize()
    shape = (N[2] + 2 * pad, N[1] + 2 * pad, N[0] + 2 * pad)
    a = [t.numpy().reshape(shape) for t in srcs]
    z, y, x = (slice(pad, pad + N[2]), slice(pad, pad + N[1]), slice(pad, pad + N[0]))
    f = [a[i][slice(pad - c[2], pad - c[2] + N[2]), slice(pad - c[1], pad - c[1] + N[1]),
              slice(pad - c[0], pad - c[0] + N[0])] for i, c in enumerate(V.D3Q19)]
    rho = np.zeros_like(f[0])
    for fi in f:
        rho = rho + fi
    for i in range(q):
        got = d_dev[i].cpu().numpy().reshape(shape)
        np.testing.assert_allclose(got[z, y, x], f[i] + omega * (rho / q - f[i]), rtol=1e-13, atol=1e-15)


def test_model_configs_of_the_validation_kernels_match_the_oracle(torch):
    lib = V._lib()
    ctx = B.Context(0, 8 << 30)
    try:
        for v in V.stencil_set()[:3] + V.lbm_set()[:2]:
            regs = lib.ws_val_regs(0 if v["kind"] == "star" else 1, v["r"] if v["kind"] == "star" else v["q"],
                                   v["fold_axis"], v["fold"])
            assert regs > 0
            cfg = V.model_config(v, regs)
            for hw in (V.hardware(None), W.a100()):
                want = oracle.estimate([cfg], hw, threads=THREADS)
                res, order = B.ws_estimate_batch(ctx, [cfg], hw)
                assert_match(res, want, what=f"validation {v['kind']} {v['B']}")
    finally:
        ctx.close()


def stream_rate(torch, lib, kind, a, b, out, nbytes, reps=3):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks, threads = sms * 16, 256
    per_pass = blocks * threads * 8
    iters = max(4, int(4e9 / per_pass))
    best = float("inf")
    for _ in range(reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        rc = lib.ws_val_stream(kind, a.data_ptr(), b.data_ptr() if kind else None, out.data_ptr() if not kind else None,
                               nbytes // 8, blocks, threads, iters, None)
        e.record()
        torch.cuda.synchronize()
        assert rc == 0
        best = min(best, s.elapsed_time(e) * 1e-3)
    return (1 if kind == 0 else 2) * per_pass * iters / best / 1e9


def test_streaming_rates_are_bounded_by_the_memory_system(torch):
    lib = V._lib()
    peak = hbm_peak_gbs()
    a = torch.rand(1 << 27, dtype=torch.float64, device="cuda")          # 1 GiB
    b = torch.empty_like(a)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    load_big = stream_rate(torch, lib, 0, a, b, out, 1 << 30)
    scale_big = stream_rate(torch, lib, 1, a, b, out, 1 << 30)
    load_l2 = stream_rate(torch, lib, 0, a, b, out, 16 << 20)
    for r in (load_big, scale_big):
        assert 0.2 * peak < r <= 1.2 * peak, (r, peak)
    assert load_l2 > 1.2 * load_big           # the L2 level of Sec. 3 lies above the DRAM level


def test_calibration_yields_a_usable_descriptor(torch):
    c = V.calibrate(0)
    peak = hbm_peak_gbs()
    l2_phys = torch.cuda.get_device_properties(0).L2_cache_size
    assert 8 << 20 < c["effective_l2_bytes"] <= 1.1 * l2_phys
    assert c["l2_level_gbs"] > c["dram_level_gbs"] > 0
    assert 0.2 * peak < c["scale_dram_gbs"] <= 1.2 * peak
    assert c["fp64_flops"] > 0
    hw = V.hardware(c)
    ctx = B.Context(0, 1 << 30)
    try:
        res, order = B.ws_estimate_batch(ctx, [W.stencil_7pt_128()], hw)
    finally:
        ctx.close()
    assert res[0]["status"] == 0 and res[0]["wave_load_sectors"] == 832 and res[0]["t_pred"] > 0
