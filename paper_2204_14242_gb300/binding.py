"""Thin Python binding of libwarpspeed (ctypes): argument marshalling only.

Every step of the estimation runs in the CUDA library; this module converts the
neutral workload descriptions into the C structs of ``include/warpspeed.h`` (numpy
structured arrays with the same layout), passes device memory and streams obtained
from PyTorch, and turns results back into numpy / dicts.  Function names follow the
C ABI.  There is no CPU fallback: if the shared library is missing or the GPU is
absent, calls raise.
"""
from __future__ import annotations

import atexit
import ctypes
import os
import threading
import weakref
from typing import List, Optional, Sequence

import numpy as np

from . import _build

# ---- struct layouts (must match include/warpspeed.h) ----------------------------------
ACCESS = np.dtype([("dx", "<i4"), ("dy", "<i4"), ("dz", "<i4"), ("is_store", "<i4"), ("dc", "<i8")], align=True)
FIELD = np.dtype([("elem_bytes", "<i4"), ("n_access", "<i4"), ("align_bytes", "<i8"), ("stride", "<i8", (3,)),
                  ("const_off", "<i8"), ("access_off", "<i8")], align=True)
CONFIG = np.dtype([("N", "<i4", (3,)), ("B", "<i4", (3,)), ("fold_axis", "<i4"), ("fold", "<i4"),
                   ("n_field", "<i4"), ("regs_per_thread", "<i4"), ("field_off", "<i8"),
                   ("flops_per_lup", "<f8"), ("wave_blocks_override", "<i4"), ("address_mode", "<i4")], align=True)
HW = np.dtype([("sms", "<i4"), ("max_threads_sm", "<i4"), ("max_blocks_sm", "<i4"), ("regs_sm", "<i4"),
               ("clock_hz", "<f8"), ("l1_bytes", "<f8"), ("l2_bytes", "<f8"), ("bw_l2", "<f8"),
               ("bw_dram", "<f8"), ("fp_peak", "<f8"), ("banks", "<i4"), ("bank_bytes", "<i4"),
               ("pair_dist_bytes", "<i4"), ("capacity_model", "<i4"), ("hit", "<f8", (4, 3))], align=True)
RESULT_INT = ["lups_block", "lups_wave", "l1_req_sectors", "l1_bank_cycles", "l1_store_sectors",
              "blk_load_sectors", "blk_load_lines", "blk_store_sectors", "blk_store_lines",
              "wave_load_sectors", "wave_load_lines", "wave_store_sectors", "wave_store_lines",
              "wave_store_req_sectors", "ov_y", "ov_z", "y_lines", "z_lines", "wave_blocks",
              "wave_first_block", "y_dist_blocks", "z_dist_blocks", "blocks_per_sm"]
RESULT_DBL = ["v_l1", "v_l2_load", "v_l2_store", "v_dram_load", "v_dram_store", "o_l1", "o_y", "o_z", "o_st",
              "t_l1", "t_l2", "t_dram", "t_fp", "t_pred", "glups"]
RESULT = np.dtype([(k, "<i8") for k in RESULT_INT] + [(k, "<f8") for k in RESULT_DBL] +
                  [("limiter", "<i4"), ("status", "<i4")], align=True)
TUNING = np.dtype([("chunk_warps", "<i4"), ("enum_threads", "<i4"), ("count_words", "<i4"),
                   ("ctas_per_sm", "<i4"), ("pass_mb", "<i4"), ("walk", "<i4")], align=True)
PLAN_SUMMARY = np.dtype([(k, "<i8") for k in (
    "candidates_ok", "fields", "groups", "passes", "enum_items", "row_items", "count_items", "access_entries",
    "interval_entries", "descriptor_bytes", "scratch_bytes", "bitmap_bytes")], align=True)
PROFILE = np.dtype([("ms_total", "<f4"), ("ms_enum", "<f4"), ("ms_count", "<f4"), ("ms_model", "<f4"),
                    ("ms_rank", "<f4"), ("ms_rows", "<f4"), ("launches", "<i4"), ("enum_items", "<i8"), ("count_items", "<i8"),
                    ("warp_instr", "<i8"), ("addresses", "<i8"), ("bitmap_bytes", "<i8"), ("passes", "<i8"),
                    ("upload_bytes", "<i8"), ("row_reds", "<i8"), ("block_addresses", "<i8"),
                    ("ms_create_host", "<f4"), ("ms_create_device", "<f4"), ("count_bytes", "<i8")], align=True)
SERVER_OPTS = np.dtype([("mem_budget", "<u8"), ("max_inflight", "<i4"), ("max_step_cfgs", "<i4"),
                        ("max_queue", "<i4"), ("reserved", "<i4")], align=True)
REQUEST = np.dtype([("cfgs", "<u8"), ("n_cfg", "<i4"), ("n_fld", "<i4"), ("fld", "<u8"), ("acc", "<u8"),
                    ("n_acc", "<i4"), ("reserved", "<i4")], align=True)
SERVER_STATS = np.dtype([("submitted", "<i8"), ("completed", "<i8"), ("rejected", "<i8"), ("steps", "<i8"),
                         ("configs_done", "<i8"), ("bytes_in_use", "<i8"), ("peak_bytes", "<i8"),
                         ("inflight_steps", "<i4"), ("queued", "<i4"), ("canceled", "<i8")], align=True)
CFG_INFO = np.dtype([("status", "<i4"), ("grid", "<i4", (3,)), ("threads", "<i4"), ("warps_per_block", "<i4"),
                     ("blocks_per_sm", "<i4"), ("n_field", "<i4"), ("total_blocks", "<i8"), ("rep_block", "<i8"),
                     ("wave_first", "<i8"), ("wave_blocks", "<i8"), ("y_lo", "<i8"), ("y_hi", "<i8"),
                     ("z_lo", "<i8"), ("z_hi", "<i8"), ("y_dist", "<i8"), ("z_dist", "<i8"),
                     ("modelled_warps", "<i8"), ("folded_loads", "<i8"), ("folded_stores", "<i8"),
                     ("scratch_bytes", "<i8")], align=True)
FIELD_INFO = np.dtype([("lo_sector", "<i8", (2,)), ("words", "<i8", (2,)), ("n_load", "<i4"), ("n_store", "<i4")],
                      align=True)
assert (CFG_INFO.itemsize, FIELD_INFO.itemsize, SERVER_STATS.itemsize) == (144, 40, 72)
assert (ACCESS.itemsize, FIELD.itemsize, CONFIG.itemsize, HW.itemsize, RESULT.itemsize) == (24, 56, 64, 176, 312)

WS_OK, WS_EINVAL, WS_ENOMEM, WS_EAGAIN, WS_ETIMEDOUT, WS_EOVERFLOW, WS_ECUDA, WS_ENOTFOUND, WS_ECANCELED = \
    0, -1, -2, -3, -4, -5, -6, -7, -8
WS_MODE_PLAIN, WS_MODE_BATCHED, WS_MODE_DIRECT = 0, 1, 2
WS_WALK_INTERVAL, WS_WALK_ADDRESS, WS_WALK_SEGMENT = 0, 1, 2
WS_ADDR_LINEAR, WS_ADDR_MULTIDIM = 0, 1

EXPORTS = ["ws_version", "ws_status_string", "ws_last_error", "ws_hw_a100", "ws_create", "ws_destroy",
           "ws_plan_create", "ws_plan_execute", "ws_plan_results", "ws_plan_device_results", "ws_plan_profile",
           "ws_autotune", "ws_plan_destroy", "ws_estimate_batch", "ws_rank", "ws_rank_key", "ws_server_create",
           "ws_server_submit", "ws_server_poll", "ws_server_stats_get", "ws_server_destroy", "ws_describe",
           "ws_describe_fields", "ws_measure_peaks", "ws_estimate_batch_noalloc", "ws_plan_dry_run",
           "ws_server_pause", "ws_server_cancel", "ws_measure_peaks2", "ws_resource_counts_get"]


class WsError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: status {code}")


_lib = None
_lock = threading.Lock()

# Live handles, closed at exit in dependency order (servers, then plans, then contexts)
# so that no worker thread or plan outlives the context it runs on.
_live = {"server": weakref.WeakSet(), "plan": weakref.WeakSet(), "ctx": weakref.WeakSet()}


@atexit.register
def _close_all():
    for kind in ("server", "plan", "ctx"):
        for obj in list(_live[kind]):
            try:
                obj.close()
            except Exception:
                pass


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Loads libwarpspeed.so.  Raises if it is missing (no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB):
            if not build_if_missing:
                raise RuntimeError(f"{_build.LIB} is missing: build it with paper_2204_14242_gb300._build.build()")
            _build.build()
        lib = ctypes.CDLL(_build.LIB)
        P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        sig = {
            "ws_version": ([], I), "ws_status_string": ([I], ctypes.c_char_p), "ws_last_error": ([], ctypes.c_char_p),
            "ws_hw_a100": ([P], None), "ws_create": ([P, I, P, ctypes.c_size_t], I), "ws_destroy": ([P], I),
            "ws_plan_create": ([P, P, I, P, I, P, I, P, P, I, P, P], I), "ws_plan_execute": ([P, I, P], I),
            "ws_plan_results": ([P, P, P, P], I), "ws_plan_device_results": ([P, P, P], I),
            "ws_plan_profile": ([P, P, P], I), "ws_autotune": ([P, P, P], I), "ws_plan_destroy": ([P], I),
            "ws_estimate_batch": ([P, P, I, P, I, P, I, P, P, P, I, P], I), "ws_rank": ([P, P, I, P, P], I),
            "ws_rank_key": ([D], D), "ws_server_create": ([P, P, P, P], I), "ws_server_submit": ([P, P, P], I),
            "ws_server_poll": ([P, ctypes.c_uint64, P, P, I64], I), "ws_server_stats_get": ([P, P], I),
            "ws_server_destroy": ([P], I), "ws_describe": ([P, I, P, I, P, I, P, P], I),
            "ws_describe_fields": ([P, P, I, P, I, P, P], I), "ws_measure_peaks": ([P, P, P], I),
            "ws_estimate_batch_noalloc": ([I, P, I, P, I, P, I, P, P, P, P], I),
            "ws_plan_dry_run": ([P, I, P, I, P, I, P, P, ctypes.c_size_t, P], I),
            "ws_server_pause": ([P, I], I), "ws_server_cancel": ([P, ctypes.c_uint64], I),
            "ws_measure_peaks2": ([P, P], I), "ws_resource_counts_get": ([P], I),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def _check(rc: int, what: str):
    if rc != WS_OK:
        err = load().ws_last_error()
        raise WsError(rc, f"{what} ({load().ws_status_string(rc).decode()}; {err.decode() if err else ''})")


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)   # torch.cuda.Stream


def _ptr(a: np.ndarray):
    return a.ctypes.data if a.size else None


# ---- marshalling ------------------------------------------------------------------------
def marshal(configs: Sequence) -> tuple:
    """Workload Config objects -> (configs, fields, accesses) structured arrays.
    Field lists shared between candidates (same Python list) are stored once."""
    fields_rows, acc_rows = [], []
    cfg = np.zeros(len(configs), CONFIG)
    seen = {}
    for i, c in enumerate(configs):
        key = id(c.fields)
        if key not in seen:
            seen[key] = len(fields_rows)
            for f in c.fields:
                fields_rows.append((f.elem_bytes, len(f.accesses), f.align, tuple(f.strides), f.const_off,
                                    len(acc_rows)))
                for a in f.accesses:
                    acc_rows.append((a.dx, a.dy, a.dz, a.is_store, a.dc))
        row = cfg[i]
        row["N"] = c.N
        row["B"] = c.B
        row["fold_axis"] = c.fold_axis
        row["fold"] = c.fold
        row["n_field"] = len(c.fields)
        row["regs_per_thread"] = c.regs_per_thread
        row["field_off"] = seen[key]
        row["flops_per_lup"] = c.flops_per_lup
        row["wave_blocks_override"] = c.wave_blocks_override
        row["address_mode"] = getattr(c, "address_mode", 0)
    fld = np.array(fields_rows, FIELD) if fields_rows else np.zeros(0, FIELD)
    acc = np.array(acc_rows, ACCESS) if acc_rows else np.zeros(0, ACCESS)
    return cfg, fld, acc


def hw_struct(hw) -> np.ndarray:
    h = np.zeros(1, HW)
    for k in ("sms", "max_threads_sm", "max_blocks_sm", "regs_sm", "clock_hz", "l1_bytes", "l2_bytes", "bw_l2",
              "bw_dram", "fp_peak", "banks", "bank_bytes", "pair_dist_bytes", "capacity_model"):
        h[0][k] = getattr(hw, k)
    h[0]["hit"] = np.array(hw.hit, np.float64)
    return h


def results_to_dicts(res: np.ndarray) -> List[dict]:
    out = []
    for r in res:
        d = {k: int(r[k]) for k in RESULT_INT}
        d.update({k: float(r[k]) for k in RESULT_DBL})
        d["limiter"] = int(r["limiter"])
        d["status"] = int(r["status"])
        out.append(d)
    return out


# ---- C ABI, same names ------------------------------------------------------------------
def ws_describe(configs=None, hw=None, arrays=None) -> np.ndarray:
    """Host-only: what the descriptor compiler makes of each candidate."""
    cfg, fld, acc = arrays if arrays is not None else marshal(configs)
    h = hw if isinstance(hw, np.ndarray) else hw_struct(hw)
    out = np.zeros(len(cfg), CFG_INFO)
    _check(load().ws_describe(_ptr(cfg), len(cfg), _ptr(fld), len(fld), _ptr(acc), len(acc), h.ctypes.data,
                              _ptr(out)), "ws_describe")
    return out


def ws_describe_fields(config, hw) -> np.ndarray:
    cfg, fld, acc = marshal([config])
    h = hw if isinstance(hw, np.ndarray) else hw_struct(hw)
    out = np.zeros(len(config.fields), FIELD_INFO)
    _check(load().ws_describe_fields(cfg.ctypes.data, _ptr(fld), len(fld), _ptr(acc), len(acc), h.ctypes.data,
                                     out.ctypes.data), "ws_describe_fields")
    return out


def ws_plan_dry_run(configs=None, hw=None, tuning=None, scratch_bytes=48 << 30, arrays=None) -> dict:
    """Sizes of the plan a batch would make, without a device (host descriptor compiler,
    list sharing, groups, passes, work items)."""
    cfg, fld, acc = arrays if arrays is not None else marshal(configs)
    h = hw if isinstance(hw, np.ndarray) else hw_struct(hw)
    tun = None
    if tuning is not None:
        tun = np.zeros(1, TUNING)
        for k, v in dict(tuning).items():
            tun[0][k] = v
    out = np.zeros(1, PLAN_SUMMARY)
    _check(load().ws_plan_dry_run(_ptr(cfg), len(cfg), _ptr(fld), len(fld), _ptr(acc), len(acc), h.ctypes.data,
                                  tun.ctypes.data if tun is not None else None, int(scratch_bytes),
                                  out.ctypes.data), "ws_plan_dry_run")
    return {k: int(out[0][k]) for k in PLAN_SUMMARY.names}


def ws_version() -> int:
    return load().ws_version()


def ws_rank_key(t: float) -> float:
    return load().ws_rank_key(float(t))


def ws_hw_a100() -> np.ndarray:
    h = np.zeros(1, HW)
    load().ws_hw_a100(h.ctypes.data)
    return h


class Context:
    """ws_ctx bound to one GPU.  The arena (memory budget) is a PyTorch device tensor."""

    def __init__(self, device: int = 0, arena_bytes: int = 4 << 30, use_torch: bool = True):
        lib = load()
        self._arena_tensor = None
        ptr = None
        if use_torch:
            import torch
            self._arena_tensor = torch.empty(arena_bytes, dtype=torch.uint8, device=f"cuda:{device}")
            ptr = self._arena_tensor.data_ptr()
        h = ctypes.c_void_p()
        _check(lib.ws_create(ctypes.byref(h), device, ptr, arena_bytes), "ws_create")
        self.handle = h
        self.device = device
        self.arena_bytes = arena_bytes
        _live["ctx"].add(self)

    def close(self):
        if self.handle:
            for kind in ("server", "plan"):
                for obj in list(_live[kind]):
                    if getattr(obj, "ctx", None) is self:
                        obj.close()
            load().ws_destroy(self.handle)
            self.handle = None
        self._arena_tensor = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ws_measure_peaks(ctx: Context) -> dict:
    pk = (ctypes.c_double * 4)()
    _check(load().ws_measure_peaks2(ctx.handle, pk), "ws_measure_peaks2")
    return {"int_ops_per_s": pk[0], "l2_red_per_s": pk[1], "l2_red64_run_per_s": pk[2]}


def ws_create(device: int = 0, arena_bytes: int = 4 << 30) -> Context:
    return Context(device, arena_bytes)


def ws_destroy(ctx: Context) -> None:
    ctx.close()


class Plan:
    """ws_plan: candidates compiled into device-resident descriptors."""

    def __init__(self, ctx: Context, configs=None, hw=None, segments=None, tuning=None, arrays=None):
        lib = load()
        if arrays is None:
            arrays = marshal(configs)
        self.cfg, self.fld, self.acc = arrays
        self.hw = hw if isinstance(hw, np.ndarray) else hw_struct(hw)
        self.n = len(self.cfg)
        seg = None
        nseg = 0
        if segments is not None:
            seg = np.ascontiguousarray(np.asarray(segments, np.int32))
            nseg = len(seg) - 1
        tun = None
        if tuning is not None:
            tun = np.zeros(1, TUNING)
            for k, v in dict(tuning).items():
                tun[0][k] = v
        h = ctypes.c_void_p()
        _check(lib.ws_plan_create(ctx.handle, _ptr(self.cfg), self.n, _ptr(self.fld), len(self.fld), _ptr(self.acc),
                                  len(self.acc), self.hw.ctypes.data, _ptr(seg) if seg is not None else None, nseg,
                                  tun.ctypes.data if tun is not None else None, ctypes.byref(h)), "ws_plan_create")
        self.handle = h
        self.ctx = ctx
        _live["plan"].add(self)

    def execute(self, mode: int = WS_MODE_BATCHED, stream=None):
        _check(load().ws_plan_execute(self.handle, mode, _stream_handle(stream)), "ws_plan_execute")

    def results(self, stream=None):
        res = np.zeros(self.n, RESULT)
        order = np.zeros(self.n, np.int32)
        _check(load().ws_plan_results(self.handle, _ptr(res), _ptr(order), _stream_handle(stream)),
               "ws_plan_results")
        return res, order

    def device_results(self):
        r, o = ctypes.c_void_p(), ctypes.c_void_p()
        _check(load().ws_plan_device_results(self.handle, ctypes.byref(r), ctypes.byref(o)), "ws_plan_device_results")
        return r.value, o.value

    def profile(self, stream=None) -> dict:
        p = np.zeros(1, PROFILE)
        _check(load().ws_plan_profile(self.handle, _stream_handle(stream), p.ctypes.data), "ws_plan_profile")
        return {k: p[0][k].item() for k in PROFILE.names}

    def autotune(self, stream=None) -> dict:
        t = np.zeros(1, TUNING)
        _check(load().ws_autotune(self.handle, _stream_handle(stream), t.ctypes.data), "ws_autotune")
        return {k: int(t[0][k]) for k in TUNING.names}

    def close(self):
        if getattr(self, "handle", None):
            load().ws_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ws_plan_create(ctx, configs, hw, segments=None, tuning=None) -> Plan:
    return Plan(ctx, configs, hw, segments, tuning)


def ws_plan_execute(plan: Plan, mode: int = WS_MODE_BATCHED, stream=None):
    plan.execute(mode, stream)


def ws_plan_results(plan: Plan, stream=None):
    return plan.results(stream)


def ws_plan_profile(plan: Plan, stream=None):
    return plan.profile(stream)


def ws_autotune(plan: Plan, stream=None):
    return plan.autotune(stream)


def ws_plan_destroy(plan: Plan):
    plan.close()


def ws_estimate_batch(ctx: Context, configs=None, hw=None, mode: int = WS_MODE_BATCHED, stream=None, arrays=None):
    """Host buffers in, host results out (the library copies inputs and results)."""
    lib = load()
    cfg, fld, acc = arrays if arrays is not None else marshal(configs)
    h = hw if isinstance(hw, np.ndarray) else hw_struct(hw)
    res = np.zeros(len(cfg), RESULT)
    order = np.zeros(len(cfg), np.int32)
    _check(lib.ws_estimate_batch(ctx.handle, _ptr(cfg), len(cfg), _ptr(fld), len(fld), _ptr(acc), len(acc),
                                 h.ctypes.data, _ptr(res), _ptr(order), mode, _stream_handle(stream)),
           "ws_estimate_batch")
    return res, order


NOALLOC_SCRATCH_BYTES = 32 << 20


def ws_estimate_batch_noalloc(device: int = 0, configs=None, hw=None, stream=None, arrays=None):
    """ws_estimate_batch for callers that cannot allocate device memory: every device
    buffer comes from the library's fixed 32 MiB scratch (no context needed)."""
    lib = load()
    cfg, fld, acc = arrays if arrays is not None else marshal(configs)
    h = hw if isinstance(hw, np.ndarray) else hw_struct(hw)
    res = np.zeros(len(cfg), RESULT)
    order = np.zeros(len(cfg), np.int32)
    _check(lib.ws_estimate_batch_noalloc(device, _ptr(cfg), len(cfg), _ptr(fld), len(fld), _ptr(acc), len(acc),
                                         h.ctypes.data, _ptr(res), _ptr(order), _stream_handle(stream)),
           "ws_estimate_batch_noalloc")
    return res, order


def ws_resource_counts() -> dict:
    """CUDA resources the library has created in this process so far."""
    c = (ctypes.c_int64 * 4)()
    _check(load().ws_resource_counts_get(c), "ws_resource_counts_get")
    return {"device_allocs": c[0], "pinned_host_allocs": c[1], "streams": c[2], "events": c[3]}


def ws_rank(ctx: Context, results: np.ndarray, stream=None) -> np.ndarray:
    res = np.ascontiguousarray(results, dtype=RESULT)
    order = np.zeros(len(res), np.int32)
    _check(load().ws_rank(ctx.handle, _ptr(res), len(res), _ptr(order), _stream_handle(stream)), "ws_rank")
    return order


class Server:
    """ws_server: continuous batching of estimation requests."""

    def __init__(self, ctx: Context, hw, mem_budget: int = 0, max_inflight: int = 4, max_step_cfgs: int = 4096,
                 max_queue: int = 0):
        lib = load()
        o = np.zeros(1, SERVER_OPTS)
        o[0]["mem_budget"] = mem_budget
        o[0]["max_inflight"] = max_inflight
        o[0]["max_step_cfgs"] = max_step_cfgs
        o[0]["max_queue"] = max_queue
        self.hw = hw if isinstance(hw, np.ndarray) else hw_struct(hw)
        h = ctypes.c_void_p()
        _check(lib.ws_server_create(ctx.handle, o.ctypes.data, self.hw.ctypes.data, ctypes.byref(h)),
               "ws_server_create")
        self.handle = h
        self.ctx = ctx
        self.sizes = {}
        _live["server"].add(self)

    def submit(self, configs=None, arrays=None) -> int:
        cfg, fld, acc = arrays if arrays is not None else marshal(configs)
        r = np.zeros(1, REQUEST)
        r[0]["cfgs"] = cfg.ctypes.data
        r[0]["n_cfg"] = len(cfg)
        r[0]["fld"] = fld.ctypes.data
        r[0]["n_fld"] = len(fld)
        r[0]["acc"] = acc.ctypes.data
        r[0]["n_acc"] = len(acc)
        rid = ctypes.c_uint64()
        _check(load().ws_server_submit(self.handle, r.ctypes.data, ctypes.byref(rid)), "ws_server_submit")
        self.sizes[rid.value] = len(cfg)
        return rid.value

    def poll(self, rid: int, timeout_us: int = 0):
        """(status, results, order); results/order are None unless status == WS_OK."""
        n = self.sizes[rid]
        res = np.zeros(n, RESULT)
        order = np.zeros(n, np.int32)
        rc = load().ws_server_poll(self.handle, rid, res.ctypes.data, order.ctypes.data, int(timeout_us))
        if rc == WS_EAGAIN:
            return rc, None, None
        del self.sizes[rid]
        if rc != WS_OK:
            return rc, None, None
        return rc, res, order

    def pause(self, paused: bool = True) -> None:
        """Stops (or resumes) admitting new device steps; queued requests wait."""
        _check(load().ws_server_pause(self.handle, int(bool(paused))), "ws_server_pause")

    def cancel(self, rid: int) -> int:
        """Withdraws a queued request: WS_OK (its poll then returns WS_ECANCELED),
        WS_EAGAIN if it already runs, WS_ENOTFOUND if unknown."""
        return load().ws_server_cancel(self.handle, rid)

    def stats(self) -> dict:
        s = np.zeros(1, SERVER_STATS)
        _check(load().ws_server_stats_get(self.handle, s.ctypes.data), "ws_server_stats_get")
        return {k: int(s[0][k]) for k in SERVER_STATS.names}

    def close(self):
        if getattr(self, "handle", None):
            load().ws_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ws_server_create(ctx, hw, **kw) -> Server:
    return Server(ctx, hw, **kw)


def ws_server_submit(srv: Server, configs) -> int:
    return srv.submit(configs)


def ws_server_poll(srv: Server, rid: int, timeout_us: int = 0):
    return srv.poll(rid, timeout_us)


def ws_server_destroy(srv: Server):
    srv.close()
