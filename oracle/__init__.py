"""CPU oracle of the metric estimator -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It compiles and loads ``liboracle.so`` (a plain
C++ std::set enumerator, ``oracle.cpp``) and marshals the neutral workload
descriptions into the oracle's own flat arrays.  It imports nothing from the CUDA
path and the CUDA path imports nothing from it.

Parity status per function (see the tests under ``tests/``):
  * sector / line / LUP / warp / bank counts: pinned by the numpy brute force of the
    paper's grid iteration, by closed forms (7-point block and wave, wave-depth law of
    Sec. 5.7, streaming copy, D3Q15 240 B/LUP) and by invariants;
  * layer-condition overlaps ov_y / ov_z: pinned by brute force and the 7-point closed
    form under the stated reading of the thread sets;
  * capacity model and limiters: pinned at the special cases the paper fixes
    (R_hit = 1 -> compulsory, R_hit = 0 -> request volume, lowest-limiter = max) and,
    term by term, against closed forms derived by hand for the 7-point case and a
    misaligned streaming copy (O_L1, O_y, O_z, O_st, R(O) with b, c != 0, every volume
    and limiter time; tests/test_model_pins.py, which also plants mistakes in a copy of
    this oracle and checks that the pins catch them);
  * the hit-rate coefficients are inputs: the paper prints none, so their values (not
    the function they enter) are parity unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFG_NI, FLD_NI, ACC_NI, HW_ND = 13, 8, 5, 26
INT_KEYS = ["status", "lups_block", "lups_wave", "l1_req_sectors", "l1_bank_cycles",
            "l1_store_sectors", "blk_load_sectors", "blk_load_lines", "blk_store_sectors",
            "blk_store_lines", "wave_load_sectors", "wave_load_lines", "wave_store_sectors",
            "wave_store_lines", "wave_store_req_sectors", "ov_y", "ov_z", "y_lines", "z_lines",
            "wave_blocks", "wave_first_block", "y_dist_blocks", "z_dist_blocks", "blocks_per_sm",
            "limiter"]
DBL_KEYS = ["v_l1", "v_l2_load", "v_l2_store", "v_dram_load", "v_dram_store", "o_l1", "o_y",
            "o_z", "o_st", "t_l1", "t_l2", "t_dram", "t_fp", "t_pred", "glups"]


def build(force: bool = False) -> str:
    """Compiles liboracle.so next to its source (plain g++, no FMA contraction)."""
    src = os.path.join(_HERE, "oracle.cpp")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(src),
                                                   os.path.getmtime(os.path.join(_HERE, "oracle.h")))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
           src, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            lib.orc_estimate.argtypes = [ctypes.c_int, P, P, P, P, P, P, P, ctypes.c_int]
            lib.orc_estimate.restype = ctypes.c_int
            lib.orc_rank.argtypes = [ctypes.c_int, P, P]
            lib.orc_rank.restype = ctypes.c_int
            lib.orc_rank_key.argtypes = [ctypes.c_double]
            lib.orc_rank_key.restype = ctypes.c_double
            _lib = lib
    return _lib


def flatten(configs, hw):
    """Neutral descriptions -> the oracle's flat arrays (fields deduplicated by identity)."""
    cfg_i = np.zeros((len(configs), CFG_NI), np.int64)
    cfg_d = np.zeros(len(configs), np.float64)
    flds, accs = [], []
    seen = {}
    for i, c in enumerate(configs):
        key = id(c.fields)
        if key not in seen:
            seen[key] = len(flds)
            for f in c.fields:
                flds.append([f.elem_bytes, f.align, f.strides[0], f.strides[1], f.strides[2],
                             f.const_off, len(f.accesses), len(accs)])
                for a in f.accesses:
                    accs.append([a.dx, a.dy, a.dz, a.is_store, a.dc])
        cfg_i[i] = [c.N[0], c.N[1], c.N[2], c.B[0], c.B[1], c.B[2], c.fold_axis, c.fold,
                    len(c.fields), seen[key], c.regs_per_thread, c.wave_blocks_override,
                    getattr(c, "address_mode", 0)]
        cfg_d[i] = c.flops_per_lup
    fld_i = np.array(flds, np.int64).reshape(-1, FLD_NI)
    acc_i = np.array(accs, np.int64).reshape(-1, ACC_NI)
    hw_d = np.array([hw.sms, hw.max_threads_sm, hw.max_blocks_sm, hw.regs_sm, hw.clock_hz,
                     hw.l1_bytes, hw.l2_bytes, hw.bw_l2, hw.bw_dram, hw.fp_peak, hw.banks,
                     hw.bank_bytes, hw.pair_dist_bytes, hw.capacity_model]
                    + [x for h in hw.hit for x in h], np.float64)
    assert hw_d.size == HW_ND
    return cfg_i, cfg_d, fld_i, acc_i, hw_d


def estimate_arrays(configs, hw, threads: int = 1):
    """Returns (out_i [n, 25] int64, out_d [n, 15] float64)."""
    lib = _load()
    cfg_i, cfg_d, fld_i, acc_i, hw_d = flatten(configs, hw)
    n = len(configs)
    out_i = np.zeros((n, len(INT_KEYS)), np.int64)
    out_d = np.zeros((n, len(DBL_KEYS)), np.float64)
    fld_i = np.ascontiguousarray(fld_i) if fld_i.size else np.zeros((1, FLD_NI), np.int64)
    acc_i = np.ascontiguousarray(acc_i) if acc_i.size else np.zeros((1, ACC_NI), np.int64)
    rc = lib.orc_estimate(n, cfg_i.ctypes.data, cfg_d.ctypes.data, fld_i.ctypes.data,
                          acc_i.ctypes.data, hw_d.ctypes.data, out_i.ctypes.data,
                          out_d.ctypes.data, int(threads))
    if rc != 0:
        raise ValueError(f"orc_estimate rejected its arguments ({rc})")
    return out_i, out_d


def estimate(configs, hw, threads: int = 1):
    """Returns one dict per candidate with every integer and fp64 output."""
    out_i, out_d = estimate_arrays(configs, hw, threads)
    res = []
    for i in range(len(configs)):
        d = {k: int(out_i[i, j]) for j, k in enumerate(INT_KEYS)}
        d.update({k: float(out_d[i, j]) for j, k in enumerate(DBL_KEYS)})
        res.append(d)
    return res


def rank(t_pred):
    lib = _load()
    t = np.ascontiguousarray(np.asarray(t_pred, np.float64))
    order = np.zeros(len(t), np.int32)
    if lib.orc_rank(len(t), t.ctypes.data, order.ctypes.data) != 0:
        raise ValueError("orc_rank rejected its arguments")
    return order


def rank_key(t: float) -> float:
    return _load().orc_rank_key(float(t))
