"""Brute-force counter for tiny grids, written the way the paper evaluates its visitors.

Sec. 4.2 of the paper enumerates thread indices with numpy's ``meshgrid`` and
deduplicates addresses with ``unique``; this module does exactly that, vectorised,
for one candidate at a time.  It is independent of the C++ oracle (different
language, different data flow) and is used only to pin it on grids of at most a
few thousand threads.
"""
from __future__ import annotations

import numpy as np


def _grid(c):
    fy = c.fold if c.fold_axis == 1 else 1
    fz = c.fold if c.fold_axis == 2 else 1
    g = (-(-c.N[0] // c.B[0]), -(-c.N[1] // (c.B[1] * fy)), -(-c.N[2] // (c.B[2] * fz)))
    return g


def _blocks_per_sm(c, hw):
    T = c.B[0] * c.B[1] * c.B[2]
    warps = -(-T // 32)
    b = min(hw.max_blocks_sm, hw.max_threads_sm // (32 * warps))
    if c.regs_per_thread > 0:
        b = min(b, hw.regs_sm // (c.regs_per_thread * 32 * warps))
    return b


def thread_groups(c, hw):
    """Block ids of the representative block, wave, y set and z set."""
    g = _grid(c)
    total = g[0] * g[1] * g[2]
    W = c.wave_blocks_override if c.wave_blocks_override > 0 else hw.sms * _blocks_per_sm(c, hw)
    weff = min(W, total)
    rep = g[0] // 2 + g[0] * (g[1] // 2 + g[1] * (g[2] // 2))
    s = min(W * (rep // W), total - weff)
    wave = np.arange(s, s + weff, dtype=np.int64)
    by = (wave // g[0]) % g[1]
    bz = wave // (g[0] * g[1])
    yset = np.setdiff1d(wave[by >= 1] - g[0], wave)
    zset = np.setdiff1d(np.setdiff1d(wave[bz >= 1] - g[0] * g[1], wave), yset)
    return dict(grid=g, rep=np.array([rep], np.int64), wave=wave, y=yset, z=zset, s=s, weff=weff)


def threads(c, g, block_ids):
    """meshgrid over (block, thread): first folded point, #valid folded points, warp id."""
    T = c.B[0] * c.B[1] * c.B[2]
    nw = -(-T // 32)
    blk, tid = np.meshgrid(block_ids, np.arange(nw * 32, dtype=np.int64), indexing="ij")
    blk, tid = blk.ravel(), tid.ravel()
    exists = tid < T
    bx, by, bz = blk % g[0], (blk // g[0]) % g[1], blk // (g[0] * g[1])
    tx, ty, tz = tid % c.B[0], (tid // c.B[0]) % c.B[1], tid // (c.B[0] * c.B[1])
    p = [bx * c.B[0] + tx, by * c.B[1] + ty, bz * c.B[2] + tz]
    if c.fold_axis:
        p[c.fold_axis] = p[c.fold_axis] * c.fold
    inside = exists & (p[0] < c.N[0]) & (p[1] < c.N[1]) & (p[2] < c.N[2])
    kv = np.where(inside, 1, 0)
    if c.fold_axis:
        kv = np.where(inside, np.minimum(c.fold, c.N[c.fold_axis] - p[c.fold_axis]), 0)
    # warp = 32 consecutive threads of one block, numbered globally
    warp = np.searchsorted(block_ids, blk) * nw + tid // 32
    lane = tid % 32
    return p, kv, warp, lane


def folded(c, offs):
    """Union over the folded points of the offsets: {o + k*e_fold}."""
    out = set()
    for o in offs:
        for k in range(c.fold):
            e = [0, 0, 0]
            if c.fold_axis:
                e[c.fold_axis] = k
            out.add((o[0] + e[0], o[1] + e[1], o[2] + e[2], o[3]))
    return sorted(out)


def needed(c, offs, o, kv):
    m = np.zeros(kv.shape, bool)
    for k in range(c.fold):
        e = [0, 0, 0]
        if c.fold_axis:
            e[c.fold_axis] = k
        if (o[0] - e[0], o[1] - e[1], o[2] - e[2], o[3]) in offs:
            m |= k < kv
    return m


def addresses(f, p, o):
    s = f.strides
    e = s[0] * (p[0] + o[0]) + s[1] * (p[1] + o[1]) + s[2] * (p[2] + o[2]) + f.const_off + o[3]
    return f.align + f.elem_bytes * e


def wave_keys(c, f, p, o, unit):
    """Sector (unit 32) or line (unit 128) identities of the wave-level sets.  Linear
    mode: the address divided by the unit.  Multi-dimensional address space (Sec. 4.4.1):
    the tuple (innermost coordinate in bytes // unit, y, z) without the base alignment,
    packed into one integer (tiny grids only)."""
    if getattr(c, "address_mode", 0) == 0:
        return np.floor_divide(addresses(f, p, o), unit)
    xe = f.strides[0] * (p[0] + o[0]) + f.const_off + o[3]
    xu = np.floor_divide(f.elem_bytes * xe, unit)
    yy, zz = p[1] + o[1], p[2] + o[2]
    assert np.all(np.abs(xu) < (1 << 29)) and np.all(np.abs(yy) < 1000) and np.all(np.abs(zz) < 1000)
    return (xu + (1 << 30)) + (1 << 31) * ((yy + 1024) + 2048 * (zz + 1024))


def bank_cycles(addrs, hw):
    words = np.unique(np.floor_divide(addrs, hw.bank_bytes))
    cycles, i = 0, 0
    while i < len(words):
        j = i
        while j < len(words) and (words[j] - words[i]) * hw.bank_bytes < hw.pair_dist_bytes:
            j += 1
        cycles += int(np.bincount(np.mod(words[i:j], hw.banks), minlength=hw.banks).max())
        i = j
    return cycles


def count(c, hw):
    """All integer outputs of the estimator for one candidate."""
    grp = thread_groups(c, hw)
    g = grp["grid"]
    res = dict(lups_block=0, lups_wave=0, l1_req_sectors=0, l1_bank_cycles=0, l1_store_sectors=0,
               blk_load_sectors=0, blk_load_lines=0, blk_store_sectors=0, blk_store_lines=0,
               wave_load_sectors=0, wave_load_lines=0, wave_store_sectors=0, wave_store_lines=0,
               wave_store_req_sectors=0, ov_y=0, ov_z=0, y_lines=0, z_lines=0,
               wave_blocks=grp["weff"], wave_first_block=grp["s"],
               y_dist_blocks=int(grp["s"] - grp["y"][0]) if len(grp["y"]) else 0,
               z_dist_blocks=int(grp["s"] - grp["z"][0]) if len(grp["z"]) else 0,
               blocks_per_sm=_blocks_per_sm(c, hw))
    th = {k: threads(c, g, grp[k]) for k in ("rep", "wave", "y", "z")}
    res["lups_block"] = int(th["rep"][1].sum())
    res["lups_wave"] = int(th["wave"][1].sum())
    for f in c.fields:
        loads = {(a.dx, a.dy, a.dz, a.dc) for a in f.accesses if not a.is_store}
        stores = {(a.dx, a.dy, a.dz, a.dc) for a in f.accesses if a.is_store}
        sets = {}
        for level in ("rep", "wave", "y", "z"):
            p, kv, warp, lane = th[level]
            for st, offs in ((0, loads), (1, stores)):
                if st and level in ("y", "z"):
                    continue
                all_s, all_l = [], []
                for o in folded(c, offs):
                    m = needed(c, offs, o, kv)
                    a = addresses(f, p, o)[m]
                    if level == "rep":
                        ks, kl = np.floor_divide(a, 32), np.floor_divide(a, 128)
                    else:
                        ks, kl = wave_keys(c, f, p, o, 32)[m], wave_keys(c, f, p, o, 128)[m]
                    all_s.append(ks)
                    all_l.append(kl)
                    if level in ("rep", "wave"):
                        wsec = np.unique(np.stack([warp[m], ks]), axis=1)
                        if level == "rep":
                            res["l1_store_sectors" if st else "l1_req_sectors"] += wsec.shape[1]
                        elif st:
                            res["wave_store_req_sectors"] += wsec.shape[1]
                    if level == "rep":
                        hw_id = warp[m] * 2 + lane[m] // 16
                        for h in np.unique(hw_id):
                            res["l1_bank_cycles"] += bank_cycles(a[hw_id == h], hw)
                ks = np.concatenate(all_s) if all_s else np.zeros(0, np.int64)
                kl = np.concatenate(all_l) if all_l else np.zeros(0, np.int64)
                sets[(level, st)] = (np.unique(ks), np.unique(kl))
        res["blk_load_sectors"] += len(sets[("rep", 0)][0])
        res["blk_load_lines"] += len(sets[("rep", 0)][1])
        res["blk_store_sectors"] += len(sets[("rep", 1)][0])
        res["blk_store_lines"] += len(sets[("rep", 1)][1])
        res["wave_load_sectors"] += len(sets[("wave", 0)][0])
        res["wave_load_lines"] += len(sets[("wave", 0)][1])
        res["wave_store_sectors"] += len(sets[("wave", 1)][0])
        res["wave_store_lines"] += len(sets[("wave", 1)][1])
        w, y, z = sets[("wave", 0)][0], sets[("y", 0)][0], sets[("z", 0)][0]
        res["ov_y"] += len(np.intersect1d(w, y))
        res["ov_z"] += len(np.setdiff1d(np.intersect1d(w, z), y))
        res["y_lines"] += len(sets[("y", 0)][1])
        res["z_lines"] += len(sets[("z", 0)][1])
    return res
