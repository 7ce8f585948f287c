"""Seeded synthetic workloads: code-generation candidates for the metric estimator.

This module only *describes* inputs.  It holds none of the estimator's arithmetic
(no addresses, sectors, waves or volumes are computed here), so both the CUDA path
and the CPU oracle can be fed from it without sharing any of the method.

A candidate configuration is what a stencil code generator hands to the estimator
(Sec. 1.2 of the paper: address expressions, launch configuration, field sizes and
alignments).  Every address expression is affine in the thread's grid point:

    addr = align + elem_bytes * (sum_d stride_d * (p_d + o_d) + const_off + dc)

where p is the grid point a thread updates and (o, dc) is the access.

Workload families (all fp64 unless stated, x contiguous, row-major):
  * stencil_7pt_128      3D 7-point star, 128^3, block 32x4x1, wave of 8 blocks
  * stencil_25pt_sweep   3D 25-point star (radius 4), 640x512x512 (x = 640), 151
                         block shapes x 5 folding variants = 755 candidates
  * lbm_sweep            27 D3Q27 pull arrays + 15 D3Q15 phase-field arrays, 256^3,
                         same 755 candidates
  * mixed_set            seeded random stencils (star/box, radius 1-4, 5-125 offsets,
                         1-27 arrays, fp32/fp64, domains 64..1024 per axis)
  * request_stream       Poisson arrivals of candidate lists built from mixed_set-style
                         stencils (16-512 candidates, log-uniform)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field as dc_field
from typing import List, Sequence, Tuple

# --------------------------------------------------------------------------------------
# descriptors
# --------------------------------------------------------------------------------------

FOLD_NONE, FOLD_Y, FOLD_Z = 0, 1, 2


@dataclass(frozen=True)
class Access:
    """One relative field access: grid offset (dx, dy, dz) plus an extra element offset dc."""
    dx: int
    dy: int
    dz: int
    is_store: int = 0
    dc: int = 0


@dataclass
class Field:
    """One array.  Fields never alias (Sec. 4.3); the base pointer is replaced by `align`."""
    elem_bytes: int
    accesses: List[Access]
    align: int = 0
    strides: Tuple[int, int, int] = (1, 0, 0)
    const_off: int = 0


@dataclass
class Config:
    """One code-generation candidate (launch configuration + fields)."""
    N: Tuple[int, int, int]
    B: Tuple[int, int, int]
    fields: List[Field]
    fold_axis: int = FOLD_NONE
    fold: int = 1
    flops_per_lup: float = 0.0
    regs_per_thread: int = 0
    wave_blocks_override: int = 0
    name: str = ""
    address_mode: int = 0        # 0 linear addresses, 1 multi-dimensional address space (Sec. 4.4.1)


@dataclass
class Hardware:
    """Modelled GPU (Table 1 of the paper).  Defaults: A100-SXM4-40G.

    Values not printed in the paper: max_blocks_sm (32, an A100 datasheet value) and
    regs_sm (65536).  fp_peak = 3.5 Flop/B machine balance x 1400 GB/s (Sec. 5.2).
    hit[i] = (a, b, c) of R(O) = a*exp(-b*exp(-c*O)) for L1, L2 y-layer, L2 z-layer,
    L2 store (Sec. 4.4); the paper prints no coefficients, these are illustrative.
    """
    sms: int = 108
    max_threads_sm: int = 2048
    max_blocks_sm: int = 32
    regs_sm: int = 65536
    clock_hz: float = 1.41e9
    l1_bytes: float = 192.0 * 1024
    l2_bytes: float = 20.0 * 1024 * 1024
    bw_l2: float = 5000e9
    bw_dram: float = 1400e9
    fp_peak: float = 4.9e12
    banks: int = 16
    bank_bytes: int = 8
    pair_dist_bytes: int = 1024
    capacity_model: int = 1
    hit: Tuple[Tuple[float, float, float], ...] = (
        (1.0, 0.01, -3.07),   # L1 redundant loads
        (1.0, 0.05, -2.0),    # L2 y-layer overlap
        (1.0, 0.01, -3.07),   # L2 z-layer overlap
        (1.0, 0.01, -3.07),   # L2 redundant (partial) stores
    )


def a100() -> Hardware:
    return Hardware()


def v100() -> Hardware:
    """V100-PCIe-32GB column of Table 1 (6 MB L2, no split).  fp_peak (half the fp64
    FMA rate, for an add-only mix) is not printed in the paper."""
    return Hardware(sms=80, clock_hz=1.38e9, l1_bytes=128.0 * 1024, l2_bytes=6.0 * 1024 * 1024,
                    bw_l2=2500e9, bw_dram=800e9, fp_peak=3.5e12)


def gb300(l2_bytes: float = 89.6e6, bw_l2: float = 15555e9, bw_dram: float = 6081e9,
          fp_peak: float = 528.8e9, clock_hz: float = 2.07e9, sms: int = 152) -> Hardware:
    """GB300 descriptor: 152 SMs, 2.07 GHz, 256 KiB L1 per SM; the defaults of the effective
    L2 size (LOAD rate above 90 % of its L2 level up to 89.6 MB), L2 bandwidth (LOAD on L2
    data sets, 15.6 TB/s), DRAM bandwidth (SCALE on data sets >= 1 GiB, 6.08 TB/s) and fp64
    rate (half of the measured 1.06 TFLOP/s FMA rate, for add-dominated stencils) are the
    values `validation.calibrate` measured on a GB300; pass others to override."""
    return Hardware(sms=sms, clock_hz=clock_hz, l1_bytes=256.0 * 1024, l2_bytes=l2_bytes, bw_l2=bw_l2,
                    bw_dram=bw_dram, fp_peak=fp_peak)


# --------------------------------------------------------------------------------------
# splitmix64 (Steele, Lea, Flood 2014; constants as published by S. Vigna)
# --------------------------------------------------------------------------------------

_M64 = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & _M64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] by rejection (no modulo bias)."""
        span = hi - lo + 1
        limit = (1 << 64) - ((1 << 64) % span)
        while True:
            x = self.next_u64()
            if x < limit:
                return lo + x % span

    def shuffle(self, xs: list) -> None:
        """Fisher-Yates, in place."""
        for i in range(len(xs) - 1, 0, -1):
            j = self.randint(0, i)
            xs[i], xs[j] = xs[j], xs[i]

    def choice(self, xs: Sequence):
        return xs[self.randint(0, len(xs) - 1)]

    def exponential(self, rate: float) -> float:
        return -math.log(1.0 - self.uniform()) / rate


# --------------------------------------------------------------------------------------
# building blocks
# --------------------------------------------------------------------------------------

def dense_strides(N: Sequence[int]) -> Tuple[int, int, int]:
    """Row-major, x contiguous, no padding."""
    return (1, N[0], N[0] * N[1])


def star_offsets(r: int) -> List[Tuple[int, int, int]]:
    """Centre plus +-1..+-r on each axis (6r+1 points)."""
    offs = [(0, 0, 0)]
    for d in range(1, r + 1):
        for s in (-d, d):
            offs += [(s, 0, 0), (0, s, 0), (0, 0, s)]
    return offs


def box_offsets(r: int) -> List[Tuple[int, int, int]]:
    """All points of the (2r+1)^3 cube, centre first."""
    offs = [(0, 0, 0)]
    for dz in range(-r, r + 1):
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                if (dx, dy, dz) != (0, 0, 0):
                    offs.append((dx, dy, dz))
    return offs


D3Q27 = [(x, y, z) for z in (-1, 0, 1) for y in (-1, 0, 1) for x in (-1, 0, 1)]
D3Q15 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)] + \
        [(x, y, z) for z in (-1, 1) for y in (-1, 1) for x in (-1, 1)]


def block_shapes() -> List[Tuple[int, int, int]]:
    """Powers of two, bx >= 4, 32 <= bx*by*bz <= 1024, bz <= 64 (CUDA limit): 151 shapes."""
    out = []
    for ez in range(0, 7):
        for ey in range(0, 11):
            for ex in range(2, 11):
                t = ex + ey + ez
                if 5 <= t <= 10:
                    out.append((1 << ex, 1 << ey, 1 << ez))
    return out


FOLD_VARIANTS = [(FOLD_NONE, 1), (FOLD_Y, 2), (FOLD_Y, 4), (FOLD_Z, 2), (FOLD_Z, 4)]


def copy_fields(N, loads, esize=8, align=0):
    """One source field read at `loads`, one destination written at 0."""
    st = dense_strides(N)
    src = Field(esize, [Access(*o) for o in loads], align=align, strides=st)
    dst = Field(esize, [Access(0, 0, 0, 1)], align=align, strides=st)
    return [src, dst]


# --------------------------------------------------------------------------------------
# the five workload families
# --------------------------------------------------------------------------------------

def stencil_7pt_128() -> Config:
    """3D 7-point star (radius 1), fp64, 128^3, block 32x4x1, no folding, wave of 8 blocks."""
    N = (128, 128, 128)
    return Config(N=N, B=(32, 4, 1), fields=copy_fields(N, star_offsets(1)),
                  flops_per_lup=7.0, wave_blocks_override=8, name="7pt_128_32x4x1")


def stencil_25pt_sweep(N=(640, 512, 512), variants=FOLD_VARIANTS) -> List[Config]:
    """3D 25-point star (radius 4), fp64: every block shape x folding variant (Sec. 5.2)."""
    fields = copy_fields(N, star_offsets(4))
    out = []
    for B in block_shapes():
        for axis, f in variants:
            out.append(Config(N=tuple(N), B=B, fields=fields, fold_axis=axis, fold=f,
                              flops_per_lup=25.0,
                              name=f"25pt_{B[0]}x{B[1]}x{B[2]}_f{'nyz'[axis]}{f}"))
    return out


def lbm_fields(N) -> List[Field]:
    """27 D3Q27 pull arrays + 15 D3Q15 phase-field arrays, each read at -c_i, written at 0."""
    st = dense_strides(N)
    fields = []
    for c in D3Q27 + D3Q15:
        fields.append(Field(8, [Access(-c[0], -c[1], -c[2], 0), Access(0, 0, 0, 1)], strides=st))
    return fields


def lbm_sweep(N=(256, 256, 256), variants=FOLD_VARIANTS) -> List[Config]:
    fields = lbm_fields(N)
    out = []
    for B in block_shapes():
        for axis, f in variants:
            out.append(Config(N=tuple(N), B=B, fields=fields, fold_axis=axis, fold=f,
                              name=f"lbm_{B[0]}x{B[1]}x{B[2]}_f{'nyz'[axis]}{f}"))
    return out


def random_stencil(rng: SplitMix64, N=None):
    """A random stencil: (fields template, N).  Offsets dealt round-robin to the arrays."""
    shape = rng.choice(("star", "box"))
    r = rng.randint(1, 4)
    pool = star_offsets(r) if shape == "star" else box_offsets(r)
    n = rng.randint(5, min(125, len(pool)))
    rest = pool[1:]
    rng.shuffle(rest)
    offs = [pool[0]] + rest[:n - 1]
    rng.shuffle(offs)
    A = min(rng.randint(1, 27), n)
    esize = rng.choice((4, 8))
    if N is None:
        N = (rng.randint(64, 1024), rng.randint(64, 1024), rng.randint(64, 1024))
    st = dense_strides(N)
    per = [[] for _ in range(A)]
    for i, o in enumerate(offs):
        per[i % A].append(Access(*o))
    fields = [Field(esize, acc, strides=st) for acc in per]
    fields.append(Field(esize, [Access(0, 0, 0, 1)], strides=st))
    return fields, tuple(N), float(n), f"{shape}{r}_n{n}_a{A}_e{esize}"


def mixed_set(n: int = 20000, seed: int = 20221) -> List[Config]:
    """Seeded mixed candidates: each one a fresh random stencil, shape and folding."""
    rng = SplitMix64(seed)
    shapes = block_shapes()
    out = []
    for i in range(n):
        fields, N, flops, tag = random_stencil(rng)
        B = rng.choice(shapes)
        axis, f = rng.choice(FOLD_VARIANTS)
        out.append(Config(N=N, B=B, fields=fields, fold_axis=axis, fold=f, flops_per_lup=flops,
                          name=f"mix{i}_{tag}"))
    return out


@dataclass
class Request:
    arrival_s: float
    configs: List[Config]
    tag: str = ""


def request_stream(n_requests: int = 10000, rate_hz: float = 200.0, seed: int = 20222,
                   kmin: int = 16, kmax: int = 512) -> List[Request]:
    """Poisson arrivals; each request = one random stencil x k candidate (shape, fold) pairs,
    k log-uniform in [kmin, kmax], drawn without replacement from the 755-candidate family."""
    rng = SplitMix64(seed)
    family = [(B, v) for B in block_shapes() for v in FOLD_VARIANTS]
    t = 0.0
    out = []
    lk0, lk1 = math.log(kmin), math.log(kmax + 1)
    for i in range(n_requests):
        t += rng.exponential(rate_hz)
        fields, N, flops, tag = random_stencil(rng)
        k = min(kmax, max(kmin, int(math.exp(lk0 + (lk1 - lk0) * rng.uniform()))))
        idx = list(range(len(family)))
        rng.shuffle(idx)
        cfgs = []
        for j in idx[:k]:
            B, (axis, f) = family[j]
            cfgs.append(Config(N=N, B=B, fields=fields, fold_axis=axis, fold=f,
                               flops_per_lup=flops, name=f"req{i}_{j}"))
        out.append(Request(arrival_s=t, configs=cfgs, tag=tag))
    return out
