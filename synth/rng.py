"""Seeded, counter-based random numbers for synthetic workloads.

Holds none of the filtering arithmetic: it only draws numbers.  Both the
CUDA path's tests/bench and the oracle's tests take their inputs from here.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used counter-style: draw i of stream s
under seed S is mix(key(S, s) + (i + 1) * GAMMA), where mix is SplitMix64's
output function and key(S, s) = mix(S ^ (s * STREAM_MULT)).  Uniforms take
the top 53 bits; normals use the Box-Muller transform (Box and Muller, 1958)
in FP64, with draws 2p and 2p+1 giving normals 2p and 2p+1.

Everything is written on torch int64 tensors (two's-complement wrap-around
multiply, logical shifts by masking), so the same function runs on the CPU
and on the GPU.  Integer draws are bit-identical across devices; FP64
normals can differ in the last bit between devices' libm, which is why the
oracle is always fed the exact tensor the GPU path consumed.
"""
from __future__ import annotations

import math

import torch

_M64 = (1 << 64) - 1


def _i64(v: int) -> int:
    v &= _M64
    return v - (1 << 64) if v >= (1 << 63) else v


GAMMA = _i64(0x9E3779B97F4A7C15)
_C1 = _i64(0xBF58476D1CE4E5B9)
_C2 = _i64(0x94D049BB133111EB)
STREAM_MULT = _i64(0xD1B54A32D192ED03)

# stream ids used by the workloads
STREAM_SIGNAL = 1
STREAM_LENGTHS = 2
STREAM_SECTIONS = 3
STREAM_FILTER = 4
STREAM_STATE = 5
STREAM_MISC = 6

CHUNK = 1 << 22


def _srl(z: torch.Tensor, s: int) -> torch.Tensor:
    """Logical right shift of int64 bit patterns."""
    return (z >> s) & ((1 << (64 - s)) - 1)


def mix_t(z: torch.Tensor) -> torch.Tensor:
    z = (z ^ _srl(z, 30)) * _C1
    z = (z ^ _srl(z, 27)) * _C2
    return z ^ _srl(z, 31)


def mix_py(z: int) -> int:
    """Pure-Python SplitMix64 output function on unsigned 64-bit ints."""
    z &= _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def stream_key(seed: int, stream: int) -> int:
    return _i64(mix_py((seed & _M64) ^ ((stream * 0xD1B54A32D192ED03) & _M64)))


def raw_u64(seed: int, stream: int, start: int, n: int, device="cpu") -> torch.Tensor:
    """Draws start..start+n-1 as int64 bit patterns."""
    key = stream_key(seed, stream)
    idx = torch.arange(start + 1, start + n + 1, dtype=torch.int64, device=device)
    return mix_t(idx * GAMMA + key)


def raw_u64_py(seed: int, stream: int, i: int) -> int:
    key = stream_key(seed, stream) & _M64
    return mix_py((key + (i + 1) * 0x9E3779B97F4A7C15) & _M64)


def uniform(seed: int, stream: int, n: int, start: int = 0, device="cpu") -> torch.Tensor:
    """U(0, 1) doubles, never exactly 0 or 1."""
    out = torch.empty(n, dtype=torch.float64, device=device)
    for o in range(0, n, CHUNK):
        m = min(CHUNK, n - o)
        r = raw_u64(seed, stream, start + o, m, device)
        out[o:o + m] = (_srl(r, 11).to(torch.float64) + 0.5) * (2.0 ** -53)
    return out


def normal(seed: int, stream: int, n: int, start: int = 0, device="cpu",
           dtype=torch.float32) -> torch.Tensor:
    """N(0, 1) via Box-Muller in FP64, rounded once to ``dtype``.
    ``start`` must be even (normals come in pairs)."""
    assert start % 2 == 0
    out = torch.empty(n, dtype=dtype, device=device)
    for o in range(0, n, CHUNK):
        m = min(CHUNK, n - o)
        npair = (m + 1) // 2
        u = uniform(seed, stream, 2 * npair, start=start + o, device=device).view(npair, 2)
        rad = torch.sqrt(-2.0 * torch.log(u[:, 0]))
        ang = (2.0 * math.pi) * u[:, 1]
        z = torch.stack((rad * torch.cos(ang), rad * torch.sin(ang)), dim=1).reshape(-1)[:m]
        out[o:o + m] = z.to(dtype)
    return out


def randint(seed: int, stream: int, n: int, lo: int, hi: int, start: int = 0,
            device="cpu") -> torch.Tensor:
    """Integers uniform in [lo, hi] inclusive: floor(u * span) on a 53-bit
    uniform u in [0, 1) (bias below span * 2^-53)."""
    span = hi - lo + 1
    assert 0 < span < (1 << 40)
    r = raw_u64(seed, stream, start, n, device)
    u = _srl(r, 11).to(torch.float64) * (2.0 ** -53)
    return lo + torch.floor(u * span).to(torch.int64)
