"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module only draws numbers; it holds none of the method's arithmetic (no
stencils, no solves, no time stepping), so both the CPU oracle and the CUDA path
may take their inputs from it without sharing any computation.

Random stream: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014).  Value k (0-based) of the stream for `seed` is
the SplitMix64 finaliser applied to ``seed + (k + 1) * 0x9E3779B97F4A7C15``
(mod 2^64); a uniform double on [0, 1) is the top 53 bits times 2^-53.  Fields
are drawn in row-major index order (``c[j * nx + i]``), batched solver arrays in
interleaved order (``x[i * batch + s]``).  The paper does not fix a generator;
it only states the distributions (uniform initial conditions, Sec. 3.5.4 and
Chapter 7; diagonally dominant random systems, Sec. 4.2.5).
"""
from __future__ import annotations

import numpy as np

GOLDEN = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Values ``offset .. offset+count-1`` of the SplitMix64 stream of ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, count: int, lo: float, hi: float, offset: int = 0) -> np.ndarray:
    """``count`` doubles uniform on [lo, hi) from stream ``seed`` starting at ``offset``."""
    u = (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def field(seed: int, ny: int, nx: int, lo: float, hi: float) -> np.ndarray:
    """A (ny, nx) row-major field of i.i.d. uniform values (initial conditions)."""
    return uniform(seed, ny * nx, lo, hi).reshape(ny, nx)


def uniform_torch(seed: int, count: int, lo: float, hi: float, device="cuda", offset: int = 0):
    """Same numbers as :func:`uniform`, generated with torch int64 ops on ``device``.

    Used for the large batched-solver inputs, where drawing on the host would
    dominate set-up time.  Logical right shifts are emulated with masks because
    torch shifts int64 arithmetically; products wrap modulo 2^64 as in C.
    """
    import torch

    def s64(v: int) -> int:
        v &= 0xFFFFFFFFFFFFFFFF
        return v - (1 << 64) if v >= (1 << 63) else v

    def lsr(z, s):
        return (z >> s) & ((1 << (64 - s)) - 1)

    k = torch.arange(offset + 1, offset + count + 1, dtype=torch.int64, device=device)
    z = k * s64(GOLDEN) + s64(seed)
    z = (z ^ lsr(z, 30)) * s64(_M1)
    z = (z ^ lsr(z, 27)) * s64(_M2)
    z = z ^ lsr(z, 31)
    u = lsr(z, 11).to(torch.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def diag_dominant_penta(seed: int, n: int, batch: int):
    """Random cyclic pentadiagonal coefficients, interleaved ``[i * batch + s]``.

    Off-diagonals a, b, d, e ~ U[-1, 1] (the cyclic corner entries included);
    diagonal c = (1.5 + 0.5 u) * (|a| + |b| + |d| + |e|) with u ~ U[0, 1], so every
    row is strictly diagonally dominant by a factor of at least 1.5, which is the
    stability condition the paper states for LU without pivoting (Sec. 4.2.5).
    Streams: a, b, d, e, u take consecutive blocks of ``n * batch`` values.
    """
    cnt = n * batch
    a = uniform(seed, cnt, -1.0, 1.0, 0 * cnt)
    b = uniform(seed, cnt, -1.0, 1.0, 1 * cnt)
    d = uniform(seed, cnt, -1.0, 1.0, 2 * cnt)
    e = uniform(seed, cnt, -1.0, 1.0, 3 * cnt)
    u = uniform(seed, cnt, 0.0, 1.0, 4 * cnt)
    c = (1.5 + 0.5 * u) * (np.abs(a) + np.abs(b) + np.abs(d) + np.abs(e))
    return a, b, c, d, e


def diag_dominant_tri(seed: int, n: int, batch: int):
    """Random cyclic tridiagonal coefficients, interleaved; b = (1.5 + 0.5u)(|a| + |c|)."""
    cnt = n * batch
    a = uniform(seed, cnt, -1.0, 1.0, 0 * cnt)
    c = uniform(seed, cnt, -1.0, 1.0, 1 * cnt)
    u = uniform(seed, cnt, 0.0, 1.0, 2 * cnt)
    b = (1.5 + 0.5 * u) * (np.abs(a) + np.abs(c))
    return a, b, c
