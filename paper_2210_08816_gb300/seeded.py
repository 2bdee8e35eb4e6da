"""Seeded synthetic inputs shared by the CUDA path's callers and the oracle's tests.

This module holds random numbers only: a counter-based SplitMix64 stream
(Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014) turned into N(0,1) samples by the Box-Muller transform.  It holds
none of the discretisation's arithmetic; each side builds its own grid,
boundary conditions and projections from what it is given here.

Every value is a pure function of (seed, stream, index), so a field drawn at
256^3 and the same field drawn at 32^3 share nothing, but two draws with the
same key are bit-identical on every machine.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (the finaliser applied to the running state)."""
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _stream_base(seed: int, stream: int) -> np.uint64:
    key = np.array([(int(seed) & 0xFFFFFFFF) << 20 | (int(stream) & 0xFFFFF)], dtype=np.uint64)
    return _mix64(key)[0]


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles in (0,1): the n first outputs of the SplitMix64 stream keyed by (seed, stream)."""
    base = _stream_base(seed, stream)
    out = np.empty(n, dtype=np.float64)
    chunk = 1 << 22
    with np.errstate(over="ignore"):
        for s in range(0, n, chunk):
            e = min(n, s + chunk)
            ctr = np.arange(s + 1, e + 1, dtype=np.uint64)
            state = base + ctr * _GAMMA
            z = _mix64(state)
            out[s:e] = ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)
    return out


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n N(0,1) doubles by Box-Muller on consecutive pairs of the uniform stream."""
    m = (n + 1) // 2
    u = uniform(seed, stream, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    t = 2.0 * np.pi * u2
    z = np.empty(2 * m, dtype=np.float64)
    z[0::2] = r * np.cos(t)
    z[1::2] = r * np.sin(t)
    return z[:n]


def normal_fields(seed: int, shape: tuple[int, int, int], sigma: float = 1.0,
                  first_stream: int = 0) -> list[np.ndarray]:
    """Four N(0, sigma^2) arrays of `shape` (nz, ny, nx), streams first_stream..first_stream+3.

    Raw random numbers: no boundary condition is applied here.  Callers zero
    what their layout requires (the wall slots of the face-normal velocities).
    """
    n = int(np.prod(shape))
    return [sigma * normal(seed, first_stream + f, n).reshape(shape) for f in range(4)]
