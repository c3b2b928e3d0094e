"""SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) as a counter-based generator.

The generator with state x outputs mix64(x + (i+1)*GAMMA) as its i-th value
(0-based), where mix64 is the published finalizer. The sketches address it
as u(seed, stream, idx): the idx-th output of the generator whose initial
state is mix64(seed + stream*GAMMA) (all arithmetic mod 2^64). The CUDA
library implements the same published definition on its own; the sketch
parameters are therefore bit-identical on both sides.

Streams: 1 sparse-sign rows, 2 sparse-sign signs, 3 SRHT diagonal D,
4 SRHT row sample P, 5 Gaussian entries.
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MASK = (1 << 64) - 1
STREAM_SPARSE_ROWS = 1
STREAM_SPARSE_SIGNS = 2
STREAM_SRHT_D = 3
STREAM_SRHT_P = 4
STREAM_GAUSS = 5


def mix64_int(z: int) -> int:
    """SplitMix64 output finalizer on a Python int (mod 2^64)."""
    z &= MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def u_int(seed: int, stream: int, idx: int) -> int:
    """u(seed, stream, idx) on Python ints."""
    state = mix64_int((seed + stream * GAMMA) & MASK)
    return mix64_int((state + (idx + 1) * GAMMA) & MASK)


def _mix64_np(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def u(seed: int, stream: int, idx) -> np.ndarray:
    """Vectorised u(seed, stream, idx) for an integer array idx (uint64 result)."""
    state = np.uint64(mix64_int((seed + stream * GAMMA) & MASK))
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64_np(state + (idx + np.uint64(1)) * np.uint64(GAMMA))


def mulhi32(x32: np.ndarray, r: int) -> np.ndarray:
    """floor(x32 * r / 2^32) for 32-bit values x32 (uint64 array) and r < 2^32."""
    return (np.asarray(x32, dtype=np.uint64) * np.uint64(r)) >> np.uint64(32)


def mulhi64_int(x: int, r: int) -> int:
    """floor(x * r / 2^64) on Python ints (Lemire's range reduction)."""
    return (x * r) >> 64
