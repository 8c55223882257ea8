"""Seeded synthetic coarse-channel voltages shared by the oracle, the tests and bench.py.

This module holds no correlator arithmetic: it draws counter-based Gaussian noise
(SplitMix64 + Box-Muller) and adds complex sinusoids (a common point source, or
per-path test tones as in the paper's hand-crafted test vectors, Sec. 3.1), then
rounds half-to-even and clips to int8.  The heavy lifting is in ``synth.c``,
compiled once into ``libsynth.so`` beside it.

Voltage layout: int8 ``[block][path][block_samples][2]`` (re, im); path = 2*tile + pol.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

FS = 1_280_000.0          # coarse-channel sample rate, Sec. 2.5
BLOCK_SAMPLES = 64_000    # samples per path per 50 ms data block, Sec. 2.5
SKY_FREQ_HZ = 139.52e6    # coarse channel 109 x 1.28 MHz, inside the 70-300 MHz band (Sec. 2.1)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile synth.c into libsynth.so (gcc, OpenMP)."""
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fno-math-errno", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.synth_voltages.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_longlong, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_int, dp, dp, dp,
                                       ctypes.POINTER(ctypes.c_int), dp, ctypes.c_double,
                                       ctypes.c_longlong, ctypes.c_void_p]
        lib.synth_voltages.restype = None
        lib.synth_uniform.argtypes = [ctypes.c_uint64, ctypes.c_longlong, dp]
        lib.synth_uniform.restype = None
        _lib = lib
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def uniform(seed: int, n: int) -> np.ndarray:
    """n counter-based uniforms in [0, 1) for the given seed."""
    out = np.empty(n, dtype=np.float64)
    if n:
        _load().synth_uniform(ctypes.c_uint64(seed & (2**64 - 1)), n, _dptr(out))
    return out


def voltages(seed: int, n_paths: int, n_samples: int, *, block_samples: int = BLOCK_SAMPLES,
             sigma: float = 16.0, tones=None, delay_c01=None, delay_poly=None, sky_freq_hz: float = 0.0,
             sample0: int = 0, out: np.ndarray | None = None) -> np.ndarray:
    """Synthetic int8 voltages, shape (n_blocks, n_paths, block_samples, 2).

    tones: list of (freq_hz, amplitude, phase_rad, path) with path = -1 for a signal
    common to every path (delayed per path by its delay polynomial), else the one path
    carrying it.
    delay_poly: float64 [n_paths, 3] of (c0 [s], c1 [s/s], c2 [s/s^2]) or None;
    delay_c01: float64 [n_paths, 2] of (c0, c1), the same with c2 = 0 (one of the two).
    """
    if n_samples % block_samples:
        raise ValueError("n_samples must be a whole number of blocks")
    n_blocks = n_samples // block_samples
    tones = list(tones or [])
    f = np.array([t[0] for t in tones] or [0.0], dtype=np.float64)
    a = np.array([t[1] for t in tones] or [0.0], dtype=np.float64)
    ph = np.array([t[2] for t in tones] or [0.0], dtype=np.float64)
    pa = np.array([t[3] for t in tones] or [0], dtype=np.int32)
    d = None
    if delay_c01 is not None and delay_poly is not None:
        raise ValueError("give delay_c01 or delay_poly, not both")
    if delay_c01 is not None:
        d = np.zeros((n_paths, 3))
        d[:, :2] = np.asarray(delay_c01, dtype=np.float64).reshape(n_paths, 2)
    elif delay_poly is not None:
        d = np.ascontiguousarray(np.asarray(delay_poly, dtype=np.float64).reshape(n_paths, 3))
    if out is None:
        out = np.empty((n_blocks, n_paths, block_samples, 2), dtype=np.int8)
    assert out.dtype == np.int8 and out.flags.c_contiguous and out.size == n_blocks * n_paths * block_samples * 2
    _load().synth_voltages(ctypes.c_uint64(seed & (2**64 - 1)), n_paths, n_blocks, block_samples, sigma,
                           len(tones), _dptr(f), _dptr(a), _dptr(ph),
                           pa.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dptr(d), sky_freq_hz,
                           sample0, out.ctypes.data)
    return out


def point_source_tones(seed: int, sigma: float = 16.0, rel_rms: float = 0.3, n_grid: int = 32):
    """A common broadband point source: equal-amplitude tones on every odd multiple of
    Fs/n_grid (bin-centred for every FFT length that is a multiple of n_grid), seeded
    random phases, total rms rel_rms*sigma per component."""
    us = [u for u in range(-(n_grid // 2) + 1, n_grid // 2) if u % 2]
    amp = rel_rms * sigma * np.sqrt(2.0 / len(us))
    ph = 2 * np.pi * uniform(seed ^ 0x70757265, len(us))
    return [(u * FS / n_grid, amp, float(ph[i]), -1) for i, u in enumerate(us)]


def tile_delays_fixed(n_tiles: int, max_s: float = 50e-9) -> np.ndarray:
    """Fixed per-tile delays evenly spread over [0, max_s]; both pols of a tile share
    them.  Returns float64 [n_paths, 3] polynomial (c0, c1, c2)."""
    d = np.zeros((2 * n_tiles, 3))
    for t in range(n_tiles):
        d[2 * t:2 * t + 2, 0] = max_s * t / max(n_tiles - 1, 1)
    return d


def tile_delays_linear(seed: int, n_tiles: int, max_c0: float = 50e-9, max_c1: float = 5e-9) -> np.ndarray:
    """Seeded linear per-tile delays: c0 in U[0, max_c0], c1 in U[-max_c1, max_c1]."""
    u = uniform(seed ^ 0x64656C61, 2 * n_tiles)
    d = np.zeros((2 * n_tiles, 3))
    for t in range(n_tiles):
        d[2 * t:2 * t + 2, 0] = max_c0 * u[2 * t]
        d[2 * t:2 * t + 2, 1] = max_c1 * (2 * u[2 * t + 1] - 1)
    return d


def path_delays_quadratic(seed: int, n_tiles: int, duration_s: float, max_c0: float = 50e-9,
                          max_c1: float = 5e-9, end_c2: float = 20e-9) -> np.ndarray:
    """Seeded quadratic delays, a different polynomial for every signal path (the x and
    y pols of a tile included): c0 in U[0, max_c0], c1 in U[-max_c1, max_c1] and c2 in
    U[-1, 1] * end_c2 / duration_s^2, so the quadratic term alone reaches up to end_c2
    seconds by the end of a call of duration_s.  Returns float64 [n_paths, 3]."""
    n = 2 * n_tiles
    u = uniform(seed ^ 0x71756164, 3 * n).reshape(n, 3)
    d = np.empty((n, 3))
    d[:, 0] = max_c0 * u[:, 0]
    d[:, 1] = max_c1 * (2 * u[:, 1] - 1)
    d[:, 2] = end_c2 / (duration_s * duration_s) * (2 * u[:, 2] - 1)
    return d
