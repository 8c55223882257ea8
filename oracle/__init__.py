"""FP64 CPU oracle of the MWAX FX correlator's GPU stage (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline leg may import
this package.  It is independent of the CUDA library: ``oracle.c`` is plain C
compiled with gcc, and nothing here touches the GPU path.

Every function follows the paper's definition step by step (Sec. 2.5-2.7, see
``oracle.c``).  Parity status per function (what pins it is in tests/test_oracle_*.py):
  dft / fft          pinned: numpy.fft, impulse and tone closed forms, direct DFT
  avg_weights        pinned: hand-derived tables in tests/golden/avg_weights.txt
  spectra (delay)    pinned: closed-form tone phase with and without correction
  correlate          pinned: Parseval identity (exact int64 RHS), tone ordering test,
                     Hermitian full matrix, point-source closed form (statistical)
  correlate_int      pinned: numpy int64 brute force, linearity (2x input -> 4x)
  correlate_sampled  pinned: equals correlate element by element
Conventions the paper leaves open (sign of the sky-frequency phase term, baseline
order inside MWAX_ORDER, edge half-channels) follow the readings stated in the
design notes; those readings are not pinned by the paper itself.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

FS = 1_280_000.0
_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None


class _Desc(ctypes.Structure):
    _fields_ = [("n_tiles", ctypes.c_int), ("fft_len", ctypes.c_int), ("fine_avg", ctypes.c_int),
                ("int_frames", ctypes.c_longlong), ("n_samples", ctypes.c_longlong),
                ("block_samples", ctypes.c_int), ("sky_freq_hz", ctypes.c_double),
                ("dc_exclude", ctypes.c_int)]


@dataclass
class Desc:
    """One correlation job: T tiles, N-point frames, fscrunch F, K frames per integration."""
    n_tiles: int
    fft_len: int
    fine_avg: int
    int_frames: int
    n_samples: int
    block_samples: int = 64_000
    sky_freq_hz: float = 0.0
    dc_exclude: int = 1

    @property
    def n_paths(self):
        return 2 * self.n_tiles

    @property
    def n_baselines(self):
        return self.n_tiles * (self.n_tiles + 1) // 2

    @property
    def n_chan_out(self):
        return self.fft_len // self.fine_avg

    @property
    def n_ints(self):
        return self.n_samples // (self.int_frames * self.fft_len)

    def c(self):
        return _Desc(self.n_tiles, self.fft_len, self.fine_avg, self.int_frames, self.n_samples,
                     self.block_samples, self.sky_freq_hz, self.dc_exclude)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc -O2, OpenMP, no fast-math)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        vp, dp = ctypes.c_void_p, ctypes.POINTER(_Desc)
        lib.ora_dft.argtypes = [ctypes.c_int, vp, vp]
        lib.ora_fft.argtypes = [ctypes.c_int, vp, vp]
        lib.ora_avg_weights.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp]
        lib.ora_avg_weights.restype = ctypes.c_double
        lib.ora_spectra.argtypes = [dp, vp, vp, ctypes.c_int, ctypes.c_longlong, ctypes.c_longlong, vp]
        lib.ora_correlate.argtypes = [dp, vp, vp, vp, vp]
        lib.ora_correlate.restype = ctypes.c_int
        lib.ora_xmatrix.argtypes = [dp, vp, vp, ctypes.c_longlong, ctypes.c_int, vp]
        lib.ora_xmatrix.restype = ctypes.c_int
        lib.ora_correlate_sampled.argtypes = [dp, vp, vp, ctypes.c_longlong, vp, vp]
        lib.ora_correlate_sampled.restype = ctypes.c_int
        lib.ora_correlate_int.argtypes = [dp, vp, vp, vp]
        lib.ora_correlate_int.restype = ctypes.c_int
        lib.ora_baseline_tiles.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int)]
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _delay(d: Desc, delay):
    if delay is None:
        return None
    a = np.ascontiguousarray(np.asarray(delay, dtype=np.float64).reshape(d.n_paths, 3))
    return a


def dft(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.complex128)
    X = np.empty_like(x)
    _load().ora_dft(len(x), _p(x), _p(X))
    return X


def fft(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.complex128)
    X = np.empty_like(x)
    _load().ora_fft(len(x), _p(x), _p(X))
    return X


def avg_weights(N: int, F: int, dc_exclude: int, j: int):
    """(weights over the N ultrafine channels, weight sum) for output channel j."""
    w = np.empty(N, dtype=np.float64)
    s = _load().ora_avg_weights(N, F, dc_exclude, j, _p(w))
    return w, s


def baseline_tiles(T: int, b: int):
    i, j = ctypes.c_int(), ctypes.c_int()
    _load().ora_baseline_tiles(T, b, ctypes.byref(i), ctypes.byref(j))
    return i.value, j.value


def spectra(d: Desc, volt: np.ndarray, delay, path: int, m0: int, nm: int) -> np.ndarray:
    """Y[m, c] for frames [m0, m0+nm) of one path (FFT, shift, delay correction)."""
    volt = np.ascontiguousarray(volt, dtype=np.int8)
    Y = np.empty((nm, d.fft_len), dtype=np.complex128)
    dl = _delay(d, delay)
    _load().ora_spectra(ctypes.byref(d.c()), _p(volt), _p(dl), path, m0, nm, _p(Y))
    return Y


def correlate(d: Desc, volt: np.ndarray, delay=None):
    """(vis complex128 [ints, B, M, 4], weights float64 [ints, B, 4])."""
    volt = np.ascontiguousarray(volt, dtype=np.int8)
    vis = np.empty((d.n_ints, d.n_baselines, d.n_chan_out, 4), dtype=np.complex128)
    wts = np.empty((d.n_ints, d.n_baselines, 4), dtype=np.float64)
    dl = _delay(d, delay)
    rc = _load().ora_correlate(ctypes.byref(d.c()), _p(volt), _p(dl), _p(vis), _p(wts))
    if rc:
        raise ValueError(f"oracle rejected the job (rc={rc})")
    return vis, wts


def xmatrix(d: Desc, volt: np.ndarray, delay, w: int, c: int) -> np.ndarray:
    volt = np.ascontiguousarray(volt, dtype=np.int8)
    C = np.empty((d.n_paths, d.n_paths), dtype=np.complex128)
    dl = _delay(d, delay)
    rc = _load().ora_xmatrix(ctypes.byref(d.c()), _p(volt), _p(dl), w, c, _p(C))
    if rc:
        raise ValueError(f"oracle rejected the job (rc={rc})")
    return C


def correlate_sampled(d: Desc, volt: np.ndarray, delay, req) -> np.ndarray:
    """req: int array [R, 4] of (integration, baseline, channel, pol) -> complex128 [R]."""
    volt = np.ascontiguousarray(volt, dtype=np.int8)
    req = np.ascontiguousarray(np.asarray(req, dtype=np.int64).reshape(-1, 4))
    out = np.empty(len(req), dtype=np.complex128)
    dl = _delay(d, delay)
    rc = _load().ora_correlate_sampled(ctypes.byref(d.c()), _p(volt), _p(dl), len(req), _p(req), _p(out))
    if rc:
        raise ValueError(f"oracle rejected the job (rc={rc})")
    return out


def correlate_int(d: Desc, volt: np.ndarray):
    """Integer mode: (vis int64 [ints, B, 4, 2], weights float64 [ints, B, 4])."""
    volt = np.ascontiguousarray(volt, dtype=np.int8)
    vis = np.empty((d.n_ints, d.n_baselines, 4, 2), dtype=np.int64)
    wts = np.empty((d.n_ints, d.n_baselines, 4), dtype=np.float64)
    rc = _load().ora_correlate_int(ctypes.byref(d.c()), _p(volt), _p(vis), _p(wts))
    if rc:
        raise ValueError(f"oracle rejected the job (rc={rc})")
    return vis, wts


# ------------------------------------------------------------------ roadmap extensions
class _Ext(ctypes.Structure):
    _fields_ = [("sample_rate_hz", ctypes.c_double), ("keep_bins", ctypes.c_int),
                ("delay_table", ctypes.c_void_p), ("table_step", ctypes.c_longlong),
                ("table_steps", ctypes.c_longlong), ("passband", ctypes.c_void_p),
                ("zero_flags", ctypes.c_void_p), ("normalise", ctypes.c_int)]


@dataclass
class Ext:
    """Roadmap extensions (Sec. 4): sample rate / kept bins (oversampled channels, 4.5),
    tabulated delays [n_paths, steps] of `table_step` samples (2.4.1, 4.3), passband gains
    per ultrafine channel (4.2), zeroing flags [n_blocks, n_paths] and normalisation (4.1)."""
    sample_rate_hz: float = 0.0
    keep_bins: int = 0
    delay_table: np.ndarray | None = None
    table_step: int = 6400
    passband: np.ndarray | None = None
    zero_flags: np.ndarray | None = None
    normalise: int = 0

    def c(self, d: Desc):
        keep = []
        tab = None
        if self.delay_table is not None:
            tab = np.ascontiguousarray(np.asarray(self.delay_table, dtype=np.float64).reshape(d.n_paths, -1))
            keep.append(tab)
        pb = None
        if self.passband is not None:
            pb = np.ascontiguousarray(np.asarray(self.passband, dtype=np.float64).reshape(d.fft_len))
            keep.append(pb)
        fl = None
        if self.zero_flags is not None:
            fl = np.ascontiguousarray(np.asarray(self.zero_flags, dtype=np.uint8).reshape(-1, d.n_paths))
            keep.append(fl)
        e = _Ext(self.sample_rate_hz, self.keep_bins, _p(tab), self.table_step,
                 0 if tab is None else tab.shape[1], _p(pb), _p(fl), self.normalise)
        return e, keep

    def n_chan_out(self, d: Desc):
        return (self.keep_bins or d.fft_len) // d.fine_avg


def _load_ext():
    lib = _load()
    if not hasattr(lib, "_ext_ready"):
        vp, dp, ep = ctypes.c_void_p, ctypes.POINTER(_Desc), ctypes.POINTER(_Ext)
        lib.ora_avg_weights_keep.argtypes = [ctypes.c_int] * 5 + [vp]
        lib.ora_avg_weights_keep.restype = ctypes.c_double
        lib.ora_spectra_ext.argtypes = [dp, ep, vp, vp, ctypes.c_int, ctypes.c_longlong, ctypes.c_longlong, vp]
        lib.ora_occupancy.argtypes = [dp, ep, ctypes.c_longlong, ctypes.c_int, ctypes.c_int]
        lib.ora_occupancy.restype = ctypes.c_double
        lib.ora_correlate_ext.argtypes = [dp, ep, vp, vp, vp, vp]
        lib.ora_correlate_ext.restype = ctypes.c_int
        lib.ora_correlate_int_ext.argtypes = [dp, ep, vp, vp, vp]
        lib.ora_correlate_int_ext.restype = ctypes.c_int
        lib._ext_ready = True
    return lib


def avg_weights_keep(N: int, keep: int, F: int, dc_exclude: int, j: int):
    w = np.empty(N, dtype=np.float64)
    s = _load_ext().ora_avg_weights_keep(N, keep, F, dc_exclude, j, _p(w))
    return w, s


def spectra_ext(d: Desc, e: Ext, volt: np.ndarray, delay, path: int, m0: int, nm: int) -> np.ndarray:
    volt = np.ascontiguousarray(volt, dtype=np.int8)
    Y = np.empty((nm, d.fft_len), dtype=np.complex128)
    ce, keep = e.c(d)
    _load_ext().ora_spectra_ext(ctypes.byref(d.c()), ctypes.byref(ce), _p(volt), _p(_delay(d, delay)), path, m0, nm,
                                _p(Y))
    return Y


def occupancy(d: Desc, e: Ext, w: int, p: int, q: int) -> float:
    ce, keep = e.c(d)
    return _load_ext().ora_occupancy(ctypes.byref(d.c()), ctypes.byref(ce), w, p, q)


def correlate_ext(d: Desc, e: Ext, volt: np.ndarray, delay=None):
    """(vis complex128 [ints, B, M, 4] with M = kept bins / F, weights float64 [ints, B, 4])."""
    volt = np.ascontiguousarray(volt, dtype=np.int8)
    M = e.n_chan_out(d)
    vis = np.empty((d.n_ints, d.n_baselines, M, 4), dtype=np.complex128)
    wts = np.empty((d.n_ints, d.n_baselines, 4), dtype=np.float64)
    ce, keep = e.c(d)
    rc = _load_ext().ora_correlate_ext(ctypes.byref(d.c()), ctypes.byref(ce), _p(volt), _p(_delay(d, delay)),
                                       _p(vis), _p(wts))
    if rc:
        raise ValueError(f"oracle rejected the job (rc={rc})")
    return vis, wts


def correlate_int_ext(d: Desc, e: Ext, volt: np.ndarray):
    volt = np.ascontiguousarray(volt, dtype=np.int8)
    vis = np.empty((d.n_ints, d.n_baselines, 4, 2), dtype=np.int64)
    wts = np.empty((d.n_ints, d.n_baselines, 4), dtype=np.float64)
    ce, keep = e.c(d)
    rc = _load_ext().ora_correlate_int_ext(ctypes.byref(d.c()), ctypes.byref(ce), _p(volt), _p(vis), _p(wts))
    if rc:
        raise ValueError(f"oracle rejected the job (rc={rc})")
    return vis, wts


def beamform(d: Desc, volt: np.ndarray, beam_table: np.ndarray, table_step: int = 6400, int_frames: int = 0,
             sample_rate_hz: float = 0.0):
    """Tied-array beams (Sec. 4.4): (beams complex128 [n_beams, 2, frames, N],
    Stokes I power [n_beams, n_det, N], incoherent [n_det, 2, N]); the detected outputs
    are empty when int_frames is 0.  beam_table: float64 [n_beams, n_paths, steps] s."""
    lib = _load()
    if not hasattr(lib, "_beam_ready"):
        vp = ctypes.c_void_p
        lib.ora_beamform.argtypes = [ctypes.POINTER(_Desc), ctypes.c_double, vp, ctypes.c_int, vp, ctypes.c_longlong,
                                     ctypes.c_longlong, ctypes.c_longlong, vp, vp, vp]
        lib.ora_beamform.restype = ctypes.c_int
        lib._beam_ready = True
    volt = np.ascontiguousarray(volt, dtype=np.int8)
    tab = np.ascontiguousarray(np.asarray(beam_table, dtype=np.float64))
    nb = tab.shape[0]
    tab = tab.reshape(nb, d.n_paths, -1)
    frames = d.n_samples // d.fft_len
    n_det = frames // int_frames if int_frames > 0 else 0
    beams = np.empty((nb, 2, frames, d.fft_len), dtype=np.complex128)
    power = np.empty((nb, n_det, d.fft_len))
    incoh = np.empty((n_det, 2, d.fft_len))
    rc = lib.ora_beamform(ctypes.byref(d.c()), sample_rate_hz, _p(volt), nb, _p(tab), table_step, tab.shape[2],
                          int_frames, _p(beams), _p(power), _p(incoh))
    if rc:
        raise ValueError(f"oracle rejected the job (rc={rc})")
    return beams, power, incoh
