"""Python binding of the MWAX B300 correlator C ABI (``include/mwax.h``).

Argument marshalling only: every step of the correlation runs in ``libmwax.so``'s CUDA
kernels.  PyTorch supplies device memory and streams.  There is no fallback: if the
library is missing or no GPU is usable, the calls raise.

    plan = mwax_plan_create_ex(PlanDesc(n_tiles=256, fft_len=128, fine_avg=4, int_time_s=0.5,
                                        samples_per_call=10_240_000, precision=MWAX_FP32))
    out = empty_output(plan)                 # torch uint8 buffer on the current device
    mwax_correlate(plan, volt, delay, out)   # volt: int8 [blocks, paths, block_samples, 2]
    vis, weights = split_output(plan, out)   # views: complex64 [ints, B, M, 4], float32 [ints, B, 4]
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _build

MWAX_OK, MWAX_EINVAL, MWAX_ENOMEM, MWAX_ECUDA, MWAX_EUNSUPPORTED, MWAX_ETIMEOUT = range(6)
MWAX_FP32, MWAX_FP16, MWAX_FP8, MWAX_INT8, MWAX_FP16X3 = range(5)
PRECISIONS = {"fp32": MWAX_FP32, "fp16": MWAX_FP16, "fp8": MWAX_FP8, "int8": MWAX_INT8, "fp16x3": MWAX_FP16X3}
FS = 1_280_000.0
BLOCK_SAMPLES = 64_000

LIB_PATH = _build.LIB


class MwaxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"mwax status {status}: {msg}")
        self.status = status


class _CDesc(ctypes.Structure):
    _fields_ = [("n_tiles", ctypes.c_int), ("fft_len", ctypes.c_int), ("fine_avg", ctypes.c_int),
                ("int_time_s", ctypes.c_double), ("samples_per_call", ctypes.c_longlong),
                ("block_samples", ctypes.c_int), ("precision", ctypes.c_int), ("sky_freq_hz", ctypes.c_double),
                ("keep_dc", ctypes.c_int), ("workspace_limit", ctypes.c_size_t),
                ("sample_rate_hz", ctypes.c_double), ("keep_bins", ctypes.c_int)]


class _BeamDesc(ctypes.Structure):
    _fields_ = [("n_tiles", ctypes.c_int), ("fft_len", ctypes.c_int), ("n_beams", ctypes.c_int),
                ("samples_per_call", ctypes.c_longlong), ("block_samples", ctypes.c_int),
                ("sky_freq_hz", ctypes.c_double), ("sample_rate_hz", ctypes.c_double),
                ("table_step_samples", ctypes.c_longlong), ("int_frames", ctypes.c_int),
                ("workspace_limit", ctypes.c_size_t), ("engine", ctypes.c_int)]


class _Call(ctypes.Structure):
    _fields_ = [("voltages", ctypes.c_void_p), ("delay_poly", ctypes.c_void_p), ("delay_table", ctypes.c_void_p),
                ("table_steps", ctypes.c_longlong), ("table_step_samples", ctypes.c_longlong),
                ("zero_flags", ctypes.c_void_p), ("normalise", ctypes.c_int), ("vis_out", ctypes.c_void_p)]


class _CInfo(ctypes.Structure):
    _fields_ = [("n_paths", ctypes.c_int), ("n_baselines", ctypes.c_longlong), ("n_chan_out", ctypes.c_int),
                ("frames_per_int", ctypes.c_longlong), ("n_ints", ctypes.c_longlong),
                ("input_bytes", ctypes.c_size_t), ("vis_set_bytes", ctypes.c_size_t),
                ("weights_bytes", ctypes.c_size_t), ("output_bytes", ctypes.c_size_t),
                ("workspace_bytes", ctypes.c_size_t), ("precision", ctypes.c_int),
                ("x_flop_alg", ctypes.c_double), ("x_flop_issued", ctypes.c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("fstep_variant", ctypes.c_int), ("run_len", ctypes.c_int), ("window", ctypes.c_int),
                ("ms", ctypes.c_double)]

    def __repr__(self):
        return (f"Tuning(fstep_variant={self.fstep_variant}, run_len={self.run_len}, window={self.window}, "
                f"ms={self.ms:.3f})")


class _ServerDesc(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("n_lanes", ctypes.c_int), ("workspace_limit", ctypes.c_size_t)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong), ("failed", ctypes.c_longlong),
                ("queued", ctypes.c_longlong), ("in_flight", ctypes.c_longlong), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double), ("deadline_misses", ctypes.c_longlong),
                ("hbm_in_use", ctypes.c_size_t), ("cold_starts", ctypes.c_longlong), ("p50_warm_ms", ctypes.c_double),
                ("p99_warm_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


@dataclass
class PlanDesc:
    n_tiles: int
    fft_len: int
    fine_avg: int
    int_time_s: float
    samples_per_call: int = 0
    block_samples: int = 0
    precision: int = MWAX_FP32
    sky_freq_hz: float = 0.0
    keep_dc: int = 0
    workspace_limit: int = 0
    sample_rate_hz: float = 0.0
    keep_bins: int = 0

    def c(self) -> _CDesc:
        return _CDesc(self.n_tiles, self.fft_len, self.fine_avg, self.int_time_s, self.samples_per_call,
                      self.block_samples, int(self.precision), self.sky_freq_hz, self.keep_dc, self.workspace_limit,
                      self.sample_rate_hz, self.keep_bins)


_lib = None
SYMBOLS = ("mwax_plan_create", "mwax_plan_create_ex", "mwax_plan_get_info", "mwax_plan_output_bytes",
           "mwax_plan_input_bytes", "mwax_plan_set_stream", "mwax_correlate", "mwax_correlate_host",
           "mwax_correlate_host_async",
           "mwax_plan_sync", "mwax_plan_set_wait_limit", "mwax_plan_destroy", "mwax_last_error", "mwax_version",
           "mwax_plan_enable_timing",
           "mwax_plan_stage_times", "mwax_plan_autotune", "mwax_plan_set_tuning", "mwax_plan_get_tuning",
           "mwax_batch_create", "mwax_batch_set_stream", "mwax_batch_set_graphs", "mwax_batch_correlate",
           "mwax_batch_sync", "mwax_batch_destroy", "mwax_server_create", "mwax_server_submit", "mwax_server_poll",
           "mwax_server_wait", "mwax_server_drain", "mwax_server_get_stats", "mwax_server_reset_stats",
           "mwax_server_destroy",
           "mwax_correlate_noalloc", "mwax_correlate_ex", "mwax_plan_set_passband", "mwax_beam_create",
           "mwax_beam_set_stream", "mwax_beam_output_bytes", "mwax_beam_form", "mwax_beam_sync", "mwax_beam_destroy",
           "mwax_probe_fma")


def load_library(path: str | None = None):
    """Load libmwax.so (building it first if the sources are newer and nvcc is present)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if _build.stale():
        try:
            _build.build()
        except (OSError, FileNotFoundError) as e:  # no nvcc: use what is there, or fail
            if not os.path.exists(path):
                raise ImportError(f"libmwax.so missing and cannot be built: {e}") from e
    if not os.path.exists(path):
        raise ImportError(f"libmwax.so not found at {path}; run `python -m paper_2303_11557_b300._build`")
    lib = ctypes.CDLL(path)
    vp, st = ctypes.c_void_p, ctypes.c_int
    lib.mwax_plan_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int]
    lib.mwax_plan_create.restype = vp
    lib.mwax_plan_create_ex.argtypes = [ctypes.POINTER(_CDesc)]
    lib.mwax_plan_create_ex.restype = vp
    lib.mwax_plan_get_info.argtypes = [vp, ctypes.POINTER(_CInfo)]
    lib.mwax_plan_get_info.restype = st
    lib.mwax_plan_output_bytes.argtypes = [vp]
    lib.mwax_plan_output_bytes.restype = ctypes.c_size_t
    lib.mwax_plan_input_bytes.argtypes = [vp]
    lib.mwax_plan_input_bytes.restype = ctypes.c_size_t
    lib.mwax_plan_set_stream.argtypes = [vp, vp]
    lib.mwax_plan_set_stream.restype = st
    lib.mwax_correlate.argtypes = [vp, vp, vp, vp]
    lib.mwax_correlate.restype = st
    lib.mwax_correlate_host.argtypes = [vp, vp, vp, vp]
    lib.mwax_correlate_host.restype = st
    lib.mwax_correlate_host_async.argtypes = [vp, vp, vp, vp]
    lib.mwax_correlate_host_async.restype = st
    lib.mwax_plan_sync.argtypes = [vp]
    lib.mwax_plan_sync.restype = st
    lib.mwax_plan_set_wait_limit.argtypes = [vp, ctypes.c_uint]
    lib.mwax_plan_set_wait_limit.restype = st
    lib.mwax_probe_fma.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp]
    lib.mwax_probe_fma.restype = ctypes.c_longlong
    lib.mwax_plan_destroy.argtypes = [vp]
    lib.mwax_plan_destroy.restype = None
    lib.mwax_last_error.argtypes = []
    lib.mwax_last_error.restype = ctypes.c_char_p
    lib.mwax_plan_enable_timing.argtypes = [vp, ctypes.c_int]
    lib.mwax_plan_enable_timing.restype = st
    lib.mwax_plan_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
    lib.mwax_plan_stage_times.restype = st
    lib.mwax_plan_autotune.argtypes = [vp, vp, vp, vp, ctypes.POINTER(Tuning)]
    lib.mwax_plan_autotune.restype = st
    lib.mwax_plan_set_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
    lib.mwax_plan_set_tuning.restype = st
    lib.mwax_plan_get_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
    lib.mwax_plan_get_tuning.restype = st
    lib.mwax_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int]
    lib.mwax_batch_create.restype = vp
    lib.mwax_batch_set_stream.argtypes = [vp, vp]
    lib.mwax_batch_set_stream.restype = st
    lib.mwax_batch_set_graphs.argtypes = [vp, ctypes.c_int]
    lib.mwax_batch_set_graphs.restype = st
    lib.mwax_batch_correlate.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp)]
    lib.mwax_batch_correlate.restype = st
    lib.mwax_batch_sync.argtypes = [vp]
    lib.mwax_batch_sync.restype = st
    lib.mwax_batch_destroy.argtypes = [vp]
    lib.mwax_batch_destroy.restype = None
    lib.mwax_server_create.argtypes = [ctypes.POINTER(_ServerDesc)]
    lib.mwax_server_create.restype = vp
    lib.mwax_server_submit.argtypes = [vp, ctypes.POINTER(_CDesc), vp, vp, vp, ctypes.c_double]
    lib.mwax_server_submit.restype = ctypes.c_longlong
    lib.mwax_server_poll.argtypes = [vp, ctypes.c_longlong]
    lib.mwax_server_poll.restype = ctypes.c_int
    lib.mwax_server_wait.argtypes = [vp, ctypes.c_longlong]
    lib.mwax_server_wait.restype = st
    lib.mwax_server_drain.argtypes = [vp]
    lib.mwax_server_drain.restype = st
    lib.mwax_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
    lib.mwax_server_get_stats.restype = st
    lib.mwax_server_reset_stats.argtypes = [vp]
    lib.mwax_server_reset_stats.restype = st
    lib.mwax_server_destroy.argtypes = [vp]
    lib.mwax_server_destroy.restype = None
    lib.mwax_correlate_noalloc.argtypes = [ctypes.POINTER(_CDesc), vp, vp, vp, vp]
    lib.mwax_correlate_noalloc.restype = st
    lib.mwax_correlate_ex.argtypes = [vp, ctypes.POINTER(_Call)]
    lib.mwax_correlate_ex.restype = st
    lib.mwax_plan_set_passband.argtypes = [vp, vp]
    lib.mwax_plan_set_passband.restype = st
    lib.mwax_beam_create.argtypes = [ctypes.POINTER(_BeamDesc)]
    lib.mwax_beam_create.restype = vp
    lib.mwax_beam_set_stream.argtypes = [vp, vp]
    lib.mwax_beam_set_stream.restype = st
    lib.mwax_beam_output_bytes.argtypes = [vp, ctypes.c_int]
    lib.mwax_beam_output_bytes.restype = ctypes.c_size_t
    lib.mwax_beam_form.argtypes = [vp, vp, vp, ctypes.c_longlong, vp, vp, vp]
    lib.mwax_beam_form.restype = st
    lib.mwax_beam_sync.argtypes = [vp]
    lib.mwax_beam_sync.restype = st
    lib.mwax_beam_destroy.argtypes = [vp]
    lib.mwax_beam_destroy.restype = None
    lib.mwax_version.argtypes = []
    lib.mwax_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


def mwax_last_error() -> str:
    return load_library().mwax_last_error().decode()


def mwax_version() -> str:
    return load_library().mwax_version().decode()


def _check(status: int):
    if status != MWAX_OK:
        raise MwaxError(status, mwax_last_error())


class Plan:
    """Owns one mwax_plan*; destroyed with the object."""

    def __init__(self, handle: int, desc: PlanDesc):
        self.handle = handle
        self.desc = desc

    @property
    def info(self) -> dict:
        """mwax_plan_info as a dict, read afresh (issued flops follow the tuning)."""
        info = _CInfo()
        _check(load_library().mwax_plan_get_info(self.handle, ctypes.byref(info)))
        return {k: getattr(info, k) for k, _ in _CInfo._fields_}

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.mwax_plan_destroy(h)

    def close(self):
        self.__del__()

    # convenience accessors
    n_ints = property(lambda self: self.info["n_ints"])
    n_baselines = property(lambda self: self.info["n_baselines"])
    n_chan_out = property(lambda self: self.info["n_chan_out"])
    output_bytes = property(lambda self: self.info["output_bytes"])
    input_bytes = property(lambda self: self.info["input_bytes"])


def mwax_plan_create(n_tiles: int, fft_len: int, int_time_s: float, fine_avg: int) -> Plan:
    h = load_library().mwax_plan_create(n_tiles, fft_len, int_time_s, fine_avg)
    if not h:
        raise MwaxError(MWAX_EINVAL, mwax_last_error())
    return Plan(h, PlanDesc(n_tiles, fft_len, fine_avg, int_time_s))


def mwax_plan_create_ex(desc: PlanDesc) -> Plan:
    cd = desc.c()
    h = load_library().mwax_plan_create_ex(ctypes.byref(cd))
    if not h:
        err = mwax_last_error()
        code = MWAX_EUNSUPPORTED if "not built" in err else MWAX_EINVAL
        raise MwaxError(code, err)
    return Plan(h, desc)


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _delay_arg(delay, plan: Plan, device: bool):
    """delay polynomial -> (pointer, keepalive).  float64 [n_paths, 3] host or device."""
    if delay is None:
        return None, None
    n = 2 * plan.desc.n_tiles
    if isinstance(delay, np.ndarray):
        d = np.ascontiguousarray(delay, dtype=np.float64)
        if d.size != 3 * n:
            raise ValueError("delay_poly must hold n_paths x 3 float64")
        return d.ctypes.data, d
    import torch
    if delay.dtype != torch.float64 or delay.numel() != 3 * n or not delay.is_contiguous():
        raise ValueError("delay_poly must be a contiguous float64 tensor of n_paths x 3")
    return delay.data_ptr(), delay


def mwax_plan_set_stream(plan: Plan, stream=None):
    """Enqueue the plan's work on a torch.cuda.Stream (default: torch's current stream)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(load_library().mwax_plan_set_stream(plan.handle, ctypes.c_void_p(s.cuda_stream)))


def mwax_correlate(plan: Plan, voltages, delay_poly, vis_out):
    """voltages: CUDA int8 tensor, plan.input_bytes; vis_out: CUDA tensor of plan.output_bytes."""
    if not voltages.is_cuda or not vis_out.is_cuda:
        raise ValueError("mwax_correlate takes device tensors; use mwax_correlate_host for host memory")
    if voltages.numel() * voltages.element_size() != plan.input_bytes or not voltages.is_contiguous():
        raise ValueError(f"voltages must be a contiguous buffer of {plan.input_bytes} bytes")
    if vis_out.numel() * vis_out.element_size() < plan.output_bytes:
        raise ValueError(f"vis_out must hold {plan.output_bytes} bytes")
    dptr, keep = _delay_arg(delay_poly, plan, True)
    _check(load_library().mwax_correlate(plan.handle, _ptr(voltages), dptr, _ptr(vis_out)))
    return keep


def mwax_correlate_host(plan: Plan, voltages, delay_poly, vis_out):
    """Host buffers (numpy or CPU tensors, pinned for full bandwidth); synchronous."""
    dptr, keep = _delay_arg(delay_poly, plan, False)
    _check(load_library().mwax_correlate_host(plan.handle, _ptr(voltages), dptr, _ptr(vis_out)))
    return keep


def mwax_correlate_host_async(plan: Plan, voltages, delay_poly, vis_out):
    """Streaming host call (pinned buffers): enqueue and return; the next call's upload
    overlaps this one's correlation.  Keep the buffers until mwax_plan_sync()."""
    dptr, keep = _delay_arg(delay_poly, plan, False)
    _check(load_library().mwax_correlate_host_async(plan.handle, _ptr(voltages), dptr, _ptr(vis_out)))
    return keep


def mwax_plan_sync(plan: Plan):
    _check(load_library().mwax_plan_sync(plan.handle))


def mwax_probe_fma(blocks: int, iters: int, sink, stream=None) -> int:
    """Enqueue the FP32 FMA throughput probe on the stream; returns the FMAs enqueued."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    n = load_library().mwax_probe_fma(blocks, iters, _ptr(sink), ctypes.c_void_p(s.cuda_stream))
    if n < 0:
        raise MwaxError(MWAX_EINVAL, "FMA probe launch failed")
    return n


def mwax_plan_set_wait_limit(plan: Plan, kilocycles: int):
    """Bound of the plan's device-side waits (x 1000 SM cycles; 0 = default ~1 s)."""
    _check(load_library().mwax_plan_set_wait_limit(plan.handle, kilocycles))


def mwax_plan_enable_timing(plan: Plan, enable: bool = True):
    _check(load_library().mwax_plan_enable_timing(plan.handle, int(bool(enable))))


STAGES = ("init", "fstep", "xstep")


def mwax_plan_stage_times(plan: Plan):
    """{stage: (milliseconds, launches)} since the last call (waits for the plan's stream)."""
    ms = (ctypes.c_double * 3)()
    n = (ctypes.c_longlong * 3)()
    _check(load_library().mwax_plan_stage_times(plan.handle, ms, n))
    return {STAGES[i]: (ms[i], n[i]) for i in range(3)}


def mwax_plan_autotune(plan: Plan, voltages, delay_poly, vis_out) -> Tuning:
    """Time the plan's launch choices on these device buffers and keep the fastest."""
    dptr, keep = _delay_arg(delay_poly, plan, True)
    t = Tuning()
    _check(load_library().mwax_plan_autotune(plan.handle, _ptr(voltages), dptr, _ptr(vis_out), ctypes.byref(t)))
    return t


def mwax_plan_set_tuning(plan: Plan, tuning: Tuning):
    _check(load_library().mwax_plan_set_tuning(plan.handle, ctypes.byref(tuning)))


def mwax_plan_get_tuning(plan: Plan) -> Tuning:
    t = Tuning()
    _check(load_library().mwax_plan_get_tuning(plan.handle, ctypes.byref(t)))
    return t


class Batch:
    """A set of plans correlated together (one persistent X-step launch per round, CUDA
    graph replay).  Keeps references to its plans."""

    def __init__(self, plans, stream=None, graphs: bool = True):
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p.handle for p in self.plans])
        h = load_library().mwax_batch_create(arr, len(self.plans))
        if not h:
            raise MwaxError(MWAX_EINVAL, mwax_last_error())
        self.handle = h
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(load_library().mwax_batch_set_stream(h, ctypes.c_void_p(s.cuda_stream)))
        _check(load_library().mwax_batch_set_graphs(h, int(graphs)))

    def correlate(self, voltages, delays, outs):
        n = len(self.plans)
        V = (ctypes.c_void_p * n)(*[_ptr(v) for v in voltages])
        O = (ctypes.c_void_p * n)(*[_ptr(o) for o in outs])
        D = None
        if delays is not None:
            D = (ctypes.c_void_p * n)(*[None if d is None else _ptr(d) for d in delays])
        _check(load_library().mwax_batch_correlate(self.handle, V, D, O))

    def sync(self):
        _check(load_library().mwax_batch_sync(self.handle))

    def close(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.mwax_batch_destroy(h)

    def __del__(self):
        self.close()


class Server:
    """Real-time serving loop (native scheduler thread in libmwax.so).  Host buffers
    passed to submit() are kept referenced until the request completes."""

    def __init__(self, hbm_budget: int = 0, n_lanes: int = 0, workspace_limit: int = 0):
        d = _ServerDesc(hbm_budget, n_lanes, workspace_limit)
        h = load_library().mwax_server_create(ctypes.byref(d))
        if not h:
            raise MwaxError(MWAX_ECUDA, mwax_last_error())
        self.handle = h
        self._keep = {}

    def submit(self, desc: PlanDesc, voltages, delay_poly, vis_out, deadline_s: float = 0.0) -> int:
        cd = desc.c()
        d = None
        if delay_poly is not None:
            d = np.ascontiguousarray(delay_poly, dtype=np.float64) if isinstance(delay_poly, np.ndarray) else delay_poly
        rid = load_library().mwax_server_submit(self.handle, ctypes.byref(cd), _ptr(voltages), _ptr(d), _ptr(vis_out),
                                                 deadline_s)
        if rid < 0:
            raise MwaxError(MWAX_EINVAL, mwax_last_error())
        self._keep[rid] = (voltages, d, vis_out)
        return rid

    def poll(self, rid: int) -> int:
        return load_library().mwax_server_poll(self.handle, rid)

    def wait(self, rid: int):
        _check(load_library().mwax_server_wait(self.handle, rid))
        self._keep.pop(rid, None)

    def drain(self):
        _check(load_library().mwax_server_drain(self.handle))
        self._keep.clear()

    def reset_stats(self):
        _check(load_library().mwax_server_reset_stats(self.handle))

    def stats(self) -> dict:
        st = ServerStats()
        _check(load_library().mwax_server_get_stats(self.handle, ctypes.byref(st)))
        return st.as_dict()

    def close(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.mwax_server_destroy(h)

    def __del__(self):
        self.close()


def mwax_correlate_noalloc(desc: PlanDesc, voltages, delay_poly, vis_out, stream=None):
    """Allocation-free FP32 call for small jobs (device buffers; see include/mwax.h)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    cd = desc.c()
    keep = delay_poly if delay_poly is None or not isinstance(delay_poly, np.ndarray) else \
        np.ascontiguousarray(delay_poly, dtype=np.float64)
    _check(load_library().mwax_correlate_noalloc(ctypes.byref(cd), _ptr(voltages), _ptr(keep), _ptr(vis_out),
                                                 ctypes.c_void_p(s.cuda_stream)))


def _array_arg(x, dtype):
    """(pointer, keepalive) of a numpy array (host) or torch tensor (host or device)."""
    if x is None:
        return None, None
    if isinstance(x, np.ndarray):
        a = np.ascontiguousarray(x, dtype=dtype)
        return a.ctypes.data, a
    if not x.is_contiguous():
        raise ValueError("tables and flags must be contiguous")
    return x.data_ptr(), x


def mwax_correlate_ex(plan: Plan, voltages, vis_out, delay_poly=None, delay_table=None, table_step_samples=0,
                      zero_flags=None, normalise=False):
    """Extended call: tabulated delays [n_paths, steps] (float64 s), zeroing flags
    [n_blocks, n_paths] (uint8) with occupancy weights, optional normalisation."""
    if not voltages.is_cuda or not vis_out.is_cuda:
        raise ValueError("mwax_correlate_ex takes device voltages and output")
    if voltages.numel() * voltages.element_size() != plan.input_bytes or not voltages.is_contiguous():
        raise ValueError(f"voltages must be a contiguous buffer of {plan.input_bytes} bytes")
    if vis_out.numel() * vis_out.element_size() < plan.output_bytes:
        raise ValueError(f"vis_out must hold {plan.output_bytes} bytes")
    dptr, keep_d = _delay_arg(delay_poly, plan, True)
    n = 2 * plan.desc.n_tiles
    tptr, keep_t = _array_arg(delay_table, np.float64)
    steps = 0
    if delay_table is not None:
        steps = (delay_table.size if isinstance(delay_table, np.ndarray) else delay_table.numel()) // n
        if steps * n != (delay_table.size if isinstance(delay_table, np.ndarray) else delay_table.numel()):
            raise ValueError("delay_table must hold n_paths x steps float64")
    fptr, keep_f = _array_arg(zero_flags, np.uint8)
    call = _Call(_ptr(voltages), dptr, tptr, steps, int(table_step_samples), fptr, int(bool(normalise)),
                 _ptr(vis_out))
    _check(load_library().mwax_correlate_ex(plan.handle, ctypes.byref(call)))
    return keep_d, keep_t, keep_f


def mwax_plan_set_passband(plan: Plan, gain=None):
    """De-ripple gains per ultrafine channel (float32 [fft_len], channel order), None = flat."""
    g = None if gain is None else np.ascontiguousarray(gain, dtype=np.float32)
    if g is not None and g.size != plan.desc.fft_len:
        raise ValueError("passband gain must hold fft_len values")
    _check(load_library().mwax_plan_set_passband(plan.handle, _ptr(g)))


class Beamformer:
    """Tied-array multibeam beamformer (Sec. 4.4); owns one mwax_beamformer*."""

    def __init__(self, n_tiles: int, fft_len: int, n_beams: int, samples_per_call: int, *, block_samples: int = 0,
                 sky_freq_hz: float = 0.0, sample_rate_hz: float = 0.0, table_step_samples: int = 0,
                 int_frames: int = 0, workspace_limit: int = 0, engine: int = 0):
        """engine: 0 = tensor cores (FP16 hi/lo pairs, FP32-level error), 1 = FP32 CUDA cores."""
        lib = load_library()
        self.desc = _BeamDesc(n_tiles, fft_len, n_beams, samples_per_call, block_samples, sky_freq_hz, sample_rate_hz,
                              table_step_samples, int_frames, workspace_limit, engine)
        h = lib.mwax_beam_create(ctypes.byref(self.desc))
        if not h:
            raise MwaxError(MWAX_EINVAL, mwax_last_error())
        self.handle = h
        self.n_paths, self.fft_len, self.n_beams = 2 * n_tiles, fft_len, n_beams
        self.frames = samples_per_call // fft_len
        self.n_det = self.frames // int_frames if int_frames else 0

    def set_stream(self, stream=None):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(load_library().mwax_beam_set_stream(self.handle, ctypes.c_void_p(s.cuda_stream)))

    def output_bytes(self, which: int) -> int:
        return load_library().mwax_beam_output_bytes(self.handle, which)

    def form(self, voltages, beam_delay, beams_out, power_out=None, incoh_out=None):
        """beam_delay: float64 [n_beams, n_paths, steps] (numpy or torch); outputs device tensors."""
        ptr, keep = _array_arg(beam_delay, np.float64)
        numel = beam_delay.size if isinstance(beam_delay, np.ndarray) else beam_delay.numel()
        steps = numel // (self.n_beams * self.n_paths)
        if steps < 1 or steps * self.n_beams * self.n_paths != numel:
            raise ValueError("beam_delay must hold n_beams x n_paths x steps float64")
        _check(load_library().mwax_beam_form(self.handle, _ptr(voltages), ptr, steps, _ptr(beams_out),
                                             _ptr(power_out), _ptr(incoh_out)))
        return keep

    def sync(self):
        _check(load_library().mwax_beam_sync(self.handle))

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.mwax_beam_destroy(h)


def mwax_plan_destroy(plan: Plan):
    plan.close()


def empty_output(plan: Plan, device=None):
    import torch
    return torch.empty(plan.output_bytes, dtype=torch.uint8, device=device or "cuda")


def split_output(plan: Plan, out):
    """Views of a call's output: (vis, weights).

    Float precisions: vis complex64 [ints, B, M, 4]; MWAX_INT8: vis int64 [ints, B, 4, 2].
    weights: float32 [ints, B, 4]."""
    info = plan.info
    n_ints, B, M = info["n_ints"], info["n_baselines"], info["n_chan_out"]
    per = info["vis_set_bytes"] + info["weights_bytes"]
    if isinstance(out, np.ndarray):
        raw = out.reshape(-1)[: n_ints * per].reshape(n_ints, per)
        vis_raw, w_raw = raw[:, : info["vis_set_bytes"]], raw[:, info["vis_set_bytes"]:]
        if info["precision"] == MWAX_INT8:
            vis = vis_raw.copy().view(np.int64).reshape(n_ints, B, 4, 2)
        else:
            vis = vis_raw.copy().view(np.complex64).reshape(n_ints, B, M, 4)
        return vis, w_raw.copy().view(np.float32).reshape(n_ints, B, 4)
    import torch
    raw = out.reshape(-1)[: n_ints * per].view(n_ints, per)
    vis_raw, w_raw = raw[:, : info["vis_set_bytes"]], raw[:, info["vis_set_bytes"]:]
    if info["precision"] == MWAX_INT8:
        vis = vis_raw.contiguous().view(torch.int64).view(n_ints, B, 4, 2)
    else:
        vis = vis_raw.contiguous().view(torch.float32).view(n_ints, B, M, 4, 2)
        vis = torch.view_as_complex(vis)
    return vis, w_raw.contiguous().view(torch.float32).view(n_ints, B, 4)
