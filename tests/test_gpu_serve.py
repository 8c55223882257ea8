"""Serving loop: requests of mixed shapes and precisions (FP16 / FP8 / INT8 / FP32
selectable per request) submitted while others run are admitted as lanes and HBM free up;
every result must equal the same request run alone, bit for bit, and each request's result
alone must match the FP64 oracle at its precision's bar (integer mode bit-exact)."""
import numpy as np
import pytest

import paper_2303_11557_b300 as mw
import synth
from _parity import check_output_vs_oracle, workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

REQS = [
    (24, 128, 4, 0.05, 128_000, mw.MWAX_FP16),
    (10, 1, 1, 0.05, 128_000, mw.MWAX_INT8),
    (40, 640, 10, 0.1, 128_000, mw.MWAX_FP8),
    (24, 128, 4, 0.05, 128_000, mw.MWAX_FP16),
    (16, 32, 1, 0.025, 64_000, mw.MWAX_FP32),
    (60, 128, 4, 0.05, 64_000, mw.MWAX_FP16),
    (10, 1, 1, 0.05, 128_000, mw.MWAX_INT8),
    (24, 128, 4, 0.05, 128_000, mw.MWAX_FP16),
]


def _desc(T, N, F, t, S, prec):
    return mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=t, samples_per_call=S, precision=prec,
                       sky_freq_hz=synth.SKY_FREQ_HZ, workspace_limit=256 << 20)


@pytest.mark.parametrize("budget_mb,lanes", [(0, 4), (160, 3)])
def test_server_mix_equals_alone(budget_mb, lanes):
    inputs, alone = [], []
    for k, (T, N, F, t, S, prec) in enumerate(REQS):
        volt, delay = workload(900 + k, T, S, delay=None if prec == mw.MWAX_INT8 else "quadratic")
        hv = torch.from_numpy(volt.reshape(-1)).pin_memory()
        hd = None if delay is None else np.ascontiguousarray(delay)
        plan = mw.mwax_plan_create_ex(_desc(T, N, F, t, S, prec))
        mw.mwax_plan_set_stream(plan)
        o = mw.empty_output(plan)
        mw.mwax_correlate(plan, hv.cuda(), None if hd is None else torch.from_numpy(hd).cuda(), o)
        mw.mwax_plan_sync(plan)
        alone.append(o.cpu().numpy().copy())
        vis, w = mw.split_output(plan, alone[-1])
        check_output_vs_oracle(T, N, F, t, S, prec, volt, hd, vis, w)
        inputs.append((hv, hd, plan.output_bytes))
        plan.close()
    srv = mw.Server(hbm_budget=budget_mb << 20, n_lanes=lanes)
    outs, ids = [], []
    for k, ((T, N, F, t, S, prec), (hv, hd, ob)) in enumerate(zip(REQS, inputs)):
        out = torch.empty(ob, dtype=torch.uint8).pin_memory()
        outs.append(out)
        ids.append(srv.submit(_desc(T, N, F, t, S, prec), hv, hd, out, deadline_s=8.0))
    srv.drain()
    st = srv.stats()
    assert st["completed"] == len(REQS) and st["failed"] == 0 and st["queued"] == 0
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    for k, (o, ref) in enumerate(zip(outs, alone)):
        assert srv.poll(ids[k]) == 1
        assert np.array_equal(o.numpy(), ref), f"request {k} differs"
    srv.close()


def test_plan_cache_ignores_descriptor_padding():
    # The server caches plans per shape.  Three requests of one shape whose descriptors
    # differ only in their padding bytes (a C caller need not initialise those) must share
    # one plan: one cold start, the rest served from the cache.
    import ctypes
    T, N, F, t, S = 8, 128, 4, 0.05, 64_000
    desc = _desc(T, N, F, t, S, mw.MWAX_FP16)
    volt, _ = workload(990, T, S, delay=None)
    hv = torch.from_numpy(volt.reshape(-1)).pin_memory()
    plan = mw.mwax_plan_create_ex(desc)
    nbytes = plan.output_bytes
    plan.close()
    out = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    srv = mw.Server(n_lanes=1)
    lib = mw.load_library()
    src = desc.c()
    size = ctypes.sizeof(type(src))
    assert size > sum(ctypes.sizeof(ty) for _, ty in type(src)._fields_)   # the struct has padding
    keep = []
    for fill in (0x00, 0xFF, 0x5A):
        raw = (ctypes.c_ubyte * size)(*([fill] * size))
        cd = type(src).from_buffer(raw)
        for name, _ in type(src)._fields_:
            setattr(cd, name, getattr(src, name))
        keep.append(raw)
        rid = lib.mwax_server_submit(srv.handle, ctypes.byref(cd), ctypes.c_void_p(hv.data_ptr()), None,
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_double(8.0))
        assert rid >= 0
        srv.wait(rid)
    st = srv.stats()
    assert st["completed"] == 3 and st["failed"] == 0
    assert st["cold_starts"] == 1, st
    srv.close()
