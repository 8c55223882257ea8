"""Batched correlation (many coarse channels of mixed shapes and precisions in one
schedule with one persistent X-step launch per round and tensor-core kernel mode,
CUDA-graph replay) and the autotuner.  Each plan's result in the batch must equal its result alone, bit for bit,
and that result must match the FP64 oracle at its precision's bar (integer mode bit-exact);
the largest configuration shapes (512 tiles at N = 6400 and 1280) are checked on sampled
outputs."""
import numpy as np
import pytest

import oracle
import paper_2303_11557_b300 as mw
import synth
from _parity import (TOL_BY_PREC, check_output_vs_oracle, oracle_desc, parity_error, sample_requests,
                     sampled_error, workload)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# (tiles, N, fscrunch, integration s, samples per call, precision, workspace MB); small
# workspaces give some plans several launch groups (rounds) or split integrations
MIX = [
    (20, 128, 4, 0.05, 128_000, mw.MWAX_FP16, 12),
    (40, 32, 1, 0.025, 64_000, mw.MWAX_FP16, 8),
    (9, 640, 10, 0.1, 128_000, mw.MWAX_FP8, 1024),
    (66, 128, 1, 0.05, 64_000, mw.MWAX_FP16, 1024),
    (12, 64, 2, 0.05, 64_000, mw.MWAX_FP32, 4),
    (30, 1, 1, 0.025, 64_000, mw.MWAX_INT8, 1024),
    (70, 6400, 50, 0.05, 64_000, mw.MWAX_FP8, 1024),
    (24, 128, 4, 0.05, 128_000, mw.MWAX_FP16X3, 16),
    (16, 64, 2, 0.05, 64_000, mw.MWAX_FP16X3, 1024),   # two hi/lo plans: one launch, two jobs
    (20, 1, 1, 0.05, 64_000, mw.MWAX_INT8, 1024),      # two integer-mode plans likewise
]


def _inputs():
    vs, ds, plans, host = [], [], [], []
    for k, (T, N, F, t, S, prec, ws) in enumerate(MIX):
        volt, delay = workload(500 + k, T, S, delay=None if prec == mw.MWAX_INT8 else "quadratic")
        plans.append(mw.mwax_plan_create_ex(mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=t,
                                                        samples_per_call=S, precision=prec,
                                                        sky_freq_hz=synth.SKY_FREQ_HZ,
                                                        workspace_limit=ws << 20)))
        vs.append(torch.from_numpy(volt.reshape(-1)).cuda())
        ds.append(None if delay is None else torch.from_numpy(delay).cuda())
        host.append((volt, delay))
    return plans, vs, ds, host


def test_batch_equals_alone_and_graph_replay():
    plans, vs, ds, host = _inputs()
    alone = []
    for k, (p, v, d) in enumerate(zip(plans, vs, ds)):
        mw.mwax_plan_set_stream(p)
        o = mw.empty_output(p)
        o.fill_(0xAB)   # poison: every byte must be written
        mw.mwax_correlate(p, v, d, o)
        mw.mwax_plan_sync(p)
        alone.append(o.cpu().numpy().copy())
        # the result alone against the FP64 oracle (so batch == alone == oracle)
        T, N, F, t, S, prec, _ = MIX[k]
        vis, w = mw.split_output(p, alone[-1])
        check_output_vs_oracle(T, N, F, t, S, prec, host[k][0], host[k][1], vis, w)
    b = mw.Batch(plans)
    outs = [mw.empty_output(p) for p in plans]
    for call in range(3):                       # eager, capture + replay, replay
        for o in outs:
            o.fill_(0x77)
        b.correlate(vs, ds, outs)
        b.sync()
        for i, (o, ref) in enumerate(zip(outs, alone)):
            assert np.array_equal(o.cpu().numpy(), ref), f"plan {i} differs in batch call {call}"
    b.close()


def test_autotune_keeps_parity():
    T, N, F, t, S = 24, 128, 4, 0.05, 128_000
    volt, delay = workload(600, T, S, delay="linear")
    for prec, tol in ((mw.MWAX_FP16, 2e-3), (mw.MWAX_FP32, 1e-5), (mw.MWAX_FP16X3, 1e-5)):
        p = mw.mwax_plan_create_ex(mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=t, samples_per_call=S,
                                               precision=prec, sky_freq_hz=synth.SKY_FREQ_HZ))
        mw.mwax_plan_set_stream(p)
        v = torch.from_numpy(volt.reshape(-1)).cuda()
        d = torch.from_numpy(delay).cuda()
        o = mw.empty_output(p)
        best = mw.mwax_plan_autotune(p, v, d, o)
        assert best.ms > 0 and best.fstep_variant in (0, 1, 2) and best.window in (128, 256)
        got = mw.mwax_plan_get_tuning(p)
        assert (got.fstep_variant, got.run_len, got.window) == (best.fstep_variant, best.run_len, best.window)
        o.fill_(0)
        mw.mwax_correlate(p, v, d, o)
        mw.mwax_plan_sync(p)
        vis, _ = mw.split_output(p, o)
        ref, _ = oracle.correlate(oracle_desc(T, N, F, t, S), volt, delay)
        assert parity_error(vis.cpu().numpy(), ref, T).max() <= tol
        # every candidate choice is correct, not just the fastest
        for fv in (0, 1, 2):
            for w in (128, 256):
                for rl in (1, 3, 32):
                    mw.mwax_plan_set_tuning(p, mw.Tuning(fv, rl, w, 0.0))
                    mw.mwax_correlate(p, v, d, o)
                    mw.mwax_plan_sync(p)
                    vis, _ = mw.split_output(p, o)
                    assert parity_error(vis.cpu().numpy(), ref, T).max() <= tol


# configuration-shaped channels of the 24-channel batch: 512 tiles at the two large FFT
# lengths, 1 s of data each (0.5 / 0.25 s integrations), FP16 as the batch benchmark runs
BIG = [
    (512, 6400, 200, 0.5, 1_280_000, mw.MWAX_FP16),
    (512, 1280, 40, 0.25, 1_280_000, mw.MWAX_FP16),
    (128, 32, 1, 0.25, 1_280_000, mw.MWAX_FP16),
]


@pytest.mark.slow
def test_batch_config_shapes_sampled_vs_oracle():
    plans, vs, ds, host = [], [], [], []
    for k, (T, N, F, t, S, prec) in enumerate(BIG):
        volt, delay = workload(700 + k, T, S, delay="quadratic")
        plans.append(mw.mwax_plan_create_ex(mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=t,
                                                        samples_per_call=S, precision=prec,
                                                        sky_freq_hz=synth.SKY_FREQ_HZ)))
        vs.append(torch.from_numpy(volt.reshape(-1)).cuda())
        ds.append(torch.from_numpy(delay).cuda())
        host.append((volt, delay))
    b = mw.Batch(plans)
    outs = [mw.empty_output(p) for p in plans]
    for o in outs:
        o.fill_(0xAB)
    b.correlate(vs, ds, outs)
    b.sync()
    for k, (T, N, F, t, S, prec) in enumerate(BIG):
        vis, w = mw.split_output(plans[k], outs[k])
        vis = vis.cpu().numpy()
        assert np.all(w.cpu().numpy() == 1.0) and np.all(np.isfinite(vis))
        n_ints, M = vis.shape[0], vis.shape[2]
        req, n_main, tiles = sample_requests(0xB16 + k, T, [0, n_ints - 1], M, 16)
        want = oracle.correlate_sampled(oracle_desc(T, N, F, t, S), host[k][0], host[k][1], req)
        got = vis[req[:, 0], req[:, 1], req[:, 2], req[:, 3]]
        err = sampled_error(got, want, req, n_main, tiles, T)
        assert err.max() <= TOL_BY_PREC[prec], f"channel {k}: max err {err.max():.3e}"
    b.close()
    for p in plans:
        p.close()
