"""Integer mode (no FFT, 1.28 MHz channels): the tcgen05 path must equal the oracle's
exact int64 sums bit for bit."""
import numpy as np
import pytest

import oracle
import paper_2303_11557_b300 as mw
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def run_int8(T, int_time_s, n_samples, volt, block_samples=64_000, workspace_limit=0):
    desc = mw.PlanDesc(n_tiles=T, fft_len=1, fine_avg=1, int_time_s=int_time_s, samples_per_call=n_samples,
                       block_samples=block_samples, precision=mw.MWAX_INT8, workspace_limit=workspace_limit)
    plan = mw.mwax_plan_create_ex(desc)
    mw.mwax_plan_set_stream(plan)
    out = mw.empty_output(plan)
    out.fill_(0x5A)
    mw.mwax_correlate(plan, torch.from_numpy(volt.reshape(-1)).cuda(), None, out)
    mw.mwax_plan_sync(plan)
    vis, w = mw.split_output(plan, out)
    od = oracle.Desc(n_tiles=T, fft_len=1, fine_avg=1, int_frames=int(round(int_time_s * synth.FS)),
                     n_samples=n_samples, block_samples=block_samples)
    ref, rw = oracle.correlate_int(od, volt)
    return vis.cpu().numpy(), w.cpu().numpy(), ref, rw


@pytest.mark.parametrize("T,t_int,S", [(16, 0.05, 128_000), (100, 0.025, 64_000), (5, 0.1, 128_000)])
def test_int8_bit_exact(T, t_int, S):
    volt = synth.voltages(0xD00D + T, 2 * T, S, sigma=40.0, tones=synth.point_source_tones(T, sigma=40.0))
    vis, w, ref, rw = run_int8(T, t_int, S, volt)
    assert np.array_equal(vis, ref)
    assert np.all(w == 1.0)


def test_int8_ragged_chunks():
    # 64,000 - 1 sample integrations are not possible; use 12,800-sample integrations
    # (50 chunks of 256) in 3,200-sample blocks, plus a chunked workspace
    T, S, bs = 7, 64_000, 3_200
    volt = synth.voltages(77, 2 * T, S, block_samples=bs, sigma=30.0)
    vis, _, ref, _ = run_int8(T, 0.01, S, volt, block_samples=bs, workspace_limit=2 * 14 * 4000 * 2)
    assert np.array_equal(vis, ref)


def test_int8_worst_case_magnitude():
    # every sample -128 - 128i: each product contributes 2 * 128^2; 0.1 s sums reach
    # 4.19e9 > 2^31, exercising the exact chunk bound and the int64 output
    T, S = 3, 128_000
    volt = np.full((S // 64_000, 2 * T, 64_000, 2), -128, dtype=np.int8)
    vis, _, ref, _ = run_int8(T, 0.1, S, volt)
    assert np.array_equal(vis, ref)
    assert ref[0, 0, 0, 0] == 128_000 * 2 * 128 * 128
