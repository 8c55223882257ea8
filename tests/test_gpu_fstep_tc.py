"""The tensor-core F-steps (F-step variants 2, 3 and 4) against the FP64 oracle: the four-step
DFT (two DFT-matrix products on tcgen05, N = 80 x 80 = 6400 and 80 x 16 = 1280, FP16
operands out) and the 128-row F-step (stage A on tcgen05, a radix-5/2 stage B in registers,
N = 128 x 50 and 128 x 10) at the FP16 and FP8 bars, the direct DFT product (N = 32, 64,
128) in every float form at its bar, and the direct DFT with the frames on the accumulator
lanes (N = 32, 64, 128) at the FP16 and FP8 bars: frame counts that leave ragged items and items that straddle two
integrations or data blocks, per-path quadratic delays, zeroed data blocks, and the same
plan with the CUDA-core F-step for comparison."""
import numpy as np
import pytest

import oracle
import paper_2303_11557_b300 as mw
import synth
from _parity import oracle_desc, parity_error, workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {mw.MWAX_FP16: 2e-3, mw.MWAX_FP8: 3e-2}
PRECS = [pytest.param(mw.MWAX_FP16, id="fp16"), pytest.param(mw.MWAX_FP8, id="fp8")]


def _run(desc, volt, delay, variant, flags=None):
    plan = mw.mwax_plan_create_ex(desc)
    mw.mwax_plan_set_stream(plan)
    t = mw.mwax_plan_get_tuning(plan)
    mw.mwax_plan_set_tuning(plan, mw.Tuning(variant, t.run_len, t.window, 0.0))
    out = mw.empty_output(plan)
    out.fill_(0xAB)
    dv = torch.from_numpy(volt.reshape(-1)).cuda()
    dd = None if delay is None else torch.from_numpy(delay).cuda()
    if flags is None:
        mw.mwax_correlate(plan, dv, dd, out)
    else:
        mw.mwax_correlate_ex(plan, dv, out, delay_poly=dd, zero_flags=torch.from_numpy(flags).cuda())
    mw.mwax_plan_sync(plan)
    vis, w = mw.split_output(plan, out)
    res = vis.cpu().numpy(), w.cpu().numpy()
    plan.close()
    return res


VARIANTS = [pytest.param(2, id="fourstep"), pytest.param(3, id="row128")]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N,F,K", [(6400, 50, 203), (1280, 10, 203), (1280, 40, 250)])
def test_tensor_core_fstep_parity(variant, prec, N, F, K):
    # K frames per integration, 2 integrations: odd K leaves a frame pair (6400) split across
    # the integrations, K not a multiple of 8 leaves 8-frame groups (1280) that straddle them
    T = 6
    bs = K * N
    volt, delay = workload(0x7C + N + K, T, 2 * bs, block_samples=bs, delay="quadratic")
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=K * N / synth.FS, samples_per_call=2 * bs,
                       block_samples=bs, sky_freq_hz=synth.SKY_FREQ_HZ, precision=prec)
    vis, w = _run(desc, volt, delay, variant)
    ref, rw = oracle.correlate(oracle_desc(T, N, F, K * N / synth.FS, 2 * bs, block_samples=bs), volt, delay)
    assert np.array_equal(w, rw.astype(np.float32))
    err = parity_error(vis, ref, T)
    assert np.all(np.isfinite(vis)) and err.max() <= TOL[prec], f"max err {err.max():.3e}"
    # the CUDA-core F-step on the same plan: both within the bar, and close to each other
    vis0, _ = _run(desc, volt, delay, 0)
    assert parity_error(vis0, ref, T).max() <= TOL[prec]
    assert parity_error(vis, vis0.astype(np.complex128), T).max() <= TOL[prec]


@pytest.mark.parametrize("variant", VARIANTS)
def test_tensor_core_fstep_zeroed_blocks_and_many_paths(variant):
    # 40 tiles (80 paths: several path items per CTA), 10 blocks of 5 frames (N = 6400), a
    # seeded tenth of the blocks flagged as zeroed: the F-step reads them as zero
    T, N, F, K, bs = 40, 6400, 200, 50, 32_000
    S = 2 * K * N
    volt, delay = workload(0x7D, T, S, block_samples=bs, delay="quadratic")
    flags = (np.random.default_rng(7).random((S // bs, 2 * T)) < 0.1).astype(np.uint8)
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=K * N / synth.FS, samples_per_call=S,
                       block_samples=bs, sky_freq_hz=synth.SKY_FREQ_HZ, precision=mw.MWAX_FP16)
    vis, w = _run(desc, volt, delay, variant, flags=flags)
    ref, rw = oracle.correlate_ext(oracle_desc(T, N, F, K * N / synth.FS, S, block_samples=bs),
                                   oracle.Ext(zero_flags=flags), volt, delay)
    assert np.allclose(w, rw, atol=1e-6)
    err = parity_error(vis, ref, T)
    assert np.all(np.isfinite(vis)) and err.max() <= 2e-3, f"max err {err.max():.3e}"


# ---------------------------------------------------------------- direct-DFT tensor-core F-step
TOL_ALL = {mw.MWAX_FP32: 1e-5, mw.MWAX_FP16: 2e-3, mw.MWAX_FP8: 3e-2, mw.MWAX_FP16X3: 1e-5}
ALL_FLOAT = [pytest.param(mw.MWAX_FP32, id="fp32"), pytest.param(mw.MWAX_FP16, id="fp16"),
             pytest.param(mw.MWAX_FP8, id="fp8"), pytest.param(mw.MWAX_FP16X3, id="fp16x3")]


@pytest.mark.parametrize("prec", ALL_FLOAT)
@pytest.mark.parametrize("N,F,K,bs", [(128, 4, 200, 6400), (64, 2, 250, 16_000), (32, 1, 250, 8000)])
def test_direct_dft_fstep_parity(prec, N, F, K, bs):
    # 128-frame items straddle the two integrations (K is not a multiple of 128) and data
    # blocks smaller than an item (bulk copies split at block boundaries); per-path
    # quadratic delays; every float form (FP16 DFT matrix for FP16 / FP8 operands, an FP16
    # hi/lo pair for FP32 and hi/lo operands)
    T = 7
    S = 2 * K * N
    assert S % bs == 0
    volt, delay = workload(0x7E + N + prec, T, S, block_samples=bs, delay="quadratic")
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=K * N / synth.FS, samples_per_call=S,
                       block_samples=bs, sky_freq_hz=synth.SKY_FREQ_HZ, precision=prec)
    vis, w = _run(desc, volt, delay, 2)
    ref, rw = oracle.correlate(oracle_desc(T, N, F, K * N / synth.FS, S, block_samples=bs), volt, delay)
    assert np.array_equal(w, rw.astype(np.float32))
    err = parity_error(vis, ref, T)
    assert np.all(np.isfinite(vis)) and err.max() <= TOL_ALL[prec], f"max err {err.max():.3e}"


def test_direct_dft_fstep_zeroed_blocks_fp32():
    T, N, F, K, bs = 9, 128, 4, 400, 6400
    S = 2 * K * N
    volt, delay = workload(0x7F, T, S, block_samples=bs, delay="quadratic")
    flags = (np.random.default_rng(8).random((S // bs, 2 * T)) < 0.15).astype(np.uint8)
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=K * N / synth.FS, samples_per_call=S,
                       block_samples=bs, sky_freq_hz=synth.SKY_FREQ_HZ, precision=mw.MWAX_FP32)
    vis, w = _run(desc, volt, delay, 2, flags=flags)
    ref, rw = oracle.correlate_ext(oracle_desc(T, N, F, K * N / synth.FS, S, block_samples=bs),
                                   oracle.Ext(zero_flags=flags), volt, delay)
    assert np.allclose(w, rw, atol=1e-6)
    err = parity_error(vis, ref, T)
    assert np.all(np.isfinite(vis)) and err.max() <= 1e-5, f"max err {err.max():.3e}"


# ---------------------------------------------------------------- frames-on-lanes direct DFT
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N,F,K,bs", [(128, 4, 200, 6400), (64, 2, 250, 16_000), (32, 1, 250, 8000),
                                      (128, 4, 500, 64_000)])
def test_frames_on_lanes_fstep_parity(prec, N, F, K, bs):
    # F-step variant 4: 128-frame items straddle the two integrations and data blocks of
    # fewer than 128 frames (several copies per item); per-path quadratic delays
    T = 7
    S = 2 * K * N
    assert S % bs == 0
    volt, delay = workload(0x80 + N + prec + K, T, S, block_samples=bs, delay="quadratic")
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=K * N / synth.FS, samples_per_call=S,
                       block_samples=bs, sky_freq_hz=synth.SKY_FREQ_HZ, precision=prec)
    vis, w = _run(desc, volt, delay, 4)
    ref, rw = oracle.correlate(oracle_desc(T, N, F, K * N / synth.FS, S, block_samples=bs), volt, delay)
    assert np.array_equal(w, rw.astype(np.float32))
    err = parity_error(vis, ref, T)
    assert np.all(np.isfinite(vis)) and err.max() <= TOL[prec], f"max err {err.max():.3e}"


@pytest.mark.parametrize("prec", PRECS)
def test_frames_on_lanes_fstep_zeroed_blocks(prec):
    T, N, F, K, bs = 9, 128, 4, 400, 6400
    S = 2 * K * N
    volt, delay = workload(0x81, T, S, block_samples=bs, delay="quadratic")
    flags = (np.random.default_rng(9).random((S // bs, 2 * T)) < 0.15).astype(np.uint8)
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=K * N / synth.FS, samples_per_call=S,
                       block_samples=bs, sky_freq_hz=synth.SKY_FREQ_HZ, precision=prec)
    vis, w = _run(desc, volt, delay, 4, flags=flags)
    ref, rw = oracle.correlate_ext(oracle_desc(T, N, F, K * N / synth.FS, S, block_samples=bs),
                                   oracle.Ext(zero_flags=flags), volt, delay)
    assert np.allclose(w, rw, atol=1e-6)
    err = parity_error(vis, ref, T)
    assert np.all(np.isfinite(vis)) and err.max() <= TOL[prec], f"max err {err.max():.3e}"


@pytest.mark.parametrize("N,F,variant,per_call", [(128, 4, 0, lambda slots: 1), (128, 4, 4, lambda slots: 2),
                                                   (1280, 10, 3, lambda slots: 3 * slots)],
                         ids=["radix32", "frames-on-lanes", "row128"])
def test_fstep_kernel_count_per_call(N, F, variant, per_call):
    """The plan's launch count is the number of kernels: the frames-on-lanes F-step launches
    its frame-term kernel too, the 128-row F-step a frame-term kernel, the F kernel and the
    transpose per integration slot (two slots per call here, one launch group)."""
    T, bs = 4, 64_000
    S = 2 * bs
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=bs / synth.FS, samples_per_call=S,
                       block_samples=bs, sky_freq_hz=synth.SKY_FREQ_HZ, precision=mw.MWAX_FP16)
    plan = mw.mwax_plan_create_ex(desc)
    mw.mwax_plan_set_stream(plan)
    t = mw.mwax_plan_get_tuning(plan)
    mw.mwax_plan_set_tuning(plan, mw.Tuning(variant, t.run_len, t.window, 0.0))
    out = mw.empty_output(plan)
    volt = torch.from_numpy(synth.voltages(5, 2 * T, S, block_samples=bs).reshape(-1)).cuda()
    mw.mwax_plan_stage_times(plan)
    mw.mwax_correlate(plan, volt, None, out)
    counts = mw.mwax_plan_stage_times(plan)
    plan.close()
    assert counts["fstep"][1] == per_call(2)


def test_workspace_bytes_count_fstep_scratch():
    """The plan's reported device memory includes the F-step scratch: choosing the
    frames-on-lanes F-step adds its frame-term table (32 bytes per frame of a launch), and
    the 128-row F-step's plans hold theirs from creation."""
    T, bs = 4, 64_000
    S = 2 * bs
    desc = mw.PlanDesc(n_tiles=T, fft_len=128, fine_avg=4, int_time_s=bs / synth.FS, samples_per_call=S,
                       block_samples=bs, sky_freq_hz=synth.SKY_FREQ_HZ, precision=mw.MWAX_FP16)
    plan = mw.mwax_plan_create_ex(desc)
    w0 = plan.info["workspace_bytes"]
    t = mw.mwax_plan_get_tuning(plan)
    mw.mwax_plan_set_tuning(plan, mw.Tuning(4, t.run_len, t.window, 0.0))
    w1 = plan.info["workspace_bytes"]
    plan.close()
    frames = S // 128   # every frame of the call in one launch group
    assert w1 - w0 == 2 * T * ((frames + 127) // 128) * 128 * 32
    d2 = mw.PlanDesc(n_tiles=T, fft_len=1280, fine_avg=10, int_time_s=bs / synth.FS, samples_per_call=S,
                     block_samples=bs, sky_freq_hz=synth.SKY_FREQ_HZ, precision=mw.MWAX_FP16)
    p2 = mw.mwax_plan_create_ex(d2)
    info = p2.info
    p2.close()
    # operands: 2 slots x N x 2 planes x paths x Kpad (50 frames -> 128) x 2 bytes; the
    # scratch: one slot of frame-major tiles, 7 groups of 8 frames x N words per path
    operands = 2 * 1280 * 2 * (2 * T) * 128 * 2
    assert info["workspace_bytes"] >= operands + (2 * T) * 7 * 8 * 1280 * 4
