"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by element
on the same seeded inputs.  Bar (per result, relative to the parallel-pol autos of the
same channel and integration): FP32 <= 1e-5, FP16 (tcgen05) <= 2e-3, FP8-e4m3 (tcgen05,
per-path-per-channel-group scales) <= 3e-2."""
import numpy as np
import pytest

import oracle
import paper_2303_11557_b300 as mw
import synth
from _parity import oracle_desc, parity_error, workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# FP16 hi/lo pairs (three tensor-core products per term, chunked two-level sums) are held to
# the FP32 bar
TOL = {mw.MWAX_FP32: 1e-5, mw.MWAX_FP16: 2e-3, mw.MWAX_FP8: 3e-2, mw.MWAX_FP16X3: 1e-5}
FLOAT_PRECS = [pytest.param(mw.MWAX_FP32, id="fp32"), pytest.param(mw.MWAX_FP16, id="fp16"),
               pytest.param(mw.MWAX_FP8, id="fp8"), pytest.param(mw.MWAX_FP16X3, id="fp16x3")]


def run_gpu(desc: mw.PlanDesc, volt: np.ndarray, delay):
    plan = mw.mwax_plan_create_ex(desc)
    mw.mwax_plan_set_stream(plan)
    dv = torch.from_numpy(volt.reshape(-1)).cuda()
    out = mw.empty_output(plan)
    out.fill_(0xAB)   # poison: every byte must be written
    dd = None if delay is None else torch.from_numpy(np.ascontiguousarray(delay, dtype=np.float64)).cuda()
    mw.mwax_correlate(plan, dv, dd, out)
    mw.mwax_plan_sync(plan)
    vis, w = mw.split_output(plan, out)
    return vis.cpu().numpy(), w.cpu().numpy(), plan


def check(desc, volt, delay, tol=None):
    vis, w, plan = run_gpu(desc, volt, delay)
    od = oracle_desc(desc.n_tiles, desc.fft_len, desc.fine_avg, desc.int_time_s, volt.shape[0] * volt.shape[2],
                     block_samples=volt.shape[2], sky=desc.sky_freq_hz, keep_dc=desc.keep_dc)
    ref, rw = oracle.correlate(od, volt, delay)
    assert vis.shape == ref.shape
    assert np.array_equal(w, rw.astype(np.float32))
    err = parity_error(vis, ref, desc.n_tiles)
    tol = tol or TOL[desc.precision]
    assert np.all(np.isfinite(vis))
    assert err.max() <= tol, f"max err {err.max():.3e} (median {np.median(err):.3e})"
    # autos: XX/YY imaginary parts are exactly zero, real parts non-negative
    T = desc.n_tiles
    ab = [i * (2 * T - i + 1) // 2 for i in range(T)]
    assert np.all(vis[:, ab][..., [0, 3]].imag == 0)
    assert np.all(vis[:, ab][..., [0, 3]].real >= 0)
    return err


@pytest.mark.parametrize("prec", FLOAT_PRECS)
def test_16_tiles_0p4s_no_averaging(prec):
    # 16 tiles x 2 pols, 0.4 s at 1.28 MS/s, 128-point FFT, no averaging, fixed 0-50 ns delays
    T, N, F, t_int = 16, 128, 1, 0.4
    volt, delay = workload(0x4D574158, T, 512_000)
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=t_int, samples_per_call=512_000,
                       sky_freq_hz=synth.SKY_FREQ_HZ, precision=prec)
    check(desc, volt, delay)


@pytest.mark.parametrize("prec", FLOAT_PRECS)
@pytest.mark.parametrize("T", [40, 100])
def test_ragged_tiles_and_averaging(prec, T):
    # 80 / 200 paths: full tile blocks plus a ragged one; even fscrunch, 2 integrations
    N, F, t_int = 32, 4, 0.1
    volt, delay = workload(7, T, 256_000, delay="linear")
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=t_int, samples_per_call=256_000,
                       sky_freq_hz=synth.SKY_FREQ_HZ, precision=prec)
    check(desc, volt, delay)


@pytest.mark.parametrize("prec", FLOAT_PRECS)
def test_ragged_frames_odd_fscrunch_keep_dc(prec):
    # 1000 frames per integration (not a multiple of the frame chunks), F = 2, DC kept
    T, N, F, t_int = 5, 16, 2, 0.0125
    volt, delay = workload(8, T, 64_000, block_samples=16_000, delay="linear")
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=t_int, samples_per_call=64_000,
                       block_samples=16_000, sky_freq_hz=synth.SKY_FREQ_HZ, keep_dc=1, precision=prec)
    check(desc, volt, delay)


@pytest.mark.parametrize("prec", FLOAT_PRECS)
def test_odd_frames_per_integration(prec):
    # 201 frames per integration: frame pairs straddle the integrations' boundary at odd K
    # indices (the FP16 store pairs neighbouring frames only inside one slot at even K)
    T, N, F, K = 5, 128, 4, 201
    bs = K * N
    volt, delay = workload(13, T, 2 * bs, block_samples=bs, delay="linear")
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=K * N / synth.FS, samples_per_call=2 * bs,
                       block_samples=bs, sky_freq_hz=synth.SKY_FREQ_HZ, precision=prec)
    check(desc, volt, delay)


@pytest.mark.parametrize("prec", FLOAT_PRECS)
@pytest.mark.parametrize("N,F", [(16, 1), (32, 1), (64, 8), (128, 4), (256, 1), (512, 16), (640, 5), (1280, 10),
                                 (3200, 64), (6400, 50)])
def test_fft_lengths(N, F, prec):
    # e4m3 rounding is ~3.6 % rms per element and averages down as 1/sqrt(frames x bins):
    # the FP8 cases get 200 frames (about 1 % expected error) instead of 40
    T, K = 3, (200 if prec == mw.MWAX_FP8 else 40)
    bs = K * N
    volt, delay = workload(100 + N, T, 2 * bs, block_samples=bs, delay="linear")
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=K * N / synth.FS, samples_per_call=2 * bs,
                       block_samples=bs, sky_freq_hz=synth.SKY_FREQ_HZ, precision=prec)
    check(desc, volt, delay)


@pytest.mark.parametrize("prec", FLOAT_PRECS)
@pytest.mark.parametrize("N,F", [(128, 4), (1280, 10)])
def test_quadratic_per_path_delays(prec, N, F):
    # tau_p(t) = c0 + c1 t + c2 t^2 evaluated in FP64 at every frame centre (Sec. 4.3), a
    # different polynomial on every signal path (x and y of one tile differ), through both
    # FFT kernel families (two-pass radix-32 at N = 128, generic Stockham at N = 1280);
    # 1.6 s of data so the c2 t^2 terms reach 20 ns, i.e. ~18 rad of fringe at 139.5 MHz
    T, t_int, S = 24, 0.4, 2_048_000
    if N not in _QUAD:   # one workload and oracle run per N, shared by the four forms
        volt, delay = workload(0xC2 + N, T, S, delay="quadratic")
        _QUAD[N] = (volt, delay, oracle.correlate(oracle_desc(T, N, F, t_int, S), volt, delay)[0])
    volt, delay, ref = _QUAD[N]
    assert np.all(delay[0::2] != delay[1::2]) and np.abs(delay[:, 2]).max() * 1.6 ** 2 > 10e-9
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=t_int, samples_per_call=S,
                       sky_freq_hz=synth.SKY_FREQ_HZ, precision=prec)
    vis, _, plan = run_gpu(desc, volt, delay)
    err = parity_error(vis, ref, T)
    assert np.all(np.isfinite(vis)) and err.max() <= TOL[prec], f"max err {err.max():.3e}"
    plan.close()


_QUAD = {}


@pytest.mark.parametrize("prec", [pytest.param(mw.MWAX_FP32, id="fp32"), pytest.param(mw.MWAX_FP16X3, id="fp16x3")])
def test_one_8s_integration(prec):
    # the longest integration of the configurations: 80,000 frames of 128 points summed into
    # each visibility (FP32 bar: the two-level sums of both FP32-level forms must hold it
    # over 16x the frames of the 0.5 s cases)
    T, N, F, t_int, S = 6, 128, 4, 8.0, 10_240_000
    volt, delay = workload(15, T, S, delay="linear")
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=t_int, samples_per_call=S,
                       sky_freq_hz=synth.SKY_FREQ_HZ, precision=prec)
    check(desc, volt, delay)


@pytest.mark.parametrize("prec", FLOAT_PRECS)
def test_no_delay_and_zero_delay_identical(prec):
    T, N = 4, 64
    volt, _ = workload(9, T, 64_000, delay=None)
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=2, int_time_s=0.05, sky_freq_hz=synth.SKY_FREQ_HZ,
                       precision=prec)
    a, _, _ = run_gpu(desc, volt, None)
    b, _, _ = run_gpu(desc, volt, np.zeros((2 * T, 3)))
    assert np.array_equal(a, b)
    check(desc, volt, None)


@pytest.mark.parametrize("prec", FLOAT_PRECS)
@pytest.mark.parametrize("limit_frames", [1, 0])
def test_workspace_grouping_and_chunking(limit_frames, prec):
    # limit_frames=1: two integrations per launch group; 0: each integration split in
    # chunks of 896 frames (4000 = 4 x 896 + 416: a short, zero-padded last chunk)
    T, N, F = 6, 32, 2
    volt, delay = workload(10, T, 512_000, delay="linear")
    elem = {mw.MWAX_FP32: 4, mw.MWAX_FP16: 2, mw.MWAX_FP8: 1, mw.MWAX_FP16X3: 4}[prec]
    per_frame = N * 2 * (2 * T) * elem
    K = 4000
    limit = (2 * ((K + 127) // 128 * 128) * per_frame) if limit_frames else 1000 * per_frame
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=0.1, samples_per_call=512_000,
                       sky_freq_hz=synth.SKY_FREQ_HZ, workspace_limit=limit, precision=prec)
    check(desc, volt, delay)


@pytest.mark.parametrize("prec", FLOAT_PRECS)
def test_no_fft_float_mode(prec):
    T = 3
    volt, delay = workload(11, T, 64_000, delay="linear")
    desc = mw.PlanDesc(n_tiles=T, fft_len=1, fine_avg=1, int_time_s=0.0125, samples_per_call=64_000,
                       sky_freq_hz=synth.SKY_FREQ_HZ, precision=prec)
    check(desc, volt, delay)


def test_host_path_matches_device_path():
    T, N, F = 8, 128, 4
    volt, delay = workload(12, T, 640_000, delay="linear")
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=0.25, samples_per_call=640_000,
                       sky_freq_hz=synth.SKY_FREQ_HZ)
    vis_d, w_d, plan = run_gpu(desc, volt, delay)
    host_out = torch.empty(plan.output_bytes, dtype=torch.uint8).pin_memory()
    host_in = torch.from_numpy(volt.reshape(-1)).pin_memory()
    mw.mwax_correlate_host(plan, host_in, np.ascontiguousarray(delay), host_out)
    vis_h, w_h = mw.split_output(plan, host_out.numpy())
    assert np.array_equal(vis_h, vis_d) and np.array_equal(w_h, w_d)


def test_host_async_two_in_flight():
    # streaming host calls: three sub-observations enqueued back to back (the staging sets
    # alternate, the third reuses the first's), each equal to the device path on its input
    T, N, F = 8, 128, 4
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=0.25, samples_per_call=640_000,
                       sky_freq_hz=synth.SKY_FREQ_HZ)
    inputs = [workload(20 + k, T, 640_000, delay="linear") for k in range(3)]
    want = [run_gpu(desc, v, d)[0] for v, d in inputs]
    plan = mw.mwax_plan_create_ex(desc)
    mw.mwax_plan_set_stream(plan)
    hins = [torch.from_numpy(v.reshape(-1)).pin_memory() for v, _ in inputs]
    houts = [torch.zeros(plan.output_bytes, dtype=torch.uint8).pin_memory() for _ in inputs]
    keep = [mw.mwax_correlate_host_async(plan, hins[k], np.ascontiguousarray(inputs[k][1]), houts[k])
            for k in range(3)]
    mw.mwax_plan_sync(plan)
    for k in range(3):
        vis, _ = mw.split_output(plan, houts[k].numpy())
        assert np.array_equal(vis, want[k])
    del keep


@pytest.mark.parametrize("prec", [pytest.param(mw.MWAX_FP16, id="fp16"), pytest.param(mw.MWAX_FP8, id="fp8"),
                                  pytest.param(mw.MWAX_FP16X3, id="fp16x3")])
@pytest.mark.parametrize("run_len", [1, 5])
def test_tensor_core_window_128(prec, run_len):
    # 128-column tiles: the persistent X-step alternates two TMEM accumulator pairs (the
    # MMAs of a group run while the previous group is drained); 40 tiles = 80 paths give
    # several 128 x 128 tiles and a ragged one; FP8 needs >= 200 frames (see test_fft_lengths).
    # The hi/lo pair form always runs 128-column tiles; here with short runs.
    T, N, F, t_int = 80, 64, 2, 0.01
    volt, delay = workload(14, T, 64_000, block_samples=6400, delay="linear")
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=t_int, samples_per_call=64_000,
                       block_samples=6400, sky_freq_hz=synth.SKY_FREQ_HZ, precision=prec)
    plan = mw.mwax_plan_create_ex(desc)
    mw.mwax_plan_set_stream(plan)
    t0 = mw.mwax_plan_get_tuning(plan)
    mw.mwax_plan_set_tuning(plan, mw.Tuning(t0.fstep_variant, run_len, 128, 0.0))
    dv = torch.from_numpy(volt.reshape(-1)).cuda()
    out = mw.empty_output(plan)
    out.fill_(0xAB)
    mw.mwax_correlate(plan, dv, torch.from_numpy(delay).cuda(), out)
    mw.mwax_plan_sync(plan)
    vis, w = mw.split_output(plan, out)
    vis = vis.cpu().numpy()
    ref, _ = oracle.correlate(oracle_desc(T, N, F, t_int, 64_000, block_samples=6400), volt, delay)
    err = parity_error(vis, ref, T)
    assert np.all(np.isfinite(vis)) and err.max() <= TOL[prec], f"max err {err.max():.3e}"
    plan.close()
