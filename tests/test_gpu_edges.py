"""Edge sizes of the array: one tile (two signal paths, a single baseline holding the two
autos and the xy cross) against the full oracle, and 512 tiles (1,024 paths, the largest
array of the serving mix; 524,800 path pairs) against per-output oracle samples.  Same
bars as the other parity tests; the integer mode bit-exact."""
import numpy as np
import pytest

import oracle
import paper_2303_11557_b300 as mw
import synth
from _parity import oracle_desc, parity_error, sample_requests, sampled_error, workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {mw.MWAX_FP32: 1e-5, mw.MWAX_FP16: 2e-3, mw.MWAX_FP8: 3e-2, mw.MWAX_FP16X3: 1e-5}
FLOAT = [pytest.param(mw.MWAX_FP32, id="fp32"), pytest.param(mw.MWAX_FP16, id="fp16"),
         pytest.param(mw.MWAX_FP8, id="fp8"), pytest.param(mw.MWAX_FP16X3, id="fp16x3")]


def run(desc, volt, delay):
    plan = mw.mwax_plan_create_ex(desc)
    mw.mwax_plan_set_stream(plan)
    out = mw.empty_output(plan)
    out.fill_(0xAB)
    dd = None if delay is None else torch.from_numpy(np.ascontiguousarray(delay)).cuda()
    mw.mwax_correlate(plan, torch.from_numpy(volt.reshape(-1)).cuda(), dd, out)
    mw.mwax_plan_sync(plan)
    vis, w = mw.split_output(plan, out)
    res = vis.cpu().numpy(), w.cpu().numpy()
    plan.close()
    return res


@pytest.mark.parametrize("prec", FLOAT)
def test_one_tile(prec):
    T, N, F, t, S = 1, 64, 2, 0.05, 128_000
    volt, delay = workload(70, T, S, delay="linear")
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=t, samples_per_call=S,
                       sky_freq_hz=synth.SKY_FREQ_HZ, precision=prec)
    vis, w = run(desc, volt, delay)
    ref, rw = oracle.correlate(oracle_desc(T, N, F, t, S), volt, delay)
    assert vis.shape == ref.shape == (2, 1, N // F, 4) and np.all(w == 1.0)
    assert parity_error(vis, ref, T).max() <= TOL[prec]
    assert np.all(vis[..., [0, 3]].imag == 0)


def test_one_tile_int8():
    T, S = 1, 64_000
    volt = synth.voltages(71, 2 * T, S, sigma=40.0)
    desc = mw.PlanDesc(n_tiles=T, fft_len=1, fine_avg=1, int_time_s=0.025, samples_per_call=S,
                       precision=mw.MWAX_INT8)
    vis, _ = run(desc, volt, None)
    ref, _ = oracle.correlate_int(oracle.Desc(n_tiles=T, fft_len=1, fine_avg=1, int_frames=32_000, n_samples=S), volt)
    assert np.array_equal(vis, ref)


@pytest.fixture(scope="module")
def array_512():
    T, S = 512, 64_000
    volt, delay = workload(72, T, S, delay="linear")
    return T, S, volt, delay


@pytest.mark.parametrize("prec", FLOAT)
def test_512_tiles_sampled(prec, array_512):
    T, S, volt, delay = array_512
    N, F, t = 32, 2, 0.025              # 1000 frames per integration, 2 integrations
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=t, samples_per_call=S,
                       sky_freq_hz=synth.SKY_FREQ_HZ, precision=prec)
    vis, w = run(desc, volt, delay)
    assert vis.shape == (2, T * (T + 1) // 2, N // F, 4) and np.all(w == 1.0)
    req, n_main, tiles = sample_requests(0x512 + prec, T, [0, 1], N // F, 40)
    want = oracle.correlate_sampled(oracle_desc(T, N, F, t, S), volt, delay, req)
    got = vis[req[:, 0], req[:, 1], req[:, 2], req[:, 3]]
    err = sampled_error(got, want, req, n_main, tiles, T)
    assert np.all(np.isfinite(got)) and err.max() <= TOL[prec], f"max err {err.max():.3e}"


def test_512_tiles_int8_sampled(array_512):
    T, S, volt, _ = array_512
    desc = mw.PlanDesc(n_tiles=T, fft_len=1, fine_avg=1, int_time_s=0.025, samples_per_call=S,
                       precision=mw.MWAX_INT8)
    vis, _ = run(desc, volt, None)               # int64 [ints, B, 4, 2]
    req, n_main, _ = sample_requests(0x5128, T, [0, 1], 1, 40)
    req = req[:n_main]
    want = oracle.correlate_sampled(oracle.Desc(n_tiles=T, fft_len=1, fine_avg=1, int_frames=32_000, n_samples=S),
                                    volt, None, req)
    got = vis[req[:, 0], req[:, 1], req[:, 3]]
    assert np.array_equal(got[:, 0], want.real.astype(np.int64))
    assert np.array_equal(got[:, 1], want.imag.astype(np.int64))


@pytest.mark.parametrize("prec,issued_pairs,frames", [
    (mw.MWAX_FP32, 64 * 64 * 23 // 32, 4000),    # one diagonal 64 x 64 tile, 9 of 32 sub-blocks skipped
    (mw.MWAX_FP16, 128 * 128, 4000),            # one 128 x 128 MMA tile (rows and columns past n = 32)
    (mw.MWAX_FP8, 128 * 128, 4032),             # K blocks of 64 frames
    (mw.MWAX_FP16X3, 128 * 128, 4000)])
def test_plan_info_flop_counts(prec, issued_pairs, frames):
    # 16 tiles, 0.4 s, N = 128, F = 1: 528 unique pairs, 4,000 frames, 128 channels each
    # fed by one bin (no run shares a boundary channel)
    plan = mw.mwax_plan_create_ex(mw.PlanDesc(n_tiles=16, fft_len=128, fine_avg=1, int_time_s=0.4,
                                              samples_per_call=512_000, precision=prec))
    info = plan.info
    assert info["x_flop_alg"] == 8.0 * 528 * 4000 * 128
    assert info["x_flop_issued"] == 8.0 * issued_pairs * frames * 128
    plan.close()
