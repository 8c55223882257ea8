"""GPU parity of the roadmap extensions (Sec. 2.4, 4.1-4.3, 4.5) through the C ABI against
the FP64 oracle's extended correlation, on seeded inputs: zeroing flags with occupancy
weights and normalisation, tabulated 5 ms-style delays, passband de-ripple gains and
oversampled coarse channels.  Same bars as the base parity tests (FP32 and FP16 hi/lo pairs
1e-5, FP16 2e-3 of the autos; int8 bit-exact); weights to FP32 rounding of the exact
fractions."""
import numpy as np
import pytest

import oracle
import paper_2303_11557_b300 as mw
import synth
from _parity import workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {mw.MWAX_FP32: 1e-5, mw.MWAX_FP16: 2e-3, mw.MWAX_FP16X3: 1e-5}


def ext_parity(vis, ref, T):
    """parity_error over the extended output; entries whose oracle autos are zero (paths
    fully flagged) must be exactly zero on both sides and are left out of the metric."""
    auto_b = np.array([i * (2 * T - i + 1) // 2 for i in range(T)])
    ti = np.concatenate([[i] * (T - i) for i in range(T)])
    tj = np.concatenate([np.arange(i, T) for i in range(T)])
    errs = []
    for pol in range(4):
        a, e = pol >> 1, pol & 1
        ap = np.abs(ref[..., 3 * a].real)[:, auto_b[ti], :]
        aq = np.abs(ref[..., 3 * e].real)[:, auto_b[tj], :]
        den = np.sqrt(ap * aq)
        zero = den == 0
        assert np.all(ref[..., pol][zero] == 0) and np.all(vis[..., pol][zero] == 0)
        errs.append((np.abs(vis[..., pol] - ref[..., pol])[~zero] / den[~zero]))
    return np.concatenate(errs)


def run_ex(desc, volt, **kw):
    plan = mw.mwax_plan_create_ex(desc)
    mw.mwax_plan_set_stream(plan)
    if "passband" in kw:
        mw.mwax_plan_set_passband(plan, kw.pop("passband"))
    dv = torch.from_numpy(volt.reshape(-1)).cuda()
    out = mw.empty_output(plan)
    out.fill_(0xAB)
    for k in ("delay_poly", "delay_table", "zero_flags"):
        if kw.get(k) is not None and kw.pop(f"{k}_on_device", True):
            kw[k] = torch.from_numpy(np.ascontiguousarray(kw[k])).cuda()
        kw.pop(f"{k}_on_device", None)
    keep = mw.mwax_correlate_ex(plan, dv, out, **kw)
    mw.mwax_plan_sync(plan)
    del keep
    vis, w = mw.split_output(plan, out)
    return vis.cpu().numpy(), w.cpu().numpy()


def odesc(desc, volt):
    fs = desc.sample_rate_hz or synth.FS
    K = int(round(desc.int_time_s * fs)) // desc.fft_len
    return oracle.Desc(n_tiles=desc.n_tiles, fft_len=desc.fft_len, fine_avg=desc.fine_avg, int_frames=K,
                       n_samples=volt.shape[0] * volt.shape[2], block_samples=volt.shape[2],
                       sky_freq_hz=desc.sky_freq_hz, dc_exclude=0 if desc.keep_dc else 1)


def flags_for(seed, n_blocks, n_paths, frac=0.15, dead=None):
    rng = np.random.default_rng(seed)
    f = (rng.random((n_blocks, n_paths)) < frac).astype(np.uint8)
    if dead is not None:
        blocks, path = dead
        f[blocks, path] = 1
    return f


@pytest.mark.parametrize("prec", [mw.MWAX_FP32, mw.MWAX_FP16, mw.MWAX_FP16X3], ids=["fp32", "fp16", "fp16x3"])
@pytest.mark.parametrize("normalise", [0, 1], ids=["raw", "normalised"])
def test_zero_flags_weights(prec, normalise):
    # 5 ms blocks, 0.1 s integrations: 20 blocks per integration; path 5 dead for all of
    # integration 1, 15 % of the other blocks zeroed, garbage left under the flags
    T, N, F, bs = 8, 128, 4, 6400
    S = 2 * 128_000
    volt, delay = workload(0x4D574159, T, S, block_samples=bs, delay="linear")
    flags = flags_for(3, S // bs, 2 * T, dead=(slice(20, 40), 5))
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=0.1, samples_per_call=S, block_samples=bs,
                       sky_freq_hz=synth.SKY_FREQ_HZ, precision=prec)
    vis, w = run_ex(desc, volt, delay_poly=delay, zero_flags=flags, normalise=normalise)
    ref, rw = oracle.correlate_ext(odesc(desc, volt), oracle.Ext(zero_flags=flags, normalise=normalise), volt, delay)
    np.testing.assert_allclose(w, rw, rtol=1e-7, atol=0)
    assert (rw == 0).any() and (rw < 1).mean() > 0.5          # the flags do bite
    err = ext_parity(vis, ref, T)
    assert err.max() <= TOL[prec], f"max err {err.max():.3e}"


def test_zero_flags_int8_exact():
    T, bs = 8, 6400
    S = 4 * 32_000
    volt, _ = workload(7, T, S, block_samples=bs, delay=None, sigma=40.0)
    flags = flags_for(9, S // bs, 2 * T, frac=0.2, dead=(slice(5, 10), 3))
    desc = mw.PlanDesc(n_tiles=T, fft_len=1, fine_avg=1, int_time_s=0.025, samples_per_call=S, block_samples=bs,
                       precision=mw.MWAX_INT8)
    vis, w = run_ex(desc, volt, zero_flags=flags, zero_flags_on_device=False)
    ref, rw = oracle.correlate_int_ext(odesc(desc, volt), oracle.Ext(zero_flags=flags), volt)
    assert np.array_equal(vis, ref)
    np.testing.assert_allclose(w, rw, rtol=1e-7, atol=0)


@pytest.mark.parametrize("N,bs", [(128, 64_000), (512, 64_000), (640, 64_000), (1, 6400)],
                         ids=["N128", "N512-straddling", "N640-generic", "N1-unpack"])
def test_delay_table(N, bs):
    # one fractional delay per path per 5 ms step, varying step to step (fringe stopping,
    # Sec. 4.3); at N = 512 frames straddle steps and take the one holding their centre
    T = 8
    S = 2 * 128_000 if N > 1 else 2 * 64_000
    F = 4 if N > 1 else 1
    t_int = 0.1 if N > 1 else 0.05
    volt, _ = workload(0x4D574158 + N, T, S, block_samples=bs, delay="linear")
    steps = S // 6400
    rng = np.random.default_rng(N)
    tab = rng.uniform(0, 50e-9, (2 * T, 1)) + rng.uniform(-2e-9, 2e-9, (2 * T, steps)).cumsum(axis=1)
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=t_int, samples_per_call=S, block_samples=bs,
                       sky_freq_hz=synth.SKY_FREQ_HZ)
    vis, w = run_ex(desc, volt, delay_table=tab, table_step_samples=6400)
    ref, _ = oracle.correlate_ext(odesc(desc, volt), oracle.Ext(delay_table=tab, table_step=6400), volt, None)
    err = ext_parity(vis, ref, T)
    assert err.max() <= TOL[mw.MWAX_FP32], f"max err {err.max():.3e}"
    assert np.all(w == 1.0)


def test_delay_table_from_host_fp16():
    T, N, S = 8, 128, 128_000
    volt, _ = workload(31, T, S, delay="linear")
    tab = np.random.default_rng(1).uniform(0, 50e-9, (2 * T, S // 6400))
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=4, int_time_s=0.1, samples_per_call=S,
                       sky_freq_hz=synth.SKY_FREQ_HZ, precision=mw.MWAX_FP16)
    vis, _ = run_ex(desc, volt, delay_table=tab, delay_table_on_device=False)
    ref, _ = oracle.correlate_ext(odesc(desc, volt), oracle.Ext(delay_table=tab, table_step=6400), volt, None)
    assert ext_parity(vis, ref, T).max() <= TOL[mw.MWAX_FP16]


@pytest.mark.parametrize("prec", [mw.MWAX_FP32, mw.MWAX_FP16, mw.MWAX_FP16X3], ids=["fp32", "fp16", "fp16x3"])
def test_passband_deripple(prec):
    # inverse of a rippled passband with rolled-off edges: gains 0.9 .. 1.9
    T, N, F, S = 8, 128, 4, 128_000
    volt, delay = workload(44, T, S, delay="linear")
    u = np.arange(N) - N // 2
    resp = (1 + 0.03 * np.cos(2 * np.pi * u / 21.0)) * (1 - 0.45 * (np.abs(u) / (N / 2)) ** 6)
    g = (1.0 / resp).astype(np.float32)
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=0.1, samples_per_call=S,
                       sky_freq_hz=synth.SKY_FREQ_HZ, precision=prec)
    vis, _ = run_ex(desc, volt, delay_poly=delay, passband=g)
    ref, _ = oracle.correlate_ext(odesc(desc, volt), oracle.Ext(passband=g.astype(np.float64)), volt, delay)
    assert ext_parity(vis, ref, T).max() <= TOL[prec]


@pytest.mark.parametrize("prec", [mw.MWAX_FP32, mw.MWAX_FP16, mw.MWAX_FP16X3], ids=["fp32", "fp16", "fp16x3"])
def test_oversampled_channel(prec):
    # 32/25 oversampled coarse channel: 1.6384 MS/s, N = 128 keeps the central 100 bins,
    # F = 4 -> 25 output channels; integration of 1000 frames = 78.125 ms
    fs, T, N, keep, F = 1.6384e6, 8, 128, 100, 4
    S = 2 * 128_000
    volt, delay = workload(55, T, S, delay="linear")
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=128_000 / fs, samples_per_call=S,
                       sky_freq_hz=synth.SKY_FREQ_HZ, precision=prec, sample_rate_hz=fs, keep_bins=keep)
    plan = mw.mwax_plan_create_ex(desc)
    assert plan.info["n_chan_out"] == keep // F
    vis, _ = run_ex(desc, volt, delay_poly=delay)
    ref, _ = oracle.correlate_ext(odesc(desc, volt), oracle.Ext(sample_rate_hz=fs, keep_bins=keep), volt, delay)
    assert vis.shape == ref.shape
    assert ext_parity(vis, ref, T).max() <= TOL[prec]


def test_everything_at_once():
    T, N, F, bs = 8, 256, 8, 6400
    S = 2 * 128_000
    volt, _ = workload(66, T, S, block_samples=bs, delay="linear")
    flags = flags_for(5, S // bs, 2 * T, frac=0.1)
    tab = np.random.default_rng(2).uniform(0, 50e-9, (2 * T, S // 3200))
    g = np.linspace(0.8, 1.2, N).astype(np.float32)
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=0.1, samples_per_call=S, block_samples=bs,
                       sky_freq_hz=synth.SKY_FREQ_HZ)
    vis, w = run_ex(desc, volt, delay_table=tab, table_step_samples=3200, zero_flags=flags, normalise=1, passband=g)
    e = oracle.Ext(delay_table=tab, table_step=3200, passband=g.astype(np.float64), zero_flags=flags, normalise=1)
    ref, rw = oracle.correlate_ext(odesc(desc, volt), e, volt, None)
    np.testing.assert_allclose(w, rw, rtol=1e-7)
    assert ext_parity(vis, ref, T).max() <= TOL[mw.MWAX_FP32]


def test_extended_call_errors():
    T, S = 2, 64_000
    desc = mw.PlanDesc(n_tiles=T, fft_len=128, fine_avg=4, int_time_s=0.05, samples_per_call=S)
    plan = mw.mwax_plan_create_ex(desc)
    mw.mwax_plan_set_stream(plan)
    v = torch.zeros(plan.input_bytes, dtype=torch.int8, device="cuda")
    out = mw.empty_output(plan)
    poly = np.zeros((2 * T, 3))
    tab = np.zeros((2 * T, 10))
    with pytest.raises(mw.MwaxError, match="exclusive"):
        mw.mwax_correlate_ex(plan, v, out, delay_poly=poly, delay_table=tab)
    with pytest.raises(mw.MwaxError, match=r"\(0, 2\]"):
        mw.mwax_plan_set_passband(plan, np.zeros(128, np.float32))
    i8 = mw.mwax_plan_create_ex(mw.PlanDesc(n_tiles=T, fft_len=1, fine_avg=1, int_time_s=0.05, samples_per_call=S,
                                            precision=mw.MWAX_INT8))
    mw.mwax_plan_set_stream(i8)
    o8 = mw.empty_output(i8)
    with pytest.raises(mw.MwaxError, match="normalise"):
        mw.mwax_correlate_ex(i8, v, o8, zero_flags=np.zeros((1, 2 * T), np.uint8), normalise=True)
    with pytest.raises(mw.MwaxError, match="exact integers"):
        mw.mwax_plan_set_passband(i8, np.ones(1, np.float32))
