"""Full-size parity: the 256-tile, 8 s sub-observation (512 signal paths, 10.24 M int8
complex samples per path, 128-point FFT, 0.5 s integrations averaged by 4) run exactly
as the benchmark runs it (same plan description and 48 GiB workspace, so the same
launches; the delays are a different quadratic polynomial on every signal path), checked
against the FP64 oracle on sampled outputs that the oracle computes one
by one: random (integration, baseline, channel, pol) entries plus the parallel-pol
autocorrelations that the parity metric divides by.  Bars as in the small-case tests:
FP32 and FP16 hi/lo pairs 1e-5, FP16 2e-3, FP8 3e-2 of the auto scale; the integer mode
(no FFT, 1 s integrations) bit-exact."""
import numpy as np
import pytest

import oracle
import paper_2303_11557_b300 as mw
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
torch = pytest.importorskip("torch")

T, N, F, T_INT, S = 256, 128, 4, 0.5, 10_240_000
SEED = 0x4D574159
WORKSPACE = 48 << 30   # as bench.py: all 16 integrations' operands resident, one launch each
TOL = {mw.MWAX_FP32: 1e-5, mw.MWAX_FP16: 2e-3, mw.MWAX_FP8: 3e-2, mw.MWAX_FP16X3: 1e-5}


@pytest.fixture(scope="module")
def full_input():
    # every signal path its own quadratic delay polynomial (c2 t^2 up to 20 ns by 8 s), the
    # source delayed by the same polynomials
    delay = synth.path_delays_quadratic(SEED, T, S / synth.FS)
    volt = np.empty((S // 64_000, 2 * T, 64_000, 2), dtype=np.int8)
    synth.voltages(SEED, 2 * T, S, tones=synth.point_source_tones(SEED), delay_poly=delay,
                   sky_freq_hz=synth.SKY_FREQ_HZ, out=volt)
    dev = torch.from_numpy(volt.reshape(-1)).cuda()
    yield volt, delay, dev
    del dev
    torch.cuda.empty_cache()


def auto_baseline(i):
    return i * (2 * T - i + 1) // 2 + 0


def sample_requests(seed, n_ints, M, per_int, ints):
    """Random (w, b, j, pol) entries in the given integrations, plus the autos (xx or yy
    of both tiles, same w and j) each one's parity metric needs."""
    rng = np.random.default_rng(seed)
    B = T * (T + 1) // 2
    req = []
    for w in ints:
        for _ in range(per_int):
            i = int(rng.integers(0, T))
            j = int(rng.integers(i, T))
            b = i * (2 * T - i + 1) // 2 + (j - i)
            req.append((w, b, int(rng.integers(0, M)), int(rng.integers(0, 4))))
    autos = set()
    for w, b, c, pol in req:
        i, j = tiles_of(b)
        autos.add((w, auto_baseline(i), c, 3 * (pol >> 1)))
        autos.add((w, auto_baseline(j), c, 3 * (pol & 1)))
    assert all(0 <= r[1] < B for r in req)
    return np.array(req + sorted(autos), dtype=np.int64), len(req)


def tiles_of(b):
    i = 0
    while b >= T - i:
        b -= T - i
        i += 1
    return i, i + b


def metric(got, want, req, n_main):
    lookup = {tuple(r): k for k, r in enumerate(req.tolist())}
    errs = []
    for k in range(n_main):
        w, b, c, pol = req[k].tolist()
        i, j = tiles_of(b)
        ap = want[lookup[(w, auto_baseline(i), c, 3 * (pol >> 1))]].real
        aq = want[lookup[(w, auto_baseline(j), c, 3 * (pol & 1))]].real
        errs.append(abs(got[k] - want[k]) / np.sqrt(abs(ap) * abs(aq)))
    return np.array(errs)


@pytest.mark.parametrize("prec", [pytest.param(mw.MWAX_FP32, id="fp32"), pytest.param(mw.MWAX_FP16, id="fp16"),
                                  pytest.param(mw.MWAX_FP8, id="fp8"), pytest.param(mw.MWAX_FP16X3, id="fp16x3")])
def test_fullsize_sampled(prec, full_input):
    volt, delay, dev = full_input
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=T_INT, samples_per_call=S,
                       sky_freq_hz=synth.SKY_FREQ_HZ, precision=prec, workspace_limit=WORKSPACE)
    plan = mw.mwax_plan_create_ex(desc)
    mw.mwax_plan_set_stream(plan)
    out = mw.empty_output(plan)
    out.fill_(0xAB)
    mw.mwax_correlate(plan, dev, torch.from_numpy(delay).cuda(), out)
    mw.mwax_plan_sync(plan)
    vis, w = mw.split_output(plan, out)
    vis = vis.cpu().numpy()
    assert np.all(w.cpu().numpy() == 1.0)
    n_ints, M = vis.shape[0], vis.shape[2]
    assert (n_ints, M) == (16, 32)
    # first, a middle and the last integration
    req, n_main = sample_requests(0x5A + prec, n_ints, M, 24, [0, 7, 15])
    od = oracle.Desc(n_tiles=T, fft_len=N, fine_avg=F, int_frames=int(T_INT * synth.FS) // N, n_samples=S,
                     sky_freq_hz=synth.SKY_FREQ_HZ)
    want = oracle.correlate_sampled(od, volt, delay, req)
    got = vis[req[:, 0], req[:, 1], req[:, 2], req[:, 3]]
    err = metric(got, want, req, n_main)
    assert np.all(np.isfinite(got))
    assert err.max() <= TOL[prec], f"max err {err.max():.3e} (median {np.median(err):.3e})"
    plan.close()


def test_fullsize_int8_sampled_exact(full_input):
    # integer mode at 1.28 MHz: 1 s integrations (1.28 M frames of one sample), no delay
    volt, _, dev = full_input
    desc = mw.PlanDesc(n_tiles=T, fft_len=1, fine_avg=1, int_time_s=1.0, samples_per_call=S,
                       precision=mw.MWAX_INT8, workspace_limit=WORKSPACE)
    plan = mw.mwax_plan_create_ex(desc)
    mw.mwax_plan_set_stream(plan)
    out = mw.empty_output(plan)
    out.fill_(0x5A)
    mw.mwax_correlate(plan, dev, None, out)
    mw.mwax_plan_sync(plan)
    vis, w = mw.split_output(plan, out)
    vis = vis.cpu().numpy()                      # int64 [ints, B, 4, 2]
    assert vis.shape[0] == 8 and np.all(w.cpu().numpy() == 1.0)
    rng = np.random.default_rng(0x1E8)
    req = []
    for wi in (0, 7):
        for _ in range(12):
            i = int(rng.integers(0, T))
            j = int(rng.integers(i, T))
            req.append((wi, i * (2 * T - i + 1) // 2 + (j - i), 0, int(rng.integers(0, 4))))
    req = np.array(req, dtype=np.int64)
    od = oracle.Desc(n_tiles=T, fft_len=1, fine_avg=1, int_frames=1_280_000, n_samples=S)
    want = oracle.correlate_sampled(od, volt, None, req)   # integer sums < 2^53: exact in FP64
    got = vis[req[:, 0], req[:, 1], req[:, 3]]
    assert np.array_equal(got[:, 0], want.real.astype(np.int64))
    assert np.array_equal(got[:, 1], want.imag.astype(np.int64))
    assert np.all(want.real == np.round(want.real)) and np.all(want.imag == np.round(want.imag))
    plan.close()
