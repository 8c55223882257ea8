"""Pins of the oracle's full correlation (Sec. 2.5-2.7) against what the paper and the
mathematics fix, never against a retyped copy of its own formulas:

* Parseval (exact identity): with no delay and F = 1 the channel sum of C_pq equals
  N * sum_s x_p[s] conj(x_q[s]), computed here in exact int64 from the voltages;
* the paper's own hand-crafted test vectors (Sec. 3.1): per-path pure tones that are
  exactly representable in int8 give closed-form visibilities at the right channel,
  baseline and polarisation and zero elsewhere;
* delay correction (Sec. 2.5.1, 4.3): closed-form fringe phase of a delayed tone,
  and zero phase once corrected, for static, linear and quadratic per-path delays
  (the last through every oracle route that evaluates the polynomial);
* a full cross-power matrix is Hermitian with real, non-negative autos;
* closed-form expectation of a noise + point-source workload (statistical);
* integer mode against numpy int64 brute force, and 2x input -> exactly 4x output.
"""
import os

import numpy as np
import pytest

import oracle
import synth

FS = synth.FS
GOLDEN_ORDER = os.path.join(os.path.dirname(__file__), "golden", "mwax_order_T3.txt")


def _order_table():
    rows = []
    for line in open(GOLDEN_ORDER):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        head, body = line.split("|")
        b, i, j = (int(v) for v in head.split())
        toks = body.split()
        pq = []
        for k in range(4):
            p = int(toks[2 * k].split(":")[1])
            q = int(toks[2 * k + 1])
            pq.append((p, q))
        rows.append((b, i, j, pq))
    return rows


def _x(volt, d, p):
    """Complex int64 time series of path p from the block-major int8 array."""
    v = volt[:, p, :, :].reshape(-1, 2).astype(np.int64)
    return v[:, 0] + 1j * v[:, 1], v


def test_baseline_order_golden():
    for b, i, j, _ in _order_table():
        assert oracle.baseline_tiles(3, b) == (i, j)


@pytest.mark.parametrize("N,T,K,bs", [(8, 2, 16, 128), (16, 3, 10, 160), (10, 2, 12, 120)])
def test_parseval_exact(N, T, K, bs):
    d = oracle.Desc(n_tiles=T, fft_len=N, fine_avg=1, int_frames=K, n_samples=2 * K * N, block_samples=bs)
    volt = synth.voltages(11 + N, 2 * T, d.n_samples, block_samples=bs, sigma=40.0)
    vis, wts = oracle.correlate(d, volt)
    assert np.all(wts == 1.0)
    for b, (i, j) in enumerate([(i, j) for i in range(T) for j in range(i, T)]):
        for pol in range(4):
            p, q = 2 * i + (pol >> 1), 2 * j + (pol & 1)
            _, vp = _x(volt, d, p)
            _, vq = _x(volt, d, q)
            for w in range(d.n_ints):
                sl = slice(w * K * N, (w + 1) * K * N)
                ar, ai, br, bi = vp[sl, 0], vp[sl, 1], vq[sl, 0], vq[sl, 1]
                re = int(np.sum(ar * br + ai * bi)) * N
                im = int(np.sum(ai * br - ar * bi)) * N
                got = vis[w, b, :, pol].sum()
                assert abs(got.real - re) <= 1e-9 * max(1, abs(re)) + 1e-6
                assert abs(got.imag - im) <= 1e-9 * max(1, abs(re)) + 1e-6


def _exact_tone_volt(N, amps, bins, quarter_turns, n_samples, bs):
    """Tones exactly representable in int8: bins in {0, +-N/4, N/2}, phases k*pi/2."""
    n = len(amps)
    volt = np.zeros((n_samples // bs, n, bs, 2), np.int8)
    s = np.arange(n_samples)
    for p in range(n):
        z = amps[p] * np.exp(1j * (np.pi / 2) * quarter_turns[p]) * np.exp(2j * np.pi * bins[p] * s / N)
        z = np.round(z.real) + 1j * np.round(z.imag)
        assert np.max(np.abs(z - amps[p] * np.exp(1j * (np.pi / 2) * quarter_turns[p])
                             * np.exp(2j * np.pi * bins[p] * s / N))) < 1e-9
        volt[:, p, :, 0] = z.real.reshape(-1, bs)
        volt[:, p, :, 1] = z.imag.reshape(-1, bs)
    return volt


def test_tone_vectors_ordering_exact():
    # Sec. 3.1: each path carries a pure tone at a selectable fine channel; the result
    # must sit at the right channel, baseline and polarisation with no cross-talk.
    N, K, T = 16, 8, 3
    amps = [3, 5, 7, 11, 13, 17]
    bins = [N // 4, 0, -N // 4, N // 4, N // 2, 0]   # paths 0 & 3 share a bin, 1 & 5 too
    turns = [0, 1, 2, 3, 1, 0]
    d = oracle.Desc(n_tiles=T, fft_len=N, fine_avg=1, int_frames=K, n_samples=K * N * 2, block_samples=64)
    volt = _exact_tone_volt(N, amps, bins, turns, d.n_samples, 64)
    vis, _ = oracle.correlate(d, volt)
    expect = np.zeros_like(vis)
    for b, i, j, pq in _order_table():
        for pol, (p, q) in enumerate(pq):
            if bins[p] % N == bins[q] % N:
                c = (bins[p] + N // 2) % N if bins[p] != N // 2 else 0   # u = N/2 is u = -N/2
                expect[:, b, c, pol] = K * N * N * amps[p] * amps[q] * np.exp(1j * np.pi / 2 * (turns[p] - turns[q]))
    assert np.max(np.abs(vis - expect)) < 1e-9 * np.max(np.abs(expect))


@pytest.mark.parametrize("N", [16, 128])
def test_delay_fringe_closed_form(N):
    # Sec. 2.5.1 / 4.3: a common tone delayed by a static tau_p shows the fringe phase
    # -2 pi (nu + f)(tau_p - tau_q) across a baseline; multiplying the spectra by
    # exp(+2 pi i (nu + f) tau_p) removes it.
    T, K = 2, 64
    nu = synth.SKY_FREQ_HZ
    u0 = N // 4 - 1
    f0 = u0 * FS / N
    delay = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [13e-9, 0.0, 0.0], [47e-9, 0.0, 0.0]])
    bs = 16 * N
    d = oracle.Desc(n_tiles=T, fft_len=N, fine_avg=1, int_frames=K, n_samples=2 * K * N, block_samples=bs,
                    sky_freq_hz=nu)
    volt = synth.voltages(3, 4, d.n_samples, block_samples=bs, sigma=0.0, tones=[(f0, 100.0, 0.4, -1)],
                          delay_c01=delay[:, :2], sky_freq_hz=nu)
    c0 = u0 + N // 2
    raw, _ = oracle.correlate(d, volt, None)
    cor, _ = oracle.correlate(d, volt, delay)
    scale = K * N * N * 1e4
    for b, (i, j) in enumerate([(0, 0), (0, 1), (1, 1)]):
        for pol in range(4):
            p, q = 2 * i + (pol >> 1), 2 * j + (pol & 1)
            want = -2 * np.pi * (nu + f0) * (delay[p, 0] - delay[q, 0])
            for w in range(d.n_ints):
                got = np.angle(raw[w, b, c0, pol])
                assert abs(np.angle(np.exp(1j * (got - want)))) < 2e-3
                assert abs(np.angle(cor[w, b, c0, pol])) < 2e-3
                assert abs(abs(cor[w, b, c0, pol]) - scale) < 2e-2 * scale


@pytest.mark.parametrize("N", [16, 128])
def test_delay_tracking_frame_centre(N):
    # Fringe stopping (Sec. 4.3): a delay that drifts in time is evaluated once per
    # frame.  Sampling tau(t) at the frame centre t_m = (m + 1/2) N / Fs leaves no
    # residual phase; sampling it at the frame start would leave
    # pi (nu + f) c1 N / Fs radians (0.09 rad at N = 128, 0.01 rad at N = 16).
    T, K = 2, 64
    nu = synth.SKY_FREQ_HZ
    u0 = N // 4 - 1
    f0 = u0 * FS / N
    delay = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [13e-9, 2e-6, 0.0], [47e-9, -1.5e-6, 0.0]])
    bs = 16 * N
    d = oracle.Desc(n_tiles=T, fft_len=N, fine_avg=1, int_frames=K, n_samples=2 * K * N, block_samples=bs,
                    sky_freq_hz=nu)
    volt = synth.voltages(4, 4, d.n_samples, block_samples=bs, sigma=0.0, tones=[(f0, 100.0, 1.1, -1)],
                          delay_c01=delay[:, :2], sky_freq_hz=nu)
    c0 = u0 + N // 2
    cor, _ = oracle.correlate(d, volt, delay)
    scale = K * N * N * 1e4
    for b in range(3):
        for pol in range(4):
            for w in range(d.n_ints):
                assert abs(np.angle(cor[w, b, c0, pol])) < 2e-3
                assert abs(abs(cor[w, b, c0, pol]) - scale) < 2e-2 * scale


@pytest.mark.parametrize("N", [16, 128])
@pytest.mark.parametrize("route", ["correlate", "sampled", "ext"])
def test_delay_quadratic_per_path_closed_form(N, route):
    # Sec. 2.5.1 / 4.3 with the full delay polynomial tau_p(t) = c0 + c1 t + c2 t^2, a
    # different one on each signal path (x and y of a tile differ too).  One frame per
    # integration, so each visibility is a single frame's product: uncorrected, a common
    # bin-centred tone shows the closed-form fringe -2 pi (nu + f)(tau_p(t_m) - tau_q(t_m))
    # at the frame centre t_m = (m + 1/2) N / Fs; corrected, no phase is left.  Over the
    # 6.4 ms call the c2 t^2 terms alone turn the fringe by up to ~1 rad, and c2 t (a
    # dropped power) by ~100 rad.  Residual of the frame-centre sampling: the half-sample
    # offset of the frame's mean time, 2 pi (nu + f) |tau_p' - tau_q'| / (2 Fs) < 1e-3 rad;
    # int8 rounding (variance 1/12 per component) adds phase noise of rms
    # sqrt(2) / (a sqrt(12 N)) per single-frame cross product, allowed 5 times over.
    T, S = 2, 8192
    nu = synth.SKY_FREQ_HZ
    u0 = N // 4 - 1
    f0 = u0 * FS / N
    delay = np.array([[5e-9, 0.8e-6, 3e-5], [20e-9, -1.0e-6, -2.5e-5],
                      [13e-9, 0.6e-6, 2e-5], [47e-9, -0.4e-6, -3e-5]])
    d = oracle.Desc(n_tiles=T, fft_len=N, fine_avg=1, int_frames=1, n_samples=S, block_samples=S,
                    sky_freq_hz=nu)
    volt = synth.voltages(6, 4, S, block_samples=S, sigma=0.0, tones=[(f0, 100.0, 0.7, -1)],
                          delay_poly=delay, sky_freq_hz=nu)
    c0 = u0 + N // 2
    frames = S // N
    t = (np.arange(frames) + 0.5) * N / FS
    tau = delay[:, 0][:, None] + delay[:, 1][:, None] * t + delay[:, 2][:, None] * t * t   # [path, frame]
    if route == "correlate":
        raw, _ = oracle.correlate(d, volt, None)
        cor, _ = oracle.correlate(d, volt, delay)
        pick = lambda v, w, b, pol: v[w, b, c0, pol]
    elif route == "ext":
        raw, _ = oracle.correlate_ext(d, oracle.Ext(), volt, None)
        cor, _ = oracle.correlate_ext(d, oracle.Ext(), volt, delay)
        pick = lambda v, w, b, pol: v[w, b, c0, pol]
    else:
        req = np.array([(w, b, c0, pol) for w in range(frames) for b in range(3) for pol in range(4)], dtype=np.int64)
        look = {tuple(r): k for k, r in enumerate(req.tolist())}
        raw = oracle.correlate_sampled(d, volt, None, req)
        cor = oracle.correlate_sampled(d, volt, delay, req)
        pick = lambda v, w, b, pol: v[look[(w, b, c0, pol)]]
    scale = N * N * 1e4
    tol = 1e-3 + 5 * np.sqrt(2) / (100.0 * np.sqrt(12 * N))
    quad_turn = 0.0
    for b, (i, j) in enumerate([(0, 0), (0, 1), (1, 1)]):
        for pol in range(4):
            p, q = 2 * i + (pol >> 1), 2 * j + (pol & 1)
            for w in range(frames):
                want = -2 * np.pi * (nu + f0) * (tau[p, w] - tau[q, w])
                got = np.angle(pick(raw, w, b, pol))
                assert abs(np.angle(np.exp(1j * (got - want)))) < tol
                assert abs(np.angle(pick(cor, w, b, pol))) < tol
                assert abs(abs(pick(cor, w, b, pol)) - scale) < 2e-2 * scale
                quad_turn = max(quad_turn, abs(2 * np.pi * (nu + f0) * (delay[p, 2] - delay[q, 2]) * t[w] ** 2))
    assert quad_turn > 0.5   # the quadratic term moves the fringe far beyond the tolerance


def test_hermitian_full_matrix():
    T, N, K = 3, 32, 40
    d = oracle.Desc(n_tiles=T, fft_len=N, fine_avg=1, int_frames=K, n_samples=K * N, block_samples=K * N,
                    sky_freq_hz=synth.SKY_FREQ_HZ)
    volt = synth.voltages(5, 2 * T, d.n_samples, block_samples=K * N, tones=synth.point_source_tones(5))
    delay = synth.tile_delays_fixed(T)
    for c in (0, 5, N // 2, N - 1):
        C = oracle.xmatrix(d, volt, delay, 0, c)
        assert np.max(np.abs(C - C.conj().T)) <= 1e-12 * np.max(np.abs(C))
        assert np.all(np.diag(C).imag == 0.0)
        assert np.all(np.diag(C).real >= 0.0)


def test_point_source_closed_form():
    # Noise (sigma per component) plus a common comb of bin-centred tones with fixed
    # per-tile delays 0-50 ns.  Expected per frame and bin:
    #   E[Y_p conj(Y_q)] = N^2 a^2 e^{-2 pi i (nu+f)(tau_p - tau_q)} on tone bins (p != q),
    #   E[|Y_p|^2]       = N (2 sigma^2 + 2/12) (+ N^2 a^2 on tone bins),
    # the 2/12 being the variance of rounding to integers.  Tolerance: 6 standard errors.
    T, N, K, sigma = 4, 32, 4000, 16.0
    nu = synth.SKY_FREQ_HZ
    tones = synth.point_source_tones(9, sigma=sigma, rel_rms=1.0)
    a = tones[0][1]
    delay = synth.tile_delays_fixed(T)
    d = oracle.Desc(n_tiles=T, fft_len=N, fine_avg=1, int_frames=K, n_samples=K * N, block_samples=K * N,
                    sky_freq_hz=nu)
    volt = synth.voltages(9, 2 * T, d.n_samples, block_samples=K * N, sigma=sigma, tones=tones,
                          delay_c01=delay[:, :2], sky_freq_hz=nu)
    raw, _ = oracle.correlate(d, volt, None)
    cor, _ = oracle.correlate(d, volt, delay)
    tone_c = sorted(int(round(f * N / FS)) + N // 2 for f, *_ in tones)
    noise_c = [c for c in range(N) if c not in tone_c]
    noise_auto = N * (2 * sigma**2 + 2 / 12)
    sig = N * N * a * a
    pairs = [(i, j) for i in range(T) for j in range(i, T)]
    autos_noise = []
    for b, (i, j) in enumerate(pairs):
        for pol in range(4):
            p, q = 2 * i + (pol >> 1), 2 * j + (pol & 1)
            for c in range(N):
                on = c in tone_c
                f = (c - N // 2) * FS / N
                if p == q:
                    want = K * (noise_auto + (sig if on else 0.0))
                    se = want / np.sqrt(K)
                    assert abs(raw[0, b, c, pol] - want) < 6 * se
                    if not on:
                        autos_noise.append(raw[0, b, c, pol].real)
                else:
                    auto = noise_auto + (sig if on else 0.0)
                    se = np.sqrt(K) * auto
                    dtau = delay[p, 0] - delay[q, 0]
                    want_raw = K * sig * np.exp(-2j * np.pi * (nu + f) * dtau) if on else 0.0
                    want_cor = K * sig if on else 0.0
                    assert abs(raw[0, b, c, pol] - want_raw) < 6 * se
                    assert abs(cor[0, b, c, pol] - want_cor) < 6 * se
    # pooled noise-only autos pin the absolute FFT scale (factor N) to ~0.1%
    m = np.mean(autos_noise) / (K * noise_auto)
    assert abs(m - 1.0) < 6 / np.sqrt(K * len(autos_noise))


def test_correlate_sampled_matches_full():
    T, N, F, K = 3, 20, 4, 30
    d = oracle.Desc(n_tiles=T, fft_len=N, fine_avg=F, int_frames=K, n_samples=3 * K * N, block_samples=200,
                    sky_freq_hz=synth.SKY_FREQ_HZ)
    volt = synth.voltages(21, 2 * T, d.n_samples, block_samples=200, tones=synth.point_source_tones(21))
    delay = synth.tile_delays_linear(21, T)
    vis, _ = oracle.correlate(d, volt, delay)
    rng = np.random.default_rng(0)
    req = np.stack([rng.integers(0, d.n_ints, 40), rng.integers(0, d.n_baselines, 40),
                    rng.integers(0, d.n_chan_out, 40), rng.integers(0, 4, 40)], 1)
    got = oracle.correlate_sampled(d, volt, delay, req)
    want = vis[req[:, 0], req[:, 1], req[:, 2], req[:, 3]]
    assert np.array_equal(got, want)


def test_averaging_real_input_mirror():
    # Real-valued voltages (im = 0) have Hermitian spectra, so V(-f) = conj V(f):
    # with odd M output channel j mirrors channel M-1-j exactly (Sec. 2.6 symmetry).
    T, N, F, K = 2, 20, 4, 25
    d = oracle.Desc(n_tiles=T, fft_len=N, fine_avg=F, int_frames=K, n_samples=K * N, block_samples=K * N)
    volt = synth.voltages(31, 2 * T, d.n_samples, block_samples=K * N)
    volt[..., 1] = 0
    vis, _ = oracle.correlate(d, volt)
    M = N // F
    assert M % 2 == 1
    for j in range(M):
        # the top edge bin (u = N/2) does not exist, so channel M-1 lacks one half-bin
        # that channel 0 has; compare the interior channels only
        if j in (0, M - 1):
            continue
        assert np.max(np.abs(vis[:, :, j, :] - np.conj(vis[:, :, M - 1 - j, :]))) < 1e-9 * np.max(np.abs(vis))


def test_int_mode_exact_and_linear():
    T, K = 3, 1000
    d = oracle.Desc(n_tiles=T, fft_len=1, fine_avg=1, int_frames=K, n_samples=4 * K, block_samples=500)
    volt = synth.voltages(41, 2 * T, d.n_samples, block_samples=500, sigma=30.0)
    vis, wts = oracle.correlate_int(d, volt)
    assert np.all(wts == 1.0)
    for b, i, j, pq in _order_table():
        for pol, (p, q) in enumerate(pq):
            _, vp = _x(volt, d, p)
            _, vq = _x(volt, d, q)
            for w in range(d.n_ints):
                sl = slice(w * K, (w + 1) * K)
                ar, ai, br, bi = vp[sl, 0], vp[sl, 1], vq[sl, 0], vq[sl, 1]
                assert vis[w, b, pol, 0] == np.sum(ar * br + ai * bi)
                assert vis[w, b, pol, 1] == np.sum(ai * br - ar * bi)
    # linearity: halve to |x| <= 63, then doubling the input multiplies every product by 4
    small = (volt // 2).astype(np.int8)
    v1, _ = oracle.correlate_int(d, small)
    v2, _ = oracle.correlate_int(d, (small * 2).astype(np.int8))
    assert np.array_equal(v2, 4 * v1)
    # the float path at N = 1 agrees with the integer path
    vf, _ = oracle.correlate(d, volt)
    assert np.array_equal(vf[:, :, 0, :].real, vis[..., 0].astype(float))
    assert np.array_equal(vf[:, :, 0, :].imag, vis[..., 1].astype(float))
