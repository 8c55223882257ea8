"""Pins of the oracle's roadmap extensions (Sec. 2.4, 4) against what the paper and the
mathematics fix, and against the already-pinned base oracle -- never against a retyped
copy of the extension's own formulas:

* with every extension off, the extended oracle is the base oracle bit for bit;
* zeroing flags (Sec. 2.4.2, 4.1): occupancy weights have a closed form when whole
  blocks of one path are flagged; flagged data is excluded whatever it holds (equal to
  the base oracle on input zeroed there); normalisation divides by that weight;
* tabulated delays (Sec. 2.4.1, 4.3): a table of constant rows equals the constant
  polynomial; with one frame per table step and the table sampled at frame centres it
  equals the polynomial path; a tone's corrected phase follows each step's value;
* passband de-ripple (Sec. 4.2): spectra are the base spectra times the channel gain,
  visibilities scale by its square;
* oversampled channels (Sec. 4.5): hand-derived averaging weights over the kept band,
  a bin-centred tone at the oversampled rate lands in its channel, tones outside the
  kept band leave no trace in the output.
"""
import numpy as np
import pytest

import oracle
import synth


def _desc(T=2, N=8, F=1, K=8, ints=2, bs=64, sky=0.0):
    return oracle.Desc(n_tiles=T, fft_len=N, fine_avg=F, int_frames=K, n_samples=ints * K * N, block_samples=bs,
                       sky_freq_hz=sky)


def _volt(d, seed=5, sigma=30.0):
    return synth.voltages(seed, d.n_paths, d.n_samples, block_samples=d.block_samples, sigma=sigma)


def test_extensions_off_is_base_oracle():
    d = _desc(T=3, N=16, F=4, K=6, ints=2, bs=96, sky=139.52e6)
    v = _volt(d)
    delay = synth.tile_delays_linear(3, 3)
    base, bw = oracle.correlate(d, v, delay)
    ext, ew = oracle.correlate_ext(d, oracle.Ext(), v, delay)
    assert np.array_equal(base, ext) and np.array_equal(bw, ew)
    for F in (1, 2, 4, 8):
        for j in range(16 // F):
            assert np.array_equal(oracle.avg_weights_keep(16, 16, F, 1, j)[0], oracle.avg_weights(16, F, 1, j)[0])


# ------------------------------------------------------------------ zeroing flags
def test_occupancy_closed_form():
    # 4 integrations of 8 frames of 8 samples, blocks of 16 samples: 4 blocks per integration
    d = _desc(T=3, N=8, K=8, ints=4, bs=16)
    n_blocks = d.n_samples // d.block_samples
    flags = np.zeros((n_blocks, d.n_paths), np.uint8)
    flags[0, 1] = 1                     # integration 0: path 1 loses 1 of 4 blocks
    flags[5:7, 4] = 1                   # integration 1: path 4 loses 2 of 4 blocks
    flags[9, 4] = 1                     # integration 2: paths 4 and 5 lose the same block
    flags[9, 5] = 1
    flags[12:16, 2] = 1                 # integration 3: path 2 loses everything
    e = oracle.Ext(zero_flags=flags)
    lost = {0: {1: {0}}, 1: {4: {1, 2}}, 2: {4: {1}, 5: {1}}, 3: {2: {0, 1, 2, 3}}}
    for w in range(4):
        for p in range(d.n_paths):
            for q in range(d.n_paths):
                gone = lost[w].get(p, set()) | lost[w].get(q, set())
                assert oracle.occupancy(d, e, w, p, q) == (4 - len(gone)) / 4


def test_flagged_data_is_excluded_and_normalised():
    d = _desc(T=2, N=8, F=2, K=8, ints=2, bs=16, sky=139.52e6)
    v = _volt(d, seed=9)
    n_blocks = d.n_samples // d.block_samples
    rng = np.random.default_rng(4)
    flags = (rng.random((n_blocks, d.n_paths)) < 0.3).astype(np.uint8)
    flags[4:8, 3] = 1                                   # path 3 absent for all of integration 1
    zeroed = v.copy()
    for b in range(n_blocks):
        for p in range(d.n_paths):
            if flags[b, p]:
                zeroed[b, p] = 0
    delay = synth.tile_delays_linear(8, 2)
    base, _ = oracle.correlate(d, zeroed, delay)
    got, wts = oracle.correlate_ext(d, oracle.Ext(zero_flags=flags), v, delay)
    assert np.array_equal(got, base)                    # garbage under the flags is ignored
    normed, wts2 = oracle.correlate_ext(d, oracle.Ext(zero_flags=flags, normalise=1), v, delay)
    assert np.array_equal(wts, wts2)
    for w in range(d.n_ints):
        for b in range(d.n_baselines):
            for pol in range(4):
                o = wts[w, b, pol]
                if o == 0.0:
                    assert np.all(normed[w, b, :, pol] == 0) and np.all(got[w, b, :, pol] == 0)
                else:
                    np.testing.assert_allclose(normed[w, b, :, pol] * o, got[w, b, :, pol], rtol=1e-12, atol=1e-9)
    # baselines with path 3 (tile 1, pol y) have zero weight in integration 1
    for b, (i, j) in enumerate([(0, 0), (0, 1), (1, 1)]):
        for pol in range(4):
            p, q = 2 * i + (pol >> 1), 2 * j + (pol & 1)
            if 3 in (p, q):
                assert wts[1, b, pol] == 0.0


def test_int_mode_flags_brute_force():
    d = _desc(T=2, N=1, F=1, K=40, ints=3, bs=20)
    v = _volt(d, seed=3, sigma=50.0)
    n_blocks = d.n_samples // d.block_samples
    flags = np.zeros((n_blocks, d.n_paths), np.uint8)
    flags[1, 0] = flags[2, 2] = flags[3, 2] = flags[5, 1] = 1
    vis, wts = oracle.correlate_int_ext(d, oracle.Ext(zero_flags=flags), v)
    z = v.astype(np.int64).copy()
    for b in range(n_blocks):
        z[b, flags[b].astype(bool)] = 0
    x = z[..., 0] + 1j * z[..., 1]                      # [blk, path, s]
    x = np.concatenate(list(x), axis=1)                 # [path, samples]
    for w in range(3):
        sl = slice(w * 40, (w + 1) * 40)
        for b, (i, j) in enumerate([(0, 0), (0, 1), (1, 1)]):
            for pol in range(4):
                p, q = 2 * i + (pol >> 1), 2 * j + (pol & 1)
                s = np.sum(x[p, sl] * np.conj(x[q, sl]))
                assert vis[w, b, pol, 0] == int(round(s.real)) and vis[w, b, pol, 1] == int(round(s.imag))
                blocks = range(2 * w, 2 * w + 2)
                good = sum(1 for k in blocks if not flags[k, p] and not flags[k, q])
                assert wts[w, b, pol] == good / 2


# ------------------------------------------------------------------ delay table
def test_constant_table_equals_constant_polynomial():
    d = _desc(T=2, N=16, F=2, K=5, ints=2, bs=80, sky=139.52e6)
    v = _volt(d, seed=21)
    c0 = np.array([3e-9, 17e-9, 40e-9, 8e-9])
    poly = np.zeros((4, 3))
    poly[:, 0] = c0
    tab = np.repeat(c0[:, None], 7, axis=1)
    a, _ = oracle.correlate(d, v, poly)
    b, _ = oracle.correlate_ext(d, oracle.Ext(delay_table=tab, table_step=32), v, None)
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-9 * np.abs(a).max())


def test_table_one_frame_per_step_equals_polynomial():
    # N = table step: every frame has its own entry; sampling the polynomial at frame
    # centres must reproduce the polynomial path (catches step-index off-by-ones)
    N = 32
    d = _desc(T=2, N=N, F=1, K=6, ints=2, bs=N * 6, sky=139.52e6)
    v = _volt(d, seed=22)
    poly = synth.tile_delays_linear(7, 2, max_c0=400e-9, max_c1=2e-3)
    frames = d.n_samples // N
    t = (np.arange(frames) + 0.5) * N / synth.FS
    tab = poly[:, :1] + poly[:, 1:2] * t[None, :]
    a, _ = oracle.correlate(d, v, poly)
    b, _ = oracle.correlate_ext(d, oracle.Ext(delay_table=tab, table_step=N), v, None)
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-9 * np.abs(a).max())


def test_table_tone_phase_per_step():
    # a bin-centred tone; each step's fractional delay gives frame phase
    # e^{+2 pi i (nu + f_u) tau_step} (Sec. 2.5.1) relative to the uncorrected spectrum.
    # Steps of 24 samples do not hold whole 16-sample frames: frame m takes the step
    # holding its centre time (m + 1/2) N / Fs, not the one holding its first sample.
    N, step = 16, 24
    d = _desc(T=1, N=N, F=1, K=16, ints=1, bs=256, sky=139.52e6)
    u0 = 3
    s = np.arange(d.n_samples)
    x = np.round(40 * np.exp(2j * np.pi * u0 * s / N))
    v = np.zeros((1, 2, 256, 2), np.int8)
    v[0, 0, :, 0], v[0, 0, :, 1] = x.real, x.imag
    v[0, 1] = v[0, 0]
    tab = np.array([np.arange(11) * 4e-9 + 1e-9, np.zeros(11)])
    Y0 = oracle.spectra(d, v, None, 0, 0, 16)
    Y = oracle.spectra_ext(d, oracle.Ext(delay_table=tab, table_step=step), v, None, 0, 0, 16)
    c = u0 + N // 2
    for m in range(16):
        centre = (m + 0.5) * N                       # in samples
        tau = tab[0, int(np.floor(centre / step))]
        want = np.exp(2j * np.pi * (d.sky_freq_hz + u0 * synth.FS / N) * tau)
        np.testing.assert_allclose(Y[m, c] / Y0[m, c], want, rtol=1e-12)


# ------------------------------------------------------------------ passband gains
def test_passband_scales_spectra_and_visibilities():
    N = 16
    d = _desc(T=2, N=N, F=1, K=6, ints=1, bs=96, sky=139.52e6)
    v = _volt(d, seed=30)
    g = 1.0 + 0.05 * np.cos(np.arange(N) * 0.9)
    delay = synth.tile_delays_linear(2, 2)
    for p in range(4):
        np.testing.assert_allclose(oracle.spectra_ext(d, oracle.Ext(passband=g), v, delay, p, 0, 6),
                                   oracle.spectra(d, v, delay, p, 0, 6) * g[None, :], rtol=1e-13, atol=1e-9)
    a, _ = oracle.correlate(d, v, delay)
    b, _ = oracle.correlate_ext(d, oracle.Ext(passband=g), v, delay)
    np.testing.assert_allclose(b, a * (g ** 2)[None, None, :, None], rtol=1e-12, atol=1e-9)


# ------------------------------------------------------------------ oversampled channels
def test_keep_weights_hand_derived():
    # N = 8, keep = 6 (u in [-3, 2]), F = 2, M = 3, centre j0 = 1, DC excluded:
    #   j = 0: centre u = -2 -> u -3 (1/2), -2 (1), -1 (1/2): sum 2
    #   j = 1: centre u =  0 -> u -1 (1/2), 0 (DC, 0), 1 (1/2): sum 1
    #   j = 2: centre u =  2 -> u  1 (1/2), 2 (1), 3 dropped: sum 1.5
    want = {0: ({-3: .5, -2: 1, -1: .5}, 2.0), 1: ({-1: .5, 0: 0, 1: .5}, 1.0), 2: ({1: .5, 2: 1}, 1.5)}
    for j, (ws, tot) in want.items():
        w, s = oracle.avg_weights_keep(8, 6, 2, 1, j)
        exp = np.zeros(8)
        for u, x in ws.items():
            exp[u + 4] = x
        assert np.array_equal(w, exp) and s == tot


def test_oversampled_tone_and_discarded_band():
    # coarse channel sampled at 32/25 x 1.28 MS/s; N = 32 keeps the central 25 bins
    fs = 1.6384e6
    N, keep = 32, 24
    d = _desc(T=1, N=N, F=1, K=8, ints=1, bs=256, sky=0.0)
    s = np.arange(d.n_samples)
    inside, outside = 5, 14                        # u = 14 lies outside [-12, 11]
    x = np.round(30 * np.exp(2j * np.pi * inside * s / N) + 30 * np.exp(2j * np.pi * outside * s / N))
    v = np.zeros((1, 2, 256, 2), np.int8)
    v[0, 0, :, 0], v[0, 0, :, 1] = x.real, x.imag
    v[0, 1] = v[0, 0]
    e = oracle.Ext(sample_rate_hz=fs, keep_bins=keep)
    vis, _ = oracle.correlate_ext(d, e, v, None)
    assert vis.shape[2] == keep
    auto = vis[0, 0, :, 0].real                    # xx auto over the kept channels
    j_in = inside + keep // 2
    assert np.argmax(auto) == j_in
    # the out-of-band tone contributes nothing: rounding noise only elsewhere
    others = np.delete(auto, j_in)
    assert others.max() < 1e-3 * auto[j_in]
    # delay correction at the oversampled rate: a common delay on both paths with the
    # second path uncorrected gives the fringe e^{+2 pi i f_u tau}, f_u = u fs / N
    tau = 300e-9
    poly = np.array([[tau, 0, 0], [0, 0, 0]])
    vd, _ = oracle.correlate_ext(d, e, v, poly)
    ph = np.angle(vd[0, 0, j_in, 1] / vis[0, 0, j_in, 1])
    want = np.angle(np.exp(2j * np.pi * inside * fs / N * tau))
    assert abs(np.angle(np.exp(1j * (ph - want)))) < 1e-9
