"""Pins of the oracle's tied-array beamformer (Sec. 4.4) against independent routines and
the already-pinned correlator -- never against a retyped copy of its own formula:

* zero steering delays: each beam is numpy's FFT of the tiles' summed voltages
  (linearity of the DFT), channel-shifted;
* a single tile steered with a delay table is that path's delay-corrected spectrum from
  the (pinned) extended correlator oracle;
* detected Stokes I equals the correlator's cross-power matrix summed over each pol's
  paths with the steering phase differences (|sum_p y_p|^2 = sum_pq y_p conj(y_q)), and
  the incoherent beam equals the sum of the correlator's autos;
* steering towards a delayed point source adds it coherently: the matched beam holds
  ~T^2 times one tile's signal power, a mis-steered beam does not.
"""
import numpy as np

import oracle
import synth


def _desc(T, N, frames, bs, sky=synth.SKY_FREQ_HZ, K=None):
    return oracle.Desc(n_tiles=T, fft_len=N, fine_avg=1, int_frames=K or frames, n_samples=frames * N,
                       block_samples=bs, sky_freq_hz=sky)


def _series(volt, p):
    v = volt[:, p].reshape(-1, 2).astype(np.float64)
    return v[:, 0] + 1j * v[:, 1]


def test_zero_delay_beam_is_fft_of_sum():
    T, N, frames, bs = 3, 16, 12, 64
    d = _desc(T, N, frames, bs)
    v = synth.voltages(2, 2 * T, frames * N, block_samples=bs, sigma=25.0)
    tab = np.zeros((2, 2 * T, 1))
    beams, _, _ = oracle.beamform(d, v, tab, table_step=6400)
    for a in range(2):
        x = sum(_series(v, 2 * t + a) for t in range(T)).reshape(frames, N)
        want = np.fft.fftshift(np.fft.fft(x, axis=1), axes=1)
        for b in range(2):
            np.testing.assert_allclose(beams[b, a], want, rtol=0, atol=1e-9 * np.abs(want).max())


def test_single_tile_beam_is_corrected_spectrum():
    N, frames, bs, step = 32, 10, 160, 48           # steps of 48 samples split 32-sample frames
    d = _desc(1, N, frames, bs)
    v = synth.voltages(3, 2, frames * N, block_samples=bs, sigma=25.0)
    tab = np.random.default_rng(0).uniform(0, 80e-9, (2, 7))
    beams, _, _ = oracle.beamform(d, v, tab[None], table_step=step)
    e = oracle.Ext(delay_table=tab, table_step=step)
    for a in range(2):
        want = oracle.spectra_ext(d, e, v, None, a, 0, frames)
        np.testing.assert_allclose(beams[0, a], want, rtol=0, atol=1e-9 * np.abs(want).max())


def test_detected_power_matches_correlator():
    T, N, K, ints, bs = 3, 16, 6, 2, 96
    frames = K * ints
    d = _desc(T, N, frames, bs, K=K)
    v = synth.voltages(4, 2 * T, frames * N, block_samples=bs, sigma=20.0)
    rng = np.random.default_rng(1)
    tab = rng.uniform(0, 60e-9, (2, 2 * T, 1))       # constant delays per beam and path
    _, power, incoh = oracle.beamform(d, v, tab, int_frames=K)
    fs = synth.FS
    for w in range(ints):
        for c in range(N):
            C = oracle.xmatrix(d, v, None, w, c)     # uncorrected cross-power of channel c
            f = (c - N // 2) * fs / N
            for b in range(2):
                ph = np.exp(2j * np.pi * (d.sky_freq_hz + f) * tab[b, :, 0])
                want = 0.0
                for a in range(2):
                    idx = np.arange(a, 2 * T, 2)
                    want += np.real(ph[idx] @ C[np.ix_(idx, idx)] @ np.conj(ph[idx]))
                np.testing.assert_allclose(power[b, w, c], want, rtol=1e-10)
            for a in range(2):
                want = sum(C[p, p].real for p in range(a, 2 * T, 2))
                np.testing.assert_allclose(incoh[w, a, c], want, rtol=1e-12)


def test_steering_adds_a_delayed_source_coherently():
    T, N, frames, bs = 8, 32, 64, 2048
    d = _desc(T, N, frames, bs)
    delays = synth.tile_delays_linear(9, T, max_c0=400e-9, max_c1=0.0)   # random per-tile signal delays
    tones = synth.point_source_tones(9, sigma=4.0, rel_rms=3.0)  # source well above the noise
    v = synth.voltages(9, 2 * T, frames * N, block_samples=bs, sigma=4.0, tones=tones,
                       delay_c01=delays[:, :2], sky_freq_hz=d.sky_freq_hz)
    tab = np.stack([delays[:, :1], np.zeros((2 * T, 1)), delays[::-1, :1]])   # matched, zero, wrong
    _, power, incoh = oracle.beamform(d, v, tab, int_frames=frames)
    src = [c for c in range(N) if (c - N // 2) % 2]               # channels holding the comb
    matched, unsteered, wrong = (power[b, 0, src].sum() for b in range(3))
    one_tile = incoh[0, :, src].sum() / T                          # signal + noise of one tile
    # signal (rms 12 per component) adds in amplitude over T tiles, noise (rms 4) in power:
    # matched / (T^2 one_tile) = (288 T^2 + 32 T) / (320 T^2) ~ 0.91 for T = 8
    assert 0.8 * T * T * one_tile < matched < 1.0 * T * T * one_tile
    assert unsteered < 0.3 * matched and wrong < 0.3 * matched
