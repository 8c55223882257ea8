"""Shared helpers of the GPU parity tests: workloads and the parity metric."""
import numpy as np

import oracle
import synth


def parity_error(vis_gpu, vis_ora, T):
    """err = |V_gpu - V_ora| / sqrt(V_ora,pp V_ora,qq), the autos being the parallel-pol
    autocorrelations of the same channel and integration (scale-free).
    vis_*: complex [ints, B, M, 4] in MWAX_ORDER.  Returns the error array."""
    B = T * (T + 1) // 2
    auto_b = np.array([i * (2 * T - i + 1) // 2 for i in range(T)])
    ti = np.concatenate([[i] * (T - i) for i in range(T)])
    tj = np.concatenate([np.arange(i, T) for i in range(T)])
    assert len(ti) == B
    err = np.empty(vis_ora.shape, dtype=np.float64)
    for pol in range(4):
        a, e = pol >> 1, pol & 1
        ap = np.abs(vis_ora[..., 3 * a].real)[:, auto_b[ti], :]   # xx (0) or yy (3) of tile i
        aq = np.abs(vis_ora[..., 3 * e].real)[:, auto_b[tj], :]
        err[..., pol] = np.abs(vis_gpu[..., pol] - vis_ora[..., pol]) / np.sqrt(ap * aq)
    return err


def workload(seed, T, n_samples, *, block_samples=64_000, delay="fixed", sky=synth.SKY_FREQ_HZ,
             sigma=16.0, rel_rms=0.3):
    """Seeded noise + point-source voltages and the per-path delay polynomial.
    delay: "fixed" (per tile, 0-50 ns), "linear" (per tile, c0 + c1 t), "quadratic" (a
    different c0 + c1 t + c2 t^2 on every path, c2 t^2 reaching 20 ns by the end of the
    call) or None (no correction; the source still carries the fixed delays)."""
    if delay == "fixed":
        dpoly = synth.tile_delays_fixed(T)
    elif delay == "linear":
        dpoly = synth.tile_delays_linear(seed, T)
    elif delay == "quadratic":
        dpoly = synth.path_delays_quadratic(seed, T, n_samples / synth.FS)
    else:
        dpoly = None
    src = dpoly if dpoly is not None else synth.tile_delays_fixed(T)
    volt = synth.voltages(seed, 2 * T, n_samples, block_samples=block_samples, sigma=sigma,
                          tones=synth.point_source_tones(seed, sigma=sigma, rel_rms=rel_rms),
                          delay_poly=src, sky_freq_hz=sky)
    return volt, dpoly


def oracle_desc(T, N, F, int_time_s, n_samples, block_samples=64_000, sky=synth.SKY_FREQ_HZ, keep_dc=0):
    K = int(round(int_time_s * synth.FS)) // N
    return oracle.Desc(n_tiles=T, fft_len=N, fine_avg=F, int_frames=K, n_samples=n_samples,
                       block_samples=block_samples, sky_freq_hz=sky, dc_exclude=0 if keep_dc else 1)


def baseline_index(T, i, j):
    return i * (2 * T - i + 1) // 2 + (j - i)


def sample_requests(seed, T, ints, M, per_int):
    """Random (integration, baseline, channel, pol) entries, plus the parallel-pol autos
    (same integration and channel) that the parity metric of each one divides by.
    Returns (requests int64 [R, 4] with the random entries first, their number, and the
    tile pair (i, j) of each random entry)."""
    rng = np.random.default_rng(seed)
    req = []
    for w in ints:
        for _ in range(per_int):
            i = int(rng.integers(0, T))
            j = int(rng.integers(i, T))
            req.append((w, baseline_index(T, i, j), int(rng.integers(0, M)), int(rng.integers(0, 4)), i, j))
    autos = set()
    for w, _, c, pol, i, j in req:
        autos.add((w, baseline_index(T, i, i), c, 3 * (pol >> 1)))
        autos.add((w, baseline_index(T, j, j), c, 3 * (pol & 1)))
    main = [r[:4] for r in req]
    return np.array(main + sorted(autos), dtype=np.int64), len(main), [(r[4], r[5]) for r in req]


def sampled_error(got, want, req, n_main, tiles, T):
    """The parity metric on sampled outputs (autos taken from the oracle's samples)."""
    look = {tuple(r): k for k, r in enumerate(req.tolist())}
    err = []
    for k in range(n_main):
        w, _, c, pol = req[k].tolist()
        i, j = tiles[k]
        ap = abs(want[look[(w, baseline_index(T, i, i), c, 3 * (pol >> 1))]].real)
        aq = abs(want[look[(w, baseline_index(T, j, j), c, 3 * (pol & 1))]].real)
        err.append(abs(got[k] - want[k]) / np.sqrt(ap * aq))
    return np.array(err)


# parity bars per precision (MWAX_* values: FP32 0, FP16 1, FP8 2, INT8 3, FP16X3 4)
TOL_BY_PREC = {0: 1e-5, 1: 2e-3, 2: 3e-2, 4: 1e-5}


def check_output_vs_oracle(T, N, F, int_time_s, n_samples, prec, volt, delay, vis, weights, keep_dc=0):
    """A call's split output (vis, weights as numpy) against the full FP64 oracle on the
    same inputs: integer mode bit-exact, float forms within their bar.  Returns the max
    parity error (0 for the integer mode)."""
    od = oracle_desc(T, N, F, int_time_s, n_samples, block_samples=volt.shape[2], keep_dc=keep_dc)
    if prec == 3:
        ref, rw = oracle.correlate_int(od, volt)
        assert np.array_equal(vis, ref), "integer mode differs from the oracle"
        assert np.array_equal(weights, rw.astype(np.float32))
        return 0.0
    ref, rw = oracle.correlate(od, volt, delay)
    assert vis.shape == ref.shape and np.array_equal(weights, rw.astype(np.float32))
    assert np.all(np.isfinite(vis))
    err = parity_error(vis, ref, T).max()
    assert err <= TOL_BY_PREC[prec], f"max err {err:.3e} (bar {TOL_BY_PREC[prec]:.0e})"
    return err
