"""The FP8 form's two scale sources against the FP64 oracle at the FP8 bar: e4m3 written by
the F-step with the plan's static per-group scales (the bound 181.02 N max gain of a group,
F-step variants 0 and 3), and e4m3 quantised from an FP16 F-step with measured per-path
maxima (variant 2).  Inputs at both ends of the range: a full-scale square-wave tone on
an FFT bin (every path; each sample near the int8 corner 127 (+-1 +-i) in the quadrant of
the tone's phase, so the bin reaches about 0.88 of the bound and nothing may saturate; a
little seeded noise keeps every channel's autocorrelation, the metric's scale, non-zero;
the tone sits 0.013 bin off centre so that its phase turns from frame to frame: a tone
repeating the same value in every frame would repeat the same e4m3 rounding, a bias of up
to 2^-4 that the bar, set for noise-like skies, does not cover) and a weak noise floor
(sigma 2: the values sit low in e4m3's range)."""
import numpy as np
import pytest

import paper_2303_11557_b300 as mw
import synth
from _parity import check_output_vs_oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _tone_volt(T, N, S, bs, k0, seed=0xF8):
    """Full-scale square-wave complex tone at bin k0: the int8 corner 127 (+-1 +-i) in the
    quadrant of exp(2 pi i k0 n / N), plus seeded noise (sigma 3, clipped to int8), on
    every path."""
    n = np.arange(S)
    ph = 2.0 * np.pi * (k0 + 0.013) * n / N
    rng = np.random.default_rng(seed)
    v = np.empty((S // bs, 2 * T, bs, 2), np.int8)
    for b in range(S // bs):
        sl = slice(b * bs, (b + 1) * bs)
        for q in range(2 * T):
            nz = rng.normal(0.0, 3.0, (bs, 2))
            v[b, q, :, 0] = np.clip(np.rint(np.where(np.cos(ph[sl]) >= 0.0, 127.0, -127.0) + nz[:, 0]), -128, 127)
            v[b, q, :, 1] = np.clip(np.rint(np.where(np.sin(ph[sl]) >= 0.0, 127.0, -127.0) + nz[:, 1]), -128, 127)
    return v


def _run(desc, volt, variant):
    plan = mw.mwax_plan_create_ex(desc)
    mw.mwax_plan_set_stream(plan)
    t = mw.mwax_plan_get_tuning(plan)
    mw.mwax_plan_set_tuning(plan, mw.Tuning(variant, t.run_len, t.window, 0.0))
    out = mw.empty_output(plan)
    out.fill_(0xAB)
    mw.mwax_correlate(plan, torch.from_numpy(volt.reshape(-1)).cuda(), None, out)
    mw.mwax_plan_sync(plan)
    vis, w = mw.split_output(plan, out)
    res = vis.cpu().numpy(), w.cpu().numpy()
    plan.close()
    return res


CASES = [pytest.param(128, 4, 0, id="n128-fstep-e4m3"), pytest.param(1280, 10, 3, id="n1280-row128-e4m3"),
         pytest.param(1280, 10, 2, id="n1280-fourstep-maxima")]


@pytest.mark.parametrize("N,F,variant", CASES)
@pytest.mark.parametrize("signal", ["tone", "weak"])
def test_fp8_scales_full_scale_tone_and_weak_floor(N, F, variant, signal):
    T, bs = 4, 64_000
    S = 2 * bs
    if signal == "tone":
        volt = _tone_volt(T, N, S, bs, k0=N // 4 + 3)
    else:
        volt = synth.voltages(0xF8 + N, 2 * T, S, block_samples=bs, sigma=2.0)
    int_time = bs / synth.FS
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=int_time, samples_per_call=S, block_samples=bs,
                       sky_freq_hz=synth.SKY_FREQ_HZ, precision=mw.MWAX_FP8)
    vis, w = _run(desc, volt, variant)
    check_output_vs_oracle(T, N, F, int_time, S, mw.MWAX_FP8, volt, None, vis, w)
