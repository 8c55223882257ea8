"""GPU parity of the tied-array beamformer (Sec. 4.4) through the C ABI against the FP64
oracle on seeded inputs: coherent beams element by element (relative to the beam's own
power scale per channel), detected Stokes I and the incoherent beam (relative), at the
FP32 bar for both engines (tensor cores from FP16 hi/lo pairs, and FP32 CUDA cores).
Covers tables whose steps split frames, more beams than one CTA's group, ragged tile
counts and frame counts that are not multiples of the CTA's frame block."""
import numpy as np
import pytest

import oracle
import paper_2303_11557_b300 as mw
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-5


ENGINES = [pytest.param(0, id="tensor"), pytest.param(1, id="cuda")]


def run(T, N, nb, S, bs, step, int_frames, seed, steps_extra=0, host_table=False, engine=0):
    tones = synth.point_source_tones(seed, sigma=16.0, rel_rms=0.5)
    delays = synth.tile_delays_linear(seed, T, max_c0=400e-9, max_c1=0.0)
    volt = synth.voltages(seed, 2 * T, S, block_samples=bs, sigma=16.0, tones=tones, delay_c01=delays[:, :2],
                          sky_freq_hz=synth.SKY_FREQ_HZ)
    steps = -(-S // step) + steps_extra
    rng = np.random.default_rng(seed)
    tab = rng.uniform(0, 400e-9, (nb, 2 * T, 1)) + rng.uniform(-3e-9, 3e-9, (nb, 2 * T, steps)).cumsum(axis=2)
    tab[0] = delays[:, :1]                                   # beam 0 points at the source
    bf = mw.Beamformer(T, N, nb, S, block_samples=bs, sky_freq_hz=synth.SKY_FREQ_HZ, table_step_samples=step,
                       int_frames=int_frames, engine=engine)
    bf.set_stream()
    dv = torch.from_numpy(volt.reshape(-1)).cuda()
    beams = torch.empty(bf.output_bytes(0), dtype=torch.uint8, device="cuda")
    power = torch.empty(max(4, bf.output_bytes(1)), dtype=torch.uint8, device="cuda") if int_frames else None
    incoh = torch.empty(max(4, bf.output_bytes(2)), dtype=torch.uint8, device="cuda") if int_frames else None
    t = tab if host_table else torch.from_numpy(tab).cuda()
    bf.form(dv, t, beams, None if power is None else power.view(torch.float32),
            None if incoh is None else incoh.view(torch.float32))
    bf.sync()
    frames = S // N
    B = torch.view_as_complex(beams.view(torch.float32).view(nb, 2, frames, N, 2)).cpu().numpy()
    d = oracle.Desc(n_tiles=T, fft_len=N, fine_avg=1, int_frames=frames, n_samples=S, block_samples=bs,
                    sky_freq_hz=synth.SKY_FREQ_HZ)
    rb, rp, ri = oracle.beamform(d, volt, tab, table_step=step, int_frames=int_frames)
    # coherent beams: error relative to the rms beam amplitude of that beam/pol/channel
    scale = np.sqrt(np.mean(np.abs(rb) ** 2, axis=2, keepdims=True))
    err = np.abs(B - rb) / scale
    assert err.max() <= TOL, f"beam err {err.max():.3e}"
    if int_frames:
        nd = frames // int_frames
        P = power.view(torch.float32)[: nb * nd * N].view(nb, nd, N).cpu().numpy()
        I = incoh.view(torch.float32)[: nd * 2 * N].view(nd, 2, N).cpu().numpy()
        assert np.abs(P - rp).max() / np.abs(rp).max() <= TOL
        np.testing.assert_allclose(I, ri, rtol=TOL)
        # the beam steered at the source collects more power than the others
        assert rp[0].sum() > rp[1:].sum(axis=(1, 2)).max()
    return err


@pytest.mark.parametrize("engine", ENGINES)
def test_beams_n128(engine):
    run(T=16, N=128, nb=4, S=64_000 * 2, bs=64_000, step=6400, int_frames=100, seed=11, engine=engine)


@pytest.mark.parametrize("engine", ENGINES)
def test_beams_n512_split_frames_many_beams(engine):
    # 512-sample frames straddle 6,400-sample steps; 11 beams = two CUDA-core beam groups
    run(T=12, N=512, nb=11, S=64_000, bs=64_000, step=6400, int_frames=25, seed=12, engine=engine)


@pytest.mark.parametrize("engine", ENGINES)
def test_beams_n32_ragged_tiles_host_table(engine):
    # T = 19 is not a multiple of the 16-tile chunk; table longer than needed; host table;
    # 200 frames per 3,200-sample step: two units of the tensor-core engine's 128 frames
    run(T=19, N=32, nb=3, S=32_000, bs=6400, step=3200, int_frames=0, seed=13, steps_extra=5, host_table=True,
        engine=engine)


@pytest.mark.parametrize("engine", ENGINES)
def test_beams_n6400_one_frame_per_step(engine):
    run(T=8, N=6400, nb=2, S=64_000 * 2, bs=64_000, step=6400, int_frames=4, seed=14, engine=engine)


def test_beams_tensor_engine_many_tiles_and_beams():
    # 70 tiles (two 64-tile K chunks, the second ragged) and 20 beams (two 16-beam groups),
    # a 7,000-sample step (not a multiple of the 128-point frame: steps split frames)
    run(T=70, N=128, nb=20, S=64_000, bs=64_000, step=7000, int_frames=50, seed=15, engine=0)


def test_beamformer_errors():
    with pytest.raises(mw.MwaxError):
        mw.Beamformer(4, 1, 2, 64_000)                       # no FFT: not a beamformer length
    with pytest.raises(mw.MwaxError):
        mw.Beamformer(4, 128, 0, 64_000)                     # no beams
    bf = mw.Beamformer(4, 128, 2, 64_000)                    # no int_frames: no detected outputs
    bf.set_stream()
    v = torch.zeros(64_000 * 8 * 2, dtype=torch.int8, device="cuda")
    out = torch.empty(bf.output_bytes(0), dtype=torch.uint8, device="cuda")
    pw = torch.empty(16, dtype=torch.float32, device="cuda")
    with pytest.raises(mw.MwaxError, match="int_frames"):
        bf.form(v, np.zeros((2, 8, 10)), out, pw)
