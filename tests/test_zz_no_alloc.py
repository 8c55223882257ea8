"""The allocation-free entry point, for callers that cannot allocate device memory
(a process whose GPU memory belongs to another allocator, a plug-in forbidden to
allocate, a service that bans allocation after start-up), against the regular plan-based
call and against the FP64 oracle: two calls in a row on different inputs over the shared
device arrays, each within the FP32 bar (1e-5 of the auto scale) of both, for a delay
polynomial that is absent, in host memory or in device memory, and for two averaging
shapes; the size limit and the alignment rule are enforced.  Collected last (file name)
so a failure here cannot hide any other test's result."""
import numpy as np
import pytest

import paper_2303_11557_b300 as mw
import synth
from _parity import check_output_vs_oracle, parity_error, workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _plan_result(desc, volt, delay):
    plan = mw.mwax_plan_create_ex(desc)
    mw.mwax_plan_set_stream(plan)
    out = mw.empty_output(plan)
    dd = None if delay is None else torch.from_numpy(delay).cuda()
    mw.mwax_correlate(plan, torch.from_numpy(volt.reshape(-1)).cuda(), dd, out)
    mw.mwax_plan_sync(plan)
    vis, w = mw.split_output(plan, out)
    res = vis.cpu().numpy(), w.cpu().numpy(), plan.output_bytes
    plan.close()
    return res


@pytest.mark.parametrize("where", ["none", "host", "device"])
@pytest.mark.parametrize("F,keep_dc", [(1, 0), (4, 1)])
def test_noalloc_matches_plan_and_oracle_on_two_calls(where, F, keep_dc):
    T, N, t, S = 12, 128, 0.05, 128_000
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=t, samples_per_call=S,
                       sky_freq_hz=synth.SKY_FREQ_HZ, keep_dc=keep_dc)
    for seed in (1201, 1202):   # second call: new data over the shared device arrays
        volt, delay = workload(seed, T, S, delay=None if where == "none" else "quadratic")
        ref, ref_w, nbytes = _plan_result(desc, volt, delay)
        out = torch.empty(nbytes, dtype=torch.uint8, device="cuda").fill_(0xCD)
        d_arg = {"none": None, "host": delay, "device": None if delay is None else torch.from_numpy(delay).cuda()}[where]
        mw.mwax_correlate_noalloc(desc, torch.from_numpy(volt.reshape(-1)).cuda(), d_arg, out)
        torch.cuda.synchronize()
        n_ints, B, M = ref.shape[0], ref.shape[1], ref.shape[2]
        per = B * M * 32 + B * 16
        raw = out.cpu().numpy().reshape(n_ints, per)
        vis = raw[:, :B * M * 32].copy().view(np.complex64).reshape(n_ints, B, M, 4)
        w = raw[:, B * M * 32:].copy().view(np.float32).reshape(n_ints, B, 4)
        assert np.array_equal(w, ref_w) and np.all(w == 1.0)   # all weights 0 would flag a device timeout
        assert parity_error(vis, ref, T).max() <= 1e-5
        check_output_vs_oracle(T, N, F, t, S, mw.MWAX_FP32, volt, delay, vis, w, keep_dc=keep_dc)


def test_noalloc_rejects_jobs_beyond_its_arrays():
    desc = mw.PlanDesc(n_tiles=32, fft_len=512, fine_avg=1, int_time_s=0.2, samples_per_call=512_000)
    out = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    volt = torch.zeros(512_000 * 64 * 2, dtype=torch.int8, device="cuda")
    with pytest.raises(mw.MwaxError) as ei:
        mw.mwax_correlate_noalloc(desc, volt, None, out)
    assert ei.value.status == mw.MWAX_EINVAL and "32 MiB" in str(ei.value)


def test_noalloc_rejects_misaligned_buffers():
    T, N, S = 2, 64, 64_000
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=1, int_time_s=0.05, samples_per_call=S)
    volt = torch.zeros(S * 2 * T * 2 + 16, dtype=torch.int8, device="cuda")
    out = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    for v, o in ((volt[1:1 + S * 2 * T * 2], out), (volt[:S * 2 * T * 2], out[4:])):
        with pytest.raises(mw.MwaxError) as ei:
            mw.mwax_correlate_noalloc(desc, v, None, o)
        assert ei.value.status == mw.MWAX_EINVAL and "aligned" in str(ei.value)
