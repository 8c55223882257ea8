"""Failure detection without a GPU fault: every device-side wait of the X-step kernels is
bounded.  A plan whose bound is set to 1,000 cycles cannot finish its tensor-core X-step
(one accumulator group alone takes far longer), so a wait runs out: the kernel raises its
abort flag, lets its own TMA loads and MMAs in flight complete (a fixed ~2 s drain bound
that does not follow the limit), frees its tensor memory and returns, and
mwax_plan_sync() reports MWAX_ETIMEOUT.  The same plan, with the default bound restored,
then runs again on the same context and matches the FP64 oracle."""
import numpy as np
import pytest

import paper_2303_11557_b300 as mw
import synth
from _parity import check_output_vs_oracle, workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = [
    pytest.param(mw.MWAX_FP16, 128, 4, id="fp16"),
    pytest.param(mw.MWAX_FP16X3, 128, 4, id="fp16x3"),
    pytest.param(mw.MWAX_INT8, 1, 1, id="int8"),
]


def _run(plan, volt_d, delay_d):
    out = mw.empty_output(plan)
    out.fill_(0xAB)
    mw.mwax_correlate(plan, volt_d, delay_d, out)
    return out


@pytest.mark.parametrize("prec,N,F", CASES)
def test_wait_bound_runs_out_then_plan_recovers(prec, N, F):
    T, t, S = 24, 0.05, 128_000
    volt, delay = workload(0x71 + prec, T, S, delay=None if prec == mw.MWAX_INT8 else "quadratic")
    plan = mw.mwax_plan_create_ex(mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=t, samples_per_call=S,
                                              precision=prec, sky_freq_hz=synth.SKY_FREQ_HZ))
    mw.mwax_plan_set_stream(plan)
    vd = torch.from_numpy(volt.reshape(-1)).cuda()
    dd = None if delay is None else torch.from_numpy(delay).cuda()
    mw.mwax_plan_set_wait_limit(plan, 1)
    _run(plan, vd, dd)
    with pytest.raises(mw.MwaxError) as ei:
        mw.mwax_plan_sync(plan)
    assert ei.value.status == mw.MWAX_ETIMEOUT
    # the status word was cleared by the sync; the default bound gives a correct result
    mw.mwax_plan_set_wait_limit(plan, 0)
    out = _run(plan, vd, dd)
    mw.mwax_plan_sync(plan)
    vis, w = mw.split_output(plan, out)
    check_output_vs_oracle(T, N, F, t, S, prec, volt, delay, vis.cpu().numpy(), w.cpu().numpy())
    plan.close()


def test_fp32_tiny_wait_bound_reports_or_completes_then_recovers():
    # The CUDA-core FP32 X-step waits only for its own TMA ring, which may keep up even
    # at 1,000 cycles: either outcome is allowed, but a wait that ran out must be
    # reported, and the plan must work afterwards.
    T, N, F, t, S = 24, 128, 4, 0.05, 128_000
    volt, delay = workload(0x70, T, S, delay="quadratic")
    plan = mw.mwax_plan_create_ex(mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=F, int_time_s=t, samples_per_call=S,
                                              sky_freq_hz=synth.SKY_FREQ_HZ))
    mw.mwax_plan_set_stream(plan)
    vd, dd = torch.from_numpy(volt.reshape(-1)).cuda(), torch.from_numpy(delay).cuda()
    mw.mwax_plan_set_wait_limit(plan, 1)
    _run(plan, vd, dd)
    try:
        mw.mwax_plan_sync(plan)
    except mw.MwaxError as e:
        assert e.status == mw.MWAX_ETIMEOUT
    mw.mwax_plan_set_wait_limit(plan, 0)
    out = _run(plan, vd, dd)
    mw.mwax_plan_sync(plan)
    vis, w = mw.split_output(plan, out)
    check_output_vs_oracle(T, N, F, t, S, mw.MWAX_FP32, volt, delay, vis.cpu().numpy(), w.cpu().numpy())
    plan.close()
