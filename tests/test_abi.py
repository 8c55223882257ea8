"""The C-ABI library builds, loads and exports every entry point its header declares,
and rejects invalid plans with the documented status before touching the GPU."""
import os
import re

import pytest

import paper_2303_11557_b300 as mw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?\w[\w\s\*]*?\b(mwax_\w+)\s*\(", src, re.M))
    return names


def test_library_exports_every_declared_symbol():
    lib = mw.load_library()
    names = _declared()
    assert "mwax_correlate" in names and "mwax_plan_create" in names
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert set(mw.SYMBOLS) <= names


def test_version_and_no_error():
    assert "sm_103a" in mw.mwax_version()


@pytest.mark.parametrize("args,frag", [
    (dict(n_tiles=0, fft_len=128, fine_avg=1, int_time_s=0.4), "n_tiles"),
    (dict(n_tiles=4, fft_len=128, fine_avg=3, int_time_s=0.4), "fine_avg"),
    (dict(n_tiles=4, fft_len=128, fine_avg=1, int_time_s=0.4000001), "whole number"),
    (dict(n_tiles=4, fft_len=6400, fine_avg=1, int_time_s=0.001), "frames"),
    (dict(n_tiles=4, fft_len=128, fine_avg=1, int_time_s=0.4, samples_per_call=600_000), "multiple"),
    (dict(n_tiles=4, fft_len=128, fine_avg=1, int_time_s=0.4, block_samples=100), "block_samples"),
    (dict(n_tiles=4, fft_len=128, fine_avg=1, int_time_s=0.4, precision=mw.MWAX_INT8), "MWAX_INT8"),
    (dict(n_tiles=4, fft_len=128, fine_avg=1, int_time_s=0.4, precision=9), "precision"),
    (dict(n_tiles=4, fft_len=128, fine_avg=4, int_time_s=0.4, keep_bins=102), "keep_bins"),
    (dict(n_tiles=4, fft_len=128, fine_avg=4, int_time_s=0.4, keep_bins=132), "keep_bins"),
    (dict(n_tiles=4, fft_len=128, fine_avg=4, int_time_s=0.4, sample_rate_hz=-1.0), "sample_rate_hz"),
    # 0.1 s at 1,638,401 samples/s is not a whole number of samples
    (dict(n_tiles=4, fft_len=128, fine_avg=4, int_time_s=0.1, sample_rate_hz=1.6384e6 + 1), "whole number"),
])
def test_invalid_plans_rejected(args, frag):
    with pytest.raises(mw.MwaxError) as ei:
        mw.mwax_plan_create_ex(mw.PlanDesc(**args))
    assert ei.value.status == mw.MWAX_EINVAL
    assert frag in str(ei.value)


def test_unsupported_fft_length():
    with pytest.raises(mw.MwaxError) as ei:
        mw.mwax_plan_create_ex(mw.PlanDesc(n_tiles=2, fft_len=100, fine_avg=1, int_time_s=0.05))
    assert ei.value.status == mw.MWAX_EUNSUPPORTED
