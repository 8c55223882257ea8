"""Host-side check of the arithmetic the FP16 hi/lo pair form (MWAX_FP16X3) relies on,
with numpy's IEEE half precision: a pre-scaled FP32 spectral value v is held as
hi = fp16(v), lo = fp16(v - hi), and a complex product is formed from the FP16 parts as
Ah Bh + Ah Bl + Al Bh (the Al Bl term dropped).  Every FP16 x FP16 product is exact in FP32
(11 x 11 significant bits), so the only errors are the representation of v and the dropped
term; both are checked against float64 here.  No GPU."""
import numpy as np

RNG = np.random.default_rng(0xF16)


def split(v: np.ndarray):
    """hi = fp16(v), lo = fp16(v - hi); v - hi is exact in FP32."""
    v = v.astype(np.float32)
    hi = v.astype(np.float16)
    lo = (v - hi.astype(np.float32)).astype(np.float16)
    return hi, lo


def operand_values(n: int) -> np.ndarray:
    # pre-scaled FFT outputs: |v| up to 2^15, with a spread of magnitudes down to ~1
    mag = np.exp2(RNG.uniform(0.0, 15.0, n))
    return (RNG.choice([-1.0, 1.0], n) * mag).astype(np.float32)


def test_pair_represents_value_to_22_bits():
    v = operand_values(200_000)
    hi, lo = split(v)
    rep = hi.astype(np.float64) + lo.astype(np.float64)
    # hi carries 11 significant bits, lo the next 11 (its own rounding: half an ulp of lo)
    assert np.all(np.abs(rep - v.astype(np.float64)) <= np.abs(v.astype(np.float64)) * 2.0 ** -22)
    # the remainder is exactly representable in FP32 (no rounding in v - hi)
    d = v.astype(np.float64) - hi.astype(np.float64)
    assert np.array_equal(d.astype(np.float32).astype(np.float64), d)


def test_fp16_products_exact_in_fp32():
    a = operand_values(100_000).astype(np.float16)
    b = operand_values(100_000).astype(np.float16)
    exact = a.astype(np.float64) * b.astype(np.float64)
    assert np.array_equal((a.astype(np.float32) * b.astype(np.float32)).astype(np.float64), exact)


def test_three_product_complex_term_at_fp32_level():
    n = 100_000
    ar, ai, br, bi = (operand_values(n) for _ in range(4))
    (arh, arl), (aih, ail), (brh, brl), (bih, bil) = (split(x) for x in (ar, ai, br, bi))
    f = lambda x: x.astype(np.float64)
    # Re, Im of A conj(B) from the three products per real term, as the MMAs form them
    re = (f(arh) * f(brh) + f(arh) * f(brl) + f(arl) * f(brh)) + (f(aih) * f(bih) + f(aih) * f(bil) + f(ail) * f(bih))
    im = (f(aih) * f(brh) + f(aih) * f(brl) + f(ail) * f(brh)) - (f(arh) * f(bih) + f(arh) * f(bil) + f(arl) * f(bih))
    re_x = f(ar) * f(br) + f(ai) * f(bi)
    im_x = f(ai) * f(br) - f(ar) * f(bi)
    scale = np.sqrt((f(ar) ** 2 + f(ai) ** 2) * (f(br) ** 2 + f(bi) ** 2))   # |A| |B|
    err = np.maximum(np.abs(re - re_x), np.abs(im - im_x)) / scale
    # representation (2 x 2^-22 per factor) plus the dropped lo x lo term (2^-22 x 2^-22)
    assert err.max() < 4.0 * 2.0 ** -22, err.max()
    # and it is far better than one FP16 product per term (the FP16 form's operands)
    re16 = f(ar.astype(np.float16)) * f(br.astype(np.float16)) + f(ai.astype(np.float16)) * f(bi.astype(np.float16))
    assert np.median(np.abs(re16 - re_x) / scale) > 100 * np.median(np.abs(re - re_x) / scale)
