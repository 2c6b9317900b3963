"""The split-FP16 product used by the tensor-core GEMM steps by default,
checked on the CPU with FP16 rounding from numpy (IEEE binary16, round to
nearest even, as the kernels' FP32 -> FP16 conversion).  Each tensor is first
scaled by a power of two so that its largest modulus lies in [2^14, 2^15);
each scaled FP32 value x is h + l with h = fp16(x), l = fp16(x - h); a real
product keeps h h' + h l' + l h' (three MMAs), dropping l l'.  Claims: x - h
is exact in FP32; h + l holds x to 2^-22 of |x| while l is a normal FP16
number (and to 2^-25 absolutely below that, far under the scaled maximum's
FP32 ulp); the three kept products give x y to 2^-20 of |x y|; dropping any
of them loses the low half."""
import numpy as np

RNG = np.random.default_rng(20171215)


def fp16(x):
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float32)


def split2(x):
    x = np.asarray(x, dtype=np.float32)
    h = fp16(x)
    r = (x - h).astype(np.float32)
    return h, fp16(r), r


def scaled_samples(n=200000, lo=-24, hi=15):
    # moduli 2^lo .. 2^hi: the range a tensor scaled to a maximum in
    # [2^14, 2^15) occupies down to 2^-38 of its maximum
    mant = RNG.uniform(1.0, 2.0, n)
    expo = RNG.integers(lo, hi, n)
    sign = RNG.choice([-1.0, 1.0], n)
    return (sign * mant * 2.0 ** expo).astype(np.float32)


def test_fp16_rounding_is_nearest_even():
    assert fp16(np.float32(1.0 + 2 ** -11)) == 1.0                 # halfway, 1.0 is even
    assert fp16(np.float32(1.0 + 3 * 2 ** -11)) == 1.0 + 2 ** -9    # halfway, up to even
    assert fp16(np.float32(2 ** 15)) == 2 ** 15
    x = scaled_samples(20000, -14, 15)
    e = np.abs(fp16(x).astype(np.float64) - x) / np.abs(x.astype(np.float64))
    assert e.max() <= 2.0 ** -11


def test_two_terms_hold_22_bits():
    x = scaled_samples()
    h, l, r = split2(x)
    xd = x.astype(np.float64)
    # the difference is exact in FP32
    assert np.array_equal(r.astype(np.float64), xd - h.astype(np.float64))
    err = np.abs(h.astype(np.float64) + l.astype(np.float64) - xd)
    normal_l = np.abs(r) >= 2.0 ** -14
    assert np.all(err[normal_l] <= 2.0 ** -22 * np.abs(xd[normal_l]))
    # below the normal range of l: half of FP16's smallest subnormal
    assert np.all(err <= np.maximum(2.0 ** -22 * np.abs(xd), 2.0 ** -25))


def test_three_term_products_reach_20_bits():
    x = scaled_samples(200000, 8, 15)
    y = scaled_samples(200000, 8, 15)
    (hx, lx, _), (hy, ly, _) = split2(x), split2(y)
    f = lambda a: a.astype(np.float64)
    three = f(hx) * f(hy) + f(hx) * f(ly) + f(lx) * f(hy)
    exact = f(x) * f(y)
    rel = np.abs(three - exact) / np.abs(exact)
    assert rel.max() <= 2.0 ** -20
    # the high terms alone are FP16's 11 bits
    assert (np.abs(f(hx) * f(hy) - exact) / np.abs(exact)).max() > 2.0 ** -13


def test_small_values_lose_only_absolute_accuracy():
    # entries far below the tensor's maximum (2^14 .. 2^15): the error stays
    # below 2^-25 absolute, i.e. 2^-39 of the maximum
    x = scaled_samples(50000, -24, -3)
    h, l, _ = split2(x)
    err = np.abs(h.astype(np.float64) + l.astype(np.float64) - x.astype(np.float64))
    assert err.max() <= 2.0 ** -25


def test_complex_product_with_negated_imaginary_part():
    ar, ai, br, bi = (scaled_samples(100000, 8, 15) for _ in range(4))
    sar, sai, sbr, sbi = (split2(v)[:2] for v in (ar, ai, br, bi))
    nai = tuple(-t for t in sai)
    assert all(np.array_equal(a, b) for a, b in zip(split2(-ai)[:2], nai))

    def prod(a, b):
        f = lambda t: t.astype(np.float64)
        return f(a[0]) * f(b[0]) + f(a[0]) * f(b[1]) + f(a[1]) * f(b[0])

    re = prod(sar, sbr) + prod(nai, sbi)
    im = prod(sar, sbi) + prod(sai, sbr)
    a = ar.astype(np.float64) + 1j * ai.astype(np.float64)
    b = br.astype(np.float64) + 1j * bi.astype(np.float64)
    z = a * b
    assert np.max(np.abs(re + 1j * im - z) / (np.abs(a) * np.abs(b))) <= 2.0 ** -19
