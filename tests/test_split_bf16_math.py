"""The split-BF16 product used by the tensor-core GEMM steps, checked on the CPU
with BF16 rounding written out (round to nearest even on the upper 16 bits of
an FP32 value).  Each FP32 value x is x0 + x1 + x2, x0 = bf16(x),
x1 = bf16(x - x0), x2 = bf16(x - x0 - x1); a product keeps the six term
products x_i y_j with i + j <= 2.  Claims: the differences are exact in FP32
and the three terms give x back exactly (8 significant bits each, 24 in all:
FP32's), and the six products give x y to 2^-24 of |x y|, the FP32 level the
kernel's accuracy rests on."""
import numpy as np

RNG = np.random.default_rng(20171214)


def bf16(x: np.ndarray) -> np.ndarray:
    """FP32 -> nearest BF16 (ties to even), returned as FP32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def split3(x: np.ndarray):
    x = np.asarray(x, dtype=np.float32)
    x0 = bf16(x)
    r1 = (x - x0).astype(np.float32)
    x1 = bf16(r1)
    r2 = (r1 - x1).astype(np.float32)
    x2 = bf16(r2)
    return x0, x1, x2, r1, r2


def samples(n=200000):
    mant = RNG.uniform(1.0, 2.0, n)
    expo = RNG.integers(-40, 40, n)
    sign = RNG.choice([-1.0, 1.0], n)
    return (sign * mant * 2.0 ** expo).astype(np.float32)


def test_bf16_rounding_is_nearest_even():
    # values exactly representable stay; halfway cases go to the even neighbour
    assert bf16(np.float32(1.0)) == 1.0
    assert bf16(np.float32(1.0 + 2 ** -8)) == 1.0               # halfway, 1.0 is even
    assert bf16(np.float32(1.0 + 3 * 2 ** -8)) == 1.0 + 2 ** -6  # halfway, rounds up to even
    assert bf16(np.float32(1.0 + 2 ** -7 + 2 ** -20)) == 1.0 + 2 ** -7
    x = samples(10000)
    e = np.abs(bf16(x).astype(np.float64) - x) / np.abs(x.astype(np.float64))
    assert e.max() <= 2.0 ** -8   # half an ulp of an 8-bit significand


def test_three_terms_reconstruct_fp32():
    x = samples()
    x0, x1, x2, r1, r2 = split3(x)
    xd = x.astype(np.float64)
    # the differences are exact in FP32
    assert np.array_equal(r1.astype(np.float64), xd - x0.astype(np.float64))
    assert np.array_equal(r2.astype(np.float64), r1.astype(np.float64) - x1.astype(np.float64))
    rec = x0.astype(np.float64) + x1.astype(np.float64) + x2.astype(np.float64)
    assert np.array_equal(rec, xd)
    # each term is at most about 2^-8 of the one before
    nz = x1 != 0
    assert np.all(np.abs(x1[nz]) <= 2.0 ** -7 * np.abs(x0[nz]))
    nz = x2 != 0
    assert np.all(np.abs(x2[nz]) <= 2.0 ** -7 * np.abs(x1[nz]))


def test_six_term_products_reach_fp32_accuracy():
    x, y = samples(), samples()
    xs, ys = split3(x)[:3], split3(y)[:3]
    six = sum(xs[i].astype(np.float64) * ys[j].astype(np.float64)
              for i in range(3) for j in range(3) if i + j <= 2)
    exact = x.astype(np.float64) * y.astype(np.float64)
    rel = np.abs(six - exact) / np.abs(exact)
    assert rel.max() <= 2.0 ** -24
    # two terms per value would not do: the error is near 2^-17
    two = sum(xs[i].astype(np.float64) * ys[j].astype(np.float64)
              for i in range(2) for j in range(2) if i + j <= 1)
    assert (np.abs(two - exact) / np.abs(exact)).max() > 2.0 ** -20


def test_complex_product_with_negated_imaginary_part():
    # re = ar br - ai bi with -ai split by flipping the sign of its terms
    ar, ai, br, bi = samples(), samples(), samples(), samples()
    sar, sai, sbr, sbi = (split3(v)[:3] for v in (ar, ai, br, bi))
    nai = tuple(-t for t in sai)
    assert all(np.array_equal(a, b) for a, b in zip(split3(-ai)[:3], nai))

    def prod(a, b):
        return sum(a[i].astype(np.float64) * b[j].astype(np.float64)
                   for i in range(3) for j in range(3) if i + j <= 2)

    re = prod(sar, sbr) + prod(nai, sbi)
    im = prod(sar, sbi) + prod(sai, sbr)
    a = ar.astype(np.float64) + 1j * ai.astype(np.float64)
    b = br.astype(np.float64) + 1j * bi.astype(np.float64)
    z = a * b
    scale = np.abs(a) * np.abs(b)
    assert np.max(np.abs(re + 1j * im - z) / scale) <= 2.0 ** -23
