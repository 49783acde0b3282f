"""Integer-pipe arithmetic of the kernels, checked on the CPU in IEEE
arithmetic (which the device follows for these operations).

* FastDiv, the index division: q = trunc(float(x) * float(1/d)) corrected
  once by the sign of x - q d, over the domain the kernels use it on:
  d < 2^14 and x < 2^28.
* f64_to_f32 / f32_to_f64, the binary64 <-> binary32 conversions written on
  the IEEE 754 encodings: they must equal the round-to-nearest-even
  conversion and the exact widening (numpy's astype) on every normal value,
  including ties, carries into the exponent and the edges of the range."""
import numpy as np


def fastdiv(x, d):
    x = np.asarray(x, np.uint64)
    inv = np.float32(1.0) / np.float32(d)
    q = np.floor(x.astype(np.float32) * inv).astype(np.int64)
    rem = x.astype(np.int64) - q * int(d)
    q = np.where(rem < 0, q - 1, np.where(rem >= d, q + 1, q))
    rem = np.where(rem < 0, rem + d, np.where(rem >= d, rem - d, rem))
    return q, rem


def test_fastdiv_exact_on_the_kernels_domain():
    rng = np.random.default_rng(0)
    divisors = np.unique(np.concatenate([np.arange(1, 2050), 2 ** np.arange(14) - 1,
                                         2 ** np.arange(14), rng.integers(1, 2 ** 14, 2000)]))
    divisors = divisors[divisors >= 1]
    for d in divisors:
        d = int(d)
        limit = min(2 ** 28, d * 2 ** 20)          # x / d < 2^20 and x < 2^28
        x = np.concatenate([rng.integers(0, limit, 4000, dtype=np.int64),
                            np.arange(0, min(limit, 3 * d)),
                            # multiples of d and their neighbours, where truncation bites
                            ((rng.integers(0, limit // d, 500, dtype=np.int64) * d)[:, None]
                             + np.array([-1, 0, 1])[None, :]).ravel()])
        x = x[(x >= 0) & (x < limit)]
        q, r = fastdiv(x, d)
        assert np.array_equal(q, x // d), d
        assert np.array_equal(r, x % d), d


def test_one_correction_step_suffices():
    """The float quotient is within one of the true one before correction."""
    rng = np.random.default_rng(1)
    for d in (3, 7, 511, 1023, 2047, 4095, 16383):
        x = rng.integers(0, min(2 ** 28, d * 2 ** 20), 200000, dtype=np.int64)
        inv = np.float32(1.0) / np.float32(d)
        q0 = np.floor(x.astype(np.float32) * inv).astype(np.int64)
        assert np.max(np.abs(q0 - x // d)) <= 1


def f64_to_f32_bits(x):
    """The device routine on the encodings (numpy uint64 arithmetic)."""
    b = np.asarray(x, np.float64).view(np.uint64)
    out = np.empty(b.shape, np.float32)
    zero = (b << np.uint64(1)) == 0
    e = ((b >> np.uint64(52)) & np.uint64(0x7ff)).astype(np.int64) - 1023 + 127
    hw = ~zero & ((e <= 0) | (e >= 255))
    fast = ~zero & ~hw
    mant = ((b >> np.uint64(29)) & np.uint64(0x7fffff)).astype(np.uint64)
    rest = (b & np.uint64(0x1fffffff)).astype(np.uint64)
    f = ((b >> np.uint64(32)) & np.uint64(0x80000000)) | (np.clip(e, 0, 255).astype(np.uint64) << np.uint64(23)) | mant
    up = (rest > 0x10000000) | ((rest == 0x10000000) & ((mant & np.uint64(1)) == 1))
    f = f + up.astype(np.uint64)
    out[fast] = f[fast].astype(np.uint32).view(np.float32)
    out[zero] = (b[zero] >> np.uint64(32)).astype(np.uint32).view(np.float32)
    out[hw] = np.asarray(x, np.float64)[hw].astype(np.float32)
    return out


def f32_to_f64_bits(v):
    b = np.asarray(v, np.float32).view(np.uint32).astype(np.uint64)
    e = (b >> np.uint64(23)) & np.uint64(0xff)
    zero = (b & np.uint64(0x7fffffff)) == 0
    hw = ~zero & ((e == 0) | (e == 255))
    hi = (b & np.uint64(0x80000000)) | ((e + np.uint64(1023 - 127)) << np.uint64(20)) | ((b & np.uint64(0x7fffff)) >> np.uint64(3))
    lo = (b & np.uint64(7)) << np.uint64(29)
    out = ((hi << np.uint64(32)) | lo).view(np.float64).copy()
    out[zero] = ((b[zero] & np.uint64(0x80000000)) << np.uint64(32)).view(np.float64)
    out[hw] = np.asarray(v, np.float32)[hw].astype(np.float64)
    return out


def test_f64_to_f32_matches_round_to_nearest_even():
    rng = np.random.default_rng(2)
    x = np.concatenate([
        rng.standard_normal(200000) * 10.0 ** rng.integers(-40, 40, 200000),
        rng.uniform(-1, 1, 100000),
        [0.0, -0.0, 1.0, -1.0, 3.4028234663852886e38, 1.1754943508222875e-38, 1e-45, 1e39],
    ])
    # exact ties and their neighbours: a float32 value plus half an ulp
    f = rng.uniform(1, 2, 20000).astype(np.float32).astype(np.float64)
    ulp = np.spacing(f.astype(np.float32)).astype(np.float64)
    x = np.concatenate([x, f + ulp / 2, f - ulp / 2, f + ulp / 2 + ulp * 2 ** -20,
                        [np.nextafter(np.float64(np.float32(3.4028235e38)), 0)]])
    with np.errstate(over="ignore"):
        want = x.astype(np.float32)
        got = f64_to_f32_bits(x)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_f32_to_f64_is_exact_widening():
    rng = np.random.default_rng(3)
    v = np.concatenate([rng.integers(0, 2 ** 32, 500000, dtype=np.uint64).astype(np.uint32).view(np.float32),
                        np.array([0.0, -0.0, 1.0, 1e-45, -1e-40], np.float32)])
    v = v[np.isfinite(v)]
    assert np.array_equal(f32_to_f64_bits(v).view(np.uint64), v.astype(np.float64).view(np.uint64))
