"""The float-reciprocal division of the kernels' index arithmetic (FastDiv):
q = trunc(float(x) * float(1/d)) corrected once by the sign of x - q d.
Checked here in IEEE float32 arithmetic, which the device follows for these
operations (round-to-nearest conversion, product and reciprocal), over the
domain the kernels use it on: d < 2^14 and x < 2^28."""
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
