"""The split compensation of the atomic force paths (edge, and the reactions of the Newton vertex path),
emulated in numpy FP32 on the CPU: each term t is split into q = (t + 1.5*2^15) - 1.5*2^15, its value rounded
to a multiple of 2^-8, and the remainder t - q; the q are summed in one FP32 accumulator and the remainders
in another.  These checks pin the arithmetic facts the kernels rely on:

- q is t rounded to the nearest multiple of 2^-8 (ties to even) for |t| < 2^14, and t - q is exact in FP32;
- FP32 sums of the q are exact, so independent of the order of the additions, while they stay below 2^16;
- hi + lo then carries the exact sum of the terms to far below the 1e-5 force-error bar.
"""
import numpy as np

MAGIC = np.float32(49152.0)  # 1.5 * 2^23 * 2^-8
SPLIT_MAX = np.float32(16384.0)
f32 = np.float32


def split(t):
    t = np.asarray(t, dtype=np.float32)
    q = np.where(np.abs(t) < SPLIT_MAX, (t + MAGIC) - MAGIC, t).astype(np.float32)
    return q, (t - q).astype(np.float32)


def fsum32(values):
    """Sequential FP32 sum, as a chain of atomic additions would form it in one order."""
    s = f32(0.0)
    for v in values:
        s = f32(s + f32(v))
    return s


def test_grid_part_is_round_to_nearest_multiple():
    rng = np.random.default_rng(11)
    t = np.concatenate([rng.normal(0, 30, 200000), rng.uniform(-16383, 16383, 200000),
                        (rng.integers(-4000, 4000, 1000) + 0.5) / 256.0]).astype(np.float32)  # exact ties
    q, r = split(t)
    want = np.round(t.astype(np.float64) * 256.0) / 256.0  # numpy rounds half to even
    assert np.array_equal(q.astype(np.float64), want)
    assert np.all(np.abs(r) <= 2.0 ** -9)
    # the remainder is exact: q + r == t in exact arithmetic
    assert np.array_equal(q.astype(np.float64) + r.astype(np.float64), t.astype(np.float64))


def test_large_terms_go_to_the_grid_accumulator_whole():
    t = np.array([16384.0, -20000.5, 1.0e6, -16384.0], dtype=np.float32)
    q, r = split(t)
    assert np.array_equal(q, t) and np.all(r == 0.0)


def test_grid_sums_do_not_depend_on_order():
    rng = np.random.default_rng(12)
    t = (rng.standard_t(3, 500) * 20.0).astype(np.float32)  # heavy-tailed, like pair forces
    q, _ = split(t)
    assert np.abs(q.astype(np.float64)).sum() < 2 ** 16  # every partial sum, in any order, stays below 2^16
    sums = {float(fsum32(q[rng.permutation(t.size)])) for _ in range(8)}
    assert len(sums) == 1
    # exact: equal to the FP64 sum of the same grid parts
    assert sums.pop() == float(q.astype(np.float64).sum())
    # plain FP32 sums of the terms themselves do depend on the order
    plain = {float(fsum32(t[rng.permutation(t.size)])) for _ in range(8)}
    assert len(plain) > 1


def test_grid_part_plus_remainder_carries_the_exact_sum():
    rng = np.random.default_rng(13)
    worst = 0.0
    for _ in range(50):
        k = int(rng.integers(20, 120))  # contributions to one particle
        t = (rng.standard_t(3, k) * 20.0).astype(np.float32)
        q, r = split(t)
        order = rng.permutation(k)
        hi, lo = fsum32(q[order]), fsum32(r[order])
        exact = t.astype(np.float64).sum()
        worst = max(worst, abs((float(hi) + float(lo)) - exact))
    # against forces of order 1-100 (F_rms ~ 20 in the LJ liquid) this is below 1e-9 relative
    assert worst < 1e-7
