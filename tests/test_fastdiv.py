"""Division by invariant integers (Granlund & Montgomery, PLDI 1994) as used
for stencil coordinates: for d >= 1, l = ceil(log2 d), m = floor(2^32
(2^l - d) / d) + 1, every x < 2^31 satisfies x // d == (umulhi(x, m) + x) >> l
and m fits in 32 bits.  The GPU parity tests exercise the device code on odd
and even grid sides; this pins the formula itself on many divisors."""
import random


def make(d):
    l = 0
    while (1 << l) < d:
        l += 1
    m = ((1 << 32) * ((1 << l) - d)) // d + 1
    return m, l


def test_fast_division_exact():
    rng = random.Random(0)
    ds = list(range(1, 1500)) + [rng.randint(1, (1 << 31) - 1) for _ in range(1500)]
    ds += [1 << k for k in range(31)] + [(1 << k) - 1 for k in range(1, 31)]
    for d in ds:
        m, l = make(d)
        assert 0 < m < (1 << 32)
        xs = [0, 1, d - 1, d, d + 1, (1 << 31) - 1] + [rng.randint(0, (1 << 31) - 1) for _ in range(200)]
        for x in xs:
            if x < (1 << 31):
                assert ((((x * m) >> 32) + x) >> l) == x // d, (x, d)
