"""The integration kernel's colour running average divides by 2 (w + 1),
w = 0..255 the colour weight, through a multiply-high by ceil(2^32 / d)
(Granlund and Montgomery's division by invariant integers).  Check on the CPU,
for every divisor and every dividend the blend can produce (< 2^17), that the
quotient equals floor division exactly."""
import numpy as np


def test_multiply_high_division_exact_for_colour_blend():
    n = np.arange(0, 1 << 17, dtype=np.uint64)
    # the largest dividend of the blend: 2 (255 * 255 + 255) + 255 + 1
    assert 2 * (255 * 255 + 255) + 256 < (1 << 17)
    for w in range(256):
        d = 2 * (w + 1)
        m = ((1 << 32) + d - 1) // d
        q = (n * np.uint64(m)) >> np.uint64(32)
        assert np.array_equal(q, n // np.uint64(d)), w
