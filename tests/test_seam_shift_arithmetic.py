"""The binary32 identities behind the seam-shifted staging of the pair tiles.

A tile whose halo crosses a periodic seam of a box [0, L) stages the
coordinates on one side of the seam shifted by L. The kernels rely on:
- x - L is exact for L/2 <= x < L (Sterbenz), and adding L back gives x;
- the plain difference of the staged coordinates of a pair across the seam
  equals the periodic displacement x_a - x_b -/+ L rounded once, which is
  what the per-pair seam path obtains with a two-sum (the image shift
  applied to the rounded difference, the rounding error added back).
Checked here with numpy binary32 arithmetic on random coordinates near the
seam, for the box lengths the workloads use and a few others.
"""
import numpy as np
import pytest

f32 = np.float32


def two_sum_periodic(xa, xb, L):
    """The per-pair seam path: s = xa - xb, its rounding error by Knuth's
    two-sum, the image shift applied to s (exact), the error added back."""
    s = f32(xa - xb)
    bb = f32(s - xa)
    e = f32(f32(xa - f32(s - bb)) + f32(f32(-xb) - bb))
    half = f32(L / 2)
    if s > half:
        t = f32(s - L)
    elif s < -half:
        t = f32(s + L)
    else:
        return s
    return f32(t + e)


@pytest.mark.parametrize("L", [1.0, 0.75, 3.0, 1.0e-3])
def test_seam_shift_matches_two_sum(L):
    rng = np.random.default_rng(11)
    L = f32(L)
    reach = f32(0.05) * L
    for _ in range(20000):
        # a near the top of the box, b near the bottom (a pair across the high seam)
        xa = f32(L - f32(rng.uniform(0, 1)) * reach)
        xb = f32(f32(rng.uniform(0, 1)) * reach)
        if xa >= L:
            xa = np.nextafter(L, f32(0))
        # high-seam tile: own cells at x - L, wrapped cells at x
        sa = f32(xa - L)
        assert float(sa) == float(xa) - float(L)          # exact
        assert f32(sa + L) == xa                           # the cell math recovers x
        d_shift = f32(sa - xb)
        assert d_shift == two_sum_periodic(xa, xb, L)
        # low-seam tile: own cells at x, wrapped cells (near L) at x - L
        sb = f32(xa - L)
        d_low = f32(xb - sb)
        assert d_low == two_sum_periodic(xb, xa, L)


def test_shift_not_exact_below_half():
    # below L/2 the subtraction rounds for most coordinates: why a high-seam
    # tile needs its halo in the upper half of the box
    rng = np.random.default_rng(12)
    L = f32(1.0)
    x = rng.uniform(0.01, 0.4, 1000).astype(np.float32)
    inexact = np.sum((x - L).astype(np.float64) != x.astype(np.float64) - 1.0)
    assert inexact > 500
