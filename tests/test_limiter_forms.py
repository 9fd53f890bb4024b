"""The slope limiter of Sec. 3.1 in the two forms the code uses.

The oracle takes alpha_i = min(1, min_j psi_ij) with psi_ij = (phi_max -
phi_i) / dphi_ij for dphi_ij > 0, (phi_min - phi_i) / dphi_ij for
dphi_ij < 0 and 1 for dphi_ij = 0.  The GPU kernels take the same number as
1 / max(1, max_j dphi_ij r), with r = 1 / (phi_max - phi_i) for dphi > 0 and
r = -1 / (phi_i - phi_min) for dphi < 0 formed once per cell, and fmax
ignoring the NaN that 0 * inf gives for dphi = 0.  This checks the two
agree, including the edge cases: the cell is the neighbourhood's maximum or
minimum (an infinite r, alpha = 0 where dphi points past it), dphi = 0, and
all dphi of one sign.
"""
import numpy as np


def alpha_division(phi_i, phi_max, phi_min, dphi):
    a = 1.0
    for d in dphi:
        if d > 0:
            psi = (phi_max - phi_i) / d
        elif d < 0:
            psi = (phi_min - phi_i) / d
        else:
            psi = 1.0
        a = min(a, psi)
    return a


def alpha_reciprocal(phi_i, phi_max, phi_min, dphi):
    with np.errstate(divide="ignore", invalid="ignore"):
        rmx = np.float64(1.0) / np.float64(phi_max - phi_i)
        rmn = np.float64(-1.0) / np.float64(phi_i - phi_min)
        b = np.float64(0.0)
        for d in dphi:
            b = np.fmax(b, np.float64(d) * (rmx if d > 0 else rmn))
        return float(np.float64(1.0) / np.fmax(np.float64(1.0), b))


def test_forms_agree_on_random_neighbourhoods():
    rng = np.random.default_rng(7)
    for _ in range(2000):
        k = int(rng.integers(4, 20))
        phi_i = rng.normal()
        nb = phi_i + rng.normal(size=k)
        phi_max, phi_min = max(phi_i, nb.max()), min(phi_i, nb.min())
        dphi = rng.normal(size=k) * rng.choice([0.1, 1.0, 10.0])
        a = alpha_division(phi_i, phi_max, phi_min, dphi)
        b = alpha_reciprocal(phi_i, phi_max, phi_min, dphi)
        assert abs(a - b) <= 4e-16 * max(1.0, a), (a, b)
        assert 0.0 <= b <= 1.0


def test_extremal_cell_gives_zero_where_dphi_points_past_it():
    # the cell is the maximum: any dphi > 0 leaves the allowed range
    assert alpha_reciprocal(2.0, 2.0, 1.0, [0.5, -0.1]) == 0.0
    assert alpha_division(2.0, 2.0, 1.0, [0.5, -0.1]) == 0.0
    # the cell is the minimum: any dphi < 0 does
    assert alpha_reciprocal(1.0, 2.0, 1.0, [0.1, -0.5]) == 0.0
    # an extremal cell whose dphi point only inward keeps its slope
    assert alpha_reciprocal(2.0, 2.0, 1.0, [-0.3, -0.2]) == 1.0


def test_zero_dphi_is_ignored():
    # dphi = 0 against an infinite reciprocal is NaN, which fmax drops
    assert alpha_reciprocal(2.0, 2.0, 2.0, [0.0, 0.0]) == 1.0
    assert alpha_reciprocal(1.5, 2.0, 1.0, [0.0, 0.25]) == 1.0
    assert abs(alpha_reciprocal(1.5, 2.0, 1.0, [0.0, 1.0]) - 0.5) < 1e-16


def test_limited_extrapolation_stays_within_the_bounds():
    rng = np.random.default_rng(8)
    for _ in range(500):
        phi_i = rng.normal()
        nb = phi_i + rng.normal(size=12)
        phi_max, phi_min = max(phi_i, nb.max()), min(phi_i, nb.min())
        dphi = rng.normal(size=12) * 3.0
        b = alpha_reciprocal(phi_i, phi_max, phi_min, dphi)
        face = phi_i + b * dphi
        span = phi_max - phi_min
        assert np.all(face <= phi_max + 4e-16 * span + 1e-300)
        assert np.all(face >= phi_min - 4e-16 * span - 1e-300)
