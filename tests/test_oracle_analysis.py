"""Pins of the oracle's dose-comparison tools: the 3-D gamma index of Sec. II.D (Low et al.),
R80 and the per-voxel z-scores.  Each is checked against a closed form or a brute-force
definition on tiny grids.  CPU only."""
import itertools
import math

import numpy as np
import pytest

from oracle import analysis as A


def _brute_gamma2(ref, ev, voxel, dose_pct, dta, threshold, search):
    """All voxel pairs, no search box: gamma^2 from its definition."""
    nz, ny, nx = ref.shape
    d = [v * 10.0 for v in voxel]
    tol = dose_pct / 100.0 * ref.max()
    out = np.full(ref.shape, np.inf)
    for iz, iy, ix in itertools.product(range(nz), range(ny), range(nx)):
        if not ref[iz, iy, ix] > threshold * ref.max():
            continue
        best = math.inf
        for jz, jy, jx in itertools.product(range(nz), range(ny), range(nx)):
            r2 = ((jx - ix) * d[0]) ** 2 + ((jy - iy) * d[1]) ** 2 + ((jz - iz) * d[2]) ** 2
            if r2 <= search * search:
                best = min(best, r2 / dta ** 2 + (ev[jz, jy, jx] - ref[iz, iy, ix]) ** 2 / tol ** 2)
        out[iz, iy, ix] = best
    return out


@pytest.mark.parametrize("shape,voxel,search", [((5, 6, 7), (0.1, 0.1, 0.1), 3.0),
                                                ((4, 7, 6), (0.125, 0.125, 0.25), 3.0),
                                                ((3, 5, 9), (0.1, 0.2, 0.15), 4.5),
                                                ((1, 1, 11), (0.1, 0.1, 0.1), 2.5)])
def test_gamma_equals_brute_force_on_tiny_grids(shape, voxel, search):
    rng = np.random.default_rng(sum(shape))
    ref = rng.uniform(0, 1, shape)
    ev = ref * rng.uniform(0.95, 1.05, shape) + rng.normal(0, 0.02, shape)
    g2, m = A.gamma_index(ref, ev, voxel, 2.0, 2.0, 0.1, search)
    bf = _brute_gamma2(ref, ev, voxel, 2.0, 2.0, 0.1, search)
    assert np.array_equal(np.isinf(g2), np.isinf(bf))
    assert np.allclose(g2[m], bf[m], rtol=1e-12, atol=0)
    assert m.sum() == (ref > 0.1 * ref.max()).sum()


def test_gamma_of_identical_doses_is_zero():
    rng = np.random.default_rng(1)
    ref = rng.uniform(0, 1, (6, 7, 8))
    g2, m = A.gamma_index(ref, ref, (0.2, 0.2, 0.2))
    assert np.all(g2[m] == 0.0) and np.all(np.isinf(g2[~m]))
    assert A.gamma_pass_rate(ref, ref, (0.2, 0.2, 0.2)) == 1.0


@pytest.mark.parametrize("scale,gamma", [(1.01, 0.5), (1.019, 0.95), (1.03, 1.5), (0.97, 1.5)])
def test_gamma_of_a_scaled_flat_field_is_the_dose_term(scale, gamma):
    """A uniform field scaled by s: every neighbour has the same evaluated dose, so
    gamma = |s - 1| / 2 %, exactly the dose term."""
    ref = np.full((7, 8, 9), 2.5)
    g2, m = A.gamma_index(ref, ref * scale, (0.1, 0.1, 0.1))
    assert m.all()
    assert np.allclose(np.sqrt(g2), gamma, rtol=1e-9)


def test_scaled_dose_fails_exactly_where_it_exceeds_two_thirds_of_max():
    """Two flat levels, 1.0 and 0.5, each wider than the search radius, scaled by 1.03:
    the difference 0.03 D exceeds 2 % of the maximum iff D > 2/3 max."""
    ref = np.full((12, 6, 6), 0.5)
    ref[:6] = 1.0
    g2, m = A.gamma_index(ref, ref * 1.03, (0.1, 0.1, 0.1))
    far = np.ones(ref.shape, bool)
    far[3:9] = False                       # within 3 mm of the step between the levels
    ok = A.gamma_passes(g2)
    assert np.all(~ok[:3][far[:3]]) and np.all(ok[9:][far[9:]])


@pytest.mark.parametrize("shift,voxel,expected", [((0, 0, 1), (0.1, 0.1, 0.1), 0.5),
                                                  ((0, 0, 1), (0.1, 0.1, 0.25), 0.5),
                                                  ((1, 0, 0), (0.1, 0.1, 0.25), 1.25),
                                                  ((0, 1, 1), (0.1, 0.2, 0.1), math.sqrt(0.25 + 1.0)),
                                                  ((0, 1, 1), (0.125, 0.125, 0.25), math.sqrt(2 * 1.25 ** 2) / 2),
                                                  ((1, 1, 0), (0.125, 0.125, 0.25), math.sqrt(2.5 ** 2 + 1.25 ** 2) / 2)])
def test_gamma_of_a_shifted_random_field_is_the_shift_distance(shift, voxel, expected):
    """A random field shifted by k voxels, with a dose criterion so tight (1e-6 %) that only
    the matching voxel has a finite-looking dose term: gamma = |shift| / dta where the shift
    lies in the search sphere (catches swapped axes: the voxels are anisotropic)."""
    rng = np.random.default_rng(7)
    ref = rng.uniform(0.5, 1.0, (10, 10, 10))
    kz, ky, kx = shift
    ev = np.roll(ref, (kz, ky, kx), axis=(0, 1, 2))
    g2, m = A.gamma_index(ref, ev, voxel, dose_pct=1e-6, search_mm=4.0)
    inner = (slice(1, -1),) * 3
    g = np.sqrt(g2[inner])
    assert np.allclose(g, expected, rtol=1e-9)


def test_shifted_gaussian_passes_at_two_mm():
    """A 1 mm shift of a smooth Gaussian field passes everywhere at 2 %/2 mm."""
    z, y, x = np.meshgrid(*(np.arange(40) - 19.5 for _ in range(3)), indexing="ij")
    ref = np.exp(-(x ** 2 + y ** 2 + z ** 2) / (2 * 6.0 ** 2))
    ev = np.exp(-((x - 1) ** 2 + y ** 2 + z ** 2) / (2 * 6.0 ** 2))
    assert A.gamma_pass_rate(ref, ev, (0.1, 0.1, 0.1)) == 1.0
    # a 4 mm shift of the same field (twice the distance criterion) does not
    ev4 = np.exp(-((x - 4) ** 2 + y ** 2 + z ** 2) / (2 * 6.0 ** 2))
    assert A.gamma_pass_rate(ref, ev4, (0.1, 0.1, 0.1)) < 0.9


def test_gamma_threshold_and_empty_selection():
    ref = np.zeros((4, 4, 4))
    ref[1, 1, 1] = 1.0
    ref[2, 2, 2] = 0.05                    # below 10 % of max: not evaluated
    g2, m = A.gamma_index(ref, ref, (0.1, 0.1, 0.1))
    assert m.sum() == 1 and m[1, 1, 1]
    assert math.isnan(A.gamma_pass_rate(np.zeros((3, 3, 3)), np.zeros((3, 3, 3)), (0.1, 0.1, 0.1)))


def test_r80_of_a_linear_falloff():
    """Plateau at 1 then a linear fall of 0.1 per voxel: 80 % is reached two voxel centres
    after the last plateau voxel."""
    idd = np.concatenate([np.ones(10), 1.0 - 0.1 * np.arange(1, 11)])
    dz = 0.2
    assert A.r80(idd, dz) == pytest.approx((9 + 0.5) * dz + 2 * dz, abs=1e-12)
    assert A.r80(idd, dz, z0=1.0) == pytest.approx(1.0 + 11.5 * dz, abs=1e-12)


def test_zscores_select_and_scale():
    Da = np.array([1.0, 2.0, 0.01, 5.0])
    Db = np.array([1.5, 2.0, 0.0, 4.0])
    sa = np.array([0.3, 0.1, 0.1, 0.6])
    sb = np.array([0.4, 0.2, 0.1, 0.8])
    z = A.zscores(Da, sa, Db, sb, frac_of_max=0.1)
    assert np.allclose(z, [-0.5 / 0.5, 0.0, 1.0 / 1.0])


def test_let_stats_ratio_estimator():
    """LET_d = sum num / sum den; a constant ratio across groups has zero spread; and the
    ratio estimator's error matches the spread of LET_d over many independent repeats."""
    den = np.array([[1.0, 2.0, 3.0, 4.0], [0.0, 0.0, 0.0, 0.0]])
    num = 2.5 * den
    let, sig = A.let_stats(num, den)
    assert let[0] == 2.5 and sig[0] == 0.0 and let[1] == 0.0 and sig[1] == 0.0
    # a hand-worked case: num (3, 5), den (1, 1): LET 4, deviations (-1, +1): var = 2 * 2 / 4
    let, sig = A.let_stats(np.array([[3.0, 5.0]]), np.array([[1.0, 1.0]]))
    assert let[0] == 4.0 and sig[0] == pytest.approx(1.0)
    rng = np.random.default_rng(3)
    reps, B, n = 4000, 20, 50
    lets, sigs = [], []
    for _ in range(reps):
        e = rng.exponential(1.0, (B, n))                  # deposits
        L = 2.0 + rng.exponential(3.0, (B, n))            # their LET
        l, s = A.let_stats((e * L).sum(1)[None, :], e.sum(1)[None, :])
        lets.append(l[0])
        sigs.append(s[0])
    assert np.mean(sigs) == pytest.approx(np.std(lets), rel=0.05)
