"""Pins of the oracle's Moliere multiple-scattering option (Bethe's form of Moliere's theory,
an alternative to the paper's Highland width, Sec. II.A.2): the tabulated distribution
functions against an independent double quadrature and against their closed-form values at
the origin, their normalisation, the characteristic angle from fundamental constants, the
B equation, and the width of transported protons against Highland's fit.  CPU only."""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import oracle as O
from paper_1409_8336_gb300 import workloads as W

EULER = 0.5772156649015329


def _f(n, t):
    """f_n(t) = (1/n!) int_0^inf u J0(t u) exp(-u^2/4) [(u^2/4) ln(u^2/4)]^n du, with J0."""
    def g(u):
        y = 0.25 * u * u
        return u * special.j0(t * u) * math.exp(-y) * (y * math.log(y) if y > 0 else 0.0) ** n
    return integrate.quad(g, 0.0, 16.0, limit=400, epsabs=1e-12)[0] / math.factorial(n)


@pytest.mark.parametrize("v", [0.3, 0.7, 1.5, 3.0, 6.0])
def test_distribution_functions_equal_independent_quadrature(v):
    """F_n(v) = int_0^v f_n(t) t dt by an outer quadrature over the J0 form of f_n (the oracle
    uses the J1 form and Simpson's rule)."""
    for n in (1, 2):
        ref = integrate.quad(lambda t: _f(n, t) * t, 0.0, v, limit=200, epsabs=1e-10)[0]
        assert O.f("or_moliere_F")(v, n) == pytest.approx(ref, abs=2e-6), (n, v)
    assert O.f("or_moliere_F")(v, 0) == pytest.approx(1.0 - math.exp(-v * v), rel=1e-15)


def test_values_at_the_origin_are_the_closed_forms():
    """Near 0, F_n(v) = f_n(0) v^2 / 2 with f1(0) = 2 (1 - gamma) and f2(0) = Gamma''(3)
    = 2 [psi(3)^2 + psi'(3)]."""
    v = 0.02
    f1_0 = 2.0 * (1.0 - EULER)
    psi3, dpsi3 = 1.5 - EULER, math.pi ** 2 / 6.0 - 1.25
    f2_0 = 2.0 * (psi3 ** 2 + dpsi3)
    assert 2.0 * O.f("or_moliere_F")(v, 1) / v ** 2 == pytest.approx(f1_0, rel=2e-3)
    assert 2.0 * O.f("or_moliere_F")(v, 2) / v ** 2 == pytest.approx(f2_0, rel=2e-3)
    assert f1_0 == pytest.approx(0.84557, abs=1e-5) and f2_0 == pytest.approx(2.49293, abs=1e-5)


def test_normalisation_and_single_scattering_tail():
    """F1 and F2 return to 0 at large v (f0 alone carries the normalisation), F1 approaching
    -1/v^2 from its Rutherford tail f1 ~ 2 v^-4; for B >= 4.5 the distribution function is
    monotone."""
    F = O.f("or_moliere_F")
    for v in (6.0, 8.0):
        assert F(v, 1) == pytest.approx(-1.0 / v ** 2, rel=0.08)
        assert abs(F(v, 2)) < 2.0 / v ** 2
    vs = np.linspace(0.0, 8.0, 801)
    for B in (4.5, 8.0, 15.0):
        cdf = np.array([F(v, 0) + F(v, 1) / B + F(v, 2) / B ** 2 for v in vs])
        assert np.all(np.diff(cdf) >= -1e-9), B


def test_characteristic_angle_and_b_equation():
    """chi_c^2 from fundamental constants (4 pi N_A r_e^2 (m_e c^2)^2 x sum w Z(Z+1)/A /
    (p beta c)^2), and B solving B - ln B = ln(chi_c^2 / (exp(2 gamma - 1) chi_a^2))."""
    prob = W.water_box((4, 4, 4), 0.1)
    E, x = 100.0, 0.1
    chic2, B = O.moliere_params(prob, 0, E, x)
    NA, re_cm, me = 6.02214076e23, 2.8179403262e-13, 0.51099895
    mp = 938.272088
    pc = math.sqrt(E * E + 2 * E * mp)
    beta = pc / (E + mp)
    wH, wO = 0.111894, 0.888106
    zz = wH * 1 * 2 / 1.00794 + wO * 8 * 9 / 15.9994
    ref = 4 * math.pi * NA * re_cm ** 2 * me ** 2 * x * zz / (pc * beta) ** 2
    assert chic2 == pytest.approx(ref, rel=1e-4)
    # screening angle, log-averaged over the elements with weights w Z(Z+1)/A
    hbarc_fm, a0_fm = 197.3269804, 52917.721090
    lna = 0.0
    for w, Z, A in ((wH, 1, 1.00794), (wO, 8, 15.9994)):
        chi0 = hbarc_fm / (0.885 * a0_fm) * Z ** (1 / 3) / pc
        alpha = Z / (137.035999 * beta)
        lna += w * Z * (Z + 1) / A * math.log(chi0 ** 2 * (1.13 + 3.76 * alpha ** 2))
    lna /= zz
    b = math.log(chic2) - lna - (2 * EULER - 1)
    assert B - math.log(B) == pytest.approx(b, abs=1e-9)
    assert 8 < B < 14
    # a very thin layer: the expansion's validity limit B = 4.5
    assert O.moliere_params(prob, 0, E, 1e-7)[1] == 4.5


def test_transported_width_against_highland():
    """Protons through 1 cm of water (no energy-loss straggling, no nuclear interactions):
    the projected angle's central 98 % has an RMS within 11 % of Highland's fit to Moliere
    (without the paper's 1.07), and the large-angle tail is heavier than a Gaussian's."""
    E0, t = 150.0, 1.0
    flags = W.NO_STRAGGLING | W.NO_ELASTIC | W.NO_INELASTIC | W.MOLIERE
    p = W.water_box((10, 1, 1), 1.0, np.array([W.spot_row(E0, sigma=0.0)]), n_batches=2, flags=flags)
    p = p.with_(voxel=(1000.0, 1000.0, t / 10), origin=(-500.0, -500.0, 0.0))
    n = 30000
    _, _, _, esc = O.run(p, n, 9, escapes=n)
    thx = np.arctan2(esc[:, 4], esc[:, 6])
    th0 = O.f("or_highland_theta0")(E0, t, 36.08294323509874) / 1.07
    lo, hi = np.percentile(thx, [1, 99])
    core = thx[(thx > lo) & (thx < hi)]
    assert core.std() == pytest.approx(th0, rel=0.11)
    sd = thx.std()
    assert np.mean(np.abs(thx) > 3 * sd) > 2 * 0.0027
