"""Pins of the oracle's transport loop (Sec. II.A.3) against results fixed by the physics:
deterministic CSDA depth-dose, the Highland angular width and the random-hinge lateral spread,
Bohr energy-loss variance, interaction probabilities from the cross-sections, and per-history
energy conservation.  CPU only."""
import math

import numpy as np
import pytest
from scipy import integrate, optimize, stats

from oracle import oracle as O
from paper_1409_8336_gb300 import workloads as W

N_A = 6.02214076e23
WATER_ZA = 0.111894 * 1 / 1.00794 + 0.888106 * 8 / 15.9994
ALL_OFF = W.NO_STRAGGLING | W.NO_MCS | W.NO_ELASTIC | W.NO_INELASTIC


def _S(E):
    return O.f("or_mass_stopping_power")(E, WATER_ZA, 75.0)


def _R(E):
    S1 = _S(1.0)
    if E <= 1.0:
        return 2 * math.sqrt(E) / S1
    return 2 / S1 + integrate.quad(lambda x: 1 / _S(x), 1.0, E, epsabs=0, epsrel=1e-12, limit=200)[0]


def _E_of_R(R):
    if R <= 0:
        return 0.0
    S1 = _S(1.0)
    if R <= 2 / S1:
        return (0.5 * R * S1) ** 2
    return optimize.brentq(lambda e: _R(e) - R, 1.0, 400.0, xtol=1e-13, rtol=1e-14)


def slab(nz, dz, E0, flags, lateral=1000.0):
    p = W.water_box((nz, 1, 1), 1.0, np.array([W.spot_row(E0, sigma=0.0)]), n_batches=2, flags=flags)
    return p.with_(voxel=(lateral, lateral, dz), origin=(-lateral / 2, -lateral / 2, 0.0))


def test_csda_depth_dose_is_deterministic_and_exact():
    E0, dz = 150.0, 0.1
    p = W.water_box((200, 3, 3), dz, np.array([W.spot_row(E0, sigma=0.0)]), n_batches=2, flags=ALL_OFF)
    n = 8
    tally, tot, _ = O.run(p, n, 1)
    idd = tally.sum(1).reshape(p.shape).sum((1, 2)) / n
    R0 = _R(E0)
    k_stop = int(R0 // dz)
    ref = np.zeros(200)
    for k in range(k_stop + 1):
        ref[k] = _E_of_R(R0 - k * dz) - _E_of_R(R0 - (k + 1) * dz)
    assert np.allclose(idd, ref, rtol=1e-8, atol=1e-9)
    assert tot["deposited"] == pytest.approx(n * E0, rel=1e-13)
    assert R0 == pytest.approx(15.7726, rel=1e-4)


def test_highland_width_and_random_hinge_spread():
    E0, t = 100.0, 1.0
    p = slab(1, t, E0, W.NO_STRAGGLING | W.NO_ELASTIC | W.NO_INELASTIC)
    n = 40000
    _, _, _, esc = O.run(p, n, 3, escapes=n)
    assert len(esc) == n
    th0 = O.f("or_highland_theta0")(E0, t, 36.08294323509874)
    thx = np.arctan2(esc[:, 4], esc[:, 6])
    thy = np.arctan2(esc[:, 5], esc[:, 6])
    for th in (thx, thy):
        v = th.var()
        assert abs(v / th0 ** 2 - 1) < 3 * math.sqrt(2 / n) + 0.01
        assert stats.kstest(th / th0, "norm").pvalue > 1e-3
    # random hinge: lateral displacement (1 - tau) t theta has variance theta0^2 t^2 / 3
    vx = esc[:, 1].var()
    assert abs(vx / (th0 ** 2 * t * t / 3) - 1) < 3 * math.sqrt(2 * 9 / 5 / n) + 0.01


def test_bohr_straggling_variance_and_mean_loss():
    E0, t = 100.0, 1.0
    p = slab(1, t, E0, W.NO_MCS | W.NO_ELASTIC | W.NO_INELASTIC)
    n = 40000
    _, _, _, esc = O.run(p, n, 4, escapes=n)
    Eo = esc[:, 0]
    var = O.f("or_bohr_variance")(E0, 1.0, WATER_ZA, t)
    assert abs(Eo.var() / var - 1) < 3 * math.sqrt(2 / n) + 0.005
    assert abs(Eo.mean() - _E_of_R(_R(E0) - t)) < 3 * math.sqrt(var / n)


def test_interaction_frequencies_follow_cross_sections():
    E0, t = 150.0, 0.2
    p = slab(1, t, E0, W.NO_STRAGGLING | W.NO_MCS)
    n = 600000
    _, tot, _ = O.run(p, n, 5)
    si, se = O.f("or_sigma_inelastic"), O.f("or_sigma_elastic")
    nH = 0.111894 * N_A / 1.00794
    nO = 0.888106 * N_A / 15.9994

    def expected(fn):
        # the proton's energy along the path from the range-energy relation
        return integrate.quad(lambda s: (nH * fn(1, 1, _E_of_R(_R(E0) - s)) + nO * fn(8, 16, _E_of_R(_R(E0) - s)))
                              * 1e-27, 0, t)[0]

    mu_in, mu_el = n * expected(si), n * expected(se)
    assert abs(tot["inelastic"] - mu_in) < 3.5 * math.sqrt(mu_in)
    assert abs(tot["elastic"] - mu_el) < 3.5 * math.sqrt(mu_el) + 0.01 * mu_el


def test_survival_probability_against_non_elastic_attenuation():
    E0, t = 150.0, 5.0
    p = slab(50, t / 50, E0, W.NO_STRAGGLING | W.NO_MCS | W.NO_ELASTIC)
    n = 100000
    _, tot, _ = O.run(p, n, 6)
    nO = 0.888106 * N_A / 15.9994
    si = O.f("or_sigma_inelastic")
    mu = integrate.quad(lambda s: nO * si(8, 16, _E_of_R(_R(E0) - s)) * 1e-27, 0, t)[0]
    P = 1 - math.exp(-mu)
    assert abs(tot["inelastic"] / n - P) < 3 * math.sqrt(P * (1 - P) / n) + 1e-4


def test_nonelastic_events_per_history_in_a_typical_plan():
    """Sec. I (footnote): about 1e6 non-elastic events are expected for 1e7 proton histories of
    a typical plan.  The CT plan (40 layers of 70-180 MeV in tissue, bone and lung) gives
    roughly 0.1 per history (read as 0.05-0.2)."""
    p = W.config3(shape=(100, 128, 128), n_layers=40)
    n = 1500
    _, tot, _ = O.run(p, n, 13)
    per = tot["inelastic"] / n
    assert 0.05 <= per <= 0.2, per


@pytest.mark.parametrize("cfg", [2, 3])
def test_energy_conservation_per_history(cfg):
    if cfg == 2:
        p, n = W.config2(), 300
    else:
        p, n = W.config3(shape=(40, 64, 64), n_layers=4), 300
    tally, tot, hl = O.run(p, n, 7, ledger=True)
    res = hl[:, 0] - hl[:, 1] - hl[:, 2] - hl[:, 3]
    assert np.all(np.abs(res) <= 1e-6 * np.maximum(hl[:, 0], 1e-12))
    assert tally.sum() == pytest.approx(tot["deposited"], rel=1e-12)
    assert tot["inelastic"] > 0 and tot["elastic"] > 0


def test_results_depend_only_on_seed():
    p = W.config1()
    a, _, _ = O.run(p, 300, 11)
    b, _, _ = O.run(p, 300, 11)
    c, _, _ = O.run(p, 300, 12)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)
    # a history's contribution does not depend on which other histories run (ranges split)
    d1, _, _ = O.run(p, 300, 11, h_begin=0, h_end=150)
    d2, _, _ = O.run(p, 300, 11, h_begin=150, h_end=300)
    assert np.allclose(d1 + d2, a, rtol=1e-12, atol=1e-12)


def test_parallel_runner_equals_serial():
    p = W.config1()
    a, ta = O.run_parallel(p, 3000, 13, procs=3)
    b, tb, _ = O.run(p, 3000, 13)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-9)
    assert ta["inelastic"] == tb["inelastic"] and ta["steps"] == tb["steps"]


def test_let_d_in_csda_is_the_voxel_energy_loss_per_length():
    """Straggling, MCS and nuclear off: each voxel is crossed by one step of length dz, so
    LET_d there is the CSDA energy lost in the voxel over dz (and E/R_left in the voxel
    where the proton stops), from the independent range quadrature.  The LET weights are
    the dose deposits themselves."""
    E0, dz = 150.0, 0.1
    p = W.water_box((200, 3, 3), dz, np.array([W.spot_row(E0, sigma=0.0)]), n_batches=2, flags=ALL_OFF)
    tally, num, den, tot = O.run_let(p, 4, 1)
    assert np.allclose(den, tally, rtol=1e-14, atol=0)
    let = num.sum(1).reshape(p.shape).sum((1, 2)) / np.maximum(den.sum(1).reshape(p.shape).sum((1, 2)), 1e-300)
    R0 = _R(E0)
    k_stop = int(R0 // dz)
    for k in range(k_stop):
        dE = _E_of_R(R0 - k * dz) - _E_of_R(R0 - (k + 1) * dz)
        assert let[k] == pytest.approx(0.1 * dE / dz, rel=1e-7), k
    Ek = _E_of_R(R0 - k_stop * dz)
    assert let[k_stop] == pytest.approx(0.1 * Ek / (R0 - k_stop * dz), rel=1e-6)
    assert np.all(let[k_stop + 1:] == 0)
    # entrance LET against the tabulated stopping power of water (keV/um = 0.1 MeV cm^2/g at 1 g/cm^3)
    assert let[0] == pytest.approx(0.1 * _S(E0), rel=2e-3)


def test_let_d_weights_only_proton_energy_losses():
    """With nuclear interactions the dose also holds recoil and fragment deposits, which carry
    no LET: the LET weights stay below the dose tally, and the dose-averaged LET rises towards
    the Bragg peak.  At the entrance it is the primaries' stopping power without nuclear
    interactions and above it with them: slow secondary protons raise it."""
    p = W.water_box((60, 1, 1), 0.25, np.array([W.spot_row(120.0, sigma=0.0)]), n_batches=2)
    p = p.with_(voxel=(1000.0, 1000.0, 0.25), origin=(-500.0, -500.0, 0.0))
    tally, num, den, tot = O.run_let(p, 3000, 2)
    assert tot["inelastic"] > 0 and tot["elastic"] > 0
    assert np.all(den <= tally * (1 + 1e-12) + 1e-12)
    assert den.sum() < tally.sum()
    let = num.sum(1) / np.maximum(den.sum(1), 1e-300)
    peak = int(np.argmax(tally.sum(1)))
    assert let[peak] > 3 * let[0]
    _, num0, den0, _ = O.run_let(p.with_(flags=W.NO_ELASTIC | W.NO_INELASTIC), 3000, 2)
    let0 = num0.sum(1)[0] / den0.sum(1)[0]
    E_mid = _E_of_R(_R(120.0) - 0.125)                 # mean energy in the first voxel
    assert let0 == pytest.approx(0.1 * _S(E_mid), rel=0.01)
    assert let[0] > 1.05 * let0
