"""Pins of the oracle's Vavilov straggling option (the paper uses Bohr's Gaussian; this is
the optional Vavilov form): the characteristic function of the Bethe collision spectrum
against the moments it must have, against a collision-by-collision simulation, and against
the Gaussian limit; the table and its sampler; and the transported energy spread.  CPU only."""
import ctypes as C

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from oracle import vavilov as V
from paper_1409_8336_gb300 import workloads as W


@pytest.mark.parametrize("kappa,b2", [(0.001, 0.2), (0.003, 0.0), (0.01, 0.0), (0.05, 0.3), (0.5, 0.1), (3.0, 0.45),
                                     (10.0, 0.2)])
def test_density_has_unit_mass_zero_mean_and_the_spectrum_variance(kappa, b2):
    """Var = int eps^2 w(eps) d eps = xi eps_max (1 - beta^2/2), i.e. kappa (1 - beta^2/2) in
    units of eps_max^2 (worked by hand from the spectrum)."""
    y, f, dy = V.density(kappa, b2)
    assert f.sum() * dy == pytest.approx(1.0, abs=1e-6)
    mean = (y * f).sum() * dy
    assert abs(mean) < 1e-6 * max(1.0, np.sqrt(kappa))
    var = ((y - mean) ** 2 * f).sum() * dy
    assert var == pytest.approx(kappa * (1.0 - 0.5 * b2), rel=2e-4)


def _collisions(kappa, b2, n, rng, xc=1e-3):
    """Centred loss (units of eps_max) from collisions one by one: Poisson many transfers
    x = eps/eps_max above xc from the spectrum kappa (1/x^2 - b2/x) (1/x^2 by inversion, then
    acceptance 1 - b2 x), minus their exact mean; transfers below xc are left out (their
    variance is kappa xc^2 / 2, negligible)."""
    lam = kappa * ((1.0 / xc - 1.0) - b2 * np.log(1.0 / xc))
    mean = kappa * (np.log(1.0 / xc) - b2 * (1.0 - xc))
    out = np.empty(n)
    for i in range(n):
        m = rng.poisson(lam)
        got = []
        while sum(len(g) for g in got) < m:
            u = rng.uniform(size=(2, 2 * m + 8))
            x = 1.0 / (1.0 / xc - u[0] * (1.0 / xc - 1.0))
            got.append(x[u[1] < 1.0 - b2 * x])
        out[i] = np.concatenate(got)[:m].sum() - mean if m else -mean
    return out


@pytest.mark.parametrize("kappa,b2", [(0.05, 0.3), (0.5, 0.1)])
def test_distribution_equals_collision_by_collision_simulation(kappa, b2):
    rng = np.random.default_rng(7)
    sample = _collisions(kappa, b2, 3000, rng)
    y, f, dy = V.density(kappa, b2)
    cdf = np.cumsum(f) * dy
    ks = stats.kstest(sample, lambda q: np.interp(q, y + 0.5 * dy, cdf)).statistic
    assert ks < 1.63 / np.sqrt(len(sample))          # 1 % critical value


def test_thin_layer_distribution_equals_collision_by_collision_simulation():
    """kappa = 0.001 (a 0.1 mm step in lung at 200 MeV): the Landau-like core is about kappa
    eps_max wide, so the simulation keeps transfers down to x = 1e-7 (some 1e4 per sample; the
    omitted ones add a variance kappa x_c, 1e-3 of the core's squared width) and the table's
    quantiles are compared with the simulation's over the body of the distribution."""
    kappa, b2, xc, n = 0.001, 0.35, 1e-7, 2000
    rng = np.random.default_rng(11)
    lam = kappa * ((1.0 / xc - 1.0) - b2 * np.log(1.0 / xc))
    mean = kappa * (np.log(1.0 / xc) - b2 * (1.0 - xc))
    m = rng.poisson(lam, size=n)
    sample = np.empty(n)
    for i in range(n):
        u = rng.uniform(size=(2, int(1.3 * m[i]) + 16))
        x = 1.0 / (1.0 / xc - u[0] * (1.0 / xc - 1.0))
        x = x[u[1] < 1.0 - b2 * x][: m[i]]
        assert len(x) == m[i]
        sample[i] = x.sum() - mean
    y, f, dy = V.density(kappa, b2)
    cdf = np.cumsum(f) * dy
    ks = stats.kstest(sample, lambda q: np.interp(q, y + 0.5 * dy, cdf)).statistic
    assert ks < 1.63 / np.sqrt(n)                    # 1 % critical value
    # the table row (units of xi, centred on its truncated mean) holds the density's quantiles
    T = V.table()
    u = np.array([0.05, 0.25, 0.5, 0.75, 0.95])
    z_tab = np.array([float(V.sample_z(T, np.array(kappa), b2, q)) for q in u])
    z_den = np.interp(u, cdf, y + 0.5 * dy) / kappa
    assert np.all(np.abs(z_den - z_tab - np.median(z_den - z_tab)) < 0.05), (z_den, z_tab)
    # below the old lower end of the table the spread keeps growing as kappa falls
    s_tab = [float(V.sample_z(T, np.array(k), b2, 0.75)) - float(V.sample_z(T, np.array(k), b2, 0.25))
             for k in (0.001, 0.01)]
    assert s_tab[0] > s_tab[1] * 0.9


def test_large_kappa_approaches_the_gaussian():
    u = V.U0 + np.arange(V.NU) * (1 - 2 * V.U0) / (V.NU - 1)
    sel = (u > 0.1) & (u < 0.9)
    for b2 in (0.0, 0.3):
        z = V.quantiles(10.0, b2)
        s = np.sqrt((1 - 0.5 * b2) / 10.0)
        assert np.max(np.abs(z[sel] - stats.norm.ppf(u[sel]) * s)) < 0.05 * s


def test_table_rows_are_centred_and_the_samplers_agree():
    T = V.table()
    assert T.shape == (V.NB, V.NK, V.NU)
    trap = (0.5 * (T[..., 0] + T[..., -1]) + T[..., 1:-1].sum(axis=-1)) / (V.NU - 1)
    assert np.abs(trap).max() < 1e-9
    assert np.all(np.diff(T, axis=-1) >= 0)          # quantile functions
    L = O.lib()
    O._ensure_vavilov(L)
    rng = np.random.default_rng(3)
    for _ in range(50):
        kappa, b2, u = np.exp(rng.uniform(np.log(0.0005), np.log(12))), rng.uniform(0, 0.55), rng.uniform()
        assert L.or_vavilov_z(kappa, b2, u) == pytest.approx(float(V.sample_z(T, np.array(kappa), b2, u)), abs=1e-12)


def test_step_parameters():
    """xi = (K/2)(Z/A) rho x / beta^2 and kappa = xi / T_max with T_max = 2 m c^2 beta^2 gamma^2 /
    (1 + 2 gamma m/M + (m/M)^2), for 100 MeV protons over 1.5 mm of water."""
    L = O.lib()
    xi, ka = C.c_double(), C.c_double()
    L.or_vavilov_params(100.0, 1.0, 0.5551, 0.15, C.byref(xi), C.byref(ka))
    me, mp = 0.51099895, 938.272088
    g = 1 + 100.0 / mp
    b2 = 1 - 1 / g ** 2
    tmax = 2 * me * b2 * g * g / (1 + 2 * g * me / mp + (me / mp) ** 2)
    assert xi.value == pytest.approx(0.5 * 0.307075 * 0.5551 * 0.15 / b2, rel=1e-12)
    assert ka.value == pytest.approx(xi.value / tmax, rel=1e-12)
    assert 0.2 < ka.value < 0.4                       # the Vavilov regime


def test_transported_spread_keeps_mean_and_variance_and_gains_the_tail():
    """1 cm of water at 100 MeV in ten 1 mm steps (kappa ~ 0.3), scattering and nuclear
    interactions off: the exit energy has the same mean and (up to the tabulated tails) the
    same variance as with Bohr's Gaussian, and the low-energy tail of Vavilov's distribution."""
    res = {}
    base = W.NO_MCS | W.NO_ELASTIC | W.NO_INELASTIC
    for name, flags in (("bohr", base), ("vavilov", base | W.VAVILOV)):
        p = W.water_box((10, 1, 1), 1.0, np.array([W.spot_row(100.0, sigma=0.0)]), n_batches=2, flags=flags)
        p = p.with_(voxel=(1000.0, 1000.0, 0.1), origin=(-500.0, -500.0, 0.0))
        n = 20000
        _, _, _, esc = O.run(p, n, 9, escapes=n)
        res[name] = esc[:, 0]
    b, v = res["bohr"], res["vavilov"]
    se = np.sqrt(b.var() / len(b) + v.var() / len(v))
    assert abs(b.mean() - v.mean()) < 4 * se
    assert v.std() == pytest.approx(b.std(), rel=0.03)
    assert stats.skew(v) < -0.2 and abs(stats.skew(b)) < 0.1


def test_library_builds_the_same_table_independently():
    """The library's host code builds its own table (its own sine/cosine integrals and Fourier
    transform, no device needed): it equals the oracle's to float precision."""
    from paper_1409_8336_gb300 import engine

    G = engine.debug_vavilov_table()
    T = V.table()
    assert G.shape == T.shape
    assert np.abs(G - T).max() <= 1e-5 * max(1.0, np.abs(T).max())
