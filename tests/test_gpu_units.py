"""Single routines on the device against the CPU oracle on identical inputs (GPU)."""
import math

import numpy as np
import pytest
from scipy import stats

from conftest import golden
from oracle import oracle as O
from paper_1409_8336_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[False, True], ids=["ieee", "fastmath"])
def eng(request):
    from paper_1409_8336_gb300 import Engine, build

    build.build()
    e = Engine(device=0, n_batches=10, fast_math=request.param)
    p = W.config3(shape=(16, 32, 32), n_layers=2)
    e.load_problem(p)
    yield e, p
    e.close()


@pytest.mark.parametrize("fast", [False, True], ids=["ieee", "fastmath"])
def test_philox_device_matches_known_answers_and_oracle(fast):
    from paper_1409_8336_gb300 import debug_philox

    for row in golden("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        assert list(debug_philox(np.array([v[0:4]]), np.array(v[4:6]), fast)[0]) == v[6:10]
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(512, 4), dtype=np.uint64).astype(np.uint32)
    key = np.array([0x12345678, 0x9abcdef0], dtype=np.uint32)
    dev = debug_philox(ctr, key, fast)
    for c, d in zip(ctr[:64], dev[:64]):
        assert O.philox([int(x) for x in c], [int(x) for x in key]) == [int(x) for x in d]


def test_range_tables_match_oracle(eng):
    e, p = eng
    E = np.geomspace(0.12, 290.0, 200)
    for m in range(len(p.materials)):
        r, eb = e.debug_tables(m, E)
        info = O.material_info(p, m)
        # the scaled materials share the reference water table (Eq. 1 / Eq. 2)
        base = 0 if not p.materials[m].get("own_table") else m
        ref = np.array([O.range_csda(p, base, x) for x in E])
        tol = 1e-4 if e.fast_math else 2e-5
        assert np.allclose(r, ref, rtol=tol, atol=1e-9), (m, np.max(np.abs(r / ref - 1)))
        assert np.allclose(eb, E, rtol=1.5 * tol), (m, np.max(np.abs(eb / E - 1)))
        assert info["f"] > 0


@pytest.mark.parametrize("nuc,E", [(0, 150.0), (3, 150.0), (3, 20.0), (6, 230.0), (1, 70.0)])
def test_elastic_kinematics_match_oracle(eng, nuc, E):
    e, p = eng
    Z, A = p.nuclides[nuc][0], p.nuclides[nuc][1]
    u = np.random.default_rng(nuc).uniform(size=(2000, 3)).astype(np.float32).astype(np.float64)
    dev = e.debug_elastic(nuc, E, u)
    ref = np.array([O.elastic(Z, A, E, row) for row in u[:300]])
    tol = 1e-3 if e.fast_math else 2e-4
    assert np.allclose(dev[:300, 0], ref[:, 0], rtol=tol / 2, atol=tol * E)
    assert np.allclose(dev[:300, 1], ref[:, 1], atol=tol)
    assert np.allclose(dev[:300, 4], ref[:, 4], atol=tol)
    assert np.allclose(dev[:, 0] + dev[:, 2], E, rtol=1e-6)


@pytest.mark.parametrize("nuc,E", [(3, 200.0), (5, 200.0), (1, 90.0), (6, 150.0)])
def test_cascade_events_match_oracle(eng, nuc, E):
    e, p = eng
    Z, A = p.nuclides[nuc][0], p.nuclides[nuc][1]
    n, seed, pid0 = 4000, 17, 1000
    ds, dp = e.debug_inc(nuc, E, seed, pid0, n)
    os_, op, _ = O.inc_batch(Z, A, E, seed, pid0, n)
    # identical random streams: most events take the same discrete path
    same = np.mean((ds[:, 0] == os_[:, 0]) & (np.abs(dp[:, 0, 1] - op[:, 0, 1]) < 1e-3 * E))
    assert same > 0.5, same
    # distributions agree (KS) for proton and neutron spectra and excitation left over
    for sp in (0, 1):
        dT = dp[:, :, 1][(dp[:, :, 0] == sp) & (np.arange(dp.shape[1])[None, :] < ds[:, :1])]
        oT = op[:, :, 1][(op[:, :, 0] == sp) & (np.arange(op.shape[1])[None, :] < os_[:, :1])]
        assert stats.ks_2samp(dT, oT).pvalue > 1e-3
        assert abs(len(dT) - len(oT)) < 4 * math.sqrt(len(oT)) + 10
    # device events conserve charge, baryon number and energy
    spec = {0: (0, 1), 1: (1, 1), 2: (1, 2), 3: (1, 3), 4: (2, 3), 5: (2, 4)}
    for i in range(0, n, 7):
        k = int(ds[i, 0])
        if ds[i, 7]:
            continue
        sps = dp[i, :k, 0].astype(int)
        assert sum(spec[s][0] for s in sps) + ds[i, 1] == Z + 1
        assert sum(spec[s][1] for s in sps) + ds[i, 2] == A + 1
        assert dp[i, :k, 1].sum() + ds[i, 3] + ds[i, 4] + ds[i, 5] == pytest.approx(E, abs=2e-4)


def test_event_generator_totals_equal_the_events_it_runs(eng):
    """The event-generator entry point runs the transport's event code with the same random
    streams: its totals equal the sums over the same events run one by one (counts exactly;
    energies to 1e-6, since the same inlined event code compiled into two kernels may fuse
    multiply-adds differently)."""
    e, p = eng
    n, seed, pid0, E = 3000, 17, 1000, 200.0
    y = e.nonelastic_events(3, E, n, seed, pid0)
    ds, dp = e.debug_inc(3, E, seed, pid0, n)
    assert y["events"] == n
    assert y["transparent"] == int(ds[:, 7].sum())
    assert y["retries"] == int(ds[:, 6].sum())
    live = np.arange(dp.shape[1])[None, :] < ds[:, :1]
    for k, name in enumerate(("n", "p", "d", "t", "He3", "alpha")):
        sel = live & (dp[:, :, 0] == k)
        assert y["count"][name] == int(sel.sum()), name
        assert y["energy"][name] == pytest.approx(dp[:, :, 1][sel].sum(), rel=1e-6, abs=n * 2.0 ** -24)
    ok = ds[:, 7] == 0
    assert y["residual_T"] == pytest.approx(ds[ok, 3].sum(), rel=1e-6, abs=n * 2.0 ** -24)
    assert y["excitation_left"] == pytest.approx(ds[ok, 4].sum(), rel=1e-6, abs=n * 2.0 ** -24)
    assert y["ms"] > 0


@pytest.mark.parametrize("nuc", [3, 5], ids=["O16", "Ca40"])
def test_event_generator_yields_match_oracle(eng, nuc):
    """Table I's reactions (p-16O and p-40Ca at 200 MeV): mean multiplicities and emitted
    energies per event from 2e5 device events against 2e4 oracle events, within 5 standard
    errors."""
    e, p = eng
    Z, A = p.nuclides[nuc][0], p.nuclides[nuc][1]
    E = 200.0
    y = e.nonelastic_events(nuc, E, 200_000, 23)
    os_, op, _ = O.inc_batch(Z, A, E, 29, 0, 20_000)
    live = np.arange(op.shape[1])[None, :] < os_[:, :1]
    ng = y["events"]
    for k, name in ((0, "n"), (1, "p"), (5, "alpha")):
        sel = live & (op[:, :, 0] == k)
        per_ev_n = sel.sum(1)
        per_ev_T = np.where(sel, op[:, :, 1], 0.0).sum(1)
        for gv, ov in ((y["count"][name] / ng, per_ev_n), (y["energy"][name] / ng, per_ev_T)):
            se = ov.std() * np.sqrt(1 / len(ov) + 1 / ng)
            assert abs(gv - ov.mean()) < 5 * se + 1e-9, (name, gv, ov.mean(), se)


def test_profile_modes_time_what_they_say_and_leave_the_dose_alone():
    """Timing events around every launch, around the primary-transport launches only, or
    none: the same run gives the same tallies; the light mode times the primary launches
    and nothing else; an unknown mode is refused."""
    from paper_1409_8336_gb300 import Engine, PmcError

    p = W.config2()
    e = Engine(device=0, n_batches=10, fast_math=True, block_size=192)
    e.load_problem(p)
    doses, profs = [], []
    for mode in ("all", "primary", "off"):
        e.enable_profile(mode != "off", primary_only=(mode == "primary"))
        e.transport(50_000, 21)
        profs.append(e.read_profile()[0])
        doses.append(e.read_dose())
    full, light, off = profs
    assert all(full[k]["launches"] > 0 for k in full)
    assert light["transport_primary"]["launches"] == full["transport_primary"]["launches"]
    assert light["transport_primary"]["ms"] > 0.0
    assert all(light[k]["launches"] == 0 for k in light if k != "transport_primary")
    assert all(off[k]["launches"] == 0 for k in off)
    for d, s in doses[1:]:
        assert np.array_equal(d, doses[0][0]) and np.array_equal(s, doses[0][1])
    with pytest.raises(PmcError):
        e._check(e._L.pmc_enable_profile(e._ctx, 3))
    e.close()
