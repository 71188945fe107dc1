"""Dose-averaged LET scored on the GPU against the oracle (Sec. IV: LET_d computed together
with the dose).  Deterministic CSDA transport checks the per-step scoring rule voxel by voxel;
full physics is compared by per-voxel z-scores of LET_d with the ratio-estimator errors of
both sides, as the dose is."""
import numpy as np
import pytest

from oracle import analysis as A
from oracle import oracle as O
from paper_1409_8336_gb300 import workloads as W

pytestmark = pytest.mark.gpu
FIX = 2.0 ** -24
ALL_OFF = W.NO_STRAGGLING | W.NO_MCS | W.NO_ELASTIC | W.NO_INELASTIC


def _gpu(prob, n, seed, fast=False):
    from paper_1409_8336_gb300 import Engine

    e = Engine(device=0, n_batches=prob.n_batches, physics_flags=prob.flags, fast_math=fast)
    e.load_problem(prob)
    e.enable_let(True)
    e.transport(n, seed)
    out = {"tally": e.read_tally(), "ledger": e.read_ledger()}
    out["num"], out["den"] = e.read_let_tally()
    out["let"], out["let_sigma"] = e.read_let()
    out["dose"], _ = e.read_dose()
    e.close()
    return out


@pytest.mark.parametrize("fast", [False, True], ids=["ieee", "fastmath"])
def test_let_csda_matches_oracle_voxel_by_voxel(fast):
    p = W.water_box((200, 3, 3), 0.1, np.array([W.spot_row(150.0, sigma=0.0)]), n_batches=2, flags=ALL_OFF)
    g = _gpu(p, 64, 1, fast)
    assert np.array_equal(g["den"], g["tally"])        # every deposit is a proton energy loss
    _, num, den, _ = O.run_let(p, 64, 1)
    lo, _ = A.let_stats(num, den)
    Lg = g["let"].reshape(p.shape)[:, 1, 1]
    Lo = lo.reshape(p.shape)[:, 1, 1]
    stop = int(np.nonzero(Lo)[0][-1])
    assert int(np.nonzero(Lg)[0][-1]) == stop
    tol = 2e-3 if fast else 5e-4
    assert np.allclose(Lg[:stop - 2], Lo[:stop - 2], rtol=tol), np.max(np.abs(Lg / np.maximum(Lo, 1e-30) - 1)[:stop - 2])
    # the LET_d the kernel reports equals the ratio of its own tallies
    lg2, _ = A.let_stats(g["num"].astype(np.float64), g["den"].astype(np.float64))
    assert np.allclose(g["let"], lg2, rtol=1e-12, atol=0)


def test_let_heterogeneous_slab_matches_oracle():
    """128^3 slab phantom (water / bone / lung / water, Ti insert), 70/150/230 MeV, full
    physics, 50 groups: LET_d z-scores within 3 sigma for >= 99 % of the voxels above 10 % of
    the maximum dose, and the device's error estimate equals the group formula."""
    prob = W.config2(n_batches=50)
    n = 1_000_000
    g = _gpu(prob, n, 9)
    tally, tot, num, den = O.run_parallel(prob, n, 9, let=True)
    lo, so = A.let_stats(num, den)
    lg, sg = A.let_stats(g["num"].astype(np.float64), g["den"].astype(np.float64))
    assert np.allclose(g["let"], lg, rtol=1e-12, atol=0)
    # the device forms the group deviations in single precision: agreement to ~1e-5 of LET_d
    assert np.all(np.abs(g["let_sigma"] - sg) <= 1e-3 * sg + 1e-5 * lg + 1e-12)
    Dg = g["tally"].sum(1).astype(np.float64)
    m = Dg > 0.1 * Dg.max()
    den_ = np.sqrt(sg[m] ** 2 + so[m] ** 2)
    z = (lg[m] - lo[m]) / np.where(den_ > 0, den_, np.inf)
    frac = np.mean(np.abs(z) <= 3.0)
    info = dict(frac=frac, voxels=int(m.sum()), mean_let_gpu=float(lg[m].mean()), mean_let_oracle=float(lo[m].mean()))
    assert frac >= 0.99, info
    # the weights are the protons' share of the dose: below the dose (up to the fixed-point
    # remainders of elastic events on hydrogen, a few hundred 2^-24 MeV units each), above
    # most of it
    assert np.all(g["den"] <= g["tally"] * (1 + 1e-5) + 4096)
    assert 0.9 * g["tally"].sum() < g["den"].sum() < g["tally"].sum()
    # LET_d rises from the entrance towards the end of the 70 MeV protons' range (in the
    # bone slab, 3-5 cm), diluted by the dose of the 150 and 230 MeV beams
    axis = lg.reshape(prob.shape)[:, 64, 64]
    assert axis[15:34].max() > 1.5 * axis[2]


def test_let_off_leaves_transport_unchanged_and_read_fails():
    """Scoring LET changes no history.  The LET-scoring build of the kernels is compiled
    separately from the plain one, and the compiler may fuse a multiply-add into an FMA in one
    and not the other, so a few histories can take an equally valid, different path: the two
    doses are compared within their statistical errors, and each build reproduces itself bit
    for bit.  The same steps of the plain run (the CSDA test above) score LET with the dose
    tally equal to the LET denominator."""
    from paper_1409_8336_gb300 import Engine, PmcError

    prob = W.config1()
    e = Engine(device=0, n_batches=prob.n_batches)
    e.load_problem(prob)
    n = 20_000
    e.transport(n, 5)
    t0 = e.read_tally()
    L0 = e.read_ledger()
    with pytest.raises(PmcError):
        e.read_let()
    e.enable_let(True)
    e.transport(n, 5)
    t1 = e.read_tally()
    L1 = e.read_ledger()
    e.transport(n, 5)
    assert np.array_equal(e.read_tally(), t1)          # deterministic with LET on
    assert L1["incident"] == L0["incident"]            # the same primaries
    D0, s0 = A.batch_stats(t0.astype(np.float64) * FIX)
    D1, s1 = A.batch_stats(t1.astype(np.float64) * FIX)
    z = A.zscores(D0, s0, D1, s1)
    assert np.mean(np.abs(z) <= 3.0) >= 0.99
    assert abs(L1["deposited"] - L0["deposited"]) <= 1e-3 * L0["incident"]
    e.enable_let(False)
    e.transport(n, 5)
    assert np.array_equal(e.read_tally(), t0)          # and back: the plain build again
    with pytest.raises(PmcError):
        e.read_let()
    e.close()
