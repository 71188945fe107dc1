"""Degenerate and ragged inputs of the transport against the oracle (GPU).

A single history and a handful (fewer than a warp), a proton born below the cutoff E_cut
(Sec. II.A.3: it deposits where it is), a spot outside the grid (it leaves at once), a beam
running exactly along voxel faces and edges (the index of a position on a face is the floor,
the tie-break both sides take), a one-voxel phantom, an oblique beam, the smallest and largest
group counts, and the calls that must be refused."""
import numpy as np
import pytest

from oracle import analysis as A
from oracle import oracle as O
from paper_1409_8336_gb300 import workloads as W

pytestmark = pytest.mark.gpu
FIX = 2.0 ** -24
CSDA = W.NO_STRAGGLING | W.NO_MCS | W.NO_ELASTIC | W.NO_INELASTIC


def _gpu(prob, n, seed, ledger=0, fast=False):
    from paper_1409_8336_gb300 import Engine

    e = Engine(device=0, n_batches=prob.n_batches, physics_flags=prob.flags, fast_math=fast)
    e.load_problem(prob)
    e.set_launch(256, 0)
    if ledger:
        e.enable_history_ledger(ledger)
    e.transport(n, seed)
    out = {"tally": e.read_tally(), "ledger": e.read_ledger()}
    out["dose"], out["sigma"] = e.read_dose()
    if ledger:
        out["hist"] = e.read_history_ledger(ledger)
    e.close()
    return out


@pytest.mark.parametrize("n", [1, 2, 31, 33])
def test_a_few_histories(n):
    """Fewer histories than a warp, and a warp plus one: each history's incident energy equals
    the oracle's (same spot sampling) and its energy closes to 1e-6."""
    p = W.config2()
    g = _gpu(p, n, 3, ledger=n)
    _, _, ho = O.run(p, n, 3, ledger=True)
    h = g["hist"].astype(np.float64) * FIX
    assert np.allclose(h[:, 0], ho[:, 0], rtol=1e-6)
    assert np.all(np.abs(h[:, 0] - h[:, 1:].sum(1)) <= 1e-6 * h[:, 0])
    L = g["ledger"]
    assert L["histories"] == n and L["dropped"] == 0 and L["errors"] == 0


def test_spots_without_histories():
    """A zero-weight spot, and spots left without histories by the largest-remainder split: the
    device's spot table holds only the spots with histories, and every history keeps its
    identity and spot (incident energies equal the oracle's history by history)."""
    spots = np.array([W.spot_row(100.0, sigma=0.3), W.spot_row(150.0, sigma=0.3, weight=0.0),
                      W.spot_row(200.0, sigma=0.3, weight=1e-9)])
    p = W.water_box((64, 16, 16), 0.5, spots, n_batches=2)
    n = 300
    g = _gpu(p, n, 4, ledger=n)
    _, _, ho = O.run(p, n, 4, ledger=True)
    h = g["hist"].astype(np.float64) * FIX
    assert np.allclose(h[:, 0], ho[:, 0], rtol=1e-6)
    assert np.allclose(h[:, 0], 100.0, rtol=1e-6)
    assert g["ledger"]["incident"] * FIX == pytest.approx(100.0 * n, rel=1e-7)


def test_proton_born_below_the_cutoff_deposits_in_its_voxel():
    p = W.water_box((8, 8, 8), 0.5, np.array([W.spot_row(0.05, x=0.1, y=-0.3, sigma=0.0)]), n_batches=2)
    n = 100
    g = _gpu(p, n, 1)
    t = g["tally"].sum(1).reshape(p.shape)
    ix, iy = int(np.floor((0.1 + 2.0) / 0.5)), int(np.floor((-0.3 + 2.0) / 0.5))
    assert t[0, iy, ix] == n * round(0.05 * 2 ** 24)
    assert t.sum() == t[0, iy, ix]
    ref, _, _ = O.run(p, n, 1)
    assert ref.sum(1).reshape(p.shape)[0, iy, ix] == pytest.approx(n * 0.05, rel=1e-7)


def test_spot_outside_the_grid_leaves_at_birth():
    p = W.water_box((8, 8, 8), 0.5, np.array([W.spot_row(100.0, x=5.0, y=0.0, sigma=0.0)]), n_batches=2)
    g = _gpu(p, 500, 1)
    L = g["ledger"]
    assert L["deposited"] == 0 and L["escaped"] == L["incident"] and L["steps"] == 0
    assert not g["tally"].any()


@pytest.mark.parametrize("fast", [False, True], ids=["ieee", "fastmath"])
def test_beam_along_voxel_faces_and_edges(fast):
    """A sigma-0 beam at x = y = 0, the common edge of four voxel columns: without scattering it
    travels exactly on two face planes for its whole range.  CSDA: the same stopping voxel and
    depth-dose as the oracle, in the column the floor of the position gives.  With full physics
    from the same edge: no particle runs out of steps, and the energy closes."""
    p = W.water_box((150, 8, 8), 0.1, np.array([W.spot_row(120.0, sigma=0.0)]), n_batches=2, flags=CSDA)
    g = _gpu(p, 64, 1, fast=fast)
    ref, _, _ = O.run(p, 64, 1)
    tg = g["tally"].sum(1).reshape(p.shape) * FIX
    to = ref.sum(1).reshape(p.shape)
    # one column on each side (the floor of a position on the face; single and double precision
    # may round 0.4 / 0.1 to either side of 4, so the column itself is not compared)
    cg = np.unravel_index(np.argmax(tg.sum(0)), tg.shape[1:])
    co = np.unravel_index(np.argmax(to.sum(0)), to.shape[1:])
    assert tg[:, cg[0], cg[1]].sum() == pytest.approx(tg.sum(), rel=1e-12)
    assert to[:, co[0], co[1]].sum() == pytest.approx(to.sum(), rel=1e-12)
    assert all(k in (3, 4) for k in (*cg, *co))
    dg, do = tg[:, cg[0], cg[1]], to[:, co[0], co[1]]
    stop = int(np.nonzero(do)[0][-1])
    assert int(np.nonzero(dg)[0][-1]) == stop
    tol = 1e-3 if fast else 2e-4
    assert np.allclose(dg[: stop - 2], do[: stop - 2], rtol=tol)
    full = _gpu(p.with_(flags=0), 20000, 2, fast=fast)
    L = full["ledger"]
    assert L["errors"] == 0 and L["dropped"] == 0
    assert abs(L["incident"] - L["deposited"] - L["escaped"] - L["binding"]) < 1e-6 * L["incident"]


def test_one_voxel_phantom():
    """A single 8 cm water voxel, 100 MeV (range 7.7 cm): the deposited energy per history
    against the oracle's within their statistical errors."""
    p = W.water_box((1, 1, 1), 8.0, np.array([W.spot_row(100.0, sigma=0.5)]), n_batches=10)
    n = 40000
    g = _gpu(p, n, 5, ledger=n)
    _, _, ho = O.run(p, n, 5, ledger=True)
    dg, do = g["hist"][:, 1].astype(np.float64) * FIX, ho[:, 1]
    se = np.sqrt(dg.var() / n + do.var() / n)
    assert abs(dg.mean() - do.mean()) < 4 * se
    L = g["ledger"]
    assert L["errors"] == 0 and abs(L["incident"] - L["deposited"] - L["escaped"] - L["binding"]) < 1e-6 * L["incident"]


def test_oblique_beam():
    """A beam entering at 40 degrees to the axis: depth-dose against the oracle (z-scores)."""
    d = (np.sin(np.radians(40.0)), 0.0, np.cos(np.radians(40.0)))
    p = W.water_box((64, 32, 48), 0.25, np.array([W.spot_row(120.0, x=-3.0, sigma=0.3, direction=d)]), n_batches=20)
    n = 200_000
    g = _gpu(p, n, 7)
    ref, _ = O.run_parallel(p, n, 7)
    Dg, sg = A.batch_stats(g["tally"].astype(np.float64) * FIX)
    Do, so = A.batch_stats(ref)
    z = A.zscores(Dg, sg, Do, so)
    assert np.mean(np.abs(z) <= 3.0) >= 0.99
    assert g["ledger"]["errors"] == 0


@pytest.mark.parametrize("B", [2, 1024])
def test_smallest_and_largest_group_counts(B):
    """The batch statistics at the smallest and largest number of groups against the group
    formula on the same tallies."""
    p = W.water_box((32, 8, 8), 0.5, np.array([W.spot_row(80.0, sigma=0.5)]), n_batches=B)
    g = _gpu(p, 4096, 9)
    Dt, st = A.batch_stats(g["tally"].astype(np.float64) * FIX)
    vol = float(np.float32(0.5)) ** 3
    dose = A.to_gray(Dt, p.rho.ravel().astype(np.float64), vol)
    sig = A.to_gray(st, p.rho.ravel().astype(np.float64), vol)
    assert np.allclose(g["dose"], dose, rtol=1e-9, atol=0)
    m = dose > 0.05 * dose.max()
    # the device sums the spread in single precision: over 1024 groups to about 1e-4
    assert np.allclose(g["sigma"][m], sig[m], rtol=1e-3 if B > 100 else 1e-4, atol=1e-6 * dose.max())


def test_refused_calls():
    from paper_1409_8336_gb300 import Engine, PmcError

    p = W.water_box((8, 8, 8), 0.5)
    e = Engine(device=0, n_batches=2)
    with pytest.raises(PmcError):
        e.transport(100, 1)                      # nothing loaded
    e.load_problem(p)
    for bad in (0, 2 ** 32):
        with pytest.raises(PmcError) as ex:
            e.transport(bad, 1)
        assert ex.value.code == -1
    e.clear_spots()
    with pytest.raises(PmcError):
        e.transport(100, 1)                      # no spots
    e.close()


def test_drain_waits_are_bounded_and_the_context_recovers():
    """The drain of the secondary generations waits for work only boundedly: a drain made to
    count one item that never comes (so it never sees its work finished) returns PMC_E_TIMEOUT
    instead of hanging, with the run's real work done, and the same context then transports
    exactly as a fresh one does."""
    from paper_1409_8336_gb300 import Engine
    from paper_1409_8336_gb300.engine import ERRORS

    prob = W.config1()
    n, seed = 3000, 9
    e = Engine(device=0, n_batches=prob.n_batches)
    e.load_problem(prob)
    e.set_launch(256, 0)
    assert ERRORS[e.debug_drain_waits(n, seed)] == "PMC_E_TIMEOUT"
    L = e.read_ledger()
    assert L["errors"] > 0 and L["dropped"] == 0
    assert abs(L["incident"] - L["deposited"] - L["escaped"] - L["binding"]) < 1e-6 * L["incident"]
    e.transport(n, seed)
    t = e.read_tally()
    assert e.read_ledger()["errors"] == 0
    e.close()
    assert np.array_equal(t, _gpu(prob, n, seed)["tally"])
