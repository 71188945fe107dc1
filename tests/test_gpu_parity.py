"""End-to-end parity of the CUDA path against the CPU oracle on the same seeded inputs (GPU).

Criteria (from the method's accuracy targets): per-voxel z-scores within 3 sigma of the
combined statistical error for >= 99 % of voxels above 10 % of the maximum, R80 within
0.1 mm, 2 %/2 mm 3-D gamma >= 99 %, bit-reproducible tallies for a fixed seed, and
per-history energy conservation to 1e-6 of the incident energy."""
import numpy as np
import pytest

from oracle import analysis as A
from oracle import oracle as O
from paper_1409_8336_gb300 import workloads as W

pytestmark = pytest.mark.gpu
FIX = 2.0 ** -24


_ORACLE = {}


@pytest.fixture(params=[False, True], ids=["ieee", "fastmath"])
def fast(request):
    """Both builds of the engine: IEEE single precision and -use_fast_math."""
    return request.param


def oracle_parallel(prob, n, seed):
    key = (prob.name, prob.shape, len(prob.spots), prob.flags, n, seed)
    if key not in _ORACLE:
        _ORACLE[key] = O.run_parallel(prob, n, seed)
    return _ORACLE[key]


def run_gpu(prob, n, seed, ledger=0, escapes=0, block=0, chunk=0, fast=False):
    from paper_1409_8336_gb300 import Engine

    e = Engine(device=0, n_batches=prob.n_batches, physics_flags=prob.flags, fast_math=fast)
    e.load_problem(prob)
    if block or chunk:
        e.set_launch(block, chunk)
    if ledger:
        e.enable_history_ledger(ledger)
    if escapes:
        e.enable_escape_record(escapes)
    e.transport(n, seed)
    out = {"tally": e.read_tally(), "ledger": e.read_ledger()}
    out["dose"], out["sigma"] = e.read_dose()
    if ledger:
        out["hist"] = e.read_history_ledger(ledger)
    if escapes:
        out["esc"] = e.read_escape_record()
    e.close()
    return out


def compare(prob, n, seed, fast, min_z=0.99, gamma_min=0.99, r80_tol=0.01):
    """n is chosen so that the statistical noise of both runs stays well below the 2 % gamma
    dose criterion in the voxels above 10 % of the maximum: two independent oracle runs of
    1e5-2e5 histories pass only 94-99 % at 2 %/2 mm, i.e. at that size the gamma test measures
    the noise.  The oracle side runs over all host cores (history ranges, spawned workers)."""
    g = run_gpu(prob, n, seed, fast=fast)
    ref, tot = oracle_parallel(prob, n, seed)
    Dg, sg = A.batch_stats(g["tally"].astype(np.float64) * FIX)
    Do, so = A.batch_stats(ref)
    z = A.zscores(Dg, sg, Do, so)
    frac = np.mean(np.abs(z) <= 3.0)
    dz = prob.voxel[2]
    r80g = A.r80(A.depth_dose(Dg.reshape(prob.shape)), dz)
    r80o = A.r80(A.depth_dose(Do.reshape(prob.shape)), dz)
    gam = A.gamma_pass_rate(Do.reshape(prob.shape), Dg.reshape(prob.shape), prob.voxel)
    L = g["ledger"]
    bal = (L["incident"] - L["deposited"] - L["escaped"] - L["binding"]) / L["incident"]
    info = dict(z_frac=frac, r80_gpu=r80g, r80_oracle=r80o, gamma=gam, ledger=bal, gpu=L, oracle=tot)
    assert frac >= min_z, info
    assert abs(r80g - r80o) <= r80_tol, info
    assert gam >= gamma_min, info
    assert abs(bal) < 1e-6, info
    assert L["dropped"] == 0 and L["errors"] == 0
    # event counts agree with the oracle's within their Poisson spread
    for k in ("elastic", "inelastic"):
        assert abs(L[k] - tot[k]) <= 5 * np.sqrt(tot[k] + 1) + 0.02 * tot[k], (k, L[k], tot[k])
    return g, info


def test_csda_only_matches_oracle_voxel_by_voxel(fast):
    flags = W.NO_STRAGGLING | W.NO_MCS | W.NO_ELASTIC | W.NO_INELASTIC
    p = W.water_box((200, 3, 3), 0.1, np.array([W.spot_row(150.0, sigma=0.0)]), n_batches=2, flags=flags)
    g = run_gpu(p, 64, 1, fast=fast)
    ref, _, _ = O.run(p, 64, 1)
    dg = g["tally"].sum(1).reshape(p.shape).sum((1, 2)) * FIX / 64
    do = ref.sum(1).reshape(p.shape).sum((1, 2)) / 64
    stop = int(np.nonzero(do)[0][-1])
    assert int(np.nonzero(dg)[0][-1]) == stop                      # stops in the same voxel
    # plateau voxels agree to single-precision rounding (no drift of the range) ...
    tol = 1e-3 if fast else 2e-4
    assert np.allclose(dg[: stop - 2], do[: stop - 2], rtol=tol), np.max(np.abs(dg / np.maximum(do, 1e-30) - 1)[: stop - 2])
    # ... and the energy deposited up to any depth differs by < 0.03 MeV, a few micrometres of
    # range at the stopping powers near the end of range
    assert np.max(np.abs(np.cumsum(dg - do))) < 0.03
    assert dg.sum() == pytest.approx(150.0, rel=1e-7)


def test_water_pencil_beam_150mev(fast):
    """64x64x128 water of 2 mm, 150 MeV, sigma 3 mm, full physics."""
    compare(W.config1(), 1_000_000, 1, fast)


def test_heterogeneous_slab_three_energies(fast):
    """128^3 slab phantom of 1.5 mm (water/bone/lung/water + Ti), 70/150/230 MeV."""
    compare(W.config2(), 1_000_000, 2, fast)


def test_ct_plan_hu_path(fast):
    """HU volume with the 6-bin table, a 4-layer plan of 200 spots."""
    p = W.config3(shape=(60, 64, 64), n_layers=4)
    compare(p, 1_000_000, 3, fast)


def test_tally_is_bit_reproducible(fast):
    p = W.config2()
    a = run_gpu(p, 30000, 5, fast=fast)["tally"]
    b = run_gpu(p, 30000, 5, block=128, chunk=7001, fast=fast)["tally"]
    assert np.array_equal(a, b)
    c = run_gpu(p, 30000, 6, fast=fast)["tally"]
    assert not np.array_equal(a, c)


def test_history_ledger_conserves_energy(fast):
    p = W.config2()
    n = 4000
    g = run_gpu(p, n, 9, ledger=n, fast=fast)
    h = g["hist"].astype(np.float64) * FIX
    res = h[:, 0] - h[:, 1] - h[:, 2] - h[:, 3]
    assert np.all(np.abs(res) <= 1e-6 * h[:, 0]), np.max(np.abs(res) / h[:, 0])
    # sampled histories: the incident energies equal the oracle's history by history
    _, _, ho = O.run(p, n, 9, ledger=True)
    assert np.allclose(h[:, 0], ho[:, 0], rtol=1e-6)


def test_full_size_slab_run_sampled_against_oracle(fast):
    """The slab workload at its full 1e6 histories, in the bench's launch configuration: the
    first 2000 histories' ledgers against the oracle's, and conservation over the whole run."""
    p = W.config2()
    n = 1_000_000
    g = run_gpu(p, n, 1, ledger=2000, fast=fast)
    L = g["ledger"]
    assert L["dropped"] == 0 and L["errors"] == 0
    assert abs(L["incident"] - L["deposited"] - L["escaped"] - L["binding"]) < 1e-6 * L["incident"]
    h = g["hist"].astype(np.float64) * FIX
    _, _, ho = O.run(p, n, 1, h_begin=0, h_end=2000, ledger=True)
    ho = ho[:2000]
    assert np.allclose(h[:, 0], ho[:, 0], rtol=1e-6)
    # deposited energy per history: most histories follow the same path on both sides
    close = np.abs(h[:, 1] - ho[:, 1]) <= 1e-3 * ho[:, 0]
    assert close.mean() > 0.8, close.mean()
    assert abs(h[:, 1].mean() - ho[:, 1].mean()) < 4 * ho[:, 1].std() / np.sqrt(2000)


def test_escape_record_angular_spread_matches_highland(fast):
    p = W.water_box((1, 1, 1), 1000.0, np.array([W.spot_row(100.0, sigma=0.0)]), n_batches=2,
                    flags=W.NO_STRAGGLING | W.NO_ELASTIC | W.NO_INELASTIC)
    p = p.with_(voxel=(1000.0, 1000.0, 1.0), origin=(-500.0, -500.0, 0.0))
    n = 40000
    g = run_gpu(p, n, 3, escapes=n, fast=fast)
    esc = g["esc"]
    assert len(esc) == n
    th0 = O.f("or_highland_theta0")(100.0, 1.0, 36.08294323509874)
    thx = np.arctan2(esc[:, 4], esc[:, 6])
    assert abs(thx.var() / th0 ** 2 - 1) < 3 * np.sqrt(2 / n) + 0.01
    assert abs(esc[:, 1].var() / (th0 ** 2 / 3) - 1) < 3 * np.sqrt(2 * 9 / 5 / n) + 0.01


def test_statistics_kernel_matches_batch_formula(fast):
    """Dose (Gy) and its standard error from the device's statistics kernel against the
    ten-group formula applied to the same tallies on the host."""
    p = W.config2()
    g = run_gpu(p, 50000, 4, fast=fast)
    Dt, st = A.batch_stats(g["tally"].astype(np.float64) * FIX)
    vx = [float(np.float32(x)) for x in p.voxel]          # the engine keeps voxel sizes in single precision
    vol = vx[0] * vx[1] * vx[2]
    rho = p.rho.ravel().astype(np.float64)
    dose = A.to_gray(Dt, rho, vol)
    sig = A.to_gray(st, rho, vol)
    assert np.allclose(g["dose"], dose, rtol=1e-9, atol=0)
    m = dose > 0.01 * dose.max()
    assert np.allclose(g["sigma"][m], sig[m], rtol=1e-4, atol=1e-6 * dose.max())


def test_full_size_ct_plan_sampled_against_oracle():
    """The CT plan at full size: 256x256x160 int16 HU at 1 mm, 2000 spots over 40 layers,
    1e7 histories in one transport.  Conservation over the whole run; the ledgers of histories
    sampled from several spots against the oracle, history by history."""
    from paper_1409_8336_gb300 import Engine

    p = W.config3()
    n = 10_000_000
    e = Engine(device=0, n_batches=p.n_batches, fast_math=True)
    e.load_problem(p)
    cnt = O.allocate_histories(p, n).astype(np.int64)
    first = np.concatenate([[0], np.cumsum(cnt)[:-1]])
    k = 150
    e.enable_history_ledger(int(first[1500] + k))
    e.transport(n, 17)
    L = e.read_ledger()
    h = e.read_history_ledger(int(first[1500] + k)).astype(np.float64) * FIX
    e.close()
    assert L["dropped"] == 0 and L["errors"] == 0
    assert abs(L["incident"] - L["deposited"] - L["escaped"] - L["binding"]) < 1e-6 * L["incident"]
    for s in (0, 700, 1500):
        h0, h1 = int(first[s]), int(first[s]) + k
        _, _, ho = O.run(p, n, 17, h_begin=h0, h_end=h1, ledger=True)
        # spot sampling is identical history by history ...
        assert np.allclose(h[h0:h1, 0], ho[h0:h1, 0], rtol=1e-6)
        res = h[h0:h1, 0] - h[h0:h1, 1:].sum(1)
        assert np.all(np.abs(res) <= 1e-6 * h[h0:h1, 0])
        # ... and the deposited energy agrees in distribution.  At these energies the hinge's
        # second leg and the distance to the voxel face differ by ~1e-8 cm, below single-
        # precision rounding, so the two sides take equally valid but different crossing
        # decisions and the histories decorrelate.
        dg, do = h[h0:h1, 1], ho[h0:h1, 1]
        se = np.sqrt(dg.var() / k + do.var() / k)
        assert abs(dg.mean() - do.mean()) < 4 * se + 1e-9, (s, dg.mean(), do.mean(), se)


def test_full_size_ct_plan_dose_against_oracle():
    """The CT plan at full size, in the benchmark's launch configuration (fast-math build,
    autotuned launch shape, one graph launch): 256x256x160 int16 HU at 1 mm, 2000 spots over
    40 layers of 70-180 MeV, 1e7 histories, against the oracle's 1e7 histories over all host
    cores on the full grid: z-scores within 3 sigma for >= 99 % of voxels above 10 % of the
    maximum, R80 within 0.1 mm, 2 %/2 mm gamma >= 99 %, ledger closure, event counts."""
    compare(W.config3(), 10_000_000, 19, True)
