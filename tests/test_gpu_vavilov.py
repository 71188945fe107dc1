"""The Vavilov straggling option on the GPU against the oracle: the energies of protons
leaving thin water and titanium slabs (Kolmogorov-Smirnov, mean, spread and the skewed
low-energy tail), and the full pencil-beam dose in water by the same criteria as the default
physics."""
import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_1409_8336_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _slab(E0, t, mat):
    """A slab of thickness t (cm) in ten layers, laterally unbounded, one pencil beam; only
    energy loss and its straggling."""
    flags = W.NO_MCS | W.NO_ELASTIC | W.NO_INELASTIC | W.VAVILOV
    p = W.water_box((10, 1, 1), 1.0, np.array([W.spot_row(E0, sigma=0.0)]), n_batches=2, flags=flags)
    p = p.with_(voxel=(1000.0, 1000.0, t / 10), origin=(-500.0, -500.0, 0.0))
    if mat == "Ti":
        p = p.with_(materials=[W.WATER, W.TITANIUM], mat=np.full(p.shape, 1, np.uint8),
                    rho=np.full(p.shape, 4.5, np.float32))
    return p


@pytest.mark.parametrize("fast", [False, True], ids=["ieee", "fastmath"])
@pytest.mark.parametrize("E0,t,mat", [(100.0, 1.0, "water"), (200.0, 2.0, "water"), (70.0, 0.3, "Ti")])
def test_exit_energies_match_oracle(fast, E0, t, mat):
    from paper_1409_8336_gb300 import Engine

    p = _slab(E0, t, mat)
    n = 40000
    e = Engine(device=0, n_batches=2, physics_flags=p.flags, fast_math=fast)
    e.load_problem(p)
    e.enable_escape_record(n)
    e.transport(n, 3)
    g = e.read_escape_record()[:, 0]
    e.close()
    o = O.run(p, n, 4, escapes=n)[3][:, 0]
    assert len(g) == n and len(o) == n
    assert stats.ks_2samp(g, o).pvalue > 1e-3
    se = np.sqrt(g.var() / n + o.var() / n)
    assert abs(g.mean() - o.mean()) < 4 * se
    assert g.std() == pytest.approx(o.std(), rel=0.03)
    assert stats.skew(g) < -0.1 and abs(stats.skew(g) - stats.skew(o)) < 0.15


def test_pencil_beam_dose_with_vavilov():
    """64x64x128 water of 2 mm, 150 MeV, full physics with Vavilov straggling, 1e6 histories:
    z-scores, R80 and 2 %/2 mm gamma against the oracle."""
    from oracle import analysis as A
    from paper_1409_8336_gb300 import Engine

    prob = W.config1(flags=W.VAVILOV)
    n = 1_000_000
    e = Engine(device=0, n_batches=prob.n_batches, physics_flags=prob.flags, fast_math=True)
    e.load_problem(prob)
    e.transport(n, 21)
    tally = e.read_tally()
    L = e.read_ledger()
    e.close()
    ref, tot = O.run_parallel(prob, n, 21)
    Dg, sg = A.batch_stats(tally.astype(np.float64) * 2.0 ** -24)
    Do, so = A.batch_stats(ref)
    z = A.zscores(Dg, sg, Do, so)
    frac = np.mean(np.abs(z) <= 3.0)
    dz = prob.voxel[2]
    r80g = A.r80(A.depth_dose(Dg.reshape(prob.shape)), dz)
    r80o = A.r80(A.depth_dose(Do.reshape(prob.shape)), dz)
    gam = A.gamma_pass_rate(Do.reshape(prob.shape), Dg.reshape(prob.shape), prob.voxel)
    info = dict(z=frac, r80=(r80g, r80o), gamma=gam)
    assert frac >= 0.99, info
    assert abs(r80g - r80o) <= 0.01, info
    assert gam >= 0.99, info
    assert abs(L["incident"] - L["deposited"] - L["escaped"] - L["binding"]) < 1e-6 * L["incident"]
