"""GPU 3-D gamma index (Sec. II.D, Low et al.) against the oracle's gamma, voxel by voxel.

Both compute gamma^2 in FP64 with the same operations in the same order, so the GPU's
float32 gamma map must equal the float32 square root of the oracle's gamma^2 exactly, and
the counts of evaluated and passing voxels must be equal."""
import numpy as np
import pytest

from oracle import analysis as A
from paper_1409_8336_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _oracle_map(ref, ev, voxel, dose_pct=2.0, dta=2.0, threshold=0.1, search=None):
    g2, m = A.gamma_index(ref, ev, voxel, dose_pct, dta, threshold, search)
    g = np.full(ref.shape, -1.0, dtype=np.float32)
    g[m] = np.sqrt(g2[m]).astype(np.float32)
    return g, int(m.sum()), int(A.gamma_passes(g2[m]).sum())


def _smooth_pair(shape, seed, noise=0.01, shift=(0.0, 0.0, 0.0)):
    """A dose-like field (sum of Gaussian blobs) and a perturbed, shifted copy."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ref = np.zeros(shape)
    ev = np.zeros(shape)
    for _ in range(4):
        c = rng.uniform(0, 1, 3) * np.array(shape)
        s = rng.uniform(0.1, 0.3, 3) * np.array(shape) + 1.0
        a = rng.uniform(0.5, 1.0)
        ref += a * np.exp(-(((z - c[0]) / s[0]) ** 2 + ((y - c[1]) / s[1]) ** 2 + ((x - c[2]) / s[2]) ** 2) / 2)
        ev += a * np.exp(-(((z - c[0] - shift[0]) / s[0]) ** 2 + ((y - c[1] - shift[1]) / s[1]) ** 2
                           + ((x - c[2] - shift[2]) / s[2]) ** 2) / 2)
    ev *= 1.0 + noise * rng.standard_normal(shape)
    return ref, ev


CASES = [  # shape, voxel (cm), dose %, dta mm, threshold, search mm (None = 1.5 dta)
    ((23, 29, 37), (0.1, 0.1, 0.1), 2.0, 2.0, 0.1, None),
    ((16, 40, 40), (0.125, 0.125, 0.25), 2.0, 2.0, 0.1, None),   # the paper's CT voxel size
    ((9, 13, 1), (0.2, 0.15, 0.1), 3.0, 3.0, 0.0, 6.0),
    ((1, 1, 300), (0.1, 0.1, 0.05), 1.0, 1.0, 0.05, None),
    ((33, 17, 65), (0.05, 0.05, 0.05), 2.0, 2.0, 0.1, None),     # 0.5 mm voxels: many offsets
]


@pytest.mark.parametrize("case", CASES, ids=[str(c[0]) for c in CASES])
def test_gamma_map_equals_oracle(case):
    from paper_1409_8336_gb300 import gamma_index

    shape, voxel, pct, dta, thr, search = case
    shift = tuple(0.0 if n == 1 else s for n, s in zip(shape, (0.4, -0.7, 0.9)))   # none along a flat axis
    ref, ev = _smooth_pair(shape, seed=sum(shape), noise=0.015, shift=shift)
    go, n_eval, n_pass = _oracle_map(ref, ev, voxel, pct, dta, thr, search)
    g, rate = gamma_index(ref, ev, voxel, pct, dta, thr, search or 0.0)
    assert np.array_equal(g, go)
    assert rate == pytest.approx(n_pass / n_eval, abs=0, rel=1e-15)
    assert 0.0 < rate < 1.0                  # both passing and failing voxels


def test_gamma_of_engine_doses_equals_oracle():
    """Two dose maps of the slab phantom from the engine at different seeds."""
    from paper_1409_8336_gb300 import Engine, gamma_index

    prob = W.config2()
    eng = Engine(device=0, n_batches=prob.n_batches)
    eng.load_problem(prob)
    maps = []
    for seed in (5, 6):
        eng.transport(200_000, seed)
        maps.append(eng.read_dose()[0].reshape(prob.shape))
    eng.close()
    go, n_eval, n_pass = _oracle_map(maps[0], maps[1], prob.voxel)
    g, rate = gamma_index(maps[0], maps[1], prob.voxel)
    assert np.array_equal(g, go)
    assert rate == n_pass / n_eval


def test_gamma_full_size_ct_grid_and_device_entry():
    """The 256 x 256 x 160 CT grid at 1 mm, device-resident doses on a side stream,
    through the workspace entry point: the map and the counts equal the oracle's."""
    import torch

    from paper_1409_8336_gb300 import GammaIndex

    shape, voxel = (160, 256, 256), (0.1, 0.1, 0.1)
    ref, ev = _smooth_pair(shape, seed=3, noise=0.02, shift=(1.0, 0.5, -0.5))
    go, n_eval, n_pass = _oracle_map(ref, ev, voxel)
    gi = GammaIndex(voxel)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        r = torch.from_numpy(ref).to("cuda", non_blocking=False)
        e = torch.from_numpy(ev).to("cuda", non_blocking=False)
        g = torch.empty(shape, dtype=torch.float32, device="cuda")
    s.synchronize()
    gi(r, e, g, stream=s)
    s.synchronize()
    assert gi.counts() == (n_eval, n_pass)
    assert np.array_equal(g.cpu().numpy(), go)
    gi(r, r, None, stream=s)                  # identical doses, no map: every voxel passes
    s.synchronize()
    assert gi.counts() == (n_eval, n_eval)


def test_gamma_degenerate_inputs():
    from paper_1409_8336_gb300 import gamma_index

    z = np.zeros((4, 5, 6))
    g, rate = gamma_index(z, z, (0.1, 0.1, 0.1))
    assert np.isnan(rate) and np.all(g == -1.0)
    one = np.zeros((1, 1, 1)) + 3.0
    g, rate = gamma_index(one, one * 1.01, (0.1, 0.1, 0.1))
    go, _, _ = _oracle_map(one, one * 1.01, (0.1, 0.1, 0.1))
    assert rate == 1.0 and np.array_equal(g, go) and abs(g[0, 0, 0] - 0.5) < 1e-6
