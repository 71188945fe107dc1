"""The multi-plan stream: many plans through one GPU, several at a time, admitted by a
device-memory budget.  Every plan's dose must be bit-identical to running the plan alone
through the single-plan transport (the random numbers of a history depend only on its
identity and the seed, and the tallies are integers), whatever the concurrency, the budget
or the order in which plans finish."""
import numpy as np
import pytest

from paper_1409_8336_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _plans(n_plans=6, seed=11):
    """Small CT plans (2 mm voxels, 24-48 voxels a side) with 20-300 spots and 2e4-8e4
    histories; three phantoms shared between them."""
    rng = np.random.default_rng(seed)
    phantoms = [W.ct_phantom(shape, 0.2, seed + k) for k, shape in
                enumerate([(24, 32, 32), (40, 48, 48), (32, 40, 24)])]
    mats = [W.WATER, W.AIR, W.LUNG, W.BONE_LO, W.CORTICAL_BONE, W.TITANIUM]
    out = []
    for i in range(n_plans):
        hu = phantoms[i % len(phantoms)]
        nz, ny, nx = hu.shape
        rows = [W.spot_row(float(rng.uniform(60, 160)), x=float(rng.uniform(-1.5, 1.5)),
                           y=float(rng.uniform(-1.5, 1.5)), sigma=0.3, weight=float(rng.lognormal(0, 0.5)))
                for _ in range(int(rng.integers(20, 300)))]
        prob = W.Problem(W.NUCLIDES, mats, hu.shape, (0.2, 0.2, 0.2), (-nx * 0.1, -ny * 0.1, 0.0), np.array(rows),
                         hu=hu, hu_bins=list(W.HU_BINS), n_batches=10, name="plan%d" % i)
        out.append((prob, int(rng.integers(20_000, 80_000)), 1000 + i))
    return out


def _alone(plans, mode=0, params=None):
    from paper_1409_8336_gb300 import Engine

    ref = []
    e = Engine(device=0, n_batches=10, block_size=256)
    e.load_materials(plans[0][0].nuclides, plans[0][0].materials, plans[0][0].hu_bins)
    if params is not None:
        e.surrogate_load(params)
    for prob, n, seed in plans:
        e.load_phantom(prob.shape, prob.voxel, prob.origin, hu=prob.hu)
        e.clear_spots()
        e.add_spots(prob.spots)
        e.transport(n, seed, mode=mode)
        ref.append((e.read_dose(), e.read_ledger()))
    e.close()
    return ref


def _stream(plans, slots, budget, mode=0, params=None):
    from paper_1409_8336_gb300 import PlanStream

    s = PlanStream(device=0, slots=slots, budget_bytes=budget, n_batches=10)
    p0 = plans[0][0]
    s.load_materials(p0.nuclides, p0.materials, p0.hu_bins)
    if params is not None:
        s.load_surrogate(params)
    fps = [s.plan_bytes(prob, n, mode) for prob, n, _ in plans]
    rc, res = s.run(plans, mode)
    s.close()
    return rc, res, fps


def _same(res, ref):
    for r, ((d, sg), led) in zip(res, ref):
        assert r["status"] == 0
        assert np.array_equal(r["dose"], d)
        assert np.array_equal(r["sigma"], sg)
        for k in ("incident", "deposited", "escaped", "binding", "steps", "inelastic", "elastic"):
            assert r["ledger"][k] == led[k], k


def test_concurrent_plans_equal_plans_run_alone():
    plans = _plans()
    ref = _alone(plans)
    rc, res, _ = _stream(plans, slots=3, budget=8 << 30)
    assert rc == 0
    _same(res, ref)
    assert len({r["slot"] for r in res}) > 1                 # more than one slot served plans
    # with room for all of them, plans overlapped in time
    overlap = sum(1 for a in res for b in res if a is not b and a["t_admit_ms"] < b["t_end_ms"] and
                  b["t_admit_ms"] < a["t_end_ms"])
    assert overlap > 0


def test_memory_budget_bounds_what_is_admitted():
    """A budget that holds the largest plan but not two of them: the plans run one at a
    time (admitted bytes never exceed the budget) and give the same doses."""
    plans = _plans(seed=12)
    ref = _alone(plans)
    from paper_1409_8336_gb300 import PlanStream

    s = PlanStream(device=0, slots=3, budget_bytes=1 << 40)
    fps = [s.plan_bytes(p, n) for p, n, _ in plans]
    s.close()
    budget = max(fps) + min(fps) // 2
    rc, res, _ = _stream(plans, slots=3, budget=budget)
    assert rc == 0
    _same(res, ref)
    events = sorted([(r["t_admit_ms"], r["device_bytes"]) for r in res] + [(r["t_end_ms"], -r["device_bytes"])
                                                                            for r in res])
    level = 0
    for _, b in events:
        level += b
        assert level <= budget
    assert all(r["device_bytes"] == f for r, f in zip(res, fps))


def test_oversized_plan_is_refused_and_the_rest_run():
    plans = _plans(n_plans=4, seed=13)
    ref = _alone(plans)
    from paper_1409_8336_gb300 import PlanStream, PmcError

    s = PlanStream(device=0, slots=2, budget_bytes=1 << 40)
    fps = [s.plan_bytes(p, n) for p, n, _ in plans]
    s.close()
    big = int(np.argmax(fps))
    budget = sorted(fps)[-2] + 1                             # everything but the largest fits
    rc, res, _ = _stream(plans, slots=2, budget=budget)
    assert rc != 0 and res[big]["status"] == PmcError(-2, "").code == -2 and res[big]["slot"] == -1
    _same([r for i, r in enumerate(res) if i != big], [x for i, x in enumerate(ref) if i != big])


def test_surrogate_form_in_the_stream():
    from paper_1409_8336_gb300 import Engine

    plans = _plans(n_plans=4, seed=14)
    e = Engine(device=0, n_batches=10, block_size=256)
    p0 = plans[0][0]
    e.load_materials(p0.nuclides, p0.materials, p0.hu_bins)
    e.train_surrogate(n_events=200_000, epochs=1, batch=4096, seed=3)
    params = e.surrogate_params()
    e.close()
    ref = _alone(plans, mode=1, params=params)
    rc, res, _ = _stream(plans, slots=2, budget=8 << 30, mode=1, params=params)
    assert rc == 0
    _same(res, ref)
