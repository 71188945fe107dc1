"""The learned stand-in of the event generator on the GPU: gradients of the hand-written
forward/backward kernels against the FP64 reference, event summaries against the oracle's
cascade, training, and transport with the trained network against the full cascade."""
import math
import time

import numpy as np
import pytest
from scipy import stats

from oracle import analysis as A
from oracle import mlp
from oracle import oracle as O
from paper_1409_8336_gb300 import workloads as W

pytestmark = pytest.mark.gpu
FIX = 2.0 ** -24


@pytest.fixture(scope="module")
def trained():
    from paper_1409_8336_gb300 import Engine

    prob = W.config2()
    e = Engine(device=0, n_batches=10, fast_math=True)
    e.load_problem(prob)
    t0 = time.perf_counter()
    res = e.train_surrogate(n_events=10_000_000, epochs=2, batch=8192, lr=1e-3, seed=4)
    res["seconds"] = time.perf_counter() - t0
    params = e.surrogate_params()
    yield e, prob, res, params
    e.close()


def test_gradients_match_fp64_reference():
    from paper_1409_8336_gb300 import Engine

    e = Engine(device=0, n_batches=10)
    e.load_problem(W.config2())
    rng = np.random.default_rng(3)
    rows = 96
    p = np.concatenate([np.concatenate([rng.normal(0, np.sqrt(2.0 / mlp.DIMS[i]), mlp.DIMS[i] * mlp.DIMS[i + 1]),
                                        rng.normal(0, 0.05, mlp.DIMS[i + 1])]) for i in range(5)]).astype(np.float32)
    x = rng.normal(size=(rows, 32)).astype(np.float32)
    y = rng.normal(size=(rows, 16)).astype(np.float32)
    tau = rng.uniform(0.05, 0.95, size=(rows, 16)).astype(np.float32)
    mask = (rng.uniform(size=(rows, 16)) < 0.7).astype(np.float32)
    loss, g, yh = e.surrogate_grad(p, x, y, tau, mask)
    lo, go, yo = mlp.grad(p.astype(np.float64), x.astype(np.float64), y, tau, mask, round_bf16=True)
    e.close()
    assert np.allclose(yh, yo, rtol=2e-2, atol=2e-2 * np.abs(yo).max())
    assert loss == pytest.approx(lo, rel=1e-2)
    # per layer: relative error of the gradient in the Frobenius norm
    o = 0
    for i in range(5):
        for n in (mlp.DIMS[i] * mlp.DIMS[i + 1], mlp.DIMS[i + 1]):
            a, b = g[o:o + n], go[o:o + n]
            assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b) + 1e-7, (i, n, np.linalg.norm(a - b) / np.linalg.norm(b))
            o += n


@pytest.mark.parametrize("rows", [1, 128, 129, 1000, 40_000])
def test_tensor_core_network_matches_fp64_reference(rows):
    """The event stage's network on the 5th-generation tensor cores (tcgen05, 128-row tiles,
    accumulators in tensor memory) against the FP64 reference with the same BF16 roundings of
    weights and layer inputs: one partial tile, exactly one, one plus one row, a ragged tail,
    and more tiles than blocks."""
    from paper_1409_8336_gb300 import Engine

    e = Engine(device=0, n_batches=10)
    e.load_problem(W.config2())
    rng = np.random.default_rng(11)
    p = np.concatenate([np.concatenate([rng.normal(0, np.sqrt(2.0 / mlp.DIMS[i]), mlp.DIMS[i] * mlp.DIMS[i + 1]),
                                        rng.normal(0, 0.05, mlp.DIMS[i + 1])]) for i in range(5)]).astype(np.float32)
    e.surrogate_load(p)
    x = rng.normal(size=(rows, 32)).astype(np.float32)
    y = e.surrogate_infer(x)
    e.close()
    _, ref = mlp.forward(p.astype(np.float64), x.astype(np.float64), round_bf16=True)
    scale = np.abs(ref).max()
    err = np.abs(y - ref)
    assert np.all(np.isfinite(y))
    assert err.max() <= 2e-2 * scale, err.max() / scale
    assert np.median(err) <= 2e-3 * scale


def test_tensor_core_waits_are_bounded_and_the_context_recovers():
    """With the MMAs withheld every mbarrier wait of the pipeline runs out: the call returns
    PMC_E_TIMEOUT instead of hanging, and the same context then computes correctly."""
    from paper_1409_8336_gb300 import Engine
    from paper_1409_8336_gb300.engine import ERRORS

    e = Engine(device=0, n_batches=10)
    e.load_problem(W.config2())
    rng = np.random.default_rng(12)
    p = np.concatenate([np.concatenate([rng.normal(0, np.sqrt(2.0 / mlp.DIMS[i]), mlp.DIMS[i] * mlp.DIMS[i + 1]),
                                        rng.normal(0, 0.05, mlp.DIMS[i + 1])]) for i in range(5)]).astype(np.float32)
    e.surrogate_load(p)
    assert ERRORS[e.debug_surrogate_waits()] == "PMC_E_TIMEOUT"
    x = rng.normal(size=(300, 32)).astype(np.float32)
    y = e.surrogate_infer(x)
    e.close()
    _, ref = mlp.forward(p.astype(np.float64), x.astype(np.float64), round_bf16=True)
    assert np.abs(y - ref).max() <= 2e-2 * np.abs(ref).max()


def test_event_summaries_match_oracle_cascade():
    from paper_1409_8336_gb300 import Engine

    prob = W.config2()
    e = Engine(device=0, n_batches=10)
    e.load_problem(prob)
    seed = 11
    d = e.surrogate_dataset(20000, seed)
    e.close()
    assert stats.kstest((d[:, 0] - 10) / 240, "uniform").pvalue > 1e-3
    assert set(np.unique(d[:, 1]).astype(int)) == set(range(6))
    assert np.all(d[:, 2] >= 0) and np.all((d[:, 3:7] >= 0) & (d[:, 3:7] <= 1))
    assert np.all(np.abs(d[:, 7:11]) <= 1) and np.all(d[:, 11] >= 0)
    assert np.all(d[:, 3:7].sum(1) + d[:, 11] <= 1 + 1e-5)             # energy out <= energy in
    # the same events from the oracle: identical random streams, summarised the same way
    slots = [i for i, n in enumerate(prob.nuclides) if n[1] >= 2]
    same = 0
    for i in range(300):
        Z, Aa = prob.nuclides[slots[int(d[i, 1])]][:2]
        s_, pr, _ = O.inc_batch(Z, Aa, float(d[i, 0]), seed, i, 1)
        k = int(s_[0, 0])
        T = pr[0, :k, 1]
        sp = pr[0, :k, 0].astype(int)
        np_or = int(np.sum((sp == 1) & (T > 0.1)))
        same += np_or == int(d[i, 2])
    assert same >= 0.7 * 300, same


def test_training_reduces_the_pinball_loss(trained):
    _, _, res, params = trained
    assert res["steps"] > 1000
    assert res["last_loss"] < 0.8 * res["first_loss"], res
    assert np.all(np.isfinite(params))


def test_surrogate_spectra_against_cascade(trained):
    """Secondary-proton spectra of the trained network (sampled on the FP64 reference with the
    trained weights) against the cascade's, per target: KS statistics."""
    e, prob, _, params = trained
    d = e.surrogate_dataset(60000, 99)
    rng = np.random.default_rng(5)
    ks_T, ks_n = [], []
    for slot in range(6):
        rows = d[d[:, 1] == slot][:4000]
        n = len(rows)
        X = np.zeros((n, 32))
        X[:, 0] = (rows[:, 0] - 130) / 120
        X[np.arange(n), 1 + slot] = 1
        X[:, 7] = -1
        X[:, 8:18] = rng.uniform(size=(n, 10))
        q_np = mlp.forward(params, X)[1][:, 0]
        np_s = np.clip(np.floor(q_np + 0.5), 0, 4)
        X[:, 7] = np_s / 4
        y2 = mlp.forward(params, X)[1]
        T_s = (np.clip(y2[:, 1], 0, None) * rows[:, 0])[np_s >= 1]
        T_c = (rows[:, 3] * rows[:, 0])[rows[:, 2] >= 1]
        ks_T.append(stats.ks_2samp(T_s, T_c).statistic)
        ks_n.append(abs(np.mean(np_s) - np.mean(np.minimum(rows[:, 2], 4))))
    print("KS leading-proton energy per target:", np.round(ks_T, 3), "mean multiplicity error:", np.round(ks_n, 3))
    assert max(ks_T) < 0.15 and max(ks_n) < 0.3


def test_surrogate_transport_gamma_and_speed(trained):
    """The slab workload, 1e6 histories: dose with the trained network against the full cascade
    (2 %/2 mm gamma >= 98 %), energy bookkeeping, and the throughput gained."""
    e, prob, _, params = trained
    n = 1_000_000
    out = {}
    for mode in (0, 1):
        e.enable_profile(True)
        e.transport(n, 7, mode=mode)
        t = []
        for k in range(3):
            t0 = time.perf_counter()
            e.transport(n, 7, mode=mode)
            t.append(time.perf_counter() - t0)
        prof, _ = e.read_profile()
        D, sg = A.batch_stats(e.read_tally().astype(np.float64) * FIX)
        out[mode] = dict(D=D.reshape(prob.shape), t=min(t), led=e.read_ledger(), cascade_ms=prof["cascade"]["ms"])
    L = out[1]["led"]
    assert L["dropped"] == 0 and L["errors"] == 0
    assert abs(L["incident"] - L["deposited"] - L["escaped"] - L["binding"]) < 1e-6 * L["incident"]
    gam = A.gamma_pass_rate(out[0]["D"], out[1]["D"], prob.voxel)
    r80f = A.r80(A.depth_dose(out[0]["D"]), prob.voxel[2])
    r80s = A.r80(A.depth_dose(out[1]["D"]), prob.voxel[2])
    print("gamma %.4f, R80 full %.3f surrogate %.3f, event stage %.3f -> %.3f ms, transport %.2f -> %.2f ms" % (
        gam, r80f, r80s, out[0]["cascade_ms"], out[1]["cascade_ms"], 1e3 * out[0]["t"], 1e3 * out[1]["t"]))
    assert gam >= 0.98
    assert abs(r80f - r80s) < 0.02
    assert out[1]["cascade_ms"] < out[0]["cascade_ms"]
    # what the trained network gains over the method without it (the full cascade): the same
    # dose within 2 %/2 mm at a higher transport throughput, the event stage faster
    assert out[1]["t"] < out[0]["t"]


def event_stage_ks(e, prob, n_per_target=10000, seed=123):
    """The shipped event kernels on the same events: the learned stand-in's tensor-core event
    kernel against the cascade and evaporation kernels, per target nucleus, with E uniform in
    10-250 MeV.  Per target: KS statistic of the leading proton's energy and polar cosine, of all
    emitted protons' energies and cosines (the cascade's four most energetic per event, as the
    network has four slots), mean multiplicity (capped at four) and mean local deposit / E."""
    targets = [i for i, nu in enumerate(prob.nuclides) if nu[1] >= 2]
    rng = np.random.default_rng(seed)
    out = {}
    for t in targets:
        E = rng.uniform(10.0, 250.0, n_per_target)
        nuc = np.full(n_per_target, t, dtype=np.int32)
        res = {}
        for mode in (0, 1):
            pr, loc = e.debug_event_stage(mode, nuc, E, seed + t)
            ev = pr[:, 0].astype(np.int64)
            order = np.lexsort((-pr[:, 1], ev))
            pr, ev = pr[order], ev[order]
            first = np.r_[True, ev[1:] != ev[:-1]]
            rank = np.arange(len(ev)) - np.maximum.accumulate(np.where(first, np.arange(len(ev)), 0))
            top4 = pr[rank < 4]
            mult = np.bincount(ev, minlength=n_per_target)
            res[mode] = dict(lead_T=pr[first, 1] / E[ev[first]], lead_c=pr[first, 2], T=top4[:, 1] / E[top4[:, 0].astype(int)],
                             c=top4[:, 2], mult=np.minimum(mult, 4).mean(), local=np.mean(loc / E))
        a, b = res[0], res[1]
        Z, A_ = prob.nuclides[t][:2]
        out["%d-%d" % (Z, A_)] = {
            "ks_leading_T": float(stats.ks_2samp(a["lead_T"], b["lead_T"]).statistic),
            "ks_leading_cos": float(stats.ks_2samp(a["lead_c"], b["lead_c"]).statistic),
            "ks_T": float(stats.ks_2samp(a["T"], b["T"]).statistic),
            "ks_cos": float(stats.ks_2samp(a["c"], b["c"]).statistic),
            "multiplicity": [float(a["mult"]), float(b["mult"])],
            "local_over_E": [float(a["local"]), float(b["local"])]}
    return out


def test_event_stage_kernel_against_cascade_kernel(trained):
    """The secondary spectra of the shipped surrogate event kernel (row building from the
    events' own random streams, BF16 network on tcgen05, multiplicity rounding, clamping and
    energy scaling) against those of the cascade kernels on the same events, per target."""
    e, prob, _, _ = trained
    ks = event_stage_ks(e, prob)
    for k, v in ks.items():
        print(k, {kk: (np.round(vv, 3).tolist() if isinstance(vv, list) else round(vv, 3)) for kk, vv in v.items()})
    assert len(ks) == 6
    for k, v in ks.items():
        assert v["ks_leading_T"] < 0.08 and v["ks_T"] < 0.08, (k, v)
        assert v["ks_leading_cos"] < 0.08 and v["ks_cos"] < 0.08, (k, v)
        assert abs(v["multiplicity"][0] - v["multiplicity"][1]) < 0.15, (k, v)
        assert abs(v["local_over_E"][0] - v["local_over_E"][1]) < 0.05, (k, v)
