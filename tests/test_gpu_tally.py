"""The fixed-point dose tally, pinned bit for bit (GPU).

Sec. II.B.3: dose tallies are updated by atomic operations.  Here they are 64-bit integers in
units of 2^-24 MeV.  With the debug deposit log on, the engine records every deposit of a small
run as the energies it was computed from; the tally must equal the integer sum of
llrint(e 2^24) over those records, entry by entry, with nothing lost to the atomics and every
deposit at its voxel and group.  The logging build of the transport kernel must produce the
same tally as the production one."""
import numpy as np
import pytest

from paper_1409_8336_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _fixed(e):
    # llrint(e 2^24), round half to even: numpy's rint on exact products (e 2^24 < 2^53)
    return np.rint(e * 2.0 ** 24).astype(np.int64)


def _run(prob, n, seed, fast, log_cap=0, block=0):
    from paper_1409_8336_gb300 import Engine

    e = Engine(device=0, n_batches=prob.n_batches, physics_flags=prob.flags, fast_math=fast)
    e.load_problem(prob)
    if block:
        e.set_launch(block, 0)
    if log_cap:
        e.enable_deposit_log(log_cap)
    e.transport(n, seed)
    out = {"tally": e.read_tally(), "ledger": e.read_ledger()}
    if log_cap:
        out["log"] = e.read_deposit_log()
    e.close()
    return out


@pytest.mark.parametrize("fast", [False, True], ids=["ieee", "fastmath"])
@pytest.mark.parametrize("workload", ["slab", "ct"])
def test_tally_equals_integer_sum_of_logged_deposits(fast, workload):
    if workload == "slab":
        prob, n = W.config2(), 1000          # 70/150/230 MeV through water, bone, lung, titanium
    else:
        prob, n = W.config3(shape=(60, 64, 64), n_layers=4), 1000   # int16 HU path
    g = _run(prob, n, 31, fast, log_cap=1 << 21, block=128)
    log = g["log"]
    L = g["ledger"]
    assert len(log) > 50 * n and L["dropped"] == 0 and L["errors"] == 0
    assert L["inelastic"] > 0 and L["elastic"] > 0 and L["secondaries"] > 0   # cascade deposits logged too
    B = prob.n_batches
    q = _fixed(log["e"][:, 0]) - _fixed(log["e"][:, 1]) - _fixed(log["e"][:, 2])
    assert np.all((log["voxel"] >= 0) & (log["voxel"] < prob.n_voxels))
    assert np.all((log["group"] >= 0) & (log["group"] < B))
    ref = np.zeros(prob.n_voxels * B, dtype=np.int64)
    np.add.at(ref, log["voxel"].astype(np.int64) * B + log["group"], q)
    tally = g["tally"].reshape(-1)
    bad = np.flatnonzero(ref != tally)
    assert bad.size == 0, (bad[:10], ref[bad[:10]], tally[bad[:10]])
    assert int(q.sum()) == L["deposited"]
    # the logging kernel computes what the production kernel does
    plain = _run(prob, n, 31, fast, block=128)
    assert np.array_equal(plain["tally"], g["tally"])
    # and the launch shape changes nothing either
    other = _run(prob, n, 31, fast, block=256)
    assert np.array_equal(other["tally"], g["tally"])


def test_deposit_log_overflow_is_reported():
    from paper_1409_8336_gb300 import Engine, PmcError

    prob = W.config1()
    e = Engine(device=0, n_batches=prob.n_batches)
    e.load_problem(prob)
    e.enable_deposit_log(1000)
    e.transport(200, 5)
    with pytest.raises(PmcError) as ex:
        e.read_deposit_log()
    assert ex.value.code == -3       # PMC_E_QUEUE_OVERFLOW
    e.enable_deposit_log(0)
    e.close()
