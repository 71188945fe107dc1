"""The transport entry point that allocates no device memory gives the same results as the
allocating one.

It exists for callers that cannot call cudaMalloc during a dose calculation (a host callback
or real-time loop that must not stall on the allocator, or an application whose own pool owns
the device memory).  Its scratch is a static device array shared by every call on a device,
so the test makes two calls in a row with different seeds: the second must not see anything
the first left behind.  This file is collected last so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

from paper_1409_8336_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fast", [False, True], ids=["ieee", "fastmath"])
def test_noalloc_transport_matches_transport_on_two_calls(fast):
    import torch

    from paper_1409_8336_gb300 import Engine

    prob = W.config2()
    n = 150_000                      # several no-allocation sub-groups of 65536 histories
    seeds = (21, 22)
    ref = Engine(device=0, n_batches=prob.n_batches, fast_math=fast)
    ref.load_problem(prob)
    expected = []
    for s in seeds:
        ref.transport(n, s)
        d, sg = ref.read_dose()
        expected.append((ref.read_tally(), d, sg, ref.read_ledger()))
    ref.close()

    eng = Engine(device=0, n_batches=prob.n_batches, fast_math=fast)
    eng.load_problem(prob)
    nv, B = prob.n_voxels, prob.n_batches
    tally = torch.empty(nv * B, dtype=torch.int64, device="cuda")
    dose = torch.empty(nv, dtype=torch.float64, device="cuda")
    sigma = torch.empty(nv, dtype=torch.float64, device="cuda")
    for s, (t_ref, d_ref, s_ref, l_ref) in zip(seeds, expected):
        tally.fill_(-1)
        eng.transport_noalloc(n, s, tally.data_ptr(), dose.data_ptr(), sigma.data_ptr())
        torch.cuda.synchronize()
        t = tally.cpu().numpy().reshape(nv, B)
        # integer tallies: identical, since each history's random numbers depend on its identity only
        assert np.array_equal(t, t_ref)
        assert np.allclose(dose.cpu().numpy(), d_ref, rtol=1e-12, atol=0)
        assert np.allclose(sigma.cpu().numpy(), s_ref, rtol=1e-12, atol=0)
        led = eng.read_ledger()
        for k in ("incident", "deposited", "escaped", "binding", "steps", "inelastic"):
            assert led[k] == l_ref[k], k
        assert led["dropped"] == 0 and led["errors"] == 0
    eng.close()


def test_noalloc_rejects_too_many_spots():
    from paper_1409_8336_gb300 import Engine, PmcError

    import torch

    prob = W.water_box((8, 8, 8), 0.5)
    eng = Engine(device=0, n_batches=2)
    eng.load_problem(prob)
    eng.clear_spots()
    eng.add_spots(np.array([W.spot_row(100.0, x=0.0, y=0.0)] * 5000))
    tally = torch.empty(prob.n_voxels * 2, dtype=torch.int64, device="cuda")
    with pytest.raises(PmcError, match="no-allocation limit"):
        eng.transport_noalloc(10000, 1, tally.data_ptr())
    eng.close()
