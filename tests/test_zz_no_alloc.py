"""The transport entry point that allocates no device memory gives the same results as the
allocating one.

It exists for callers that cannot call cudaMalloc during a dose calculation (a real-time loop
that must not stall on the allocator, or an application whose own pool owns the device
memory).  Its scratch is a static device array shared by every call on a device, so the test
makes two calls in a row with different seeds: the second must not see anything the first left
behind.  Two host threads making their first calls at once (in a fresh process) both get the
allocating entry point's tally: the array's address is looked up once per device and the calls
are serialised.  This file is collected last so that a run stopping at the first failure has
already run every other test."""
import os
import subprocess
import sys

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


_TWO_THREADS = r"""
import sys, threading
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_1409_8336_gb300 import Engine
from paper_1409_8336_gb300 import workloads as W

prob = W.config1()
n, seed = 20000, 41
ref = Engine(device=0, n_batches=prob.n_batches)
ref.load_problem(prob)
ref.transport(n, seed)
expected = ref.read_tally().reshape(-1)
ref.close()
engines, outs = [], []
for _ in range(2):
    e = Engine(device=0, n_batches=prob.n_batches)
    e.load_problem(prob)
    engines.append(e)
    outs.append(torch.full((prob.n_voxels * prob.n_batches,), -1, dtype=torch.int64, device="cuda"))
torch.cuda.synchronize()
gate = threading.Barrier(2)
errors = []

def first_call(e, t):
    try:
        gate.wait()
        e.transport_noalloc(n, seed, t.data_ptr())
    except Exception as ex:  # reported below
        errors.append(repr(ex))

th = [threading.Thread(target=first_call, args=(engines[i], outs[i])) for i in range(2)]
for t in th:
    t.start()
for t in th:
    t.join()
torch.cuda.synchronize()
assert not errors, errors
for t in outs:
    assert np.array_equal(t.cpu().numpy(), expected)
for e in engines:
    e.close()
print("TWO_THREADS_OK")
"""


def test_noalloc_first_calls_from_two_threads():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _TWO_THREADS, root], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "TWO_THREADS_OK" in r.stdout, (r.stdout[-2000:], r.stderr[-4000:])
