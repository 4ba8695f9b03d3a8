"""Failure detection without a GPU fault: the bounded mbarrier wait that every
asynchronous-copy and tensor-core kernel of the library uses gives up after
its poll limit, flags DGR_STATUS_TIMEOUT in the status word the host reads,
and leaves the context usable.  The wait is made to run out on purpose on an
mbarrier nothing arrives at, with nothing in flight (dgr_test_bounded_wait);
no trap, fault or endless loop is involved."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2411_04844_b300 import dgr, synth
from tests._common import oracle_grid, rel_l2

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.mark.parametrize("polls", [1, 1000])
def test_bounded_wait_gives_up_flags_timeout_and_the_context_survives(polls):
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    gave_up = torch.full((1,), -1, dtype=torch.int32, device=DEV)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dgr.dgr_test_bounded_wait(polls, status, gave_up)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    print(f"{polls} unsuccessful polls: {dt * 1e3:.3f} ms")
    assert dt < 5.0  # the wait ends by its own limit
    assert int(gave_up) == 1
    assert int(status) & dgr.DGR_STATUS_TIMEOUT
    # the context still runs work correctly afterwards
    gs = synth.GridSpec((24, 20, 16), 1.0, (-12.0, -10.0, -8.0))
    f = synth.gaussian_field(synth.rng_for(1, 91), 50, gs, ("loguniform", 0.6, 2.5))
    grid = dgr.Grid.of(gs)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=DEV)
    ws = dgr.Workspace(dgr.make_plan(grid, f.n, 200000, 200000))
    vol = torch.empty(gs.shape, device=DEV)
    dgr.dgr_voxelize(grid, T(f.mu), T(f.s), T(f.q), T(f.rho), 3.0, vol, ws)
    torch.cuda.synchronize()
    assert dgr.dgr_status(ws) == 0
    vo = O.voxelize(oracle_grid(gs), f.mu, f.s, f.q, f.rho, 3.0)
    assert rel_l2(vol.cpu().numpy(), vo) <= 1e-5


def test_bounded_wait_rejects_limits_beyond_the_kernels_own():
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    gave_up = torch.zeros(1, dtype=torch.int32, device=DEV)
    for bad in (0, (1 << 18) + 1):
        with pytest.raises(dgr.DgrError):
            dgr.dgr_test_bounded_wait(bad, status, gave_up)
