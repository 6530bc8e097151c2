"""Failure detection on the GPU without a fault: the grid barriers of the
persistent iteration kernel wait at most a bounded number of polls, and a wait
that runs out is reported as AMPCG_ERR_TIMEOUT instead of hanging.  The test
makes a wait run out with a block that never arrives (a flag nothing sets) and
a short poll limit, then checks the status and that the device stays usable."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2505_04155_b300")


@pytest.mark.parametrize("nblocks", [2, 8])
def test_barrier_passes_when_every_block_arrives(nblocks):
    assert P.barrier_check(nblocks, -1, 1 << 16) == P.OK


@pytest.mark.parametrize("nblocks,absent", [(2, 1), (2, 0), (8, 5)])
def test_barrier_wait_runs_out_when_a_block_never_arrives(nblocks, absent):
    assert P.barrier_check(nblocks, absent, 2000) == P.ERR_TIMEOUT
    assert "gave up" in P.load_library().ampcg_last_error().decode()


def test_device_usable_after_a_timed_out_wait():
    assert P.barrier_check(4, 2, 500) == P.ERR_TIMEOUT
    a = W.poisson2d(16)
    b = torch.as_tensor(W.rhs_uniform(a.n, 0), device="cuda")
    s = P.Solver(a.rowptr, a.col, a.val)
    x, info = s.solve(b, tol=1e-10, maxit=500, policy=P.Policy.pcg64())
    s.close()
    assert info.status == P.OK and info.true_relres <= 1.01e-10
    assert P.barrier_check(4, -1, 1 << 16) == P.OK
