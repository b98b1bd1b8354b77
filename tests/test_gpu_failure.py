"""Failure detection without a GPU fault: the bounded waits of the grid
barrier that the cooperative solvers use between phases.  A block that
never arrives (made on purpose, by a launch argument) makes every other
block's wait run out after a short budget; the kernel ends, the error flag
is set, and the context stays usable for the next solve."""
import numpy as np
import pytest
import torch

import oracle
from paper_2601_13994_b300 import _lib as L
from paper_2601_13994_b300 import inputs as I
from paper_2601_13994_b300 import sla
from tests.gpu_util import csr, rel, to_dev

pytestmark = pytest.mark.gpu


def _selftest(blocks, absent, budget, rounds):
    word = torch.zeros(4, dtype=torch.int32, device="cuda")
    rc = L.lib().sla_selftest_grid_barrier(blocks, absent, budget, rounds, word.data_ptr(),
                                           torch.cuda.current_stream().cuda_stream)
    assert rc == L.SLA_OK, rc
    torch.cuda.synchronize()
    return [int(v) for v in word.cpu()]


def test_every_block_passes_when_all_arrive():
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for blocks in (1, 7, sms, 2 * sms):
        timed_out, passed, count, err = _selftest(blocks, -1, 4_000_000_000, 50)
        assert (timed_out, passed, err) == (0, blocks, 0)
        assert count == 50 * blocks   # the counter only grows


def test_missing_block_makes_the_waits_run_out_and_the_context_survives():
    # about 1 ms of budget at the B300's clock; block 3 never arrives
    timed_out, passed, count, err = _selftest(64, 3, 2_000_000, 5)
    assert timed_out == 63 and passed == 0 and err == 1
    assert count == 63                 # every present block arrived at the first barrier
    # the device still works: a cooperative solve right after
    rp, c, v = I.poisson2d(40)
    b = I.rhs_uniform(1600, 5)
    x, info = sla.cg(csr(rp, c), to_dev(v), to_dev(b), rtol=1e-10)
    xo, _ = oracle.pcg(rp, c, v, b, rtol=1e-13)
    assert info.status == 0 and rel(x.cpu().numpy(), xo) <= 1e-8
