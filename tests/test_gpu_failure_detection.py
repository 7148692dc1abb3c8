"""Failure detection without a GPU fault: the kernels' waits are bounded.  A wait that nothing satisfies
(an mbarrier no one arrives on) gives up after its limit, sets the error word and returns; the host reads
the status and the context stays usable for the next solve."""
import numpy as np
import pytest

from tests.helpers import have_gpu

pytestmark = pytest.mark.gpu

if have_gpu():
    import torch
    from paper_1903_11357_gb300 import dgasm as dg


def test_bounded_wait_gives_up_and_context_survives():
    gave_up, ms = dg.selftest_bounded_wait(5.0)
    assert gave_up
    assert 2.0 <= ms <= 1000.0
    # the same context solves a problem afterwards
    from tests.test_gpu_parity import build_case, dev
    c = build_case(200, 2, 2, 4, 8)
    x = torch.zeros(len(c["b"]), dtype=torch.float64, device="cuda")
    rc, st = c["P"].solve(dev(c["b"]), x)
    assert rc == 0 and st[0]["converged"]
    xs = np.linalg.solve(c["A"].toarray(), c["b"])
    assert np.linalg.norm(x.cpu().numpy() - xs) <= 1e-6 * np.linalg.norm(xs)


def test_bounded_wait_rejects_bad_limits():
    with pytest.raises(dg.DgasmError):
        dg.selftest_bounded_wait(0.0)
    with pytest.raises(dg.DgasmError):
        dg.selftest_bounded_wait(5000.0)
