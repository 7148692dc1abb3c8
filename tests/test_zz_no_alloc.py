"""The allocation-free entry point dgasm_system_spmv_dot_noalloc, for callers that cannot allocate device
memory (inside a stream capture, under another runtime's allocator, in real-time loops): its y = A x must
equal the regular dgasm_system_spmv output and its x^T A x the inner product of x with that output, on two
calls in a row (the shared fixed scratch must be left ready for the next call).  Kept in its own file so
that it is collected last."""
import ctypes as C

import numpy as np
import pytest

from tests.helpers import have_gpu, mesh

pytestmark = pytest.mark.gpu

if have_gpu():
    import torch
    from paper_1903_11357_gb300 import dgasm as dg


@pytest.mark.parametrize("n,p", [(300, 2), (1200, 3)])
def test_spmv_dot_noalloc_matches_regular_entry_point(n, p):
    m = mesh(n, 21)
    S = dg.System(dg.Mesh.from_polymesh(m, np.ones(n)), p, 10.0)
    rng = np.random.default_rng(7)
    x = torch.tensor(rng.standard_normal(S.ndof), dtype=torch.float64, device="cuda")
    y_ref = torch.zeros_like(x)
    S.spmv(x, y_ref)                      # regular entry point (also uploads the matrix)
    torch.cuda.synchronize()
    ref_dot = float(torch.dot(x, y_ref))
    for call in range(2):
        y = torch.full_like(x, float("nan"))
        d = torch.zeros(1, dtype=torch.float64, device="cuda")
        rc = dg.lib().dgasm_system_spmv_dot_noalloc(S.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                                    C.c_void_p(d.data_ptr()), None)
        assert rc == 0, dg.last_error()
        torch.cuda.synchronize()
        assert torch.equal(y, y_ref), f"call {call}"
        assert abs(float(d) - ref_dot) <= 1e-12 * abs(ref_dot), f"call {call}"


def test_spmv_dot_noalloc_needs_uploaded_matrix():
    m = mesh(64, 22)
    S = dg.System(dg.Mesh.from_polymesh(m, np.ones(64)), 1, 10.0)
    x = torch.zeros(S.ndof, dtype=torch.float64, device="cuda")
    rc = dg.lib().dgasm_system_spmv_dot_noalloc(S.h, C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()),
                                                C.c_void_p(x.data_ptr()), None)
    assert rc == dg.EINVAL and "not on the device" in dg.last_error()
