"""The allocation-free entry point dgasm_system_spmv_dot_noalloc.  It is there for callers that must not
allocate device memory once they run: code whose device memory belongs to another runtime's caching
allocator, and real-time loops whose memory is fixed at start-up.  Its y = A x must equal the regular
dgasm_system_spmv output bit for bit and its x^T A x the inner product of x with that output (to 1e-12), on
two calls in a row (the shared fixed scratch must be left ready for the next call); a counting allocator
installed through dgasm_set_allocator must see no allocation and no free during those calls.  Kept in its
own file, named so that pytest collects it last."""
import ctypes as C
import gc

import numpy as np
import pytest

from tests.helpers import have_gpu, mesh

pytestmark = pytest.mark.gpu

if have_gpu():
    import torch
    from paper_1903_11357_gb300 import dgasm as dg


class CountingAllocator:
    """Device allocator hooks that count every call and hand out nothing (an allocation attempt fails with
    DGASM_ENOMEM and is counted); installed only around calls that must not allocate."""

    def __init__(self):
        self.allocs = 0
        self.frees = 0
        self._a = dg.ALLOC_FN(self._alloc)
        self._f = dg.FREE_FN(self._free)

    def _alloc(self, nbytes, stream, user):
        self.allocs += 1
        return None

    def _free(self, ptr, stream, user):
        self.frees += 1

    def __enter__(self):
        gc.disable()   # no library object may be destroyed (and free through these hooks) in the window
        dg.check(dg.lib().dgasm_set_allocator(C.cast(self._a, C.c_void_p), C.cast(self._f, C.c_void_p), None))
        return self

    def __exit__(self, *exc):
        dg.check(dg.lib().dgasm_set_allocator(None, None, None))
        gc.enable()
        return False


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
    ys = [torch.full_like(x, float("nan")) for _ in range(2)]
    ds = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in range(2)]
    with CountingAllocator() as hooks:
        for call in range(2):
            S.spmv_dot_noalloc(x, ys[call], ds[call])
            torch.cuda.synchronize()
    assert hooks.allocs == 0 and hooks.frees == 0
    for call in range(2):
        assert torch.equal(ys[call], y_ref), f"call {call}"
        assert abs(float(ds[call]) - ref_dot) <= 1e-12 * abs(ref_dot), f"call {call}"


def test_spmv_dot_noalloc_rejects_bad_calls():
    m = mesh(64, 22)
    S = dg.System(dg.Mesh.from_polymesh(m, np.ones(64)), 1, 10.0)
    x = torch.zeros(S.ndof, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    L = dg.lib()
    rc = L.dgasm_system_spmv_dot_noalloc(S.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                         C.c_void_p(d.data_ptr()), None)
    assert rc == dg.EINVAL and "not on the device" in dg.last_error()
    S.spmv(x, y)
    torch.cuda.synchronize()
    # y aliasing x, and xAx inside y
    rc = L.dgasm_system_spmv_dot_noalloc(S.h, C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()),
                                         C.c_void_p(d.data_ptr()), None)
    assert rc == dg.EINVAL and "overlap" in dg.last_error()
    rc = L.dgasm_system_spmv_dot_noalloc(S.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                         C.c_void_p(y.data_ptr() + 8), None)
    assert rc == dg.EINVAL and "overlap" in dg.last_error()
    with pytest.raises(ValueError):
        S.spmv_dot_noalloc(x[:-1], y, d)
