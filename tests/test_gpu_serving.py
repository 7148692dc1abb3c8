"""Continuous-batching server: requests of different sizes and degrees admitted as slots and memory
free up; every result equals the same solve run alone (bitwise: each problem's arithmetic and
reduction order do not depend on the batch)."""
import numpy as np
import pytest

from tests.helpers import have_gpu, mesh

pytestmark = pytest.mark.gpu

if have_gpu():
    import torch
    from paper_1903_11357_gb300 import dgasm as dg


def make_system(n, seed, p):
    m = mesh(n, seed)
    rng = np.random.default_rng(seed)
    M = dg.Mesh.from_polymesh(m, 10.0 ** rng.uniform(0, 3, n))
    return dg.System(M, p, 10.0)


def rhs(S, k, seed):
    r = np.random.default_rng(seed).standard_normal((k, S.ndof))
    return torch.tensor(r if k > 1 else r[0], dtype=torch.float64, device="cuda")


CASES = [(256, 1, 2, 4, 16, 1, "fp64"), (400, 2, 3, 4, 16, 2, "fp32"), (300, 3, 1, 2, 8, 3, "fp64"),
         (500, 4, 2, 8, 32, 1, "bf16"), (200, 5, 4, 2, 8, 2, "fp64")]


def alone(S, nsub, ncoarse, b, precision):
    P = dg.Prec(S, nsub, ncoarse, 1, precision=precision)
    x = torch.zeros_like(b)
    rc, st = P.solve(b, x)
    assert rc == 0
    return x


def test_results_equal_alone_and_in_the_mix():
    systems = [make_system(n, s, p) for (n, s, p, *_ ) in CASES]
    bs = [rhs(S, c[5], 10 + i) for i, (S, c) in enumerate(zip(systems, CASES))]
    refs = [alone(S, c[3], c[4], b, c[6]) for S, c, b in zip(systems, CASES, bs)]
    sv = dg.Server(hbm_budget=8 << 30, max_slots=3)
    xs = [torch.zeros_like(b) for b in bs]
    tickets = [sv.submit(S, c[3], c[4], 1, b, x, precision=c[6]) for S, c, b, x in zip(systems, CASES, bs, xs)]
    for t, x, ref in zip(tickets, xs, refs):
        rc, st = sv.wait(t, 60000)
        assert rc == 0 and all(s["converged"] for s in st)
        assert torch.equal(x, ref)
    stats = sv.stats()
    assert stats["done"] == len(CASES) and stats["bytes_in_use"] == 0
    sv.close()


def test_admission_by_memory_budget_and_errors():
    S = make_system(400, 7, 3)
    P = dg.Prec(S, 4, 16, 1)
    need = P.footprint()
    sv = dg.Server(hbm_budget=int(need * 2.5), max_slots=4)   # room for one request at a time
    bs = [rhs(S, 1, 20 + i) for i in range(3)]
    xs = [torch.zeros_like(b) for b in bs]
    ts = [sv.submit(S, 4, 16, 1, b, x) for b, x in zip(bs, xs)]
    for t in ts:
        rc, st = sv.wait(t, 60000)
        assert rc == 0
    ref = alone(S, 4, 16, bs[2], "fp64")
    assert torch.equal(ref, xs[2])
    assert sv.stats()["stalls"] > 0
    tiny = dg.Server(hbm_budget=1 << 20, max_slots=1)
    with pytest.raises(dg.DgasmError) as e:
        tiny.submit(S, 4, 16, 1, bs[0], xs[0])
    assert e.value.code == dg.ETOOBIG
    tiny.close()
    assert sv.poll(123456)[0] == dg.ENOTFOUND
    sv.close()


def test_cancel_queued_request():
    S = make_system(600, 8, 3)
    sv = dg.Server(hbm_budget=8 << 30, max_slots=1)
    bs = [rhs(S, 1, 30 + i) for i in range(4)]
    xs = [torch.zeros_like(b) for b in bs]
    ts = [sv.submit(S, 4, 16, 1, b, x) for b, x in zip(bs, xs)]
    rc = sv.cancel(ts[-1])
    assert rc in (dg.OK, dg.PENDING)
    out = sv.wait(ts[-1], 60000)[0]
    assert out in (dg.ECANCELLED, dg.OK)
    for t in ts[:-1]:
        assert sv.wait(t, 60000)[0] == 0
    sv.close()


def test_restarts_from_the_true_residual_in_the_mix():
    """A tight tolerance makes the recursive residual run ahead of b - A x, so requests restart from the
    true residual (residual replacement) while others come and go; each result still equals the solve
    alone and meets the tolerance in both senses."""
    cases = [(300, 21, 3, 4, 16, 1), (400, 22, 2, 4, 16, 2), (250, 23, 3, 2, 8, 1), (350, 24, 2, 4, 8, 3)]
    systems = [make_system(n, s, p) for (n, s, p, *_) in cases]
    bs = [rhs(S, c[5], 30 + i) for i, (S, c) in enumerate(zip(systems, cases))]
    refs = []
    for S, c, b in zip(systems, cases, bs):
        P = dg.Prec(S, c[3], c[4], 1)
        x = torch.zeros_like(b)
        rc, st = P.solve(b, x, rtol=1e-12)
        assert rc == 0 and all(s["true_relres"] <= 1e-12 for s in st)
        refs.append(x)
    sv = dg.Server(hbm_budget=8 << 30, max_slots=2)
    xs = [torch.zeros_like(b) for b in bs]
    tickets = [sv.submit(S, c[3], c[4], 1, b, x, rtol=1e-12) for S, c, b, x in zip(systems, cases, bs, xs)]
    for t, x, ref in zip(tickets, xs, refs):
        rc, st = sv.wait(t, 60000)
        assert rc == 0 and all(s["converged"] and s["true_relres"] <= 1e-12 for s in st)
        assert torch.equal(x, ref)
    sv.close()


def test_server_keeps_the_system_of_a_pending_request():
    """The server reads a request's system until it finishes: the binding holds the reference, so a
    system the caller no longer names is not destroyed under a queued request."""
    import gc
    ref_S = make_system(300, 9, 2)
    b = rhs(ref_S, 1, 40)
    ref = alone(ref_S, 4, 16, b, "fp64")
    sv = dg.Server(hbm_budget=8 << 30, max_slots=1)
    xs = [torch.zeros_like(b) for _ in range(3)]
    ts = [sv.submit(make_system(300, 9, 2), 4, 16, 1, b, x) for x in xs]   # temporaries only
    gc.collect()
    for t, x in zip(ts, xs):
        rc, st = sv.wait(t, 60000)
        assert rc == 0 and st[0]["converged"]
        assert torch.equal(x, ref)
    sv.close()
