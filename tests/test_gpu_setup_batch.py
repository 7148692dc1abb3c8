"""dgasm_setup_batch: preconditioners of several problems built at once (host plans on the worker threads, each
problem's device work on its own streams) must be the ones dgasm_setup builds one at a time, bit for bit, in
every precision mode and in the element-block case; a failing problem fails the whole call and is named."""
import numpy as np
import pytest

from tests.helpers import f_sin, have_gpu, mesh

pytestmark = pytest.mark.gpu

if have_gpu():
    import torch
    from paper_1903_11357_gb300 import dgasm as dg


def _system(n, seed, p, contrast=1.0):
    m = mesh(n, seed)
    rho = np.ones(n)
    if contrast != 1.0:
        rho = np.where(np.arange(n) % 2 == 0, 1.0, contrast)
    return dg.System(dg.Mesh.from_polymesh(m, rho), p, 10.0, f=f_sin)


def _problems():
    specs = [(600, 51, 2, 4, 16, "fp64", 1.0), (1200, 52, 3, 8, 32, "fp32", 1e2), (900, 53, 1, 4, 16, "bf16", 1.0),
             (700, 54, 2, 6, 24, "tf32", 1.0), (400, 55, 2, 400, 16, "fp64", 1.0), (1500, 56, 4, 6, 24, "fp32", 1.0)]
    return [dict(system=_system(n, seed, p, c), nsub=nsub, ncoarse=nc, precision=prec)
            for n, seed, p, nsub, nc, prec, c in specs]


def test_setup_batch_equals_setup_one_at_a_time():
    probs = _problems()
    batch = dg.setup_batch(probs)
    alone = [dg.Prec(**pr) for pr in probs]
    for i, (pb, pa, pr) in enumerate(zip(batch, alone, probs)):
        assert pb.info()["nsub"] == pa.info()["nsub"], i
        np.testing.assert_array_equal(pb.partition()[0], pa.partition()[0])
        r = torch.tensor(np.random.default_rng(i).standard_normal((2, pr["system"].ndof)), dtype=torch.float64,
                         device="cuda")
        zb, za = torch.zeros_like(r), torch.zeros_like(r)
        pb.apply(r, zb)
        pa.apply(r, za)
        assert torch.equal(zb, za), f"problem {i}: apply differs"
        b = torch.tensor(pr["system"].rhs(), dtype=torch.float64, device="cuda")
        xb, xa = torch.zeros_like(b), torch.zeros_like(b)
        rcb, sb = pb.solve(b, xb, rtol=1e-8)
        rca, sa = pa.solve(b, xa, rtol=1e-8)
        assert rcb == 0 and rca == 0
        assert sb[0]["iters"] == sa[0]["iters"], i
        assert torch.equal(xb, xa), f"problem {i}: solve differs"


def test_many_small_problems_at_once_equal_one_at_a_time():
    # more problems than worker threads, so that setups queue behind one another on the workers
    probs = [dict(system=_system(300 + 40 * i, 60 + i, 1 + i % 3), nsub=2 + i % 4, ncoarse=8 + 4 * (i % 3),
                  precision=["fp64", "fp32", "bf16"][i % 3]) for i in range(24)]
    batch = dg.setup_batch(probs)
    for i, (pb, pr) in enumerate(zip(batch, probs)):
        pa = dg.Prec(**pr)
        r = torch.tensor(np.random.default_rng(100 + i).standard_normal(pr["system"].ndof), dtype=torch.float64,
                         device="cuda")
        zb, za = torch.zeros_like(r), torch.zeros_like(r)
        pb.apply(r, zb)
        pa.apply(r, za)
        assert torch.equal(zb, za), f"problem {i}: apply differs"


def test_setup_batch_twice_in_a_row_and_batched_solve():
    probs = _problems()[:3]
    first = dg.setup_batch(probs)
    second = dg.setup_batch(probs)
    bs = [torch.tensor(pr["system"].rhs(), dtype=torch.float64, device="cuda") for pr in probs]
    xs1 = [torch.zeros_like(b) for b in bs]
    xs2 = [torch.zeros_like(b) for b in bs]
    assert dg.solve_batch(first, bs, xs1)[0] == 0
    assert dg.solve_batch(second, bs, xs2)[0] == 0
    for a, b in zip(xs1, xs2):
        assert torch.equal(a, b)


def test_setup_batch_fails_whole_and_names_the_problem():
    probs = _problems()[:3]
    probs[1] = dict(probs[1], p_c=9)   # coarse degree above p: rejected by the plan
    with pytest.raises(dg.DgasmError) as e:
        dg.setup_batch(probs)
    assert e.value.code == dg.EINVAL
    assert "problem 1" in str(e.value)
