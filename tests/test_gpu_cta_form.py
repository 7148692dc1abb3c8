"""The two forms of the FP32 and BF16 local-solve launches: a cluster of two CTAs per subdomain item, or one CTA
of twice the warps per item (which the library takes when a launch's pairs would not all fit on the GPU at
once).  Both add the same products in the same order, so solves and preconditioner applications must agree bit
for bit, alone and in a batch large enough for the automatic choice to switch forms."""
import numpy as np
import pytest

from tests.helpers import f_sin, have_gpu, mesh

pytestmark = pytest.mark.gpu

if have_gpu():
    import torch
    from paper_1903_11357_gb300 import dgasm as dg


def _prec(n, seed, p, nsub, ncoarse, precision):
    m = mesh(n, seed)
    S = dg.System(dg.Mesh.from_polymesh(m, np.ones(n)), p, 10.0, f=f_sin)
    P = dg.Prec(S, nsub, ncoarse, 1, precision=precision)
    P.set_local_variant("sweeps")   # the envelope sweeps: the kernel whose launch form is under test
    return S, P


def _solve(P, B, form, kc=None):
    dg.set_local_cta_form(form)
    try:
        if kc is not None:
            P.set_rhs_chunk(B.shape[0], kc)
        X = torch.zeros_like(B)
        rc, st = P.solve(B, X, rtol=1e-8)
        Z = torch.zeros_like(B)
        P.apply(B, Z)
        torch.cuda.synchronize()
    finally:
        dg.set_local_cta_form("auto")
    assert rc == 0
    return X, Z, [s["iters"] for s in st]


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("nrhs,kc", [(1, None), (4, 4), (4, 1)])
def test_one_cta_form_equals_pair_bitwise(precision, nrhs, kc):
    S, P = _prec(1200, 31, 3, 8, 32, precision)
    B = torch.tensor(np.random.default_rng(5).standard_normal((nrhs, S.ndof)), dtype=torch.float64, device="cuda")
    if nrhs == 1:
        B = B[0].contiguous()
    xp, zp, ip = _solve(P, B, "pair", kc)
    xo, zo, io = _solve(P, B, "one", kc)
    assert ip == io
    assert torch.equal(xp, xo) and torch.equal(zp, zo)


def test_automatic_form_in_a_large_batch_equals_alone():
    # 6 problems x 16 subdomains = 96 items: more pairs than fit at once (the batch takes one CTA per item),
    # while each problem alone (16 items) runs as pairs
    cases = [_prec(1024, 40 + i, 2, 16, 64, "fp32") for i in range(6)]
    bs = [torch.tensor(np.random.default_rng(i).standard_normal(S.ndof), dtype=torch.float64, device="cuda")
          for i, (S, _) in enumerate(cases)]
    alone = []
    for (S, P), b in zip(cases, bs):
        x = torch.zeros_like(b)
        rc, _ = P.solve(b, x, rtol=1e-8)
        assert rc == 0
        alone.append(x)
    xs = [torch.zeros_like(b) for b in bs]
    rc, _ = dg.solve_batch([P for _, P in cases], bs, xs, rtol=1e-8)
    assert rc == 0
    for a, x in zip(alone, xs):
        assert torch.equal(a, x)


def test_form_rejects_unknown_values():
    assert dg.lib().dgasm_set_local_cta_form(3) == dg.EINVAL
    assert dg.lib().dgasm_set_local_cta_form(-1) == dg.EINVAL
