"""SIPG assembly on the device (dgasm_assemble_device) against the host assembly and the oracle.

Both library paths compute the same terms with the same rules in the same order per entry; the device
contracts products into FMAs, so blocks agree to rounding: max |device - host| <= 1e-13 max |A| (the entries are
sums of a few hundred terms).  Against the oracle (scipy sparse, its own quadrature code) the bound is 1e-12
relative, as for the host assembly.  The load vector is the host's on both paths.
"""
import numpy as np
import pytest

from oracle import sipg
from synth.coeff import checker_per_subdomain
from tests.helpers import f_sin, have_gpu, mesh

pytestmark = pytest.mark.gpu

if have_gpu():
    import torch
    from paper_1903_11357_gb300 import dgasm as dg


def dense_blocks(S):
    rowptr, col, vals = S.blocks()
    return rowptr, col, vals


@pytest.mark.parametrize("n,p", [(256, 1), (300, 2), (600, 3), (200, 4), (120, 6), (64, 8)])
def test_device_blocks_match_host(n, p):
    m = mesh(n, 4)
    sub, _ = dg.Mesh.from_polymesh(m, np.ones(n)).partition(4, 0)
    M = dg.Mesh.from_polymesh(m, checker_per_subdomain(m, sub, 1e3))
    H = dg.System(M, p, 10.0, f=f_sin)
    D = dg.System(M, p, 10.0, f=f_sin, device=True)
    rh, ch, vh = dense_blocks(H)
    rd, cd, vd = dense_blocks(D)
    assert np.array_equal(rh, rd) and np.array_equal(ch, cd)
    assert np.abs(vd - vh).max() <= 1e-13 * np.abs(vh).max()
    assert np.array_equal(H.rhs(), D.rhs())


def test_device_assembly_matches_oracle():
    n, p = 150, 3
    m = mesh(n, 6)
    rho = np.random.default_rng(3).uniform(1.0, 100.0, n)
    D = dg.System(dg.Mesh.from_polymesh(m, rho), p, 10.0, f=f_sin, device=True)
    A, b, _ = sipg.assemble(m, rho, p, 10.0, f_sin)
    rowptr, col, vals = D.blocks()
    nb = (p + 1) * (p + 2) // 2
    Ad = np.zeros((n * nb, n * nb))
    for e in range(n):
        for k in range(rowptr[e], rowptr[e + 1]):
            Ad[e * nb:(e + 1) * nb, col[k] * nb:(col[k] + 1) * nb] = vals[k]
    Ao = A.toarray()
    assert np.abs(Ad - Ao).max() <= 1e-12 * np.abs(Ao).max()
    assert np.linalg.norm(D.rhs() - b) <= 1e-12 * np.linalg.norm(b)


def test_solve_on_device_assembled_system():
    m = mesh(1024, 2)
    M = dg.Mesh.from_polymesh(m, np.ones(1024))
    out = []
    for device in (False, True):
        S = dg.System(M, 3, 10.0, f=f_sin, device=device)
        P = dg.Prec(S, 4, 16, 1)
        b = torch.tensor(S.rhs(), dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        rc, st = P.solve(b, x, rtol=1e-8)
        assert rc == 0 and st[0]["true_relres"] <= 1e-8
        out.append((st[0]["iters"], x))
    assert abs(out[0][0] - out[1][0]) <= 1
    assert float(torch.linalg.norm(out[0][1] - out[1][1]) / torch.linalg.norm(out[0][1])) <= 1e-9
