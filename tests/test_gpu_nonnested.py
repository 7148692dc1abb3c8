"""Non-nested coarse spaces on the GPU path (Eq. R0T with an independent coarse Voronoi mesh, Example 4):
parity with the oracle and the paper's trends.

Tolerances as in the nested parity tests: the preconditioner application agrees with the oracle to 1e-11
relative (the same sums of products in another order, plus the pieces below 1e-12 |kappa| that both sides
drop); FP64 solutions agree to 1e-10 at equal iteration counts, and iteration counts to +-1.
"""
import numpy as np
import pytest

from oracle import partition, pcg, schwarz, sipg
from oracle.geometry import build_geometry
from synth.voronoi import voronoi_mesh
from tests.helpers import f_sin, have_gpu, mesh, paper_table

pytestmark = pytest.mark.gpu

if have_gpu():
    import torch
    from paper_1903_11357_gb300 import dgasm as dg


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def build_case(nf, nc, p, q, nsub, seed_f=1, seed_c=21, precision="fp64"):
    fm, cm = mesh(nf, seed_f), mesh(nc, seed_c)
    M = dg.Mesh.from_polymesh(fm, np.ones(nf))
    CM = dg.Mesh.from_polymesh(cm, np.ones(nc))
    S = dg.System(M, p, 10.0, f=f_sin)
    P = dg.Prec(S, nsub, 0, q, precision=precision, coarse_mesh=CM)
    A, b, g = sipg.assemble(fm, np.ones(nf), p, 10.0, f_sin)
    osub = partition.subdomains(g.centroid, nsub)
    O = schwarz.build(A, fm, g, p, osub, None, q, coarse=(cm, build_geometry(cm)))
    return dict(S=S, P=P, A=A, b=b, O=O, CM=CM)


@pytest.mark.parametrize("nf,nc,p,q,nsub", [(300, 20, 2, 1, 4), (200, 12, 3, 3, 4), (256, 30, 1, 1, 8),
                                            (150, 40, 2, 2, 150)])
def test_apply_matches_oracle(nf, nc, p, q, nsub):
    c = build_case(nf, nc, p, q, nsub)
    assert c["P"].info()["nagg"] == nc
    r = np.random.default_rng(2).standard_normal(c["A"].shape[0])
    z = torch.zeros_like(dev(r))
    c["P"].apply(dev(r), z)
    torch.cuda.synchronize()
    ref = c["O"].apply(r)
    assert np.linalg.norm(z.cpu().numpy() - ref) <= 1e-11 * np.linalg.norm(ref)


def test_solve_parity_fp64():
    c = build_case(256, 16, 2, 1, 4)
    ref = pcg.pcg(c["A"], c["b"], c["O"].apply, rtol=1e-8)
    x = torch.zeros(len(c["b"]), dtype=torch.float64, device="cuda")
    rc, st = c["P"].solve(dev(c["b"]), x, rtol=1e-8)
    assert rc == 0 and st[0]["converged"] and st[0]["true_relres"] <= 1.1e-8
    assert abs(st[0]["iters"] - ref.iters) <= 1
    rc, st2 = c["P"].solve(dev(c["b"]), x, fixed_iters=ref.iters)
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-10 * np.linalg.norm(ref.x)
    assert st[0]["kappa"] == pytest.approx(pcg.condition_estimate(ref), rel=0.05)


def test_mixed_precision_and_batch_with_nested():
    nn32 = build_case(300, 20, 2, 1, 4, precision="fp32")
    x = torch.zeros(len(nn32["b"]), dtype=torch.float64, device="cuda")
    rc, st = nn32["P"].solve(dev(nn32["b"]), x, rtol=1e-8)
    assert rc == 0 and st[0]["true_relres"] <= 1e-8
    # a non-nested problem batched next to a nested one gives the same bits as alone
    nn = build_case(256, 16, 2, 1, 4)
    m = mesh(200, 3)
    S2 = dg.System(dg.Mesh.from_polymesh(m, np.ones(200)), 3, 10.0, f=f_sin)
    P2 = dg.Prec(S2, 2, 8, 1)
    bs = [dev(nn["b"]), dev(S2.rhs())]
    alone = []
    for P, b in zip([nn["P"], P2], bs):
        xa = torch.zeros_like(b)
        P.solve(b, xa)
        alone.append(xa)
    xs = [torch.zeros_like(b) for b in bs]
    rc, st = dg.solve_batch([nn["P"], P2], bs, xs)
    assert rc == 0
    for a, b in zip(alone, xs):
        assert torch.equal(a, b)


def K_nonnested(nh, nH, p):
    """Example 4's setting: subdomains = fine elements, an independently generated coarse Voronoi mesh,
    q = p, rho = 1, N(0, 1) right-hand side."""
    fm, cm = voronoi_mesh(nh, 1), voronoi_mesh(nH, 7)
    S = dg.System(dg.Mesh.from_polymesh(fm, np.ones(nh)), p, 10.0)
    P = dg.Prec(S, nh, 0, p, coarse_mesh=dg.Mesh.from_polymesh(cm, np.ones(nH)))
    b = torch.tensor(np.random.default_rng(0).standard_normal(S.ndof), dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    rc, st = P.solve(b, x, rtol=1e-8)
    assert rc == 0 and st[0]["converged"] and st[0]["true_relres"] <= 1e-8
    return st[0]["kappa"], st[0]["iters"]


def test_example4_trends_p1():
    T = paper_table(4, 1)   # the paper's non-nested table (Example 4, p = q = 1)
    k_1024_64, _ = K_nonnested(1024, 64, 1)
    k_4096_256, _ = K_nonnested(4096, 256, 1)
    k_4096_64, it_4096_64 = K_nonnested(4096, 64, 1)
    # N_h / N_H fixed (paper 100.89 / 106.42) and N_h x 4 at fixed N_H (paper 411.02 / 106.42): same ratios
    assert 1 / 1.5 <= (k_4096_256 / k_1024_64) / (T[4096, 256][0] / T[1024, 64][0]) <= 1.5
    assert 0.6 <= (k_4096_64 / k_1024_64) / (T[4096, 64][0] / T[1024, 64][0]) <= 1.6
    assert 0.5 * T[4096, 64][1] <= it_4096_64 <= 2.0 * T[4096, 64][1]   # paper: 167 iterations


def test_server_mixes_nested_and_nonnested_requests():
    """A non-nested request admitted next to a nested one gives the bits of its solve alone."""
    nn = build_case(256, 16, 2, 1, 4)
    m = mesh(300, 3)
    S2 = dg.System(dg.Mesh.from_polymesh(m, np.ones(300)), 3, 10.0, f=f_sin)
    b1, b2 = dev(nn["b"]), dev(S2.rhs())
    x1a = torch.zeros_like(b1)
    nn["P"].solve(b1, x1a)
    x2a = torch.zeros_like(b2)
    dg.Prec(S2, 4, 16, 1).solve(b2, x2a)
    sv = dg.Server(hbm_budget=4 << 30, max_slots=2)
    x1, x2 = torch.zeros_like(b1), torch.zeros_like(b2)
    t1 = sv.submit(nn["S"], 4, 0, 1, b1, x1, coarse_mesh=nn["CM"])
    t2 = sv.submit(S2, 4, 16, 1, b2, x2)
    for t in (t1, t2):
        rc, st = sv.wait(t, 60000)
        assert rc == 0 and all(s["converged"] for s in st)
    assert torch.equal(x1, x1a) and torch.equal(x2, x2a)
    sv.close()
