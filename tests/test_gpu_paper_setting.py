"""The paper's experimental setting on the GPU path (Sec. 7): subdomains = fine elements, nested coarse
spaces (RCB agglomerates) at q = p, rho = 1, C_sigma = 10, rtol 1e-8 from a zero initial guess.

The same trends as the oracle's pins (tests/test_oracle_trends.py), at sizes the oracle is too slow for:
K(P_ad) about constant when N_h / N_H is fixed, and growing about 4x when N_h quadruples at fixed N_H
(the paper's Example 2 table, tests/golden/paper_example2_p1.txt; Remark 6.6's H/h dependence)."""
import numpy as np
import pytest

from synth.voronoi import voronoi_mesh
from tests.helpers import have_gpu, paper_table

pytestmark = pytest.mark.gpu

if have_gpu():
    import torch
    from paper_1903_11357_gb300 import dgasm as dg


def K_and_iters(nh, nH, p):
    m = voronoi_mesh(nh, 1)
    S = dg.System(dg.Mesh.from_polymesh(m, np.ones(nh)), p, 10.0)
    b = torch.tensor(np.random.default_rng(0).standard_normal(S.ndof), dtype=torch.float64, device="cuda")
    P = dg.Prec(S, nh, nH, p)
    x = torch.zeros_like(b)
    rc, st = P.solve(b, x, rtol=1e-8)
    assert rc == 0 and st[0]["converged"] and st[0]["true_relres"] <= 1e-8
    return st[0]["kappa"], st[0]["iters"]


def test_paper_setting_trends_p1():
    T = paper_table(2, 1)   # the paper's nested-grid table (Example 2, p = q = 1)
    k_1024_64, _ = K_and_iters(1024, 64, 1)
    k_4096_256, _ = K_and_iters(4096, 256, 1)
    k_4096_64, it_4096_64 = K_and_iters(4096, 64, 1)
    # N_h / N_H fixed (paper 83.77 / 73.42) and N_h x 4 at fixed N_H (paper 261.36 / 73.42): same ratios
    assert 1 / 1.5 <= (k_4096_256 / k_1024_64) / (T[4096, 256][0] / T[1024, 64][0]) <= 1.5
    assert 0.6 <= (k_4096_64 / k_1024_64) / (T[4096, 64][0] / T[1024, 64][0]) <= 1.6
    assert 0.5 * T[4096, 64][1] <= it_4096_64 <= 2.0 * T[4096, 64][1]   # paper: 163 iterations


def test_paper_setting_degree():
    k1, _ = K_and_iters(1024, 64, 1)
    k3, _ = K_and_iters(1024, 64, 3)
    assert 1.5 <= k3 / k1 <= 16.0                         # Example 5: sub-quadratic growth in p
