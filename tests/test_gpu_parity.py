"""GPU parity: the CUDA path (through the C-ABI) against the CPU oracle on the same seeded inputs.

Tolerances: FP64 mode solutions agree with the oracle to a relative L2 difference of 1e-10 when both
run the same number of iterations, and iteration counts under the 1e-8 stop test agree within +-1.
Operator-level checks (SpMV, preconditioner application) agree to 1e-12 relative: both sides compute
the same sums of products of the same FP64 numbers in different orders.
"""
import numpy as np
import pytest

from oracle import partition, pcg, schwarz, sipg
from oracle.geometry import build_geometry
from synth.coeff import checker_per_subdomain
from tests.helpers import f_sin, have_gpu, mesh

pytestmark = pytest.mark.gpu

if have_gpu():
    import torch
    from paper_1903_11357_gb300 import dgasm as dg


def build_case(n, seed, p, nsub, ncoarse, q=1, contrast=1.0, precision="fp64"):
    m = mesh(n, seed)
    M0 = dg.Mesh.from_polymesh(m, np.ones(n))
    sub, _ = M0.partition(nsub, 0)
    rho = checker_per_subdomain(m, sub, contrast) if contrast != 1.0 else np.ones(n)
    M = dg.Mesh.from_polymesh(m, rho)
    S = dg.System(M, p, 10.0, f=f_sin)
    P = dg.Prec(S, nsub, ncoarse, q, precision=precision)
    A, b, g = sipg.assemble(m, rho, p, 10.0, f_sin)
    osub = partition.subdomains(g.centroid, nsub)
    oagg = partition.agglomerates(g.centroid, osub, nsub, ncoarse) if ncoarse else None
    O = schwarz.build(A, m, g, p, osub, oagg, q)
    return dict(m=m, M=M, S=S, P=P, A=A, b=b, O=O, rho=rho)


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("n,p", [(256, 2), (600, 3)])
def test_spmv_matches_oracle(n, p):
    c = build_case(n, 3, p, 4, 0)
    x = np.random.default_rng(0).standard_normal(c["A"].shape[0])
    y = torch.zeros_like(dev(x))
    c["S"].spmv(dev(x), y)
    torch.cuda.synchronize()
    ref = c["A"] @ x
    assert np.abs(y.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("n,p,nsub,ncoarse,q", [(256, 2, 4, 16, 1), (600, 3, 8, 32, 1), (300, 2, 5, 0, 1),
                                                 (400, 3, 4, 16, 2), (150, 1, 1, 0, 1)])
def test_preconditioner_apply_matches_oracle(n, p, nsub, ncoarse, q):
    c = build_case(n, 7, p, nsub, ncoarse, q)
    r = np.random.default_rng(1).standard_normal(c["A"].shape[0])
    z = torch.zeros_like(dev(r))
    c["P"].apply(dev(r), z)
    torch.cuda.synchronize()
    ref = c["O"].apply(r)
    assert np.linalg.norm(z.cpu().numpy() - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("n,p,ncoarse,q", [(256, 2, 16, 1), (200, 3, 8, 2), (120, 1, 0, 1)])
def test_element_blocks_apply_matches_oracle(n, p, ncoarse, q):
    """Subdomains = elements (the setting of the paper's experiments): explicit inverses of the
    diagonal blocks instead of envelope factors."""
    c = build_case(n, 5, p, n, ncoarse, q)
    assert c["P"].info()["stream_tiles"] == 0
    r = np.random.default_rng(2).standard_normal(c["A"].shape[0])
    z = torch.zeros_like(dev(r))
    c["P"].apply(dev(r), z)
    torch.cuda.synchronize()
    ref = c["O"].apply(r)
    assert np.linalg.norm(z.cpu().numpy() - ref) <= 1e-11 * np.linalg.norm(ref)


def test_element_blocks_solve_parity():
    c = build_case(256, 1, 2, 256, 16)
    ref = pcg.pcg(c["A"], c["b"], c["O"].apply, rtol=1e-8)
    x = torch.zeros(len(c["b"]), dtype=torch.float64, device="cuda")
    rc, st = c["P"].solve(dev(c["b"]), x, rtol=1e-8)
    assert rc == 0 and st[0]["converged"] and abs(st[0]["iters"] - ref.iters) <= 1
    assert st[0]["true_relres"] <= 1e-8
    rc, st2 = c["P"].solve(dev(c["b"]), x, fixed_iters=ref.iters)
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-10 * np.linalg.norm(ref.x)
    assert st[0]["kappa"] == pytest.approx(pcg.condition_estimate(ref), rel=0.05)
    # two right-hand sides through the same block inverses
    B = np.random.default_rng(3).standard_normal((2, len(c["b"])))
    X = torch.zeros(2, len(c["b"]), dtype=torch.float64, device="cuda")
    rc, stm = c["P"].solve(dev(B), X, rtol=1e-8)
    assert rc == 0
    for j in range(2):
        xs = np.linalg.solve(c["A"].toarray(), B[j])
        assert np.linalg.norm(X[j].cpu().numpy() - xs) <= 1e-6 * np.linalg.norm(xs)


def test_partition_used_matches_oracle():
    c = build_case(256, 1, 2, 4, 16)
    sub, agg = c["P"].partition()
    g = build_geometry(c["m"])
    osub = partition.subdomains(g.centroid, 4)
    assert np.array_equal(sub, osub)
    assert np.array_equal(agg, partition.agglomerates(g.centroid, osub, 4, 16))


@pytest.mark.parametrize("contrast", [1.0, 1e4])
def test_cfg1_solve_parity_fp64(contrast):
    """256 Voronoi cells, p = 2, 4 RCB subdomains, 16 agglomerates at q = 1 (the small configuration)."""
    c = build_case(256, 1, 2, 4, 16, 1, contrast)
    ref = pcg.pcg(c["A"], c["b"], c["O"].apply, rtol=1e-8)
    x = torch.zeros(len(c["b"]), dtype=torch.float64, device="cuda")
    rc, st = c["P"].solve(dev(c["b"]), x, rtol=1e-8)
    assert rc == 0 and st[0]["converged"]
    assert abs(st[0]["iters"] - ref.iters) <= 1
    assert st[0]["true_relres"] <= 1.1e-8
    # equal iteration counts: solutions agree to 1e-10
    rc, st2 = c["P"].solve(dev(c["b"]), x, fixed_iters=ref.iters)
    xr = x.cpu().numpy()
    assert np.linalg.norm(xr - ref.x) <= 1e-10 * np.linalg.norm(ref.x)
    assert st2[0]["iters"] == ref.iters
    K = pcg.condition_estimate(ref)
    assert st[0]["kappa"] == pytest.approx(K, rel=0.05)


def test_multi_rhs_equals_single():
    """Several right-hand sides share one pass over the factors; the local solve groups its accumulation
    chains per right-hand-side count, so results agree with one-at-a-time solves to rounding."""
    c = build_case(300, 4, 2, 4, 16)
    rng = np.random.default_rng(5)
    B = rng.standard_normal((3, len(c["b"])))
    X = torch.zeros(3, len(c["b"]), dtype=torch.float64, device="cuda")
    rc, st = c["P"].solve(dev(B), X, rtol=1e-8)
    assert rc == 0 and len(st) == 3
    for j in range(3):
        x1 = torch.zeros(len(c["b"]), dtype=torch.float64, device="cuda")
        rc1, st1 = c["P"].solve(dev(B[j]), x1, rtol=1e-8)
        assert abs(st1[0]["iters"] - st[j]["iters"]) <= 1
        assert float(torch.linalg.norm(x1 - X[j])) <= 1e-9 * float(torch.linalg.norm(x1))


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_mixed_precision_reaches_tolerance(precision):
    c = build_case(256, 1, 2, 4, 16, 1, 1e4, precision=precision)
    x = torch.zeros(len(c["b"]), dtype=torch.float64, device="cuda")
    rc, st = c["P"].solve(dev(c["b"]), x, rtol=1e-8)
    assert rc == 0 and st[0]["converged"] and st[0]["true_relres"] <= 1e-8
    xs = np.linalg.solve(c["A"].toarray(), c["b"])
    assert np.linalg.norm(x.cpu().numpy() - xs) <= 1e-6 * np.linalg.norm(xs)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_true_residual_meets_tolerance_high_contrast(precision):
    # p = 4 and contrast 1e6: the recursive residual drifts from b - A x; the solve restarts from the
    # true residual until both meet rtol
    m = mesh(1024, 3)
    sub, _ = dg.Mesh.from_polymesh(m, np.ones(1024)).partition(16, 0)
    S = dg.System(dg.Mesh.from_polymesh(m, checker_per_subdomain(m, sub, 1e6)), 4, 10.0, f=f_sin)
    P = dg.Prec(S, 16, 64, 1, precision=precision)
    b = dev(S.rhs())
    x = torch.zeros_like(b)
    rc, st = P.solve(b, x, rtol=1e-8)
    assert rc == 0 and st[0]["converged"] and st[0]["true_relres"] <= 1e-8 and st[0]["relres"] <= 1e-8
    assert 0.0 < st[0]["kappa"] < 1e6


def test_initial_guess():
    c = build_case(256, 1, 2, 4, 16, 1, 1e4)
    b = dev(c["b"])
    x = torch.zeros_like(b)
    rc, st = c["P"].solve(b, x)
    assert rc == 0
    # from the converged solution: nothing to do, x comes back unchanged
    x2 = x.clone()
    rc, st2 = c["P"].solve(b, x2, x0_given=True)
    assert rc == 0 and st2[0]["iters"] == 0 and torch.equal(x2, x)
    # from a perturbed guess: the same solution, fewer iterations than from zero
    g = torch.Generator(device="cpu").manual_seed(7)
    x3 = x + 1e-4 * torch.randn(x.shape, generator=g, dtype=torch.float64).cuda()
    rc, st3 = c["P"].solve(b, x3, x0_given=True)
    assert rc == 0 and st3[0]["true_relres"] <= 1e-8 and st3[0]["iters"] <= st[0]["iters"]
    assert float(torch.linalg.norm(x3 - x)) <= 1e-6 * float(torch.linalg.norm(x))
    # a zero right-hand side gives zero whatever the guess
    x4 = torch.ones_like(x)
    rc, st4 = c["P"].solve(torch.zeros_like(b), x4, x0_given=True)
    assert rc == 0 and float(x4.abs().max()) == 0.0


def test_zero_rhs_and_one_subdomain():
    c = build_case(200, 2, 2, 1, 0)
    x = torch.ones(len(c["b"]), dtype=torch.float64, device="cuda")
    rc, st = c["P"].solve(torch.zeros_like(x), x)
    assert rc == 0 and st[0]["iters"] == 0 and float(x.abs().max()) == 0.0
    rc, st = c["P"].solve(dev(c["b"]), x)
    assert st[0]["iters"] == 1 and st[0]["true_relres"] < 1e-10


def test_batch_equals_alone():
    # the third problem runs with subdomains = elements (block inverses) next to two envelope problems
    cases = [build_case(256, 1, 2, 4, 16), build_case(300, 2, 3, 4, 8), build_case(200, 3, 1, 2, 8),
             build_case(180, 4, 2, 180, 12)]
    xs_alone = []
    for c in cases:
        x = torch.zeros(len(c["b"]), dtype=torch.float64, device="cuda")
        c["P"].solve(dev(c["b"]), x)
        xs_alone.append(x)
    bs = [dev(c["b"]) for c in cases]
    xs = [torch.zeros_like(b) for b in bs]
    rc, st = dg.solve_batch([c["P"] for c in cases], bs, xs)
    assert rc == 0
    for a, b in zip(xs_alone, xs):
        assert torch.equal(a, b)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_eight_right_hand_sides_equal_single_solves(precision):
    """The widest right-hand-side block (8 vectors, more than the persistent vector kernel's warps per CTA):
    every column takes the same iterations and reaches the same solution as its own single-vector solve
    (the same products in the same order; 1e-13 leaves room only for contraction differences)."""
    c = build_case(600, 5, 2, 4, 16, precision=precision)
    B = np.random.default_rng(9).standard_normal((8, len(c["b"])))
    X = torch.zeros_like(dev(B))
    rc, st = c["P"].solve(dev(B), X, rtol=1e-8)
    assert rc == 0 and all(s["converged"] for s in st)
    for j in range(8):
        x = torch.zeros(len(c["b"]), dtype=torch.float64, device="cuda")
        rc1, st1 = c["P"].solve(dev(B[j]), x, rtol=1e-8)
        assert rc1 == 0 and st1[0]["iters"] == st[j]["iters"], (j, st1[0]["iters"], st[j]["iters"])
        assert float(torch.linalg.norm(X[j] - x) / torch.linalg.norm(x)) <= 1e-13


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_rhs_chunk_choices_give_identical_solutions(precision):
    """1 or 4 right-hand sides per local-solve item: the same products in the same order for every vector,
    so the tuner's (timing-dependent) choice cannot change a solution."""
    c = build_case(300, 4, 2, 4, 16, precision=precision)
    B = dev(np.random.default_rng(8).standard_normal((3, len(c["b"]))))
    out = {}
    for kc in (1, 4):
        c["P"].set_rhs_chunk(3, kc)
        X = torch.zeros_like(B)
        rc, st = c["P"].solve(B, X, rtol=1e-8)
        assert rc == 0
        out[kc] = (X, [s["iters"] for s in st])
    assert torch.equal(out[1][0], out[4][0]) and out[1][1] == out[4][1]
    c["P"].set_rhs_chunk(3, 0)
    assert c["P"].rhs_chunk(3) == 0
    X = torch.zeros_like(B)
    rc, st = c["P"].solve(B, X, rtol=1e-8)
    assert rc == 0 and c["P"].rhs_chunk(3) in (1, 4)
    assert torch.equal(X, out[1][0])


@pytest.mark.parametrize("variant", ["sweeps", "inverse"])
@pytest.mark.parametrize("n,p,nsub,ncoarse,q", [(64, 8, 2, 4, 1), (80, 6, 4, 8, 2)])
def test_high_degree_apply_and_solve_match_oracle(n, p, nsub, ncoarse, q, variant):
    """The largest blocks the library takes (p = 8: 45 dofs per element, the widest SpMV and envelope rows).
    Two backward-stable Cholesky factorisations of the same matrix differ by up to about kappa * 2^-53 relative,
    and at p = 8 the Jacobi-scaled subdomain matrices reach kappa ~ 1e8 (p = 3: ~4e3), so the apply bound is
    10 * kappa_max * 2^-53 with kappa_max measured here on the oracle's local and coarse matrices.

    Solves (Sec. 7 stop test): at the oracle's iteration count k_o the two iterates agree to 1e-10 (8.8e-10 seen
    at p = 8 comes from the same kappa amplification, so the bound there is the apply bound times 10).  Near
    the tolerance the residual history can stay within rounding of rtol for several iterations (p = 6 here: the
    oracle's 1.18, 1.07, 1.15, 1.07, 0.91 e-8 at iterations 203-207), and two FP64 recursions whose iterates
    agree to that bound then stop a few iterations apart: at p = 8 ||A|| ||x|| / ||b|| is large enough that the
    residual norms differ by up to about half of rtol.  So the library's stopping iteration k_g and the
    oracle's k_o are compared through the residuals both recursions carry, at every iteration k from
    min(k_g, k_o) - 1 to max(k_g, k_o): eta_k = | ||r_k|| - ||r_k^oracle|| | / ||b|| must be explained by the
    iterates' difference, eta_k <= (||A (x_k - x_k^oracle)|| + gap_k + gap_k^oracle) / ||b|| (triangle inequality;
    gap = || r_k - (b - A x_k) ||, the drift of each recursion from its true residual), and each stop must be a
    stop of the other history up to eta = max eta_k (the oracle's residual at k_g and the library's at k_o are
    <= rtol + eta).  Both local-solve variants (sweeps and explicit inverses) are checked."""
    c = build_case(n, 2, p, nsub, ncoarse, q)
    c["P"].set_local_variant(variant)
    A, O = c["A"].tocsr(), c["O"]
    kmax = 0.0
    for M in [A[idx][:, idx].toarray() for idx in O.local_dofs] + [O.A0]:
        d = 1.0 / np.sqrt(np.diag(M))
        ev = np.linalg.eigvalsh(M * d[:, None] * d[None, :])
        kmax = max(kmax, ev[-1] / ev[0])
    apply_bound = 10.0 * kmax * 2.0 ** -53
    r = np.random.default_rng(4).standard_normal(A.shape[0])
    z = torch.zeros_like(dev(r))
    c["P"].apply(dev(r), z)
    torch.cuda.synchronize()
    ref = O.apply(r)
    assert np.linalg.norm(z.cpu().numpy() - ref) <= apply_bound * np.linalg.norm(ref)
    b = c["b"]
    oref = pcg.pcg(A, b, O.apply, rtol=1e-8)
    ko = oref.iters
    xk = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    c["P"].solve(dev(b), xk, fixed_iters=ko)
    xk = xk.cpu().numpy()
    assert np.linalg.norm(xk - oref.x) <= max(1e-10, 10.0 * apply_bound) * np.linalg.norm(oref.x)
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    rc, st = c["P"].solve(dev(b), x, rtol=1e-8)
    assert rc == 0 and st[0]["converged"] and st[0]["true_relres"] <= 1e-8
    kg = st[0]["iters"]
    bn = np.linalg.norm(b)
    etas = []
    rel_g, rel_o = {}, {}
    for k in range(min(kg, ko) - 1, max(kg, ko) + 1):
        xf = torch.zeros(len(b), dtype=torch.float64, device="cuda")
        _, sf = c["P"].solve(dev(b), xf, fixed_iters=k)
        xg = xf.cpu().numpy()
        ok = pcg.pcg(A, b, O.apply, fixed_iters=k)
        rel_g[k], rel_o[k] = sf[0]["relres"], ok.resid[-1]
        gap_g = abs(rel_g[k] - np.linalg.norm(b - A @ xg) / bn)
        gap_o = abs(rel_o[k] - np.linalg.norm(b - A @ ok.x) / bn)
        eta_k = abs(rel_g[k] - rel_o[k])
        assert eta_k <= 1.01 * (np.linalg.norm(A @ (xg - ok.x)) / bn + gap_g + gap_o), k
        etas.append(eta_k)
    eta = max(etas)
    assert rel_o[kg] <= 1e-8 + eta and rel_g[ko] <= 1e-8 + eta, (kg, ko, eta)
