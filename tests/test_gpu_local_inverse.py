"""Local solves by explicit subdomain inverses (Sec. 3, local solvers z_i = A_i^{-1} r_i): the variant for small
subdomains, selected per preconditioner (dgasm_prec_set_local_variant) or by the first solve's measurement.

Tolerances: in FP64 the inverse is formed by the same backward-stable substitutions as the sweeps, so B r agrees
with the oracle's to 1e-11 as the sweeps do (subdomain condition numbers ~4e3 at p = 2); in FP32 both variants
differ from the oracle's FP64 B r by up to about kappa * 2^-24, so the bound is 10 * kappa_max * 2^-24 with
kappa_max measured on the oracle's Jacobi-scaled subdomain matrices.  Solves: FP64 parity as for the sweeps
(equal iteration counts within one, x at the oracle's count to 1e-10)."""
import numpy as np
import pytest

from oracle import pcg
from tests.helpers import have_gpu, mesh

pytestmark = pytest.mark.gpu

if have_gpu():
    import torch
    from paper_1903_11357_gb300 import dgasm as dg
    from tests.test_gpu_parity import build_case, dev


def kappa_max_local(c):
    A, O = c["A"].tocsr(), c["O"]
    kmax = 0.0
    for idx in O.local_dofs:
        M = A[idx][:, idx].toarray()
        d = 1.0 / np.sqrt(np.diag(M))
        ev = np.linalg.eigvalsh(M * d[:, None] * d[None, :])
        kmax = max(kmax, ev[-1] / ev[0])
    return kmax


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_inverse_variant_apply_matches_oracle(precision):
    c = build_case(256, 1, 2, 4, 16, precision=precision)   # 256 cells, p = 2, 4 subdomains of ~384 dofs
    r = np.random.default_rng(3).standard_normal(c["A"].shape[0])
    ref = c["O"].apply(r)
    if precision == "fp64":
        bound = 1e-11
    else:
        bound = 10.0 * kappa_max_local(c) * 2.0 ** (-24 if precision == "fp32" else -8)
    out = {}
    for variant in ("sweeps", "inverse"):
        c["P"].set_local_variant(variant)
        assert c["P"].local_variant() == variant
        z = torch.zeros_like(dev(r))
        c["P"].apply(dev(r), z)
        torch.cuda.synchronize()
        out[variant] = z.cpu().numpy()
        assert np.linalg.norm(out[variant] - ref) <= bound * np.linalg.norm(ref), variant


def test_inverse_variant_solve_parity_fp64():
    c = build_case(256, 1, 2, 4, 16)
    c["P"].set_local_variant("inverse")
    ref = pcg.pcg(c["A"], c["b"], c["O"].apply, rtol=1e-8)
    x = torch.zeros(len(c["b"]), dtype=torch.float64, device="cuda")
    rc, st = c["P"].solve(dev(c["b"]), x, rtol=1e-8)
    assert rc == 0 and st[0]["converged"] and st[0]["true_relres"] <= 1e-8
    assert abs(st[0]["iters"] - ref.iters) <= 1
    rc, st2 = c["P"].solve(dev(c["b"]), x, fixed_iters=ref.iters)
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-10 * np.linalg.norm(ref.x)
    assert c["P"].local_variant() == "inverse"


def test_variant_tuner_picks_one_and_solves():
    c = build_case(300, 4, 2, 4, 16)
    assert c["P"].local_variant() == "tune"
    x = torch.zeros(len(c["b"]), dtype=torch.float64, device="cuda")
    rc, st = c["P"].solve(dev(c["b"]), x, rtol=1e-8)
    assert rc == 0 and st[0]["converged"] and st[0]["true_relres"] <= 1e-8
    assert c["P"].local_variant() in ("sweeps", "inverse")


def test_inverse_variant_in_a_batch_equals_alone():
    cases = [build_case(256, 1, 2, 4, 16), build_case(300, 2, 3, 4, 8), build_case(200, 3, 1, 2, 8)]
    cases[0]["P"].set_local_variant("inverse")
    cases[1]["P"].set_local_variant("sweeps")
    cases[2]["P"].set_local_variant("inverse")
    alone = []
    for c in cases:
        x = torch.zeros(len(c["b"]), dtype=torch.float64, device="cuda")
        rc, _ = c["P"].solve(dev(c["b"]), x)
        assert rc == 0
        alone.append(x)
    bs = [dev(c["b"]) for c in cases]
    xs = [torch.zeros_like(b) for b in bs]
    rc, _ = dg.solve_batch([c["P"] for c in cases], bs, xs)
    assert rc == 0
    for a, b in zip(alone, xs):
        assert torch.equal(a, b)


def test_inverse_variant_refuses_large_subdomains():
    m = mesh(600, 6)
    S = dg.System(dg.Mesh.from_polymesh(m, np.ones(600)), 3, 10.0)
    P = dg.Prec(S, 1, 0, 1)   # one subdomain of 6000 dofs
    with pytest.raises(dg.DgasmError):
        P.set_local_variant("inverse")
    P.set_local_variant("sweeps")
    assert P.local_variant() == "sweeps"
