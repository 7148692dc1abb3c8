"""The TF32 and BF16 precision modes: trailing updates of the local tile Cholesky (Sec. 3, local solvers) on the
tensor cores (tcgen05; split TF32 operands, or BF16 operands split in three, FP32 accumulation).

The kernel itself is pinned against a plain float64 numpy product of the same float32 tiles.  Split TF32
(v = hi + lo, three MMAs per k-step) keeps about 21 bits of each product, and the tensor cores accumulate the
32 products of a k-loop in FP32, so an entry's error is bounded by about 32 * 2^-22 of the sum of the absolute
products; the test allows 2^-16 of (|C| + sum |products|).  A single-pass TF32 product (2^-11) or any layout
mistake fails it.  The BF16 kernel splits each FP32 entry exactly into three BF16 parts (8 bits each) and keeps
the six products down to the order 2^-16 of the part sizes, so its products carry about 23 bits: the same bound
holds, and a single BF16 pass (2^-8) or a two-part split (2^-15 with the FP32 accumulation) fails it.  The mode as a whole is checked against the library's FP64 and FP32 modes: its
preconditioner may differ from FP64's by a few times FP32's difference (at most 20 times), and its solves
reach the 1e-8 true residual within two iterations of FP32's.
"""
import numpy as np
import pytest

from synth.coeff import checker_per_subdomain
from tests.helpers import f_sin, have_gpu, mesh

pytestmark = pytest.mark.gpu

if have_gpu():
    import torch
    from paper_1903_11357_gb300 import dgasm as dg


def lower_tiles(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(((n + 1) * (n + 2) // 2, 32, 32)).astype(np.float32)


def tid(I, J):
    return I * (I + 1) // 2 + J


@pytest.mark.parametrize("kind", ["tf32", "bf16"])
@pytest.mark.parametrize("n", [1, 4, 5, 9, 13])
def test_tc_update_matches_float64_product(n, kind):
    t = lower_tiles(n, 100 + n)
    out = dg.selftest_tc_update(t, kind=kind)
    for I in range(n + 1):
        for J in range(I + 1):
            k = tid(I, J)
            if J == 0:   # the panel and the diagonal tile of step 0 are read, not written
                assert np.array_equal(out[k], t[k])
                continue
            a = t[tid(I, 0)].astype(np.float64)
            b = t[tid(J, 0)].astype(np.float64)
            ref = t[k].astype(np.float64) - a @ b.T
            scale = np.abs(t[k]).astype(np.float64) + np.abs(a) @ np.abs(b).T
            err = np.abs(out[k].astype(np.float64) - ref)
            assert (err <= 2.0 ** -16 * scale).all(), (I, J, float((err / scale).max()))


def test_tc_update_rejects_bad_arguments():
    with pytest.raises(ValueError):
        dg.selftest_tc_update(np.zeros((4, 32, 32), np.float32))   # not a triangular count


def _case(precision, contrast=1e4):
    m = mesh(1024, 3)
    sub, _ = dg.Mesh.from_polymesh(m, np.ones(1024)).partition(4, 0)
    S = dg.System(dg.Mesh.from_polymesh(m, checker_per_subdomain(m, sub, contrast)), 3, 10.0, f=f_sin)
    return S, dg.Prec(S, 4, 16, 1, precision=precision)


def test_tf32_mode_apply_and_solve_track_fp32():
    """256-element subdomains (the bench's size): panels of up to ~10 tiles, so the update blocks include
    row blocks past the first and column blocks past the eighth tile."""
    r = None
    z = {}
    res = {}
    for prec in ("fp64", "fp32", "tf32"):
        S, P = _case(prec)
        b = torch.tensor(S.rhs(), dtype=torch.float64, device="cuda")
        if r is None:
            r = torch.tensor(np.random.default_rng(5).standard_normal(len(b)), dtype=torch.float64, device="cuda")
        zz = torch.zeros_like(r)
        P.apply(r, zz)
        x = torch.zeros_like(b)
        rc, st = P.solve(b, x, rtol=1e-8)
        torch.cuda.synchronize()
        z[prec] = zz.cpu().numpy()
        res[prec] = (rc, st[0], x.cpu().numpy())
    e32 = np.linalg.norm(z["fp32"] - z["fp64"]) / np.linalg.norm(z["fp64"])
    etc = np.linalg.norm(z["tf32"] - z["fp64"]) / np.linalg.norm(z["fp64"])
    # FP32 factors already differ from FP64 by ~1e-4 here (ill-conditioned subdomain matrices); split TF32
    # keeps ~21 bits per product against FP32's 24, so its error may be a few times FP32's, not more
    print(f"apply rel. error vs FP64: fp32 {e32:.3e} tf32 {etc:.3e}; iterations fp64 {res['fp64'][1]['iters']} "
          f"fp32 {res['fp32'][1]['iters']} tf32 {res['tf32'][1]['iters']}")
    assert etc <= 20 * e32 + 1e-12 and etc <= 1e-2, (etc, e32)
    rc, st, x = res["tf32"]
    assert rc == 0 and st["converged"] and st["true_relres"] <= 1e-8
    assert abs(st["iters"] - res["fp32"][1]["iters"]) <= 2
    x64 = res["fp64"][2]
    assert np.linalg.norm(x - x64) <= 1e-6 * np.linalg.norm(x64)


def test_bf16_mode_factorises_on_the_tensor_cores_and_solves():
    """BF16 mode: the trailing updates on the tensor cores with BF16 operands (three-part split), the solve
    streams in BF16; the outer FP64 PCG reaches the 1e-8 true residual within 10 % of FP32's iterations and its
    solution agrees with FP64's to 1e-6."""
    res = {}
    for prec in ("fp64", "fp32", "bf16"):
        S, P = _case(prec)   # P of the last mode (bf16) is kept
        b = torch.tensor(S.rhs(), dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        rc, st = P.solve(b, x, rtol=1e-8)
        torch.cuda.synchronize()
        res[prec] = (rc, st[0], x.cpu().numpy())
    rc, st, x = res["bf16"]
    assert rc == 0 and st["converged"] and st["true_relres"] <= 1e-8
    assert P.info()["tc_fallback"] == 0   # the tensor-core factorisation held
    assert st["iters"] <= 1.1 * res["fp32"][1]["iters"] + 1
    x64 = res["fp64"][2]
    assert np.linalg.norm(x - x64) <= 1e-6 * np.linalg.norm(x64)
