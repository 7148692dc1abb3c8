"""Host-side checks of libdgasm.so (no GPU): it loads, exports every entry point of include/dgasm.h, answers
NULL arguments with DGASM_EINVAL, validates meshes, and its partition, SIPG assembly and non-nested R_0^T agree
with the oracle."""
import ctypes

import numpy as np
import pytest

from oracle import partition, pcg, sipg
from paper_1903_11357_gb300 import dgasm as dg
from synth.coeff import checker_per_subdomain
from synth.voronoi import PolyMesh, quad_mesh
from tests.helpers import f_sin, mesh


def test_library_loads_and_exports_header_symbols():
    L = dg.lib()
    names = dg.exported_symbols()
    assert "dgasm_solve" in names and "dgasm_setup" in names and "dgasm_submit" in names
    for n in names:
        assert hasattr(L, n), n


# every entry point with NULL handles and buffers: an argument check answers before any CUDA call
NULL_CALLS = {
    "dgasm_setup": (None, None, None),
    "dgasm_setup_batch": (0, None, None, None),
    "dgasm_prec_apply": (None, 1, None, None, None),
    "dgasm_prec_set_rhs_chunk": (None, 1, 1),
    "dgasm_prec_get_rhs_chunk": (None, 1, None),
    "dgasm_prec_partition": (None, None, None),
    "dgasm_prec_footprint": (None, None),
    "dgasm_prec_info": (None, None),
    "dgasm_solve": (None, 1, None, None, None, None),
    "dgasm_solve_batch": (0, None, None, None, None, None, None),
    "dgasm_system_spmv": (None, None, None, None),
    "dgasm_system_spmv_dot_noalloc": (None, None, None, None, None),
    "dgasm_system_dofs": (None, None, None),
    "dgasm_system_rhs": (None, None),
    "dgasm_system_blocks": (None, None, None, None, None),
    "dgasm_mesh_info": (None, None, None, None),
    "dgasm_mesh_centroids": (None, None),
    "dgasm_partition": (None, 4, 0, None, None),
    "dgasm_submit": (None, None, None, 1, None, None, None, None),
    "dgasm_poll": (None, 0, None),
    "dgasm_wait": (None, 0, 0, None),
    "dgasm_cancel": (None, 0),
    "dgasm_server_stats": (None, None, None, None, None),
    "dgasm_nonnested_prolongation": (None, None, 1, 1, None, None, None, None),
    "dgasm_selftest_plan": (None, 4, None, None),
    "dgasm_selftest_tc_update": (0, None, None),
    "dgasm_lanczos": (0, None, None, None, None),
}


def test_every_entry_rejects_null_arguments():
    """Each entry point answers NULL handles or buffers with DGASM_EINVAL and a message naming the problem, and
    each destroy accepts NULL; none of these calls reaches the GPU."""
    L = dg.lib()
    buf = ctypes.create_string_buffer(512)
    calls = dict(NULL_CALLS)
    calls["dgasm_assemble"] = (None, 3, 10.0, dg.RHS_FN(), None, None)
    calls["dgasm_assemble_device"] = (None, 3, 10.0, dg.RHS_FN(), None, None, None)
    for name, args in calls.items():
        assert getattr(L, name)(*args) == dg.EINVAL, name
        L.dgasm_last_error(buf, 512)
        assert buf.value, name
    L.dgasm_last_error(buf, 512)
    assert buf.value.startswith(b"dgasm_assemble_device")
    for name in ("dgasm_prec_destroy", "dgasm_system_destroy", "dgasm_mesh_destroy", "dgasm_server_destroy"):
        assert getattr(L, name)(None) == dg.OK, name


def test_binding_refuses_mismatched_vector_shapes():
    """The library reads and writes k * ndof doubles through each vector pointer, so the binding checks shapes
    before any call: a wrong length, different vector counts or a wrong host dtype never reach the library."""
    import torch
    assert dg._nvec(10, torch.zeros(10), torch.zeros(10)) == 1
    assert dg._nvec(10, torch.zeros(3, 10), torch.zeros(3, 10)) == 3
    for a, b in [(torch.zeros(9), torch.zeros(10)), (torch.zeros(2, 10), torch.zeros(3, 10)),
                 (torch.zeros(10, 2), torch.zeros(10, 2)), (torch.zeros(2, 2, 10), torch.zeros(2, 2, 10))]:
        with pytest.raises(ValueError):
            dg._nvec(10, a, b)
    P = dg.Prec.__new__(dg.Prec)   # no device: only the checks in front of the call run
    P.ndof, P.h = 10, None
    with pytest.raises(ValueError):
        P.solve(np.zeros(9), np.zeros(10), host_buffers=True)
    with pytest.raises(TypeError):
        P.solve(np.zeros(10, np.float32), np.zeros(10), host_buffers=True)
    with pytest.raises(dg.DgasmError) as e:   # shapes agree: the library refuses the NULL handle
        P.solve(np.zeros(10), np.zeros(10), host_buffers=True)
    assert e.value.code == dg.EINVAL


def test_mesh_validation_errors():
    sq = quad_mesh(1)
    with pytest.raises(dg.DgasmError) as e:
        dg.Mesh(sq.xy, sq.poly_ptr, sq.poly_vtx[::-1].copy(), [1.0])
    assert e.value.code == dg.EINVAL and "area" in str(e.value)
    with pytest.raises(dg.DgasmError):
        dg.Mesh(sq.xy, sq.poly_ptr, sq.poly_vtx, [0.0])
    with pytest.raises(dg.DgasmError):
        dg.Mesh(sq.xy, sq.poly_ptr, np.array([0, 1, 3, 7], np.int32), [1.0])
    bad = PolyMesh(xy=np.array([[0, 0], [1, 0], [0, 1.0]]), poly_ptr=np.array([0, 2], np.int32),
                   poly_vtx=np.array([0, 1], np.int32))
    with pytest.raises(dg.DgasmError):
        dg.Mesh(bad.xy, bad.poly_ptr, bad.poly_vtx, [1.0])


def test_faces_counted():
    m = mesh(200, 3)
    M = dg.Mesh.from_polymesh(m, np.ones(200))
    ne, nfi, nfb = M.info()
    from oracle.geometry import build_geometry
    g = build_geometry(m)
    assert ne == 200 and nfi == sum(1 for f in g.faces if f[1] >= 0) and nfb == sum(1 for f in g.faces if f[1] < 0)


@pytest.mark.parametrize("n,nsub,ncoarse", [(256, 4, 16), (300, 7, 20), (500, 16, 5), (1024, 4, 64), (64, 64, 8)])
def test_partition_matches_oracle(n, nsub, ncoarse):
    m = mesh(n, n)
    M = dg.Mesh.from_polymesh(m, np.ones(n))
    sub, agg = M.partition(nsub, ncoarse)
    from oracle.geometry import build_geometry
    g = build_geometry(m)
    assert np.array_equal(M.centroids(), g.centroid)
    osub = partition.subdomains(g.centroid, nsub)
    assert np.array_equal(sub, osub)
    assert np.array_equal(agg, partition.agglomerates(g.centroid, osub, nsub, ncoarse))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_assembly_matches_oracle(p):
    m = mesh(96, 5)
    sub, _ = dg.Mesh.from_polymesh(m, np.ones(96)).partition(6, 0)
    rho = checker_per_subdomain(m, sub, 1e4)
    M = dg.Mesh.from_polymesh(m, rho)
    S = dg.System(M, p, 10.0, f=f_sin)
    A, b, _ = sipg.assemble(m, rho, p, 10.0, f_sin)
    rowptr, col, vals = S.blocks()
    npb = S.np
    Ad = A.toarray()
    L = np.zeros_like(Ad)
    for e in range(96):
        for k in range(rowptr[e], rowptr[e + 1]):
            L[e * npb:(e + 1) * npb, col[k] * npb:(col[k] + 1) * npb] = vals[k]
    assert np.abs(L - Ad).max() <= 1e-13 * np.abs(Ad).max()
    assert np.abs(S.rhs() - b).max() <= 1e-13 * np.abs(b).max()


def test_assemble_rejects_bad_degree():
    m = mesh(16, 1)
    M = dg.Mesh.from_polymesh(m, np.ones(16))
    with pytest.raises(dg.DgasmError):
        dg.System(M, 0)
    with pytest.raises(dg.DgasmError):
        dg.System(M, 9)


def test_lanczos_matches_oracle():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((30, 30))
    A = A @ A.T + 30 * np.eye(30)
    res = pcg.pcg(A, rng.standard_normal(30), lambda r: r.copy(), rtol=1e-12)
    lo_o, hi_o = pcg.lanczos_extremes(res.alphas, res.betas[:len(res.alphas) - 1])
    lo, hi = dg.lanczos(res.alphas, res.betas[:len(res.alphas) - 1])
    assert lo == pytest.approx(lo_o, rel=1e-10) and hi == pytest.approx(hi_o, rel=1e-10)


def test_last_error_roundtrip():
    buf = ctypes.create_string_buffer(64)
    dg.lib().dgasm_partition(None, 1, 0, None, None)
    assert dg.lib().dgasm_last_error(buf, 64) == dg.EINVAL
    assert b"NULL" in buf.value


@pytest.mark.parametrize("nf,nc,p,q", [(300, 20, 2, 1), (200, 12, 3, 3), (150, 40, 2, 2)])
def test_nonnested_prolongation_matches_oracle(nf, nc, p, q):
    """The library's host R_0^T of a non-nested coarse mesh (the blocks dgasm_setup uploads) against the
    oracle's, computed independently from Eq. R0T."""
    from oracle import schwarz
    from oracle.basis import n_basis
    from oracle.geometry import build_geometry
    fm, cm = mesh(nf, 1), mesh(nc, 21)
    F = dg.Mesh.from_polymesh(fm, np.ones(nf))
    Cm = dg.Mesh.from_polymesh(cm, np.ones(nc))
    ptr, col, blk = dg.nonnested_prolongation(F, Cm, p, q)
    nb, nq = n_basis(p), n_basis(q)
    L = np.zeros((nf * nb, nc * nq))
    for e in range(nf):
        assert np.all(np.diff(col[ptr[e]:ptr[e + 1]]) > 0)   # ascending coarse cells
        for t in range(ptr[e], ptr[e + 1]):
            L[e * nb:(e + 1) * nb, col[t] * nq:(col[t] + 1) * nq] = blk[t]
    O = schwarz.prolongation_nonnested(fm, build_geometry(fm), cm, build_geometry(cm), p, q).toarray()
    assert np.abs(L - O).max() <= 1e-12 * np.abs(O).max()
    with pytest.raises(dg.DgasmError):
        dg.nonnested_prolongation(F, Cm, 2, 3)   # q > p


@pytest.mark.parametrize("n,p,nsub", [(256, 2, 4), (600, 3, 8), (400, 4, 2), (300, 1, 16), (200, 3, 1)])
def test_plan_self_check(n, p, nsub):
    """Tensor-core update groups cover the Cholesky update tasks, and the solve streams and run tables
    match the tile envelope, on subdomains of 1 to 32 tile rows."""
    S = dg.System(dg.Mesh.from_polymesh(mesh(n, 5), np.ones(n)), p, 10.0)
    violations, checks = dg.selftest_plan(S, nsub)
    assert violations == 0 and checks > 0


def test_nonnested_prolongation_rejects_a_non_convex_coarse_cell():
    fm = mesh(60, 1)
    F = dg.Mesh.from_polymesh(fm, np.ones(60))
    # two cells of the unit square: an L-shaped (non-convex) cell and the square that completes it
    xy = np.array([[0, 0], [1, 0], [1, 0.5], [0.5, 0.5], [0.5, 1], [0, 1], [1, 1]], float)
    cm = PolyMesh(xy=xy, poly_ptr=np.array([0, 6, 10], np.int32),
                  poly_vtx=np.array([0, 1, 2, 3, 4, 5, 3, 2, 6, 4], np.int32))
    Cm = dg.Mesh.from_polymesh(cm, np.ones(2))
    with pytest.raises(dg.DgasmError, match="not convex"):
        dg.nonnested_prolongation(F, Cm, 2, 1)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without libdgasm.so every call raises instead of computing anything."""
    monkeypatch.setattr(dg, "_lib", None)
    monkeypatch.setattr(dg, "LIB_PATH", str(tmp_path / "libdgasm.so"))
    with pytest.raises(RuntimeError, match="missing"):
        dg.lib()
    with pytest.raises(RuntimeError, match="missing"):
        dg.Mesh.from_polymesh(mesh(32, 1), np.ones(32))


def test_partitions_and_plans_from_concurrent_threads_match_serial():
    """The host plan's loops run on one shared worker pool: partitions computed from several threads at once
    (ctypes releases the interpreter lock during each call) equal the serial ones, and plans built
    concurrently pass their self-check."""
    import threading
    n = 3000
    m = mesh(n, 11)
    M = dg.Mesh.from_polymesh(m, np.ones(n))
    cases = [(64, 256), (16, 64), (7, 30), (5, 3)]
    ref = {c: M.partition(*c) for c in cases}
    S = dg.System(M, 2, 10.0)
    got, checks, errors = {}, {}, []

    def work(i):
        try:
            c = cases[i % len(cases)]
            for _ in range(3):
                got[(i, c)] = M.partition(*c)
            checks[i] = dg.selftest_plan(S, c[0])
        except Exception as e:   # reported below
            errors.append(repr(e))

    th = [threading.Thread(target=work, args=(i,)) for i in range(8)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    for (i, c), (sub, agg) in got.items():
        assert np.array_equal(sub, ref[c][0]) and np.array_equal(agg, ref[c][1]), (i, c)
    assert all(v == 0 and k > 0 for v, k in checks.values()), checks


def test_no_unordered_legacy_stream_writes_in_library_sources():
    """The library's kernels run on non-blocking streams, which the legacy default stream does not order with.
    A plain cudaMemset, or a cudaMemcpy from the host, is queued on that legacy stream and can land after kernels
    issued later on another stream.  Two such gaps were found (the upload of plan arrays, the clear of a new
    Krylov workspace); this scan keeps new ones out: every plain cudaMemset or host-to-device cudaMemcpy in the
    sources must sit in a function listed here, each of which orders it (a legacy-stream wait, or kernels that run
    on the legacy stream themselves)."""
    import os
    import re
    allowed = {"upload", "dgasm_selftest_bounded_wait", "selftest_tc"}
    src = os.path.join(os.path.dirname(dg.__file__), "csrc")
    bad = []
    for name in sorted(os.listdir(src)):
        if not name.endswith((".cu", ".cpp", ".h")):
            continue
        func = None
        for lineno, line in enumerate(open(os.path.join(src, name)), 1):
            m = re.match(r"^(?:extern \"C\" )?(?:static )?[\w:<>*& ]+?\b(\w+)\(", line)
            if m and not line.startswith((" ", "\t", "//", "#")):
                func = m.group(1)
            plain_set = re.search(r"\bcudaMemset\(", line)
            plain_h2d = re.search(r"\bcudaMemcpy\(", line) and "cudaMemcpyDeviceToHost" not in line
            if (plain_set or plain_h2d) and func not in allowed:
                bad.append(f"{name}:{lineno} in {func}: {line.strip()}")
    assert not bad, "\n".join(bad)
