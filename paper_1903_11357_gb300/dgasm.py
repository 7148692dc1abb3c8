"""ctypes binding of the dgasm C-ABI (include/dgasm.h): argument marshalling only.

Every numerical step runs inside libdgasm.so.  Device arrays are passed as torch CUDA tensors
(their data pointers); host arrays as numpy arrays.  If the shared library has not been built,
``lib()`` raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libdgasm.so")

OK, PENDING = 0, 1
EINVAL, ENOMEM, ENOTSPD, ENOCONV, ENAN, ECUDA, ETIMEOUT, ETOOBIG, ECANCELLED, ENOTFOUND = range(-1, -11, -1)
FP64, FP32, TF32, BF16 = 0, 1, 2, 3
PRECISIONS = {"fp64": FP64, "fp32": FP32, "tf32": TF32, "bf16": BF16}

RHS_FN = C.CFUNCTYPE(None, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p)
# device allocator hooks of dgasm_set_allocator: alloc(bytes, stream, user) -> pointer, free(ptr, stream, user)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class SetupOpts(C.Structure):
    _fields_ = [("nsub", C.c_int), ("ncoarse", C.c_int), ("p_c", C.c_int),
                ("sub_of_elem", C.POINTER(C.c_int)), ("agg_of_elem", C.POINTER(C.c_int)),
                ("precision", C.c_int), ("stream", C.c_void_p), ("coarse_mesh", C.c_void_p)]


class SolveOpts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("maxit", C.c_int), ("fixed_iters", C.c_int), ("x0_given", C.c_int),
                ("host_buffers", C.c_int), ("stream", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("converged", C.c_int), ("relres", C.c_double), ("true_relres", C.c_double),
                ("lambda_min", C.c_double), ("lambda_max", C.c_double), ("kappa", C.c_double),
                ("solve_ms", C.c_double), ("launches", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class PrecInfo(C.Structure):
    _fields_ = [("nsub", C.c_int), ("nagg", C.c_int), ("n0", C.c_int), ("precision", C.c_int),
                ("local_dofs", C.c_int64), ("local_tiles", C.c_int64), ("stream_tiles", C.c_int64),
                ("factor_flops", C.c_int64),
                ("nnzb", C.c_int64), ("plan_ms", C.c_double), ("setup_ms", C.c_double),
                ("setup_launches", C.c_int), ("tc_fallback", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class DgasmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dgasm error {code}: {msg}")
        self.code = code


_lib = None


def lib():
    """The loaded libdgasm.so; raises if it has not been built (no CPU fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libdgasm.so is missing ({LIB_PATH}); build it with "
                               "`python -m paper_1903_11357_gb300.build`")
        L = C.CDLL(LIB_PATH)
        vp, ip, dp, i64p = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_int64)
        sig = {
            "dgasm_last_error": [C.c_char_p, C.c_size_t],
            "dgasm_mesh_create": [C.c_int, dp, C.c_int, ip, ip, dp, C.POINTER(vp)],
            "dgasm_mesh_info": [vp, ip, ip, ip],
            "dgasm_mesh_centroids": [vp, dp],
            "dgasm_mesh_destroy": [vp],
            "dgasm_partition": [vp, C.c_int, C.c_int, ip, ip],
            "dgasm_assemble": [vp, C.c_int, C.c_double, RHS_FN, vp, C.POINTER(vp)],
            "dgasm_assemble_device": [vp, C.c_int, C.c_double, RHS_FN, vp, vp, C.POINTER(vp)],
            "dgasm_system_dofs": [vp, i64p, ip],
            "dgasm_system_rhs": [vp, dp],
            "dgasm_system_blocks": [vp, i64p, ip, ip, dp],
            "dgasm_system_spmv": [vp, vp, vp, vp],
            "dgasm_system_destroy": [vp],
            "dgasm_setup": [vp, C.POINTER(SetupOpts), C.POINTER(vp)],
            "dgasm_setup_batch": [C.c_int, C.POINTER(vp), C.POINTER(C.POINTER(SetupOpts)), C.POINTER(vp)],
            "dgasm_prec_apply": [vp, C.c_int, vp, vp, vp],
            "dgasm_prec_partition": [vp, ip, ip],
            "dgasm_prec_footprint": [vp, i64p],
            "dgasm_prec_set_rhs_chunk": [vp, C.c_int, C.c_int],
            "dgasm_nonnested_prolongation": [vp, vp, C.c_int, C.c_int, i64p, ip, ip, dp],
            "dgasm_selftest_plan": [vp, C.c_int, i64p, i64p],
            "dgasm_prec_get_rhs_chunk": [vp, C.c_int, ip],
            "dgasm_prec_set_local_variant": [vp, C.c_int],
            "dgasm_prec_get_local_variant": [vp, ip],
            "dgasm_prec_destroy": [vp],
            "dgasm_solve": [vp, C.c_int, vp, vp, C.POINTER(SolveOpts), C.POINTER(Stats)],
            "dgasm_solve_batch": [C.c_int, C.POINTER(vp), ip, C.POINTER(vp), C.POINTER(vp), C.POINTER(SolveOpts),
                                  C.POINTER(Stats)],
            "dgasm_lanczos": [C.c_int, dp, dp, dp, dp],
            "dgasm_set_allocator": [vp, vp, vp],
            "dgasm_prec_info": [vp, C.c_void_p],
            "dgasm_profile_enable": [C.c_int],
            "dgasm_selftest_bounded_wait": [C.c_double, C.POINTER(C.c_int), dp],
            "dgasm_selftest_tc_update": [C.c_int, vp, vp],
            "dgasm_selftest_tc_update_bf16": [C.c_int, vp, vp],
            "dgasm_profile_read": [C.c_int, dp, i64p, C.c_int],
            "dgasm_server_create": [C.c_size_t, C.c_int, vp, C.POINTER(vp)],
            "dgasm_submit": [vp, vp, C.POINTER(SetupOpts), C.c_int, vp, vp, C.POINTER(SolveOpts),
                             C.POINTER(C.c_uint64)],
            "dgasm_poll": [vp, C.c_uint64, C.POINTER(Stats)],
            "dgasm_wait": [vp, C.c_uint64, C.c_int, C.POINTER(Stats)],
            "dgasm_cancel": [vp, C.c_uint64],
            "dgasm_server_stats": [vp, i64p, i64p, i64p, i64p],
            "dgasm_server_destroy": [vp],
            "dgasm_system_spmv_dot_noalloc": [vp, vp, vp, vp, vp],
            "dgasm_probe_fp64": [ip, dp, dp],
            "dgasm_set_local_cta_form": [C.c_int],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        _lib = L
    return _lib


def exported_symbols():
    """Names of the entry points declared in include/dgasm.h."""
    import re
    with open(os.path.join(os.path.dirname(_HERE), "include", "dgasm.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"\bint\s+(dgasm_\w+)\s*\(", text)))


def last_error() -> str:
    buf = C.create_string_buffer(512)
    lib().dgasm_last_error(buf, 512)
    return buf.value.decode()


def check(code):
    if code < 0:
        raise DgasmError(code, last_error())
    return code


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _stream_ptr(stream):
    if stream is None:
        return None
    return C.c_void_p(int(getattr(stream, "cuda_stream", stream)))


def _dev_ptr(t):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _nvec(ndof, *arrays, host=False):
    """Vector count k of arrays shaped (ndof,) or (k, ndof), the same for all of them.  The library reads and
    writes k * ndof doubles through each pointer, so a shape that does not match is refused here instead of
    running past the end of a buffer."""
    k = None
    for a in arrays:
        if host and not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
            raise TypeError("expected a C-contiguous float64 numpy array")
        shape = tuple(a.shape)
        if len(shape) not in (1, 2) or shape[-1] != ndof:
            raise ValueError(f"expected shape ({ndof},) or (k, {ndof}), got {shape}")
        kk = 1 if len(shape) == 1 else shape[0]
        if k is not None and kk != k:
            raise ValueError(f"input and output hold different numbers of vectors ({k} and {kk})")
        k = kk
    return k


class Mesh:
    def __init__(self, xy, poly_ptr, poly_vtx, rho):
        self._xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1)
        ptr = np.ascontiguousarray(poly_ptr, dtype=np.int32)
        vtx = np.ascontiguousarray(poly_vtx, dtype=np.int32)
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        self.ne = len(ptr) - 1
        h = C.c_void_p()
        check(lib().dgasm_mesh_create(len(self._xy) // 2, _dp(self._xy), self.ne, _ip(ptr), _ip(vtx), _dp(rho),
                                      C.byref(h)))
        self.h = h

    @classmethod
    def from_polymesh(cls, m, rho):
        return cls(m.xy, m.poly_ptr, m.poly_vtx, rho)

    def info(self):
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        check(lib().dgasm_mesh_info(self.h, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def centroids(self):
        out = np.empty(2 * self.ne)
        check(lib().dgasm_mesh_centroids(self.h, _dp(out)))
        return out.reshape(-1, 2)

    def partition(self, nsub, ncoarse=0):
        sub = np.empty(self.ne, np.int32)
        agg = np.empty(self.ne, np.int32)
        check(lib().dgasm_partition(self.h, nsub, ncoarse, _ip(sub), _ip(agg)))
        return sub, (agg if ncoarse > 0 else None)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.dgasm_mesh_destroy(self.h)
            self.h = None


class System:
    def __init__(self, mesh: Mesh, p: int, c_sigma: float = 10.0, f=None, device=False, stream=None):
        """device=True assembles the matrix on the GPU (dgasm_assemble_device)."""
        self.mesh = mesh  # keeps the mesh alive
        self.p = p
        h = C.c_void_p()
        cb = RHS_FN()
        if f is not None:
            def _cb(n, xy, out, user):
                pts = np.ctypeslib.as_array(xy, shape=(n, 2))
                o = np.ctypeslib.as_array(out, shape=(n,))
                o[:] = f(pts)
            cb = RHS_FN(_cb)
        self._cb = cb
        if device:
            check(lib().dgasm_assemble_device(mesh.h, p, c_sigma, cb, None, _stream_ptr(stream), C.byref(h)))
        else:
            check(lib().dgasm_assemble(mesh.h, p, c_sigma, cb, None, C.byref(h)))
        self.h = h
        n = C.c_int64()
        npb = C.c_int()
        check(lib().dgasm_system_dofs(h, C.byref(n), C.byref(npb)))
        self.ndof, self.np = n.value, npb.value

    def rhs(self):
        b = np.empty(self.ndof)
        check(lib().dgasm_system_rhs(self.h, _dp(b)))
        return b

    def blocks(self):
        nnzb = C.c_int64()
        check(lib().dgasm_system_blocks(self.h, C.byref(nnzb), None, None, None))
        rowptr = np.empty(self.mesh.ne + 1, np.int32)
        col = np.empty(nnzb.value, np.int32)
        vals = np.empty(nnzb.value * self.np * self.np)
        check(lib().dgasm_system_blocks(self.h, C.byref(nnzb), _ip(rowptr), _ip(col), _dp(vals)))
        return rowptr, col, vals.reshape(-1, self.np, self.np)

    def spmv(self, x, y, stream=None):
        if _nvec(self.ndof, x, y) != 1 or x.dim() != 1:
            raise ValueError("spmv takes one vector")
        check(lib().dgasm_system_spmv(self.h, _dev_ptr(x), _dev_ptr(y), _stream_ptr(stream)))

    def spmv_dot_noalloc(self, x, y, out, stream=None):
        """y = A x and out[0] = x^T A x with no device allocation (dgasm_system_spmv_dot_noalloc; asynchronous
        on the stream).  The matrix must already be on the device (spmv or a Prec uploads it)."""
        import torch
        if _nvec(self.ndof, x, y) != 1 or x.dim() != 1:
            raise ValueError("spmv_dot_noalloc takes one vector")
        if not (isinstance(out, torch.Tensor) and out.numel() >= 1):
            raise ValueError("out must hold at least one double")
        check(lib().dgasm_system_spmv_dot_noalloc(self.h, _dev_ptr(x), _dev_ptr(y), _dev_ptr(out),
                                                  _stream_ptr(stream)))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.dgasm_system_destroy(self.h)
            self.h = None


class Prec:
    def __init__(self, system: System, nsub: int, ncoarse: int, p_c: int = 1, precision="fp64", sub_of_elem=None,
                 agg_of_elem=None, stream=None, coarse_mesh=None):
        """coarse_mesh: a Mesh of the same domain carrying a non-nested coarse space (ncoarse is ignored)."""
        o = self._options(system, nsub, ncoarse, p_c, precision, sub_of_elem, agg_of_elem, stream, coarse_mesh)
        h = C.c_void_p()
        check(lib().dgasm_setup(system.h, C.byref(o), C.byref(h)))
        self.h = h

    def _options(self, system, nsub, ncoarse, p_c, precision, sub_of_elem, agg_of_elem, stream, coarse_mesh):
        """dgasm_setup_opts for this preconditioner; the arrays it points into are kept on the object."""
        self.system = system
        self.ndof = system.ndof
        self._coarse = coarse_mesh
        o = SetupOpts()
        if coarse_mesh is not None:
            o.coarse_mesh = coarse_mesh.h
        o.nsub, o.ncoarse, o.p_c = nsub, ncoarse, p_c
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self._sub = self._agg = None
        if sub_of_elem is not None:
            self._sub = np.ascontiguousarray(sub_of_elem, np.int32)
            o.sub_of_elem = _ip(self._sub)
        if agg_of_elem is not None:
            self._agg = np.ascontiguousarray(agg_of_elem, np.int32)
            o.agg_of_elem = _ip(self._agg)
        o.stream = _stream_ptr(stream)
        return o

    def set_rhs_chunk(self, nrhs, kc):
        """Right-hand sides per local-solve item for nrhs-vector solves: 1, 4, or 0 to let the first solve
        measure both."""
        check(lib().dgasm_prec_set_rhs_chunk(self.h, int(nrhs), int(kc)))

    def rhs_chunk(self, nrhs):
        v = C.c_int()
        check(lib().dgasm_prec_get_rhs_chunk(self.h, int(nrhs), C.byref(v)))
        return v.value

    LOCAL_VARIANTS = {"tune": 0, "sweeps": 1, "inverse": 2}

    def set_local_variant(self, variant):
        """Local solves by the envelope sweeps ("sweeps"), by explicit subdomain inverses ("inverse", small
        subdomains only), or "tune" to let the first solve measure both (dgasm_prec_set_local_variant)."""
        v = self.LOCAL_VARIANTS[variant] if isinstance(variant, str) else int(variant)
        check(lib().dgasm_prec_set_local_variant(self.h, v))

    def local_variant(self):
        v = C.c_int()
        check(lib().dgasm_prec_get_local_variant(self.h, C.byref(v)))
        return {0: "tune", 1: "sweeps", 2: "inverse"}[v.value]

    def apply(self, r, z, stream=None):
        k = _nvec(self.ndof, r, z)
        check(lib().dgasm_prec_apply(self.h, k, _dev_ptr(r), _dev_ptr(z), _stream_ptr(stream)))

    def partition(self):
        ne = self.system.mesh.ne
        sub = np.empty(ne, np.int32)
        agg = np.full(ne, -1, np.int32)
        check(lib().dgasm_prec_partition(self.h, _ip(sub), _ip(agg)))
        return sub, agg

    def info(self):
        i = PrecInfo()
        check(lib().dgasm_prec_info(self.h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in i._fields_}

    def footprint(self):
        b = C.c_int64()
        check(lib().dgasm_prec_footprint(self.h, C.byref(b)))
        return b.value

    def solve(self, b, x, rtol=1e-8, maxit=10000, fixed_iters=0, stream=None, host_buffers=False, x0_given=False):
        """b, x: (k, ndof) or (ndof,) float64 CUDA tensors (numpy arrays if host_buffers; views of pinned
        memory, e.g. torch.zeros(n, dtype=torch.float64).pin_memory().numpy(), copy fastest); with x0_given
        x holds the initial guess on entry.  Returns (return code, [stats dict per right-hand side])."""
        o = SolveOpts(rtol=rtol, maxit=maxit, fixed_iters=fixed_iters, x0_given=1 if x0_given else 0,
                      host_buffers=1 if host_buffers else 0, stream=_stream_ptr(stream))
        k = _nvec(self.ndof, b, x, host=host_buffers)
        if host_buffers:
            bp, xp = C.c_void_p(b.ctypes.data), C.c_void_p(x.ctypes.data)
        else:
            bp, xp = _dev_ptr(b), _dev_ptr(x)
        st = (Stats * k)()
        rc = lib().dgasm_solve(self.h, k, bp, xp, C.byref(o), st)
        if rc < 0 and rc != ENOCONV:
            check(rc)
        return rc, [s.as_dict() for s in st]

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.dgasm_prec_destroy(self.h)
            self.h = None


def setup_batch(problems):
    """Preconditioners of several problems built at once (dgasm_setup_batch): problems is a list of dicts of
    Prec's arguments (system, nsub, ncoarse and optionally p_c, precision, sub_of_elem, agg_of_elem, stream,
    coarse_mesh).  Returns one Prec per problem, each the same as Prec(**problem) would build."""
    n = len(problems)
    if n < 1:
        raise ValueError("no problems")
    precs, opts = [], []
    for pr in problems:
        P = Prec.__new__(Prec)
        P.h = None
        a = dict(p_c=1, precision="fp64", sub_of_elem=None, agg_of_elem=None, stream=None, coarse_mesh=None)
        a.update(pr)
        opts.append(P._options(a["system"], a["nsub"], a["ncoarse"], a["p_c"], a["precision"], a["sub_of_elem"],
                               a["agg_of_elem"], a["stream"], a["coarse_mesh"]))
        precs.append(P)
    systems = (C.c_void_p * n)(*[P.system.h.value for P in precs])
    op = (C.POINTER(SetupOpts) * n)(*[C.pointer(o) for o in opts])
    hs = (C.c_void_p * n)()
    check(lib().dgasm_setup_batch(n, systems, op, hs))
    for P, h in zip(precs, hs):
        P.h = C.c_void_p(h)
    return precs


def solve_batch(precs, bs, xs, rtol=1e-8, maxit=10000, fixed_iters=0, stream=None, x0_given=False):
    n = len(precs)
    if len(bs) != n or len(xs) != n:
        raise ValueError("one b and one x per preconditioner")
    hs = (C.c_void_p * n)(*[p.h.value for p in precs])
    ks = np.array([_nvec(p.ndof, b, x) for p, b, x in zip(precs, bs, xs)], np.int32)
    bp = (C.c_void_p * n)(*[_dev_ptr(b).value for b in bs])
    xp = (C.c_void_p * n)(*[_dev_ptr(x).value for x in xs])
    o = SolveOpts(rtol=rtol, maxit=maxit, fixed_iters=fixed_iters, x0_given=1 if x0_given else 0, host_buffers=0,
                  stream=_stream_ptr(stream))
    st = (Stats * int(ks.sum()))()
    rc = lib().dgasm_solve_batch(n, hs, _ip(ks), bp, xp, C.byref(o), st)
    if rc < 0 and rc != ENOCONV:
        check(rc)
    return rc, [s.as_dict() for s in st]


def lanczos(alphas, betas):
    a = np.ascontiguousarray(alphas, np.float64)
    b = np.ascontiguousarray(betas if len(betas) else [0.0], np.float64)
    lo, hi = C.c_double(), C.c_double()
    check(lib().dgasm_lanczos(len(a), _dp(a), _dp(b), C.byref(lo), C.byref(hi)))
    return lo.value, hi.value


def selftest_bounded_wait(limit_ms=5.0):
    """Runs the kernels' bounded-wait failure path on purpose (a wait nothing satisfies); returns
    (gave_up, device ms)."""
    g = C.c_int()
    ms = C.c_double()
    check(lib().dgasm_selftest_bounded_wait(float(limit_ms), C.byref(g), C.byref(ms)))
    return bool(g.value), ms.value


def nonnested_prolongation(fine: "Mesh", coarse: "Mesh", p: int, q: int):
    """R_0^T of a non-nested coarse mesh (host): (ptr [ne+1], col [npair], blocks [npair, n_p, n_q])."""
    n = C.c_int64()
    check(lib().dgasm_nonnested_prolongation(fine.h, coarse.h, p, q, C.byref(n), None, None, None))
    ptr = np.empty(fine.ne + 1, np.int32)
    col = np.empty(n.value, np.int32)
    nb, nq = (p + 1) * (p + 2) // 2, (q + 1) * (q + 2) // 2
    blk = np.empty(n.value * nb * nq)
    check(lib().dgasm_nonnested_prolongation(fine.h, coarse.h, p, q, C.byref(n), _ip(ptr), _ip(col), _dp(blk)))
    return ptr, col, blk.reshape(-1, nb, nq)


def selftest_plan(system: "System", nsub: int):
    """Host plan consistency check: (violations, entries compared)."""
    v, n = C.c_int64(), C.c_int64()
    check(lib().dgasm_selftest_plan(system.h, int(nsub), C.byref(v), C.byref(n)))
    return v.value, n.value


def selftest_tc_update(tiles, kind="tf32"):
    """One tensor-core trailing-update step (C_IJ -= L_I0 L_J0^T, 1 <= J <= I <= n) on a dense lower tile
    matrix: `tiles` is a float32 array of shape ((n+1)(n+2)/2, 32, 32), tile (I, J) at I(I+1)/2 + J; returns
    the updated array.  kind: "tf32" (the TF32 mode's kernel) or "bf16" (the BF16 mode's)."""
    t = np.ascontiguousarray(tiles, dtype=np.float32)
    m = t.shape[0]
    n = int(round((-3 + np.sqrt(1 + 8 * m)) / 2))
    if t.shape[1:] != (32, 32) or (n + 1) * (n + 2) // 2 != m:
        raise ValueError("tiles must have shape ((n+1)(n+2)/2, 32, 32)")
    out = np.empty_like(t)
    fn = lib().dgasm_selftest_tc_update_bf16 if kind == "bf16" else lib().dgasm_selftest_tc_update
    check(fn(n, t.ctypes.data, out.ctypes.data))
    return out


PROFILE_KINDS = ["spmv", "update", "local", "coarse", "pupdate", "chol_diag", "chol_panel", "chol_update"]


def profile_enable(on=True, kinds=None):
    """Time kernel launches with CUDA events: every kind (on=True), none (on=False), or only the
    named kinds (kinds: iterable of names from PROFILE_KINDS)."""
    if not on:
        mask = 0
    elif kinds is None:
        mask = (1 << len(PROFILE_KINDS)) - 1
    else:
        mask = 0
        for k in kinds:
            mask |= 1 << PROFILE_KINDS.index(k)
    check(lib().dgasm_profile_enable(mask))


def profile_read(reset=False):
    """{kind: (total_ms, launches)} accumulated since the last reset."""
    out = {}
    for i, name in enumerate(PROFILE_KINDS):
        ms, n = C.c_double(), C.c_int64()
        check(lib().dgasm_profile_read(i, C.byref(ms), C.byref(n), 1 if reset else 0))
        out[name] = (ms.value, n.value)
    return out


class Server:
    """Continuous-batching solve server (dgasm_server_*)."""

    def __init__(self, hbm_budget: int, max_slots: int, stream=None):
        h = C.c_void_p()
        check(lib().dgasm_server_create(int(hbm_budget), int(max_slots), _stream_ptr(stream), C.byref(h)))
        self.h = h
        self._keep = {}

    def submit(self, system: System, nsub, ncoarse, p_c, b, x, precision="fp64", rtol=1e-8, maxit=10000,
               sub_of_elem=None, agg_of_elem=None, coarse_mesh=None):
        o = SetupOpts()
        o.nsub, o.ncoarse, o.p_c = nsub, ncoarse, p_c
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        keep = [b, x, system]   # the server reads the system until the request finishes
        if coarse_mesh is not None:
            keep.append(coarse_mesh)
            o.coarse_mesh = coarse_mesh.h
        if sub_of_elem is not None:
            a = np.ascontiguousarray(sub_of_elem, np.int32)
            keep.append(a)
            o.sub_of_elem = _ip(a)
        if agg_of_elem is not None:
            a = np.ascontiguousarray(agg_of_elem, np.int32)
            keep.append(a)
            o.agg_of_elem = _ip(a)
        so = SolveOpts(rtol=rtol, maxit=maxit, fixed_iters=0, x0_given=0, host_buffers=0, stream=None)
        k = _nvec(system.ndof, b, x)
        t = C.c_uint64()
        check(lib().dgasm_submit(self.h, system.h, C.byref(o), k, _dev_ptr(b), _dev_ptr(x), C.byref(so), C.byref(t)))
        self._keep[t.value] = (keep, k)
        return t.value

    def _result(self, ticket, rc, st):
        if rc == PENDING:
            return rc, None
        keep = self._keep.pop(ticket, None)
        k = keep[1] if keep else 1
        if rc < 0 and rc != ENOCONV:
            return rc, None
        return rc, [st[i].as_dict() for i in range(k)]

    def poll(self, ticket):
        st = (Stats * 8)()
        rc = lib().dgasm_poll(self.h, ticket, st)
        return self._result(ticket, rc, st)

    def wait(self, ticket, timeout_ms=-1):
        st = (Stats * 8)()
        rc = lib().dgasm_wait(self.h, ticket, int(timeout_ms), st)
        if rc == ETIMEOUT:
            return rc, None
        return self._result(ticket, rc, st)

    def cancel(self, ticket):
        return lib().dgasm_cancel(self.h, ticket)

    def stats(self):
        v = [C.c_int64() for _ in range(4)]
        check(lib().dgasm_server_stats(self.h, *[C.byref(x) for x in v]))
        return dict(zip(["done", "rounds", "stalls", "bytes_in_use"], [x.value for x in v]))

    def close(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.dgasm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


def probe_fp64():
    """FP64 FMA issue rate of the current device (dgasm_probe_fp64): (SM count, FMA per clock per SM, TFLOP/s)."""
    n = C.c_int()
    r = C.c_double()
    t = C.c_double()
    check(lib().dgasm_probe_fp64(C.byref(n), C.byref(r), C.byref(t)))
    return n.value, r.value, t.value


def set_local_cta_form(form):
    """FP32/BF16 local-solve launches: "auto" (pairs while they all fit at once, else one CTA per item), "one"
    or "pair" (dgasm_set_local_cta_form; process-wide; results are the same bits in every form)."""
    check(lib().dgasm_set_local_cta_form({"auto": 0, "one": 1, "pair": 2}[form]))
