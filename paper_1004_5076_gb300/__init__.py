"""Python binding of the scabem C-ABI (include/scabem.h).

Argument marshalling only: every computation runs in the CUDA library
``libscabem.so`` built in this directory (``build.py``).  Importing this
package does not load the library; the first call does, and raises if it is
missing.  There is no CPU fallback.

Data buffers may be torch tensors (device or host) or numpy arrays (host);
complex64 / complex128 arrays are passed as interleaved (re, im) pointers.
Streams: pass ``stream=`` an integer handle or a ``torch.cuda.Stream``;
the default is torch's current stream when torch has CUDA, else 0.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(_HERE, "libscabem.so")
_lib = None

SCABEM_C64, SCABEM_C128 = 0, 1
SIGMA_MONOMIAL, SIGMA_PER_QPOINT, SIGMA_BSPLINE = 0, 1, 2
STATUS = {
    0: "SCABEM_OK", -1: "SCABEM_E_ARG", -2: "SCABEM_E_MESH", -3: "SCABEM_E_DEVICE", -4: "SCABEM_E_NOMEM",
    -5: "SCABEM_E_NOCONV", -6: "SCABEM_E_BREAKDOWN", -7: "SCABEM_E_NONFINITE", -8: "SCABEM_E_TIMEOUT",
}


class ScabemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Media(C.Structure):
    _fields_ = [("eps_i", C.c_double), ("mu_i", C.c_double), ("eps_e", C.c_double), ("mu_e", C.c_double),
                ("lambda0", C.c_double)]


class GridOpts(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("h", C.c_double), ("origin", C.c_double * 3), ("p", C.c_int32),
                ("q", C.c_int32), ("r_near", C.c_double), ("prec_mask", C.c_int32), ("transverse", C.c_int32)]


class Sigma(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nseg", C.c_int32), ("seg", C.POINTER(C.c_double)),
                ("per_qpoint", C.POINTER(C.c_double)), ("x0", C.c_double), ("L", C.c_double),
                ("axis", C.c_int32), ("ncoef", C.c_int32), ("coef", C.POINTER(C.c_double))]


class Source(C.Structure):
    _fields_ = [("kind", C.c_int32), ("side", C.c_int32), ("pos", C.c_double * 3), ("dir", C.c_double * 3),
                ("pol", C.c_double * 3), ("b", C.c_double)]


class SolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("restart", C.c_int32), ("maxit", C.c_int32), ("refine_tol", C.c_double),
                ("max_refine", C.c_int32), ("prec", C.c_int32), ("transpose", C.c_int32)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("refinements", C.c_int32), ("relres", C.c_double), ("status", C.c_int32)]


class Poynting(C.Structure):
    _fields_ = [("xc", C.c_double), ("core", C.c_double * 2), ("box", C.c_double * 2), ("slab", C.c_double),
                ("n", C.c_int32)]


class Circulant(C.Structure):
    _fields_ = [("axis", C.c_int32), ("x0", C.c_double), ("dx", C.c_double), ("first", C.c_int32),
                ("count", C.c_int32), ("kind", C.c_int32)]


class Probe(C.Structure):
    _fields_ = [("axis", C.c_int32), ("comp", C.c_int32), ("p0", C.c_double * 3), ("t0", C.c_double),
                ("t1", C.c_double), ("npts", C.c_int32), ("beta_lo", C.c_double), ("beta_hi", C.c_double),
                ("nbeta", C.c_int32)]


EXPORTS = [
    "scabem_mesh_create", "scabem_mesh_info", "scabem_mesh_edges", "scabem_mesh_destroy", "scabem_op_create",
    "scabem_op_info", "scabem_op_destroy", "scabem_set_sigma", "scabem_apply", "scabem_rhs", "scabem_solve",
    "scabem_fields", "scabem_reflection", "scabem_last_error", "scabem_rhs_noalloc", "scabem_profile",
    "scabem_profile_read",
]


def lib():
    """Load libscabem.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIBPATH):
        raise RuntimeError(f"CUDA library not built: {LIBPATH} missing (run paper_1004_5076_gb300/build.py)")
    L = C.CDLL(LIBPATH)
    vp, i64, i32, dp = C.c_void_p, C.c_int64, C.c_int32, C.POINTER(C.c_double)
    L.scabem_mesh_create.argtypes = [vp, i64, vp, i64, vp, C.POINTER(vp)]
    L.scabem_mesh_info.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
    L.scabem_mesh_edges.argtypes = [vp, vp, vp, vp]
    L.scabem_mesh_destroy.argtypes = [vp]
    L.scabem_mesh_destroy.restype = None
    L.scabem_op_create.argtypes = [vp, C.POINTER(Media), C.POINTER(GridOpts), vp, C.POINTER(vp)]
    L.scabem_op_info.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
    L.scabem_op_grid_info.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i32)]
    L.scabem_op_destroy.argtypes = [vp]
    L.scabem_op_destroy.restype = None
    L.scabem_set_sigma.argtypes = [vp, C.POINTER(Sigma)]
    L.scabem_apply.argtypes = [vp, vp, vp, i32, i64, i32, vp]
    L.scabem_apply_adjoint.argtypes = [vp, vp, vp, i32, i64, i32, vp]
    L.scabem_selftest_wait_limit.argtypes = [vp, vp]
    L.scabem_grid_plan.argtypes = [vp, C.c_double, i32, C.c_double, C.POINTER(GridOpts)]
    L.scabem_decay_fit.argtypes = [vp, vp, i32, C.c_double, C.c_double, i32, C.c_double, C.c_double, i32, vp, vp]
    L.scabem_decay_rate.argtypes = [vp, vp, i32, i64, C.POINTER(Probe), C.c_double, C.c_double, i32,
                                    C.POINTER(Source), vp, vp]
    L.scabem_sigma_gradient.argtypes = [vp, vp, vp, C.POINTER(Source), i32, C.POINTER(Sigma), vp, vp]
    L.scabem_rhs.argtypes = [vp, C.POINTER(Source), i32, vp, i64, i32, vp]
    L.scabem_solve.argtypes = [vp, vp, vp, i32, i64, C.POINTER(SolveOpts), vp, C.POINTER(SolveInfo)]
    L.scabem_fields.argtypes = [vp, vp, i32, i64, vp, i32, C.POINTER(Source), vp, vp]
    L.scabem_reflection.argtypes = [vp, vp, i32, i64, C.POINTER(Probe), C.POINTER(Source), vp, vp]
    L.scabem_rhs_noalloc.argtypes = [vp, C.POINTER(Source), i32, vp, i64, i32, vp]
    L.scabem_profile.argtypes = [vp, i32, i32]
    L.scabem_profile_read.argtypes = [vp, vp, C.POINTER(i64)]
    L.scabem_peak_fma.argtypes = [i32, C.POINTER(C.c_double), vp]
    L.scabem_fields_eh.argtypes = [vp, vp, i32, i64, vp, i32, i32, C.POINTER(Source), vp, vp, vp]
    L.scabem_set_precond_circulant.argtypes = [vp, vp, C.POINTER(Circulant), vp]
    L.scabem_autotune.argtypes = [vp, i32, i32, vp, vp]
    L.scabem_precond_apply.argtypes = [vp, vp, vp, i32, i64, i32, vp]
    L.scabem_poynting_rate.argtypes = [vp, vp, i32, i64, C.POINTER(Poynting), C.POINTER(Source), vp, vp]
    L.scabem_last_error.argtypes = []
    L.scabem_last_error.restype = C.c_char_p
    _lib = L
    return L


def _check(rc):
    if rc != 0:
        raise ScabemError(rc, lib().scabem_last_error().decode())


def _ptr(a):
    """Data pointer of a torch tensor or numpy array (must be contiguous)."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("buffer must be contiguous")
        if (hasattr(a, "is_conj") and a.is_conj()) or (hasattr(a, "is_neg") and a.is_neg()):
            raise ValueError("tensor has a pending conjugate/negation bit: call resolve_conj() / resolve_neg()")
        return C.c_void_p(a.data_ptr())
    a = np.asarray(a)
    if not a.flags["C_CONTIGUOUS"] and not a.flags["F_CONTIGUOUS"]:
        raise ValueError("buffer must be contiguous")
    return C.c_void_p(a.ctypes.data)


def _stream(stream):
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return C.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


# ------------------------------------------------------------------ C-ABI, same names
def scabem_mesh_create(V, T, region):
    V = np.ascontiguousarray(V, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.int32)
    region = np.ascontiguousarray(region, dtype=np.int32)
    h = C.c_void_p()
    _check(lib().scabem_mesh_create(_ptr(V), len(V), _ptr(T), len(T), _ptr(region), C.byref(h)))
    return h


def scabem_mesh_info(mesh):
    a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
    _check(lib().scabem_mesh_info(mesh, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def scabem_mesh_edges(mesh):
    nL, nR, _ = scabem_mesh_info(mesh)
    ne = nL + nR
    ev = np.zeros((ne, 2), np.int64)
    et = np.zeros((ne, 2), np.int64)
    ec = np.zeros(ne, np.int32)
    _check(lib().scabem_mesh_edges(mesh, _ptr(ev), _ptr(et), _ptr(ec)))
    return ev, et, ec


def scabem_mesh_destroy(mesh):
    lib().scabem_mesh_destroy(mesh)


TRANSVERSE = {"auto": 0, "fft": 1, "direct": 2}


def scabem_op_create(mesh, media, n, h, origin, p=3, q=6, r_near=0.0, prec_mask=3, stream=None, transverse="auto"):
    md = Media(*media)
    tv = TRANSVERSE[transverse] if isinstance(transverse, str) else int(transverse)
    go = GridOpts((C.c_int32 * 3)(*n), h, (C.c_double * 3)(*origin), p, q, r_near, prec_mask, tv)
    op = C.c_void_p()
    _check(lib().scabem_op_create(mesh, C.byref(md), C.byref(go), _stream(stream), C.byref(op)))
    return op


def scabem_grid_plan(mesh, h_max, p=3, near_h=2.05):
    """Grid options for scabem_op_create from the mesh's bounding box (see the header)."""
    go = GridOpts()
    _check(lib().scabem_grid_plan(mesh, h_max, p, near_h, C.byref(go)))
    return {"n": tuple(go.n), "h": go.h, "origin": tuple(go.origin), "p": go.p, "q": go.q, "r_near": go.r_near,
            "prec_mask": go.prec_mask, "transverse": go.transverse}


def scabem_op_info(op):
    a, b, c, d = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
    _check(lib().scabem_op_info(op, C.byref(a), C.byref(b), C.byref(c), C.byref(d)))
    return {"near_pairs": a.value, "near_bytes_c64": b.value, "near_bytes_c128": c.value, "qpoints": d.value}


def scabem_op_grid_info(op):
    a, b, c = C.c_int64(), C.c_int64(), C.c_int32()
    _check(lib().scabem_op_grid_info(op, C.byref(a), C.byref(b), C.byref(c)))
    return {"covered_points": a.value, "active_columns": b.value, "transverse_direct": bool(c.value)}


def scabem_op_destroy(op):
    lib().scabem_op_destroy(op)


def scabem_set_sigma(op, segments=None, per_qpoint=None, bspline=None):
    """segments: list of (x0, L, sigma0 [S], d, axis, dir); or per_qpoint (nt*q) [S];
    or bspline = (x0, L, axis, coef) with coef the cubic B-spline coefficients [S]."""
    if bspline is not None:
        x0, L, axis, coef = bspline
        cf = np.ascontiguousarray(coef, dtype=np.float64).reshape(-1)
        sg = Sigma(SIGMA_BSPLINE, 0, None, None, float(x0), float(L), int(axis), len(cf),
                   cf.ctypes.data_as(C.POINTER(C.c_double)))
        _check(lib().scabem_set_sigma(op, C.byref(sg)))
        return
    if per_qpoint is not None:
        arr = np.ascontiguousarray(per_qpoint, dtype=np.float64).reshape(-1)
        sg = Sigma(SIGMA_PER_QPOINT, 0, None, arr.ctypes.data_as(C.POINTER(C.c_double)))
        _check(lib().scabem_set_sigma(op, C.byref(sg)))
        return
    seg = np.ascontiguousarray(np.asarray(segments if segments else [], dtype=np.float64).reshape(-1))
    sg = Sigma(SIGMA_MONOMIAL, len(seg) // 6, seg.ctypes.data_as(C.POINTER(C.c_double)) if len(seg) else None,
               None)
    _check(lib().scabem_set_sigma(op, C.byref(sg)))


def scabem_apply(op, x, y, nrhs=1, ld=None, prec=SCABEM_C128, stream=None):
    if ld is None:
        ld = x.shape[0]
    _check(lib().scabem_apply(op, _ptr(x), _ptr(y), nrhs, ld, prec, _stream(stream)))


def scabem_apply_adjoint(op, y, x, nrhs=1, ld=None, prec=SCABEM_C128, stream=None):
    """x = A^T y (transpose, no conjugation)."""
    if ld is None:
        ld = y.shape[0]
    _check(lib().scabem_apply_adjoint(op, _ptr(y), _ptr(x), nrhs, ld, prec, _stream(stream)))


def scabem_selftest_wait_limit(op, stream=None):
    """Run the bounded-wait self-test; returns the status code (SCABEM_E_TIMEOUT expected)."""
    return lib().scabem_selftest_wait_limit(op, _stream(stream))


def make_source(kind, side=0, pos=(0, 0, 0), dir=(1, 0, 0), pol=(0, 1, 0), b=0.0):
    kinds = {"planewave": 0, "dipole": 1, "beam": 2}
    k = kinds[kind] if isinstance(kind, str) else int(kind)
    s = {"i": 0, "e": 1}.get(side, side)
    return Source(k, int(s), (C.c_double * 3)(*pos), (C.c_double * 3)(*dir), (C.c_double * 3)(*pol), b)


def scabem_rhs(op, sources, b, ld=None, prec=SCABEM_C128, stream=None):
    arr = (Source * len(sources))(*sources)
    if ld is None:
        ld = b.shape[0]
    _check(lib().scabem_rhs(op, arr, len(sources), _ptr(b), ld, prec, _stream(stream)))


def scabem_rhs_noalloc(op, sources, b, ld=None, prec=SCABEM_C128, stream=None):
    """scabem_rhs without any device allocation (b must be a device buffer).

    For callers that cannot allocate device memory while they run; the
    library keeps the scratch in one fixed device array (meshes of at most
    32768 triangles), shared by all calls, so calls must not overlap on the GPU.
    """
    arr = (Source * len(sources))(*sources)
    if ld is None:
        ld = b.shape[0]
    _check(lib().scabem_rhs_noalloc(op, arr, len(sources), _ptr(b), ld, prec, _stream(stream)))


def scabem_solve(op, b, x, nrhs=1, ld=None, tol=1e-6, restart=60, maxit=2000, refine_tol=1e-8, max_refine=10,
                 prec=SCABEM_C128, stream=None, transpose=False):
    """Solve A x = b (or A^T x = b with transpose=True); x holds the initial guess."""
    if ld is None:
        ld = b.shape[0]
    o = SolveOpts(tol, restart, maxit, refine_tol, max_refine, prec, 1 if transpose else 0)
    info = (SolveInfo * max(nrhs, 1))()
    rc = lib().scabem_solve(op, _ptr(b), _ptr(x), nrhs, ld, C.byref(o), _stream(stream), info)
    out = [{"iters": i.iters, "refinements": i.refinements, "relres": i.relres, "status": i.status}
           for i in info[:nrhs]]
    _check(rc)
    return out


def scabem_sigma_gradient(op, x, lam, sources=(), segments=None, bspline=None, per_qpoint=False, stream=None):
    """g_i = sum_p dsigma_p/dc_i d(lam^T (A x - b))/dsigma_p for the parameters of
    a profile: bspline = (x0, L, axis, ncoef) -> ncoef values; segments (the
    monomial list) -> one value per segment (d / d sigma0); per_qpoint -> Q values."""
    arr = (Source * max(len(sources), 1))(*sources)
    if bspline is not None:
        x0, L, axis, ncoef = bspline
        basis = Sigma(SIGMA_BSPLINE, 0, None, None, float(x0), float(L), int(axis), int(ncoef), None)
        n = int(ncoef)
        keep = None
    elif segments is not None:
        seg = np.ascontiguousarray(np.asarray(segments, dtype=np.float64).reshape(-1))
        basis = Sigma(SIGMA_MONOMIAL, len(seg) // 6, seg.ctypes.data_as(C.POINTER(C.c_double)), None)
        n = len(seg) // 6
        keep = seg
    elif per_qpoint:
        basis = Sigma(SIGMA_PER_QPOINT, 0, None, None)
        n = scabem_op_info(op)["qpoints"]
        keep = None
    else:
        raise ValueError("give bspline, segments or per_qpoint")
    out = np.zeros(2 * max(n, 1), dtype=np.float64)
    _check(lib().scabem_sigma_gradient(op, _ptr(x), _ptr(lam), arr, len(sources), C.byref(basis), _ptr(out),
                                       _stream(stream)))
    del keep
    return out[0::2][:n] + 1j * out[1::2][:n]


def scabem_fields(op, x, pts, inc=None, nrhs=1, ld=None, stream=None):
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    if ld is None:
        ld = x.shape[0]
    E = np.zeros((nrhs, len(pts), 3), np.complex128)
    _check(lib().scabem_fields(op, _ptr(x), nrhs, ld, _ptr(pts), len(pts), C.byref(inc) if inc else None, _ptr(E),
                               _stream(stream)))
    return E


def scabem_autotune(op, prec=SCABEM_C64, nrhs=1, stream=None):
    """Time the operator's runtime shapes and keep the fastest: returns
    {"ms": best, "ms_initial": ..., "direct": bool, "axis0_lines": int}."""
    out = np.zeros(4, np.float64)
    _check(lib().scabem_autotune(op, int(prec), int(nrhs), _stream(stream), _ptr(out)))
    return {"ms": out[0], "ms_initial": out[1], "direct": bool(out[2]), "axis0_lines": int(out[3])}


def scabem_set_precond_circulant(op, mesh, axis=0, x0=0.0, dx=1.0, first=1, count=0, kind="strang", stream=None):
    """Circulant preconditioner (kind "strang" or "chan") on regular slices first .. first+count-1
    (count = 0 removes it)."""
    c = Circulant(int(axis), float(x0), float(dx), int(first), int(count), {"strang": 0, "chan": 1}[kind])
    _check(lib().scabem_set_precond_circulant(op, mesh, C.byref(c), _stream(stream)))


def scabem_precond_apply(op, v, z, nrhs=1, ld=None, transpose=False, stream=None):
    """z = M^-1 v with the solver's preconditioner (complex128 device buffers)."""
    if ld is None:
        ld = v.shape[-1] if nrhs > 1 else v.shape[0]
    _check(lib().scabem_precond_apply(op, _ptr(v), _ptr(z), nrhs, ld, 1 if transpose else 0, _stream(stream)))


def scabem_fields_eh(op, x, pts, side=0, inc=None, nrhs=1, ld=None, stream=None):
    """(E, H) of the interior (side 0, plus inc) or exterior (side 1) current set at pts:
    two arrays (nrhs, npts, 3) complex128."""
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    if ld is None:
        ld = x.shape[0]
    E = np.zeros((nrhs, len(pts), 3), np.complex128)
    H = np.zeros_like(E)
    _check(lib().scabem_fields_eh(op, _ptr(x), nrhs, ld, _ptr(pts), len(pts), int(side),
                                  C.byref(inc) if inc else None, _ptr(E), _ptr(H), _stream(stream)))
    return E, H


def scabem_poynting_rate(op, x, xc, core, box, slab, n=10, inc=None, nrhs=1, ld=None, stream=None):
    """Decay rate by Poynting's theorem at x = xc: per right-hand side
    (alpha [1/um], loss per length, side flux per length, cross-section flux)."""
    if ld is None:
        ld = x.shape[0]
    pp = Poynting(float(xc), (C.c_double * 2)(*core), (C.c_double * 2)(*box), float(slab), int(n))
    out = np.zeros((nrhs, 4), np.float64)
    _check(lib().scabem_poynting_rate(op, _ptr(x), nrhs, ld, C.byref(pp), C.byref(inc) if inc else None, _ptr(out),
                                      _stream(stream)))
    return out


def scabem_reflection(op, x, axis, comp, p0, t0, t1, npts, beta_lo, beta_hi, nbeta, inc=None, nrhs=1, ld=None,
                      stream=None):
    if ld is None:
        ld = x.shape[0]
    pr = Probe(axis, comp, (C.c_double * 3)(*p0), t0, t1, npts, beta_lo, beta_hi, nbeta)
    out = np.zeros((nrhs, 6), np.float64)
    _check(lib().scabem_reflection(op, _ptr(x), nrhs, ld, C.byref(pr), C.byref(inc) if inc else None, _ptr(out),
                                   _stream(stream)))
    return out


def scabem_decay_fit(t, E, alpha_lo, alpha_hi, nalpha, beta_lo, beta_hi, nbeta, stream=None):
    """Decay-rate fit of samples E(t) (host arrays); returns
    {alpha, beta, relative residual, Re(c/a), Im(c/a), |a|}."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    E = np.ascontiguousarray(E, dtype=np.complex128)
    out = np.zeros(6, np.float64)
    _check(lib().scabem_decay_fit(t.ctypes.data, E.ctypes.data, len(t), alpha_lo, alpha_hi, nalpha, beta_lo,
                                  beta_hi, nbeta, out.ctypes.data, _stream(stream)))
    return out


def scabem_decay_rate(op, x, axis, comp, p0, t0, t1, npts, alpha_lo, alpha_hi, nalpha, beta_lo, beta_hi, nbeta,
                      inc=None, nrhs=1, ld=None, stream=None):
    """Decay-rate fit of the interior field component on a probe line, per right-hand side."""
    if ld is None:
        ld = x.shape[0]
    pr = Probe(axis, comp, (C.c_double * 3)(*p0), t0, t1, npts, beta_lo, beta_hi, nbeta)
    out = np.zeros((nrhs, 6), np.float64)
    _check(lib().scabem_decay_rate(op, _ptr(x), nrhs, ld, C.byref(pr), alpha_lo, alpha_hi, nalpha,
                                   C.byref(inc) if inc else None, _ptr(out), _stream(stream)))
    return out


STAGES = ["summaries", "projection", "fft_axis0_fwd", "fft_planes_green", "fft_axis0_inv", "points"]


def scabem_profile(op, enable=True, max_applies=1024):
    _check(lib().scabem_profile(op, int(bool(enable)), max_applies))


def scabem_profile_read(op):
    ms = np.zeros(len(STAGES), np.float64)
    n = C.c_int64()
    _check(lib().scabem_profile_read(op, _ptr(ms), C.byref(n)))
    return dict(zip(STAGES, ms.tolist())), n.value


def scabem_peak_fma(prec=SCABEM_C128, stream=None):
    """Measured FMA-pipe peak in TFLOP/s: FP64 (prec=SCABEM_C128) or packed FP32x2 (SCABEM_C64)."""
    v = C.c_double()
    _check(lib().scabem_peak_fma(int(prec), C.byref(v), _stream(stream)))
    return v.value


def scabem_last_error():
    return lib().scabem_last_error().decode()
