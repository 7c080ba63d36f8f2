"""ORACLE — test infrastructure only.

A plain FP64 CPU restatement (``rfo.c``) of the paper's discrete two-phase
model, its BiCGSTAB + geometric-multigrid stage solver and the LIMEX step
(arXiv 2506.04763, Secs. 2-5).  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / reference leg of ``bench.py`` may import this
package.  It shares no code with the CUDA library; the two meet only through
plain arrays in the natural vertex order documented in ``rfo.h``.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rfo.c")
_HDR = os.path.join(_HERE, "rfo.h")
_SO = os.path.join(_HERE, "librfo.so")

JACOBI, GS8 = 0, 1


def build(force=False):
    """Compile the oracle with gcc (no contraction of a*b+c into fma)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        # idle OpenMP threads sleep instead of spinning, so that two processes
        # running the oracle at once do not starve each other
        os.environ.setdefault("OMP_WAIT_POLICY", "PASSIVE")
        _lib = ctypes.CDLL(_SO)
        _declare(_lib)
    return _lib


class _Model(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("h", ctypes.c_double * 3),
                ("g", ctypes.c_double * 3), ("rho_w", ctypes.c_double), ("rho_n", ctypes.c_double),
                ("mu_w", ctypes.c_double), ("mu_n", ctypes.c_double), ("S_wr", ctypes.c_double),
                ("S_nr", ctypes.c_double), ("lam", ctypes.c_double),
                ("K", ctypes.c_void_p), ("phi", ctypes.c_void_p), ("pd", ctypes.c_void_p),
                ("dir", ctypes.c_void_p), ("pw_dir", ctypes.c_void_p), ("q_in", ctypes.c_void_p),
                ("scheme", ctypes.c_int), ("nlaws", ctypes.c_int), ("kr_laws", ctypes.c_void_p),
                ("cell_law", ctypes.c_void_p)]

KR_BROOKS_COREY, KR_POLY = 0, 1


class _LimexOpts(ctypes.Structure):
    _fields_ = [("kappa", ctypes.c_int), ("tol", ctypes.c_double), ("rho", ctypes.c_double),
                ("fac_min", ctypes.c_double), ("fac_max", ctypes.c_double), ("nlevels", ctypes.c_int),
                ("smoother", ctypes.c_int), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("omega", ctypes.c_double), ("rtol", ctypes.c_double), ("maxit", ctypes.c_int)]


class _LimexInfo(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("H_new", ctypes.c_double), ("accepted", ctypes.c_int),
                ("solves", ctypes.c_int), ("iterations", ctypes.c_int)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double


def _declare(L):
    sig = {
        "rfo_set_threads": (None, [_I]),
        "rfo_get_threads": (_I, []),
        "rfo_brooks_corey": (None, [_P, _D, _P]),
        "rfo_shat": (None, [_P, _D, _D, _D, _P]),
        "rfo_kr_law": (None, [_P, _I, _D, _P]),
        "rfo_pdmin": (None, [_P, _P]),
        "rfo_phiv": (None, [_P, _P]),
        "rfo_assemble": (None, [_P, _P, _P, _P, _P]),
        "rfo_storage": (None, [_P, _P, _P]),
        "rfo_ie_step": (_I, [_P, _P, _D, _P, _P, _P]),
        "rfo_make_A": (None, [_I, _I, _P, _P, _D, _P]),
        "rfo_spmv": (None, [_I, _P, _P, _P, _P]),
        "rfo_residual": (None, [_I, _P, _P, _P, _P, _P]),
        "rfo_jacobi": (None, [_I, _P, _P, _P, _P, _P, _D]),
        "rfo_gs_sweep": (None, [_I, _P, _P, _P, _P, _I]),
        "rfo_restrict": (None, [_I, _P, _P, _P, _P, _P, _P]),
        "rfo_prolong_add": (None, [_I, _P, _P, _P, _P, _P, _P]),
        "rfo_galerkin": (None, [_I, _P, _P, _P, _P, _P, _P]),
        "rfo_lu_factor": (_I, [_I, _P, _P]),
        "rfo_lu_solve": (None, [_I, _P, _P, _P]),
        "rfo_gmg_create": (_P, [_I, _P, _P, _P, _I, _I, _I, _I, _D]),
        "rfo_gmg_free": (None, [_P]),
        "rfo_gmg_nlevels": (_I, [_P]),
        "rfo_gmg_level_dims": (None, [_P, _I, _P]),
        "rfo_gmg_level_matrix": (None, [_P, _I, _P]),
        "rfo_gmg_vcycle": (None, [_P, _P, _P]),
        "rfo_gmg32_create": (_P, [_P]),
        "rfo_gmg32_free": (None, [_P]),
        "rfo_gmg32_vcycle": (None, [_P, _P, _P]),
        "rfo_bicgstab": (_I, [_I, _P, _P, _P, _P, _P, _D, _I, _P, _P]),
        "rfo_extrapolate": (None, [_I, _P, _I, _P, _P, _P]),
        "rfo_h1_seminorm2": (_D, [_I, _P, _P, _P, _I]),
        "rfo_lumped_l2norm2": (_D, [_I, _P, _P, _P, _I]),
        "rfo_limex_step": (_I, [_P, _P, _D, _P, _P, _P]),
        "rfo_limex_run": (_I, [_P, _P, _D, _P, _P, _P, _P, _I]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _dims(n):
    return (ctypes.c_int * 3)(*[int(t) for t in n])


class Model:
    """Holds a problem description (the dict made by ``inputs``) as a C struct."""

    def __init__(self, prob):
        self.prob = prob
        self.dim = int(prob["dim"])
        self.n = tuple(int(t) for t in prob["n"])
        self.nv = self.n[0] * self.n[1] * self.n[2]
        self.nb = 27 if self.dim == 3 else 9
        self._keep = {k: _f64(prob[k]) for k in ("K", "phi", "pd", "pw_dir")}
        self._keep["dir"] = np.ascontiguousarray(prob["dir"], dtype=np.uint8)
        q = prob.get("q_in")
        self._keep["q_in"] = _f64(q) if q is not None else None
        s = _Model()
        s.dim = self.dim
        s.n = (ctypes.c_int * 3)(*self.n)
        s.h = (ctypes.c_double * 3)(*[float(t) for t in prob["h"]])
        s.g = (ctypes.c_double * 3)(*[float(t) for t in prob["g"]])
        for k in ("rho_w", "rho_n", "mu_w", "mu_n", "S_wr", "S_nr"):
            setattr(s, k, float(prob[k]))
        s.lam = float(prob["lam"])
        for k in ("K", "phi", "pd", "dir", "pw_dir", "q_in"):
            setattr(s, k, _p(self._keep[k]))
        s.scheme = int(prob.get("scheme", 0))
        laws = prob.get("kr_laws")
        if laws is not None:
            self._keep["kr_laws"] = _f64(np.asarray(laws, dtype=np.float64).reshape(-1, 6))
            self._keep["cell_law"] = np.ascontiguousarray(prob["cell_law"], dtype=np.uint8)
            s.nlaws = len(self._keep["kr_laws"])
            s.kr_laws = _p(self._keep["kr_laws"])
            s.cell_law = _p(self._keep["cell_law"])
        self.s = s

    @property
    def ref(self):
        return ctypes.byref(self.s)


def set_threads(n):
    """OpenMP threads of the oracle's per-vertex loops (results are bitwise
    the same for any count)."""
    lib().rfo_set_threads(int(n))


def get_threads():
    return int(lib().rfo_get_threads())


def brooks_corey(model, Se):
    out = np.zeros(6)
    lib().rfo_brooks_corey(model.ref, float(Se), _p(out))
    return out


def kr_law(model, cell, Se):
    """(k_rw, dk_rw/dS_e, k_rn, dk_rn/dS_e) of the medium of `cell`."""
    out = np.zeros(4)
    lib().rfo_kr_law(model.ref, int(cell), float(Se), _p(out))
    return out


def shat(model, Se, pd_cell, pdmin):
    out = np.zeros(2)
    lib().rfo_shat(model.ref, float(Se), float(pd_cell), float(pdmin), _p(out))
    return out


def pdmin(model):
    out = np.zeros(model.nv)
    lib().rfo_pdmin(model.ref, _p(out))
    return out


def phiv(model):
    out = np.zeros(model.nv)
    lib().rfo_phiv(model.ref, _p(out))
    return out


def storage(model, u):
    """Storage terms [nv, 2] = (m_w, m_n) per vertex (kg)."""
    u = _f64(u)
    out = np.zeros((model.nv, 2))
    lib().rfo_storage(model.ref, _p(u), _p(out))
    return out


def assemble(model, u, jacobian=True):
    """Returns (F [2nv], J [nv, nb, 4] or None, mdiag [nv, 2] or None)."""
    u = _f64(u)
    F = np.zeros(2 * model.nv)
    J = np.zeros((model.nv, model.nb, 4)) if jacobian else None
    md = np.zeros((model.nv, 2)) if jacobian else None
    lib().rfo_assemble(model.ref, _p(u), _p(F), _p(J), _p(md))
    return F, J, md


def make_A(J, mdiag, shift):
    J = _f64(J)
    A = np.zeros_like(J)
    lib().rfo_make_A(J.shape[0], J.shape[1], _p(J), _p(_f64(mdiag)), float(shift), _p(A))
    return A


def spmv(dim, n, A, x):
    x = _f64(x)
    y = np.zeros_like(x)
    lib().rfo_spmv(dim, _dims(n), _p(_f64(A)), _p(x), _p(y))
    return y


def residual(dim, n, A, b, x):
    r = np.zeros(len(b))
    lib().rfo_residual(dim, _dims(n), _p(_f64(A)), _p(_f64(b)), _p(_f64(x)), _p(r))
    return r


def jacobi(dim, n, A, b, x, omega):
    out = np.zeros(len(b))
    lib().rfo_jacobi(dim, _dims(n), _p(_f64(A)), _p(_f64(b)), _p(_f64(x)), _p(out), float(omega))
    return out


def gs_sweep(dim, n, A, b, x, forward=True):
    x = _f64(x).copy()
    lib().rfo_gs_sweep(dim, _dims(n), _p(_f64(A)), _p(_f64(b)), _p(x), int(bool(forward)))
    return x


def restrict(dim, nf, dmf, nc, dmc, r):
    out = np.zeros(2 * int(np.prod(nc)))
    lib().rfo_restrict(dim, _dims(nf), _p(np.ascontiguousarray(dmf, np.uint8)), _dims(nc),
                       _p(np.ascontiguousarray(dmc, np.uint8)), _p(_f64(r)), _p(out))
    return out


def prolong_add(dim, nf, dmf, nc, dmc, xc, xf):
    xf = _f64(xf).copy()
    lib().rfo_prolong_add(dim, _dims(nf), _p(np.ascontiguousarray(dmf, np.uint8)), _dims(nc),
                          _p(np.ascontiguousarray(dmc, np.uint8)), _p(_f64(xc)), _p(xf))
    return xf


def galerkin(dim, nf, dmf, Af, nc, dmc):
    nb = 27 if dim == 3 else 9
    Ac = np.zeros((int(np.prod(nc)), nb, 4))
    lib().rfo_galerkin(dim, _dims(nf), _p(np.ascontiguousarray(dmf, np.uint8)), _p(_f64(Af)),
                       _dims(nc), _p(np.ascontiguousarray(dmc, np.uint8)), _p(Ac))
    return Ac


def lu_solve_dense(M, b):
    M = _f64(M).copy()
    N = M.shape[0]
    piv = np.zeros(N, dtype=np.int32)
    rc = lib().rfo_lu_factor(N, _p(M), _p(piv))
    if rc != 0:
        raise np.linalg.LinAlgError("singular")
    x = _f64(b).copy()
    lib().rfo_lu_solve(N, _p(M), _p(piv), _p(x))
    return x


class GMG:
    def __init__(self, dim, n, A0, dmask, nlevels, smoother=JACOBI, nu1=2, nu2=2, omega=0.8):
        self.dim, self.n = dim, tuple(n)
        self._A0 = _f64(A0)
        self._dm = np.ascontiguousarray(dmask, np.uint8)
        self.h = lib().rfo_gmg_create(dim, _dims(n), _p(self._A0), _p(self._dm), int(nlevels),
                                      int(smoother), int(nu1), int(nu2), float(omega))

    def __del__(self):
        if getattr(self, "h", None):
            lib().rfo_gmg_free(self.h)
            self.h = None

    @property
    def nlevels(self):
        return lib().rfo_gmg_nlevels(self.h)

    def level_dims(self, level):
        n = (ctypes.c_int * 3)()
        lib().rfo_gmg_level_dims(self.h, level, n)
        return tuple(n)

    def level_matrix(self, level):
        n = self.level_dims(level)
        nb = 27 if self.dim == 3 else 9
        A = np.zeros((int(np.prod(n)), nb, 4))
        lib().rfo_gmg_level_matrix(self.h, level, _p(A))
        return A

    def vcycle(self, b):
        x = np.zeros(len(b))
        lib().rfo_gmg_vcycle(self.h, _p(_f64(b)), _p(x))
        return x


class GMG32:
    """FP32 emulation of a GMG hierarchy's V-cycle (float storage and sums)."""

    def __init__(self, gmg):
        self.gmg = gmg   # keeps the double hierarchy alive
        self.h = lib().rfo_gmg32_create(gmg.h)

    def __del__(self):
        if getattr(self, "h", None):
            lib().rfo_gmg32_free(self.h)
            self.h = None

    def vcycle(self, b):
        b32 = np.ascontiguousarray(b, dtype=np.float32)
        x = np.zeros(len(b32), dtype=np.float32)
        lib().rfo_gmg32_vcycle(self.h, _p(b32), _p(x))
        return x.astype(np.float64)


def bicgstab(dim, n, A, gmg, b, rtol=1e-10, maxit=200):
    x = np.zeros(len(b))
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = lib().rfo_bicgstab(dim, _dims(n), _p(_f64(A)), gmg.h if gmg is not None else None,
                            _p(_f64(b)), _p(x), float(rtol), int(maxit), ctypes.byref(it), ctypes.byref(rr))
    return x, dict(status=st, iterations=it.value, relres=rr.value)


def extrapolate(T1, nseq):
    T1 = _f64(T1)
    kappa, length = T1.shape
    ns = np.ascontiguousarray(nseq, dtype=np.int32)
    Tkk = np.zeros(length)
    Tkk1 = np.zeros(length)
    lib().rfo_extrapolate(kappa, _p(ns), length, _p(T1), _p(Tkk), _p(Tkk1))
    return Tkk, Tkk1


def h1_seminorm2(dim, n, h, q, stride=1):
    return lib().rfo_h1_seminorm2(dim, _dims(n), _p(_f64(h)), _p(_f64(q)), int(stride))


def lumped_l2norm2(dim, n, h, q, stride=1):
    return lib().rfo_lumped_l2norm2(dim, _dims(n), _p(_f64(h)), _p(_f64(q)), int(stride))


def limex_step(model, u0, H, kappa=4, tol=1e-3, rho=0.75, fac_min=0.2, fac_max=4.0, nlevels=4,
               smoother=JACOBI, nu1=2, nu2=2, omega=0.8, rtol=1e-10, maxit=200):
    o = _LimexOpts(kappa, tol, rho, fac_min, fac_max, nlevels, smoother, nu1, nu2, omega, rtol, maxit)
    info = _LimexInfo()
    u_out = np.zeros(2 * model.nv)
    st = lib().rfo_limex_step(model.ref, _p(_f64(u0)), float(H), ctypes.byref(o), _p(u_out), ctypes.byref(info))
    return u_out, dict(status=st, eps=info.eps, H_new=info.H_new, accepted=info.accepted,
                       solves=info.solves, iterations=info.iterations)


class _LimexRunOpts(ctypes.Structure):
    _fields_ = [("step", _LimexOpts), ("t_end", ctypes.c_double), ("H_max", ctypes.c_double),
                ("max_steps", ctypes.c_int), ("max_rejects", ctypes.c_int), ("hold_after_reject", ctypes.c_int)]


class _LimexRunInfo(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("H_next", ctypes.c_double), ("accepted", ctypes.c_int),
                ("rejected", ctypes.c_int), ("solves", ctypes.c_int), ("iterations", ctypes.c_int),
                ("steps", ctypes.c_int)]


def limex_run(model, u0, H0, steps=0, t_end=0.0, H_max=0.0, max_rejects=50, hold_after_reject=True, kappa=4,
              tol=1e-3, rho=0.75, fac_min=0.2, fac_max=4.0, nlevels=4, smoother=JACOBI, nu1=2, nu2=2, omega=0.8,
              rtol=1e-10, maxit=200, hist_cap=1000):
    """Adaptive LIMEX integration (rfo_limex_run): returns (u, info, history)
    with history rows (H, eps, accepted) per attempted step."""
    o = _LimexRunOpts(_LimexOpts(kappa, tol, rho, fac_min, fac_max, nlevels, smoother, nu1, nu2, omega, rtol, maxit),
                      float(t_end), float(H_max), int(steps), int(max_rejects), int(bool(hold_after_reject)))
    info = _LimexRunInfo()
    u_out = np.zeros(2 * model.nv)
    hist = np.zeros((hist_cap, 3))
    st = lib().rfo_limex_run(model.ref, _p(_f64(u0)), float(H0), ctypes.byref(o), _p(u_out), ctypes.byref(info),
                             _p(hist), int(hist_cap))
    n = min(info.steps, hist_cap)
    return u_out, dict(status=st, t=info.t, H_next=info.H_next, accepted=info.accepted, rejected=info.rejected,
                       solves=info.solves, iterations=info.iterations, steps=info.steps), hist[:n].copy()


class _IeOpts(ctypes.Structure):
    _fields_ = [("atol", ctypes.c_double), ("rtol", ctypes.c_double), ("max_newton", ctypes.c_int),
                ("nlevels", ctypes.c_int), ("smoother", ctypes.c_int), ("nu1", ctypes.c_int),
                ("nu2", ctypes.c_int), ("omega", ctypes.c_double), ("lin_rtol", ctypes.c_double),
                ("lin_maxit", ctypes.c_int), ("max_ls", ctypes.c_int)]


class _IeInfo(ctypes.Structure):
    _fields_ = [("newton", ctypes.c_int), ("linear", ctypes.c_int), ("res0", ctypes.c_double),
                ("res", ctypes.c_double)]


def ie_step(model, u_old, H, atol=1e-8, rtol=1e-6, max_newton=20, nlevels=4, smoother=JACOBI, nu1=2, nu2=2,
            omega=0.8, lin_rtol=1e-10, lin_maxit=400, max_ls=0):
    """One implicit Euler step solved by Newton's method (rfo_ie_step)."""
    o = _IeOpts(atol, rtol, max_newton, nlevels, smoother, nu1, nu2, omega, lin_rtol, lin_maxit, max_ls)
    info = _IeInfo()
    u_out = np.zeros(2 * model.nv)
    st = lib().rfo_ie_step(model.ref, _p(_f64(u_old)), float(H), ctypes.byref(o), _p(u_out), ctypes.byref(info))
    return u_out, dict(status=st, newton=info.newton, linear=info.linear, res0=info.res0, res=info.res)
