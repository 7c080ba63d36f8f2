"""GB300 (sm_103a) LIMEX stage solver for two-phase porous-media flow.

Thin ctypes binding of the C ABI in ``include/rf.h`` (``librf.so``, built
in-tree by ``paper_2506_04763_gb300.build``).  The functions ``rf_*`` keep the
ABI's names and only marshal arguments; every step of the path runs in the
library's CUDA kernels.  PyTorch supplies device memory (as the library's
allocator and for user tensors) and streams.  There is no CPU fallback: if the
library or a GPU is missing, the calls raise.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librf.so")

RF_OK, RF_EINVAL, RF_ENOMEM, RF_ECUDA, RF_ENOTCONV, RF_EBREAKDOWN, RF_ENONFINITE, RF_ETIMEOUT = range(8)
RF_SMOOTH_JACOBI, RF_SMOOTH_GS8 = 0, 1
RF_PREC_FP64, RF_PREC_FP32, RF_PREC_FP16 = 0, 1, 2
RF_OP_SPMV, RF_OP_VCYCLE, RF_OP_SMOOTH, RF_OP_RESIDUAL, RF_OP_RESTRICT, RF_OP_PROLONG, RF_OP_COARSE = range(7)
RF_NOALLOC_MAX_N = 512
RF_SCHEME_SHAT_STORAGE, RF_SCHEME_DARCY_UPWIND = 1, 2
PROF_CLASSES = ["spmv64", "smooth_fine", "resid_fine", "transfer", "coarse_levels", "vector"]


class RFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("rf status %d (%s): %s" % (status, _status_name(status), msg))
        self.status = status


def _status_name(s):
    return ["ok", "invalid argument", "out of memory", "CUDA error", "not converged", "breakdown",
            "non-finite", "timeout"][s] if 0 <= s < 8 else "unknown"


# ------------------------------------------------------------------ structs
class rf_grid_desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int64 * 3), ("h", ctypes.c_double * 3),
                ("g", ctypes.c_double * 3)]


class rf_fluids(ctypes.Structure):
    _fields_ = [("rho_w", ctypes.c_double), ("rho_n", ctypes.c_double), ("mu_w", ctypes.c_double),
                ("mu_n", ctypes.c_double)]


class rf_materials(ctypes.Structure):
    _fields_ = [("S_wr", ctypes.c_double), ("S_nr", ctypes.c_double), ("lam", ctypes.c_double),
                ("K", ctypes.c_void_p), ("phi", ctypes.c_void_p), ("pd", ctypes.c_void_p)]


class rf_bc(ctypes.Structure):
    _fields_ = [("dir_pw", ctypes.c_void_p), ("pw_dir", ctypes.c_void_p), ("q_in", ctypes.c_void_p)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class rf_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


class rf_gmg_opts(ctypes.Structure):
    _fields_ = [("nlevels", ctypes.c_int), ("smoother", ctypes.c_int), ("nu1", ctypes.c_int),
                ("nu2", ctypes.c_int), ("omega", ctypes.c_double), ("precision", ctypes.c_int),
                ("autotune", ctypes.c_int)]


RF_OUTER_FP64, RF_OUTER_DF32 = 0, 1
OUTERS = {"fp64": RF_OUTER_FP64, "df32": RF_OUTER_DF32}


class rf_solve_opts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_it", ctypes.c_int), ("outer", ctypes.c_int)]


class rf_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("relres", ctypes.c_double), ("status", ctypes.c_int),
                ("restarts", ctypes.c_int)]


class rf_limex_opts(ctypes.Structure):
    _fields_ = [("kappa", ctypes.c_int), ("tol", ctypes.c_double), ("rho", ctypes.c_double),
                ("fac_min", ctypes.c_double), ("fac_max", ctypes.c_double), ("gmg", rf_gmg_opts),
                ("solve", rf_solve_opts)]


class rf_limex_run_opts(ctypes.Structure):
    _fields_ = [("step", rf_limex_opts), ("t_end", ctypes.c_double), ("H_max", ctypes.c_double),
                ("max_steps", ctypes.c_int), ("max_rejects", ctypes.c_int), ("hold_after_reject", ctypes.c_int)]


class rf_limex_run_info(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("H_next", ctypes.c_double), ("accepted", ctypes.c_int),
                ("rejected", ctypes.c_int), ("solves", ctypes.c_int), ("iterations", ctypes.c_int),
                ("steps", ctypes.c_int), ("status", ctypes.c_int)]


class rf_ie_opts(ctypes.Structure):
    _fields_ = [("atol", ctypes.c_double), ("rtol", ctypes.c_double), ("max_newton", ctypes.c_int),
                ("gmg", rf_gmg_opts), ("solve", rf_solve_opts), ("max_ls", ctypes.c_int)]


class rf_ie_info(ctypes.Structure):
    _fields_ = [("newton", ctypes.c_int), ("linear", ctypes.c_int), ("res0", ctypes.c_double),
                ("res", ctypes.c_double), ("status", ctypes.c_int)]


class rf_limex_info(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("H_new", ctypes.c_double), ("accepted", ctypes.c_int),
                ("solves", ctypes.c_int), ("iterations", ctypes.c_int), ("status", ctypes.c_int)]


# exported symbols of include/rf.h and their signatures
_P, _I, _D, _I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
SIGNATURES = {
    "rf_grid_create": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "rf_grid_destroy": (None, [_P]),
    "rf_grid_nv": (_I64, [_P]),
    "rf_assemble": (_I, [_P, _P, _I, _P, _P]),
    "rf_grid_set_scheme": (_I, [_P, _I]),
    "rf_grid_set_kr_laws": (_I, [_P, _I, _P, _P, _P]),
    "rf_barrier_check": (_I, [_I, _I, _D, _P, _P]),
    "rf_gmg_setup": (_I, [_P, _P, _I, _P, _P]),
    "rf_solve": (_I, [_P, _I, _P, _P, _P, _P, _P]),
    "rf_limex_step": (_I, [_P, _P, _D, _P, _P, _P]),
    "rf_limex_step_batched": (_I, [_P, _P, _P, _I, _P, _P, _I, _P]),
    "rf_limex_run": (_I, [_P, _P, _D, _P, _P, _P, _I, _P]),
    "rf_ie_step": (_I, [_P, _P, _D, _P, _P, _P]),
    "rf_phase_mass": (_I, [_P, _P, _P, _P]),
    "rf_export_jacobian": (_I, [_P, _P, _P, _P]),
    "rf_export_level": (_I, [_P, _I, _I, _P, _P, _P]),
    "rf_export_rows": (_I, [_P, _P, _I, _P, _P, _P]),
    "rf_apply": (_I, [_P, _I, _I, _I, _P, _P, _P, _P]),
    "rf_dense_inverse_noalloc": (_I, [_I, _P, _P, _P]),
    "rf_profile": (_I, [_P, _I]),
    "rf_profile_read": (_I, [_P, _I, _P, _P, _P]),
    "rf_fp64_fma_rate": (_I, [_P, _P]),
    "rf_launch_count": (_I64, []),
    "rf_status_string": (ctypes.c_char_p, [_I]),
    "rf_last_error": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """Load librf.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("librf.so is not built: run `python -m paper_2506_04763_gb300.build` "
                               "(needs nvcc); this package has no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != RF_OK:
        raise RFError(status, lib().rf_last_error().decode(errors="replace"))


# ------------------------------------------------------------------ ABI wrappers (same names)
def rf_grid_create(desc, fluids, mat, bc, alloc, stream):
    h = ctypes.c_void_p()
    _check(lib().rf_grid_create(ctypes.byref(desc), ctypes.byref(fluids), ctypes.byref(mat),
                                ctypes.byref(bc) if bc is not None else None,
                                ctypes.byref(alloc) if alloc is not None else None, stream, ctypes.byref(h)))
    return h.value


def rf_grid_destroy(grid):
    lib().rf_grid_destroy(grid)


def rf_assemble(grid, u_ptr, want_jacobian, F_ptr, stream):
    _check(lib().rf_assemble(grid, u_ptr, int(want_jacobian), F_ptr, stream))


def rf_grid_set_scheme(grid, scheme):
    _check(lib().rf_grid_set_scheme(grid, int(scheme)))


def rf_grid_set_kr_laws(grid, laws, cell_law, stream=None):
    """laws: [nlaws, 6] rows {kind, a_w, n_w, a_n, b_n, c_n}; cell_law: one
    law index per cell (natural cell order).  laws=None: Brooks-Corey
    everywhere."""
    if laws is None:
        _check(lib().rf_grid_set_kr_laws(grid, 0, None, None, stream))
        return
    t = np.ascontiguousarray(np.asarray(laws, dtype=np.float64).reshape(-1, 6))
    c = np.ascontiguousarray(cell_law, dtype=np.uint8)
    _check(lib().rf_grid_set_kr_laws(grid, len(t), t.ctypes.data, c.ctypes.data, stream))


def rf_gmg_setup(grid, shifts, opts, stream):
    arr = (ctypes.c_double * len(shifts))(*[float(s) for s in shifts])
    _check(lib().rf_gmg_setup(grid, arr, len(shifts), ctypes.byref(opts), stream))


def rf_solve(grid, shift, b_ptr, x_ptr, opts, stream):
    info = rf_solve_info()
    st = lib().rf_solve(grid, int(shift), b_ptr, x_ptr, ctypes.byref(opts), ctypes.byref(info), stream)
    if st not in (RF_OK, RF_ENOTCONV):
        _check(st)
    return st, info


def rf_limex_step(grid, u_ptr, H, opts, stream):
    info = rf_limex_info()
    st = lib().rf_limex_step(grid, u_ptr, float(H), ctypes.byref(opts), ctypes.byref(info), stream)
    if st not in (RF_OK, RF_ENOTCONV):
        _check(st)
    return st, info


def rf_ie_step(grid, u_ptr, H, opts, stream):
    info = rf_ie_info()
    st = lib().rf_ie_step(grid, u_ptr, float(H), ctypes.byref(opts), ctypes.byref(info), stream)
    if st not in (RF_OK, RF_ENOTCONV):
        _check(st)
    return st, info


def rf_limex_step_batched(grids, u_ptrs, H, opts, max_concurrent, stream):
    n = len(grids)
    ga = (ctypes.c_void_p * n)(*grids)
    ua = (ctypes.c_void_p * n)(*u_ptrs)
    ha = (ctypes.c_double * n)(*[float(h) for h in H])
    oa = (rf_limex_opts * n)(*opts)
    infos = (rf_limex_info * n)()
    st = lib().rf_limex_step_batched(ga, ua, ha, n, oa, infos, int(max_concurrent), stream)
    if st not in (RF_OK, RF_ENOTCONV):
        _check(st)
    return st, list(infos)


def limex_step_batched(grids, us, H, kappa=4, tol=1e-3, rho=0.75, fac_min=0.2, fac_max=4.0, gmg=None, rtol=1e-10,
                       max_it=200, outer="fp64", max_concurrent=0, stream=None):
    """LIMEX steps of an ensemble of Grid objects, run concurrently by the
    library.  gmg: one rf_gmg_opts or a list (one per grid)."""
    n = len(grids)
    gm = gmg if isinstance(gmg, (list, tuple)) else [gmg if gmg is not None else gmg_opts(4)] * n
    Hs = H if isinstance(H, (list, tuple)) else [H] * n
    opts = [rf_limex_opts(int(kappa), float(tol), float(rho), float(fac_min), float(fac_max), gm[i],
                          rf_solve_opts(float(rtol), int(max_it), OUTERS.get(outer, outer))) for i in range(n)]
    st, infos = rf_limex_step_batched([g.handle for g in grids], [_ptr(u) for u in us], Hs, opts, max_concurrent,
                                      _stream_handle(stream))
    return st, [dict(status=i.status, eps=i.eps, H_new=i.H_new, accepted=i.accepted, solves=i.solves,
                     iterations=i.iterations) for i in infos]


def rf_export_jacobian(grid, J_host, md_host, stream):
    _check(lib().rf_export_jacobian(grid, J_host, md_host, stream))


def rf_export_level(grid, level, shift, A_host, dims_host, stream):
    _check(lib().rf_export_level(grid, int(level), int(shift), A_host, dims_host, stream))


def rf_apply(grid, op, level, shift, in0, in1, out, stream):
    _check(lib().rf_apply(grid, int(op), int(level), int(shift), in0, in1, out, stream))


def rf_profile(grid, enable):
    _check(lib().rf_profile(grid, int(enable)))


def rf_profile_read(grid, cls):
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    by = ctypes.c_double()
    _check(lib().rf_profile_read(grid, int(cls), ctypes.byref(ms), ctypes.byref(n), ctypes.byref(by)))
    return ms.value, n.value, by.value


def rf_barrier_check(rounds, extra=0, limit_s=1.0, stream=None):
    """Status of rf_barrier_check (not raised: RF_ETIMEOUT is the expected
    answer for extra=1) and the launch's block count."""
    nb = ctypes.c_int()
    st = lib().rf_barrier_check(int(rounds), int(extra), float(limit_s), ctypes.byref(nb), _stream_handle(stream))
    return int(st), nb.value


def rf_fp64_fma_rate(stream=None):
    """Measured FP64 FMA/s of the current GPU (rf_fp64_fma_rate)."""
    v = ctypes.c_double()
    _check(lib().rf_fp64_fma_rate(_stream_handle(stream), ctypes.byref(v)))
    return v.value


def rf_launch_count():
    return int(lib().rf_launch_count())


def rf_status_string(s):
    return lib().rf_status_string(int(s)).decode()


def rf_last_error():
    return lib().rf_last_error().decode(errors="replace")


# ------------------------------------------------------------------ convenience layer
def _ptr(a):
    """Device pointer of a torch tensor or host pointer of a numpy array (contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return a.data_ptr()


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _torch_allocator():
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0)
        except Exception:
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    a = rf_allocator(ALLOC_FN(_alloc), FREE_FN(_free), None)
    return a


SMOOTHERS = {"jacobi": RF_SMOOTH_JACOBI, "gs8": RF_SMOOTH_GS8, "gs": RF_SMOOTH_GS8}
PRECISIONS = {"fp64": RF_PREC_FP64, "fp32": RF_PREC_FP32, "fp16": RF_PREC_FP16}


def gmg_opts(nlevels, smoother="jacobi", nu1=2, nu2=2, omega=0.8, precision="fp32", autotune=False):
    return rf_gmg_opts(int(nlevels), SMOOTHERS.get(smoother, smoother), int(nu1), int(nu2), float(omega),
                       PRECISIONS.get(precision, precision), int(bool(autotune)))


class Grid:
    """A problem on the GPU.  ``prob`` is a dict as made by
    ``paper_2506_04763_gb300.inputs`` (grid, fluids, Brooks-Corey parameters,
    per-cell K/phi/p_d, Dirichlet mask and values, optional sources)."""

    def __init__(self, prob, allocator="torch", stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA GPU is required (no CPU fallback)")
        self.prob = prob
        self.dim = int(prob["dim"])
        self.n = tuple(int(t) for t in prob["n"])
        self.nv = self.n[0] * self.n[1] * self.n[2]
        self.nb = 27 if self.dim == 3 else 9
        self.stream = _stream_handle(stream)
        desc = rf_grid_desc(self.dim, (ctypes.c_int64 * 3)(*self.n), (ctypes.c_double * 3)(*prob["h"]),
                            (ctypes.c_double * 3)(*prob["g"]))
        fl = rf_fluids(prob["rho_w"], prob["rho_n"], prob["mu_w"], prob["mu_n"])
        keep = {k: np.ascontiguousarray(prob[k], np.float64) for k in ("K", "phi", "pd", "pw_dir")}
        keep["dir"] = np.ascontiguousarray(prob["dir"], np.uint8)
        keep["q_in"] = None if prob.get("q_in") is None else np.ascontiguousarray(prob["q_in"], np.float64)
        mat = rf_materials(prob["S_wr"], prob["S_nr"], prob["lam"], _ptr(keep["K"]), _ptr(keep["phi"]),
                           _ptr(keep["pd"]))
        bc = rf_bc(_ptr(keep["dir"]), _ptr(keep["pw_dir"]), _ptr(keep["q_in"]))
        # "torch": PyTorch's caching allocator; None: cudaMalloc; or an rf_allocator
        self._alloc = _torch_allocator() if allocator == "torch" else allocator
        self.handle = rf_grid_create(desc, fl, mat, bc, self._alloc, self.stream)
        if int(prob.get("scheme", 0)):
            self.set_scheme(prob["scheme"])
        if prob.get("kr_laws") is not None:
            self.set_kr_laws(prob["kr_laws"], prob["cell_law"])

    def close(self):
        if getattr(self, "handle", None):
            rf_grid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- wrappers over the ABI (tensors on the GPU, or numpy arrays on the host)
    def assemble(self, u, jacobian=True, F=None):
        rf_assemble(self.handle, _ptr(u), jacobian, _ptr(F), self.stream)
        return F

    def set_scheme(self, scheme):
        """Discretisation variant bits (SCHEME_SHAT_STORAGE, SCHEME_DARCY_UPWIND)."""
        rf_grid_set_scheme(self.handle, scheme)

    def set_kr_laws(self, laws, cell_law):
        """Per-medium relative permeability laws (rows {kind, a_w, n_w, a_n,
        b_n, c_n}) and each cell's law index; laws=None: Brooks-Corey."""
        rf_grid_set_kr_laws(self.handle, laws, cell_law, self.stream)

    def gmg_setup(self, shifts, opts):
        rf_gmg_setup(self.handle, list(shifts), opts, self.stream)

    def solve(self, shift, b, x, rtol=1e-10, max_it=200, outer="fp64"):
        o = rf_solve_opts(float(rtol), int(max_it), OUTERS.get(outer, outer))
        st, info = rf_solve(self.handle, shift, _ptr(b), _ptr(x), o, self.stream)
        return dict(status=st, iterations=info.iterations, relres=info.relres, restarts=info.restarts)

    def limex_step(self, u, H, kappa=4, tol=1e-3, rho=0.75, fac_min=0.2, fac_max=4.0, gmg=None, rtol=1e-10,
                   max_it=200, outer="fp64"):
        gmg = gmg if gmg is not None else gmg_opts(4)
        o = rf_limex_opts(int(kappa), float(tol), float(rho), float(fac_min), float(fac_max), gmg,
                          rf_solve_opts(float(rtol), int(max_it), OUTERS.get(outer, outer)))
        st, info = rf_limex_step(self.handle, _ptr(u), H, o, self.stream)
        return dict(status=st, eps=info.eps, H_new=info.H_new, accepted=info.accepted, solves=info.solves,
                    iterations=info.iterations)

    def ie_step(self, u, H, atol=1e-8, rtol=1e-6, max_newton=20, gmg=None, lin_rtol=1e-10, max_it=200,
                outer="fp64", max_ls=0):
        """One implicit Euler step solved by Newton's method (rf_ie_step)."""
        gmg = gmg if gmg is not None else gmg_opts(4)
        o = rf_ie_opts(float(atol), float(rtol), int(max_newton), gmg,
                       rf_solve_opts(float(lin_rtol), int(max_it), OUTERS.get(outer, outer)), int(max_ls))
        st, info = rf_ie_step(self.handle, _ptr(u), H, o, self.stream)
        return dict(status=st, newton=info.newton, linear=info.linear, res0=info.res0, res=info.res)

    def limex_run(self, u, H0, steps=None, tol=1e-3, rho=0.75, H_max=None, gmg=None, rtol=1e-10, max_it=200,
                  outer="fp64", kappa=4, max_rejects=50, t_end=None, hold_after_reject=True, hist_cap=100000,
                  fac_min=0.2, fac_max=4.0):
        """Adaptive LIMEX integration (rf_limex_run): `steps` accepted steps
        and/or up to time `t_end`, from state u (updated in place).  Returns
        (t, history) with one dict per attempted step (H, eps, accepted)."""
        if steps is None and t_end is None:
            raise ValueError("give steps or t_end")
        gmg = gmg if gmg is not None else gmg_opts(4)
        step = rf_limex_opts(int(kappa), float(tol), float(rho), float(fac_min), float(fac_max), gmg,
                             rf_solve_opts(float(rtol), int(max_it), OUTERS.get(outer, outer)))
        o = rf_limex_run_opts(step, float(t_end or 0.0), float(H_max or 0.0), int(steps or 0), int(max_rejects),
                              int(bool(hold_after_reject)))
        info = rf_limex_run_info()
        hist = np.zeros((int(hist_cap), 3))
        st = lib().rf_limex_run(self.handle, _ptr(u), float(H0), ctypes.byref(o), ctypes.byref(info), _ptr(hist),
                                int(hist_cap), self.stream)
        if st == RF_ENOTCONV and info.rejected > max_rejects:
            raise RuntimeError("LIMEX: more than %d rejected steps" % max_rejects)
        if st not in (RF_OK, RF_ENOTCONV):
            _check(st)
        n = min(info.steps, int(hist_cap))
        self.last_run = dict(t=info.t, H_next=info.H_next, accepted=info.accepted, rejected=info.rejected,
                             solves=info.solves, iterations=info.iterations, steps=info.steps, status=st)
        return info.t, [dict(H=float(h[0]), eps=float(h[1]), accepted=int(h[2])) for h in hist[:n]]

    def phase_mass(self, u):
        """(water, NAPL) mass in kg of state u (lumped storage)."""
        out = np.zeros(2)
        _check(lib().rf_phase_mass(self.handle, _ptr(u), _ptr(out), self.stream))
        return float(out[0]), float(out[1])

    def profile(self, enable):
        rf_profile(self.handle, enable)

    def profile_read(self):
        return {name: dict(zip(("ms", "launches", "bytes"), rf_profile_read(self.handle, c)))
                for c, name in enumerate(PROF_CLASSES)}

    def export_jacobian(self):
        J = np.zeros((self.nv, self.nb, 4))
        md = np.zeros((self.nv, 2))
        rf_export_jacobian(self.handle, _ptr(J), _ptr(md), self.stream)
        return J, md

    def export_rows(self, vertices):
        v = np.ascontiguousarray(vertices, dtype=np.int64)
        J = np.zeros((len(v), self.nb, 4))
        md = np.zeros((len(v), 2))
        _check(lib().rf_export_rows(self.handle, _ptr(v), len(v), _ptr(J), _ptr(md), self.stream))
        return J, md

    def export_level(self, level, shift):
        dims = (ctypes.c_int64 * 3)()
        # size of the level first: at most nv
        buf = np.zeros(self.nv * self.nb * 4)
        rf_export_level(self.handle, level, shift, _ptr(buf), ctypes.addressof(dims), self.stream)
        n = tuple(int(t) for t in dims)
        nvl = n[0] * n[1] * n[2]
        return buf[:nvl * self.nb * 4].reshape(nvl, self.nb, 4).copy(), n

    def apply(self, op, level, shift, in0, in1=None, out_len=None):
        in0 = np.ascontiguousarray(in0, np.float64)
        in1 = None if in1 is None else np.ascontiguousarray(in1, np.float64)
        out = np.zeros(out_len if out_len is not None else 2 * self.nv)
        rf_apply(self.handle, op, level, shift, _ptr(in0), _ptr(in1), _ptr(out), self.stream)
        return out
