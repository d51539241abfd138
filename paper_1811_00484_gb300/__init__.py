"""Python binding of libvie, the Tucker-compressed FFT-VIE library.

Argument marshalling only: every array operation runs in the CUDA library
behind ``include/vie.h`` (loaded with ctypes from this package directory).
PyTorch supplies device memory and the current CUDA stream.  There is no
CPU path: without ``libvie.so`` the import fails, and without a GPU every
compute call fails.

Arrays are torch tensors on the GPU, C-contiguous, complex64 (the FP32
path) or complex128 (the FP64 path):
  vector fields  [B, 3, n1, n2, n3]   (a leading B may be omitted for B = 1)
  scalar fields  [n1, n2, n3]
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvie.so")

VIE_OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "out of memory",
          4: "no convergence", 5: "numerical failure", 6: "device wait timed out"}
VIE_C64, VIE_C128 = 0, 1
PATHS = {"tucker": 0, "uncompressed": 1, "tucker_cp": 2}
RANK_RULES = {"tail": 0, "sigma_max": 1}
VIE_STORE_UNCOMPRESSED, VIE_SELF_TERM_PV, VIE_REBUILD_SIMT, VIE_SETUP_FACTORWISE = 1, 2, 4, 8
VIE_REBUILD_TCGEN05 = 16
REBUILD_KERNELS = {0: "in_cta", 1: "simt", 2: "mma_sync", 3: "tcgen05"}
VIE_SOLVE_ADJOINT, VIE_SOLVE_RHS_INCIDENT, VIE_SOLVE_X0 = 1, 2, 4
COMPONENTS = ("xx", "xy", "xz", "yy", "yz", "zz")

# every symbol include/vie.h declares
EXPORTS = ("vie_tucker_compress", "vie_op_info", "vie_op_export", "vie_green_spectrum",
           "vie_reserve", "vie_matvec", "vie_matvec_adjoint", "vie_apply_system",
           "vie_total_field", "vie_solve", "vie_contrast_gradient", "vie_incident_dipole",
           "vie_destroy", "vie_status_string", "vie_last_error", "vie_profile_start",
           "vie_profile_stop", "vie_matvec_noalloc", "vie_matvec_multi", "vie_autotune",
           "vie_solve_multi", "vie_tucker_cp", "vie_cp_export", "vie_selftest_bounded_wait",
           "vie_matvec_multi_ex")


class VieError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))


class Grid(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_int), ("n2", ctypes.c_int), ("n3", ctypes.c_int),
                ("h", ctypes.c_double), ("freq_hz", ctypes.c_double)]


class OpInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("P", ctypes.c_int * 3), ("ranks", (ctypes.c_int * 3) * 6),
                ("tucker_bytes", ctypes.c_size_t), ("tucker_bytes_full", ctypes.c_size_t),
                ("slab_bytes", ctypes.c_size_t), ("rebuild_scratch_bytes", ctypes.c_size_t),
                ("uncompressed_bytes", ctypes.c_size_t), ("workspace_bytes", ctypes.c_size_t),
                ("has_uncompressed", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("line_threads", ctypes.c_int * 4), ("tuned_batch", ctypes.c_int),
                ("rebuild_kernel", ctypes.c_int), ("cp_rank", ctypes.c_int),
                ("cp_rel_err", ctypes.c_double * 6), ("cp_sweeps", ctypes.c_int * 6),
                ("cp_bytes", ctypes.c_size_t), ("device_bytes_tucker", ctypes.c_size_t),
                ("device_bytes_spectra", ctypes.c_size_t), ("matvec_workspace_bytes", ctypes.c_size_t),
                ("solver_workspace_bytes", ctypes.c_size_t), ("setup_scratch_bytes", ctypes.c_size_t),
                ("rebuild_tiles", ctypes.c_int * 2)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int), ("max_outer", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_refine", ctypes.c_int), ("path", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("refine", ctypes.c_int), ("orth", ctypes.c_int)]


class ProfileEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_longlong),
                ("ms", ctypes.c_double), ("bytes", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("converged", ctypes.c_int), ("refine_steps", ctypes.c_int),
                ("iterations", ctypes.c_int), ("matvecs", ctypes.c_int),
                ("relres", ctypes.c_double), ("history", ctypes.c_double * 65)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python paper_1811_00484_gb300/build.py`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, ci, cd = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    pd = ctypes.POINTER(ctypes.c_double)
    sig = {
        "vie_tucker_compress": [ctypes.POINTER(Grid), cd, ci, ci, vp, ctypes.POINTER(vp)],
        "vie_op_info": [vp, ctypes.POINTER(OpInfo)],
        "vie_op_export": [vp, ci, pd, pd, pd, pd, pd, pd, pd, vp],
        "vie_green_spectrum": [ctypes.POINTER(Grid), ci, ci, vp, vp],
        "vie_reserve": [vp, ci],
        "vie_matvec": [vp, vp, vp, ci, ci, ci, vp],
        "vie_matvec_adjoint": [vp, vp, vp, ci, ci, ci, vp],
        "vie_matvec_noalloc": [vp, vp, vp, ci, vp],
        "vie_matvec_multi": [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                             ctypes.POINTER(ci), ci, vp],
        "vie_matvec_multi_ex": [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                ctypes.POINTER(ci), ci, ci, vp],
        "vie_autotune": [vp, ci, vp],
        "vie_tucker_cp": [vp, ci, cd, ci, ctypes.c_ulonglong, vp],
        "vie_cp_export": [vp, ci, pd, pd, pd, pd, ctypes.POINTER(ci), vp],
        "vie_solve_multi": [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                            ctypes.POINTER(vp), ctypes.POINTER(ci), ci, ci, ci,
                            ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), vp],
        "vie_apply_system": [vp, vp, vp, vp, ci, ci, ci, ci, vp],
        "vie_total_field": [vp, vp, vp, vp, ci, ci, ci, vp],
        "vie_solve": [vp, vp, vp, vp, ci, ci, ci, ctypes.POINTER(SolveOpts),
                      ctypes.POINTER(SolveInfo), vp],
        "vie_contrast_gradient": [vp, vp, vp, vp, ci, cd, ci, vp],
        "vie_incident_dipole": [vp, pd, ci, vp, ci, vp],
        "vie_destroy": [vp],
        "vie_profile_start": [ctypes.c_uint],
        "vie_profile_stop": [ctypes.POINTER(ProfileEntry), ci, ctypes.POINTER(ci)],
        "vie_status_string": [ci],
        "vie_selftest_bounded_wait": [ci, cd, vp],
        "vie_last_error": [],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ci
    lib.vie_destroy.restype = None
    lib.vie_status_string.restype = ctypes.c_char_p
    lib.vie_last_error.restype = ctypes.c_char_p
    return lib


lib = _load()


def _check(status, where):
    if status != VIE_OK:
        detail = lib.vie_last_error().decode(errors="replace")
        raise VieError(status, where, detail)


def _torch():
    import torch
    return torch


def _stream():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _precision(t):
    torch = _torch()
    if t.dtype == torch.complex64:
        return VIE_C64
    if t.dtype == torch.complex128:
        return VIE_C128
    raise TypeError(f"expected complex64 or complex128, got {t.dtype}")


def _dev(t, name, shape_tail=None):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape_tail is not None and tuple(t.shape[-len(shape_tail):]) != tuple(shape_tail):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected [..., {shape_tail}]")
    return ctypes.c_void_p(t.data_ptr())


def _batch(t, n):
    if t.dim() == 4:
        return 1
    if t.dim() == 5:
        return t.shape[0]
    raise ValueError(f"vector field must be [3, {n}] or [B, 3, {n}]")


class Operator:
    """The compressed J-block operator of a uniform grid (vie_tucker_compress)."""

    def __init__(self, n, h, freq_hz, tol, rank_rule="tail", store_uncompressed=False,
                 self_term="full", rebuild="tensor_cores", setup="spectrum"):
        # "tensor_cores" (= "mma_sync"): warp-level mma.sync; "tcgen05": tcgen05.mma
        # with TMEM accumulators where the grid fits it; "simt": FP32 FMAs
        if rebuild not in ("tensor_cores", "mma_sync", "tcgen05", "simt"):
            raise ValueError("rebuild must be 'tensor_cores', 'mma_sync', 'tcgen05' or 'simt'")
        if setup not in ("spectrum", "factorwise"):
            raise ValueError("setup must be 'spectrum' or 'factorwise'")
        if isinstance(n, int):
            n = (n, n, n)
        self.n = tuple(int(v) for v in n)
        self.h, self.freq_hz, self.tol = float(h), float(freq_hz), float(tol)
        self._grid = Grid(self.n[0], self.n[1], self.n[2], self.h, self.freq_hz)
        flags = (VIE_STORE_UNCOMPRESSED if store_uncompressed else 0) | \
                (VIE_SELF_TERM_PV if self_term == "pv" else 0) | \
                (VIE_REBUILD_SIMT if rebuild == "simt" else 0) | \
                (VIE_REBUILD_TCGEN05 if rebuild == "tcgen05" else 0) | \
                (VIE_SETUP_FACTORWISE if setup == "factorwise" else 0)
        handle = ctypes.c_void_p()
        _check(lib.vie_tucker_compress(ctypes.byref(self._grid), self.tol, RANK_RULES[rank_rule],
                                       flags, _stream(), ctypes.byref(handle)),
               "vie_tucker_compress")
        self._h = handle

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib.vie_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- introspection -----------------------------------------------------
    def info(self):
        inf = OpInfo()
        _check(lib.vie_op_info(self._h, ctypes.byref(inf)), "vie_op_info")
        return {"n": tuple(inf.n), "P": tuple(inf.P),
                "ranks": [tuple(inf.ranks[c]) for c in range(6)],
                "tucker_bytes": inf.tucker_bytes, "tucker_bytes_full": inf.tucker_bytes_full,
                "slab_bytes": inf.slab_bytes, "rebuild_scratch_bytes": inf.rebuild_scratch_bytes,
                "uncompressed_bytes": inf.uncompressed_bytes,
                "workspace_bytes": inf.workspace_bytes,
                "has_uncompressed": bool(inf.has_uncompressed), "max_batch": inf.max_batch,
                "line_threads": tuple(inf.line_threads), "tuned_batch": inf.tuned_batch,
                "rebuild_kernel": REBUILD_KERNELS[inf.rebuild_kernel],
                "cp_rank": inf.cp_rank, "cp_rel_err": tuple(inf.cp_rel_err),
                "cp_sweeps": tuple(inf.cp_sweeps), "cp_bytes": inf.cp_bytes,
                "device_bytes_tucker": inf.device_bytes_tucker,
                "device_bytes_spectra": inf.device_bytes_spectra,
                "matvec_workspace_bytes": inf.matvec_workspace_bytes,
                "solver_workspace_bytes": inf.solver_workspace_bytes,
                "setup_scratch_bytes": inf.setup_scratch_bytes,
                "rebuild_tiles": tuple(inf.rebuild_tiles)}

    def export(self, c):
        """(core, [U1, U2, U3], [sigma1, sigma2, sigma3]) of component c as complex128 numpy."""
        inf = self.info()
        r = inf["ranks"][c]
        P = inf["P"]
        core = np.zeros(r, dtype=np.complex128)
        U = [np.zeros((P[q], r[q]), dtype=np.complex128) for q in range(3)]
        S = [np.zeros(P[q] // 2 + 1, dtype=np.float64) for q in range(3)]
        dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        _check(lib.vie_op_export(self._h, c, dp(core), dp(U[0]), dp(U[1]), dp(U[2]),
                                 dp(S[0]), dp(S[1]), dp(S[2]), _stream()), "vie_op_export")
        return core, U, S

    def tucker_cp(self, rank, tol=1e-9, max_iter=500, seed=0):
        """Algorithm 2: CP-ALS with `rank` terms on each HOSVD core (vie_tucker_cp);
        afterwards path="tucker_cp" applies eq. (17).  Returns the relative core
        errors of the six components."""
        _check(lib.vie_tucker_cp(self._h, int(rank), float(tol), int(max_iter), int(seed), _stream()),
               "vie_tucker_cp")
        return self.info()["cp_rel_err"]

    def cp_export(self, c):
        """([W1, W2, W3], rel_err, sweeps) of component c as complex128 numpy (all P_q rows)."""
        inf = self.info()
        R, P = inf["cp_rank"], inf["P"]
        W = [np.zeros((P[q], R), dtype=np.complex128) for q in range(3)]
        err = ctypes.c_double()
        sw = ctypes.c_int()
        dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        _check(lib.vie_cp_export(self._h, c, dp(W[0]), dp(W[1]), dp(W[2]), ctypes.byref(err),
                                 ctypes.byref(sw), _stream()), "vie_cp_export")
        return W, err.value, sw.value

    def reserve(self, max_batch):
        _check(lib.vie_reserve(self._h, int(max_batch)), "vie_reserve")

    def autotune(self, batch=1):
        """Pick the FFT stages' CTA sizes by timing matvecs at `batch`, and the tcgen05
        rebuild's tile shape (vie_autotune); returns the stages' CTA sizes."""
        _check(lib.vie_autotune(self._h, int(batch), _stream()), "vie_autotune")
        return self.info()["line_threads"]

    # -- operator applications ---------------------------------------------
    def _out(self, like, out):
        torch = _torch()
        return torch.empty_like(like) if out is None else out

    def matvec(self, J, path="tucker", out=None):
        """Y = G J."""
        B = _batch(J, self.n)
        Y = self._out(J, out)
        _check(lib.vie_matvec(self._h, _dev(J, "J", self.n), _dev(Y, "out", self.n), B,
                              PATHS[path], _precision(J), _stream()), "vie_matvec")
        return Y

    def matvec_adjoint(self, Y, path="tucker", out=None):
        """X = G^H Y."""
        B = _batch(Y, self.n)
        X = self._out(Y, out)
        _check(lib.vie_matvec_adjoint(self._h, _dev(Y, "Y", self.n), _dev(X, "out", self.n), B,
                                      PATHS[path], _precision(Y), _stream()), "vie_matvec_adjoint")
        return X

    def apply_system(self, chi, w, adjoint=False, path="tucker", out=None):
        """A w = w - chi (G w), or A^H w."""
        B = _batch(w, self.n)
        o = self._out(w, out)
        _check(lib.vie_apply_system(self._h, _dev(chi, "chi", self.n), _dev(w, "w", self.n),
                                    _dev(o, "out", self.n), B, int(bool(adjoint)), PATHS[path],
                                    _precision(w), _stream()), "vie_apply_system")
        return o

    def total_field(self, einc, w, path="tucker", out=None):
        """E = e_inc + G w."""
        B = _batch(w, self.n)
        E = self._out(w, out)
        _check(lib.vie_total_field(self._h, _dev(einc, "einc", self.n), _dev(w, "w", self.n),
                                   _dev(E, "out", self.n), B, PATHS[path], _precision(w),
                                   _stream()), "vie_total_field")
        return E

    def solve(self, chi, rhs, incident=True, adjoint=False, x0=None, tol=1e-6, restart=50,
              max_outer=200, inner_tol=None, max_refine=20, path="tucker", use_graph=True,
              refine=True, orth=1, out=None, raise_on_failure=True):
        """Solve A w = b (or A^H w = b); b = chi * rhs when ``incident``.  Returns (w, info)."""
        B = _batch(rhs, self.n)
        w = self._out(rhs, out)
        flags = (VIE_SOLVE_ADJOINT if adjoint else 0) | (VIE_SOLVE_RHS_INCIDENT if incident else 0)
        if x0 is not None:
            w.copy_(x0)
            flags |= VIE_SOLVE_X0
        opts = _solve_opts(tol, restart, max_outer, inner_tol, max_refine, path, use_graph, refine,
                           orth)
        inf = SolveInfo()
        st = lib.vie_solve(self._h, _dev(chi, "chi", self.n), _dev(rhs, "rhs", self.n),
                           _dev(w, "w", self.n), B, flags, _precision(rhs), ctypes.byref(opts),
                           ctypes.byref(inf), _stream())
        info = _solve_info(inf, st)
        if st != VIE_OK and (raise_on_failure or st != 4):
            _check(st, "vie_solve")
        return w, info

    def contrast_gradient(self, lam, E, scale=2.0, out=None):
        """grad = scale * sum_b sum_a lam conj(E)."""
        torch = _torch()
        B = _batch(E, self.n)
        g = torch.empty(self.n, dtype=E.dtype, device=E.device) if out is None else out
        _check(lib.vie_contrast_gradient(self._h, _dev(lam, "lam", self.n), _dev(E, "E", self.n),
                                         _dev(g, "grad", self.n), B, float(scale), _precision(E),
                                         _stream()), "vie_contrast_gradient")
        return g

    def incident_dipole(self, sources, dtype=None, device="cuda"):
        """Fields [B, 3, n1, n2, n3] of unit z-dipoles at ``sources`` [B, 3] (metres)."""
        torch = _torch()
        src = np.ascontiguousarray(np.asarray(sources, dtype=np.float64).reshape(-1, 3))
        B = src.shape[0]
        dtype = dtype or torch.complex64
        out = torch.empty((B, 3) + self.n, dtype=dtype, device=device)
        _check(lib.vie_incident_dipole(self._h, src.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       B, _dev(out, "out"), _precision(out), _stream()),
               "vie_incident_dipole")
        return out


PROFILE_FAMILIES = ("line_x", "line_y", "fused_tucker", "fused_stored", "line_iy", "line_ix",
                    "tucker_rebuild", "arnoldi_dots", "arnoldi_update", "arnoldi_small", "fp64_vector",
                    "setup", "matvec_fp64")


def _solve_opts(tol, restart, max_outer, inner_tol, max_refine, path, use_graph, refine, orth):
    if inner_tol is None:
        # the first inner solve aims below the target, so that FP32 rounding of its
        # residual estimate does not cost a second refinement step
        inner_tol = max(0.5 * tol, 5e-6) if refine else tol
    return SolveOpts(float(tol), int(restart), int(max_outer), float(inner_tol), int(max_refine),
                     PATHS[path], int(bool(use_graph)), int(bool(refine)), int(orth))


def _solve_info(inf, st):
    return {"converged": bool(inf.converged), "refine_steps": inf.refine_steps,
            "iterations": inf.iterations, "matvecs": inf.matvecs, "relres": inf.relres,
            "history": list(inf.history[:inf.refine_steps + 1]), "status": st}


def solve_multi(ops, chis, rhss, incident=True, adjoint=False, tol=1e-6, restart=50, max_outer=200,
                inner_tol=None, max_refine=20, path="tucker", use_graph=True, refine=True, orth=1):
    """Independent solves on several operators (grids may differ), run concurrently
    (vie_solve_multi).  Returns [(w, info)] in the order of ``ops``."""
    torch = _torch()
    count = len(ops)
    if len(chis) != count or len(rhss) != count:
        raise ValueError("one contrast and one right-hand side per operator")
    dtypes = {r.dtype for r in rhss}
    if len(dtypes) != 1:
        raise TypeError("all right-hand sides must share one dtype")
    ws = [torch.empty_like(r) for r in rhss]
    flags = (VIE_SOLVE_ADJOINT if adjoint else 0) | (VIE_SOLVE_RHS_INCIDENT if incident else 0)
    opts = _solve_opts(tol, restart, max_outer, inner_tol, max_refine, path, use_graph, refine, orth)
    infs = (SolveInfo * count)()
    hs = (ctypes.c_void_p * count)(*[op._h.value for op in ops])
    cp = (ctypes.c_void_p * count)(*[_dev(c, "chi", op.n).value for op, c in zip(ops, chis)])
    rp = (ctypes.c_void_p * count)(*[_dev(r, "rhs", op.n).value for op, r in zip(ops, rhss)])
    wp = (ctypes.c_void_p * count)(*[_dev(w, "w", op.n).value for op, w in zip(ops, ws)])
    bs = (ctypes.c_int * count)(*[_batch(r, op.n) for op, r in zip(ops, rhss)])
    st = lib.vie_solve_multi(hs, cp, rp, wp, bs, count, flags, _precision(rhss[0]),
                             ctypes.byref(opts), infs, _stream())
    _check(st, "vie_solve_multi")
    return [(w, _solve_info(infs[p], VIE_OK)) for p, w in enumerate(ws)]


MULTI_MODES = {"persistent": 0, "staged": 1}


def matvec_multi(ops, Js, outs=None, mode="persistent"):
    """Y_p = G_p J_p for several operators (grids may differ): one persistent
    cooperative launch over all stages (mode "persistent") or one launch per
    stage ("staged")."""
    torch = _torch()
    count = len(ops)
    if len(Js) != count:
        raise ValueError("one current per operator")
    outs = [torch.empty_like(J) for J in Js] if outs is None else outs
    for J in Js:
        if J.dtype != torch.complex64:
            raise TypeError("vie_matvec_multi takes complex64")
    hs = (ctypes.c_void_p * count)(*[op._h.value for op in ops])
    jp = (ctypes.c_void_p * count)(*[_dev(J, "J", op.n).value for op, J in zip(ops, Js)])
    yp = (ctypes.c_void_p * count)(*[_dev(Y, "out", op.n).value for op, Y in zip(ops, outs)])
    bs = (ctypes.c_int * count)(*[_batch(J, op.n) for op, J in zip(ops, Js)])
    _check(lib.vie_matvec_multi_ex(hs, jp, yp, bs, count, MULTI_MODES[mode], _stream()),
           "vie_matvec_multi_ex")
    return outs


def profile_start(families=None):
    """Start per-kernel-family event timing (vie_profile_start); None = every family."""
    mask = 0xFFFFFFFF if families is None else \
        sum(1 << PROFILE_FAMILIES.index(f) for f in families)
    _check(lib.vie_profile_start(ctypes.c_uint(mask)), "vie_profile_start")


def profile_stop():
    """Stop timing; {family: {"launches", "ms", "bytes"}} of the families that ran."""
    buf = (ProfileEntry * 32)()
    n = ctypes.c_int()
    _check(lib.vie_profile_stop(buf, 32, ctypes.byref(n)), "vie_profile_stop")
    return {buf[i].name.decode(): {"launches": buf[i].launches, "ms": buf[i].ms,
                                   "bytes": buf[i].bytes} for i in range(n.value)}


def green_spectrum(n, h, freq_hz, c, self_term="full", device="cuda"):
    """The FFT'd circulant component c (complex128 [P1, P2, P3]) as the setup forms it."""
    torch = _torch()
    if isinstance(n, int):
        n = (n, n, n)
    g = Grid(n[0], n[1], n[2], float(h), float(freq_hz))
    out = torch.empty(tuple(2 * v for v in n), dtype=torch.complex128, device=device)
    _check(lib.vie_green_spectrum(ctypes.byref(g), int(c), VIE_SELF_TERM_PV if self_term == "pv" else 0,
                                  _dev(out, "out"), _stream()), "vie_green_spectrum")
    return out


from .autograd import SolveFields, solve_fields  # noqa: E402,F401
