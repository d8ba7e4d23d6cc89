"""ctypes binding of libct (the C ABI declared in include/ct.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Vectors may be torch tensors (CUDA or CPU) or numpy arrays; they
must be float32 and contiguous.  CUDA tensors are used in place on the
current torch stream of their device; host buffers go through the library's
synchronous staging path.  There is no CPU fallback: if libct.so is missing
the first call raises.

The module-level ``ct_*`` functions mirror the C entry points one to one;
``Matrix`` is a small convenience wrapper around a matrix handle.
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libct.so")

CT_OK = 0
CT_ERR_ARG = -1
CT_ERR_CUDA = -2
CT_ERR_OOM = -3
CT_ERR_BREAKDOWN = -4
CT_ERR_NONFINITE = -5
CT_ERR_TIMEOUT = -6
CT_ERR_UNSUPPORTED = -7

CT_VAL_FP32 = 0
CT_VAL_FP16_ROWSCALE = 1
CT_KEEP_FP32_COPY = 4
CT_F64_FP64_PIPE = 8

CT_FOURIER_FUSED = 0
CT_FOURIER_GRIDDING = 1

SYMBOLS = (
    "ct_build_matrix",
    "ct_matrix_info",
    "ct_destroy_matrix",
    "ct_forward",
    "ct_adjoint",
    "ct_forward_f64",
    "ct_adjoint_f64",
    "ct_cg_solve",
    "ct_cg_solve_noalloc",
    "ct_split_bregman",
    "ct_split_bregman_ragged",
    "ct_chambolle_pock",
    "ct_set_spmm_unroll",
    "ct_get_spmm_unroll",
    "ct_time_cg_kernels",
    "ct_get_tuning",
    "ct_set_tuning",
    "ct_tune",
    "ct_set_wait_limit",
    "ct_normal_f64",
    "ct_matrix_export",
    "ct_matrix_export_fp16",
    "ct_surrogate_stencil",
    "ct_build_fourier",
    "ct_fourier_forward",
    "ct_fourier_adjoint",
    "ct_fourier_normal",
    "ct_fourier_data",
    "ct_status_string",
    "ct_last_error",
)


class Geometry(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32),
        ("n_angles_total", ctypes.c_int32),
        ("keep_every", ctypes.c_int32),
        ("n_bins", ctypes.c_int32),
    ]


class CgParams(ctypes.Structure):
    _fields_ = [
        ("c_id", ctypes.c_double),
        ("c_ata", ctypes.c_double),
        ("c_grad", ctypes.c_double),
        ("max_iters", ctypes.c_int32),
        ("rel_tol", ctypes.c_double),
        ("surrogate_r", ctypes.c_int32),
        ("refresh_every", ctypes.c_int32),
        ("surrogate_square", ctypes.c_int32),
    ]


class CgStats(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int32),
        ("final_rel_res", ctypes.c_double),
        ("status", ctypes.c_int32),
    ]


class SbParams(ctypes.Structure):
    _fields_ = [
        ("alpha", ctypes.c_double),
        ("lambda_", ctypes.c_double),
        ("outer_iters", ctypes.c_int32),
        ("inner_cg_iters", ctypes.c_int32),
        ("stop_rel_update", ctypes.c_double),
        ("surrogate_r", ctypes.c_int32),
        ("refresh_every", ctypes.c_int32),
        ("surrogate_square", ctypes.c_int32),
        ("cg_rel_tol", ctypes.c_double),
    ]


class CpParams(ctypes.Structure):
    _fields_ = [
        ("alpha", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("theta", ctypes.c_double),
        ("outer_iters", ctypes.c_int32),
        ("inner_cg_iters", ctypes.c_int32),
    ]


class FourierParams(ctypes.Structure):
    _fields_ = [
        ("m_sp", ctypes.c_int32),
        ("tau", ctypes.c_double),
        ("mode", ctypes.c_int32),
    ]


class SbStats(ctypes.Structure):
    _fields_ = [
        ("outer_done", ctypes.c_int32),
        ("first_update_l1", ctypes.c_double),
        ("last_update_l1", ctypes.c_double),
        ("status", ctypes.c_int32),
    ]


class Tuning(ctypes.Structure):
    _fields_ = [
        ("fwd_warps", ctypes.c_int32),
        ("fwd_unroll", ctypes.c_int32),
        ("op_ctas", ctypes.c_int32),
        ("op_pixels", ctypes.c_int32),
        ("spmm_unroll", ctypes.c_int32),
    ]


class CtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (status_string(code), code, msg))
        self.code = code


_lib = None


def lib():
    """Loads libct.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "libct.so not found at %s; build it with __graft_entry__.build()" % LIB_PATH
            )
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
        P = ctypes.POINTER
        L.ct_build_matrix.argtypes = [P(Geometry), u32, P(vp)]
        L.ct_matrix_info.argtypes = [vp, P(i64), P(i64), P(i64)]
        L.ct_destroy_matrix.argtypes = [vp]
        L.ct_destroy_matrix.restype = None
        L.ct_forward.argtypes = [vp, vp, vp, i32, vp]
        L.ct_adjoint.argtypes = [vp, vp, vp, i32, vp]
        L.ct_forward_f64.argtypes = [vp, vp, vp, i32, vp]
        L.ct_adjoint_f64.argtypes = [vp, vp, vp, i32, vp]
        L.ct_cg_solve.argtypes = [vp, P(CgParams), vp, vp, i32, P(CgStats), vp]
        L.ct_cg_solve_noalloc.argtypes = [vp, P(CgParams), vp, vp, P(CgStats), vp]
        L.ct_split_bregman.argtypes = [vp, P(SbParams), vp, vp, i32, P(SbStats), vp]
        L.ct_split_bregman_ragged.argtypes = [i32, vp, vp, vp, P(SbParams), vp, vp]
        L.ct_chambolle_pock.argtypes = [vp, P(CpParams), vp, vp, i32, P(SbStats), vp]
        L.ct_set_spmm_unroll.argtypes = [vp, i32, i32]
        L.ct_get_spmm_unroll.argtypes = [vp, i32, P(i32)]
        L.ct_time_cg_kernels.argtypes = [vp, ctypes.c_double, ctypes.c_double, i32, vp, vp]
        L.ct_get_tuning.argtypes = [vp, i32, P(Tuning)]
        L.ct_set_tuning.argtypes = [vp, i32, P(Tuning)]
        L.ct_tune.argtypes = [vp, i32, vp]
        L.ct_set_wait_limit.argtypes = [i64, i32]
        L.ct_normal_f64.argtypes = [vp, ctypes.c_double, ctypes.c_double, vp, vp, i32, vp]
        L.ct_matrix_export.argtypes = [vp, i32, vp, vp, vp]
        L.ct_matrix_export_fp16.argtypes = [vp, vp, vp]
        L.ct_surrogate_stencil.argtypes = [vp, i32, i32, i32, vp, vp, vp, P(i32)]
        L.ct_build_fourier.argtypes = [P(Geometry), P(FourierParams), P(vp)]
        L.ct_fourier_forward.argtypes = [vp, vp, vp, vp]
        L.ct_fourier_adjoint.argtypes = [vp, vp, vp, vp]
        L.ct_fourier_normal.argtypes = [vp, vp, vp, vp]
        L.ct_fourier_data.argtypes = [vp, vp, vp, vp]
        L.ct_status_string.argtypes = [ctypes.c_int]
        L.ct_status_string.restype = ctypes.c_char_p
        L.ct_last_error.argtypes = []
        L.ct_last_error.restype = ctypes.c_char_p
        for name in SYMBOLS:
            if name not in ("ct_destroy_matrix", "ct_status_string", "ct_last_error"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def status_string(code):
    return lib().ct_status_string(code).decode()


def _check(code):
    if code != CT_OK:
        raise CtError(code, lib().ct_last_error().decode())
    return code


def _vec(x, f64=False):
    """(pointer, stream handle) of a contiguous float32 (or float64) tensor or array."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(x, torch.Tensor):
        want = torch.float64 if f64 else torch.float32
        if x.dtype != want or not x.is_contiguous():
            raise TypeError("expected a contiguous %s tensor" % want)
        stream = torch.cuda.current_stream(x.device).cuda_stream if x.is_cuda else 0
        return x.data_ptr(), stream
    if isinstance(x, np.ndarray):
        want = np.float64 if f64 else np.float32
        if x.dtype != want or not x.flags["C_CONTIGUOUS"]:
            raise TypeError("expected a C-contiguous %s array" % np.dtype(want).name)
        return x.ctypes.data, 0
    raise TypeError("expected a torch tensor or numpy array, got %r" % type(x))


# ---------------------------------------------------------------------------
# one-to-one mirrors of the C entry points
# ---------------------------------------------------------------------------
def ct_build_matrix(geometry, flags=0):
    h = ctypes.c_void_p()
    _check(lib().ct_build_matrix(ctypes.byref(geometry), flags, ctypes.byref(h)))
    return h


def ct_matrix_info(h):
    r, c, z = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().ct_matrix_info(h, ctypes.byref(r), ctypes.byref(c), ctypes.byref(z)))
    return r.value, c.value, z.value


def ct_destroy_matrix(h):
    lib().ct_destroy_matrix(h)


def ct_forward(h, x, y, batch, stream=None):
    px, sx = _vec(x)
    py, _ = _vec(y)
    return _check(lib().ct_forward(h, px, py, batch, sx if stream is None else stream))


def ct_adjoint(h, y, x, batch, stream=None):
    py, sy = _vec(y)
    px, _ = _vec(x)
    return _check(lib().ct_adjoint(h, py, px, batch, sy if stream is None else stream))


def ct_forward_f64(h, x, y, batch, stream=None):
    px, sx = _vec(x, f64=True)
    py, _ = _vec(y, f64=True)
    return _check(lib().ct_forward_f64(h, px, py, batch, sx if stream is None else stream))


def ct_adjoint_f64(h, y, x, batch, stream=None):
    py, sy = _vec(y, f64=True)
    px, _ = _vec(x, f64=True)
    return _check(lib().ct_adjoint_f64(h, py, px, batch, sy if stream is None else stream))


def ct_normal_f64(h, alpha, lam, x, out, batch, stream=None):
    px, sx = _vec(x, f64=True)
    po, _ = _vec(out, f64=True)
    return _check(lib().ct_normal_f64(h, alpha, lam, px, po, batch, sx if stream is None else stream))


def ct_cg_solve(h, params, rhs, u, batch, stats=None, stream=None):
    pr, sr = _vec(rhs)
    pu, _ = _vec(u)
    sp = ctypes.byref(stats) if stats is not None else None
    return _check(lib().ct_cg_solve(h, ctypes.byref(params), pr, pu, batch, sp, sr if stream is None else stream))


def ct_cg_solve_noalloc(h, params, rhs, u, stats=None, stream=None):
    """ct_cg_solve for one slice on the library's fixed scratch array (no allocation)."""
    pr, sr = _vec(rhs)
    pu, _ = _vec(u)
    sp = ctypes.byref(stats) if stats is not None else None
    return _check(lib().ct_cg_solve_noalloc(h, ctypes.byref(params), pr, pu, sp, sr if stream is None else stream))


def ct_split_bregman(h, params, f, u, batch, stats=None, stream=None):
    pf, sf = _vec(f)
    pu, _ = _vec(u)
    sp = ctypes.byref(stats) if stats is not None else None
    return _check(lib().ct_split_bregman(h, ctypes.byref(params), pf, pu, batch, sp, sf if stream is None else stream))


def ct_chambolle_pock(h, params, g, u, batch, stats=None, stream=None):
    pg, sg = _vec(g)
    pu, _ = _vec(u)
    sp = ctypes.byref(stats) if stats is not None else None
    return _check(lib().ct_chambolle_pock(h, ctypes.byref(params), pg, pu, batch, sp, sg if stream is None else stream))


def ct_split_bregman_ragged(handles, params, fs, us, stats=None, stream=None):
    """One call over len(handles) problems: (handles[i], fs[i], us[i]); stats:
    None or a ctypes array of len(handles) SbStats."""
    count = len(handles)
    if not (len(fs) == len(us) == count):
        raise ValueError("handles, fs and us must have the same length")
    hs = (ctypes.c_void_p * count)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    pf = (ctypes.c_void_p * count)()
    pu = (ctypes.c_void_p * count)()
    sf = None
    for i in range(count):
        pf[i], s_i = _vec(fs[i])
        pu[i], _ = _vec(us[i])
        sf = s_i if sf is None else sf
    sp = stats if stats is not None else None
    return _check(lib().ct_split_bregman_ragged(count, hs, pf, pu, ctypes.byref(params), sp,
                                                sf if stream is None else stream))


def ct_time_cg_kernels(h, c_ata, c_grad, reps, stream=None):
    """Mean ms per launch of the CG step's kernels: [A p, Op(p) fused into
    A^T, u/r update, direction update]."""
    ms = (ctypes.c_double * 4)()
    if stream is None:
        import torch

        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _check(lib().ct_time_cg_kernels(h, c_ata, c_grad, reps, ms, stream))
    return list(ms)


def ct_get_tuning(h, batch):
    t = Tuning()
    _check(lib().ct_get_tuning(h, batch, ctypes.byref(t)))
    return {k: getattr(t, k) for k, _ in Tuning._fields_}


def ct_set_tuning(h, batch, **fields):
    t = Tuning(**fields)
    return _check(lib().ct_set_tuning(h, batch, ctypes.byref(t)))


def ct_tune(h, batch, stream=None):
    if stream is None:
        import torch

        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return _check(lib().ct_tune(h, batch, stream))


def ct_set_wait_limit(polls, hold_first=False):
    """Bounded-wait limit of the persistent ragged kernel (polls <= 0: the
    default); hold_first makes the next persistent call run out of its waits."""
    return _check(lib().ct_set_wait_limit(int(polls), int(bool(hold_first))))


def ct_matrix_export(h, which):
    rows, cols, nnz = ct_matrix_info(h)
    n_rows = rows if which == 0 else cols
    rp = np.zeros(n_rows + 1, dtype=np.int64)
    ci = np.zeros(nnz, dtype=np.int32)
    va = np.zeros(nnz, dtype=np.float32)
    _check(lib().ct_matrix_export(h, which, rp.ctypes.data, ci.ctypes.data, va.ctypes.data))
    return rp, ci, va


def ct_matrix_export_fp16(h):
    rows, _, nnz = ct_matrix_info(h)
    q = np.zeros(nnz, dtype=np.uint16)
    s = np.zeros(rows, dtype=np.float32)
    _check(lib().ct_matrix_export_fp16(h, q.ctypes.data, s.ctypes.data))
    return q, s


def ct_surrogate_stencil(h, r, square=False):
    cnt = ctypes.c_int32()
    lib().ct_surrogate_stencil(h, r, int(square), 0, None, None, None, ctypes.byref(cnt))
    n = cnt.value
    if n <= 0:
        _check(CT_ERR_ARG)
    di = np.zeros(n, dtype=np.int32)
    dj = np.zeros(n, dtype=np.int32)
    w = np.zeros(n, dtype=np.float64)
    _check(lib().ct_surrogate_stencil(h, r, int(square), n, di.ctypes.data, dj.ctypes.data,
                                      w.ctypes.data, ctypes.byref(cnt)))
    return {(int(a), int(b)): float(v) for a, b, v in zip(di, dj, w)}


def ct_build_fourier(geometry, params):
    h = ctypes.c_void_p()
    _check(lib().ct_build_fourier(ctypes.byref(geometry), ctypes.byref(params), ctypes.byref(h)))
    return h


def ct_fourier_forward(h, x, y, stream=None):
    """y (2J floats, complex interleaved) = F x."""
    px, sx = _vec(x)
    py, _ = _vec(y)
    return _check(lib().ct_fourier_forward(h, px, py, sx if stream is None else stream))


def ct_fourier_adjoint(h, y, x, stream=None):
    """x = Re(F^H y)."""
    py, sy = _vec(y)
    px, _ = _vec(x)
    return _check(lib().ct_fourier_adjoint(h, py, px, sy if stream is None else stream))


def ct_fourier_normal(h, x, out, stream=None):
    """out = Re(F^H F x)."""
    px, sx = _vec(x)
    po, _ = _vec(out)
    return _check(lib().ct_fourier_normal(h, px, po, sx if stream is None else stream))


def ct_fourier_data(h, f, fhat, stream=None):
    """fhat (2J floats, complex interleaved) = DFTs of the sinogram's projections."""
    pf, sf = _vec(f)
    ph, _ = _vec(fhat)
    return _check(lib().ct_fourier_data(h, pf, ph, sf if stream is None else stream))


def _is_f64(x):
    dt = getattr(x, "dtype", None)
    return str(dt) in ("torch.float64", "float64")


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------
class Matrix:
    """A = M R and A^T for one geometry, resident on the current CUDA device."""

    def __init__(self, n, n_angles_total, keep_every, n_bins, flags=CT_VAL_FP32):
        self.geometry = Geometry(n, n_angles_total, keep_every, n_bins)
        self.flags = flags
        self.handle = ct_build_matrix(self.geometry, flags)
        self.rows, self.cols, self.nnz = ct_matrix_info(self.handle)
        self.n = n

    def close(self):
        if self.handle is not None:
            ct_destroy_matrix(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _batch(self, x, length):
        total = int(np.prod(x.shape))
        if total % length:
            raise ValueError("vector size %d is not a multiple of %d" % (total, length))
        return total // length

    def forward(self, x, y):
        """y = A x; float64 tensors use the FP64-vector entry point."""
        fn = ct_forward_f64 if _is_f64(x) else ct_forward
        fn(self.handle, x, y, self._batch(x, self.cols))
        return y

    def adjoint(self, y, x):
        """x = A^T y; float64 tensors use the FP64-vector entry point."""
        fn = ct_adjoint_f64 if _is_f64(y) else ct_adjoint
        fn(self.handle, y, x, self._batch(y, self.rows))
        return x

    def cg_solve(self, rhs, u, c_id, c_ata, c_grad, max_iters, rel_tol=0.0, surrogate_r=0,
                 refresh_every=0, square=False):
        p = CgParams(c_id, c_ata, c_grad, max_iters, rel_tol, surrogate_r, refresh_every, int(square))
        st = CgStats()
        ct_cg_solve(self.handle, p, rhs, u, self._batch(u, self.cols), st)
        return {"iters": st.iters, "final_rel_res": st.final_rel_res, "status": st.status}

    def split_bregman(self, f, u, alpha, lam, outer, inner, stop_rel_update=0.0, surrogate_r=0,
                      refresh_every=0, square=False, stats=True, cg_rel_tol=0.0):
        p = SbParams(alpha, lam, outer, inner, stop_rel_update, surrogate_r, refresh_every, int(square), cg_rel_tol)
        st = SbStats() if stats else None
        ct_split_bregman(self.handle, p, f, u, self._batch(u, self.cols), st)
        if st is None:
            return None
        return {"outer_done": st.outer_done, "first_update_l1": st.first_update_l1,
                "last_update_l1": st.last_update_l1, "status": st.status}

    def chambolle_pock(self, g, u, alpha, tau, sigma, outer, inner, theta=1.0, stats=True):
        """Primal-dual TV reconstruction (one slice): u in = initial guess, out = result."""
        p = CpParams(alpha, tau, sigma, theta, outer, inner)
        st = SbStats() if stats else None
        ct_chambolle_pock(self.handle, p, g, u, self._batch(u, self.cols), st)
        if st is None:
            return None
        return {"outer_done": st.outer_done, "first_update_l1": st.first_update_l1,
                "last_update_l1": st.last_update_l1, "status": st.status}

    def set_spmm_unroll(self, batch, unroll):
        """Pins the batched products' staged-entry unroll (4 or 8; 0 = automatic)."""
        _check(lib().ct_set_spmm_unroll(self.handle, batch, unroll))

    def spmm_unroll(self, batch):
        """The batched products' unroll for this batch size (0 = not chosen yet)."""
        v = ctypes.c_int32()
        _check(lib().ct_get_spmm_unroll(self.handle, batch, ctypes.byref(v)))
        return v.value

    def export(self, which=0):
        return ct_matrix_export(self.handle, which)

    def export_fp16(self):
        return ct_matrix_export_fp16(self.handle)

    def surrogate_stencil(self, r, square=False):
        return ct_surrogate_stencil(self.handle, r, square)


class FourierMatrix(Matrix):
    """The Fourier-domain data term of one geometry (Sec. 2, Eq. four_obj),
    gridded with window half-width m_sp (Sec. 3.1) and, in fused mode, the
    precomputed matrix of Eq. fusedop.  cg_solve, split_bregman,
    chambolle_pock and surrogate_stencil work as on a Matrix (one slice);
    forward/adjoint are the complex F and Re(F^H)."""

    def __init__(self, n, n_angles_total, keep_every, n_bins, m_sp=6, tau=0.0, mode=CT_FOURIER_FUSED):
        self.geometry = Geometry(n, n_angles_total, keep_every, n_bins)
        self.flags = 0
        self.params = FourierParams(m_sp, tau, mode)
        self.handle = ct_build_fourier(self.geometry, self.params)
        self.rows, self.cols, self.nnz = ct_matrix_info(self.handle)
        self.n = n

    def forward(self, x, y):
        """y (2 * rows floats: complex samples, interleaved) = F x."""
        ct_fourier_forward(self.handle, x, y)
        return y

    def adjoint(self, y, x):
        """x = Re(F^H y)."""
        ct_fourier_adjoint(self.handle, y, x)
        return x

    def normal(self, x, out):
        """out = Re(F^H F x)."""
        ct_fourier_normal(self.handle, x, out)
        return out

    def data(self, f, fhat):
        """fhat (2 * rows floats) = the DFTs of the sinogram f's projections."""
        ct_fourier_data(self.handle, f, fhat)
        return fhat


def split_bregman_ragged(matrices, fs, us, alpha, lam, outer, inner, stop_rel_update=0.0, surrogate_r=0,
                         refresh_every=0, square=False, stats=True, cg_rel_tol=0.0):
    """Split Bregman over problems of possibly different geometries in one
    call: problem i reconstructs us[i] (N_i*N_i, in = initial guess) from
    fs[i] with matrices[i].  Returns per-problem stats (or None)."""
    p = SbParams(alpha, lam, outer, inner, stop_rel_update, surrogate_r, refresh_every, int(square), cg_rel_tol)
    st = (SbStats * len(matrices))() if stats else None
    ct_split_bregman_ragged([m.handle for m in matrices], p, fs, us, st)
    if st is None:
        return None
    return [{"outer_done": s.outer_done, "first_update_l1": s.first_update_l1,
             "last_update_l1": s.last_update_l1, "status": s.status} for s in st]
