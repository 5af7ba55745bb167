"""Thin Python binding of the C ABI in include/mixfft.h.

Argument marshalling only: every step of the computation runs in the CUDA
library libmixfft.so.  PyTorch supplies the device workspace and the CUDA
stream; numpy arrays are passed as host pointers.  If the library has not been
built, importing this module raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# MF_LIBRARY=debug selects the bounds-checking build (build.build(debug=True)),
# MF_LIBRARY=trace the phase-timestamp build (build.build(trace=True))
LIB_PATH = os.path.join(_HERE, {"debug": "libmixfft_debug.so", "trace": "libmixfft_trace.so"}.get(
    os.environ.get("MF_LIBRARY", ""), "libmixfft.so"))

MF_OK, MF_INVALID_ARG, MF_NOT_CONVERGED, MF_CG_BREAKDOWN = 0, 1, 2, 3
MF_NONPOSITIVE_J, MF_CUDA_ERROR, MF_DEVICE_TIMEOUT, MF_NO_WORKSPACE = 4, 5, 6, 7
MF_TOO_LARGE = 8
MF_FP64, MF_FP32_INNER = 0, 1
MF_NEOHOOKE, MF_SVK_CUBIC = 0, 1
MF_OUTER_DOUBLE_WORD, MF_OUTER_FP64 = 0, 1
MF_PROJ_FP32, MF_PROJ_OUTER, MF_PROJ_AUTO = 0, 1, 2
MF_PRED_UNIFORM, MF_PRED_EXTRAPOLATE, MF_PRED_QUADRATIC = 0, 1, 2
MF_TRACE_STEP_START, MF_TRACE_STEP_BEGIN, MF_TRACE_FIRST_CONSTITUTIVE, MF_TRACE_FIRST_RESIDUAL = 1, 2, 3, 4
MF_TRACE_ITER_START, MF_TRACE_NEWTON_PRE, MF_TRACE_CG_INIT, MF_TRACE_CG_LOOP = 10, 11, 12, 13
MF_TRACE_PROJECTION, MF_TRACE_DEFLATION, MF_TRACE_UPDATE, MF_TRACE_NEWTON_POST = 14, 15, 16, 17
MF_TRACE_FBAR, MF_TRACE_CONSTITUTIVE, MF_TRACE_RESIDUAL, MF_TRACE_CONS_SWITCH = 18, 19, 20, 21
MF_TRACE_NEWTON_LOOP, MF_TRACE_STEP_END = 30, 31

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: run paper_1901_06531_gb300.build.build() first")

_lib = ctypes.CDLL(LIB_PATH)
_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_sz = ctypes.c_size_t

_lib.mf_create.argtypes = [ctypes.POINTER(_vp), _i, _i, _i, _i, _vp]
_lib.mf_workspace_bytes.argtypes = [_vp]
_lib.mf_workspace_bytes.restype = _sz
_lib.mf_bind_workspace.argtypes = [_vp, _vp, _sz]
_lib.mf_set_material.argtypes = [_vp, _i, _i, _vp, _vp, _vp, _vp]
_lib.mf_set_F.argtypes = [_vp, _vp]
_lib.mf_solve.argtypes = [_vp, _i, _vp, _vp, _d, _d, _d, _i, _i, _vp, _vp, _vp]
_lib.mf_get_fields.argtypes = [_vp, _vp, _vp]
_lib.mf_save_F.argtypes = [_vp, _vp]
_lib.mf_load_F.argtypes = [_vp, _vp]
_lib.mf_solve_batch.argtypes = [_i, _vp, _i, _vp, _vp, _d, _d, _d, _i, _i, _vp, _vp, _vp, _vp]
_lib.mf_constitutive.argtypes = [_vp]
_lib.mf_stress.argtypes = [_vp, _vp]
_lib.mf_get_tangent.argtypes = [_vp, _vp]
_lib.mf_matvec.argtypes = [_vp, _vp, _vp, _vp]
_lib.mf_residual.argtypes = [_vp, _vp, _vp, _vp, _vp]
_lib.mf_residual_noalloc.argtypes = [_i, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp]
_lib.mf_time_kernels.argtypes = [_vp, _vp, _i, _i, _vp]
_lib.mf_cufft_workspace_bytes.argtypes = [_vp]
_lib.mf_cufft_workspace_bytes.restype = _sz
_lib.mf_cufft_bind.argtypes = [_vp, _vp, _sz]
_lib.mf_matvec_cufft.argtypes = [_vp, _vp, _vp, _vp]
_lib.mf_time_cufft.argtypes = [_vp, _vp, _i, _vp]
_lib.mf_kernel_launches.argtypes = []
_lib.mf_kernel_launches.restype = ctypes.c_longlong
_lib.mf_sync.argtypes = [_vp]
_lib.mf_autotune.argtypes = [_vp, _vp, _vp, _vp, _vp]
_lib.mf_set_outer_arith.argtypes = [_vp, _i]
_lib.mf_set_inexact_newton.argtypes = [_vp, _i]
_lib.mf_set_predictor.argtypes = [_vp, _i]
_lib.mf_probe_fma.argtypes = [_i, _vp]
_lib.mf_debug_report.argtypes = [_vp, _vp, _vp, _vp]
_lib.mf_debug_selftest.argtypes = []
_lib.mf_trace_read.argtypes = [_i, _vp, _vp, _vp]
_lib.mf_set_xy_split.argtypes = [_vp, _i]
_lib.mf_set_xy_persistent.argtypes = [_vp, _i]
_lib.mf_set_xy_cluster.argtypes = [_vp, _i]
_lib.mf_xy_schedule.argtypes = [_vp, _vp, _vp, _vp]
_lib.mf_set_projection_arith.argtypes = [_vp, _i]
_lib.mf_selftest_wait_timeout.argtypes = [_i]
_lib.mf_adjoint.argtypes = [_vp, _vp, _vp, _vp, _d, _d, _i, _vp, _vp, _vp, _vp]
_lib.mf_last_cuda_error.argtypes = []
_lib.mf_last_cuda_error.restype = ctypes.c_char_p
_lib.mf_status_string.argtypes = [_i]
_lib.mf_status_string.restype = ctypes.c_char_p
_lib.mf_destroy.argtypes = [_vp]
_lib.mf_destroy.restype = None

EXPORTED = ["mf_create", "mf_workspace_bytes", "mf_bind_workspace", "mf_set_material", "mf_set_F",
            "mf_solve", "mf_solve_batch", "mf_get_fields", "mf_save_F", "mf_load_F", "mf_constitutive",
            "mf_stress", "mf_get_tangent", "mf_matvec", "mf_residual", "mf_residual_noalloc",
            "mf_time_kernels", "mf_cufft_workspace_bytes", "mf_cufft_bind", "mf_matvec_cufft",
            "mf_time_cufft", "mf_kernel_launches", "mf_sync", "mf_autotune", "mf_adjoint",
            "mf_set_outer_arith", "mf_set_xy_split", "mf_set_xy_persistent", "mf_set_xy_cluster", "mf_xy_schedule", "mf_set_projection_arith",
            "mf_set_inexact_newton", "mf_set_predictor", "mf_probe_fma", "mf_debug_report", "mf_debug_selftest", "mf_trace_read", "mf_selftest_wait_timeout", "mf_last_cuda_error",
            "mf_status_string", "mf_destroy"]


def probe_fma(precision):
    """mf_probe_fma: measured FMA throughput of the current device, TFLOP/s."""
    out = np.zeros(1)
    _check("mf_probe_fma", _lib.mf_probe_fma(precision, _ptr(out)))
    return float(out[0])


def debug_report():
    """mf_debug_report: (failed bounds checks since the last call, first
    failure's source line, index, extent); count -1 in a release build."""
    cnt = ctypes.c_longlong(0)
    line = ctypes.c_int(0)
    idx = ctypes.c_longlong(0)
    ext = ctypes.c_longlong(0)
    _check("mf_debug_report", _lib.mf_debug_report(ctypes.byref(cnt), ctypes.byref(line), ctypes.byref(idx),
                                                   ctypes.byref(ext)))
    return cnt.value, line.value, idx.value, ext.value


def debug_selftest():
    """mf_debug_selftest: status (MF_OK in a debug build, MF_INVALID_ARG in a
    release build)."""
    return int(_lib.mf_debug_selftest())


# phase ids of mf_trace_read (include/mixfft.h, mf_trace_phase)
TRACE_PHASES = {v: k[len("MF_TRACE_"):].lower() for k, v in dict(globals()).items() if k.startswith("MF_TRACE_")}


def trace_read(cap=65536):
    """mf_trace_read: (timestamps in ns, phase ids) recorded since the last
    call by a trace build (MF_LIBRARY=trace); raises in a release build."""
    t = np.zeros(cap, dtype=np.uint64)
    ids = np.zeros(cap, dtype=np.int32)
    n = ctypes.c_int(0)
    _check("mf_trace_read", _lib.mf_trace_read(cap, _ptr(t), _ptr(ids), ctypes.byref(n)))
    k = min(n.value, cap)
    return t[:k].copy(), ids[:k].copy()


def kernel_launches():
    """mf_kernel_launches: kernels launched by the library in this process."""
    return int(_lib.mf_kernel_launches())


def residual_noalloc(nx, ny, nz, P, mask, pbar, b, stream=None):
    """mf_residual_noalloc: b = -G*(P - P-bar) in FP64 with no device
    allocation (for callers that cannot allocate at this point).  P, b: torch
    CUDA float64 tensors of 9N values owned by the caller; returns <P>.
    Calls sharing the library's static scratch must not overlap on the GPU."""
    import torch
    assert P.dtype == torch.float64 and b.dtype == torch.float64
    assert P.is_contiguous() and b.is_contiguous() and P.numel() == b.numel() == 9 * nx * ny * nz
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    pb = _c64(pbar)
    meanP = np.zeros(9)
    st = stream if stream is not None else torch.cuda.current_stream()
    _check("mf_residual_noalloc", _lib.mf_residual_noalloc(nx, ny, nz, _vp(P.data_ptr()), _ptr(m), _ptr(pb),
                                                           _vp(b.data_ptr()), _ptr(meanP),
                                                           _vp(st.cuda_stream)))
    return meanP


def solve_batch(contexts, masks, targets, tol_newton=1e-8, tol_cg=1e-10, cg_rel=1e-4, max_newton=50,
                max_cg=5000):
    """mf_solve_batch: the same number of load steps on every context at once.
    masks, targets: (n, nsteps, 9).  Returns a dict of (n, nsteps, ...) arrays
    and the per-cell status; raises on the first failure after all cells
    have been driven to their end."""
    n = len(contexts)
    masks = np.ascontiguousarray(masks, dtype=np.uint8).reshape(n, -1, 9)
    targets = _c64(targets).reshape(n, -1, 9)
    nsteps = masks.shape[1]
    Fbar = np.zeros((n, nsteps, 9))
    Pbar = np.zeros((n, nsteps, 9))
    iters = np.zeros((n, nsteps, 2), dtype=np.int32)
    status = np.zeros(n, dtype=np.int32)
    handles = (_vp * n)(*[c.h.value for c in contexts])
    st = _lib.mf_solve_batch(n, ctypes.cast(handles, _vp), nsteps, _ptr(masks), _ptr(targets), tol_newton, tol_cg,
                             cg_rel, max_newton, max_cg, _ptr(Fbar), _ptr(Pbar), _ptr(iters), _ptr(status))
    out = {"Fbar": Fbar, "Pbar": Pbar, "newton": iters[..., 0].astype(np.int64),
           "cg": iters[..., 1].astype(np.int64), "status": status}
    _check("mf_solve_batch", st)
    return out


class MixFFTError(RuntimeError):
    def __init__(self, call, status):
        self.status = status
        msg = _lib.mf_status_string(status).decode()
        if status == MF_CUDA_ERROR:
            msg += " [" + _lib.mf_last_cuda_error().decode() + "]"
        super().__init__(f"{call}: {msg} (status {status})")


def _check(call, status):
    if status != MF_OK:
        raise MixFFTError(call, status)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_vp)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Context:
    """One periodic cell on the current CUDA device (mf_create ... mf_destroy).

    precision: MF_FP64 or MF_FP32_INNER.  stream: a torch.cuda.Stream or None
    (the current stream).  The workspace is one torch uint8 tensor.
    """

    def __init__(self, nx, ny, nz, precision=MF_FP64, stream=None, device=None):
        import torch
        self.torch = torch
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.precision = precision
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = _vp()
        _check("mf_create", _lib.mf_create(ctypes.byref(h), nx, ny, nz, precision,
                                           _vp(self.stream.cuda_stream)))
        self.h = h
        nbytes = int(_lib.mf_workspace_bytes(h))
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        _check("mf_bind_workspace", _lib.mf_bind_workspace(h, _vp(aligned), nbytes))
        self.inner_dtype = torch.float32 if precision == MF_FP32_INNER else torch.float64

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            _lib.mf_destroy(h)
            self.h = None

    # -- problem set-up --------------------------------------------------
    def set_material(self, model, params, phase, rot=None, scale=None):
        params = _c64(params)
        phase = np.ascontiguousarray(phase, dtype=np.int32)
        rot = None if rot is None else _c64(rot)
        scale = None if scale is None else _c64(scale)
        nphase = params.shape[0]
        self.nphase = nphase
        _check("mf_set_material", _lib.mf_set_material(self.h, model, nphase, _ptr(params), _ptr(rot),
                                                       _ptr(phase), _ptr(scale)))

    def set_F(self, F=None):
        F = None if F is None else _c64(F)
        _check("mf_set_F", _lib.mf_set_F(self.h, _ptr(F)))

    # -- load history ----------------------------------------------------
    def solve(self, mask, target, tol_newton=1e-8, tol_cg=1e-10, cg_rel=1e-4, max_newton=50,
              max_cg=5000):
        mask = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1, 9)
        target = _c64(target).reshape(-1, 9)
        n = mask.shape[0]
        Fbar = np.zeros((n, 9))
        Pbar = np.zeros((n, 9))
        iters = np.zeros((n, 2), dtype=np.int32)
        st = _lib.mf_solve(self.h, n, _ptr(mask), _ptr(target), tol_newton, tol_cg, cg_rel,
                           max_newton, max_cg, _ptr(Fbar), _ptr(Pbar), _ptr(iters))
        _check("mf_solve", st)
        return {"Fbar": Fbar, "Pbar": Pbar, "newton": iters[:, 0].astype(np.int64),
                "cg": iters[:, 1].astype(np.int64)}

    def get_fields(self):
        F = np.empty((9,) + self.shape)
        P = np.empty((9,) + self.shape)
        _check("mf_get_fields", _lib.mf_get_fields(self.h, _ptr(F), _ptr(P)))
        return F, P

    def save_F(self, out=None):
        """mf_save_F: the current F into a torch FP64 CUDA tensor (9, nz, ny, nx)."""
        if out is None:
            out = self.torch.empty((9,) + self.shape, dtype=self.torch.float64, device=self.device)
        assert out.dtype == self.torch.float64 and out.is_contiguous() and out.numel() == 9 * self.N
        _check("mf_save_F", _lib.mf_save_F(self.h, _vp(out.data_ptr())))
        return out

    def load_F(self, F):
        """mf_load_F: replace the current F by a torch FP64 CUDA tensor of 9N values."""
        assert F.dtype == self.torch.float64 and F.is_contiguous() and F.numel() == 9 * self.N
        _check("mf_load_F", _lib.mf_load_F(self.h, _vp(F.data_ptr())))

    # -- operator level --------------------------------------------------
    def constitutive(self):
        _check("mf_constitutive", _lib.mf_constitutive(self.h))

    def stress(self):
        """mf_stress: P at the current F (no tangent); returns <P>."""
        meanP = np.zeros(9)
        _check("mf_stress", _lib.mf_stress(self.h, _ptr(meanP)))
        return meanP

    def get_tangent(self):
        K = np.empty((45,) + self.shape)
        _check("mf_get_tangent", _lib.mf_get_tangent(self.h, _ptr(K)))
        return K

    def matvec(self, x, y, mask):
        """y = G*(K : x); x, y: torch CUDA tensors of 9N values of the inner dtype."""
        assert x.dtype == self.inner_dtype and y.dtype == self.inner_dtype
        assert x.is_contiguous() and y.is_contiguous() and x.numel() == 9 * self.N == y.numel()
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        _check("mf_matvec", _lib.mf_matvec(self.h, _vp(x.data_ptr()), _vp(y.data_ptr()), _ptr(m)))

    def residual(self, mask, pbar, b):
        """b = -G*(P - P-bar) in FP64 into the torch tensor b; returns <P>."""
        assert b.dtype == self.torch.float64 and b.is_contiguous() and b.numel() == 9 * self.N
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        pb = _c64(pbar)
        meanP = np.zeros(9)
        _check("mf_residual", _lib.mf_residual(self.h, _ptr(m), _ptr(pb), _vp(b.data_ptr()),
                                               _ptr(meanP)))
        return meanP

    def time_kernels(self, mask, reps=20, graph=False):
        """Mean ms per launch of the four kernels of a CG iteration (tangent
        pass, x-y forward, z-pass, x-y inverse with residual update), each
        after an L2 flush; graph: timed as back-to-back graph nodes (see
        mf_time_kernels)."""
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        ms = np.zeros(4, dtype=np.float32)
        _check("mf_time_kernels", _lib.mf_time_kernels(self.h, _ptr(m), reps, 1 if graph else 0, _ptr(ms)))
        return ms.astype(np.float64)

    # -- cuFFT comparison path -------------------------------------------
    def cufft_bind(self):
        nbytes = int(_lib.mf_cufft_workspace_bytes(self.h))
        if nbytes == 0:
            raise MixFFTError("mf_cufft_workspace_bytes", MF_CUDA_ERROR)
        self.cufft_buffer = self.torch.empty(nbytes + 256, dtype=self.torch.uint8, device=self.device)
        aligned = (self.cufft_buffer.data_ptr() + 255) & ~255
        _check("mf_cufft_bind", _lib.mf_cufft_bind(self.h, _vp(aligned), nbytes))

    def matvec_cufft(self, x, y, mask):
        assert x.dtype == self.inner_dtype and y.dtype == self.inner_dtype
        assert x.is_contiguous() and y.is_contiguous() and x.numel() == 9 * self.N == y.numel()
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        _check("mf_matvec_cufft", _lib.mf_matvec_cufft(self.h, _vp(x.data_ptr()), _vp(y.data_ptr()), _ptr(m)))

    def time_cufft(self, mask, reps=20):
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        ms = np.zeros(3, dtype=np.float32)
        _check("mf_time_cufft", _lib.mf_time_cufft(self.h, _ptr(m), reps, _ptr(ms)))
        return ms.astype(np.float64)

    def autotune(self):
        """mf_autotune: returns (chosen z-pass tile width, ms per width 4/8/16,
        x-y forward schedule (0 one block per plane, 1 persistent, 2 cluster), ms of
        the forward pass per plane and persistent; mf_xy_schedule has all timings)."""
        zs = np.zeros(1, dtype=np.int32)
        ms = np.zeros(3, dtype=np.float32)
        xy = np.zeros(1, dtype=np.int32)
        xyms = np.full(2, -1.0, dtype=np.float32)
        _check("mf_autotune", _lib.mf_autotune(self.h, _ptr(zs), _ptr(ms), _ptr(xy), _ptr(xyms)))
        return int(zs[0]), ms.astype(np.float64), int(xy[0]), xyms.astype(np.float64)

    def adjoint(self, mask, wF, wP, tol_cg=1e-11, cg_rel=0.0, max_cg=20000, dscale=None):
        """mf_adjoint at the current (converged) F: returns (J, dJ/d(mu, lam)
        per phase as an (nphase, 2) array, CG iterations).  dscale: a torch
        FP64 CUDA tensor of N values that receives dJ/ds_v, or None."""
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        wF = _c64(wF)
        wP = _c64(wP)
        J = np.zeros(1)
        nphase = getattr(self, "nphase", 0)
        grad = np.zeros((max(nphase, 1), 2))
        its = np.zeros(1, dtype=np.int32)
        if dscale is not None:
            assert dscale.dtype == self.torch.float64 and dscale.is_contiguous() and dscale.numel() == self.N
        _check("mf_adjoint", _lib.mf_adjoint(self.h, _ptr(m), _ptr(wF), _ptr(wP), tol_cg, cg_rel, max_cg,
                                             _ptr(J), _ptr(grad),
                                             None if dscale is None else _vp(dscale.data_ptr()), _ptr(its)))
        return float(J[0]), grad[:nphase], int(its[0])

    def set_xy_split(self, split):
        """mf_set_xy_split: 0 fused x-y plane kernels, 1 separate row/column kernels."""
        _check("mf_set_xy_split", _lib.mf_set_xy_split(self.h, int(split)))

    def set_projection_arith(self, arith):
        """mf_set_projection_arith: MF_PROJ_FP32, MF_PROJ_OUTER or MF_PROJ_AUTO (default) for the
        projection of each FP32 correction."""
        _check("mf_set_projection_arith", _lib.mf_set_projection_arith(self.h, int(arith)))

    def set_xy_persistent(self, on):
        """mf_set_xy_persistent: 1 persistent bulk-copy FP32 x-y forward kernel, 0 one block per plane."""
        _check("mf_set_xy_persistent", _lib.mf_set_xy_persistent(self.h, int(on)))

    def set_xy_cluster(self, which):
        """mf_set_xy_cluster: two-CTA cluster FP32 x-y kernels, bit 0 forward, bit 1 inverse."""
        _check("mf_set_xy_cluster", _lib.mf_set_xy_cluster(self.h, int(which)))

    def xy_schedule(self):
        """mf_xy_schedule: (forward schedule 0/1/2, inverse schedule 0/2, the autotuner's
        ms for forward per plane / persistent / cluster and inverse per plane / cluster)."""
        f = np.zeros(1, np.int32)
        i = np.zeros(1, np.int32)
        ms = np.zeros(5, np.float32)
        _check("mf_xy_schedule", _lib.mf_xy_schedule(self.h, _ptr(f), _ptr(i), _ptr(ms)))
        return int(f[0]), int(i[0]), ms

    def set_outer_arith(self, arith):
        """mf_set_outer_arith: MF_OUTER_DOUBLE_WORD or MF_OUTER_FP64."""
        _check("mf_set_outer_arith", _lib.mf_set_outer_arith(self.h, arith))

    def set_predictor(self, kind):
        """mf_set_predictor: MF_PRED_UNIFORM (default), MF_PRED_EXTRAPOLATE or MF_PRED_QUADRATIC."""
        _check("mf_set_predictor", _lib.mf_set_predictor(self.h, int(kind)))

    def set_inexact_newton(self, on):
        """mf_set_inexact_newton: the FP32-inner forcing sequence for the CG
        solves of an FP64 context (1) or the absolute CG tolerance (0)."""
        _check("mf_set_inexact_newton", _lib.mf_set_inexact_newton(self.h, int(on)))

    def sync(self):
        _check("mf_sync", _lib.mf_sync(self.h))


def selftest_wait_timeout(max_polls=1000):
    """mf_selftest_wait_timeout: the library's status for a bounded device
    wait that runs out (MF_DEVICE_TIMEOUT when the mechanism works)."""
    return int(_lib.mf_selftest_wait_timeout(int(max_polls)))
