"""Python binding of librve.so, the GB300 (sm_103a) implementation of one
strain increment of FFT-Galerkin homogenisation with lower-order
strain-gradient crystal plasticity (Haouala, Lucarini, LLorca, Segurado,
arXiv:1910.01946).

This module only marshals arguments: every step of the increment runs in the
library's CUDA kernels.  PyTorch provides the device workspace and the CUDA
stream.  The functions ``rve_*`` mirror the C ABI of ``include/rve.h`` one to
one; ``RVE`` wraps a handle.  Importing works without a GPU; any call into the
library raises if librve.so has not been built or no CUDA device is present.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librve.so")

RVE_OK, RVE_EINVAL, RVE_ENOMEM, RVE_ECUDA = 0, 1, 2, 3
RVE_ENOCONV_LOCAL, RVE_ENOCONV_CG, RVE_ENOCONV_NEWTON, RVE_ENAN, RVE_ETIMEOUT = 4, 5, 6, 7, 8
STATUS_NAMES = {0: "RVE_OK", 1: "RVE_EINVAL", 2: "RVE_ENOMEM", 3: "RVE_ECUDA", 4: "RVE_ENOCONV_LOCAL",
                5: "RVE_ENOCONV_CG", 6: "RVE_ENOCONV_NEWTON", 7: "RVE_ENAN", 8: "RVE_ETIMEOUT"}

FIELDS = {"F": (0, 9), "P": (1, 9), "FP": (2, 9), "S": (3, 6), "SIGMA": (4, 9), "RHO_SSD": (5, 12),
          "RHO_GND": (6, 12), "RHO_GND18": (7, 18), "NYE": (8, 9), "VM": (9, 1), "TAUC": (10, 12),
          "DGAM": (11, 12), "TANGENT": (12, 81), "GRAIN": (13, 1), "P_EVAL": (14, 9), "S_EVAL": (15, 6)}

MAX_NEWTON_LOG = 64
KERNELS = ("fft_x_r2c", "fft_y", "fft_z_op", "fft_x_c2r", "constitutive", "hardening", "tangent_apply",
           "cg_update", "reduce", "other", "stencil", "tangent_build", "fft_curl", "fft_y_inv")


class rve_material(C.Structure):
    _fields_ = [("C11", C.c_double), ("C12", C.c_double), ("C44", C.c_double), ("b", C.c_double),
                ("mu", C.c_double), ("tau0", C.c_double), ("alpha", C.c_double), ("q", C.c_double * 6),
                ("q_normalise", C.c_int32), ("gdot0", C.c_double), ("n", C.c_double), ("K", C.c_double),
                ("yc", C.c_double), ("rho0_total", C.c_double), ("gnd_enabled", C.c_int32)]


class rve_options(C.Structure):
    _fields_ = [("L", C.c_double), ("newton_tol", C.c_double), ("cg_tol", C.c_double),
                ("local_tol", C.c_double), ("max_newton", C.c_int32), ("max_cg", C.c_int32),
                ("max_local", C.c_int32), ("max_halvings", C.c_int32), ("extrapolate", C.c_int32),
                ("precision", C.c_int32), ("cg_adaptive", C.c_int32), ("krylov", C.c_int32),
                ("graphs", C.c_int32), ("tma", C.c_int32), ("autotune", C.c_int32), ("stencils", C.c_int32),
                ("continuation", C.c_int32)]


class rve_step_info(C.Structure):
    _fields_ = [("converged", C.c_int32), ("newton_iters", C.c_int32), ("cg_iters_total", C.c_int32),
                ("local_max_iters", C.c_int32), ("local_failures", C.c_int32), ("halvings", C.c_int32),
                ("bicgstab_solves", C.c_int32), ("load_stages", C.c_int32), ("local_iters_total", C.c_int64),
                ("local_evals_total", C.c_int64),
                ("residual", C.c_double), ("seconds", C.c_double), ("cg_iters", C.c_int32 * MAX_NEWTON_LOG),
                ("residuals", C.c_double * (MAX_NEWTON_LOG + 1))]


_SIGS = {
    "rve_workspace_bytes": (C.c_size_t, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]),
    "rve_create": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int,
                             C.POINTER(rve_material), C.POINTER(rve_options), C.c_void_p, C.c_size_t,
                             C.c_void_p, C.POINTER(C.c_void_p)]),
    "rve_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                           C.POINTER(rve_step_info)]),
    "rve_step_batch": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p]),
    "rve_get_macro_stress": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "rve_get_fields": (C.c_int, [C.c_void_p, C.c_uint32, C.c_void_p, C.c_size_t, C.c_int]),
    "rve_set_fields": (C.c_int, [C.c_void_p, C.c_uint32, C.c_void_p, C.c_size_t, C.c_int]),
    "rve_eval_hardening": (C.c_int, [C.c_void_p]),
    "rve_eval_nye": (C.c_int, [C.c_void_p, C.c_int]),
    "rve_eval_constitutive": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "rve_project": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rve_checkpoint_bytes": (C.c_size_t, [C.c_void_p]),
    "rve_checkpoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "rve_restore": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "rve_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "rve_get_tuning": (C.c_int, [C.c_void_p, C.c_void_p]),
    "rve_kernel_stats": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "rve_set_wait_limit": (C.c_int, [C.c_void_p, C.c_uint32]),
    "rve_time_fft": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double)]),
    "rve_project_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_double, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p]),
    "rve_sensitivity_bytes": (C.c_size_t, [C.c_void_p]),
    "rve_sensitivity_enable": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_double]),
    "rve_get_stress_sensitivity": (C.c_int, [C.c_void_p, C.c_void_p]),
    "rve_last_error": (C.c_char_p, [C.c_void_p]),
    "rve_destroy": (None, [C.c_void_p]),
}
EXPORTED = tuple(_SIGS)

_lib = None


def load_library(path: str = LIB_PATH):
    """Load librve.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1910_01946_gb300._build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class RVEError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# ---- thin wrappers with the C names ---------------------------------------
def rve_workspace_bytes(n0, n1, n2, n_grains, precision=0):
    return load_library().rve_workspace_bytes(n0, n1, n2, n_grains, precision)


def rve_create(grain_id, n0, n1, n2, quat, n_grains, mat, opt, d_workspace, ws_bytes, stream):
    handle = C.c_void_p()
    st = load_library().rve_create(_ptr(grain_id), n0, n1, n2, _ptr(quat), n_grains, C.byref(mat), C.byref(opt),
                                   C.c_void_p(d_workspace), ws_bytes, C.c_void_p(stream), C.byref(handle))
    return st, handle


def rve_step(h, dFbar, mask, Pbar, dt, info=None):
    return load_library().rve_step(h, _ptr(dFbar), _ptr(mask), _ptr(Pbar), dt,
                                   C.byref(info) if info is not None else None)


def rve_step_batch(handles, dFbar, mask, Pbar, dt, infos=None, status=None):
    """handles: sequence of handle pointers; dFbar, Pbar: (n, 9) float64;
    mask: (n, 9) uint8; dt: (n,) float64; infos: ctypes array of rve_step_info
    or None; status: (n,) int32 array or None."""
    n = len(handles)
    harr = (C.c_void_p * n)(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    return load_library().rve_step_batch(harr, n, _ptr(dFbar), _ptr(mask), _ptr(Pbar), _ptr(dt),
                                         C.cast(infos, C.c_void_p) if infos is not None else None,
                                         _ptr(status) if status is not None else None)


def step_batch(rves, dFbar, mask, Pbar, dt):
    """Advance RVE objects by one increment each, concurrently (their own streams).
    dFbar, Pbar: (n, 9); mask: (9,) or (n, 9); dt: scalar or (n,).  Returns the
    per-handle step dictionaries; raises on the first failed status."""
    n = len(rves)
    dF = np.ascontiguousarray(np.broadcast_to(np.asarray(dFbar, dtype=np.float64).reshape(-1, 9), (n, 9)))
    Pb = np.ascontiguousarray(np.broadcast_to(np.asarray(Pbar, dtype=np.float64).reshape(-1, 9), (n, 9)))
    mk = np.ascontiguousarray(np.broadcast_to(np.asarray(mask, dtype=np.uint8).reshape(-1, 9), (n, 9)))
    dts = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64).reshape(-1), (n,)))
    infos = (rve_step_info * n)()
    status = np.zeros(n, dtype=np.int32)
    rve_step_batch([r.h for r in rves], dF, mk, Pb, dts, infos, status)
    out = []
    for i, r in enumerate(rves):
        inf = infos[i]
        out.append(dict(status=int(status[i]), converged=bool(inf.converged), newton_iters=inf.newton_iters,
                        cg_iters_total=inf.cg_iters_total, local_iters_total=inf.local_iters_total,
                        local_evals_total=inf.local_evals_total, residual=inf.residual, seconds=inf.seconds))
        if status[i] != RVE_OK:
            raise RVEError(int(status[i]), f"rve_step_batch[{i}]: {rve_last_error(r.h)}")
    return out


def rve_get_macro_stress(h, P, sig):
    return load_library().rve_get_macro_stress(h, _ptr(P), _ptr(sig))


def rve_get_fields(h, which, dst_ptr, nbytes, dst_is_device):
    return load_library().rve_get_fields(h, which, C.c_void_p(dst_ptr), nbytes, dst_is_device)


def rve_set_fields(h, which, src_ptr, nbytes, src_is_device):
    return load_library().rve_set_fields(h, which, C.c_void_p(src_ptr), nbytes, src_is_device)


def rve_eval_hardening(h):
    return load_library().rve_eval_hardening(h)


def rve_eval_constitutive(h, dt):
    it, nf = C.c_int32(), C.c_int32()
    st = load_library().rve_eval_constitutive(h, dt, C.byref(it), C.byref(nf))
    return st, it.value, nf.value


def rve_project(h, mask, d_X, d_Y):
    return load_library().rve_project(h, _ptr(mask), C.c_void_p(d_X), C.c_void_p(d_Y))


def rve_checkpoint_bytes(h):
    return load_library().rve_checkpoint_bytes(h)


def rve_checkpoint(h, buf):
    return load_library().rve_checkpoint(h, _ptr(buf), buf.nbytes)


def rve_restore(h, buf):
    return load_library().rve_restore(h, _ptr(buf), buf.nbytes)


def rve_profile(h, enable):
    return load_library().rve_profile(h, int(enable))


def rve_kernel_stats(h, launches, ms):
    return load_library().rve_kernel_stats(h, _ptr(launches), _ptr(ms))


def rve_project_noalloc(n0, n1, n2, L, mask, d_X, d_Y, stream):
    """Y = G*(X) with the library's static scratch (no allocation; asynchronous on `stream`)."""
    return load_library().rve_project_noalloc(n0, n1, n2, float(L), _ptr(mask), C.c_void_p(d_X),
                                              C.c_void_p(d_Y), C.c_void_p(stream))


PARAMS = ("tau0", "K", "alpha", "b")   # order of the sensitivity parameters


def rve_sensitivity_bytes(h):
    return load_library().rve_sensitivity_bytes(h)


def rve_sensitivity_enable(h, d_workspace, nbytes, tol=0.0):
    return load_library().rve_sensitivity_enable(h, C.c_void_p(d_workspace), nbytes, float(tol))


def rve_get_stress_sensitivity(h, out):
    return load_library().rve_get_stress_sensitivity(h, _ptr(out))


def rve_last_error(h):
    s = load_library().rve_last_error(h)
    return s.decode() if s else ""


def rve_destroy(h):
    load_library().rve_destroy(h)


# ---- handle wrapper ---------------------------------------------------------
DEFAULT_OPTIONS = dict(newton_tol=1e-11, cg_tol=1e-11, local_tol=1e-14, max_newton=100, max_cg=2000,
                       max_local=60, max_halvings=12, extrapolate=1, precision=0, cg_adaptive=1, krylov=0, graphs=1, tma=1, autotune=0,
                       stencils=0, continuation=2)


def make_material(m) -> rve_material:
    """From an object or dict with the fields of rvegen.Material."""
    g = (lambda k: m[k]) if isinstance(m, dict) else (lambda k: getattr(m, k))
    out = rve_material()
    for k in ("C11", "C12", "C44", "b", "mu", "tau0", "alpha", "gdot0", "n", "K", "yc", "rho0_total"):
        setattr(out, k, float(g(k)))
    for i, v in enumerate(g("q")):
        out.q[i] = float(v)
    out.q_normalise = 1 if g("q_normalise") else 0
    out.gnd_enabled = 1 if g("gnd_enabled") else 0
    return out


def make_options(L, **kw) -> rve_options:
    d = dict(DEFAULT_OPTIONS)
    d.update(kw)
    o = rve_options()
    o.L = float(L)
    for k, v in d.items():
        setattr(o, k, v)
    return o


class RVE:
    """One voxelised polycrystal on one GPU.

    grain_id: int array of numpy shape (n2, n1, n0) (x fastest); quat:
    (n_grains, 4) unit quaternions (w, x, y, z); mat: rvegen.Material-like;
    L: RVE edge along x [m].  The workspace is a torch uint8 tensor on
    ``device``; the stream is torch's current stream on that device.
    """

    def __init__(self, grain_id, quat, mat, L, device="cuda:0", stream=None, own_stream=False, **options):
        import torch
        lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the GB300 path has no CPU fallback")
        self.torch = torch
        self.device = torch.device(device)
        gid = np.ascontiguousarray(grain_id, dtype=np.int32)
        self.shape = gid.shape
        n2, n1, n0 = gid.shape
        self.n = (n0, n1, n2)
        self.nvox = gid.size
        q = np.ascontiguousarray(quat, dtype=np.float64).reshape(-1, 4)
        self.n_grains = q.shape[0]
        self.mat = make_material(mat)
        self.opt = make_options(L, **options)
        self.ws_bytes = lib.rve_workspace_bytes(n0, n1, n2, self.n_grains, self.opt.precision)
        if self.ws_bytes == 0:
            raise RVEError(RVE_EINVAL, f"unsupported grid {self.n} / grains {self.n_grains}")
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
            if stream is not None:
                self.stream = stream
            elif own_stream:          # a stream of its own (concurrent batched steps)
                self.stream = torch.cuda.Stream(self.device)
            else:
                self.stream = torch.cuda.current_stream(self.device)
        st, h = rve_create(gid, n0, n1, n2, q, self.n_grains, self.mat, self.opt, self.workspace.data_ptr(),
                           self.ws_bytes, self.stream.cuda_stream)
        if st != RVE_OK:
            raise RVEError(st, "rve_create failed")
        self.h = h

    def _check(self, st, what):
        if st != RVE_OK:
            raise RVEError(st, f"{what}: {rve_last_error(self.h)}")

    def step(self, dFbar, mask, Pbar, dt, check=True):
        info = rve_step_info()
        st = rve_step(self.h, np.ascontiguousarray(dFbar, dtype=np.float64).reshape(9),
                      np.ascontiguousarray(mask, dtype=np.uint8).reshape(9),
                      np.ascontiguousarray(Pbar, dtype=np.float64).reshape(9), float(dt), info)
        out = dict(status=st, converged=bool(info.converged), newton_iters=info.newton_iters,
                   # a failed step also reports the Krylov iterations of the iteration that failed
                   cg_iters=list(info.cg_iters[:min(info.newton_iters + (0 if info.converged else 1),
                                                    MAX_NEWTON_LOG)]),
                   cg_iters_total=info.cg_iters_total, local_max_iters=info.local_max_iters,
                   local_failures=info.local_failures, halvings=info.halvings, residual=info.residual,
                   local_iters_total=info.local_iters_total, local_evals_total=info.local_evals_total,
                   bicgstab_solves=info.bicgstab_solves, load_stages=info.load_stages,
                   residuals=list(info.residuals[:min(info.newton_iters, MAX_NEWTON_LOG) + 1]),
                   seconds=info.seconds)
        if check:
            self._check(st, "rve_step")
        return out

    def enable_sensitivity(self, tol=0.0):
        """Carry d/d(tau0, K, alpha, b) through every following increment (the
        current state is taken as parameter-independent); workspace from torch."""
        n = rve_sensitivity_bytes(self.h)
        with self.torch.cuda.device(self.device):
            self.sens_workspace = self.torch.empty(n + 256, dtype=self.torch.uint8, device=self.device)
        base = self.sens_workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        self._check(rve_sensitivity_enable(self.h, aligned, n, tol), "rve_sensitivity_enable")

    def set_wait_limit(self, polls: int):
        """Poll limit of the per-tile wait in the staged FP32 tangent apply (0: give up at once)."""
        self._check(load_library().rve_set_wait_limit(self.h, int(polls)), "rve_set_wait_limit")

    def time_fft(self, nf=3, fp32=False, reps=20):
        """Average device milliseconds of one forward + inverse FFT of nf fields
        (the hand-written transforms alone, on the handle's buffers)."""
        ms = C.c_double()
        self._check(load_library().rve_time_fft(self.h, int(nf), int(bool(fp32)), int(reps), C.byref(ms)),
                    "rve_time_fft")
        return ms.value

    def tuning(self):
        """Launch shapes in use: divergence grid cap, FFT fill targets (x, y, z passes), staged FP32
        apply, autotuned."""
        out = np.zeros(6, dtype=np.int32)
        self._check(load_library().rve_get_tuning(self.h, _ptr(out)), "rve_get_tuning")
        return dict(div_blocks=int(out[0]), fft_fill=int(out[1]), tma=bool(out[2]), autotuned=bool(out[3]),
                    fft_fill_y=int(out[4]), fft_fill_z=int(out[5]))

    def stress_sensitivity(self):
        """d<P>/d theta of the last increment, shape (4, 3, 3), theta = PARAMS."""
        out = np.zeros(36)
        self._check(rve_get_stress_sensitivity(self.h, out), "rve_get_stress_sensitivity")
        return out.reshape(4, 3, 3)

    def macro_stress(self):
        P, s = np.zeros(9), np.zeros(9)
        self._check(rve_get_macro_stress(self.h, P, s), "rve_get_macro_stress")
        return P.reshape(3, 3), s.reshape(3, 3)

    def field(self, name, device=False):
        """Field as numpy (n2, n1, n0, ncomp) (device=False) or a torch tensor (ncomp, nvox)."""
        which, nc = FIELDS[name]
        dt = np.int32 if name == "GRAIN" else np.float64
        if device:
            t = self.torch.empty((nc, self.nvox), dtype=self.torch.int32 if name == "GRAIN" else self.torch.float64,
                                 device=self.device)
            self._check(rve_get_fields(self.h, which, t.data_ptr(), t.numel() * t.element_size(), 1), "get_fields")
            return t
        a = np.empty((nc, self.nvox), dtype=dt)
        self._check(rve_get_fields(self.h, which, a.ctypes.data, a.nbytes, 0), "get_fields")
        return np.moveaxis(a.reshape((nc,) + self.shape), 0, -1)

    def set_field(self, name, arr):
        """Set F, FP or RHO_SSD from numpy (n2, n1, n0, ncomp)."""
        which, nc = FIELDS[name]
        a = np.ascontiguousarray(np.moveaxis(np.asarray(arr, dtype=np.float64).reshape(self.shape + (nc,)), -1, 0))
        self._check(rve_set_fields(self.h, which, a.ctypes.data, a.nbytes, 0), "set_fields")

    def eval_hardening(self):
        self._check(rve_eval_hardening(self.h), "rve_eval_hardening")

    def eval_nye(self, scheme=0):
        """Nye tensor of the committed Fp into field NYE: scheme 0 rotated (the
        method's), 1 standard spectral derivative (for comparison)."""
        self._check(load_library().rve_eval_nye(self.h, int(scheme)), "rve_eval_nye")

    def eval_constitutive(self, dt):
        st, it, nf = rve_eval_constitutive(self.h, float(dt))
        self._check(st, "rve_eval_constitutive")
        return it, nf

    def project(self, mask, X, Y=None):
        """G*(X) for a device tensor X of shape (9, nvox), float64."""
        Y = self.torch.empty_like(X) if Y is None else Y
        assert X.dtype == self.torch.float64 and X.is_contiguous() and X.numel() == 9 * self.nvox
        self._check(rve_project(self.h, np.ascontiguousarray(mask, dtype=np.uint8).reshape(9), X.data_ptr(),
                                Y.data_ptr()), "rve_project")
        return Y

    def profile(self, enable: bool):
        """Reset the kernel counters; time every launch with CUDA events while enabled."""
        self._check(rve_profile(self.h, enable), "rve_profile")

    def kernel_stats(self):
        """{kernel category: (launches, device milliseconds)} since the last profile() call."""
        n = np.zeros(len(KERNELS), dtype=np.int64)
        ms = np.zeros(len(KERNELS), dtype=np.float64)
        self._check(rve_kernel_stats(self.h, n, ms), "rve_kernel_stats")
        return {k: (int(n[i]), float(ms[i])) for i, k in enumerate(KERNELS)}

    def checkpoint(self) -> np.ndarray:
        buf = np.empty(rve_checkpoint_bytes(self.h), dtype=np.uint8)
        self._check(rve_checkpoint(self.h, buf), "rve_checkpoint")
        return buf

    def restore(self, buf: np.ndarray):
        self._check(rve_restore(self.h, np.ascontiguousarray(buf, dtype=np.uint8)), "rve_restore")

    def close(self):
        if getattr(self, "h", None):
            rve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
