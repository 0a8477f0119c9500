"""Python binding of the sqrtba C ABI (include/sqrtba.h).

Square root bundle adjustment (Demmel et al., CVPR 2021) on GB300: the
binding only marshals arguments; every step of the solver runs in the CUDA
kernels of libsqrtba.so.  There is no CPU fallback: if the library has not
been built, importing works but any call raises BAError.

    from paper_2103_01843_gb300 import Problem
    with Problem(cams, pts, obs_cam, obs_pt, obs_xy) as p:
        reports = p.solve()
        cams, pts = p.get_params()

Function names follow the C ABI (ba_create -> Problem(), ba_linearize ->
Problem.linearize, ...).  PyTorch, when used, only supplies the CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsqrtba.so")

BA_OK = 0
STATUS_NAMES = {0: "BA_OK", 1: "BA_ERR_INVALID_ARG", 2: "BA_ERR_OOM", 3: "BA_ERR_CUDA",
                4: "BA_ERR_STATE", 5: "BA_ERR_NUMERIC", 6: "BA_ERR_TIMEOUT"}


class BAError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("lambda0", ctypes.c_double), ("max_lm_iters", ctypes.c_int32),
                ("func_tol", ctypes.c_double), ("max_cg_iters", ctypes.c_int32),
                ("cg_eta", ctypes.c_double), ("use_graph", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("use_learned", ctypes.c_int32),
                ("pipeline_stages", ctypes.c_int32), ("target_cost", ctypes.c_double),
                ("precond_from_blocks", ctypes.c_int32), ("implicit_blocks", ctypes.c_int32),
                ("huber_delta", ctypes.c_double), ("schur_explicit", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class PcgReport(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("stop_reason", ctypes.c_int32),
                ("residual_norm", ctypes.c_double), ("rhs_norm", ctypes.c_double),
                ("learned", ctypes.c_int32), ("warm_start", ctypes.c_int32),
                ("precond_fallbacks", ctypes.c_int32), ("precond_exact", ctypes.c_int32)]


class LmReport(ctypes.Structure):
    _fields_ = [("iteration", ctypes.c_int32), ("accepted", ctypes.c_int32),
                ("relinearized", ctypes.c_int32), ("cg_iters", ctypes.c_int32),
                ("stop", ctypes.c_int32), ("pcg_stop_reason", ctypes.c_int32),
                ("cost", ctypes.c_double), ("new_cost", ctypes.c_double),
                ("model_cost", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("rho", ctypes.c_double), ("precond_fallbacks", ctypes.c_int32),
                ("precond_exact", ctypes.c_int32)]


class LmState(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("nu", ctypes.c_double),
                ("iteration", ctypes.c_int32), ("stopped", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("n_cam", ctypes.c_int32), ("n_pt", ctypes.c_int32), ("n_obs", ctypes.c_int64),
                ("a_pool_floats", ctypes.c_int64), ("sum_k2", ctypes.c_int64),
                ("k_max", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64)]


class Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 8), ("count", ctypes.c_int64 * 8),
                ("kernel_launches", ctypes.c_int64), ("h2d_bytes", ctypes.c_int64),
                ("d2h_bytes", ctypes.c_int64)]


class TuneReport(ctypes.Structure):
    _fields_ = [("ksmall", ctypes.c_int32), ("small_bytes", ctypes.c_int32),
                ("matvec_ms", ctypes.c_double), ("default_ms", ctypes.c_double),
                ("tune_ms", ctypes.c_double), ("pc_ksmall", ctypes.c_int32),
                ("pc_small_bytes", ctypes.c_int32), ("ns", ctypes.c_int32), ("y_smem", ctypes.c_int32),
                ("pc_ns", ctypes.c_int32), ("big8_kmax", ctypes.c_int32)]


class ProblemDesc(ctypes.Structure):
    _fields_ = [("cams", ctypes.POINTER(ctypes.c_double)), ("n_cam", ctypes.c_int32),
                ("pts", ctypes.POINTER(ctypes.c_double)), ("n_pt", ctypes.c_int32),
                ("obs_cam", ctypes.POINTER(ctypes.c_int32)), ("obs_pt", ctypes.POINTER(ctypes.c_int32)),
                ("obs_xy", ctypes.POINTER(ctypes.c_double)), ("n_obs", ctypes.c_int64)]


class BatchReport(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("accepted", ctypes.c_int32),
                ("cg_iters", ctypes.c_int32), ("stop", ctypes.c_int32),
                ("initial_cost", ctypes.c_double), ("final_cost", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("solve_ms", ctypes.c_double)]


class BatchSummary(ctypes.Structure):
    _fields_ = [("n_problems", ctypes.c_int32), ("lm_iterations", ctypes.c_int32),
                ("tuned_ksmall", ctypes.c_int32), ("tuned_small_bytes", ctypes.c_int32),
                ("total_ms", ctypes.c_double), ("tune_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64)]


PROFILE_SLOTS = ("linearize", "damp", "precond", "matvec", "unused", "backsub", "cost")


def _struct_dict(s):
    return {name.rstrip("_"): getattr(s, name) for name, _ in s._fields_ if not name.startswith("reserved")}


_lib = None
_lock = threading.Lock()

_P = ctypes.c_void_p
_d = ctypes.POINTER(ctypes.c_double)
_f = ctypes.POINTER(ctypes.c_float)
_i32 = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.POINTER(ctypes.c_int64)

# name -> argtypes (restype ba_status = int unless noted)
_SIGS = {
    "ba_create": [_d, ctypes.c_int32, _d, ctypes.c_int32, _i32, _i32, _d, ctypes.c_int64,
                  ctypes.POINTER(Options), _P, ctypes.POINTER(_P)],
    "ba_destroy": [_P],
    "ba_linearize": [_P],
    "ba_marginalize_qr": [_P, ctypes.c_double],
    "ba_linearize_damped": [_P, ctypes.c_double],
    "ba_pcg_solve": [_P, ctypes.POINTER(PcgReport)],
    "ba_backsubstitute": [_P, _d],
    "ba_eval_cost": [_P, ctypes.c_int32, _d],
    "ba_lm_step": [_P, ctypes.POINTER(LmReport)],
    "ba_solve": [_P, ctypes.POINTER(LmReport), ctypes.c_int32, _i32],
    "ba_get_params": [_P, _d, _d],
    "ba_set_params": [_P, _d, _d],
    "ba_get_state": [_P, ctypes.POINTER(LmState)],
    "ba_set_options": [_P, ctypes.POINTER(Options)],
    "ba_set_state": [_P, ctypes.POINTER(LmState)],
    "ba_get_info": [_P, ctypes.POINTER(Info)],
    "ba_set_profiling": [_P, ctypes.c_int32],
    "ba_get_profile": [_P, ctypes.POINTER(Profile)],
    "ba_eval_cost_noalloc": [_P, ctypes.c_int32, _P, ctypes.c_int32, _P, _P, _P, ctypes.c_int64, _P, _P],
    "ba_autotune": [_P, ctypes.POINTER(TuneReport)],
    "ba_batch_create": [ctypes.POINTER(ProblemDesc), ctypes.c_int32, ctypes.POINTER(Options), _P,
                        ctypes.POINTER(_P)],
    "ba_batch_destroy": [_P],
    "ba_batch_solve": [_P, ctypes.POINTER(BatchReport), ctypes.POINTER(BatchSummary)],
    "ba_batch_restart": [_P],
    "ba_batch_get_params": [_P, ctypes.c_int32, _d, _d],
    "ba_batch_set_profiling": [_P, ctypes.c_int32],
    "ba_batch_get_profile": [_P, ctypes.POINTER(Profile)],
    "ba_batch_get_info": [_P, ctypes.POINTER(Info)],
    "ba_batch_iterations": [_P, ctypes.c_int32, _i32, _f, _i32],
    "ba_mlp_create": [_f, _P, ctypes.POINTER(_P)],
    "ba_mlp_destroy": [_P],
    "ba_mlp_get_params": [_P, _f],
    "ba_mlp_forward": [_P, _P, ctypes.c_int32, _P],
    "ba_mlp_prepare": [_P, _P, _P, _P, _P, ctypes.c_int32, _P, _P],
    "ba_mlp_loss_grad": [_P, _P, _P, ctypes.c_int32, _d, _f],
    "ba_mlp_train_step": [_P, _P, _P, ctypes.c_int32, ctypes.c_float, _d],
    "ba_set_learned": [_P, _P],
    "ba_learned_fallbacks": [_P, _i64],
    "ba_debug_export_order": [_P, _i32, _i64, _i64, _i32],
    "ba_debug_export_landmark": [_P, ctypes.c_int32, ctypes.c_int32, _f, _f, _f, _f, _i32],
    "ba_debug_export_damping": [_P, _f, _f],
    "ba_debug_export_jacobians": [_P, _f, _f, _f],
    "ba_debug_export_rcs_diag": [_P, _f, _f],
    "ba_debug_matvec": [_P, _f, _f],
    "ba_debug_fail_matvec": [_P, ctypes.c_int32, ctypes.c_double],
    "ba_debug_export_step": [_P, _f, _f],
}


def lib():
    """The loaded libsqrtba.so; raises BAError if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise BAError(3, f"{LIB_PATH} is missing: build it with "
                                 "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(LIB_PATH)
            for name, args in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            L.ba_default_options.argtypes = [ctypes.POINTER(Options)]
            L.ba_default_options.restype = None
            L.ba_last_error.argtypes = [_P]
            L.ba_last_error.restype = ctypes.c_char_p
            L.ba_batch_last_error.argtypes = [_P]
            L.ba_batch_last_error.restype = ctypes.c_char_p
            L.ba_mlp_last_error.argtypes = [_P]
            L.ba_mlp_last_error.restype = ctypes.c_char_p
            _lib = L
    return _lib


def exported_symbols():
    """Names the binding expects the library to export."""
    return sorted(list(_SIGS) + ["ba_default_options", "ba_last_error", "ba_batch_last_error",
                                 "ba_mlp_last_error"])


def default_options(**kw):
    o = Options()
    lib().ba_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(a, t):
    return a.ctypes.data_as(t)


def _devptr(x):
    """Device address of a tensor-like object (data_ptr()) or an int."""
    return int(x.data_ptr()) if hasattr(x, "data_ptr") else int(x)


def eval_cost_noalloc(cams, pts, obs_cam, obs_pt, obs_xy, out, n_cam=None, n_pt=None, n_obs=None, stream=None):
    """ba_eval_cost_noalloc: E of device-resident FP32 data written to the
    device double `out`, with no device allocation.  Arguments are CUDA
    tensors (or raw device addresses with explicit sizes); enqueued on
    `stream` without synchronising."""
    n_cam = n_cam if n_cam is not None else cams.shape[0]
    n_pt = n_pt if n_pt is not None else pts.shape[0]
    n_obs = n_obs if n_obs is not None else obs_cam.shape[0]
    rc = lib().ba_eval_cost_noalloc(_devptr(cams), int(n_cam), _devptr(pts), int(n_pt), _devptr(obs_cam),
                                    _devptr(obs_pt), _devptr(obs_xy), int(n_obs), _devptr(out),
                                    _P(stream) if stream else None)
    if rc != BA_OK:
        raise BAError(rc, lib().ba_last_error(None).decode())


class Problem:
    """One bundle-adjustment problem resident on the GPU (ba_create)."""

    def __init__(self, cams, pts, obs_cam, obs_pt, obs_xy, options=None, stream=None, **kw):
        L = lib()
        self._cams = np.ascontiguousarray(cams, np.float64)
        self._pts = np.ascontiguousarray(pts, np.float64)
        oc = np.ascontiguousarray(obs_cam, np.int32)
        op = np.ascontiguousarray(obs_pt, np.int32)
        xy = np.ascontiguousarray(obs_xy, np.float64)
        self.n_cam, self.n_pt, self.n_obs = self._cams.shape[0], self._pts.shape[0], oc.shape[0]
        opt = options if options is not None else default_options(**kw)
        h = _P()
        st = _P(stream) if stream else None
        rc = L.ba_create(_ptr(self._cams, _d), self.n_cam, _ptr(self._pts, _d), self.n_pt,
                         _ptr(oc, _i32), _ptr(op, _i32), _ptr(xy, _d), self.n_obs,
                         ctypes.byref(opt), st, ctypes.byref(h))
        if rc != BA_OK:
            raise BAError(rc, L.ba_last_error(None).decode())
        self.h = h
        self.options = opt

    @classmethod
    def from_scene(cls, scene, **kw):
        return cls(scene.cams, scene.pts, scene.obs_cam, scene.obs_pt, scene.obs_xy, **kw)

    # --- lifetime -------------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            lib().ba_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != BA_OK:
            raise BAError(rc, lib().ba_last_error(self.h).decode())

    # --- the hot path -----------------------------------------------------------
    def linearize(self):
        self._check(lib().ba_linearize(self.h))

    def linearize_damped(self, lam):
        self._check(lib().ba_linearize_damped(self.h, float(lam)))

    def marginalize_qr(self, lam):
        self._check(lib().ba_marginalize_qr(self.h, float(lam)))

    def pcg_solve(self):
        r = PcgReport()
        self._check(lib().ba_pcg_solve(self.h, ctypes.byref(r)))
        return _struct_dict(r)

    def backsubstitute(self):
        m = ctypes.c_double()
        self._check(lib().ba_backsubstitute(self.h, ctypes.byref(m)))
        return m.value

    def eval_cost(self, candidate=False):
        c = ctypes.c_double()
        self._check(lib().ba_eval_cost(self.h, 1 if candidate else 0, ctypes.byref(c)))
        return c.value

    def lm_step(self):
        r = LmReport()
        self._check(lib().ba_lm_step(self.h, ctypes.byref(r)))
        return _struct_dict(r)

    def set_target_cost(self, target):
        """Stop the LM after an accepted step with cost <= target (0: off)."""
        self.options.target_cost = float(target)
        self._check(lib().ba_set_options(self.h, ctypes.byref(self.options)))

    def solve(self, max_reports=1000):
        reps = (LmReport * max_reports)()
        n = ctypes.c_int32()
        self._check(lib().ba_solve(self.h, reps, max_reports, ctypes.byref(n)))
        return [_struct_dict(r) for r in reps[: min(n.value, max_reports)]]

    # --- state ------------------------------------------------------------------
    def get_params(self):
        c = np.empty((self.n_cam, 9))  # every element is written by the call
        p = np.empty((self.n_pt, 3))
        self._check(lib().ba_get_params(self.h, _ptr(c, _d), _ptr(p, _d)))
        return c, p

    def set_params(self, cams, pts):
        c = np.ascontiguousarray(cams, np.float64)
        p = np.ascontiguousarray(pts, np.float64)
        assert c.shape == (self.n_cam, 9) and p.shape == (self.n_pt, 3)
        self._check(lib().ba_set_params(self.h, _ptr(c, _d), _ptr(p, _d)))

    def get_state(self):
        s = LmState()
        self._check(lib().ba_get_state(self.h, ctypes.byref(s)))
        return _struct_dict(s)

    def set_state(self, lam, nu, iteration, stopped=False):
        s = LmState(lam, nu, iteration, 1 if stopped else 0)
        self._check(lib().ba_set_state(self.h, ctypes.byref(s)))

    def info(self):
        i = Info()
        self._check(lib().ba_get_info(self.h, ctypes.byref(i)))
        return _struct_dict(i)

    def autotune(self):
        r = TuneReport()
        self._check(lib().ba_autotune(self.h, ctypes.byref(r)))
        return _struct_dict(r)

    def set_learned(self, model):
        """Attach a Mlp (None detaches); the model must outlive its use."""
        self._model = model
        self._check(lib().ba_set_learned(self.h, model.h if model is not None else None))

    def learned_fallbacks(self):
        c = ctypes.c_int64()
        self._check(lib().ba_learned_fallbacks(self.h, ctypes.byref(c)))
        return c.value

    def set_profiling(self, enable=True):
        self._check(lib().ba_set_profiling(self.h, 1 if enable else 0))

    def profile(self):
        pr = Profile()
        self._check(lib().ba_get_profile(self.h, ctypes.byref(pr)))
        out = {name: dict(ms=pr.ms[i], count=pr.count[i]) for i, name in enumerate(PROFILE_SLOTS)}
        out.update(kernel_launches=pr.kernel_launches, h2d_bytes=pr.h2d_bytes, d2h_bytes=pr.d2h_bytes)
        return out

    # --- inspection exports -------------------------------------------------------
    def export_order(self):
        perm = np.zeros(self.n_obs, np.int32)
        pt_off = np.zeros(self.n_pt + 1, np.int64)
        cam_off = np.zeros(self.n_cam + 1, np.int64)
        cam_list = np.zeros(self.n_obs, np.int32)
        self._check(lib().ba_debug_export_order(self.h, _ptr(perm, _i32), _ptr(pt_off, _i64),
                                                _ptr(cam_off, _i64), _ptr(cam_list, _i32)))
        return perm, pt_off, cam_off, cam_list

    def export_landmark(self, j, k_cap=256, top_only=False):
        """Landmark j's top rows, A_j, c_j and rotations (top_only: the top
        rows alone, the only part the implicit storage exports: it rebuilds
        them from its records)."""
        top = np.zeros(3 * (9 * k_cap + 4), np.float32)
        a = np.zeros(2 * k_cap * 9 * k_cap if not top_only else 1, np.float32)
        c = np.zeros(2 * k_cap, np.float32)
        rot = np.zeros(12, np.float32)
        k = ctypes.c_int32()
        none = ctypes.POINTER(ctypes.c_float)()
        self._check(lib().ba_debug_export_landmark(
            self.h, int(j), int(k_cap), _ptr(top, _f), none if top_only else _ptr(a, _f),
            none if top_only else _ptr(c, _f), none if top_only else _ptr(rot, _f), ctypes.byref(k)))
        k = k.value
        n = 9 * k
        out = dict(k=k, top=top[: 3 * (n + 4)].reshape(3, n + 4))
        if not top_only:
            out.update(a=a[: 2 * k * n].reshape(2 * k, n), c=c[: 2 * k], rot=rot.reshape(6, 2))
        return out

    def set_options(self, **kw):
        """Change options of the live problem (ba_set_options)."""
        opt = Options.from_buffer_copy(self.options)
        for key, val in kw.items():
            setattr(opt, key, val)
        self._check(lib().ba_set_options(self.h, ctypes.byref(opt)))
        self.options = opt

    def export_damping(self):
        dp2 = np.zeros(9 * self.n_cam, np.float32)
        dl2 = np.zeros(3 * self.n_pt, np.float32)
        self._check(lib().ba_debug_export_damping(self.h, _ptr(dp2, _f), _ptr(dl2, _f)))
        return dp2.reshape(-1, 9), dl2.reshape(-1, 3)

    def export_jacobians(self):
        r = np.zeros(2 * self.n_obs, np.float32)
        jp = np.zeros(18 * self.n_obs, np.float32)
        jl = np.zeros(6 * self.n_obs, np.float32)
        self._check(lib().ba_debug_export_jacobians(self.h, _ptr(r, _f), _ptr(jp, _f), _ptr(jl, _f)))
        return r.reshape(-1, 2), jp.reshape(-1, 2, 9), jl.reshape(-1, 2, 3)

    def export_rcs_diag(self):
        m = np.zeros(81 * self.n_cam, np.float32)
        g = np.zeros(9 * self.n_cam, np.float32)
        self._check(lib().ba_debug_export_rcs_diag(self.h, _ptr(m, _f), _ptr(g, _f)))
        return m.reshape(-1, 9, 9), g.reshape(-1, 9)

    def matvec(self, v):
        v = np.ascontiguousarray(v, np.float32).ravel()
        y = np.zeros_like(v)
        self._check(lib().ba_debug_matvec(self.h, _ptr(v, _f), _ptr(y, _f)))
        return y

    def debug_fail_matvec(self, tile, wait_ms=1.0):
        """Failure test hook: later matvecs leave `tile` of the first CTA
        unissued and give up waiting after wait_ms (tile < 0 restores)."""
        self._check(lib().ba_debug_fail_matvec(self.h, int(tile), float(wait_ms)))

    def export_step(self):
        dp = np.zeros(9 * self.n_cam, np.float32)
        dl = np.zeros(3 * self.n_pt, np.float32)
        self._check(lib().ba_debug_export_step(self.h, _ptr(dp, _f), _ptr(dl, _f)))
        return dp.reshape(-1, 9), dl.reshape(-1, 3)


class Batch:
    """Independent problems solved together (ba_batch_create).  `problems`
    is a sequence of (cams, pts, obs_cam, obs_pt, obs_xy) tuples or objects
    with those attributes, indices local to each problem."""

    def __init__(self, problems, options=None, stream=None, **kw):
        L = lib()
        self._keep = []
        descs = (ProblemDesc * len(problems))()
        self.sizes = []
        for i, pr in enumerate(problems):
            if not isinstance(pr, tuple):
                pr = (pr.cams, pr.pts, pr.obs_cam, pr.obs_pt, pr.obs_xy)
            c = np.ascontiguousarray(pr[0], np.float64)
            x = np.ascontiguousarray(pr[1], np.float64)
            oc = np.ascontiguousarray(pr[2], np.int32)
            op = np.ascontiguousarray(pr[3], np.int32)
            xy = np.ascontiguousarray(pr[4], np.float64)
            self._keep += [c, x, oc, op, xy]
            descs[i] = ProblemDesc(_ptr(c, _d), c.shape[0], _ptr(x, _d), x.shape[0], _ptr(oc, _i32),
                                   _ptr(op, _i32), _ptr(xy, _d), oc.shape[0])
            self.sizes.append((c.shape[0], x.shape[0], oc.shape[0]))
        opt = options if options is not None else default_options(**kw)
        h = _P()
        rc = L.ba_batch_create(descs, len(problems), ctypes.byref(opt), _P(stream) if stream else None,
                               ctypes.byref(h))
        self._keep = []
        if rc != BA_OK:
            raise BAError(rc, L.ba_batch_last_error(None).decode())
        self.h = h
        self.options = opt

    def close(self):
        if getattr(self, "h", None):
            lib().ba_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != BA_OK:
            raise BAError(rc, lib().ba_batch_last_error(self.h).decode())

    def solve(self):
        n = len(self.sizes)
        reps = (BatchReport * n)()
        summ = BatchSummary()
        self._check(lib().ba_batch_solve(self.h, reps, ctypes.byref(summ)))
        return [_struct_dict(r) for r in reps], _struct_dict(summ)

    def restart(self):
        self._check(lib().ba_batch_restart(self.h))

    def set_profiling(self, enable=True):
        self._check(lib().ba_batch_set_profiling(self.h, 1 if enable else 0))

    def profile(self):
        pr = Profile()
        self._check(lib().ba_batch_get_profile(self.h, ctypes.byref(pr)))
        out = {name: dict(ms=pr.ms[i], count=pr.count[i]) for i, name in enumerate(PROFILE_SLOTS)}
        out.update(kernel_launches=pr.kernel_launches, h2d_bytes=pr.h2d_bytes, d2h_bytes=pr.d2h_bytes)
        return out

    def info(self):
        i = Info()
        self._check(lib().ba_batch_get_info(self.h, ctypes.byref(i)))
        return _struct_dict(i)

    def iterations(self):
        """(active problems at the start, ms) of each LM iteration of the last solve."""
        n = ctypes.c_int32()
        self._check(lib().ba_batch_iterations(self.h, 0, None, None, ctypes.byref(n)))
        m = n.value
        act = np.zeros(max(m, 1), np.int32)
        ms = np.zeros(max(m, 1), np.float32)
        self._check(lib().ba_batch_iterations(self.h, m, _ptr(act, _i32), _ptr(ms, _f), ctypes.byref(n)))
        return act[:m].tolist(), ms[:m].tolist()

    def get_params(self, i):
        nc, npt, _ = self.sizes[i]
        c = np.zeros((nc, 9))
        p = np.zeros((npt, 3))
        self._check(lib().ba_batch_get_params(self.h, int(i), _ptr(c, _d), _ptr(p, _d)))
        return c, p


MLP_PARAMS = 150582
MLP_IN, MLP_OUT, MLP_AUX = 19, 54, 72


class Mlp:
    """The learned warm start / preconditioner model (ba_mlp_*).  Device
    arguments are CUDA tensors (float32 / int32, contiguous) or raw device
    addresses; parameters are host float32 arrays of MLP_PARAMS values."""

    def __init__(self, params, stream=None):
        L = lib()
        prm = np.ascontiguousarray(params, np.float32).ravel()
        assert prm.size == MLP_PARAMS
        h = _P()
        rc = L.ba_mlp_create(_ptr(prm, _f), _P(stream) if stream else None, ctypes.byref(h))
        if rc != BA_OK:
            raise BAError(rc, L.ba_mlp_last_error(None).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().ba_mlp_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != BA_OK:
            raise BAError(rc, lib().ba_mlp_last_error(self.h).decode())

    def params(self):
        out = np.zeros(MLP_PARAMS, np.float32)
        self._check(lib().ba_mlp_get_params(self.h, _ptr(out, _f)))
        return out

    def forward(self, feats, out):
        self._check(lib().ba_mlp_forward(self.h, _devptr(feats), int(feats.shape[0]), _devptr(out)))

    def prepare(self, M, g, xstar, count, feats, aux):
        self._check(lib().ba_mlp_prepare(self.h, _devptr(M), _devptr(g), _devptr(xstar) if xstar is not None else None,
                                         _devptr(count), int(count.shape[0]), _devptr(feats), _devptr(aux)))

    def loss_grad(self, feats, aux, with_grads=True):
        loss = ctypes.c_double()
        grads = np.zeros(MLP_PARAMS, np.float32) if with_grads else None
        self._check(lib().ba_mlp_loss_grad(self.h, _devptr(feats), _devptr(aux), int(feats.shape[0]),
                                           ctypes.byref(loss), _ptr(grads, _f) if with_grads else None))
        return loss.value, grads

    def train_step(self, feats, aux, lr):
        loss = ctypes.c_double()
        self._check(lib().ba_mlp_train_step(self.h, _devptr(feats), _devptr(aux), int(feats.shape[0]),
                                            float(lr), ctypes.byref(loss)))
        return loss.value


def mlp_params_flat(params):
    """Flatten [(W, b), ...] (the oracle's layout) into the C-ABI order."""
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params]).astype(np.float32)


def mlp_params_unflat(flat, sizes=(19, 256, 256, 256, 54)):
    out, o = [], 0
    for i, n in zip(sizes[:-1], sizes[1:]):
        W = np.asarray(flat[o:o + n * i], np.float64).reshape(n, i)
        o += n * i
        b = np.asarray(flat[o:o + n], np.float64)
        o += n
        out.append((W, b))
    return out
