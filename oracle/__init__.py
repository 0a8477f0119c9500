"""FP64 CPU oracle for square root bundle adjustment (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use this package.  It is a plain Schur-complement
Levenberg-Marquardt solver in double precision (``oracle.c``), independent of
the CUDA library: it shares no code, header or constant table with it.

Functions and the passages of the paper they follow:
  residual / rotmat / compose / apply_update : BAL camera model (Sec. 6.2),
      left-multiplicative rotation increment (reading, no paper text)
  cost           : E = sum ||r||^2, Eq. ba_energy
  sort_obs       : residuals grouped by landmark (Sec. 5.1)
  damping_diag   : D^2 = diag(J^T J) (Sec. 4.1), clamped to [1e-6, 1e32]
  rcs_dense/diag : damped Schur complement H~, b~ (Sec. 4.2, end of Sec. 4.4)
  landmark_sc    : one landmark's contribution to H~ and b~ (Eq. red_H, red_b)
  linear_step    : dense or block-Jacobi PCG solve of the RCS (Sec. 5.4, 6.1)
                   and back substitution (Eq. backsub_sc)
  rcs_matvec     : products with H~ (block-sparse assembly)
  backsub_given  : back substitution and model cost for a given pose step
  pcg_dense      : the same block-Jacobi PCG and stop rules on a dense SPD matrix
                   (Sec. 6.1 forcing sequence, Nash-Sofer reading)
  lm_decide      : accept/reject and damping update of one LM iteration
                   (Sec. 6.1, Nielsen's rule as the reading)
  lm             : the Levenberg-Marquardt loop of Sec. 6.1
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.POINTER(ctypes.c_int64)


class Options(ctypes.Structure):
    _fields_ = [("lambda0", ctypes.c_double), ("max_iters", ctypes.c_int32),
                ("func_tol", ctypes.c_double), ("max_cg", ctypes.c_int32),
                ("cg_eta", ctypes.c_double), ("dense", ctypes.c_int32),
                ("target_cost", ctypes.c_double)]


class Iter(ctypes.Structure):
    _fields_ = [("cost", ctypes.c_double), ("new_cost", ctypes.c_double),
                ("model_cost", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("rho", ctypes.c_double), ("cg_iters", ctypes.c_int32),
                ("accepted", ctypes.c_int32)]


def build(force=False):
    """Compile oracle.c with gcc into oracle/_build/liboracle.so."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp]
    try:  # OpenMP host threads where the toolchain has them, else one thread
        subprocess.check_call(base + ["-fopenmp", "-lm"], stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(base + ["-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def set_threads(n):
    """Host threads of the oracle's parallel loops (1 by default); results do
    not depend on it.  Returns the count in effect."""
    lib().orc_set_threads(ctypes.c_int32(max(1, int(n))))
    return max(1, int(n))


def max_threads():
    """Processors OpenMP sees (1 when built without OpenMP)."""
    return int(lib().orc_max_threads())


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _lib.orc_cost.restype = ctypes.c_double
            _lib.orc_max_threads.restype = ctypes.c_int32
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _huber(delta):
    """Huber parameter of the next call (reading of Sec. 6.2's robust norm as
    IRLS; 0 = squared norm)."""
    lib().orc_set_huber(ctypes.c_double(float(delta)))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32a(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _problem(s):
    cams, pts = _f64(s.cams), _f64(s.pts)
    oc, op, xy = _i32a(s.obs_cam), _i32a(s.obs_pt), _f64(s.obs_xy)
    return cams, pts, oc, op, xy


def _args(cams, pts, oc, op, xy):
    return (ctypes.c_int32(cams.shape[0]), _p(cams, _d), ctypes.c_int32(pts.shape[0]),
            _p(pts, _d), ctypes.c_int64(oc.shape[0]), _p(oc, _i32), _p(op, _i32), _p(xy, _d))


class OracleError(RuntimeError):
    pass


def _check(rc, what):
    if rc != 0:
        raise OracleError(f"oracle {what} failed with status {rc}")


def rotmat(w):
    w = _f64(w)
    R = np.zeros(9)
    lib().orc_rotmat(_p(w, _d), _p(R, _d))
    return R.reshape(3, 3)


def compose(dw, w):
    dw, w = _f64(dw), _f64(w)
    out = np.zeros(3)
    lib().orc_compose(_p(dw, _d), _p(w, _d), _p(out, _d))
    return out


def residual(cam, X, z):
    """Residual (2,), pose Jacobian (2, 9), landmark Jacobian (2, 3)."""
    cam, X, z = _f64(cam), _f64(X), _f64(z)
    r, Jp, Jl = np.zeros(2), np.zeros(18), np.zeros(6)
    lib().orc_residual(_p(cam, _d), _p(X, _d), _p(z, _d), _p(r, _d), _p(Jp, _d), _p(Jl, _d))
    return r, Jp.reshape(2, 9), Jl.reshape(2, 3)


def apply_update(cams, dcams, pts, dpts):
    cams, dcams, pts, dpts = _f64(cams), _f64(dcams), _f64(pts), _f64(dpts)
    co, po = np.zeros_like(cams), np.zeros_like(pts)
    lib().orc_apply_update(ctypes.c_int32(cams.shape[0]), _p(cams, _d), _p(dcams, _d),
                           ctypes.c_int32(pts.shape[0]), _p(pts, _d), _p(dpts, _d),
                           _p(co, _d), _p(po, _d))
    return co, po


def cost(s, cams=None, pts=None, huber_delta=0.0):
    _huber(huber_delta)
    c, p, oc, op, xy = _problem(s)
    if cams is not None:
        c = _f64(cams)
    if pts is not None:
        p = _f64(pts)
    return float(lib().orc_cost(*_args(c, p, oc, op, xy)))


def sort_obs(n_cam, n_pt, obs_cam, obs_pt):
    """(status, perm, pt_off, cam_off, cam_list) ordering by (landmark, camera)."""
    oc, op = _i32a(obs_cam), _i32a(obs_pt)
    n = oc.shape[0]
    perm = np.zeros(max(n, 1), np.int32)
    pt_off = np.zeros(n_pt + 1, np.int64)
    cam_off = np.zeros(n_cam + 1, np.int64)
    cam_list = np.zeros(max(n, 1), np.int32)
    rc = lib().orc_sort_obs(ctypes.c_int32(n_cam), ctypes.c_int32(n_pt), ctypes.c_int64(n),
                            _p(oc, _i32), _p(op, _i32), _p(perm, _i32), _p(pt_off, _i64),
                            _p(cam_off, _i64), _p(cam_list, _i32))
    return rc, perm[:n], pt_off, cam_off, cam_list[:n]


def damping_diag(s, cams=None, pts=None, huber_delta=0.0):
    _huber(huber_delta)
    c, p, oc, op, xy = _problem(s)
    c = c if cams is None else _f64(cams)
    p = p if pts is None else _f64(pts)
    Dp2, Dl2 = np.zeros(9 * c.shape[0]), np.zeros(3 * p.shape[0])
    _check(lib().orc_damping_diag(*_args(c, p, oc, op, xy), _p(Dp2, _d), _p(Dl2, _d)), "damping_diag")
    return Dp2.reshape(-1, 9), Dl2.reshape(-1, 3)


def rcs_dense(s, lam, cams=None, pts=None, huber_delta=0.0):
    """Dense damped Schur complement H~ (9 n_cam square) and b~."""
    _huber(huber_delta)
    c, p, oc, op, xy = _problem(s)
    c = c if cams is None else _f64(cams)
    p = p if pts is None else _f64(pts)
    n = 9 * c.shape[0]
    H, bt = np.zeros((n, n)), np.zeros(n)
    _check(lib().orc_rcs_dense(*_args(c, p, oc, op, xy), ctypes.c_double(lam), _p(H, _d),
                               _p(bt, _d)), "rcs_dense")
    return H, bt


def rcs_diag(s, lam, cams=None, pts=None, huber_delta=0.0):
    """Per-camera 9x9 diagonal blocks of H~ and b~ (block-sparse assembly)."""
    _huber(huber_delta)
    c, p, oc, op, xy = _problem(s)
    c = c if cams is None else _f64(cams)
    p = p if pts is None else _f64(pts)
    M, bt = np.zeros((c.shape[0], 9, 9)), np.zeros(9 * c.shape[0])
    _check(lib().orc_rcs_diag(*_args(c, p, oc, op, xy), ctypes.c_double(lam), _p(M, _d),
                              _p(bt, _d)), "rcs_diag")
    return M, bt.reshape(-1, 9)


def landmark_sc(s, lam, j, k_cap=256, cams=None, pts=None, huber_delta=0.0):
    """Landmark j's damped SC pieces: S (9k, 9k), b~_j (9k), H_ll + lam D_l^2, ||c_j||^2."""
    _huber(huber_delta)
    c, p, oc, op, xy = _problem(s)
    c = c if cams is None else _f64(cams)
    p = p if pts is None else _f64(pts)
    S = np.zeros((9 * k_cap) ** 2)
    bts, Hll, cc, k = np.zeros(9 * k_cap), np.zeros(9), np.zeros(1), np.zeros(1, np.int32)
    _check(lib().orc_landmark_sc(*_args(c, p, oc, op, xy), ctypes.c_double(lam),
                                 ctypes.c_int32(j), ctypes.c_int32(k_cap), _p(S, _d), _p(bts, _d),
                                 _p(Hll, _d), _p(cc, _d), _p(k, _i32)), "landmark_sc")
    n = 9 * int(k[0])
    return S[: n * n].reshape(n, n), bts[:n], Hll.reshape(3, 3), float(cc[0])


def rcs_matvec(s, lam, V, cams=None, pts=None, huber_delta=0.0):
    """Rows of H~ V^T: y_m = H~ v_m for each row v_m of V (m, 9 n_cam)."""
    _huber(huber_delta)
    c, p, oc, op, xy = _problem(s)
    c = c if cams is None else _f64(cams)
    p = p if pts is None else _f64(pts)
    V = np.atleast_2d(_f64(V))
    Y = np.zeros_like(V)
    _check(lib().orc_rcs_matvec(*_args(c, p, oc, op, xy), ctypes.c_double(lam), ctypes.c_int32(V.shape[0]),
                                _p(V, _d), _p(Y, _d)), "rcs_matvec")
    return Y


def backsub_given(s, lam, dp, cams=None, pts=None, huber_delta=0.0):
    """Landmark step for a given pose step dp (Eq. backsub_sc) and L(dx)."""
    _huber(huber_delta)
    c, p, oc, op, xy = _problem(s)
    c = c if cams is None else _f64(cams)
    p = p if pts is None else _f64(pts)
    dp = _f64(dp).ravel()
    dl = np.zeros(3 * p.shape[0])
    m = ctypes.c_double()
    _check(lib().orc_backsub_given(*_args(c, p, oc, op, xy), ctypes.c_double(lam), _p(dp, _d),
                                   _p(dl, _d), ctypes.byref(m)), "backsub_given")
    return dl.reshape(-1, 3), m.value


def options(lambda0=1e-4, max_iters=50, func_tol=1e-6, max_cg=500, cg_eta=0.1, dense=False,
            target_cost=0.0):
    return Options(lambda0, max_iters, func_tol, max_cg, cg_eta, 1 if dense else 0, target_cost)


def linear_step(s, lam, dense=True, max_cg=500, cg_eta=0.1, cams=None, pts=None, huber_delta=0.0):
    """One damped step: dict(dp (n_cam,9), dl (n_pt,3), model_cost, cost, cg_iters)."""
    _huber(huber_delta)
    c, p, oc, op, xy = _problem(s)
    c = c if cams is None else _f64(cams)
    p = p if pts is None else _f64(pts)
    opt = options(max_cg=max_cg, cg_eta=cg_eta, dense=dense)
    dp, dl = np.zeros(9 * c.shape[0]), np.zeros(3 * p.shape[0])
    model, E, cg = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    _check(lib().orc_linear_step(*_args(c, p, oc, op, xy), ctypes.c_double(lam), ctypes.byref(opt),
                                 _p(dp, _d), _p(dl, _d), ctypes.byref(model), ctypes.byref(E),
                                 ctypes.byref(cg)), "linear_step")
    return dict(dp=dp.reshape(-1, 9), dl=dl.reshape(-1, 3), model_cost=model.value,
                cost=E.value, cg_iters=cg.value)


def pcg_dense(H, g, max_it=500, eta=0.1):
    """Block-Jacobi PCG on a dense SPD H (9m square): (x, iterations, Q_0..Q_i, status)."""
    H, g = _f64(H), _f64(g).ravel()
    n = g.shape[0]
    assert n % 9 == 0 and H.shape == (n, n)
    x = np.zeros(n)
    Q = np.zeros(max_it + 1)
    st = ctypes.c_int32()
    it = lib().orc_pcg_dense(ctypes.c_int32(n // 9), _p(H, _d), _p(g, _d), ctypes.c_int32(max_it),
                             ctypes.c_double(eta), _p(x, _d), _p(Q, _d), ctypes.byref(st))
    return x, int(it), Q[: it + 1].copy(), int(st.value)


def lm_decide(E, E_new, model, lam, nu, func_tol=1e-6, target_cost=0.0):
    """One LM decision: dict(accepted, stop, rho, lam, nu) after the update."""
    lam_c, nu_c = ctypes.c_double(lam), ctypes.c_double(nu)
    stop, rho = ctypes.c_int32(), ctypes.c_double()
    acc = lib().orc_lm_decide(ctypes.c_double(E), ctypes.c_double(E_new), ctypes.c_double(model),
                              ctypes.c_double(func_tol), ctypes.c_double(target_cost),
                              ctypes.byref(lam_c), ctypes.byref(nu_c), ctypes.byref(stop),
                              ctypes.byref(rho))
    return dict(accepted=bool(acc), stop=bool(stop.value), rho=rho.value, lam=lam_c.value,
                nu=nu_c.value)


def lm(s, cams=None, pts=None, huber_delta=0.0, **kw):
    """Run the LM loop; returns (cams, pts, log list of dicts)."""
    _huber(huber_delta)
    c, p, oc, op, xy = _problem(s)
    c = (c if cams is None else _f64(cams)).copy()
    p = (p if pts is None else _f64(pts)).copy()
    opt = options(**kw)
    log = (Iter * max(1, opt.max_iters))()
    n = ctypes.c_int32()
    _check(lib().orc_lm(*_args(c, p, oc, op, xy), ctypes.byref(opt), log, ctypes.byref(n)), "lm")
    out = [dict(cost=e.cost, new_cost=e.new_cost, model_cost=e.model_cost, lam=e.lambda_,
                rho=e.rho, cg_iters=e.cg_iters, accepted=bool(e.accepted)) for e in log[: n.value]]
    return c, p, out
