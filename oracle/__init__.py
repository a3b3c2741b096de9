"""FP64 CPU oracle for the STORM control step -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this package.  It wraps ``storm_oracle.c`` (plain sequential C in double
precision) through ctypes and shares no code with the CUDA library.  Inputs are
plain numpy arrays, e.g. those drawn by ``paper_2104_13542_b300.workloads``.

Parity status: every routine is pinned by the CPU tests under ``tests/``
(closed forms, invariants, special cases, brute force); see each C routine's
comment for its pin.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "storm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libstorm_oracle.so")
NTERMS = 11


def build(force: bool = False) -> str:
    """Compile the oracle with gcc -O2 (no fast-math; OpenMP for the optional
    particle-parallel rollout loop) into oracle/libstorm_oracle.so."""
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC),
                                               os.path.getmtime(_SRC[:-2] + ".h")):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC,
                               "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_up = C.POINTER(C.c_uint32)


class _Robot(C.Structure):
    _fields_ = [("dof", C.c_int), ("dh", _dp), ("q_min", _dp), ("q_max", _dp),
                ("n_spheres", C.c_int), ("sphere_link", _ip), ("sphere", _dp),
                ("n_pairs", C.c_int), ("pairs", _ip)]


class _World(C.Structure):
    _fields_ = [("n_boxes", C.c_int), ("boxes", _dp), ("n_spheres", C.c_int),
                ("spheres", _dp)]


class _Arch(C.Structure):
    _fields_ = [("enc", C.c_int), ("h1", C.c_int), ("h2", C.c_int), ("h3", C.c_int)]


# surrogate architectures: (encoding, h1, h2, h3)
ARCH_DISTANCE = (0, 256, 256, 256)   # theta / 3 encoding, three 256-wide layers
ARCH_JOINTNERF = (1, 256, 128, 64)   # [sin theta, cos theta] encoding, [256, 128, 64] (Sec. 4.2)


class _Params(C.Structure):
    _fields_ = [("N", C.c_int), ("H", C.c_int), ("K", C.c_int), ("n_knots", C.c_int),
                ("sampler", C.c_int), ("n_null", C.c_int), ("dt", _dp),
                ("beta", C.c_double), ("gamma", C.c_double), ("alpha_mu", C.c_double),
                ("alpha_sigma", C.c_double), ("sigma_min", C.c_double),
                ("w_pos", C.c_double), ("w_rot", C.c_double), ("w_stop", C.c_double),
                ("w_joint", C.c_double), ("w_manip", C.c_double), ("w_coll", C.c_double),
                ("w_smooth", C.c_double), ("pos_axis_w", C.c_double * 3),
                ("rot_axis_w", C.c_double * 3), ("rot_mode", C.c_int), ("k_jl", C.c_double),
                ("k_m", C.c_double), ("qdd_max", C.c_double), ("seed", C.c_uint64),
                ("instance", C.c_uint32), ("grad_steps", C.c_int), ("grad_eta", C.c_double),
                ("filter", C.c_int), ("comb", C.c_double * 3), ("mix_bspline", C.c_double),
                ("w_ee_vel", C.c_double), ("w_ee_acc", C.c_double), ("ee_vel_max", C.c_double),
                ("ee_acc_max", C.c_double), ("w_ball", C.c_double), ("gravity", C.c_double * 3),
                ("tray_center", C.c_double * 3), ("ball", _dp), ("halton_scramble", C.c_int),
                ("mlp_mode", C.c_int), ("mlp_params", _dp), ("mlp_enc", C.c_int), ("mlp_h1", C.c_int),
                ("mlp_h2", C.c_int), ("mlp_h3", C.c_int), ("mlp_margin", C.c_double)]


def set_threads(n: int) -> None:
    """Threads of the rollout's particle loop (1 = sequential; same bits for any count)."""
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def _declare(L):
    L.orc_set_threads.argtypes = [C.c_int]
    L.orc_set_threads.restype = None
    L.orc_get_threads.restype = C.c_int
    L.orc_philox4x32_10.argtypes = [_up, _up, _up]
    L.orc_uniform_from_bits.argtypes = [C.c_uint32]
    L.orc_uniform_from_bits.restype = C.c_double
    L.orc_box_muller.argtypes = [C.c_double, C.c_double, _dp, _dp]
    L.orc_noise_philox.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                   C.c_longlong, _dp]
    L.orc_radical_inverse.argtypes = [C.c_uint64, C.c_int]
    L.orc_radical_inverse.restype = C.c_double
    L.orc_nth_prime.argtypes = [C.c_int]
    L.orc_nth_prime.restype = C.c_int
    L.orc_norm_ppf.argtypes = [C.c_double]
    L.orc_norm_ppf.restype = C.c_double
    L.orc_noise_halton.argtypes = [C.c_int, C.c_int, C.c_int, _dp]
    L.orc_noise_halton_ex.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64, _dp]
    L.orc_radical_inverse_scrambled.argtypes = [C.c_uint64, C.c_int, C.c_int]
    L.orc_radical_inverse_scrambled.restype = C.c_double
    L.orc_halton_multiplier.argtypes = [C.c_uint64, C.c_int, C.c_int]
    L.orc_halton_multiplier.restype = C.c_int
    L.orc_bspline_basis.argtypes = [C.c_int, C.c_int, _dp]
    L.orc_smooth_controls.argtypes = [C.POINTER(_Params), C.c_int, _dp, _dp, _dp, _dp]
    L.orc_integrate.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp]
    L.orc_fk.argtypes = [C.POINTER(_Robot), _dp, _dp]
    L.orc_jacobian.argtypes = [C.POINTER(_Robot), _dp, _dp]
    L.orc_det.argtypes = [C.c_int, _dp]
    L.orc_det.restype = C.c_double
    L.orc_manipulability.argtypes = [_dp, C.c_int]
    L.orc_manipulability.restype = C.c_double
    L.orc_quat_from_rot.argtypes = [_dp, _dp]
    L.orc_rot_from_quat.argtypes = [_dp, _dp]
    L.orc_box_sdf.argtypes = [_dp, _dp]
    L.orc_box_sdf.restype = C.c_double
    L.orc_self_min_sd.argtypes = [C.POINTER(_Robot), _dp]
    L.orc_self_min_sd.restype = C.c_double
    L.orc_world_min_sd.argtypes = [C.POINTER(_Robot), C.POINTER(_World), _dp]
    L.orc_world_min_sd.restype = C.c_double
    L.orc_running_cost.argtypes = [C.POINTER(_Robot), C.POINTER(_World), C.POINTER(_Params),
                                   _dp, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
    L.orc_rollout.argtypes = [C.POINTER(_Robot), C.POINTER(_World), C.POINTER(_Params),
                              _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    L.orc_rollout.restype = C.c_int
    L.orc_update.argtypes = [C.POINTER(_Params), C.c_int, _dp, _dp, _dp, _dp, _dp]
    L.orc_update.restype = C.c_int
    L.orc_shift.argtypes = [C.c_int, C.c_int, _dp]
    L.orc_step.argtypes = [C.POINTER(_Robot), C.POINTER(_World), C.POINTER(_Params), _dp, _dp,
                           C.c_uint32, _dp, _dp, _dp, _dp]
    L.orc_step.restype = C.c_int
    L.orc_running_cost_grad.argtypes = [C.POINTER(_Robot), C.POINTER(_World), C.POINTER(_Params),
                                        _dp, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    L.orc_integrate_adjoint.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp]
    L.orc_cost_grad.argtypes = [C.POINTER(_Robot), C.POINTER(_World), C.POINTER(_Params), _dp, _dp,
                                _dp, _dp, _dp, _dp, _dp, _dp]
    L.orc_cost_grad.restype = C.c_int
    L.orc_mlp_param_count.restype = C.c_long
    L.orc_mlp_arch_param_count.argtypes = [C.POINTER(_Arch)]
    L.orc_mlp_arch_param_count.restype = C.c_long
    L.orc_mlp_arch_encode.argtypes = [C.POINTER(_Arch), _dp, C.c_int, _dp]
    L.orc_mlp_arch_forward.argtypes = [C.POINTER(_Arch), _dp, _dp, C.c_int, C.c_int, C.c_int, _dp]
    L.orc_mlp_arch_loss_grad.argtypes = [C.POINTER(_Arch), _dp, _dp, _dp, C.c_int, C.c_int, C.c_int, _dp]
    L.orc_mlp_arch_loss_grad.restype = C.c_double
    L.orc_bf16_round.argtypes = [C.c_float]
    L.orc_bf16_round.restype = C.c_float
    L.orc_mlp_forward.argtypes = [_dp, _dp, C.c_int, C.c_int, C.c_int, _dp]
    L.orc_mlp_loss_grad.argtypes = [_dp, _dp, _dp, C.c_int, C.c_int, C.c_int, _dp]
    L.orc_mlp_loss_grad.restype = C.c_double
    L.orc_self_min_sd_theta.argtypes = [C.POINTER(_Robot), _dp]
    L.orc_self_min_sd_theta.restype = C.c_double
    L.orc_comb_filter.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp]
    L.orc_ee_twist.argtypes = [C.POINTER(_Robot), _dp, _dp, _dp, _dp, _dp]
    L.orc_ball_states.argtypes = [C.POINTER(_Robot), C.POINTER(_Params), _dp, _dp, _dp, _dp]
    L.orc_ball_states.restype = C.c_int


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def _iptr(a):
    return a.ctypes.data_as(_ip)


# --------------------------------------------------------------------------- primitives

def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(c.ctypes.data_as(_up), k.ctypes.data_as(_up), out.ctypes.data_as(_up))
    return out


def uniform_from_bits(x: int) -> float:
    return lib().orc_uniform_from_bits(int(x))


def box_muller(u1: float, u2: float):
    z0, z1 = C.c_double(), C.c_double()
    lib().orc_box_muller(u1, u2, C.byref(z0), C.byref(z1))
    return z0.value, z1.value


def noise_philox(seed, step, instance, it, tag, count) -> np.ndarray:
    out = np.zeros(int(count))
    lib().orc_noise_philox(int(seed), int(step), int(instance), int(it), int(tag), int(count),
                           _ptr(out))
    return out


def radical_inverse(i: int, base: int) -> float:
    return lib().orc_radical_inverse(int(i), int(base))


def nth_prime(n: int) -> int:
    return lib().orc_nth_prime(int(n))


def norm_ppf(p: float) -> float:
    return lib().orc_norm_ppf(float(p))


def noise_halton(N, S, d, scramble=False, seed=0) -> np.ndarray:
    out = np.zeros((N, S, d))
    lib().orc_noise_halton_ex(N, S, d, int(bool(scramble)), int(seed), _ptr(out))
    return out


def radical_inverse_scrambled(i: int, base: int, mult: int) -> float:
    return lib().orc_radical_inverse_scrambled(int(i), int(base), int(mult))


def halton_multiplier(seed: int, dim: int, base: int) -> int:
    return int(lib().orc_halton_multiplier(int(seed), int(dim), int(base)))


def comb_filter(c, eps) -> np.ndarray:
    """Comb filter of eps (H x d) along the horizon with coefficients c (3,)."""
    e = _f64(eps)
    H, d = e.shape
    out = np.zeros((H, d))
    lib().orc_comb_filter(H, d, _ptr(_f64(c)), _ptr(e), _ptr(out))
    return out


def bspline_basis(H, S) -> np.ndarray:
    out = np.zeros((H, S))
    lib().orc_bspline_basis(H, S, _ptr(out))
    return out


def mlp_param_count() -> int:
    return int(lib().orc_mlp_param_count())


def bf16_round(x: float) -> float:
    return float(lib().orc_bf16_round(float(x)))


def mlp_forward(params, theta, bf16=True) -> np.ndarray:
    params, theta = _f64(params), _f64(theta)
    B, dof = theta.shape
    y = np.zeros(B)
    lib().orc_mlp_forward(_ptr(params), _ptr(theta), B, dof, int(bf16), _ptr(y))
    return y


def mlp_arch_param_count(arch) -> int:
    return int(lib().orc_mlp_arch_param_count(C.byref(_Arch(*arch))))


def mlp_arch_encode(arch, theta) -> np.ndarray:
    th = _f64(theta)
    x = np.zeros(16)
    lib().orc_mlp_arch_encode(C.byref(_Arch(*arch)), _ptr(th), th.shape[0], _ptr(x))
    return x


def mlp_arch_forward(arch, params, theta, bf16=True) -> np.ndarray:
    params, theta = _f64(params), _f64(theta)
    B, dof = theta.shape
    y = np.zeros(B)
    lib().orc_mlp_arch_forward(C.byref(_Arch(*arch)), _ptr(params), _ptr(theta), B, dof, int(bf16), _ptr(y))
    return y


def mlp_arch_loss_grad(arch, params, theta, target, bf16=True):
    params, theta, target = _f64(params), _f64(theta), _f64(target)
    B, dof = theta.shape
    g = np.zeros(mlp_arch_param_count(arch))
    loss = lib().orc_mlp_arch_loss_grad(C.byref(_Arch(*arch)), _ptr(params), _ptr(theta), _ptr(target), B, dof,
                                        int(bf16), _ptr(g))
    return loss, g


def mlp_loss_grad(params, theta, target, bf16=True):
    params, theta, target = _f64(params), _f64(theta), _f64(target)
    B, dof = theta.shape
    g = np.zeros(mlp_param_count())
    loss = lib().orc_mlp_loss_grad(_ptr(params), _ptr(theta), _ptr(target), B, dof, int(bf16),
                                   _ptr(g))
    return loss, g


def integrate_adjoint(dt, g_theta, g_theta_dot, g_u):
    dt = _f64(dt)
    g_theta, g_theta_dot, g_u = _f64(g_theta), _f64(g_theta_dot), _f64(g_u)
    H, d = g_u.shape
    out = np.zeros((H, d))
    lib().orc_integrate_adjoint(H, d, _ptr(dt), _ptr(g_theta), _ptr(g_theta_dot), _ptr(g_u),
                                _ptr(out))
    return out


def integrate(dt, state, u):
    dt, state, u = _f64(dt), _f64(state), _f64(u)
    H, d = u.shape
    th = np.zeros((H, d))
    thd = np.zeros((H, d))
    lib().orc_integrate(H, d, _ptr(dt), _ptr(state), _ptr(u), _ptr(th), _ptr(thd))
    return th, thd


def det(A) -> float:
    A = _f64(A)
    return lib().orc_det(A.shape[0], _ptr(A))


def manipulability(J) -> float:
    J = _f64(J)
    return lib().orc_manipulability(_ptr(J), J.shape[1])


def quat_from_rot(Rm) -> np.ndarray:
    Rm = _f64(Rm)
    q = np.zeros(4)
    lib().orc_quat_from_rot(_ptr(Rm), _ptr(q))
    return q


def rot_from_quat(q) -> np.ndarray:
    q = _f64(q)
    Rm = np.zeros((3, 3))
    lib().orc_rot_from_quat(_ptr(q), _ptr(Rm))
    return Rm


def box_sdf(p, box) -> float:
    return lib().orc_box_sdf(_ptr(_f64(p)), _ptr(_f64(box)))


# --------------------------------------------------------------------------- model-level

class Oracle:
    """Holds one workload's robot / world / params in the oracle's own structs."""

    def __init__(self, robot, world, params):
        self.robot, self.world, self.params = robot, world, params
        self._keep = []
        self.d = int(robot.dh.shape[0])
        self.R = self._robot(robot)
        self.W = self._world(world)
        self.P = self._params(params)

    def _hold(self, a):
        self._keep.append(a)
        return a

    def _robot(self, r):
        dh = self._hold(_f64(r.dh))
        qmin = self._hold(_f64(r.q_min))
        qmax = self._hold(_f64(r.q_max))
        link = self._hold(np.ascontiguousarray(r.sphere_link, dtype=np.int32))
        sph = self._hold(_f64(r.spheres).reshape(-1, 4))
        pairs = self._hold(np.ascontiguousarray(np.asarray(r.pairs, dtype=np.int32).reshape(-1, 2)))
        return _Robot(dh.shape[0], _ptr(dh), _ptr(qmin), _ptr(qmax), sph.shape[0], _iptr(link),
                      _ptr(sph), pairs.shape[0], _iptr(pairs))

    def _world(self, w):
        boxes = self._hold(_f64(w.boxes).reshape(-1, 6))
        sph = self._hold(_f64(w.spheres).reshape(-1, 4))
        return _World(boxes.shape[0], _ptr(boxes), sph.shape[0], _ptr(sph))

    def _params(self, p):
        dt = self._hold(_f64(p.dt))
        assert dt.shape[0] == p.H
        s = _Params()
        s.N, s.H, s.K, s.n_knots = p.N, p.H, p.K, p.n_knots
        s.sampler, s.n_null, s.dt = p.sampler, p.n_null, _ptr(dt)
        s.beta, s.gamma, s.alpha_mu, s.alpha_sigma = p.beta, p.gamma, p.alpha_mu, p.alpha_sigma
        s.sigma_min = p.sigma_min
        s.w_pos, s.w_rot, s.w_stop, s.w_joint = p.w_pos, p.w_rot, p.w_stop, p.w_joint
        s.w_manip, s.w_coll, s.w_smooth = p.w_manip, p.w_coll, p.w_smooth
        s.pos_axis_w[:] = list(p.pos_axis_w)
        s.rot_axis_w[:] = list(p.rot_axis_w)
        s.rot_mode, s.k_jl, s.k_m, s.qdd_max = p.rot_mode, p.k_jl, p.k_m, p.qdd_max
        s.seed, s.instance = int(p.seed), int(p.instance)
        s.grad_steps, s.grad_eta = int(p.grad_steps), float(p.grad_eta)
        s.filter, s.mix_bspline = int(p.filter), float(p.mix_bspline)
        s.comb[:] = [float(c) for c in p.comb]
        s.w_ee_vel, s.w_ee_acc = float(p.w_ee_vel), float(p.w_ee_acc)
        s.ee_vel_max, s.ee_acc_max = float(p.ee_vel_max), float(p.ee_acc_max)
        s.w_ball = float(p.w_ball)
        s.gravity[:] = [float(g) for g in p.gravity]
        s.tray_center[:] = [float(c) for c in p.tray_center]
        s.ball = None
        s.halton_scramble = int(p.halton_scramble)
        s.mlp_mode, s.mlp_params = 0, None
        return s

    def set_surrogate(self, arch, params, margin=None):
        """The learned self-collision network (Sec. 4.2) in the rollout's self term:
        with `margin`, a gate (the exact check only where the predicted distance is
        below it); without, the Eq. 13 cost max(0, net) with no exact check.
        `params` = None restores the exact check."""
        if params is None:
            self.P.mlp_mode, self.P.mlp_params = 0, None
            return
        self._mlp = _f64(params).ravel()
        assert self._mlp.size == mlp_arch_param_count(arch)
        self.P.mlp_params = _ptr(self._mlp)
        self.P.mlp_enc, self.P.mlp_h1, self.P.mlp_h2, self.P.mlp_h3 = (int(a) for a in arch)
        self.P.mlp_mode = 2 if margin is None else 1
        self.P.mlp_margin = 0.0 if margin is None else float(margin)

    def set_ball(self, pos, vel):
        """Ball position and velocity (world frame) at the current robot state."""
        self._ball = _f64(np.concatenate([np.asarray(pos, float).ravel(), np.asarray(vel, float).ravel()]))
        assert self._ball.shape == (6,)
        self.P.ball = _ptr(self._ball)

    @property
    def n_noise(self):
        p = self.params
        return p.n_knots if (p.filter == 0 and p.n_knots > 0) else p.H

    # -- stages
    def noise(self, step: int, it: int) -> np.ndarray:
        p = self.params
        if p.sampler == 1:
            return noise_halton(p.N, self.n_noise, self.d, p.halton_scramble, p.seed)
        return noise_philox(p.seed, step, p.instance, it, 0,
                            p.N * self.n_noise * self.d).reshape(p.N, self.n_noise, self.d)

    def fk(self, theta) -> np.ndarray:
        th = _f64(theta)
        frames = np.zeros((self.d + 1, 4, 4))
        lib().orc_fk(C.byref(self.R), _ptr(th), _ptr(frames))
        return frames

    def ee_twist(self, theta, theta_dot, theta_ddot):
        """(X_dot, X_ddot) of Eq. 8, each [linear; angular] (6,)."""
        frames = self.fk(theta)
        xd, xdd = np.zeros(6), np.zeros(6)
        lib().orc_ee_twist(C.byref(self.R), _ptr(frames), _ptr(_f64(theta_dot)),
                           _ptr(_f64(theta_ddot)), _ptr(xd), _ptr(xdd))
        return xd, xdd

    def ball_states(self, state, theta):
        """Ball position and velocity in the end-effector frame along one rollout (H x 3 each)."""
        H = self.params.H
        xb, vb = np.zeros((H, 3)), np.zeros((H, 3))
        rc = lib().orc_ball_states(C.byref(self.R), C.byref(self.P), _ptr(_f64(state)),
                                   _ptr(_f64(theta)), _ptr(xb), _ptr(vb))
        if rc != 0:
            raise ValueError("no ball state set")
        return xb, vb

    def jacobian(self, theta) -> np.ndarray:
        frames = self.fk(theta)
        J = np.zeros((6, self.d))
        lib().orc_jacobian(C.byref(self.R), _ptr(frames), _ptr(J))
        return J

    def self_min_sd(self, theta) -> float:
        frames = self.fk(theta)
        return lib().orc_self_min_sd(C.byref(self.R), _ptr(frames))

    def self_min_sd_theta(self, theta) -> float:
        return lib().orc_self_min_sd_theta(C.byref(self.R), _ptr(_f64(theta)))

    def world_min_sd(self, theta) -> float:
        frames = self.fk(theta)
        return lib().orc_world_min_sd(C.byref(self.R), C.byref(self.W), _ptr(frames))

    def running_cost(self, goal, h, theta_h, theta_dot_h, u_h, u_prev):
        terms = np.zeros(NTERMS)
        tot = C.c_double()
        lib().orc_running_cost(C.byref(self.R), C.byref(self.W), C.byref(self.P),
                               _ptr(_f64(goal)), int(h), _ptr(_f64(theta_h)),
                               _ptr(_f64(theta_dot_h)), _ptr(_f64(u_h)), _ptr(_f64(u_prev)),
                               _ptr(terms), C.byref(tot))
        return terms, tot.value

    def controls(self, mu, sigma, eps) -> np.ndarray:
        p = self.params
        u = np.zeros((p.N, p.H, self.d))
        lib().orc_smooth_controls(C.byref(self.P), self.d, _ptr(_f64(mu)), _ptr(_f64(sigma)),
                                  _ptr(_f64(eps)), _ptr(u))
        return u

    def rollout(self, state, goal, mu, sigma, eps) -> dict:
        p, d = self.params, self.d
        out = dict(u=np.zeros((p.N, p.H, d)), theta=np.zeros((p.N, p.H, d)),
                   theta_dot=np.zeros((p.N, p.H, d)), ee=np.zeros((p.N, p.H, 3, 4)),
                   terms=np.zeros((p.N, p.H, NTERMS)), cost=np.zeros((p.N, p.H)),
                   C=np.zeros(p.N))
        rc = lib().orc_rollout(C.byref(self.R), C.byref(self.W), C.byref(self.P),
                               _ptr(_f64(state)), _ptr(_f64(goal)), _ptr(_f64(mu)),
                               _ptr(_f64(sigma)), _ptr(_f64(eps)), _ptr(out["u"]),
                               _ptr(out["theta"]), _ptr(out["theta_dot"]), _ptr(out["ee"]),
                               _ptr(out["terms"]), _ptr(out["cost"]), _ptr(out["C"]))
        if rc != 0:
            raise ValueError(f"orc_rollout failed: {rc}")
        return out

    def running_cost_grad(self, goal, h, theta_h, theta_dot_h, u_h, u_prev):
        d = self.d
        g = [np.zeros(d) for _ in range(4)]
        lib().orc_running_cost_grad(C.byref(self.R), C.byref(self.W), C.byref(self.P),
                                    _ptr(_f64(goal)), int(h), _ptr(_f64(theta_h)),
                                    _ptr(_f64(theta_dot_h)), _ptr(_f64(u_h)), _ptr(_f64(u_prev)),
                                    *[_ptr(x) for x in g])
        return g

    def cost_grad(self, state, goal, mu, sigma, eps, per_particle=False):
        """J(mu) = mean_n C_n and dJ/dmu (H x d), noise eps fixed."""
        p = self.params
        grad = np.zeros((p.H, self.d))
        J = C.c_double()
        dcdu = np.zeros((p.N, p.H, self.d)) if per_particle else None
        rc = lib().orc_cost_grad(C.byref(self.R), C.byref(self.W), C.byref(self.P),
                                 _ptr(_f64(state)), _ptr(_f64(goal)), _ptr(_f64(mu)),
                                 _ptr(_f64(sigma)), _ptr(_f64(eps)), _ptr(grad), C.byref(J),
                                 _ptr(dcdu))
        if rc != 0:
            raise ValueError("orc_cost_grad failed")
        return (J.value, grad, dcdu) if per_particle else (J.value, grad)

    def update(self, Ctot, u, mu, sigma):
        mu = _f64(mu).copy()
        sigma = _f64(sigma).copy()
        w = np.zeros(self.params.N)
        st = lib().orc_update(C.byref(self.P), self.d, _ptr(_f64(Ctot)), _ptr(_f64(u)), _ptr(mu),
                              _ptr(sigma), _ptr(w))
        return mu, sigma, st, w

    def step(self, state, goal, step, mu, sigma):
        mu = _f64(mu).copy()
        sigma = _f64(sigma).copy()
        cmd = np.zeros(self.d)
        best = C.c_double()
        st = lib().orc_step(C.byref(self.R), C.byref(self.W), C.byref(self.P), _ptr(_f64(state)),
                            _ptr(_f64(goal)), int(step), _ptr(mu), _ptr(sigma), _ptr(cmd),
                            C.byref(best))
        return cmd, mu, sigma, st, best.value


def from_workload(wl) -> Oracle:
    return Oracle(wl.robot, wl.world, wl.params)
