"""ctypes binding of ``libstorm_b300.so`` (the C ABI declared in ``include/storm.h``).

Argument marshalling only: every step of the control path runs in the CUDA
library.  PyTorch supplies device memory and the CUDA stream.  There is no CPU
fallback: if the library is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
LIB_PATH = os.path.join(_HERE, "libstorm_b300.so")
_SOURCES = [os.path.join(_HERE, "csrc", f) for f in sorted(os.listdir(os.path.join(_HERE, "csrc")))
            if f.endswith((".cu", ".cuh"))] + [os.path.join(_ROOT, "include", "storm.h")]

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
              "-Xcompiler", "-fPIC", "-shared"]

STORM_OK = 0
STORM_WARN_DEGENERATE = 1
STORM_ERR_INVALID_ARG = -1
STORM_ERR_CUDA = -2
STORM_ERR_OOM = -3
STORM_ERR_NONFINITE = -4
STORM_ERR_TIMEOUT = -5
STORM_ERR_STATE = -6
STORM_MAP_CTA = 0
STORM_MAP_WARP = 1
STORM_MAP_WARP_PAIR = 2
STORM_MAP_WARP_QUAD = 3
NTERMS = 11

EXPORTED = [
    "storm_create", "storm_destroy", "storm_status_string", "storm_last_error", "storm_reset",
    "storm_step", "storm_step_async", "storm_sync", "storm_device_io", "storm_shift",
    "storm_sample_noise", "storm_generate_rollouts", "storm_update_distribution", "storm_get_distribution",
    "storm_set_distribution", "storm_set_world", "storm_forward_kinematics", "storm_get_state",
    "storm_set_state", "storm_rollout_costs_noalloc", "storm_set_launch", "storm_get_launch", "storm_set_launch_warp", "storm_get_launch_mapping",
    "storm_ee_twist", "storm_set_ball", "storm_set_launch_warp_pair", "storm_set_launch_warp_quad",
    "storm_autotune", "storm_cost_grad", "storm_batch_create", "storm_batch_destroy",
    "storm_batch_last_error", "storm_batch_sizes", "storm_batch_step", "storm_batch_step_resident",
    "storm_batch_device_io", "storm_batch_sync", "storm_batch_get_distribution",
    "storm_batch_set_distribution", "storm_batch_autotune", "storm_batch_get_launch",
    "storm_batch_set_launch", "storm_batch_set_launch_warp", "storm_batch_get_launch_mapping",
    "storm_set_dependent_launch", "storm_get_dependent_launch",
    "storm_mlp_create", "storm_mlp_destroy", "storm_mlp_last_error", "storm_mlp_get_params",
    "storm_mlp_set_params", "storm_mlp_predict", "storm_mlp_loss_grad", "storm_mlp_train",
    "storm_self_distance", "storm_set_surrogate", "storm_set_broadphase", "storm_set_trace",
    "storm_mlp_create_arch", "storm_mlp_param_count", "storm_set_surrogate_cost",
    "storm_philox_words", "storm_mlp_wait_probe", "storm_mlp_predict_layers", "storm_fp32_peak",
    "storm_mlp_predict_async",
]
MLP_PARAMS = 135937


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile csrc/storm.cu for sm_103a into the package directory."""
    newest = max(os.path.getmtime(s) for s in _SOURCES)
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < newest:
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["nvcc", *NVCC_FLAGS, "-I", os.path.join(_ROOT, "include"), "-o", tmp,
               os.path.join(_HERE, "csrc", "storm.cu")]
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int)


class storm_robot(C.Structure):
    _fields_ = [("dof", C.c_int), ("dh", _dp), ("q_min", _dp), ("q_max", _dp),
                ("n_spheres", C.c_int), ("sphere_link", _ip), ("spheres", _dp),
                ("n_pairs", C.c_int), ("pairs", _ip)]


class storm_world(C.Structure):
    _fields_ = [("n_boxes", C.c_int), ("boxes", _dp), ("n_spheres", C.c_int), ("spheres", _dp)]


class storm_params(C.Structure):
    _fields_ = [("N", C.c_int), ("H", C.c_int), ("K", C.c_int), ("n_knots", C.c_int),
                ("sampler", C.c_int), ("n_null", C.c_int), ("dt", _dp), ("beta", C.c_double),
                ("gamma", C.c_double), ("alpha_mu", C.c_double), ("alpha_sigma", C.c_double),
                ("sigma_init", C.c_double), ("sigma_min", C.c_double), ("w_pos", C.c_double),
                ("w_rot", C.c_double), ("w_stop", C.c_double), ("w_joint", C.c_double),
                ("w_manip", C.c_double), ("w_coll", C.c_double), ("w_smooth", C.c_double),
                ("pos_axis_w", C.c_double * 3), ("rot_axis_w", C.c_double * 3),
                ("rot_mode", C.c_int), ("k_jl", C.c_double), ("k_m", C.c_double),
                ("qdd_max", C.c_double), ("seed", C.c_uint64), ("instance", C.c_uint32),
                ("grad_steps", C.c_int), ("grad_eta", C.c_double), ("filter", C.c_int),
                ("comb", C.c_double * 3), ("mix_bspline", C.c_double), ("w_ee_vel", C.c_double),
                ("w_ee_acc", C.c_double), ("ee_vel_max", C.c_double), ("ee_acc_max", C.c_double),
                ("w_ball", C.c_double), ("gravity", C.c_double * 3), ("tray_center", C.c_double * 3),
                ("halton_scramble", C.c_int)]


class storm_step_info(C.Structure):
    _fields_ = [("best_cost", C.c_float), ("mean_weighted_cost", C.c_float),
                ("status", C.c_int), ("step", C.c_uint32)]


_lib = None


def lib():
    """Load the library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.storm_create.argtypes = [C.POINTER(storm_robot), C.POINTER(storm_world),
                                   C.POINTER(storm_params), vp, C.POINTER(vp)]
        L.storm_destroy.argtypes = [vp]
        L.storm_destroy.restype = None
        L.storm_status_string.argtypes = [C.c_int]
        L.storm_status_string.restype = C.c_char_p
        L.storm_last_error.argtypes = [vp]
        L.storm_last_error.restype = C.c_char_p
        L.storm_reset.argtypes = [vp]
        L.storm_step.argtypes = [vp, _fp, _fp, _fp, C.POINTER(storm_step_info)]
        L.storm_step_async.argtypes = [vp, vp, vp, vp]
        L.storm_sync.argtypes = [vp, C.POINTER(storm_step_info)]
        L.storm_device_io.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp)]
        L.storm_shift.argtypes = [vp]
        L.storm_generate_rollouts.argtypes = [vp, vp, vp, C.c_uint32, C.c_int, vp, vp, vp, vp, vp,
                                              vp, vp]
        L.storm_update_distribution.argtypes = [vp, vp, vp, vp]
        L.storm_sample_noise.argtypes = [vp, C.c_uint32, C.c_int, vp]
        L.storm_philox_words.argtypes = [vp, C.c_uint32, C.c_int, C.c_uint32, C.c_int, vp]
        L.storm_mlp_wait_probe.argtypes = [vp, C.c_uint]
        L.storm_fp32_peak.argtypes = [C.c_int, C.POINTER(C.c_float), C.POINTER(C.c_float)]
        L.storm_get_distribution.argtypes = [vp, _fp, _fp]
        L.storm_set_distribution.argtypes = [vp, _fp, _fp]
        L.storm_set_world.argtypes = [vp, C.POINTER(storm_world)]
        L.storm_forward_kinematics.argtypes = [vp, vp, C.c_int, vp]
        L.storm_get_state.argtypes = [vp, vp, C.POINTER(C.c_size_t)]
        L.storm_set_state.argtypes = [vp, vp, C.c_size_t]
        L.storm_set_launch.argtypes = [vp, C.c_int, C.c_int]
        L.storm_get_launch.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.storm_set_launch_warp.argtypes = [vp, C.c_int]
        L.storm_set_launch_warp_pair.argtypes = [vp, C.c_int]
        L.storm_set_launch_warp_quad.argtypes = [vp, C.c_int]
        L.storm_ee_twist.argtypes = [vp, vp, vp, vp, C.c_int, vp, vp]
        L.storm_set_ball.argtypes = [vp, C.POINTER(C.c_float)]
        L.storm_get_launch_mapping.argtypes = [vp]
        L.storm_autotune.argtypes = [vp, C.POINTER(C.c_float)]
        L.storm_cost_grad.argtypes = [vp, vp, vp, vp, C.c_uint32, C.c_int, vp, vp, vp]
        ip = C.POINTER(C.c_int)
        L.storm_batch_create.argtypes = [C.c_int, C.POINTER(storm_robot), C.POINTER(storm_world),
                                         C.POINTER(storm_params), vp, C.POINTER(vp)]
        L.storm_batch_destroy.argtypes = [vp]
        L.storm_batch_destroy.restype = None
        L.storm_batch_last_error.argtypes = [vp]
        L.storm_batch_last_error.restype = C.c_char_p
        L.storm_batch_sizes.argtypes = [vp, ip, ip]
        L.storm_batch_step.argtypes = [vp, _fp, _fp, _fp, ip]
        L.storm_batch_step_resident.argtypes = [vp]
        L.storm_batch_device_io.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp)]
        L.storm_batch_sync.argtypes = [vp]
        L.storm_batch_get_distribution.argtypes = [vp, C.c_int, _fp, _fp]
        L.storm_batch_set_distribution.argtypes = [vp, C.c_int, _fp, _fp]
        L.storm_batch_autotune.argtypes = [vp, C.POINTER(C.c_float)]
        L.storm_batch_get_launch.argtypes = [vp, ip, ip]
        L.storm_batch_set_launch.argtypes = [vp, C.c_int, C.c_int]
        L.storm_batch_set_launch_warp.argtypes = [vp, C.c_int]
        L.storm_batch_get_launch_mapping.argtypes = [vp]
        L.storm_set_dependent_launch.argtypes = [vp, C.c_int]
        L.storm_get_dependent_launch.argtypes = [vp]
        L.storm_mlp_create.argtypes = [C.c_uint64, vp, C.POINTER(vp)]
        L.storm_mlp_create_arch.argtypes = [C.c_uint64, C.c_int, vp, C.POINTER(vp)]
        L.storm_mlp_param_count.argtypes = [vp]
        L.storm_set_surrogate_cost.argtypes = [vp, vp]
        L.storm_mlp_destroy.argtypes = [vp]
        L.storm_mlp_destroy.restype = None
        L.storm_mlp_last_error.argtypes = [vp]
        L.storm_mlp_last_error.restype = C.c_char_p
        L.storm_mlp_get_params.argtypes = [vp, _fp]
        L.storm_mlp_set_params.argtypes = [vp, _fp]
        L.storm_mlp_predict.argtypes = [vp, vp, C.c_int, C.c_int, vp]
        L.storm_mlp_predict_layers.argtypes = [vp, vp, C.c_int, C.c_int, vp]
        L.storm_mlp_predict_async.argtypes = [vp, vp, C.c_int, C.c_int, vp]
        L.storm_mlp_loss_grad.argtypes = [vp, vp, vp, C.c_int, C.c_int, _fp, _fp]
        L.storm_mlp_train.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_float,
                                      C.c_uint64, _fp]
        L.storm_self_distance.argtypes = [vp, vp, C.c_int, vp]
        L.storm_set_surrogate.argtypes = [vp, vp, C.c_double]
        L.storm_set_broadphase.argtypes = [vp, C.c_int]
        L.storm_set_trace.argtypes = [vp, vp]
        _lib = L
    return _lib


def fp32_peak(iters: int = 8192) -> dict:
    """storm_fp32_peak: measured FP32 FMA TFLOP/s of the current device (scalar and
    paired FMA instructions)."""
    a, b = C.c_float(), C.c_float()
    rc = lib().storm_fp32_peak(int(iters), C.byref(a), C.byref(b))
    if rc != 0:
        raise StormError(rc, "storm_fp32_peak failed")
    return {"scalar_tflops": a.value, "paired_tflops": b.value}


def status_string(code: int) -> str:
    return lib().storm_status_string(int(code)).decode()


class StormError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{status_string(code)} ({code}): {msg}")
        self.code = code


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _p(a, t=_dp):
    return a.ctypes.data_as(t)


def _dptr(t):
    """Raw device pointer of a CUDA tensor, or None."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


class _Marshal:
    """Keeps the numpy buffers behind the ctypes structs alive."""

    def __init__(self):
        self.keep = []

    def hold(self, a):
        self.keep.append(a)
        return a

    def robot(self, r):
        dh = self.hold(_f64(r.dh))
        qmin, qmax = self.hold(_f64(r.q_min)), self.hold(_f64(r.q_max))
        link = self.hold(np.ascontiguousarray(r.sphere_link, dtype=np.int32))
        sph = self.hold(_f64(r.spheres).reshape(-1, 4))
        pairs = self.hold(np.ascontiguousarray(np.asarray(r.pairs, dtype=np.int32).reshape(-1, 2)))
        return storm_robot(dh.shape[0], _p(dh), _p(qmin), _p(qmax), sph.shape[0], _p(link, _ip),
                           _p(sph), pairs.shape[0], _p(pairs, _ip))

    def world(self, w):
        boxes = self.hold(_f64(w.boxes).reshape(-1, 6))
        sph = self.hold(_f64(w.spheres).reshape(-1, 4))
        return storm_world(boxes.shape[0], _p(boxes), sph.shape[0], _p(sph))

    def params(self, p):
        dt = self.hold(_f64(p.dt))
        s = storm_params()
        s.N, s.H, s.K, s.n_knots, s.sampler, s.n_null = p.N, p.H, p.K, p.n_knots, p.sampler, p.n_null
        s.dt = _p(dt)
        s.beta, s.gamma, s.alpha_mu, s.alpha_sigma = p.beta, p.gamma, p.alpha_mu, p.alpha_sigma
        s.sigma_init, s.sigma_min = p.sigma_init, p.sigma_min
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
        s.halton_scramble = int(p.halton_scramble)
        return s


class _StepIO:
    """Host buffers of Controller.step, reused across calls with their C pointers
    formed once (marshalling cost per call: two copies in, one out)."""

    def __init__(self, d):
        self.st = np.zeros(3 * d, dtype=np.float32)
        self.g = np.zeros(7, dtype=np.float32)
        self.cmd = np.zeros(d, dtype=np.float32)
        self.info = storm_step_info()
        self.p_st, self.p_g, self.p_cmd = _p(self.st, _fp), _p(self.g, _fp), _p(self.cmd, _fp)
        self.p_info = C.byref(self.info)
        self.fn = lib().storm_step


class Controller:
    """One STORM MPC handle (``storm_create`` ... ``storm_destroy``)."""

    def __init__(self, robot, world, params, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("STORM controller needs a CUDA device")
        self.torch = torch
        self.params = params
        self.d = int(robot.dh.shape[0])
        self.N, self.H = int(params.N), int(params.H)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        m = _Marshal()
        r, w, p = m.robot(robot), m.world(world), m.params(params)
        h = C.c_void_p()
        rc = lib().storm_create(C.byref(r), C.byref(w), C.byref(p),
                                C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if rc != 0:
            raise StormError(rc, "storm_create failed (see stderr)")
        self.h = h
        self._io = _StepIO(self.d)

    # ------------------------------------------------------------------ plumbing
    def _check(self, rc, allow_warn=True):
        if rc < 0 or (rc > 0 and not allow_warn):
            raise StormError(rc, lib().storm_last_error(self.h).decode())
        return rc

    def _join(self):
        """Make the handle's stream wait for work queued on torch's current stream."""
        self.stream.wait_stream(self.torch.cuda.current_stream())

    def _empty(self, *shape):
        with self.torch.cuda.stream(self.stream):
            return self.torch.empty(shape, dtype=self.torch.float32, device="cuda")

    def close(self):
        if getattr(self, "h", None):
            lib().storm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------ control step
    def step(self, state, goal):
        """Host-buffer control step -> (cmd (d,), info dict, status)."""
        io = self._io
        if np.size(state) != 3 * self.d or np.size(goal) != 7:
            raise ValueError("state must have 3*dof values and goal 7")
        io.st[:] = np.ravel(state)  # (float32 conversion into the reused buffers)
        io.g[:] = np.ravel(goal)
        rc = io.fn(self.h, io.p_st, io.p_g, io.p_cmd, io.p_info)
        self._check(rc)
        info = io.info
        return io.cmd.copy(), dict(best_cost=info.best_cost, mean_weighted_cost=info.mean_weighted_cost,
                                   status=info.status, step=info.step), rc

    def step_async(self, state_dev, goal_dev, cmd_dev):
        self._join()
        self._check(lib().storm_step_async(self.h, _dptr(state_dev), _dptr(goal_dev),
                                           _dptr(cmd_dev)))

    def sync(self):
        info = storm_step_info()
        rc = self._check(lib().storm_sync(self.h, C.byref(info)))
        return dict(best_cost=info.best_cost, mean_weighted_cost=info.mean_weighted_cost,
                    status=info.status, step=info.step), rc

    def device_io_ptrs(self):
        s, g, c = C.c_void_p(), C.c_void_p(), C.c_void_p()
        self._check(lib().storm_device_io(self.h, C.byref(s), C.byref(g), C.byref(c)))
        return s.value, g.value, c.value

    def step_resident(self):
        """Step on inputs already in the handle's own device buffers (no copies)."""
        s, g, c = self.device_io_ptrs()
        self._check(lib().storm_step_async(self.h, C.c_void_p(s), C.c_void_p(g), C.c_void_p(c)))

    # ------------------------------------------------------------------ stages
    def shift(self):
        self._check(lib().storm_shift(self.h))

    @property
    def n_noise(self):
        return self.params.n_knots if self.params.n_knots > 0 else self.H

    def sample_noise(self, step: int, it: int):
        eps = self._empty(self.N, self.n_noise, self.d)
        self._check(lib().storm_sample_noise(self.h, int(step), int(it), _dptr(eps)))
        self.stream.synchronize()
        return eps

    def philox_words(self, step: int, it: int, first_block: int, count: int):
        """Raw Philox4x32-10 words of the noise stream (count x 4 uint32, host)."""
        import torch
        with torch.cuda.stream(self.stream):
            out = torch.empty((count, 4), dtype=torch.int32, device="cuda")
        self._check(lib().storm_philox_words(self.h, int(step), int(it), int(first_block), int(count),
                                             _dptr(out)))
        self.stream.synchronize()
        return out.cpu().numpy().view(np.uint32)

    def generate_rollouts(self, state_dev, goal_dev, step: int, it: int, debug: bool = True):
        N, H, d = self.N, self.H, self.d
        out = dict(u=self._empty(N, H, d), C=self._empty(N))
        if debug:
            out.update(theta=self._empty(N, H, d), theta_dot=self._empty(N, H, d),
                       ee=self._empty(N, H, 3, 4), terms=self._empty(N, H, NTERMS),
                       cost=self._empty(N, H))
        self._join()
        g = out.get
        self._check(lib().storm_generate_rollouts(
            self.h, _dptr(state_dev), _dptr(goal_dev), int(step), int(it), _dptr(out["u"]),
            _dptr(g("theta")), _dptr(g("theta_dot")), _dptr(g("ee")), _dptr(g("terms")),
            _dptr(g("cost")), _dptr(out["C"])))
        self.stream.synchronize()
        return out

    def cost_grad(self, mean_dev, state_dev, goal_dev, step: int, it: int, want_C=False):
        """J(mu) (1-element tensor) and dJ/dmu (H x d) for the noise of (step, it)."""
        grad = self._empty(self.H, self.d)
        J = self._empty(1)
        Cn = self._empty(self.N) if want_C else None
        self._join()
        self._check(lib().storm_cost_grad(self.h, _dptr(state_dev), _dptr(goal_dev),
                                          _dptr(mean_dev.contiguous()), int(step), int(it),
                                          _dptr(grad), _dptr(J), _dptr(Cn)))
        self.torch.cuda.current_stream().wait_stream(self.stream)
        return (J, grad, Cn) if want_C else (J, grad)

    def update_distribution(self, C_dev, u_dev, want_weights=True):
        w = self._empty(self.N) if want_weights else None
        self._join()
        self._check(lib().storm_update_distribution(self.h, _dptr(C_dev), _dptr(u_dev), _dptr(w)))
        self.stream.synchronize()
        return w

    def get_distribution(self):
        mu = np.zeros((self.H, self.d), dtype=np.float32)
        sg = np.zeros(self.d, dtype=np.float32)
        self._check(lib().storm_get_distribution(self.h, _p(mu, _fp), _p(sg, _fp)))
        return mu, sg

    def set_distribution(self, mu=None, sigma=None):
        m = None if mu is None else _f32(mu).reshape(self.H, self.d)
        s = None if sigma is None else _f32(sigma).reshape(self.d)
        self._check(lib().storm_set_distribution(self.h, None if m is None else _p(m, _fp),
                                                 None if s is None else _p(s, _fp)))

    def set_world(self, world):
        m = _Marshal()
        w = m.world(world)
        self._check(lib().storm_set_world(self.h, C.byref(w)))

    def reset(self):
        self._check(lib().storm_reset(self.h))

    def forward_kinematics(self, theta_dev):
        n = theta_dev.shape[0]
        ee = self._empty(n, 3, 4)
        self._join()
        self._check(lib().storm_forward_kinematics(self.h, _dptr(theta_dev), int(n), _dptr(ee)))
        self.stream.synchronize()
        return ee

    def set_launch(self, particles_per_cta: int, threads: int):
        """CTA-wide mapping with this shape."""
        self._check(lib().storm_set_launch(self.h, int(particles_per_cta), int(threads)))

    def set_launch_warp(self, warps_per_cta: int):
        """Warp mapping (one lane per (particle, step)) with this many warps per CTA."""
        self._check(lib().storm_set_launch_warp(self.h, int(warps_per_cta)))

    def set_launch_warp_pair(self, pairs_per_cta: int):
        """Warp-pair mapping (a cost warp and a collision warp per particle group)."""
        self._check(lib().storm_set_launch_warp_pair(self.h, int(pairs_per_cta)))

    def set_launch_warp_quad(self, groups_per_cta: int):
        """Warp-quad mapping (cost, world + manipulability and two self-collision warps per group)."""
        self._check(lib().storm_set_launch_warp_quad(self.h, int(groups_per_cta)))

    def launch_mapping(self) -> str:
        m = lib().storm_get_launch_mapping(self.h)
        if m < 0:
            self._check(m)
        return {STORM_MAP_WARP: "warp", STORM_MAP_WARP_PAIR: "pair", STORM_MAP_WARP_QUAD: "quad"}.get(m, "cta")

    def set_dependent_launch(self, on: bool):
        """Programmatic dependent launch of the step graph's rollouts and updates."""
        self._check(lib().storm_set_dependent_launch(self.h, 1 if on else 0))

    def dependent_launch(self) -> bool:
        return bool(self._check(lib().storm_get_dependent_launch(self.h)))

    def ee_twist(self, theta_dev, theta_dot_dev, theta_ddot_dev):
        """(X_dot, X_ddot) of Eq. 8 for count configurations: two count x 6 tensors."""
        n = theta_dev.shape[0]
        xd, xdd = self._empty(n, 6), self._empty(n, 6)
        self._join()
        self._check(lib().storm_ee_twist(self.h, _dptr(theta_dev.contiguous()), _dptr(theta_dot_dev.contiguous()),
                                         _dptr(theta_ddot_dev.contiguous()), int(n), _dptr(xd), _dptr(xdd)))
        self.stream.synchronize()
        return xd, xdd

    def set_ball(self, pos, vel):
        """Ball position and velocity (world frame) for the next steps."""
        b = np.ascontiguousarray(np.concatenate([np.ravel(pos), np.ravel(vel)]), dtype=np.float32)
        assert b.shape == (6,)
        self._check(lib().storm_set_ball(self.h, b.ctypes.data_as(C.POINTER(C.c_float))))

    def set_trace(self, trace_dev):
        """trace_dev: int64 CUDA tensor of 7 entries (phase stamps in ns) or None."""
        self._check(lib().storm_set_trace(self.h, _dptr(trace_dev)))
        self._trace = trace_dev

    def set_broadphase(self, on: bool):
        self._check(lib().storm_set_broadphase(self.h, int(bool(on))))

    def get_launch(self):
        a, b = C.c_int(), C.c_int()
        self._check(lib().storm_get_launch(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def autotune(self) -> float:
        t = C.c_float()
        self._check(lib().storm_autotune(self.h, C.byref(t)))
        return t.value

    def self_distance(self, theta_dev):
        """Exact minimum self-pair signed distance for each row of theta_dev (count x dof)."""
        n = int(theta_dev.shape[0])
        out = self._empty(n)
        self._join()
        self._check(lib().storm_self_distance(self.h, _dptr(theta_dev.contiguous()), n, _dptr(out)))
        self.stream.synchronize()
        return out

    def set_surrogate_cost(self, mlp):
        """Self term = max(0, mlp(theta)) (Eq. 13), mlp predicting penetration depth; None stops it."""
        self._check(lib().storm_set_surrogate_cost(self.h, mlp.h if mlp is not None else None))
        self._mlp = mlp

    def set_surrogate(self, mlp, margin: float = 0.05):
        self._check(lib().storm_set_surrogate(self.h, mlp.h if mlp is not None else None,
                                              float(margin)))
        self._mlp = mlp  # keep the network alive while attached

    def get_state(self) -> bytes:
        n = C.c_size_t(0)
        self._check(lib().storm_get_state(self.h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._check(lib().storm_get_state(self.h, buf, C.byref(n)))
        return buf.raw[: n.value]

    def set_state(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        self._check(lib().storm_set_state(self.h, buf, len(blob)))


def rollout_costs_noalloc(robot, world, params, state_dev, goal_dev, mean_dev, sigma_dev,
                          step: int, it: int, Ctot_dev, stream=None) -> int:
    """storm_rollout_costs_noalloc: rollout totals with no device allocation in the
    library (static scratch).  All tensors are caller-owned CUDA tensors."""
    L = lib()
    vp = C.c_void_p
    L.storm_rollout_costs_noalloc.argtypes = [C.POINTER(storm_robot), C.POINTER(storm_world),
                                              C.POINTER(storm_params), vp, vp, vp, vp,
                                              C.c_uint32, C.c_int, vp, vp]
    m = _Marshal()
    r, w, p = m.robot(robot), m.world(world), m.params(params)
    s = C.c_void_p(stream.cuda_stream) if stream is not None else None
    return L.storm_rollout_costs_noalloc(C.byref(r), C.byref(w), C.byref(p), _dptr(state_dev),
                                         _dptr(goal_dev), _dptr(mean_dev), _dptr(sigma_dev),
                                         int(step), int(it), _dptr(Ctot_dev), s)


def _storm_cost_function():
    import torch

    class StormCost(torch.autograd.Function):
        """J(mu) of a controller's rollouts as a differentiable function of the
        mean control sequence; backward is the library's adjoint kernel."""

        @staticmethod
        def forward(ctx, mean, controller, state_dev, goal_dev, step, it):
            J, grad = controller.cost_grad(mean.detach().float(), state_dev, goal_dev, step, it)
            ctx.save_for_backward(grad)
            return J.reshape(())

        @staticmethod
        def backward(ctx, gJ):
            (grad,) = ctx.saved_tensors
            return gJ * grad, None, None, None, None, None

    return StormCost


_StormCost = None


def storm_cost(mean, controller, state_dev, goal_dev, step: int = 0, it: int = 0):
    """Differentiable J(mu): ``storm_cost(mu, ctl, state, goal).backward()``."""
    global _StormCost
    if _StormCost is None:
        _StormCost = _storm_cost_function()
    return _StormCost.apply(mean, controller, state_dev, goal_dev, step, it)


class BatchController:
    """Many uneven controllers stepped together (storm_batch_* C ABI)."""

    def __init__(self, robots, worlds, params, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("STORM batch needs a CUDA device")
        self.torch = torch
        n = len(robots)
        self.n = n
        self.dofs = [int(r.dh.shape[0]) for r in robots]
        self.shapes = [(int(p.H), int(r.dh.shape[0])) for r, p in zip(robots, params)]
        self.stream = stream if stream is not None else torch.cuda.Stream()
        m = _Marshal()
        R = (storm_robot * n)(*[m.robot(r) for r in robots])
        Wd = (storm_world * n)(*[m.world(w) for w in worlds])
        P = (storm_params * n)(*[m.params(p) for p in params])
        h = C.c_void_p()
        rc = lib().storm_batch_create(n, R, Wd, P, C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if rc != 0:
            raise StormError(rc, "storm_batch_create failed (see stderr)")
        self.h = h
        a, b = C.c_int(), C.c_int()
        lib().storm_batch_sizes(self.h, C.byref(a), C.byref(b))
        self.state_floats, self.cmd_floats = a.value, b.value

    def _check(self, rc):
        if rc < 0:
            raise StormError(rc, lib().storm_batch_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            lib().storm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def step(self, states, goals):
        """states: list of (3, dof_i) arrays; goals: (n, 7) -> (list of cmds, statuses)."""
        st = _f32(np.concatenate([np.asarray(s, np.float32).reshape(-1) for s in states]))
        g = _f32(goals).reshape(-1)
        cmds = np.zeros(self.cmd_floats, dtype=np.float32)
        statuses = np.zeros(self.n, dtype=np.int32)
        self._check(lib().storm_batch_step(self.h, _p(st, _fp), _p(g, _fp), _p(cmds, _fp),
                                           statuses.ctypes.data_as(C.POINTER(C.c_int))))
        out, o = [], 0
        for d in self.dofs:
            out.append(cmds[o:o + d].copy())
            o += d
        return out, statuses

    def step_resident(self):
        self._check(lib().storm_batch_step_resident(self.h))

    def sync(self):
        self._check(lib().storm_batch_sync(self.h))

    def get_distribution(self, i):
        H, d = self.shapes[i]
        mu = np.zeros((H, d), dtype=np.float32)
        sg = np.zeros(d, dtype=np.float32)
        self._check(lib().storm_batch_get_distribution(self.h, i, _p(mu, _fp), _p(sg, _fp)))
        return mu, sg

    def autotune(self):
        t = C.c_float()
        self._check(lib().storm_batch_autotune(self.h, C.byref(t)))
        return t.value

    def get_launch(self):
        a, b = C.c_int(), C.c_int()
        self._check(lib().storm_batch_get_launch(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def set_launch(self, items_per_tile: int, threads: int):
        """CTA-wide mapping of the batched rollout."""
        self._check(lib().storm_batch_set_launch(self.h, int(items_per_tile), int(threads)))

    def set_launch_warp(self, warps_per_cta: int):
        """Warp mapping of the batched rollout (the default)."""
        self._check(lib().storm_batch_set_launch_warp(self.h, int(warps_per_cta)))

    def launch_mapping(self) -> str:
        return {STORM_MAP_CTA: "cta", STORM_MAP_WARP: "warp"}[
            self._check(lib().storm_batch_get_launch_mapping(self.h))]


MLP_ARCHS = {"distance": 0, "jointnerf": 1}


class SurrogateMLP:
    """A learned self-collision network (storm_mlp_* C ABI): arch "distance"
    (theta / 3 encoding, 256-256-256) or "jointnerf" (the paper's [sin, cos]
    encoding, 256-128-64)."""

    def __init__(self, seed: int = 0, stream=None, arch: str = "distance"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the surrogate network needs a CUDA device")
        self.torch = torch
        self.arch = arch
        self.stream = stream if stream is not None else torch.cuda.Stream()
        h = C.c_void_p()
        rc = lib().storm_mlp_create_arch(int(seed), MLP_ARCHS[arch], C.c_void_p(self.stream.cuda_stream),
                                         C.byref(h))
        if rc != 0:
            raise StormError(rc, "storm_mlp_create failed (see stderr)")
        self.h = h
        self.n_params = int(lib().storm_mlp_param_count(self.h))

    def _check(self, rc):
        if rc < 0:
            raise StormError(rc, lib().storm_mlp_last_error(self.h).decode())
        return rc

    def _sync_in(self):
        self.stream.wait_stream(self.torch.cuda.current_stream())

    def close(self):
        if getattr(self, "h", None):
            lib().storm_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        self._check(lib().storm_mlp_get_params(self.h, _p(out, _fp)))
        return out

    def set_params(self, params):
        p = _f32(params).reshape(-1)
        assert p.size == self.n_params
        self._check(lib().storm_mlp_set_params(self.h, _p(p, _fp)))

    def predict(self, theta_dev, layers: bool = False, out=None, wait: bool = True):
        """Predictions for theta_dev (count x dof): the fused whole-network kernel,
        or with layers=True the layer-by-layer kernels of the training pass.
        wait=False (fused kernel only) enqueues on the network's stream and
        returns at once."""
        n, dof = int(theta_dev.shape[0]), int(theta_dev.shape[1])
        if out is None:
            with self.torch.cuda.stream(self.stream):
                out = self.torch.empty(n, dtype=self.torch.float32, device="cuda")
        self._sync_in()
        if layers:
            fn = lib().storm_mlp_predict_layers
        else:
            fn = lib().storm_mlp_predict if wait else lib().storm_mlp_predict_async
        self._check(fn(self.h, _dptr(theta_dev.contiguous()), n, dof, _dptr(out)))
        return out

    def wait_probe(self, limit_us: int) -> int:
        """storm_mlp_wait_probe: the bounded tensor-core wait run out on purpose;
        returns the status (STORM_ERR_TIMEOUT when the bound works)."""
        return int(lib().storm_mlp_wait_probe(self.h, int(limit_us)))

    def loss_grad(self, theta_dev, target_dev):
        n, dof = int(theta_dev.shape[0]), int(theta_dev.shape[1])
        loss = np.zeros(1, dtype=np.float32)
        grad = np.zeros(self.n_params, dtype=np.float32)
        self._sync_in()
        self._check(lib().storm_mlp_loss_grad(self.h, _dptr(theta_dev.contiguous()),
                                              _dptr(target_dev.contiguous()), n, dof,
                                              _p(loss, _fp), _p(grad, _fp)))
        return float(loss[0]), grad

    def train(self, theta_dev, target_dev, batch=4096, epochs=4, lr=1e-3, seed=0):
        n, dof = int(theta_dev.shape[0]), int(theta_dev.shape[1])
        losses = np.zeros(epochs, dtype=np.float32)
        self._sync_in()
        self._check(lib().storm_mlp_train(self.h, _dptr(theta_dev.contiguous()),
                                          _dptr(target_dev.contiguous()), n, dof, int(batch),
                                          int(epochs), float(lr), int(seed), _p(losses, _fp)))
        return losses
