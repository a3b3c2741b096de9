"""Shared helpers of the GPU parity tests: tolerance model and array plumbing.

Tolerances (FP32 GPU against the FP64 oracle):
  * joint states, end-effector poses: 1e-5 relative with scale 1 (rad, m)
  * cost terms and weighted costs: 1e-4 relative to max |c_hat| (Eq. 15)
  * the manipulability term jumps from (1 - k_m) to 0 at m = k_m (Eq. 12):
    items whose oracle score lies within 1e-4 of k_m may take the other branch
    in FP32; they are counted, must stay below 0.1 % of all items, and are
    excluded from the cost comparison
  * updated mean / sigma: 1e-4 relative, widened by kappa / 1e-5 where
    kappa = max|C_hat| * 2^-23 / beta (FP32 cost error amplified by the
    exponential weights, Eq. 6); the distribution update alone, fed identical
    inputs, is held to 1e-5
"""
import numpy as np
import torch

import oracle

TOL_STATE = 1e-5
TOL_COST = 1e-4
TOL_UPDATE = 1e-5


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(np.asarray(a, dtype=np.float32)), device="cuda")


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def f32(a):
    """The FP32 value both sides see (inputs are handed to the GPU as float)."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def max_rel(g, o, scale):
    g, o = np.asarray(g, np.float64), np.asarray(o, np.float64)
    if g.size == 0:
        return 0.0
    return float(np.max(np.abs(g - o)) / max(scale, 1e-30))


def kappa(C, beta):
    C = np.asarray(C)
    C = C[np.isfinite(C)]
    if beta <= 0 or C.size == 0:
        return 0.0
    return float(np.max(np.abs(C)) * 2.0 ** -23 / beta)


def mu_tolerance(C, beta):
    return 1e-4 * max(1.0, kappa(C, beta) / 1e-5)


def manip_flips(orc, theta, k_m, g_terms, o_terms, band=1e-4):
    """Items where the two sides disagree on the manipulability branch.
    Returns (mask of flipped items, all flips within the band)."""
    gm = g_terms[..., 4] > 0
    om = o_terms[..., 4] > 0
    flip = gm != om
    ok = True
    for idx in zip(*np.nonzero(flip)):
        m = oracle.manipulability(orc.jacobian(theta[idx]))
        ok &= abs(m - k_m) < band
    return flip, ok
