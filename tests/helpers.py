"""Shared helpers of the GPU tests: seeded cases, the oracle's reference step,
relative errors and the support-flip rule."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2207_11669_gb300 import synth


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def make_case(m, n_i, r, *, seed=0, k=None, density=0.05, amp=10.0, factor_std=1.0,
              rho=1e-2, lam=None):
    """A seeded instance plus identical float32 starting points for both sides."""
    n_i = np.asarray(n_i, np.int64)
    n = int(n_i.sum())
    k = r if k is None else k
    inst = synth.make_instance(m, n, k, seed=seed, density=density, amp=amp,
                               factor_std=factor_std, n_i=n_i)
    lam = 1.0 / np.sqrt(m) if lam is None else lam
    U0 = synth.gaussian_u0(m, r, seed)
    V0 = O.init_v0(inst.M, U0.astype(np.float64), rho).astype(np.float32)
    return dict(inst=inst, M=inst.M, n_i=n_i, r=r, rho=rho, lam=lam, U0=U0, V0=V0)


def r_error_bound(M, U, V, r):
    """Bound on |R_fp32 - R_exact| for R = M - U V^T formed with an FP32
    length-r FMA chain and one subtraction: (r + 2) u (|M| + |U||V|^T)."""
    u = 2.0 ** -24
    return (r + 2) * u * (np.abs(M).astype(np.float64)
                          + np.abs(U.astype(np.float64)) @ np.abs(V.astype(np.float64)).T)


def support_flips(S_gpu, S_ref, R_ref, lam, eps):
    """Entries whose support differs, and those among them NOT explained by
    being within 1e-5*lambda (+ the FP32 error of R) of the threshold."""
    flip = (S_gpu != 0) != (S_ref != 0)
    near = np.abs(np.abs(R_ref) - lam) <= 1e-5 * lam + eps
    return int(flip.sum()), int((flip & ~near).sum())
