"""Pins of the FP64 unrolled-network oracle and its hand-derived adjoint."""
import numpy as np
import pytest

import oracle as O
from oracle import unrolled as UN
from paper_2207_11669_gb300 import synth


def tiny(seed=3, m=12, n=14, k=2, lam=0.35, rho=0.05, K=3):
    inst = synth.make_instance(m, n, k, seed=seed, density=0.1, amp=3.0, factor_std=1.0, E=2)
    U0 = synth.gaussian_u0(m, k, seed).astype(np.float64) * 2.0
    V0 = O.init_v0(inst.M, U0, rho)
    return inst, U0, V0, lam, rho, K


def kink_margin(M, traj, lam, rho, theta):
    """Smallest distance of |R| to lambda_k over the steps (FD is only valid away from it)."""
    a = theta[0]
    mg = np.inf
    for kk in range(len(a)):
        U, V = traj[kk]
        R = M - U @ V.T
        mg = min(mg, np.min(np.abs(np.abs(R) - lam * np.exp(a[kk]))))
    return mg


def test_untrained_network_is_plain_iterations():
    inst, U0, V0, lam, rho, K = tiny()
    theta = (np.zeros(K), np.zeros(K), np.ones(K))
    loss, traj = UN.unrolled_forward(inst.M, U0, V0, inst.A, inst.B, lam, rho, theta)
    U, V, S, _, _ = O.dcf_run(inst.M, inst.n_i, U0, V0, rho, lam, K)
    assert np.max(np.abs(traj[-1][0] - U)) < 1e-10
    assert np.max(np.abs(traj[-1][1] - V)) < 1e-10


def test_factor_loss_matches_dense():
    inst, U0, V0, lam, rho, K = tiny()
    L0 = inst.A.astype(np.float64) @ inst.B.T.astype(np.float64)
    d = np.sum((U0 @ V0.T - L0) ** 2) / np.sum(L0 ** 2)
    assert abs(UN.factor_loss(U0, V0, inst.A, inst.B) - d) < 1e-10


@pytest.mark.parametrize("seed", [3, 5])
def test_adjoint_matches_central_differences(seed):
    inst, U0, V0, lam, rho, K = tiny(seed=seed)
    g = np.random.default_rng(seed)
    theta = (g.uniform(-0.3, 0.3, K), g.uniform(-0.3, 0.3, K), g.uniform(0.6, 1.2, K))
    loss, traj = UN.unrolled_forward(inst.M, U0, V0, inst.A, inst.B, lam, rho, theta)
    assert kink_margin(inst.M, traj, lam, rho, theta) > 1e-4
    (ga, gb, gc), _ = UN.unrolled_backward(inst.M, traj, inst.A, inst.B, lam, rho, theta)
    h = 1e-6
    grads = (ga, gb, gc)
    for which in range(3):
        for kk in range(K):
            tp = [t.copy() for t in theta]
            tm = [t.copy() for t in theta]
            tp[which][kk] += h
            tm[which][kk] -= h
            lp, _ = UN.unrolled_forward(inst.M, U0, V0, inst.A, inst.B, lam, rho, tp)
            lm, _ = UN.unrolled_forward(inst.M, U0, V0, inst.A, inst.B, lam, rho, tm)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grads[which][kk]) <= 1e-6 * max(1.0, abs(fd)), (which, kk, fd,
                                                                              grads[which][kk])


def test_adjoint_wrt_start_point_matches_central_differences():
    inst, U0, V0, lam, rho, K = tiny(seed=7)
    theta = (np.full(K, 0.1), np.full(K, -0.2), np.full(K, 0.9))
    loss, traj = UN.unrolled_forward(inst.M, U0, V0, inst.A, inst.B, lam, rho, theta)
    _, (Ubar, Vbar) = UN.unrolled_backward(inst.M, traj, inst.A, inst.B, lam, rho, theta)
    h = 1e-6
    for (i, j) in [(0, 0), (3, 1), (11, 0)]:
        Up, Um = U0.copy(), U0.copy()
        Up[i, j] += h
        Um[i, j] -= h
        lp, _ = UN.unrolled_forward(inst.M, Up, V0, inst.A, inst.B, lam, rho, theta)
        lm, _ = UN.unrolled_forward(inst.M, Um, V0, inst.A, inst.B, lam, rho, theta)
        assert abs((lp - lm) / (2 * h) - Ubar[i, j]) < 1e-6 * max(1.0, abs(Ubar[i, j]))
    for (i, j) in [(0, 0), (5, 1), (13, 0)]:
        Vp, Vm = V0.copy(), V0.copy()
        Vp[i, j] += h
        Vm[i, j] -= h
        lp, _ = UN.unrolled_forward(inst.M, U0, Vp, inst.A, inst.B, lam, rho, theta)
        lm, _ = UN.unrolled_forward(inst.M, U0, Vm, inst.A, inst.B, lam, rho, theta)
        assert abs((lp - lm) / (2 * h) - Vbar[i, j]) < 1e-6 * max(1.0, abs(Vbar[i, j]))


def _fd_residual(backward_fn, seed=3):
    """Largest |FD - adjoint| over the parameters, for a given backward function."""
    inst, U0, V0, lam, rho, K = tiny(seed=seed)
    g = np.random.default_rng(seed)
    theta = (g.uniform(-0.3, 0.3, K), g.uniform(-0.3, 0.3, K), g.uniform(0.6, 1.2, K))
    loss, traj = UN.unrolled_forward(inst.M, U0, V0, inst.A, inst.B, lam, rho, theta)
    grads = backward_fn(inst.M, traj, inst.A, inst.B, lam, rho, theta)[0]
    h, res = 1e-6, 0.0
    for which in range(3):
        for kk in range(K):
            tp = [t.copy() for t in theta]
            tm = [t.copy() for t in theta]
            tp[which][kk] += h
            tm[which][kk] -= h
            lp, _ = UN.unrolled_forward(inst.M, U0, V0, inst.A, inst.B, lam, rho, tp)
            lm, _ = UN.unrolled_forward(inst.M, U0, V0, inst.A, inst.B, lam, rho, tm)
            res = max(res, abs((lp - lm) / (2 * h) - grads[which][kk]))
    return res


def _mutated_backward(mutation):
    orig = UN.step_backward

    def step_backward(cache, Ubar_n, Vbar_n):
        c = dict(cache)
        if mutation == "no_mask":
            c["lam"] = -1.0          # treats every entry as clamped
        Ub, Vb, lb, rb, ab = orig(c, Ubar_n, Vbar_n)
        if mutation == "rho_sign":
            rb = -rb
        if mutation == "drop_alpha_term":
            ab = 0.0
        return Ub, Vb, lb, rb, ab

    def backward(*args, **kw):
        saved = UN.step_backward
        UN.step_backward = step_backward
        try:
            return UN.unrolled_backward(*args, **kw)
        finally:
            UN.step_backward = saved
    return backward


@pytest.mark.parametrize("mutation", ["no_mask", "rho_sign", "drop_alpha_term"])
def test_planted_adjoint_mistakes_are_caught(mutation):
    assert _fd_residual(UN.unrolled_backward) < 1e-6
    assert _fd_residual(_mutated_backward(mutation)) > 1e-4
