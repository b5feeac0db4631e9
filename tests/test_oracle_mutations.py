"""Planted mistakes in the oracle must fail the pins.

Each case swaps one oracle function for a copy with a plausible mistake (a
dropped term, a wrong sign, a wrong weight) and checks that the pin that
guards it reports a large residual.  The mistakes live only in this file.
"""
import numpy as np
import pytest

import oracle as O
from tests import pins


def _hard_threshold_s_step(M, U, V, lam):
    R = M - U @ V.T
    return np.where(np.abs(R) > lam, R, 0.0)


def _flipped_s_step(M, U, V, lam):
    return -O.s_step(M, U, V, lam)


def _v_step_no_rho(M, S, U, rho):
    return O.v_step(M, S, U, 0.0)


def _v_step_half_rho(M, S, U, rho):
    return O.v_step(M, S, U, 0.5 * rho)


def _v_step_ignores_S(M, S, U, rho):
    return O.v_step(M, np.zeros_like(M), U, rho)


def _u_exact_no_rho(Ms, Ss, Vs, rho):
    return O.u_step_exact(Ms, Ss, Vs, 1e-12)


def _u_exact_ignores_S(Ms, Ss, Vs, rho):
    return O.u_step_exact(Ms, [np.zeros_like(S) for S in Ss], Vs, rho)


def _grad_no_share(M_i, U, V_i, S_i, rho, n_i, n):
    return rho * U + (U @ V_i.T + S_i - M_i) @ V_i


def _grad_wrong_sign(M_i, U, V_i, S_i, rho, n_i, n):
    return rho * (n_i / n) * U + (U @ V_i.T - S_i - M_i) @ V_i


def _huber_no_offset(x, lam):
    a = np.abs(np.asarray(x, dtype=float))
    return float(np.sum(np.where(a <= lam, 0.5 * a * a, lam * a)))


def _local_no_share(M_i, U, V_i, S_i, rho, lam, n_i, n):
    return O.local_objective(M_i, U, V_i, S_i, rho, lam, n_i, n) \
        - 0.5 * rho * (n_i / n) * float(np.sum(U * U))


def _weighted_fedavg_iteration(M, n_i, U, V, rho, lam, *, u_mode=0, eta=0.0, local_steps=1):
    # averages the client U_i with weights n_i/n instead of 1/E
    off = O.block_offsets(n_i)
    n = int(off[-1])
    acc = np.zeros_like(U)
    for i in range(len(n_i)):
        Mi = M[:, off[i]:off[i + 1]]
        Si = O.s_step(Mi, U, V[off[i]:off[i + 1]], lam)
        Vi = O.v_step(Mi, Si, U, rho)
        acc += (n_i[i] / n) * (U - eta * O.grad_U_local(Mi, U, Vi, Si, rho, int(n_i[i]), n))
    return acc, None, None


def _fedavg_no_share(Ms, Ss, Vs, U, rho, eta, n_i, n):
    # drops the n_i/n share of the rho term in every client's gradient
    acc = np.zeros_like(U)
    for M, S, V in zip(Ms, Ss, Vs):
        acc += U - eta * (rho * U + (U @ V.T + S - M) @ V)
    return acc / len(Ms)


def _fedavg_weighted(Ms, Ss, Vs, U, rho, eta, n_i, n):
    # weights the client results by n_i/n instead of the unweighted mean
    acc = np.zeros_like(U)
    for M, S, V, ni in zip(Ms, Ss, Vs, n_i):
        acc += (ni / n) * (U - eta * O.grad_U_local(M, U, V, S, rho, ni, n))
    return acc


def _local_steps_round_U(M, n_i, U, V, rho, lam, *, u_mode=0, eta=0.0, local_steps=1):
    # S and V of every local step use the round's U, not the client's own U_i
    off = O.block_offsets(n_i)
    n = int(off[-1])
    Us, Vs, Ss = [], [], []
    for i in range(len(n_i)):
        Mi = M[:, off[i]:off[i + 1]]
        Ui, Vi = U.copy(), V[off[i]:off[i + 1]].copy()
        for _ in range(local_steps):
            Si = O.s_step(Mi, U, Vi, lam)
            Vi = O.v_step(Mi, Si, U, rho)
            Ui = Ui - eta * O.grad_U_local(Mi, Ui, Vi, Si, rho, int(n_i[i]), n)
        Us.append(Ui)
        Vs.append(Vi)
        Ss.append(Si)
    return sum(Us) / len(Us), np.vstack(Vs), np.hstack(Ss)


def _local_steps_average_each_step(M, n_i, U, V, rho, lam, *, u_mode=0, eta=0.0,
                                   local_steps=1):
    # the server averages after every local step instead of once after K
    off = O.block_offsets(n_i)
    n = int(off[-1])
    E = len(n_i)
    Vs = [V[off[i]:off[i + 1]].copy() for i in range(E)]
    Ss = [None] * E
    for _ in range(local_steps):
        acc = np.zeros_like(U)
        for i in range(E):
            Mi = M[:, off[i]:off[i + 1]]
            Ss[i] = O.s_step(Mi, U, Vs[i], lam)
            Vs[i] = O.v_step(Mi, Ss[i], U, rho)
            acc += U - eta * O.grad_U_local(Mi, U, Vs[i], Ss[i], rho, int(n_i[i]), n)
        U = acc / E
    return U, np.vstack(Vs), np.hstack(Ss)


def _local_steps_stale_V(M, n_i, U, V, rho, lam, *, u_mode=0, eta=0.0, local_steps=1):
    # every local step restarts its S-step from the round's V_i
    off = O.block_offsets(n_i)
    n = int(off[-1])
    Us, Vs, Ss = [], [], []
    for i in range(len(n_i)):
        Mi = M[:, off[i]:off[i + 1]]
        Ui = U.copy()
        V0 = V[off[i]:off[i + 1]]
        for _ in range(local_steps):
            Si = O.s_step(Mi, Ui, V0, lam)
            Vi = O.v_step(Mi, Si, Ui, rho)
            Ui = Ui - eta * O.grad_U_local(Mi, Ui, Vi, Si, rho, int(n_i[i]), n)
        Us.append(Ui)
        Vs.append(Vi)
        Ss.append(Si)
    return sum(Us) / len(Us), np.vstack(Vs), np.hstack(Ss)


def _sv_one_factor(X, Y):
    # forgets the right factor's triangular part
    return np.linalg.svd(np.linalg.qr(np.asarray(X, float), mode="r"), compute_uv=False)


def _sv_error_first(sigma, sigma0, k):
    # divides by the largest value of L0 instead of the k-th
    d = np.abs(np.asarray(sigma)[:len(sigma0)] - np.asarray(sigma0)[:len(sigma)])
    return float(np.max(d) / np.max(sigma0))


def _check_sv(fn):
    g = np.random.default_rng(93)
    X, Y = g.standard_normal((30, 5)), g.standard_normal((40, 5))
    d = np.linalg.svd(X @ Y.T, compute_uv=False)[:5]
    return float(np.max(np.abs(fn(X, Y) - d)) / d[0])


def _check_sv_err(fn):
    return abs(fn([3.0, 2.0, 0.5], [3.0, 2.0], 2) - 0.25) + \
        abs(fn([3.1, 1.8], [3.0, 2.0, 1.0], 3) - 1.0)


CASES = [
    ("s_hard", lambda: pins.check_s_step(_hard_threshold_s_step)),
    ("s_sign", lambda: pins.check_s_step(_flipped_s_step)),
    ("v_no_rho", lambda: pins.check_v_step(_v_step_no_rho)),
    ("v_half_rho", lambda: pins.check_v_step(_v_step_half_rho)),
    ("v_ignores_S", lambda: pins.check_v_step(_v_step_ignores_S)),
    ("u_no_rho", lambda: pins.check_u_step_exact(_u_exact_no_rho, O.objective)),
    ("u_ignores_S", lambda: pins.check_u_step_exact(_u_exact_ignores_S, O.objective)),
    ("grad_no_share", lambda: pins.check_grad_U_local(_grad_no_share, O.local_objective)),
    ("grad_sign", lambda: pins.check_grad_U_local(_grad_wrong_sign, O.local_objective)),
    ("huber_offset", lambda: pins.check_huber(_huber_no_offset)),
    ("local_share", lambda: pins.check_local_split(_local_no_share, O.objective)),
    ("fedavg_weights", lambda: pins.check_fedavg_is_global_gd(
        _weighted_fedavg_iteration, O.objective, O.s_step, O.v_step)),
    ("fedavg_fn_no_share", lambda: pins.check_u_step_fedavg(_fedavg_no_share,
                                                            O.local_objective)),
    ("fedavg_fn_weighted", lambda: pins.check_u_step_fedavg(_fedavg_weighted,
                                                            O.local_objective)),
    ("fedavg_fn_no_share_gd", lambda: pins.check_u_step_fedavg_is_global_gd(
        _fedavg_no_share, O.objective)),
    ("local_round_U", lambda: pins.check_local_steps(
        _local_steps_round_U, O.local_objective, O.s_step, O.v_step, K=3)),
    ("local_avg_each_step", lambda: pins.check_local_steps(
        _local_steps_average_each_step, O.local_objective, O.s_step, O.v_step, K=3)),
    ("local_avg_each_step_indep", lambda: pins.check_clients_independent(
        _local_steps_average_each_step, K=3)),
    ("local_stale_V", lambda: pins.check_local_steps(
        _local_steps_stale_V, O.local_objective, O.s_step, O.v_step, K=3)),
    ("sv_one_factor", lambda: _check_sv(_sv_one_factor)),
    ("sv_error_first", lambda: _check_sv_err(_sv_error_first)),
]


@pytest.mark.parametrize("name,run", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_is_caught(name, run):
    assert run() > 1e-4
