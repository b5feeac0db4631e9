"""Pins of the FP64 oracle against what the paper and the mathematics fix."""
import numpy as np
import pytest

import oracle as O
from paper_2207_11669_gb300 import synth
from tests import pins

TOL = 1e-9


def test_s_step_is_l1_prox():
    assert pins.check_s_step(O.s_step) < TOL


def test_soft_threshold_ties_give_zero():
    lam = 0.25
    R = np.array([lam, -lam, 0.0, lam * (1 + 1e-12), -3.0])
    S = O.soft_threshold(R, lam)
    assert S[0] == 0.0 and S[1] == 0.0 and S[2] == 0.0
    assert S[3] > 0.0 and S[4] == -3.0 + lam


def test_huber_is_min_over_S():
    assert pins.check_huber(O.huber) < 1e-8


def test_huber_form_equals_objective_at_optimal_S():
    """§2.2 eq. cancelV: substituting the optimal S turns the §1 objective into
    the Huber form."""
    p = pins.small_problem(11)
    M, U, V, rho, lam = p["M"], p["U"], p["V"], p["rho"], p["lam"]
    S = O.s_step(M, U, V, lam)
    a = O.objective(M, U, V, S, rho, lam)
    b = O.objective_huber(M, U, V, rho, lam)
    assert abs(a - b) <= 1e-12 * abs(a)


def test_v_step_is_ridge_regression():
    assert pins.check_v_step(O.v_step) < 1e-10


def test_u_step_exact_zero_gradient():
    assert pins.check_u_step_exact(O.u_step_exact, O.objective) < 1e-6


def test_local_objectives_sum_to_objective():
    assert pins.check_local_split(O.local_objective, O.objective) < 1e-13


def test_grad_U_local_matches_finite_differences():
    assert pins.check_grad_U_local(O.grad_U_local, O.local_objective) < 1e-6


def test_fedavg_k1_is_one_global_gradient_step():
    assert pins.check_fedavg_is_global_gd(O.dcf_iteration, O.objective, O.s_step,
                                          O.v_step) < 1e-7


def test_u_step_fedavg_matches_finite_difference_client_steps():
    assert pins.check_u_step_fedavg(O.u_step_fedavg, O.local_objective) < 1e-7


def test_u_step_fedavg_k1_is_one_global_gradient_step():
    assert pins.check_u_step_fedavg_is_global_gd(O.u_step_fedavg, O.objective) < 1e-7


@pytest.mark.parametrize("K", [1, 2, 3])
def test_local_steps_follow_algorithm_1(K):
    assert pins.check_local_steps(O.dcf_iteration, O.local_objective, O.s_step,
                                  O.v_step, K=K) < 1e-7


@pytest.mark.parametrize("K", [2, 5])
def test_local_steps_clients_meet_only_in_the_average(K):
    assert pins.check_clients_independent(O.dcf_iteration, K=K) < 1e-12


def test_local_steps_k1_equals_fedavg_function():
    """The K = 1 branch of the round and u_step_fedavg on the round's own
    (V_t, S_t) give the same U."""
    p = pins.small_problem(12)
    M, U, V, rho, lam, n_i = p["M"], p["U"], p["V"], p["rho"], p["lam"], p["n_i"]
    U1, V1, S1 = O.dcf_iteration(M, n_i, U, V, rho, lam, u_mode=1, eta=0.02)
    off = O.block_offsets(n_i)
    E = len(n_i)
    U2 = O.u_step_fedavg([M[:, off[i]:off[i + 1]] for i in range(E)],
                         [S1[:, off[i]:off[i + 1]] for i in range(E)],
                         [V1[off[i]:off[i + 1]] for i in range(E)],
                         U, rho, 0.02, n_i, M.shape[1])
    assert np.max(np.abs(U1 - U2)) < 1e-13


def test_ridge_solve_matches_dense_solve():
    g = np.random.default_rng(3)
    A = g.standard_normal((6, 6))
    G = A @ A.T + 0.1 * np.eye(6)
    B = g.standard_normal((10, 6))
    X = O.ridge_solve(G, B)
    assert np.max(np.abs(X @ G - B)) < 1e-10


@pytest.mark.parametrize("u_mode", [0, 1])
def test_objective_monotone_in_exact_mode(u_mode):
    """Exact mode: S, V and U are each exact block minimisers, so the §1
    objective never rises inside an iteration.  (Gradient mode with a small
    step also descends here.)"""
    p = pins.small_problem(21, m=12, n=15, r=3, E=3)
    M, U, V, rho, lam, n_i = p["M"], p["U"], p["V"], p["rho"], p["lam"], p["n_i"]
    S = O.s_step(M, U, V, lam)
    F_prev = O.objective(M, U, V, np.zeros_like(M), rho, lam)
    for t in range(15):
        S = O.s_step(M, U, V, lam)
        F1 = O.objective(M, U, V, S, rho, lam)
        V = O.v_step(M, S, U, rho)
        F2 = O.objective(M, U, V, S, rho, lam)
        off = O.block_offsets(n_i)
        if u_mode == 0:
            Ms = [M[:, off[i]:off[i + 1]] for i in range(len(n_i))]
            Ss = [S[:, off[i]:off[i + 1]] for i in range(len(n_i))]
            Vs = [V[off[i]:off[i + 1]] for i in range(len(n_i))]
            U = O.u_step_exact(Ms, Ss, Vs, rho)
        else:
            U = O.u_step_fedavg([M[:, off[i]:off[i + 1]] for i in range(len(n_i))],
                                [S[:, off[i]:off[i + 1]] for i in range(len(n_i))],
                                [V[off[i]:off[i + 1]] for i in range(len(n_i))],
                                U, rho, 1e-3, n_i, M.shape[1])
        F3 = O.objective(M, U, V, S, rho, lam)
        tol = 1e-10 * abs(F_prev)
        assert F1 <= F_prev + tol and F2 <= F1 + tol and F3 <= F2 + tol
        F_prev = F3


def test_iteration_order_matches_block_updates():
    """dcf_iteration performs S(U_{t-1},V_{t-1}) -> V(U_{t-1},S_t) -> U(V_t,S_t)."""
    p = pins.small_problem(31)
    M, U, V, rho, lam, n_i = p["M"], p["U"], p["V"], p["rho"], p["lam"], p["n_i"]
    U1, V1, S1 = O.dcf_iteration(M, n_i, U, V, rho, lam)
    S = O.s_step(M, U, V, lam)
    Vn = O.v_step(M, S, U, rho)
    Un = O.u_step_exact([M], [S], [Vn], rho)
    assert np.max(np.abs(S1 - S)) < 1e-12
    assert np.max(np.abs(V1 - Vn)) < 1e-10
    assert np.max(np.abs(U1 - Un)) < 1e-10


def test_exact_mode_is_partition_invariant():
    """E = 1 (centralised alternating minimisation, CF-PCA of §4.2) and E = 4
    clients give the same iterates in exact-consensus mode."""
    p = pins.small_problem(41, m=10, n=16, r=3, E=4)
    M, U, V, rho, lam = p["M"], p["U"], p["V"], p["rho"], p["lam"]
    a = O.dcf_run(M, [16], U, V, rho, lam, 8)
    b = O.dcf_run(M, [3, 5, 4, 4], U, V, rho, lam, 8)
    for x, y in zip(a[:3], b[:3]):
        assert np.max(np.abs(x - y)) < 1e-9


def test_zero_padding_of_rank_is_exact():
    """Extra all-zero columns of U and V stay exactly zero and leave the other
    columns unchanged (the r x r solves are block diagonal)."""
    p = pins.small_problem(51)
    M, U, V, rho, lam, n_i = p["M"], p["U"], p["V"], p["rho"], p["lam"], p["n_i"]
    Up = np.hstack([U, np.zeros((U.shape[0], 2))])
    Vp = np.hstack([V, np.zeros((V.shape[0], 2))])
    a = O.dcf_run(M, n_i, U, V, rho, lam, 5)
    b = O.dcf_run(M, n_i, Up, Vp, rho, lam, 5)
    assert np.all(b[0][:, 3:] == 0) and np.all(b[1][:, 3:] == 0)
    assert np.max(np.abs(a[0] - b[0][:, :3])) < 1e-10
    assert np.max(np.abs(a[1] - b[1][:, :3])) < 1e-10


def test_factor_metrics_match_dense():
    g = np.random.default_rng(61)
    U, V = g.standard_normal((20, 3)), g.standard_normal((30, 3))
    Up, Vp = U + 0.1 * g.standard_normal(U.shape), V + 0.1 * g.standard_normal(V.shape)
    A, B = g.standard_normal((20, 2)), g.standard_normal((30, 2))
    L, Lp, L0 = U @ V.T, Up @ Vp.T, A @ B.T
    d = np.linalg.norm(L - Lp) / np.linalg.norm(L)
    assert abs(O.factor_delta_rel(U, V, Up, Vp) - d) < 1e-10
    e = np.linalg.norm(L - L0) / np.linalg.norm(L0)
    assert abs(O.rel_err_L(U, V, A, B) - e) < 1e-10


def test_paper_err_definition():
    L0 = np.ones((2, 2))
    S0 = np.zeros((2, 2))
    assert O.paper_err(L0, S0, L0, S0) == 0.0
    assert abs(O.paper_err(2 * L0, S0, L0, S0) - 1.0) < 1e-15


def test_inner_sweeps_reach_joint_VS_argmin():
    """Repeating the S -> V sweep with U fixed converges to the unique joint
    minimiser of Algorithm 1 eq. VS_arg; checked against a quasi-Newton
    minimisation of the Huber form h(V) of §2.2 eq. cancelV."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    p = pins.small_problem(71, m=8, n=6, r=2, E=1, lam=0.4, rho=0.3)
    M, U, V, rho, lam = p["M"], p["U"], p["V"], p["rho"], p["lam"]
    for _ in range(3000):
        S = O.s_step(M, U, V, lam)
        V = O.v_step(M, S, U, rho)

    def h(v):
        Vv = v.reshape(V.shape)
        R = M - U @ Vv.T
        a = np.abs(R)
        H = np.where(a <= lam, 0.5 * R * R, lam * a - 0.5 * lam * lam)
        dH = np.clip(R, -lam, lam)
        f = 0.5 * rho * np.sum(Vv * Vv) + np.sum(H)
        g = rho * Vv - dH.T @ U
        return f, g.ravel()

    res = scipy_opt.minimize(h, np.zeros(V.size), jac=True, method="L-BFGS-B",
                             options=dict(gtol=1e-14, ftol=1e-16, maxiter=10000))
    assert np.max(np.abs(res.x.reshape(V.shape) - V)) < 1e-6


def test_planted_recovery_small():
    """A tiny well-conditioned planted instance (m = n = 40, rank 2, density
    0.05; §4.1 generator) is recovered: relative L error below 1e-3.

    The minimiser of the §1 objective is biased by lambda (on the support the
    optimal S is S* shrunk by lambda), so the recovery error must also shrink
    as lambda does; lambda = 0.01 is small enough for 1e-3 here."""
    inst = synth.make_instance(40, 40, 2, seed=5, density=0.05, amp=10.0,
                               factor_std=1.0, E=4)
    U0 = synth.gaussian_u0(40, 2, 5).astype(np.float64)
    rho = 1e-2
    V0 = O.init_v0(inst.M, U0, rho)
    L0 = inst.A.astype(np.float64) @ inst.B.T.astype(np.float64)
    errs = []
    for lam in (0.08, 0.04, 0.01):
        U, V, S, it, d = O.dcf_solve(inst.M, inst.n_i, U0, V0, rho, lam, 6000, 1e-13)
        errs.append(O.rel_err_L(U, V, inst.A, inst.B))
        assert d <= 1e-13
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-3
    assert O.paper_err(U @ V.T, S, L0, inst.S_star) < 1e-5


def test_init_v0_is_v_step_with_zero_S():
    p = pins.small_problem(81)
    M, U, rho = p["M"], p["U"], p["rho"]
    V0 = O.init_v0(M, U, rho)
    G = U.T @ U + rho * np.eye(U.shape[1])
    assert np.max(np.abs(G @ V0.T - U.T @ M)) < 1e-10


def test_singular_values_factored_match_dense_svd():
    """sigma(X Y^T) from the factors equals numpy's SVD of the dense product,
    also for a rank-deficient product (a zero column pair) and p > rank."""
    g = np.random.default_rng(91)
    X, Y = g.standard_normal((30, 6)), g.standard_normal((45, 6))
    X[:, 5] = 0.0                               # rank 5
    s = O.singular_values_factored(X, Y)
    d = np.linalg.svd(X @ Y.T, compute_uv=False)[:6]
    assert np.max(np.abs(s - d)) < 1e-12 * d[0]
    assert s[5] < 1e-12 * d[0]


def test_singular_values_factored_gauge_invariant():
    """L = X Y^T = (X T)(Y T^{-T})^T for any invertible T: the same values."""
    g = np.random.default_rng(92)
    X, Y = g.standard_normal((20, 4)), g.standard_normal((25, 4))
    T = g.standard_normal((4, 4)) + 3 * np.eye(4)
    a = O.singular_values_factored(X, Y)
    b = O.singular_values_factored(X @ T, Y @ np.linalg.inv(T).T)
    assert np.max(np.abs(a - b)) < 1e-11 * a[0]


def test_singular_value_error_definition():
    """Table 1's quantity on hand-made lists: the largest gap over all indices
    (missing values are 0), divided by the k-th value of L0."""
    assert O.singular_value_error([3.0, 2.0, 0.5], [3.0, 2.0], 2) == 0.25
    assert O.singular_value_error([3.1, 1.8], [3.0, 2.0, 1.0], 3) == 1.0
    assert O.singular_value_error([2.0, 1.0], [2.0, 1.0], 2) == 0.0
