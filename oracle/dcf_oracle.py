"""FP64 oracle of one DCF-PCA iteration and of the quantities built on it.

Test infrastructure only (see the package docstring).  Every function
restates the paper ("Distributed Robust Principal Component Analysis",
arXiv 2207.11669) in float64 numpy, in the paper's order and notation:

  objective        §1, eq. ``noncovex_problem``:
                   1/2||U V^T + S - M||_F^2 + rho/2 (||U||_F^2 + ||V||_F^2) + lambda ||S||_1
  client split     §2.1 (M = [M_1 ... M_E], M_i in R^{m x n_i});
                   §2.2 local objectives L~_i and L_i (with the n_i rho/(2n)||U||^2 share)
  S-step           §2.2, eq. ``optS`` (soft threshold of M_i - U V_i^T)
  V-step           App. B, eq. ``condition1``: (U^T U + rho I) V_i^T = U^T (M_i - S_i)
  U-step           exact consensus: the zero of sum_i grad_U L_i (App. B, Lemma 2
                   proof) -> U (sum_i V_i^T V_i + rho I) = sum_i (M_i - S_i) V_i;
                   FedAvg gradient mode: Algorithm 1, eqs. ``U_local`` and ``U_agg``
  Huber form       §2.2 eq. ``cancelV`` and App. A.2
  error metric     §4.1 "Evaluation Metric" (squared, L and S together)
  singular values  §4.2 "Upper-bound rank recovery", Table 1: the relative
                   singular-value error max_i |sigma_i(L) - sigma_i(L0)| / sigma_r(L0)

Readings of the paper taken here:
  * one alternating S -> V sweep per iteration solves the (V,S) subproblem of
    Algorithm 1 eq. ``VS_arg`` (inner = 1); S uses (U_{t-1}, V_{t-1}), V uses
    (U_{t-1}, S_t), U uses (V_t, S_t);
  * exact-consensus U-step by default, Algorithm 1's gradient step as
    ``u_mode=1`` with eta_t = eta0 / sqrt(t + 1);
  * ties |R| == lambda give S = 0;
  * the FedAvg average is unweighted even for uneven n_i (eq. ``U_agg``).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "soft_threshold", "huber", "objective", "objective_huber", "local_objective",
    "grad_U_local", "s_step", "v_step", "u_step_exact", "u_step_fedavg",
    "ridge_solve", "init_v0", "dcf_iteration", "dcf_run", "dcf_solve",
    "block_offsets", "factor_delta_rel", "rel_err_L", "paper_err",
    "singular_values_factored", "singular_value_error",
]


def _f64(x):
    return np.asarray(x, dtype=np.float64)


def block_offsets(n_i):
    """Column offsets c_i of the blocks M_i = M[:, c_i:c_i+n_i] (§2.1)."""
    n_i = np.asarray(n_i, dtype=np.int64)
    return np.concatenate([[0], np.cumsum(n_i)]).astype(np.int64)


# ---------------------------------------------------------------------------
# Elementwise pieces
# ---------------------------------------------------------------------------
def soft_threshold(R, lam):
    """S = sign(R) * max(|R| - lambda, 0)  (§2.2, eq. ``optS``).

    Entries with |R| <= lambda (ties included) give exactly 0.
    """
    R = _f64(R)
    mag = np.abs(R) - lam
    return np.where(mag > 0.0, np.sign(R) * mag, 0.0)


def huber(x, lam):
    """Elementwise Huber loss H_lambda (App. A.2), summed over all entries.

    x^2/2 on [-lambda, lambda], lambda|x| - lambda^2/2 outside.
    """
    x = _f64(x)
    a = np.abs(x)
    return float(np.sum(np.where(a <= lam, 0.5 * x * x, lam * a - 0.5 * lam * lam)))


# ---------------------------------------------------------------------------
# Objectives
# ---------------------------------------------------------------------------
def objective(M, U, V, S, rho, lam):
    """Brute-force objective of §1 eq. ``noncovex_problem``."""
    M, U, V, S = map(_f64, (M, U, V, S))
    D = U @ V.T + S - M
    return float(0.5 * np.sum(D * D) + 0.5 * rho * (np.sum(U * U) + np.sum(V * V))
                 + lam * np.sum(np.abs(S)))


def objective_huber(M, U, V, rho, lam):
    """Objective minimised over S: sum H_lambda(M - U V^T) + rho/2(||U||^2+||V||^2)
    (§2.2 eq. ``cancelV``, App. A.2)."""
    M, U, V = map(_f64, (M, U, V))
    return huber(M - U @ V.T, lam) + 0.5 * rho * (np.sum(U * U) + np.sum(V * V))


def local_objective(M_i, U, V_i, S_i, rho, lam, n_i, n):
    """L_i(U, V_i, S_i) of §2.2: L~_i + (n_i rho / 2n) ||U||_F^2."""
    M_i, U, V_i, S_i = map(_f64, (M_i, U, V_i, S_i))
    D = U @ V_i.T + S_i - M_i
    return float(0.5 * np.sum(D * D) + 0.5 * rho * np.sum(V_i * V_i)
                 + lam * np.sum(np.abs(S_i)) + 0.5 * rho * (n_i / n) * np.sum(U * U))


def grad_U_local(M_i, U, V_i, S_i, rho, n_i, n):
    """grad_U L_i = rho (n_i/n) U + (U V_i^T + S_i - M_i) V_i  (App. B, Lemma 2 proof)."""
    M_i, U, V_i, S_i = map(_f64, (M_i, U, V_i, S_i))
    return rho * (n_i / n) * U + (U @ V_i.T + S_i - M_i) @ V_i


# ---------------------------------------------------------------------------
# Block updates
# ---------------------------------------------------------------------------
def ridge_solve(G, B):
    """Solve X G = B for symmetric positive definite G (r x r) by Cholesky.

    G = L L^T; X = B G^{-1} is computed as two triangular solves on B^T.
    """
    G = _f64(G)
    B = _f64(B)
    L = np.linalg.cholesky(G)
    Y = np.linalg.solve(L, B.T)          # L Y = B^T
    Xt = np.linalg.solve(L.T, Y)         # L^T X^T = Y
    return Xt.T


def s_step(M_i, U, V_i, lam):
    """S_i = soft(M_i - U V_i^T, lambda)  (§2.2 eq. ``optS``)."""
    M_i, U, V_i = map(_f64, (M_i, U, V_i))
    return soft_threshold(M_i - U @ V_i.T, lam)


def v_step(M_i, S_i, U, rho):
    """V_i with (U^T U + rho I) V_i^T = U^T (M_i - S_i)  (App. B eq. ``condition1``;
    the same closed form as the commented V-update of §2.2)."""
    M_i, S_i, U = map(_f64, (M_i, S_i, U))
    r = U.shape[1]
    G = U.T @ U + rho * np.eye(r)
    # V_i = (M_i - S_i)^T U G^{-1}  (G symmetric)
    return ridge_solve(G, (M_i - S_i).T @ U)


def u_step_exact(Ms, Ss, Vs, rho):
    """Exact consensus U-step: U (sum_i V_i^T V_i + rho I) = sum_i (M_i - S_i) V_i.

    This is the zero of sum_i grad_U L_i with sum_i n_i/n = 1 (App. B,
    Lemma 2 proof), i.e. the minimiser over U of the objective of §1 with
    every (V_i, S_i) fixed.
    """
    r = Vs[0].shape[1]
    P = sum(_f64(M) @ _f64(V) - _f64(S) @ _f64(V) for M, S, V in zip(Ms, Ss, Vs))
    Q = sum(_f64(V).T @ _f64(V) for V in Vs)
    return ridge_solve(Q + rho * np.eye(r), P)


def u_step_fedavg(Ms, Ss, Vs, U, rho, eta, n_i, n):
    """Algorithm 1: U_i = U - eta grad_U L_i(U, V_i, S_i) (eq. ``U_local``),
    then U <- (1/E) sum_i U_i (eq. ``U_agg``)."""
    E = len(Ms)
    U = _f64(U)
    acc = np.zeros_like(U)
    for M, S, V, ni in zip(Ms, Ss, Vs, n_i):
        acc += U - eta * grad_U_local(M, U, V, S, rho, ni, n)
    return acc / E


def init_v0(M, U0, rho):
    """V0 from one S = 0 sweep: V0 = M^T U0 (U0^T U0 + rho I)^{-1}.

    Algorithm 1 leaves the initial V_i unspecified ("randomly"); this reading
    takes the V-step of App. B eq. ``condition1`` with S = 0.
    """
    M = _f64(M)
    return v_step(M, np.zeros_like(M), U0, rho)


# ---------------------------------------------------------------------------
# One iteration and runs
# ---------------------------------------------------------------------------
def dcf_iteration(M, n_i, U, V, rho, lam, *, u_mode=0, eta=0.0, local_steps=1):
    """One communication round t of DCF-PCA over the E client blocks.

    Returns (U_t, V_t, S_t) where S_t = soft(M - U_{t-1} V_{t-1}^T) is the S
    that the round computed (§2.2 eq. ``optS``), V_t the V-step on S_t with
    U_{t-1}, and U_t the consensus update.

    u_mode 0: exact consensus (see :func:`u_step_exact`); local_steps must be 1.
    u_mode 1: Algorithm 1 with K = local_steps local steps per client:
              for k < K: S_i <- soft(M_i - U_i V_i^T); V_i <- V-step(U_i, S_i);
                         U_i <- U_i - eta grad_U L_i(U_i, V_i, S_i);
              then U_t = (1/E) sum_i U_i.
    """
    M = _f64(M)
    U = _f64(U)
    V = _f64(V)
    off = block_offsets(n_i)
    E = len(n_i)
    n = int(off[-1])
    Ms = [M[:, off[i]:off[i + 1]] for i in range(E)]
    V_new = np.empty_like(V)
    S_new = np.empty_like(M)
    if u_mode == 0:
        if local_steps != 1:
            raise ValueError("exact consensus takes one local step")
        Ss, Vs = [], []
        for i in range(E):                                   # each client i (concurrently)
            S_i = s_step(Ms[i], U, V[off[i]:off[i + 1]], lam)
            V_i = v_step(Ms[i], S_i, U, rho)
            Ss.append(S_i)
            Vs.append(V_i)
        U_new = u_step_exact(Ms, Ss, Vs, rho)               # server consensus
    else:
        Us = []
        Ss, Vs = [], []
        for i in range(E):
            U_i = U.copy()
            V_i = V[off[i]:off[i + 1]].copy()
            for _ in range(local_steps):
                S_i = s_step(Ms[i], U_i, V_i, lam)
                V_i = v_step(Ms[i], S_i, U_i, rho)
                U_i = U_i - eta * grad_U_local(Ms[i], U_i, V_i, S_i, rho, int(n_i[i]), n)
            Us.append(U_i)
            Ss.append(S_i)
            Vs.append(V_i)
        U_new = sum(Us) / E                                  # eq. U_agg
    for i in range(E):
        V_new[off[i]:off[i + 1]] = Vs[i]
        S_new[:, off[i]:off[i + 1]] = Ss[i]
    return U_new, V_new, S_new


def dcf_run(M, n_i, U0, V0, rho, lam, iters, *, u_mode=0, eta0=0.0, local_steps=1,
            callback=None):
    """``iters`` rounds from (U0, V0); returns (U, V, S, U_prev, V_prev)."""
    U, V = _f64(U0), _f64(V0)
    U_prev, V_prev, S = U, V, None
    for t in range(iters):
        eta = eta0 / np.sqrt(t + 1.0)
        U_prev, V_prev = U, V
        U, V, S = dcf_iteration(M, n_i, U, V, rho, lam, u_mode=u_mode, eta=eta,
                                local_steps=local_steps)
        if callback is not None:
            callback(t, U, V, S)
    return U, V, S, U_prev, V_prev


def factor_delta_rel(U, V, U_prev, V_prev):
    """||U V^T - U_p V_p^T||_F / ||U V^T||_F evaluated through r x r Grams."""
    U, V, U_prev, V_prev = map(_f64, (U, V, U_prev, V_prev))
    a = np.sum((U.T @ U) * (V.T @ V))
    b = np.sum((U.T @ U_prev) * (V.T @ V_prev))
    c = np.sum((U_prev.T @ U_prev) * (V_prev.T @ V_prev))
    d2 = max(a - 2.0 * b + c, 0.0)
    return float(np.sqrt(d2 / a)) if a > 0 else float("inf")


def dcf_solve(M, n_i, U0, V0, rho, lam, max_iter, tol, *, u_mode=0, eta0=0.0,
              local_steps=1):
    """Run rounds until ||L_t - L_{t-1}||_F / ||L_t||_F <= tol or max_iter.

    The paper runs a fixed number of rounds T; the stopping rule is this
    build's reading.  Returns (U, V, S, iterations, last relative change).
    """
    U, V = _f64(U0), _f64(V0)
    S = None
    d = float("inf")
    for t in range(max_iter):
        eta = eta0 / np.sqrt(t + 1.0)
        U_new, V_new, S = dcf_iteration(M, n_i, U, V, rho, lam, u_mode=u_mode, eta=eta,
                                        local_steps=local_steps)
        d = factor_delta_rel(U_new, V_new, U, V)
        U, V = U_new, V_new
        if d <= tol:
            return U, V, S, t + 1, d
    return U, V, S, max_iter, d


# ---------------------------------------------------------------------------
# Metrics
# ---------------------------------------------------------------------------
def rel_err_L(U, V, A, B):
    """||U V^T - A B^T||_F / ||A B^T||_F, evaluated through r x r Grams."""
    U, V, A, B = map(_f64, (U, V, A, B))
    a = np.sum((U.T @ U) * (V.T @ V))
    b = np.sum((U.T @ A) * (V.T @ B))
    c = np.sum((A.T @ A) * (B.T @ B))
    return float(np.sqrt(max(a - 2.0 * b + c, 0.0) / c))


def paper_err(L, S, L0, S0):
    """(||L - L0||^2 + ||S - S0||^2) / (||L0||^2 + ||S0||^2)  (§4.1, squared)."""
    L, S, L0, S0 = map(_f64, (L, S, L0, S0))
    return float((np.sum((L - L0) ** 2) + np.sum((S - S0) ** 2))
                 / (np.sum(L0 ** 2) + np.sum(S0 ** 2)))


def singular_values_factored(X, Y):
    """Singular values of L = X Y^T (X: N1 x p, Y: N2 x p), descending, from the
    factors alone: X = Q_x R_x and Y = Q_y R_y (Householder QR), so that
    L = Q_x (R_x R_y^T) Q_y^T with orthonormal Q's and the singular values of L
    are those of the p x p matrix R_x R_y^T (an SVD)."""
    X, Y = _f64(X), _f64(Y)
    Rx = np.linalg.qr(X, mode="r")
    Ry = np.linalg.qr(Y, mode="r")
    return np.linalg.svd(Rx @ Ry.T, compute_uv=False)


def singular_value_error(sigma, sigma0, k):
    """Table 1 of §4.2: max_i |sigma_i(L) - sigma_i(L0)| / sigma_k(L0), with k the
    rank of L0, over every index either list has (a missing value is 0)."""
    sigma = np.sort(_f64(sigma))[::-1]
    sigma0 = np.sort(_f64(sigma0))[::-1]
    n = max(len(sigma), len(sigma0))
    a = np.zeros(n)
    b = np.zeros(n)
    a[:len(sigma)] = sigma
    b[:len(sigma0)] = sigma0
    return float(np.max(np.abs(a - b)) / sigma0[k - 1])
