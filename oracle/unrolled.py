"""FP64 oracle of the learned unrolled DCF network and of its adjoint.

Test infrastructure only (see the package docstring).

Network (the learned form of K rounds of Algorithm 1 with the exact consensus
U-step; parameters per step k):
    lambda_k = lambda * exp(a_k),  rho_k = rho * exp(b_k),  alpha_k = c_k
    R   = M - U V^T,  C = clamp(R, -lambda_k, lambda_k),  X = U V^T + C
                                            (S-step of §2.2 eq. optS: X = M - S)
    G   = U^T U + rho_k I,  W = U G^{-1},  V' = X^T W
                                            (V-step, App. B eq. condition1)
    P   = X V',  H = V'^T V' + rho_k I,  U* = P H^{-1}
                                            (exact consensus U-step)
    U'  = U + alpha_k (U* - U)              (relaxation; alpha = 1 is the plain step)
At a = b = 0, c = 1 the network is K plain iterations (pinned against dcf_run).

Loss (factor space): sum_{k=1..K} w_k ||U_k V_k^T - L*||_F^2 / ||L*||_F^2 with
L* = A B^T and increasing weights w_k = 2k / (K (K + 1)).

The adjoint below is the hand-derived reverse mode of one step, applied from
the last step to the first with every step recomputed from its checkpoint
(U_k, V_k).  It is pinned by central finite differences of the forward loss.
"""
from __future__ import annotations

import numpy as np

__all__ = ["loss_weights", "unrolled_forward", "unrolled_backward", "step_forward",
           "step_backward", "factor_loss", "factor_loss_grad"]


def _f64(x):
    return np.asarray(x, dtype=np.float64)


def loss_weights(K):
    k = np.arange(1, K + 1, dtype=np.float64)
    return 2.0 * k / (K * (K + 1))


def factor_loss(U, V, A, B):
    """||U V^T - A B^T||_F^2 / ||A B^T||_F^2 through r x r Grams."""
    U, V, A, B = map(_f64, (U, V, A, B))
    a = np.sum((U.T @ U) * (V.T @ V))
    b = np.sum((U.T @ A) * (V.T @ B))
    c = np.sum((A.T @ A) * (B.T @ B))
    return float((a - 2.0 * b + c) / c)


def factor_loss_grad(U, V, A, B):
    """Gradient of factor_loss with respect to U and V."""
    U, V, A, B = map(_f64, (U, V, A, B))
    c = np.sum((A.T @ A) * (B.T @ B))
    gU = 2.0 * (U @ (V.T @ V) - A @ (B.T @ V)) / c
    gV = 2.0 * (V @ (U.T @ U) - B @ (A.T @ U)) / c
    return gU, gV


def step_forward(M, U, V, lam, rho, alpha):
    """One network step; returns (U', V') and the intermediates of the adjoint."""
    M, U, V = map(_f64, (M, U, V))
    r = U.shape[1]
    L = U @ V.T
    R = M - L
    C = np.clip(R, -lam, lam)
    X = L + C
    G = U.T @ U + rho * np.eye(r)
    Ginv = np.linalg.inv(G)
    W = U @ Ginv
    Vn = X.T @ W
    P = X @ Vn
    H = Vn.T @ Vn + rho * np.eye(r)
    Hinv = np.linalg.inv(H)
    Us = P @ Hinv
    Un = U + alpha * (Us - U)
    cache = dict(R=R, X=X, Ginv=Ginv, W=W, Vn=Vn, Hinv=Hinv, Us=Us, U=U, V=V, lam=lam,
                 rho=rho, alpha=alpha)
    return Un, Vn, cache


def step_backward(cache, Ubar_n, Vbar_n):
    """Reverse mode of step_forward: returns (Ubar, Vbar, lam_bar, rho_bar, alpha_bar)."""
    R, X, Ginv, W, Vn = cache["R"], cache["X"], cache["Ginv"], cache["W"], cache["Vn"]
    Hinv, Us, U, V = cache["Hinv"], cache["Us"], cache["U"], cache["V"]
    lam, alpha = cache["lam"], cache["alpha"]
    sym = lambda Z: 0.5 * (Z + Z.T)
    # U' = (1 - alpha) U + alpha U*
    alpha_bar = float(np.sum(Ubar_n * (Us - U)))
    Us_bar = alpha * Ubar_n
    Ubar = (1.0 - alpha) * Ubar_n
    # U* = P H^{-1}
    P_bar = Us_bar @ Hinv
    H_bar = sym(-(Us.T @ Us_bar) @ Hinv)
    rho_bar = float(np.trace(H_bar))
    # H = V'^T V' + rho I
    Vn_bar = Vbar_n + 2.0 * Vn @ H_bar
    # P = X V'
    X_bar = P_bar @ Vn.T
    Vn_bar = Vn_bar + X.T @ P_bar
    # V' = X^T W
    X_bar = X_bar + W @ Vn_bar.T
    W_bar = X @ Vn_bar
    # W = U G^{-1},  G = U^T U + rho I
    Ubar = Ubar + W_bar @ Ginv
    G_bar = sym(-(W.T @ W_bar) @ Ginv)
    Ubar = Ubar + 2.0 * U @ G_bar
    rho_bar += float(np.trace(G_bar))
    # X = U V^T + clamp(M - U V^T, -lam, lam)
    outside = np.abs(R) > lam
    D = np.where(outside, X_bar, 0.0)
    Ubar = Ubar + D @ V
    Vbar = D.T @ U
    lam_bar = float(np.sum(np.where(outside, X_bar * np.sign(R), 0.0)))
    return Ubar, Vbar, lam_bar, rho_bar, alpha_bar


def unrolled_forward(M, U0, V0, A, B, lam, rho, theta, weights=None):
    """theta = (a, b, c) arrays of length K.  Returns (loss, [(U_k, V_k)] k=0..K)."""
    a, b, c = (np.asarray(t, dtype=np.float64) for t in theta)
    K = len(a)
    w = loss_weights(K) if weights is None else np.asarray(weights, np.float64)
    U, V = _f64(U0), _f64(V0)
    traj = [(U, V)]
    loss = 0.0
    for k in range(K):
        U, V, _ = step_forward(M, U, V, lam * np.exp(a[k]), rho * np.exp(b[k]), c[k])
        traj.append((U, V))
        loss += w[k] * factor_loss(U, V, A, B)
    return float(loss), traj


def unrolled_backward(M, traj, A, B, lam, rho, theta, weights=None):
    """Gradient of the loss with respect to (a, b, c), and to (U0, V0)."""
    a, b, c = (np.asarray(t, dtype=np.float64) for t in theta)
    K = len(a)
    w = loss_weights(K) if weights is None else np.asarray(weights, np.float64)
    ga, gb, gc = np.zeros(K), np.zeros(K), np.zeros(K)
    Ubar = np.zeros_like(traj[0][0])
    Vbar = np.zeros_like(traj[0][1])
    for k in range(K - 1, -1, -1):
        Uk1, Vk1 = traj[k + 1]
        gU, gV = factor_loss_grad(Uk1, Vk1, A, B)
        Ubar = Ubar + w[k] * gU
        Vbar = Vbar + w[k] * gV
        lam_k, rho_k = lam * np.exp(a[k]), rho * np.exp(b[k])
        _, _, cache = step_forward(M, traj[k][0], traj[k][1], lam_k, rho_k, c[k])
        Ubar, Vbar, lb, rb, ab = step_backward(cache, Ubar, Vbar)
        ga[k], gb[k], gc[k] = lb * lam_k, rb * rho_k, ab
    return (ga, gb, gc), (Ubar, Vbar)
