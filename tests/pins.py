"""Checks that pin the oracle to facts the paper and the mathematics fix.

Each ``check_*`` takes the oracle function(s) it checks and returns a
residual (0 when the fact holds).  The pins never call the function they
check to produce the expected value: they evaluate a different route to
the same fact (an optimality condition, a brute-force minimisation, a
finite-difference gradient of the brute-force objective, a Householder QR
least-squares solve).  ``test_oracle_mutations.py`` plants mistakes in the
oracle and asserts that these residuals then become large.
"""
from __future__ import annotations

import numpy as np


def rng(seed):
    return np.random.default_rng(seed)


def small_problem(seed=0, m=9, n=11, r=3, E=3, lam=0.3, rho=0.05):
    g = rng(seed)
    M = g.standard_normal((m, n)) + np.where(g.random((m, n)) < 0.1,
                                             g.uniform(-4, 4, (m, n)), 0.0)
    U = g.standard_normal((m, r))
    V = g.standard_normal((n, r))
    base = n // E
    n_i = np.full(E, base)
    n_i[: n - base * E] += 1
    return dict(M=M, U=U, V=V, n_i=n_i, lam=lam, rho=rho, r=r)


# --- S-step: the prox of lambda ||.||_1 ---------------------------------------
def check_s_step(s_step, seed=1):
    """Subgradient conditions of min_S 1/2||R - S||^2 + lambda ||S||_1 entrywise,
    and the minimum located by brute force on a fine grid."""
    p = small_problem(seed)
    M, U, V, lam = p["M"], p["U"], p["V"], p["lam"]
    R = M - U @ V.T
    S = s_step(M, U, V, lam)
    res = 0.0
    nz = S != 0
    # S != 0  =>  R - S = lambda sign(S)
    res = max(res, float(np.max(np.abs((R - S)[nz] - lam * np.sign(S[nz])), initial=0.0)))
    # S == 0  =>  |R| <= lambda
    res = max(res, float(np.max(np.abs(R[~nz]) - lam, initial=-1.0)))
    # brute force on a grid around R for a few entries
    for (a, j) in [(0, 0), (1, 3), (4, 5), (8, 10)]:
        grid = np.linspace(-8, 8, 160001)
        f = 0.5 * (R[a, j] - grid) ** 2 + lam * np.abs(grid)
        res = max(res, abs(grid[np.argmin(f)] - S[a, j]) - 1e-4)
    return max(res, 0.0)


# --- Huber identity -----------------------------------------------------------
def check_huber(huber, seed=2):
    """min_s 1/2 (x - s)^2 + lambda |s| = H_lambda(x), by brute force per entry,
    plus H's defining values: H(0)=0, continuity and slope lambda outside."""
    g = rng(seed)
    lam = 0.7
    xs = np.concatenate([g.uniform(-3, 3, 25), [0.0, lam, -lam, 2 * lam]])
    grid = np.linspace(-6, 6, 240001)
    res = 0.0
    for x in xs:
        brute = np.min(0.5 * (x - grid) ** 2 + lam * np.abs(grid))
        res = max(res, abs(huber(np.array([x]), lam) - brute))
    res = max(res, abs(huber(np.array([0.0]), lam)))
    # slope lambda for |x| > lambda
    res = max(res, abs((huber(np.array([3.0]), lam) - huber(np.array([2.0]), lam)) - lam))
    return res


# --- V-step: ridge regression ---------------------------------------------------
def check_v_step(v_step, seed=3):
    """V-step against an augmented least-squares solve by Householder QR:
    min_v ||U v - x||^2 + rho ||v||^2 for every column x of M - S."""
    p = small_problem(seed)
    M, U, rho = p["M"], p["U"], p["rho"]
    g = rng(seed + 100)
    S = np.where(g.random(M.shape) < 0.2, g.standard_normal(M.shape), 0.0)
    V = v_step(M, S, U, rho)
    r = U.shape[1]
    Aug = np.vstack([U, np.sqrt(rho) * np.eye(r)])
    Qm, Rm = np.linalg.qr(Aug)
    X = M - S
    res = 0.0
    for j in range(M.shape[1]):
        rhs = np.concatenate([X[:, j], np.zeros(r)])
        v = np.linalg.solve(Rm, Qm.T @ rhs)
        res = max(res, float(np.max(np.abs(v - V[j]))))
    # App. B (Lemma 4 proof): rho V = Lambda^T U with Lambda = M - U V^T - S
    Lam = M - U @ V.T - S
    res = max(res, float(np.max(np.abs(rho * V - Lam.T @ U))))
    return res


# --- U-step (exact consensus): zero gradient of the brute-force objective -------------
def fd_grad(f, X, h=1e-6):
    G = np.zeros_like(X)
    for idx in np.ndindex(X.shape):
        Xp = X.copy()
        Xm = X.copy()
        Xp[idx] += h
        Xm[idx] -= h
        G[idx] = (f(Xp) - f(Xm)) / (2 * h)
    return G


def check_u_step_exact(u_step_exact, objective, seed=4):
    """The exact consensus U minimises the §1 objective over U with every
    (V_i, S_i) fixed: its finite-difference gradient vanishes, and it equals
    the QR least-squares solution of [V; sqrt(rho) I] U^T = [(M - S)^T; 0]."""
    p = small_problem(seed)
    M, V, rho, lam, n_i = p["M"], p["V"], p["rho"], p["lam"], p["n_i"]
    g = rng(seed + 7)
    S = np.where(g.random(M.shape) < 0.2, g.standard_normal(M.shape), 0.0)
    off = np.concatenate([[0], np.cumsum(n_i)])
    Ms = [M[:, off[i]:off[i + 1]] for i in range(len(n_i))]
    Ss = [S[:, off[i]:off[i + 1]] for i in range(len(n_i))]
    Vs = [V[off[i]:off[i + 1]] for i in range(len(n_i))]
    U = u_step_exact(Ms, Ss, Vs, rho)
    G = fd_grad(lambda X: objective(M, X, V, S, rho, lam), U)
    res = float(np.max(np.abs(G)) / max(1.0, np.max(np.abs(U))))
    r = V.shape[1]
    Aug = np.vstack([V, np.sqrt(rho) * np.eye(r)])
    Qm, Rm = np.linalg.qr(Aug)
    rhs = np.vstack([(M - S).T, np.zeros((r, M.shape[0]))])
    Ut = np.linalg.solve(Rm, Qm.T @ rhs)
    res = max(res, float(np.max(np.abs(Ut.T - U))))
    return res


# --- local objectives and their gradient ------------------------------------------------
def check_local_split(local_objective, objective, seed=5):
    """sum_i L_i(U, V_i, S_i) equals the §1 objective (the separability of §2.2)."""
    p = small_problem(seed)
    M, U, V, rho, lam, n_i = p["M"], p["U"], p["V"], p["rho"], p["lam"], p["n_i"]
    g = rng(seed + 1)
    S = np.where(g.random(M.shape) < 0.2, g.standard_normal(M.shape), 0.0)
    n = M.shape[1]
    off = np.concatenate([[0], np.cumsum(n_i)])
    tot = sum(local_objective(M[:, off[i]:off[i + 1]], U, V[off[i]:off[i + 1]],
                              S[:, off[i]:off[i + 1]], rho, lam, int(n_i[i]), n)
              for i in range(len(n_i)))
    return abs(tot - objective(M, U, V, S, rho, lam)) / abs(tot)


def check_grad_U_local(grad_U_local, local_objective, seed=6):
    """grad_U L_i against central finite differences of L_i itself."""
    p = small_problem(seed)
    M, U, V, rho, lam, n_i = p["M"], p["U"], p["V"], p["rho"], p["lam"], p["n_i"]
    g = rng(seed + 1)
    S = np.where(g.random(M.shape) < 0.2, g.standard_normal(M.shape), 0.0)
    n = M.shape[1]
    c0, c1 = 0, int(n_i[0])
    Mi, Vi, Si = M[:, c0:c1], V[c0:c1], S[:, c0:c1]
    G = grad_U_local(Mi, U, Vi, Si, rho, int(n_i[0]), n)
    Gfd = fd_grad(lambda X: local_objective(Mi, X, Vi, Si, rho, lam, int(n_i[0]), n), U)
    return float(np.max(np.abs(G - Gfd)) / max(1.0, np.max(np.abs(Gfd))))


def check_fedavg_is_global_gd(dcf_iteration, objective, s_step, v_step, seed=7):
    """Algorithm 1 with K = 1: the FedAvg of the clients' U_i equals one global
    gradient step U - (eta/E) grad_U F(U, V_t, S_t) (§2.2, the K = 1 remark),
    the gradient taken by finite differences of the brute-force objective."""
    p = small_problem(seed)
    M, U, V, rho, lam, n_i = p["M"], p["U"], p["V"], p["rho"], p["lam"], p["n_i"]
    eta = 0.01
    U1, V1, S1 = dcf_iteration(M, n_i, U, V, rho, lam, u_mode=1, eta=eta)
    S_ref = s_step(M, U, V, lam)
    V_ref = v_step(M, S_ref, U, rho)
    G = fd_grad(lambda X: objective(M, X, V_ref, S_ref, rho, lam), U)
    U_ref = U - eta / len(n_i) * G
    return float(np.max(np.abs(U1 - U_ref)))


# --- FedAvg U-step of Algorithm 1, and its K > 1 local steps --------------------------
def _split(M, V, S, n_i):
    off = np.concatenate([[0], np.cumsum(n_i)])
    E = len(n_i)
    return ([M[:, off[i]:off[i + 1]] for i in range(E)],
            [V[off[i]:off[i + 1]] for i in range(E)],
            [S[:, off[i]:off[i + 1]] for i in range(E)])


def check_u_step_fedavg(u_step_fedavg, local_objective, seed=8):
    """Algorithm 1 eqs. U_local and U_agg with the (V_i, S_i) fixed: every client
    takes U - eta grad_U L_i, the gradient by central finite differences of the
    brute-force L_i of §2.2 (which carries the rho n_i/(2n) ||U||^2 share), and the
    server takes the unweighted mean of the E results."""
    p = small_problem(seed, m=8, n=13, r=3, E=3)
    M, U, V, rho, lam, n_i = p["M"], p["U"], p["V"], p["rho"], p["lam"], p["n_i"]
    n_i = np.array([2, 4, 7])          # uneven shares n_i / n
    g = rng(seed + 1)
    S = np.where(g.random(M.shape) < 0.2, g.standard_normal(M.shape), 0.0)
    n = M.shape[1]
    Ms, Vs, Ss = _split(M, V, S, n_i)
    eta = 0.03
    got = u_step_fedavg(Ms, Ss, Vs, U, rho, eta, n_i, n)
    ref = np.zeros_like(U)
    for Mi, Vi, Si, ni in zip(Ms, Vs, Ss, n_i):
        G = fd_grad(lambda X: local_objective(Mi, X, Vi, Si, rho, lam, int(ni), n), U)
        ref += U - eta * G
    ref /= len(n_i)
    return float(np.max(np.abs(got - ref)))


def check_u_step_fedavg_is_global_gd(u_step_fedavg, objective, seed=9):
    """With the clients' (V_i, S_i) fixed and K = 1, the unweighted FedAvg of the
    client steps is one global gradient step U - (eta/E) grad_U F of the §1
    objective (the K = 1 remark of §2.2), F's gradient by finite differences."""
    p = small_problem(seed, m=7, n=12, r=2, E=4)
    M, U, V, rho, lam, n_i = p["M"], p["U"], p["V"], p["rho"], p["lam"], p["n_i"]
    n_i = np.array([1, 2, 4, 5])
    g = rng(seed + 1)
    S = np.where(g.random(M.shape) < 0.2, g.standard_normal(M.shape), 0.0)
    Ms, Vs, Ss = _split(M, V, S, n_i)
    eta = 0.02
    got = u_step_fedavg(Ms, Ss, Vs, U, rho, eta, n_i, M.shape[1])
    G = fd_grad(lambda X: objective(M, X, V, S, rho, lam), U)
    return float(np.max(np.abs(got - (U - eta / len(n_i) * G))))


def check_local_steps(dcf_iteration, local_objective, s_step, v_step, K=3, seed=10):
    """Algorithm 1 with K local steps: each client i starts from the round's U and
    its own V_i; at every local step S_i and V_i are recomputed from the client's
    CURRENT U_i (eq. VS_arg with one S -> V sweep), then U_i moves by -eta times the
    finite-difference gradient of the brute-force L_i at (U_i, V_i, S_i)
    (eq. U_local).  Only after the K steps does the server average the U_i
    (eq. U_agg).  V and S returned are each client's last local V_i and S_i."""
    p = small_problem(seed, m=8, n=14, r=3, E=3)
    M, U, V, rho, lam = p["M"], p["U"], p["V"], p["rho"], p["lam"]
    n_i = np.array([3, 5, 6])
    n = M.shape[1]
    eta = 0.05
    U1, V1, S1 = dcf_iteration(M, n_i, U, V, rho, lam, u_mode=1, eta=eta, local_steps=K)
    off = np.concatenate([[0], np.cumsum(n_i)])
    U_acc = np.zeros_like(U)
    res = 0.0
    for i in range(len(n_i)):
        Mi = M[:, off[i]:off[i + 1]]
        Ui = U.copy()
        Vi = V[off[i]:off[i + 1]].copy()
        for _ in range(K):
            Si = s_step(Mi, Ui, Vi, lam)
            Vi = v_step(Mi, Si, Ui, rho)
            G = fd_grad(lambda X: local_objective(Mi, X, Vi, Si, rho, lam, int(n_i[i]), n),
                        Ui)
            Ui = Ui - eta * G
        U_acc += Ui
        res = max(res, float(np.max(np.abs(V1[off[i]:off[i + 1]] - Vi))))
        res = max(res, float(np.max(np.abs(S1[:, off[i]:off[i + 1]] - Si))))
    res = max(res, float(np.max(np.abs(U1 - U_acc / len(n_i)))))
    return res


def check_clients_independent(dcf_iteration, K=4, seed=11):
    """The clients of Algorithm 1 run their K local steps on their own data only
    and meet once, in the unweighted mean of eq. U_agg.  With two blocks of equal
    width (share n_i/n = 1/2 each), a round over [M_1, X] must therefore return
    U = (U_1 + U_2)/2 where U_1 is the round over the identical pair [M_1, M_1]
    (both clients take M_1's trajectory, so their mean is that trajectory) and U_2
    the round over [X, X]; the V and S blocks of [M_1, X] are those of the
    matching pairs.  Averaging inside the local loop breaks this for K > 1."""
    p = small_problem(seed, m=7, n=10, r=2, E=2)
    M, U, V, rho, lam = p["M"], p["U"], p["V"], p["rho"], p["lam"]
    w = 5
    M1, X = M[:, :w], M[:, w:]
    V1, VX = V[:w], V[w:]
    eta = 0.04
    kw = dict(u_mode=1, eta=eta, local_steps=K)
    Ua, Va, Sa = dcf_iteration(M, [w, w], U, V, rho, lam, **kw)
    U1, V11, S11 = dcf_iteration(np.hstack([M1, M1]), [w, w], U, np.vstack([V1, V1]),
                                 rho, lam, **kw)
    U2, VXX, SXX = dcf_iteration(np.hstack([X, X]), [w, w], U, np.vstack([VX, VX]),
                                 rho, lam, **kw)
    res = float(np.max(np.abs(2.0 * Ua - (U1 + U2))))
    res = max(res, float(np.max(np.abs(Va[:w] - V11[:w]))),
              float(np.max(np.abs(Va[w:] - VXX[w:]))))
    res = max(res, float(np.max(np.abs(Sa[:, :w] - S11[:, :w]))),
              float(np.max(np.abs(Sa[:, w:] - SXX[:, w:]))))
    # the identical pair: both clients end in the same state
    res = max(res, float(np.max(np.abs(V11[:w] - V11[w:]))))
    return res
