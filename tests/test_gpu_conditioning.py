"""Ill-conditioned ridge systems against the FP64 oracle.

The V-step solves with U^T U + rho I (App. B eq. condition1) and the U-step
with V^T V + rho I.  With a small rho and nearly collinear columns of U both
are ill-conditioned and rounding errors are amplified by their condition
numbers.  The library estimates the 1-norm condition number of each system
as it inverts it; above 100 the inverse is formed in double-float and handed
on as a float pair, W = U G^{-1}, V_{t-1}^T V_t applied to U_{t-1} and the
Grams of V use compensated products (the FP32 rounding of every product
kept), so that the rounding of W and V to FP32 storage is what is left.  An
FP64 computation in which only W and V are rounded to FP32
(``fp32_w_reference``) shows that floor.  The checks: U and V within 1e-4 of
the oracle up to kappa ~ 1.4e6 on every path, V within 1e-4 and U within 1e-3
at kappa ~ 1.4e8, the estimate reported by dcf_get_conditioning within a
factor 4 of numpy's 1-norm condition number (below 1e6, where the FP32
inverse it is read from is accurate to kappa 2^-24), and a well-conditioned
problem on the FP32 route.
"""
import numpy as np
import pytest

import oracle as O
from paper_2207_11669_gb300 import dcf
from tests.helpers import make_case, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_11669_gb300 import build
    build.build()


def collinear_case(eps, rho, r=8, m=300, n_i=(100, 76, 140), seed=3):
    """U0 with its second column within eps of its first (relative), rho small."""
    case = make_case(m, list(n_i), r, seed=seed, rho=rho)
    U0 = case["U0"].astype(np.float64)
    g = np.random.default_rng(seed + 2)
    U0[:, 1] = U0[:, 0] + eps * g.standard_normal(m) / np.sqrt(m)
    U0 = U0.astype(np.float32)
    case["U0"] = U0
    case["V0"] = O.init_v0(case["M"], U0.astype(np.float64), rho).astype(np.float32)
    G = U0.astype(np.float64).T @ U0.astype(np.float64) + rho * np.eye(r)
    return case, float(np.linalg.cond(G, 1))


def fp32_w_reference(case):
    """One iteration in FP64 except that W = U (U^T U + rho I)^{-1} and the new V
    are rounded to FP32 (test-side numpy, a model of the GPU's storage)."""
    M, U0, V0, rho, lam = case["M"], case["U0"], case["V0"], case["rho"], case["lam"]
    S = O.s_step(M, U0, V0, lam)
    X = M - S
    U = U0.astype(np.float64)
    Gi = np.linalg.inv(U.T @ U + rho * np.eye(U.shape[1]))
    W = (U @ Gi).astype(np.float32).astype(np.float64)
    V = (X.T @ W).astype(np.float32).astype(np.float64)
    Un = (X @ V) @ np.linalg.inv(V.T @ V + rho * np.eye(U.shape[1]))
    return Un, V


@pytest.mark.parametrize("path", [dcf.PATH_GENERAL, dcf.PATH_FUSED, dcf.PATH_TC2])
@pytest.mark.parametrize("eps,rho", [
    (3e-2, 1e-6),     # kappa ~ 5e3
    (1e-2, 1e-6),     # kappa ~ 4.4e4
    (1e-3, 1e-6),     # kappa ~ 1.4e6
    (1e-4, 1e-8),     # kappa ~ 1.4e8: recorded
])
def test_one_step_parity_ill_conditioned(eps, rho, path):
    case, kappa = collinear_case(eps, rho)
    s = dcf.Solver(case["M"].shape[0], case["n_i"], case["r"], case["rho"], case["lam"],
                   path=path)
    s.load(case["M"])
    s.load_init(case["U0"], case["V0"])
    s.step(1)
    U, V = s.factors()
    kg, kh = s.conditioning()
    s.close()
    Uo, Vo, _ = O.dcf_iteration(case["M"], case["n_i"], case["U0"], case["V0"], case["rho"],
                                case["lam"])
    Uw, Vw = fp32_w_reference(case)
    eu, ev = rel(U, Uo), rel(V, Vo)
    euw, evw = rel(Uw, Uo), rel(Vw, Vo)
    print(f"\npath {path} kappa_1(U^T U + rho I) = {kappa:.2e} (estimate {kg:.2e}; V side "
          f"{kh:.2e}): rel err U {eu:.2e}, V {ev:.2e} "
          f"(FP64 with W, V rounded to FP32: U {euw:.2e}, V {evw:.2e})")
    assert np.all(np.isfinite(U)) and np.all(np.isfinite(V))
    # the estimate is of the G of the new U; the case's kappa is of U0's G
    U64 = U.astype(np.float64)
    kap_new = float(np.linalg.cond(U64.T @ U64 + case["rho"] * np.eye(U.shape[1]), 1))
    if kap_new < 1e6:   # FP32-route inverse within ~kappa 2^-24 of the true one
        assert kap_new / 4 <= kg <= 4 * kap_new
    else:
        assert kg > 100.0
    assert ev <= 1e-4
    assert eu <= (1e-4 if kappa < 1e7 else 1e-3)


@pytest.mark.parametrize("r", [8, 16, 32, 64])
def test_well_conditioned_problem_takes_the_fp32_route(r):
    """Each padded rank has its own FP32 route (one-warp Gauss-Jordan up to 32,
    the factorisation-based one at 64); the estimate must be right on all."""
    case = make_case(300, [100, 76, 140], r, seed=5)
    s = dcf.Solver(300, case["n_i"], r, case["rho"], case["lam"], path=dcf.PATH_GENERAL)
    s.load(case["M"])
    s.load_init(case["U0"], case["V0"])
    s.step(1)
    U, V = s.factors()
    kg, kh, route_g, route_h = s.conditioning(routes=True)
    s.close()
    U64, V64 = U.astype(np.float64), V.astype(np.float64)
    kap = float(np.linalg.cond(U64.T @ U64 + case["rho"] * np.eye(r), 1))
    kap_h = float(np.linalg.cond(V64.T @ V64 + case["rho"] * np.eye(r), 1))
    print(f"\nr {r}: kappa_1 {kap:.3g}, estimate {kg:.3g} (route {route_g}); V side "
          f"{kap_h:.3g}, estimate {kh:.3g} (route {route_h})")
    assert kap / 4 <= kg <= 4 * kap
    assert kap_h / 4 <= kh <= 4 * kap_h
    assert kg < 100.0 and route_g == 0
    assert route_h == (0 if kh < 100.0 else 1)
