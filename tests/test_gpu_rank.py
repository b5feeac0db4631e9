"""Upper-bound rank (§2.2 "Problems with Unknown Exact Rank", §4.2 "Upper-bound
rank recovery", Table 1): the factor rank p is an upper bound on the truth's
rank k, and the recovered L is judged by its singular values.

dcf_singular_values computes them on the device (FP64 Gram matrices, cyclic
Jacobi); the oracle takes the QR of each factor and an SVD of the p x p core.
Both must agree on the same factors to FP64 rounding of the squared values,
and on whole runs from identical starting points within the 1e-3 bar of L.
Table 1's printed errors are context only (the paper gives no rho, lambda, T or
seed): the tests print the quantity for the paper's n = 200, p = 2r setting
without pinning it to the printed 0.0286.
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


def solver_for(case, path=dcf.PATH_AUTO):
    s = dcf.Solver(case["M"].shape[0], case["n_i"], case["r"], case["rho"], case["lam"],
                   path=path)
    s.load(case["M"])
    s.load_init(case["U0"], case["V0"])
    return s


@pytest.mark.parametrize("m,n_i,p,k,path", [
    (200, [50, 50, 50, 50], 20, 10, dcf.PATH_AUTO),     # the paper's n = 200, p = 2r
    (300, [100, 77, 140], 13, 5, dcf.PATH_GENERAL),     # ragged p, padded rank 16
    (257, [300, 211], 64, 30, dcf.PATH_AUTO),           # p = 64, the largest rank
    (96, [40, 33], 3, 7, dcf.PATH_GENERAL),             # p below the truth's rank
])
def test_singular_values_match_oracle_on_same_factors(m, n_i, p, k, path):
    case = make_case(m, n_i, p, k=k, seed=m + p, amp=10.0)
    s = solver_for(case, path)
    s.step(7)
    U, V = s.factors()
    s.set_truth(case["inst"].A, case["inst"].B)
    sig, sig0, err = s.singular_values(with_truth=True)
    s.close()
    ref = O.singular_values_factored(U, V)[:p]
    ref0 = O.singular_values_factored(case["inst"].A, case["inst"].B)[:k]
    # squared singular values agree to FP64 rounding of the Gram route
    assert np.max(np.abs(sig ** 2 - ref ** 2)) <= 1e-10 * ref[0] ** 2
    assert np.max(np.abs(sig0 ** 2 - ref0 ** 2)) <= 1e-10 * ref0[0] ** 2
    assert np.all(np.diff(sig) <= 0) and np.all(sig >= 0)
    assert abs(err - O.singular_value_error(ref, ref0, k)) <= 1e-6 * max(1.0, err)


def test_singular_values_without_truth_and_state_errors():
    case = make_case(128, [64, 64], 8, seed=4)
    s = solver_for(case)
    s.step(2)
    sig, sig0, err = s.singular_values()
    assert sig0 is None and err is None and sig.shape == (8,)
    with pytest.raises(dcf.DcfError) as e:
        dcf.dcf_singular_values(s.h, 8, 4)          # sigma0 requested, no truth registered
    assert e.value.status == dcf.DCF_ESTATE
    s.close()


def test_upper_bound_rank_recovery_paper_setting():
    """§4.2: m = n = 200, truth rank r = 0.05 n = 10, s = 0.05, factor rank
    p = 0.1 n = 20, lambda = 1/sqrt(n) and a unit nuclear-norm weight rho = 1
    (the paper states neither; with rho = 1e-2 the surplus components are not
    suppressed, see the design notes).  The GPU run and the oracle run from
    identical starting points reach the same L (1e-3) and the same Table 1
    error (1e-3), the spectrum beyond the truth's rank collapses
    (sigma_{r+1} / sigma_r small, the figure's reading), and the error is small."""
    case = make_case(200, [50, 50, 50, 50], 20, k=10, seed=2207, amp=10.0, factor_std=1.0,
                     rho=1.0)
    T = 300
    s = solver_for(case)
    s.step(T)
    U, V = s.factors()
    s.set_truth(case["inst"].A, case["inst"].B)
    sig, sig0, err = s.singular_values(with_truth=True)
    s.close()
    Uo, Vo, _, _, _ = O.dcf_run(case["M"], case["n_i"], case["U0"], case["V0"], case["rho"],
                                case["lam"], T)
    ref = O.singular_values_factored(Uo, Vo)
    ref0 = O.singular_values_factored(case["inst"].A, case["inst"].B)[:10]
    err_o = O.singular_value_error(ref, ref0, 10)
    assert rel(U @ V.T, Uo @ Vo.T) <= 1e-3
    assert np.max(np.abs(sig - ref)) <= 1e-3 * ref[0]
    assert abs(err - err_o) <= 1e-3
    assert sig[10] / sig[9] < 1e-3
    assert err < 0.05
    print(f"\nTable 1 setting n=200 r=10 p=20: relative singular-value error {err:.4f} "
          f"(oracle {err_o:.4f}; the paper prints 0.0286 with unstated rho, lambda, T); "
          f"sigma_11/sigma_10 = {sig[10] / sig[9]:.2e}")
