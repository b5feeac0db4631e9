"""K > 1 local steps of Algorithm 1 (FedAvg mode) on the GPU against the oracle.

Each client i iterates K times on its own block with its own U_i (S-step and
V-step from U_i, then U_i <- U_i - eta_t grad_U L_i), and the server averages
the U_i once per round (Algorithm 1, eqs. VS_arg, U_local, U_agg).  The oracle's
branch for this (``dcf_iteration(..., u_mode=1, local_steps=K)``) is pinned on
the CPU by finite-difference client steps and by client independence.

Tolerances as in the other parity tests: relative Frobenius error <= 1e-4 on
U, V and the S of the last local step after one round from identical float32
starting points, <= 1e-3 on L after several rounds.  The ablation of §4.3
("Number of local iterations"): more local steps reach the stopping tolerance
in far fewer rounds.
"""
import numpy as np
import pytest

import oracle as O
from paper_2207_11669_gb300 import dcf, synth
from tests.helpers import make_case, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_11669_gb300 import build
    build.build()


def path_ok(path, m, r):
    if path == dcf.PATH_FUSED:
        return r <= 32 and m % 4 == 0 and (m + 255) // 256 <= 16
    if path == dcf.PATH_TC2:
        return m % 4 == 0
    return True


def stable_eta0(case, scale=0.3):
    """A step size well inside the stable range of every client's gradient step:
    scale / the largest eigenvalue of the start's V_i^T V_i over the clients."""
    off = O.block_offsets(case["n_i"])
    V = case["V0"].astype(np.float64)
    lmax = max(np.linalg.eigvalsh(V[off[i]:off[i + 1]].T @ V[off[i]:off[i + 1]]).max()
               for i in range(len(case["n_i"])))
    return scale / lmax


def gpu_run(case, K, eta0, path, rounds):
    s = dcf.Solver(case["M"].shape[0], case["n_i"], case["r"], case["rho"], case["lam"],
                   u_mode=1, eta0=eta0, local_steps=K, path=path)
    s.load(case["M"])
    s.load_init(case["U0"], case["V0"])
    s.step(rounds)
    return s


@pytest.mark.parametrize("path", [dcf.PATH_GENERAL, dcf.PATH_FUSED, dcf.PATH_TC2])
@pytest.mark.parametrize("K", [2, 10])
@pytest.mark.parametrize("m,n_i,r", [
    (300, [100, 77, 140], 16),        # ragged rows and blocks
    (512, [300, 211, 150, 97], 8),    # four uneven clients, padded rank
    (260, [300, 211], 40),            # R = 64
])
def test_one_round_parity(m, n_i, r, K, path):
    if not path_ok(path, m, r):
        pytest.skip("shape outside this path")
    case = make_case(m, n_i, r, seed=m + K)
    eta0 = stable_eta0(case)
    s = gpu_run(case, K, eta0, path, 1)
    assert s.path == path
    U, V = s.factors()
    obj, dL, it = s.stats()
    S_gpu = np.hstack([s.LS(i)[1] for i in range(len(n_i))])
    s.close()
    Uo, Vo, So, Up, Vp = O.dcf_run(case["M"], n_i, case["U0"], case["V0"], case["rho"],
                                   case["lam"], 1, u_mode=1, eta0=eta0, local_steps=K)
    assert it == 1
    assert rel(U, Uo) <= 1e-4 and rel(V, Vo) <= 1e-4
    assert rel(S_gpu, So) <= 1e-4
    # the round's objective at (U_{t-1}, V_{t-1}, S of the first local step)
    ref_obj = O.objective_huber(case["M"], case["U0"], case["V0"], case["rho"], case["lam"])
    assert abs(obj - ref_obj) <= 1e-4 * abs(ref_obj)
    ref_dL = O.factor_delta_rel(Uo, Vo, Up, Vp)
    assert abs(dL - ref_dL) <= 1e-3 * ref_dL + 1e-6


@pytest.mark.parametrize("path", [dcf.PATH_GENERAL, dcf.PATH_FUSED])
def test_several_rounds_parity(path):
    case = make_case(384, [120, 64, 200, 90], 12, seed=5)
    eta0 = stable_eta0(case)
    s = gpu_run(case, 5, eta0, path, 6)
    U, V = s.factors()
    s.close()
    Uo, Vo, _, _, _ = O.dcf_run(case["M"], case["n_i"], case["U0"], case["V0"], case["rho"],
                                case["lam"], 6, u_mode=1, eta0=eta0, local_steps=5)
    assert rel(U @ V.T, Uo @ Vo.T) <= 1e-3


def test_k1_is_the_plain_fedavg_round():
    """local_steps = 1 in FedAvg mode is the existing single-step round; K = 1 through
    the oracle's local-step branch gives the same iterate."""
    case = make_case(256, [100, 156], 8, seed=9)
    eta0 = stable_eta0(case)
    s = gpu_run(case, 1, eta0, dcf.PATH_AUTO, 2)
    U, V = s.factors()
    s.close()
    Uo, Vo, _, _, _ = O.dcf_run(case["M"], case["n_i"], case["U0"], case["V0"], case["rho"],
                                case["lam"], 2, u_mode=1, eta0=eta0, local_steps=1)
    assert rel(U, Uo) <= 1e-4 and rel(V, Vo) <= 1e-4


def test_more_local_steps_need_fewer_rounds():
    """§4.3 "Number of local iterations" (m = n = 500, E = 10 clients): with the
    same step size, K = 10 local steps per round reach the stopping tolerance
    in far fewer communication rounds than K = 1.  The rounds of the GPU runs
    match the oracle's within a few rounds."""
    m = n = 500
    E, k = 10, 25
    inst = synth.make_instance(m, n, k, seed=11, density=0.05, amp=10.0,
                               factor_std=1.0 / np.sqrt(k), E=E)
    U0 = synth.gaussian_u0(m, k, 11)
    rho, lam, eta0, tol = 1e-2, 1.0 / np.sqrt(m), 0.05, 1e-4
    V0 = O.init_v0(inst.M, U0.astype(np.float64), rho).astype(np.float32)
    rounds = {}
    for K in (1, 10):
        s = dcf.Solver(m, inst.n_i, k, rho, lam, max_iter=400, tol=tol, u_mode=1, eta0=eta0,
                       local_steps=K)
        s.load(inst.M)
        s.load_init(U0, V0)
        it, dL, conv = s.solve()
        assert conv
        U, V = s.factors()
        s.close()
        _, _, _, it_o, _ = O.dcf_solve(inst.M, inst.n_i, U0, V0, rho, lam, 400, tol, u_mode=1,
                                       eta0=eta0, local_steps=K)
        assert dL <= tol
        assert abs(it - it_o) <= max(3, 0.05 * it_o)
        assert O.rel_err_L(U, V, inst.A, inst.B) < 0.05
        rounds[K] = it
    assert rounds[10] * 2 < rounds[1]
    print(f"\nrounds to dL <= {tol}: K=1 {rounds[1]}, K=10 {rounds[10]}")


def test_local_steps_validation():
    import torch
    case = make_case(128, [64, 64], 8, seed=3)
    with pytest.raises(dcf.DcfError) as e:
        dcf.Solver(128, [64, 64], 8, 1e-2, 0.1, u_mode=0, local_steps=3)   # exact mode
    assert e.value.status == dcf.DCF_EINVAL
    s = gpu_run(case, 3, stable_eta0(case), dcf.PATH_AUTO, 1)
    Mt = torch.from_numpy(np.ascontiguousarray(case["M"].T)).cuda()
    with pytest.raises(dcf.DcfError) as e:
        s.reload_async(Mt)
    assert e.value.status == dcf.DCF_EINVAL
    s.close()
