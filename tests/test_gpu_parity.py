"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: relative Frobenius error <= 1e-4 on U, V and S after one step
from identical float32 starting points; <= 1e-3 on L = U V^T after several
steps and at convergence; the S support identical except where the oracle's
|R| lies within 1e-5*lambda (plus the FP32 rounding bound of R) of lambda.
"""
import numpy as np
import pytest

import oracle as O
from paper_2207_11669_gb300 import dcf
from tests.helpers import make_case, rel, r_error_bound, support_flips

pytestmark = pytest.mark.gpu

SHAPES = [
    # (m, n_i, r): the 200x200 E=4 workload, ragged rows/columns, each padded rank
    (200, [50, 50, 50, 50], 5),
    (300, [100, 77, 140], 16),
    (129, [33, 64, 31], 32),
    (257, [300, 211], 40),
    (64, [10, 9, 11], 8),
    (1000, [700, 1300, 517], 32),
    (260, [300, 211], 40),          # R = 64 on the two-pass tensor-core path
    (4100, [150, 170], 6),          # 17 slabs: past the fused kernel's cluster
]


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_11669_gb300 import build
    build.build()
    torch.cuda.init()


def fused_ok(m, r):
    return r <= 32 and m % 4 == 0 and (m + 255) // 256 <= 16


def small_ok(m, n, r):
    # the whole-solve kernel's shared memory (M with leading dimension m + 1,
    # two copies of U and V, W, the r x r workspace) within one SM
    R = 8 if r <= 8 else 16
    smem = (10 * R * R * 8 + 2048 + 2 * R * R * 4 + 512 * 8 + ((m + 1) * n * 4 + 15) // 16 * 16
            + 4 * (3 * m * R + 2 * n * R))
    return r <= 16 and smem + 2048 <= 232448


def path_ok(path, m, r, n=None):
    if path == dcf.PATH_FUSED:
        return fused_ok(m, r)
    if path == dcf.PATH_TC2:
        return m % 4 == 0
    if path == dcf.PATH_SMALL:
        return small_ok(m, n, r)
    return True


PATHS = [dcf.PATH_GENERAL, dcf.PATH_FUSED, dcf.PATH_TC2, dcf.PATH_SMALL]


def gpu_solver(case, **kw):
    s = dcf.Solver(case["M"].shape[0], case["n_i"], case["r"], case["rho"], case["lam"], **kw)
    s.load(case["M"])
    s.load_init(case["U0"], case["V0"])
    return s


def oracle_step(case, iters=1, **kw):
    return O.dcf_run(case["M"], case["n_i"], case["U0"], case["V0"], case["rho"], case["lam"],
                     iters, **kw)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("m,n_i,r", SHAPES)
def test_one_step_parity(m, n_i, r, path):
    if not path_ok(path, m, r, sum(n_i)):
        pytest.skip("shape outside this path")
    case = make_case(m, n_i, r, seed=m + r)
    s = gpu_solver(case, path=path)
    assert s.path == path
    s.step(1)
    U, V = s.factors()
    U1, V1, S1, U0, V0 = oracle_step(case, 1)
    assert rel(U, U1) <= 1e-4
    assert rel(V, V1) <= 1e-4
    off = O.block_offsets(case["n_i"])
    S_gpu = np.concatenate([s.LS(i)[1] for i in range(len(n_i))], axis=1)
    assert rel(S_gpu, S1) <= 1e-4
    R_ref = case["M"].astype(np.float64) - case["U0"].astype(np.float64) @ case["V0"].T.astype(
        np.float64)
    eps = r_error_bound(case["M"], case["U0"], case["V0"], r)
    flips, bad = support_flips(S_gpu, S1, R_ref, case["lam"], eps)
    assert bad == 0, (flips, bad)
    s.close()


@pytest.mark.parametrize("path", PATHS)
def test_fedavg_step_parity(path):
    if path == dcf.PATH_SMALL:
        pytest.skip("the whole-solve kernel runs the exact U-step")
    case = make_case(300, [100, 77, 140], 16, seed=3)
    s = gpu_solver(case, u_mode=1, eta0=0.01, path=path)
    s.step(3)
    U, V = s.factors()
    Uo, Vo, *_ = oracle_step(case, 3, u_mode=1, eta0=0.01)
    assert rel(U, Uo) <= 1e-4
    assert rel(V, Vo) <= 1e-4
    s.close()


@pytest.mark.parametrize("path", PATHS)
def test_several_steps_L_parity(path):
    case = make_case(200, [50] * 4, 5, seed=7)
    s = gpu_solver(case, path=path)
    s.step(10)
    U, V = s.factors()
    Uo, Vo, *_ = oracle_step(case, 10)
    assert rel(U @ V.T, Uo @ Vo.T) <= 1e-3
    s.close()


@pytest.mark.parametrize("path", PATHS)
def test_converged_L_parity_and_support(path):
    """The 200 x 200, E = 4 workload run to convergence on both sides.  The GPU
    solve stops at a relative change of 1e-6: FP32 iterates settle into a
    rounding-level cycle near 1e-7 on some paths, which the change metric (formed
    from the Grams of the change itself) resolves rather than rounding to zero."""
    case = make_case(200, [50] * 4, 5, seed=20220723)
    s = gpu_solver(case, max_iter=400, tol=1e-6, path=path)
    it, d, ok = s.solve()
    assert ok and d <= 1e-6, (it, d)
    U, V = s.factors()
    Uo, Vo, So, ito, do = O.dcf_solve(case["M"], case["n_i"], case["U0"], case["V0"],
                                      case["rho"], case["lam"], 400, 1e-7)
    assert rel(U @ V.T, Uo @ Vo.T) <= 1e-3
    S_gpu = np.concatenate([s.LS(i)[1] for i in range(4)], axis=1)
    # S at convergence: flips only where the oracle's |R| is within the threshold
    # band widened by the difference of the two residuals
    R_ref = case["M"].astype(np.float64) - Uo @ Vo.T
    R_gpu = case["M"].astype(np.float64) - U.astype(np.float64) @ V.T.astype(np.float64)
    eps = np.abs(R_gpu - R_ref) + r_error_bound(case["M"], U, V, 5)
    flips, bad = support_flips(S_gpu, So, R_ref, case["lam"], eps)
    assert bad == 0, (flips, bad)
    s.close()


def test_fused_path_is_chosen_automatically():
    case = make_case(300, [100, 77, 140], 16, seed=21)
    s = gpu_solver(case)
    assert s.path == dcf.PATH_FUSED
    s.close()
    case = make_case(257, [300, 211], 40, seed=21)
    s = gpu_solver(case)
    assert s.path == dcf.PATH_GENERAL          # m % 4 != 0: no tensor map
    s.close()
    case = make_case(260, [300, 211], 40, seed=21)
    s = gpu_solver(case)
    assert s.path == dcf.PATH_TC2              # r > 32
    s.close()
    case = make_case(4100, [150, 170], 6, seed=21)
    s = gpu_solver(case)
    assert s.path == dcf.PATH_TC2              # more than 16 slabs
    s.close()
    with pytest.raises(dcf.DcfError):
        dcf.Solver(257, [300, 211], 40, 1e-2, 0.1, path=dcf.PATH_TC2)
    case = make_case(200, [50] * 4, 5, seed=21)
    s = gpu_solver(case)
    assert s.path == dcf.PATH_FUSED             # the whole-solve path is on request only
    s.close()
    with pytest.raises(dcf.DcfError):
        dcf.Solver(300, [100, 77, 140], 16, 1e-2, 0.1, path=dcf.PATH_SMALL)


def test_whole_solve_one_launch_equals_single_steps():
    """dcf_step(n) on the whole-solve path is one launch of n iterations; it
    must give the bits of n launches of one iteration each (the r x r state
    is rebuilt from U and V, which are written back exactly)."""
    case = make_case(200, [50] * 4, 5, seed=31)
    a = gpu_solver(case, path=dcf.PATH_SMALL)
    b = gpu_solver(case, path=dcf.PATH_SMALL)
    a.step(7)
    for _ in range(7):
        b.step(1)
    Ua, Va = a.factors()
    Ub, Vb = b.factors()
    assert np.array_equal(Ua, Ub) and np.array_equal(Va, Vb)
    assert a.stats() == b.stats()
    a.close()
    b.close()
    with pytest.raises(dcf.DcfError):
        dcf.Solver(257, [300, 211], 40, 1e-2, 0.1, path=dcf.PATH_FUSED)


def test_init_sweep_parity():
    case = make_case(257, [300, 211], 40, seed=11)
    s = dcf.Solver(257, case["n_i"], 40, case["rho"], case["lam"])
    s.load(case["M"])
    s.load_init(case["U0"])          # V0 from the S = 0 sweep on the GPU
    U, V = s.factors()
    assert rel(V, case["V0"]) <= 1e-5
    assert np.array_equal(U, case["U0"])
    s.close()


@pytest.mark.parametrize("path", PATHS)
def test_partition_invariance_on_gpu(path):
    if not path_ok(path, 300, 16, 317):
        pytest.skip("shape outside this path")
    case = make_case(300, [100, 77, 140], 16, seed=5)
    a = gpu_solver(case, path=path)
    case1 = dict(case, n_i=np.array([317]))
    b = gpu_solver(case1, path=path)
    a.step(4)
    b.step(4)
    Ua, Va = a.factors()
    Ub, Vb = b.factors()
    assert np.array_equal(Ua, Ub) and np.array_equal(Va, Vb)
    a.close()
    b.close()


@pytest.mark.parametrize("path", PATHS)
def test_stats_and_rel_err(path):
    case = make_case(200, [50] * 4, 5, seed=9)
    s = gpu_solver(case, path=path)
    s.set_truth(case["inst"].A, case["inst"].B)
    s.step(2)
    obj, dL, it = s.stats()
    U2, V2, S2, U1, V1 = oracle_step(case, 2)
    assert it == 2
    assert abs(obj - O.objective_huber(case["M"], U1, V1, case["rho"], case["lam"])) <= 1e-4 * abs(obj)
    assert abs(dL - O.factor_delta_rel(U2, V2, U1, V1)) <= 1e-3 * dL + 1e-7
    U, V = s.factors()
    assert abs(s.rel_err() - O.rel_err_L(U, V, case["inst"].A, case["inst"].B)) <= 1e-5
    s.close()


@pytest.mark.parametrize("path", PATHS)
def test_get_LS_blocks_and_privacy(path):
    if not path_ok(path, 132, 32, 128):
        pytest.skip("shape outside this path")
    case = make_case(132, [33, 64, 31], 32, seed=13)
    s = gpu_solver(case, path=path)
    s.step(2)
    U2, V2, S2, U1, V1 = oracle_step(case, 2)
    off = O.block_offsets(case["n_i"])
    for i in range(3):
        L, S = s.LS(i)
        assert rel(L, U2 @ V2[off[i]:off[i + 1]].T) <= 1e-4
        assert rel(S, S2[:, off[i]:off[i + 1]]) <= 1e-4
    dcf.dcf_set_private(s.h, 1, True)
    with pytest.raises(dcf.DcfError) as e:
        s.LS(1)
    assert e.value.status == dcf.DCF_EPRIVATE
    s.close()


def test_errors_are_status_codes():
    with pytest.raises(dcf.DcfError) as e:
        dcf.Solver(10, [5, 5], 0, 1e-2, 0.1)
    assert e.value.status == dcf.DCF_EINVAL
    with pytest.raises(dcf.DcfError):
        dcf.Solver(10, [5, 5], 3, -1.0, 0.1)
    s = dcf.Solver(16, [8, 8], 3, 1e-2, 0.1)
    with pytest.raises(dcf.DcfError) as e:
        s.step(1)
    assert e.value.status == dcf.DCF_ESTATE
    M = np.ones((16, 16), np.float32, order="F")
    M[3, 4] = np.nan
    with pytest.raises(dcf.DcfError) as e:
        s.load(M)
    assert e.value.status == dcf.DCF_ENONFINITE
    s.close()


def test_default_init_is_seeded_gaussian():
    M = np.asfortranarray(np.random.default_rng(0).standard_normal((512, 256)).astype(np.float32))
    a = dcf.Solver(512, [128, 128], 8, 1e-2, 0.05, seed=42)
    a.load(M)
    b = dcf.Solver(512, [128, 128], 8, 1e-2, 0.05, seed=42)
    b.load(M)
    Ua, _ = a.factors()
    Ub, _ = b.factors()
    assert np.array_equal(Ua, Ub)
    assert abs(Ua.mean()) < 0.01 and abs(Ua.var() * 512 - 1.0) < 0.1
    a.close()
    b.close()


@pytest.mark.parametrize("path", PATHS)
def test_borrowed_device_matrix_matches_host_copy(path):
    import torch
    if not path_ok(path, 300, 16, 317):
        pytest.skip("shape outside this path")
    case = make_case(300, [100, 77, 140], 16, seed=17)
    Mt = torch.from_numpy(np.ascontiguousarray(case["M"].T)).cuda()   # (n, m) = M column-major
    s1 = gpu_solver(case, path=path)
    s2 = dcf.Solver(300, case["n_i"], 16, case["rho"], case["lam"], path=path)
    s2.load(Mt)
    s2.load_init(case["U0"], case["V0"])
    s1.step(2)
    s2.step(2)
    assert np.array_equal(s1.factors()[0], s2.factors()[0])
    s1.close()
    s2.close()


@pytest.mark.parametrize("path", PATHS)
def test_reload_continues_from_the_current_factors(path):
    """dcf_reload_blocks: two steps on M, new values M' copied in, one more
    step equals one oracle round on M' from the factors the GPU held."""
    import torch
    m, n_i, r = 120, [40, 37, 50], 16
    if not path_ok(path, m, r, sum(n_i)):
        pytest.skip("shape outside this path")
    case = make_case(m, n_i, r, seed=23)
    case2 = make_case(m, n_i, r, seed=24)
    s = gpu_solver(case, path=path)
    s.step(2)
    Ua, Va = s.factors()
    s.reload(case2["M"])                           # host blocks
    s.step(1)
    U, V = s.factors()
    U1, V1, S1, _, _ = O.dcf_run(case2["M"], n_i, Ua, Va, case2["rho"], case2["lam"], 1)
    assert rel(U, U1) <= 1e-4
    assert rel(V, V1) <= 1e-4
    S_gpu = np.concatenate([s.LS(i)[1] for i in range(len(n_i))], axis=1)
    assert rel(S_gpu, S1) <= 1e-4
    # device blocks: back to M, then one more step, against the oracle again
    Ub, Vb = U, V
    s.reload(torch.from_numpy(np.ascontiguousarray(case["M"].T)).cuda())
    s.step(1)
    U, V = s.factors()
    U2, V2, _, _, _ = O.dcf_run(case["M"], n_i, Ub, Vb, case["rho"], case["lam"], 1)
    assert rel(U, U2) <= 1e-4
    assert rel(V, V2) <= 1e-4
    s.close()


def test_reload_errors():
    import torch
    case = make_case(200, [50, 50, 50, 50], 5, seed=3)
    s = dcf.Solver(200, case["n_i"], 5, case["rho"], case["lam"])
    with pytest.raises(dcf.DcfError) as e:
        s.reload(case["M"])                        # nothing loaded yet
    assert e.value.status == dcf.DCF_ESTATE
    Mt = torch.from_numpy(np.ascontiguousarray(case["M"].T)).cuda()
    s.load(Mt)                                     # borrowed
    with pytest.raises(dcf.DcfError) as e:
        s.reload(case["M"])
    assert e.value.status == dcf.DCF_ESTATE
    s.load(case["M"])                              # own copy
    s.step(1)
    bad = case["M"].copy()
    bad[7, 11] = np.nan
    with pytest.raises(dcf.DcfError) as e:
        s.reload(bad)
    assert e.value.status == dcf.DCF_ENONFINITE
    with pytest.raises(dcf.DcfError) as e:
        s.step(1)                                  # the rejected values are never iterated on
    assert e.value.status == dcf.DCF_ESTATE
    s.load(case["M"])
    s.step(1)
    s.close()


@pytest.mark.parametrize("path", PATHS)
def test_async_reload_continues_from_the_current_factors(path):
    """dcf_reload_blocks_async: the new values are copied behind the enqueued
    work into a second buffer; the next step reads them (oracle from the
    factors the GPU held), a second call before a step replaces the first, and
    the S of the step comes from the new values."""
    m, n_i, r = 120, [40, 37, 50], 16
    if not path_ok(path, m, r, sum(n_i)):
        pytest.skip("shape outside this path")
    case = make_case(m, n_i, r, seed=31)
    case2 = make_case(m, n_i, r, seed=32)
    case3 = make_case(m, n_i, r, seed=33)
    s = gpu_solver(case, path=path)
    s.step(2)
    Ua, Va = s.factors()
    s.reload_async(case3["M"])
    s.reload_async(case2["M"])                     # replaces the first
    s.step(1)
    U, V = s.factors()
    U1, V1, S1, _, _ = O.dcf_run(case2["M"], n_i, Ua, Va, case2["rho"], case2["lam"], 1)
    assert rel(U, U1) <= 1e-4
    assert rel(V, V1) <= 1e-4
    S_gpu = np.concatenate([s.LS(i)[1] for i in range(len(n_i))], axis=1)
    assert rel(S_gpu, S1) <= 1e-4
    # alternate buffers for a few more steps: each reads the matrix copied before it
    for q, c in enumerate([case, case3, case2]):
        Ub, Vb = s.factors()
        s.reload_async(c["M"])
        s.step(1)
        U, V = s.factors()
        U2, V2, _, _, _ = O.dcf_run(c["M"], n_i, Ub, Vb, c["rho"], c["lam"], 1)
        assert rel(U, U2) <= 1e-4, q
        assert rel(V, V2) <= 1e-4, q
    s.close()


def test_async_reload_of_nonfinite_values_stops_the_solve():
    case = make_case(200, [50, 50, 50, 50], 5, seed=4)
    s = dcf.Solver(200, case["n_i"], 5, case["rho"], case["lam"])
    s.load(case["M"])
    s.step(1)
    U0, _ = s.factors()
    bad = case["M"].copy()
    bad[3, 150] = np.inf
    s.reload_async(bad)
    s.step(2)                                      # no iteration runs on the rejected values
    with pytest.raises(dcf.DcfError) as e:
        s.stats()
    assert e.value.status == dcf.DCF_ENONFINITE
    assert np.array_equal(s.factors()[0], U0)
    s.load(case["M"])                              # a full load starts over
    s.step(1)
    s.stats()
    s.close()
