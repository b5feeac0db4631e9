"""Parity of batched problems (dcf_batch_*) with the FP64 oracle.

Instances of up to 4096 rows run their pass over M on the tensor-core kernel
(one cluster per instance, m padded to a multiple of 4 with zero rows), the
others on the general passes; both kinds share a batch below.

Each instance of a batch must compute what the oracle computes for it alone:
relative Frobenius error <= 1e-4 on U and V after one step from identical
float32 starting points, <= 1e-3 after several steps, and every instance of a
solved batch at or below its tolerance.  Shapes mix the three padded ranks
(8, 16, 32), ragged m and uneven column blocks.
"""
import numpy as np
import pytest

import oracle as O
from paper_2207_11669_gb300 import dcf
from tests.helpers import make_case, rel

pytestmark = pytest.mark.gpu

SHAPES = [
    # (m, n_i, r)
    (64, [40, 33, 50], 3),
    (200, [50, 50, 50, 50], 5),
    (257, [300, 211], 12),
    (130, [70, 90, 65, 81, 30], 16),
    (300, [100, 77, 140], 20),
    (96, [64, 64], 32),
    (513, [129, 700], 8),
    (4100, [150, 170], 6),      # past the tensor-core kernel's 4096 rows: general passes
]


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_11669_gb300 import build
    build.build()
    torch.cuda.init()


def cases(seed0=0):
    return [make_case(m, n_i, r, seed=seed0 + 17 * q + m, density=0.05, amp=5.0)
            for q, (m, n_i, r) in enumerate(SHAPES)]


def batch_of(cs, load_init=True, **kw):
    probs = [dict(m=c["M"].shape[0], n_i=c["n_i"], r=c["r"], rho=c["rho"], lam=c["lam"])
             for c in cs]
    b = dcf.Batch(probs, **kw)
    for q, c in enumerate(cs):
        b.load(q, c["M"])
        if load_init:
            b.load_init(q, c["U0"], c["V0"])
    return b


def test_one_step_matches_oracle():
    cs = cases()
    b = batch_of(cs)
    b.step(1)
    for q, c in enumerate(cs):
        U, V = b.factors(q)
        U1, V1, S1, _, _ = O.dcf_run(c["M"], c["n_i"], c["U0"], c["V0"], c["rho"], c["lam"], 1)
        assert rel(U, U1) <= 1e-4, (q, rel(U, U1))
        assert rel(V, V1) <= 1e-4, (q, rel(V, V1))
    b.close()


def test_several_steps_match_oracle_and_single_handles():
    cs = cases(seed0=5)
    b = batch_of(cs)
    b.step(6)
    for q, c in enumerate(cs):
        U, V = b.factors(q)
        U6, V6, _, _, _ = O.dcf_run(c["M"], c["n_i"], c["U0"], c["V0"], c["rho"], c["lam"], 6)
        L = U.astype(np.float64) @ V.T.astype(np.float64)
        L6 = U6 @ V6.T
        assert rel(L, L6) <= 1e-3, (q, rel(L, L6))
        s = dcf.Solver(c["M"].shape[0], c["n_i"], c["r"], c["rho"], c["lam"],
                       path=dcf.PATH_GENERAL)
        s.load(c["M"])
        s.load_init(c["U0"], c["V0"])
        s.step(6)
        Us, Vs = s.factors()
        # same per-item arithmetic; only the column-split grouping of the P
        # partials may differ (the tuner's choice), so agreement is to rounding
        Ls = Us.astype(np.float64) @ Vs.T.astype(np.float64)
        assert rel(L, Ls) <= 1e-4, (q, rel(L, Ls))
        _, _, it = b.stats(q)
        assert it == 6
        s.close()
    b.close()


def test_solve_stops_each_instance_at_its_tolerance():
    cs = cases(seed0=9)
    b = batch_of(cs, max_iter=1500, tol=1e-5)
    its, nconv = b.solve()
    assert nconv == len(cs), [(q, b.stats(q)) for q in range(len(cs))]
    for q in range(len(cs)):
        _, dL, it = b.stats(q)
        assert dL <= 1e-5
        assert it == its[q] and it >= 1
    # stopped instances stay where they stopped
    U_before = [b.factors(q)[0] for q in range(len(cs))]
    b.step(2)
    for q in range(len(cs)):
        assert np.array_equal(b.factors(q)[0], U_before[q])
    # the converged point agrees with the oracle's solve to the 1e-3 bar on L
    c = cs[1]
    U, V = b.factors(1)
    Uo, Vo, _, _ = O.dcf_solve(c["M"], c["n_i"], c["U0"], c["V0"], c["rho"], c["lam"], 400,
                               1e-5)[:4]
    L = U.astype(np.float64) @ V.T.astype(np.float64)
    assert rel(L, Uo @ Vo.T) <= 1e-3
    b.close()


def test_default_start_point_and_tuner():
    cs = cases(seed0=3)
    b = batch_of(cs, load_init=False, seed=11)
    report = b.tune(reps=2)
    assert "chosen" in report
    b.step(3)
    for q in range(len(cs)):
        o, dL, it = b.stats(q)
        assert it == 3 and np.isfinite(o) and np.isfinite(dL)
    b.close()


def test_errors():
    c = make_case(64, [30, 30], 4, seed=1)
    with pytest.raises(dcf.DcfError) as e:
        dcf.Batch([dict(m=64, n_i=[30, 30], r=40, rho=1e-2, lam=0.1)])
    assert e.value.status == dcf.DCF_EINVAL
    b = dcf.Batch([dict(m=64, n_i=[30, 30], r=4, rho=1e-2, lam=0.1)] * 2)
    b.load(0, c["M"])
    with pytest.raises(dcf.DcfError) as e:
        b.step(1)                      # instance 1 has no M
    assert e.value.status == dcf.DCF_ESTATE
    with pytest.raises(dcf.DcfError) as e:
        b.load(5, c["M"])
    assert e.value.status == dcf.DCF_EINVAL
    b.close()


def test_more_problems_than_clusters():
    """400 problems of 64 rows need three waves of the tensor-core kernel (one
    cluster each, 152 clusters per launch on this GPU)."""
    cs = [make_case(64, [40, 30], 4, seed=500 + q, density=0.05, amp=5.0) for q in range(400)]
    b = batch_of(cs)
    b.step(2)
    for q in (0, 151, 152, 303, 399):
        c = cs[q]
        U, V = b.factors(q)
        U2, V2, _, _, _ = O.dcf_run(c["M"], c["n_i"], c["U0"], c["V0"], c["rho"], c["lam"], 2)
        L = U.astype(np.float64) @ V.T.astype(np.float64)
        assert rel(L, U2 @ V2.T) <= 1e-4, (q, rel(L, U2 @ V2.T))
    b.close()


def collinear_instance(m, n_i, r, eps, rho, seed):
    """An instance whose U0 has two nearly collinear columns (the second within
    eps of the first, relative), so that U0^T U0 + rho I is ill-conditioned."""
    c = make_case(m, n_i, r, seed=seed, rho=rho, density=0.05, amp=5.0)
    U0 = c["U0"].astype(np.float64)
    g = np.random.default_rng(seed + 2)
    U0[:, 1] = U0[:, 0] + eps * g.standard_normal(m) / np.sqrt(m)
    c["U0"] = U0.astype(np.float32)
    c["V0"] = O.init_v0(c["M"], c["U0"].astype(np.float64), rho).astype(np.float32)
    G = c["U0"].astype(np.float64).T @ c["U0"].astype(np.float64) + rho * np.eye(r)
    return c, float(np.linalg.cond(G, 1))


def test_ill_conditioned_instances_take_the_double_float_route():
    """Ill-conditioned instances next to a well-conditioned one in one batch:
    the batched tails, Grams, rows and images switch to the compensated route
    per instance (from the instance's own condition estimate) and every
    instance still meets 1e-4 after one step."""
    specs = [((300, [100, 76, 140], 8), 1e-3, 1e-6),     # tensor-core table mode, R = 8
             ((257, [200, 99], 12), 1e-3, 1e-6),         # R = 16
             ((520, [180, 190], 24), 1e-2, 1e-6),        # R = 32
             ((4100, [150, 170], 6), 1e-3, 1e-6)]        # general passes
    cs, kaps = [], []
    for q, (shape, eps, rho) in enumerate(specs):
        c, k = collinear_instance(*shape, eps, rho, seed=40 + q)
        cs.append(c)
        kaps.append(k)
    cs.append(make_case(200, [50, 50, 50, 50], 5, seed=7, density=0.05, amp=5.0))
    kaps.append(None)
    b = batch_of(cs)
    b.step(1)
    for q, c in enumerate(cs):
        U, V = b.factors(q)
        U1, V1, _, _, _ = O.dcf_run(c["M"], c["n_i"], c["U0"], c["V0"], c["rho"], c["lam"], 1)
        print(f"\ninstance {q}: kappa_1(U0^T U0 + rho I) {kaps[q] if kaps[q] else 0:.2e}: "
              f"rel err U {rel(U, U1):.2e}, V {rel(V, V1):.2e}")
        assert rel(U, U1) <= 1e-4, (q, rel(U, U1))
        assert rel(V, V1) <= 1e-4, (q, rel(V, V1))
    b.close()
