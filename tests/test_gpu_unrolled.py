"""Parity of the GPU learned unrolled network and its adjoint with the FP64 oracle.

Tolerances.  The forward pass runs the plain FP32 iteration kernels, whose one-step
error is below 1e-4 (relative Frobenius); over K = 4 steps the factors stay
within 1e-3 of the oracle's trajectory.  The loss is a relative squared error
evaluated from FP64 Grams of FP32 factors: relative 1e-3 (loss values here are
1e-3 .. 1e-1).  Gradients are FP32 streams with FP64 r x r algebra: relative
2e-3 in norm per parameter vector and for the start-point gradients.  Entries
of R within the FP32 rounding of R of a threshold may take the other branch of
the clamp; the instances below have margins well above that bound.
"""
import numpy as np
import pytest

from oracle import unrolled as UN
from paper_2207_11669_gb300 import dcf
from tests.helpers import make_case, rel

pytestmark = pytest.mark.gpu

K = 4
CASES = [
    # (m, n_i, r, k_truth)
    (200, [50, 50, 50, 50], 5, 5),
    (300, [100, 77, 140], 16, 12),
    (128, [33, 64, 31], 32, 20),
    (64, [10, 9, 11], 8, 3),
    # m not a multiple of 4 (4-byte copies of M in the adjoint kernels; general
    # path only) and column splits of several 32-column chunks
    (130, [2600, 2403], 12, 6),
]
PATHS = [dcf.PATH_GENERAL, dcf.PATH_FUSED]


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


def theta_of(seed, K=K):
    g = np.random.default_rng(seed)
    return (g.uniform(-0.3, 0.3, K), g.uniform(-0.5, 0.5, K), g.uniform(0.7, 1.3, K))


def case_of(m, n_i, r, k):
    return make_case(m, n_i, r, seed=1000 + m + r, k=k, density=0.05, amp=5.0,
                     lam=2.0 / np.sqrt(m))


def solver_of(case, path):
    s = dcf.Solver(case["M"].shape[0], case["n_i"], case["r"], case["rho"], case["lam"],
                   path=path)
    s.load(case["M"])
    s.load_init(case["U0"], case["V0"])
    s.set_truth(case["inst"].A, case["inst"].B)
    return s


def oracle_run(case, theta):
    inst = case["inst"]
    U0 = case["U0"].astype(np.float64)
    V0 = case["V0"].astype(np.float64)
    loss, traj = UN.unrolled_forward(inst.M, U0, V0, inst.A, inst.B, case["lam"], case["rho"],
                                     theta)
    grads, start = UN.unrolled_backward(inst.M, traj, inst.A, inst.B, case["lam"], case["rho"],
                                        theta)
    terms = [UN.factor_loss(U, V, inst.A, inst.B) for (U, V) in traj[1:]]
    return loss, np.array(terms), traj, grads, start


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("m,n_i,r,k", CASES)
def test_forward_and_adjoint_match_oracle(m, n_i, r, k, path):
    if path == dcf.PATH_FUSED and not fused_ok(m, r):
        pytest.skip("shape outside the fused path")
    case = case_of(m, n_i, r, k)
    theta = theta_of(m + r)
    s = solver_of(case, path)
    tot, terms = s.unrolled_forward(*theta)
    U, V = s.factors()
    ga, gb, gc, gU, gV = s.unrolled_backward(K, start_grads=True)
    loss, oterms, traj, (oa, ob, oc), (oU, oV) = oracle_run(case, theta)
    assert abs(tot - loss) <= 1e-3 * loss
    assert np.all(np.abs(terms - oterms) <= 1e-3 * oterms)
    assert rel(U, traj[-1][0]) <= 1e-3
    assert rel(V, traj[-1][1]) <= 1e-3
    assert rel(ga, oa) <= 2e-3, (ga, oa)
    assert rel(gb, ob) <= 2e-3, (gb, ob)
    assert rel(gc, oc) <= 2e-3, (gc, oc)
    assert rel(gU, oU) <= 2e-3
    assert rel(gV, oV) <= 2e-3
    s.close()


@pytest.mark.parametrize("path", PATHS)
def test_untrained_network_is_plain_steps(path):
    m, n_i, r, k = CASES[1]
    case = case_of(m, n_i, r, k)
    if path == dcf.PATH_FUSED and not fused_ok(m, r):
        pytest.skip("shape outside the fused path")
    s1 = solver_of(case, path)
    s1.unrolled_forward(np.zeros(K), np.zeros(K), np.ones(K), want_loss=False)
    s2 = solver_of(case, path)
    s2.step(K)
    U1, V1 = s1.factors()
    U2, V2 = s2.factors()
    # same kernels, same order, same (U^T U + rho I)^{-1}: identical bits
    assert np.array_equal(U1, U2)
    assert np.array_equal(V1, V2)
    s1.close()
    s2.close()


def test_plain_refinement_after_forward():
    """After the network, dcf_step continues with the plain lambda and rho."""
    m, n_i, r, k = CASES[0]
    case = case_of(m, n_i, r, k)
    theta = theta_of(7)
    s = solver_of(case, dcf.PATH_GENERAL)
    s.unrolled_forward(*theta)
    s.step(3)
    U, V = s.factors()
    _, _, traj, _, _ = oracle_run(case, theta)
    import oracle as O
    U3, V3, _, _, _ = O.dcf_run(case["M"], case["n_i"], traj[-1][0], traj[-1][1], case["rho"],
                                case["lam"], 3)
    assert rel(U, U3) <= 1e-3
    assert rel(V, V3) <= 1e-3
    s.close()


def test_loss_terms_agree_with_rel_err():
    m, n_i, r, k = CASES[0]
    case = case_of(m, n_i, r, k)
    s = solver_of(case, dcf.PATH_GENERAL)
    _, terms = s.unrolled_forward(*theta_of(11))
    assert abs(np.sqrt(terms[-1]) - s.rel_err()) <= 1e-5 + 1e-4 * s.rel_err()
    s.close()


def test_errors():
    m, n_i, r, k = CASES[0]
    case = case_of(m, n_i, r, k)
    s = dcf.Solver(m, n_i, r, case["rho"], case["lam"])
    s.load(case["M"])
    with pytest.raises(dcf.DcfError) as e:
        s.unrolled_backward(K)
    assert e.value.status == dcf.DCF_ESTATE
    with pytest.raises(dcf.DcfError) as e:
        s.unrolled_forward(*theta_of(1))          # a loss without truth factors
    assert e.value.status == dcf.DCF_ESTATE
    s.unrolled_forward(*theta_of(1), want_loss=False)
    with pytest.raises(dcf.DcfError) as e:
        s.unrolled_backward(K)                    # forward ran without the loss
    assert e.value.status == dcf.DCF_ESTATE
    with pytest.raises(dcf.DcfError) as e:
        s.unrolled_forward(np.array([np.nan] * K), np.zeros(K), np.ones(K), want_loss=False)
    assert e.value.status == dcf.DCF_EINVAL
    s.close()
    s = dcf.Solver(m, n_i, r, case["rho"], case["lam"], u_mode=1, eta0=0.1)
    s.load(case["M"])
    with pytest.raises(dcf.DcfError) as e:
        s.unrolled_forward(*theta_of(1), want_loss=False)
    assert e.value.status == dcf.DCF_EINVAL
    s.close()
    big = make_case(96, [40, 40], 40, seed=5)
    s = dcf.Solver(96, [40, 40], 40, big["rho"], big["lam"])
    s.load(big["M"])
    with pytest.raises(dcf.DcfError) as e:
        s.unrolled_forward(*theta_of(1), want_loss=False)
    assert e.value.status == dcf.DCF_EINVAL
    s.close()


def test_training_lowers_the_loss():
    """A few Adam steps on GPU gradients lower the network's loss."""
    import torch
    from paper_2207_11669_gb300.unrolled import UnrolledDCF, train
    probs = []
    for seed in range(3):
        case = make_case(256, [128, 128, 128, 128], 8, seed=50 + seed, k=8, density=0.05,
                         amp=5.0, lam=2.0 / 16)
        s = solver_of(case, dcf.PATH_GENERAL)
        probs.append((s, (case["U0"], case["V0"])))
    net = UnrolledDCF(3)
    hist = train(net, probs, steps=15, lr=0.1)
    assert hist[-1] < 0.9 * hist[0], hist
    for s, _ in probs:
        s.close()


def test_trained_network_reaches_the_fixed_point_in_fewer_steps():
    """The committed parameters (trained on the GPU by train_unrolled) on a
    held-out problem of their workload: K network steps plus plain refinement
    reach 1e-4 of the plain method's fixed point in fewer total iterations than
    the plain iteration alone, and the untrained network gains nothing."""
    import json
    import os
    import torch
    from paper_2207_11669_gb300 import synth
    from paper_2207_11669_gb300.unrolled import fixed_point, steps_to_tolerance
    path = os.path.join(os.path.dirname(dcf.__file__), "learned_theta.json")
    th = json.load(open(path))
    theta = (np.array(th["a"]), np.array(th["b"]), np.array(th["c"]))
    Kn = th["K"]
    inst = synth.learned_instance(7, "test")
    m, n = inst.M.shape
    U0 = synth.gaussian_u0(m, 16, 123456)
    Mt = torch.from_numpy(np.ascontiguousarray(inst.M.T)).cuda()
    s = dcf.Solver(m, inst.n_i, 16, synth.LEARNED_RHO, synth.LEARNED_LAMBDA)
    s.load(Mt)
    Uf, Vf = fixed_point(s, U0, 1500)
    s.set_truth(Uf, Vf)
    n_plain = steps_to_tolerance(s, U0, 1e-4, 1000)
    n_ref = steps_to_tolerance(s, U0, 1e-4, 1000, theta)
    n_untrained = steps_to_tolerance(s, U0, 1e-4, 1000,
                                     (np.zeros(Kn), np.zeros(Kn), np.ones(Kn)))
    assert n_plain <= 1000
    assert Kn + n_ref < n_plain, (Kn, n_ref, n_plain)
    assert Kn + n_untrained >= n_plain - 1        # K plain steps are just plain steps
    s.close()
