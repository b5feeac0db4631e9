"""The allocation-free iteration (dcf_iterate_noalloc).

Some callers may not let a library allocate device memory: frameworks that
hand out all device memory from their own pools, and latency-critical loops
where cudaMalloc/cudaFree would synchronise the device.  For them this entry
point takes all scratch from a fixed array inside the library.  Two calls in a
row must reproduce two dcf_step iterations of the general path from the same
start, and the FP64 oracle's two rounds, within the tolerance of the other
parity tests (relative Frobenius error 1e-4).  The shared array keeps the
previous call's contents, so calls with a smaller rank after a larger one
(rank padding r < R) are checked against the oracle as well.  This file is
collected last so that a failure here stops a -x run only after every other
test has run.
"""
import numpy as np
import pytest

import oracle as O
from paper_2207_11669_gb300 import dcf
from tests.helpers import make_case, rel

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_11669_gb300 import build
    build.build()


def _two_noalloc_calls(case, m, n, r):
    """Two dcf_iterate_noalloc calls in a row on device copies of the case."""
    import torch
    dev = torch.device("cuda")
    Md = torch.from_numpy(np.ascontiguousarray(case["M"].T)).to(dev)   # column-major M
    Ua = torch.from_numpy(np.ascontiguousarray(case["U0"])).to(dev)
    Va = torch.from_numpy(np.ascontiguousarray(case["V0"])).to(dev)
    Ub, Vb = torch.empty_like(Ua), torch.empty_like(Va)
    Uc, Vc = torch.empty_like(Ua), torch.empty_like(Va)
    stream = torch.cuda.current_stream().cuda_stream
    assert dcf.dcf_iterate_noalloc(Md, m, n, r, case["rho"], case["lam"], Ua, Va, Ub, Vb,
                                   stream) == dcf.DCF_OK
    assert dcf.dcf_iterate_noalloc(Md, m, n, r, case["rho"], case["lam"], Ub, Vb, Uc, Vc,
                                   stream) == dcf.DCF_OK
    torch.cuda.synchronize()
    return (Ub.cpu().numpy(), Vb.cpu().numpy()), (Uc.cpu().numpy(), Vc.cpu().numpy())


def _oracle_two_rounds(case):
    U1, V1, _ = O.dcf_iteration(case["M"], case["n_i"], case["U0"], case["V0"],
                                case["rho"], case["lam"])
    U2, V2, _ = O.dcf_iteration(case["M"], case["n_i"], U1, V1, case["rho"], case["lam"])
    return (U1, V1), (U2, V2)


def test_noalloc_matches_dcf_step_twice():
    case = make_case(300, [100, 77, 140], 16, seed=31)
    m, n, r = 300, int(case["n_i"].sum()), 16
    ref = dcf.Solver(m, case["n_i"], r, case["rho"], case["lam"], path=dcf.PATH_GENERAL)
    ref.load(case["M"])
    ref.load_init(case["U0"], case["V0"])
    ref.step(1)
    U1, V1 = ref.factors()
    ref.step(1)
    U2, V2 = ref.factors()
    ref.close()
    (Ub, Vb), (Uc, Vc) = _two_noalloc_calls(case, m, n, r)
    assert rel(Ub, U1) <= TOL and rel(Vb, V1) <= TOL
    assert rel(Uc, U2) <= TOL and rel(Vc, V2) <= TOL
    (Uo1, Vo1), (Uo2, Vo2) = _oracle_two_rounds(case)
    assert rel(Ub, Uo1) <= TOL and rel(Vb, Vo1) <= TOL
    assert rel(Uc, Uo2) <= TOL and rel(Vc, Vo2) <= TOL


@pytest.mark.parametrize("m,n_i,r", [
    (300, [100, 77, 140], 16),    # R = 16, fills the rank: leaves the array dirty
    (257, [64, 99], 12),          # R = 16 with 4 zero-padded columns, after r = 16
    (131, [70, 61], 5),           # R = 8 with 3 padded columns
    (400, [200, 190], 32),        # R = 32 (one V-Gram CTA per SM)
    (211, [90, 45], 12),          # R = 16 again, after R = 32
])
def test_noalloc_matches_oracle_after_other_sizes(m, n_i, r):
    """Runs in the order listed, on the one shared array: each call must clear
    the padding and state the previous, differently sized call left behind."""
    case = make_case(m, n_i, r, seed=7 * m + r)
    n = int(np.sum(n_i))
    (Ub, Vb), (Uc, Vc) = _two_noalloc_calls(case, m, n, r)
    (Uo1, Vo1), (Uo2, Vo2) = _oracle_two_rounds(case)
    assert rel(Ub, Uo1) <= TOL and rel(Vb, Vo1) <= TOL
    assert rel(Uc, Uo2) <= TOL and rel(Vc, Vo2) <= TOL


def test_noalloc_rejects_problems_beyond_the_scratch_array():
    import torch
    dev = torch.device("cuda")
    t = torch.zeros(16, device=dev)
    # m = 4096, n = 65536, r = 32 needs far more than the fixed 16 MiB array
    st = dcf.dcf_iterate_noalloc(t, 4096, 65536, 32, 1e-2, 1 / 64, t, t, t, t, 0)
    assert st == dcf.DCF_EINVAL
