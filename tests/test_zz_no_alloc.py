"""The allocation-free iteration (dcf_iterate_noalloc) against dcf_step.

Callers that cannot let a library allocate device memory (graph capture,
latency-critical loops, frameworks with their own pools) use this entry
point; it takes all scratch from a fixed array inside the library.  Two
calls in a row must reproduce two dcf_step iterations of the general path
from the same start, within the tolerance of the other parity tests.  This
file is collected last so that a failure here stops a -x run only after
every other test has run.
"""
import numpy as np
import pytest

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


def test_noalloc_matches_dcf_step_twice():
    import torch
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
    assert rel(Ub.cpu().numpy(), U1) <= 1e-4 and rel(Vb.cpu().numpy(), V1) <= 1e-4
    assert rel(Uc.cpu().numpy(), U2) <= 1e-4 and rel(Vc.cpu().numpy(), V2) <= 1e-4


def test_noalloc_rejects_problems_beyond_the_scratch_array():
    import torch
    dev = torch.device("cuda")
    t = torch.zeros(16, device=dev)
    # m = 4096, n = 65536, r = 32 needs far more than the fixed 16 MiB array
    st = dcf.dcf_iterate_noalloc(t, 4096, 65536, 32, 1e-2, 1 / 64, t, t, t, t, 0)
    assert st == dcf.DCF_EINVAL
