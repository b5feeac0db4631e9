"""The sparsity x rank sweep of §4.2 (the phase-transition figure) as one batch.

Every cell of the grid (truth rank r = 0.05n .. 0.2n, S* density s = 0.05 ..
0.3, m = n = 160 so that r = 0.2n stays within the batched path's rank 32) is
an independent problem of one dcf_batch, solved together to a relative
change of 1e-6 (at most 500 iterations).  Checks: the batch reproduces the
FP64 oracle run from the same start on sampled cells (the relative error of L
against the planted L* within 1e-3 where the method recovers L*, and a failed
recovery where the oracle fails); the easy corner (small r, small s) is
recovered and the hard corner (r = 0.2n, s = 0.3) is not, as in the figure.
"""
import numpy as np
import pytest

import oracle as O
from paper_2207_11669_gb300 import dcf, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_11669_gb300 import build
    build.build()


def start_point(cell):
    inst = synth.make_instance(cell["m"], cell["n"], cell["k"], seed=cell["seed"],
                               density=cell["density"], amp=cell["amp"],
                               factor_std=cell["factor_std"], n_i=cell["n_i"])
    U0 = synth.gaussian_u0(cell["m"], cell["r"], cell["seed"])
    V0 = O.init_v0(inst.M, U0.astype(np.float64), cell["rho"]).astype(np.float32)
    return inst, U0, V0


@pytest.fixture(scope="module")
def phase_run():
    cells = synth.phase_grid()
    probs = [dict(m=c["m"], n_i=c["n_i"], r=c["r"], rho=c["rho"], lam=c["lam"]) for c in cells]
    b = dcf.Batch(probs, max_iter=500, tol=1e-6, seed=3)
    insts = []
    for q, c in enumerate(cells):
        inst, U0, V0 = start_point(c)
        b.load(q, inst.M)
        b.load_init(q, U0, V0)
        insts.append((inst, U0, V0))
    its, nconv = b.solve()
    errs = []
    for q, (inst, _, _) in enumerate(insts):
        U, V = b.factors(q)
        errs.append(O.rel_err_L(U, V, inst.A, inst.B))
    b.close()
    return cells, insts, np.array(errs), its


def test_phase_corners(phase_run):
    cells, _, errs, _ = phase_run
    by = {(c["cell"][0], c["cell"][1]): e for c, e in zip(cells, errs)}
    assert by[(0.05, 0.05)] < 0.03
    assert by[(0.2, 0.3)] > 1.0
    table = "\n".join(
        f"r={ra:5.3f}n " + " ".join(f"{by[(ra, s)]:8.3f}" for s in synth.PHASE_DENSITIES)
        for ra in synth.PHASE_RANKS)
    print("\nrelative L error, rows r, columns s = "
          + " ".join(f"{s:.2f}" for s in synth.PHASE_DENSITIES) + "\n" + table)


@pytest.mark.parametrize("ratio,dens", [(0.05, 0.05), (0.1, 0.15), (0.05, 0.3), (0.2, 0.05)])
def test_phase_cells_match_oracle(phase_run, ratio, dens):
    cells, insts, errs, its = phase_run
    q = next(i for i, c in enumerate(cells) if c["cell"][:2] == (ratio, dens))
    c = cells[q]
    inst, U0, V0 = insts[q]
    Uo, Vo, _, it_o, _ = O.dcf_solve(inst.M, c["n_i"], U0, V0, c["rho"], c["lam"], 500, 1e-6)
    e_o = O.rel_err_L(Uo, Vo, inst.A, inst.B)
    if e_o < 0.2:
        assert abs(errs[q] - e_o) <= 1e-3 * max(e_o, 1e-2)
    else:
        assert errs[q] > 0.2
