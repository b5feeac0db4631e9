"""Parity at the full sizes of the benchmark workloads, in the launch
configuration that bench.py times (path chosen automatically, M borrowed from
a torch CUDA tensor, graph-launched steps; the batched problems tuned and
stepped together; the learned network with its trained parameters).

Where the FP64 oracle finishes the whole output in seconds it checks all of
it (medium workload, learned network).  Elsewhere it checks sampled outputs
that it computes one by one: the V-step is separable by columns (§2.2, App. B
eq. condition1) and the U-step by rows once every V_i is known (App. B), so
the oracle's own s_step / v_step / u_step_exact run on column and row subsets.
Tolerances as in test_gpu_parity: 1e-4 relative Frobenius on U, V and S after
one step, 1e-3 on L after several.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from oracle import unrolled as UN
from paper_2207_11669_gb300 import dcf, synth
from tests.helpers import rel

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_11669_gb300 import build
    build.build()
    torch.cuda.init()


def borrowed(M):
    import torch
    return torch.from_numpy(np.ascontiguousarray(M.T)).cuda()     # (n, m): M column-major


def test_medium_workload_full_output():
    """m = 4096, n = 65536 in 16 uneven blocks, r = 32: every entry of U, V after
    one step, S of the first and last block, and L after three steps."""
    import torch
    wl = synth.workload_medium()
    inst = wl.instance()
    M, n_i = inst.M, inst.n_i
    U0 = synth.gaussian_u0(wl.m, wl.r, wl.seed)
    V0 = O.init_v0(M, U0.astype(np.float64), wl.rho).astype(np.float32)
    Mt = borrowed(M)
    stream = torch.cuda.current_stream()
    s = dcf.Solver(wl.m, n_i, wl.r, wl.rho, wl.lam, max_iter=wl.iters, tol=0.0,
                   stream=stream.cuda_stream)
    s.load(Mt)
    s.load_init(U0, V0)
    assert s.path == dcf.PATH_FUSED
    s.step(1)
    U, V = s.factors()
    off = O.block_offsets(n_i)
    S_first = s.LS(0)[1]
    S_last = s.LS(len(n_i) - 1)[1]
    s.step(2)
    U3, V3 = s.factors()
    s.close()
    del Mt

    seen = {}

    def keep(t, Ut, Vt, St):
        if t == 0:
            seen["U"], seen["V"] = Ut, Vt
            seen["S0"] = St[:, off[0]:off[1]].copy()
            seen["S1"] = St[:, off[-2]:off[-1]].copy()

    Uo, Vo, _, _, _ = O.dcf_run(M, n_i, U0, V0, wl.rho, wl.lam, 3, callback=keep)
    assert rel(U, seen["U"]) <= 1e-4
    assert rel(V, seen["V"]) <= 1e-4
    assert rel(S_first, seen["S0"]) <= 1e-4
    assert rel(S_last, seen["S1"]) <= 1e-4
    L_gpu = U3.astype(np.float64) @ V3.T.astype(np.float64)
    assert rel(L_gpu, Uo @ Vo.T) <= 1e-3


def test_large_workload_sampled_columns_and_rows():
    """m = 16384, n = 262144 in 64 uneven blocks, r = 64 (the two-pass tensor-core
    path).  After one step: V' on three whole blocks, 1024 random columns and the
    last strip, against the oracle's S- and V-steps on those columns; U on 64
    rows (slab edges among them) against the oracle's exact U-step of those rows,
    with the oracle's S of those rows and the step's V'."""
    import torch
    wl = synth.workload_large()
    inst = wl.instance()
    M, n_i = inst.M, inst.n_i
    m, n, r = wl.m, wl.n, wl.r
    U0 = synth.gaussian_u0(m, r, wl.seed)
    g = np.random.default_rng(wl.seed + 11)
    V0 = (g.standard_normal((n, r)) * wl.factor_std).astype(np.float32)
    Mt = borrowed(M)
    stream = torch.cuda.current_stream()
    s = dcf.Solver(m, n_i, r, wl.rho, wl.lam, max_iter=wl.iters, tol=0.0,
                   stream=stream.cuda_stream)
    s.load(Mt)
    s.load_init(U0, V0)
    assert s.path == dcf.PATH_TC2
    s.step(1)
    U, V = s.factors()
    s.close()
    del Mt
    torch.cuda.empty_cache()

    off = O.block_offsets(n_i)
    blocks = [0, len(n_i) // 2, len(n_i) - 1]
    cols = np.unique(np.concatenate(
        [np.arange(off[b], off[b + 1]) for b in blocks]
        + [g.choice(n, 1024, replace=False), np.arange(n - 128, n)]))
    Mc = M[:, cols]
    Sc = O.s_step(Mc, U0, V0[cols], wl.lam)
    Vc = O.v_step(Mc, Sc, U0, wl.rho)
    assert rel(V[cols], Vc) <= 1e-4

    rows = np.unique(np.concatenate([[0, 255, 256, 4095, 4096, m - 256, m - 1],
                                     g.choice(m, 57, replace=False)]))
    Mr = np.ascontiguousarray(M[rows, :])
    Sr = O.s_step(Mr, U0[rows], V0, wl.lam)
    Ur = O.u_step_exact([Mr], [Sr], [V], wl.rho)
    assert rel(U[rows], Ur) <= 1e-4


def test_batched_workload_sampled_instances():
    """All 512 problems of the batched workload loaded, tuned and stepped
    together; two problems of every (padded rank, cluster size) group, the
    largest, the smallest and the last one start from oracle start points and
    are checked after one step."""
    import torch
    shapes = synth.batched_instance_shapes(512, seed=synth.SEED_BASE + 2)
    probs = [dict(m=sh["m"], n_i=sh["n_i"], r=sh["r"], rho=sh["rho"], lam=sh["lam"])
             for sh in shapes]

    def group(sh):
        R = 16 if sh["r"] <= 16 else 32
        slabs = ((sh["m"] + 3) // 4 * 4 + 255) // 256
        return R, 2 if slabs <= 2 else 4

    picks = {}
    for q, sh in enumerate(shapes):
        lst = picks.setdefault(group(sh), [])
        if len(lst) < 2:
            lst.append(q)
    size = [sh["m"] * sh["n"] for sh in shapes]
    sample = sorted(set(sum(picks.values(), []) + [int(np.argmax(size)), int(np.argmin(size)),
                                                   len(shapes) - 1]))
    assert len(picks) == 4

    def instance(sh):
        return synth.make_instance(sh["m"], sh["n"], sh["k"], seed=sh["seed"],
                                   density=sh["density"], amp=sh["amp"],
                                   factor_std=sh["factor_std"], n_i=sh["n_i"])

    stream = torch.cuda.current_stream()
    b = dcf.Batch(probs, max_iter=1000, tol=0.0, seed=7, stream=stream.cuda_stream)
    starts = {}
    for q, sh in enumerate(shapes):
        inst = instance(sh)
        Mt = borrowed(inst.M)
        b.load(q, Mt)
        if q in sample:
            U0 = synth.gaussian_u0(sh["m"], sh["r"], sh["seed"])
            V0 = O.init_v0(inst.M, U0.astype(np.float64), sh["rho"]).astype(np.float32)
            b.load_init(q, U0, V0)
            starts[q] = (U0, V0)
        torch.cuda.synchronize()
        del Mt
    b.tune(reps=3)
    b.step(1)
    for q in sample:
        sh = shapes[q]
        U, V = b.factors(q)
        U0, V0 = starts[q]
        U1, V1, _, _, _ = O.dcf_run(instance(sh).M, sh["n_i"], U0, V0, sh["rho"], sh["lam"], 1)
        assert rel(U, U1) <= 1e-4, (q, group(sh), rel(U, U1))
        assert rel(V, V1) <= 1e-4, (q, group(sh), rel(V, V1))
    b.close()


def test_learned_workload_full_size_forward_and_adjoint():
    """The learned network at its workload's size (m = 1024, n = 16384 in 8
    blocks, r = 16) with the trained parameters (K = 10): loss terms, final
    factors and every gradient against the oracle's unrolled forward and
    adjoint.  Tolerances as in test_gpu_unrolled."""
    import torch
    with open(os.path.join(ROOT, "paper_2207_11669_gb300", "learned_theta.json")) as f:
        th = json.load(f)
    theta = (np.array(th["a"]), np.array(th["b"]), np.array(th["c"]))
    K = len(theta[0])
    inst = synth.learned_instance(0, "test")
    m, n = inst.M.shape
    r, rho, lam = 16, synth.LEARNED_RHO, synth.LEARNED_LAMBDA
    U0 = synth.gaussian_u0(m, r, 7000 + 100000)
    V0 = O.init_v0(inst.M, U0.astype(np.float64), rho).astype(np.float32)
    Mt = borrowed(inst.M)
    stream = torch.cuda.current_stream()
    s = dcf.Solver(m, inst.n_i, r, rho, lam, stream=stream.cuda_stream)
    s.load(Mt)
    s.load_init(U0, V0)
    s.set_truth(inst.A, inst.B)
    tot, terms = s.unrolled_forward(*theta)
    U, V = s.factors()
    ga, gb, gc, gU, gV = s.unrolled_backward(K, start_grads=True)
    s.close()
    del Mt

    loss, traj = UN.unrolled_forward(inst.M, U0.astype(np.float64), V0.astype(np.float64),
                                     inst.A, inst.B, lam, rho, theta)
    (oa, ob, oc), (oU, oV) = UN.unrolled_backward(inst.M, traj, inst.A, inst.B, lam, rho, theta)
    oterms = np.array([UN.factor_loss(Ut, Vt, inst.A, inst.B) for (Ut, Vt) in traj[1:]])
    assert abs(tot - loss) <= 1e-3 * loss
    assert np.all(np.abs(terms - oterms) <= 1e-3 * oterms)
    assert rel(U, traj[-1][0]) <= 1e-3
    assert rel(V, traj[-1][1]) <= 1e-3
    assert rel(ga, oa) <= 2e-3, (ga, oa)
    assert rel(gb, ob) <= 2e-3, (gb, ob)
    assert rel(gc, oc) <= 2e-3, (gc, oc)
    assert rel(gU, oU) <= 2e-3
    assert rel(gV, oV) <= 2e-3
