"""Train the parameters of the learned unrolled network on generated problems.

The network (K steps with per-step lambda_k = lambda e^{a_k}, rho_k = rho e^{b_k}
and relaxation c_k) is trained on the GPU with the library's forward and
hand-written reverse pass (``UnrolledLoss``).  Its target on each problem is
the plain method's fixed point (the plain iteration run to convergence), so
that the network is a fast proposal that the plain iteration then finishes.

    python -m paper_2207_11669_gb300.train_unrolled --out theta.json

writes {"K", "a", "b", "c", "loss_history", ...}.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import dcf, synth
from .unrolled import UnrolledDCF, fixed_point, train


def make_problems(count, split, fp_iters, stream):
    probs = []
    for q in range(count):
        inst = synth.learned_instance(q, split)
        m, n = inst.M.shape
        U0 = synth.gaussian_u0(m, 16, 7000 + q + (0 if split == "train" else 100000))
        Mt = torch.from_numpy(np.ascontiguousarray(inst.M.T)).cuda()
        s = dcf.Solver(m, inst.n_i, 16, synth.LEARNED_RHO, synth.LEARNED_LAMBDA, stream=stream)
        s.load(Mt)
        Uf, Vf = fixed_point(s, U0, fp_iters)
        s.set_truth(Uf, Vf)
        probs.append((s, (U0, None), Mt))
    return probs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--problems", type=int, default=64)
    ap.add_argument("--per-step", type=int, default=64,
                    help="problems per Adam step (the batch of 64 of the learned workload)")
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--lr", type=float, default=0.05)
    ap.add_argument("--fp-iters", type=int, default=1500)
    args = ap.parse_args()
    torch.cuda.init()
    stream = torch.cuda.current_stream().cuda_stream
    t0 = time.time()
    probs = make_problems(args.problems, "train", args.fp_iters, stream)
    t_setup = time.time() - t0
    net = UnrolledDCF(synth.LEARNED_K)
    opt = torch.optim.Adam(net.parameters(), lr=args.lr)
    hist = []
    t0 = time.time()
    rng = np.random.default_rng(0)
    step_s = []
    for it in range(args.steps):
        ts = time.time()
        pick = rng.choice(len(probs), size=min(args.per_step, len(probs)), replace=False)
        opt.zero_grad()
        total = 0.0
        for q in pick:
            s, start, _ = probs[q]
            loss = net(s, start) / len(pick)
            loss.backward()
            total += float(loss.detach())
        opt.step()
        torch.cuda.synchronize()
        step_s.append(time.time() - ts)
        hist.append(total)
        print(f"step {it}: loss {total:.4e} ({step_s[-1]:.3f} s)", flush=True)
    t_train = time.time() - t0
    a, b, c = net.theta()
    out = {"K": synth.LEARNED_K, "a": a.tolist(), "b": b.tolist(), "c": c.tolist(),
           "loss_history": hist, "problems": args.problems, "per_step": args.per_step,
           "adam_steps": args.steps, "lr": args.lr, "fixed_point_iters": args.fp_iters,
           "setup_s": t_setup, "train_s": t_train,
           "adam_step_s_median": float(np.median(step_s)),
           "workload": "m=1024, n=16384 (E=8), rank 16, density 0.10, values U[-10,10], "
                       "rho=1e-2, lambda=1/32"}
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)
    for s, _, _ in probs:
        s.close()


if __name__ == "__main__":
    main()
