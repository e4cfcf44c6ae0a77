"""Training and evaluation of the learned setup (the gauge-covariant
parallel-transport network of the C-ABI's mg_nn_* calls) on an ensemble of
seeded quenched fields.

Ensemble: a Markov chain of the heatbath (1 Kennedy-Pendleton heatbath + 4
over-relaxation per compound sweep, beta = 6.0) started from the thermalised
16^3 x 32 field of the benchmark, `spacing` compound sweeps between members,
each member's sweeps seeded by its index; members 0..n_train-1 train, the
rest are held out.

Training: for every training member the plain adaptive setup (Sec. IV) runs at
the setup mass and the network takes `steps` Adam steps against that setup's
block projector, for `rounds` passes over the members (the network never sees
a held-out field).  Evaluation on a held-out member: the plain setup and the
learned setup (network prototypes + `refine` group-refinement iterations)
are timed, each then solves at the lightest mass, and the two-grid rate of
each coarse space is measured.

Usage (one GPU):
    python -m paper_1005_3043_gb300.learned_setup train  -> writes WEIGHTS
    python -m paper_1005_3043_gb300.learned_setup eval
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "learned_setup_16x16x16x32_nv20.npy")


def ensemble(w, n, spacing=10, seed0=7000):
    """Yield n members (links) of the chain started from the workload's field."""
    import synth
    U = synth.gauge_field(w.dims, beta=w.beta, sweeps=w.sweeps, n_or=w.n_or, seed=w.seed).copy()
    for k in range(n):
        for s in range(spacing):
            synth.gauge_sweep(U, w.dims, w.beta, w.n_or, seed0 + k, s)
        yield k, U.copy()


def starts(w, n, seed):
    import synth
    return np.stack([synth.gaussian_spinor(w.dims, seed, stream=i) for i in range(n)])


def init_weights(seed):
    """Seeded initial weights: the on-site identity on the first channel of
    every layer plus small Gaussian entries (numpy Generator)."""
    rng = np.random.default_rng(seed)
    ch = (1, 8, 8, 8, 1)
    Ws = []
    for ci, co in zip(ch[:-1], ch[1:]):
        s = 0.3 / np.sqrt(9 * ci)
        W = s * (rng.standard_normal((co, ci, 9, 4, 4)) + 1j * rng.standard_normal((co, ci, 9, 4, 4)))
        for a in range(co):
            for b in range(ci):
                if a % ci == b or ci == 1:
                    W[a, b, 0] += np.eye(4) / max(ci, 1) ** 0.5
        Ws.append(W)
    return Ws


def make_params(wmg, w, prec="fp16"):
    p = wmg.mg_default_params()
    for i in range(4):
        p.block[i] = w.block[i]
    p.nvec = w.nvec
    p.setup_group, p.setup_iters, p.setup_init_relax = 4, 5, 10
    p.gcr_restart, p.tol, p.max_outer = 16, 1e-10, 4000
    p.smoother, p.smoother_steps = w.extra.get("smoother", 0), w.extra.get("smoother_steps", 4)
    p.prec_inner = {"fp32": wmg.MG_FP32, "fp16": wmg.MG_FP16, "fp64": wmg.MG_FP64}[prec]
    p.delta = 1e-4
    return p


def train(n_train=32, rounds=2, steps=20, n_starts=4, lr=2e-3, seed=11, out=WEIGHTS, log=print):
    import torch
    import paper_1005_3043_gb300 as wmg
    import synth
    from paper_1005_3043_gb300.workloads import WORKLOADS
    w = WORKLOADS["wilson_16x16x16x32_nv20_beta6_5mass"]
    wmg.build.build()
    wmg.load()
    V0 = synth.gaussian_vectors(w.dims, w.nvec, w.setup_seed)
    eta = starts(w, n_starts, 9100)
    members = list(ensemble(w, n_train))
    mg = wmg.WilsonMG(w.dims, make_params(wmg, w), stream=torch.cuda.current_stream())
    mg.nn_set_weights(init_weights(seed))
    hist = []
    t0 = time.time()
    for r in range(rounds):
        for k, U in members:
            mg.set_links(U)
            mg.set_mass(w.setup_mass())
            mg.setup(V0)
            l0, l1 = mg.nn_train(eta, steps, lr)
            hist.append((r, k, l0, l1))
            log(f"round {r} member {k}: loss {l0:.4f} -> {l1:.4f} ({time.time() - t0:.0f} s)")
    Ws = mg.nn_get_weights()
    mg.close()
    np.save(out, wmg.nn_flatten(Ws))
    return hist


def two_grid_rate(wmg, mg, w, iters=16, seed=9300):
    """Asymptotic rate of the two-grid iteration e <- e - M D e (eq. 3) with
    the library's V-cycle as M (MR(4) smoother, coarse CGNR to 1e-5 standing in
    for the exact coarse solve) and its FP64 operator as D, over the second
    half of `iters` iterations."""
    import synth
    p = mg.params
    q = wmg.MgParams.from_buffer_copy(p)
    q.smoother, q.smoother_steps, q.coarse_tol, q.max_coarse = 0, 4, 1e-5, 20000
    mg.set_params(q)
    e = synth.gaussian_spinor(w.dims, seed)
    norms = [np.linalg.norm(e)]
    for _ in range(iters):
        e = e - mg.vcycle(mg.dslash(e, wmg.MG_FP64), wmg.MG_FP32)
        norms.append(np.linalg.norm(e))
    mg.set_params(p)
    h = iters // 2
    return float((norms[iters] / norms[h]) ** (1.0 / (iters - h)))


def evaluate(n_train=32, n_eval=16, refine=(0, 1, 2), weights=WEIGHTS, with_rate=True, log=print):
    """Setups compared on held-out members n_train .. n_train + n_eval - 1 at the
    lightest mass: "plain" (random starts, 10 relaxations, 5 refinement
    iterations: the Sec. IV schedule), "plain_r{r}" (random starts, 10
    relaxations, r iterations), "learned_r{r}" (network prototypes, no
    relaxation, r iterations) and "learned_relax_r{r}" (network prototypes,
    10 relaxations, r iterations).  Per setup: its device time, the outer
    iterations and time of one solve, and the two-grid rate."""
    import torch
    import paper_1005_3043_gb300 as wmg
    import synth
    from paper_1005_3043_gb300.workloads import WORKLOADS
    w = WORKLOADS["wilson_16x16x16x32_nv20_beta6_5mass"]
    wmg.build.build()
    wmg.load()
    V0 = synth.gaussian_vectors(w.dims, w.nvec, w.setup_seed)
    eta = starts(w, w.nvec, 9200)
    b = synth.gaussian_spinor(w.dims, w.source_seed, stream=0)
    m = w.masses()[-1]
    st = torch.cuda.current_stream()
    base = make_params(wmg, w)
    mg = wmg.WilsonMG(w.dims, base, stream=st)
    mg.nn_set_weights(wmg.nn_unflatten(np.load(weights)))
    variants = [("plain", False, 10, 5)] + [(f"plain_r{r}", False, 10, r) for r in refine] + \
               [(f"learned_r{r}", True, 0, r) for r in refine] + [(f"learned_relax_r{r}", True, 10, r) for r in refine]
    rows = []
    for k, U in ensemble(w, n_train + n_eval):
        if k < n_train:
            continue
        mg.set_links(U)
        row = {"member": k}
        for name, learned, relax, iters in variants:
            p = wmg.MgParams.from_buffer_copy(base)
            p.setup_init_relax, p.setup_iters = relax, iters
            mg.set_params(p)
            mg.set_mass(w.setup_mass())
            if learned:
                mg.setup_learned(eta, refine_iters=iters)
            else:
                mg.setup(V0)
            mg.set_mass(m)
            x, info = mg.solve(b)
            row[name] = {"setup_ms": info["setup_ms"], "outer_iters": info["outer_iters"], "status": info["status"],
                         "solve_ms": info["solve_ms"], "true_rel_res": info["true_rel_res"]}
            if with_rate:
                row[name]["two_grid_rate"] = two_grid_rate(wmg, mg, w)
        mg.set_params(base)
        rows.append(row)
        log(json.dumps(row))
    mg.close()
    return rows


if __name__ == "__main__":
    if sys.argv[1] == "train":
        train()
    elif sys.argv[1] == "eval":
        evaluate()
