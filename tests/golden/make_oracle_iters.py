"""Work counts of the FP64 oracle on a workload: the oracle's adaptive setup at
the workload's setup mass, then one solve per mass of the sweep (the same
inputs as the benchmark step).  Recorded per solve: outer MG-GCR iterations,
coarse CG iterations and fine operator applications; for the setup: its fine
operator applications and coarse CG iterations (they depend on how good the
prototypes become, which only the whole setup shows).  The benchmark's CPU
baseline times the oracle's unit costs on the machine it runs on and scales
them by these counts.  Calls only oracle/ and synth/.

usage: python tests/golden/make_oracle_iters.py <workload name>
       -> tests/golden/<workload name>_oracle_iters.txt
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
import synth  # noqa: E402
from paper_1005_3043_gb300.workloads import WORKLOADS  # noqa: E402

SETUP_ITERS = {"wilson_8x8x8x8_nv8_beta6": 3}   # the 8^4 configuration's 3 sweeps; otherwise Sec. IV's 5


def smoother(w):
    """(smoother, steps) of the workload: 0 = MR steps, 1 = one GMRES(steps)."""
    return int(w.extra.get("smoother", 0)), int(w.extra.get("smoother_steps", 4))


def main(name):
    w = WORKLOADS[name]
    oracle.build()
    U = synth.gauge_field(w.dims, beta=w.beta, sweeps=w.sweeps, n_or=w.n_or, seed=w.seed)
    V0 = synth.gaussian_vectors(w.dims, w.nvec, w.setup_seed)
    t0 = time.time()
    sm, steps = smoother(w)
    po = oracle.make_params(w.dims, w.block, nv=w.nvec, m=w.setup_mass(), gcr_restart=16, tol=1e-10, max_outer=20000,
                            smoother=sm, mr_steps=steps)
    Vs, P, A, st, sinfo = oracle.setup_counted(po, U, V0, init_relax=10, n_iter=SETUP_ITERS.get(name, 5),
                                               group_size=4)
    assert st == 0
    t_setup = time.time() - t0
    print(f"setup {t_setup:.0f} s", flush=True)
    iters, rels, coarse, mvs = [], [], [], []
    for i, m in enumerate(w.masses()):
        b = synth.gaussian_spinor(w.dims, w.source_seed, stream=i)
        po = oracle.make_params(w.dims, w.block, nv=w.nvec, m=m, gcr_restart=16, tol=1e-10, max_outer=20000,
                                smoother=sm, mr_steps=steps)
        A_m = oracle.coarse_build(U, P, m, w.dims, w.block)
        t = time.time()
        x, info = oracle.gcr_solve(po, U, P, A_m, b)
        iters.append(int(info["outer_iters"]))
        rels.append(float(info["true_rel_res"]))
        coarse.append(int(info["coarse_iters"]))
        mvs.append(int(info["fine_matvecs"]))
        print(f"m {m:.10f}: {info['outer_iters']} outer iterations, true rel res {info['true_rel_res']:.3e}, "
              f"{time.time() - t:.0f} s", flush=True)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}_oracle_iters.txt")
    with open(out, "w") as f:
        f.write(f"# {name}: oracle setup ({SETUP_ITERS.get(name, 5)} refinement iterations per group of 4) "
                f"at m = {w.setup_mass():.10f}, then one FP64 MG-GCR(16) solve per mass to 1e-10; "
                f"smoother {'GMRES(%d)' % steps if sm else '%d MR steps' % steps}\n")
        f.write(f"# masses {w.masses()}\n# true relative residuals {rels}\n# setup {t_setup:.0f} s\n")
        f.write("outer_iters " + " ".join(map(str, iters)) + "\n")
        f.write("coarse_iters " + " ".join(map(str, coarse)) + "\n")
        f.write("fine_matvecs " + " ".join(map(str, mvs)) + "\n")
        f.write(f"setup_fine_matvecs {sinfo['fine_matvecs']}\nsetup_coarse_iters {sinfo['coarse_iters']}\n")
    print(open(out).read())


if __name__ == "__main__":
    main(sys.argv[1])
