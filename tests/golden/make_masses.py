"""Compute Re(lambda_min) of D(m=0) for the seeded quenched workloads.

Calls only the oracle's Wilson operator (eq. 2) and scipy's ARPACK
(implicitly restarted Arnoldi, which='SR').  Since D(m) = D(0) + m exactly,
the bare mass giving Re(lambda_min) = target is m = target - Re(lambda_min(D(0))).

usage: python tests/golden/make_masses.py c1|c2  -> writes tests/golden/<name>_mass.txt
"""
import os
import sys
import time

import numpy as np
import scipy.sparse.linalg as sla

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
import synth  # noqa: E402

WORKLOADS = {
    "c1": dict(L=(8, 8, 8, 8), seed=1001),
    "c2": dict(L=(16, 16, 16, 32), seed=2001),
}


def re_lambda_min(L, U, k=6, ncv=60, tol=1e-9):
    V = oracle.volume(L)
    count = [0]
    t0 = time.time()

    def mv(v):
        count[0] += 1
        if count[0] % 500 == 0:
            print(f"  {count[0]} matvecs, {time.time() - t0:.0f} s", flush=True)
        return oracle.dslash(U, v.reshape(V, 4, 3), 0.0, L).ravel()

    op = sla.LinearOperator((V * 12, V * 12), dtype=np.complex128, matvec=mv)
    ev = sla.eigs(op, k=k, which="SR", ncv=ncv, tol=tol, return_eigenvectors=False)
    return float(np.min(ev.real)), ev


if __name__ == "__main__":
    name = sys.argv[1]
    w = WORKLOADS[name]
    U = synth.gauge_field(w["L"], beta=6.0, sweeps=200, n_or=4, seed=w["seed"])
    t = time.time()
    big = oracle.volume(w["L"]) > 100000
    # on large lattices the left edge of the spectrum is dense and ARPACK
    # stagnates when asked for several converged pairs: ask for the leftmost
    # pair only, with a larger Krylov space and a residual tolerance of 1e-3
    # relative (the eigenvalue error is far below the residual for the real,
    # isolated edge modes found on the smaller lattice)
    lam, ev = re_lambda_min(w["L"], U, k=2 if big else 6, ncv=80 if big else 60, tol=1e-3 if big else 1e-9)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}_mass.txt")
    with open(out, "w") as f:
        f.write(f"# {name}: L={w['L']} beta=6.0 sweeps=200 n_or=4 seed={w['seed']}\n")
        f.write(f"# plaquette {synth.plaquette(U, w['L']):.12f} sha1 {synth.checksum(U)}\n")
        f.write(f"# eigenvalues (which=SR): {np.sort_complex(ev)}\n")
        f.write(f"# ARPACK time {time.time() - t:.1f} s\n")
        f.write(f"re_lambda_min_m0 {lam:.10f}\n")
    print(open(out).read())
