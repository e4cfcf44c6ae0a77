"""Small seeded fields shared by the tests (all from synth, no method arithmetic)."""
import numpy as np

import synth


def rough_gauge(L, seed=11, sweeps=3, beta=6.0):
    """A few heatbath sweeps from a hot start: rough, cheap, deterministic."""
    return synth.gauge_field(L, beta=beta, sweeps=sweeps, n_or=1, seed=seed, cache=False)


def dense_from_apply(apply, n):
    """Columns of a linear map given as a function on flat complex vectors."""
    M = np.zeros((n, n), dtype=np.complex128)
    for k in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[k] = 1.0
        M[:, k] = apply(e)
    return M


# 8^4 quenched field at beta = 6.0 (hot start, 200 x (1 heatbath + 4 OR)), seed 1001.
# Re lambda_min(D(m=0)) = 0.7985754 for this field (ARPACK, which='SR', on the
# oracle operator; see tests/golden/c1_mass.txt), so m = 0.01 - 0.7985754.
C1_RE_LAMBDA_MIN_M0 = 0.7985754005


def c1_workload():
    L, B, nv = (8, 8, 8, 8), (4, 4, 4, 4), 8
    U = synth.gauge_field(L, beta=6.0, sweeps=200, n_or=4, seed=1001)
    return L, B, nv, U, 0.01 - C1_RE_LAMBDA_MIN_M0
