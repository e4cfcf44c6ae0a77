"""Red-black (even-odd) preconditioned CG on the GPU, through the C-ABI, against
the oracle's red-black CG (the comparison solver of Sec. IV) on identical
seeded inputs: FP64 iterates after a fixed number of CG iterations to 1e-10,
converged FP64 and mixed FP32/FP64 solves to a true residual <= 1e-10
recomputed with the oracle's operator, iteration counts against the oracle's."""
import numpy as np
import pytest

import oracle
import paper_1005_3043_gb300 as wmg
import synth
from tests._fields import c1_workload, rough_gauge

pytestmark = pytest.mark.gpu


def maxrel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def params(B=(2, 2, 2, 2)):
    p = wmg.mg_default_params()
    for i in range(4):
        p.block[i] = B[i]
    p.nvec = 2
    p.setup_group = 2
    return p


@pytest.fixture(scope="module", autouse=True)
def _built():
    wmg.build.build()
    wmg.load()


# several thread blocks with a ragged tail (Vh = 384, 1536), periodic and antiperiodic t
CASES = [((4, 4, 4, 12), (2, 2, 2, 2), 1), ((8, 4, 6, 4), (2, 2, 2, 2), 0), ((8, 8, 8, 8), (4, 4, 4, 4), 1)]


@pytest.mark.parametrize("L,B,tap", CASES)
@pytest.mark.parametrize("k", [1, 5, 20])
def test_fixed_iterations_fp64_match_oracle(L, B, tap, k):
    U = rough_gauge(L, seed=41)
    m = -0.35
    b = synth.gaussian_spinor(L, 42)
    x_ref, it_ref, mv_ref, rel_ref, _ = oracle.eo_cg(U, b, m, L, 1e-30, k, tap=tap)
    assert it_ref == k
    with wmg.WilsonMG(L, params(B), t_antiperiodic=tap) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        x, info = mg.solve_eo_cg(b, tol=1e-30, maxit=k, prec=wmg.MG_FP64)
    assert info["status"] == wmg.MG_ERR_NOT_CONVERGED and info["outer_iters"] == k
    assert maxrel(x, x_ref) < 1e-10, maxrel(x, x_ref)
    assert info["true_rel_res"] == pytest.approx(rel_ref, rel=1e-8)
    # one pass stopped by maxit: Dhat and Dhat^dag per iteration, plus the
    # right-hand side, the first Dhat^dag, x_o and the residual check
    assert info["fine_matvecs"] == mv_ref == 2 * k + 4, (info["fine_matvecs"], mv_ref)


@pytest.mark.parametrize("prec", [wmg.MG_FP64, wmg.MG_FP32])
def test_converged_solve_near_critical_8x8x8x8(prec):
    """The 8^4 beta = 6.0 field at Re(lambda_min) = 0.01: true residual <= 1e-10
    with the oracle's operator; FP64 iterations within 1 % (and 2) of the
    oracle's, mixed precision within 5 % (its FP32 CG replaces its residual
    by the FP64 one every factor 10 of reduction and keeps its direction)."""
    L, B, nv, U, m = c1_workload()
    b = synth.gaussian_spinor(L, 7)
    x_ref, it_ref, _, rel_ref, st_ref = oracle.eo_cg(U, b, m, L, 1e-10, 100000)
    assert st_ref == 0
    with wmg.WilsonMG(L, params(B)) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        x, info = mg.solve_eo_cg(b, tol=1e-10, maxit=100000, prec=prec)
    assert info["status"] == 0
    res = np.linalg.norm(b - oracle.dslash(U, x, m, L)) / np.linalg.norm(b)
    assert res <= 1e-10, res
    assert info["true_rel_res"] == pytest.approx(res, rel=1e-3)
    slack = max(2, 0.01 * it_ref) if prec == wmg.MG_FP64 else 0.05 * it_ref
    assert abs(info["outer_iters"] - it_ref) <= slack, (info["outer_iters"], it_ref)
    if prec == wmg.MG_FP32:
        assert info["restarts"] >= 2
    assert info["dslash_bytes"] > 0 and info["solve_ms"] > 0


def test_zero_source_and_odd_extent():
    L = (4, 4, 4, 4)
    U = rough_gauge(L, seed=43)
    with wmg.WilsonMG(L, params()) as mg:
        mg.set_links(U)
        mg.set_mass(-0.2)
        x, info = mg.solve_eo_cg(np.zeros((256, 4, 3), complex), prec=wmg.MG_FP32)
        assert info["status"] == 0 and info["outer_iters"] == 0 and not np.any(x)
    L = (4, 4, 4, 3)
    p = params((2, 2, 2, 1))
    with wmg.WilsonMG(L, p) as mg:
        mg.set_links(rough_gauge(L, seed=44))
        with pytest.raises(wmg.MGError) as ei:
            mg.solve_eo_cg(synth.gaussian_spinor(L, 1))
        assert ei.value.status == wmg.MG_ERR_INVALID_ARG
