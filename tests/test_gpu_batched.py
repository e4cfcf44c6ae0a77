"""Batched right-hand sides: the tensor-core coarse stencil on an RHS panel and
the lockstep batched MG-GCR solve, against the FP64 CPU oracle."""
import numpy as np
import pytest

import oracle
import paper_1005_3043_gb300 as wmg
import synth
from tests._fields import c1_workload, rough_gauge

pytestmark = pytest.mark.gpu


def maxrel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def params(nv, B=(4, 4, 4, 4), **kw):
    p = wmg.mg_default_params()
    for i in range(4):
        p.block[i] = B[i]
    p.nvec = nv
    p.setup_group = kw.pop("setup_group", min(4, nv))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("L,B,nv,nrhs", [((8, 8, 8, 8), (4, 4, 4, 4), 8, 5),
                                         ((8, 8, 8, 8), (4, 4, 4, 4), 8, 16),
                                         ((4, 4, 4, 8), (2, 2, 2, 2), 8, 33),
                                         ((8, 8, 8, 8), (4, 4, 4, 4), 24, 12)])
def test_batched_coarse_stencil(L, B, nv, nrhs):
    """Tensor cores (FP16 operator, hi+lo panel, FP32 accumulation) and the FP64 SIMT
    reference against the oracle's D_c and D_c^dag, one RHS at a time.

    The tensor-core product is held to 1e-5 per source against the oracle's
    stencil with the operator's real and imaginary parts rounded to FP16 (the
    kernel's embedding, no scale) and the source unrounded: the hi + lo split
    keeps the source to ~2^-22 and the FP32 sums add ~1e-6.  The same check on
    a source rounded to FP16 alone (a kernel without the lo MMAs) is shown to
    fail by more than 10x that tolerance, so the split itself is tested."""
    wmg.build.build()
    U = rough_gauge(L, seed=5)
    m = -0.2
    V0 = synth.gaussian_vectors(L, nv, 91)
    P, st = oracle.block_orthonormalize(V0, L, B)
    A = oracle.coarse_build(U, P, m, L, B)
    # the tensor-core embedding: real and imaginary parts each rounded to FP16
    A16 = A.real.astype(np.float16).astype(np.float64) + 1j * A.imag.astype(np.float16).astype(np.float64)
    Lc = oracle.coarse_dims(L, B)
    Vc = oracle.volume(Lc)
    x = synth.gaussian(nrhs * Vc * 2 * nv, 92, 0).reshape(nrhs, Vc, 2 * nv)
    x[1 % nrhs] *= 1e-6                          # sources of very different scale in one panel
    with wmg.WilsonMG(L, params(nv, B)) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        mg.set_null_vectors(V0)
        for dag in (False, True):
            ref = np.stack([(oracle.coarse_apply_dag if dag else oracle.coarse_apply)(A, x[i], Lc) for i in range(nrhs)])
            y64 = mg.coarse_batched(x, dagger=dag, impl=1)
            assert maxrel(y64, ref) < 1e-12
            ytc = mg.coarse_batched(x, dagger=dag, impl=0)
            apply = oracle.coarse_apply_dag if dag else oracle.coarse_apply
            ref16 = np.stack([apply(A16, x[i], Lc) for i in range(nrhs)])
            for i in range(nrhs):                # per source, relative to its own size
                assert maxrel(ytc[i], ref16[i]) < 1e-5, (dag, i, maxrel(ytc[i], ref16[i]))
                # the FP16 operator itself is 2^-11 away from D_c
                assert maxrel(ytc[i], ref[i]) < 2e-3, (dag, i, maxrel(ytc[i], ref[i]))
                # negative control: the hi half alone (FP16-rounded source, each
                # source scaled to max |x| = 1 first as the library does)
                sc = np.abs(x[i].view(np.float64)).max()
                xh = (x[i].real / sc).astype(np.float16).astype(np.float64) + \
                    1j * (x[i].imag / sc).astype(np.float16).astype(np.float64)
                assert maxrel(apply(A16, xh * sc, Lc), ref16[i]) > 1e-4


def test_batched_solve_matches_single_solves():
    L, B, nv, U, m = c1_workload()
    V0 = synth.gaussian_vectors(L, nv, 2001)
    po = oracle.make_params(L, B, nv=nv, m=m)
    _, P, A, st = oracle.setup(po, U, V0, init_relax=10, n_iter=3, group_size=4)
    Vs = _
    nrhs = 6
    V = oracle.volume(L)
    b = np.stack([synth.gaussian_spinor(L, 7, stream=i) for i in range(nrhs - 2)] +
                 [synth.point_source(L, 0, 0, 0), synth.point_source(L, 77, 3, 2)])
    with wmg.WilsonMG(L, params(nv, B, prec_inner=wmg.MG_FP32, delta=1e-4)) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        mg.set_null_vectors(Vs)
        x, infos = mg.solve_batched(b)
        single = [mg.solve(b[i])[1] for i in range(nrhs)]
    for i in range(nrhs):
        assert infos[i]["status"] == 0
        res = np.linalg.norm(b[i] - oracle.dslash(U, x[i], m, L)) / np.linalg.norm(b[i])
        assert res <= 1e-10, (i, res)
        # same method per source; the FP16 coarse operator changes the preconditioner only slightly
        assert abs(infos[i]["outer_iters"] - single[i]["outer_iters"]) <= max(3, 0.15 * single[i]["outer_iters"])


def test_batched_solve_with_gmres_smoother():
    """The lockstep batched solve with one GMRES(8) post-smoothing per cycle and
    the FP16-storage mode: every source reaches 1e-10, iteration counts close to
    the single-source solves."""
    L, B, nv, U, m = c1_workload()
    V0 = synth.gaussian_vectors(L, nv, 2001)
    po = oracle.make_params(L, B, nv=nv, m=m, smoother=1, mr_steps=8)
    Vs, P, A, st = oracle.setup(po, U, V0, init_relax=10, n_iter=3, group_size=4)
    assert st == 0
    nrhs = 4
    b = np.stack([synth.gaussian_spinor(L, 7, stream=i) for i in range(nrhs - 1)] + [synth.point_source(L, 0, 1, 2)])
    with wmg.WilsonMG(L, params(nv, B, prec_inner=wmg.MG_FP16, delta=1e-4, smoother=1, smoother_steps=8)) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        mg.set_null_vectors(Vs)
        x, infos = mg.solve_batched(b)
        single = [mg.solve(b[i])[1] for i in range(nrhs)]
    for i in range(nrhs):
        assert infos[i]["status"] == 0
        res = np.linalg.norm(b[i] - oracle.dslash(U, x[i], m, L)) / np.linalg.norm(b[i])
        assert res <= 1e-10, (i, res)
        assert abs(infos[i]["outer_iters"] - single[i]["outer_iters"]) <= max(3, 0.2 * single[i]["outer_iters"])


def test_batched_solve_deep_coarse_iterations_16x16x16x32():
    """At the lightest 16^3x32 mass with the GMRES(12) setup the coarse CG runs
    hundreds of iterations per cycle and its vectors shrink far below 1: the
    tensor-core split of the panel into FP16 hi + lo must stay out of the FP16
    subnormal range (per-column power-of-two scaling).  Batched and single solves
    then take the same outer iterations and all reach 1e-10."""
    from paper_1005_3043_gb300.workloads import WORKLOADS
    w = WORKLOADS["wilson_16x16x16x32_nv20_beta6_5mass"]
    U = synth.gauge_field(w.dims, beta=w.beta, sweeps=w.sweeps, n_or=w.n_or, seed=w.seed)
    V0 = synth.gaussian_vectors(w.dims, w.nvec, w.setup_seed)
    b = np.stack([synth.point_source(w.dims, 0, 0, 2), synth.gaussian_spinor(w.dims, w.source_seed, stream=102)])
    m = w.masses()[-1]
    p = params(w.nvec, w.block, prec_inner=wmg.MG_FP16, delta=1e-4, setup_group=4, setup_iters=5,
               smoother=1, smoother_steps=12, max_outer=300)
    with wmg.WilsonMG(w.dims, p) as mg:
        mg.set_links(U)
        mg.set_mass(w.setup_mass())
        mg.setup(V0)
        mg.set_mass(m)
        x, infos = mg.solve_batched(b)
        single = [mg.solve(b[i])[1] for i in range(len(b))]
    for i in range(len(b)):
        assert infos[i]["status"] == 0, infos[i]
        res = np.linalg.norm(b[i] - oracle.dslash(U, x[i], m, w.dims)) / np.linalg.norm(b[i])
        assert res <= 1e-10, (i, res)
        assert abs(infos[i]["outer_iters"] - single[i]["outer_iters"]) <= 2
