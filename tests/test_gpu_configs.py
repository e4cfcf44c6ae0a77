"""The other configurations at their full sizes, as parity cases: the 24^3 x 64
lattice with Nv = 24 (the many-right-hand-side configuration) and the 32^3 x 96
lattice with three levels.  Oracle inputs come from the seeded generators only;
where the oracle cannot follow the whole computation at this size the check is a
property that holds at any size (a solve's true residual recomputed with the
oracle's operator, orthonormality of the level-2 prolongator)."""
import numpy as np
import pytest

import oracle
import paper_1005_3043_gb300 as wmg
import synth
from paper_1005_3043_gb300.workloads import WORKLOADS

pytestmark = pytest.mark.gpu


def maxrel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def field(w):
    U = synth.gauge_field(w.dims, beta=w.beta, sweeps=w.sweeps, n_or=w.n_or, seed=w.seed)
    assert abs(synth.plaquette(U, w.dims) - w.plaquette) < 1e-10
    return U


def params(w, **kw):
    p = wmg.mg_default_params()
    for i in range(4):
        p.block[i] = w.block[i]
    p.nvec = w.nvec
    p.setup_group = 4
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.fixture(scope="module", autouse=True)
def _built():
    wmg.build.build()
    wmg.load()


def test_24x24x24x64_dslash_and_batched_stencil():
    """Eq. 2 on the whole 24^3 x 64 heatbath field (FP64 1e-12, FP32 1e-5 against
    the oracle); D_c of random prototypes against the oracle's Galerkin build
    (1e-12); the tensor-core stencil on a 16-column panel against the oracle's
    stencil with the FP16-rounded operator (1e-5 per column), D_c and D_c^dag."""
    w = WORKLOADS["wilson_24x24x24x64_nv24_beta6_76rhs"]
    U = field(w)
    m = w.setup_mass()
    psi = synth.gaussian_spinor(w.dims, 41)
    ref = oracle.dslash(U, psi, m, w.dims)
    V0 = synth.gaussian_vectors(w.dims, w.nvec, 42)
    P, st = oracle.block_orthonormalize(V0, w.dims, w.block)
    assert st == 0
    A = oracle.coarse_build(U, P, m, w.dims, w.block)
    del P
    A16 = A.real.astype(np.float16).astype(np.float64) + 1j * A.imag.astype(np.float16).astype(np.float64)
    Lc = oracle.coarse_dims(w.dims, w.block)
    Vc = oracle.volume(Lc)
    nrhs = 16
    x = synth.gaussian(nrhs * Vc * 2 * w.nvec, 43, 0).reshape(nrhs, Vc, 2 * w.nvec)
    # FP64 inner precision: D_c is built with FP64 products (the FP32/FP16 modes
    # build it with FP32 products, ~4e-9 relative), so the tensor-core stencil
    # sees the same FP16 rounding of the operator as the oracle's reference
    with wmg.WilsonMG(w.dims, params(w, prec_inner=wmg.MG_FP64)) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        assert maxrel(mg.dslash(psi, wmg.MG_FP64), ref) < 1e-12
        assert maxrel(mg.dslash(psi, wmg.MG_FP32), ref) < 1e-5
        mg.set_null_vectors(V0)
        assert maxrel(mg.coarse_op(), A) < 1e-12
        for dag in (False, True):
            apply = oracle.coarse_apply_dag if dag else oracle.coarse_apply
            ytc = mg.coarse_batched(x, dagger=dag, impl=0)
            for i in (0, 7, 15):
                assert maxrel(ytc[i], apply(A16, x[i], Lc)) < 1e-5, (dag, i)


def test_32x32x32x96_three_level_solve():
    """Three levels (4^4 then 2^4 aggregates, Nv = 24 then 32) on the 32^3 x 96
    heatbath field, MG_FP16 inner precision: the adaptive setup of both levels,
    then a point source solved to 1e-10, its residual recomputed on the host
    with the oracle's operator; the level-2 prolongator orthonormal on sampled
    level-2 aggregates (P2^dag P2 = I per aggregate and chirality)."""
    w = WORKLOADS["wilson_32x32x32x96_nv24_nv32_3level"]
    U = field(w)
    m = w.extra["mass"]
    p = params(w, prec_inner=wmg.MG_FP16, smoother=1, smoother_steps=w.extra["smoother_steps"],
               gcr_restart=w.extra["gcr_restart"], tol=1e-10, max_outer=2000, delta=1e-4,
               setup_iters=w.extra.get("setup_iters", 5), setup_init_relax=10, levels=3,
               nvec2=w.extra["nvec2"], smoother_steps1=4, cycles1=2)
    for i in range(4):
        p.block2[i] = w.extra["block2"][i]
    V0 = synth.gaussian_vectors(w.dims, w.nvec, w.setup_seed)
    b = synth.point_source(w.dims, 0, 0, 0)
    with wmg.WilsonMG(w.dims, p) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        mg.setup(V0)
        V2 = synth.gaussian(w.extra["nvec2"] * mg.Vc * mg.nc, w.setup_seed + 2, 0).reshape(w.extra["nvec2"], mg.Vc, mg.nc)
        mg.setup_level2(V2)
        x, info = mg.solve(b)
        P2 = mg.level2_prolongator()
    assert info["status"] == 0, info
    assert np.linalg.norm(b - oracle.dslash(U, x, m, w.dims)) <= 1e-10 * np.linalg.norm(b)
    # P2 (nv2, Vc1, 2 nv1): per level-2 aggregate and chirality the nv2 columns are orthonormal
    nv1, nv2, B2 = w.nvec, w.extra["nvec2"], w.extra["block2"]
    Lc1 = oracle.coarse_dims(w.dims, w.block)
    i1 = np.arange(oracle.volume(Lc1))
    c = [i1 % Lc1[0], (i1 // Lc1[0]) % Lc1[1], (i1 // (Lc1[0] * Lc1[1])) % Lc1[2], i1 // (Lc1[0] * Lc1[1] * Lc1[2])]
    Lc2 = [Lc1[k] // B2[k] for k in range(4)]
    X2 = (c[0] // B2[0]) + Lc2[0] * ((c[1] // B2[1]) + Lc2[1] * ((c[2] // B2[2]) + Lc2[2] * (c[3] // B2[3])))
    for x2 in (0, int(X2.max()) // 2, int(X2.max())):
        sites = np.where(X2 == x2)[0]
        for s in (0, 1):
            Q = P2[:, sites, s * nv1:(s + 1) * nv1].reshape(nv2, -1)
            assert np.abs(Q.conj() @ Q.T - np.eye(nv2)).max() < 1e-10
