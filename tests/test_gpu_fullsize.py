"""Coarse CGNR parity at the 16^3 x 32 shapes the benchmark runs (4^4 aggregates,
Nv = 20: Vc = 512 coarse sites, nc = 40 dof per site), on the default on-chip
kernel with the FP16 operator in tensor memory (products on the tensor cores:
128 rows per CTA in one MMA tile, the 8 rows past it on the CUDA cores, every
one of the 152 CTAs owning units) and on the CUDA-core form (three 32-column
TMEM chunks per thread), in both iteration forms,
against the oracle's CGLS (Sec. IV: CG on the normal equations of the
coarsest operator) on the oracle's own D_c rounded by the FP16 storage rule.

The library builds D_c in FP64 here (an FP64 context) from the same
prototypes, so both sides round the same FP64 entries to FP16; the oracle's
operator, prototypes and every expected value come from the oracle alone."""
import numpy as np
import pytest

import oracle
import paper_1005_3043_gb300 as wmg
import synth
from paper_1005_3043_gb300.workloads import WORKLOADS
from tests.test_gpu_cgls import quantise16

pytestmark = pytest.mark.gpu

W = WORKLOADS["wilson_16x16x16x32_nv20_beta6_5mass"]
SHIFT = -0.5


def maxrel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


@pytest.fixture(scope="module", autouse=True)
def _built():
    wmg.build.build()
    wmg.load()


@pytest.fixture(scope="module")
def c2():
    L, B, nv = W.dims, W.block, W.nvec
    U = synth.gauge_field(L, beta=W.beta, sweeps=W.sweeps, n_or=W.n_or, seed=W.seed)
    m = W.masses()[-1]
    V0 = synth.gaussian_vectors(L, nv, W.setup_seed)
    Lc = oracle.coarse_dims(L, B)
    rc = synth.gaussian(oracle.volume(Lc) * 2 * nv, 8, 0).reshape(-1, 2 * nv)
    # (a) the random starts as prototypes: well-conditioned blocks, so the
    # library's and the oracle's P agree to ~1e-13 and every FP16 rounding of D_c agrees
    P, st = oracle.block_orthonormalize(V0, L, B)
    assert st == 0
    A_rand = oracle.coarse_build(U, P, m, L, B)
    # (b) the first step of the setup (Sec. IV): 10 relaxation steps on D v = 0
    # from each random start, by the oracle's MR smoother -- a D_c with small
    # singular values that needs many CG iterations
    Vr = np.empty_like(V0)
    for i in range(nv):
        e, _ = oracle.mr(U, V0[i].copy(), -oracle.dslash(U, V0[i], m, L), m, L, 10, 0.9)
        Vr[i] = e / np.linalg.norm(e)
    P, st = oracle.block_orthonormalize(Vr, L, B)
    assert st == 0
    # built at m - 0.5 (the same prototypes; D_c(m') = D_c(m) + (m' - m) I by
    # eq. 4): the shift takes its smallest singular values near zero, so CG
    # needs ~460 iterations to 1e-3, the depth of the benchmark's coarse solves
    A_relax = oracle.coarse_build(U, P, m + SHIFT, L, B)
    return dict(L=L, B=B, nv=nv, m=m, U=U, Lc=Lc, rc=rc, V_rand=V0, A16_rand=quantise16(A_rand), V_relax=Vr,
                A16_relax=quantise16(A_relax))


def _mg(c, V, form, shift=0.0, kernel=0):
    p = wmg.mg_default_params()
    for i in range(4):
        p.block[i] = c["B"][i]
    p.nvec = c["nv"]
    p.setup_group = 4
    p.prec_inner = wmg.MG_FP64        # D_c built in FP64 from the prototypes
    p.coarse_kernel = kernel
    p.coarse_form = form
    mg = wmg.WilsonMG(c["L"], p)
    mg.set_links(c["U"])
    mg.set_mass(c["m"] + shift)
    mg.set_null_vectors(V)
    return mg


# after 25 steps the random-prototype D_c (4 iterations to 1e-3) sits at the
# FP32 rounding floor, where iterates of two FP32 CGs drift apart slowly
FIXED_K_TOL = {1: 1e-5, 6: 1e-5, 25: 1e-4}


# coarse_kernel -> MG_CK_* id at this size: 0 (default) the tensor-memory
# operator with tensor-core products, 4 with CUDA-core products
TMEM_KERNELS = {0: 4, 4: 3}


@pytest.mark.parametrize("kernel", [0, 4])
@pytest.mark.parametrize("form", [0, 1])
def test_fixed_iterations_16x16x16x32_tmem(c2, form, kernel):
    with _mg(c2, c2["V_rand"], form, kernel=kernel) as mg:
        for k, tol in FIXED_K_TOL.items():
            y_ref, it_ref, _ = oracle.cgnr(c2["A16_rand"], c2["rc"], c2["Lc"], 0.0, k)
            y, it, _ = mg.coarse_solve(c2["rc"], 0.0, k, wmg.MG_FP16)
            assert mg.coarse_kernel() == TMEM_KERNELS[kernel], wmg.COARSE_KERNELS[mg.coarse_kernel()]
            assert it == it_ref == k
            assert maxrel(y, y_ref) < tol, (k, maxrel(y, y_ref))


@pytest.mark.parametrize("kernel", [0, 4])
@pytest.mark.parametrize("form", [0, 1])
def test_converged_solve_16x16x16x32_tmem(c2, form, kernel):
    """On the relaxed-prototype D_c at the shifted mass: iterates after 6, 25
    and 100 steps (a complex64 numpy CGLS on these entries stays within 5e-7
    of the FP64 one up to k = 100), then the solve to 1e-3 with an iteration
    count within 2 % (and 2) of the oracle's on the same FP16 entries (the
    complex64 CGLS takes 460 against 459), and the kernel's residual honest
    when recomputed in FP64 with that operator."""
    A16 = c2["A16_relax"]
    y_ref, it_ref, _ = oracle.cgnr(A16, c2["rc"], c2["Lc"], 1e-3, 20000)
    assert it_ref > 300, it_ref           # deep enough to exercise many exchanges
    with _mg(c2, c2["V_relax"], form, SHIFT, kernel) as mg:
        for k, tol in ((6, 1e-5), (25, 1e-5), (100, 1e-4)):
            y_k, _, _ = oracle.cgnr(A16, c2["rc"], c2["Lc"], 0.0, k)
            y, it, _ = mg.coarse_solve(c2["rc"], 0.0, k, wmg.MG_FP16)
            assert it == k and maxrel(y, y_k) < tol, (k, maxrel(y, y_k))
        y, it, rel = mg.coarse_solve(c2["rc"], 1e-3, 20000, wmg.MG_FP16)
        assert mg.coarse_kernel() == TMEM_KERNELS[kernel]
    assert rel <= 1e-3
    assert abs(it - it_ref) <= max(2, 0.02 * it_ref), (it, it_ref)
    true_rel = np.linalg.norm(c2["rc"] - oracle.coarse_apply(A16, y, c2["Lc"])) / np.linalg.norm(c2["rc"])
    assert true_rel <= 1.5e-3, true_rel


@pytest.mark.parametrize("kernel", [0, 4])
def test_scale_invariance_16x16x16x32_tmem(c2, kernel):
    """CGLS is linear in its right-hand side: y(lam rc) = lam y(rc) with the same
    iterates.  The tensor-core form rescales each aggregate's operand by a power
    of two before its FP16 hi/lo split, so right-hand sides far outside the FP16
    range (lam = 2^-40, 2^40; |lam rc|^2 stays inside the FP32 range of the CG
    scalars) give the same iterates as lam = 1, scaled by lam (powers of two:
    exactly); a zero right-hand side gives y = 0 in zero iterations."""
    with _mg(c2, c2["V_rand"], 0, kernel=kernel) as mg:
        y1, it1, _ = mg.coarse_solve(c2["rc"], 0.0, 6, wmg.MG_FP16)
        for lam in (2.0 ** -40, 2.0 ** 40):
            y, it, _ = mg.coarse_solve(lam * c2["rc"], 0.0, 6, wmg.MG_FP16)
            assert it == it1 == 6
            assert maxrel(y / lam, y1) < 1e-6, (lam, maxrel(y / lam, y1))
        y0, it0, _ = mg.coarse_solve(np.zeros_like(c2["rc"]), 1e-3, 100, wmg.MG_FP16)
        assert it0 == 0 and not np.any(y0)
        assert mg.coarse_kernel() == TMEM_KERNELS[kernel]
