"""GPU (CUDA, through the C-ABI) against the FP64 CPU oracle on identical seeded
inputs.  Tolerances: 1e-12 relative for FP64 single operator applications,
1e-5 for FP32; every solve reaches a true FP64 relative residual <= 1e-10,
recomputed here with the oracle's own operator."""
import numpy as np
import pytest

import oracle
import paper_1005_3043_gb300 as wmg
import synth
from tests._fields import c1_workload, rough_gauge

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


def maxrel(a, b):
    """max elementwise |a-b| relative to max |b| (elementwise comparison)."""
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def make_params(nv, B=(4, 4, 4, 4), **kw):
    p = wmg.mg_default_params()
    for i in range(4):
        p.block[i] = B[i]
    p.nvec = nv
    p.setup_group = kw.pop("setup_group", min(4, nv))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.fixture(scope="module", autouse=True)
def _built():
    wmg.build.build()
    wmg.load()


# lattices: several 256-site tiles, a ragged grid tail, non-cubic extents, degenerate coarse extents
DSLASH_CASES = [
    ((8, 8, 8, 8), (4, 4, 4, 4)),
    ((4, 4, 4, 4), (4, 4, 4, 4)),          # one block, coarse extent 1
    ((6, 4, 2, 10), (2, 2, 2, 2)),         # V = 480: ragged last thread block
    ((4, 8, 4, 12), (2, 4, 2, 4)),
]


@pytest.mark.parametrize("L,B", DSLASH_CASES)
def test_dslash_parity(L, B):
    U = rough_gauge(L, seed=3)
    psi = synth.gaussian_spinor(L, 17)
    m = -0.42
    ref = oracle.dslash(U, psi, m, L)
    with wmg.WilsonMG(L, make_params(2, B)) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        assert maxrel(mg.dslash(psi, wmg.MG_FP64), ref) < TOL64
        assert maxrel(mg.dslash(psi, wmg.MG_FP32), ref) < TOL32


@pytest.mark.parametrize("B", [(2, 2, 2, 2), (4, 4, 4, 4)])   # per-site kernel / aggregate-staged kernel
def test_dslash_periodic_t_and_free_field(B):
    L = (4, 4, 4, 8)
    U = synth.unit_gauge(L)
    psi = synth.gaussian_spinor(L, 5)
    with wmg.WilsonMG(L, make_params(1, B), t_antiperiodic=0) as mg:
        mg.set_links(U)
        mg.set_mass(0.3)
        ref = oracle.dslash(U, psi, 0.3, L, tap=0)
        assert maxrel(mg.dslash(psi), ref) < TOL64
        assert maxrel(mg.dslash(psi, wmg.MG_FP32), ref) < TOL32


def _level(L, B, nv, seed=21, m=-0.2, sweeps=3):
    U = rough_gauge(L, seed=seed, sweeps=sweeps)
    V0 = synth.gaussian_vectors(L, nv, seed + 100)
    P, st = oracle.block_orthonormalize(V0, L, B)
    assert st == 0
    A = oracle.coarse_build(U, P, m, L, B)
    return U, V0, P, A


@pytest.mark.parametrize("L,B,nv", [((8, 8, 8, 8), (4, 4, 4, 4), 4),
                                    ((4, 4, 4, 8), (2, 2, 2, 4), 3),
                                    ((4, 4, 4, 4), (4, 4, 4, 4), 2)])
def test_block_ortho_restrict_prolong_coarse_parity(L, B, nv):
    m = -0.2
    U, V0, P, A = _level(L, B, nv, m=m)
    Lc = oracle.coarse_dims(L, B)
    Vc = oracle.volume(Lc)
    with wmg.WilsonMG(L, make_params(nv, B)) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        mg.set_null_vectors(V0)
        assert maxrel(mg.prolongator(), P) < TOL64
        assert maxrel(mg.coarse_op(), A) < TOL64
        r = synth.gaussian_spinor(L, 33)
        rc_ref = oracle.restrict(P, r, L, B)
        assert maxrel(mg.restrict(r), rc_ref) < TOL64
        assert maxrel(mg.restrict(r, wmg.MG_FP32), rc_ref) < TOL32
        y = synth.gaussian(Vc * 2 * nv, 34, 0).reshape(Vc, 2 * nv)
        e_ref = oracle.prolong(P, y, L, B)
        assert maxrel(mg.prolong(y), e_ref) < TOL64
        assert maxrel(mg.prolong(y, wmg.MG_FP32), e_ref) < TOL32
        c_ref = oracle.coarse_apply(A, y, Lc)
        cd_ref = oracle.coarse_apply_dag(A, y, Lc)
        assert maxrel(mg.coarse(y), c_ref) < TOL64
        assert maxrel(mg.coarse(y, dagger=True), cd_ref) < TOL64
        assert maxrel(mg.coarse(y, prec=wmg.MG_FP32), c_ref) < TOL32
        assert maxrel(mg.coarse(y, dagger=True, prec=wmg.MG_FP32), cd_ref) < TOL32
        # mass change shifts the coarse diagonal exactly (P^dag P = I)
        mg.set_mass(m + 0.05)
        assert maxrel(mg.coarse_op(), oracle.coarse_build(U, P, m + 0.05, L, B)) < TOL64


def test_mr_parity():
    L = (8, 4, 4, 8)
    U = rough_gauge(L, seed=4)
    m, w = -0.3, 0.9
    e = synth.gaussian_spinor(L, 1)
    r = synth.gaussian_spinor(L, 2)
    e_ref, r_ref = oracle.mr(U, e, r, m, L, 4, w)
    with wmg.WilsonMG(L, make_params(2, (4, 4, 4, 4))) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        e64, r64 = mg.mr(e, r, 4)
        assert maxrel(e64, e_ref) < TOL64 and maxrel(r64, r_ref) < TOL64
        e32, r32 = mg.mr(e, r, 4, wmg.MG_FP32)
        assert maxrel(e32, e_ref) < 1e-4 and maxrel(r32, r_ref) < 1e-4


def test_coarse_solve_parity():
    L, B, nv = (8, 8, 8, 8), (4, 4, 4, 4), 4
    m = -0.2
    U, V0, P, A = _level(L, B, nv, m=m)
    Lc = oracle.coarse_dims(L, B)
    rc = synth.gaussian(oracle.volume(Lc) * 2 * nv, 8, 0).reshape(-1, 2 * nv)
    with wmg.WilsonMG(L, make_params(nv, B)) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        mg.set_null_vectors(V0)
        for k in (1, 7, 25):                         # fixed iteration counts (tol = 0)
            y_ref, it_ref, _ = oracle.cgnr(A, rc, Lc, 0.0, k)
            y, it, _ = mg.coarse_solve(rc, 0.0, k)
            assert it == it_ref == k
            assert maxrel(y, y_ref) < 1e-10
        y_ref, it_ref, rel_ref = oracle.cgnr(A, rc, Lc, 1e-3, 5000)
        y, it, rel = mg.coarse_solve(rc, 1e-3, 5000)
        assert rel <= 1e-3 and abs(it - it_ref) <= 1
        y32, it32, rel32 = mg.coarse_solve(rc, 1e-3, 5000, wmg.MG_FP32)
        assert rel32 <= 1e-3


def test_vcycle_parity():
    L, B, nv = (8, 8, 8, 8), (4, 4, 4, 4), 4
    m = -0.2
    U, V0, P, A = _level(L, B, nv, m=m)
    r = synth.gaussian_spinor(L, 12)
    po = oracle.make_params(L, B, nv=nv, m=m, coarse_tol=0.0, coarse_maxit=30)
    z_ref, _ = oracle.vcycle(po, U, P, A, r)
    with wmg.WilsonMG(L, make_params(nv, B, coarse_tol=0.0, max_coarse=30)) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        mg.set_null_vectors(V0)
        assert maxrel(mg.vcycle(r), z_ref) < 1e-10
        assert maxrel(mg.vcycle(r, wmg.MG_FP32), z_ref) < 1e-4


def _true_rel(U, x, b, m, L):
    return np.linalg.norm(b - oracle.dslash(U, x, m, L)) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def c1():
    L, B, nv, U, m = c1_workload()
    V0 = synth.gaussian_vectors(L, nv, 2001)
    po = oracle.make_params(L, B, nv=nv, m=m)
    Vs, P, A, st = oracle.setup(po, U, V0, init_relax=10, n_iter=3, group_size=4)
    assert st == 0
    return dict(L=L, B=B, nv=nv, U=U, m=m, V0=V0, Vs=Vs, P=P, A=A, po=po)


def test_solve_fp64_matches_oracle(c1):
    L, B, nv, U, m = c1["L"], c1["B"], c1["nv"], c1["U"], c1["m"]
    b = synth.gaussian_spinor(L, 7)
    x_ref, info_ref = oracle.gcr_solve(c1["po"], U, c1["P"], c1["A"], b)
    with wmg.WilsonMG(L, make_params(nv, B)) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        mg.set_null_vectors(c1["Vs"])
        x, info = mg.solve(b)
    assert info["status"] == 0 and info_ref["status"] == 0
    assert _true_rel(U, x, b, m, L) <= 1e-10
    assert abs(info["true_rel_res"] - _true_rel(U, x, b, m, L)) < 1e-12
    assert abs(info["outer_iters"] - info_ref["outer_iters"]) <= 2
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-7


def test_solve_into_caller_buffer(c1):
    """The host-buffer solve writing into a caller's array (pinned host memory
    here) gives the same solution as the one it allocates; a wrong-sized or
    wrong-typed array is refused before any work."""
    import torch
    L, B, nv, U, m = c1["L"], c1["B"], c1["nv"], c1["U"], c1["m"]
    b = synth.gaussian_spinor(L, 7)
    out = torch.zeros(b.shape, dtype=torch.complex128, pin_memory=True)
    with wmg.WilsonMG(L, make_params(nv, B)) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        mg.set_null_vectors(c1["Vs"])
        x, info = mg.solve(b)
        x2, info2 = mg.solve(b, out=out.numpy())
        with pytest.raises(ValueError):
            mg.solve(b, out=np.zeros(b.size - 1, dtype=np.complex128))
        with pytest.raises(ValueError):
            mg.solve(b, out=np.zeros(b.shape, dtype=np.complex64))
    assert np.shares_memory(x2, out.numpy())
    assert info2["status"] == 0 and info2["outer_iters"] == info["outer_iters"]
    assert np.abs(x2 - x).max() <= 1e-13 * np.abs(x).max()


def test_launch_timer_classes(c1):
    """The launch timer tracks the selected kernel classes only; the selection
    cannot change while recorded launches are unread, and an empty one is refused."""
    L, B, nv, U, m = c1["L"], c1["B"], c1["nv"], c1["U"], c1["m"]
    b = synth.gaussian_spinor(L, 7)
    with wmg.WilsonMG(L, make_params(nv, B, prec_inner=wmg.MG_FP32, delta=1e-4)) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        mg.set_null_vectors(c1["Vs"])
        mg.profile_classes(["coarse_solve"])
        mg.profile_enable(True)
        mg.solve(b)
        with pytest.raises(RuntimeError):
            mg.profile_classes(["dslash"])          # unread launches pending
        one, iters = mg.profile_read()
        assert one["coarse_solve"][1] > 0 and iters > 0
        assert all(v == (0.0, 0) for k, v in one.items() if k != "coarse_solve")
        mg.profile_classes(wmg.KERNEL_CLASSES)
        mg.solve(b)
        every, _ = mg.profile_read()
        mg.profile_enable(False)
        assert every["coarse_solve"][1] == one["coarse_solve"][1]
        assert every["dslash"][1] > 0 and every["krylov"][1] > 0
        with pytest.raises(RuntimeError):
            mg.profile_classes([])


def test_solve_fp32_inner_reaches_fp64_residual(c1):
    L, B, nv, U, m = c1["L"], c1["B"], c1["nv"], c1["U"], c1["m"]
    b = synth.gaussian_spinor(L, 7)
    with wmg.WilsonMG(L, make_params(nv, B, prec_inner=wmg.MG_FP32, delta=1e-4)) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        mg.set_null_vectors(c1["Vs"])
        x, info = mg.solve(b)
    assert info["status"] == 0
    assert _true_rel(U, x, b, m, L) <= 1e-10


def test_setup_fp64_matches_oracle(c1):
    L, B, nv, U, m = c1["L"], c1["B"], c1["nv"], c1["U"], c1["m"]
    with wmg.WilsonMG(L, make_params(nv, B, setup_iters=3)) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        mg.setup(c1["V0"])
        Vg = mg.null_vectors()
        Pg = mg.prolongator()
        Ag = mg.coarse_op()
        b = synth.gaussian_spinor(L, 9)
        x, info = mg.solve(b)
    # same algorithm, FP64 on both sides: prototypes agree unless a coarse stopping
    # test landed on the other side of its threshold
    d = max(np.linalg.norm(Vg[i] - c1["Vs"][i]) for i in range(nv))
    assert d < 1e-6
    # its prolongator and Galerkin D_c agree with the oracle's setup output to the
    # same order (the oracle's own P and D_c, nothing computed from GPU output)
    assert maxrel(Pg, c1["P"]) < 1e-5
    assert maxrel(Ag, c1["A"]) < 1e-5
    assert info["status"] == 0 and _true_rel(U, x, b, m, L) <= 1e-10


def test_setup_two_grid_factor_matches_oracle(c1):
    """Setup quality by eq. 3: the asymptotic two-grid rate (||e_40|| / ||e_20||)^(1/20)
    of the GPU's own FP64 setup (its V-cycle with the MR(4) smoother, coarse CGNR
    to 1e-12 standing in for the exact solve) agrees with the oracle's setup
    measured by the oracle (exact coarse solve) to 10 % relative."""
    L, B, nv, U, m = c1["L"], c1["B"], c1["nv"], c1["U"], c1["m"]
    e0 = synth.gaussian_spinor(L, 2002)
    _, n_ref = oracle.two_grid_factor(c1["po"], U, c1["P"], c1["A"], e0, 40)
    rate_ref = (n_ref[40] / n_ref[20]) ** (1 / 20)
    p = make_params(nv, B, setup_iters=3, smoother=0, smoother_steps=4, coarse_tol=1e-12, max_coarse=100000)
    with wmg.WilsonMG(L, p) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        mg.setup(c1["V0"])
        e = e0.copy()
        norms = [np.linalg.norm(e)]
        for _ in range(40):
            e = e + mg.vcycle(-mg.dslash(e, wmg.MG_FP64), wmg.MG_FP64)
            norms.append(np.linalg.norm(e))
    rate = (norms[40] / norms[20]) ** (1 / 20)
    assert rate < 1 and abs(rate - rate_ref) <= 0.1 * rate_ref, (rate, rate_ref)


def test_mass_sweep_reuses_setup(c1):
    L, B, nv, U, m = c1["L"], c1["B"], c1["nv"], c1["U"], c1["m"]
    b = synth.gaussian_spinor(L, 11)
    with wmg.WilsonMG(L, make_params(nv, B, prec_inner=wmg.MG_FP32, delta=1e-4)) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        mg.set_null_vectors(c1["Vs"])
        iters = []
        for mm in (m + 0.09, m + 0.04, m + 0.02, m):
            mg.set_mass(mm)
            x, info = mg.solve(b)
            assert info["status"] == 0 and _true_rel(U, x, b, mm, L) <= 1e-10
            iters.append(info["outer_iters"])
    assert iters[0] <= iters[-1]


def test_edge_cases(c1):
    L, B, nv, U, m = c1["L"], c1["B"], c1["nv"], c1["U"], c1["m"]
    with wmg.WilsonMG(L, make_params(nv, B)) as mg:
        with pytest.raises(wmg.MGError) as ei:
            mg.solve(np.zeros((mg.V, 4, 3)))         # no links yet
        assert ei.value.status == wmg.MG_ERR_NOT_SETUP
        mg.set_links(U)
        mg.set_mass(m)
        bad = c1["Vs"].copy()
        bad[1] = bad[0] * 2.0                         # rank-deficient prototypes
        with pytest.raises(wmg.MGError) as ei:
            mg.set_null_vectors(bad)
        assert ei.value.status == wmg.MG_ERR_NUMERIC
        mg.set_null_vectors(c1["Vs"])
        x, info = mg.solve(np.zeros((mg.V, 4, 3)))    # b = 0
        assert info["status"] == 0 and np.abs(x).max() == 0
        p = make_params(nv, B, max_outer=2)
        mg.set_params(p)
        x, info = mg.solve(synth.gaussian_spinor(L, 3))
        assert info["status"] == wmg.MG_ERR_NOT_CONVERGED and info["outer_iters"] == 2
        mg.set_params(make_params(nv, B))
        b = synth.gaussian_spinor(L, 3)
        b[5, 1, 2] = np.nan
        with pytest.raises(wmg.MGError) as ei:
            mg.solve(b)
        assert ei.value.status == wmg.MG_ERR_NUMERIC
    with pytest.raises(wmg.MGError) as ei:
        wmg.WilsonMG((8, 8, 8, 6), make_params(nv, B))   # 6 not divisible by 4
    assert ei.value.status == wmg.MG_ERR_INVALID_ARG


def test_fp16_coarse_storage(c1):
    """MG_FP16: FP16 coarse operator (per-block scale) in the coarse CGNR.  The coarse
    residual against the exact D_c stays at the FP16 storage level; every solve still
    reaches a true FP64 residual of 1e-10."""
    L, B, nv, U, m = c1["L"], c1["B"], c1["nv"], c1["U"], c1["m"]
    Lc = oracle.coarse_dims(L, B)
    with wmg.WilsonMG(L, make_params(nv, B, prec_inner=wmg.MG_FP16, delta=1e-4)) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        mg.set_null_vectors(c1["Vs"])
        A = c1["A"]                                  # the oracle's D_c of the same setup
        rc = synth.gaussian(mg.Vc * mg.nc, 41, 0).reshape(mg.Vc, mg.nc)
        y16, it16, rel16 = mg.coarse_solve(rc, 1e-3, 5000, wmg.MG_FP16)
        assert rel16 <= 1e-3
        true_rel = np.linalg.norm(rc - oracle.coarse_apply(A, y16, Lc)) / np.linalg.norm(rc)
        assert true_rel < 1e-2, true_rel
        b = synth.gaussian_spinor(L, 7)
        x, info = mg.solve(b)
    assert info["status"] == 0
    assert _true_rel(U, x, b, m, L) <= 1e-10


def test_fp16_fine_storage_dslash_and_mr():
    """MG_FP16 smoother storage: spinors in FP16 with one FP32 scale per site and
    FP16 links.  The oracle error of a single application is at the FP16
    rounding level (2^-11 relative per stored entry, a few entries per output);
    the bound 4e-3 is reported, not a parity claim; MR steps reduce the residual
    as in FP64 to the same precision."""
    L = (8, 4, 4, 8)
    U = rough_gauge(L, seed=4)
    m, w = -0.3, 0.9
    psi = synth.gaussian_spinor(L, 17)
    ref = oracle.dslash(U, psi, m, L)
    e = synth.gaussian_spinor(L, 1)
    r = synth.gaussian_spinor(L, 2)
    e_ref, r_ref = oracle.mr(U, e, r, m, L, 4, w)
    with wmg.WilsonMG(L, make_params(2, (4, 4, 4, 4))) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        err = maxrel(mg.dslash(psi, wmg.MG_FP16), ref)
        assert 1e-5 < err < 4e-3, err             # FP16-rounded, but close
        e16, r16 = mg.mr(e, r, 4, wmg.MG_FP16)
    assert maxrel(e16, e_ref) < 1e-2 and maxrel(r16, r_ref) < 1e-2
    # the residual it returns is the residual of the e it returns (to FP16 storage)
    r_true = r + oracle.dslash(U, e, m, L) - oracle.dslash(U, e16, m, L)
    assert maxrel(r16, r_true) < 1e-2


@pytest.mark.parametrize("smoother", [0, 1])
@pytest.mark.parametrize("smoother_fp16", [1, 2])
def test_fp16_mode_solve_with_each_smoother_storage(c1, smoother_fp16, smoother):
    """MG_FP16 solves with the smoother's storage in FP16 (1) or FP32 (2) — the MR
    smoother's spinors and links, or the GMRES(8) smoother's Arnoldi basis — all
    reach a true FP64 residual of 1e-10."""
    L, B, nv, U, m = c1["L"], c1["B"], c1["nv"], c1["U"], c1["m"]
    b = synth.gaussian_spinor(L, 7)
    steps = 8 if smoother else 4
    with wmg.WilsonMG(L, make_params(nv, B, prec_inner=wmg.MG_FP16, delta=1e-4, smoother_fp16=smoother_fp16,
                                     smoother=smoother, smoother_steps=steps)) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        mg.set_null_vectors(c1["Vs"])
        x, info = mg.solve(b)
    assert info["status"] == 0
    assert _true_rel(U, x, b, m, L) <= 1e-10


@pytest.mark.parametrize("steps", [4, 8])
def test_vcycle_parity_gmres_smoother(steps):
    """V(0, GMRES(k)) cycle: one GMRES(k) post-smoothing application scaled by
    omega (Sec. III-IV) against the oracle's, fixed coarse iterations."""
    L, B, nv = (8, 8, 8, 8), (4, 4, 4, 4), 4
    m = -0.2
    U, V0, P, A = _level(L, B, nv, m=m)
    r = synth.gaussian_spinor(L, 12)
    po = oracle.make_params(L, B, nv=nv, m=m, coarse_tol=0.0, coarse_maxit=30, smoother=1, mr_steps=steps)
    z_ref, _ = oracle.vcycle(po, U, P, A, r)
    with wmg.WilsonMG(L, make_params(nv, B, coarse_tol=0.0, max_coarse=30, smoother=1, smoother_steps=steps)) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        mg.set_null_vectors(V0)
        assert maxrel(mg.vcycle(r), z_ref) < 1e-10
        assert maxrel(mg.vcycle(r, wmg.MG_FP32), z_ref) < 1e-4


def test_solve_gmres_smoother_matches_oracle(c1):
    """MG-GCR with the GMRES(8) smoother: FP64 iteration count within 2 of the
    oracle's, the FP16-storage mode reaches the same 1e-10 true residual."""
    L, B, nv, U, m = c1["L"], c1["B"], c1["nv"], c1["U"], c1["m"]
    b = synth.gaussian_spinor(L, 7)
    po = oracle.make_params(L, B, nv=nv, m=m, smoother=1, mr_steps=8)
    x_ref, info_ref = oracle.gcr_solve(po, U, c1["P"], c1["A"], b)
    for prec, delta in ((wmg.MG_FP64, 0.0), (wmg.MG_FP16, 1e-4)):
        with wmg.WilsonMG(L, make_params(nv, B, prec_inner=prec, delta=delta, smoother=1, smoother_steps=8)) as mg:
            mg.set_links(U)
            mg.set_mass(m)
            mg.set_null_vectors(c1["Vs"])
            x, info = mg.solve(b)
        assert info["status"] == 0
        assert _true_rel(U, x, b, m, L) <= 1e-10
        assert abs(info["outer_iters"] - info_ref["outer_iters"]) <= (2 if prec == wmg.MG_FP64 else 6)


def test_gmres_smoother_edge_cases():
    """GMRES(1) is one MR step (same minimiser over span{r}); invalid smoother
    parameters are rejected."""
    L, B, nv = (8, 8, 8, 8), (4, 4, 4, 4), 4
    m = -0.2
    U, V0, P, A = _level(L, B, nv, m=m)
    r = synth.gaussian_spinor(L, 12)
    outs = []
    for sm in (0, 1):
        with wmg.WilsonMG(L, make_params(nv, B, coarse_tol=0.0, max_coarse=10, smoother=sm, smoother_steps=1)) as mg:
            mg.set_links(U)
            mg.set_mass(m)
            mg.set_null_vectors(V0)
            outs.append(mg.vcycle(r))
    assert maxrel(outs[1], outs[0]) < 1e-11
    for bad in ({"smoother": 2}, {"smoother": 1, "smoother_steps": 17}):
        with pytest.raises(wmg.MGError):
            wmg.WilsonMG(L, make_params(nv, B, **bad))
