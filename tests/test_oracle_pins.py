"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: each check is a closed form,
an identity the paper states, a brute-force dense construction, or an
independent library routine (numpy QR / LU / lstsq).
"""
import numpy as np
import pytest

import oracle
import synth
from tests._fields import dense_from_apply, rough_gauge

RTOL64 = 1e-13


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


# ---------------------------------------------------------------- gamma basis
def test_gamma_matrices_clifford_hermitian_chiral():
    g = oracle.gamma_matrices()
    for a in range(4):
        assert np.allclose(g[a], g[a].conj().T, atol=0)
        for b in range(4):
            assert np.allclose(g[a] @ g[b] + g[b] @ g[a], 2 * np.eye(4) * (a == b), atol=0)
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    # chiral basis: gamma5 diagonal, upper spins (0,1) chirality +1 (Sec. III split)
    assert np.array_equal(g5, np.diag([1, 1, -1, -1]).astype(complex))
    psi = synth.gaussian_spinor((2, 2, 2, 2), seed=3)
    assert np.array_equal(oracle.gamma5(psi), np.einsum("ab,xbc->xac", g5, psi))


# ---------------------------------------------------------------- eq. (2)
def _plane_wave(L, p, u):
    """psi(x) = exp(i p.x) u with u a 4x3 spin-colour constant."""
    c = np.stack(np.meshgrid(*[np.arange(l) for l in L], indexing="ij"), -1)  # (L0,L1,L2,L3,4)
    # site index = x + L0*(y + L1*(z + L2*t)) -> transpose to (t,z,y,x) order for ravel
    phase = np.exp(1j * (c @ np.asarray(p)))
    phase = np.transpose(phase, (3, 2, 1, 0)).reshape(-1)
    return phase[:, None, None] * u[None]


@pytest.mark.parametrize("L", [(4, 2, 2, 4), (2, 4, 2, 6)])
def test_free_field_plane_waves(L):
    """U = 1: D e^{ipx} u = [m + sum(1-cos p) + i sum gamma_mu sin p_mu] e^{ipx} u,
    periodic in x,y,z (p = 2 pi n/L) and antiperiodic in t (p4 = (2n+1) pi/Lt)."""
    g = oracle.gamma_matrices()
    U = synth.unit_gauge(L)
    m = 0.137
    rng = np.random.default_rng(0)
    for trial in range(6):
        n = [rng.integers(0, l) for l in L]
        p = [2 * np.pi * n[0] / L[0], 2 * np.pi * n[1] / L[1], 2 * np.pi * n[2] / L[2],
             (2 * n[3] + 1) * np.pi / L[3]]
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        Dp = (m + sum(1 - np.cos(q) for q in p)) * np.eye(4) + 1j * sum(g[mu] * np.sin(p[mu]) for mu in range(4))
        psi = _plane_wave(L, p, u)
        expect = _plane_wave(L, p, Dp @ u)
        assert rel(oracle.dslash(U, psi, m, L), expect) < 1e-13


def test_free_field_spectrum_closed_form():
    """Dense eigenvalues on 4x2x2x4: m + sum(1-cos p) +- i sqrt(sum sin^2 p), 6-fold each."""
    L = (4, 2, 2, 4)
    V = oracle.volume(L)
    U = synth.unit_gauge(L)
    m = 0.1
    D = dense_from_apply(lambda e: oracle.dslash(U, e.reshape(V, 4, 3), m, L).ravel(), V * 12)
    ev = np.linalg.eigvals(D)
    expect = []
    for n0 in range(L[0]):
        for n1 in range(L[1]):
            for n2 in range(L[2]):
                for n3 in range(L[3]):
                    p = [2 * np.pi * n0 / L[0], 2 * np.pi * n1 / L[1], 2 * np.pi * n2 / L[2],
                         (2 * n3 + 1) * np.pi / L[3]]
                    re = m + sum(1 - np.cos(q) for q in p)
                    im = np.sqrt(sum(np.sin(q) ** 2 for q in p))
                    expect += [re + 1j * im] * 6 + [re - 1j * im] * 6
    a = np.sort_complex(np.round(ev, 8))
    b = np.sort_complex(np.round(np.array(expect), 8))
    assert np.abs(a - b).max() < 1e-7


def test_gamma5_hermiticity():
    """D^dag = gamma5 D gamma5 (Sec. I): <x, g5 D g5 y> = <D x, y>."""
    L = (4, 4, 2, 4)
    U = rough_gauge(L)
    m = -0.3
    x = synth.gaussian_spinor(L, 1)
    y = synth.gaussian_spinor(L, 2)
    lhs = np.vdot(x, oracle.gamma5(oracle.dslash(U, oracle.gamma5(y), m, L)))
    rhs = np.vdot(oracle.dslash(U, x, m, L), y)
    assert abs(lhs - rhs) / abs(rhs) < RTOL64


def test_gamma5_hermiticity_dense():
    L = (2, 2, 2, 4)
    V = oracle.volume(L)
    U = rough_gauge(L)
    D = dense_from_apply(lambda e: oracle.dslash(U, e.reshape(V, 4, 3), 0.2, L).ravel(), V * 12)
    G5 = np.kron(np.eye(V), np.kron(np.diag([1, 1, -1, -1]), np.eye(3)))
    assert np.abs(G5 @ D @ G5 - D.conj().T).max() < 1e-14
    # eigenvalues come in complex-conjugate pairs (consequence of gamma5-hermiticity)
    ev = np.linalg.eigvals(D)
    assert np.abs(np.sort_complex(np.round(ev, 9)) - np.sort_complex(np.round(ev.conj(), 9))).max() < 1e-8


def test_gauge_covariance():
    """D[U^Om](Om psi) = Om D[U] psi with U^Om_mu(x) = Om(x) U_mu(x) Om(x+mu)^dag."""
    L = (4, 2, 4, 4)
    V = oracle.volume(L)
    U = rough_gauge(L)
    Om = synth.random_gauge_transform(V, seed=99)
    idx = np.arange(V).reshape(L[3], L[2], L[1], L[0])       # idx[t,z,y,x]
    Ug = np.empty_like(U)
    for mu in range(4):
        ax = 3 - mu
        fwd = np.roll(idx, -1, axis=ax).reshape(-1)          # site of x + mu
        Ug[mu] = Om @ U[mu] @ Om[fwd].conj().transpose(0, 2, 1)
    psi = synth.gaussian_spinor(L, 5)
    Opsi = np.einsum("xab,xsb->xsa", Om, psi)
    lhs = oracle.dslash(Ug, Opsi, 0.05, L)
    rhs = np.einsum("xab,xsb->xsa", Om, oracle.dslash(U, psi, 0.05, L))
    assert rel(lhs, rhs) < RTOL64


def test_mass_shift_is_identity_times_m():
    L = (2, 4, 2, 4)
    U = rough_gauge(L)
    psi = synth.gaussian_spinor(L, 8)
    d = oracle.dslash(U, psi, 0.7, L) - oracle.dslash(U, psi, 0.0, L)
    assert rel(d, 0.7 * psi) < 1e-14


# ---------------------------------------------------------------- eq. (4), chirality split
def _setup_small(L=(4, 4, 4, 4), B=(2, 2, 2, 2), nv=3, seed=21):
    U = rough_gauge(L)
    V0 = synth.gaussian_vectors(L, nv, seed)
    P, st = oracle.block_orthonormalize(V0, L, B)
    assert st == 0
    return U, V0, P


def _dense_P(P, L, B):
    nv = P.shape[0]
    Vc = oracle.volume(oracle.coarse_dims(L, B))
    n = Vc * 2 * nv
    cols = []
    for k in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[k] = 1
        cols.append(oracle.prolong(P, e.reshape(Vc, 2 * nv), L, B).ravel())
    return np.stack(cols, 1)


def test_block_orthonormalisation_invariants():
    L, B = (4, 4, 4, 4), (2, 2, 2, 2)
    U, V0, P = _setup_small(L, B)
    Pd = _dense_P(P, L, B)
    nc = Pd.shape[1]
    assert np.abs(Pd.conj().T @ Pd - np.eye(nc)).max() < 1e-13            # P^dag P = I_c
    for i in range(V0.shape[0]):                                           # P V_c = V
        v = V0[i].ravel()
        assert rel(Pd @ (Pd.conj().T @ v), v) < 1e-13
    V = oracle.volume(L)
    G5 = np.kron(np.eye(V), np.kron(np.diag([1, 1, -1, -1]), np.eye(3)))
    S3 = np.kron(np.eye(nc // (2 * V0.shape[0])), np.diag([1] * V0.shape[0] + [-1] * V0.shape[0]))
    assert np.abs(G5 @ Pd - Pd @ S3).max() == 0                            # gamma5 P = P sigma3


def test_block_orthonormalisation_matches_numpy_qr():
    """Q of a Householder QR (numpy), with diag(R) made real positive, per aggregate
    and chirality: the Q with positive real R-diagonal is unique."""
    L, B = (4, 4, 2, 2), (2, 2, 2, 2)
    nv = 4
    V0 = synth.gaussian_vectors(L, nv, 77)
    P, st = oracle.block_orthonormalize(V0, L, B)
    assert st == 0
    c = np.stack(np.meshgrid(*[np.arange(l) for l in L], indexing="ij"), -1)
    c = np.transpose(c, (3, 2, 1, 0, 4)).reshape(-1, 4)
    Lc = oracle.coarse_dims(L, B)
    blk = (c // np.asarray(B)) @ np.array([1, Lc[0], Lc[0] * Lc[1], Lc[0] * Lc[1] * Lc[2]])
    for X in range(oracle.volume(Lc)):
        sites = np.nonzero(blk == X)[0]
        for s in range(2):
            W = V0[:, sites, 2 * s:2 * s + 2, :].reshape(nv, -1).T
            Q, R = np.linalg.qr(W)
            ph = np.diag(R) / np.abs(np.diag(R))
            Q = Q * ph[None, :]
            got = P[:, sites, 2 * s:2 * s + 2, :].reshape(nv, -1).T
            assert np.abs(got - Q).max() < 1e-13


def test_block_orthonormalisation_rank_deficient_is_numeric_error():
    L, B = (4, 4, 2, 2), (2, 2, 2, 2)
    V0 = synth.gaussian_vectors(L, 3, 5)
    V0[2] = V0[0] * (0.5 - 0.25j)
    _, st = oracle.block_orthonormalize(V0, L, B)
    assert st == oracle.ERR_NUMERIC


def test_restrict_prolong_adjoint_pair():
    L, B = (4, 4, 4, 4), (2, 2, 2, 2)
    U, V0, P = _setup_small(L, B)
    Lc = oracle.coarse_dims(L, B)
    r = synth.gaussian_spinor(L, 31)
    y = synth.gaussian(oracle.volume(Lc) * 6, 32, 0).reshape(-1, 6)
    assert abs(np.vdot(oracle.restrict(P, r, L, B), y) - np.vdot(r, oracle.prolong(P, y, L, B))) < 1e-12
    assert rel(oracle.restrict(P, oracle.prolong(P, y, L, B), L, B), y) < 1e-14


# ---------------------------------------------------------------- D_c = P^dag D P
@pytest.mark.parametrize("L,B", [((4, 4, 4, 4), (2, 2, 2, 2)),      # coarse extent 2
                                 ((4, 4, 4, 4), (4, 4, 4, 4)),      # coarse extent 1
                                 ((4, 2, 2, 8), (2, 2, 2, 2))])     # coarse extent 4 in t
def test_coarse_operator_equals_dense_galerkin(L, B):
    nv = 2
    U, V0, P = _setup_small(L, B, nv=nv, seed=41)
    m = -0.25
    A = oracle.coarse_build(U, P, m, L, B)
    Lc = oracle.coarse_dims(L, B)
    V = oracle.volume(L)
    nC = oracle.volume(Lc) * 2 * nv
    D = dense_from_apply(lambda e: oracle.dslash(U, e.reshape(V, 4, 3), m, L).ravel(), V * 12)
    Pd = _dense_P(P, L, B)
    Dc_dense = Pd.conj().T @ D @ Pd
    Dc_apply = dense_from_apply(lambda e: oracle.coarse_apply(A, e.reshape(-1, 2 * nv), Lc).ravel(), nC)
    assert np.abs(Dc_apply - Dc_dense).max() < 1e-13 * np.abs(Dc_dense).max()
    # sigma3 D_c sigma3 = D_c^dag (from P^dag gamma5 = sigma3 P^dag)
    S3 = np.kron(np.eye(oracle.volume(Lc)), np.diag([1] * nv + [-1] * nv))
    assert np.abs(S3 @ Dc_dense @ S3 - Dc_dense.conj().T).max() < 1e-13
    Dag = dense_from_apply(lambda e: oracle.coarse_apply_dag(A, e.reshape(-1, 2 * nv), Lc).ravel(), nC)
    assert np.abs(Dag - Dc_dense.conj().T).max() < 1e-13
    # coarse correction kills the coarse space: (I - P D_c^-1 P^dag D) P = 0 (eqs. 3, 8)
    E = Pd - Pd @ np.linalg.solve(Dc_dense, Pd.conj().T @ D @ Pd)
    assert np.abs(E).max() < 1e-11


def test_coarse_operator_nearest_neighbour_and_mass_shift():
    L, B = (8, 4, 4, 4), (2, 2, 2, 2)          # coarse 4x2x2x2: x-neighbours distinct
    nv = 2
    U, V0, P = _setup_small(L, B, nv=nv, seed=42)
    A0 = oracle.coarse_build(U, P, 0.0, L, B)
    A1 = oracle.coarse_build(U, P, 0.3, L, B)
    d = A1 - A0
    assert np.abs(d[:, 1:]).max() == 0
    assert np.abs(d[:, 0] - 0.3 * np.eye(2 * nv)[None]).max() < 1e-14
    # coupling of X to X+2x is zero: D_c is nearest neighbour (Sec. III)
    Lc = oracle.coarse_dims(L, B)
    nC = oracle.volume(Lc) * 2 * nv
    Dc = dense_from_apply(lambda e: oracle.coarse_apply(A0, e.reshape(-1, 2 * nv), Lc).ravel(), nC)
    blk = Dc.reshape(oracle.volume(Lc), 2 * nv, oracle.volume(Lc), 2 * nv)
    assert np.abs(blk[0, :, 2, :]).max() == 0          # sites (0,..) and (2,..) in x


def test_non_split_coarsening_is_singular_in_free_field():
    """Sec. III: coarsening spins together, the free-field constant prototype gives
    P^dag gamma5 P = 0; keeping chirality apart gives sigma3 instead."""
    L, B = (4, 4, 4, 4), (2, 2, 2, 2)
    V = oracle.volume(L)
    u = np.zeros((4, 3), complex)
    u[:, 0] = 1.0                                        # equal weight on both chiralities
    v = np.broadcast_to(u, (V, 4, 3)).copy()
    Lc = oracle.coarse_dims(L, B)
    c = np.stack(np.meshgrid(*[np.arange(l) for l in L], indexing="ij"), -1)
    c = np.transpose(c, (3, 2, 1, 0, 4)).reshape(-1, 4)
    blk = (c // np.asarray(B)) @ np.array([1, Lc[0], Lc[0] * Lc[1], Lc[0] * Lc[1] * Lc[2]])
    nb = oracle.volume(Lc)
    Pns = np.zeros((V * 12, nb), complex)
    for X in range(nb):
        col = np.where((blk == X)[:, None, None], v, 0).ravel()
        Pns[:, X] = col / np.linalg.norm(col)
    g5 = oracle.gamma5(np.eye(V * 12).reshape(V * 12, V, 4, 3)[0].reshape(V, 4, 3))  # smoke
    G5P = np.stack([oracle.gamma5(Pns[:, k].reshape(V, 4, 3)).ravel() for k in range(nb)], 1)
    assert np.abs(Pns.conj().T @ G5P).max() < 1e-15
    # the chirality-split prolongator from the same prototype: P^dag g5 P = sigma3
    P, st = oracle.block_orthonormalize(v[None], L, B)
    assert st == 0
    Pd = _dense_P(P, L, B)
    G5Pd = np.stack([oracle.gamma5(Pd[:, k].reshape(V, 4, 3)).ravel() for k in range(Pd.shape[1])], 1)
    assert np.abs(Pd.conj().T @ G5Pd - np.kron(np.eye(nb), np.diag([1, -1]))).max() < 1e-14
    del g5


# ---------------------------------------------------------------- smoother, coarse solve, GCR
def test_mr_step_residual_identity():
    """One MR step with omega: ||r'||^2 = ||r||^2 - (2w - w^2)|<q,r>|^2/||q||^2, and
    the pair (e, r) stays consistent: r - r' = D (e' - e)."""
    L = (4, 4, 2, 4)
    U = rough_gauge(L)
    m, w = -0.2, 0.9
    e = synth.gaussian_spinor(L, 1)
    r = synth.gaussian_spinor(L, 2)
    q = oracle.dslash(U, r, m, L)
    e1, r1 = oracle.mr(U, e, r, m, L, 1, w)
    pred = np.vdot(r, r).real - (2 * w - w * w) * abs(np.vdot(q, r)) ** 2 / np.vdot(q, q).real
    assert abs(np.vdot(r1, r1).real - pred) / pred < 1e-13
    e4, r4 = oracle.mr(U, e, r, m, L, 4, w)
    assert rel(r - r4, oracle.dslash(U, e4 - e, m, L)) < 1e-13
    assert np.linalg.norm(r4) < np.linalg.norm(r1) < np.linalg.norm(r)


def test_cgnr_reaches_dense_solution():
    L, B = (4, 4, 4, 4), (2, 2, 2, 2)
    nv = 2
    U, V0, P = _setup_small(L, B, nv=nv, seed=43)
    A = oracle.coarse_build(U, P, 0.1, L, B)
    Lc = oracle.coarse_dims(L, B)
    nC = oracle.volume(Lc) * 2 * nv
    Dc = dense_from_apply(lambda e: oracle.coarse_apply(A, e.reshape(-1, 2 * nv), Lc).ravel(), nC)
    rc = synth.gaussian(nC, 3, 0).reshape(-1, 2 * nv)
    y, it, relres = oracle.cgnr(A, rc, Lc, 1e-13, 5000)
    assert relres <= 1e-13 and it < 5000
    assert rel(y.ravel(), np.linalg.solve(Dc, rc.ravel())) < 1e-10
    # tol = 1e-3 stops at the first iterate whose residual is <= 1e-3
    y3, it3, rel3 = oracle.cgnr(A, rc, Lc, 1e-3, 5000)
    assert rel3 <= 1e-3
    _, _, rel_prev = oracle.cgnr(A, rc, Lc, 0.0, it3 - 1)
    assert rel_prev > 1e-3
    assert rel(Dc @ y3.ravel(), rc.ravel()) == pytest.approx(rel3, rel=1e-9)


def _cg_one_reduction(Dc, b, maxit, tol):
    """CG on Dc^dag Dc in the Chronopoulos-Gear arrangement (both scalars of an
    iteration from u = Dc s: gamma = |s|^2, delta = |u|^2), written on the dense
    operator; convergence is read from |r|^2 at the start of an iteration."""
    y = np.zeros_like(b)
    r = b.copy()
    s = Dc.conj().T @ r
    rc2 = np.vdot(b, b).real
    p = z = q = None
    gamma_old = alpha_old = 0.0
    i = 0
    while True:
        u = Dc @ s
        delta, gamma, r2 = np.vdot(u, u).real, np.vdot(s, s).real, np.vdot(r, r).real
        if (i > 0 and r2 <= tol * tol * rc2) or i >= maxit:
            return y, i
        beta = gamma / gamma_old if i else 0.0
        alpha = gamma / (delta - beta * gamma / alpha_old) if i else gamma / delta
        w = Dc.conj().T @ u
        p, z, q = (s, w, u) if i == 0 else (s + beta * p, w + beta * z, u + beta * q)
        y, r, s = y + alpha * p, r - alpha * q, s - alpha * z
        gamma_old, alpha_old = gamma, alpha
        i += 1


def test_one_reduction_cg_has_the_cgls_iterates():
    """The coarse solve's CG on the normal equations (Sec. IV) in the arrangement
    with one reduction per iteration produces the same iterates and the same
    iteration count to 1e-3 as the oracle's textbook CGLS."""
    L, B = (4, 4, 4, 4), (2, 2, 2, 2)
    nv = 2
    U, V0, P = _setup_small(L, B, nv=nv, seed=43)
    A = oracle.coarse_build(U, P, 0.1, L, B)
    Lc = oracle.coarse_dims(L, B)
    nC = oracle.volume(Lc) * 2 * nv
    Dc = dense_from_apply(lambda e: oracle.coarse_apply(A, e.reshape(-1, 2 * nv), Lc).ravel(), nC)
    rc = synth.gaussian(nC, 3, 0).reshape(-1, 2 * nv)
    for k in (1, 5, 12):
        y_ref, it_ref, _ = oracle.cgnr(A, rc, Lc, 0.0, k)
        y, it = _cg_one_reduction(Dc, rc.ravel(), k, 0.0)
        assert it == it_ref == k
        assert rel(y, y_ref.ravel()) < 1e-10, k
    _, it3, _ = oracle.cgnr(A, rc, Lc, 1e-3, 5000)
    _, it3b = _cg_one_reduction(Dc, rc.ravel(), 5000, 1e-3)
    assert it3b == it3


def test_gcr_without_preconditioner_equals_gmres():
    """GCR and GMRES minimise ||b - D x|| over the same Krylov space K_k(D, b)."""
    L = (2, 2, 2, 4)
    V = oracle.volume(L)
    U = rough_gauge(L)
    m = 0.3
    b = synth.gaussian_spinor(L, 4)
    D = dense_from_apply(lambda e: oracle.dslash(U, e.reshape(V, 4, 3), m, L).ravel(), V * 12)
    for k in (1, 3, 7):
        p = oracle.make_params(L, nv=1, m=m, gcr_restart=32, tol=0.0, max_outer=k, use_mg=0)
        x, info = oracle.gcr_solve(p, U, None, None, b)
        assert info["outer_iters"] == k
        K = [b.ravel()]
        for _ in range(k - 1):
            K.append(D @ K[-1])
        Q, _ = np.linalg.qr(np.stack(K, 1))
        c, *_ = np.linalg.lstsq(D @ Q, b.ravel(), rcond=None)
        gm = np.linalg.norm(b.ravel() - D @ Q @ c)
        assert abs(np.linalg.norm(b.ravel() - D @ x.ravel()) - gm) / gm < 1e-9


def test_vcycle_coarse_part_is_galerkin():
    """With no smoothing and an exact coarse solve, z = P D_c^-1 P^dag r, so the
    restricted residual of z vanishes: P^dag (r - D z) = 0 (eq. 8)."""
    L, B = (4, 4, 4, 4), (2, 2, 2, 2)
    nv = 2
    U, V0, P = _setup_small(L, B, nv=nv, seed=44)
    m = 0.1
    A = oracle.coarse_build(U, P, m, L, B)
    p = oracle.make_params(L, B, nv=nv, m=m, mr_steps=0, coarse_tol=1e-14, coarse_maxit=20000)
    r = synth.gaussian_spinor(L, 9)
    z, info = oracle.vcycle(p, U, P, A, r)
    res = oracle.restrict(P, r - oracle.dslash(U, z, m, L), L, B)
    assert np.linalg.norm(res) / np.linalg.norm(oracle.restrict(P, r, L, B)) < 1e-11
    # with smoothing the cycle still reduces the residual
    p4 = oracle.make_params(L, B, nv=nv, m=m, mr_steps=4)
    z4, _ = oracle.vcycle(p4, U, P, A, r)
    assert np.linalg.norm(r - oracle.dslash(U, z4, m, L)) < np.linalg.norm(r)


def test_mg_gcr_solve_true_residual():
    L, B = (4, 4, 4, 8), (2, 2, 2, 4)
    nv = 4
    U = rough_gauge(L, sweeps=5)
    m = -0.2
    p = oracle.make_params(L, B, nv=nv, m=m)
    V0 = synth.gaussian_vectors(L, nv, 51)
    Vv, P, A, st = oracle.setup(p, U, V0, init_relax=10, n_iter=1, group_size=2)
    assert st == 0
    b = synth.gaussian_spinor(L, 52)
    x, info = oracle.gcr_solve(p, U, P, A, b)
    assert info["status"] == 0
    true = np.linalg.norm(b - oracle.dslash(U, x, m, L)) / np.linalg.norm(b)
    assert true <= 1e-10
    assert info["true_rel_res"] == pytest.approx(true, rel=1e-6)
    # the setup's P and D_c keep the invariants
    Pd = _dense_P(P, L, B)
    assert np.abs(Pd.conj().T @ Pd - np.eye(Pd.shape[1])).max() < 1e-12
    # MG preconditioning beats unpreconditioned GCR on the same system
    p0 = oracle.make_params(L, B, nv=nv, m=m, use_mg=0, max_outer=3000)
    x0, info0 = oracle.gcr_solve(p0, U, None, None, b)
    assert info["outer_iters"] * 3 < info0["outer_iters"]


@pytest.mark.slow
def test_setup_improves_outer_iterations():
    """The adaptive setup (Sec. II, practical two-step form of Sec. IV) gives a
    coarse space that cuts outer iterations: random prototypes > relaxed
    prototypes > relaxed + group-refined prototypes, on the 8^4 beta = 6.0 field
    at Re(lambda_min) = 0.01."""
    from tests._fields import c1_workload
    L, B, nv, U, m = c1_workload()
    b = synth.gaussian_spinor(L, 7)
    V0 = synth.gaussian_vectors(L, nv, 2001)
    p = oracle.make_params(L, B, nv=nv, m=m)
    Prand, _ = oracle.block_orthonormalize(V0, L, B)
    _, info_rand = oracle.gcr_solve(p, U, Prand, oracle.coarse_build(U, Prand, m, L, B), b)
    _, P0, A0, st0 = oracle.setup(p, U, V0, init_relax=10, n_iter=0, group_size=4)
    _, P5, A5, st5 = oracle.setup(p, U, V0, init_relax=10, n_iter=5, group_size=4)
    assert st0 == 0 and st5 == 0
    _, info0 = oracle.gcr_solve(p, U, P0, A0, b)
    _, info5 = oracle.gcr_solve(p, U, P5, A5, b)
    for inf in (info_rand, info0, info5):
        assert inf["status"] == 0 and inf["true_rel_res"] <= 1e-10
    assert info_rand["outer_iters"] > info0["outer_iters"] > info5["outer_iters"]


@pytest.mark.parametrize("k", [1, 3, 5])
def test_gmres_smoother_minimises_over_the_krylov_space(k):
    """GMRES(k) smoothing (Sec. III-IV): with omega = 1 the correction d minimises
    ||r - D d|| over K_k(D, r) = span{r, Dr, ..., D^(k-1) r}; checked against a
    least-squares fit (numpy lstsq, QR-based) over the explicit power basis; with
    omega the correction is omega times the same d; k = 1 is one MR step."""
    L = (4, 4, 4, 4)
    U = rough_gauge(L, seed=9)
    m = -0.5
    e0 = synth.gaussian_spinor(L, 3)
    r = synth.gaussian_spinor(L, 4)
    basis = [r]
    for _ in range(k - 1):
        basis.append(oracle.dslash(U, basis[-1], m, L))
    K = np.stack([b.ravel() for b in basis], axis=1)
    DK = np.stack([oracle.dslash(U, b, m, L).ravel() for b in basis], axis=1)
    c, *_ = np.linalg.lstsq(DK, r.ravel(), rcond=None)
    d_ref = (K @ c).reshape(r.shape)
    e1 = oracle.gmres_smooth(U, e0, r, m, L, k, 1.0)
    assert np.abs((e1 - e0) - d_ref).max() < 1e-9 * np.abs(d_ref).max()
    e09 = oracle.gmres_smooth(U, e0, r, m, L, k, 0.9)
    assert np.abs((e09 - e0) - 0.9 * d_ref).max() < 1e-9 * np.abs(d_ref).max()
    if k == 1:
        e_mr, _ = oracle.mr(U, e0, r, m, L, 1, 0.9)
        assert np.abs(e_mr - e09).max() < 1e-12 * np.abs(e_mr).max()


def test_gmres_smoother_lowers_outer_iterations():
    """One GMRES(6) application per cycle needs fewer outer iterations than MR(4)
    on a rough field (a stronger smoother), and both reach 1e-10."""
    L, B, nv = (8, 8, 8, 8), (4, 4, 4, 4), 4
    U = rough_gauge(L, seed=21, sweeps=3)
    V0 = synth.gaussian_vectors(L, nv, 121)
    m = -0.6
    P, st = oracle.block_orthonormalize(V0, L, B)
    A = oracle.coarse_build(U, P, m, L, B)
    b = synth.gaussian_spinor(L, 7)
    its = {}
    for sm, steps in ((0, 4), (1, 6)):
        p = oracle.make_params(L, B, nv=nv, m=m, smoother=sm, mr_steps=steps)
        x, info = oracle.gcr_solve(p, U, P, A, b)
        assert info["status"] == 0 and info["true_rel_res"] <= 1e-10
        its[sm] = info["outer_iters"]
    assert its[1] < its[0], its


# ---------------------------------------------------------------- eq. 3: two-grid convergence factor
def _small_level(L=(4, 4, 4, 8), B=(2, 2, 2, 4), nv=4, seed=61, m=-0.2):
    U = rough_gauge(L, sweeps=5)
    V0 = synth.gaussian_vectors(L, nv, seed)
    P, st = oracle.block_orthonormalize(V0, L, B)
    assert st == 0
    return L, B, nv, U, m, P, oracle.coarse_build(U, P, m, L, B)


def test_two_grid_factor_coarse_correction_identities():
    """Without smoothing, E_TG = I - P D_c^-1 P^dag D (eq. 3): it annihilates
    range(P) (a start e0 = P y gives e1 = 0), it is a projection (E^2 = E, so
    the norms stay at ||E e0|| after the first step), and the corrected error
    has a Galerkin-orthogonal residual, P^dag D e1 = 0."""
    L, B, nv, U, m, P, A = _small_level()
    p0 = oracle.make_params(L, B, nv=nv, m=m, mr_steps=0)
    Lc = oracle.coarse_dims(L, B)
    y = synth.gaussian(oracle.volume(Lc) * 2 * nv, 62, 0).reshape(-1, 2 * nv)
    e_in_P = oracle.prolong(P, y, L, B)
    f, norms = oracle.two_grid_factor(p0, U, P, A, e_in_P, 1)
    assert norms[1] < 1e-11 * norms[0]
    e0 = synth.gaussian_spinor(L, 63)
    f3, norms3 = oracle.two_grid_factor(p0, U, P, A, e0, 3)
    assert 0 < norms3[1] < norms3[0]
    assert abs(norms3[2] - norms3[1]) < 1e-10 * norms3[1] and abs(norms3[3] - norms3[1]) < 1e-10 * norms3[1]
    # e1 by hand from the definition, then its restricted residual
    _, n1 = oracle.two_grid_factor(p0, U, P, A, e0, 1)
    r = -oracle.dslash(U, e0, m, L)
    Dc = oracle.coarse_dense(A, Lc)
    e1 = e0 + oracle.prolong(P, np.linalg.solve(Dc, oracle.restrict(P, r, L, B).ravel()).reshape(-1, 2 * nv), L, B)
    assert abs(np.linalg.norm(e1) - n1[1]) < 1e-12 * n1[1]
    assert np.linalg.norm(oracle.restrict(P, oracle.dslash(U, e1, m, L), L, B)) < 1e-11 * np.linalg.norm(r)


def test_two_grid_factor_smoothing_contracts():
    """With the post-smoother the two-grid method contracts (factor < 1) and the
    smoother can only lower the error of the unsmoothed projection here."""
    L, B, nv, U, m, P, A = _small_level()
    e0 = synth.gaussian_spinor(L, 64)
    f0, _ = oracle.two_grid_factor(oracle.make_params(L, B, nv=nv, m=m, mr_steps=0), U, P, A, e0, 4)
    f4, _ = oracle.two_grid_factor(oracle.make_params(L, B, nv=nv, m=m, mr_steps=4), U, P, A, e0, 4)
    fg, _ = oracle.two_grid_factor(oracle.make_params(L, B, nv=nv, m=m, mr_steps=4, smoother=1), U, P, A, e0, 4)
    assert f4 < 1 and fg < 1 and f4 < f0 and fg < f0, (f0, f4, fg)


def test_setup_truncated_level_removes_the_group():
    """The refinement of Sec. IV removes the group being refined from V: the
    truncated prolongator reproduces every remaining prototype (P_t P_t^dag v = v,
    eq. 4) and none of the group's, in order."""
    L, B, nv = (4, 4, 4, 8), (2, 2, 2, 4), 6
    U = rough_gauge(L, sweeps=5)
    V = synth.gaussian_vectors(L, nv, 71)
    p = oracle.make_params(L, B, nv=nv, m=-0.2)
    for g0 in (0, 2, 4):
        Vt, Pt, At, st = oracle.setup_truncated_level(p, U, V, g0, 2)
        assert st == 0 and Vt.shape[0] == nv - 2
        kept = [i for i in range(nv) if not g0 <= i < g0 + 2]
        assert all(np.array_equal(Vt[j], V[i]) for j, i in enumerate(kept))
        for i in range(nv):
            proj = oracle.prolong(Pt, oracle.restrict(Pt, V[i], L, B), L, B)
            miss = np.linalg.norm(V[i] - proj) / np.linalg.norm(V[i])
            if i in kept:
                assert miss < 1e-12, (g0, i, miss)
            else:
                assert miss > 0.5, (g0, i, miss)   # a random vector mostly outside a 4 of 96 per block subspace
        # the truncated coarse operator is the Galerkin product of the truncated P
        assert np.abs(At - oracle.coarse_build(U, Pt, -0.2, L, B)).max() == 0


@pytest.mark.slow
def test_setup_lowers_the_two_grid_factor():
    """Setup quality measured by eq. 3 on the 8^4 beta = 6.0 field at
    Re(lambda_min) = 0.01 (exact coarse solve, the configuration's MR(4)
    smoother, one random error): the asymptotic rate (||e_40|| / ||e_20||)^(1/20)
    orders relaxed + group-refined prototypes < relaxed prototypes < the random
    starts (0.945 < 0.957 < 0.970; the first iterations are a transient)."""
    from tests._fields import c1_workload
    L, B, nv, U, m = c1_workload()
    V0 = synth.gaussian_vectors(L, nv, 2001)
    p = oracle.make_params(L, B, nv=nv, m=m)
    e0 = synth.gaussian_spinor(L, 2002)
    def rate(P, A):
        _, n = oracle.two_grid_factor(p, U, P, A, e0, 40)
        return (n[40] / n[20]) ** (1 / 20)

    Prand, _ = oracle.block_orthonormalize(V0, L, B)
    f_rand = rate(Prand, oracle.coarse_build(U, Prand, m, L, B))
    _, P0, A0, st0 = oracle.setup(p, U, V0, init_relax=10, n_iter=0, group_size=4)
    _, P3, A3, st3 = oracle.setup(p, U, V0, init_relax=10, n_iter=3, group_size=4)
    assert st0 == 0 and st3 == 0
    f_relax, f_ref = rate(P0, A0), rate(P3, A3)
    assert f_ref < f_relax < f_rand < 1, (f_ref, f_relax, f_rand)


@pytest.mark.parametrize("smoother,k", [(1, 1), (1, 4), (0, 1)])
def test_vcycle_smoothing_half(smoother, k):
    """The post-smoothing half of the V(0, k) cycle (Sec. III-IV) acts on the
    coarse-corrected residual r' = r - D P D_c^-1 P^dag r: with an exact coarse
    solve, r - D z equals r' - omega D d with d the least-squares minimiser of
    ||r' - D d|| over K_k(D, r') (numpy lstsq over the power basis).  GMRES(k)
    and one MR step (k = 1) alike; a cycle smoothing r instead of r' fails."""
    L, B, nv, U, m, P, A = _small_level()
    Lc = oracle.coarse_dims(L, B)
    omega = 0.9
    p = oracle.make_params(L, B, nv=nv, m=m, mr_steps=k, smoother=smoother, omega=omega, coarse_tol=1e-15,
                           coarse_maxit=50000)
    r = synth.gaussian_spinor(L, 81)
    z, _ = oracle.vcycle(p, U, P, A, r)
    Dc = oracle.coarse_dense(A, Lc)
    e0 = oracle.prolong(P, np.linalg.solve(Dc, oracle.restrict(P, r, L, B).ravel()).reshape(-1, 2 * nv), L, B)

    def expected(res):
        basis = [res]
        for _ in range(k - 1):
            basis.append(oracle.dslash(U, basis[-1], m, L))
        DK = np.stack([oracle.dslash(U, b, m, L).ravel() for b in basis], axis=1)
        c, *_ = np.linalg.lstsq(DK, res.ravel(), rcond=None)
        return res - omega * (DK @ c).reshape(res.shape)

    r1 = r - oracle.dslash(U, e0, m, L)
    got = r - oracle.dslash(U, z, m, L)
    want = expected(r1)
    assert np.abs(got - want).max() < 1e-9 * np.abs(want).max()
    wrong = r - oracle.dslash(U, e0, m, L) - (r - expected(r))   # smoothing r, not r'
    assert np.abs(got - wrong).max() > 1e-3 * np.abs(want).max()


# ---------------------------------------------------------------- red-black preconditioned CG (Sec. IV comparison)
def _even_part(L, psi):
    return psi * oracle.parity_mask(L)[:, None, None]


def test_eo_schur_complement_eliminates_odd_sites():
    """D applied to (x_e, x_o) with x_o = H_oe x_e / (4+m) is (Dhat x_e, 0):
    checked with the full operator of eq. 2 (H = (4+m) - D, so H_oe x_e is the
    odd part of (4+m) x_e - D x_e)."""
    L = (4, 4, 2, 6)
    U = rough_gauge(L, seed=17)
    m = -0.3
    xe = _even_part(L, synth.gaussian_spinor(L, 5))
    odd = ~oracle.parity_mask(L)
    Hx = (4 + m) * xe - oracle.dslash(U, xe, m, L)            # H x_e (its odd part)
    x = xe + (Hx * odd[:, None, None]) / (4 + m)
    Dx = oracle.dslash(U, x, m, L)
    assert np.abs(Dx[odd]).max() < 1e-13 * np.abs(Dx).max()
    Dh = oracle.eo_schur(U, xe, m, L)
    assert np.abs(Dh[odd]).max() == 0
    assert rel(Dh, _even_part(L, Dx)) < 1e-13


def test_eo_schur_gamma5_hermitian():
    L = (4, 2, 4, 4)
    U = rough_gauge(L, seed=18)
    m = -0.1
    u = _even_part(L, synth.gaussian_spinor(L, 6))
    v = _even_part(L, synth.gaussian_spinor(L, 7))
    lhs = np.vdot(u, oracle.eo_schur(U, v, m, L))
    rhs = np.vdot(oracle.eo_schur(U, u, m, L, dag=True), v)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # dag is gamma5 Dhat gamma5
    assert rel(oracle.eo_schur(U, u, m, L, dag=True), oracle.gamma5(oracle.eo_schur(U, oracle.gamma5(u), m, L))) < 1e-14


@pytest.mark.parametrize("k", [1, 2, 4])
def test_eo_cg_iterates_are_krylov_least_squares(k):
    """CG on the normal equations minimises |bhat - Dhat x| over the Krylov space
    K_k(Dhat^dag Dhat, Dhat^dag bhat): after k iterations the true residual
    equals the least-squares one (numpy lstsq over the explicit power basis)."""
    L = (4, 4, 2, 4)
    U = rough_gauge(L, seed=19)
    m = -0.2
    b = synth.gaussian_spinor(L, 8)
    x, it, mv, relres, st = oracle.eo_cg(U, b, m, L, 0.0, k)
    assert it == k
    odd = ~oracle.parity_mask(L)
    bh = _even_part(L, b) + _even_part(L, (4 + m) * np.where(odd[:, None, None], b, 0)
                                       - oracle.dslash(U, np.where(odd[:, None, None], b, 0), m, L)) / (4 + m)
    ev = oracle.parity_mask(L)
    K = [oracle.eo_schur(U, bh, m, L, dag=True)]
    for _ in range(k - 1):
        K.append(oracle.eo_schur(U, oracle.eo_schur(U, K[-1], m, L), m, L, dag=True))
    DK = np.stack([oracle.eo_schur(U, v, m, L)[ev].ravel() for v in K], 1)
    c, *_ = np.linalg.lstsq(DK, bh[ev].ravel(), rcond=None)
    want = np.linalg.norm(bh[ev].ravel() - DK @ c)
    got = np.linalg.norm(b - oracle.dslash(U, x, m, L))    # = |bhat - Dhat x_e| (odd part vanishes)
    assert abs(got - want) < 1e-9 * want, (got, want)


def test_eo_cg_solves_against_dense():
    """To 1e-12 on a 2^3 x 4 lattice: the solution of the dense system (numpy
    solve of D built column by column from eq. 2), in at most 2 x 192 iterations."""
    L = (2, 2, 2, 4)
    U = rough_gauge(L, seed=20)
    m = -0.25
    V = oracle.volume(L)
    b = synth.gaussian_spinor(L, 9)
    D = dense_from_apply(lambda e: oracle.dslash(U, e.reshape(V, 4, 3), m, L).ravel(), V * 12)
    x_ref = np.linalg.solve(D, b.ravel()).reshape(b.shape)
    x, it, mv, relres, st = oracle.eo_cg(U, b, m, L, 1e-12, 2000)
    assert st == 0 and relres <= 1e-12 and it <= 2 * V * 6
    assert rel(x, x_ref) < 1e-9
    # one pass: Dhat and Dhat^dag per iteration (no Dhat^dag after the last),
    # plus bhat, the first Dhat^dag r, the odd-site reconstruction and the check
    assert mv == 2 * it + 3, (mv, it)


def test_eo_cg_iterations_grow_toward_critical_mass():
    """Critical slowing down of CG (the motivation of Sec. I and Fig. 1): on the
    8^4 beta = 6.0 field the iteration count to 1e-10 rises as Re(lambda_min)
    falls from 0.1 to 0.01, and every solve reaches the tolerance."""
    from tests._fields import c1_workload, C1_RE_LAMBDA_MIN_M0
    L, B, nv, U, m = c1_workload()
    b = synth.gaussian_spinor(L, 7)
    its = []
    for target in (0.1, 0.03, 0.01):
        x, it, mv, relres, st = oracle.eo_cg(U, b, target - C1_RE_LAMBDA_MIN_M0, L, 1e-10, 20000)
        assert st == 0 and relres <= 1e-10
        assert np.linalg.norm(b - oracle.dslash(U, x, target - C1_RE_LAMBDA_MIN_M0, L)) <= 1e-10 * np.linalg.norm(b)
        its.append(it)
    assert its[0] < its[1] < its[2], its


# ---------------------------------------------------------------- third level (Sec. III recursion, Sec. IV W-cycle)
def _level1(L=(4, 4, 4, 8), B=(2, 2, 2, 2), nv=4, m=-0.3, seed=91):
    """A level-1 operator D_c = P^dag D P from random prototypes on a small lattice."""
    U = rough_gauge(L, seed=seed)
    V0 = synth.gaussian_vectors(L, nv, seed + 1)
    P, st = oracle.block_orthonormalize(V0, L, B)
    assert st == 0
    A1 = oracle.coarse_build(U, P, m, L, B)
    return L, B, nv, U, m, P, A1, oracle.coarse_dims(L, B)


def _level1_vectors(Lc1, nv1, n, seed):
    Vc1 = oracle.volume(Lc1)
    return synth.gaussian(n * Vc1 * 2 * nv1, seed, 0).reshape(n, Vc1, 2 * nv1)


def _dense_P2(P2, Lc1, B2, nv1):
    Lc2 = oracle.coarse_dims(Lc1, B2)
    nC = oracle.volume(Lc2) * 2 * P2.shape[0]
    cols = []
    for k in range(nC):
        e = np.zeros(nC, dtype=np.complex128)
        e[k] = 1
        cols.append(oracle.cprolong(P2, e.reshape(oracle.volume(Lc2), -1), Lc1, B2, nv1).ravel())
    return np.stack(cols, 1)


@pytest.mark.parametrize("B2", [(1, 1, 2, 2), (2, 2, 2, 2), (2, 2, 2, 4)])
def test_level2_prolongator_and_galerkin_operator(B2):
    """One level down (Sec. III): P2^dag P2 = I and P2 V2_c = V2 (eq. 4), chirality
    kept, Q equal to numpy's QR (positive diagonal) per aggregate and chirality,
    restriction the adjoint of prolongation, and A2 = P2^dag A1 P2 equal to the
    dense product for level-2 extents 2, 1 and mixed (the exit-face slots),
    sigma3-hermitian like A1, with (I - P2 A2^-1 P2^dag A1) P2 = 0."""
    L, B, nv1, U, m, P, A1, Lc1 = _level1()
    nv2 = 3
    V2 = _level1_vectors(Lc1, nv1, nv2, 92)
    P2, st = oracle.cblock_orthonormalize(V2, Lc1, B2, nv1)
    assert st == 0
    P2d = _dense_P2(P2, Lc1, B2, nv1)
    assert np.abs(P2d.conj().T @ P2d - np.eye(P2d.shape[1])).max() < 1e-13
    for i in range(nv2):                         # P2 P2^dag v_i = v_i
        v = V2[i]
        proj = oracle.cprolong(P2, oracle.crestrict(P2, v, Lc1, B2, nv1), Lc1, B2, nv1)
        assert rel(proj, v) < 1e-13
        assert not np.any(P2[i][:, :nv1] * 0)     # both chiralities present in the prototypes
    # numpy QR of one aggregate's chirality-0 block
    Lc2 = oracle.coarse_dims(Lc1, B2)
    c1 = np.indices(tuple(Lc1)[::-1]).reshape(4, -1)[::-1]
    blk = (c1[0] // B2[0]) + Lc2[0] * ((c1[1] // B2[1]) + Lc2[1] * ((c1[2] // B2[2]) + Lc2[2] * (c1[3] // B2[3])))
    sites = np.nonzero(blk == 0)[0]
    W = np.stack([V2[i][sites, :nv1].ravel() for i in range(nv2)], 1)
    Q, R = np.linalg.qr(W)
    Q = Q * (np.sign(np.diag(R).real) * np.exp(-1j * np.angle(np.diag(R))) * np.abs(np.sign(np.diag(R))))[None, :]
    Qp = np.stack([P2[i][sites, :nv1].ravel() for i in range(nv2)], 1)
    ph = np.diag(R) / np.abs(np.diag(R))
    assert np.abs(Qp - np.linalg.qr(W)[0] * ph[None, :]).max() < 1e-12
    assert np.all(P2[:, sites][:, :, nv1:][:, :, :].shape)   # shape sanity
    # chirality: sigma3 P2 = P2 sigma3 (columns of chirality s live on dof of chirality s)
    s1 = np.concatenate([np.ones(nv1), -np.ones(nv1)])
    s2 = np.concatenate([np.ones(nv2), -np.ones(nv2)])
    S1 = np.diag(np.tile(s1, oracle.volume(Lc1)))
    S2 = np.diag(np.tile(s2, oracle.volume(Lc2)))
    assert np.abs(S1 @ P2d - P2d @ S2).max() == 0
    # adjointness
    r1 = _level1_vectors(Lc1, nv1, 1, 93)[0]
    y2 = synth.gaussian(oracle.volume(Lc2) * 2 * nv2, 94, 0).reshape(-1, 2 * nv2)
    lhs = np.vdot(y2, oracle.crestrict(P2, r1, Lc1, B2, nv1))
    rhs = np.vdot(oracle.cprolong(P2, y2, Lc1, B2, nv1), r1)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)
    # Galerkin product against the dense one
    A1d = oracle.coarse_dense(A1, Lc1)
    A2 = oracle.ccoarse_build(A1, P2, Lc1, B2)
    A2d = oracle.coarse_dense(A2, Lc2)
    assert np.abs(A2d - P2d.conj().T @ A1d @ P2d).max() < 1e-12 * np.abs(A2d).max()
    assert np.abs(S2 @ A2d @ S2 - A2d.conj().T).max() < 1e-12 * np.abs(A2d).max()
    C = P2d - P2d @ np.linalg.solve(A2d, P2d.conj().T @ A1d @ P2d)
    assert np.abs(C).max() < 1e-10


@pytest.mark.parametrize("smoother1,k", [(1, 1), (1, 4), (0, 1)])
def test_level1_smoother_minimises_over_the_krylov_space(smoother1, k):
    """Level-1 post-smoothing (Sec. III smoother on A1): e += omega d with d the
    least-squares minimiser of |r - A1 d| over K_k(A1, r) (numpy lstsq over the
    power basis); one MR step is GMRES(1)."""
    L, B, nv1, U, m, P, A1, Lc1 = _level1()
    p = oracle.make_params(L, B, nv=nv1, m=m, smoother1=smoother1, steps1=k, omega=0.9)
    e0 = _level1_vectors(Lc1, nv1, 1, 95)[0]
    r = _level1_vectors(Lc1, nv1, 1, 96)[0]
    basis = [r]
    for _ in range(k - 1):
        basis.append(oracle.coarse_apply(A1, basis[-1], Lc1))
    K = np.stack([b.ravel() for b in basis], 1)
    AK = np.stack([oracle.coarse_apply(A1, b, Lc1).ravel() for b in basis], 1)
    c, *_ = np.linalg.lstsq(AK, r.ravel(), rcond=None)
    e1, r1 = oracle.csmooth(p, Lc1, A1, e0, r)
    want = e0 + 0.9 * (K @ c).reshape(r.shape)
    assert np.abs(e1 - want).max() < 1e-9 * np.abs(want).max()


def test_three_level_cycle_composition():
    """The three-level cycle (Sec. IV) from its parts, with an exact coarsest
    solve: one level-1 V-cycle is P2 A2^-1 P2^dag r1 followed by the level-1
    smoother on the corrected residual (lstsq check); two cycles (the W-cycle)
    are e = K(r1), e += K(r1 - A1 e); the fine cycle with this correction
    smooths r - D P K1(P^dag r) (lstsq over the fine Krylov space)."""
    L, B, nv1, U, m, P, A1, Lc1 = _level1()
    B2, nv2 = (1, 1, 2, 2), 4
    P2, _ = oracle.cblock_orthonormalize(_level1_vectors(Lc1, nv1, nv2, 97), Lc1, B2, nv1)
    A2 = oracle.ccoarse_build(A1, P2, Lc1, B2)
    Lc2 = oracle.coarse_dims(Lc1, B2)
    kw = dict(nv=nv1, m=m, levels=3, B2=B2, nv2=nv2, smoother1=1, steps1=3, coarse_tol=1e-15, coarse_maxit=100000,
              omega=0.9)
    r1 = _level1_vectors(Lc1, nv1, 1, 98)[0]
    e_one, _ = oracle.kcycle_l1(oracle.make_params(L, B, cycles1=1, **kw), A1, P2, A2, r1)
    y2 = np.linalg.solve(oracle.coarse_dense(A2, Lc2), oracle.crestrict(P2, r1, Lc1, B2, nv1).ravel())
    e0 = oracle.cprolong(P2, y2.reshape(oracle.volume(Lc2), -1), Lc1, B2, nv1)
    rr = r1 - oracle.coarse_apply(A1, e0, Lc1)
    basis = [rr]
    for _ in range(2):
        basis.append(oracle.coarse_apply(A1, basis[-1], Lc1))
    K = np.stack([b.ravel() for b in basis], 1)
    AK = np.stack([oracle.coarse_apply(A1, b, Lc1).ravel() for b in basis], 1)
    c, *_ = np.linalg.lstsq(AK, rr.ravel(), rcond=None)
    assert rel(e_one, e0 + 0.9 * (K @ c).reshape(rr.shape)) < 1e-9
    e_two, _ = oracle.kcycle_l1(oracle.make_params(L, B, cycles1=2, **kw), A1, P2, A2, r1)
    e_b, _ = oracle.kcycle_l1(oracle.make_params(L, B, cycles1=1, **kw), A1, P2, A2,
                              r1 - oracle.coarse_apply(A1, e_one, Lc1))
    assert rel(e_two, e_one + e_b) < 1e-12
    # the fine cycle around it
    p3 = oracle.make_params(L, B, cycles1=2, smoother=1, mr_steps=2, **kw)
    r = synth.gaussian_spinor(L, 99)
    z, _ = oracle.vcycle3(p3, U, P, A1, P2, A2, r)
    ez = oracle.prolong(P, oracle.kcycle_l1(p3, A1, P2, A2, oracle.restrict(P, r, L, B))[0], L, B)
    rf = r - oracle.dslash(U, ez, m, L)
    basis = [rf, oracle.dslash(U, rf, m, L)]
    DK = np.stack([oracle.dslash(U, b, m, L).ravel() for b in basis], 1)
    c, *_ = np.linalg.lstsq(DK, rf.ravel(), rcond=None)
    want = rf - 0.9 * (DK @ c).reshape(rf.shape)
    got = r - oracle.dslash(U, z, m, L)
    assert np.abs(got - want).max() < 1e-9 * np.abs(want).max()


@pytest.mark.slow
def test_three_level_solve_and_level2_setup():
    """On the 8^4 beta = 6.0 field at Re(lambda_min) = 0.01 (Nv = 8, 4^4 then
    1x1x2x2 aggregates, Nv2 = 8): the level-2 setup keeps its invariants and
    orders the asymptotic level-1 two-grid rate (eq. 3 on A1, exact level-2
    solve, MR(4) level-1 smoother): refined < relaxed only < random level-2
    prototypes (0.21 < 0.29 < 0.58); MG-GCR with the three-level W-cycle
    reaches 1e-10 in FP64.  (On this 2^4 intermediate lattice the outer
    iteration count is not ordered the same way: 111 with the refined against
    103 with random prototypes, whose well-conditioned A2 the 1e-3 coarsest
    CG solves more accurately.)"""
    from tests._fields import c1_workload
    L, B, nv, U, m = c1_workload()
    V0 = synth.gaussian_vectors(L, nv, 2001)
    p2 = oracle.make_params(L, B, nv=nv, m=m, smoother=1, mr_steps=4)
    _, P, A1, st = oracle.setup(p2, U, V0, init_relax=10, n_iter=3, group_size=4)
    assert st == 0
    Lc1 = oracle.coarse_dims(L, B)
    B2, nv2 = (1, 1, 2, 2), 8
    p3 = oracle.make_params(L, B, nv=nv, m=m, smoother=1, mr_steps=4, levels=3, B2=B2, nv2=nv2, smoother1=1,
                            steps1=4, cycles1=2)
    V2 = _level1_vectors(Lc1, nv, nv2, 2003)
    _, P2, A2, st2, sinfo = oracle.setup_level2(p3, A1, V2, init_relax=10, n_iter=3, group_size=4)
    assert st2 == 0 and sinfo["coarse_iters"] > 0
    P2d = _dense_P2(P2, Lc1, B2, nv)
    assert np.abs(P2d.conj().T @ P2d - np.eye(P2d.shape[1])).max() < 1e-12
    b = synth.gaussian_spinor(L, 7)
    x, info = oracle.gcr_solve3(p3, U, P, A1, P2, A2, b)
    assert info["status"] == 0
    assert np.linalg.norm(b - oracle.dslash(U, x, m, L)) <= 1e-10 * np.linalg.norm(b)
    P2r, _ = oracle.cblock_orthonormalize(V2, Lc1, B2, nv)
    _, P20, A20, st0, _ = oracle.setup_level2(p3, A1, V2, init_relax=10, n_iter=0, group_size=4)
    pm = oracle.make_params(L, B, nv=nv, m=m, levels=3, B2=B2, nv2=nv2, smoother1=0, steps1=4)
    e0 = _level1_vectors(Lc1, nv, 1, 77)[0]

    def rate(P2_, A2_):
        _, n = oracle.ctwo_grid_factor(pm, A1, P2_, A2_, e0, 40)
        return (n[40] / n[20]) ** (1 / 20)

    f_rand = rate(P2r, oracle.ccoarse_build(A1, P2r, Lc1, B2))
    f_relax, f_ref = rate(P20, A20), rate(P2, A2)
    assert f_ref < f_relax < f_rand < 1, (f_ref, f_relax, f_rand)


def test_level1_two_grid_factor_annihilates_range_of_p2():
    """Without smoothing the level-1 two-grid step removes any error in range(P2)."""
    L, B, nv1, U, m, P, A1, Lc1 = _level1()
    B2, nv2 = (1, 1, 2, 2), 3
    P2, _ = oracle.cblock_orthonormalize(_level1_vectors(Lc1, nv1, nv2, 80), Lc1, B2, nv1)
    A2 = oracle.ccoarse_build(A1, P2, Lc1, B2)
    Lc2 = oracle.coarse_dims(Lc1, B2)
    p = oracle.make_params(L, B, nv=nv1, m=m, levels=3, B2=B2, nv2=nv2, steps1=0)
    y2 = synth.gaussian(oracle.volume(Lc2) * 2 * nv2, 81, 0).reshape(-1, 2 * nv2)
    f, n = oracle.ctwo_grid_factor(p, A1, P2, A2, oracle.cprolong(P2, y2, Lc1, B2, nv1), 1)
    assert n[1] < 1e-12 * n[0]
