"""CPU oracle for the adaptive multigrid Wilson-Dirac solve (arXiv:1005.3043).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg import this package; the product path
never does.  It wraps ``oracle.c`` (plain FP64 C, one function per step of the
method, each citing the paper passage it restates) through ctypes.

Parity status per function (what pins it; see the tests):
  dslash            free-field plane-wave eigenvalues, gamma5-hermiticity, gauge
                    covariance, mass shift, dense brute force (eq. 2)
  block_orthonormalize / restrict / prolong
                    P^dag P = I, P V_c = V (eq. 4), gamma5 P = P sigma3,
                    Q of numpy's QR up to phases
  coarse_build / coarse_apply
                    dense P^dag D P brute force, sigma3 D_c sigma3 = D_c^dag,
                    mass shift, (I - P D_c^-1 P^dag D) P = 0 (eqs. 3, 8),
                    nearest-neighbour sparsity, non-split singularity
  mr                exact residual-decrease identity per step
  cgnr              reaches the dense LU solution; CGLS orthogonality
  gcr_solve         with M = I equals GMRES residuals; true residual <= tol
  vcycle            coarse part Galerkin (P^dag (r - D z) = 0); smoothing half
                    equal to the least-squares correction over K_k(D, r') of
                    the coarse-corrected residual r' (numpy lstsq)
  setup             parity unpinned as a bit pattern (iterative, nonlinear);
                    pinned by the invariants of its outputs, by the two-grid
                    convergence factor (refined < relaxed only < random
                    prototypes) and by its truncated level (the refined group
                    is outside range(P_t), every other prototype inside)
  eo_schur / eo_cg  red-black preconditioned CG (the comparison of Sec. IV):
                    D applied to (x_e, H_oe x_e / (4+m)) is (Dhat x_e, 0);
                    gamma5-hermiticity of Dhat; CG iterates equal the
                    least-squares solution over the Krylov space (numpy
                    lstsq); dense solve on a small lattice; true residual
  cblock_orthonormalize / crestrict / cprolong / ccoarse_build (level 2)
                    P2^dag P2 = I, P2 V2_c = V2, sigma3 kept, numpy QR,
                    adjointness, dense P2^dag A1 P2 for level-2 extents 2, 1
                    and mixed, (I - P2 A2^-1 P2^dag A1) P2 = 0
  csmooth / kcycle_l1 / vcycle3 / gcr_solve3 / setup_level2
                    level-1 smoother = lstsq over K_k(A1, r); the W-cycle
                    equals its composition from single V-cycles; the fine
                    cycle smooths r - D P K1(P^dag r) (lstsq); the 3-level
                    solve reaches 1e-10; the level-2 setup lowers the level-1
                    two-grid rate (refined < relaxed < random)
  two_grid_factor   eq. 3 with an exact coarse solve: a start in range(P)
                    is annihilated, the unsmoothed E_TG is a projection, the
                    corrected residual is Galerkin-orthogonal to range(P)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_NOT_CONVERGED, ERR_NUMERIC = 0, -1, -4, -5


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fcx-limited-range", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int * 4), ("B", ctypes.c_int * 4), ("nv", ctypes.c_int),
                ("tap", ctypes.c_int), ("m", ctypes.c_double), ("mr_steps", ctypes.c_int),
                ("omega", ctypes.c_double), ("coarse_tol", ctypes.c_double),
                ("coarse_maxit", ctypes.c_int), ("gcr_restart", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_outer", ctypes.c_int), ("use_mg", ctypes.c_int),
                ("smoother", ctypes.c_int), ("levels", ctypes.c_int), ("B2", ctypes.c_int * 4),
                ("nv2", ctypes.c_int), ("smoother1", ctypes.c_int), ("steps1", ctypes.c_int),
                ("cycles1", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int), ("coarse_iters", ctypes.c_int),
                ("fine_matvecs", ctypes.c_int), ("restarts", ctypes.c_int),
                ("true_rel_res", ctypes.c_double), ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
            lib.or_gamma_matrices.argtypes = [P]
            lib.or_dslash.argtypes = [P, I, P, D, P, P]
            lib.or_gamma5.argtypes = [I64, P, P]
            lib.or_dot.argtypes = [I64, P, P, P]
            lib.or_block_orthonormalize.argtypes = [P, P, I, P, P]
            lib.or_block_orthonormalize.restype = I
            lib.or_restrict.argtypes = [P, P, I, P, P, P]
            lib.or_prolong.argtypes = [P, P, I, P, P, P]
            lib.or_coarse_build.argtypes = [P, P, I, I, P, D, P, P]
            lib.or_coarse_apply.argtypes = [P, I, P, P, P]
            lib.or_coarse_apply_dag.argtypes = [P, I, P, P, P]
            lib.or_mr.argtypes = [P, I, P, D, I, D, P, P]
            lib.or_gmres_smooth.argtypes = [P, I, P, D, I, D, P, P]
            lib.or_cgnr.argtypes = [P, I, P, P, P, D, I, P]
            lib.or_cgnr.restype = I
            lib.or_vcycle.argtypes = [P, P, P, P, P, P, P]
            lib.or_gcr_solve.argtypes = [P, P, P, P, P, P, P]
            lib.or_gcr_solve.restype = I
            lib.or_setup.argtypes = [P, P, P, I, I, I, P, P]
            lib.or_setup.restype = I
            lib.or_cblock_orthonormalize.argtypes = [P, P, I, I, P, P]
            lib.or_cblock_orthonormalize.restype = I
            lib.or_crestrict.argtypes = [P, P, I, I, P, P, P]
            lib.or_cprolong.argtypes = [P, P, I, I, P, P, P]
            lib.or_ccoarse_build.argtypes = [P, P, I, I, P, P, P]
            lib.or_csmooth.argtypes = [P, P, P, P, P]
            lib.or_kcycle_l1.argtypes = [P, P, P, P, P, P, P]
            lib.or_setup_level2.argtypes = [P, P, P, I, I, I, P, P, P]
            lib.or_setup_level2.restype = I
            lib.or_vcycle3.argtypes = [P, P, P, P, P, P, P, P, P]
            lib.or_gcr_solve3.argtypes = [P, P, P, P, P, P, P, P, P]
            lib.or_gcr_solve3.restype = I
            lib.or_setup_counted.argtypes = [P, P, P, I, I, I, P, P, P]
            lib.or_setup_counted.restype = I
            lib.or_setup_truncated_level.argtypes = [P, P, P, I, I, P, P, P]
            lib.or_setup_truncated_level.restype = I
            lib.or_eo_schur.argtypes = [P, I, P, D, I, P, P]
            lib.or_eo_cg.argtypes = [P, I, P, D, P, P, D, I, P, P, P]
            lib.or_eo_cg.restype = I
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "array must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _i4(L) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(L, dtype=np.int32).reshape(4))


def volume(L) -> int:
    return int(np.prod(np.asarray(L, dtype=np.int64)))


def coarse_dims(L, B):
    return tuple(int(l) // int(b) for l, b in zip(L, B))


def gamma_matrices() -> np.ndarray:
    g = np.zeros((4, 4, 4), dtype=np.complex128)
    _load().or_gamma_matrices(_p(g))
    return g


def dslash(U, psi, m: float, L, tap: int = 1) -> np.ndarray:
    """D(U) psi, eq. (2).  U (4,V,3,3), psi (V,4,3)."""
    U, psi = _c(U), _c(psi)
    out = np.empty_like(psi)
    _load().or_dslash(_p(_i4(L)), int(tap), _p(U), float(m), _p(psi), _p(out))
    return out


def gamma5(psi) -> np.ndarray:
    psi = _c(psi)
    out = np.empty_like(psi)
    _load().or_gamma5(psi.shape[0], _p(psi), _p(out))
    return out


def block_orthonormalize(Vecs, L, B):
    """Returns (P, status).  Vecs (Nv,V,4,3) -> P (Nv,V,4,3)."""
    Vecs = _c(Vecs)
    P = np.empty_like(Vecs)
    st = _load().or_block_orthonormalize(_p(_i4(L)), _p(_i4(B)), Vecs.shape[0], _p(Vecs), _p(P))
    return P, st


def restrict(P, r, L, B) -> np.ndarray:
    P, r = _c(P), _c(r)
    nv = P.shape[0]
    Vc = volume(coarse_dims(L, B))
    rc = np.empty((Vc, 2 * nv), dtype=np.complex128)
    _load().or_restrict(_p(_i4(L)), _p(_i4(B)), nv, _p(P), _p(r), _p(rc))
    return rc


def prolong(P, yc, L, B) -> np.ndarray:
    P, yc = _c(P), _c(yc)
    nv = P.shape[0]
    e = np.empty(P.shape[1:], dtype=np.complex128)
    _load().or_prolong(_p(_i4(L)), _p(_i4(B)), nv, _p(P), _p(yc), _p(e))
    return e


def coarse_build(U, P, m: float, L, B, tap: int = 1) -> np.ndarray:
    """A[Xc, 9, nc, nc] = P^dag D P in nearest-neighbour form."""
    U, P = _c(U), _c(P)
    nv = P.shape[0]
    nc = 2 * nv
    Vc = volume(coarse_dims(L, B))
    A = np.empty((Vc, 9, nc, nc), dtype=np.complex128)
    _load().or_coarse_build(_p(_i4(L)), _p(_i4(B)), nv, int(tap), _p(U), float(m), _p(P), _p(A))
    return A


def coarse_apply(A, x, Lc) -> np.ndarray:
    A, x = _c(A), _c(x)
    y = np.empty_like(x)
    _load().or_coarse_apply(_p(_i4(Lc)), A.shape[-1], _p(A), _p(x), _p(y))
    return y


def coarse_apply_dag(A, x, Lc) -> np.ndarray:
    A, x = _c(A), _c(x)
    y = np.empty_like(x)
    _load().or_coarse_apply_dag(_p(_i4(Lc)), A.shape[-1], _p(A), _p(x), _p(y))
    return y


def mr(U, e, r, m: float, L, nsteps: int, omega: float, tap: int = 1):
    """nsteps MR steps; returns updated (e, r)."""
    e, r = _c(e).copy(), _c(r).copy()
    _load().or_mr(_p(_i4(L)), int(tap), _p(_c(U)), float(m), int(nsteps), float(omega), _p(e), _p(r))
    return e, r


def gmres_smooth(U, e, r, m: float, L, k: int, omega: float, tap: int = 1):
    """One GMRES(k) smoothing application: returns e + omega * argmin over K_k(D, r) of ||r - D d||."""
    e, r = _c(e).copy(), _c(r)
    _load().or_gmres_smooth(_p(_i4(L)), int(tap), _p(_c(U)), float(m), int(k), float(omega), _p(e), _p(r))
    return e


def cgnr(A, rc, Lc, tol: float, maxit: int):
    """Returns (y, iterations, final relative residual)."""
    A, rc = _c(A), _c(rc)
    y = np.empty_like(rc)
    rel = ctypes.c_double(0)
    it = _load().or_cgnr(_p(_i4(Lc)), A.shape[-1], _p(A), _p(rc), _p(y), float(tol), int(maxit),
                         ctypes.byref(rel))
    return y, it, rel.value


def make_params(L, B=(4, 4, 4, 4), nv=8, m=0.0, tap=1, mr_steps=4, omega=0.9, coarse_tol=1e-3,
                coarse_maxit=10000, gcr_restart=16, tol=1e-10, max_outer=1000, use_mg=1, smoother=0,
                levels=2, B2=(2, 2, 2, 2), nv2=0, smoother1=1, steps1=4, cycles1=2) -> Params:
    p = Params()
    for i in range(4):
        p.L[i] = int(L[i]); p.B[i] = int(B[i])
    p.nv, p.tap, p.m = int(nv), int(tap), float(m)
    p.mr_steps, p.omega = int(mr_steps), float(omega)
    p.coarse_tol, p.coarse_maxit = float(coarse_tol), int(coarse_maxit)
    p.gcr_restart, p.tol, p.max_outer, p.use_mg = int(gcr_restart), float(tol), int(max_outer), int(use_mg)
    p.smoother = int(smoother)
    p.levels, p.nv2 = int(levels), int(nv2)
    for i in range(4):
        p.B2[i] = int(B2[i])
    p.smoother1, p.steps1, p.cycles1 = int(smoother1), int(steps1), int(cycles1)
    return p


def vcycle(params: Params, U, P, A, r):
    U, P, A, r = _c(U), _c(P), _c(A), _c(r)
    z = np.empty_like(r)
    info = Info()
    _load().or_vcycle(ctypes.byref(params), _p(U), _p(P), _p(A), _p(r), _p(z), ctypes.byref(info))
    return z, info.as_dict()


def gcr_solve(params: Params, U, P, A, b):
    """Returns (x, info dict).  P, A may be None when params.use_mg == 0."""
    U, b = _c(U), _c(b)
    if P is None:
        P = np.zeros((1, 1), dtype=np.complex128)
        A = np.zeros((1, 1), dtype=np.complex128)
    P, A = _c(P), _c(A)
    x = np.empty_like(b)
    info = Info()
    _load().or_gcr_solve(ctypes.byref(params), _p(U), _p(P), _p(A), _p(b), _p(x), ctypes.byref(info))
    return x, info.as_dict()


def setup(params: Params, U, V0, init_relax: int, n_iter: int, group_size: int = 4):
    """Adaptive setup from random starts V0 (Nv,V,4,3): init_relax relaxation steps,
    then group refinement with n_iter truncated-MG iterations per group.
    Returns (V, P, A, status)."""
    U = _c(U)
    Vv = _c(V0).copy()
    nv = Vv.shape[0]
    assert nv == params.nv
    Lc = coarse_dims(list(params.L), list(params.B))
    P = np.empty_like(Vv)
    A = np.empty((volume(Lc), 9, 2 * nv, 2 * nv), dtype=np.complex128)
    st = _load().or_setup(ctypes.byref(params), _p(U), _p(Vv), int(init_relax), int(n_iter),
                         int(group_size), _p(P), _p(A))
    return Vv, P, A, st


def setup_counted(params: Params, U, V0, init_relax: int, n_iter: int, group_size: int = 4):
    """setup() that also returns its work: (V, P, A, status, info) with
    info['fine_matvecs'] the operator applications of the relaxation and the
    truncated cycles and info['coarse_iters'] their coarse CG iterations."""
    U = _c(U)
    Vv = _c(V0).copy()
    nv = Vv.shape[0]
    assert nv == params.nv
    Lc = coarse_dims(list(params.L), list(params.B))
    P = np.empty_like(Vv)
    A = np.empty((volume(Lc), 9, 2 * nv, 2 * nv), dtype=np.complex128)
    info = Info()
    st = _load().or_setup_counted(ctypes.byref(params), _p(U), _p(Vv), int(init_relax), int(n_iter),
                                  int(group_size), _p(P), _p(A), ctypes.byref(info))
    return Vv, P, A, st, info.as_dict()


def setup_truncated_level(params: Params, U, V, g0: int, group_size: int):
    """The truncated level the group refinement of Sec. IV builds for group
    g0 .. g0 + group_size - 1: (Vt, Pt, At, status) with Vt the prototypes
    without the group, Pt their block orthonormalisation (eq. 4) and
    At = Pt^dag D Pt.  The same C routine serves the setup itself."""
    U, V = _c(U), _c(V)
    nv = V.shape[0]
    assert nv == params.nv
    nt = nv - group_size
    Lc = coarse_dims(list(params.L), list(params.B))
    Vt = np.empty((nt,) + V.shape[1:], dtype=np.complex128)
    Pt = np.empty_like(Vt)
    At = np.empty((volume(Lc), 9, 2 * nt, 2 * nt), dtype=np.complex128)
    st = _load().or_setup_truncated_level(ctypes.byref(params), _p(U), _p(V), int(g0), int(group_size), _p(Vt),
                                          _p(Pt), _p(At))
    return Vt, Pt, At, st


def coarse_dense(A, Lc) -> np.ndarray:
    """D_c as a dense (Vc nc) x (Vc nc) matrix, column by column from coarse_apply."""
    A = _c(A)
    nC = A.shape[0] * A.shape[-1]
    M = np.empty((nC, nC), dtype=np.complex128)
    for k in range(nC):
        e = np.zeros(nC, dtype=np.complex128)
        e[k] = 1.0
        M[:, k] = coarse_apply(A, e.reshape(A.shape[0], A.shape[-1]), Lc).ravel()
    return M


def two_grid_factor(params: Params, U, P, A, e0, k: int):
    """Two-grid convergence factor (||E_TG^k e0|| / ||e0||)^(1/k) of eq. 3,
    E_TG = S (I - P (P^dag D P)^-1 P^dag D), with the coarse system solved
    exactly (dense LU of D_c, numpy) and S the post-smoother of the cycle
    (params.smoother: mr_steps MR steps, or one GMRES(mr_steps) application,
    under-relaxed by params.omega).  The iteration is the two-grid method on
    D x = 0 with x = e: coarse correction e <- e + P D_c^-1 P^dag (-D e), then
    the smoother on (e, -D e).  Returns (factor, [||e_j|| for j = 0..k])."""
    U, P, A = _c(U), _c(P), _c(A)
    L, B = list(params.L), list(params.B)
    m, tap = params.m, params.tap
    Lc = coarse_dims(L, B)
    from scipy.linalg import lu_factor, lu_solve
    lu = lu_factor(coarse_dense(A, Lc))   # exact coarse solve (small coarse grids only)
    e = _c(e0).copy()
    norms = [float(np.linalg.norm(e))]
    for _ in range(k):
        r = -dslash(U, e, m, L, tap)
        y = lu_solve(lu, restrict(P, r, L, B).ravel()).reshape(volume(Lc), -1)
        e = e + prolong(P, y, L, B)
        if params.mr_steps > 0:
            r = -dslash(U, e, m, L, tap)
            if params.smoother == 1:
                e = gmres_smooth(U, e, r, m, L, params.mr_steps, params.omega, tap)
            else:
                e, _ = mr(U, e, r, m, L, params.mr_steps, params.omega, tap)
        norms.append(float(np.linalg.norm(e)))
    return (norms[-1] / norms[0]) ** (1.0 / k), norms


def parity_mask(L) -> np.ndarray:
    """(V,) bool, True on the even sites ((x + y + z + t) mod 2 = 0)."""
    c = np.indices(tuple(L)[::-1]).reshape(4, -1)[::-1]    # c[mu] per lexicographic site
    return (c.sum(0) % 2) == 0


def eo_schur(U, xe, m: float, L, dag: bool = False, tap: int = 1) -> np.ndarray:
    """Dhat xe = (4+m) xe - H_eo H_oe xe / (4+m) on the even sites (dag:
    gamma5 Dhat gamma5), the Schur complement of the red-black preconditioned
    CG that Sec. IV compares against; xe read on the even sites."""
    xe = _c(xe)
    out = np.empty_like(xe)
    _load().or_eo_schur(_p(_i4(L)), int(tap), _p(_c(U)), float(m), int(bool(dag)), _p(xe), _p(out))
    return out


def eo_cg(U, b, m: float, L, tol: float, maxit: int, tap: int = 1):
    """Red-black preconditioned CG (CGLS on the even-site Schur complement) for
    D x = b: returns (x, iterations, matvecs, true relative residual, status)."""
    b = _c(b)
    x = np.empty_like(b)
    it, mv, rel = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0)
    st = _load().or_eo_cg(_p(_i4(L)), int(tap), _p(_c(U)), float(m), _p(b), _p(x), float(tol), int(maxit),
                          ctypes.byref(it), ctypes.byref(mv), ctypes.byref(rel))
    return x, it.value, mv.value, rel.value, st


# ---------------------------------------------------------------- third level (Sec. III recursion, Sec. IV W-cycle)
def cblock_orthonormalize(V2, Lc1, B2, nv1: int):
    """Level-1 vectors V2 (nv2, Vc1, 2 nv1) -> (P2, status): eq. 4 one level down,
    per level-2 aggregate and chirality (dof a of chirality a // nv1)."""
    V2 = _c(V2)
    P2 = np.empty_like(V2)
    st = _load().or_cblock_orthonormalize(_p(_i4(Lc1)), _p(_i4(B2)), int(nv1), int(V2.shape[0]), _p(V2), _p(P2))
    return P2, st


def crestrict(P2, r1, Lc1, B2, nv1: int) -> np.ndarray:
    P2, r1 = _c(P2), _c(r1)
    Lc2 = coarse_dims(Lc1, B2)
    out = np.empty((volume(Lc2), 2 * P2.shape[0]), dtype=np.complex128)
    _load().or_crestrict(_p(_i4(Lc1)), _p(_i4(B2)), int(nv1), int(P2.shape[0]), _p(P2), _p(r1), _p(out))
    return out


def cprolong(P2, y2, Lc1, B2, nv1: int) -> np.ndarray:
    P2, y2 = _c(P2), _c(y2)
    out = np.empty((volume(Lc1), 2 * nv1), dtype=np.complex128)
    _load().or_cprolong(_p(_i4(Lc1)), _p(_i4(B2)), int(nv1), int(P2.shape[0]), _p(P2), _p(y2), _p(out))
    return out


def ccoarse_build(A1, P2, Lc1, B2) -> np.ndarray:
    """A2 = P2^dag A1 P2 in nearest-neighbour form (slots by the face a term leaves through)."""
    A1, P2 = _c(A1), _c(P2)
    nv1, nv2 = A1.shape[-1] // 2, P2.shape[0]
    Lc2 = coarse_dims(Lc1, B2)
    A2 = np.empty((volume(Lc2), 9, 2 * nv2, 2 * nv2), dtype=np.complex128)
    _load().or_ccoarse_build(_p(_i4(Lc1)), _p(_i4(B2)), int(nv1), int(nv2), _p(A1), _p(P2), _p(A2))
    return A2


def csmooth(params: Params, Lc1, A1, e, r):
    """Level-1 post-smoothing (params.smoother1: MR or GMRES(steps1), omega) on (e, r); returns (e, r)."""
    e, r = _c(e).copy(), _c(r).copy()
    _load().or_csmooth(ctypes.byref(params), _p(_i4(Lc1)), _p(_c(A1)), _p(e), _p(r))
    return e, r


def kcycle_l1(params: Params, A1, P2, A2, r1):
    """The three-level method's coarse-grid correction: params.cycles1 level-1
    V-cycles on A1 e = r1 from e = 0.  Returns (e1, info)."""
    r1 = _c(r1)
    e1 = np.empty_like(r1)
    info = Info()
    _load().or_kcycle_l1(ctypes.byref(params), _p(_c(A1)), _p(_c(P2)), _p(_c(A2)), _p(r1), _p(e1),
                         ctypes.byref(info))
    return e1, info.as_dict()


def setup_level2(params: Params, A1, V2, init_relax: int, n_iter: int, group_size: int = 4):
    """Adaptive setup of level 2 on the operator A1 from random level-1 starts V2
    (nv2, Vc1, 2 nv1): returns (V2, P2, A2, status, info)."""
    A1 = _c(A1)
    V = _c(V2).copy()
    Lc1 = coarse_dims(list(params.L), list(params.B))
    Lc2 = coarse_dims(Lc1, list(params.B2))
    nv2 = V.shape[0]
    assert nv2 == params.nv2
    P2 = np.empty_like(V)
    A2 = np.empty((volume(Lc2), 9, 2 * nv2, 2 * nv2), dtype=np.complex128)
    info = Info()
    st = _load().or_setup_level2(ctypes.byref(params), _p(A1), _p(V), int(init_relax), int(n_iter), int(group_size),
                                 _p(P2), _p(A2), ctypes.byref(info))
    return V, P2, A2, st, info.as_dict()


def vcycle3(params: Params, U, P, A, P2, A2, r):
    r = _c(r)
    z = np.empty_like(r)
    info = Info()
    _load().or_vcycle3(ctypes.byref(params), _p(_c(U)), _p(_c(P)), _p(_c(A)), _p(_c(P2)), _p(_c(A2)), _p(r), _p(z),
                       ctypes.byref(info))
    return z, info.as_dict()


def gcr_solve3(params: Params, U, P, A, P2, A2, b):
    """Flexible GCR preconditioned by the three-level W-cycle: returns (x, info)."""
    b = _c(b)
    x = np.empty_like(b)
    info = Info()
    _load().or_gcr_solve3(ctypes.byref(params), _p(_c(U)), _p(_c(P)), _p(_c(A)), _p(_c(P2)), _p(_c(A2)), _p(b),
                          _p(x), ctypes.byref(info))
    return x, info.as_dict()


def ctwo_grid_factor(params: Params, A1, P2, A2, e0, k: int):
    """Eq. 3 one level down: the two-grid method of levels 1 and 2 on A1 e = 0
    with the level-2 system solved exactly (dense LU of A2, scipy) and the
    level-1 post-smoother (params.smoother1, steps1, omega): e <- e + P2 A2^-1
    P2^dag (-A1 e), then the smoother on (e, -A1 e).  Returns (factor over k
    iterations, [||e_j||, j = 0..k])."""
    from scipy.linalg import lu_factor, lu_solve
    A1, P2, A2 = _c(A1), _c(P2), _c(A2)
    Lc1 = coarse_dims(list(params.L), list(params.B))
    B2 = list(params.B2)
    Lc2 = coarse_dims(Lc1, B2)
    nv1 = A1.shape[-1] // 2
    lu = lu_factor(coarse_dense(A2, Lc2))
    e = _c(e0).copy()
    norms = [float(np.linalg.norm(e))]
    for _ in range(k):
        r = -coarse_apply(A1, e, Lc1)
        y = lu_solve(lu, crestrict(P2, r, Lc1, B2, nv1).ravel()).reshape(volume(Lc2), -1)
        e = e + cprolong(P2, y, Lc1, B2, nv1)
        if params.steps1 > 0:
            e, _ = csmooth(params, Lc1, A1, e, -coarse_apply(A1, e, Lc1))
        norms.append(float(np.linalg.norm(e)))
    return (norms[-1] / norms[0]) ** (1.0 / k), norms
