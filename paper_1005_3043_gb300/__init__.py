"""GB300-native adaptive multigrid solver for the lattice Wilson-Dirac equation
D(U) psi = b (Babich et al., arXiv:1005.3043).

This module is a thin ctypes binding of the C-ABI in ``include/wilson_mg.h``:
the functions keep the C names and only marshal arguments (numpy arrays for
host buffers, torch tensors or integer addresses for device buffers, torch
streams).  Every numerical step runs in the CUDA kernels of
``_build/libwilson_mg.so``; if that library is missing the import of any entry
point fails loudly -- there is no CPU path.

Layouts (boundary): links ``U[mu, site, a, b]``, spinors ``psi[site, spin, colour]``,
complex128, site = x + L0*(y + L1*(z + L2*t)).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build_mod

MG_OK = 0
MG_ERR_INVALID_ARG = -1
MG_ERR_NOT_SETUP = -2
MG_ERR_OOM = -3
MG_ERR_NOT_CONVERGED = -4
MG_ERR_NUMERIC = -5
MG_ERR_TIMEOUT = -6
MG_ERR_CUDA = -7
MG_FP64 = 0
MG_FP32 = 1
MG_FP16 = 2

LIB_PATH = _build_mod.LIB


class MgParams(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int * 4), ("nvec", ctypes.c_int), ("setup_init_relax", ctypes.c_int),
                ("setup_iters", ctypes.c_int), ("setup_group", ctypes.c_int), ("smoother_steps", ctypes.c_int),
                ("omega", ctypes.c_double), ("gcr_restart", ctypes.c_int), ("tol", ctypes.c_double),
                ("coarse_tol", ctypes.c_double), ("max_outer", ctypes.c_int), ("max_coarse", ctypes.c_int),
                ("delta", ctypes.c_double), ("prec_inner", ctypes.c_int), ("coarse_check", ctypes.c_int),
                ("coarse_kernel", ctypes.c_int), ("smoother", ctypes.c_int), ("smoother_fp16", ctypes.c_int),
                ("coarse_form", ctypes.c_int), ("levels", ctypes.c_int), ("block2", ctypes.c_int * 4),
                ("nvec2", ctypes.c_int), ("smoother_steps1", ctypes.c_int), ("cycles1", ctypes.c_int)]


class MgSolveInfo(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int), ("coarse_iters", ctypes.c_int), ("fine_matvecs", ctypes.c_int),
                ("restarts", ctypes.c_int), ("true_rel_res", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("status", ctypes.c_int), ("setup_ms", ctypes.c_double), ("dslash_bytes", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


_lib = None

# name -> (argtypes, restype)
_P, _I, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
_SIGS = {
    "mg_default_params": ([_P], _I),
    "mg_create": ([_P, _I, _P, _P, _P], _I),
    "mg_destroy": ([_P], None),
    "mg_set_links": ([_P, _P], _I),
    "mg_set_links_device": ([_P, _P, _P], _I),
    "mg_set_mass": ([_P, _D], _I),
    "mg_set_params": ([_P, _P], _I),
    "mg_setup": ([_P, _P], _I),
    "mg_setup_device": ([_P, _P], _I),
    "mg_set_null_vectors": ([_P, _P, _I], _I),
    "mg_get_prolongator": ([_P, _P], _I),
    "mg_get_null_vectors": ([_P, _P], _I),
    "mg_setup_level2": ([_P, _P], _I),
    "mg_nn_set_weights": ([_P, _P, _I], _I),
    "mg_nn_get_weights": ([_P, _P, _I], _I),
    "mg_nn_forward": ([_P, _P, _P, _I], _I),
    "mg_nn_loss_grad": ([_P, _P, _I, _P, _P], _I),
    "mg_nn_train": ([_P, _P, _I, _I, _D, _P, _P], _I),
    "mg_setup_learned": ([_P, _P, _I], _I),
    "mg_set_level2_vectors": ([_P, _P], _I),
    "mg_get_level2_prolongator": ([_P, _P], _I),
    "mg_get_level2_op": ([_P, _P], _I),
    "mg_kcycle": ([_P, _P, _P, _I], _I),
    "mg_get_coarse_op": ([_P, _P], _I),
    "mg_solve": ([_P, _P, _P, _P], _I),
    "mg_solve_device": ([_P, _P, _P, _P], _I),
    "mg_solve_batched": ([_P, _P, _P, _I, _P], _I),
    "mg_solve_batched_device": ([_P, _P, _P, _I, _P], _I),
    "mg_apply_coarse_batched": ([_P, _P, _P, _I, _I, _I], _I),
    "mg_solve_eo_cg": ([_P, _P, _P, _D, _I, _I, _P], _I),
    "mg_solve_eo_cg_device": ([_P, _P, _P, _D, _I, _I, _P], _I),
    "mg_apply_dslash": ([_P, _P, _P, _I], _I),
    "mg_restrict": ([_P, _P, _P, _I], _I),
    "mg_prolong": ([_P, _P, _P, _I], _I),
    "mg_apply_coarse": ([_P, _P, _P, _I, _I], _I),
    "mg_mr": ([_P, _P, _P, _I, _I], _I),
    "mg_coarse_solve": ([_P, _P, _P, _D, _I, _I, _P, _P], _I),
    "mg_coarse_solve_noalloc": ([_P, _P, _P, _D, _I, _P, _P], _I),
    "mg_vcycle": ([_P, _P, _P, _I], _I),
    "mg_time_dslash": ([_P, _I, _I, _P, _P], _I),
    "mg_time_coarse_floor": ([_P, _I, _P, _P], _I),
    "mg_time_coarse_batched": ([_P, _I, _I, _P, _P, _P], _I),
    "mg_time_dslash_cold": ([_P, _I, _I, _P, ctypes.c_size_t, _P, _P], _I),
    "mg_profile_enable": ([_P, _I], _I),
    "mg_profile_read": ([_P, _P, _P, _P], _I),
    "mg_profile_classes": ([_P, ctypes.c_uint], _I),
    "mg_kernel_launches": ([], ctypes.c_longlong),
    "mg_coarse_kernel": ([ctypes.c_void_p], ctypes.c_int),
    "mg_check_wait_timeout": ([_P, _I, ctypes.c_longlong], _I),
    "mg_status_string": ([_I], ctypes.c_char_p),
    "mg_last_error": ([_P], ctypes.c_char_p),
}
EXPORTED = tuple(_SIGS)


def load(path: str | None = None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library {p} is missing: run paper_1005_3043_gb300.build.build() first")
        lib = ctypes.CDLL(p)
        for name, (args, res) in _SIGS.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


def status_string(status: int) -> str:
    return load().mg_status_string(int(status)).decode()


def _err(ctx) -> str:
    return load().mg_last_error(ctx).decode() if ctx else ""


def _check(status: int, ctx=None, allow=()):
    if status != MG_OK and status not in allow:
        raise MGError(status, _err(ctx))
    return status


def _host(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dev_ptr(t) -> int:
    """Device address of a torch tensor (or an int address)."""
    if isinstance(t, int):
        return t
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device buffers must be contiguous CUDA tensors")
    return t.data_ptr()


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------------ C-ABI, same names
def mg_default_params() -> MgParams:
    p = MgParams()
    _check(load().mg_default_params(ctypes.byref(p)))
    return p


def mg_create(dims, t_antiperiodic: int = 1, params: MgParams | None = None, stream=None):
    p = params or mg_default_params()
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    out = ctypes.c_void_p()
    _check(load().mg_create(d, int(t_antiperiodic), ctypes.byref(p), _stream_ptr(stream), ctypes.byref(out)))
    return out


def mg_destroy(ctx) -> None:
    if ctx:
        load().mg_destroy(ctx)


def mg_set_links(ctx, U) -> None:
    _check(load().mg_set_links(ctx, _ptr(_host(U))), ctx)


def mg_set_links_device(ctx, U_dev, stream=None) -> None:
    """Links from device memory (boundary layout, complex128), ordered on ``stream``."""
    _check(load().mg_set_links_device(ctx, _dev_ptr(U_dev), _stream_ptr(stream)), ctx)


def mg_set_mass(ctx, m: float) -> None:
    _check(load().mg_set_mass(ctx, float(m)), ctx)


def mg_set_params(ctx, params: MgParams) -> None:
    _check(load().mg_set_params(ctx, ctypes.byref(params)), ctx)


def mg_setup(ctx, V0) -> None:
    _check(load().mg_setup(ctx, _ptr(_host(V0))), ctx)


def mg_setup_device(ctx, V0_dev) -> None:
    _check(load().mg_setup_device(ctx, _dev_ptr(V0_dev)), ctx)


def mg_set_null_vectors(ctx, V) -> None:
    V = _host(V)
    _check(load().mg_set_null_vectors(ctx, _ptr(V), int(V.shape[0])), ctx)


def mg_get_prolongator(ctx, nv: int, V: int) -> np.ndarray:
    out = np.empty((nv, V, 4, 3), dtype=np.complex128)
    _check(load().mg_get_prolongator(ctx, _ptr(out)), ctx)
    return out


def mg_get_null_vectors(ctx, nv: int, V: int) -> np.ndarray:
    out = np.empty((nv, V, 4, 3), dtype=np.complex128)
    _check(load().mg_get_null_vectors(ctx, _ptr(out)), ctx)
    return out


NN_PARAMS = 20736   # complex weights of the learned setup's network (layers 1-8-8-8-1)
NN_CHANNELS = (1, 8, 8, 8, 1)


def nn_flatten(Ws) -> np.ndarray:
    """Layer weight arrays [Cout, Cin, 9, 4, 4] -> the flat complex vector of the C-ABI."""
    return np.concatenate([np.ascontiguousarray(W, dtype=np.complex128).ravel() for W in Ws])


def nn_unflatten(w) -> list:
    out, o = [], 0
    for ci, co in zip(NN_CHANNELS[:-1], NN_CHANNELS[1:]):
        n = co * ci * 144
        out.append(np.asarray(w[o:o + n]).reshape(co, ci, 9, 4, 4))
        o += n
    return out


def mg_nn_set_weights(ctx, Ws) -> None:
    w = _host(nn_flatten(Ws) if isinstance(Ws, (list, tuple)) else Ws)
    _check(load().mg_nn_set_weights(ctx, _ptr(w), int(w.size)), ctx)


def mg_nn_get_weights(ctx) -> list:
    w = np.empty(NN_PARAMS, dtype=np.complex128)
    _check(load().mg_nn_get_weights(ctx, _ptr(w), NN_PARAMS), ctx)
    return nn_unflatten(w)


def mg_nn_forward(ctx, etas) -> np.ndarray:
    e = _host(etas)
    v = np.empty_like(e)
    _check(load().mg_nn_forward(ctx, _ptr(e), _ptr(v), int(e.shape[0])), ctx)
    return v


def mg_nn_loss_grad(ctx, etas, grad: bool = True):
    e = _host(etas)
    loss = ctypes.c_double(0)
    g = np.empty(NN_PARAMS, dtype=np.complex128) if grad else None
    _check(load().mg_nn_loss_grad(ctx, _ptr(e), int(e.shape[0]), ctypes.byref(loss), _ptr(g) if grad else None), ctx)
    return loss.value, (nn_unflatten(g) if grad else None)


def mg_nn_train(ctx, etas, steps: int, lr: float):
    e = _host(etas)
    l0, l1 = ctypes.c_double(0), ctypes.c_double(0)
    _check(load().mg_nn_train(ctx, _ptr(e), int(e.shape[0]), int(steps), float(lr), ctypes.byref(l0),
                              ctypes.byref(l1)), ctx)
    return l0.value, l1.value


def mg_setup_learned(ctx, etas, refine_iters: int = 0) -> None:
    _check(load().mg_setup_learned(ctx, _ptr(_host(etas)), int(refine_iters)), ctx)


def mg_setup_level2(ctx, V2) -> None:
    _check(load().mg_setup_level2(ctx, _ptr(_host(V2))), ctx)


def mg_set_level2_vectors(ctx, V2) -> None:
    _check(load().mg_set_level2_vectors(ctx, _ptr(_host(V2))), ctx)


def mg_get_level2_prolongator(ctx, nv2: int, Vc1: int, nc1: int) -> np.ndarray:
    out = np.empty((nv2, Vc1, nc1), dtype=np.complex128)
    _check(load().mg_get_level2_prolongator(ctx, _ptr(out)), ctx)
    return out


def mg_get_level2_op(ctx, Vc2: int, nc2: int) -> np.ndarray:
    out = np.empty((Vc2, 9, nc2, nc2), dtype=np.complex128)
    _check(load().mg_get_level2_op(ctx, _ptr(out)), ctx)
    return out


def mg_kcycle(ctx, r1, prec: int = MG_FP64) -> np.ndarray:
    r1 = _host(r1)
    e1 = np.empty_like(r1)
    _check(load().mg_kcycle(ctx, _ptr(r1), _ptr(e1), int(prec)), ctx)
    return e1


def mg_get_coarse_op(ctx, Vc: int, nc: int) -> np.ndarray:
    out = np.empty((Vc, 9, nc, nc), dtype=np.complex128)
    _check(load().mg_get_coarse_op(ctx, _ptr(out)), ctx)
    return out


def mg_solve(ctx, b, out=None):
    """Host solve: returns (x, info dict).  NOT_CONVERGED is reported in info.
    ``out``: an optional contiguous complex128 host array of b's size (e.g. a
    view of pinned memory) that receives x."""
    b = _host(b)
    if out is None:
        x = np.empty_like(b)
    else:
        x = out
        if not isinstance(x, np.ndarray) or x.dtype != np.complex128 or not x.flags.c_contiguous or x.size != b.size:
            raise ValueError("out must be a contiguous complex128 array of the source's size")
    info = MgSolveInfo()
    _check(load().mg_solve(ctx, _ptr(b), _ptr(x), ctypes.byref(info)), ctx, allow=(MG_ERR_NOT_CONVERGED,))
    return x, info.as_dict()


def mg_solve_device(ctx, b_dev, x_dev) -> dict:
    info = MgSolveInfo()
    _check(load().mg_solve_device(ctx, _dev_ptr(b_dev), _dev_ptr(x_dev), ctypes.byref(info)), ctx,
           allow=(MG_ERR_NOT_CONVERGED,))
    return info.as_dict()


def mg_solve_batched(ctx, b):
    """b (nrhs, V, 4, 3) host -> (x, [info dicts])."""
    b = _host(b)
    nrhs = b.shape[0]
    x = np.empty_like(b)
    infos = (MgSolveInfo * nrhs)()
    _check(load().mg_solve_batched(ctx, _ptr(b), _ptr(x), nrhs, infos), ctx, allow=(MG_ERR_NOT_CONVERGED,))
    return x, [i.as_dict() for i in infos]


def mg_solve_batched_device(ctx, b_dev, x_dev, nrhs: int):
    infos = (MgSolveInfo * nrhs)()
    _check(load().mg_solve_batched_device(ctx, _dev_ptr(b_dev), _dev_ptr(x_dev), int(nrhs), infos), ctx,
           allow=(MG_ERR_NOT_CONVERGED,))
    return [i.as_dict() for i in infos]


def mg_solve_eo_cg(ctx, b, tol: float = 1e-10, maxit: int = 100000, prec: int = MG_FP32):
    """Red-black preconditioned CG (host buffers): returns (x, info dict)."""
    b = _host(b)
    x = np.empty_like(b)
    info = MgSolveInfo()
    _check(load().mg_solve_eo_cg(ctx, _ptr(b), _ptr(x), float(tol), int(maxit), int(prec), ctypes.byref(info)), ctx,
           allow=(MG_ERR_NOT_CONVERGED,))
    return x, info.as_dict()


def mg_solve_eo_cg_device(ctx, b_dev, x_dev, tol: float = 1e-10, maxit: int = 100000, prec: int = MG_FP32) -> dict:
    info = MgSolveInfo()
    _check(load().mg_solve_eo_cg_device(ctx, _dev_ptr(b_dev), _dev_ptr(x_dev), float(tol), int(maxit), int(prec),
                                        ctypes.byref(info)), ctx, allow=(MG_ERR_NOT_CONVERGED,))
    return info.as_dict()


def mg_apply_coarse_batched(ctx, x, dagger: bool = False, impl: int = 0) -> np.ndarray:
    """x (nrhs, Vc, nc) host -> y (nrhs, Vc, nc); impl 0 tensor cores, 1 SIMT FP64."""
    x = _host(x)
    y = np.empty_like(x)
    _check(load().mg_apply_coarse_batched(ctx, _ptr(x), _ptr(y), int(x.shape[0]), int(bool(dagger)), int(impl)), ctx)
    return y


def mg_apply_dslash(ctx, psi, prec: int = MG_FP64) -> np.ndarray:
    psi = _host(psi)
    out = np.empty_like(psi)
    _check(load().mg_apply_dslash(ctx, _ptr(psi), _ptr(out), int(prec)), ctx)
    return out


def mg_restrict(ctx, r, Vc: int, nc: int, prec: int = MG_FP64) -> np.ndarray:
    r = _host(r)
    out = np.empty((Vc, nc), dtype=np.complex128)
    _check(load().mg_restrict(ctx, _ptr(r), _ptr(out), int(prec)), ctx)
    return out


def mg_prolong(ctx, yc, V: int, prec: int = MG_FP64) -> np.ndarray:
    yc = _host(yc)
    out = np.empty((V, 4, 3), dtype=np.complex128)
    _check(load().mg_prolong(ctx, _ptr(yc), _ptr(out), int(prec)), ctx)
    return out


def mg_apply_coarse(ctx, x, dagger: bool = False, prec: int = MG_FP64) -> np.ndarray:
    x = _host(x)
    out = np.empty_like(x)
    _check(load().mg_apply_coarse(ctx, _ptr(x), _ptr(out), int(bool(dagger)), int(prec)), ctx)
    return out


def mg_mr(ctx, e, r, nsteps: int, prec: int = MG_FP64):
    e = _host(e).copy()
    r = _host(r).copy()
    _check(load().mg_mr(ctx, _ptr(e), _ptr(r), int(nsteps), int(prec)), ctx)
    return e, r


def mg_coarse_solve(ctx, rc, tol: float, maxit: int, prec: int = MG_FP64):
    rc = _host(rc)
    y = np.empty_like(rc)
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0)
    _check(load().mg_coarse_solve(ctx, _ptr(rc), _ptr(y), float(tol), int(maxit), int(prec), ctypes.byref(it),
                                  ctypes.byref(rel)), ctx)
    return y, it.value, rel.value


def mg_coarse_solve_noalloc(ctx, rc_dev, y_dev, tol: float, maxit: int):
    """Allocation-free FP64 coarse solve on device buffers; returns (iters, final_rel)."""
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0)
    _check(load().mg_coarse_solve_noalloc(ctx, _dev_ptr(rc_dev), _dev_ptr(y_dev), float(tol), int(maxit),
                                          ctypes.byref(it), ctypes.byref(rel)), ctx)
    return it.value, rel.value


def mg_vcycle(ctx, r, prec: int = MG_FP64) -> np.ndarray:
    r = _host(r)
    z = np.empty_like(r)
    _check(load().mg_vcycle(ctx, _ptr(r), _ptr(z), int(prec)), ctx)
    return z


def mg_time_dslash(ctx, prec: int = MG_FP32, reps: int = 50):
    ms = ctypes.c_double(0)
    nbytes = ctypes.c_double(0)
    _check(load().mg_time_dslash(ctx, int(prec), int(reps), ctypes.byref(ms), ctypes.byref(nbytes)), ctx)
    return ms.value, nbytes.value


def mg_time_coarse_floor(ctx, rounds: int = 200):
    """(us per round of the two tagged coarse stencils alone, us per exchange alone)."""
    a = ctypes.c_double(0)
    b = ctypes.c_double(0)
    _check(load().mg_time_coarse_floor(ctx, int(rounds), ctypes.byref(a), ctypes.byref(b)), ctx)
    return a.value, b.value


def mg_time_coarse_batched(ctx, nrhs: int, reps: int = 20):
    """(ms per launch, algorithmic bytes, useful flops) of the tensor-core batched coarse stencil."""
    ms, nb, fl = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
    _check(load().mg_time_coarse_batched(ctx, int(nrhs), int(reps), ctypes.byref(ms), ctypes.byref(nb),
                                         ctypes.byref(fl)), ctx)
    return ms.value, nb.value, fl.value


def mg_time_dslash_cold(ctx, flush_ptr: int, flush_bytes: int, prec: int = MG_FP32, reps: int = 20):
    """Mean dslash time with the L2 flushed (a device buffer of flush_bytes overwritten) before each launch."""
    ms = ctypes.c_double(0)
    nbytes = ctypes.c_double(0)
    _check(load().mg_time_dslash_cold(ctx, int(prec), int(reps), ctypes.c_void_p(flush_ptr), ctypes.c_size_t(flush_bytes),
                                      ctypes.byref(ms), ctypes.byref(nbytes)), ctx)
    return ms.value, nbytes.value


KERNEL_CLASSES = ("dslash", "coarse_solve", "restrict", "prolong", "block_ortho", "coarse_build", "krylov",
                  "true_residual")


def mg_kernel_launches() -> int:
    return int(load().mg_kernel_launches())


COARSE_KERNELS = {-1: "none", 0: "k_cgnr_persistent (operator from global memory)",
                  1: "k_cgls_onchip (operator resident in shared memory)",
                  2: "k_cgls_onchip (operator streamed through shared memory)",
                  3: "k_cgls_onchip (operator resident in tensor memory, products on the CUDA cores)",
                  4: "k_cgls_onchip (operator resident in tensor memory, products on the tensor cores)"}


def mg_coarse_kernel(ctx) -> int:
    return int(load().mg_coarse_kernel(ctx))


def mg_check_wait_timeout(ctx, kind: int, spin_limit: int = 20000) -> int:
    """Status of one bounded device wait driven to give up (MG_ERR_TIMEOUT expected)."""
    return int(load().mg_check_wait_timeout(ctx, int(kind), int(spin_limit)))


def mg_profile_enable(ctx, on: bool = True) -> None:
    _check(load().mg_profile_enable(ctx, int(bool(on))), ctx)


def mg_profile_classes(ctx, classes) -> None:
    """Track only the given kernel classes (names of KERNEL_CLASSES) while profiling."""
    mask = 0
    for c in classes:
        mask |= 1 << KERNEL_CLASSES.index(c)
    _check(load().mg_profile_classes(ctx, mask), ctx)


def mg_profile_read(ctx):
    """({class: (total ms, launches)}, coarse CG iterations) since the last read."""
    n = len(KERNEL_CLASSES)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int * n)()
    cit = ctypes.c_double(0)
    _check(load().mg_profile_read(ctx, ms, cnt, ctypes.byref(cit)), ctx)
    return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_CLASSES)}, cit.value


class WilsonMG:
    """Owning wrapper: ``with WilsonMG(dims, params) as mg: mg.set_links(U); ...``."""

    def __init__(self, dims, params: MgParams | None = None, t_antiperiodic: int = 1, stream=None):
        self.dims = tuple(int(x) for x in dims)
        self.params = params or mg_default_params()
        self.ctx = mg_create(self.dims, t_antiperiodic, self.params, stream)
        self.V = int(np.prod(self.dims))
        self.Vc = int(np.prod([d // b for d, b in zip(self.dims, self.params.block)]))
        self.nv = self.params.nvec
        self.nc = 2 * self.nv

    def close(self):
        if self.ctx:
            mg_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_links(self, U):
        mg_set_links(self.ctx, U)

    def set_links_device(self, U_dev, stream=None):
        mg_set_links_device(self.ctx, U_dev, stream)

    def set_mass(self, m):
        mg_set_mass(self.ctx, m)

    def set_params(self, p: MgParams):
        mg_set_params(self.ctx, p)
        self.params = p

    def setup(self, V0):
        mg_setup(self.ctx, V0)

    def setup_device(self, V0_dev):
        mg_setup_device(self.ctx, V0_dev)

    def set_null_vectors(self, V):
        mg_set_null_vectors(self.ctx, V)

    @property
    def Vc2(self):
        return int(np.prod([d // b // c for d, b, c in zip(self.dims, self.params.block, self.params.block2)]))

    def nn_set_weights(self, Ws):
        mg_nn_set_weights(self.ctx, Ws)

    def nn_get_weights(self):
        return mg_nn_get_weights(self.ctx)

    def nn_forward(self, etas):
        return mg_nn_forward(self.ctx, etas)

    def nn_loss_grad(self, etas, grad=True):
        return mg_nn_loss_grad(self.ctx, etas, grad)

    def nn_train(self, etas, steps, lr):
        return mg_nn_train(self.ctx, etas, steps, lr)

    def setup_learned(self, etas, refine_iters=0):
        mg_setup_learned(self.ctx, etas, refine_iters)

    def setup_level2(self, V2):
        mg_setup_level2(self.ctx, V2)

    def set_level2_vectors(self, V2):
        mg_set_level2_vectors(self.ctx, V2)

    def level2_prolongator(self):
        return mg_get_level2_prolongator(self.ctx, self.params.nvec2, self.Vc, self.nc)

    def level2_op(self):
        return mg_get_level2_op(self.ctx, self.Vc2, 2 * self.params.nvec2)

    def kcycle(self, r1, prec=MG_FP64):
        return mg_kcycle(self.ctx, r1, prec)

    def prolongator(self):
        return mg_get_prolongator(self.ctx, self.nv, self.V)

    def null_vectors(self):
        return mg_get_null_vectors(self.ctx, self.nv, self.V)

    def coarse_op(self):
        return mg_get_coarse_op(self.ctx, self.Vc, self.nc)

    def solve(self, b, out=None):
        return mg_solve(self.ctx, b, out)

    def solve_device(self, b_dev, x_dev):
        return mg_solve_device(self.ctx, b_dev, x_dev)

    def solve_batched(self, b):
        return mg_solve_batched(self.ctx, b)

    def solve_batched_device(self, b_dev, x_dev, nrhs):
        return mg_solve_batched_device(self.ctx, b_dev, x_dev, nrhs)

    def solve_eo_cg(self, b, tol=1e-10, maxit=100000, prec=MG_FP32):
        return mg_solve_eo_cg(self.ctx, b, tol, maxit, prec)

    def solve_eo_cg_device(self, b_dev, x_dev, tol=1e-10, maxit=100000, prec=MG_FP32):
        return mg_solve_eo_cg_device(self.ctx, b_dev, x_dev, tol, maxit, prec)

    def coarse_batched(self, x, dagger=False, impl=0):
        return mg_apply_coarse_batched(self.ctx, x, dagger, impl)

    def dslash(self, psi, prec=MG_FP64):
        return mg_apply_dslash(self.ctx, psi, prec)

    def restrict(self, r, prec=MG_FP64):
        return mg_restrict(self.ctx, r, self.Vc, self.nc, prec)

    def prolong(self, yc, prec=MG_FP64):
        return mg_prolong(self.ctx, yc, self.V, prec)

    def coarse(self, x, dagger=False, prec=MG_FP64):
        return mg_apply_coarse(self.ctx, x, dagger, prec)

    def mr(self, e, r, nsteps, prec=MG_FP64):
        return mg_mr(self.ctx, e, r, nsteps, prec)

    def coarse_solve(self, rc, tol, maxit, prec=MG_FP64):
        return mg_coarse_solve(self.ctx, rc, tol, maxit, prec)

    def vcycle(self, r, prec=MG_FP64):
        return mg_vcycle(self.ctx, r, prec)

    def profile_enable(self, on=True):
        mg_profile_enable(self.ctx, on)

    def profile_read(self):
        return mg_profile_read(self.ctx)

    def profile_classes(self, classes):
        mg_profile_classes(self.ctx, classes)

    def time_dslash(self, prec=MG_FP32, reps=50):
        return mg_time_dslash(self.ctx, prec, reps)

    def time_coarse_floor(self, rounds=200):
        return mg_time_coarse_floor(self.ctx, rounds)

    def time_coarse_batched(self, nrhs, reps=20):
        return mg_time_coarse_batched(self.ctx, nrhs, reps)

    def time_dslash_cold(self, flush_ptr: int, flush_bytes: int, prec=MG_FP32, reps=20):
        return mg_time_dslash_cold(self.ctx, flush_ptr, flush_bytes, prec, reps)

    def coarse_kernel(self) -> int:
        """MG_CK_* id of the coarse CGNR kernel the last coarse solve ran."""
        return mg_coarse_kernel(self.ctx)
