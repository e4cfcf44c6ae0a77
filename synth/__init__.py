"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This package holds no arithmetic of the multigrid method.  It builds
``synth.c`` (Philox4x32-10 random numbers, Gaussian fields, a quenched
Wilson-gauge heatbath) into a small shared library and exposes:

* :func:`gaussian_spinor`, :func:`gaussian_vectors` -- seeded complex Gaussian
  fields (sources and the random starts of the adaptive setup);
* :func:`point_source` -- a delta source at one site, spin and colour;
* :func:`gauge_field` -- SU(3) links from a hot start followed by ``sweeps``
  compound sweeps (1 Kennedy-Pendleton heatbath + ``n_or`` over-relaxation),
  cached on disk because the workloads reuse them;
* :func:`random_gauge_transform` -- Omega(x) in SU(3), for covariance checks.

Layouts (also the C-ABI boundary's): site = x + L0*(y + L1*(z + L2*t)),
links ``U[mu, site, a, b]``, spinors ``psi[site, spin, colour]``, complex128.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsynth.so")
_CACHE = os.environ.get("SYNTH_CACHE_DIR", os.path.join(_BUILD, "cache"))
_lock = threading.Lock()
_lib = None

# bump when synth.c changes the numbers it produces (invalidates the cache)
GENERATOR_VERSION = 1


def build(force: bool = False) -> str:
    """Compile synth.c with gcc (no FMA contraction, OpenMP) into _build/."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            lib.synth_philox4x32_10.argtypes = [P, P, P]
            lib.synth_log.argtypes = [ctypes.c_double]
            lib.synth_log.restype = ctypes.c_double
            lib.synth_gaussian.argtypes = [P, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32]
            lib.synth_gauge_hot.argtypes = [P, P, ctypes.c_uint64]
            lib.synth_gauge_unit.argtypes = [P, P]
            lib.synth_gauge_sweep.argtypes = [P, P, ctypes.c_double, ctypes.c_int, ctypes.c_uint64, ctypes.c_int]
            lib.synth_plaquette.argtypes = [P, P]
            lib.synth_plaquette.restype = ctypes.c_double
            lib.synth_random_su3_field.argtypes = [P, ctypes.c_int64, ctypes.c_uint64]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _dims(L):
    L = np.ascontiguousarray(np.asarray(L, dtype=np.int32))
    assert L.shape == (4,) and (L > 0).all()
    return L


def philox4x32_10(counter, key) -> np.ndarray:
    """One Philox4x32-10 block: 4 uint32 counter words, 2 uint32 key words."""
    lib = _load()
    c = np.ascontiguousarray(np.asarray(counter, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib.synth_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def log(x: float) -> float:
    """The generator's own natural logarithm (series, no libm)."""
    return _load().synth_log(float(x))


def gaussian(n_complex: int, seed: int, stream: int) -> np.ndarray:
    """n complex128 numbers, real and imaginary parts independent N(0,1)."""
    out = np.empty(n_complex, dtype=np.complex128)
    _load().synth_gaussian(_ptr(out), int(n_complex), int(seed) & (2**64 - 1), int(stream) & 0xFFFFFFFF)
    return out


def volume(L) -> int:
    return int(np.prod(np.asarray(L, dtype=np.int64)))


def gaussian_spinor(L, seed: int, stream: int = 0) -> np.ndarray:
    """Gaussian fine spinor field, shape (V, 4, 3) complex128."""
    V = volume(L)
    return gaussian(V * 12, seed, stream).reshape(V, 4, 3)


def gaussian_vectors(L, n: int, seed: int, stream0: int = 1000) -> np.ndarray:
    """n independent Gaussian fine fields, shape (n, V, 4, 3) (setup random starts)."""
    return np.stack([gaussian_spinor(L, seed, stream0 + i) for i in range(n)])


def point_source(L, site: int, spin: int, colour: int) -> np.ndarray:
    V = volume(L)
    b = np.zeros((V, 4, 3), dtype=np.complex128)
    b[site, spin, colour] = 1.0
    return b


def unit_gauge(L) -> np.ndarray:
    V = volume(L)
    U = np.empty((4, V, 3, 3), dtype=np.complex128)
    _load().synth_gauge_unit(_ptr(U), _ptr(_dims(L)))
    return U


def hot_gauge(L, seed: int) -> np.ndarray:
    """Independent Haar-like random SU(3) on every link (hot start, 0 sweeps)."""
    V = volume(L)
    U = np.empty((4, V, 3, 3), dtype=np.complex128)
    _load().synth_gauge_hot(_ptr(U), _ptr(_dims(L)), int(seed))
    return U


def gauge_sweep(U: np.ndarray, L, beta: float, n_or: int, seed: int, sweep: int) -> None:
    _load().synth_gauge_sweep(_ptr(U), _ptr(_dims(L)), float(beta), int(n_or), int(seed), int(sweep))


def plaquette(U: np.ndarray, L) -> float:
    return _load().synth_plaquette(_ptr(U), _ptr(_dims(L)))


def _cache_path(L, beta, sweeps, n_or, seed) -> str:
    tag = f"v{GENERATOR_VERSION}_L{'x'.join(map(str, L))}_b{beta!r}_s{sweeps}_or{n_or}_seed{seed}"
    h = hashlib.sha1(tag.encode()).hexdigest()[:10]
    return os.path.join(_CACHE, f"gauge_{tag}_{h}.npy")


def gauge_field(L, beta: float = 6.0, sweeps: int = 200, n_or: int = 4, seed: int = 1,
                cache: bool = True) -> np.ndarray:
    """Quenched SU(3) links: hot start, then `sweeps` x (1 heatbath + n_or OR).

    Shape (4, V, 3, 3) complex128.  Deterministic in (L, beta, sweeps, n_or, seed)
    and bitwise identical on x86-64 and aarch64.
    """
    L = tuple(int(x) for x in L)
    path = _cache_path(L, beta, sweeps, n_or, seed)
    if cache and os.path.exists(path):
        return np.load(path)
    U = hot_gauge(L, seed)
    for s in range(sweeps):
        gauge_sweep(U, L, beta, n_or, seed, s)
    if cache:
        os.makedirs(_CACHE, exist_ok=True)
        tmp = path + f".tmp{os.getpid()}.npy"
        np.save(tmp, U)
        os.replace(tmp, path)
    return U


def random_gauge_transform(V: int, seed: int) -> np.ndarray:
    """Omega[site] in SU(3), shape (V, 3, 3)."""
    Om = np.empty((V, 3, 3), dtype=np.complex128)
    _load().synth_random_su3_field(_ptr(Om), int(V), int(seed))
    return Om


def checksum(a: np.ndarray) -> str:
    """sha1 of the raw bytes: detects any bit difference between machines."""
    return hashlib.sha1(np.ascontiguousarray(a).tobytes()).hexdigest()
