"""Boundary entry points on the GPU, through the C-ABI: link upload from device
memory on a caller's stream, the solve-info fields, and the bounded device
waits (each wait driven to give up with a short poll limit must return
MG_ERR_TIMEOUT and leave the context usable)."""
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


@pytest.fixture(scope="module", autouse=True)
def _built():
    wmg.build.build()
    wmg.load()


def test_set_links_device_on_caller_stream():
    """Links uploaded from a device buffer on a side stream give the same
    operator as the host upload (eq. 2 against the oracle to 1e-12); the buffer
    is overwritten on that stream right after the call, which the stream
    ordering of the entry point must make harmless."""
    import torch
    L = (8, 4, 4, 8)
    U = rough_gauge(L, seed=21)
    psi = synth.gaussian_spinor(L, 22)
    m = -0.37
    ref = oracle.dslash(U, psi, m, L)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        dU = torch.from_numpy(np.ascontiguousarray(U).view(np.float64).ravel().copy()).to("cuda", non_blocking=False)
    with wmg.WilsonMG(L, params(2, (2, 2, 2, 2))) as mg:
        mg.set_links_device(dU, side)
        with torch.cuda.stream(side):
            dU.zero_()                         # ordered after the conversion on `side`
        side.synchronize()
        mg.set_mass(m)
        assert maxrel(mg.dslash(psi, wmg.MG_FP64), ref) < 1e-12
        assert maxrel(mg.dslash(psi, wmg.MG_FP32), ref) < 1e-5


def test_solve_info_setup_time_and_dslash_bytes():
    L, B, nv, U, m = c1_workload()
    V0 = synth.gaussian_vectors(L, nv, 2001)
    b = synth.gaussian_spinor(L, 7)
    with wmg.WilsonMG(L, params(nv, B, prec_inner=wmg.MG_FP32, delta=1e-4)) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        mg.setup(V0)
        x, info = mg.solve(b)
    assert info["status"] == 0 and info["setup_ms"] > 0
    V = int(np.prod(L))
    # every application moves at least the FP32 bytes of some and at most the FP64 bytes of all
    assert 248 * V * info["fine_matvecs"] <= info["dslash_bytes"] <= 960 * V * info["fine_matvecs"]


@pytest.mark.parametrize("kind", [0, 1, 2, 3])
def test_bounded_wait_gives_up_and_context_stays_usable(kind):
    """kind 0: epoch exchange with one publisher missing; 1: counter grid
    barrier with one arrival missing; 2: mbarrier transaction never completed;
    3: epoch-tagged entry never written.  Each gives up after the short poll
    limit with MG_ERR_TIMEOUT; the same context then applies D correctly."""
    L = (4, 4, 4, 8)
    U = rough_gauge(L, seed=31)
    psi = synth.gaussian_spinor(L, 32)
    m = -0.3
    with wmg.WilsonMG(L, params(2, (2, 2, 2, 2))) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        st = wmg.mg_check_wait_timeout(mg.ctx, kind, 20000)
        assert st == wmg.MG_ERR_TIMEOUT, wmg.status_string(st)
        assert maxrel(mg.dslash(psi, wmg.MG_FP64), oracle.dslash(U, psi, m, L)) < 1e-12
        # a second probe on the same context behaves the same way
        assert wmg.mg_check_wait_timeout(mg.ctx, kind, 20000) == wmg.MG_ERR_TIMEOUT
