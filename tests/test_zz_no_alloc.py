"""The allocation-free coarse solve (mg_coarse_solve_noalloc) against the
regular coarse solve (mg_coarse_solve) through the C-ABI.

The allocation-free entry point is for callers that cannot allocate device
memory when they call (another framework owns the allocator, or allocation
is not allowed where they run); its scratch is a file-scope device array.
This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process."""
import numpy as np
import pytest

import paper_1005_3043_gb300 as wmg
import synth
from tests._fields import rough_gauge

pytestmark = pytest.mark.gpu


def test_noalloc_coarse_solve_matches_regular_two_calls():
    import torch
    wmg.build.build()
    L, B, nv = (8, 8, 8, 8), (4, 4, 4, 4), 4
    U = rough_gauge(L, seed=21)
    V0 = synth.gaussian_vectors(L, nv, 121)
    p = wmg.mg_default_params()
    p.nvec, p.setup_group = nv, 2
    with wmg.WilsonMG(L, p, stream=torch.cuda.current_stream()) as mg:
        mg.set_links(U)
        mg.set_mass(-0.2)
        mg.set_null_vectors(V0)
        for call in range(2):                       # the shared scratch keeps the last call's contents
            rc = synth.gaussian(mg.Vc * mg.nc, 300 + call, 0).reshape(mg.Vc, mg.nc)
            y_ref, it_ref, rel_ref = mg.coarse_solve(rc, 1e-3, 5000, wmg.MG_FP64)
            rc_dev = torch.from_numpy(rc.view(np.float64)).cuda()
            y_dev = torch.zeros_like(rc_dev)
            it, rel = wmg.mg_coarse_solve_noalloc(mg.ctx, rc_dev, y_dev, 1e-3, 5000)
            y = y_dev.cpu().numpy().view(np.complex128)
            assert it == it_ref
            assert abs(rel - rel_ref) <= 1e-12
            assert np.abs(y - y_ref).max() / np.abs(y_ref).max() < 1e-12
        # sizes beyond the stated maximum are rejected with a clear error:
        # 16x16x16x8 with 2^4 aggregates and Nv = 20 has 2048 x 40 = 81920 coarse entries
    Lb, Bb, nvb = (16, 16, 16, 8), (2, 2, 2, 2), 20
    pb = wmg.mg_default_params()
    for i in range(4):
        pb.block[i] = Bb[i]
    pb.nvec, pb.setup_group = nvb, 4
    with wmg.WilsonMG(Lb, pb) as big:
        big.set_links(synth.unit_gauge(Lb))
        big.set_null_vectors(synth.gaussian_vectors(Lb, nvb, 5))
        assert big.Vc * big.nc > 65536
        rc_big = torch.zeros(big.Vc * big.nc * 2, dtype=torch.float64, device="cuda")
        with pytest.raises(wmg.MGError) as ei:
            wmg.mg_coarse_solve_noalloc(big.ctx, rc_big, torch.zeros_like(rc_big), 1e-3, 10)
        assert ei.value.status == wmg.MG_ERR_INVALID_ARG
        assert "allocation-free limit" in str(ei.value)
