"""The learned setup on the GPU, through the C-ABI, against the oracle's network
(oracle/learned.py) on identical seeded inputs: the forward pass (FP32 kernels
against FP64, 1e-5), the Wilson operator of eq. 2 as a special case of the
network (the transport conventions), the loss and its gradient, that Adam steps
lower the loss, and that the learned setup feeds a converging MG-GCR solve."""
import numpy as np
import pytest

import oracle
import oracle.learned as nn
import paper_1005_3043_gb300 as wmg
import synth
from tests._fields import rough_gauge

pytestmark = pytest.mark.gpu


def maxrel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def params(nv, B, **kw):
    p = wmg.mg_default_params()
    for i in range(4):
        p.block[i] = B[i]
    p.nvec = nv
    p.setup_group = kw.pop("setup_group", 2)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.fixture(scope="module", autouse=True)
def _built():
    wmg.build.build()
    wmg.load()


@pytest.mark.parametrize("L,tap", [((4, 4, 4, 8), 1), ((8, 4, 2, 4), 0)])
def test_forward_matches_oracle(L, tap):
    U = rough_gauge(L, seed=61)
    Ws = nn.init_weights(62)
    etas = np.stack([synth.gaussian_spinor(L, 63, stream=i) for i in range(2)])
    with wmg.WilsonMG(L, params(2, (2, 2, 2, 2)), t_antiperiodic=tap) as mg:
        mg.set_links(U)
        mg.nn_set_weights(Ws)
        v = mg.nn_forward(etas)
        back = mg.nn_get_weights()
    for i in range(2):
        ref = nn.forward(Ws, U, etas[i], L, tap)[-1][0]
        assert maxrel(v[i], ref) < 1e-5, maxrel(v[i], ref)
    assert all(np.array_equal(a, b) for a, b in zip(back, Ws))


def test_network_with_wilson_weights_is_eq2():
    """Layer 1 with (4+m) on site and -(1 -/+ gamma_mu)/2 on the hops into
    channel 0, layers 2-4 the identity on channel 0: the network is D(U)."""
    L = (4, 4, 4, 8)
    U = rough_gauge(L, seed=64)
    m = -0.31
    g = oracle.gamma_matrices()
    Ws = [np.zeros((co, ci, 9, 4, 4), complex) for ci, co in zip(wmg.NN_CHANNELS[:-1], wmg.NN_CHANNELS[1:])]
    Ws[0][0, 0, 0] = (4 + m) * np.eye(4)
    for mu in range(4):
        Ws[0][0, 0, 1 + 2 * mu] = -0.5 * (np.eye(4) - g[mu])
        Ws[0][0, 0, 2 + 2 * mu] = -0.5 * (np.eye(4) + g[mu])
    for k in (1, 2, 3):
        Ws[k][0, 0, 0] = np.eye(4)
    psi = synth.gaussian_spinor(L, 65)
    with wmg.WilsonMG(L, params(2, (2, 2, 2, 2))) as mg:
        mg.set_links(U)
        mg.nn_set_weights(Ws)
        v = mg.nn_forward(psi[None])[0]
    assert maxrel(v, oracle.dslash(U, psi, m, L)) < 1e-5


def test_loss_and_gradient_match_oracle():
    L, B, nv = (4, 4, 4, 8), (2, 2, 2, 2), 4
    U = rough_gauge(L, seed=66)
    V = synth.gaussian_vectors(L, nv, 67)
    P, st = oracle.block_orthonormalize(V, L, B)
    assert st == 0
    etas = np.stack([synth.gaussian_spinor(L, 68, stream=i) for i in range(3)])
    Ws = nn.init_weights(69)
    l_ref, G_ref = nn.loss_and_grad(Ws, U, list(etas), P, L, B)
    with wmg.WilsonMG(L, params(nv, B)) as mg:
        mg.set_links(U)
        mg.set_mass(-0.3)
        mg.set_null_vectors(V)
        mg.nn_set_weights(Ws)
        l, G = mg.nn_loss_grad(etas)
    assert abs(l - l_ref) < 1e-5 * l_ref, (l, l_ref)
    for k in range(4):
        assert maxrel(G[k], G_ref[k]) < 1e-4, (k, maxrel(G[k], G_ref[k]))


def test_training_lowers_the_loss_and_learned_setup_solves():
    """On the 8^4 beta = 6.0 field: Adam steps against the plain setup's
    projector lower the loss; the learned prototypes (with one refinement
    iteration) give a P and D_c with which MG-GCR reaches 1e-10."""
    from tests._fields import c1_workload
    L, B, nv, U, m = c1_workload()
    V0 = synth.gaussian_vectors(L, nv, 2001)
    etas = np.stack([synth.gaussian_spinor(L, 70, stream=i) for i in range(nv)])
    b = synth.gaussian_spinor(L, 7)
    p = params(nv, B, setup_group=4, smoother=1, smoother_steps=4, prec_inner=wmg.MG_FP32, delta=1e-4)
    with wmg.WilsonMG(L, p) as mg:
        mg.set_links(U)
        mg.set_mass(m)
        mg.setup(V0)
        mg.nn_set_weights(nn.init_weights(71))
        l0, _ = mg.nn_train(etas[:2], 1, 1e-3)
        _, l1 = mg.nn_train(etas[:2], 30, 1e-3)
        assert l1 < l0, (l0, l1)
        mg.setup_learned(etas, refine_iters=1)
        x, info = mg.solve(b)
    assert info["status"] == 0 and info["setup_ms"] > 0
    assert np.linalg.norm(b - oracle.dslash(U, x, m, L)) <= 1e-10 * np.linalg.norm(b)
