"""Pins of the learned-setup oracle (oracle/learned.py): the gauge-covariant
parallel-transport convolution that stands in for the random-start relaxation
of the Sec. IV setup.  Each check is independent of the network code: the
Wilson operator of eq. 2 (the oracle's C routine) as a special case of one
layer, gauge covariance under a random SU(3) transform, the gradient against
central finite differences of the loss, and the projector's algebra."""
import numpy as np
import pytest

import oracle
import oracle.learned as nn
import synth
from tests._fields import rough_gauge


def _wilson_weights(m):
    """One-channel layer weights that make the layer eq. 2: (4+m) on site,
    -(1 - gamma_mu)/2 forward, -(1 + gamma_mu)/2 backward."""
    g = oracle.gamma_matrices()
    W = np.zeros((1, 1, 9, 4, 4), dtype=np.complex128)
    W[0, 0, 0] = (4 + m) * np.eye(4)
    for mu in range(4):
        W[0, 0, 1 + 2 * mu] = -0.5 * (np.eye(4) - g[mu])
        W[0, 0, 2 + 2 * mu] = -0.5 * (np.eye(4) + g[mu])
    return W


@pytest.mark.parametrize("tap", [0, 1])
def test_layer_with_wilson_weights_is_eq2(tap):
    L = (4, 2, 6, 4)
    U = rough_gauge(L, seed=31)
    psi = synth.gaussian_spinor(L, 32)
    m = -0.37
    out = nn.layer(_wilson_weights(m), U, psi[None], L, tap)[0]
    ref = oracle.dslash(U, psi, m, L, tap)
    assert np.abs(out - ref).max() < 1e-13 * np.abs(ref).max()


def test_network_is_gauge_covariant():
    """U_mu(x) -> G(x) U_mu(x) G(x+mu)^dag, eta -> G eta: the output becomes G v."""
    L = (4, 4, 2, 4)
    V = oracle.volume(L)
    U = rough_gauge(L, seed=33)
    G = synth.random_gauge_transform(V, 34)
    Ug = np.empty_like(U)
    c = np.indices(tuple(L)[::-1]).reshape(4, -1)[::-1]
    for mu in range(4):
        cc = c.copy()
        cc[mu] = (cc[mu] + 1) % L[mu]
        nxt = cc[0] + L[0] * (cc[1] + L[1] * (cc[2] + L[2] * cc[3]))
        Ug[mu] = np.einsum("xab,xbc,xdc->xad", G, U[mu], G[nxt].conj())
    eta = synth.gaussian_spinor(L, 35)
    Ws = nn.init_weights(36)
    v = nn.forward(Ws, U, eta, L)[-1][0]
    vg = nn.forward(Ws, Ug, np.einsum("xab,xsb->xsa", G, eta), L)[-1][0]
    assert np.abs(vg - np.einsum("xab,xsb->xsa", G, v)).max() < 1e-12 * np.abs(v).max()


def test_gradient_matches_finite_differences():
    """dLoss/dh along a random weight direction D equals Re<G, D> (G the
    returned gradient, 2 dLoss/d conj W) to central-difference accuracy."""
    L, B = (4, 4, 4, 4), (2, 2, 2, 2)
    U = rough_gauge(L, seed=37)
    P, st = oracle.block_orthonormalize(synth.gaussian_vectors(L, 3, 38), L, B)
    assert st == 0
    etas = [synth.gaussian_spinor(L, 39, stream=i) for i in range(2)]
    Ws = nn.init_weights(40, channels=(1, 2, 2, 1))
    l0, G = nn.loss_and_grad(Ws, U, etas, P, L, B)
    assert abs(l0 - nn.loss(Ws, U, etas, P, L, B)) < 1e-14
    rng = np.random.default_rng(41)
    D = [rng.standard_normal(W.shape) + 1j * rng.standard_normal(W.shape) for W in Ws]
    h = 1e-5
    lp = nn.loss([W + h * d for W, d in zip(Ws, D)], U, etas, P, L, B)
    lm = nn.loss([W - h * d for W, d in zip(Ws, D)], U, etas, P, L, B)
    fd = (lp - lm) / (2 * h)
    an = sum(np.vdot(g, d).real for g, d in zip(G, D))
    assert abs(fd - an) < 1e-6 * abs(an), (fd, an)


def test_projector_algebra():
    """(1 - P P^dag) is an orthogonal projector; its loss is 0 on range(P) and
    1 on vectors orthogonal to it."""
    L, B = (4, 4, 4, 4), (2, 2, 2, 2)
    V0 = synth.gaussian_vectors(L, 3, 42)
    P, _ = oracle.block_orthonormalize(V0, L, B)
    x = synth.gaussian_spinor(L, 43)
    r = nn.project_out(P, x, L, B)
    assert np.abs(nn.project_out(P, r, L, B) - r).max() < 1e-13 * np.abs(r).max()
    assert abs(np.vdot(r, x - r)) < 1e-12 * np.vdot(x, x).real
    assert np.abs(nn.project_out(P, V0[1], L, B)).max() < 1e-13 * np.abs(V0[1]).max()
