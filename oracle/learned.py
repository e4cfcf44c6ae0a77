"""CPU oracle of the learned setup (test infrastructure, like the rest of
``oracle/``): a gauge-covariant parallel-transport convolution network that
maps the links and random starts to prototype vectors for the adaptive setup.

The paper's setup (Sec. IV) begins with 10 relaxation steps applied to each of
20 random vectors; each relaxation step is a polynomial in the hopping term of
eq. 2 applied to the random vector.  The learned replacement keeps that form:
a stack of layers, each a sum over the nine stencil directions d (0: the site
itself, +-mu: its neighbours) of a learned 4x4 complex spin matrix applied
after parallel transport by the links,

    out[a](x) = sum_b sum_d W[a, b, d] (T_d in[b])(x),
    (T_0 p)(x) = p(x),  (T_{+mu} p)(x) = U_mu(x) p(x + mu),
    (T_{-mu} p)(x) = U_mu(x - mu)^dag p(x - mu)

(with the antiperiodic sign on hops across the t boundary, as in eq. 2), on
channels a, b.  Colour is only ever touched by the links, so the layer is
gauge covariant: with U_mu(x) -> G(x) U_mu(x) G(x + mu)^dag and p -> G p the
output transforms as G out.  Four layers with 1 -> 8 -> 8 -> 8 -> 1 channels.

Training signal: the prototypes of the plain adaptive setup (Sec. IV) define
a block projector Pi = P P^dag (eq. 4); the loss of an output v is the part of
it outside that space, |(1 - Pi) v|^2 / |v|^2, averaged over the outputs.

Everything here is plain numpy in complex128, vectorised over sites only.
Parity: pinned by gauge covariance, by the adjoint identity <W, grad> against
finite differences of the loss, and by the linearity / stencil structure of a
single layer against a dense brute-force construction on a tiny lattice.
"""
from __future__ import annotations

import numpy as np

from . import prolong, restrict

CHANNELS = (1, 8, 8, 8, 1)


def _shift(p, L, mu, step):
    """p(x + step * mu) for every site x (p: (..., V, 4, 3) in lexicographic
    order x fastest), periodic index shift."""
    shape = p.shape[:-3] + tuple(L[::-1]) + (4, 3)
    q = p.reshape(shape)
    axis = len(p.shape[:-3]) + (3 - mu)
    return np.roll(q, -step, axis=axis).reshape(p.shape)


def _tsign(L, mu, step, tap):
    """(V,) factor -1 where the hop from x to x + step * mu crosses the t boundary."""
    V = int(np.prod(L))
    s = np.ones(V)
    if mu == 3 and tap:
        t = np.arange(V) // (L[0] * L[1] * L[2])
        s[(t == L[3] - 1) if step > 0 else (t == 0)] = -1.0
    return s


def transport(U, p, L, d, tap=1):
    """(T_d p) for d = 0 (identity), 1 + 2 mu (+mu), 2 + 2 mu (-mu); p (..., V, 4, 3)."""
    if d == 0:
        return p
    mu = (d - 1) // 2
    fwd = (d % 2) == 1
    if fwd:
        q = _shift(p, L, mu, +1)
        out = np.einsum("xab,...xsb->...xsa", U[mu], q)
    else:
        q = _shift(p, L, mu, -1)
        Ub = _link_shift(U[mu], L, mu, -1)               # U_mu(x - mu)
        out = np.einsum("xba,...xsb->...xsa", Ub.conj(), q)
    sg = _tsign(L, mu, +1 if fwd else -1, tap)
    return out * sg[:, None, None]


def _link_shift(Umu, L, mu, step):
    """Umu(x + step * mu) for every site x; Umu (V, 3, 3)."""
    q = Umu.reshape(tuple(L[::-1]) + (3, 3))
    return np.roll(q, -step, axis=3 - mu).reshape(-1, 3, 3)


def transport_adj(U, p, L, d, tap=1):
    """The adjoint of T_d: T_{+mu}^dag = T_{-mu}, T_{-mu}^dag = T_{+mu}, T_0^dag = T_0."""
    if d == 0:
        return p
    return transport(U, p, L, d + 1 if d % 2 == 1 else d - 1, tap)


def layer(W, U, inp, L, tap=1):
    """out[a] = sum_b sum_d W[a, b, d] (T_d inp[b]); W (Cout, Cin, 9, 4, 4), inp (Cin, V, 4, 3)."""
    cout = W.shape[0]
    out = np.zeros((cout,) + inp.shape[1:], dtype=np.complex128)
    for d in range(9):
        t = transport(U, inp, L, d, tap)                      # (Cin, V, 4, 3)
        out += np.einsum("abst,bxtc->axsc", W[:, :, d], t)
    return out


def forward(Ws, U, eta, L, tap=1):
    """Network output for one random start eta (V, 4, 3): the list of layer
    activations [x0 = eta[None], x1, ..., x4] (x4 has one channel)."""
    xs = [np.asarray(eta, dtype=np.complex128)[None]]
    for W in Ws:
        xs.append(layer(W, U, xs[-1], L, tap))
    return xs


def project_out(P, v, L, B):
    """(1 - P P^dag) v with the block prolongator P (eq. 4)."""
    return v - prolong(P, restrict(P, v, L, B), L, B)


def loss(Ws, U, etas, P, L, B, tap=1):
    """Mean over the random starts of |(1 - P P^dag) v|^2 / |v|^2, v = network(eta)."""
    tot = 0.0
    for eta in etas:
        v = forward(Ws, U, eta, L, tap)[-1][0]
        r = project_out(P, v, L, B)
        tot += np.vdot(r, r).real / np.vdot(v, v).real
    return tot / len(etas)


def loss_and_grad(Ws, U, etas, P, L, B, tap=1):
    """The loss and its gradient with respect to every weight, by the adjoint
    (reverse) pass.  For complex weights the gradient G is the Wirtinger
    derivative 2 dLoss/d(conj W): a small step W -> W - h G lowers the loss by
    h Re<G, G> to first order."""
    grads = [np.zeros_like(W) for W in Ws]
    tot = 0.0
    for eta in etas:
        xs = forward(Ws, U, eta, L, tap)
        v = xs[-1][0]
        vv = np.vdot(v, v).real
        r = project_out(P, v, L, B)
        rr = np.vdot(r, r).real
        tot += rr / vv
        # d(rr / vv)/d conj(v) = (Q v) / vv - rr v / vv^2 with Q = 1 - P P^dag (Q^2 = Q = Q^dag)
        g = (r / vv - rr * v / vv ** 2)[None]
        for k in range(len(Ws) - 1, -1, -1):
            W, xin = Ws[k], xs[k]
            gin = np.zeros_like(xin)
            for d in range(9):
                t = transport(U, xin, L, d, tap)
                # out[a] += W[a,b,d] t[b]: dL/dconj(W[a,b,d])_{st} = sum_{x,c} g[a](x)_s conj(t[b](x)_t)
                grads[k][:, :, d] += 2 * np.einsum("axsc,bxtc->abst", g, t.conj())
                # back to the input: t[b] receives sum_a W[a,b,d]^dag g[a]; then T_d^dag
                gt = np.einsum("abts,axtc->bxsc", W[:, :, d].conj(), g)
                gin += transport_adj(U, gt, L, d, tap)
            g = gin
    n = len(etas)
    return tot / n, [G / n for G in grads]


def init_weights(seed, channels=CHANNELS, scale=None):
    """Seeded initial weights: the identity spin matrix on the on-site term of
    every channel pair (a = b or the one-channel ends) scaled to keep norms,
    plus Gaussian noise of width scale on every entry (numpy Generator)."""
    rng = np.random.default_rng(seed)
    Ws = []
    for cin, cout in zip(channels[:-1], channels[1:]):
        s = scale if scale is not None else 0.3 / np.sqrt(9 * cin)
        W = s * (rng.standard_normal((cout, cin, 9, 4, 4)) + 1j * rng.standard_normal((cout, cin, 9, 4, 4)))
        for a in range(cout):
            for b in range(cin):
                if a % cin == b or cin == 1:
                    W[a, b, 0] += np.eye(4) / max(cin, 1) ** 0.5
        Ws.append(W)
    return Ws
