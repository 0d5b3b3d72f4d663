"""CPU FP64 oracle: the learned G-shell preconditioner network.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call
this module; only tests, the package's smoke check and the benchmark's CPU
baseline leg use it.  It shares no code with the CUDA library.

The paper's G-space diagonal preconditioner M(G) = 1/((G^2 - E)^2 + dE^2)
(Sec. II.C, under the M' equation) depends on |G| alone.  The learned variant
scales it per band i and per kinetic-energy shell s of the plane waves:

    W_G = M(G) * exp(z_{i, s(G)}) * R_G,    z_{i,s} = f(features_{i,s})

with f a multilayer perceptron 4 -> 128 -> 128 -> 128 -> 1 (tanh hidden
activations, linear output; the last layer starts at zero so the untrained
network reproduces M(G) exactly).  Features of (band i, shell s):

    f0 = (centre kinetic energy of shell s) / ecut
    f1 = log10( mean_{G in s} |R_G|^2 / mean_G |R_G|^2 )   (shell share of the residual)
    f2 = d_i / 0.1 Ha,  d_i = <x_i, (H-E) x_i>             (signed distance to E)
    f3 = log10(||R_i||) / 10

Training label (per band and shell): the per-shell gain that, for a
preconditioner diagonal in the shells, would turn the preconditioned residual
into the error e_i of the band -- the ratio of the error's magnitude to that
of M R in the shell, both taken as shares of their band totals,

    z*_{i,s} = clip( (1/2) log( (||e||_s^2 / ||e||^2) / (||M R||_s^2 / ||M R||^2) ),
                     log 0.1, log 10 ),

weighted by the shell's share of ||M R||^2; loss = weighted mean of
(z - z*)^2.  Only the shell-relative part matters: the search direction is
normalised before use.  (A least-squares gain Re<M R, e>_s / ||M R||_s^2 was
the first reading; its labels are dominated by the phase noise of e in the
high shells, where it drives the gain to zero, and a network trained on them
lost iterations on held-out boxes.  The magnitude ratio is the gain a diagonal
operator with e = K R would have.)  Parameters are a flat float vector in the order
W1[128][4], b1[128], W2[128][128], b2[128], W3[128][128], b3[128], W4[128], b4.
"""
from __future__ import annotations

import numpy as np

SIZES = (4, 128, 128, 128, 1)


def n_params():
    n = 0
    for a, b in zip(SIZES[:-1], SIZES[1:]):
        n += a * b + b
    return n


def unpack(theta):
    """Flat parameter vector -> [(W, b)] with W of shape (out, in)."""
    out = []
    o = 0
    for a, b in zip(SIZES[:-1], SIZES[1:]):
        W = theta[o:o + a * b].reshape(b, a)
        o += a * b
        bb = theta[o:o + b]
        o += b
        out.append((W, bb))
    return out


def init_params(seed=0):
    """Uniform(-1/sqrt(in), 1/sqrt(in)) hidden layers, zero output layer."""
    rng = np.random.default_rng(seed)
    parts = []
    for li, (a, b) in enumerate(zip(SIZES[:-1], SIZES[1:])):
        lim = 1.0 / np.sqrt(a)
        if li == len(SIZES) - 2:
            W = np.zeros((b, a))
            bb = np.zeros(b)
        else:
            W = rng.uniform(-lim, lim, size=(b, a))
            bb = rng.uniform(-lim, lim, size=b)
        parts += [W.ravel(), bb]
    return np.concatenate(parts)


def forward(theta, F):
    """z = f(F) for features F (n, 4); returns z (n,) and the activations."""
    layers = unpack(theta)
    acts = [F]
    h = F
    for li, (W, b) in enumerate(layers):
        pre = h @ W.T + b
        h = np.tanh(pre) if li < len(layers) - 1 else pre
        acts.append(h)
    return h[:, 0], acts


def bf16_round(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    a = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((a + 0x7FFF + ((a >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(theta, F):
    """The forward pass with the operands of the two 128 x 128 layers in BF16, as
    an inference on tensor cores with BF16 inputs takes it: W2, W3 and the
    activations that enter them (layers 1 and 2) rounded to BF16, W1 and W4
    rounded to BF16, products accumulated and everything else in FP64."""
    (W1, b1), (W2, b2), (W3, b3), (W4, b4) = unpack(theta)
    h1 = np.tanh(F @ bf16_round(W1).T + b1)
    h2 = np.tanh(bf16_round(h1) @ bf16_round(W2).T + b2)
    h3 = np.tanh(bf16_round(h2) @ bf16_round(W3).T + b3)
    return (h3 @ bf16_round(W4).T + b4)[:, 0]


def loss_and_grad(theta, F, zt, wt):
    """Weighted MSE sum(w (z - z*)^2) / sum(w) and its gradient (backprop)."""
    z, acts = forward(theta, F)
    layers = unpack(theta)
    sw = np.sum(wt)
    r = z - zt
    loss = np.sum(wt * r * r) / sw
    g = (2.0 * wt * r / sw)[:, None]          # dL/dz, (n, 1)
    grads = []
    for li in range(len(layers) - 1, -1, -1):
        W, b = layers[li]
        h_in = acts[li]
        gW = g.T @ h_in
        gb = g.sum(axis=0)
        grads.append((gW, gb))
        if li > 0:
            g = (g @ W) * (1.0 - acts[li] ** 2)   # through tanh of layer li-1's output
    grads.reverse()
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat


def adam_step(theta, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015); returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def shell_index(kin, ecut, nshell):
    """Shell of each plane wave: uniform bins of |q|^2/2 over [0, ecut]."""
    return np.minimum((kin / ecut * nshell).astype(np.int64), nshell - 1)


def features_and_labels(kin, ecut, nshell, M, R, E_err, d, shell):
    """Features (nb*nshell, 4), labels and weights for bands with residual
    rows R[i], errors E_err[i], distances d[i]; shells with no residual weight
    get weight 0."""
    nb = R.shape[0]
    MR = M[None, :] * R
    F = np.zeros((nb, nshell, 4))
    num = np.zeros((nb, nshell))
    den = np.zeros((nb, nshell))
    centres = (np.arange(nshell) + 0.5) / nshell
    r2 = np.abs(R) ** 2
    mean_all = r2.mean(axis=1)
    for s in range(nshell):
        sel = shell == s
        if not np.any(sel):
            continue
        ms = r2[:, sel].mean(axis=1)
        F[:, s, 0] = centres[s]
        F[:, s, 1] = np.log10(np.maximum(ms, 1e-300) / np.maximum(mean_all, 1e-300))
        F[:, s, 2] = d / 0.1
        F[:, s, 3] = np.log10(np.maximum(np.linalg.norm(R, axis=1), 1e-300)) / 10.0
        num[:, s] = np.sum(np.abs(E_err[:, sel]) ** 2, axis=1)
        den[:, s] = np.sum(np.abs(MR[:, sel]) ** 2, axis=1)
    ntot = num.sum(axis=1, keepdims=True)
    dtot = den.sum(axis=1, keepdims=True)
    a = np.where(ntot > 0, num / np.maximum(ntot, 1e-300), 0.0)
    wt = np.where(dtot > 0, den / np.maximum(dtot, 1e-300), 0.0)
    lo, hi = np.log(0.1), np.log(10.0)
    with np.errstate(divide="ignore"):
        z = np.where(a > 0, 0.5 * np.log(np.maximum(a, 1e-300) / np.maximum(wt, 1e-300)), lo)
    zt = np.where(wt > 0, np.clip(z, lo, hi), 0.0)
    F[:, :, 1] = np.maximum(F[:, :, 1], -30.0)
    return F.reshape(-1, 4), zt.ravel(), wt.ravel()
