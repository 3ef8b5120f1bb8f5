"""FP64 reference of the learned WENO weights (test infrastructure only).

Plain numpy, one sample at a time where it matters, written to be checked
against the definitions below by eye.  Only tests/ and the benchmark's CPU
legs may import it; it shares no code with the CUDA library.

Network (one per characteristic field s = 0..6, 1 379 parameters each):
    h1 = gelu(W1 x + b1)      W1: 32x6,  b1: 32
    h2 = gelu(W2 h1 + b2)     W2: 32x32, b2: 32
    z  = W3 h2 + b3           W3: 3x32,  b3: 3
    omega = softmax(z)
gelu(t) = t sigma(1.702 t) = t/2 (1 + tanh(0.851 t)), the sigmoid form of the
GELU (its inner argument is linear in t, so on the GPU it folds into the
layer's weights).
Flat parameter order per field: W1 (row-major), b1, W2, b2, W3, b3.

Input of one side of one interface: the six split characteristic fluxes of
the stencil cells i-2..i+3 (the '-' side reversed, so one network serves
both), normalised x = (v - mean v) / (max|v - mean v| + 1e-12).  omega_0 and
omega_2 replace the Jiang-Shu weights in phi_N (Sec. 2.1).

Training loss of one record (normalised candidate fluxes q_k of the three
third-order sub-stencils, normalised target T of the exact reconstruction):
    (sum_k omega_k q_k - T)^2 + lam * sum_k d_k log(d_k / omega_k),
d = (0.1, 0.6, 0.3).
"""
from __future__ import annotations

import numpy as np

D_LIN = np.array([0.1, 0.6, 0.3])
NIN, NH, NOUT = 6, 32, 3
NPARAM = NH * NIN + NH + NH * NH + NH + NOUT * NH + NOUT      # 1379
NFIELD = 7
K_GELU = 1.702          # gelu(t) = t sigma(K t)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + NH * NIN].reshape(NH, NIN); o += NH * NIN
    b1 = p[o:o + NH]; o += NH
    W2 = p[o:o + NH * NH].reshape(NH, NH); o += NH * NH
    b2 = p[o:o + NH]; o += NH
    W3 = p[o:o + NOUT * NH].reshape(NOUT, NH); o += NOUT * NH
    b3 = p[o:o + NOUT]; o += NOUT
    assert o == NPARAM
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])


def gelu(t):
    return 0.5 * t * (1.0 + np.tanh(0.5 * K_GELU * t))


def gelu_grad(t):
    sig = 0.5 * (1.0 + np.tanh(0.5 * K_GELU * t))         # sigma(K t)
    return sig + K_GELU * t * sig * (1.0 - sig)


def softmax(z):
    e = np.exp(z - z.max(axis=-1, keepdims=True))
    return e / e.sum(axis=-1, keepdims=True)


def forward(p, x):
    """omega for inputs x (..., 6); also the intermediate values."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    a1 = x @ W1.T + b1
    h1 = gelu(a1)
    a2 = h1 @ W2.T + b2
    h2 = gelu(a2)
    z = h2 @ W3.T + b3
    return softmax(z), (x, a1, h1, a2, h2, z)


def record_loss(omega, q, T, lam):
    y = (omega * q).sum(axis=-1)
    kl = (D_LIN * (np.log(D_LIN) - np.log(omega))).sum(axis=-1)
    return (y - T) ** 2 + lam * kl


def loss_and_grad(p, x, q, T, lam):
    """Mean loss over records and its gradient by hand-written backprop."""
    n = x.shape[0]
    W1, b1, W2, b2, W3, b3 = unpack(p)
    om, (x, a1, h1, a2, h2, z) = forward(p, x)
    y = (om * q).sum(axis=1)
    L = record_loss(om, q, T, lam).mean()
    # dL/domega (per record, mean over records)
    dom = (2.0 * (y - T))[:, None] * q - lam * D_LIN[None, :] / om
    dom /= n
    # softmax Jacobian: dz_j = om_j (dom_j - sum_k om_k dom_k)
    dz = om * (dom - (om * dom).sum(axis=1, keepdims=True))
    gW3 = dz.T @ h2
    gb3 = dz.sum(axis=0)
    dh2 = dz @ W3
    da2 = dh2 * gelu_grad(a2)
    gW2 = da2.T @ h1
    gb2 = da2.sum(axis=0)
    dh1 = da2 @ W2
    da1 = dh1 * gelu_grad(a1)
    gW1 = da1.T @ x
    gb1 = da1.sum(axis=0)
    return L, pack(gW1, gb1, gW2, gb2, gW3, gb3)


def normalise(v):
    v = np.asarray(v, dtype=np.float64)
    m = v.mean(axis=-1, keepdims=True)
    d = v - m
    return d / (np.abs(d).max(axis=-1, keepdims=True) + 1e-12)


def candidates(f5):
    """Third-order sub-stencil fluxes at i+1/2 from f_{i-2..i+2}."""
    f = np.asarray(f5, dtype=np.float64)
    q0 = (2 * f[..., 0] - 7 * f[..., 1] + 11 * f[..., 2]) / 6
    q1 = (-f[..., 1] + 5 * f[..., 2] + 2 * f[..., 3]) / 6
    q2 = (2 * f[..., 2] + 5 * f[..., 3] - f[..., 4]) / 6
    return np.stack([q0, q1, q2], axis=-1)


def detector(D4, kappa):
    """Jump detector on the four differences phi_N reads: fires when the
    largest exceeds kappa times the mean magnitude of the other three."""
    a = np.abs(np.asarray(D4, dtype=np.float64))
    mx = a.max(axis=-1)
    others = (a.sum(axis=-1) - mx) / 3.0
    return mx > kappa * others + 1e-300


def smoothness_indicators(D4):
    """IS_0..2 of the Jiang-Shu weights (Sec. 2.1) on the four differences
    phi_N reads, as printed there."""
    a, b, c, d = (float(v) for v in D4)
    return (13.0 * (a - b) ** 2 + 3.0 * (a - 3.0 * b) ** 2,
            13.0 * (b - c) ** 2 + 3.0 * (b + c) ** 2,
            13.0 * (c - d) ** 2 + 3.0 * (3.0 * c - d) ** 2)


def rough(D4, smooth, eps=1e-6):
    """The smoothness gate: the network's weights are used only where the
    smoothness indicators spread by more than the ratio `smooth`,
    (eps + max IS) > smooth (eps + min IS); returns (decision, relative
    distance from the threshold)."""
    IS = smoothness_indicators(D4)
    lhs, rhs = eps + max(IS), smooth * (eps + min(IS))
    return lhs > rhs, abs(lhs - rhs) / max(rhs, lhs, 1e-300)


def phi_n_weights(a, b, c, d, w0, w2):
    return w0 * (a - 2 * b + c) / 3.0 + (w2 - 0.5) * (b - 2 * c + d) / 6.0


def linear_params():
    """Parameters whose output is omega = d for every input (W3 = 0,
    b3 = log d): the learned flux then is the linear upwind-biased flux."""
    rng = np.random.default_rng(0)
    W1 = rng.standard_normal((NH, NIN)) * 0.3
    b1 = np.zeros(NH)
    W2 = rng.standard_normal((NH, NH)) * 0.2
    b2 = np.zeros(NH)
    W3 = np.zeros((NOUT, NH))
    b3 = np.log(D_LIN)
    return pack(W1, b1, W2, b2, W3, b3)


def interface_flux_learned(Us, gamma, params, kappa=4.0, pjump=0.5, margins=None, smooth=0.0):
    """Eq. FWENO flux at i+1/2 (rotated frame, stencil cells i-2..i+3, 6x8)
    with the Jiang-Shu weights replaced by the network's (params: 7 x 1379)
    wherever neither detector fires: the jump detector on the side's four
    differences, or a pressure ratio max p / min p > 1 + pjump over the six
    cells (then every field falls back to Jiang-Shu); and, with smooth > 0,
    only where the side's smoothness indicators spread by more than the
    ratio `smooth` (see `rough`).  Same steps as the
    oracle's orc_interface_flux otherwise.  With a list `margins`, the
    smallest relative distance of any detector input from its threshold is
    appended to it (how far the decisions are from flipping)."""
    import oracle as O

    Us = np.asarray(Us, dtype=np.float64).reshape(6, 8)
    params = np.asarray(params, dtype=np.float64).reshape(NFIELD, NPARAM)
    SYS = [0, 1, 2, 3, 5, 6, 7]
    W = np.array([O.cons_to_prim(u, gamma) for u in Us])
    F = np.array([O.flux_n(u, gamma) for u in Us])
    lk = np.empty((6, 7))
    for k in range(6):
        cf, ca, cs = O.wave_speeds(W[k], gamma)
        u = W[k][1]
        lk[k] = [u - cf, u - ca, u - cs, u, u + cs, u + ca, u + cf]
    lam, RU, LU, _ = O.eigen(0.5 * (W[2] + W[3]), gamma)
    p = W[:, 7]
    pfire = p.max() > (1.0 + pjump) * p.min()
    margin = abs(p.max() - (1.0 + pjump) * p.min()) / ((1.0 + pjump) * p.min())
    corr = np.empty(7)
    for s in range(7):
        alpha = max(abs(lam[s]), np.abs(lk[:, s]).max())
        w = np.array([LU[s] @ Us[k][SYS] for k in range(6)])
        g = np.array([LU[s] @ F[k][SYS] for k in range(6)])
        gp = 0.5 * (g + alpha * w)
        gm = 0.5 * (g - alpha * w)
        dp = np.diff(gp)
        dm = np.diff(gm)
        # '+' side: D_{i-3/2..i+3/2}; '-' side: D_{i+5/2..i-1/2}
        Dp = dp[0:4]
        Dm = dm[[4, 3, 2, 1]]
        out = []
        for D, v in ((Dp, gp), (Dm, gm[::-1])):
            a = np.abs(D)
            thr = kappa * (a.sum() - a.max()) / 3.0
            margin = min(margin, abs(a.max() - thr) / (thr + 1e-300))
            use_net, m_s = rough(D, smooth)
            if smooth > 0.0:
                margin = min(margin, m_s)
            if pfire or detector(D, kappa) or not use_net:
                out.append(O.phi_n(*D))
            else:
                om, _ = forward(params[s], normalise(v))
                out.append(phi_n_weights(*D, om[0], om[2]))
        corr[s] = -out[0] + out[1]
    Fh = np.empty(8)
    for f in range(7):
        q = SYS[f]
        Fh[q] = (-F[1][q] + 7 * F[2][q] + 7 * F[3][q] - F[4][q]) / 12.0 + RU[f] @ corr
    Fh[4] = 0.0
    if margins is not None:
        margins.append(margin)
    return Fh
