"""FP64 NumPy oracle of the learned correction network used as an inner
preconditioner for the shifted systems B_k = lambda_k I + tau K(a) of Sec. 4
(variable coefficient, where the sine transform no longer applies).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The network is a 4-level convolutional correction with the multigrid's own
grid hierarchy (m_{l+1} = (m_l - 1)/2, bilinear prolongation P and
full-weighting restriction R = P^T/4 as its fixed up- and down-sampling):

    level 0:  h0 = relu(conv(x, W0)); s0 = relu(conv(h0, W1))
    level 1:  s1 = relu(conv(R s0, W2))
    level 2:  s2 = relu(conv(R s1, W3))
    level 3:  s3 = relu(conv(R s2, W4))
    up:       u2 = relu(conv(P s3 + s2, W5))
              u1 = relu(conv(P u2 + s1, W6))
              u0 = relu(conv(P u1 + s0, W7))
    output:   y = conv(u0, W8)           (2 channels: real and imaginary part)

Every conv is a 3 x 3 correlation with zero padding and no bias; a weight
tensor W has shape [3][3][C_in][C_out] and out[co](y, x) = sum_{dy,dx,ci}
W[dy+1][dx+1][ci][co] in[ci](y+dy, x+dx).  Activations are [C][m][m].

The network runs one level below the fine grid.  For a fine residual r
(the residual left by one V-cycle), r_c = R_0 r is restricted to the grid
of spacing 2h.  The input channels (5) are r_c / s (real and imaginary
parts), log a at the coarse nodes (centred), and the real and imaginary
parts of lambda_k as constant planes; s is the root-mean-square of r_c.  The
correction is e = P_0 (s c_k (y_0 + i y_1)) with c_k = 1 / |lambda_k +
tau a_mean 2 pi^2|, the size of B_k^{-1} on the smoothest mode.  Training
minimises the relative error ||e - e*||^2 / ||e*||^2 to pairs
(r, e* = B_k^{-1} r) that the multigrid generates.
"""
from __future__ import annotations

import math

import numpy as np

from .bec_oracle import mg_prolongation

N_LAYERS = 9
C_IN = 5
C_OUT = 2


def layer_shapes(C: int):
    """(C_in, C_out) of the 9 convolutions."""
    return [(C_IN, C), (C, C), (C, C), (C, C), (C, C), (C, C), (C, C), (C, C), (C, C_OUT)]


def init_params(C: int, seed: int = 0):
    """He-normal initialisation, last layer scaled down."""
    rng = np.random.default_rng(seed)
    ps = []
    for i, (ci, co) in enumerate(layer_shapes(C)):
        std = math.sqrt(2.0 / (9 * ci)) * (0.1 if i == N_LAYERS - 1 else 1.0)
        ps.append(rng.standard_normal((3, 3, ci, co)) * std)
    return ps


def conv3x3(x: np.ndarray, W: np.ndarray) -> np.ndarray:
    """out[co] = sum_{dy,dx,ci} W[dy+1, dx+1, ci, co] x[ci](y+dy, x+dx), zero padding."""
    C_in, m, _ = x.shape
    xp = np.zeros((C_in, m + 2, m + 2))
    xp[:, 1:-1, 1:-1] = x
    out = np.zeros((W.shape[3], m, m))
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            patch = xp[:, 1 + dy:1 + dy + m, 1 + dx:1 + dx + m]           # [ci][m][m]
            out += np.einsum("io,iyx->oyx", W[dy + 1, dx + 1], patch)
    return out


def relu(x):
    return np.maximum(x, 0.0)


class Transfers:
    """Per-level bilinear prolongation and full-weighting restriction."""

    def __init__(self, m: int, levels: int = 4):
        self.sizes = [m]
        for _ in range(levels - 1):
            self.sizes.append((self.sizes[-1] - 1) // 2)
        self.P = [mg_prolongation(self.sizes[l + 1]) for l in range(levels - 1)]
        self.R = [(P.T / 4.0).tocsr() for P in self.P]

    def restrict(self, l: int, x: np.ndarray) -> np.ndarray:
        mc = self.sizes[l + 1]
        return np.stack([(self.R[l] @ c.reshape(-1)).reshape(mc, mc) for c in x])

    def prolong(self, l: int, x: np.ndarray) -> np.ndarray:
        mf = self.sizes[l]
        return np.stack([(self.P[l] @ c.reshape(-1)).reshape(mf, mf) for c in x])


def forward(params, x: np.ndarray, tr: Transfers) -> np.ndarray:
    """The network of the module docstring on one input [5][m][m]."""
    W = params
    h0 = relu(conv3x3(x, W[0]))
    s0 = relu(conv3x3(h0, W[1]))
    s1 = relu(conv3x3(tr.restrict(0, s0), W[2]))
    s2 = relu(conv3x3(tr.restrict(1, s1), W[3]))
    s3 = relu(conv3x3(tr.restrict(2, s2), W[4]))
    u2 = relu(conv3x3(tr.prolong(2, s3) + s2, W[5]))
    u1 = relu(conv3x3(tr.prolong(1, u2) + s1, W[6]))
    u0 = relu(conv3x3(tr.prolong(0, u1) + s0, W[7]))
    return conv3x3(u0, W[8])


def coarse_log_a(log_a_nodes: np.ndarray, mc: int) -> np.ndarray:
    """log a at the nodes of the grid of spacing 2h (fine node (2i+2, 2j+2) of
    the (m+2)^2 node array), centred by the mean over all fine nodes."""
    la = log_a_nodes[2:2 + 2 * mc:2, 2:2 + 2 * mc:2]
    return la - float(np.mean(log_a_nodes))


def features(rc: np.ndarray, la_c: np.ndarray, lam: complex):
    """Input planes and the residual scale s for one coarse complex residual."""
    s = math.sqrt(float(np.mean(np.abs(rc) ** 2)))
    s = s if s > 0 else 1.0
    mc = rc.shape[0]
    x = np.stack([rc.real / s, rc.imag / s, la_c, np.full((mc, mc), lam.real),
                  np.full((mc, mc), lam.imag)])
    return x, s


def output_scale(lam: complex, tau: float, a_mean: float) -> float:
    return 1.0 / abs(lam + tau * a_mean * 2.0 * math.pi ** 2)


class LearnedCorrection:
    """Fine grid m, network grid (m-1)/2 with 4 levels."""

    def __init__(self, m: int, log_a_nodes: np.ndarray, tau: float):
        self.m = m
        self.mc = (m - 1) // 2
        self.P0 = mg_prolongation(self.mc)
        self.R0 = (self.P0.T / 4.0).tocsr()
        self.tr = Transfers(self.mc)
        self.la_c = coarse_log_a(log_a_nodes, self.mc)
        self.a_mean = float(np.mean(np.exp(log_a_nodes)))
        self.tau = tau

    def __call__(self, params, r: np.ndarray, lam: complex) -> np.ndarray:
        """e = P_0 (s c_k (y_0 + i y_1)) for a fine complex residual r [m][m]."""
        mc = self.mc
        rc = (self.R0 @ r.reshape(-1)).reshape(mc, mc)
        x, s = features(rc, self.la_c, lam)
        y = forward(params, x, self.tr)
        c = s * output_scale(lam, self.tau, self.a_mean)
        ec = c * (y[0] + 1j * y[1])
        return (self.P0 @ ec.reshape(-1)).reshape(self.m, self.m)


def loss(params, samples, lc: LearnedCorrection) -> float:
    """Mean over samples (r, lam, e*) of ||e - e*||^2 / ||e*||^2."""
    tot = 0.0
    for r, lam, et in samples:
        e = lc(params, r, lam)
        tot += float(np.sum(np.abs(e - et) ** 2) / np.sum(np.abs(et) ** 2))
    return tot / len(samples)


def correct(params, lc: LearnedCorrection, A, b: np.ndarray, x: np.ndarray, lam: complex,
            omega: float = 0.8, net=None):
    """One judged learned correction of an iterate x of A x = b (A = B_k on the
    fine grid, vectors flattened), in three steps:
      1. x1 = x + e, e = the network's correction of the residual b - A x
         (``net(res, lam)`` in place of the network when given);
      2. x2 = x1 + omega D^{-1} (b - A x1): one damped-Jacobi sweep, the
         post-smoothing that follows any prolonged coarse-grid correction in
         multigrid (Sec. 4's multigrid, Example 2's one post-smoothing step),
         removing what the bilinear P_0 adds at high frequencies;
      3. x <- x + alpha (x2 - x) with the complex alpha that minimises
         ||b - A (x + alpha d)||, d = x2 - x:
         alpha = <A d, res> / <A d, A d>, <u, v> = u^H v.
    Step 3 is the judge: the residual norm never grows, and alpha = 0 (the
    V-cycle's iterate kept) when A d = 0.  Returns (x_new, ||res_new|| /
    ||res||)."""
    m = lc.m
    res = b - A @ x
    e = (net(res, lam) if net is not None else lc(params, res.reshape(m, m), lam)).reshape(-1)
    x1 = x + e
    x2 = x1 + omega * (b - A @ x1) / A.diagonal()
    d = x2 - x
    Ad = A @ d
    dd = float(np.vdot(Ad, Ad).real)
    alpha = complex(np.vdot(Ad, res)) / dd if dd > 0 else 0.0
    xn = x + alpha * d
    rn = float(np.linalg.norm(b - A @ xn))
    r0 = float(np.linalg.norm(res))
    return xn, (rn / r0 if r0 > 0 else 0.0)


def forward_sign_eigs(N: int, eps: float) -> np.ndarray:
    """lambda'_k = 1 - eps^{1/N} e^{-2 pi i k / N}, k = 0..N/2: the eigenvalues of
    the backward-Euler epsilon-circulant paired with a forward-sign (e^{-})
    DFT over time (the conjugates of Sec. 4's lambda_k)."""
    k = np.arange(N // 2 + 1)
    return 1.0 - eps ** (1.0 / N) * np.exp(-2j * np.pi * k / N)


def apply_Pinv_learned(y: np.ndarray, h, lc: LearnedCorrection, params, tau: float, eps: float,
                       omega: float = 0.8, nu1: int = 1, nu2: int = 1, ratios=None, net=None):
    """P_eps^{-1} y by Sec. 4's three steps with Step 2 done, per frequency,
    by one V-cycle (``mg_vcycle``) and then the judged learned correction
    (``correct``).  The network is not conjugation-equivariant, so the route is
    defined on the half spectrum of a forward-sign real DFT (k = 0..N/2 with
    lambda'_k of ``forward_sign_eigs``); the other frequencies are the
    conjugates (a real result), and the imaginary parts at k = 0 and N/2 are
    dropped, as by a complex-to-real inverse DFT.  BDF1 only.  When given,
    ``ratios`` receives ||res_new|| / ||res|| per frequency, and ``net``
    replaces the network as in ``correct``."""
    from .bec_oracle import eps_scaling, mg_vcycle
    N = y.shape[0]
    Y = y.reshape(N, -1).astype(np.float64)
    d = eps_scaling(N, eps)
    yt = np.fft.rfft(d[:, None] * Y, axis=0)                            # Step 1
    lam = forward_sign_eigs(N, eps)
    zt = np.empty_like(yt)
    A0 = [h.op(0, lk, tau) for lk in lam]
    for k in range(N // 2 + 1):                                          # Step 2
        x = mg_vcycle(h, lam[k], tau, yt[k], omega, nu1, nu2)
        zt[k], q = correct(params, lc, A0[k], yt[k], x, lam[k], omega, net)
        if ratios is not None:
            ratios.append(q)
    z = np.fft.irfft(zt, n=N, axis=0) / d[:, None]                      # Step 3
    return z.reshape(y.shape)
