"""FP64 NumPy oracle of the learned correction used as an inner preconditioner
for the shifted systems B_k = lambda_k I + tau K(a) of Sec. 4 (variable
coefficient, where the sine transform no longer applies).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The correction is applied after one multigrid V-cycle to the residual r it
left.  Two properties are built in, whatever the weights:

(i) It is LINEAR in r: for a fixed coefficient a and frequency k it is a
fixed complex-linear map, so P_eps^{-1} stays a fixed linear operator and
the outer Krylov method keeps its acceleration.

(ii) Its dependence on the frequency is ANALYTIC in lambda_k.  Step 3
multiplies time step j by eps^{-j/N}.  Write an inner solve's frequency
dependence as a series in z = eps^{1/N} e^{-2 pi i k/N} (lambda_k = 1 - z
for backward Euler).  Non-negative powers of z act causally in time and
come back unamplified; a negative power, which any dependence on conj(z)
brings in (on Re lambda, Im lambda or |lambda| separately, or on
conj(r)), links the first time steps to the last ones and comes back
amplified by up to 1/eps.  The exact shifted inverse, the V-cycle and the
Jacobi sweep are rational in lambda, with poles at lambda = -(positive),
outside the circle |z| = eps^{1/N}, so they have no such part.  The
correction is therefore a sum of such terms, with fixed poles and residue
maps that do not depend on k (the partial-fraction form of
(lambda M + tau K)^{-1} = sum over modes of phi phi^T / (lambda + tau mu)):

    ec_k = sum_j w_j(lambda_k) Nc_j(x),   w_j(lambda) = sigma_j / (lambda + sigma_j)

with poles sigma_j = sigma_0 rho^j, j = 0..7, log-spaced from the smoothest
mode's shift sigma_0 = tau a_mean 2 pi^2 to the largest eigenvalue
2 tau a_mean (m + 1)^2 of the 5-point operator on the grid of spacing 2h.

The residue maps are REAL operators, applied to the real and the imaginary
part of the residual alike: Nc_j(x) = N_j(Re x) + i N_j(Im x), with N one
network of one real plane on the grid of spacing 2h (the multigrid's level
1), 4 levels, and the multigrid's own bilinear prolongation P and
full-weighting restriction R = P^T/4 as its down- and up-sampling:

    rc = R_0 r;   x = rc / sigma_0;   for v = Re x and v = Im x (1 channel):
    h0 = conv(v, W0) G0;           s0 = conv(h0, W1) G1
    s1 = conv(R s0, W2) G2;        s2 = conv(R s1, W3) G3;   s3 = conv(R s2, W4) G4
    u2 = conv(P s3 + s2, W5) G5;   u1 = conv(P u2 + s1, W6) G6
    u0 = conv(P u1 + s0, W7) G7;   N(v) = conv(u0, W8)       (8 channels)
    Nc_j(x) = N_j(Re x) + i N_j(Im x),   e = P_0 ec

Every conv is a 3 x 3 correlation with zero padding and no bias; a weight
tensor W has shape [3][3][C_in][C_out].  Real residue operators make the
correction complex-linear and give it the symmetry of the exact inverse,
ec(conj lambda, conj r) = conj ec(lambda, r).  The route evaluates only
k = 0..N/2 and takes the conjugates for the other half of the spectrum, so
without that symmetry the correction would jump between a map and its
conjugate at k = 0 and k = N/2: a dependence on k that is not analytic,
see (ii).  (A network mixing the two planes with free weights is only
real-linear, N(x) = M x + M' conj(x), with M' a dependence on conj(r).)
The gates depend on the coefficient alone and multiply each channel of a
layer's output point by point:

    G_i = 1 + tanh(conv(relu(conv(la_l, A1_i)), A2_i))

with la_l the centred log a on the layer's level l (levels of the gated
layers: 0 0 1 2 3 2 1 0).  They let the correction adapt to a while staying
linear in r and independent of k.

Training target: the exact coarse-grid correction ec* = B_{k,1}^{-1} R_0 r,
B_{k,1} = lambda_k M_1 + tau K_1 the Galerkin operator of level 1; loss =
mean over samples of ||ec - ec*||^2 / ||ec*||^2.  After the correction one
damped-Jacobi sweep follows (the post-smoothing of a prolonged correction),
and the step from the V-cycle's iterate is scaled by one complex alpha, the
same for every frequency (a per-frequency step would again depend on k
non-analytically), fixed by one calibration apply: the minimal-residual
step over all frequencies on a fixed right-hand side.  Then the multigrid
judges the result: power iterations on the error operator I - M_k A_k of
the V-cycle alone and of the corrected preconditioner estimate their
spectral radii, and unless the corrected one's largest radius over k is the
smaller, alpha = 0, which keeps the V-cycle's result (the multigrid is the
fallback).
"""
from __future__ import annotations

import math

import numpy as np

from .bec_oracle import mg_prolongation

N_LAYERS = 9
N_GATED = 8
N_POLES = 8
C_IN = 1
C_OUT = N_POLES
NA = 8            # hidden channels of an a-gate
GATE_LEVEL = (0, 0, 1, 2, 3, 2, 1, 0)


def layer_shapes(C: int):
    """(C_in, C_out) of the 9 convolutions of the residual path."""
    return [(C_IN, C), (C, C), (C, C), (C, C), (C, C), (C, C), (C, C), (C, C), (C, C_OUT)]


def param_shapes(C: int):
    """Shapes of every parameter array in the order of the flat weight vector:
    W0..W8, A1_0..A1_7, A2_0..A2_7."""
    out = [(3, 3, ci, co) for ci, co in layer_shapes(C)]
    out += [(3, 3, 1, NA)] * N_GATED + [(3, 3, NA, C)] * N_GATED
    return out


def num_params(C: int) -> int:
    return sum(int(np.prod(s)) for s in param_shapes(C))


def unflatten(w, C: int) -> dict:
    """The parameter dict {"W", "A1", "A2"} of a flat vector."""
    arrs, off = [], 0
    for s in param_shapes(C):
        n = int(np.prod(s))
        arrs.append(np.asarray(w[off:off + n], dtype=np.float64).reshape(s))
        off += n
    g = N_GATED
    return {"W": arrs[:9], "A1": arrs[9:9 + g], "A2": arrs[9 + g:9 + 2 * g]}


def flatten(params: dict) -> np.ndarray:
    parts = params["W"] + params["A1"] + params["A2"]
    return np.concatenate([np.asarray(p, dtype=np.float64).reshape(-1) for p in parts])


def init_params(C: int, seed: int = 0, gate_scale: float = 0.0) -> dict:
    """Seeded initialisation: W normal with std sqrt(1 / (9 C_in)) (the last
    layer scaled by 0.1), A1 std 0.3; A2 normal with std gate_scale (0: every
    gate starts at 1)."""
    rng = np.random.default_rng(seed)
    W = []
    for i, (ci, co) in enumerate(layer_shapes(C)):
        std = math.sqrt(1.0 / (9 * ci)) * (0.1 if i == N_LAYERS - 1 else 1.0)
        W.append(rng.standard_normal((3, 3, ci, co)) * std)
    A1 = [rng.standard_normal((3, 3, 1, NA)) * 0.3 for _ in range(N_GATED)]
    A2 = [rng.standard_normal((3, 3, NA, C)) * gate_scale for _ in range(N_GATED)]
    return {"W": W, "A1": A1, "A2": A2}


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


def coarse_log_a(log_a_nodes: np.ndarray, mc: int) -> np.ndarray:
    """log a at the nodes of the grid of spacing 2h (fine node (2i+2, 2j+2) of
    the (m+2)^2 node array), centred by the mean over all fine nodes."""
    la = log_a_nodes[2:2 + 2 * mc:2, 2:2 + 2 * mc:2]
    return la - float(np.mean(log_a_nodes))


def level_log_a(la0: np.ndarray, tr: Transfers):
    """The centred log a on the network's 4 levels: level 0 as given, level
    l + 1 the full-weighting restriction of level l."""
    out = [la0]
    for l in range(len(tr.sizes) - 1):
        out.append(tr.restrict(l, out[-1][None])[0])
    return out


def a_gates(params: dict, la_levels) -> list:
    """GA_i = 1 + tanh(conv(relu(conv(la_l, A1_i)), A2_i)), [C][m_l][m_l]."""
    out = []
    for i in range(N_GATED):
        la = la_levels[GATE_LEVEL[i]][None]
        out.append(1.0 + np.tanh(conv3x3(relu(conv3x3(la, params["A1"][i])), params["A2"][i])))
    return out


def pole_shifts(tau: float, a_mean: float, m: int) -> np.ndarray:
    """sigma_j = sigma_0 rho^j, j = 0..N_POLES-1: sigma_0 = tau a_mean 2 pi^2
    (the shift of the smoothest mode) up to sigma_top = 2 tau a_mean (m+1)^2
    (tau a_mean 8 / (2h)^2, the largest eigenvalue of the 5-point operator on
    the grid of spacing 2h, h = 1 / (m+1))."""
    s0 = tau * a_mean * 2.0 * math.pi ** 2
    top = 2.0 * tau * a_mean * (m + 1) ** 2
    return s0 * (top / s0) ** (np.arange(N_POLES) / (N_POLES - 1))


def pole_weights(lam: complex, sig: np.ndarray) -> np.ndarray:
    """w_j = sigma_j / (lambda + sigma_j)."""
    return sig / (lam + sig)


def forward(params: dict, x: np.ndarray, GA: list, tr: Transfers) -> np.ndarray:
    """The residual path of the module docstring on one real input plane
    [1][m][m], with the gates GA (list of [C][m_l][m_l]); returns the
    N_POLES output planes N_j."""
    W = params["W"]
    G = GA
    h0 = conv3x3(x, W[0]) * G[0]
    s0 = conv3x3(h0, W[1]) * G[1]
    s1 = conv3x3(tr.restrict(0, s0), W[2]) * G[2]
    s2 = conv3x3(tr.restrict(1, s1), W[3]) * G[3]
    s3 = conv3x3(tr.restrict(2, s2), W[4]) * G[4]
    u2 = conv3x3(tr.prolong(2, s3) + s2, W[5]) * G[5]
    u1 = conv3x3(tr.prolong(1, u2) + s1, W[6]) * G[6]
    u0 = conv3x3(tr.prolong(0, u1) + s0, W[7]) * G[7]
    return conv3x3(u0, W[8])


class LearnedCorrection:
    """Fine grid m, network grid (m-1)/2 with 4 levels."""

    def __init__(self, m: int, log_a_nodes: np.ndarray, tau: float):
        self.m = m
        self.mc = (m - 1) // 2
        self.P0 = mg_prolongation(self.mc)
        self.R0 = (self.P0.T / 4.0).tocsr()
        self.tr = Transfers(self.mc)
        self.la_c = coarse_log_a(log_a_nodes, self.mc)
        self.la_levels = level_log_a(self.la_c, self.tr)
        self.a_mean = float(np.mean(np.exp(log_a_nodes)))
        self.tau = tau
        self.sig = pole_shifts(tau, self.a_mean, m)

    def residues(self, params: dict, rc: np.ndarray) -> np.ndarray:
        """Nc_j(x) = N_j(Re x) + i N_j(Im x), x = rc / sigma_0, for j =
        0..N_POLES-1 ([N_POLES][mc][mc] complex) from the coarse residual rc."""
        GA = a_gates(params, self.la_levels)
        x = rc / self.sig[0]
        return forward(params, x.real[None], GA, self.tr) + 1j * forward(params, x.imag[None], GA, self.tr)

    def coarse(self, params: dict, r: np.ndarray, lam: complex) -> np.ndarray:
        """ec (complex [mc][mc]) for a fine complex residual r [m][m]."""
        mc = self.mc
        rc = (self.R0 @ r.reshape(-1)).reshape(mc, mc)
        w = pole_weights(lam, self.sig)
        return np.tensordot(w, self.residues(params, rc), axes=1)

    def __call__(self, params: dict, r: np.ndarray, lam: complex) -> np.ndarray:
        """e = P_0 ec on the fine grid [m][m]."""
        ec = self.coarse(params, r, lam)
        return (self.P0 @ ec.reshape(-1)).reshape(self.m, self.m)


def coarse_target(h, lam: complex, tau: float, r: np.ndarray) -> np.ndarray:
    """The exact coarse-grid correction B_{k,1}^{-1} R_0 r (level 1 of the
    multigrid hierarchy h), [mc][mc] complex."""
    import scipy.sparse.linalg as spla
    mc = h.sizes[1]
    rc = h.R[0] @ r.reshape(-1)
    return spla.spsolve(h.op(1, lam, tau).tocsc(), rc).reshape(mc, mc)


def loss(params: dict, samples, lc: LearnedCorrection) -> float:
    """Mean over samples (r, lam, ec*) of ||ec - ec*||^2 / ||ec*||^2 on the
    coarse grid."""
    tot = 0.0
    for r, lam, et in samples:
        ec = lc.coarse(params, r, lam)
        tot += float(np.sum(np.abs(ec - et) ** 2) / np.sum(np.abs(et) ** 2))
    return tot / len(samples)


def correct(params, lc: LearnedCorrection, A, b: np.ndarray, x: np.ndarray, lam: complex,
            alpha: complex, omega: float = 0.8, net=None):
    """The corrected iterate of x (the V-cycle's) for A x = b (A = B_k on the
    fine grid, vectors flattened): x1 = x + e with e the correction of the
    residual b - A x (``net(res, lam)`` in place of the network when given),
    x2 = x1 + omega D^{-1} (b - A x1) (one damped-Jacobi sweep), and the
    result x + alpha (x2 - x).  Returns (x_new, x2)."""
    m = lc.m
    res = b - A @ x
    e = (net(res, lam) if net is not None else lc(params, res.reshape(m, m), lam)).reshape(-1)
    x1 = x + e
    x2 = x1 + omega * (b - A @ x1) / A.diagonal()
    return x + alpha * (x2 - x), x2


def minimal_residual_step(A, b: np.ndarray, x: np.ndarray, x2: np.ndarray):
    """alpha = <A d, res> / <A d, A d>, d = x2 - x, res = b - A x (<u, v> = u^H v):
    the complex step that minimises ||b - A (x + alpha d)||; 0 when A d = 0 or
    the sums are not finite.  Returns (alpha, ||res_new|| / ||res||)."""
    res = b - A @ x
    Ad = A @ (x2 - x)
    dd = float(np.vdot(Ad, Ad).real)
    cr = complex(np.vdot(Ad, res))
    ok = dd > 0 and math.isfinite(dd) and math.isfinite(cr.real) and math.isfinite(cr.imag)
    alpha = cr / dd if ok else 0.0
    rr = float(np.vdot(res, res).real)
    after = max(rr - abs(cr) ** 2 / dd, 0.0) if ok else rr
    return alpha, (math.sqrt(after / rr) if rr > 0 else 0.0)


MASK64 = (1 << 64) - 1


def splitmix64(z: np.ndarray) -> np.ndarray:
    """The SplitMix64 output function (Steele, Lea and Flood, 2014) on uint64."""
    z = (z + np.uint64(0x9E3779B97F4A7C15)) & np.uint64(MASK64)
    z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & np.uint64(MASK64)
    z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & np.uint64(MASK64)
    return z ^ (z >> np.uint64(31))


CALIBRATION_KEY = 0xCA11B8A7E5EED001


def calibration_rhs(K: int, J: int) -> np.ndarray:
    """The fixed right-hand side of the calibration apply, [K][J] complex:
    value i of the interleaved (re, im) array is (t >> 40) 2^-23 - 1 with
    t = splitmix64(key ^ splitmix64(i)), uniform in [-1, 1) and exactly
    representable in FP32 and FP64."""
    with np.errstate(over="ignore"):
        i = np.arange(2 * K * J, dtype=np.uint64)
        t = splitmix64(np.uint64(CALIBRATION_KEY) ^ splitmix64(i))
    v = (t >> np.uint64(40)).astype(np.float64) * 2.0 ** -23 - 1.0
    v = v.reshape(K, J, 2)
    return v[..., 0] + 1j * v[..., 1]


def forward_sign_eigs(N: int, eps: float) -> np.ndarray:
    """lambda'_k = 1 - eps^{1/N} e^{-2 pi i k / N}, k = 0..N/2: the eigenvalues of
    the backward-Euler epsilon-circulant paired with a forward-sign (e^{-})
    DFT over time (the conjugates of Sec. 4's lambda_k)."""
    k = np.arange(N // 2 + 1)
    return 1.0 - eps ** (1.0 / N) * np.exp(-2j * np.pi * k / N)


JUDGE_ITERS = 10


def judge_radii(h, lc: LearnedCorrection, params, tau: float, eps: float, N: int, alpha,
                omega: float = 0.8, nu1: int = 1, nu2: int = 1, net=None, iters: int = JUDGE_ITERS):
    """The judge's estimates of the spectral radius of E_k = I - M_k A_k per
    frequency k = 0..N/2: `iters` power iterations v <- E_k v / ||E_k v|| from
    the calibration right-hand side normalised, the last ||E_k v||; once for
    M_k the V-cycle alone and once for the corrected preconditioner (V-cycle,
    correction, sweep, step alpha).  Returns (rho_vcycle, rho_corrected)."""
    from .bec_oracle import mg_vcycle
    lam = forward_sign_eigs(N, eps)
    m = lc.m
    B = calibration_rhs(N // 2 + 1, m * m)
    out = np.zeros((2, N // 2 + 1))
    for k in range(N // 2 + 1):
        A = h.op(0, lam[k], tau)
        for arm in (0, 1):
            v = B[k] / np.linalg.norm(B[k])
            for _ in range(iters):
                r = -(A @ v)
                z = mg_vcycle(h, lam[k], tau, r, omega, nu1, nu2)
                if arm == 1:
                    z, _ = correct(params, lc, A, r, z, lam[k], alpha, omega, net)
                v = v + z
                rho = float(np.linalg.norm(v))
                if rho > 0.0:
                    v = v / rho
            out[arm, k] = rho
    return out[0], out[1]


def calibrate(h, lc: LearnedCorrection, params, tau: float, eps: float, N: int,
              omega: float = 0.8, nu1: int = 1, nu2: int = 1, net=None, judge: bool = True):
    """The one step alpha for all frequencies from one calibration apply: the
    V-cycle and the correction on calibration_rhs at every k = 0..N/2, then
    the minimal-residual step of the stacked system, alpha = sum_k <A_k d_k,
    res_k> / sum_k ||A_k d_k||^2 (0 when the sums vanish or are not finite).
    With judge, the multigrid then judges the corrected preconditioner
    (judge_radii): unless its largest radius estimate over k is below the
    V-cycle's, alpha = 0.  Returns (alpha, ratios, radii): ratios[k] =
    ||res_k - alpha A_k d_k|| / ||res_k|| for the minimal-residual alpha,
    radii = judge_radii's pair (None without judge)."""
    from .bec_oracle import mg_vcycle
    lam = forward_sign_eigs(N, eps)
    m = lc.m
    B = calibration_rhs(N // 2 + 1, m * m)
    pairs = []
    for k in range(N // 2 + 1):
        A = h.op(0, lam[k], tau)
        x = mg_vcycle(h, lam[k], tau, B[k], omega, nu1, nu2)
        _, x2 = correct(params, lc, A, B[k], x, lam[k], 0.0, omega, net)
        pairs.append((B[k] - A @ x, A @ (x2 - x)))
    dd = sum(float(np.vdot(Ad, Ad).real) for _, Ad in pairs)
    cr = sum(complex(np.vdot(Ad, res)) for res, Ad in pairs)
    ok = dd > 0 and math.isfinite(dd) and math.isfinite(cr.real) and math.isfinite(cr.imag)
    alpha = cr / dd if ok else 0.0
    ratios = [float(np.linalg.norm(res - alpha * Ad) / np.linalg.norm(res)) for res, Ad in pairs]
    radii = None
    if judge:
        radii = judge_radii(h, lc, params, tau, eps, N, alpha, omega, nu1, nu2, net)
        if not radii[1].max() < radii[0].max():
            alpha = 0.0
    return alpha, np.array(ratios), radii


def apply_Pinv_learned(y: np.ndarray, h, lc: LearnedCorrection, params, tau: float, eps: float,
                       alpha, omega: float = 0.8, nu1: int = 1, nu2: int = 1, net=None):
    """P_eps^{-1} y by Sec. 4's three steps with Step 2 done, per frequency, by
    one V-cycle (``mg_vcycle``) and then the correction with the fixed step
    alpha (``correct``).  The route is defined on the half spectrum of a
    forward-sign real DFT (k = 0..N/2 with lambda'_k of
    ``forward_sign_eigs``); the other frequencies are the conjugates (a real
    result), and the imaginary parts at k = 0 and N/2 are dropped, as by a
    complex-to-real inverse DFT.  BDF1 only.  ``net`` replaces the network as
    in ``correct``."""
    from .bec_oracle import eps_scaling, mg_vcycle
    N = y.shape[0]
    Y = y.reshape(N, -1).astype(np.float64)
    d = eps_scaling(N, eps)
    yt = np.fft.rfft(d[:, None] * Y, axis=0)                            # Step 1
    lam = forward_sign_eigs(N, eps)
    zt = np.empty_like(yt)
    for k in range(N // 2 + 1):                                          # Step 2
        A = h.op(0, lam[k], tau)
        x = mg_vcycle(h, lam[k], tau, yt[k], omega, nu1, nu2)
        zt[k], _ = correct(params, lc, A, yt[k], x, lam[k], alpha, omega, net)
    z = np.fft.irfft(zt, n=N, axis=0) / d[:, None]                      # Step 3
    return z.reshape(y.shape)
