"""Pins of the learned-correction oracle (oracle/learned_oracle.py): the
convolution against scipy.signal.correlate2d, the transfers against the
multigrid oracle's P and R, the gates against loops written from their
definition, complex-linearity in the residual and the conjugation symmetry
of real residue operators, analyticity in the shift (Cauchy-Riemann), the
poles against Lanczos eigenvalues and the sign of their weights, the
coarse-grid target against a dense solve, the loss's normalisation, the step
and calibration rules, the calibration generator against SplitMix64's
published first output, and the whole learned P_eps^{-1} against banded LU
with an exact correction."""
import math

import numpy as np
import pytest
import scipy.signal as ss
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
from oracle import learned_oracle as LO


def sp_identity(n):
    return sp.identity(n, format="csr")


def _varcoef_case(m=15, seed=11):
    rng = np.random.default_rng(seed)
    log_a = 0.5 * rng.standard_normal((m + 2, m + 2))
    K = O.fd_stiffness_varcoef(np.exp(log_a))
    return log_a, K


def test_conv3x3_is_a_zero_padded_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 9, 9))
    W = rng.standard_normal((3, 3, 3, 4))
    out = LO.conv3x3(x, W)
    for co in range(4):
        ref = sum(ss.correlate2d(x[ci], W[:, :, ci, co], mode="same", boundary="fill")
                  for ci in range(3))
        np.testing.assert_allclose(out[co], ref, atol=1e-12)


def test_transfers_match_the_multigrid_operators():
    tr = LO.Transfers(31)
    assert tr.sizes == [31, 15, 7, 3]
    h = O.MGHierarchy(O.fd_stiffness(2, 31), 31)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 31, 31))
    np.testing.assert_allclose(tr.restrict(0, x)[1].reshape(-1), h.R[0] @ x[1].reshape(-1), atol=1e-14)
    y = rng.standard_normal((2, 3, 3))
    np.testing.assert_allclose(tr.prolong(2, y)[0].reshape(-1), h.P[2] @ y[0].reshape(-1), atol=1e-14)


def test_parameter_layout():
    C = 4
    ps = LO.init_params(C, seed=2, gate_scale=0.3)
    w = LO.flatten(ps)
    assert w.size == LO.num_params(C)
    back = LO.unflatten(w, C)
    for key in ("W", "A1", "A2"):
        for a, b in zip(ps[key], back[key]):
            np.testing.assert_array_equal(a, b)
    assert back["W"][0].shape == (3, 3, 1, C) and back["W"][8].shape == (3, 3, C, LO.N_POLES)
    assert back["A2"][7].shape == (3, 3, LO.NA, C) and len(back) == 3


def _conv_loops(x, W):
    """3 x 3 zero-padded correlation by loops over every output point."""
    ci_n, m, _ = x.shape
    co_n = W.shape[3]
    out = np.zeros((co_n, m, m))
    for co in range(co_n):
        for yy in range(m):
            for xx in range(m):
                s = 0.0
                for ci in range(ci_n):
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            if 0 <= yy + dy < m and 0 <= xx + dx < m:
                                s += W[dy + 1, dx + 1, ci, co] * x[ci, yy + dy, xx + dx]
                out[co, yy, xx] = s
    return out


def test_gates_follow_their_definition():
    """GA_i against loops written from the definition, on a 7 x 7 network
    grid; and all gates are exactly 1 when A2 = 0."""
    C = 3
    ps = LO.init_params(C, seed=3, gate_scale=0.4)
    tr = LO.Transfers(7)
    rng = np.random.default_rng(4)
    la = LO.level_log_a(rng.standard_normal((7, 7)) * 0.7, tr)
    GA = LO.a_gates(ps, la)
    for i in (0, 2, 4):
        lv = LO.GATE_LEVEL[i]
        z = _conv_loops(np.maximum(_conv_loops(la[lv][None], ps["A1"][i]), 0.0), ps["A2"][i])
        np.testing.assert_allclose(GA[i], 1.0 + np.tanh(z), rtol=1e-13, atol=1e-14)
    flat = LO.init_params(C, seed=3, gate_scale=0.0)
    assert all(np.all(g == 1.0) for g in LO.a_gates(flat, la))
    # the level fields are restrictions of level 0
    np.testing.assert_allclose(la[1], tr.restrict(0, la[0][None])[0])


def test_correction_is_linear_in_the_residual_and_lives_on_the_coarse_grid():
    m = 31
    rng = np.random.default_rng(5)
    log_a = rng.standard_normal((m + 2, m + 2)) * 0.3
    lc = LO.LearnedCorrection(m, log_a, 1 / 16)
    assert lc.mc == 15 and lc.tr.sizes == [15, 7, 3, 1]
    ps = LO.init_params(4, seed=4, gate_scale=0.5)
    lam = 0.4 - 0.3j
    r1 = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    r2 = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    e1, e2 = lc(ps, r1, lam), lc(ps, r2, lam)
    e12 = lc(ps, 2.5 * r1 - 0.75 * r2, lam)
    np.testing.assert_allclose(e12, 2.5 * e1 - 0.75 * e2, rtol=1e-11, atol=1e-13 * np.abs(e12).max())
    # complex-linear, not only real-linear
    ez = lc(ps, (0.6 - 1.3j) * r1, lam)
    np.testing.assert_allclose(ez, (0.6 - 1.3j) * e1, rtol=1e-11, atol=1e-13 * np.abs(ez).max())
    # the correction is a prolongation of a coarse field
    ec = lc.coarse(ps, r1, lam)
    np.testing.assert_allclose(e1.reshape(-1), lc.P0 @ ec.reshape(-1), atol=1e-14)
    # coarse log a samples the nodes (2i+2, 2j+2), centred
    assert abs(lc.la_c[0, 0] - (log_a[2, 2] - log_a.mean())) < 1e-15
    # no last layer: no correction
    z = dict(ps, W=ps["W"][:8] + [np.zeros_like(ps["W"][8])])
    assert np.all(lc(z, r1, lam) == 0.0)


def test_residues_are_real_operators():
    """Nc_j(x) = N_j(Re x) + i N_j(Im x): a real residual gives real residues,
    the residues of conj(r) are the conjugates, and the correction has the
    symmetry of the exact inverse, ec(conj lambda, conj r) = conj ec(lambda,
    r), which the half-spectrum evaluation relies on; ec is the
    pole-weighted sum of the residues."""
    m = 31
    rng = np.random.default_rng(8)
    lc = LO.LearnedCorrection(m, rng.standard_normal((m + 2, m + 2)) * 0.3, 1 / 16)
    ps = LO.init_params(4, seed=2, gate_scale=0.4)
    r = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    rc = (lc.R0 @ r.reshape(-1)).reshape(lc.mc, lc.mc)
    nc = lc.residues(ps, rc)
    assert nc.shape == (LO.N_POLES, lc.mc, lc.mc) and np.abs(nc).max() > 1e-3
    assert np.all(lc.residues(ps, rc.real + 0j).imag == 0.0)
    np.testing.assert_allclose(lc.residues(ps, np.conj(rc)), np.conj(nc), rtol=1e-13,
                               atol=1e-15 * np.abs(nc).max())
    lam = 0.5 - 0.2j
    ec = lc.coarse(ps, r, lam)
    np.testing.assert_allclose(lc.coarse(ps, np.conj(r), np.conj(lam)), np.conj(ec), rtol=1e-13,
                               atol=1e-15 * np.abs(ec).max())
    w = lc.sig / (lam + lc.sig)
    np.testing.assert_allclose(ec, sum(w[j] * nc[j] for j in range(LO.N_POLES)), rtol=1e-12,
                               atol=1e-14 * np.abs(ec).max())
    # one forward pass per plane: the real part's residues come from Re x alone
    y = LO.forward(ps, (rc.real / lc.sig[0])[None], LO.a_gates(ps, lc.la_levels), lc.tr)
    np.testing.assert_allclose(nc.real, y, rtol=1e-13, atol=1e-15 * np.abs(y).max())


def test_correction_is_analytic_in_the_shift():
    """ec(lambda) satisfies the Cauchy-Riemann equations: its difference
    quotients along a real and along an imaginary step agree (d ec / d
    conj(lambda) = 0), at points of the backward-Euler circle and off it,
    with gates away from 1.  A dependence on Re lambda, Im lambda or
    |lambda| separately fails this by O(1)."""
    m = 15
    rng = np.random.default_rng(22)
    lc = LO.LearnedCorrection(m, rng.standard_normal((m + 2, m + 2)) * 0.4, 1 / 32)
    ps = LO.init_params(4, seed=23, gate_scale=0.4)
    r = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    d = 1e-5
    for lam in (0.02 - 0.01j, 0.6 + 0.9j, 1.9 - 0.1j, 0.3 + 0.0j):
        dre = (lc.coarse(ps, r, lam + d) - lc.coarse(ps, r, lam - d)) / (2 * d)
        dim = (lc.coarse(ps, r, lam + 1j * d) - lc.coarse(ps, r, lam - 1j * d)) / (2j * d)
        assert np.abs(dre).max() > 1e-6
        assert np.abs(dre - dim).max() <= 1e-6 * np.abs(dre).max(), lam


def test_pole_weights_are_bounded_on_the_right_half_plane():
    """w_j = sigma_j / (lambda + sigma_j) with sigma_j > 0: |w_j| < 1 where
    Re lambda > 0 (every lambda_k of backward Euler, 1 - eps^{1/N}
    e^{-2 pi i k/N}), w_j -> 1 as lambda -> 0 and -> 0 as |lambda| grows (a
    pole on the wrong side, sigma_j / (lambda - sigma_j), breaks the bound
    near lambda = sigma_j)."""
    sig = LO.pole_shifts(1 / 64, 1.3, 127)
    assert np.all(sig > 0) and np.all(np.diff(sig) > 0)
    lam = np.concatenate([LO.forward_sign_eigs(64, 1 / 16), LO.forward_sign_eigs(256, 1 / 32),
                          sig[:3]])
    for l in lam:
        w = LO.pole_weights(l, sig)
        assert np.all(np.abs(w) < 1.0)
    np.testing.assert_allclose(LO.pole_weights(1e-12, sig), 1.0, rtol=1e-9)
    assert np.all(np.abs(LO.pole_weights(1e9, sig)) < 1e-3)


def test_coarse_target_solves_the_galerkin_system():
    m, tau, lam = 31, 1 / 16, 0.2 + 0.5j
    log_a, K = _varcoef_case(m, 6)
    h = O.MGHierarchy(K, m)
    r = np.random.default_rng(7).standard_normal((m, m)) + 1j
    et = LO.coarse_target(h, lam, tau, r)
    B1 = (lam * h.M[1] + tau * h.K[1]).toarray()
    np.testing.assert_allclose(B1 @ et.reshape(-1), h.R[0] @ r.reshape(-1), rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(et.reshape(-1), np.linalg.solve(B1, h.R[0] @ r.reshape(-1)),
                               rtol=1e-10)


def test_loss_is_the_mean_of_the_per_sample_relative_errors():
    """Zero output (last layer 0) gives 1 per sample; with targets 2 ec and
    -ec the per-sample values are 1/4 and 4, and the loss is their mean,
    2.125 (a ratio of sums, or a norm that is not squared, gives another
    number)."""
    m = 15
    rng = np.random.default_rng(30)
    lc = LO.LearnedCorrection(m, 0.3 * rng.standard_normal((m + 2, m + 2)), 1 / 16)
    ps = LO.init_params(4, seed=31, gate_scale=0.2)
    zero = dict(ps, W=ps["W"][:8] + [np.zeros_like(ps["W"][8])])
    r1 = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    r2 = 5.0 * (rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m)))
    l1, l2 = 0.3 - 0.2j, 1.1 + 0.4j
    e1, e2 = lc.coarse(ps, r1, l1), lc.coarse(ps, r2, l2)
    assert np.abs(e1).max() > 0 and np.abs(e2).max() > 0
    assert LO.loss(zero, [(r1, l1, e1), (r2, l2, 3.0 * e2)], lc) == pytest.approx(1.0, abs=1e-15)
    assert LO.loss(ps, [(r1, l1, e1)], lc) == pytest.approx(0.0, abs=1e-28)
    assert LO.loss(ps, [(r1, l1, 2.0 * e1)], lc) == pytest.approx(0.25, rel=1e-13)
    assert LO.loss(ps, [(r1, l1, 2.0 * e1), (r2, l2, -e2)], lc) == pytest.approx(2.125, rel=1e-13)


@pytest.mark.parametrize("a", [0.5, 2.0])
def test_poles_span_the_spectrum_of_the_coarse_operator(a):
    """For a constant coefficient the poles run from the shift of the
    smoothest mode to the largest eigenvalue on the grid of spacing 2h, both
    found by Lanczos on assembled matrices (no formula): sigma_0 = tau a 2 pi^2
    against tau mu_min of the fine 5-point K(a) (the continuum value, O(h^2)
    off: pi^2 h^2 / 12 < 2.5e-4), and sigma_top = 2 tau a (m+1)^2 against
    tau mu_max of the 5-point K(a) on the 2h grid (1 - mu_max / (8 a / (2h)^2)
    = sin^2(pi h) = O(h^2), 2.4e-3 here); the poles are geometric."""
    m, N = 63, 32
    tau = 1.0 / N
    K = O.fd_stiffness_varcoef(np.full((m + 2, m + 2), a))
    mu_min = float(spla.eigsh(K.tocsc(), k=1, sigma=0.0, which="LM", return_eigenvectors=False)[0])
    mc = (m - 1) // 2
    Kc = O.fd_stiffness_varcoef(np.full((mc + 2, mc + 2), a))
    mu_max = float(spla.eigsh(Kc.tocsc(), k=1, which="LA", return_eigenvectors=False)[0])
    lc = LO.LearnedCorrection(m, np.full((m + 2, m + 2), math.log(a)), tau)
    assert lc.a_mean == pytest.approx(a, rel=1e-14)
    sig = lc.sig
    assert sig.size == LO.N_POLES
    assert sig[0] == pytest.approx(tau * mu_min, rel=2.5e-4)
    assert tau * mu_max <= sig[-1] <= tau * mu_max * (1 + 3e-3)
    np.testing.assert_allclose(sig[1:] / sig[:-1], sig[1] / sig[0], rtol=1e-12)


def test_correction_with_an_exact_network_lands_on_the_solution():
    """With e = B^{-1} res in place of the network, x + e is the exact solution,
    the smoothing sweep leaves it there, alpha = 1 keeps it, and the
    calibration's minimal-residual step is 1 with a zero residual ratio."""
    m, tau, lam = 15, 1 / 16, 0.3 - 0.2j
    log_a, K = _varcoef_case(m)
    A = (lam * sp_identity(m * m) + tau * K).tocsc()
    lc = LO.LearnedCorrection(m, log_a, tau)
    rng = np.random.default_rng(12)
    b = rng.standard_normal(m * m) + 1j * rng.standard_normal(m * m)
    x = rng.standard_normal(m * m) + 1j * rng.standard_normal(m * m)
    exact = lambda res, lam_: spla.spsolve(A, res.reshape(-1))
    xn, x2 = LO.correct(None, lc, A, b, x, lam, 1.0, net=exact)
    sol = spla.spsolve(A, b)
    np.testing.assert_allclose(xn, sol, rtol=1e-11, atol=1e-12)
    alpha, q = LO.minimal_residual_step(A, b, x, x2)
    assert abs(alpha - 1.0) < 1e-10 and q < 1e-10


def test_minimal_residual_step_minimises_along_its_direction():
    m, tau, lam = 15, 1 / 16, 0.05 + 0.01j
    _, K = _varcoef_case(m, 13)
    A = (lam * sp_identity(m * m) + tau * K).tocsr()
    rng = np.random.default_rng(14)
    b = rng.standard_normal(m * m) + 1j * rng.standard_normal(m * m)
    x = rng.standard_normal(m * m) + 1j * rng.standard_normal(m * m)
    x2 = x + rng.standard_normal(m * m) + 1j * rng.standard_normal(m * m)
    alpha, q = LO.minimal_residual_step(A, b, x, x2)
    f = lambda al: np.linalg.norm(b - A @ (x + al * (x2 - x)))
    best = f(alpha)
    assert abs(best / np.linalg.norm(b - A @ x) - q) < 1e-12
    for da in (1e-3, -1e-3, 1e-3j, -1e-3j, 0.05, -0.05j):
        assert f(alpha + da * max(abs(alpha), 1e-3)) >= best
    # no direction: the fallback alpha = 0
    assert LO.minimal_residual_step(A, b, x, x)[0] == 0.0


def test_zero_network_step_solves_a_diagonal_system_exactly():
    """For a diagonal B and a zero network, x2 - x = omega D^{-1} res and
    B (x2 - x) = omega res, so the minimal-residual step is 1/omega and the
    step lands on the exact solution for any omega."""
    m = 15
    rng = np.random.default_rng(16)
    dg = rng.uniform(0.5, 3.0, m * m) + 1j * rng.uniform(-1, 1, m * m)
    A = sp.diags(dg).tocsr()
    lc = LO.LearnedCorrection(m, np.zeros((m + 2, m + 2)), 1 / 16)
    b = rng.standard_normal(m * m) + 1j * rng.standard_normal(m * m)
    zero = lambda res, lam_: np.zeros(m * m, complex)
    x0 = np.zeros(m * m, complex)
    for omega in (0.8, 0.5, 1.3):
        _, x2 = LO.correct(None, lc, A, b, x0, 0.5, 0.0, omega, net=zero)
        alpha, _ = LO.minimal_residual_step(A, b, x0, x2)
        assert alpha == pytest.approx(1.0 / omega, rel=1e-13)
        xn, _ = LO.correct(None, lc, A, b, x0, 0.5, alpha, omega, net=zero)
        np.testing.assert_allclose(xn, b / dg, rtol=1e-13)


def test_calibration_generator():
    """SplitMix64's published first output for state 0 (0xe220a8397b1dcdaf),
    the map to [-1, 1) with values exact in FP32, determinism, and the
    interleaved (re, im) order of the generated array."""
    out = LO.splitmix64(np.array([0], dtype=np.uint64))
    assert int(out[0]) == 0xE220A8397B1DCDAF
    v = LO.calibration_rhs(3, 50)
    assert v.shape == (3, 50)
    parts = np.stack([v.real, v.imag])
    assert parts.min() >= -1.0 and parts.max() < 1.0
    assert np.all(parts.astype(np.float32).astype(np.float64) == parts)
    np.testing.assert_array_equal(v, LO.calibration_rhs(3, 50))
    # element (k, q): indices 2 (k J + q) and 2 (k J + q) + 1, from Python integers
    M = (1 << 64) - 1

    def mix(z):
        z = (z + 0x9E3779B97F4A7C15) & M
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        return z ^ (z >> 31)
    k, q = 2, 17
    i = 2 * (k * 50 + q)
    re = (mix(LO.CALIBRATION_KEY ^ mix(i)) >> 40) * 2.0 ** -23 - 1.0
    im = (mix(LO.CALIBRATION_KEY ^ mix(i + 1)) >> 40) * 2.0 ** -23 - 1.0
    assert v[k, q] == re + 1j * im


def test_learned_pinv_with_an_exact_network_is_the_exact_inverse():
    """With exact shifted solves in place of the network and alpha = 1 the
    learned route is P_eps^{-1} itself: this pins the forward-sign pairing of
    lambda'_k, the half spectrum and the complex-to-real inverse against
    banded LU; the calibration then finds alpha = 1."""
    m, N, eps = 15, 8, 0.1
    tau = 1.0 / N
    log_a, K = _varcoef_case(m, 17)
    h = O.MGHierarchy(K, m)
    lc = LO.LearnedCorrection(m, log_a, tau)
    y = np.random.default_rng(18).standard_normal((N, m, m))
    exact = lambda res, lam_: spla.spsolve((lam_ * sp_identity(m * m) + tau * K).tocsc(),
                                           res.reshape(-1))
    alpha, ratios, (rho_v, rho_c) = LO.calibrate(h, lc, None, tau, eps, N, net=exact)
    assert abs(alpha - 1.0) < 1e-10 and np.all(ratios < 1e-9)
    # the judge keeps it: I - M B vanishes for the exact inverse
    assert np.all(rho_c < 1e-9) and np.all((rho_v > 0.01) & (rho_v < 1.0))
    z = LO.apply_Pinv_learned(y, h, lc, None, tau, eps, alpha, net=exact)
    ref = O.apply_Pinv_lu(y, sp_identity(m * m), K, tau, eps)
    np.testing.assert_allclose(z, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
    np.testing.assert_allclose(LO.forward_sign_eigs(N, eps), np.conj(O.eps_circulant_eigs(N, eps)[:N // 2 + 1]),
                               atol=1e-15)


def test_learned_pinv_with_zero_steps_is_the_multigrid_route():
    """alpha = 0 keeps the V-cycle's iterates: the route is then the
    multigrid P_eps^{-1} (the fallback); with the calibrated step it is
    linear in y."""
    m, N, eps = 15, 8, 0.05
    tau = 1.0 / N
    log_a, K = _varcoef_case(m, 19)
    h = O.MGHierarchy(K, m)
    lc = LO.LearnedCorrection(m, log_a, tau)
    ps = LO.init_params(4, seed=21, gate_scale=0.3)
    rng = np.random.default_rng(20)
    y1, y2 = rng.standard_normal((2, N, m, m))
    z0 = LO.apply_Pinv_learned(y1, h, lc, ps, tau, eps, 0.0)
    # the multigrid route on the same half spectrum
    d = O.eps_scaling(N, eps)
    yt = np.fft.rfft(d[:, None] * y1.reshape(N, -1), axis=0)
    lam = LO.forward_sign_eigs(N, eps)
    zt = np.array([O.mg_vcycle(h, lam[k], tau, yt[k]) for k in range(N // 2 + 1)])
    ref = (np.fft.irfft(zt, n=N, axis=0) / d[:, None]).reshape(y1.shape)
    np.testing.assert_allclose(z0, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())
    alpha, _, radii = LO.calibrate(h, lc, ps, tau, eps, N, judge=False)
    assert alpha != 0.0 and radii is None
    za = LO.apply_Pinv_learned(y1, h, lc, ps, tau, eps, alpha)
    zb = LO.apply_Pinv_learned(y2, h, lc, ps, tau, eps, alpha)
    zab = LO.apply_Pinv_learned(0.5 * y1 - 2.0 * y2, h, lc, ps, tau, eps, alpha)
    np.testing.assert_allclose(zab, 0.5 * za - 2.0 * zb, rtol=1e-10, atol=1e-12 * np.abs(zab).max())


def test_judge_estimates_the_spectral_radius_and_rejects_a_harmful_correction():
    """The judge's 10 power iterations against the spectral radius of the
    dense error operator E_k = I - M_k A_k (assembled column by column,
    numpy eigenvalues) for the V-cycle at every frequency of a small case.
    A correction that is exact except on the three smoothest eigenvectors of
    K, where it is -10 times the exact one, multiplies the V-cycle's error
    there by 11.  One step alpha cannot repair it (the minimal-residual
    alpha stays near 1, fitted to the other modes), so its radius exceeds
    the V-cycle's and it is rejected: alpha = 0, and the learned P_eps^{-1}
    is the multigrid route's.  (3 times the exact correction everywhere is
    repaired by alpha near 1/3 and kept.)"""
    m, N, eps = 15, 8, 0.1
    tau = 1.0 / N
    log_a, K = _varcoef_case(m, 25)
    h = O.MGHierarchy(K, m)
    lc = LO.LearnedCorrection(m, log_a, tau)
    lam = LO.forward_sign_eigs(N, eps)
    exact = lambda res, lam_: spla.spsolve((lam_ * sp_identity(m * m) + tau * K).tocsc(),
                                           res.reshape(-1))
    rho_v, _ = LO.judge_radii(h, lc, None, tau, eps, N, 1.0, net=exact)
    for k in range(N // 2 + 1):
        A = h.op(0, lam[k], tau)
        E = np.zeros((m * m, m * m), complex)
        for j in range(m * m):
            e = np.zeros(m * m, complex)
            e[j] = 1.0
            E[:, j] = e - O.mg_vcycle(h, lam[k], tau, A @ e)
        rho = float(np.abs(np.linalg.eigvals(E)).max())
        assert abs(rho_v[k] - rho) <= 0.15 * rho, (k, rho_v[k], rho)
    over = lambda res, lam_: 3.0 * exact(res, lam_)
    alpha3, _, (rv, rc) = LO.calibrate(h, lc, None, tau, eps, N, net=over)
    assert abs(alpha3 - 1.0 / 3.0) < 0.2 and rc.max() < rv.max()
    _, Q = np.linalg.eigh(K.toarray())
    Q = Q[:, :3]
    flip = lambda res, lam_: (lambda e: e - 11.0 * Q @ (Q.T @ e))(exact(res, lam_))
    alpha, _, (rv, rc) = LO.calibrate(h, lc, None, tau, eps, N, net=flip)
    assert alpha == 0.0 and rc.max() > rv.max()
    y = np.random.default_rng(26).standard_normal((N, m, m))
    z = LO.apply_Pinv_learned(y, h, lc, None, tau, eps, alpha, net=flip)
    d = O.eps_scaling(N, eps)
    yt = np.fft.rfft(d[:, None] * y.reshape(N, -1), axis=0)
    zt = np.array([O.mg_vcycle(h, lam[k], tau, yt[k]) for k in range(N // 2 + 1)])
    ref = (np.fft.irfft(zt, n=N, axis=0) / d[:, None]).reshape(y.shape)
    np.testing.assert_allclose(z, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())
