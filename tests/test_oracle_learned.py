"""Pins of the learned-correction network oracle: the convolution against
scipy.signal.correlate2d, the transfers against the multigrid oracle's P and
R, the absence of biases (positive homogeneity) and the shapes."""
import math

import numpy as np
import pytest
import scipy.signal as ss

import oracle as O
from oracle import learned_oracle as LO


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


def test_network_has_no_bias_and_maps_shapes():
    tr = LO.Transfers(15)
    ps = LO.init_params(4, seed=2)
    assert [p.shape for p in ps][0] == (3, 3, 5, 4) and ps[-1].shape == (3, 3, 4, 2)
    x = np.random.default_rng(3).standard_normal((5, 15, 15))
    y = LO.forward(ps, x, tr)
    assert y.shape == (2, 15, 15)
    np.testing.assert_allclose(LO.forward(ps, 2.5 * x, tr), 2.5 * y, rtol=1e-12, atol=1e-14)


def test_correction_scales_with_the_residual_and_lives_on_the_coarse_grid():
    m = 31
    rng = np.random.default_rng(5)
    log_a = rng.standard_normal((m + 2, m + 2)) * 0.3
    lc = LO.LearnedCorrection(m, log_a, 1 / 16)
    assert lc.mc == 15 and lc.tr.sizes == [15, 7, 3, 1]
    ps = LO.init_params(4, seed=4)
    r = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    e1 = lc(ps, r, 0.4 - 0.3j)
    e2 = lc(ps, 3.0 * r, 0.4 - 0.3j)
    np.testing.assert_allclose(e2, 3.0 * e1, rtol=1e-12)
    # the correction is a prolongation of a coarse field
    assert np.allclose(e1.reshape(-1), lc.P0 @ np.linalg.lstsq(lc.P0.toarray(), e1.reshape(-1), rcond=None)[0])
    # coarse log a samples the nodes (2i+2, 2j+2)
    assert abs(lc.la_c[0, 0] - (log_a[2, 2] - log_a.mean())) < 1e-15


def _varcoef_case(m=15, seed=11):
    rng = np.random.default_rng(seed)
    log_a = 0.5 * rng.standard_normal((m + 2, m + 2))
    K = O.fd_stiffness_varcoef(np.exp(log_a))
    return log_a, K


def test_correction_step_is_exact_with_an_exact_network():
    """With e = B^{-1} res in place of the network, x + e is the exact solution,
    the smoothing sweep leaves it there and the minimal-residual step keeps it."""
    import scipy.sparse.linalg as spla
    m, tau, lam = 15, 1 / 16, 0.3 - 0.2j
    log_a, K = _varcoef_case(m)
    A = (lam * sp_identity(m * m) + tau * K).tocsc()
    lc = LO.LearnedCorrection(m, log_a, tau)
    rng = np.random.default_rng(12)
    b = rng.standard_normal(m * m) + 1j * rng.standard_normal(m * m)
    x = rng.standard_normal(m * m) + 1j * rng.standard_normal(m * m)
    exact = lambda res, lam_: spla.spsolve(A, res.reshape(-1))
    xn, q = LO.correct(None, lc, A, b, x, lam, net=exact)
    np.testing.assert_allclose(xn, spla.spsolve(A, b), rtol=1e-11, atol=1e-12)
    assert q < 1e-10


def test_correction_step_minimises_the_residual_along_its_direction():
    """The judged step is the minimiser over complex alpha (checked on a grid of
    alphas around it), so the residual never grows, whatever the network."""
    m, tau, lam = 15, 1 / 16, 0.05 + 0.01j
    log_a, K = _varcoef_case(m, 13)
    A = (lam * sp_identity(m * m) + tau * K).tocsr()
    lc = LO.LearnedCorrection(m, log_a, tau)
    rng = np.random.default_rng(14)
    b = rng.standard_normal(m * m) + 1j * rng.standard_normal(m * m)
    x = np.zeros(m * m, complex)
    ps = LO.init_params(4, seed=15)
    xn, q = LO.correct(ps, lc, A, b, x, lam)
    assert q <= 1.0 + 1e-14
    # the direction of the step, rebuilt from its definition
    e = lc(ps, b.reshape(m, m), lam).reshape(-1)
    d = e + 0.8 * (b - A @ e) / A.diagonal()
    alpha = np.vdot(d, xn - x) / np.vdot(d, d)
    np.testing.assert_allclose(xn, x + alpha * d, rtol=1e-12, atol=1e-14)
    f = lambda al: np.linalg.norm(b - A @ (x + al * d))
    best = f(alpha)
    assert abs(best / np.linalg.norm(b) - q) < 1e-12
    for da in (1e-3, -1e-3, 1e-3j, -1e-3j, 0.05, -0.05j):
        assert f(alpha + da * abs(alpha)) >= best
    # a hostile network (the negated exact correction) is neutralised, not followed
    import scipy.sparse.linalg as spla
    bad = lambda res, lam_: -10.0 * spla.spsolve(A.tocsc(), res.reshape(-1))
    _, qb = LO.correct(None, lc, A, b, x, lam, net=bad)
    assert qb <= 1.0 + 1e-14


def test_correction_step_solves_a_diagonal_system_exactly():
    """For a diagonal B and a zero network, d = omega D^{-1} res, B d = omega res,
    so alpha = 1/omega and the step lands on the exact solution for any omega."""
    m = 15
    rng = np.random.default_rng(16)
    dg = rng.uniform(0.5, 3.0, m * m) + 1j * rng.uniform(-1, 1, m * m)
    A = sp_diags(dg)
    lc = LO.LearnedCorrection(m, np.zeros((m + 2, m + 2)), 1 / 16)
    b = rng.standard_normal(m * m) + 1j * rng.standard_normal(m * m)
    zero = lambda res, lam_: np.zeros(m * m, complex)
    for omega in (0.8, 0.5, 1.3):
        xn, q = LO.correct(None, lc, A.tocsr(), b, np.zeros(m * m, complex), 0.5, omega, net=zero)
        np.testing.assert_allclose(xn, b / dg, rtol=1e-13)


def test_learned_pinv_with_an_exact_network_is_the_exact_inverse():
    """With exact shifted solves in place of the network the learned route is
    P_eps^{-1} itself: this pins the forward-sign pairing of lambda'_k, the
    half spectrum and the complex-to-real inverse against banded LU."""
    import scipy.sparse.linalg as spla
    m, N, eps = 15, 8, 0.1
    tau = 1.0 / N
    log_a, K = _varcoef_case(m, 17)
    h = O.MGHierarchy(K, m)
    lc = LO.LearnedCorrection(m, log_a, tau)
    y = np.random.default_rng(18).standard_normal((N, m, m))
    exact = lambda res, lam_: spla.spsolve((lam_ * sp_identity(m * m) + tau * K).tocsc(),
                                           res.reshape(-1))
    ratios = []
    z = LO.apply_Pinv_learned(y, h, lc, None, tau, eps, net=exact, ratios=ratios)
    ref = O.apply_Pinv_lu(y, sp_identity(m * m), K, tau, eps)
    np.testing.assert_allclose(z, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
    assert len(ratios) == N // 2 + 1 and max(ratios) < 1e-9
    # lambda'_k are the conjugates of the eigenvalues of Sec. 4 (k <= N/2)
    np.testing.assert_allclose(LO.forward_sign_eigs(N, eps), np.conj(O.eps_circulant_eigs(N, eps)[:N // 2 + 1]),
                               atol=1e-15)


def test_learned_pinv_never_does_worse_than_the_vcycle():
    """Per frequency the judged correction leaves a residual no larger than the
    V-cycle's (random, untrained weights)."""
    m, N, eps = 15, 8, 0.05
    tau = 1.0 / N
    log_a, K = _varcoef_case(m, 19)
    h = O.MGHierarchy(K, m)
    lc = LO.LearnedCorrection(m, log_a, tau)
    y = np.random.default_rng(20).standard_normal((N, m, m))
    ratios = []
    LO.apply_Pinv_learned(y, h, lc, LO.init_params(4, seed=21), tau, eps, ratios=ratios)
    assert all(0.0 <= q <= 1.0 + 1e-12 for q in ratios)


def sp_identity(n):
    import scipy.sparse as sp
    return sp.identity(n, format="csr")


def sp_diags(d):
    import scipy.sparse as sp
    return sp.diags(d)


def test_loss_is_the_mean_of_the_per_sample_relative_errors():
    """Zero weights give e = 0, so every sample's ||e - e*||^2 / ||e*||^2 is 1;
    with targets 2e and -e the per-sample values are 1/4 and 4, and the loss is
    their mean, 2.125 (a ratio of sums, or a norm that is not squared, gives
    another number)."""
    m = 15
    rng = np.random.default_rng(30)
    lc = LO.LearnedCorrection(m, 0.3 * rng.standard_normal((m + 2, m + 2)), 1 / 16)
    ps = LO.init_params(4, seed=31)
    zero = [np.zeros_like(w) for w in ps]
    r1 = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    r2 = 5.0 * (rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m)))
    l1, l2 = 0.3 - 0.2j, 1.1 + 0.4j
    e1, e2 = lc(ps, r1, l1), lc(ps, r2, l2)
    assert np.abs(e1).max() > 0 and np.abs(e2).max() > 0
    assert LO.loss(zero, [(r1, l1, e1), (r2, l2, 3.0 * e2)], lc) == pytest.approx(1.0, abs=1e-15)
    assert LO.loss(ps, [(r1, l1, e1)], lc) == pytest.approx(0.0, abs=1e-28)
    assert LO.loss(ps, [(r1, l1, 2.0 * e1)], lc) == pytest.approx(0.25, rel=1e-13)
    assert LO.loss(ps, [(r1, l1, 2.0 * e1), (r2, l2, -e2)], lc) == pytest.approx(2.125, rel=1e-13)


@pytest.mark.parametrize("a", [0.5, 2.0])
def test_output_scale_is_the_inverse_shifted_operator_on_its_smoothest_mode(a):
    """For a constant coefficient, the smallest eigenvalue of the 5-point K(a)
    (shift-invert Lanczos on the assembled matrix, no formula) is a mu_min,
    and |lambda + tau a mu_min|^-1 is the size of B_k^{-1} on that mode.
    output_scale uses the continuum value mu_min -> 2 pi^2, which agrees to
    O(h^2): here pi^2 h^2 / 12 < 2.5e-4 of mu_min."""
    import scipy.sparse.linalg as spla
    m, N, eps = 63, 32, 0.05
    tau = 1.0 / N
    K = O.fd_stiffness_varcoef(np.full((m + 2, m + 2), a))
    mu_min = float(spla.eigsh(K.tocsc(), k=1, sigma=0.0, which="LM", return_eigenvectors=False)[0])
    assert mu_min == pytest.approx(a * 2.0 * math.pi ** 2, rel=2.5e-4)
    for lam in LO.forward_sign_eigs(N, eps):
        ref = 1.0 / abs(lam + tau * mu_min)
        assert LO.output_scale(lam, tau, a) == pytest.approx(ref, rel=2.5e-4)
    # the route takes a_mean over the node values: constant a gives a itself
    lc = LO.LearnedCorrection(m, np.full((m + 2, m + 2), math.log(a)), tau)
    assert lc.a_mean == pytest.approx(a, rel=1e-14)
