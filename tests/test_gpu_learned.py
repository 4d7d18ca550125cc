"""The learned correction on the GPU (through the C ABI) against the NumPy
oracle of the same network (oracle/learned_oracle.py): loss and weight
gradients (checked by central finite differences of the oracle), the whole
learned P_eps^{-1} (V-cycle, linear gated correction, smoothing sweep,
calibrated step) element by element, BF16 against FP32 activations,
training by the GPU's own kernels, and what the trained correction gains
over the multigrid preconditioner without it (the A/B/C test).

Weights are seeded in the tests (oracle.init_params) and set on the GPU; no
oracle input is read back from the GPU.

Tolerance of the P_eps^{-1} parity: the multigrid route's bound 16 u
(log2(N n^2) + 8 L) / eps plus the network's 9 convolutions, each output a
sum of 9 C_in products whose rounding grows like sqrt(9 C_in) u (the
probabilistic bound of Higham and Mary for sums of random-sign terms):
16 u (log2(N n^2) + 8 L + 9 sqrt(9 C)) / eps."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from oracle import learned_oracle as LO
from workloads import grf_log_coefficient, heat_case_2d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2002_01108_gb300 import build
    build.build()


def small_problem(net_fp32, C=4, m=31, N=8, eps=0.1, seed=5):
    from paper_2002_01108_gb300 import Problem
    a = O.node_coefficient(grf_log_coefficient(seed=seed, m=m))
    p = Problem(2, m, N, route="learned", precision="fp32", a_nodes=a, net_channels=C,
                net_fp32=net_fp32, flexible=True)
    p.set_eps(eps)
    return p, a


def seeded_weights(C, seed, gate_scale):
    ps = LO.init_params(C, seed=seed, gate_scale=gate_scale)
    return ps, LO.flatten(ps).astype(np.float32)


def samples(m, B, seed):
    """Fine residuals [B][m][m] and coarse targets [B][mc][mc], complex."""
    rng = np.random.default_rng(seed)
    mc = (m - 1) // 2
    r = rng.standard_normal((B, m, m)) + 1j * rng.standard_normal((B, m, m))
    e = rng.standard_normal((B, mc, mc)) + 1j * rng.standard_normal((B, mc, mc))
    return r, e


def test_weight_count_matches_the_oracle_layout():
    p, _ = small_problem(True, 4)
    with p:
        assert p.learned_weights().size == LO.num_params(4)
    p, _ = small_problem(False, 32, m=63, N=8)
    with p:
        assert p.learned_weights().size == LO.num_params(32)


def test_loss_and_gradients_match_the_oracle():
    """FP32 activations, C = 4, gates away from 1: the GPU's loss against the
    oracle's, its gradient against central differences of the oracle's loss
    along random directions and for single weights of the residual path and
    of every kind of gate weight."""
    import torch
    m, N, eps, C = 31, 8, 0.1, 4
    p, a = small_problem(True, C, m, N, eps)
    ps, w = seeded_weights(C, 40, 0.3)
    w64 = w.astype(np.float64)
    lam = LO.forward_sign_eigs(N, eps)
    with p:
        p.set_learned_weights(w)
        lc = LO.LearnedCorrection(m, np.log(a), 1.0 / N)
        idx = [0, 2, 4]
        r, e = samples(m, 3, 7)
        loss_gpu, g = p.learned_loss_grad(idx, torch.from_numpy(r).cuda(), torch.from_numpy(e).cuda())
        S = [(r[b], lam[idx[b]], e[b]) for b in range(3)]
        L = lambda v: LO.loss(LO.unflatten(v, C), S, lc)
        loss_ref = L(w64)
        assert abs(loss_gpu - loss_ref) <= 1e-4 * loss_ref, (loss_gpu, loss_ref)
        rng = np.random.default_rng(8)
        h = 1e-4
        for _ in range(4):
            d = rng.standard_normal(w.size)
            d /= np.linalg.norm(d)
            fd = (L(w64 + h * d) - L(w64 - h * d)) / (2 * h)
            assert abs(float(g @ d) - fd) <= 2e-3 * max(abs(fd), 1e-2 * np.linalg.norm(g)), (g @ d, fd)
        shapes = LO.param_shapes(C)
        offs = np.cumsum([0] + [int(np.prod(s)) for s in shapes])
        # conv 0, 4, 8; A1_2, A2_5
        for t in (0, 4, 8, 9 + 2, 17 + 5):
            j = int(offs[t] + rng.integers(offs[t + 1] - offs[t]))
            e_j = np.zeros(w.size)
            e_j[j] = 1.0
            fd = (L(w64 + h * e_j) - L(w64 - h * e_j)) / (2 * h)
            assert abs(g[j] - fd) <= 5e-3 * max(abs(fd), 1e-3 * np.abs(g).max()), (t, g[j], fd)


def _tol(eps, N, m, C):
    U32 = 2.0 ** -24
    L = int(math.log2(m + 1))
    return 16 * U32 * (math.log2(N * (m + 1) ** 2) + 8 * L + 9 * math.sqrt(9 * C)) / eps


@pytest.mark.parametrize("m,N,eps,C,gs", [(31, 8, 0.1, 4, 0.0), (63, 16, 0.0625, 32, 0.3),
                                          (127, 4, 0.02, 32, 0.5)])
def test_learned_apply_Pinv_matches_the_oracle(m, N, eps, C, gs):
    """Seeded weights (gates 1, then gates away from 1) in the oracle's
    learned P_eps^{-1} with its own calibration, the judge off on both sides
    (so that the correction's arithmetic is what is compared); FP32
    activations.  The residual ratios of the GPU's calibration (which follow
    from its one step) match the oracle's."""
    import torch
    p, a = small_problem(True, C, m, N, eps)
    ps, w = seeded_weights(C, 50 + m, gs)
    y = np.random.default_rng(30 + m).uniform(-1, 1, (N, m, m))
    with p:
        p.set_learned_weights(w)
        p.set_learned_judge(False)
        z = p.apply_Pinv(torch.from_numpy(y).cuda())
        torch.cuda.synchronize()
        z = z.cpu().numpy()
        ratios = p.learned_residual_ratios()
        assert p.learned_fallbacks == 0
    K = O.fd_stiffness_varcoef(a)
    h = O.MGHierarchy(K, m)
    lc = LO.LearnedCorrection(m, np.log(a), 1.0 / N)
    params = LO.unflatten(w.astype(np.float64), C)
    alpha, rr, _ = LO.calibrate(h, lc, params, 1.0 / N, eps, N, judge=False)
    ref = LO.apply_Pinv_learned(y, h, lc, params, 1.0 / N, eps, alpha)
    err = float(np.max(np.abs(z - ref)) / np.max(np.abs(ref)))
    assert err <= _tol(eps, N, m, C), (err, _tol(eps, N, m, C))
    np.testing.assert_allclose(ratios, rr, atol=1e-3)
    print(f"learned P^-1 parity m={m} N={N} C={C} gates {gs}: err {err:.2e}, ratios {np.round(ratios, 3)}")


@pytest.mark.parametrize("m,N,eps,C,gs,seed", [(31, 8, 0.1, 4, 0.3, 80), (63, 16, 0.0625, 4, None, 81)])
def test_judge_matches_the_oracle(m, N, eps, C, gs, seed):
    """The judge on both sides: the GPU's power-iteration radii per
    frequency (V-cycle and corrected preconditioner) against the oracle's,
    the same decision, and the judged P_eps^{-1} element by element.  Seeded
    random weights (a correction that hurts: rejected) and zero weights (the
    V-cycle plus the sweep and step: kept).  The cases have the two maxima
    apart by more than the radii's tolerance, so that the decision is not a
    rounding tie."""
    import torch
    p, a = small_problem(True, C, m, N, eps)
    if gs is None:
        w = np.zeros(LO.num_params(C), np.float32)
    else:
        _, w = seeded_weights(C, seed, gs)
    y = np.random.default_rng(seed).uniform(-1, 1, (N, m, m))
    with p:
        p.set_learned_weights(w)
        z = p.apply_Pinv(torch.from_numpy(y).cuda())
        torch.cuda.synchronize()
        z = z.cpu().numpy()
        rv, rc, mv, mc = p.learned_judge_radii()
        fb = p.learned_fallbacks
    K = O.fd_stiffness_varcoef(a)
    h = O.MGHierarchy(K, m)
    lc = LO.LearnedCorrection(m, np.log(a), 1.0 / N)
    params = LO.unflatten(w.astype(np.float64), C)
    alpha, _, (ov, oc) = LO.calibrate(h, lc, params, 1.0 / N, eps, N)
    print(f"judge m={m}: V-cycle {ov.max():.4f} (GPU {mv:.4f}), corrected {oc.max():.4f} "
          f"(GPU {mc:.4f}), kept {alpha != 0.0} (GPU {fb == 0})")
    np.testing.assert_allclose(rv, ov, rtol=1e-3)
    np.testing.assert_allclose(rc, oc, rtol=1e-3)
    assert abs(mc - mv) > 5e-3 * mv
    assert (fb == 0) == (alpha != 0.0)
    ref = LO.apply_Pinv_learned(y, h, lc, params, 1.0 / N, eps, alpha)
    err = float(np.max(np.abs(z - ref)) / np.max(np.abs(ref)))
    assert err <= _tol(eps, N, m, C), err


def test_judge_api():
    """The judge's entry points: radii are NaN before a calibration and with
    the judge off; turning it off, on or off again recalibrates at the next
    apply (the fallback flag follows); a problem of another route has no
    judge."""
    import torch
    from paper_2002_01108_gb300 import BecError, Problem
    p, _ = small_problem(True, 4)
    _, w = seeded_weights(4, 80, 0.3)           # a correction the judge rejects (see above)
    y = torch.from_numpy(np.random.default_rng(3).uniform(-1, 1, (8, 31, 31))).cuda()
    with p:
        p.set_learned_weights(w)
        rv, rc, mv, mc = p.learned_judge_radii()
        assert np.all(np.isnan(rv)) and np.all(np.isnan(rc)) and math.isnan(mv) and math.isnan(mc)
        p.apply_Pinv(y)
        _, _, mv, mc = p.learned_judge_radii()
        assert mc > mv > 0 and p.learned_fallbacks == 1
        p.set_learned_judge(False)
        assert math.isnan(p.learned_judge_radii()[2])
        p.apply_Pinv(y)
        assert math.isnan(p.learned_judge_radii()[2]) and p.learned_fallbacks == 0
        p.set_learned_judge(True)
        p.apply_Pinv(y)
        _, _, mv2, mc2 = p.learned_judge_radii()
        assert (mv2, mc2) == (mv, mc) and p.learned_fallbacks == 1
    with Problem(2, 31, 8, route="mg", precision="fp32") as q:
        q.set_eps(0.1)
        with pytest.raises(BecError):
            q.set_learned_judge(False)


def test_bf16_activations_track_fp32():
    import torch
    m, N, eps, C = 63, 16, 0.05, 32
    r, e = samples(m, 4, 9)
    _, w = seeded_weights(C, 60, 0.3)
    losses = []
    for fp32 in (True, False):
        p, _ = small_problem(fp32, C, m, N, eps)
        with p:
            p.set_learned_weights(w)
            loss, g = p.learned_loss_grad([0, 3, 5, 8], torch.from_numpy(r).cuda(), torch.from_numpy(e).cuda())
            losses.append((loss, g))
    (l32, g32), (l16, g16) = losses
    assert abs(l16 - l32) <= 2e-2 * l32
    assert np.dot(g16, g32) / (np.linalg.norm(g16) * np.linalg.norm(g32)) > 0.95


@pytest.mark.parametrize("m", [63, 127, 255])
def test_bf16_tensor_core_network_matches_the_oracle(m):
    """BF16 activations with C = 32 run every convolution of the residual
    path on the tensor cores (tcgen05, BF16 operands and weights, FP32
    accumulation).  Their coarse correction, against the FP64 oracle network
    with the same weights: the loss with e* = the oracle's correction is the
    squared relative error.  Bound: each of the 9 layers rounds its inputs,
    weights and outputs to BF16 (u = 2^-9), the gates and transfers add a few
    more roundings of the activations: 24 u relative, worst case."""
    import torch
    N, eps, C = 16, 0.05, 32
    p, a = small_problem(False, C, m, N, eps)
    idx = [0, 3, 5, 8]
    r, _ = samples(m, 4, 11)
    ps, w = seeded_weights(C, 70, 0.3)
    lam = LO.forward_sign_eigs(N, eps)
    with p:
        p.set_learned_weights(w)
        lc = LO.LearnedCorrection(m, np.log(a), 1.0 / N)
        params = LO.unflatten(w.astype(np.float64), C)
        e_ref = np.stack([lc.coarse(params, r[b], lam[idx[b]]) for b in range(4)])
        loss, _ = p.learned_loss_grad(idx, torch.from_numpy(r).cuda(), torch.from_numpy(e_ref).cuda())
    print(f"BF16 network m={m}: relative error {math.sqrt(loss):.2e}")
    assert math.sqrt(loss) <= 24 * 2.0 ** -9


def test_bf16_tensor_core_apply_matches_the_oracle():
    """The learned P_eps^{-1} with BF16 activations, C = 32: inference runs
    every convolution on the tensor cores with each gated layer's gate
    applied in the epilogue, then the pole sum, the sweep and the calibrated
    step (judge off on both sides).  Against the FP64 oracle with the same
    seeded weights, the error is measured against the size of the
    correction's contribution, ||z_ref - z_mg|| (z_mg: the same route with
    alpha = 0): BF16 activations (u = 2^-9, 24 u per network as above) plus
    the step alpha computed from them, 48 u together."""
    import torch
    m, N, eps, C = 63, 16, 0.0625, 32
    p, a = small_problem(False, C, m, N, eps)
    _, w = seeded_weights(C, 90, 0.3)
    y = np.random.default_rng(91).uniform(-1, 1, (N, m, m))
    with p:
        p.set_learned_weights(w)
        p.set_learned_judge(False)
        z = p.apply_Pinv(torch.from_numpy(y).cuda())
        torch.cuda.synchronize()
        z = z.cpu().numpy()
    K = O.fd_stiffness_varcoef(a)
    h = O.MGHierarchy(K, m)
    lc = LO.LearnedCorrection(m, np.log(a), 1.0 / N)
    params = LO.unflatten(w.astype(np.float64), C)
    alpha, _, _ = LO.calibrate(h, lc, params, 1.0 / N, eps, N, judge=False)
    ref = LO.apply_Pinv_learned(y, h, lc, params, 1.0 / N, eps, alpha)
    mg = LO.apply_Pinv_learned(y, h, lc, params, 1.0 / N, eps, 0.0)
    corr = float(np.linalg.norm(ref - mg))
    assert corr > 1e-3 * np.linalg.norm(ref), corr          # the correction is not negligible
    err = float(np.linalg.norm(z - ref)) / corr
    print(f"BF16 tensor-core learned P^-1: error {err:.2e} of the correction's contribution")
    assert err <= 48 * 2.0 ** -9, err


def test_training_lowers_the_loss():
    m, N, eps = 63, 16, 0.05
    p, _ = small_problem(False, 32, m, N, eps)
    with p:
        hist = p.learned_train(steps=200, batch=8, lr=2e-3, seed=1)
    assert np.all(np.isfinite(hist))
    assert hist[-20:].mean() < 0.5 * hist[:5].mean(), (hist[:5], hist[-20:])


TRAIN_STEPS = 1500


def abc_arms(m, N, rtol):
    """FGMRES(30) iterations, error against sequential stepping and true
    relative residual for the three arms on a = exp(GRF) at m^2 x N: the
    multigrid preconditioner alone ("mg"), the learned route at zero
    weights ("zero": the V-cycle, the smoothing sweep and the calibrated
    step without a correction) and the learned route trained on the GPU."""
    import torch
    from paper_2002_01108_gb300 import Problem
    eps = math.sqrt(1.0 / N) / 2
    a = O.node_coefficient(grf_log_coefficient(seed=5, m=m))
    case = heat_case_2d(seed=6, m=m, N=N, eps=eps)
    f = O.build_rhs(case.u0, case.fsrc, case.tau)
    K = O.fd_stiffness_varcoef(a)
    u_ref = O.timestep_solve(f, sp.identity(K.shape[0], format="csr"), K, case.tau)
    fd = torch.from_numpy(f).cuda()
    res = {}
    for arm in ("mg", "zero", "trained"):
        route = "mg" if arm == "mg" else "learned"
        with Problem(2, m, N, route=route, precision="fp32", a_nodes=a, flexible=True) as p:
            p.set_eps(eps)
            if arm == "zero":
                p.set_learned_weights(np.zeros(p.learned_weights().size, np.float32))
            if arm == "trained":
                hist = p.learned_train(steps=TRAIN_STEPS, batch=16, lr=2e-3, seed=3)
                print(f"{m}^2 x {N} training loss", hist[:3], hist[-3:])
                assert np.all(np.isfinite(hist))
                assert hist[-50:].mean() < 0.2 * hist[:5].mean()
            if arm == "zero":
                p.set_learned_judge(False)   # the sweep and step alone, not judged
            u, info = p.gmres_solve(fd, restart=30, rtol=rtol, maxit=400, flexible=True)
            torch.cuda.synchronize()
            err = float(np.linalg.norm(u.cpu().numpy() - u_ref) / np.linalg.norm(u_ref))
            extra = ()
            if route == "learned":
                ratios = p.learned_residual_ratios()
                extra = (p.learned_fallbacks, float(np.mean(ratios)), p.learned_judge_radii()[2:])
            res[arm] = (info["iters"], err, info["true_relres"]) + extra
    print(f"A/B/C {m}^2 x {N}", res)
    for arm, (it, err, rr, *_) in res.items():
        assert rr <= 1.01 * rtol and err <= 1e-8, (arm, it, err, rr)
    return res


def test_trained_correction_gains_over_the_vcycle():
    """A/B/C at 63^2 x 32: the judge keeps the trained correction, which
    takes fewer FGMRES iterations than the V-cycle alone and than the route
    at zero weights; every arm reaches the sequential stepping solution."""
    res = abc_arms(63, 32, 1e-10)
    assert res["trained"][3] == 0, res
    assert res["trained"][0] < res["mg"][0], res
    assert res["trained"][0] < res["zero"][0], res


def test_trained_correction_gains_at_127():
    """A/B/C at 127^2 x 64, as at 63^2 x 32."""
    res = abc_arms(127, 64, 1e-10)
    assert res["trained"][3] == 0, res
    assert res["trained"][0] < res["mg"][0], res
    assert res["trained"][0] < res["zero"][0], res


def test_learned_route_at_the_workload_size():
    """The learned form at the size bench.py times: 255^2 x 256, a = exp(GRF),
    eps = sqrt(tau)/2, trained on the GPU as bench.py trains it (4000 steps,
    lr 1e-3): FGMRES(30) reaches RES 1e-8 (the benchmark's tolerance), and
    solved on to RES 1e-10 its solution equals sequential stepping to 1e-8.
    At this size the trained correction does not gain: the judge finds its
    spectral radius above the V-cycle's and falls back to the V-cycle, so the
    route takes the V-cycle's iterations.  The iteration count of the
    correction forced on (judge off) is printed beside it."""
    import torch
    from paper_2002_01108_gb300 import Problem
    m, N = 255, 256
    eps = math.sqrt(1.0 / N) / 2
    a = O.node_coefficient(grf_log_coefficient(seed=5, m=m))
    case = heat_case_2d(seed=6, m=m, N=N, eps=eps)
    f = O.build_rhs(case.u0, case.fsrc, case.tau)
    K = O.fd_stiffness_varcoef(a)
    u_ref = O.timestep_solve(f, sp.identity(K.shape[0], format="csr"), K, case.tau)
    fd = torch.from_numpy(f).cuda()
    with Problem(2, m, N, route="mg", precision="fp32", a_nodes=a, flexible=True) as p:
        p.set_eps(eps)
        _, info_mg = p.gmres_solve(fd, restart=30, rtol=1e-8, flexible=True)
    with Problem(2, m, N, route="learned", precision="fp32", a_nodes=a, flexible=True) as p:
        p.set_eps(eps)
        p.learned_train(steps=4000, batch=16, lr=1e-3, seed=3)
        p.set_learned_judge(False)
        _, info_on = p.gmres_solve(fd, restart=30, rtol=1e-8, maxit=400, flexible=True)
        p.set_learned_judge(True)
        u, info = p.gmres_solve(fd, restart=30, rtol=1e-8, flexible=True)
        assert info["converged"] == 1 and info["true_relres"] <= 1.01e-8, info
        radii = p.learned_judge_radii()
        print(f"255^2 x 256: V-cycle {info_mg['iters']} iterations, judged route {info['iters']} "
              f"(fallback {p.learned_fallbacks}, radii V-cycle {radii[2]:.3f} corrected "
              f"{radii[3]:.3f}), correction forced on {info_on['iters']}")
        assert info["iters"] <= info_mg["iters"] + 1, (info, info_mg)
        u, info = p.gmres_solve(fd, restart=30, rtol=1e-10, maxit=400, flexible=True)
        torch.cuda.synchronize()
    assert info["converged"] == 1 and info["true_relres"] <= 1.01e-10, info
    err = float(np.linalg.norm(u.cpu().numpy() - u_ref) / np.linalg.norm(u_ref))
    assert err <= 1e-8, err
