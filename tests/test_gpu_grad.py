"""Adjoint gradients (twa_grad) against the oracle's FP64 tangent and against
central finite differences with common random numbers, through the C ABI.

The FP64 GPU adjoint and the oracle tangent compute the same pathwise
derivative of the same discretised trajectories, so they agree per trajectory
to rounding (1e-8 relative here). The mixed-precision adjoints (FP32 tape,
BF16X3 or BF16X2 contractions) differ by their arithmetic only: over the short horizons
tested it stays within 1e-2 of the FP64 result, and the paired per-trajectory
difference of the two (the precision error of the estimate) is checked to be a
small fraction of the gradient's standard error.
"""
import numpy as np
import pytest

from oracle.twa_tangent import TWATangent

pytestmark = pytest.mark.gpu


def _twa():
    from paper_2608_10075_b300 import twa
    return twa


@pytest.mark.parametrize("objective", ["SpSm", "g2"])
@pytest.mark.parametrize("theta,col", [("w", 0), ("alpha", 1)])
def test_fp64_adjoint_equals_oracle_tangent(objective, theta, col):
    twa = _twa()
    N, alpha, w, G, dt, M, steps, t0 = 16, 1.0, 8.0, 1.0, 2e-3, 32, 60, 0.04
    o = TWATangent(N, alpha, w, G, dt, 0, M, theta, window_start=t0)
    o.run(steps)
    J, dJ, per = o.derivative(objective)
    with twa.TWA(N, alpha, w, G, dt, seed=0, precision="fp64", window_start=t0) as g:
        r = g.grad(objective, M, steps, checkpoint=16, per_traj=True)
    assert abs(r["J"] - J) <= 1e-9 * abs(J)
    d = r["dJ_dw"] if theta == "w" else r["dJ_dalpha"]
    assert abs(d - dJ) <= 1e-8 * max(abs(dJ), 1e-6), (d, dJ)
    assert np.max(np.abs(r["per_traj"][:, col] - per)) <= 1e-7 * max(np.max(np.abs(per)), 1e-6)


@pytest.mark.parametrize("objective", ["SpSm", "g2"])
def test_fp64_adjoint_with_sample_stride_equals_oracle_tangent(objective):
    # window samples every 4th step (steps 19, 23, ..., 59): the objective and its
    # derivatives are those of the strided window
    twa = _twa()
    N, alpha, w, G, dt, M, steps, t0, k = 16, 1.0, 8.0, 1.0, 2e-3, 24, 59, 0.03, 4
    for theta, key in (("w", "dJ_dw"), ("alpha", "dJ_dalpha")):
        o = TWATangent(N, alpha, w, G, dt, 0, M, theta, window_start=t0, sample_stride=k)
        o.run(steps)
        J, dJ, _ = o.derivative(objective)
        with twa.TWA(N, alpha, w, G, dt, seed=0, precision="fp64", window_start=t0, sample_stride=k) as g:
            r = g.grad(objective, M, steps, checkpoint=16)
        assert o.count == (steps - 15) // k
        assert abs(r["J"] - J) <= 1e-9 * abs(J)
        assert abs(r[key] - dJ) <= 1e-8 * max(abs(dJ), 1e-6), (theta, r[key], dJ)


def test_checkpoint_stride_does_not_change_the_gradient():
    twa = _twa()
    res = []
    for ck in (1, 7, 64):
        with twa.TWA(40, 0.8, 10.0, 1.0, 1e-3, seed=2, precision="fp64", window_start=0.01) as g:
            res.append(g.grad("g2", 24, 30, checkpoint=ck))
    for r in res[1:]:
        assert abs(r["dJ_dw"] - res[0]["dJ_dw"]) <= 1e-11 * abs(res[0]["dJ_dw"])
        assert abs(r["dJ_dalpha"] - res[0]["dJ_dalpha"]) <= 1e-11 * abs(res[0]["dJ_dalpha"])


def test_fp64_adjoint_matches_crn_finite_difference_on_gpu():
    # central differences of the GPU forward itself (J from twa_grad's forward run)
    twa = _twa()
    N, alpha, w, G, dt, M, steps, t0, d = 130, 1.2, 12.0, 1.0, 1e-3, 40, 40, 0.02, 1e-5
    kw = dict(seed=7, precision="fp64", window_start=t0)
    with twa.TWA(N, alpha, w, G, dt, **kw) as g:
        r = g.grad("SpSm", M, steps, checkpoint=16)
    J = {}
    for s in (+1, -1):
        with twa.TWA(N, alpha, w * (1 + s * d), G, dt, **kw) as g:
            J[("w", s)] = g.grad("SpSm", M, steps, want_alpha=False)["J"]
        with twa.TWA(N, alpha + s * d, w, G, dt, **kw) as g:
            J[("a", s)] = g.grad("SpSm", M, steps, want_alpha=False)["J"]
    fd_w = (J[("w", 1)] - J[("w", -1)]) / (2 * w * d)
    fd_a = (J[("a", 1)] - J[("a", -1)]) / (2 * d)
    assert abs(r["dJ_dw"] - fd_w) <= 1e-5 * abs(fd_w)
    assert abs(r["dJ_dalpha"] - fd_a) <= 1e-5 * abs(fd_a)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x2", "bf16b"])
@pytest.mark.parametrize("objective", ["SpSm", "g2"])
def test_mixed_adjoint_close_to_fp64(objective, prec):
    twa = _twa()
    N, alpha, w, G, dt, M, steps, t0 = 256, 1.0, 32.0, 1.0, 1e-3, 128, 40, 0.02
    out = {}
    for p in ("fp64", prec):
        with twa.TWA(N, alpha, w, G, dt, seed=1, precision=p, window_start=t0) as g:
            out[p] = g.grad(objective, M, steps, checkpoint=16)
    for k in ("dJ_dw", "dJ_dalpha"):
        a, b = out["fp64"][k], out[prec][k]
        assert abs(a - b) <= 1e-2 * abs(a) + 3 * out["fp64"][k + "_se"] * 1e-2, (k, a, b)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x2"])
@pytest.mark.parametrize("objective", ["SpSm", "g2"])
def test_mixed_adjoint_error_is_far_below_the_sampling_error(objective, prec):
    # per-trajectory gradient samples of the mixed and FP64 adjoints on the same
    # trajectories: their paired difference (the precision error) must be a small
    # fraction of the standard error the gradient is quoted with
    import math
    twa = _twa()
    N, alpha, w, G, dt, M, steps, t0 = 256, 1.0, 32.0, 1.0, 1e-3, 128, 40, 0.02
    out = {}
    for p in ("fp64", prec):
        with twa.TWA(N, alpha, w, G, dt, seed=1, precision=p, window_start=t0) as g:
            out[p] = g.grad(objective, M, steps, checkpoint=16, per_traj=True)
    for col, k in ((0, "dJ_dw"), (1, "dJ_dalpha")):
        d = out[prec]["per_traj"][:, col] - out["fp64"]["per_traj"][:, col]
        paired, paired_se = abs(float(d.mean())), float(d.std(ddof=1) / math.sqrt(M))
        assert paired + 3.0 * paired_se <= 0.2 * out["fp64"][k + "_se"], (k, paired, paired_se, out["fp64"][k + "_se"])


def test_mixed_adjoint_matches_finite_differences_at_delta_1e4():
    # central differences with common random numbers at the relative step
    # delta = 1e-4 in w, through the same BF16X3 forward run the adjoint
    # differentiates: the tensor-core images hold W / w and L / sqrt(w), so the
    # runs at w (1 +- delta) differ only in the FP32 factors w and sqrt(w) of the
    # epilogue, not by a rounding of their images of size 2^-17 / (2 delta) ~ 4 %.
    # (BF16X2 and BF16 round the state itself to BF16 for W.s: their forward map
    # is piecewise constant on the scale 2^-9, which a step of 1e-4 does not
    # resolve; their adjoints are checked against the FP64 adjoint above.)
    prec = "bf16x3"
    twa = _twa()
    N, alpha, w, G, dt, M, steps, t0, d = 256, 1.0, 32.0, 1.0, 1e-3, 128, 60, 0.03, 1e-4
    kw = dict(seed=5, precision=prec, window_start=t0)
    with twa.TWA(N, alpha, w, G, dt, **kw) as g:
        r = g.grad("SpSm", M, steps, checkpoint=16, want_alpha=False)
    J = []
    for s in (+1, -1):
        with twa.TWA(N, alpha, w * (1 + s * d), G, dt, **kw) as g:
            J.append(g.grad("SpSm", M, steps, checkpoint=16, want_alpha=False)["J"])
    fd = (J[0] - J[1]) / (2 * w * d)
    assert abs(r["dJ_dw"] - fd) <= 1e-2 * abs(fd), (r["dJ_dw"], fd)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x2", "fp32", "tf32"])
def test_tensor_core_images_do_not_depend_on_w(prec):
    # W.s and L.eta of the step at w and at 2w: the images are those of W / w
    # and L / sqrt(w), so the FP32 results scale exactly (2 is exact, and so is
    # sqrt(2) w.r.t. the same rounding of the accumulated product times the
    # factor: compare against the unit-w product times the factor)
    import torch
    twa = _twa()
    N, alpha, K = 300, 0.8, 6
    g_ = torch.Generator().manual_seed(3)
    s = torch.randn(K, N, generator=g_, dtype=torch.float64).cuda()
    out = {}
    for w in (4.0, 8.0, 4.0 * (1 + 1e-4)):
        with twa.TWA(N, alpha, w, 1.0, 1e-3, precision=prec) as g:
            out[w] = (g.contract(s, "W").cpu().numpy(), g.contract(s, "L").cpu().numpy())
    W4, L4 = out[4.0]
    W8, L8 = out[8.0]
    assert np.array_equal(W8, 2.0 * W4)
    # L: sqrt(8) / sqrt(4) = sqrt(2) is not exact in FP32; the accumulators agree,
    # so the results differ by the rounding of the two products only
    np.testing.assert_allclose(L8, np.sqrt(2.0) * L4, rtol=3e-7, atol=0)
    w1 = 4.0 * (1 + 1e-4)
    W1, L1 = out[w1]
    np.testing.assert_allclose(W1, W4 * (w1 / 4.0), rtol=3e-7, atol=0)
    np.testing.assert_allclose(L1, L4 * np.sqrt(w1 / 4.0), rtol=3e-7, atol=0)


def test_autograd_function_wraps_the_adjoint():
    import torch
    from paper_2608_10075_b300.autograd import SteadyStateObjective
    spec = dict(N=64, Gamma=1.0, dt=1e-3, seed=3, precision="fp64", window_start=0.01, M=32, steps=20,
                checkpoint=8, objective="SpSm")
    w = torch.tensor(6.0, dtype=torch.float64, requires_grad=True)
    a = torch.tensor(1.1, dtype=torch.float64, requires_grad=True)
    J = SteadyStateObjective.apply(w, a, spec)
    (2.0 * J).backward()
    twa = _twa()
    with twa.TWA(64, 1.1, 6.0, 1.0, 1e-3, seed=3, precision="fp64", window_start=0.01) as g:
        r = g.grad("SpSm", 32, 20, checkpoint=8)
    assert abs(float(J.detach()) - r["J"]) <= 1e-12 * abs(r["J"])
    assert abs(float(w.grad) - 2 * r["dJ_dw"]) <= 1e-9 * abs(r["dJ_dw"])
    assert abs(float(a.grad) - 2 * r["dJ_dalpha"]) <= 1e-9 * abs(r["dJ_dalpha"])


def test_grad_rejects_unsupported_cases():
    import math
    twa = _twa()
    with twa.TWA(8, 0.0, 1.0, 1.0, 1e-3) as g:
        with pytest.raises(twa.TWAError) as e:
            g.grad("SpSm", 4, 5)
        assert e.value.name == "TWA_EUNSUPPORTED"
        r = g.grad("SpSm", 4, 5, want_alpha=False)   # d/dw is fine at alpha = 0
        assert math.isfinite(r["dJ_dw"])
    with twa.TWA(8, 1.0, 1.0, 1.0, 1e-3, window_start=1.0) as g:
        with pytest.raises(twa.TWAError) as e:
            g.grad("SpSm", 4, 5)
        assert e.value.name == "TWA_ESTATE"
