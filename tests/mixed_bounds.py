"""Reference and error bound for per-trajectory checks of the BF16X3 path.

The mixed path draws its pump normals eta in FP32 and rounds them once to BF16
(its noise operand), then forms L.eta with the two products L_hi.eta + L_lo.eta
and W.s with the three products of the hi/lo splits, accumulating in FP32. The
rounding of eta is part of what that path computes, so a trajectory is compared
with the oracle's integrator run on the *same* BF16-rounded normals
(``BF16NoiseOracle``). What is left between the two is small and bounded term
by term (``step_bound``):

* the split of L: |L - (hi + lo)| <= 2^-18 |L| after the FP32 image (2^-24), so
  (L eta)_i is off by ~2^-17 sum_j |L_ij||eta_j|;
* the split of W and s: 3 2^-18 sum_j |W_ij||s_j| in each of the predictor and
  corrector fields;
* FP32 accumulation over K = N in steps of 16 products: (N/16) 2^-22 of the
  same absolute sums;
* the FP32 Box-Muller: the kernel's normals differ from the oracle's by ~1e-6
  relative, so an eta within 1e-5 relative of a BF16 rounding boundary may
  round the other way (2^-8 |eta_j|): those entries are found and added in full;
* FP32 state arithmetic (a few 2^-24 per component per step).

A field error dB moves the Heun step by at most ~sqrt(3)(1 + |b|) |dB| per
component of b (the step is s x b twice, |s| = sqrt(3)), and renormalisation
does not increase it. Without the BF16 rounding of eta in the reference the
differences would be 2^-9-sized; a single-term L (a dropped lo image) adds
~2^-9 sum_j L_ij eta_j, far above this bound.
"""
import math

import numpy as np

from oracle.twa_oracle import TWAOracle


def bf16(a):
    """Round-to-nearest-even BF16 of the FP32 value of `a`, returned as float64."""
    import torch
    x = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
    return x.to(torch.bfloat16).to(torch.float64).numpy()


def near_bf16_boundary(a, rel=1e-5):
    """True where a relative change of `rel` can change the BF16 rounding."""
    a = np.asarray(a, dtype=np.float64)
    return bf16(a * (1.0 - rel)) != bf16(a * (1.0 + rel))


class BF16NoiseOracle(TWAOracle):
    """The oracle's stochastic-Heun integrator with the pump normals eta rounded
    to BF16, the rounding the mixed path applies to its noise operand; the
    collective normals and all arithmetic stay FP64."""

    def noise(self, t):
        xi_x, xi_y, eta_x, eta_y = super().noise(t)
        return xi_x, xi_y, bf16(eta_x), bf16(eta_y)


# representation error of a W.s product per precision: BF16X3 splits W and s
# (three products: 3 2^-18); BF16X2 splits W but rounds s once to BF16
# (2^-9 + 2^-18); BF16L2 and BF16B round both off their two-product band
# (2 2^-9). L.eta is split (2^-17 after eta's own rounding, which the reference
# shares) except in BF16B, whose L is one BF16 product off the band (2^-9).
W_REP = {"bf16x3": 3 * 2.0 ** -18, "bf16x2": 2.0 ** -9 + 2.0 ** -18, "bf16l2": 2 * 2.0 ** -9 + 2.0 ** -18,
         "bf16b": 2 * 2.0 ** -9 + 2.0 ** -18}
L_REP = {"bf16b": 2.0 ** -9}


def step_bound(o, sx, sy, sz, prec="bf16x3"):
    """Bound, per trajectory and site, of the difference that one step of the
    mixed path (`prec`) adds between the kernel and ``BF16NoiseOracle`` o, for
    the step o is about to take from the state (sx, sy, sz)."""
    N, dt, G = o.N, o.dt, o.Gamma
    xi_x, xi_y, ex, ey = TWAOracle.noise(o, o.t)          # unrounded FP64 normals
    absL, absW = np.abs(o.L), np.abs(o.W)
    acc = (N / 16.0) * 2.0 ** -22                          # FP32 accumulation
    sd = math.sqrt(dt)
    lsum = np.maximum(np.abs(ex) @ absL.T, np.abs(ey) @ absL.T)
    dq = sd * (L_REP.get(prec, 2.0 ** -17) + 2.0 ** -24 + acc + 2e-6) * lsum
    flip_x = np.abs(ex) * near_bf16_boundary(ex)
    flip_y = np.abs(ey) * near_bf16_boundary(ey)
    dq += sd * 2.0 ** -8 * np.maximum(flip_x @ absL.T, flip_y @ absL.T)
    # pump field at the state and at the predictor (|s~| <= |s| (1 + |b|))
    wsum = np.maximum(np.abs(sx) @ absW.T, np.abs(sy) @ absW.T)
    bmax = _field_size(o, sx, sy, sz)
    dp = 0.5 * dt * (W_REP[prec] + 2.0 ** -24 + acc) * wsum * (1.0 + bmax)
    dxi = math.sqrt(G * dt) * 2e-6 * max(np.max(np.abs(xi_x)), np.max(np.abs(xi_y)))
    db = dq + dp + dxi
    return 2.0 * math.sqrt(3.0) * (1.0 + bmax) * math.sqrt(2.0) * db + 8 * 2.0 ** -24 * math.sqrt(3.0)


def _field_size(o, sx, sy, sz):
    """max |b| over trajectories and sites for the step o is about to take."""
    dxi_x, dxi_y, dchi_x, dchi_y = o.noise_increments(o.t)
    bx, by, _ = o.field(sx, sy, sz, dxi_x, dxi_y, dchi_x, dchi_y)
    return float(np.max(np.hypot(bx, by)))


def track(o_ref, run_gpu, steps, prec="bf16x3"):
    """Advance the BF16-noise oracle and the kernel step by step; after step k
    check |kernel - oracle| <= 2 x (sum of the step bounds so far) element by
    element (the factor 2 covers the growth of earlier differences over a few
    steps). run_gpu() advances the kernel one step and returns its state.
    Returns the largest ratio of difference to bound."""
    tol = 0.0
    worst = 0.0
    for _ in range(steps):
        tol = tol + step_bound(o_ref, o_ref.sx, o_ref.sy, o_ref.sz, prec)
        o_ref.run(1)
        gx, gy, gz = run_gpu()
        err = np.maximum(np.maximum(np.abs(gx - o_ref.sx), np.abs(gy - o_ref.sy)), np.abs(gz - o_ref.sz))
        ratio = float(np.max(err / (2.0 * tol)))
        assert ratio <= 1.0, (ratio, float(np.max(err)))
        worst = max(worst, ratio)
    return worst
