"""FP64 CPU oracle for the dissipative truncated-Wigner (TWA) dynamics of N spins
under collective cavity decay and the power-law correlated pump.

TEST INFRASTRUCTURE. This module is the slow, plain reference that the CUDA
path is checked against. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the product library never does
and shares no code with it.

Everything is float64 numpy, vectorised over trajectories only. A dense matmul
(BLAS) and ``numpy.linalg.cholesky`` serve as library steps; nothing is
blocked, fused or reordered beyond the definitions below.

What it follows (arxiv 2608.10075):

* Eq. (1): Lindblad model, collective decay Gamma through S^- = sum_i sigma_i^-,
  pump sum_ij w_ij/2 D[sigma_j^+, sigma_i^-].
* Eq. (2): pump matrix w_ij = w / (|i-j| + 1)^alpha, open chain.
* Sec. S1, Eq. (S1): stochastic equations of motion of the classical spins,
  with white noises <xi^a xi^b> = Gamma delta_ab (no site index: one collective
  noise per component) and <chi_i^a chi_j^b> = w_ij delta_ab.
* Sec. S1, item 3: discrete-Wigner initial sampling, s^x, s^y = +-1.
* Sec. S1, items 5-6: trajectory averages, symmetric-to-normal ordering of
  <S+S-> and <S+S+S-S->; the closing paragraph of Sec. S1: time averaging.
* Main text, "Observables and method": g2 = <S+S+S-S-> / <S+S->^2.

Readings where the paper is silent (each is also listed in the design notes):

* Integrator: stochastic Heun (predictor/corrector, Stratonovich sense, the
  same noise in both stages) followed by renormalising every spin to length
  sqrt(3). Option: the semi-implicit midpoint scheme the paper cites for its
  own runs (Mentink et al., J. Phys.: Condens. Matter 22, 176001 (2010)),
  written with the effective field of Sec. S1, ds_i = s_i x b_i: a predictor
  s~ = s + ((s + s~)/2) x b(s), then s' = s + ((s + s')/2) x b((s + s~)/2),
  each an exact rotation; the same noise in both stages.
* Noise: chi = L eta with L L^T = W (Cholesky, lower triangular); alpha = 0 uses
  the exact rank-one factor L[:, 0] = sqrt(w); alpha = inf uses sqrt(w) I.
  Per step the increments are sqrt(Gamma dt) xi_hat (collective, one per
  trajectory and component) and sqrt(dt) (L eta_hat)_i, with xi_hat, eta_hat
  standard normals drawn from Philox4x32-10.
* Random stream: Philox4x32-10 (Salmon et al., SC'11) with key (seed low word,
  seed high word) and counter (trajectory m, step t, site i, stream). Stream 0,
  i < N: pump noise eta_i; i = N: collective noise xi. Stream 1, t = 0: the
  initial signs. Two 53-bit uniforms per call, u = (k + 1/2) 2^-53, then
  Box-Muller: r = sqrt(-2 ln u1), (r cos 2 pi u2, r sin 2 pi u2) -> (x, y).
* Initial s^z is a parameter (+1 excited as in the paper, -1 ground).
* Window: the state after completed step t (time t dt) is one sample when
  t > round(t0 / dt), t0 the window start, and (t - round(t0 / dt)) is a
  multiple of the sample stride (1: every step); each trajectory's window mean
  is one sample of the ensemble; g2 is the ratio of ensemble means with a
  block-jackknife standard error.
"""
import math

import numpy as np

__all__ = [
    "philox4x32_10", "philox_normals", "initial_signs",
    "pump_matrix", "noise_factor", "spectrum",
    "TWAOracle", "observables_from_moments",
]

_MASK32 = np.uint64(0xFFFFFFFF)
# Philox4x32 multipliers and Weyl key increments (Salmon et al., SC'11, Sec. 5).
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on arrays of 32-bit words (held as uint64).

    One round maps (c0, c1, c2, c3) under key (k0, k1) to
    (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0));
    the key gains (W0, W1) between rounds.
    """
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & _MASK32 for v in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK32
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK32
    for r in range(10):
        if r > 0:
            k0 = (k0 + _W0) & _MASK32
            k1 = (k1 + _W1) & _MASK32
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def _key(seed):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.uint64(seed & 0xFFFFFFFF), np.uint64(seed >> 32)


def _uniform53(hi, lo):
    """(k + 1/2) 2^-53 with k the top 53 bits of the 64-bit word hi:lo; in (0, 1)."""
    k = ((hi << np.uint64(32)) | lo) >> np.uint64(11)
    return (k.astype(np.float64) + 0.5) * 2.0 ** -53


def philox_normals(seed, m, t, i, stream=0):
    """Two independent standard normals per counter (m, t, i, stream)."""
    k0, k1 = _key(seed)
    w0, w1, w2, w3 = philox4x32_10(m, t, i, stream, k0, k1)
    u1 = _uniform53(w0, w1)
    u2 = _uniform53(w2, w3)
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)


def initial_signs(seed, m, i):
    """Discrete-Wigner signs (Sec. S1, item 3): s^x, s^y = +-1 from the low bits
    of Philox words 0 and 1 at counter (m, 0, i, 1)."""
    k0, k1 = _key(seed)
    w0, w1, _, _ = philox4x32_10(m, 0, i, 1, k0, k1)
    sx = np.where((w0 & np.uint64(1)) == 1, 1.0, -1.0)
    sy = np.where((w1 & np.uint64(1)) == 1, 1.0, -1.0)
    return sx, sy


def pump_matrix(N, alpha, w):
    """Eq. (2): w_ij = w / (|i-j| + 1)^alpha on an open chain of N sites.

    alpha = +inf gives the local pump w delta_ij (the alpha -> inf limit the
    paper names below Eq. (2)); alpha = 0 gives the collective pump w.
    """
    d = np.abs(np.arange(N)[:, None] - np.arange(N)[None, :]).astype(np.float64)
    if math.isinf(alpha):
        return w * np.eye(N)
    return w / np.power(d + 1.0, alpha)


def noise_factor(N, alpha, w):
    """A factor L with L L^T = W for the correlated pump noise chi = L eta.

    Cholesky (lower triangular) for 0 < alpha < inf; the exact rank-one factor
    for the collective pump alpha = 0 (Cholesky breaks down there); sqrt(w) I
    for the local pump alpha = inf; zero for w = 0.
    """
    if w == 0.0:
        return np.zeros((N, N))
    if alpha == 0.0:
        L = np.zeros((N, N))
        L[:, 0] = math.sqrt(w)
        return L
    if math.isinf(alpha):
        return math.sqrt(w) * np.eye(N)
    return np.linalg.cholesky(pump_matrix(N, alpha, w))


def spectrum(N, alpha, w):
    """Largest and smallest eigenvalue of w_ij (the paper's w_max, w_min)."""
    ev = np.linalg.eigvalsh(pump_matrix(N, alpha, w))
    return float(ev[-1]), float(ev[0])


class TWAOracle:
    """Stochastic-Heun (or semi-implicit midpoint) integration of Eq. (S1) for
    trajectories m0 .. m0+M-1.

    State arrays ``sx, sy, sz`` have shape (M, N): row = trajectory, column =
    site. ``t`` counts completed steps; the Philox counter uses the global
    trajectory index and the step index, so a continuation reproduces one
    uninterrupted run exactly.
    """

    def __init__(self, N, alpha, w, Gamma, dt, seed, M, m0=0, init_sz=-1.0,
                 window_start=0.0, renormalize=True, L=None, W=None, sample_stride=1, integrator="heun"):
        self.N, self.alpha, self.w, self.Gamma, self.dt = int(N), float(alpha), float(w), float(Gamma), float(dt)
        self.seed, self.M, self.m0 = int(seed), int(M), int(m0)
        self.window_start = float(window_start)
        # samples are taken after completed step t for t > n_w, n_w = round(t0 / dt),
        # every sample_stride-th step: t = n_w + stride, n_w + 2 stride, ...
        self.n_window = int(math.floor(self.window_start / self.dt + 0.5))
        self.sample_stride = max(1, int(sample_stride))
        self.renormalize = bool(renormalize)
        if integrator not in ("heun", "midpoint"):
            raise ValueError("integrator must be 'heun' or 'midpoint'")
        self.integrator = integrator
        self.W = pump_matrix(self.N, self.alpha, self.w) if W is None else np.asarray(W, dtype=np.float64)
        self.L = noise_factor(self.N, self.alpha, self.w) if L is None else np.asarray(L, dtype=np.float64)
        mm = (self.m0 + np.arange(self.M, dtype=np.uint64))[:, None]
        ii = np.arange(self.N, dtype=np.uint64)[None, :]
        self.sx, self.sy = initial_signs(self.seed, mm, ii)
        self.sz = np.full((self.M, self.N), float(init_sz))
        self.t = 0
        # per-trajectory window sums of S^z, A, A^2, A S^z, (S^z)^2 and the count
        self.mom = np.zeros((self.M, 5))
        self.count = 0

    # -- noise of step t ---------------------------------------------------
    def noise(self, t):
        """(xi_x, xi_y) of shape (M,) and (eta_x, eta_y) of shape (M, N)."""
        mm = (self.m0 + np.arange(self.M, dtype=np.uint64))[:, None]
        ii = np.arange(self.N + 1, dtype=np.uint64)[None, :]
        gx, gy = philox_normals(self.seed, mm, np.uint64(t), ii, 0)
        return gx[:, self.N], gy[:, self.N], gx[:, : self.N], gy[:, : self.N]

    # -- right-hand side of Eq. (S1) over one step -------------------------
    def increment(self, sx, sy, sz, dxi_x, dxi_y, dchi_x, dchi_y):
        """Increment of (s^x, s^y, s^z) over dt, term by term as in Eq. (S1).

        dxi_a = xi^a dt (collective, shape (M, 1)); dchi_a = chi_i^a dt (M, N).
        """
        G, dt = self.Gamma, self.dt
        Sx = sx.sum(axis=1, keepdims=True)          # sum_j s^x_j
        Sy = sy.sum(axis=1, keepdims=True)
        Px = sx @ self.W.T                           # sum_j w_ij s^x_j
        Py = sy @ self.W.T
        dx = (0.5 * G * sz * Sx - 0.5 * sz * Px) * dt + dxi_x * sz - dchi_x * sz
        dy = (0.5 * G * sz * Sy - 0.5 * sz * Py) * dt + dxi_y * sz - dchi_y * sz
        dz = (-0.5 * G * (sx * Sx + sy * Sy) + 0.5 * (sx * Px + sy * Py)) * dt \
            - (dxi_x * sx + dxi_y * sy) + (dchi_x * sx + dchi_y * sy)
        return dx, dy, dz

    def field(self, sx, sy, sz, dxi_x, dxi_y, dchi_x, dchi_y):
        """Effective field of Sec. S1 integrated over dt, b_i = (B^y_i, -B^x_i, 0),
        so that the increment of Eq. (S1) is s_i x b_i, with
        B^a_i = 1/2 (Gamma S^a - sum_j w_ij s^a_j) dt + xi^a dt - chi_i^a dt."""
        G, dt = self.Gamma, self.dt
        Bx = 0.5 * (G * sx.sum(axis=1, keepdims=True) - sx @ self.W.T) * dt + dxi_x - dchi_x
        By = 0.5 * (G * sy.sum(axis=1, keepdims=True) - sy @ self.W.T) * dt + dxi_y - dchi_y
        return By, -Bx, np.zeros_like(Bx)

    @staticmethod
    def cayley(sx, sy, sz, bx, by, bz):
        """The s' solving s' = s + ((s + s') / 2) x b for every spin.

        With K the cross-product matrix of b (K v = b x v, so v x b = -K v) the
        equation is (I + K/2) s' = (I - K/2) s, solved spin by spin."""
        b = np.stack(np.broadcast_arrays(bx, by, bz), axis=-1)
        K = np.zeros(b.shape + (3,))
        K[..., 0, 1], K[..., 0, 2] = -b[..., 2], b[..., 1]
        K[..., 1, 0], K[..., 1, 2] = b[..., 2], -b[..., 0]
        K[..., 2, 0], K[..., 2, 1] = -b[..., 1], b[..., 0]
        eye = np.eye(3)
        v = np.stack(np.broadcast_arrays(sx, sy, sz), axis=-1)[..., None]
        out = np.linalg.solve(eye + 0.5 * K, (eye - 0.5 * K) @ v)[..., 0]
        return out[..., 0], out[..., 1], out[..., 2]

    def noise_increments(self, t):
        """Integrated noises of step t: xi^a dt with variance Gamma dt (one per
        trajectory and component, shape (M, 1)) and chi_i^a dt = sqrt(dt) (L eta^a)_i
        with covariance w_ij dt (shape (M, N))."""
        xi_x, xi_y, eta_x, eta_y = self.noise(t)
        sg = math.sqrt(self.Gamma * self.dt)
        sd = math.sqrt(self.dt)
        dxi_x, dxi_y = sg * xi_x[:, None], sg * xi_y[:, None]
        dchi_x = sd * (eta_x @ self.L.T)
        dchi_y = sd * (eta_y @ self.L.T)
        return dxi_x, dxi_y, dchi_x, dchi_y

    def step(self):
        t = self.t
        dxi_x, dxi_y, dchi_x, dchi_y = self.noise_increments(t)
        sx, sy, sz = self.sx, self.sy, self.sz
        if self.integrator == "heun":
            fx, fy, fz = self.increment(sx, sy, sz, dxi_x, dxi_y, dchi_x, dchi_y)
            px, py, pz = sx + fx, sy + fy, sz + fz        # predictor
            gx, gy, gz = self.increment(px, py, pz, dxi_x, dxi_y, dchi_x, dchi_y)
            nx, ny, nz = sx + 0.5 * (fx + gx), sy + 0.5 * (fy + gy), sz + 0.5 * (fz + gz)
        else:
            # semi-implicit midpoint: predictor with the field at s, corrector with
            # the field at the midpoint of s and the predictor
            b0 = self.field(sx, sy, sz, dxi_x, dxi_y, dchi_x, dchi_y)
            px, py, pz = self.cayley(sx, sy, sz, *b0)
            b1 = self.field(0.5 * (sx + px), 0.5 * (sy + py), 0.5 * (sz + pz), dxi_x, dxi_y, dchi_x, dchi_y)
            nx, ny, nz = self.cayley(sx, sy, sz, *b1)
        if self.renormalize:
            scale = math.sqrt(3.0) / np.sqrt(nx * nx + ny * ny + nz * nz)
            nx, ny, nz = nx * scale, ny * scale, nz * scale
        self.sx, self.sy, self.sz = nx, ny, nz
        self.t = t + 1
        if self.t > self.n_window and (self.t - self.n_window) % self.sample_stride == 0:
            self.accumulate()

    def accumulate(self):
        """Window sums of the classical collective moments (Sec. S1, items 5-6)."""
        Sx, Sy, Sz = self.sx.sum(1), self.sy.sum(1), self.sz.sum(1)
        A = 0.25 * (Sx * Sx + Sy * Sy)               # classical S+S- = |S^x + i S^y|^2 / 4
        self.mom += np.stack([Sz, A, A * A, A * Sz, Sz * Sz], axis=1)
        self.count += 1

    def run(self, steps):
        for _ in range(int(steps)):
            self.step()
        return self

    def window_means(self):
        """Per-trajectory window means, shape (M, 5): S^z, A, A^2, A S^z, (S^z)^2."""
        if self.count == 0:
            raise ValueError("no step inside the averaging window yet")
        return self.mom / self.count

    def observables(self):
        return observables_from_moments(self.window_means(), self.N)


def _g2_parts(means):
    """Normal-ordered moments from the symmetric-ordered ones (Sec. S1, item 6)."""
    Sz, A, A2, ASz, Sz2 = means
    spsm = A + 0.5 * Sz
    g2num = A2 + 2.0 * ASz - Sz / 3.0 + 0.5 * Sz2 - 4.0 / 3.0 * A
    return spsm, g2num


def observables_from_moments(samples, N, blocks=32):
    """Ensemble means and standard errors from per-trajectory window means.

    samples: (M, 5) array of per-trajectory window means of
    (S^z, A, A^2, A S^z, (S^z)^2) with A = ((S^x)^2 + (S^y)^2) / 4.
    Returns a dict of value and SE for Sz, sigma_z, SpSm, G2num (the normal-
    ordered <S+S+S-S->) and g2 (ratio of means; block-jackknife SE).
    """
    samples = np.asarray(samples, dtype=np.float64)
    M = samples.shape[0]
    spsm_s, g2n_s = _g2_parts(samples.T)

    def mean_se(x):
        se = float(np.std(x, ddof=1) / math.sqrt(M)) if M > 1 else float("nan")
        return float(np.mean(x)), se

    out = {}
    out["Sz"], out["Sz_se"] = mean_se(samples[:, 0])
    out["sigma_z"], out["sigma_z_se"] = out["Sz"] / N, out["Sz_se"] / N
    out["SpSm"], out["SpSm_se"] = mean_se(spsm_s)
    out["G2num"], out["G2num_se"] = mean_se(g2n_s)
    mu = samples.mean(axis=0)
    spsm, g2n = _g2_parts(mu)
    out["g2"] = float(g2n / (spsm * spsm))
    B = min(int(blocks), M)
    if B >= 2:
        edges = np.array([(b * M) // B for b in range(B + 1)])
        sums = np.stack([samples[edges[b]:edges[b + 1]].sum(axis=0) for b in range(B)])
        cnts = np.diff(edges).astype(np.float64)
        tot = sums.sum(axis=0)
        est = []
        for b in range(B):
            m_b = (tot - sums[b]) / (M - cnts[b])
            s_b, g_b = _g2_parts(m_b)
            est.append(g_b / (s_b * s_b))
        est = np.asarray(est)
        out["g2_se"] = float(math.sqrt((B - 1) / B * np.sum((est - est.mean()) ** 2)))
    else:
        out["g2_se"] = float("nan")
    return out
