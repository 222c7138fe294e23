"""The Toeplitz/FFT route for the pump field, through the C ABI.

The route computes sum_j w_ij s_j as a circulant-embedding convolution in FP32.
A mixed-radix FFT of length P in FP32 has a relative 2-norm error of order
log2(P) * 2^-24 (a few 1e-7 at P = 2e4); the convolution is one forward and one
inverse transform, and the spectrum lambda is rounded to FP32 once. The tests
use 2e-6 on the relative Frobenius error and 5e-6 of the largest entry
elementwise, an order of magnitude above that estimate and well below the
BF16X3 contraction's 3 * 2^-18.
"""
import math

import numpy as np
import pytest

from oracle.twa_oracle import TWAOracle, pump_matrix

pytestmark = pytest.mark.gpu


def _twa():
    from paper_2608_10075_b300 import twa
    return twa


@pytest.mark.parametrize("N,K,alpha", [(1, 3, 1.0), (7, 5, 0.5), (37, 8, 1.3), (300, 33, 1.0), (1024, 16, 2.0),
                                       (4999, 6, 0.25)])
def test_fft_field_matches_definition(N, K, alpha):
    import torch
    twa = _twa()
    rng = np.random.default_rng(N)
    s = rng.normal(size=(K, N))
    W = pump_matrix(N, alpha, N / 2.0)
    with twa.TWA(N, alpha, N / 2.0, 1.0, 1e-4, precision="bf16x3", ws_route="fft") as g:
        P = g.field(torch.tensor(s, device="cuda")).cpu().numpy()
    ref = s @ W.T
    assert np.linalg.norm(P - ref) <= 2e-6 * np.linalg.norm(ref)
    assert np.max(np.abs(P - ref)) <= 5e-6 * np.max(np.abs(ref))


def test_fft_field_full_size_sampled():
    import torch
    twa = _twa()
    N, K = 10000, 4
    rng = np.random.default_rng(9)
    s = rng.choice([-1.0, 1.0], size=(K, N))
    with twa.TWA(N, 1.0, 5000.0, 1.0, 2e-5, precision="bf16x3", ws_route="fft") as g:
        P = g.field(torch.tensor(s, device="cuda")).cpu().numpy()
    d = np.arange(N)
    for i in (0, 1, 5000, 9998, 9999):
        wrow = 5000.0 / (np.abs(i - d) + 1.0)
        ref = s @ wrow
        assert np.max(np.abs(P[:, i] - ref)) <= 5e-6 * 5000.0 * np.sum(1.0 / (d + 1.0)), (i, P[:, i], ref)


def test_fft_route_tracks_dense_route():
    # Both routes share the noise (the same BF16 normals and the same L.eta
    # kernel), so trajectories differ only by the contraction error.
    twa = _twa()
    N, M, alpha, w, dt = 300, 64, 1.0, 20.0, 1e-3
    out = {}
    for route in ("dense", "fft"):
        with twa.TWA(N, alpha, w, 1.0, dt, seed=3, precision="bf16x3", ws_route=route) as g:
            g.run(M, 5)
            out[route] = g.get_state()
    err = max(np.max(np.abs(a - b)) for a, b in zip(out["dense"], out["fft"]))
    assert err < 2e-4, err


def test_fft_route_ensemble_within_3se():
    N, alpha, w, G, dt, M, T, t0 = 256, 1.0, 32.0, 1.0, 1e-3, 512, 1.0, 0.5
    steps = int(round(T / dt))
    twa = _twa()
    o = TWAOracle(N, alpha, w, G, dt, 5, M, window_start=t0)
    o.run(steps)
    ob = o.observables()
    with twa.TWA(N, alpha, w, G, dt, seed=5, precision="bf16x3", window_start=t0, ws_route="fft") as g:
        g.run(M, steps)
        gb = g.observables()
    assert gb["samples"] == o.count
    for k in ("Sz", "SpSm", "G2num", "g2"):
        assert abs(gb[k] - ob[k]) <= 3.0 * math.hypot(gb[k + "_se"], ob[k + "_se"]), (k, gb[k], ob[k])


def test_fft_route_full_size_runs():
    # N = 10^4, M = 1024 (the benchmark's shape) on the FFT route: spins stay on
    # their sphere and the sampled trajectory follows the dense route closely.
    twa = _twa()
    N, alpha, w, G, dt, M = 10000, 1.0, 5000.0, 1.0, 2e-5, 1024
    st = {}
    for route in ("fft", "dense"):
        with twa.TWA(N, alpha, w, G, dt, seed=0, precision="bf16x3", ws_route=route) as g:
            g.run(M, 3)
            st[route] = g.get_state()
    x, y, z = st["fft"]
    assert np.max(np.abs(x * x + y * y + z * z - 3.0)) < 5e-6
    for m in (0, 511, 1023):
        err = max(np.max(np.abs(a[m] - b[m])) for a, b in zip(st["fft"], st["dense"]))
        assert err < 1e-3, (m, err)


def test_fft_route_rejects_what_it_cannot_do(monkeypatch):
    twa = _twa()
    with pytest.raises(twa.TWAError) as e:
        twa.TWA(64, 1.0, 1.0, 1.0, 1e-4, precision="fp64", ws_route="fft")
    assert e.value.name == "TWA_EUNSUPPORTED"
    monkeypatch.setenv("TWA_FFT_CLUSTER", "3")
    with pytest.raises(twa.TWAError) as e:
        twa.TWA(64, 1.0, 1.0, 1.0, 1e-4, precision="bf16x3", ws_route="fft")
    assert e.value.name == "TWA_EINVAL"


@pytest.mark.parametrize("noise", ["cholesky", "circulant"])
@pytest.mark.parametrize("N", [300, 1000, 4999, 10000])
def test_warp_local_stages_give_the_same_bits(monkeypatch, N, noise):
    # the later stages of the one-CTA transform run warp by warp (each warp owns
    # whole sub-transforms): the same butterflies as the block-wide mapping
    import torch
    twa = _twa()
    rng = np.random.default_rng(N)
    s = torch.tensor(rng.normal(size=(3, N)), device="cuda")
    out = {}
    for warp in ("1", "0"):
        monkeypatch.setenv("TWA_FFT_WARP", warp)
        with twa.TWA(N, 1.0, N / 2.0, 1.0, 2e-5, seed=2, precision="bf16x2", ws_route="fft",
                     noise_route=noise) as g:
            f = g.field(s).cpu().numpy()
            g.run(16, 4)
            out[warp] = (f, g.get_state())
    assert np.array_equal(out["1"][0], out["0"][0])
    for u, v in zip(out["1"][1], out["0"][1]):
        assert np.array_equal(u, v)


# ---------------------------------------------------------------------------
# transforms longer than one CTA's shared memory (P > 28000, N > 14001): one
# thread-block cluster of 2, 4 or 8 CTAs per trajectory, the transform spread
# over their shared memories

def _toeplitz_reference(s, alpha, w):
    """sum_j w / (1 + |i - j|)^alpha s_j for each row of s, in FP64 by a
    zero-padded numpy FFT (exact linear convolution up to FP64 rounding)."""
    K, N = s.shape
    d = np.arange(-(N - 1), N, dtype=np.float64)
    k = w / np.power(np.abs(d) + 1.0, alpha)
    n = 1 << int(math.ceil(math.log2(3 * N)))
    S = np.fft.rfft(s, n=n, axis=1)
    Kf = np.fft.rfft(k, n=n)
    full = np.fft.irfft(S * Kf[None, :], n=n, axis=1)
    return full[:, N - 1:2 * N - 1]


def _circle(g, M=2):
    """(P, CTAs per trajectory) the context reports after a one-step run."""
    g.run(M, 1)
    ob = g.observables()
    return ob["fft_length"], ob["fft_ctas"]


def test_toeplitz_reference_is_the_dense_product():
    rng = np.random.default_rng(1)
    s = rng.normal(size=(3, 301))
    W = pump_matrix(301, 0.7, 5.0)
    assert np.allclose(_toeplitz_reference(s, 0.7, 5.0), s @ W.T, rtol=0, atol=1e-11 * np.abs(s @ W.T).max())


@pytest.mark.parametrize("N,alpha,ctas", [(14002, 1.0, 2), (20000, 0.5, 2), (30001, 1.0, 4), (56002, 2.0, 8)])
def test_cluster_fft_field_matches_definition(N, alpha, ctas):
    import torch
    twa = _twa()
    K = 3
    rng = np.random.default_rng(N)
    s = rng.normal(size=(K, N))
    with twa.TWA(N, alpha, N / 2.0, 1.0, 1e-6, precision="bf16x3", ws_route="fft") as g:
        P = g.field(torch.tensor(s, device="cuda")).cpu().numpy()
        plen, c = _circle(g)
    assert c == ctas and plen % (4 * ctas) == 0 and plen >= 2 * N - 2 and plen // ctas <= 28000
    ref = _toeplitz_reference(s, alpha, N / 2.0)
    assert np.linalg.norm(P - ref) <= 2e-6 * np.linalg.norm(ref)
    assert np.max(np.abs(P - ref)) <= 5e-6 * np.max(np.abs(ref))


@pytest.mark.parametrize("ctas", [2, 4, 8])
@pytest.mark.parametrize("N", [3, 37, 1000, 10000])
def test_forced_cluster_fft_field_matches_definition(monkeypatch, N, ctas):
    # the cluster form on transforms that would fit one CTA: the stages whose
    # stride C does not divide run through the other CTAs' shared memory
    import torch
    monkeypatch.setenv("TWA_FFT_CLUSTER", str(ctas))
    twa = _twa()
    K, alpha = 5, 1.3
    rng = np.random.default_rng(N + ctas)
    s = rng.normal(size=(K, N))
    with twa.TWA(N, alpha, N / 2.0, 1.0, 1e-6, precision="bf16x3", ws_route="fft") as g:
        P = g.field(torch.tensor(s, device="cuda")).cpu().numpy()
        plen, c = _circle(g)
    assert c == ctas and plen % (4 * ctas) == 0
    ref = _toeplitz_reference(s, alpha, N / 2.0)
    assert np.linalg.norm(P - ref) <= 2e-6 * np.linalg.norm(ref)
    assert np.max(np.abs(P - ref)) <= 5e-6 * np.max(np.abs(ref))


@pytest.mark.parametrize("integrator", ["heun", "midpoint"])
def test_cluster_fft_route_tracks_one_cta(monkeypatch, integrator):
    # N = 300 on clusters of 2, 4, 8 against one CTA per trajectory: both draw
    # the same noise (dense L.eta), so trajectories differ by the transform's
    # FP32 rounding only; moments and observables come out the same
    twa = _twa()
    N, M, alpha, w, dt, steps = 300, 40, 1.0, 20.0, 1e-3, 6
    out = {}
    for ctas in (1, 2, 4, 8):
        monkeypatch.setenv("TWA_FFT_CLUSTER", str(ctas))
        with twa.TWA(N, alpha, w, 1.0, dt, seed=3, precision="bf16x3", ws_route="fft", integrator=integrator) as g:
            g.run(M, steps)
            out[ctas] = (g.get_state(), g.observables())
    for ctas in (2, 4, 8):
        err = max(np.max(np.abs(a - b)) for a, b in zip(out[1][0], out[ctas][0]))
        assert err < 2e-5, (ctas, err)
        assert out[ctas][1]["fft_ctas"] == ctas
        for k in ("Sz", "SpSm", "g2"):
            assert abs(out[ctas][1][k] - out[1][1][k]) <= 1e-4 * abs(out[1][1][k]), (ctas, k)


def test_cluster_fft_route_tracks_dense_route_at_n20000():
    twa = _twa()
    N, alpha, w, G, dt, M, steps = 20000, 1.0, 10000.0, 1.0, 1e-5, 8, 3
    st = {}
    for route in ("fft", "dense"):
        with twa.TWA(N, alpha, w, G, dt, seed=0, precision="bf16x3", ws_route=route) as g:
            g.run(M, steps)
            st[route] = g.get_state()
            if route == "fft":
                assert g.observables()["fft_ctas"] == 2
    x, y, z = st["fft"]
    assert np.max(np.abs(x * x + y * y + z * z - 3.0)) < 5e-6
    err = max(np.max(np.abs(a - b)) for a, b in zip(st["fft"], st["dense"]))
    assert err < 1e-3, err


def test_cluster_circulant_route_tracks_its_oracle():
    # N = 15000 (P = 30000 on clusters of two): every step FFT-only; trajectories
    # 0 and 5 against the oracle on the circle length the library reports
    from oracle.circulant import TWAOracleCirculant
    twa = _twa()
    N, alpha, w, G, dt, M, steps = 15000, 1.0, 7500.0, 1.0, 2e-5, 6, 2
    with twa.TWA(N, alpha, w, G, dt, seed=0, precision="bf16x3", ws_route="fft", noise_route="circulant") as g:
        g.run(M, steps)
        x, y, z = g.get_state()
        ob = g.observables()
    assert ob["fft_ctas"] == 2 and ob["fft_length"] % 8 == 0
    assert np.max(np.abs(x * x + y * y + z * z - 3.0)) < 5e-6
    for m in (0, 5):
        o = TWAOracleCirculant(N, alpha, w, G, dt, 0, 1, m0=m, P=ob["fft_length"])
        o.run(steps)
        err = max(np.max(np.abs(a[m] - b[0])) for a, b in zip((x, y, z), (o.sx, o.sy, o.sz)))
        assert err < 5e-5, (m, err)


# ---------------------------------------------------------------------------
# circulant-embedding noise draw (fully FFT step)
#
# The step is then FP32 throughout: the FFT convolution (relative error a few
# 1e-7) and the FP32 Box-Muller normals of the same Philox words the oracle turns
# into FP64 normals (32-bit against 53-bit uniforms: relative 1e-7). Over a few
# steps each spin component moves by O(sqrt(w dt)) per step, so a per-trajectory
# difference of 5e-5 is two orders above the expected 1e-7 .. 1e-6 and far
# below what any wrong frequency, scale or sign of the draw would give (O(1)).

@pytest.mark.parametrize("N,M,alpha,w,steps", [(300, 48, 1.0, 20.0, 4), (37, 20, 0.5, 4.0, 6), (38, 9, 2.0, 10.0, 3),
                                               (1, 6, 1.0, 2.0, 5), (200, 16, math.inf, 8.0, 3),
                                               (128, 16, 0.0, 3.0, 3)])
def test_circulant_route_tracks_its_oracle(N, M, alpha, w, steps):
    from oracle.circulant import TWAOracleCirculant
    twa = _twa()
    dt = 1e-3
    o = TWAOracleCirculant(N, alpha, w, 1.0, dt, 7, M)
    o.run(steps)
    with twa.TWA(N, alpha, w, 1.0, dt, seed=7, precision="bf16x3", ws_route="fft", noise_route="circulant") as g:
        g.run(M, steps)
        x, y, z = g.get_state()
    # (alpha = 0: all but one eigenvalue of the embedding vanish, and their FP64
    # rounding, different on the two sides, enters through sqrt: ~1e-7 here)
    tol = 5e-5
    for a, b in zip((x, y, z), (o.sx, o.sy, o.sz)):
        assert np.max(np.abs(a - b)) < tol, np.max(np.abs(a - b))


def test_circulant_route_ensemble_matches_the_cholesky_law():
    # same law as chi = L eta: observables agree with the Cholesky oracle within 3 SE
    N, alpha, w, G, dt, M, T, t0 = 256, 1.0, 32.0, 1.0, 1e-3, 512, 1.0, 0.5
    steps = int(round(T / dt))
    twa = _twa()
    o = TWAOracle(N, alpha, w, G, dt, 5, M, window_start=t0)
    o.run(steps)
    ob = o.observables()
    with twa.TWA(N, alpha, w, G, dt, seed=5, precision="bf16x3", window_start=t0, ws_route="fft",
                 noise_route="circulant") as g:
        g.run(M, steps)
        gb = g.observables()
    for k in ("Sz", "SpSm", "G2num", "g2"):
        assert abs(gb[k] - ob[k]) <= 3.0 * math.hypot(gb[k + "_se"], ob[k + "_se"]), (k, gb[k], ob[k])


def test_circulant_route_full_size_sampled():
    # N = 10^4, M = 1024 (the benchmark's shape): trajectories 0 and 1023 against
    # the oracle run on those two trajectories alone
    from oracle.circulant import TWAOracleCirculant
    twa = _twa()
    N, alpha, w, G, dt, M, steps = 10000, 1.0, 5000.0, 1.0, 2e-5, 1024, 2
    with twa.TWA(N, alpha, w, G, dt, seed=0, precision="bf16x3", ws_route="fft", noise_route="circulant") as g:
        g.run(M, steps)
        x, y, z = g.get_state()
    assert np.max(np.abs(x * x + y * y + z * z - 3.0)) < 5e-6
    for m in (0, 1023):
        o = TWAOracleCirculant(N, alpha, w, G, dt, 0, 1, m0=m)
        o.run(steps)
        err = max(np.max(np.abs(a[m] - b[0])) for a, b in zip((x, y, z), (o.sx, o.sy, o.sz)))
        assert err < 5e-5, (m, err)


def test_circulant_route_launches_no_contraction():
    twa = _twa()
    with twa.TWA(300, 1.0, 20.0, 1.0, 1e-3, precision="bf16x3", ws_route="fft", noise_route="circulant") as g:
        g.run(64, 1)
        g.profile(True)
        g.run(64, 3)
        p = g.profile_read()
        g.profile(False)
    assert p["noise"][1] == 3 and p["predict"][1] == 3 and p["correct"][1] == 3
    assert p["noise_factor"][1] == 0


def test_circulant_route_rejects_the_adjoint():
    twa = _twa()
    with twa.TWA(64, 1.0, 8.0, 1.0, 1e-3, precision="bf16x3", ws_route="fft", noise_route="circulant") as g:
        with pytest.raises(twa.TWAError) as e:
            g.grad("SpSm", M=8, steps=4)
    assert e.value.name == "TWA_EUNSUPPORTED"
