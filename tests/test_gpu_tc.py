"""Parity of the mixed-precision tensor-core path (tcgen05, BF16 operands, FP32
accumulation and state) with the FP64 CPU oracle, through the C ABI.

Contraction bound. Write v = hi + lo + r with hi = bf16(v), lo = bf16(v - hi):
|hi - v| <= 2^-9 |v| and |r| <= 2^-9 |v - hi| <= 2^-18 |v|. The three-term
product hi_w hi_s + hi_w lo_s + lo_w hi_s misses lo_w lo_s and the residuals,
so each product w s is off by at most ~3 * 2^-18 |w s| (plus 2^-24 from the
FP32 rounding of W), and the FP32 sum over N terms adds N 2^-24 sum |w s| in
the worst case. Single-term BF16 is off by ~2 * 2^-9 |w s| per product, and
the TF32 mode (operands rounded to nearest TF32, 2^-11 relative, products
exact and summed in FP32) by ~2 * 2^-11 |w s|. The FP32 mode is BF16X3's split
with TF32 halves: residual and dropped lo*lo term 2^-22 each, so ~3 * 2^-22
|w s| per product. The tests use these bounds with a factor of two of margin.

Trajectories. The mixed path rounds its normals to BF16 (relative 2^-9), so a
trajectory only stays close to the plain oracle's for a few steps; beyond that
the comparison is statistical: ensemble observables within 3 standard errors.
The BF16X3 trajectories are checked against the oracle run on the same
BF16-rounded normals, within the term-by-term bound of tests/mixed_bounds.py
(~2^-17 of the noise and field sums per step, plus the few normals that sit at
a BF16 rounding boundary), which a dropped lo image of L exceeds.
"""
import math

import numpy as np
import pytest

from oracle.twa_oracle import TWAOracle, noise_factor, pump_matrix
from tests.mixed_bounds import BF16NoiseOracle, bf16, track

pytestmark = pytest.mark.gpu


def _twa():
    from paper_2608_10075_b300 import twa
    return twa


def _field_check(prec, N, K, alpha, w, seed=2):
    import torch
    twa = _twa()
    rng = np.random.default_rng(seed)
    s = rng.choice([-1.0, 1.0], size=(K, N)) * rng.uniform(0.2, 1.7, size=(K, N))
    if prec in ("bf16x2", "bf16l2", "bf16b"):
        # these precisions round the operand once to BF16: give it exact BF16 values,
        # so that the check is of the W representation and the accumulation
        s = bf16(s)
    W = pump_matrix(N, alpha, w)
    with twa.TWA(N, alpha, w, 1.0, 1e-4, precision=prec) as g:
        P = g.field(torch.tensor(s, device="cuda")).cpu().numpy()
    ref = s @ W.T
    absref = np.abs(s) @ np.abs(W).T
    if prec == "bf16x3":
        bound = 2.0 * (3 * 2.0 ** -18 + 2.0 ** -24 + N * 2.0 ** -24) * absref
    elif prec == "tf32":
        bound = 2.0 * (2 * 2.0 ** -11 + N * 2.0 ** -24) * absref
    elif prec == "fp32":
        bound = 2.0 * (3 * 2.0 ** -22 + 2.0 ** -24 + N * 2.0 ** -24) * absref
    elif prec == "bf16x2":
        bound = 2.0 * (2.0 ** -18 + 2.0 ** -24 + N * 2.0 ** -24) * absref
    else:
        bound = 2.0 * (2 * 2.0 ** -9 + N * 2.0 ** -24) * absref
    err = np.abs(P - ref)
    assert np.all(err <= bound + 1e-30), float(np.max(err / absref))
    return float(np.max(err / absref))


@pytest.mark.parametrize("prec", ["bf16x3", "bf16", "tf32", "fp32", "bf16x2", "bf16l2", "bf16b"])
@pytest.mark.parametrize("N,K", [(16, 8), (300, 600), (129, 257), (1024, 512)])
def test_field_contraction_bound(prec, N, K):
    # several 128-site row tiles and 256-row column tiles, with ragged tails
    _field_check(prec, N, K, 1.0, N / 2.0)


def test_field_bf16x3_is_much_better_than_bf16():
    e3 = _field_check("bf16x3", 300, 256, 0.5, 150.0)
    et = _field_check("tf32", 300, 256, 0.5, 150.0)
    e1 = _field_check("bf16", 300, 256, 0.5, 150.0)
    assert e3 < e1 / 50
    assert e3 < et < e1   # 16, 11 and 8 significant bits


def test_fp32_mode_resolves_22_bits():
    # alpha = inf: W = w I, so every output is one product w s and the sum adds
    # only exact zeros; w = 150 is exact in every format. The FP32 split keeps
    # s to 2^-22 (+ 2^-24 from FP64 -> FP32 and the accumulator's rounding),
    # the BF16 split only to 2^-18.
    import torch
    twa = _twa()
    N, K, w = 300, 600, 150.0
    rng = np.random.default_rng(9)
    s = rng.choice([-1.0, 1.0], size=(K, N)) * rng.uniform(0.2, 1.7, size=(K, N))
    err = {}
    for prec in ("fp32", "bf16x3"):
        with twa.TWA(N, math.inf, w, 1.0, 1e-4, precision=prec) as g:
            P = g.field(torch.tensor(s, device="cuda")).cpu().numpy()
        err[prec] = float(np.max(np.abs(P - w * s) / np.abs(w * s)))
    assert err["fp32"] <= 2.0 * (2.0 ** -22 + 2.0 ** -23 + 2.0 ** -24), err
    assert err["bf16x3"] > 2.0 * err["fp32"], err


@pytest.mark.parametrize("prec", ["bf16x3", "bf16", "tf32", "fp32"])
def test_initial_state_is_exact(prec):
    twa = _twa()
    N, M = 300, 200
    o = TWAOracle(N, 1.0, 10.0, 1.0, 1e-3, 7, M, init_sz=1.0)
    with twa.TWA(N, 1.0, 10.0, 1.0, 1e-3, seed=7, precision=prec, init_state=1) as g:
        g.run(M, 0)
        gx, gy, gz = g.get_state()
    assert np.array_equal(gx, o.sx) and np.array_equal(gy, o.sy) and np.array_equal(gz, o.sz)


def _leta_bound(prec, N, absref):
    """Bound of |L.eta - kernel| for eta exactly representable in BF16 (so the
    kernel's noise operand is eta itself): the L representation error of the
    precision (BF16X3: hi + lo leaves 2^-18 after the FP32 image's 2^-24; one
    BF16 term 2^-9; TF32 2^-11; the FP32 split 2^-22) plus FP32 accumulation in
    N/16 instruction steps, with a factor of two of margin."""
    rep = {"bf16x3": 2.0 ** -18 + 2.0 ** -24, "bf16": 2.0 ** -9, "tf32": 2.0 ** -11,
           "fp32": 2.0 ** -22 + 2.0 ** -24, "bf16x2": 2.0 ** -18 + 2.0 ** -24,
           "bf16l2": 2.0 ** -18 + 2.0 ** -24, "bf16b": 2.0 ** -9}[prec]
    return 2.0 * (rep + (N / 16.0) * 2.0 ** -22) * absref


@pytest.mark.parametrize("prec", ["bf16x3", "bf16", "tf32", "fp32", "bf16x2", "bf16l2", "bf16b"])
@pytest.mark.parametrize("N,K", [(16, 8), (300, 600), (129, 257), (1024, 512)])
def test_noise_factor_contraction_bound(prec, N, K):
    # the step's L.eta arithmetic alone (twa_contract, matrix L): BF16X3 takes L
    # hi + lo against the noise rounded once to BF16 (two products)
    import torch
    twa = _twa()
    rng = np.random.default_rng(4)
    eta = bf16(rng.standard_normal((K, N)))
    L = noise_factor(N, 1.0, N / 2.0)
    with twa.TWA(N, 1.0, N / 2.0, 1.0, 1e-4, precision=prec) as g:
        P = g.contract(torch.tensor(eta, device="cuda"), matrix="L").cpu().numpy()
    ref = eta @ L.T
    absref = np.abs(eta) @ np.abs(L).T
    bound = _leta_bound(prec, N, absref)
    err = np.abs(P - ref)
    assert np.all(err <= bound + 1e-30), float(np.max(err / (absref + 1e-300)))
    if prec in ("bf16x3", "bf16x2", "bf16l2"):
        # the bound resolves the lo image: L hi alone (a dropped lo term) breaks it
        planted = eta @ bf16(L).T
        assert np.mean(np.abs(planted - ref) > bound) > 0.1


@pytest.mark.parametrize("prec,matrix", [("bf16l2", "W"), ("bf16b", "W"), ("bf16b", "L"), ("bf16l2", "L")])
def test_two_products_exactly_on_the_band(prec, matrix):
    # unit vectors as operands (exact in BF16): the contraction returns the
    # columns of W (or L) as the kernel represents them. For rows i in [u, u + 256)
    # (u a multiple of 256) the entries with j in [u - 64, u + 320) -- every entry
    # within 64 of the diagonal -- take hi + lo (~2^-16 relative); every other
    # entry is one BF16 product: the scale times bf16(entry / scale). BF16L2's L
    # is split everywhere.
    import torch
    twa = _twa()
    N, alpha, w = 1024, 1.0, 512.0
    A = pump_matrix(N, alpha, w) if matrix == "W" else noise_factor(N, alpha, w)
    scale = w if matrix == "W" else math.sqrt(w)
    with twa.TWA(N, alpha, w, 1.0, 1e-4, precision=prec) as g:
        eye = torch.eye(N, dtype=torch.float64, device="cuda")
        P = (g.field(eye) if matrix == "W" else g.contract(eye, matrix="L")).cpu().numpy()
    got = P.T                                   # got[i, j]: entry (i, j) as represented
    i = np.arange(N)[:, None]
    j = np.arange(N)[None, :]
    u = (i // 256) * 256
    band = (j >= u - 64) & (j < u + 320)
    if prec == "bf16l2" and matrix == "L":
        band = np.ones_like(band)
    nz = A != 0.0
    rel = np.abs(got - A) / np.where(nz, np.abs(A), 1.0)
    assert np.all(rel[band & nz] <= 2.0 ** -15), float(np.max(rel[band & nz]))
    assert np.all(got[~nz] == 0.0)
    if not np.any(~band & nz):
        return
    one = scale * bf16(A / scale)               # one product: the BF16 image, rescaled
    off = ~band & nz
    assert np.all(np.abs(got[off] - one[off]) <= 2.0 ** -22 * np.abs(one[off])), \
        float(np.max(np.abs(got[off] - one[off]) / np.abs(one[off])))
    assert np.max(rel[off]) > 2.0 ** -12      # and the one-term rounding is really there
    assert np.all(np.abs(i - j)[off] > 64)


def test_noise_factor_contraction_full_size_sampled():
    # N = 10^4, 2 x 1024 noise vectors (the benchmark's launch shape), BF16X3,
    # rows of L recomputed one by one
    import torch
    twa = _twa()
    N, K = 10000, 2048
    rng = np.random.default_rng(5)
    eta = bf16(rng.standard_normal((K, N)))
    with twa.TWA(N, 1.0, 5000.0, 1.0, 2e-5, precision="bf16x3") as g:
        P = g.contract(torch.tensor(eta, device="cuda"), matrix="L").cpu().numpy()
    L = noise_factor(N, 1.0, 5000.0)
    rows = np.array([0, 1, 127, 128, 129, 4999, 5000, 9871, 9998, 9999] + list(rng.choice(N, 54, replace=False)))
    Lr = L[rows]
    ref = eta @ Lr.T
    absref = np.abs(eta) @ np.abs(Lr).T
    bound = _leta_bound("bf16x3", N, absref)
    err = np.abs(P[:, rows] - ref)
    assert np.all(err <= bound), float(np.max(err / absref))
    planted = eta @ bf16(Lr).T
    assert np.mean(np.abs(planted - ref) > bound) > 0.1


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x2", "bf16l2", "bf16b"])
def test_split_noise_trajectories_track_bf16_noise_oracle(prec):
    # every entry of three consecutive steps within the derived per-step bound;
    # N = 1000 puts most of W and L off the two-product band of BF16L2 and BF16B
    twa = _twa()
    for N, M in ((300, 200), (128, 128), (45, 3), (130, 257), (1000, 40)):
        alpha, w, G, dt = 1.0, 8.0, 1.0, 2e-3
        o = BF16NoiseOracle(N, alpha, w, G, dt, 11, M)
        with twa.TWA(N, alpha, w, G, dt, seed=11, precision=prec) as g:
            def step():
                g.run(M, 1)
                return g.get_state()
            worst = track(o, step, 3, prec)
        assert worst <= 1.0


@pytest.mark.parametrize("prec,tol", [("bf16", 3e-2), ("tf32", 1e-2), ("fp32", 1e-4)])
@pytest.mark.parametrize("N,M", [(300, 200), (128, 128), (45, 3)])
def test_trajectories_track_oracle_for_a_few_steps(prec, tol, N, M):
    # Here the noise increment per site is sqrt(w dt) eta ~ 0.13 eta; rounding eta
    # to BF16 moves it by up to 2^-9 |eta|, i.e. ~1e-3 per step at |eta| ~ 4 in
    # the tail of 6e4 draws, so three steps stay within ~1e-2 of the oracle. The
    # FP32 mode keeps eta to 2^-22; what is left is the FP32 Box-Muller (32-bit
    # uniforms: ~1e-5 on the largest of 6e4 normals) and FP32 state arithmetic.
    twa = _twa()
    alpha, w, G, dt = 1.0, 8.0, 1.0, 2e-3
    o = TWAOracle(N, alpha, w, G, dt, 11, M)
    with twa.TWA(N, alpha, w, G, dt, seed=11, precision=prec) as g:
        for _ in range(3):
            o.run(1)
            g.run(M, 1)
            gx, gy, gz = g.get_state()
            err = max(np.max(np.abs(gx - o.sx)), np.max(np.abs(gy - o.sy)), np.max(np.abs(gz - o.sz)))
            assert err < tol, err
            # spins keep length sqrt(3) up to FP32 rounding
            assert np.max(np.abs(gx ** 2 + gy ** 2 + gz ** 2 - 3.0)) < 5e-6


@pytest.mark.parametrize("prec", ["bf16x3", "bf16", "tf32", "fp32", "bf16x2", "bf16l2", "bf16b"])
def test_ensemble_observables_within_3se(prec):
    # N = 256, alpha = 1, w = 32, M = 512, dt = 1e-3, T = 1, window (0.5, 1]
    N, alpha, w, G, dt, M, T, t0 = 256, 1.0, 32.0, 1.0, 1e-3, 512, 1.0, 0.5
    steps = int(round(T / dt))
    twa = _twa()
    o = TWAOracle(N, alpha, w, G, dt, 5, M, window_start=t0)
    o.run(steps)
    ob = o.observables()
    with twa.TWA(N, alpha, w, G, dt, seed=5, precision=prec, window_start=t0) as g:
        g.run(M, steps)
        gb = g.observables()
    for k in ("Sz", "SpSm", "G2num", "g2"):
        assert abs(gb[k] - ob[k]) <= 3.0 * math.hypot(gb[k + "_se"], ob[k + "_se"]), (k, gb[k], ob[k])
    assert gb["nonfinite"] == 0


def test_full_size_sampled_trajectories():
    # N = 10^4, alpha = 1, w = N/2, dt = 2e-5, M = 1024 in the launch shape the
    # benchmark times; three trajectories recomputed one by one by the oracle on
    # the same BF16-rounded normals, within the derived per-step bound.
    twa = _twa()
    N, alpha, w, G, dt, M = 10000, 1.0, 5000.0, 1.0, 2e-5, 1024
    states = []
    with twa.TWA(N, alpha, w, G, dt, seed=0, precision="bf16x3") as g:
        for _ in range(2):
            g.run(M, 1)
            states.append(g.get_state())
    for gx, gy, gz in states:
        assert np.max(np.abs(gx ** 2 + gy ** 2 + gz ** 2 - 3.0)) < 5e-6
    W = pump_matrix(N, alpha, w)
    L = np.linalg.cholesky(W)
    for m in (0, 517, 1023):
        o = BF16NoiseOracle(N, alpha, w, G, dt, 0, 1, m0=m, W=W, L=L)
        it = iter(states)
        assert track(o, lambda: tuple(a[m:m + 1] for a in next(it)), 2) <= 1.0


def test_full_size_sampled_field():
    # the contraction kernel at N = 10^4 on 2 x 1024 vectors, rows sampled one by one
    import torch
    twa = _twa()
    N, K = 10000, 2048
    rng = np.random.default_rng(3)
    s = rng.choice([-1.0, 1.0], size=(K, N))
    with twa.TWA(N, 1.0, 5000.0, 1.0, 2e-5, precision="bf16x3") as g:
        P = g.field(torch.tensor(s, device="cuda")).cpu().numpy()
    d = np.arange(N)
    for i in (0, 1, 127, 128, 4999, 9871, 9999):
        wrow = 5000.0 / (np.abs(i - d) + 1.0)
        for k in (0, 255, 256, 1500, 2047):
            ref = float(wrow @ s[k])
            bound = 2.0 * (3 * 2.0 ** -18 + (N + 1) * 2.0 ** -24) * float(np.abs(wrow) @ np.abs(s[k]))
            assert abs(P[k, i] - ref) <= bound, (i, k, P[k, i], ref)


def test_tf32_fp32_full_size_sampled_trajectories_and_fft_route():
    # the 16-wide FP32 K-stage configuration (kind::tf32 MMAs, FP32-container
    # images) at N = 10^4, M = 1024: TF32 (one term) and FP32 (three terms, eta
    # split too) on the dense route and on the FFT route (whose L.eta runs on the
    # same kernel); three trajectories by the oracle
    twa = _twa()
    N, alpha, w, G, dt, M = 10000, 1.0, 5000.0, 1.0, 2e-5, 1024
    tol = {"tf32": 1e-2, "fp32": 1e-4}
    st = {}
    for prec in tol:
        for route in ("dense", "fft"):
            with twa.TWA(N, alpha, w, G, dt, seed=0, precision=prec, ws_route=route) as g:
                g.run(M, 2)
                st[prec, route] = g.get_state()
    W = pump_matrix(N, alpha, w)
    L = np.linalg.cholesky(W)
    for gx, gy, gz in st.values():
        assert np.max(np.abs(gx ** 2 + gy ** 2 + gz ** 2 - 3.0)) < 5e-6
    for m in (0, 517, 1023):
        o = TWAOracle(N, alpha, w, G, dt, 0, 1, m0=m, W=W, L=L)
        o.run(2)
        for (prec, route), (gx, gy, gz) in st.items():
            err = max(np.max(np.abs(gx[m] - o.sx[0])), np.max(np.abs(gy[m] - o.sy[0])),
                      np.max(np.abs(gz[m] - o.sz[0])))
            assert err < tol[prec], (prec, route, m, err)


@pytest.mark.parametrize("prec", ["tf32", "fp32"])
def test_tf32_modes_reject_what_they_do_not_cover(prec, monkeypatch):
    twa = _twa()
    with twa.TWA(64, 1.0, 8.0, 1.0, 1e-3, precision=prec) as g:
        with pytest.raises(twa.TWAError) as e:
            g.grad("SpSm", 8, 4)
        assert e.value.name == "TWA_EUNSUPPORTED"
    with pytest.raises(twa.TWAError) as e:
        twa.batch_run([dict(N=32, alpha=1.0, w=4.0, Gamma=1.0, dt=1e-3, steps=4)], 8, precision=prec)
    assert e.value.name == "TWA_EUNSUPPORTED"
    monkeypatch.setenv("TWA_TC_BN", "128")
    with pytest.raises(twa.TWAError) as e:
        twa.TWA(64, 1.0, 8.0, 1.0, 1e-3, precision=prec)
    assert e.value.name == "TWA_EINVAL"


TILE_CONFIGS = {
    # (TWA_TC_PAIR, TWA_TC_KC): single CTAs and CTA pairs, 32- and 64-wide K stages,
    # four operand images or one per stage
    "one_image": [("0", "1"), ("0", "3"), ("0", "4"), ("1", "1"), ("1", "3"), ("1", "4"), ("1", "0")],
    "four_images": [("0", "1"), ("0", "0"), ("1", "1"), ("1", "0")],
}


@pytest.mark.parametrize("prec", ["bf16x2", "bf16l2", "bf16b", "bf16", "bf16x3"])
@pytest.mark.parametrize("N,M", [(300, 200), (1024, 128)])
def test_every_tile_configuration_gives_the_same_bits(monkeypatch, prec, N, M):
    # every K-stage configuration, on single CTAs or on CTA pairs (256-row
    # tcgen05.mma.cta_group::2 tiles split over two CTAs), issues the same MMAs in
    # the same K order into each accumulator row: identical states, window sums and
    # contractions. N = 300 has an odd number of 128-row tiles (a pair's second
    # tile lies past the last row) and M = 200 a ragged trajectory tile.
    import torch
    twa = _twa()
    rng = np.random.default_rng(1)
    s = torch.tensor(rng.standard_normal((5, N)), dtype=torch.float64, device="cuda")
    out = {}
    cfgs = TILE_CONFIGS["four_images" if prec == "bf16x3" else "one_image"]
    for pair, kc in cfgs:
        monkeypatch.setenv("TWA_TC_PAIR", pair)
        monkeypatch.setenv("TWA_TC_KC", kc)
        with twa.TWA(N, 1.0, 8.0, 1.0, 2e-3, seed=3, precision=prec, window_start=0.004) as g:
            g.run(M, 6)
            out[pair, kc] = (g.get_state(), g.moments(), g.field(s).cpu().numpy(), g.contract(s, "L").cpu().numpy())
    ref = out[cfgs[0]]
    for cfg in cfgs[1:]:
        got = out[cfg]
        for a, b in zip(ref[0], got[0]):
            assert np.array_equal(a, b), cfg
        for k in (1, 2, 3):
            assert np.array_equal(ref[k], got[k]), (cfg, k)


def test_tile_configuration_rejections(monkeypatch):
    twa = _twa()
    for kc in ("3", "4"):   # one operand image per stage: at most two products
        monkeypatch.setenv("TWA_TC_KC", kc)
        with pytest.raises(twa.TWAError) as e:
            twa.TWA(64, 1.0, 8.0, 1.0, 1e-3, precision="bf16x3")
        assert e.value.name == "TWA_EINVAL"
    monkeypatch.delenv("TWA_TC_KC")
    monkeypatch.setenv("TWA_TC_PAIR", "1")   # no pair configuration for the FP32 K stages
    with pytest.raises(twa.TWAError) as e:
        twa.TWA(64, 1.0, 8.0, 1.0, 1e-3, precision="tf32")
    assert e.value.name == "TWA_EINVAL"
    monkeypatch.setenv("TWA_TC_BN", "192")   # nor for 192-wide tiles
    with pytest.raises(twa.TWAError) as e:
        twa.TWA(64, 1.0, 8.0, 1.0, 1e-3, precision="bf16x2")
    assert e.value.name == "TWA_EINVAL"
