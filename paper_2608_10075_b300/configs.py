"""Parameter sets of the synthetic workloads (no arithmetic of the method).

Every workload is a point (N, alpha, w, Gamma, dt, T, M) of the model of
Eq. 1-2 with discrete-Wigner ground-state starts (x, y = +-1 from Philox seed
0, z = -1). The paper runs its own protocol (N_trj = 2^13, excited start,
Sec. S1); these are the sizes this engine is measured and checked on.
"""

SMALL_CHAIN = dict(name="N16-fp64", N=16, alpha=1.0, w=8.0, Gamma=1.0, M=1024, dt=2e-3, T=5.0, window=2.0,
                   precision="fp64")

MIXED_N1024 = dict(name="N1024-mixed", N=1024, alphas=(0.5, 1.0, 2.0), w=512.0, Gamma=1.0, M=4096, dt=1e-4, T=2.0,
                   window=1.0, precision="bf16x3")

# W and L as BF16 images, one product per entry except hi + lo within 64
# columns of the diagonal; FP32 state; the contractions take the state and the
# noise rounded once to BF16 (precision "bf16b")
LARGE_N1E4 = dict(name="N10000-bf16b", N=10000, alpha=1.0, w=5000.0, Gamma=1.0, M=1024, dt=2e-5, T=0.5,
                  window=0.2, precision="bf16b")

SCAN_POINTS = dict(name="scan96", Ns=(100, 300, 1000, 3000), alphas=(0.25, 0.5, 0.75, 1.0, 1.5, 2.0),
                   n_w=4, M=512, Gamma=1.0, T=1.0)

ADJOINT_N1024 = dict(name="N1024-adjoint", N=1024, alpha=1.0, w=256.0, Gamma=1.0, M=2048, dt=1e-4, T=2.0,
                     checkpoint=64, delta=1e-4)


def scan_points():
    """The 96 (N, alpha, w) points of the batched scan: w / Gamma at 4
    log-spaced values in [1, N]; dt = 0.02 / (N Gamma)."""
    pts = []
    for N in SCAN_POINTS["Ns"]:
        for a in SCAN_POINTS["alphas"]:
            for k in range(SCAN_POINTS["n_w"]):
                w = float(N) ** (k / (SCAN_POINTS["n_w"] - 1))
                pts.append(dict(N=N, alpha=a, w=w, Gamma=1.0, dt=0.02 / N, T=SCAN_POINTS["T"]))
    return pts
