"""Exact (brute-force) solution of the Lindblad model Eq. (1) for a few spins.

TEST INFRASTRUCTURE: used only by ``tests/`` to pin the TWA oracle against the
quantum dynamics it approximates. Dense superoperator on the full 4^N space,
so N <= 5 in practice.

Conventions: site basis {|0> = down, |1> = up}; sigma^+ = |1><0|,
sigma^- = |0><1|, sigma^z = diag(-1, +1); S^a = sum_i sigma_i^a (Eq. (1) and
the line above it). Superoperators act on column-stacked density matrices,
vec(A rho B) = (B^T kron A) vec(rho).
"""
import math

import numpy as np
import scipy.linalg

__all__ = ["spin_ops", "liouvillian", "steady_state", "expectations", "dicke_collective_steady"]


def spin_ops(N):
    """sigma_i^-, sigma_i^+, sigma_i^z for i = 0..N-1 as dense 2^N matrices."""
    sm1 = np.array([[0.0, 1.0], [0.0, 0.0]])
    sz1 = np.diag([-1.0, 1.0])
    eye = np.eye(2)

    def site(op, i):
        out = np.ones((1, 1))
        for k in range(N):
            out = np.kron(out, op if k == i else eye)
        return out

    sm = [site(sm1, i) for i in range(N)]
    sp = [m.T.copy() for m in sm]
    sz = [site(sz1, i) for i in range(N)]
    return sm, sp, sz


def liouvillian(N, W, Gamma):
    """Superoperator of Eq. (1) with pump matrix W (N x N) and collective decay Gamma."""
    sm, sp, _ = spin_ops(N)
    d = 2 ** N
    I = np.eye(d)
    Sm = sum(sm)
    Sp = sum(sp)
    # collective decay: Gamma/2 (2 S- rho S+ - {S+ S-, rho})
    SpSm = Sp @ Sm
    Lv = Gamma * np.kron(Sp.T, Sm) - 0.5 * Gamma * (np.kron(I, SpSm) + np.kron(SpSm.T, I))
    # correlated pump: sum_ij w_ij/2 (2 s_j^+ rho s_i^- - {s_i^- s_j^+, rho})
    K = np.zeros((d, d))
    for i in range(N):
        for j in range(N):
            if W[i, j] == 0.0:
                continue
            Lv += W[i, j] * np.kron(sm[i].T, sp[j])
            K += W[i, j] * (sm[i] @ sp[j])
    Lv -= 0.5 * (np.kron(I, K) + np.kron(K.T, I))
    return Lv


def steady_state(N, W, Gamma, rho0=None, T=None):
    """Long-time state exp(L T) rho0 (rho0 defaults to all spins down).

    Time evolution rather than a null-space solve, so that models with several
    stationary states (the collective pump conserves the total spin) relax
    inside the sector of the initial state.
    """
    d = 2 ** N
    if rho0 is None:
        rho0 = np.zeros((d, d))
        rho0[0, 0] = 1.0
    Lv = liouvillian(N, W, Gamma)
    if T is None:
        T = 400.0 / max(Gamma, 1e-300)
    v = scipy.linalg.expm(Lv * T) @ rho0.reshape(-1, order="F")
    rho = v.reshape(d, d, order="F")
    return 0.5 * (rho + rho.T)


def expectations(rho, N):
    """<S^z>, <S+S->, <S+S+S-S->, g2 of a density matrix."""
    sm, sp, sz = spin_ops(N)
    Sm, Sp, Sz = sum(sm), sum(sp), sum(sz)
    ez = float(np.trace(rho @ Sz))
    e2 = float(np.trace(rho @ Sp @ Sm))
    e4 = float(np.trace(rho @ Sp @ Sp @ Sm @ Sm))
    return {"Sz": ez, "SpSm": e2, "G2num": e4, "g2": e4 / (e2 * e2)}


def dicke_collective_steady(N, w, Gamma):
    """Collective pump (alpha = 0) steady state in the J = N/2 manifold.

    Detailed balance between neighbouring Dicke states (Sec. S3 of the
    supplement): populations p_{m+1} = (w / Gamma) p_m for m = -J..J. With
    S^- = J^- and J^- |J, m> = sqrt((J+m)(J-m+1)) |J, m-1>.
    """
    J = N / 2.0
    ms = np.arange(-J, J + 1.0)
    r = w / Gamma
    logp = (ms + J) * math.log(r) if r != 1.0 else np.zeros_like(ms)
    p = np.exp(logp - logp.max())
    p /= p.sum()
    a = (J + ms) * (J - ms + 1.0)
    b = a * (J + ms - 1.0) * (J - ms + 2.0)
    ez = float(np.sum(p * 2.0 * ms))
    e2 = float(np.sum(p * a))
    e4 = float(np.sum(p * b))
    return {"Sz": ez, "SpSm": e2, "G2num": e4, "g2": e4 / (e2 * e2)}
