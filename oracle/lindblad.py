"""Exact (brute-force) solution of the Lindblad model Eq. (1) for a few spins.

TEST INFRASTRUCTURE: used only by ``tests/`` to pin the TWA oracle against the
quantum dynamics it approximates. Two solvers: the dense superoperator on the
full 4^N space, evolved in time (N <= 5 in practice; any pump), and, for a
positive-definite pump matrix (alpha > 0, a unique steady state), a direct
solve restricted to the matrix elements the steady state can occupy (N <= 8).

Conventions: site basis {|0> = down, |1> = up}; sigma^+ = |1><0|,
sigma^- = |0><1|, sigma^z = diag(-1, +1); S^a = sum_i sigma_i^a (Eq. (1) and
the line above it). Superoperators act on column-stacked density matrices,
vec(A rho B) = (B^T kron A) vec(rho).
"""
import math

import numpy as np
import scipy.linalg
import scipy.sparse as sparse

__all__ = ["spin_ops", "liouvillian", "liouvillian_sparse", "steady_state", "steady_state_unique", "expectations",
           "dicke_collective_steady"]


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


def liouvillian_sparse(N, W, Gamma):
    """The superoperator of ``liouvillian`` (same terms, same vectorisation) as
    a sparse matrix, built site operator by site operator."""
    d = 2 ** N
    lower = sparse.csr_matrix(np.array([[0.0, 1.0], [0.0, 0.0]]))

    def site(i):
        left = sparse.identity(2 ** i, format="csr")
        right = sparse.identity(2 ** (N - 1 - i), format="csr")
        return sparse.kron(sparse.kron(left, lower), right, format="csr")

    sm = [site(i) for i in range(N)]
    sp = [m.T.tocsr() for m in sm]
    I = sparse.identity(d, format="csr")
    Sm = sum(sm)
    Sp = sum(sp)
    SpSm = (Sp @ Sm).tocsr()
    Lv = Gamma * sparse.kron(Sp.T, Sm) - 0.5 * Gamma * (sparse.kron(I, SpSm) + sparse.kron(SpSm.T, I))
    K = sparse.csr_matrix((d, d))
    for i in range(N):
        for j in range(N):
            if W[i, j] == 0.0:
                continue
            Lv = Lv + W[i, j] * sparse.kron(sm[i].T, sp[j], format="csr")
            K = K + W[i, j] * (sm[i] @ sp[j])
    return (Lv - 0.5 * (sparse.kron(I, K) + sparse.kron(K.T, I))).tocsr()


def steady_state_unique(N, W, Gamma):
    """The steady state of Eq. (1) for a positive-definite pump matrix, by a
    direct solve of L rho = 0 with tr rho = 1.

    With W positive definite the pump's jump operators span every single-site
    sigma_i^+, so together with their adjoints they generate the whole operator
    algebra and the steady state is unique (alpha = 0, a rank-one W, conserves
    the total spin instead: use ``steady_state`` there). Two exact reductions
    make N = 8 a small dense solve:
    - every term of Eq. (1) changes the number of up spins of the ket and of the
      bra of |a><b| by the same amount, and the unique steady state is reached
      from |0...0><0...0|, so it has rho_ab = 0 unless popcount(a) = popcount(b);
    - the superoperator is real and maps rho^T to (L rho)^T, so the unique steady
      state is real symmetric: only rho_ab with a <= b are unknowns.
    """
    if np.linalg.eigvalsh(W).min() <= 0.0:
        raise ValueError("steady_state_unique needs a positive-definite pump matrix")
    d = 2 ** N
    L = liouvillian_sparse(N, W, Gamma)
    ups = np.array([bin(a).count("1") for a in range(d)])
    idx = np.arange(d)
    a, b = np.nonzero((ups[:, None] == ups[None, :]) & (idx[:, None] <= idx[None, :]))
    col = a + d * b      # column-stacked position of rho_ab
    col_t = b + d * a    # of rho_ba, the same unknown
    rows = L[col]
    A = (rows[:, col] + rows[:, col_t]).toarray()
    diag = a == b
    A[:, diag] *= 0.5    # rho_aa was added to itself above
    A[0, :] = diag       # the trace condition replaces one (redundant) equation
    rhs = np.zeros(len(col))
    rhs[0] = 1.0
    v = scipy.linalg.solve(A, rhs)
    rho = np.zeros((d, d))
    rho[a, b] = v
    rho[b, a] = v
    return rho


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
