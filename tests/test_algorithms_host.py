"""The eliminations the kernels run, written out in numpy on small random
systems and checked against a dense solve (CPU, no GPU): the twisted block
elimination with its two-ended sweeps, the cluster kernel's row-distributed
Gauss-Jordan step, and the pivots-first FP64 panel with multipliers from the
pivot block's LU factors.  They pin the algebra the CUDA code implements (the
GPU parity tests check the kernels themselves against the oracle)."""
import numpy as np
import pytest


def _system(rng, L, S, dominance=4.0):
    A = rng.standard_normal((L, S, S)) + dominance * S * np.eye(S)
    lo = rng.standard_normal((L, S))
    up = rng.standard_normal((L, S))
    lo[0] = 0.0
    up[-1] = 0.0
    f = rng.standard_normal((L, S))
    return A, lo, up, f


def _dense(A, lo, up):
    L, S, _ = A.shape
    M = np.zeros((L * S, L * S))
    for k in range(L):
        M[k * S:(k + 1) * S, k * S:(k + 1) * S] = A[k]
        if k > 0:
            M[k * S:(k + 1) * S, (k - 1) * S:k * S] = np.diag(lo[k])
        if k + 1 < L:
            M[k * S:(k + 1) * S, (k + 1) * S:(k + 2) * S] = np.diag(up[k])
    return M


def _twisted(A, lo, up, f):
    """Elimination from both ends, meeting in the middle layer (the factor and
    sweep kernels' recurrences)."""
    L = A.shape[0]
    mid = L // 2
    inv = [None] * L
    for k in range(mid):                                   # top-down
        D = A[k] - (lo[k][:, None] * inv[k - 1] * up[k - 1][None, :] if k else 0.0)
        inv[k] = np.linalg.inv(D)
    for k in range(L - 1, mid, -1):                        # bottom-up
        E = A[k] - (up[k][:, None] * inv[k + 1] * lo[k + 1][None, :] if k < L - 1 else 0.0)
        inv[k] = np.linalg.inv(E)
    Dm = A[mid].copy()
    if mid > 0:
        Dm -= lo[mid][:, None] * inv[mid - 1] * up[mid - 1][None, :]
    if mid < L - 1:
        Dm -= up[mid][:, None] * inv[mid + 1] * lo[mid + 1][None, :]
    inv[mid] = np.linalg.inv(Dm)
    g = np.zeros_like(f)
    g[0] = f[0]
    for k in range(1, mid):
        g[k] = f[k] - lo[k] * (inv[k - 1] @ g[k - 1])
    g[L - 1] = f[L - 1]
    for k in range(L - 2, mid, -1):
        g[k] = f[k] - up[k] * (inv[k + 1] @ g[k + 1])
    y_top = inv[mid - 1] @ g[mid - 1] if mid > 0 else 0.0
    y_bot = inv[mid + 1] @ g[mid + 1] if mid < L - 1 else 0.0
    x = np.zeros_like(f)
    x[mid] = inv[mid] @ (f[mid] - lo[mid] * y_top - up[mid] * y_bot)
    for k in range(mid - 1, -1, -1):
        x[k] = inv[k] @ (g[k] - up[k] * x[k + 1])
    for k in range(mid + 1, L):
        x[k] = inv[k] @ (g[k] - lo[k] * x[k - 1])
    return x


@pytest.mark.parametrize("L", [3, 4, 7, 12])
def test_twisted_elimination_solves_the_system(L):
    rng = np.random.default_rng(L)
    A, lo, up, f = _system(rng, L, 6)
    x = _twisted(A, lo, up, f)
    ref = np.linalg.solve(_dense(A, lo, up), f.ravel()).reshape(f.shape)
    np.testing.assert_allclose(x, ref, rtol=1e-10, atol=1e-12)


def _gauss_jordan_row_panels(D, nb):
    """The cluster kernel's step: per panel the owner forms U = Dpp^-1 D[P,:] with the
    panel columns replaced by Dpp^-1, every other row r becomes
    (j in panel ? 0 : D[r][j]) - D[r][panel] U[:, j], the panel rows become U."""
    S = D.shape[0]
    D = D.copy()
    for c0 in range(0, S, nb):
        P = slice(c0, min(S, c0 + nb))
        Dinv = np.linalg.inv(D[P, P])
        U = Dinv @ D[P, :]
        U[:, P] = Dinv
        G = D[:, P].copy()
        new = D.copy()
        new[:, P] = 0.0
        new = new - G @ U
        new[P, :] = U
        D = new
    return D


@pytest.mark.parametrize("S,nb", [(5, 8), (20, 8), (37, 8), (40, 16)])
def test_cluster_gauss_jordan_inverts(S, nb):
    rng = np.random.default_rng(S + nb)
    D = rng.standard_normal((S, S)) + S * np.eye(S)
    np.testing.assert_allclose(_gauss_jordan_row_panels(D, nb) @ D, np.eye(S), atol=1e-12)


def _pivots_first(D, nb):
    """FP64 panel with its pivots chosen first (right-looking elimination of the
    unpivoted rows, multipliers kept), multipliers of every row by w U = rhs and
    G L = w, the trailing update of the column-by-column kernel; implicit pivots:
    the inverse is B[perm(i)][iperm(j)]."""
    S = D.shape[0]
    D = D.copy()
    perm = np.zeros(S, int)
    iperm = -np.ones(S, int)
    for c0 in range(0, S, nb):
        w = min(nb, S - c0)
        P = D[:, c0:c0 + w].copy()
        ip = iperm.copy()
        piv = []
        for lc in range(w):
            rows = np.where(ip < 0)[0]
            pr = rows[np.argmax(np.abs(P[rows, lc]))]
            ip[pr] = c0 + lc
            piv.append(pr)
            rows = np.where(ip < 0)[0]
            m = P[rows, lc] / P[pr, lc]
            P[np.ix_(rows, range(lc + 1, w))] -= np.outer(m, P[pr, lc + 1:w])
            P[rows, lc] = m
        for l, pr in enumerate(piv):
            perm[c0 + l] = pr
            iperm[pr] = c0 + l
        LU = P[piv, :]
        G = np.zeros((S, w))
        for r in range(S):
            rhs = np.eye(w)[piv.index(r)] if r in piv else -D[r, c0:c0 + w]
            z = np.zeros(w)
            for j in range(w):
                z[j] = (rhs[j] - z[:j] @ LU[:j, j]) / LU[j, j]
            g = z.copy()
            for i in range(w - 1, -1, -1):
                g[i] = z[i] - g[i + 1:] @ LU[i + 1:, i]
            G[r] = g
        others = [j for j in range(S) if not (c0 <= j < c0 + w)]
        U = D[piv, :][:, others]
        new = D.copy()
        for r in range(S):
            new[r, others] = G[r] @ U if r in piv else D[r, others] + G[r] @ U
        new[:, c0:c0 + w] = G
        D = new
    return D, perm, iperm


@pytest.mark.parametrize("S,nb", [(7, 4), (20, 8), (37, 8), (33, 16)])
def test_pivots_first_inverts_with_pivoting(S, nb):
    """Ragged last panels (7 = 4 + 3, 37 = 4 x 8 + 5, 33 = 2 x 16 + 1)."""
    rng = np.random.default_rng(100 + S)
    # rows scaled over many decades: partial pivoting is needed
    D = rng.standard_normal((S, S)) * np.exp(rng.uniform(-8, 8, (S, 1)))
    B, perm, iperm = _pivots_first(D, nb)
    inv = B[np.ix_(perm, iperm)]
    err = np.abs(inv @ D - np.eye(S)).max()
    # with partial pivoting the residual of the inverse stays near rounding (4e-15 to 2e-13
    # here) although the rows span 7 decades (condition 3e5 to 4e7); without pivoting it would not
    assert err < 1e-11, err
