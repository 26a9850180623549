"""Independent checks ("pins") of the oracle against what the paper and the
mathematics fix.  Each function raises AssertionError on failure so that the
mutation tests can show that a planted mistake in the oracle is caught.

None of these re-types the oracle's formula: they use finite differences,
textbook library routines on a different formulation (eigh of the
Golub-Kahan tridiagonal, lstsq, normal equations, eigh of A^T A), brute
force, or closed forms.
"""
from __future__ import annotations

import math

import numpy as np


def fd_laplacian(fun, P, h):
    """4th-order central-difference Laplacian of a scalar field, one Richardson step."""
    def lap(hh):
        out = np.zeros(P.shape[0])
        for ax in range(3):
            e = np.zeros(3)
            e[ax] = hh
            f0 = fun(P)
            fp1, fm1 = fun(P + e), fun(P - e)
            fp2, fm2 = fun(P + 2 * e), fun(P - 2 * e)
            out += (-fp2 + 16 * fp1 - 30 * f0 + 16 * fm1 - fm2) / (12 * hh * hh)
        return out
    a, b = lap(h), lap(h / 2)
    return (64 * b - a) / 63.0


def pin_mq_laplacian(mq, rng, n=400, tol=1e-8):
    """L Phi at random (X, X_c, c, k) equals the FD Laplacian of Phi(|X-X_c|) + k^2 Phi."""
    worst = 0.0
    for _ in range(n // 40):
        c = math.exp(rng.uniform(math.log(0.05), math.log(1.0)))
        k = rng.uniform(0.0, 20.0)
        Xc = rng.uniform(-1, 1, 3)
        P = Xc + rng.uniform(-1.5, 1.5, (40, 3))
        fun = lambda Q: np.sqrt(np.sum((Q - Xc) ** 2, axis=1) + c * c)
        ref = fd_laplacian(fun, P, 0.02 * c) + k * k * fun(P)
        got = mq.lphi(np.linalg.norm(P - Xc, axis=1), c, k)
        worst = max(worst, float(np.max(np.abs(got - ref) / np.abs(ref))))
    assert worst < tol, worst
    return worst


def pin_assembly_rows(mq, X, n_interior, c, k, rng, tol=1e-7):
    """Rows of A applied to random coefficients reproduce the PDE / BC operators
    applied (by finite differences) to the MQ expansion u_a = sum_j a_j Phi_j."""
    A = mq.assemble(X, n_interior, c, k)
    a = rng.normal(size=X.shape[0])

    def ua(Q):
        D = np.sqrt(((Q[:, None, :] - X[None, :, :]) ** 2).sum(-1) + c * c)
        return D @ a

    Aa = A @ a
    XI = X[:n_interior]
    ref_I = fd_laplacian(ua, XI, 0.02 * c) + k * k * ua(XI)
    ref_B = ua(X[n_interior:])
    scale = np.abs(A).max(axis=1) * np.abs(a).sum()
    err_I = np.max(np.abs(Aa[:n_interior] - ref_I) / scale[:n_interior]) if n_interior else 0.0
    err_B = np.max(np.abs(Aa[n_interior:] - ref_B) / scale[n_interior:]) if n_interior < X.shape[0] else 0.0
    assert err_I < tol and err_B < 1e-13, (err_I, err_B)
    return err_I, err_B


def pin_gkb_relations(A, f, g, tol=1e-12):
    """A Z_l = W_{l+1} C_l, A^T W_l = Z_l B_l^T, orthonormal bases, W^T f = beta_1 e_1."""
    l = g.steps_done
    W, Z, C = g.W_l1(), g.Z_l(), g.C()
    nA = np.linalg.norm(A)
    r1 = np.linalg.norm(A @ Z - W @ C) / nA
    r2 = np.linalg.norm(A.T @ W[:, :l] - Z @ C[:l, :].T) / nA
    Wv = W if g.breakdown != 2 else W[:, :l]
    o1 = np.max(np.abs(Wv.T @ Wv - np.eye(Wv.shape[1])))
    o2 = np.max(np.abs(Z.T @ Z - np.eye(l))) if l else 0.0
    e1 = np.zeros(W.shape[1])
    e1[0] = g.beta1
    r3 = np.linalg.norm(W.T @ f - e1) / g.beta1
    assert max(r1, r2, o1, o2, r3) < tol, (r1, r2, o1, o2, r3)
    return r1, r2, o1, o2, r3


def tgk_singular_values(C):
    """Singular values of C from the eigenvalues of [[0, C], [C^T, 0]] (eigh)."""
    m, n = C.shape
    T = np.zeros((m + n, m + n))
    T[:m, m:] = C
    T[m:, :m] = C.T
    ev = np.linalg.eigvalsh(T)
    return np.sort(ev[ev > 0])[::-1][:n] if np.sum(ev > 0) >= n else np.sort(np.abs(ev))[::-1][:n]


def pin_projected_svd(ps, C, beta1, tol=1e-12):
    s_ref = tgk_singular_values(C)
    e_s = np.max(np.abs(ps.sigma - s_ref)) / s_ref[0]
    l = C.shape[1]
    S = np.zeros(C.shape)
    S[:l, :l] = np.diag(ps.sigma)
    e_rec = np.linalg.norm(ps.U @ S @ ps.V.T - C) / np.linalg.norm(C)
    e_f = abs(np.sum(ps.ftil ** 2) - beta1 ** 2) / beta1 ** 2
    # f~ are the coordinates of beta_1 e_1 in the left singular basis: U f~ = beta_1 e_1
    e1 = np.zeros(C.shape[0])
    e1[0] = beta1
    e_u = np.linalg.norm(ps.U @ ps.ftil - e1) / beta1
    assert max(e_s, e_rec, e_f, e_u) < tol, (e_s, e_rec, e_f, e_u)
    return e_s, e_rec, e_f, e_u


def hat_matrix(A, lam):
    """H = A (A^T A + lam^2 I)^{-1} A^T = Q1 Q1^T with [A; lam I] = [Q1; Q2] R (QR)."""
    m, n = A.shape
    Q, _ = np.linalg.qr(np.vstack([A, lam * np.eye(n)]))
    Q1 = Q[:m]
    return Q1 @ Q1.T


def gcv_dense(C, beta1, lam):
    """GCV from the explicit hat matrix H = C (C^T C + lam^2 I)^{-1} C^T."""
    m, n = C.shape
    H = hat_matrix(C, lam)
    b = np.zeros(m)
    b[0] = beta1
    r = b - H @ b
    return float(r @ r) / (m - np.trace(H)) ** 2


def tikhonov_lstsq(C, b, lam):
    n = C.shape[1]
    M = np.vstack([C, lam * np.eye(n)])
    rhs = np.concatenate([b, np.zeros(n)])
    return np.linalg.lstsq(M, rhs, rcond=None)[0]


def tsvd_via_eigh(A, f, k):
    """TSVD solution from the eigen-decomposition of A^T A (no SVD routine)."""
    ev, V = np.linalg.eigh(A.T @ A)
    order = np.argsort(ev)[::-1]
    ev, V = ev[order], V[:, order]
    out = np.zeros(A.shape[1])
    for i in range(k):
        s = math.sqrt(ev[i])
        u = A @ V[:, i] / s
        out += (u @ f) / s * V[:, i]
    return out


def matrix_with_singular_values(s, rng):
    """A = U diag(s) V^T with Haar-random orthogonal U, V (QR of Gaussians): a
    matrix whose singular values are fixed by construction."""
    n = len(s)
    U, _ = np.linalg.qr(rng.normal(size=(n, n)))
    V, _ = np.linalg.qr(rng.normal(size=(n, n)))
    return (U * np.asarray(s)) @ V.T


def pin_full_rank(full_svd, rng):
    """Numerical rank r = #{s_i > N eps s_1} of the full SVD (Algorithm 3) on
    matrices whose rank is known by construction.  (The eigenvalues of A^T A
    resolve singular values only down to about sqrt(N eps) s_1, far above the
    N eps s_1 threshold, so they cannot decide this count; the constructions
    place every singular value far from the threshold instead.)
      1. exactly rank-deficient products B C^T (N x r times r x N): rank r;
      2. singular values 1 .. 1e-8 (r1 of them), then 30 N eps, then values at
         0.03 N eps (a few eps) and exact zeros: rank r1 + 1, so a threshold of
         eps s_1 (counting the 0.03 N eps values) or of a different scale fails."""
    eps = np.finfo(np.float64).eps
    for n, r in ((60, 23), (200, 150), (41, 40)):
        A = rng.normal(size=(n, r)) @ rng.normal(size=(r, n))
        got = full_svd(A, rng.normal(size=n)).r
        assert got == r, (n, r, got)
    for n, r1 in ((80, 30), (150, 97)):
        s = np.zeros(n)
        s[:r1] = np.logspace(0, -8, r1)
        s[r1] = 30 * n * eps
        s[r1 + 1:r1 + 6] = 0.03 * n * eps
        A = matrix_with_singular_values(s, rng)
        fs = full_svd(A, rng.normal(size=n))
        assert fs.r == r1 + 1, (n, r1, fs.r)
    return True


def pin_tsvd_gcv_curve(tsvd_full, rng):
    """The full-TSVD rank curve (reading of Algorithm 3 with eq. tsvd_solution)
    against brute force: GCV(k) = |A x_k - f|^2 / (N - k)^2 with x_k the rank-k
    TSVD solution applied to the dense A, for every k = 1..min(r, N - 1) (the
    curve has exactly that many entries), and the chosen rank its argmin.  Cases:
    full rank (r = N, so the range stops at N - 1) and an exact rank-r matrix
    (r < N, the residual then includes f's component outside range(A))."""
    for n, r in ((40, 40), (50, 31)):
        s = np.zeros(n)
        s[:r] = np.logspace(0, -6, r)
        A = matrix_with_singular_values(s, rng)
        f = rng.normal(size=n)
        t = tsvd_full(A, f)
        curve = np.asarray(t["curve"])
        kmax = min(r, n - 1)
        assert curve.shape == (kmax,), (curve.shape, kmax)
        ref = np.empty(kmax)
        for k in range(1, kmax + 1):
            x = tsvd_full(A, f, rank=k)["coef"]
            res = A @ x - f
            ref[k - 1] = float(res @ res) / (n - k) ** 2
        assert np.allclose(curve, ref, rtol=1e-8, atol=0), np.max(np.abs(curve - ref) / ref)
        assert t["rank"] == int(np.argmin(ref)) + 1
    return True
