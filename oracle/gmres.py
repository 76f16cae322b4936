"""Restarted GMRES (Saad & Schultz 1986), the iterative solver of Section 4.

Plain textbook form: Arnoldi with modified Gram-Schmidt, Givens rotations on
the Hessenberg matrix, zero initial guess, stop when ||b - A x|| / ||b|| <= tol
(estimated from the rotated residual, verified with a true residual at each
restart).  Pinned in tests/test_oracle_gmres.py against numpy.linalg.solve.
"""
import numpy as np


def gmres(apply, b, tol=1e-6, restart=100, maxit=1000):
    b = np.asarray(b, np.complex128)
    n = b.size
    x = np.zeros(n, np.complex128)
    bn = np.linalg.norm(b)
    if bn == 0:
        return x, 0, [0.0]
    hist = []
    it = 0
    r = b.copy()
    while it < maxit:
        beta = np.linalg.norm(r)
        hist.append(beta / bn)
        if beta / bn <= tol:
            break
        m = min(restart, maxit - it)
        Q = np.zeros((m + 1, n), np.complex128)
        H = np.zeros((m + 1, m), np.complex128)
        cs = np.zeros(m, np.complex128)
        sn = np.zeros(m, np.complex128)
        g = np.zeros(m + 1, np.complex128)
        g[0] = beta
        Q[0] = r / beta
        j_used = 0
        for j in range(m):
            w = apply(Q[j])
            for i in range(j + 1):
                H[i, j] = np.vdot(Q[i], w)
                w = w - H[i, j] * Q[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                Q[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = np.conj(cs[i]) * H[i, j] + np.conj(sn[i]) * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.sqrt(abs(H[j, j]) ** 2 + abs(H[j + 1, j]) ** 2)
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            it += 1
            j_used = j + 1
            hist.append(abs(g[j + 1]) / bn)
            if abs(g[j + 1]) / bn <= tol or H[j, j] == 0:
                break
        y = np.linalg.solve(np.triu(H[:j_used, :j_used]), g[:j_used])
        x = x + Q[:j_used].T @ y
        r = b - apply(x)
        if np.linalg.norm(r) / bn <= tol:
            hist.append(np.linalg.norm(r) / bn)
            break
    return x, it, hist
