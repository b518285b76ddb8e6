"""Solvers for Eq. final (oracle): dense LU and plain restarted GMRES.

The paper solves Eq. final with GMRES (Sec. IV-A, PETSc); restart length,
orthogonalisation and initial guess are not given.  Reading: GMRES(m) with
zero initial guess and modified Gram-Schmidt, stopping on ||b - A x|| /
||b||.  No preconditioner (the near-field preconditioner of Eq.
final_precond is not part of this path).

Pins: GMRES agrees with dense LU on small systems; dense LU is LAPACK.
"""
import numpy as np
import scipy.linalg as sla


def dense_solve(A, b):
    return sla.solve(A, b)


def gmres(matvec, b, rtol=1e-10, restart=30, max_iters=10000):
    """Restarted GMRES, plain Arnoldi with modified Gram-Schmidt and Givens
    rotations.  Returns (x, iterations, relative residual history)."""
    b = np.asarray(b, dtype=complex)
    n = b.shape[0]
    x = np.zeros(n, dtype=complex)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, [0.0]
    hist = [1.0]
    it = 0
    while it < max_iters:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        if beta / bnorm <= rtol:
            hist.append(beta / bnorm)
            break
        V = np.zeros((restart + 1, n), dtype=complex)
        H = np.zeros((restart + 1, restart), dtype=complex)
        cs = np.zeros(restart, dtype=complex)
        sn = np.zeros(restart, dtype=complex)
        g = np.zeros(restart + 1, dtype=complex)
        g[0] = beta
        V[0] = r / beta
        j_end = 0
        for j in range(restart):
            w = matvec(V[j])
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = np.conj(cs[i]) * H[i, j] + np.conj(sn[i]) * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.sqrt(abs(H[j, j]) ** 2 + abs(H[j + 1, j]) ** 2)
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            it += 1
            j_end = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) / bnorm <= rtol or it >= max_iters:
                break
        y = sla.solve_triangular(H[:j_end, :j_end], g[:j_end])
        x = x + V[:j_end].T @ y
        if hist[-1] <= rtol:
            r = b - matvec(x)
            if np.linalg.norm(r) / bnorm <= rtol * 10:
                break
    return x, it, hist
