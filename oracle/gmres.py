"""Restarted right-preconditioned flexible GMRES, plain numpy FP64.

Test infrastructure only (see :mod:`oracle`).

Paper: Sec. 4 solves the right-preconditioned system calA P^{-1} (P U) = F
with a GMRES-type method from x0 = 0 and stops on a relative residual.
This is the textbook flexible variant (the preconditioned vectors z_j are
stored, so P^{-1} may be inexact), with modified Gram-Schmidt and Givens
rotations, restarted every m steps.  Stopping rule: the true residual
||F - calA U||_2 / ||F||_2 <= tol, checked at every restart and at exit.
"""
import numpy as np


def fgmres(matvec, precond, F, tol=1e-10, restart=20, max_cycles=50, x0=None):
    """Right-preconditioned restarted flexible GMRES (Sec. 4, the outer solver of Example 1) with modified
    Gram-Schmidt.  Solve matvec(U) = F.  ``matvec`` and ``precond`` map arrays of F's
    shape to arrays of F's shape.  Returns (U, info) with info holding the
    total number of inner iterations ``iters``, ``cycles`` and the final true
    relative residual ``trr``."""
    F = np.asarray(F, dtype=np.float64)
    shape = F.shape
    b = F.ravel()
    nb = np.linalg.norm(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64).ravel()
    A = lambda v: np.asarray(matvec(v.reshape(shape)), dtype=np.float64).ravel()
    P = lambda v: np.asarray(precond(v.reshape(shape)), dtype=np.float64).ravel()
    iters = 0
    cycles = 0
    trr = np.linalg.norm(b - A(x)) / nb if nb > 0 else 0.0
    while trr > tol and cycles < max_cycles:
        r = b - A(x)
        beta = np.linalg.norm(r)
        m = restart
        V = np.zeros((m + 1, b.size))
        Z = np.zeros((m, b.size))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            Z[j] = P(V[j])
            w = A(Z[j])
            for i in range(j + 1):          # modified Gram-Schmidt
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):              # apply previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            d = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / d
            sn[j] = H[j + 1, j] / d
            H[j, j] = d
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            iters += 1
            j_done = j + 1
            if abs(g[j + 1]) <= tol * nb or H[j, j] == 0.0:
                break
        y = np.zeros(j_done)
        for i in range(j_done - 1, -1, -1):  # back substitution
            y[i] = (g[i] - H[i, i + 1:j_done] @ y[i + 1:]) / H[i, i]
        x = x + y @ Z[:j_done]
        cycles += 1
        trr = np.linalg.norm(b - A(x)) / nb
    return x.reshape(shape), {"iters": iters, "cycles": cycles, "trr": trr}


def bicgstab(matvec, precond, F, tol=1e-9, maxit=500, x0=None):
    """Preconditioned BiCGSTAB (van der Vorst), the outer solver of Example 2 in Sec. 4.

    The preconditioner is applied to the two search directions of each step (y = P^{-1} p, then
    y = P^{-1} s) and the iterate is updated with them, so the recurrence carries the residual of the
    original system; the iteration stops when ||r_k||_2 / ||r_0||_2 < tol (r_0 = F for x0 = 0), checked
    after each half step (the s vector) and each full step.  The paper calls its solver
    left-preconditioned; the Iter columns it prints (Tables 4-6, in half steps) are those of this form
    (the interface of the library routine it cites, with a preconditioner argument), not of BiCGSTAB on
    P^{-1} calA with the preconditioned residual monitored, which needs up to 1.5 more steps there.
    Returns (U, info) with ``iters`` (half steps / 2), ``applies`` (preconditioner applications) and
    the true relative residual ``trr``."""
    F = np.asarray(F, dtype=np.float64)
    shape = F.shape
    b = F.ravel()
    A = lambda v: np.asarray(matvec(v.reshape(shape)), dtype=np.float64).ravel()
    P = lambda v: np.asarray(precond(v.reshape(shape)), dtype=np.float64).ravel()
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64).ravel()
    r = b - A(x)
    rhat = r.copy()
    n0 = np.linalg.norm(r)
    rho = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    halves = applies = 0
    done = n0 == 0.0
    while not done and halves < 2 * maxit:
        rho_new = rhat @ r
        beta = (rho_new / rho) * (alpha / omega)
        rho = rho_new
        p = r + beta * (p - omega * v)
        y = P(p)
        applies += 1
        v = A(y)
        alpha = rho / (rhat @ v)
        x = x + alpha * y
        s = r - alpha * v
        halves += 1
        if np.linalg.norm(s) / n0 < tol:
            break
        y = P(s)
        applies += 1
        t = A(y)
        omega = (t @ s) / (t @ t)
        x = x + omega * y
        r = s - omega * t
        halves += 1
        done = np.linalg.norm(r) / n0 < tol
    nb = np.linalg.norm(b)
    trr = np.linalg.norm(b - A(x)) / nb if nb > 0 else 0.0
    return x.reshape(shape), {"iters": halves / 2.0, "applies": applies, "trr": trr}
