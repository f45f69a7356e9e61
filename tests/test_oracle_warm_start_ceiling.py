"""How much any warm start of the shifted solves could save: a ceiling for the learned initial guess (CPU).

Step (b) (Sec. 3.1) solves (lambda_n I + c T) x = zhat_n for every time frequency n by COCG with the Strang
circulant preconditioner.  The learned warm start (no counterpart in the paper) predicts x from zhat_n with a
Fourier neural operator whose spectral path keeps the 16 lowest spatial modes.  Here every guess is given the
exact solution's information, so the counts bound from below what a model of that kind could reach: starting from
the exact solution's 16 lowest Fourier modes, from its 64 lowest, and from the Strang solve itself.

Workload of the learned configuration (M = 1023, Nt = 256, alpha 1.2 / 1.5 / 1.8, kappa = 1, eps of the mixed path),
the shifted systems of the first preconditioner application (zhat of F / ||F||), FP64 COCG to 1e-6 as on the GPU.
"""
import numpy as np
import pytest

from oracle import aao, fcd, precond
from paper_2003_07020_gb300 import workloads

M, NT, KAPPA, SEED = 1023, 256, 1.0, 7


def _low_modes(x, k):
    X = np.fft.fft(x)
    keep = np.zeros_like(X)
    keep[:k] = X[:k]
    keep[-k + 1:] = X[-k + 1:]
    return np.fft.ifft(keep)


def _cocg_iterations(matvec, b, pinv, x0, tol=1e-6, maxit=200):
    """Preconditioned COCG (bilinear form u^T w) from x0; iterations until ||r|| <= tol ||b||."""
    x = x0.copy()
    r = b - matvec(x)
    nb = np.linalg.norm(b)
    if np.linalg.norm(r) <= tol * nb:
        return 0
    z = pinv(r)
    p = z.copy()
    rho = r @ z
    for it in range(1, maxit + 1):
        q = matvec(p)
        a = rho / (p @ q)
        x = x + a * p
        r = r - a * q
        if np.linalg.norm(r) <= tol * nb:
            return it
        z = pinv(r)
        rho_new = r @ z
        p = z + (rho_new / rho) * p
        rho = rho_new
    return maxit


def _totals(alpha):
    tau, h = 1.0 / NT, 1.0 / (M + 1)
    eps = max(min(0.5, 0.5 * tau), 1.0 / 16)
    g = (tau * KAPPA / h ** alpha) * fcd.fcd_weights(alpha, M)  # c g: first column of c T
    L = 2 * M + 2
    emb = np.zeros(L)
    emb[:M] = g
    emb[L - M + 1:] = g[1:][::-1]
    ehat = np.fft.fft(emb)
    _, sev = precond.strang_symbol(g, M)
    lam_all = precond.eigenvalues_C_eps(NT, eps)
    u0, f = workloads.make_inputs(M, NT, seed=SEED)[:2]
    F = aao.build_rhs(u0, f, tau)
    zhat = precond.time_dft_half(F / np.linalg.norm(F), eps)
    tot = {"zero": 0, "exact_16_modes": 0, "exact_64_modes": 0, "strang_solve": 0}
    for n in range(NT // 2 + 1):
        lam = lam_all[n]

        def mv(x):
            return lam * x + np.fft.ifft(ehat * np.fft.fft(np.concatenate([x, np.zeros(L - M)])))[:M]

        def pinv(r):
            return np.fft.ifft(np.fft.fft(r) / (lam + sev))

        b = zhat[n]
        xs = np.linalg.solve(precond.shifted_system(g, M, lam), b)
        guesses = {"zero": np.zeros(M, complex), "exact_16_modes": _low_modes(xs, 16),
                   "exact_64_modes": _low_modes(xs, 64), "strang_solve": pinv(b)}
        for k, x0 in guesses.items():
            tot[k] += _cocg_iterations(mv, b, pinv, x0)
    return tot


@pytest.mark.parametrize("alpha", [1.2, 1.5, 1.8])
def test_no_16_mode_warm_start_saves_15_percent(alpha):
    tot = _totals(alpha)
    base = tot["zero"]
    saved = {k: 1.0 - v / base for k, v in tot.items()}
    print(alpha, tot, {k: round(100 * v, 1) for k, v in saved.items()})
    # even the exact solution's 16 lowest modes save less than 15 % of the iterations (measured 10.6 / 11.6 /
    # 11.4 %): the iterations are spent on the high-frequency part of the error, which 16 modes cannot carry
    assert 0.0 < saved["exact_16_modes"] < 0.15
    # more modes help, and the model-free start x0 = (lambda I + c S)^{-1} b already saves about one iteration
    # per system (it costs one preconditioner solve and one product with the shifted matrix, about an iteration)
    assert saved["exact_64_modes"] >= saved["exact_16_modes"] - 0.02
    assert saved["strang_solve"] > saved["exact_16_modes"]
