"""Host checks of the plan's spectral tables against the oracle (no GPU).

Step (b) (Sec. 3.1) solves (lambda_n I + c T) x = zhat_n, preconditioned by the Strang circulant or the natural
tau matrix (Sec. 3.2, Eq. 3.9), after the eps-scaled time DFT of Step (a) (Eqs. 1.6a/b, 1.11).  The library builds
the numbers these steps read on the host (`build_tables` in setup.cpp): lambda_n, the scalings eps^(+-k/Nt), the
Strang eigenvalues c DFT_M(s) and the tau eigenvalues c sigma_j.  This test compiles that source for the host and
compares every table with the oracle's own construction: eigenvalues of the eps-circulant C_eps, the circulant
eigenvalues of the Strang symbol, and the diagonal of S tau(T) S^-1 with the DST-I matrix S.  A sign or an index
slip (the conjugate lambda, eps^(k/Nt) for eps^(-k/Nt), an eigenvalue off by one place) fails it.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import fcd, precond

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2003_07020_gb300", "csrc")

MAIN = r"""
#include <cstdio>
#include <cstdlib>
#include "setup.h"
int main(int argc, char** argv) {
  aao::HostTables t;
  const char* err = nullptr;
  if (!aao::build_tables(atoll(argv[1]), atoll(argv[2]), atof(argv[3]), atof(argv[4]), atof(argv[5]),
                         atof(argv[6]), t, &err)) { printf("ERR %s\n", err); return 1; }
  printf("%a %a %d\n", t.c, t.eps, (int)t.tau_ok);
  for (const auto& l : t.lambda) printf("%a %a\n", l.real(), l.imag());
  for (int64_t k = 0; k < t.Nt; ++k) printf("%a %a\n", t.scale_fwd[k], t.scale_inv[k]);
  for (int64_t k = 0; k < t.M; ++k) printf("%a\n", t.strang_eig[k]);
  if (t.tau_ok) for (int64_t k = 0; k < t.M; ++k) printf("%a\n", t.tau_eig_nat[k]);
  return 0;
}
"""


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    cxx, inc = shutil.which("g++"), _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("setup_tables")
    (d / "main.cpp").write_text(MAIN)
    out = d / "h"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", inc, "-I", CSRC, "-o", str(out), str(d / "main.cpp"),
                    os.path.join(CSRC, "setup.cpp")], check=True)
    return str(out)


def _tables(exe, M, Nt, T, alpha, kappa, eps):
    lines = subprocess.run([exe, str(M), str(Nt), repr(T), repr(alpha), repr(kappa), repr(eps)], capture_output=True,
                           text=True, check=True).stdout.split("\n")
    c, e, tau_ok = lines[0].split()
    c, e, tau_ok = float.fromhex(c), float.fromhex(e), tau_ok == "1"
    pos = 1
    half = Nt // 2 + 1
    lam = np.array([complex(*(float.fromhex(x) for x in ln.split())) for ln in lines[pos:pos + half]])
    pos += half
    sc = np.array([[float.fromhex(x) for x in ln.split()] for ln in lines[pos:pos + Nt]])
    pos += Nt
    strang = np.array([float.fromhex(x) for x in lines[pos:pos + M]])
    pos += M
    tau = np.array([float.fromhex(x) for x in lines[pos:pos + M]]) if tau_ok else None
    return c, e, lam, sc[:, 0], sc[:, 1], strang, tau


@pytest.mark.parametrize("M,Nt,T,alpha,kappa,eps", [
    (63, 64, 1.0, 1.5, 1.0, 0.0),       # eps from Sec. 4: min(0.5, 0.5 tau)
    (100, 16, 2.0, 1.2, 0.5, 0.0625),
    (255, 8, 1.0, 1.8, 2.0, 0.5),
    (1, 4, 1.0, 1.1, 1.0, 0.0),
])
def test_setup_tables_match_the_oracle(exe, M, Nt, T, alpha, kappa, eps):
    c, e, lam, sfwd, sinv, strang, tau = _tables(exe, M, Nt, T, alpha, kappa, eps)
    tau_step, h = T / Nt, 1.0 / (M + 1)
    assert np.isclose(c, tau_step * kappa / h ** alpha, rtol=1e-15)
    assert e == (eps if eps > 0 else precond.default_eps(tau_step))
    # lambda_n of C_eps (Eq. 1.6a), n = 0 .. Nt/2, and the eigenvalues of the dense C_eps contain them
    want = precond.eigenvalues_C_eps(Nt, e)[: Nt // 2 + 1]
    assert np.max(np.abs(lam - want)) <= 1e-14 * np.max(np.abs(want))
    ev = np.linalg.eigvals(precond.C_eps(Nt, e))
    assert all(np.min(np.abs(ev - l)) <= 1e-10 for l in lam)
    # Step (a) scales row k by eps^(k/Nt); Step (c) by eps^(-k/Nt) / Nt
    k = np.arange(Nt)
    assert np.allclose(sfwd, e ** (k / Nt), rtol=1e-15, atol=0)
    assert np.allclose(sinv, e ** (-k / Nt) / Nt, rtol=1e-15, atol=0)
    # Strang circulant eigenvalues of c T (reading 2)
    g = c * fcd.fcd_weights(alpha, M)
    _, sev = precond.strang_symbol(g, M)
    assert np.max(np.abs(strang - sev)) <= 1e-12 * np.max(np.abs(sev))
    # natural tau matrix eigenvalues in DST order (reading 3), when M + 1 is a power of two
    if tau is not None:
        S = precond.dst1_matrix(M)
        D = S @ precond.tau_matrix(g, M) @ np.linalg.inv(S)
        assert np.max(np.abs(D - np.diag(np.diag(D)))) <= 1e-9 * np.max(np.abs(np.diag(D)))
        assert np.max(np.abs(tau - np.diag(D))) <= 1e-10 * np.max(np.abs(tau))
    else:
        assert (M + 1) & M  # M + 1 not a power of two
