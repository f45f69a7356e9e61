"""Host checks of the exact-integer matvec's tables (no GPU).

The NTT matvec (Sec. 3.2, c T v_k by circulant embedding) reads tables that the library builds on the host
(`build_ntt_tables` in setup.cpp): the quantised stencil G_j = round(c g_j 2^(58 - e)) with c g_0 < 2^e, its
circulant embedding's number-theoretic transform modulo each of the four primes (bit-reversed, times L^-1, each
value with its Shoup companion floor(v 2^32 / p)), and Garner's constants p_a^-1 mod p_b.  This test compiles the
host source for the host, builds the tables of a few problems and recomputes every entry with an independent
pure-Python transform, and checks the bound sum_d |G_d| <= 2 G_0 + M (the sign pattern of Lemma 2.1) on which
the four-prime reconstruction relies.
"""
import math
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2003_07020_gb300", "csrc")

MAIN = r"""
#include <cstdio>
#include <cstdlib>
#include "setup.h"
int main(int argc, char** argv) {
  aao::HostTables t;
  const char* err = nullptr;
  if (!aao::build_tables(atoll(argv[1]), atoll(argv[2]), 1.0, atof(argv[3]), 1.0, 0.0, t, &err)) return 1;
  aao::build_ntt_tables(t);
  printf("%lld %d %a %a %d\n", (long long)t.L, t.logL, t.c, t.ntt_c_gscale, t.ntt_gexp);
  for (int64_t j = 0; j < t.M; ++j) printf("%a\n", t.g[j]);
  for (size_t i = 0; i < t.ntt_ghat.size(); i += 2) printf("%u %u\n", t.ntt_ghat[i], t.ntt_ghat[i + 1]);
  for (int i = 0; i < 12; ++i) printf("%u\n", t.ntt_crt[i]);
  return 0;
}
"""


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


def _constants():
    text = open(os.path.join(CSRC, "kernels.h")).read()

    def arr(name):
        s = text[text.index(name):]
        return [int(x.strip().rstrip("u")) for x in s[s.index("{") + 1:s.index("}")].split(",")]

    return arr("kNttPrime[kNttPrimes]"), arr("kNttGen[kNttPrimes]")


@pytest.fixture(scope="module")
def tables_exe(tmp_path_factory):
    cxx, inc = shutil.which("g++"), _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("ntt_tables")
    (d / "main.cpp").write_text(MAIN)
    exe = d / "h"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", inc, "-I", CSRC, "-o", str(exe), str(d / "main.cpp"),
                    os.path.join(CSRC, "setup.cpp")], check=True)
    return str(exe)


def _ntt(a, w, p):
    """Cyclic transform A_k = sum_j a_j w^(jk) mod p, natural order in and out (recursive radix 2)."""
    n = len(a)
    if n == 1:
        return list(a)
    even, odd = _ntt(a[0::2], w * w % p, p), _ntt(a[1::2], w * w % p, p)
    out, t = [0] * n, 1
    for k in range(n // 2):
        u, v = even[k], odd[k] * t % p
        out[k], out[k + n // 2] = (u + v) % p, (u - v) % p
        t = t * w % p
    return out


def _llround(x):
    """Round half away from zero, like llround (the fractional part of a double is exact)."""
    a = abs(x)
    f = math.floor(a)
    n = int(f) + (1 if a - f >= 0.5 else 0)
    return n if x >= 0 else -n


@pytest.mark.parametrize("M,Nt,alpha", [(1, 4, 1.5), (100, 8, 1.2), (1000, 16, 1.8), (8191, 8, 1.5)])
def test_ntt_tables_are_the_transforms_of_the_quantised_stencil(tables_exe, M, Nt, alpha):
    primes, gens = _constants()
    out = subprocess.run([tables_exe, str(M), str(Nt), str(alpha)], capture_output=True, text=True,
                         check=True).stdout.split("\n")
    head = out[0].split()
    L, logL, c, gscale, gexp = int(head[0]), int(head[1]), float.fromhex(head[2]), float.fromhex(head[3]), int(head[4])
    g = [float.fromhex(x) for x in out[1:1 + M]]
    rows = out[1 + M:1 + M + len(primes) * L]
    crt = [int(x) for x in out[1 + M + len(primes) * L:1 + M + len(primes) * L + 12]]
    assert L >= 2 * M - 1 and L == 1 << logL
    # quantisation: c g_0 < 2^e, G_j = round(c g_j 2^(58 - e)); the scale 2^(e - 58) is a power of two
    e = math.frexp(c * g[0])[1]
    assert gexp == e - 58 and gscale == 2.0 ** gexp
    G = [_llround(math.ldexp(c * gj, 58 - e)) for gj in g]
    assert 0 < G[0] < 2 ** 58 and all(x <= 0 for x in G[1:])
    total = G[0] + 2 * sum(abs(x) for x in G[1:])
    assert total <= 2 * G[0] + M  # so |Y| <= 2^58 (2^59 + M) < 2^117 (1 + 2^-45) for every quantised row
    P = 1
    for p in primes:
        P *= p
    assert 2 ** 58 * (2 ** 59 + M) < P // 2
    for q, (p, gen) in enumerate(zip(primes, gens)):
        w = pow(gen, (p - 1) // L, p)
        assert pow(w, L // 2, p) == p - 1  # a primitive L-th root of unity
        emb = [0] * L
        emb[0] = G[0] % p
        for j in range(1, M):
            emb[j] = emb[L - j] = G[j] % p
        S = _ntt(emb, w, p)
        Linv = pow(L, p - 2, p)
        for k in range(L):
            br = int(format(k, "0%db" % logL)[::-1], 2) if logL else 0
            v, sh = (int(x) for x in rows[q * L + k].split())
            assert v == S[br] * Linv % p, (q, k)
            assert sh == (v << 32) // p, (q, k)
    o = 0
    for a in range(len(primes) - 1):
        for b in range(a + 1, len(primes)):
            cc, sh = crt[2 * o], crt[2 * o + 1]
            assert cc * primes[a] % primes[b] == 1 and sh == (cc << 32) // primes[b]
            o += 1
