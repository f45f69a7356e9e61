// Host FP64 setup of a plan (see setup.h).
//
// Paper references: the weights g_k (Eq. 2.4), the Toeplitz Jacobian
// (Sec. 2.1), the eigenvalues lambda_n of the eps-circulant C_eps (Eq. 1.6a),
// the scaling Lambda_eps of Eq. 1.6a used by Steps (a) and (c) (Sec. 3.1),
// and the tau-matrix of Sec. 3.2 (here in its natural T - H(T) form).
#include "setup.h"

#include <utility>

#include "kernels.h"

#include <cmath>

namespace aao {

static const double kPi = 3.14159265358979323846;

void fcd_weights_recurrence(double alpha, int64_t n, double* g) {
  if (n <= 0) return;
  const double a2 = 0.5 * alpha;
  const double gh = std::tgamma(1.0 + a2);
  g[0] = std::tgamma(1.0 + alpha) / (gh * gh);
  for (int64_t k = 0; k + 1 < n; ++k) g[k + 1] = g[k] * ((double)k - a2) / (a2 + (double)k + 1.0);
}

int ilog2_exact(int64_t n) {
  if (n <= 0 || (n & (n - 1))) return -1;
  int l = 0;
  while ((int64_t(1) << l) < n) ++l;
  return l;
}

cd unit_root(int64_t m, int64_t n, int sign) {
  int64_t r = m % n;
  if (r < 0) r += n;
  if (2 * r > n) r -= n;  // angle in (-pi, pi]
  const double ang = 2.0 * kPi * (double)r / (double)n;
  return cd(std::cos(ang), sign * std::sin(ang));
}

void host_fft(std::vector<cd>& a, int sign) {
  const int64_t n = (int64_t)a.size();
  const int logn = ilog2_exact(n);
  for (int64_t i = 0, j = 0; i < n; ++i) {  // bit-reversal permutation
    if (i < j) std::swap(a[i], a[j]);
    int64_t bit = n >> 1;
    while (bit && (j & bit)) { j ^= bit; bit >>= 1; }
    j |= bit;
  }
  std::vector<cd> tw((size_t)(n / 2 > 0 ? n / 2 : 1));
  for (int64_t m = 0; m < n / 2; ++m) tw[m] = unit_root(m, n, sign);
  for (int s = 1; s <= logn; ++s) {
    const int64_t len = int64_t(1) << s, half = len >> 1, step = n / len;
    for (int64_t st = 0; st < n; st += len)
      for (int64_t j = 0; j < half; ++j) {
        const cd u = a[st + j], v = a[st + j + half] * tw[j * step];
        a[st + j] = u + v;
        a[st + j + half] = u - v;
      }
  }
}

static int64_t bitrev64(int64_t k, int logn) {
  int64_t r = 0;
  for (int b = 0; b < logn; ++b) r |= ((k >> b) & 1) << (logn - 1 - b);
  return r;
}

double default_eps(double tau, bool mixed) {
  const double e = std::min(0.5, 0.5 * tau);
  return mixed ? std::max(e, 1.0 / 16.0) : e;
}

int64_t fused_to_freq(int64_t p, int logN) {
  const int r = logN < 4 ? logN : 4;
  const int64_t R = int64_t(1) << r;
  const int64_t blk = p / R, m = p % R;
  const int64_t pos = blk * R + bitrev64(m, r);  // bit-reversed position
  return bitrev64(pos, logN);
}

void build_strang2d_q(int64_t M, int logL, bool fused_order, std::vector<cd>& Q) {
  const int64_t L = int64_t(1) << logL, ML = M * L;
  Q.assign((size_t)(L * M), cd(0, 0));
  for (int64_t row = 0; row < L; ++row) {
    const int64_t K = fused_order ? fused_to_freq(row, logL) : bitrev64(row, logL);
    // phase of the wrapped copy: exp(-2 pi i K (L - M) / L)
    const cd ph = unit_root(K * (L - M), L, -1);
    int64_t r2 = (-K * M) % L;  // z^M = exp(2 pi i r2 / L)
    if (r2 < 0) r2 += L;
    if (2 * r2 > L) r2 -= L;
    const double phi = 2.0 * kPi * (double)r2 / (double)L;
    for (int64_t k = 0; k < M; ++k) {
      // S = sum_{j<M} z^j, z = exp(2 pi i (kL - KM) / (ML)), by the half-angle form of (1 - z^M) / (1 - z)
      int64_t r1 = (k * L - K * M) % ML;
      if (r1 < 0) r1 += ML;
      if (2 * r1 > ML) r1 -= ML;
      cd S;
      if (r1 == 0) {
        S = cd((double)M, 0.0);
      } else {
        const double th = 2.0 * kPi * (double)r1 / (double)ML;
        S = std::polar(std::sin(0.5 * phi) / std::sin(0.5 * th), 0.5 * (phi - th));
      }
      Q[(size_t)(row * M + k)] = (S + ph * (S - 1.0)) / (double)ML;
    }
  }
}

bool build_tables(int64_t M, int64_t Nt, double T, double alpha, double kappa, double eps,
                  HostTables& t, const char** err) {
  if (M < 1) { *err = "M must be >= 1"; return false; }
  if (ilog2_exact(Nt) < 2) { *err = "Nt must be a power of two >= 4"; return false; }
  if (!(T > 0.0)) { *err = "T must be > 0"; return false; }
  if (!(alpha > 0.0 && alpha <= 2.0)) { *err = "alpha must be in (0, 2]"; return false; }
  if (!(kappa > 0.0)) { *err = "kappa must be > 0"; return false; }
  t.M = M;
  t.Nt = Nt;
  t.logNt = ilog2_exact(Nt);
  int64_t L = 4;
  while (L < 2 * M) L <<= 1;  // L >= 2M - 1, a power of two, at least 4
  t.L = L;
  t.logL = ilog2_exact(L);
  if (t.logL > 14) { *err = "M too large: the circulant embedding is limited to 16384 points"; return false; }
  t.tau = T / (double)Nt;
  t.h = 1.0 / (double)(M + 1);
  t.c = t.tau * kappa / std::pow(t.h, alpha);
  t.eps = eps > 0.0 ? eps : std::min(0.5, 0.5 * t.tau);
  if (!(t.eps > 0.0 && t.eps <= 1.0)) { *err = "eps must be in (0, 1]"; return false; }
  const double c = t.c;

  t.g.resize((size_t)M + 2);
  fcd_weights_recurrence(alpha, M + 2, t.g.data());

  // circulant embedding of T: e_j = g_min(j, L-j) when that index is < M, else 0
  std::vector<cd> e((size_t)L, cd(0, 0));
  for (int64_t j = 0; j < L; ++j) {
    const int64_t d = std::min(j, L - j);
    if (d < M) e[j] = t.g[d];
  }
  host_fft(e, -1);
  t.Ehat_half.resize((size_t)L / 2 + 1);
  for (int64_t m = 0; m <= L / 2; ++m) t.Ehat_half[m] = c * e[m].real() / (double)(L / 2);
  t.Ehat_f.resize((size_t)L);
  for (int64_t p = 0; p < L; ++p) t.Ehat_f[p] = c * e[fused_to_freq(p, t.logL)].real() / (double)L;

  t.tw_L.resize((size_t)L / 2);
  for (int64_t m = 0; m < L / 2; ++m) t.tw_L[m] = unit_root(m, L, -1);
  t.tw_Nt.resize((size_t)Nt / 2);
  for (int64_t m = 0; m < Nt / 2; ++m) t.tw_Nt[m] = unit_root(m, Nt, -1);

  // eigenvalues of C_eps, Eq. 1.6a: lambda_n = 3/2 - 2 eps^{1/Nt} theta^n + 1/2 eps^{2/Nt} theta^{2n}
  t.lambda.resize((size_t)Nt / 2 + 1);
  const double e1 = std::pow(t.eps, 1.0 / (double)Nt), e2 = std::pow(t.eps, 2.0 / (double)Nt);
  for (int64_t n = 0; n <= Nt / 2; ++n)
    t.lambda[n] = 1.5 - 2.0 * e1 * unit_root(n, Nt, +1) + 0.5 * e2 * unit_root(2 * n, Nt, +1);
  t.scale_fwd.resize((size_t)Nt);
  t.scale_inv.resize((size_t)Nt);
  const double le = std::log(t.eps);
  for (int64_t k = 0; k < Nt; ++k) {
    t.scale_fwd[k] = std::exp(le * (double)k / (double)Nt);
    t.scale_inv[k] = std::exp(-le * (double)k / (double)Nt) / (double)Nt;
  }

  // Strang circulant s of T: s_k = g_k (k <= M/2), g_{M-k} otherwise; its
  // eigenvalues DFT_M(s) by Bluestein's chirp-z identity with FFTs of length L.
  t.chirp.resize((size_t)M);
  for (int64_t j = 0; j < M; ++j) t.chirp[j] = unit_root((j * j) % (2 * M), 2 * M, -1);
  std::vector<cd> b((size_t)L, cd(0, 0));
  for (int64_t d = 0; d < M; ++d) {
    b[d] = std::conj(t.chirp[d]);
    if (d > 0) b[L - d] = std::conj(t.chirp[d]);
  }
  host_fft(b, -1);  // DFT_L of the chirp filter
  t.chirp_hat_f.resize((size_t)L);
  for (int64_t p = 0; p < L; ++p) t.chirp_hat_f[p] = b[fused_to_freq(p, t.logL)] / (double)L;
  std::vector<cd> a((size_t)L, cd(0, 0));
  for (int64_t k = 0; k < M; ++k) {
    const double s = (k <= M / 2) ? t.g[k] : t.g[M - k];
    a[k] = s * t.chirp[k];
  }
  host_fft(a, -1);
  for (int64_t m = 0; m < L; ++m) a[m] *= b[m];
  host_fft(a, +1);
  t.strang_eig.resize((size_t)M);
  for (int64_t k = 0; k < M; ++k) t.strang_eig[k] = c * (t.chirp[k] * a[k] / (double)L).real();

  // natural tau matrix tau(T) = T - H(T): first column q_i = g_i - g_{i+2}
  // (i <= M-3), q_{M-2} = g_{M-2}, q_{M-1} = g_{M-1}; eigenvalues
  // sigma_j = (S q)_j / sin(pi j/(M+1)), S_{jl} = sin(pi j l/(M+1)).
  t.tau_ok = (L == 2 * (M + 1));
  if (t.tau_ok) {
    std::vector<cd> y((size_t)L, cd(0, 0));
    for (int64_t l = 1; l <= M; ++l) {
      const int64_t i = l - 1;
      const double q = (i + 2 <= M - 1) ? t.g[i] - t.g[i + 2] : t.g[i];
      y[l] = q;
      y[L - l] = -q;
    }
    host_fft(y, -1);  // = -2i (S q)_j
    std::vector<double> sig((size_t)L, 0.0);
    for (int64_t j = 1; j <= M; ++j) {
      const double sq = -0.5 * y[j].imag();
      sig[j] = sq / unit_root(j, L, +1).imag();  // sin(pi j/(M+1)) = sin(2 pi j / L)
      sig[L - j] = sig[j];
    }
    t.tau_eig_nat.resize((size_t)M);
    for (int64_t j = 1; j <= M; ++j) t.tau_eig_nat[j - 1] = c * sig[j];
    t.tau_eig_f.resize((size_t)L);
    for (int64_t p = 0; p < L; ++p) {
      const int64_t f = fused_to_freq(p, t.logL);
      t.tau_eig_f[p] = (f == 0 || f == M + 1) ? 1e30 : c * sig[f];
    }
  }
  return true;
}

}  // namespace aao

extern "C" int aao_setup_coeffs_impl(double alpha, int64_t n, double* g) {
  if (n < 1 || g == nullptr || !(alpha > 0.0 && alpha <= 2.0)) return 1;
  aao::fcd_weights_recurrence(alpha, n, g);
  return 0;
}

// ---- exact-integer matvec tables -------------------------------------------------------------
namespace aao {
namespace {

uint64_t mulmod(uint64_t a, uint64_t b, uint64_t p) { return (a * b) % p; }  // a, b < 2^30
uint64_t powmod(uint64_t b, uint64_t e, uint64_t p) {
  uint64_t r = 1;
  b %= p;
  while (e) {
    if (e & 1) r = mulmod(r, b, p);
    b = mulmod(b, b, p);
    e >>= 1;
  }
  return r;
}
uint32_t shoup(uint64_t w, uint64_t p) { return (uint32_t)((w << 32) / p); }

// In-place cyclic NTT A_k = sum_j a_j w^{jk} (natural order in and out), radix 2.
void host_ntt(std::vector<uint64_t>& a, uint64_t p, uint64_t w) {
  const size_t n = a.size();
  for (size_t i = 1, j = 0; i < n; ++i) {
    size_t bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  for (size_t len = 2; len <= n; len <<= 1) {
    const uint64_t wl = powmod(w, n / len, p);
    for (size_t i = 0; i < n; i += len) {
      uint64_t wj = 1;
      for (size_t j = 0; j < len / 2; ++j) {
        const uint64_t u = a[i + j], v = mulmod(a[i + j + len / 2], wj, p);
        a[i + j] = (u + v) % p;
        a[i + j + len / 2] = (u + p - v) % p;
        wj = mulmod(wj, wl, p);
      }
    }
  }
}

}  // namespace

void build_ntt_tables(HostTables& t) {
  const int64_t L = t.L, M = t.M;
  const int logL = t.logL;
  constexpr int NP = kNttPrimes, QB = 58;
  // quantised stencil of c T: G_j = round(c g_j 2^(58 - e_g)), c g_0 = max |c g_j| < 2^e_g (c > 0).  The scale of
  // the product, 2^(e_g - 58) 2^(e_v - 58), is then a power of two, which the epilogue applies to the exponent
  // of the reconstructed integer instead of multiplying in FP64.
  int eg = 0;
  std::frexp(t.c * t.g[0], &eg);
  std::vector<int64_t> G((size_t)M);
  for (int64_t j = 0; j < M; ++j) G[j] = std::llround(std::ldexp(t.c * t.g[j], QB - eg));
  t.ntt_c_gscale = std::ldexp(1.0, eg - QB);
  t.ntt_gexp = eg - QB;
  const size_t tsz = (size_t)ntt_tw_size(logL);
  t.ntt_twf.assign((size_t)NP * tsz * 2, 0);
  t.ntt_twi.assign((size_t)NP * tsz * 2, 0);
  t.ntt_ghat.assign((size_t)NP * L * 2, 0);
  for (int q = 0; q < NP; ++q) {
    const uint64_t p = kNttPrime[q];
    const uint64_t w = powmod(kNttGen[q], (p - 1) / (uint64_t)L, p), wi = powmod(w, p - 2, p);
    // entry idx of prime q: w^e and w^-e with their Shoup companions
    auto put = [&](size_t idx, uint64_t e) {
      const size_t o = ((size_t)q * tsz + idx) * 2;
      const uint64_t a = powmod(w, e, p), b = powmod(wi, e, p);
      t.ntt_twf[o] = (uint32_t)a;
      t.ntt_twf[o + 1] = shoup(a, p);
      t.ntt_twi[o] = (uint32_t)b;
      t.ntt_twi[o + 1] = shoup(b, p);
    };
    const int rmax = logL < 4 ? logL : 4;
    for (int e = 0; e < 8; ++e) put((size_t)e, (uint64_t)e * (uint64_t)(L >> rmax));
    for (int s0 = 0; s0 < ntt_last_pass(logL); s0 += 4) {
      const int r = ntt_pass_r(logL, s0), R = 1 << r;
      const int64_t S = L >> (s0 + r);
      const size_t off = (size_t)ntt_tw_offset(logL, s0);
      for (int k = 1; k < R; ++k) {
        int bk = 0;  // bit reversal of k over r bits
        for (int bit = 0; bit < r; ++bit)
          if (k & (1 << bit)) bk |= 1 << (r - 1 - bit);
        for (int64_t j = 0; j < S; ++j) put(off + (size_t)(k - 1) * S + j, ((uint64_t)j * bk) << s0);
      }
    }
    // circulant embedding of the stencil: c_0 = G_0, c_j = c_{L-j} = G_j (1 <= j < M); its spectrum in
    // bit-reversed order times L^-1
    auto res = [&](int64_t x) { int64_t m = x % (int64_t)p; return (uint64_t)(m < 0 ? m + (int64_t)p : m); };
    const uint64_t Linv = powmod((uint64_t)L % p, p - 2, p);
    auto spectrum = [&](const std::vector<int64_t>& Gq, std::vector<uint32_t>& out) {
      std::vector<uint64_t> c((size_t)L, 0);
      c[0] = res(Gq[0]);
      for (int64_t j = 1; j < M; ++j) c[j] = c[L - j] = res(Gq[j]);
      host_ntt(c, p, w);
      for (int64_t k = 0; k < L; ++k) {
        int64_t r = 0;  // bit reversal of k over logL bits
        for (int bit = 0; bit < logL; ++bit)
          if (k & ((int64_t)1 << bit)) r |= (int64_t)1 << (logL - 1 - bit);
        const uint64_t v = mulmod(c[r], Linv, p);
        out[((size_t)q * L + k) * 2] = (uint32_t)v;
        out[((size_t)q * L + k) * 2 + 1] = shoup(v, p);
      }
    };
    spectrum(G, t.ntt_ghat);
  }
  // Garner constants p_a^-1 mod p_b (a < b) in the order (0,1) (0,2) (0,3) (1,2) (1,3) (2,3), each with its
  // Shoup companion floor(c 2^32 / p_b)
  int o = 0;
  for (int a = 0; a < NP - 1; ++a)
    for (int bq = a + 1; bq < NP; ++bq) {
      const uint64_t pb = kNttPrime[bq];
      const uint64_t c = powmod(kNttPrime[a] % pb, pb - 2, pb);
      t.ntt_crt[2 * o] = (uint32_t)c;
      t.ntt_crt[2 * o + 1] = shoup(c, pb);
      ++o;
    }
}

}  // namespace aao
