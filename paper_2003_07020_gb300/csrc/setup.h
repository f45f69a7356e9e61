// Host-side FP64 setup for a plan: FCD weights, spectra, eigenvalues and
// FFT tables.  Everything here runs once per plan on the CPU in double
// precision; the device kernels only read the tables it produces.
#pragma once
#include <complex>
#include <cstdint>
#include <vector>

namespace aao {

using cd = std::complex<double>;

// g_0 .. g_{n-1} of Eq. 2.4 by the Gamma-ratio recurrence.
void fcd_weights_recurrence(double alpha, int64_t n, double* g);

// In-place radix-2 complex FFT of length n (a power of two), natural order
// in and out.  sign = -1: sum x_j exp(-2 pi i jk/n); sign = +1: exp(+...).
void host_fft(std::vector<cd>& a, int sign);

// exp(sign * 2 pi i * m / n), with the angle reduced exactly in integers.
cd unit_root(int64_t m, int64_t n, int sign);

int ilog2_exact(int64_t n);  // -1 if n is not a power of two

struct HostTables {
  int64_t M = 0, Nt = 0, L = 0;
  int logL = 0, logNt = 0;
  double tau = 0, h = 0, c = 0, eps = 0;
  std::vector<double> g;            // g_0 .. g_{M+1}
  std::vector<double> Ehat_half;    // c * DFT_L(e)_m / (L/2), m = 0 .. L/2 (matvec, FP64 R2C form)
  std::vector<double> Ehat_f;       // c * DFT_L(e)_m / L in fused-pass order (complex-vector form)
  std::vector<cd> tw_L;             // exp(-2 pi i m / L), m < L/2
  std::vector<cd> tw_Nt;            // exp(-2 pi i m / Nt), m < Nt/2
  std::vector<cd> lambda;           // lambda_n of C_eps, n = 0 .. Nt/2
  std::vector<double> scale_fwd;    // eps^{k/Nt}
  std::vector<double> scale_inv;    // eps^{-k/Nt} / Nt
  // Strang circulant (Bluestein form)
  std::vector<double> strang_eig;   // c * DFT_M(s)_k, k < M
  std::vector<cd> chirp;            // exp(-pi i j^2 / M), j < M
  std::vector<cd> chirp_hat_f;      // DFT_L(b)_m / L in fused-pass order, b_d = conj(chirp_|d|)
  // natural tau matrix (DST form), valid when L == 2(M+1)
  std::vector<double> tau_eig_f;    // c * sigma_f in fused-pass order; 1e30 at f = 0 and f = M+1
  std::vector<double> tau_eig_nat;  // c * sigma_j, j = 1..M, stored at j - 1
  bool tau_ok = false;
  // exact integer Toeplitz product (NTT matvec): per prime q, interleaved (value, Shoup companion)
  std::vector<uint32_t> ntt_twf;    // [4][ntt_tw_size][2]: pass-ordered powers of w_q (kernels.h)
  std::vector<uint32_t> ntt_twi;    // [4][ntt_tw_size][2]: the same for w_q^-1
  std::vector<uint32_t> ntt_ghat;   // [4][L][2]: NTT of the quantised stencil embedding, bit-reversed, times L^-1
  uint32_t ntt_crt[12] = {0};       // Garner constants and their Shoup companions (see ntt.cu)
  double ntt_c_gscale = 0;          // 2^(e_g - 58): G_j = round(c g_j 2^(58 - e_g))
  int ntt_gexp = 0;                 // e_g - 58
};

// Builds the NTT matvec tables of t (after build_tables); primes and generators are
// kNttPrime / kNttGen of kernels.h.
void build_ntt_tables(HostTables& t);

// Fused-pass order of a length-2^logN spectrum (see fft_convolve): entry
// blk * R + m holds the value for bit-reversed position blk * R + bitrev_r(m)
// of the natural frequency bitrev_logN(that position), R = 2^r,
// r = min(4, logN).  Returns the natural frequency for fused index p.
int64_t fused_to_freq(int64_t p, int logN);

// The 2D Strang preconditioner's per-direction map from the reciprocal eigenvalues of an M-point
// circulant to the spectrum of its kernel wrapped into L = 2^logL points (L >= 2M - 1):
//   Q[K][k] = (1/(L M)) sum_{j<M} A[K][j] exp(+2 pi i j k / M),
//   A[K][j] = exp(-2 pi i K j / L) + [j >= 1] exp(-2 pi i K (L - M + j) / L),
// the sum over j in closed form (a geometric series).  Row r of Q (r < L, M entries each) is frequency
// K = bitrev(r) (the order of a DIF transform's output) or, if fused_order, K = fused_to_freq(r).
void build_strang2d_q(int64_t M, int logL, bool fused_order, std::vector<cd>& Q);

// Default circulant parameter when the caller passes eps <= 0: the paper's
// min(0.5, 0.5 tau) (Sec. 4) for the FP64 path; for the mixed path at least
// 1/16, which bounds cond(V_eps) = 1/eps, the factor by which Step (c)
// amplifies the FP32 errors of the shifted solves.
double default_eps(double tau, bool mixed);

// Fills every table for the 1D problem.  Returns false with a message on bad input.
bool build_tables(int64_t M, int64_t Nt, double T, double alpha, double kappa, double eps,
                  HostTables& out, const char** err);

}  // namespace aao
