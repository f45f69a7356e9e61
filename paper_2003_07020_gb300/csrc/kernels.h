// Launchers of the sm_103a kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

struct aao_fno;

namespace aao {

// ---- all-at-once matvec (FP64), matvec.cu -------------------------------------------
// w = calA v, or w = rhs - calA v when rhs != nullptr.  v is double or float.
// If sq_partial != nullptr, sq_partial[k] = sum_i w[k][i]^2 for every row k.
cudaError_t launch_matvec_f64(const double* v, const double* rhs, double* w, double* sq_partial,
                              int M, int Nt, int logL, const double* Ehalf, const double2* twL,
                              cudaStream_t s);
cudaError_t launch_matvec_f64_fin(const float* v, const double* rhs, double* w, double* sq_partial,
                                  int M, int Nt, int logL, const double* Ehalf, const double2* twL,
                                  cudaStream_t s);
size_t matvec_smem_bytes(int logL);

// ---- time DFT, Steps (a) and (c), tdft.cu -------------------------------------------
// Step (a): out[n][i] = sum_k scale[k] theta^{nk} v[k][i], n = 0..Nt/2, theta = exp(2 pi i/Nt)
// launch_tdft_fwd_f32_ff: the same with v a float-float vector (hi, lo per element; hi is used).
// Shared memory of one time-DFT CTA (all Nt rows of an 8-column tile) and the largest power-of-two
// Nt whose CTA fits in smem_limit bytes (the device's opt-in limit per block).
size_t tdft_smem_bytes(int Nt, bool fp32);
int tdft_max_Nt(bool fp32, size_t smem_limit);
cudaError_t launch_tdft_fwd_f32_ff(const float2* v, float2* out, int M, int Nt, const float* scale,
                                   const float2* twNt, cudaStream_t s);
cudaError_t launch_tdft_fwd_f32(const double* v, float2* out, int M, int Nt, const float* scale,
                                const float2* twNt, cudaStream_t s);
cudaError_t launch_tdft_fwd_f64(const double* v, double2* out, int M, int Nt, const double* scale,
                                const double2* twNt, cudaStream_t s);
// Step (c): z[k][i] = scale_inv[k] * Re sum_{n<Nt} x_n theta^{-nk}, x_{Nt-n} = conj(x_n)
cudaError_t launch_tdft_inv_f32(const float2* in, float* z, int M, int Nt, const float* scale_inv,
                                const float2* twNt, cudaStream_t s);
cudaError_t launch_tdft_inv_f32_to_f64(const float2* in, double* z, int M, int Nt,
                                       const float* scale_inv, const float2* twNt, cudaStream_t s);
cudaError_t launch_tdft_inv_f64(const double2* in, double* z, int M, int Nt, const double* scale_inv,
                                const double2* twNt, cudaStream_t s);

// ---- shifted solves, Step (b), cocg.cu -----------------------------------------------
struct CocgTables32 {
  const float2* twL;      // exp(-2 pi i m/L), m < L/2
  const float* Ebr;       // c * DFT_L(e) / L, fused-pass order
  const double2* lambda;  // lambda_n, n < nsys
  const float2* chirp;    // Strang: exp(-pi i j^2/M)
  const float2* chat_br;  // Strang: DFT_L(conj chirp filter)/L, fused-pass order
  const float* seig;      // Strang: c * eigenvalues of S
  const float* taueig_br; // tau: c * sigma_f, fused-pass order (1e30 where the DST multiplier vanishes)
  // Strang, optional: per system n, the fused-order spectrum (/L) of the length-L circulant whose
  // first M outputs apply (lambda_n I + c S)^{-1} exactly ([nsys][L]); null: Bluestein at run time
  const float2* sconv;
};
// Step (b) with the Krylov vectors in tensor memory (cocg_tm.cu): Strang by precomputed spectra, FP32,
// 4096 < M <= 8191 (L = 2^14), one system per CTA of 512 threads.  Spectra in the order of its fused
// pass: entry s holds L-frequency tm_order_freq(s).
struct CocgTmTables {
  const float2* twL;      // exp(-2 pi i m/L), m < L/2
  const float* Ebr;       // c DFT_L(e) / L (real) [L]
  const float2* sconv;    // per system, the spectra of CocgTables32::sconv [nsys][L]
  const double2* lambda;  // lambda_n
};
int tm_order_freq(int s);
bool cocg_tm_supported(int M, int logL);
size_t cocg_tm_smem_bytes();
// dst[n][s] = src[n][perm[s]] (n < nsys), dstr[s] = srcr[perm[s]], s < 2^14
cudaError_t launch_tm_gather(const float2* src, float2* dst, const float* srcr, float* dstr, const int* perm, int nsys,
                             cudaStream_t s);
// xb: [nsys][M] right-hand sides in, solutions out; iters / flags as launch_cocg_f32.
cudaError_t launch_cocg_tm(float2* xb, int M, int logL, int nsys, const CocgTmTables& tb, float tol, int maxit,
                           int* iters, int* flags, cudaStream_t s);
struct CocgTables64 {
  const double2* twL;
  const double* Ebr;
  const double2* lambda;
  const double2* chirp;
  const double2* chat_br;
  const double* seig;
  const double* taueig_br;
};
// One instance of a batched Step (b) launch (launch_cocg_batched): its right-hand sides / solutions
// xb ([nsys][M] complex), sizes, tables (Strang spectra or tau eigenvalues), tolerance and statistics.
struct CocgBatchInst {
  float2* xb;
  int M, logL, nsys;
  CocgTables32 tb;
  float tol;
  int maxit;
  int* iters;
  int* flags;
};
// Step (b) of several instances in ONE launch: CTA b solves system work[b].y of instance work[b].x with
// the register-resident COCG of CTA size nt (>= every instance's minimum; kind 1 = tau, 2 = Strang spectra).
// insts, work: device arrays; nwork CTAs; smem_logL: the largest instance's logL.
cudaError_t launch_cocg_batched(const CocgBatchInst* insts, const int2* work, int nwork, int kind, int nt,
                                int smem_logL, cudaStream_t s);
// xb: [nsys][M] complex, right-hand sides on entry, solutions on exit.
// rws, pws: [nsys][M] complex workspace.  gbuf: global FFT scratch used when
// the transform does not fit in shared memory (may be null otherwise).
// iters[n]: iterations used; flags[n] & 3: 0 ok, 1 not converged, 2 breakdown, 3 non-finite.
// x0 (optional, [nsys][M] complex, M <= 8192): learned initial guesses; system n
// starts from x0[n] only if ||b - A x0[n]|| < ||b||, and then flags[n] |= 4.
cudaError_t launch_cocg_f32(float2* xb, float2* rws, float2* pws, int M, int logL, int nsys,
                            int inner, const CocgTables32& tb, float tol, int maxit, int* iters,
                            int* flags, int grid, cudaStream_t s, const float2* x0 = nullptr,
                            int threads = 0);
// Builds CocgTables32::sconv (out: [nsys][L] complex) for M <= 8192: the first column h of
// (lambda_n I + c S)^{-1} by the Bluestein preconditioner applied to e_0, wrapped into the
// length-L circulant g (g_d = h_d, g_{L-d} = h_{M-d}), transformed to fused order and divided by L.
cudaError_t launch_strang_conv_setup(int M, int logL, int nsys, const CocgTables32& tb, float2* out,
                                     cudaStream_t s);
// Smallest CTA size (64 .. 512) of the register-resident FP32 COCG kernel for M, or 0 when
// M > 8192 (the shared-memory kernel is used); `threads` of launch_cocg_f32 may be any power
// of two from this value to 512 (0: 512).
cudaError_t launch_cocg_f64(double2* xb, double2* rws, double2* pws, double2* gbuf, int M, int logL,
                            int nsys, int inner, const CocgTables64& tb, double tol, int maxit,
                            int* iters, int* flags, int grid, cudaStream_t s);
size_t cocg_gbuf_elems_f64(int logL, int grid);
// The direct tau-matrix Step (b): xb[n] <- (lambda_n I + c tau(T))^{-1} xb[n] for every n by one DST-I
// convolution (L = 2(M+1)); iters[n] = flags[n] = 0.  FP64 uses gbuf (grid CTAs) when the transform
// does not fit in shared memory (cocg_gbuf_elems_f64 != 0).
cudaError_t launch_tau_direct_f32(float2* xb, int M, int logL, int nsys, const CocgTables32& tb, int* iters,
                                  int* flags, cudaStream_t s);
cudaError_t launch_tau_direct_f64(double2* xb, double2* gbuf, int M, int logL, int nsys, const CocgTables64& tb,
                                  int* iters, int* flags, int grid, cudaStream_t s);
int cocg_reg_min_threads(int M);
// x[i] = deterministic pseudo-random values in [-1, 1)^2 (autotuner inputs)
cudaError_t launch_fill_test_rhs(float2* x, size_t n, cudaStream_t s);

// ---- exact-integer matvec (NTT), ntt.cu ---------------------------------------------
// Four primes p < 2^30 with 2^22 | p - 1 (product ~2^119.5) and a primitive root of each.
constexpr int kNttPrimes = 4;
constexpr uint32_t kNttPrime[kNttPrimes] = {1004535809u, 998244353u, 985661441u, 943718401u};
constexpr uint32_t kNttGen[kNttPrimes] = {3u, 3u, 3u, 7u};
// Twiddle tables of the transforms, per prime and direction, in the order the passes read
// them: 8 constant roots w^(e L / Rmax) (Rmax = min(16, L)), then for every pass but the last
// (stages s0 .. s0 + r - 1, r = min(4, logL - s0), S = L >> (s0 + r)) its (2^r - 1) S external
// twiddles w^(j bitrev_r(k) 2^s0) at (k - 1) S + j, so that consecutive threads (consecutive j)
// read consecutive entries.  Each entry is (w, floor(w 2^32 / p)).
#ifdef __CUDACC__
#define AAO_HD __host__ __device__
#else
#define AAO_HD
#endif
AAO_HD inline int ntt_pass_r(int logL, int s0) { return logL - s0 < 4 ? logL - s0 : 4; }
AAO_HD inline int ntt_last_pass(int logL) { return ((logL - 1) / 4) * 4; }
AAO_HD inline int ntt_tw_offset(int logL, int s0) {
  int off = 8;
  for (int t = 0; t < s0; t += 4) {
    const int r = ntt_pass_r(logL, t);
    off += ((1 << r) - 1) * (1 << (logL - t - r));
  }
  return off;
}
AAO_HD inline int ntt_tw_size(int logL) { return ntt_tw_offset(logL, ntt_last_pass(logL)); }
#undef AAO_HD
struct NttTables {
  const uint2* twf;     // [4][ntt_tw_size(logL)] forward roots w (a primitive L-th root mod p), layout above
  const uint2* twi;     // [4][ntt_tw_size(logL)] the same for w^-1
  const uint2* ghat;    // [4][L] stencil spectrum, bit-reversed, times L^-1
  uint2 crt[6];         // Garner constants (c, floor(c 2^32 / p_b)): p0^-1 mod p1, p2, p3, p1^-1 mod p2, p3,
                        // p2^-1 mod p3
  double c_gscale;      // 2^(e_g - 58): the stencil is c g quantised, G_j = round(c g_j 2^(58 - e_g))
  int gexp;             // e_g - 58
};
// w = calA v (or rhs - calA v) with c T v_k by exact NTT convolution of the row quantised to 58 bits
// (same contract as launch_matvec_f64; sq_partial gets ntt_partials(M, Nt) per-CTA sums).  res: 6 n uint32
// scratch (4 n residues, then n int64 quantised entries, 8-byte aligned when res is); rowscale: Nt doubles.
int ntt_partials(int M, int Nt);
// The FP32-row matvec w = calA v of the mixed Arnoldi step with the first Gram-Schmidt pass fused into its
// epilogue: dots_partial[b nv + i] (b < ntt_partials(M, Nt)) = partial sums of hi(w) hi(V_i), i < nv <= 65,
// for V a float-float basis (vectors vstride elements apart) -- launch_dots_ff's sums, one read of w less.
cudaError_t launch_matvec_ntt_fin_dots(const float* v, double* w, int M, int Nt, int logL, const NttTables& t,
                                       uint32_t* res, double* rowscale, const float2* V, size_t vstride, int nv,
                                       double* dots_partial, cudaStream_t s);
cudaError_t launch_matvec_ntt(const double* v, const double* rhs, double* w, double* sq_partial, int M, int Nt,
                              int logL, const NttTables& t, uint32_t* res, double* rowscale, cudaStream_t s);
// 2D (Eq. 4.2): w = band + c_x T_x v + c_y T_y v (or rhs - that) by exact line convolutions of every time level
// quantised to 58 bits (one scale per level), tx / ty the tables of the x and y stencils; sq_partial gets
// ntt2d_partials(Mx, My, Nt) per-CTA sums.  res: ntt2d_scratch_words(Mx, My, Nt) uint32 (8-byte aligned);
// levelscale: Nt doubles.
int ntt2d_partials(int Mx, int My, int Nt);
size_t ntt2d_scratch_words(int Mx, int My, int Nt);
cudaError_t launch_matvec2d_ntt(const double* v, const double* rhs, double* w, double* sq_partial, int Mx, int My,
                                int Nt, int logLx, int logLy, const NttTables& tx, const NttTables& ty, uint32_t* res,
                                double* levelscale, cudaStream_t s);
cudaError_t launch_matvec2d_ntt_fin(const float* v, const double* rhs, double* w, double* sq_partial, int Mx, int My,
                                    int Nt, int logLx, int logLy, const NttTables& tx, const NttTables& ty,
                                    uint32_t* res, double* levelscale, cudaStream_t s);
cudaError_t launch_matvec_ntt_fin(const float* v, const double* rhs, double* w, double* sq_partial, int M, int Nt,
                                  int logL, const NttTables& t, uint32_t* res, double* rowscale, cudaStream_t s);

// ---- 2D problem, twod.cu ----------------------------------------------------------------
// w = calA v (or rhs - calA v) for K = I (x) K_x + K_y (x) I (x fastest); tmp: n doubles of scratch;
// sq (optional): per-CTA sums of squares of w, mv2d_partials(Mx, Nt, logLy) of them.
cudaError_t launch_matvec2d_f64(const double* v, const double* rhs, double* w, double* tmp, double* sq, int Mx,
                                int My, int Nt, int logLx, int logLy, const double2* twx, const double2* twy,
                                const double* Exf, const double* Eyf, cudaStream_t s);
cudaError_t launch_matvec2d_f64_fin(const float* v, const double* rhs, double* w, double* tmp, double* sq, int Mx,
                                    int My, int Nt, int logLx, int logLy, const double2* twx, const double2* twy,
                                    const double* Exf, const double* Eyf, cudaStream_t s);
size_t mv2d_partials(int Mx, int Nt, int logLy);

template <typename R> struct VecT;
template <> struct VecT<float> { using c = float2; };
template <> struct VecT<double> { using c = double2; };
// Step (b) in 2D: all systems' COCG iterations with the 2D tau preconditioner.
template <typename R> struct Cocg2dArgs {
  using C = typename VecT<R>::c;
  C *X, *Rr, *P, *Z, *Q, *Tm;  // [nsys][My][Mx]; X: rhs in, solution out
  int Mx, My, nsys, logLx, logLy;
  const C *twx, *twy;          // exp(-2 pi i m / L) tables
  const R *Exf, *Eyf;          // c * DFT(embedding) / L, fused-pass order
  const R *sxn, *syf;          // c_x sigma^x (natural), c_y sigma^y (fused, 1e30 where the DST multiplier vanishes)
  const double2* lambda;
  void* state;                 // cocg2d_state_bytes(nsys)
  double2* part;               // nsys * cocg2d_max_partials(...) partial sums
  int* active_count;           // device int
  int* host_count;             // pinned host int
  int *iters, *flags;          // per system
  double tol;
  int maxit;
  int* it_dev;                 // device int: iterations of the current graph-driven loop
  long long* loops_total;      // device counter of graph-driven iterations (launch accounting)
  C* W2;                       // 2D Strang: [nsys][My][Lx] row spectra (null: the tau preconditioner)
  const C* G2;                 // 2D Strang: [nsys][Lx][Ly] spectra of the BCCB inverses (fused y order, / (Lx Ly))
};
size_t cocg2d_state_bytes(int nsys);
// The 2D Strang spectra G[n][p][f] = sum_{l,k} Qy[f][l] Qx[p][k] / (lambda_n + sy[l] + sx[k]) (Bt: nsys My Lx
// complex scratch); Qx: [Lx][Mx], Qy: [Ly][My] (host-built, see build_strang2d_q).
cudaError_t launch_strang2d_setup_f32(const float2* Qx, const float2* Qy, const float* sx, const float* sy,
                                      const double2* lambda, int Mx, int My, int logLx, int logLy, int nsys,
                                      float2* Bt, float2* G, cudaStream_t s);
cudaError_t launch_strang2d_setup_f64(const double2* Qx, const double2* Qy, const double* sx, const double* sy,
                                      const double2* lambda, int Mx, int My, int logLx, int logLy, int nsys,
                                      double2* Bt, double2* G, cudaStream_t s);
int cocg2d_max_partials(int Mx, int My, int logLx, int logLy, int csize);
cudaError_t launch_cocg2d_f32(const Cocg2dArgs<float>& a, cudaStream_t s, int* iters_run);
cudaError_t launch_cocg2d_f64(const Cocg2dArgs<double>& a, cudaStream_t s, int* iters_run);
// The same COCG recorded into the graph that s is capturing, its iterations as a conditional WHILE node
// (body captured on body_stream): 7 start kernels + 1, then 13 kernels per iteration, no host wait.
cudaError_t capture_cocg2d_f32(const Cocg2dArgs<float>& a, cudaStream_t s, cudaStream_t body_stream);
cudaError_t capture_cocg2d_f64(const Cocg2dArgs<double>& a, cudaStream_t s, cudaStream_t body_stream);
// The direct 2D tau-matrix Step (b) (Example 2, Eq. 4.5): X[n] <- (lambda_n I + c_x tau(T_x) (x) I +
// I (x) c_y tau(T_y))^{-1} X[n] by 2D DSTs (uses Tm, Q, state; iters = flags = 0).
cudaError_t launch_tau2d_direct_f32(const Cocg2dArgs<float>& a, cudaStream_t s);
cudaError_t launch_tau2d_direct_f64(const Cocg2dArgs<double>& a, cudaStream_t s);

// ---- vector kernels (FP64), blas.cu ----------------------------------------------------
int blas_partial_blocks();
// partial[b*nv + i] = sum over block b's elements of w[e] * V[i*vstride + e]
cudaError_t launch_dots(const double* w, const double* V, size_t vstride, int nv, size_t n,
                        double* partial, cudaStream_t s);
// w -= sum_i h[i] V_i; then partial dots of the updated w with V_i
cudaError_t launch_update_dots(double* w, const double* V, size_t vstride, int nv, size_t n,
                               const double* h, double* partial, cudaStream_t s);
// w -= sum_i h[i] V_i; then partial sum of squares of the updated w
cudaError_t launch_update_norm(double* w, const double* V, size_t vstride, int nv, size_t n,
                               const double* h, double* partial, cudaStream_t s);
// out[i] = sum_b partial[b*nv + i], fixed order
cudaError_t launch_reduce_partials(const double* partial, int nblocks, int nv, double* out,
                                   cudaStream_t s);
// The same three CGS2 sweeps on a float-float basis V (hi, lo per element, mixed precision): pass-1
// dots of the FP64 w in FP32; wout = w - sum h_i V_i (float-float) with the pass-2 dots; the pass-2
// update in place with ||w||^2.  Partial sums as launch_dots.
cudaError_t launch_dots_ff(const double* w, const float2* V, size_t vstride, int nv, size_t n, double* partial,
                           cudaStream_t s);
cudaError_t launch_update_dots_ff(const double* w, float2* wout, const float2* V, size_t vstride, int nv, size_t n,
                                  const double* h, double* partial, cudaStream_t s);
cudaError_t launch_update_norm_ff(float2* w, const float2* V, size_t vstride, int nv, size_t n, const double* h,
                                  double* partial, cudaStream_t s);
// y = a x (FP64 x into a float-float y) and x *= a (float-float x); a = *a_dev if a_dev != nullptr
cudaError_t launch_scale_to_ff(float2* y, const double* x, const double* a_dev, double a, size_t n, cudaStream_t s);
cudaError_t launch_scale_ff(float2* x, const double* a_dev, double a, size_t n, cudaStream_t s);
cudaError_t launch_scale(double* out, const double* in, double a, size_t n, cudaStream_t s);
// out = (*a_dev) * in, the factor read from device memory
cudaError_t launch_scale_dev(double* out, const double* in, const double* a_dev, size_t n, cudaStream_t s);
// U += sum_j y[j] Z_j in FP64 for FP32 Z (mixed path) or FP64 Z
cudaError_t launch_zy_update_f32(double* U, const float* Z, size_t zstride, int nz, size_t n, const double* y,
                                 cudaStream_t s);
cudaError_t launch_zy_update_f64(double* U, const double* Z, size_t zstride, int nz, size_t n,
                                 const double* y, cudaStream_t s);
cudaError_t launch_build_rhs(const double* u0, const double* f, double* F, double tau, int M, int Nt,
                             cudaStream_t s);
// out = a x + b y + c z elementwise (z may be null when c = 0); out may alias x, y or z
cudaError_t launch_lincomb3(double* out, double a, const double* x, double b, const double* y, double c,
                            const double* z, size_t n, cudaStream_t s);
// The right-hand side of one Horner step of the polynomial preconditioner (Sec. 3.1):
// w = v + ((C_eps - C) (x) I) z, i.e. w = v except in time rows 0 and 1:
//   w_0 = v_0 + z_0 / 2 + (eps/2) z_{Nt-2} - 2 eps z_{Nt-1},   w_1 = v_1 + (eps/2) z_{Nt-1}.
// v: FP64 or float-float (hi + lo); z: FP64 or FP32; Ms unknowns per time level.
cudaError_t launch_poly_rhs(double* w, const void* v, bool v_ff, const void* z, bool z_f32, double eps, size_t Ms,
                            int Nt, cudaStream_t s);
cudaError_t launch_f32_to_f64(const float* in, double* out, size_t n, cudaStream_t s);

// Message reported by aao_last_error(NULL) (calls without a plan).
void set_planless_error(const std::string& msg);
// Shape of a learned warm-start model (fno.cu).
int fno_grid_size(const aao_fno* f);
int fno_max_batch(const aao_fno* f);
}  // namespace aao
