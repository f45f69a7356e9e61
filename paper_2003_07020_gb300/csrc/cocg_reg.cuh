// Register-resident FP32 COCG for Step (b) (Sec. 3.1), shared by the translation units that
// instantiate it (cocg.cu: the Bluestein Strang form; cocg_reg_tau.cu and cocg_reg_sconv.cu:
// the tau matrix and the precomputed Strang spectra, each for every CTA size and with or without
// a learned initial guess).  Splitting the instantiations keeps each file's compile short and
// lets them build in parallel.
#pragma once
#include "common.cuh"
#include "kernels.h"

namespace aao {

template <typename C> __device__ __forceinline__ C cdiv(C a, C b) {
  const auto d = b.x * b.x + b.y * b.y;
  return C{(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}

// COCG breakdown test for a bilinear product u^T w used as a divisor: it is treated as zero when
// |u^T w| <= kappa ||u|| ||w||, kappa = 64 units of roundoff, i.e. below the rounding error of
// the dot product itself, where its phase is no longer determined by the data.
template <typename R> __host__ __device__ constexpr R breakdown_rel() {
  return sizeof(R) == 4 ? (R)(64.0 / 16777216.0) : (R)(64.0 / 9007199254740992.0);
}
template <typename R>
__device__ __forceinline__ bool near_breakdown(R re, R im, R uu, R ww) {
  const R k = breakdown_rel<R>();
  return !(re * re + im * im > k * k * uu * ww);
}

// ---- spectrum providers for the fused pass: element access and blocks of R values by 16-byte loads ----
// (a thread's group of R factors is contiguous and starts at a multiple of R, so the loads are aligned)
struct RealSpec32 {  // (e_k, 0), e real
  const float* e;
  __device__ __forceinline__ float2 operator()(int k) const { return float2{__ldg(&e[k]), 0.0f}; }
  template <int R> __device__ __forceinline__ void block(int s, float2 (&f)[R]) const {
    if constexpr (R % 4 == 0) {
      const float4* e4 = reinterpret_cast<const float4*>(e + s);
#pragma unroll
      for (int m = 0; m < R / 4; ++m) {
        const float4 a = __ldg(&e4[m]);
        f[4 * m] = float2{a.x, 0.0f};
        f[4 * m + 1] = float2{a.y, 0.0f};
        f[4 * m + 2] = float2{a.z, 0.0f};
        f[4 * m + 3] = float2{a.w, 0.0f};
      }
    } else {
#pragma unroll
      for (int m = 0; m < R; ++m) f[m] = (*this)(s + m);
    }
  }
};
struct CplxSpec32 {  // complex values
  const float2* c;
  __device__ __forceinline__ float2 operator()(int k) const { return __ldg(&c[k]); }
  template <int R> __device__ __forceinline__ void block(int s, float2 (&f)[R]) const {
    if constexpr (R % 2 == 0) {
      const float4* c4 = reinterpret_cast<const float4*>(c + s);
#pragma unroll
      for (int m = 0; m < R / 2; ++m) {
        const float4 a = __ldg(&c4[m]);
        f[2 * m] = float2{a.x, a.y};
        f[2 * m + 1] = float2{a.z, a.w};
      }
    } else {
#pragma unroll
      for (int m = 0; m < R; ++m) f[m] = (*this)(s + m);
    }
  }
};

struct TauSpec32 {  // 1 / (L (lambda + sigma_p)), sigma real
  const float* sig;
  float2 lam;
  float invL;
  __device__ __forceinline__ float2 at(float sg) const {
    float2 d = lam;
    d.x += sg;
    return cdiv(float2{invL, 0}, d);
  }
  __device__ __forceinline__ float2 operator()(int p) const { return at(__ldg(&sig[p])); }
  template <int R> __device__ __forceinline__ void block(int s, float2 (&f)[R]) const {
    if constexpr (R % 4 == 0) {
      const float4* s4 = reinterpret_cast<const float4*>(sig + s);
#pragma unroll
      for (int m = 0; m < R / 4; ++m) {
        const float4 a = __ldg(&s4[m]);
        f[4 * m] = at(a.x);
        f[4 * m + 1] = at(a.y);
        f[4 * m + 2] = at(a.z);
        f[4 * m + 3] = at(a.w);
      }
    } else {
#pragma unroll
      for (int m = 0; m < R; ++m) f[m] = (*this)(s + m);
    }
  }
};

// ---- FP32 path with register-resident vectors -------------------------------------------
// NT threads (64 .. 512, chosen per problem by the autotuner of plan creation); thread t owns
// elements i = t + NT j, j < 16 (M <= 16 NT), so r and p live in registers for the whole solve
// and only x is updated in global memory.  Every variant keeps <= 128 registers per thread so
// that 512 / NT CTAs fit on an SM.
constexpr int kRegMaxThreads = 512;
constexpr int kRegElems = 16;

// The embedding length L = 32 NT, for which the first and last FFT passes (2^r0 points at stride
// S0 = L / 2^r0, a multiple of NT) only touch elements t + NT m of one thread t.
template <int NT> __host__ __device__ constexpr int own_logL() { return NT == 64 ? 11 : NT == 128 ? 12 : NT == 256 ? 13 : 14; }

// For L = 32 NT: buf[i] <- (backward(factor .* forward(x)))[i] for the thread's own elements
// i = t + NT j (j < 16) of the register vector x (element t + NT j in x[j], zero at and beyond M,
// so the upper half of the embedding is zero).  The first forward pass reads its groups
// (elements t + NT (a + k A), k < 2^r0 / 2; the rest are zero) from registers and the last backward
// pass stores only the lower half of each group, which are the thread's own elements: no staging
// sweep, no zero fill and no trailing barrier, since each thread then reads back only its own
// elements.  Starts synchronised.
template <int NT, typename F>
__device__ __forceinline__ void fft_convolve_own(float2* buf, const float2 (&x)[kRegElems], const float2* q,
                                                 F factor, const float2* pt) {
  constexpr int LOGL = own_logL<NT>(), L = 1 << LOGL;
  constexpr int r0 = (LOGL & 3) ? (LOGL & 3) : 4, R0 = 1 << r0, S0 = L / R0, A = S0 / NT;
  static_assert(S0 % NT == 0 && A * R0 / 2 == kRegElems, "first-pass groups must be thread-local");
  const int t = threadIdx.x;
  __syncthreads();
#pragma unroll
  for (int a = 0; a < A; ++a) {
    const int j0 = t + NT * a;
    float2 v[R0];
#pragma unroll
    for (int k = 0; k < R0; ++k) v[k] = k < R0 / 2 ? x[a + k * A] : float2{0, 0};
    dft<-1, r0>(v);
    if (j0 != 0) {
#pragma unroll
      for (int m = 1; m < R0; ++m) v[m] = cmul(v[m], twiddle<-1>(q, j0 * m, LOGL));
    }
#pragma unroll
    for (int m = 0; m < R0; ++m) buf[pad16(j0 + brev_c<r0>(m) * S0)] = v[m];
  }
  __syncthreads();
  fft_convolve_inner(buf, LOGL, q, LOGL, factor, pt);
#pragma unroll
  for (int a = 0; a < A; ++a) {
    const int j0 = t + NT * a;
    float2 v[R0];
#pragma unroll
    for (int m = 0; m < R0; ++m) v[m] = buf[pad16(j0 + brev_c<r0>(m) * S0)];
    if (j0 != 0) {
#pragma unroll
      for (int m = 1; m < R0; ++m) v[m] = cmul(v[m], twiddle<+1>(q, j0 * m, LOGL));
    }
    dft<+1, r0>(v);
#pragma unroll
    for (int k = 0; k < R0 / 2; ++k) buf[pad16(j0 + k * S0)] = v[k];
  }
}

// buf[i] <- (c T x)[i] (the Toeplitz product by its circulant embedding, real spectrum Ebr) for the
// thread's own elements i = t + NT j < M; starts synchronised.
template <int NT>
__device__ __forceinline__ void toeplitz_reg(float2* buf, const float2 (&x)[kRegElems], int M, int logL,
                                             const CocgTables32& tb, const float2* q, const float2* pt) {
  const RealSpec32 ef{tb.Ebr};
  if (logL == own_logL<NT>()) {
    fft_convolve_own<NT>(buf, x, q, ef, pt);
    return;
  }
  const int L = 1 << logL;
  const int t = threadIdx.x;
  __syncthreads();  // earlier readers of buf are done
#pragma unroll
  for (int j = 0; j < kRegElems; ++j) {
    const int i = t + NT * j;
    if (i < L) buf[pad16(i)] = (i < M) ? x[j] : float2{0, 0};
  }
  for (int i = t + NT * kRegElems; i < L; i += NT) buf[pad16(i)] = float2{0, 0};
  fft_convolve(buf, logL, q, logL, ef, pt);
}

// KIND 0: Strang by Bluestein (4 FFTs of L); 1: natural tau matrix by DST-I (2 FFTs); 2: Strang by
// the precomputed per-system circulant spectrum sc (2 FFTs).  The result is read by zval().
template <int KIND, int NT>
__device__ __forceinline__ void precond_reg(float2* buf, const float2 (&r)[kRegElems], int M, int logL, float2 lam,
                                            const CocgTables32& tb, const float2* q, const float2* pt,
                                            const float2* __restrict__ sc) {
  const int L = 1 << logL;
  const int t = threadIdx.x;
  if constexpr (KIND == 2) {
    const CplxSpec32 sf{sc};
    if (logL == own_logL<NT>()) {
      fft_convolve_own<NT>(buf, r, q, sf, pt);
      return;
    }
    __syncthreads();  // earlier readers of buf are done
#pragma unroll
    for (int j = 0; j < kRegElems; ++j) {
      const int i = t + NT * j;
      if (i < L) buf[pad16(i)] = (i < M) ? r[j] : float2{0, 0};
    }
    for (int i = t + NT * kRegElems; i < L; i += NT) buf[pad16(i)] = float2{0, 0};
    fft_convolve(buf, logL, q, logL, sf, pt);
  } else if constexpr (KIND == 0) {
#pragma unroll
    for (int j = 0; j < kRegElems; ++j) {
      const int i = t + NT * j;
      if (i < L) buf[pad16(i)] = (i < M) ? cmul(r[j], __ldg(&tb.chirp[i])) : float2{0, 0};
    }
    for (int i = t + NT * kRegElems; i < L; i += NT) buf[pad16(i)] = float2{0, 0};
    fft_convolve(buf, logL, q, logL, [&](int p) { return __ldg(&tb.chat_br[p]); }, pt);
    const float invM = 1.0f / (float)M;
#pragma unroll
    for (int j = 0; j < kRegElems; ++j) {
      const int k = t + NT * j;
      if (k < M) {
        float2 d = lam;
        d.x += __ldg(&tb.seig[k]);
        buf[pad16(k)] = cscale(cdiv(buf[pad16(k)], d), invM);
      } else if (k < L) {
        buf[pad16(k)] = float2{0, 0};
      }
    }
    for (int i = t + NT * kRegElems; i < L; i += NT) buf[pad16(i)] = float2{0, 0};
    fft_convolve(buf, logL, q, logL, [&](int p) { return cconj(__ldg(&tb.chat_br[p])); }, pt);
  } else {
    (void)sc;
    if (t == 0) {
      buf[pad16(0)] = float2{0, 0};
      buf[pad16(M + 1)] = float2{0, 0};
    }
#pragma unroll
    for (int j = 0; j < kRegElems; ++j) {
      const int i = t + NT * j;
      if (i < M) {
        buf[pad16(i + 1)] = r[j];
        buf[pad16(L - 1 - i)] = float2{-r[j].x, -r[j].y};
      }
    }
    const TauSpec32 tf{tb.taueig_br, lam, 1.0f / (float)L};
    fft_convolve(buf, logL, q, logL, tf, pt);
  }
}

// Element i of the preconditioned residual left in buf by precond_reg<KIND>.
template <int KIND>
__device__ __forceinline__ float2 zval(const float2* buf, const CocgTables32& tb, int i) {
  if constexpr (KIND == 0) return cmulc(buf[pad16(i)], __ldg(&tb.chirp[i]));
  else if constexpr (KIND == 1) return buf[pad16(i + 1)];
  else return buf[pad16(i)];
}

// One shifted system n: right-hand side in xb[n] on entry, COCG solution there on exit (x0b: learned
// initial guesses when WARM).  buf, q, pt: the CTA's FFT buffer and twiddle tables for logL; red: the block
// reduction scratch.  Starts and ends synchronised.
template <int KIND, bool WARM, int NT>
__device__ __forceinline__ void cocg_reg_solve(int n, float2* __restrict__ xb, const float2* __restrict__ x0b, int M,
                                               int logL, const CocgTables32& tb, float tol, int maxit,
                                               int* __restrict__ iters, int* __restrict__ flags, float2* buf,
                                               const float2* q, const float2* pt, float* red) {
  const int t = threadIdx.x;
  const double2 lamd = tb.lambda[n];
  const float2 lam{(float)lamd.x, (float)lamd.y};
  float2* x = xb + (size_t)n * M;
  const float2* sc = KIND == 2 ? tb.sconv + ((size_t)n << logL) : nullptr;
  float2 r[kRegElems], p[kRegElems];
  // The iteration runs on b / ||b||_1 (x stays in the units of b): COCG is scale invariant, and the
  // normalised vectors keep the squared norms and the breakdown products far from FP32 underflow even
  // when b is at rounding level (a frequency that Step (a) cancels).
  float b1[1] = {0};
#pragma unroll
  for (int j = 0; j < kRegElems; ++j) {
    const int i = t + NT * j;
    r[j] = (i < M) ? x[i] : float2{0, 0};
    b1[0] += fabsf(r[j].x) + fabsf(r[j].y);
  }
  block_sum<float, 1>(b1, red);
#pragma unroll
  for (int j = 0; j < kRegElems; ++j) {
    const int i = t + NT * j;
    if (i < M) x[i] = float2{0, 0};
  }
  if (!(b1[0] > 0.0f) || b1[0] > 3.0e38f) {  // zero right-hand side, or NaN / infinity in it
    if (t == 0) { iters[n] = 0; flags[n] = b1[0] == 0.0f ? 0 : 3; }
    return;
  }
  const float bs = b1[0], ibs = 1.0f / bs;
  float nb2[1] = {0};
#pragma unroll
  for (int j = 0; j < kRegElems; ++j) {
    r[j] = float2{r[j].x * ibs, r[j].y * ibs};
    nb2[0] += r[j].x * r[j].x + r[j].y * r[j].y;
  }
  block_sum<float, 1>(nb2, red);
  const float thr = tol * tol * nb2[0];
  int accepted = 0;
  if constexpr (WARM) {
    // warm start: r0 = b - (lambda I + c T) x0, kept only if ||r0|| < ||b||
    const float2* x0 = x0b + (size_t)n * M;
    float2 w[kRegElems];
#pragma unroll
    for (int j = 0; j < kRegElems; ++j) {
      const int i = t + NT * j;
      w[j] = (i < M) ? float2{x0[i].x * ibs, x0[i].y * ibs} : float2{0, 0};
    }
    toeplitz_reg<NT>(buf, w, M, logL, tb, q, pt);
    float r02[1] = {0};
#pragma unroll
    for (int j = 0; j < kRegElems; ++j) {
      const int i = t + NT * j;
      if (i < M) {
        const float2 rj = csub(r[j], cadd(buf[pad16(i)], cmul(lam, w[j])));
        r02[0] += rj.x * rj.x + rj.y * rj.y;
      }
    }
    block_sum<float, 1>(r02, red);
    if (r02[0] < nb2[0]) {  // uniform across the block
      accepted = 1;
#pragma unroll
      for (int j = 0; j < kRegElems; ++j) {
        const int i = t + NT * j;
        if (i < M) {
          r[j] = csub(r[j], cadd(buf[pad16(i)], cmul(lam, w[j])));
          x[i] = x0[i];
        }
      }
      if (r02[0] <= thr) {
        if (t == 0) { iters[n] = 0; flags[n] = 4; }
        __syncthreads();
        return;
      }
    }
    __syncthreads();
  }
  // z = P^{-1} r, p = z, rho = r^T z
  precond_reg<KIND, NT>(buf, r, M, logL, lam, tb, q, pt, sc);
  float rho2[4] = {0, 0, 0, 0};  // r^T z, |z|^2, |r|^2
#pragma unroll
  for (int j = 0; j < kRegElems; ++j) {
    const int i = t + NT * j;
    float2 z{0, 0};
    if (i < M) z = zval<KIND>(buf, tb, i);
    p[j] = z;
    rho2[0] += r[j].x * z.x - r[j].y * z.y;
    rho2[1] += r[j].x * z.y + r[j].y * z.x;
    rho2[2] += z.x * z.x + z.y * z.y;
    rho2[3] += r[j].x * r[j].x + r[j].y * r[j].y;
  }
  block_sum<float, 4>(rho2, red);
  float2 rho{rho2[0], rho2[1]};
  int it = 0, flag = 1;
  const bool bd0 = near_breakdown(rho2[0], rho2[1], rho2[2], rho2[3]);  // z^T r of the first step
  if (bd0) flag = 2;
  while (!bd0 && it < maxit) {
    // q = (lambda I + c T) p
    toeplitz_reg<NT>(buf, p, M, logL, tb, q, pt);
    float pq2[4] = {0, 0, 0, 0};  // p^T q, |p|^2, |q|^2
#pragma unroll
    for (int j = 0; j < kRegElems; ++j) {
      const int i = t + NT * j;
      if (i < M) {
        const float2 qq = cadd(buf[pad16(i)], cmul(lam, p[j]));
        pq2[0] += p[j].x * qq.x - p[j].y * qq.y;
        pq2[1] += p[j].x * qq.y + p[j].y * qq.x;
        pq2[2] += p[j].x * p[j].x + p[j].y * p[j].y;
        pq2[3] += qq.x * qq.x + qq.y * qq.y;
      }
    }
    block_sum<float, 4>(pq2, red);
    const float2 pq{pq2[0], pq2[1]};
    if (near_breakdown(pq2[0], pq2[1], pq2[2], pq2[3])) { flag = 2; break; }
    const float2 a = cdiv(rho, pq);
    const float2 ax{a.x * bs, a.y * bs};  // the step in the units of b
    float rr[1] = {0};
#pragma unroll
    for (int j = 0; j < kRegElems; ++j) {
      const int i = t + NT * j;
      if (i < M) {
        const float2 qq = cadd(buf[pad16(i)], cmul(lam, p[j]));
        x[i] = cadd(x[i], cmul(ax, p[j]));
        r[j] = csub(r[j], cmul(a, qq));
        rr[0] += r[j].x * r[j].x + r[j].y * r[j].y;
      }
    }
    block_sum<float, 1>(rr, red);
    ++it;
    if (!(rr[0] == rr[0]) || rr[0] > 1e30f * nb2[0]) { flag = 3; break; }
    if (rr[0] <= thr) { flag = 0; break; }
    precond_reg<KIND, NT>(buf, r, M, logL, lam, tb, q, pt, sc);
    float rn2[3] = {0, 0, 0};  // r^T z, |z|^2
#pragma unroll
    for (int j = 0; j < kRegElems; ++j) {
      const int i = t + NT * j;
      if (i < M) {
        const float2 z = zval<KIND>(buf, tb, i);
        rn2[0] += r[j].x * z.x - r[j].y * z.y;
        rn2[1] += r[j].x * z.y + r[j].y * z.x;
        rn2[2] += z.x * z.x + z.y * z.y;
      }
    }
    block_sum<float, 3>(rn2, red);
    const float2 rho_new{rn2[0], rn2[1]};
    // rho_new divides the next beta: |r^T z| at rounding level of ||r|| ||z|| is a breakdown
    if (near_breakdown(rn2[0], rn2[1], rn2[2], rr[0])) { flag = 2; break; }
    const float2 beta = cdiv(rho_new, rho);
    rho = rho_new;
#pragma unroll
    for (int j = 0; j < kRegElems; ++j) {
      const int i = t + NT * j;
      float2 z{0, 0};
      if (i < M) z = zval<KIND>(buf, tb, i);
      p[j] = cadd(z, cmul(beta, p[j]));
    }
    __syncthreads();
  }
  if (t == 0) { iters[n] = it; flags[n] = flag | (accepted << 2); }
  __syncthreads();
}

template <int KIND, bool WARM, int NT>
__global__ void __launch_bounds__(NT, kRegMaxThreads / NT)
    cocg_reg_kernel(float2* __restrict__ xb, const float2* __restrict__ x0b, int M, int logL, int nsys,
                    CocgTables32 tb, float tol, int maxit, int* __restrict__ iters, int* __restrict__ flags) {
  extern __shared__ unsigned char smraw[];
  __shared__ float red[4 * 32];
  float2* buf = reinterpret_cast<float2*>(smraw);
  float2* q = buf + padded_size(1 << logL);
  float2* pt = q + (1 << logL) / 4;  // per-pass twiddle tables
  const int L = 1 << logL;
  load_quarter(q, tb.twL, L / 4);
  __syncthreads();
  build_pass_tables(pt, q, logL, logL);
  for (int n = blockIdx.x; n < nsys; n += gridDim.x)
    cocg_reg_solve<KIND, WARM, NT>(n, xb, x0b, M, logL, tb, tol, maxit, iters, flags, buf, q, pt, red);
}

// Step (b) of many independent problems in one launch: CTA b solves system work[b].y of instance work[b].x
// (its sizes, tables, tolerance and buffers in insts[work[b].x]), with the same per-system code as
// cocg_reg_kernel.  Shared memory for the largest instance.
template <int KIND, int NT>
__global__ void __launch_bounds__(NT, kRegMaxThreads / NT)
    cocg_reg_batched_kernel(const CocgBatchInst* __restrict__ insts, const int2* __restrict__ work) {
  extern __shared__ unsigned char smraw[];
  __shared__ float red[4 * 32];
  const int2 w = work[blockIdx.x];
  const CocgBatchInst I = insts[w.x];
  float2* buf = reinterpret_cast<float2*>(smraw);
  float2* q = buf + padded_size(1 << I.logL);
  float2* pt = q + (1 << I.logL) / 4;
  load_quarter(q, I.tb.twL, (1 << I.logL) / 4);
  __syncthreads();
  build_pass_tables(pt, q, I.logL, I.logL);
  cocg_reg_solve<KIND, false, NT>(w.y, I.xb, nullptr, I.M, I.logL, I.tb, I.tol, I.maxit, I.iters, I.flags, buf, q,
                                  pt, red);
}

template <typename R>
static size_t cocg_smem(int logL) { return (size_t)padded_size(1 << logL) * sizeof(typename cplx_t<R>::type); }
template <typename R>
static size_t cocg_table_bytes(int logL) { return (size_t)(1 << (logL - 2)) * sizeof(typename cplx_t<R>::type); }
static inline size_t cocg_reg_smem(int logL) {
  return cocg_smem<float>(logL) + cocg_table_bytes<float>(logL) + (size_t)pass_table_size(logL) * sizeof(float2);
}

template <int KIND, bool WARM, int NT>
static cudaError_t launch_reg_one(float2* xb, const float2* x0, int M, int logL, int nsys, const CocgTables32& tb,
                                  float tol, int maxit, int* iters, int* flags, int grid, cudaStream_t s) {
  auto kern = cocg_reg_kernel<KIND, WARM, NT>;
  cudaError_t e = allow_max_dynamic_smem(kern);
  if (e != cudaSuccess) return e;
  kern<<<grid, NT, cocg_reg_smem(logL), s>>>(xb, x0, M, logL, nsys, tb, tol, maxit, iters, flags);
  return cudaGetLastError();
}

// Every CTA size (64 .. 512) and both initial-guess forms of one preconditioner kind.
template <int KIND>
static cudaError_t launch_reg_kind(float2* xb, const float2* x0, int M, int logL, int nsys, const CocgTables32& tb,
                                   float tol, int maxit, int* iters, int* flags, int grid, int nt, cudaStream_t s) {
#define AAO_REG_NT(N)                                                                                      \
  case N:                                                                                                  \
    return x0 ? launch_reg_one<KIND, true, N>(xb, x0, M, logL, nsys, tb, tol, maxit, iters, flags, grid, s) \
              : launch_reg_one<KIND, false, N>(xb, x0, M, logL, nsys, tb, tol, maxit, iters, flags, grid, s);
  switch (nt) {
    AAO_REG_NT(64)
    AAO_REG_NT(128)
    AAO_REG_NT(256)
    AAO_REG_NT(512)
    default: return cudaErrorInvalidValue;
  }
#undef AAO_REG_NT
}

// Per-kind entry points (defined in cocg_reg_tau.cu and cocg_reg_sconv.cu).
cudaError_t launch_cocg_reg_tau(float2* xb, const float2* x0, int M, int logL, int nsys, const CocgTables32& tb,
                                float tol, int maxit, int* iters, int* flags, int grid, int nt, cudaStream_t s);
cudaError_t launch_cocg_reg_sconv(float2* xb, const float2* x0, int M, int logL, int nsys, const CocgTables32& tb,
                                  float tol, int maxit, int* iters, int* flags, int grid, int nt, cudaStream_t s);

}  // namespace aao
