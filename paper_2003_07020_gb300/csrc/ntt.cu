// All-at-once matvec, Sec. 3.2, with the Toeplitz product c T v_k computed
// EXACTLY for quantised inputs by number-theoretic transforms (NTT) instead of
// FP64 FFTs (the FP64 pipe of this GPU issues ~1.6 DFMA per clock per SM; its
// integer pipes are an order of magnitude faster).
//
// Row k of v is scaled by a power of two so that its largest magnitude lies in
// [2^50, 2^51) and rounded to integers V (relative quantisation error 2^-52,
// FP64 level); the FCD stencil g is quantised the same way once at plan
// creation (G).  The linear convolution Y = G * V has |Y| < M 2^102 <= 2^115
// and is computed modulo four NTT primes p_q < 2^30 (product ~2^119.5) by
// cyclic convolution of length L >= 2M - 1 (circulant embedding), then
// reconstructed by Garner's mixed-radix CRT and converted to FP64:
// c T v_k = c 2^(e_v + e_g - 102) Y.
//
// Kernel 1 (ntt_conv_kernel): one CTA per (time row, prime): quantise the row
// mod p, forward NTT (radix-4 DIF passes in shared memory, natural order in,
// bit-reversed out), multiply by the stencil spectrum (stored bit-reversed,
// L^-1 folded in), inverse NTT (radix-4 DIT, bit-reversed in, natural out),
// write the residues of the first M outputs.
// Kernel 2 (ntt_epilogue_kernel): one CTA per row: Garner CRT of the four
// residues, scaling, the BDF band of C (Eq. 1.7), optional residual rhs - w and
// per-row sums of squares (as the FP64 matvec).
//
// Modular arithmetic: Shoup multiplication by a constant w with precomputed
// w' = floor(w 2^32 / p), lazy values in [0, 2p) (p < 2^30 keeps all sums
// below 2^32).
#include "common.cuh"
#include "kernels.h"

namespace aao {

namespace {

constexpr uint32_t kP0 = kNttPrime[0], kP1 = kNttPrime[1], kP2 = kNttPrime[2], kP3 = kNttPrime[3];
template <int Q> struct Prime;
template <> struct Prime<0> { static constexpr uint32_t p = kP0; };
template <> struct Prime<1> { static constexpr uint32_t p = kP1; };
template <> struct Prime<2> { static constexpr uint32_t p = kP2; };
template <> struct Prime<3> { static constexpr uint32_t p = kP3; };

// a * w mod p in [0, 2p) for a < 2^32, w = (w, floor(w 2^32 / p))
template <uint32_t P>
__device__ __forceinline__ uint32_t mulsh(uint32_t a, uint2 w) {
  const uint32_t q = __umulhi(a, w.y);
  return a * w.x - q * P;
}
template <uint32_t P> __device__ __forceinline__ uint32_t red2(uint32_t a) { return a >= 2 * P ? a - 2 * P : a; }
template <uint32_t P> __device__ __forceinline__ uint32_t red1(uint32_t a) { return a >= P ? a - P : a; }

// Gentleman-Sande butterfly: (x, y) -> (x + y, (x - y) w), all in [0, 2p)
template <uint32_t P>
__device__ __forceinline__ void dif2(uint32_t& x, uint32_t& y, uint2 w) {
  const uint32_t s = x + y, d = x - y + 2 * P;
  x = red2<P>(s);
  y = mulsh<P>(d, w);
}
// Cooley-Tukey butterfly: (x, y) -> (x + y w, x - y w), all in [0, 2p)
template <uint32_t P>
__device__ __forceinline__ void dit2(uint32_t& x, uint32_t& y, uint2 w) {
  const uint32_t t = mulsh<P>(y, w);
  const uint32_t s = x + t, d = x - t + 2 * P;
  x = red2<P>(s);
  y = red2<P>(d);
}

// Forward cyclic NTT X[k] = sum_j x_j w^{jk} (w a primitive L-th root, tw[e] = w^e for e < L/2),
// natural order in, bit-reversed order out.  Each radix-4 pass performs the DIF stages of half
// sizes h and h/2; an odd last stage (h = 1) is done as a radix-2 pass.
template <uint32_t P>
__device__ void ntt_dif(uint32_t* buf, int logL, const uint2* __restrict__ tw) {
  const int L = 1 << logL;
  int s = 0;
  for (; s + 2 <= logL; s += 2) {
    const int h = L >> (s + 1), hq = h >> 1;
    __syncthreads();
    for (int g = threadIdx.x; g < L / 4; g += blockDim.x) {
      const int b = g >> (logL - s - 2), j = g & (hq - 1);
      const int i0 = (b << (logL - s)) + j, i1 = i0 + hq, i2 = i0 + h, i3 = i2 + hq;
      uint32_t a0 = buf[i0], a1 = buf[i1], a2 = buf[i2], a3 = buf[i3];
      const int e1 = j << s;
      const uint2 w1 = __ldg(&tw[e1]), w2 = __ldg(&tw[e1 + (L >> 2)]), w3 = __ldg(&tw[e1 << 1]);
      dif2<P>(a0, a2, w1);
      dif2<P>(a1, a3, w2);
      dif2<P>(a0, a1, w3);
      dif2<P>(a2, a3, w3);
      buf[i0] = a0;
      buf[i1] = a1;
      buf[i2] = a2;
      buf[i3] = a3;
    }
  }
  if (s < logL) {
    __syncthreads();
    const uint2 w0 = __ldg(&tw[0]);
    for (int g = threadIdx.x; g < L / 2; g += blockDim.x) {
      uint32_t a = buf[2 * g], c = buf[2 * g + 1];
      dif2<P>(a, c, w0);
      buf[2 * g] = a;
      buf[2 * g + 1] = c;
    }
  }
  __syncthreads();
}

// Inverse (unnormalised) cyclic NTT x_j = sum_k X[k] w^{-jk} (twi[e] = w^{-e}), bit-reversed order
// in, natural order out: radix-4 DIT passes of half sizes h and 2h, an odd first stage (h = 1)
// as a radix-2 pass.
template <uint32_t P>
__device__ void ntt_dit(uint32_t* buf, int logL, const uint2* __restrict__ twi) {
  const int L = 1 << logL;
  int s = 0;
  if (logL & 1) {
    __syncthreads();
    const uint2 w0 = __ldg(&twi[0]);
    for (int g = threadIdx.x; g < L / 2; g += blockDim.x) {
      uint32_t a = buf[2 * g], c = buf[2 * g + 1];
      dit2<P>(a, c, w0);
      buf[2 * g] = a;
      buf[2 * g + 1] = c;
    }
    s = 1;
  }
  for (; s + 2 <= logL; s += 2) {
    const int h = 1 << s;
    __syncthreads();
    for (int g = threadIdx.x; g < L / 4; g += blockDim.x) {
      const int b = g >> s, j = g & (h - 1);
      const int i0 = (b << (s + 2)) + j, i1 = i0 + h, i2 = i1 + h, i3 = i2 + h;
      uint32_t a0 = buf[i0], a1 = buf[i1], a2 = buf[i2], a3 = buf[i3];
      const int e2 = j << (logL - s - 2);
      const uint2 w1 = __ldg(&twi[e2 << 1]), w2 = __ldg(&twi[e2]), w3 = __ldg(&twi[e2 + (L >> 2)]);
      dit2<P>(a0, a1, w1);
      dit2<P>(a2, a3, w1);
      dit2<P>(a0, a2, w2);
      dit2<P>(a1, a3, w3);
      buf[i0] = a0;
      buf[i1] = a1;
      buf[i2] = a2;
      buf[i3] = a3;
    }
  }
  __syncthreads();
}

template <typename TIn> __device__ __forceinline__ double ldd(const TIn* p) { return (double)__ldg(p); }

template <typename TIn, int Q>
__device__ __forceinline__ void conv_row(const TIn* __restrict__ vk, int M, int logL, double qs,
                                         const NttTables& t, uint32_t* buf, uint32_t* __restrict__ out) {
  constexpr uint32_t P = Prime<Q>::p;
  const int L = 1 << logL;
  const size_t half = (size_t)(L >> 1);
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    uint32_t r = 0;
    if (i < M) {
      const long long V = __double2ll_rn(ldd(vk + i) * qs);  // |V| <= 2^51, exact power-of-two scaling
      long long m = V % (long long)P;
      if (m < 0) m += P;
      r = (uint32_t)m;
    }
    buf[i] = r;
  }
  ntt_dif<P>(buf, logL, t.twf + Q * half);
  const uint2* gh = t.ghat + (size_t)Q * L;
  for (int k = threadIdx.x; k < L; k += blockDim.x) buf[k] = mulsh<P>(buf[k], __ldg(&gh[k]));
  ntt_dit<P>(buf, logL, t.twi + Q * half);
  for (int i = threadIdx.x; i < M; i += blockDim.x) out[i] = red1<P>(red2<P>(buf[i]));
}

// grid (Nt, 4): blockIdx.y selects the prime.  res: [4][Nt][M] residues; rowscale[k] = 2^(e_v - 51)
// (0 for a zero row, NaN for a row with a non-finite entry), written by the prime-0 CTAs.
template <typename TIn>
__global__ void __launch_bounds__(512) ntt_conv_kernel(const TIn* __restrict__ v, int M, int Nt, int logL,
                                                       NttTables t, uint32_t* __restrict__ res,
                                                       double* __restrict__ rowscale) {
  extern __shared__ uint32_t nbuf[];
  __shared__ double red[32];
  __shared__ int bad_any;
  const int k = blockIdx.x, q = blockIdx.y;
  const TIn* vk = v + (size_t)k * M;
  if (threadIdx.x == 0) bad_any = 0;
  double mx = 0.0;
  int bad = 0;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    const double a = fabs(ldd(vk + i));
    if (!(a <= 1.7976931348623157e308)) bad = 1;  // NaN or Inf
    else mx = fmax(mx, a);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __syncthreads();
  if (bad) bad_any = 1;
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  mx = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
  int ev = 0;
  if (mx > 0) frexp(mx, &ev);                // mx < 2^ev
  const double qs = mx > 0 ? ldexp(1.0, 51 - ev) : 0.0;
  if (q == 0 && threadIdx.x == 0) rowscale[k] = bad_any ? __longlong_as_double(0x7ff8000000000000ll)
                                                        : (mx > 0 ? ldexp(1.0, ev - 51) : 0.0);
  uint32_t* out = res + ((size_t)q * Nt + k) * M;
  switch (q) {
    case 0: conv_row<TIn, 0>(vk, M, logL, qs, t, nbuf, out); break;
    case 1: conv_row<TIn, 1>(vk, M, logL, qs, t, nbuf, out); break;
    case 2: conv_row<TIn, 2>(vk, M, logL, qs, t, nbuf, out); break;
    default: conv_row<TIn, 3>(vk, M, logL, qs, t, nbuf, out); break;
  }
}

// Garner's mixed-radix digits d_q of the residues, then Y = d0 + p0 (d1 + p1 (d2 + p2 d3)) in
// FP64, negative when d3 > p3/2 (|Y| < 2^115 << p0 p1 p2 p3 / 2).
__device__ __forceinline__ double crt4(uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3, const uint32_t* inv) {
  const uint64_t d0 = r0;
  const uint64_t d1 = ((uint64_t)(r1 + kP1 - (uint32_t)(d0 % kP1)) * inv[0]) % kP1;  // inv[0] = p0^-1 mod p1
  uint64_t t2 = ((uint64_t)(r2 + kP2 - (uint32_t)(d0 % kP2)) * inv[1]) % kP2;        // inv[1] = p0^-1 mod p2
  const uint64_t d2 = ((t2 + kP2 - d1 % kP2) * inv[2]) % kP2;                         // inv[2] = p1^-1 mod p2
  uint64_t t3 = ((uint64_t)(r3 + kP3 - (uint32_t)(d0 % kP3)) * inv[3]) % kP3;        // inv[3] = p0^-1 mod p3
  t3 = ((t3 + kP3 - d1 % kP3) * inv[4]) % kP3;                                        // inv[4] = p1^-1 mod p3
  const uint64_t d3 = ((t3 + kP3 - d2 % kP3) * inv[5]) % kP3;                         // inv[5] = p2^-1 mod p3
  if (d3 <= kP3 / 2)
    return (((double)d3 * kP2 + (double)d2) * kP1 + (double)d1) * kP0 + (double)d0;
  // negative: Y = -(P - Y), P - 1 - Y has the complemented digits p_q - 1 - d_q
  const double e3 = (double)(kP3 - 1 - d3), e2 = (double)(kP2 - 1 - d2), e1 = (double)(kP1 - 1 - d1),
               e0 = (double)(kP0 - 1 - d0);
  return -((((e3 * kP2 + e2) * kP1 + e1) * kP0 + e0) + 1.0);
}

template <typename TIn>
__global__ void __launch_bounds__(256) ntt_epilogue_kernel(const TIn* __restrict__ v, const double* __restrict__ rhs,
                                                           double* __restrict__ w, double* __restrict__ sq_partial,
                                                           int M, int Nt, const uint32_t* __restrict__ res,
                                                           const double* __restrict__ rowscale, NttTables t) {
  __shared__ double redb[32];
  const int k = blockIdx.x;
  const double f = t.c_gscale * rowscale[k];  // c 2^(e_g - 51) 2^(e_v - 51)
  const TIn* vk = v + (size_t)k * M;
  const TIn* vk1 = vk - M;
  const TIn* vk2 = vk - 2 * M;
  double* wk = w + (size_t)k * M;
  const double* rk = rhs ? rhs + (size_t)k * M : nullptr;
  const size_t n = (size_t)Nt * M, base = (size_t)k * M;
  double sq = 0.0;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    const double Y = crt4(res[base + i], res[n + base + i], res[2 * n + base + i], res[3 * n + base + i], t.crt);
    const double y = f * Y;
    double band;
    if (k == 0) band = ldd(vk + i);
    else if (k == 1) band = 1.5 * ldd(vk + i) - 2.0 * ldd(vk1 + i);
    else band = 1.5 * ldd(vk + i) - 2.0 * ldd(vk1 + i) + 0.5 * ldd(vk2 + i);
    double out = band + y;
    if (rk) out = rk[i] - out;
    wk[i] = out;
    sq += out * out;
  }
  if (sq_partial) {
    double a[1] = {sq};
    block_sum<double, 1>(a, redb);
    if (threadIdx.x == 0) sq_partial[k] = a[0];
  }
}

template <typename TIn>
cudaError_t launch_ntt(const TIn* v, const double* rhs, double* w, double* sq_partial, int M, int Nt, int logL,
                       const NttTables& t, uint32_t* res, double* rowscale, cudaStream_t s) {
  const size_t smem = (size_t)(1u << logL) * sizeof(uint32_t);
  cudaError_t e = allow_max_dynamic_smem(ntt_conv_kernel<TIn>);
  if (e != cudaSuccess) return e;
  ntt_conv_kernel<TIn><<<dim3(Nt, 4), 512, smem, s>>>(v, M, Nt, logL, t, res, rowscale);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ntt_epilogue_kernel<TIn><<<Nt, 256, 0, s>>>(v, rhs, w, sq_partial, M, Nt, res, rowscale, t);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_matvec_ntt(const double* v, const double* rhs, double* w, double* sq_partial, int M, int Nt,
                              int logL, const NttTables& t, uint32_t* res, double* rowscale, cudaStream_t s) {
  return launch_ntt<double>(v, rhs, w, sq_partial, M, Nt, logL, t, res, rowscale, s);
}
cudaError_t launch_matvec_ntt_fin(const float* v, const double* rhs, double* w, double* sq_partial, int M, int Nt,
                                  int logL, const NttTables& t, uint32_t* res, double* rowscale, cudaStream_t s) {
  return launch_ntt<float>(v, rhs, w, sq_partial, M, Nt, logL, t, res, rowscale, s);
}

}  // namespace aao
