// All-at-once matvec, Sec. 3.2, with the Toeplitz product c T v_k computed
// EXACTLY for quantised inputs by number-theoretic transforms (NTT) instead of
// FP64 FFTs (the FP64 pipe of this GPU issues ~1.6 DFMA per clock per SM; its
// integer pipes are an order of magnitude faster).
//
// Row k of v is scaled by a power of two so that its largest magnitude lies in
// [2^57, 2^58) and rounded to integers V (quantisation error 2^-59 of the row's
// largest entry); the FCD stencil times c (c > 0) is quantised the same way
// once at plan creation (G, G_0 <= 2^58).  The linear convolution Y = G * V is bounded by
// max|V| sum_d |G_d|, and the FCD weights have g_0 > 0 >= g_d (d >= 1) with
// sum over all d of g_d = 0 (Lemma 2.1), so sum_d |G_d| <= 2 G_0 + M (the
// rounding) and |Y| < 2^117 (1 + 2^-45).  Four NTT primes p_q < 2^30 (product
// ~2^119.5) therefore determine Y exactly: it is computed by cyclic
// convolution of length L >= 2M - 1 (circulant embedding) modulo each prime,
// reconstructed by Garner's mixed-radix CRT and rounded to FP64 once:
// c T v_k = 2^(e_v + e_g - 116) Y, the power of two applied to the exponent.
//
// Kernel 0 (ntt_quant_kernel): one CTA per time row: the row's scale and its
// int64 quantisation (the only FP64 work before the epilogue).
// Kernel 1 (ntt_conv_kernel): one CTA per (time row, prime): residues of the
// quantised row mod p, forward NTT, multiply by the stencil spectrum (stored
// bit-reversed, L^-1 folded in), inverse NTT, write the residues of the first
// M outputs.
// The transforms run in passes of r <= 4 radix-2 stages: each thread takes a
// group of 2^r elements at stride S = L / 2^(s0 + r) into registers, applies
// the 2^r-point transform with constant roots, multiplies by the external
// twiddles w^(j bitrev_r(k) 2^s0) (DIF; conjugate order for the DIT inverse)
// and stores back (natural order in, bit-reversed out, and back).  The
// twiddles are stored pass by pass in the order the threads read them
// (coalesced).  The first forward pass reads its group straight from the
// quantised row (the upper half of the embedding is zero), the last forward
// pass, the spectrum product and the first inverse pass are one register pass
// (stride 1, no external twiddles), and the last inverse pass writes the
// residues straight to global memory, so shared memory sees 2 (log2 L / 4) - 1
// read-write sweeps per row.  Shared memory is padded by one word per 32.
// Kernel 2 (ntt_epilogue_kernel): a few CTAs per row: Garner CRT of the
// residues, scaling, the BDF band of C (Eq. 1.7), optional residual rhs - w,
// per-CTA sums of squares and (Arnoldi step) the first Gram-Schmidt pass.
//
// Modular arithmetic: Shoup multiplication by a constant w with precomputed
// w' = floor(w 2^32 / p), lazy values in [0, 2p) (p < 2^30 keeps all sums
// below 2^32).
#include "common.cuh"
#include "ff.cuh"
#include "kernels.h"

namespace aao {

namespace {

constexpr int NP = kNttPrimes;
constexpr int QBITS = 58;  // quantisation: |V| < 2^58

template <int Q> struct Prime { static constexpr uint32_t p = kNttPrime[Q]; };

// a * w mod p in [0, 2p) for a < 2^32, w = (w, floor(w 2^32 / p))
template <uint32_t P>
__device__ __forceinline__ uint32_t mulsh(uint32_t a, uint2 w) {
  const uint32_t q = __umulhi(a, w.y);
  return a * w.x - q * P;
}
template <uint32_t P> __device__ __forceinline__ uint32_t red2(uint32_t a) { return a >= 2 * P ? a - 2 * P : a; }
template <uint32_t P> __device__ __forceinline__ uint32_t red1(uint32_t a) { return a >= P ? a - P : a; }
__device__ __forceinline__ int pad32(int i) { return i + (i >> 5); }

// Gentleman-Sande butterfly (x, y) -> (x + y, (x - y) w); w == 1 when ONE; all values in [0, 2p)
template <uint32_t P, bool ONE>
__device__ __forceinline__ void dif2(uint32_t& x, uint32_t& y, uint2 w) {
  const uint32_t s = x + y, d = x - y + 2 * P;
  x = red2<P>(s);
  y = ONE ? red2<P>(d) : mulsh<P>(d, w);
}
// Cooley-Tukey butterfly (x, y) -> (x + y w, x - y w)
template <uint32_t P, bool ONE>
__device__ __forceinline__ void dit2(uint32_t& x, uint32_t& y, uint2 w) {
  const uint32_t t = ONE ? y : mulsh<P>(y, w);
  const uint32_t s = x + t, d = x - t + 2 * P;
  x = red2<P>(s);
  y = red2<P>(d);
}

// The 2^r-point transforms with constant roots wint[e] = w^(e L / R): DIF (natural order in,
// bit-reversed out) and its inverse DIT.
template <uint32_t P, int r>
__device__ __forceinline__ void dif_core(uint32_t (&v)[1 << r], const uint2 (&wint)[8]) {
  constexpr int R = 1 << r;
#pragma unroll
  for (int t = 0; t < r; ++t) {
    const int half = R >> (t + 1);
#pragma unroll
    for (int k = 0; k < R; ++k) {
      if (k & half) continue;
      const int e = (k % half) << t;  // power of w^(L/R)
      if (e == 0) dif2<P, true>(v[k], v[k + half], wint[0]);
      else dif2<P, false>(v[k], v[k + half], wint[e]);
    }
  }
}
template <uint32_t P, int r>
__device__ __forceinline__ void dit_core(uint32_t (&v)[1 << r], const uint2 (&wint)[8]) {
  constexpr int R = 1 << r;
#pragma unroll
  for (int t = r - 1; t >= 0; --t) {
    const int half = R >> (t + 1);
#pragma unroll
    for (int k = 0; k < R; ++k) {
      if (k & half) continue;
      const int e = (k % half) << t;
      if (e == 0) dit2<P, true>(v[k], v[k + half], wint[0]);
      else dit2<P, false>(v[k], v[k + half], wint[e]);
    }
  }
}

// A middle forward pass of 4 stages starting at stage s0 (see the file comment); tw is this
// pass's table: w^(j bitrev_4(k) 2^s0) at (k - 1) S + j.
template <uint32_t P>
__device__ __forceinline__ void dif_pass(uint32_t* buf, int logL, int s0, const uint2* __restrict__ tw,
                                         const uint2 (&wint)[8]) {
  constexpr int r = 4, R = 16;
  const int L = 1 << logL, logS = logL - s0 - r, S = 1 << logS;
  for (int g = threadIdx.x; g < (L >> r); g += blockDim.x) {
    const int b = g >> logS, j = g & (S - 1);
    const int base = (b << (logL - s0)) + j;
    uint32_t v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = buf[pad32(base + k * S)];
    dif_core<P, r>(v, wint);
#pragma unroll
    for (int k = 0; k < R; ++k) {
      if (k) v[k] = mulsh<P>(v[k], __ldg(&tw[(k - 1) * S + j]));
      buf[pad32(base + k * S)] = v[k];
    }
  }
}

// The inverse of dif_pass with the inverse table (w^-1 in place of w).
template <uint32_t P>
__device__ __forceinline__ void dit_pass(uint32_t* buf, int logL, int s0, const uint2* __restrict__ twi,
                                         const uint2 (&wint)[8]) {
  constexpr int r = 4, R = 16;
  const int L = 1 << logL, logS = logL - s0 - r, S = 1 << logS;
  for (int g = threadIdx.x; g < (L >> r); g += blockDim.x) {
    const int b = g >> logS, j = g & (S - 1);
    const int base = (b << (logL - s0)) + j;
    uint32_t v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      v[k] = buf[pad32(base + k * S)];
      if (k) v[k] = mulsh<P>(v[k], __ldg(&twi[(k - 1) * S + j]));
    }
    dit_core<P, r>(v, wint);
#pragma unroll
    for (int k = 0; k < R; ++k) buf[pad32(base + k * S)] = v[k];
  }
}

// x mod p in [0, p) for a signed 64-bit x
template <uint32_t P> __device__ __forceinline__ uint32_t residue(long long x) {
  long long m = x % (long long)P;
  if (m < 0) m += P;
  return (uint32_t)m;
}

// The first forward pass (stages 0..3, stride S = L / 16) reading the quantised row from global
// memory: element i = j + k S is V[i] mod p for i < M, else 0 (the circulant embedding's padding;
// the plan takes L >= 2M, so the upper half of every group is zero).
template <uint32_t P>
__device__ __forceinline__ void dif_first(const long long* __restrict__ Vk, int M, uint32_t* buf, int logL,
                                          const uint2* __restrict__ tw, const uint2 (&wint)[8]) {
  constexpr int r = 4, R = 16;
  const int S = 1 << (logL - r);
  for (int j = threadIdx.x; j < S; j += blockDim.x) {
    uint32_t v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {  // L >= 2M: elements k >= R / 2 lie in the zero half
      const int i = j + k * S;
      v[k] = (k < R / 2 && i < M) ? residue<P>(__ldg(Vk + i)) : 0u;
    }
    dif_core<P, r>(v, wint);
#pragma unroll
    for (int k = 0; k < R; ++k) {
      if (k) v[k] = mulsh<P>(v[k], __ldg(&tw[(k - 1) * S + j]));
      buf[pad32(j + k * S)] = v[k];
    }
  }
}

// The last inverse pass (stages 3..0, stride S = L / 16) writing the residues of the first M
// outputs to global memory.
template <uint32_t P>
__device__ __forceinline__ void dit_last(const uint32_t* buf, int logL, int M, const uint2* __restrict__ twi,
                                         const uint2 (&wint)[8], uint32_t* __restrict__ out) {
  constexpr int r = 4, R = 16;
  const int S = 1 << (logL - r);
  for (int j = threadIdx.x; j < S; j += blockDim.x) {
    uint32_t v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      v[k] = buf[pad32(j + k * S)];
      if (k) v[k] = mulsh<P>(v[k], __ldg(&twi[(k - 1) * S + j]));
    }
    dit_core<P, r>(v, wint);
#pragma unroll
    for (int k = 0; k < R / 2; ++k) {  // L >= 2M: outputs k >= R / 2 are not needed
      const int i = j + k * S;
      if (i < M) out[i] = red1<P>(v[k]);
    }
  }
}

// The last forward pass (stride 1, so its external twiddles are all 1), the product with the
// bit-reversed stencil spectrum gh and the first inverse pass, on the same 2^r contiguous elements.
template <uint32_t P, int r>
__device__ __forceinline__ void mid_fused(uint32_t* buf, int logL, const uint2* __restrict__ gh,
                                          const uint2 (&wf)[8], const uint2 (&wi)[8]) {
  constexpr int R = 1 << r;
  const int per = 1 << (logL - r);
  for (int g = threadIdx.x; g < per; g += blockDim.x) {
    const int base = g << r;
    uint32_t v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = buf[pad32(base + k)];
    dif_core<P, r>(v, wf);
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = mulsh<P>(v[k], __ldg(&gh[base + k]));
    dit_core<P, r>(v, wi);
#pragma unroll
    for (int k = 0; k < R; ++k) buf[pad32(base + k)] = v[k];
  }
}

// wint[e] = w^(e L / 2^r) for e < 2^r / 2 from the table's constant roots w^(e L / Rmax)
template <int r>
__device__ __forceinline__ void load_roots(uint2 (&wint)[8], const uint2* __restrict__ tab, int logL) {
  const int rmax = logL < 4 ? logL : 4;
#pragma unroll
  for (int e = 0; e < 8; ++e) wint[e] = (e < (1 << r) / 2) ? __ldg(&tab[e << (rmax - r)]) : uint2{1, 0};
}

template <uint32_t P, int r>
__device__ __forceinline__ void mid_fused_roots(uint32_t* buf, int logL, const uint2* __restrict__ gh,
                                                const uint2* __restrict__ twf, const uint2* __restrict__ twi) {
  uint2 wf[8], wi[8];
  load_roots<r>(wf, twf, logL);
  load_roots<r>(wi, twi, logL);
  mid_fused<P, r>(buf, logL, gh, wf, wi);
}
template <uint32_t P>
__device__ __forceinline__ void mid_fused_any(int r, uint32_t* buf, int logL, const uint2* __restrict__ gh,
                                              const uint2* __restrict__ twf, const uint2* __restrict__ twi) {
  switch (r) {
    case 1: mid_fused_roots<P, 1>(buf, logL, gh, twf, twi); break;
    case 2: mid_fused_roots<P, 2>(buf, logL, gh, twf, twi); break;
    case 3: mid_fused_roots<P, 3>(buf, logL, gh, twf, twi); break;
    default: mid_fused_roots<P, 4>(buf, logL, gh, twf, twi); break;
  }
}

__device__ __forceinline__ double ldd(const double* p) { return __ldg(p); }

// Quantisation pre-pass, one CTA per row: V[k][i] = round(v[k][i] 2^(58 - e_v)) with the row's
// largest magnitude below 2^e_v (int64, |V| < 2^58); rowscale[k] = 2^(e_v - 58) (0 for a zero row,
// NaN for a row with a non-finite entry, whose V is left 0).
template <typename TIn>
__global__ void __launch_bounds__(512) ntt_quant_kernel(const TIn* __restrict__ v, int M, long long* __restrict__ V,
                                                        double* __restrict__ rowscale) {
  __shared__ double red[32];
  __shared__ int bad_any;
  const int k = blockIdx.x;
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
  if (mx > 0) frexp(mx, &ev);  // mx < 2^ev
  const double qs = mx > 0 && !bad_any ? ldexp(1.0, QBITS - ev) : 0.0;
  if (threadIdx.x == 0) rowscale[k] = bad_any ? __longlong_as_double(0x7ff8000000000000ll)
                                              : (mx > 0 ? ldexp(1.0, ev - QBITS) : 0.0);
  long long* Vk = V + (size_t)k * M;
  for (int i = threadIdx.x; i < M; i += blockDim.x) Vk[i] = __double2ll_rn(ldd(vk + i) * qs);  // exact scaling
}

// The quantisation pre-pass for FP32 rows (to QB bits), in integer arithmetic on the bit patterns: the row's
// largest magnitude as bits (monotone for finite values) gives e_v, and each entry m 2^E (24-bit significand m)
// becomes m 2^(E + QB - e_v), shifted left exactly or right with rounding half to even -- the same integers as
// round(v 2^(QB - e_v)), without FP64<->FP32 conversions.
template <int QB>
__global__ void __launch_bounds__(512) ntt_quant_f32_kernel(const float* __restrict__ v, int M,
                                                            long long* __restrict__ V, double* __restrict__ rowscale) {
  __shared__ unsigned int redu[32];
  const int k = blockIdx.x;
  const unsigned int* vk = reinterpret_cast<const unsigned int*>(v + (size_t)k * M);
  unsigned int amax = 0;  // >= 0x7f800000: a non-finite entry
  for (int i = threadIdx.x; i < M; i += blockDim.x) amax = max(amax, __ldg(vk + i) & 0x7fffffffu);
  amax = __reduce_max_sync(0xffffffffu, amax);
  if ((threadIdx.x & 31) == 0) redu[threadIdx.x >> 5] = amax;
  __syncthreads();
  amax = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) amax = max(amax, redu[w]);
  const bool bad = amax >= 0x7f800000u;
  int ev = 0;  // largest magnitude < 2^ev
  if (amax) ev = (amax >> 23) ? (int)(amax >> 23) - 126 : (32 - __clz((int)amax)) - 149;
  if (threadIdx.x == 0) rowscale[k] = bad ? __longlong_as_double(0x7ff8000000000000ll) : (amax ? ldexp(1.0, ev - QB) : 0.0);
  long long* Vk = V + (size_t)k * M;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    const unsigned int u = __ldg(vk + i), a = u & 0x7fffffffu;
    long long q = 0;
    if (!bad && a) {
      const unsigned int ex = a >> 23;
      const unsigned int m = ex ? ((a & 0x7fffffu) | 0x800000u) : a;
      const int sh = (ex ? (int)ex - 150 : -149) + QB - ev;  // <= QB - 24
      if (sh >= 0) {
        q = (long long)m << sh;
      } else if (sh > -26) {  // m < 2^24: a shift by 26 or more rounds to 0
        const int r = -sh;
        unsigned int qq = m >> r;
        const unsigned int rem = m & ((1u << r) - 1u), half = 1u << (r - 1);
        if (rem > half || (rem == half && (qq & 1u))) ++qq;
        q = qq;
      }
      if (u >> 31) q = -q;
    }
    Vk[i] = q;
  }
}

template <int Q>
__device__ __forceinline__ void conv_row(const long long* __restrict__ Vk, int M, int logL, const NttTables& t,
                                         const uint2* __restrict__ ghat, uint32_t* buf, uint32_t* __restrict__ out) {
  constexpr uint32_t P = Prime<Q>::p;
  const int L = 1 << logL;
  const size_t tsz = (size_t)ntt_tw_size(logL);
  const uint2* twf = t.twf + Q * tsz;
  const uint2* twi = t.twi + Q * tsz;
  const uint2* gh = ghat + (size_t)Q * L;
  const int sl = ntt_last_pass(logL);
  if (sl == 0) {  // L <= 16: one pass
    for (int i = threadIdx.x; i < L; i += blockDim.x) buf[pad32(i)] = i < M ? residue<P>(__ldg(Vk + i)) : 0u;
    __syncthreads();
    mid_fused_any<P>(logL, buf, logL, gh, twf, twi);
    __syncthreads();
    for (int i = threadIdx.x; i < M; i += blockDim.x) out[i] = red1<P>(buf[pad32(i)]);
    return;
  }
  {
    uint2 w[8];
    load_roots<4>(w, twf, logL);
    dif_first<P>(Vk, M, buf, logL, twf + 8, w);
  }
  for (int s0 = 4; s0 < sl; s0 += 4) {
    __syncthreads();
    uint2 w[8];
    load_roots<4>(w, twf, logL);
    dif_pass<P>(buf, logL, s0, twf + ntt_tw_offset(logL, s0), w);
  }
  __syncthreads();
  mid_fused_any<P>(logL - sl, buf, logL, gh, twf, twi);
  for (int s0 = sl - 4; s0 >= 4; s0 -= 4) {
    __syncthreads();
    uint2 w[8];
    load_roots<4>(w, twi, logL);
    dit_pass<P>(buf, logL, s0, twi + ntt_tw_offset(logL, s0), w);
  }
  __syncthreads();
  uint2 w[8];
  load_roots<4>(w, twi, logL);
  dit_last<P>(buf, logL, M, twi + 8, w, out);
}

// grid (Nt, NP): blockIdx.y selects the prime.  V: the quantised rows; res: [NP][Nt][M] residues.
__global__ void __launch_bounds__(512, 2) ntt_conv_kernel(const long long* __restrict__ V, int M, int Nt, int logL,
                                                       NttTables t, uint32_t* __restrict__ res) {
  extern __shared__ uint32_t nbuf[];
  const int k = blockIdx.x, q = blockIdx.y;
  const long long* Vk = V + (size_t)k * M;
  uint32_t* out = res + ((size_t)q * Nt + k) * M;
  switch (q) {
    case 0: conv_row<0>(Vk, M, logL, t, t.ghat, nbuf, out); break;
    case 1: conv_row<1>(Vk, M, logL, t, t.ghat, nbuf, out); break;
    case 2: conv_row<2>(Vk, M, logL, t, t.ghat, nbuf, out); break;
    default: conv_row<3>(Vk, M, logL, t, t.ghat, nbuf, out); break;
  }
}

// One Garner step in 32-bit arithmetic: (r - x) c mod p_B for a residue r < p_B, a digit x < p_A (one
// subtraction brings it below p_B: the four primes lie within a factor 1.07 of each other) and the constant
// c = (c, floor(c 2^32 / p_B)) by Shoup multiplication.
template <int B> __device__ __forceinline__ uint32_t gstep(uint32_t r, uint32_t x, uint2 c) {
  constexpr uint32_t P = Prime<B>::p;
  const uint32_t xr = x >= P ? x - P : x;
  const uint32_t a = r >= xr ? r - xr : r + P - xr;
  return red1<P>(mulsh<P>(a, c));
}

// Garner's mixed-radix digits d_q of the four residues r_q, then Y = d0 + p0 (d1 + p1 (d2 + p2 d3)) in
// integer arithmetic; negative when d3 > p3 / 2 (|Y| < 2^117.01, below half the product).  Returns the 64
// leading bits of |Y| with a sticky bit in bit 0 (top) and the weight of its lowest bit (|Y| ~ top 2^sh).
struct CrtTop {
  uint64_t top;
  int sh;
  bool neg;
};
__device__ __forceinline__ CrtTop crt4_top(const uint32_t (&rq)[NP], const uint2* c) {
  constexpr uint64_t p0 = Prime<0>::p, p1 = Prime<1>::p, p2 = Prime<2>::p, p3 = Prime<3>::p;
  // c: p0^-1 mod p1, p2, p3 (c[0..2]), p1^-1 mod p2, p3 (c[3..4]), p2^-1 mod p3 (c[5])
  uint32_t d[NP];
  d[0] = rq[0];
  d[1] = gstep<1>(rq[1], d[0], c[0]);
  d[2] = gstep<2>(gstep<2>(rq[2], d[0], c[1]), d[1], c[3]);
  d[3] = gstep<3>(gstep<3>(gstep<3>(rq[3], d[0], c[2]), d[1], c[4]), d[2], c[5]);
  // Y as a 3-limb integer from the mixed-radix digits; when negative, |Y| = (P - 1 - Y) + 1 with the
  // complemented digits p_q - 1 - d_q
  const uint64_t pm[NP] = {p0, p1, p2, p3};
  const bool neg = d[NP - 1] > pm[NP - 1] / 2;
  uint64_t e[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) e[q] = neg ? pm[q] - 1 - d[q] : d[q];
  uint64_t l0 = e[NP - 1], l1 = 0, l2 = 0;
#pragma unroll
  for (int q = NP - 2; q >= 0; --q) {  // (l2, l1, l0) = (l2, l1, l0) * p_q + e_q
    const uint64_t m = pm[q];
    const uint64_t lo0 = l0 * m, hi0 = __umul64hi(l0, m);
    const uint64_t lo1 = l1 * m, hi1 = __umul64hi(l1, m);
    const uint64_t n0 = lo0 + e[q];
    const uint64_t c0 = n0 < lo0;
    const uint64_t s1 = lo1 + hi0;
    uint64_t c1 = s1 < lo1;
    const uint64_t n1 = s1 + c0;
    c1 += n1 < s1;
    l2 = l2 * m + hi1 + c1;
    l1 = n1;
    l0 = n0;
  }
  if (neg) {  // + 1
    l0 += 1;
    const uint64_t cc = l0 == 0;
    l1 += cc;
    l2 += (cc && l1 == 0);
  }
  CrtTop r;
  r.neg = neg;
  if (l2) {
    const int z = __clzll(l2);
    r.top = z ? (l2 << z) | (l1 >> (64 - z)) : l2;
    const uint64_t rest = z ? (l1 << z) | l0 : (l1 | l0);
    r.top |= (rest != 0);
    r.sh = 128 - z;
  } else if (l1) {
    const int z = __clzll(l1);
    r.top = z ? (l1 << z) | (l0 >> (64 - z)) : l1;
    r.top |= (z ? (l0 << z) : l0) != 0;
    r.sh = 64 - z;
  } else {
    r.top = l0;
    r.sh = 0;
  }
  return r;
}

// (+-) top 2^(sh + E) correctly rounded to FP64.  A normal result is assembled from the bits by integer
// operations (round half to even on the 53 leading bits; a carry out of the significand moves into the
// exponent field by the addition); zero stays zero; results outside the normal range take the conversion and
// ldexp on the FP64 pipe.
__device__ __forceinline__ double crt_to_double(CrtTop t, int E) {
  if (t.top == 0) return 0.0;
  const int z = __clzll(t.top);
  const uint64_t top = t.top << z;
  const int be = t.sh - z + E + 63 + 1023;  // biased exponent of the leading bit
  if (be < 1 || be > 2045) {
    const double m = ldexp(__ull2double_rn(top), t.sh - z + E);
    return t.neg ? -m : m;
  }
  uint64_t m = top >> 11;
  m += ((top >> 10) & 1ull) & ((uint64_t)((top & 0x3ffull) != 0) | (m & 1ull));
  const uint64_t bits = ((uint64_t)(be - 1) << 52) + m;
  return __longlong_as_double((long long)(bits | ((uint64_t)t.neg << 63)));
}

// The row scale 2^(e_v - 58) as its exponent when it is a normal power of two (fast: the epilogue adds it to
// the exponent); a zero row (scale 0) or a row with a non-finite entry (scale NaN) gives fast = false and the
// epilogue multiplies by the scale instead, which keeps 0 and NaN.
__device__ __forceinline__ int pow2_exponent(double s, bool& fast) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(s);
  const int ex = (int)((b >> 52) & 0x7ffu);
  fast = (b >> 63) == 0 && (b & 0xfffffffffffffull) == 0 && ex != 0 && ex != 0x7ff;
  return ex - 1023;
}

// The BDF2 band of time row k at element i (Eq. 2.5: row 0 the BDF1 start): v_k, 1.5 v_k - 2 v_{k-1}, or
// 1.5 v_k - 2 v_{k-1} + 0.5 v_{k-2}; vk points at v_k[i], rows are `stride` apart.  FP32 rows are widened with
// the factors 2 and 1/2 folded into the exponent (two FP64 operations for a full band instead of three).
__device__ __forceinline__ double bdf_band(const double* vk, size_t stride, int k) {
  const double a = __ldg(vk);
  if (k == 0) return a;
  const double b = __ldg(vk - stride);
  if (k == 1) return fma(1.5, a, -2.0 * b);
  return fma(1.5, a, fma(-2.0, b, 0.5 * __ldg(vk - 2 * stride)));
}
__device__ __forceinline__ double bdf_band(const float* vk, size_t stride, int k) {
  const double a = f2d_bits(__ldg(vk));
  if (k == 0) return a;
  const double b2 = -f2d_exact(__ldg(vk - stride), 1);
  if (k == 1) return fma(1.5, a, b2);
  return fma(1.5, a, b2 + f2d_exact(__ldg(vk - 2 * stride), -1));
}

// Chunks per row of the epilogue: about 8 elements per thread of a 256-thread CTA, so that a matvec's
// epilogue launches several waves of CTAs instead of one CTA per row.
inline int epi_chunks(int M) { return (M + 256 * 8 - 1) / (256 * 8); }
inline int ntt2d_chunks(int Mx, int My) { return ((Mx * My) + 256 * 8 - 1) / (256 * 8); }

// Pass-1 Gram-Schmidt dots fused into the epilogue (the Arnoldi step of the mixed path): with NVMAX > 0 each
// CTA also writes the partial sums of hi(w) hi(V_i) for i < nv (V: float-float basis vectors of vstride
// elements) to dots_partial[(k chunks + c) nv + i], the FP32 first pass of CGS2.
struct FusedDots {
  const float2* V;
  size_t vstride;
  int nv;
  double* partial;
};

// grid (Nt, chunks): CTA (k, c) finishes elements [c chunk, (c + 1) chunk) of row k.
template <typename TIn, int NVMAX>
__global__ void __launch_bounds__(256) ntt_epilogue_kernel(const TIn* __restrict__ v, const double* __restrict__ rhs,
                                                           double* __restrict__ w, double* __restrict__ sq_partial,
                                                           int M, int Nt, const uint32_t* __restrict__ res,
                                                           const double* __restrict__ rowscale, NttTables t,
                                                           FusedDots fd) {
  __shared__ double redb[32];
  const int k = blockIdx.x;
  const int chunk = (M + gridDim.y - 1) / gridDim.y;
  const int i0 = blockIdx.y * chunk, i1 = min(M, i0 + chunk);
  const double rs = rowscale[k];  // 2^(e_v - 58)
  bool fast;
  const int E = t.gexp + pow2_exponent(rs, fast);
  const double f = t.c_gscale * rs;  // 2^(e_g - 58) 2^(e_v - 58), for rows whose scale is 0 or NaN
  const TIn* vk = v + (size_t)k * M;
  double* wk = w + (size_t)k * M;
  const double* rk = rhs ? rhs + (size_t)k * M : nullptr;
  const size_t n = (size_t)Nt * M, base = (size_t)k * M;
  double sq = 0.0;
  float acc[NVMAX > 0 ? NVMAX : 1];
#pragma unroll
  for (int q = 0; q < (NVMAX > 0 ? NVMAX : 1); ++q) acc[q] = 0.0f;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    uint32_t rq[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) rq[q] = res[q * n + base + i];
    float vh[NVMAX > 0 ? NVMAX : 1];
#pragma unroll
    for (int q = 0; q < NVMAX; ++q)
      if (q < fd.nv) vh[q] = __ldg(&fd.V[q * fd.vstride + base + i]).x;
    const double y = fast ? crt_to_double(crt4_top(rq, t.crt), E) : f * crt_to_double(crt4_top(rq, t.crt), 0);
    double out = bdf_band(vk + i, (size_t)M, k) + y;
    if (rk) out = rk[i] - out;
    wk[i] = out;
    if constexpr (NVMAX == 0) sq += out * out;  // the fused-dots launch has no sq_partial
    if (NVMAX > 0) {
      const float wh = ff_split(out).x;
#pragma unroll
      for (int q = 0; q < NVMAX; ++q)
        if (q < fd.nv) acc[q] = fmaf(wh, vh[q], acc[q]);
    }
  }
  if (sq_partial) {
    double a[1] = {sq};
    block_sum<double, 1>(a, redb);
    if (threadIdx.x == 0) sq_partial[(size_t)k * gridDim.y + blockIdx.y] = a[0];
  }
  if constexpr (NVMAX > 0) {
    double accd[NVMAX];
#pragma unroll
    for (int q = 0; q < NVMAX; ++q) accd[q] = (double)acc[q];
    block_partials_to<NVMAX, 256>(accd, fd.nv, fd.partial + ((size_t)k * gridDim.y + blockIdx.y) * fd.nv);
  }
}

template <typename TIn>
cudaError_t launch_ntt(const TIn* v, const double* rhs, double* w, double* sq_partial, int M, int Nt, int logL,
                       const NttTables& t, uint32_t* res, double* rowscale, cudaStream_t s,
                       FusedDots fd = FusedDots{nullptr, 0, 0, nullptr}) {
  if (fd.partial && sq_partial) return cudaErrorInvalidValue;  // the fused-dots epilogue forms no sums of squares
  const int L = 1 << logL;
  const size_t smem = (size_t)(L + L / 32 + 1) * sizeof(uint32_t);
  cudaError_t e = allow_max_dynamic_smem(ntt_conv_kernel);
  if (e != cudaSuccess) return e;
  long long* V = reinterpret_cast<long long*>(res + (size_t)NP * Nt * M);  // after the residues
  if constexpr (sizeof(TIn) == 4) ntt_quant_f32_kernel<QBITS><<<Nt, 512, 0, s>>>(v, M, V, rowscale);
  else ntt_quant_kernel<TIn><<<Nt, 512, 0, s>>>(v, M, V, rowscale);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ntt_conv_kernel<<<dim3(Nt, NP), 512, smem, s>>>(V, M, Nt, logL, t, res);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const dim3 ge(Nt, epi_chunks(M));
  if (!fd.partial) {
    ntt_epilogue_kernel<TIn, 0><<<ge, 256, 0, s>>>(v, rhs, w, sq_partial, M, Nt, res, rowscale, t, fd);
  } else {
    const int nv = fd.nv;
    if (nv <= 4) ntt_epilogue_kernel<TIn, 4><<<ge, 256, 0, s>>>(v, rhs, w, sq_partial, M, Nt, res, rowscale, t, fd);
    else if (nv <= 8) ntt_epilogue_kernel<TIn, 8><<<ge, 256, 0, s>>>(v, rhs, w, sq_partial, M, Nt, res, rowscale, t, fd);
    else if (nv <= 16) ntt_epilogue_kernel<TIn, 16><<<ge, 256, 0, s>>>(v, rhs, w, sq_partial, M, Nt, res, rowscale, t, fd);
    else if (nv <= 24) ntt_epilogue_kernel<TIn, 24><<<ge, 256, 0, s>>>(v, rhs, w, sq_partial, M, Nt, res, rowscale, t, fd);
    else if (nv <= 32) ntt_epilogue_kernel<TIn, 32><<<ge, 256, 0, s>>>(v, rhs, w, sq_partial, M, Nt, res, rowscale, t, fd);
    else ntt_epilogue_kernel<TIn, 65><<<ge, 256, 0, s>>>(v, rhs, w, sq_partial, M, Nt, res, rowscale, t, fd);
  }
  return cudaGetLastError();
}

// ---- 2D (Eq. 4.2): c_x T_x along the rows and c_y T_y along the columns of every time level, each an
// exact-integer line convolution of the level quantised to 58 bits with one scale per level -------------
// A CTA transforms lb lines of one prime in shared memory (each padded by one word per 32; lb from
// ntt2d_lines_per_cta, at most 16 and at most 96 KB): the same passes as conv_row (forward 16-point passes,
// the fused middle pass with the stencil spectrum, inverse passes), looped over the lines.
inline int ntt2d_lines_per_cta(int logL) {
  const int L = 1 << logL, bytes = (L + L / 32 + 1) * 4;
  const int b = (96 * 1024) / bytes;
  return b < 1 ? 1 : (b > 16 ? 16 : b);
}

template <uint32_t P>
__device__ __forceinline__ void bdif_pass(uint32_t* buf, int LS, int nb, int logL, int s0, const uint2* __restrict__ tw,
                                          const uint2 (&wint)[8]) {
  constexpr int r = 4, R = 16;
  const int logS = logL - s0 - r, S = 1 << logS, lper = logL - r;
  for (int gg = threadIdx.x; gg < (nb << lper); gg += blockDim.x) {
    const int line = gg >> lper, g = gg & ((1 << lper) - 1);
    const int b = g >> logS, j = g & (S - 1);
    const int base = (b << (logL - s0)) + j;
    uint32_t* bl = buf + line * LS;
    uint32_t v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = bl[pad32(base + k * S)];
    dif_core<P, r>(v, wint);
#pragma unroll
    for (int k = 0; k < R; ++k) {
      if (k) v[k] = mulsh<P>(v[k], __ldg(&tw[(k - 1) * S + j]));
      bl[pad32(base + k * S)] = v[k];
    }
  }
}

template <uint32_t P>
__device__ __forceinline__ void bdit_pass(uint32_t* buf, int LS, int nb, int logL, int s0, const uint2* __restrict__ twi,
                                          const uint2 (&wint)[8]) {
  constexpr int r = 4, R = 16;
  const int logS = logL - s0 - r, S = 1 << logS, lper = logL - r;
  for (int gg = threadIdx.x; gg < (nb << lper); gg += blockDim.x) {
    const int line = gg >> lper, g = gg & ((1 << lper) - 1);
    const int b = g >> logS, j = g & (S - 1);
    const int base = (b << (logL - s0)) + j;
    uint32_t* bl = buf + line * LS;
    uint32_t v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      v[k] = bl[pad32(base + k * S)];
      if (k) v[k] = mulsh<P>(v[k], __ldg(&twi[(k - 1) * S + j]));
    }
    dit_core<P, r>(v, wint);
#pragma unroll
    for (int k = 0; k < R; ++k) bl[pad32(base + k * S)] = v[k];
  }
}

template <uint32_t P, int r>
__device__ __forceinline__ void bmid(uint32_t* buf, int LS, int nb, int logL, const uint2* __restrict__ gh,
                                     const uint2* __restrict__ twf, const uint2* __restrict__ twi) {
  constexpr int R = 1 << r;
  uint2 wf[8], wi[8];
  load_roots<r>(wf, twf, logL);
  load_roots<r>(wi, twi, logL);
  const int lper = logL - r;
  for (int gg = threadIdx.x; gg < (nb << lper); gg += blockDim.x) {
    const int line = gg >> lper, g = gg & ((1 << lper) - 1);
    const int base = g << r;
    uint32_t* bl = buf + line * LS;
    uint32_t v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = bl[pad32(base + k)];
    dif_core<P, r>(v, wf);
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = mulsh<P>(v[k], __ldg(&gh[base + k]));
    dit_core<P, r>(v, wi);
#pragma unroll
    for (int k = 0; k < R; ++k) bl[pad32(base + k)] = v[k];
  }
}

// COL = false: line l = k My + j is row j of level k (M = Mx points, stride 1); COL = true: line l = k Mx + i
// is column i of level k (M = My points, stride Mx).  Lines are read and written so that consecutive threads
// touch consecutive addresses (along the row, or across neighbouring columns).
template <uint32_t P, bool COL>
__device__ __forceinline__ void conv_lines(const long long* __restrict__ V, int Mx, int My, int nlines, int logL,
                                           int lb, const NttTables& t, int q, uint32_t* buf,
                                           uint32_t* __restrict__ out) {
  const int L = 1 << logL, LS = L + L / 32 + 1;
  const int M = COL ? My : Mx, per = COL ? Mx : My;  // points per line, lines per level
  const size_t Ms = (size_t)Mx * My;
  const int l0 = blockIdx.x * lb;
  const int nb = min(lb, nlines - l0);
  auto addr = [&](int line, int i) -> size_t {  // element i of line l0 + line
    const int l = l0 + line, k = l / per, c = l - k * per;
    return (size_t)k * Ms + (COL ? (size_t)i * Mx + c : (size_t)c * Mx + i);
  };
  for (int idx = threadIdx.x; idx < lb * L; idx += blockDim.x) {
    const int line = COL ? idx % lb : idx / L, i = COL ? idx / lb : idx % L;
    if (line >= nb) continue;
    buf[line * LS + pad32(i)] = i < M ? residue<P>(__ldg(V + addr(line, i))) : 0u;
  }
  __syncthreads();
  const size_t tsz = (size_t)ntt_tw_size(logL);
  const uint2* twf = t.twf + (size_t)q * tsz;
  const uint2* twi = t.twi + (size_t)q * tsz;
  const uint2* gh = t.ghat + (size_t)q * L;
  const int sl = ntt_last_pass(logL);
  for (int s0 = 0; s0 < sl; s0 += 4) {
    uint2 w[8];
    load_roots<4>(w, twf, logL);
    bdif_pass<P>(buf, LS, nb, logL, s0, twf + ntt_tw_offset(logL, s0), w);
    __syncthreads();
  }
  switch (logL - sl) {
    case 1: bmid<P, 1>(buf, LS, nb, logL, gh, twf, twi); break;
    case 2: bmid<P, 2>(buf, LS, nb, logL, gh, twf, twi); break;
    case 3: bmid<P, 3>(buf, LS, nb, logL, gh, twf, twi); break;
    default: bmid<P, 4>(buf, LS, nb, logL, gh, twf, twi); break;
  }
  __syncthreads();
  for (int s0 = sl - 4; s0 >= 0; s0 -= 4) {
    uint2 w[8];
    load_roots<4>(w, twi, logL);
    bdit_pass<P>(buf, LS, nb, logL, s0, twi + ntt_tw_offset(logL, s0), w);
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < lb * M; idx += blockDim.x) {
    const int line = COL ? idx % lb : idx / M, i = COL ? idx / lb : idx % M;
    if (line >= nb) continue;
    out[addr(line, i)] = red1<P>(buf[line * LS + pad32(i)]);
  }
}

// grid (ceil(nlines / lb), NP); res: [NP][Nt Mx My] residues of this direction
template <bool COL>
__global__ void __launch_bounds__(256) ntt2d_lines_kernel(const long long* __restrict__ V, int Mx, int My, int Nt,
                                                          int logL, int lb, NttTables t, uint32_t* __restrict__ res) {
  extern __shared__ uint32_t nbuf[];
  const int q = blockIdx.y;
  const int nlines = Nt * (COL ? Mx : My);
  uint32_t* out = res + (size_t)q * Nt * Mx * My;
  switch (q) {
    case 0: conv_lines<Prime<0>::p, COL>(V, Mx, My, nlines, logL, lb, t, q, nbuf, out); break;
    case 1: conv_lines<Prime<1>::p, COL>(V, Mx, My, nlines, logL, lb, t, q, nbuf, out); break;
    case 2: conv_lines<Prime<2>::p, COL>(V, Mx, My, nlines, logL, lb, t, q, nbuf, out); break;
    default: conv_lines<Prime<3>::p, COL>(V, Mx, My, nlines, logL, lb, t, q, nbuf, out); break;
  }
}

// w = band + c_x T_x v + c_y T_y v (or rhs - that), both products reconstructed from their residues; grid
// (chunks, Nt), per-CTA sums of squares at sq_partial[k chunks + chunk]
template <typename TIn>
__global__ void __launch_bounds__(256) ntt2d_epilogue_kernel(const TIn* __restrict__ v, const double* __restrict__ rhs,
                                                             double* __restrict__ w, double* __restrict__ sq_partial,
                                                             int Ms, int Nt, const uint32_t* __restrict__ rx,
                                                             const uint32_t* __restrict__ ry,
                                                             const double* __restrict__ levelscale, NttTables tx,
                                                             NttTables ty) {
  __shared__ double redb[32];
  const int k = blockIdx.y;
  const int chunk = (Ms + gridDim.x - 1) / gridDim.x;
  const int e0 = blockIdx.x * chunk, e1 = min(Ms, e0 + chunk);
  const double ls = levelscale[k];  // 2^(e_v - 58)
  bool fast;
  const int ev = pow2_exponent(ls, fast);
  const double fx = tx.c_gscale * ls, fy = ty.c_gscale * ls;  // for levels whose scale is 0 or NaN
  const size_t n = (size_t)Nt * Ms, base = (size_t)k * Ms;
  double sq = 0.0;
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    uint32_t ax[NP], ay[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      ax[q] = rx[q * n + base + e];
      ay[q] = ry[q * n + base + e];
    }
    const double y = fast ? crt_to_double(crt4_top(ax, tx.crt), tx.gexp + ev) +
                                crt_to_double(crt4_top(ay, ty.crt), ty.gexp + ev)
                          : fx * crt_to_double(crt4_top(ax, tx.crt), 0) + fy * crt_to_double(crt4_top(ay, ty.crt), 0);
    double out = bdf_band(v + base + e, (size_t)Ms, k) + y;
    if (rhs) out = rhs[base + e] - out;
    w[base + e] = out;
    sq += out * out;
  }
  if (sq_partial) {
    double a[1] = {sq};
    block_sum<double, 1>(a, redb);
    if (threadIdx.x == 0) sq_partial[(size_t)k * gridDim.x + blockIdx.x] = a[0];
  }
}

template <typename TIn>
cudaError_t launch_ntt2d(const TIn* v, const double* rhs, double* w, double* sq_partial, int Mx, int My, int Nt,
                         int logLx, int logLy, const NttTables& tx, const NttTables& ty, uint32_t* res,
                         double* levelscale, cudaStream_t s) {
  const size_t Ms = (size_t)Mx * My, n = Ms * Nt;
  uint32_t* rx = res;
  uint32_t* ry = res + (size_t)NP * n;
  long long* V = reinterpret_cast<long long*>(res + (size_t)2 * NP * n);  // after both residue sets
  if constexpr (sizeof(TIn) == 4) ntt_quant_f32_kernel<QBITS><<<Nt, 512, 0, s>>>(v, (int)Ms, V, levelscale);
  else ntt_quant_kernel<TIn><<<Nt, 512, 0, s>>>(v, (int)Ms, V, levelscale);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int Lx = 1 << logLx, Ly = 1 << logLy;
  const int bx = ntt2d_lines_per_cta(logLx), by = ntt2d_lines_per_cta(logLy);
  const size_t smx = (size_t)bx * (Lx + Lx / 32 + 1) * sizeof(uint32_t);
  const size_t smy = (size_t)by * (Ly + Ly / 32 + 1) * sizeof(uint32_t);
  e = allow_max_dynamic_smem(ntt2d_lines_kernel<false>);
  if (e == cudaSuccess) e = allow_max_dynamic_smem(ntt2d_lines_kernel<true>);
  if (e != cudaSuccess) return e;
  ntt2d_lines_kernel<false><<<dim3((Nt * My + bx - 1) / bx, NP), 256, smx, s>>>(V, Mx, My, Nt, logLx, bx, tx, rx);
  ntt2d_lines_kernel<true><<<dim3((Nt * Mx + by - 1) / by, NP), 256, smy, s>>>(V, Mx, My, Nt, logLy, by, ty, ry);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ntt2d_epilogue_kernel<TIn><<<dim3(ntt2d_chunks(Mx, My), Nt), 256, 0, s>>>(v, rhs, w, sq_partial, (int)Ms, Nt, rx, ry,
                                                                           levelscale, tx, ty);
  return cudaGetLastError();
}

}  // namespace

int ntt_partials(int M, int Nt) { return Nt * epi_chunks(M); }

cudaError_t launch_matvec_ntt_fin_dots(const float* v, double* w, int M, int Nt, int logL, const NttTables& t,
                                       uint32_t* res, double* rowscale, const float2* V, size_t vstride, int nv,
                                       double* dots_partial, cudaStream_t s) {
  if (nv < 1 || nv > 65 || !V || !dots_partial) return cudaErrorInvalidValue;
  return launch_ntt<float>(v, nullptr, w, nullptr, M, Nt, logL, t, res, rowscale, s,
                           FusedDots{V, vstride, nv, dots_partial});
}

cudaError_t launch_matvec_ntt(const double* v, const double* rhs, double* w, double* sq_partial, int M, int Nt,
                              int logL, const NttTables& t, uint32_t* res, double* rowscale, cudaStream_t s) {
  return launch_ntt<double>(v, rhs, w, sq_partial, M, Nt, logL, t, res, rowscale, s);
}
cudaError_t launch_matvec_ntt_fin(const float* v, const double* rhs, double* w, double* sq_partial, int M, int Nt,
                                  int logL, const NttTables& t, uint32_t* res, double* rowscale, cudaStream_t s) {
  return launch_ntt<float>(v, rhs, w, sq_partial, M, Nt, logL, t, res, rowscale, s);
}

int ntt2d_partials(int Mx, int My, int Nt) { return Nt * ntt2d_chunks(Mx, My); }
size_t ntt2d_scratch_words(int Mx, int My, int Nt) { return (size_t)(2 * kNttPrimes + 2) * Mx * My * Nt; }

cudaError_t launch_matvec2d_ntt(const double* v, const double* rhs, double* w, double* sq_partial, int Mx, int My,
                                int Nt, int logLx, int logLy, const NttTables& tx, const NttTables& ty, uint32_t* res,
                                double* levelscale, cudaStream_t s) {
  return launch_ntt2d<double>(v, rhs, w, sq_partial, Mx, My, Nt, logLx, logLy, tx, ty, res, levelscale, s);
}
cudaError_t launch_matvec2d_ntt_fin(const float* v, const double* rhs, double* w, double* sq_partial, int Mx, int My,
                                    int Nt, int logLx, int logLy, const NttTables& tx, const NttTables& ty,
                                    uint32_t* res, double* levelscale, cudaStream_t s) {
  return launch_ntt2d<float>(v, rhs, w, sq_partial, Mx, My, Nt, logLx, logLy, tx, ty, res, levelscale, s);
}

}  // namespace aao
