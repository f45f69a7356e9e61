// Step (b) of Sec. 3.1 in FP32 for 4096 < M <= 8191 (L = 2^14): preconditioned COCG on
//   (lambda_n I + c T) x = b,  preconditioner (lambda_n I + c S)^{-1} (Strang, precomputed spectra),
// one shifted system per CTA of 512 threads, with the Krylov vectors in tensor memory.
//
// The register-resident kernel (cocg_reg.cuh) keeps r and p in registers, which leaves its FFT passes
// 64 registers and forces radix-16 passes (five round trips through shared memory per convolution).
// Here r and p live in TMEM (the SM's 256 KB tensor memory, 128 lanes x 512 columns of 32 bits,
// used as per-thread storage: a warp reaches the 32 lanes of its sub-partition), together with the
// thread's 31 twiddles W_L^{t m} of its first and last pass (read once per convolution half instead of
// looked up in the quarter table, whose strided reads conflict in the shared-memory banks), so the
// passes get the whole register file:
//   * first forward pass: 32 points at stride 512 (five radix-2 stages), of which the upper 16 are
//     the zero padding of the embedding, in the thread's registers;
//   * one 16-point pass at stride 32 through shared memory;
//   * the last forward pass, the spectrum product and the first backward pass: one 32-point group
//     of consecutive elements per thread;
//   * the inverse 16-point pass, and the last backward pass back into registers, keeping only the 16
//     outputs below L/2 (the thread's elements).
// Three round trips through shared memory per convolution instead of five.  Thread t owns elements
// i = t + 512 j, j < 16.  Element i of the buffer sits at i + i/32 (conflict-free for the 32-point
// groups of the fused pass).  Spectra are stored in the order of the fused pass (tm_order_freq).
// Same recurrence, stopping test, normalisation and breakdown test as the register-resident kernel.
#include <cstdint>

#include "cocg_reg.cuh"

namespace aao {
namespace {

constexpr int kTmLogL = 14, kTmL = 1 << kTmLogL, kTmNT = 512, kTmE = 16;
constexpr int kTmPadded = kTmL + kTmL / 32;
constexpr int kTmPassS = 32;                // stride of the 16-point pass (first stage 5)
constexpr int kTmTable = 15 * kTmPassS;     // its twiddles W_512^{j0 m}, [m - 1][j0]
constexpr int kTmCols = 512;                // TMEM columns allocated (r, p and 2 x 16 twiddles: 128 per thread, 4 warps per lane group)

__device__ __forceinline__ int pad32(int i) { return i + (i >> 5); }

// W_64^k = exp(-2 pi i k / 64) for a compile-time k < 32 (DIR > 0: the conjugate), from cos(2 pi k / 64),
// k <= 16, by the quarter-wave symmetries
template <int DIR> __device__ __forceinline__ float2 w64(int k) {
  constexpr float c[17] = {1.0f, 0.99518472667219688624f, 0.98078528040323044913f, 0.95694033573220886494f,
                           0.92387953251128675613f, 0.88192126434835502971f, 0.83146961230254523708f,
                           0.77301045336273696081f, 0.70710678118654752440f, 0.63439328416364549822f,
                           0.55557023301960222474f, 0.47139673682599764856f, 0.38268343236508977173f,
                           0.29028467725446236764f, 0.19509032201612826785f, 0.09801714032956060199f, 0.0f};
  const float cs = k <= 16 ? c[k] : -c[32 - k], sn = k <= 16 ? c[16 - k] : c[k - 16];
  return DIR < 0 ? float2{cs, -sn} : float2{cs, sn};
}
template <int DIR> __device__ __forceinline__ float2 w32(int k) { return w64<DIR>(2 * k); }

// 32-point DFT in registers, natural order in and out: a radix-2 split (X_{2m} from v_k + v_{k+16},
// X_{2m+1} from (v_k - v_{k+16}) W_32^k) and two 16-point DFTs.
template <int DIR> __device__ __forceinline__ void dft32(float2 (&v)[32]) {
  float2 a[16], b[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    a[k] = cadd(v[k], v[k + 16]);
    b[k] = csub(v[k], v[k + 16]);
    if (k > 0) b[k] = cmul(b[k], w32<DIR>(k));
  }
  dft<DIR, 4>(a);
  dft<DIR, 4>(b);
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    v[2 * m] = a[m];
    v[2 * m + 1] = b[m];
  }
}

// ---- tensor memory as per-thread storage --------------------------------------------------------
// A vector of 16 complex values per thread occupies 32 consecutive columns of the thread's lane.
__device__ __forceinline__ void tm_ld(uint32_t taddr, float2 (&v)[kTmE]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < kTmE; ++j) v[j] = float2{__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1])};
}

__device__ __forceinline__ void tm_st(uint32_t taddr, const float2 (&v)[kTmE]) {
  uint32_t r[32];
#pragma unroll
  for (int j = 0; j < kTmE; ++j) {
    r[2 * j] = __float_as_uint(v[j].x);
    r[2 * j + 1] = __float_as_uint(v[j].y);
  }
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};"
      :: "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
         "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
         "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
         "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tm_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// ---- the convolution ------------------------------------------------------------------------------
// v (the thread's 16 elements of a vector supported on [0, L/2)) <- the first L/2 outputs of its L-point
// cyclic convolution with the kernel whose spectrum F (or, if Fr is not null, the real spectrum Fr) is
// stored in fused-pass order.  buf: the padded
// transform buffer; pt: the 16-point pass's table; tE, tO: the TMEM addresses of the thread's twiddles
// W_L^{2 t m'} and W_L^{t (2 m' + 1)}, m' < 16.  Starts and ends synchronised.
__device__ __forceinline__ void tm_conv(float2* buf, const float2* pt, float2 (&v)[kTmE],
                                        const float2* __restrict__ F, const float* __restrict__ Fr, uint32_t tE,
                                        uint32_t tO) {
  const int t = threadIdx.x;
  // the thread's 32 spectrum values (one or two 128-byte lines) into L1 ahead of the fused pass
  if (Fr) {
    asm volatile("prefetch.global.L1 [%0];" :: "l"(Fr + (t << 5)));
  } else {
    asm volatile("prefetch.global.L1 [%0];" :: "l"(F + (t << 5)));
    asm volatile("prefetch.global.L1 [%0];" :: "l"(F + (t << 5) + 16));
  }
  // first forward pass (DIF, 32 points at stride 512, inputs 16..31 zero): output 2m' is the 16-point DFT
  // of v, output 2m'+1 that of v_k W_32^k; output m is multiplied by W_L^{t m} and stored at
  // t + bitrev_5(m) 512 (bitrev_5(2m') = bitrev_4(m'), bitrev_5(2m'+1) = 16 + bitrev_4(m'))
  {
    float2 h[16], w[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) h[k] = v[k];
    dft<-1, 4>(h);
    tm_ld(tE, w);
#pragma unroll
    for (int m = 0; m < 16; ++m) buf[pad32(t + brev_c<4>(m) * kTmNT)] = cmul(h[m], w[m]);
#pragma unroll
    for (int k = 0; k < 16; ++k) h[k] = k > 0 ? cmul(v[k], w32<-1>(k)) : v[k];
    dft<-1, 4>(h);
    tm_ld(tO, w);
#pragma unroll
    for (int m = 0; m < 16; ++m) buf[pad32(t + (16 + brev_c<4>(m)) * kTmNT)] = cmul(h[m], w[m]);
  }
  __syncthreads();
  // 16-point DIF pass, stages 5..8 (stride 32): two groups per thread
#pragma unroll 1
  for (int g = t; g < kTmL / 16; g += kTmNT) {
    const int j0 = g & (kTmPassS - 1), start = (g >> 5) << 9;
    float2 h[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) h[k] = buf[pad32(start + j0 + k * kTmPassS)];
    dft<-1, 4>(h);
    if (j0 != 0) {
#pragma unroll
      for (int m = 1; m < 16; ++m) h[m] = cmul(h[m], pt[(m - 1) * kTmPassS + j0]);
    }
#pragma unroll
    for (int m = 0; m < 16; ++m) buf[pad32(start + j0 + brev_c<4>(m) * kTmPassS)] = h[m];
  }
  __syncthreads();
  // stages 9..13 forward (32 consecutive points), the spectrum product at fused index start + m, and
  // the same stages backward
  {
    const int start = t << 5;
    float2 h[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) h[k] = buf[pad32(start + k)];
    dft32<-1>(h);
    if (Fr) {  // a real spectrum (the Toeplitz embedding's): four values per 16-byte load
      const float4* F4 = reinterpret_cast<const float4*>(Fr + start);  // 16-byte aligned: start is a multiple of 32
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const float4 f = __ldg(&F4[m]);
        h[4 * m] = cscale(h[4 * m], f.x);
        h[4 * m + 1] = cscale(h[4 * m + 1], f.y);
        h[4 * m + 2] = cscale(h[4 * m + 2], f.z);
        h[4 * m + 3] = cscale(h[4 * m + 3], f.w);
      }
    } else {  // complex: two values per load
      const float4* F4 = reinterpret_cast<const float4*>(F + start);
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const float4 f = __ldg(&F4[m]);
        h[2 * m] = cmul(h[2 * m], float2{f.x, f.y});
        h[2 * m + 1] = cmul(h[2 * m + 1], float2{f.z, f.w});
      }
    }
    dft32<+1>(h);
#pragma unroll
    for (int k = 0; k < 32; ++k) buf[pad32(start + k)] = h[k];
  }
  __syncthreads();
  // inverse of the 16-point pass
#pragma unroll 1
  for (int g = t; g < kTmL / 16; g += kTmNT) {
    const int j0 = g & (kTmPassS - 1), start = (g >> 5) << 9;
    float2 h[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) h[m] = buf[pad32(start + j0 + brev_c<4>(m) * kTmPassS)];
    if (j0 != 0) {
#pragma unroll
      for (int m = 1; m < 16; ++m) h[m] = cmulc(h[m], pt[(m - 1) * kTmPassS + j0]);
    }
    dft<+1, 4>(h);
#pragma unroll
    for (int k = 0; k < 16; ++k) buf[pad32(start + j0 + k * kTmPassS)] = h[k];
  }
  __syncthreads();
  // last backward pass: outputs k < 16 only, x_k = A_k + W_32^{-k} B_k with A, B the 16-point inverse DFTs
  // of the even and odd inputs (each multiplied by W_L^{-t m} first)
  {
    float2 h[16], w[16];
    tm_ld(tE, w);
#pragma unroll
    for (int m = 0; m < 16; ++m) h[m] = cmulc(buf[pad32(t + brev_c<4>(m) * kTmNT)], w[m]);
    dft<+1, 4>(h);
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = h[k];
    tm_ld(tO, w);
#pragma unroll
    for (int m = 0; m < 16; ++m) h[m] = cmulc(buf[pad32(t + (16 + brev_c<4>(m)) * kTmNT)], w[m]);
    dft<+1, 4>(h);
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = cadd(v[k], k > 0 ? cmul(h[k], w32<+1>(k)) : h[k]);
  }
  __syncthreads();  // the next convolution overwrites buf
}

struct TmScalars {
  float2 lam, rho;
  float bs, nb2, thr;
  uint32_t tmem;
};

// COCG on one shifted system per CTA.  The iteration alternates two kinds of step around one
// convolution (so that its code exists once): kind 0 applies the preconditioner to r (z, rho, beta,
// p = z + beta p), kind 1 the Toeplitz product to p (q = lambda p + c T p, alpha, x, r).
__global__ void __launch_bounds__(kTmNT, 1)
    cocg_tm_kernel(float2* __restrict__ xb, int M, int nsys, CocgTmTables tb, float tol, int maxit,
                   int* __restrict__ iters, int* __restrict__ flags) {
  extern __shared__ unsigned char smraw[];
  float2* buf = reinterpret_cast<float2*>(smraw);
  float2* q = buf + kTmPadded;
  float2* pt = q + kTmL / 4;
  float* red = reinterpret_cast<float*>(pt + kTmTable);
  __shared__ TmScalars sc;
  const int t = threadIdx.x, warp = t >> 5;
  const int n = blockIdx.x;
  if (n >= nsys) return;
  // TMEM: 512 columns (one CTA per SM: the shared memory allows no second one, so the allocation
  // never waits); warp w uses lanes 32 (w mod 4) .. +31 and columns 128 (w div 4) + {0: r, 32: p,
  // 64: W_L^{2 t m'}, 96: W_L^{t (2m'+1)}}
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"((uint32_t)__cvta_generic_to_shared(&sc.tmem)), "r"((uint32_t)kTmCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  load_quarter(q, tb.twL, kTmL / 4);
  tm_fence_before();
  __syncthreads();
  tm_fence_after();
  for (int idx = t; idx < kTmTable; idx += kTmNT) {  // W_512^{j0 m} = W_L^{32 j0 m}
    const int m = idx / kTmPassS + 1, j0 = idx - (m - 1) * kTmPassS;
    pt[idx] = twiddle<-1>(q, (j0 * m) << 5, kTmLogL);
  }
  const uint32_t tbase = sc.tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 128u * (uint32_t)(warp >> 2);
  const uint32_t tR = tbase, tP = tbase + 32, tE = tbase + 64, tO = tbase + 96;
  float2* const xt = xb + (size_t)n * M + t;
  const float2* const G = tb.sconv + ((size_t)n << kTmLogL);
  {
    float2 w[kTmE];
#pragma unroll
    for (int m = 0; m < kTmE; ++m) w[m] = twiddle<-1>(q, t * (2 * m), kTmLogL);
    tm_st(tE, w);
#pragma unroll
    for (int m = 0; m < kTmE; ++m) w[m] = twiddle<-1>(q, t * (2 * m + 1), kTmLogL);
    tm_st(tO, w);
  }

  // b / ||b||_1 (zero beyond M) into r; x = 0
  float2 v[kTmE];
  float b1[1] = {0};
#pragma unroll
  for (int j = 0; j < kTmE; ++j) {
    v[j] = t + kTmNT * j < M ? xt[kTmNT * j] : float2{0, 0};
    b1[0] += fabsf(v[j].x) + fabsf(v[j].y);
  }
  block_sum<float, 1>(b1, red);
  int it = 0, flag = 1;
  if (!(b1[0] > 0.0f) || b1[0] > 3.0e38f) {  // zero right-hand side, or NaN / infinity in it
    flag = b1[0] == 0.0f ? 0 : 3;
#pragma unroll
    for (int j = 0; j < kTmE; ++j)
      if (t + kTmNT * j < M) xt[kTmNT * j] = float2{0, 0};
  } else {
    {
      const float ibs = 1.0f / b1[0];
      float nb2[1] = {0};
#pragma unroll
      for (int j = 0; j < kTmE; ++j) {
        v[j] = float2{v[j].x * ibs, v[j].y * ibs};
        nb2[0] += v[j].x * v[j].x + v[j].y * v[j].y;
      }
      tm_st(tR, v);
#pragma unroll
      for (int j = 0; j < kTmE; ++j)
        if (t + kTmNT * j < M) xt[kTmNT * j] = float2{0, 0};
      block_sum<float, 1>(nb2, red);
      if (t == 0) {
        const double2 lamd = tb.lambda[n];
        sc.lam = float2{(float)lamd.x, (float)lamd.y};
        sc.bs = b1[0];
        sc.nb2 = nb2[0];
        sc.thr = tol * tol * nb2[0];
      }
    }
    int kind = 0;
    bool first = true;
#pragma unroll 1
    for (;;) {
      tm_ld(kind ? tP : tR, v);
      tm_conv(buf, pt, v, G, kind ? tb.Ebr : nullptr, tE, tO);
      if (kind == 0) {
        // z = v (zero beyond M); rho = r^T z; p = z (first step) or z + beta p
#pragma unroll
        for (int j = 0; j < kTmE; ++j)
          if (t + kTmNT * j >= M) v[j] = float2{0, 0};
        float rz[4] = {0, 0, 0, 0};  // r^T z, |z|^2, |r|^2
        {
          float2 r[kTmE];
          tm_ld(tR, r);
#pragma unroll
          for (int j = 0; j < kTmE; ++j) {
            rz[0] += r[j].x * v[j].x - r[j].y * v[j].y;
            rz[1] += r[j].x * v[j].y + r[j].y * v[j].x;
            rz[2] += v[j].x * v[j].x + v[j].y * v[j].y;
            rz[3] += r[j].x * r[j].x + r[j].y * r[j].y;
          }
        }
        block_sum<float, 4>(rz, red);
        // rho divides the next beta: |r^T z| at rounding level of ||r|| ||z|| is a breakdown
        if (near_breakdown(rz[0], rz[1], rz[2], rz[3])) { flag = 2; break; }
        const float2 rho_new{rz[0], rz[1]};
        if (!first) {
          const float2 beta = cdiv(rho_new, sc.rho);
          float2 p[kTmE];
          tm_ld(tP, p);
#pragma unroll
          for (int j = 0; j < kTmE; ++j) v[j] = cadd(v[j], cmul(beta, p[j]));
        }
        tm_st(tP, v);
        first = false;
        __syncthreads();  // every thread has read sc.rho
        if (t == 0) sc.rho = rho_new;
        if (it >= maxit) break;
        kind = 1;
      } else {
        // q = v + lambda p (zero beyond M), alpha = rho / p^T q
        const float2 lam = sc.lam;
        float pq[4] = {0, 0, 0, 0};  // p^T q, |p|^2, |q|^2
        {
          float2 p[kTmE];
          tm_ld(tP, p);
#pragma unroll
          for (int j = 0; j < kTmE; ++j) {
            v[j] = t + kTmNT * j < M ? cadd(v[j], cmul(lam, p[j])) : float2{0, 0};
            pq[0] += p[j].x * v[j].x - p[j].y * v[j].y;
            pq[1] += p[j].x * v[j].y + p[j].y * v[j].x;
            pq[2] += p[j].x * p[j].x + p[j].y * p[j].y;
            pq[3] += v[j].x * v[j].x + v[j].y * v[j].y;
          }
        }
        block_sum<float, 4>(pq, red);
        if (near_breakdown(pq[0], pq[1], pq[2], pq[3])) { flag = 2; break; }
        const float2 a = cdiv(sc.rho, float2{pq[0], pq[1]});
        float rr[1] = {0};
        {
          float2 r[kTmE];
          tm_ld(tR, r);
#pragma unroll
          for (int j = 0; j < kTmE; ++j) {
            r[j] = csub(r[j], cmul(a, v[j]));
            rr[0] += r[j].x * r[j].x + r[j].y * r[j].y;
          }
          tm_st(tR, r);
        }
        {
          const float bs = sc.bs;
          const float2 ax{a.x * bs, a.y * bs};  // the step in the units of b
          float2 p[kTmE];
          tm_ld(tP, p);
#pragma unroll
          for (int j = 0; j < kTmE; ++j)
            if (t + kTmNT * j < M) xt[kTmNT * j] = cadd(xt[kTmNT * j], cmul(ax, p[j]));
        }
        block_sum<float, 1>(rr, red);
        ++it;
        if (!(rr[0] == rr[0]) || rr[0] > 1e30f * sc.nb2) { flag = 3; break; }
        if (rr[0] <= sc.thr) { flag = 0; break; }
        kind = 0;
      }
    }
  }
  if (t == 0) { iters[n] = it; flags[n] = flag; }
  // release TMEM once every warp's accesses are complete
  tm_fence_before();
  __syncthreads();
  if (warp == 0) {
    tm_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(sc.tmem), "r"((uint32_t)kTmCols)
                 : "memory");
  }
}

}  // namespace

size_t cocg_tm_smem_bytes() {
  return ((size_t)kTmPadded + kTmL / 4 + kTmTable) * sizeof(float2) + 4 * 32 * sizeof(float);
}

bool cocg_tm_supported(int M, int logL) { return logL == kTmLogL && M > kTmL / 4 && M <= kTmL / 2; }

int tm_order_freq(int s) {
  // fused index s = 32 g + m (m the natural output index of the group's 32-point DFT) sits at
  // bit-reversed position 32 g + bitrev_5(m), i.e. natural frequency bitrev_14(32 g + bitrev_5(m))
  const int m = s & 31, start = s - m;
  int mb = 0;
  for (int b = 0; b < 5; ++b) mb |= ((m >> b) & 1) << (4 - b);
  const int pos = start + mb;
  int f = 0;
  for (int b = 0; b < kTmLogL; ++b) f |= ((pos >> b) & 1) << (kTmLogL - 1 - b);
  return f;
}

__global__ void tm_gather_kernel(const float2* __restrict__ src, float2* __restrict__ dst, const int* __restrict__ perm,
                                 int nsys) {
  const size_t tot = (size_t)kTmL * nsys;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = src[(e & ~(size_t)(kTmL - 1)) + perm[e & (kTmL - 1)]];
}

__global__ void tm_gather_real_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                      const int* __restrict__ perm) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kTmL; e += gridDim.x * blockDim.x) dst[e] = src[perm[e]];
}

cudaError_t launch_tm_gather(const float2* src, float2* dst, const float* srcr, float* dstr, const int* perm, int nsys,
                             cudaStream_t s) {
  tm_gather_kernel<<<4 * 152, 256, 0, s>>>(src, dst, perm, nsys);
  tm_gather_real_kernel<<<kTmL / 256, 256, 0, s>>>(srcr, dstr, perm);
  return cudaGetLastError();
}

cudaError_t launch_cocg_tm(float2* xb, int M, int logL, int nsys, const CocgTmTables& tb, float tol, int maxit,
                           int* iters, int* flags, cudaStream_t s) {
  if (!cocg_tm_supported(M, logL)) return cudaErrorInvalidValue;
  cudaError_t e = allow_max_dynamic_smem(cocg_tm_kernel);
  if (e != cudaSuccess) return e;
  cocg_tm_kernel<<<nsys, kTmNT, cocg_tm_smem_bytes(), s>>>(xb, M, nsys, tb, tol, maxit, iters, flags);
  return cudaGetLastError();
}

}  // namespace aao
