// Time-direction DFTs of the block-circulant preconditioner, Sec. 3.1:
//   Step (a): zhat_n = sum_k eps^{k/Nt} theta^{nk} v_k,        n = 0 .. Nt/2
//   Step (c): z_k    = eps^{-k/Nt} (1/Nt) sum_n x_n theta^{-nk}, x_{Nt-n} = conj(x_n)
// with theta = exp(2 pi i / Nt).  Only the half spectrum is kept because v
// is real (Sec. 3.2: the systems come in conjugate pairs).
//
// Each CTA owns a tile of TW spatial columns over all Nt time rows; the rows
// are read as contiguous TW-column segments (coalesced) and the column pairs
// (q, q + TW/2) are packed as one complex transform.
#include "common.cuh"
#include "kernels.h"

namespace aao {

constexpr int TW = 8;    // columns per CTA (8, 16 and 32 measured at M = 8191, Nt = 1024: 8 is fastest)
constexpr int TWH = TW / 2;
constexpr int LU = 8;    // independent global loads in flight per thread (the loads are latency-bound)

template <typename R> __device__ __forceinline__ R ldv(const double* p) { return (R)__ldg(p); }
// a float-float element hi + lo read in FP32: hi (|lo| is below half an FP32 ulp of hi)
template <typename R> __device__ __forceinline__ R ldv(const float2* p) { return (R)__ldg(p).x; }

// ---- Step (a) ----
template <typename R, typename TV>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 1) tdft_fwd_kernel(const TV* __restrict__ v,
                                                       typename cplx_t<R>::type* __restrict__ out, int M,
                                                       int logNt, const R* __restrict__ scale,
                                                       const typename cplx_t<R>::type* __restrict__ tw) {
  using C = typename cplx_t<R>::type;
  extern __shared__ unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  R* smr = reinterpret_cast<R*>(smraw);
  const int Nt = 1 << logNt;
  const int bstride = padded_size(Nt) + 1;  // odd stride: the TW/2 transforms start in different banks
  const int c0 = blockIdx.x * TW;
  C* tq = sm + TWH * bstride;
  C* pt = tq + Nt / 4;  // per-pass twiddle tables (conflict-free reads in the 16-point passes)
  load_quarter(tq, tw, Nt / 4);
  __syncthreads();
  build_pass_tables(pt, tq, logNt, logNt);
  // load y_k = scale_k v_k (real) into position bitrev(k); column cc -> transform cc % TWH, part cc / TWH
  for (int base = threadIdx.x; base < Nt * TW; base += LU * blockDim.x) {
    R vals[LU];
#pragma unroll
    for (int u = 0; u < LU; ++u) {
      const int idx = base + u * blockDim.x;
      const int k = idx / TW, col = c0 + (idx - k * TW);
      vals[u] = (idx < Nt * TW && col < M) ? ldv<R>(v + (size_t)k * M + col) : (R)0;
    }
#pragma unroll
    for (int u = 0; u < LU; ++u) {
      const int idx = base + u * blockDim.x;
      if (idx >= Nt * TW) break;
      const int k = idx / TW, cc = idx - k * TW;
      const int q = cc & (TWH - 1), part = cc / TWH;
      smr[2 * (q * bstride + pad16(bitrev(k, logNt))) + part] = vals[u] * __ldg(&scale[k]);
    }
  }
  fft_backward(sm, logNt, TWH, bstride, tq, logNt, pt);  // sum_k y_k exp(+2 pi i nk/Nt), natural order
  const int half = Nt / 2;
  for (int idx = threadIdx.x; idx < (half + 1) * TW; idx += blockDim.x) {
    const int n = idx / TW, cc = idx - n * TW;
    const int col = c0 + cc;
    if (col >= M) continue;
    const int q = cc & (TWH - 1), part = cc / TWH;
    const C Zn = sm[q * bstride + pad16(n)];
    const C Zm = sm[q * bstride + pad16((Nt - n) & (Nt - 1))];
    C X;
    if (part == 0) X = C{(R)0.5 * (Zn.x + Zm.x), (R)0.5 * (Zn.y - Zm.y)};   // (Z_n + conj Z_{-n})/2
    else X = C{(R)0.5 * (Zn.y + Zm.y), (R)-0.5 * (Zn.x - Zm.x)};          // (Z_n - conj Z_{-n})/(2i)
    out[(size_t)n * M + col] = X;
  }
}

// Step (a) for Nt >= 64 with the first four radix-2 stages in registers.  The forward (DIF, sign -)
// transform of w_k = conj(y_k) gives conj(Z_n) in bit-reversed order, so no permutation is needed at the
// input: the first pass takes 16 rows at stride Nt / 16 of one column pair straight from global memory,
// every load of the pass issued together (the tile loads of tdft_fwd_kernel wait out one memory latency per
// round of 8), scales, transforms and stores them; the remaining stages run in shared memory.
template <typename R, typename TV>
__global__ void __launch_bounds__(256, 4) tdft_fwd_reg_kernel(const TV* __restrict__ v,
                                                              typename cplx_t<R>::type* __restrict__ out, int M,
                                                              int logNt, const R* __restrict__ scale,
                                                              const typename cplx_t<R>::type* __restrict__ tw) {
  using C = typename cplx_t<R>::type;
  extern __shared__ unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int Nt = 1 << logNt, S = Nt >> 4;
  const int bstride = padded_size(Nt) + 1;
  const int c0 = blockIdx.x * TW;
  C* tq = sm + TWH * bstride;
  load_quarter(tq, tw, Nt / 4);
  __syncthreads();
  for (int gg = threadIdx.x; gg < TWH * S; gg += blockDim.x) {
    const int q = gg & (TWH - 1), j0 = gg / TWH;
    const int ca = c0 + q, cb = ca + TWH;
    C w[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int k = j0 + m * S;
      const R a = ca < M ? ldv<R>(v + (size_t)k * M + ca) : (R)0;
      const R b = cb < M ? ldv<R>(v + (size_t)k * M + cb) : (R)0;
      w[m] = C{a, -b};
    }
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const R sc = __ldg(&scale[j0 + m * S]);
      w[m] = C{w[m].x * sc, w[m].y * sc};
    }
    dft<-1, 4>(w);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      if (j0 != 0 && m != 0) w[m] = cmul(w[m], twiddle<-1>(tq, j0 * m, logNt));
      sm[q * bstride + pad16(j0 + brev_c<4>(m) * S)] = w[m];
    }
  }
  __syncthreads();
  for (int s0 = 4; s0 < logNt; s0 += 4) {
    dif_pass_any<C>(min(4, logNt - s0), sm, logNt, s0, TWH, bstride, tq, logNt);
    __syncthreads();
  }
  const int half = Nt / 2;
  for (int idx = threadIdx.x; idx < (half + 1) * TW; idx += blockDim.x) {
    const int n = idx / TW, cc = idx - n * TW;
    const int col = c0 + cc;
    if (col >= M) continue;
    const int q = cc & (TWH - 1), part = cc / TWH;
    const C Wn = sm[q * bstride + pad16(bitrev(n, logNt))];
    const C Wm = sm[q * bstride + pad16(bitrev((Nt - n) & (Nt - 1), logNt))];
    const C Zn{Wn.x, -Wn.y}, Zm{Wm.x, -Wm.y};  // Z = conj(W)
    C X;
    if (part == 0) X = C{(R)0.5 * (Zn.x + Zm.x), (R)0.5 * (Zn.y - Zm.y)};   // (Z_n + conj Z_{-n})/2
    else X = C{(R)0.5 * (Zn.y + Zm.y), (R)-0.5 * (Zn.x - Zm.x)};          // (Z_n - conj Z_{-n})/(2i)
    out[(size_t)n * M + col] = X;
  }
}

// ---- Step (c) ----
template <typename R, typename TOut>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 1) tdft_inv_kernel(const typename cplx_t<R>::type* __restrict__ in,
                                                       TOut* __restrict__ z, int M, int logNt,
                                                       const R* __restrict__ scale_inv,
                                                       const typename cplx_t<R>::type* __restrict__ tw) {
  using C = typename cplx_t<R>::type;
  extern __shared__ unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int Nt = 1 << logNt;
  const int bstride = padded_size(Nt) + 1;  // odd stride: the TW/2 transforms start in different banks
  const int c0 = blockIdx.x * TW;
  const int half = Nt / 2;
  C* tq = sm + TWH * bstride;
  C* pt = tq + Nt / 4;
  load_quarter(tq, tw, Nt / 4);
  __syncthreads();
  build_pass_tables(pt, tq, logNt, logNt);
  const int nin = (half + 1) * TWH;
  for (int base = threadIdx.x; base < nin; base += LU * blockDim.x) {
    C xa[LU], xb[LU];
#pragma unroll
    for (int u = 0; u < LU; ++u) {
      const int idx = base + u * blockDim.x;
      const int n = idx / TWH, q = idx - n * TWH;
      const int ca = c0 + q, cb = c0 + q + TWH;
      xa[u] = (idx < nin && ca < M) ? in[(size_t)n * M + ca] : C{0, 0};
      xb[u] = (idx < nin && cb < M) ? in[(size_t)n * M + cb] : C{0, 0};
    }
#pragma unroll
    for (int u = 0; u < LU; ++u) {
      const int idx = base + u * blockDim.x;
      if (idx >= nin) break;
      const int n = idx / TWH, q = idx - n * TWH;
      C Xa = xa[u], Xb = xb[u];
      if (n == 0 || n == half) { Xa.y = 0; Xb.y = 0; }
      sm[q * bstride + pad16(n)] = C{Xa.x - Xb.y, Xa.y + Xb.x};                  // Xa + i Xb
      if (n != 0 && n != half) sm[q * bstride + pad16(Nt - n)] = C{Xa.x + Xb.y, Xb.x - Xa.y};  // conj Xa + i conj Xb
    }
  }
  fft_forward(sm, logNt, TWH, bstride, tq, logNt, pt);  // sum_n Z_n exp(-2 pi i nk/Nt), bit-reversed
  for (int idx = threadIdx.x; idx < Nt * TW; idx += blockDim.x) {
    const int k = idx / TW, cc = idx - k * TW;
    const int col = c0 + cc;
    if (col >= M) continue;
    const int q = cc & (TWH - 1), part = cc / TWH;
    const C Zk = sm[q * bstride + pad16(bitrev(k, logNt))];
    const R val = (part == 0 ? Zk.x : Zk.y) * __ldg(&scale_inv[k]);
    z[(size_t)k * M + col] = (TOut)val;
  }
}

static int ilog2i(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }

template <typename R>
static size_t tdft_smem(int Nt) {
  return ((size_t)TWH * (padded_size(Nt) + 1) + (size_t)(Nt / 4) + (size_t)pass_table_size(ilog2i(Nt))) *
         sizeof(typename cplx_t<R>::type);
}


size_t tdft_smem_bytes(int Nt, bool fp32) { return fp32 ? tdft_smem<float>(Nt) : tdft_smem<double>(Nt); }

int tdft_max_Nt(bool fp32, size_t smem_limit) {
  int best = 0;
  for (int Nt = 4; Nt <= (1 << 16); Nt *= 2)
    if (tdft_smem_bytes(Nt, fp32) <= smem_limit) best = Nt;
  return best;
}

template <typename R, typename TV>
static cudaError_t fwd(const TV* v, typename cplx_t<R>::type* out, int M, int Nt, const R* scale,
                       const typename cplx_t<R>::type* tw, cudaStream_t s) {
  const size_t smem = tdft_smem<R>(Nt);
  if constexpr (sizeof(R) == 4) {
    if (Nt >= 64) {
      cudaError_t e = allow_max_dynamic_smem(tdft_fwd_reg_kernel<R, TV>);
      if (e != cudaSuccess) return e;
      tdft_fwd_reg_kernel<R, TV><<<(M + TW - 1) / TW, 256, smem, s>>>(v, out, M, ilog2i(Nt), scale, tw);
      return cudaGetLastError();
    }
  }
  cudaError_t e = allow_max_dynamic_smem(tdft_fwd_kernel<R, TV>);
  if (e != cudaSuccess) return e;
  tdft_fwd_kernel<R, TV><<<(M + TW - 1) / TW, 256, smem, s>>>(v, out, M, ilog2i(Nt), scale, tw);
  return cudaGetLastError();
}

template <typename R, typename TOut>
static cudaError_t inv(const typename cplx_t<R>::type* in, TOut* z, int M, int Nt, const R* scale_inv,
                       const typename cplx_t<R>::type* tw, cudaStream_t s) {
  const size_t smem = tdft_smem<R>(Nt);
  cudaError_t e = allow_max_dynamic_smem(tdft_inv_kernel<R, TOut>);
  if (e != cudaSuccess) return e;
  tdft_inv_kernel<R, TOut><<<(M + TW - 1) / TW, 256, smem, s>>>(in, z, M, ilog2i(Nt), scale_inv, tw);
  return cudaGetLastError();
}

cudaError_t launch_tdft_fwd_f32(const double* v, float2* out, int M, int Nt, const float* scale,
                                const float2* twNt, cudaStream_t s) {
  return fwd<float, double>(v, out, M, Nt, scale, twNt, s);
}
cudaError_t launch_tdft_fwd_f32_ff(const float2* v, float2* out, int M, int Nt, const float* scale,
                                   const float2* twNt, cudaStream_t s) {
  return fwd<float, float2>(v, out, M, Nt, scale, twNt, s);
}
cudaError_t launch_tdft_fwd_f64(const double* v, double2* out, int M, int Nt, const double* scale,
                                const double2* twNt, cudaStream_t s) {
  return fwd<double, double>(v, out, M, Nt, scale, twNt, s);
}
cudaError_t launch_tdft_inv_f32(const float2* in, float* z, int M, int Nt, const float* scale_inv,
                                const float2* twNt, cudaStream_t s) {
  return inv<float, float>(in, z, M, Nt, scale_inv, twNt, s);
}
cudaError_t launch_tdft_inv_f32_to_f64(const float2* in, double* z, int M, int Nt, const float* scale_inv,
                                       const float2* twNt, cudaStream_t s) {
  return inv<float, double>(in, z, M, Nt, scale_inv, twNt, s);
}
cudaError_t launch_tdft_inv_f64(const double2* in, double* z, int M, int Nt, const double* scale_inv,
                                const double2* twNt, cudaStream_t s) {
  return inv<double, double>(in, z, M, Nt, scale_inv, twNt, s);
}

}  // namespace aao
