// Device helpers shared by the sm_103a kernels: complex arithmetic, the
// in-shared-memory radix-2^r FFT engine, and deterministic block reductions.
//
// FFT conventions (used by every kernel of the library):
//   * forward  = DIF, X_k = sum_j x_j exp(-2 pi i jk/N), natural order in,
//                bit-reversed order out;
//   * backward = DIT, x_j = sum_k X_k exp(+2 pi i jk/N) (no 1/N), bit-reversed
//                order in, natural order out.
// A convolution therefore never permutes: DIF, multiply by a kernel
// spectrum stored in bit-reversed order, DIT.
//
// Shared-memory layout: element i of a transform lives at pad(i) =
// i + (i >> 4), which makes the unit-stride last pass free of bank conflicts.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace aao {

template <typename R> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };

template <typename T> __device__ __forceinline__ T cadd(T a, T b) { return T{a.x + b.x, a.y + b.y}; }
template <typename T> __device__ __forceinline__ T csub(T a, T b) { return T{a.x - b.x, a.y - b.y}; }
template <typename T> __device__ __forceinline__ T cmul(T a, T b) {
  return T{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * conj(b)
template <typename T> __device__ __forceinline__ T cmulc(T a, T b) {
  return T{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <typename T, typename R> __device__ __forceinline__ T cscale(T a, R s) { return T{a.x * s, a.y * s}; }
template <typename T> __device__ __forceinline__ T cconj(T a) { return T{a.x, -a.y}; }

__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }
__host__ __device__ inline int padded_size(int n) { return n + (n >> 4); }

__device__ __forceinline__ int bitrev(int k, int logN) { return (int)(__brev((unsigned)k) >> (32 - logN)); }

// One DIF pass of r radix-2 stages (global stages s0 .. s0+r-1) over `batch`
// transforms of length N = 2^logN stored at buf[b*bstride + pad16(i)].
// tw[m << twshift] = exp(-2 pi i m / N) for m < N/2.
template <typename T, int r>
__device__ __forceinline__ void dif_pass(T* buf, int logN, int s0, int batch, int bstride,
                                         const T* __restrict__ tw, int twshift) {
  const int S = 1 << (logN - s0 - r);
  const int per = 1 << (logN - r);
  for (int g = threadIdx.x; g < batch * per; g += blockDim.x) {
    const int b = g >> (logN - r);
    const int gi = g & (per - 1);
    const int j0 = gi & (S - 1);
    const int start = (gi >> (logN - s0 - r)) << (logN - s0);
    T* base = buf + b * bstride;
    T v[1 << r];
#pragma unroll
    for (int k = 0; k < (1 << r); ++k) v[k] = base[pad16(start + j0 + k * S)];
#pragma unroll
    for (int t = 0; t < r; ++t) {
      const int hk = 1 << (r - t - 1);
#pragma unroll
      for (int k = 0; k < (1 << r); ++k) {
        if (k & hk) continue;
        const int j = j0 + (k & (hk - 1)) * S;
        const T a = v[k], c = v[k + hk];
        v[k] = cadd(a, c);
        v[k + hk] = cmul(csub(a, c), __ldg(&tw[(j << (s0 + t)) << twshift]));
      }
    }
#pragma unroll
    for (int k = 0; k < (1 << r); ++k) base[pad16(start + j0 + k * S)] = v[k];
  }
}

// The inverse of dif_pass (stages s0+r-1 down to s0, conjugate twiddles).
template <typename T, int r>
__device__ __forceinline__ void dit_pass(T* buf, int logN, int s0, int batch, int bstride,
                                         const T* __restrict__ tw, int twshift) {
  const int S = 1 << (logN - s0 - r);
  const int per = 1 << (logN - r);
  for (int g = threadIdx.x; g < batch * per; g += blockDim.x) {
    const int b = g >> (logN - r);
    const int gi = g & (per - 1);
    const int j0 = gi & (S - 1);
    const int start = (gi >> (logN - s0 - r)) << (logN - s0);
    T* base = buf + b * bstride;
    T v[1 << r];
#pragma unroll
    for (int k = 0; k < (1 << r); ++k) v[k] = base[pad16(start + j0 + k * S)];
#pragma unroll
    for (int t = r - 1; t >= 0; --t) {
      const int hk = 1 << (r - t - 1);
#pragma unroll
      for (int k = 0; k < (1 << r); ++k) {
        if (k & hk) continue;
        const int j = j0 + (k & (hk - 1)) * S;
        const T a = v[k];
        const T c = cmulc(v[k + hk], __ldg(&tw[(j << (s0 + t)) << twshift]));
        v[k] = cadd(a, c);
        v[k + hk] = csub(a, c);
      }
    }
#pragma unroll
    for (int k = 0; k < (1 << r); ++k) base[pad16(start + j0 + k * S)] = v[k];
  }
}

// The first pass takes the leftover logN mod 4 stages so that every later
// pass has stride >= 16 (or exactly 1 for the last one).
__device__ __forceinline__ int first_pass_stages(int logN) {
  const int rem = logN & 3;
  return rem ? rem : 4;
}

// Forward FFT (DIF) of `batch` transforms; ends with __syncthreads().
template <typename T>
__device__ void fft_forward(T* buf, int logN, int batch, int bstride, const T* __restrict__ tw, int twshift) {
  int s0 = 0;
  int r = first_pass_stages(logN);
  while (s0 < logN) {
    switch (r) {
      case 1: dif_pass<T, 1>(buf, logN, s0, batch, bstride, tw, twshift); break;
      case 2: dif_pass<T, 2>(buf, logN, s0, batch, bstride, tw, twshift); break;
      case 3: dif_pass<T, 3>(buf, logN, s0, batch, bstride, tw, twshift); break;
      default: dif_pass<T, 4>(buf, logN, s0, batch, bstride, tw, twshift); break;
    }
    __syncthreads();
    s0 += r;
    r = 4;
  }
}

// Backward FFT (DIT, unnormalised) of `batch` transforms; ends with __syncthreads().
template <typename T>
__device__ void fft_backward(T* buf, int logN, int batch, int bstride, const T* __restrict__ tw, int twshift) {
  const int r0 = first_pass_stages(logN);
  int s0 = logN - 4;
  while (s0 >= r0) {
    dit_pass<T, 4>(buf, logN, s0, batch, bstride, tw, twshift);
    __syncthreads();
    s0 -= 4;
  }
  switch (r0) {
    case 1: dit_pass<T, 1>(buf, logN, 0, batch, bstride, tw, twshift); break;
    case 2: dit_pass<T, 2>(buf, logN, 0, batch, bstride, tw, twshift); break;
    case 3: dit_pass<T, 3>(buf, logN, 0, batch, bstride, tw, twshift); break;
    default: dit_pass<T, 4>(buf, logN, 0, batch, bstride, tw, twshift); break;
  }
  __syncthreads();
}

// Block-wide sum of NV values per thread; the result is valid in every thread.
// Deterministic: fixed shuffle tree, then a fixed-order sum over warps.
// `scratch` must hold NV * 32 values of R.  Ends synchronised.
template <typename R, int NV>
__device__ __forceinline__ void block_sum(R (&v)[NV], R* scratch) {
#pragma unroll
  for (int q = 0; q < NV; ++q)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) scratch[q * 32 + warp] = v[q];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    R s = 0;
    for (int w = 0; w < nw; ++w) s += scratch[q * 32 + w];
    v[q] = s;
  }
  __syncthreads();
}

}  // namespace aao
