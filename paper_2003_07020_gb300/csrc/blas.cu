// Vector kernels for the flexible GMRES driver: classical Gram-Schmidt with
// re-orthogonalisation (two passes) fused into three sweeps, in FP64 or on a
// float-float basis (mixed precision), the
// solution update U += Z y, the right-hand side of Eq. 12, and deterministic
// two-stage reductions (per-block partial sums, then a fixed-order sum).
#include <mutex>
#include <set>
#include <utility>

#include "common.cuh"
#include "ff.cuh"
#include "kernels.h"

namespace aao {

cudaError_t allow_max_dynamic_smem_impl(const void* kern) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({kern, dev})) return cudaSuccess;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess) done.insert({kern, dev});
  return e;
}

constexpr int kBlasThreads = 256;
constexpr int kBlasBlocks = 152 * 4;
constexpr int kMaxVec = 65;

int blas_partial_blocks() { return kBlasBlocks; }

// Block partial sums of NV-vectors held per thread (runtime nv <= kMaxVec):
// writes partial[blockIdx.x * nv + i].
template <int NVMAX>
__device__ __forceinline__ void block_partials(double (&acc)[NVMAX], int nv, double* partial) {
  __shared__ double sred[kBlasThreads / 32][kMaxVec];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < NVMAX; ++i) {
    if (i >= nv) break;
    double v = acc[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sred[warp][i] = v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    double s = 0;
    for (int w = 0; w < kBlasThreads / 32; ++w) s += sred[w][i];
    partial[(size_t)blockIdx.x * nv + i] = s;
  }
}

template <int NVMAX>
__global__ void __launch_bounds__(kBlasThreads) dots_kernel(const double* __restrict__ w, const double* __restrict__ V,
                                                            size_t vstride, int nv, size_t n,
                                                            double* __restrict__ partial) {
  double acc[NVMAX];
#pragma unroll
  for (int i = 0; i < NVMAX; ++i) acc[i] = 0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double we = w[e];
#pragma unroll
    for (int i = 0; i < NVMAX; ++i)
      if (i < nv) acc[i] = fma(we, __ldg(&V[i * vstride + e]), acc[i]);
  }
  block_partials(acc, nv, partial);
}

template <int NVMAX>
__global__ void __launch_bounds__(kBlasThreads) update_dots_kernel(double* __restrict__ w, const double* __restrict__ V,
                                                                   size_t vstride, int nv, size_t n,
                                                                   const double* __restrict__ h,
                                                                   double* __restrict__ partial) {
  __shared__ double hs[NVMAX];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = h[i];
  __syncthreads();
  double acc[NVMAX];
#pragma unroll
  for (int i = 0; i < NVMAX; ++i) acc[i] = 0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double vv[NVMAX];
    double we = w[e];
#pragma unroll
    for (int i = 0; i < NVMAX; ++i)
      if (i < nv) { vv[i] = __ldg(&V[i * vstride + e]); we = fma(-hs[i], vv[i], we); }
    w[e] = we;
#pragma unroll
    for (int i = 0; i < NVMAX; ++i)
      if (i < nv) acc[i] = fma(we, vv[i], acc[i]);
  }
  __syncthreads();
  block_partials(acc, nv, partial);
}

template <int NVMAX>
__global__ void __launch_bounds__(kBlasThreads) update_norm_kernel(double* __restrict__ w, const double* __restrict__ V,
                                                                   size_t vstride, int nv, size_t n,
                                                                   const double* __restrict__ h,
                                                                   double* __restrict__ partial) {
  __shared__ double hs[NVMAX];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = h[i];
  __syncthreads();
  double acc[1] = {0};
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double we = w[e];
#pragma unroll
    for (int i = 0; i < NVMAX; ++i)
      if (i < nv) we = fma(-hs[i], __ldg(&V[i * vstride + e]), we);
    w[e] = we;
    acc[0] = fma(we, we, acc[0]);
  }
  __syncthreads();
  block_partials(acc, 1, partial);
}

// ---- float-float basis (mixed precision): arithmetic in ff.cuh -------------------------------

// CGS2 pass 1 on the float-float basis: partial sums of hi(V_i) w in FP32.  Its error (~1e-6 of
// sum |terms|) only leaves components along V_i that the second pass removes.
template <int NVMAX>
__global__ void __launch_bounds__(kBlasThreads) dots_ff_kernel(const double* __restrict__ w,
                                                               const float2* __restrict__ V, size_t vstride, int nv,
                                                               size_t n, double* __restrict__ partial) {
  float acc[NVMAX];
#pragma unroll
  for (int i = 0; i < NVMAX; ++i) acc[i] = 0.0f;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    float vh[NVMAX];  // loads issued before the split's branch
#pragma unroll
    for (int i = 0; i < NVMAX; ++i)
      if (i < nv) vh[i] = __ldg(&V[i * vstride + e]).x;
    const float we = ff_split(w[e]).x;
#pragma unroll
    for (int i = 0; i < NVMAX; ++i)
      if (i < nv) acc[i] = fmaf(we, vh[i], acc[i]);
  }
  double accd[NVMAX];
#pragma unroll
  for (int i = 0; i < NVMAX; ++i) accd[i] = (double)acc[i];
  block_partials(accd, nv, partial);
}

// CGS2 pass 2: wout = w - sum_i h_i V_i in float-float (the FP64 w split once), then partial sums
// of V_i . wout accumulated in float-float (the second-pass coefficients are small corrections of
// large cancelling terms and need the extra precision).
template <int NVMAX>
__global__ void __launch_bounds__(kBlasThreads) update_dots_ff_kernel(const double* __restrict__ w,
                                                                      float2* __restrict__ wout,
                                                                      const float2* __restrict__ V, size_t vstride,
                                                                      int nv, size_t n,
                                                                      const double* __restrict__ h,
                                                                      double* __restrict__ partial) {
  __shared__ float2 hs[NVMAX];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = ff_from_double(h[i]);
  __syncthreads();
  float2 acc[NVMAX];
#pragma unroll
  for (int i = 0; i < NVMAX; ++i) acc[i] = float2{0.0f, 0.0f};
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    float2 vv[NVMAX];  // all loads of the element issued before the split and the dependent update chain
#pragma unroll
    for (int i = 0; i < NVMAX; ++i)
      if (i < nv) vv[i] = __ldg(&V[i * vstride + e]);
    float2 wf = ff_split(w[e]);
#pragma unroll
    for (int i = 0; i < NVMAX; ++i)
      if (i < nv) wf = ff_add(wf, ff_neg(ff_mul(hs[i], vv[i])));
    wout[e] = wf;
#pragma unroll
    for (int i = 0; i < NVMAX; ++i)
      if (i < nv) acc[i] = ff_add(acc[i], ff_mul(wf, vv[i]));
  }
  double accd[NVMAX];
#pragma unroll
  for (int i = 0; i < NVMAX; ++i) accd[i] = ff_to_double(acc[i]);
  __syncthreads();
  block_partials(accd, nv, partial);
}

// CGS2 update of pass 2 in place on the float-float w, and the partial sums of ||w||^2.
template <int NVMAX>
__global__ void __launch_bounds__(kBlasThreads) update_norm_ff_kernel(float2* __restrict__ w,
                                                                      const float2* __restrict__ V, size_t vstride,
                                                                      int nv, size_t n,
                                                                      const double* __restrict__ h,
                                                                      double* __restrict__ partial) {
  __shared__ float2 hs[NVMAX];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = ff_from_double(h[i]);
  __syncthreads();
  float2 acc{0.0f, 0.0f};
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    float2 vv[NVMAX];  // all loads of the element issued before the dependent update chain
#pragma unroll
    for (int i = 0; i < NVMAX; ++i)
      if (i < nv) vv[i] = __ldg(&V[i * vstride + e]);
    float2 wf = w[e];
#pragma unroll
    for (int i = 0; i < NVMAX; ++i)
      if (i < nv) wf = ff_add(wf, ff_neg(ff_mul(hs[i], vv[i])));
    w[e] = wf;
    acc = ff_add(acc, ff_mul(wf, wf));
  }
  double accd[1] = {ff_to_double(acc)};
  __syncthreads();
  block_partials(accd, 1, partial);
}

// U += sum_j y_j Z_j for the FP32 Z of the mixed path, in FP64 (the update must keep FP64 accuracy: an error
// d in U shows in the residual as calA d, and ||c T|| is ~4e4 at M = 8191, so a float-float sum would put
// ~1e-10 into the true residual); Z_j is widened exactly from its bits (f2d_bits), not by the FP64-pipe
// conversion, so the FP64 pipe does one FMA per element and vector.
template <int NZMAX>
__global__ void __launch_bounds__(kBlasThreads) zy_f32_kernel(double* __restrict__ U, const float* __restrict__ Z,
                                                              size_t zstride, int nz, size_t n,
                                                              const double* __restrict__ y) {
  __shared__ double ys[NZMAX];
  for (int i = threadIdx.x; i < nz; i += blockDim.x) ys[i] = y[i];
  __syncthreads();
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    float zz[NZMAX];
#pragma unroll
    for (int j = 0; j < NZMAX; ++j)
      if (j < nz) zz[j] = __ldg(&Z[j * zstride + e]);
    double u = U[e];
#pragma unroll
    for (int j = 0; j < NZMAX; ++j)
      if (j < nz) u = fma(ys[j], f2d_bits(zz[j]), u);
    U[e] = u;
  }
}

// y = a x into the float-float basis from an FP64 vector; a = *a_dev if a_dev, else a.
__global__ void scale_to_ff_kernel(float2* __restrict__ y, const double* __restrict__ x,
                                   const double* __restrict__ a_dev, double a, size_t n) {
  const double s = a_dev ? *a_dev : a;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    y[e] = ff_from_double(s * x[e]);
}

// x *= a in place on a float-float vector; a = *a_dev if a_dev, else a.
__global__ void scale_ff_kernel(float2* __restrict__ x, const double* __restrict__ a_dev, double a, size_t n) {
  const float2 s = ff_from_double(a_dev ? *a_dev : a);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    x[e] = ff_mul(x[e], s);
}

__global__ void reduce_partials_kernel(const double* __restrict__ partial, int nblocks, int nv,
                                       double* __restrict__ out) {
  __shared__ double s[256];
  for (int i = 0; i < nv; ++i) {
    double a = 0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) a += partial[(size_t)b * nv + i];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[i] = s[0];
    __syncthreads();
  }
}

__global__ void scale_kernel(double* __restrict__ out, const double* __restrict__ in, double a, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    out[e] = a * in[e];
}

__global__ void scale_dev_kernel(double* __restrict__ out, const double* __restrict__ in,
                                 const double* __restrict__ a_dev, size_t n) {
  const double a = *a_dev;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    out[e] = a * in[e];
}

template <typename TZ, int NZMAX>
__global__ void __launch_bounds__(kBlasThreads) zy_kernel(double* __restrict__ U, const TZ* __restrict__ Z,
                                                          size_t zstride, int nz, size_t n,
                                                          const double* __restrict__ y) {
  __shared__ double ys[NZMAX];
  for (int i = threadIdx.x; i < nz; i += blockDim.x) ys[i] = y[i];
  __syncthreads();
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double u = U[e];
#pragma unroll 4
    for (int j = 0; j < nz; ++j) u = fma(ys[j], (double)__ldg(&Z[j * zstride + e]), u);
    U[e] = u;
  }
}

__global__ void build_rhs_kernel(const double* __restrict__ u0, const double* __restrict__ f, double* __restrict__ F,
                                 double tau, int M, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double v = tau * f[e];
    if (e < (size_t)M) v += u0[e];
    else if (e < 2 * (size_t)M) v -= 0.5 * u0[e - M];
    F[e] = v;
  }
}

__global__ void f32_to_f64_kernel(const float* __restrict__ in, double* __restrict__ out, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    out[e] = (double)in[e];
}

// out = a x + b y + c z (z unused when null); each element is read before it is written, so out may
// alias any input
__global__ void lincomb3_kernel(double* out, double a, const double* x, double b, const double* y, double c,
                                const double* z, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double v = a * x[e] + b * y[e];
    if (z) v += c * z[e];
    out[e] = v;
  }
}

template <typename TV> __device__ __forceinline__ double ld_any(const TV* p, size_t e);
template <> __device__ __forceinline__ double ld_any<double>(const double* p, size_t e) { return p[e]; }
template <> __device__ __forceinline__ double ld_any<float>(const float* p, size_t e) { return f2d_bits(p[e]); }
template <> __device__ __forceinline__ double ld_any<float2>(const float2* p, size_t e) {
  const float2 v = p[e];
  return f2d_bits(v.x) + f2d_bits(v.y);
}

// w = v + ((C_eps - C) (x) I) z: rows 0 and 1 carry the wrap-around terms of C_eps (Eq. 1.11) and the
// difference 3/2 - 1 of the first diagonal entry; every other row is v.
template <typename TV, typename TZ>
__global__ void poly_rhs_kernel(double* __restrict__ w, const TV* __restrict__ v, const TZ* __restrict__ z,
                                double eps, size_t Ms, int Nt) {
  const size_t n = Ms * (size_t)Nt;
  const size_t r2 = (size_t)(Nt - 2) * Ms, r1 = (size_t)(Nt - 1) * Ms;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double val = ld_any<TV>(v, e);
    if (e < Ms)
      val += 0.5 * ld_any<TZ>(z, e) + 0.5 * eps * ld_any<TZ>(z, r2 + e) - 2.0 * eps * ld_any<TZ>(z, r1 + e);
    else if (e < 2 * Ms)
      val += 0.5 * eps * ld_any<TZ>(z, r1 + (e - Ms));
    w[e] = val;
  }
}

// Dispatch on the number of vectors with a few compile-time caps.
#define AAO_NV_DISPATCH(KERNEL, nv, ...)                                                          \
  do {                                                                                            \
    if (nv <= 4) KERNEL<4><<<kBlasBlocks, kBlasThreads, 0, s>>>(__VA_ARGS__);                     \
    else if (nv <= 8) KERNEL<8><<<kBlasBlocks, kBlasThreads, 0, s>>>(__VA_ARGS__);                \
    else if (nv <= 16) KERNEL<16><<<kBlasBlocks, kBlasThreads, 0, s>>>(__VA_ARGS__);              \
    else if (nv <= 24) KERNEL<24><<<kBlasBlocks, kBlasThreads, 0, s>>>(__VA_ARGS__);              \
    else if (nv <= 32) KERNEL<32><<<kBlasBlocks, kBlasThreads, 0, s>>>(__VA_ARGS__);              \
    else if (nv <= kMaxVec) KERNEL<kMaxVec><<<kBlasBlocks, kBlasThreads, 0, s>>>(__VA_ARGS__);    \
    else return cudaErrorInvalidValue;                                                            \
  } while (0)

cudaError_t launch_dots(const double* w, const double* V, size_t vstride, int nv, size_t n, double* partial,
                        cudaStream_t s) {
  AAO_NV_DISPATCH(dots_kernel, nv, w, V, vstride, nv, n, partial);
  return cudaGetLastError();
}
cudaError_t launch_update_dots(double* w, const double* V, size_t vstride, int nv, size_t n, const double* h,
                               double* partial, cudaStream_t s) {
  AAO_NV_DISPATCH(update_dots_kernel, nv, w, V, vstride, nv, n, h, partial);
  return cudaGetLastError();
}
cudaError_t launch_update_norm(double* w, const double* V, size_t vstride, int nv, size_t n, const double* h,
                               double* partial, cudaStream_t s) {
  AAO_NV_DISPATCH(update_norm_kernel, nv, w, V, vstride, nv, n, h, partial);
  return cudaGetLastError();
}
cudaError_t launch_dots_ff(const double* w, const float2* V, size_t vstride, int nv, size_t n, double* partial,
                           cudaStream_t s) {
  AAO_NV_DISPATCH(dots_ff_kernel, nv, w, V, vstride, nv, n, partial);
  return cudaGetLastError();
}
cudaError_t launch_update_dots_ff(const double* w, float2* wout, const float2* V, size_t vstride, int nv, size_t n,
                                  const double* h, double* partial, cudaStream_t s) {
  AAO_NV_DISPATCH(update_dots_ff_kernel, nv, w, wout, V, vstride, nv, n, h, partial);
  return cudaGetLastError();
}
cudaError_t launch_update_norm_ff(float2* w, const float2* V, size_t vstride, int nv, size_t n, const double* h,
                                  double* partial, cudaStream_t s) {
  AAO_NV_DISPATCH(update_norm_ff_kernel, nv, w, V, vstride, nv, n, h, partial);
  return cudaGetLastError();
}
cudaError_t launch_scale_to_ff(float2* y, const double* x, const double* a_dev, double a, size_t n, cudaStream_t s) {
  scale_to_ff_kernel<<<kBlasBlocks, kBlasThreads, 0, s>>>(y, x, a_dev, a, n);
  return cudaGetLastError();
}
cudaError_t launch_scale_ff(float2* x, const double* a_dev, double a, size_t n, cudaStream_t s) {
  scale_ff_kernel<<<kBlasBlocks, kBlasThreads, 0, s>>>(x, a_dev, a, n);
  return cudaGetLastError();
}
cudaError_t launch_reduce_partials(const double* partial, int nblocks, int nv, double* out, cudaStream_t s) {
  reduce_partials_kernel<<<1, 256, 0, s>>>(partial, nblocks, nv, out);
  return cudaGetLastError();
}
cudaError_t launch_scale(double* out, const double* in, double a, size_t n, cudaStream_t s) {
  scale_kernel<<<kBlasBlocks, kBlasThreads, 0, s>>>(out, in, a, n);
  return cudaGetLastError();
}
cudaError_t launch_scale_dev(double* out, const double* in, const double* a_dev, size_t n, cudaStream_t s) {
  scale_dev_kernel<<<kBlasBlocks, kBlasThreads, 0, s>>>(out, in, a_dev, n);
  return cudaGetLastError();
}
cudaError_t launch_zy_update_f32(double* U, const float* Z, size_t zstride, int nz, size_t n, const double* y,
                                 cudaStream_t s) {
  AAO_NV_DISPATCH(zy_f32_kernel, nz, U, Z, zstride, nz, n, y);
  return cudaGetLastError();
}
cudaError_t launch_zy_update_f64(double* U, const double* Z, size_t zstride, int nz, size_t n, const double* y,
                                 cudaStream_t s) {
  if (nz > kMaxVec) return cudaErrorInvalidValue;
  zy_kernel<double, kMaxVec><<<kBlasBlocks, kBlasThreads, 0, s>>>(U, Z, zstride, nz, n, y);
  return cudaGetLastError();
}
cudaError_t launch_build_rhs(const double* u0, const double* f, double* F, double tau, int M, int Nt,
                             cudaStream_t s) {
  build_rhs_kernel<<<kBlasBlocks, kBlasThreads, 0, s>>>(u0, f, F, tau, M, (size_t)M * Nt);
  return cudaGetLastError();
}
cudaError_t launch_lincomb3(double* out, double a, const double* x, double b, const double* y, double c,
                            const double* z, size_t n, cudaStream_t s) {
  lincomb3_kernel<<<kBlasBlocks, kBlasThreads, 0, s>>>(out, a, x, b, y, c, z, n);
  return cudaGetLastError();
}
cudaError_t launch_poly_rhs(double* w, const void* v, bool v_ff, const void* z, bool z_f32, double eps, size_t Ms,
                            int Nt, cudaStream_t s) {
  if (v_ff && z_f32)
    poly_rhs_kernel<float2, float><<<kBlasBlocks, kBlasThreads, 0, s>>>(w, (const float2*)v, (const float*)z, eps,
                                                                         Ms, Nt);
  else if (v_ff)
    poly_rhs_kernel<float2, double><<<kBlasBlocks, kBlasThreads, 0, s>>>(w, (const float2*)v, (const double*)z, eps,
                                                                          Ms, Nt);
  else if (z_f32)
    poly_rhs_kernel<double, float><<<kBlasBlocks, kBlasThreads, 0, s>>>(w, (const double*)v, (const float*)z, eps,
                                                                         Ms, Nt);
  else
    poly_rhs_kernel<double, double><<<kBlasBlocks, kBlasThreads, 0, s>>>(w, (const double*)v, (const double*)z, eps,
                                                                          Ms, Nt);
  return cudaGetLastError();
}
cudaError_t launch_f32_to_f64(const float* in, double* out, size_t n, cudaStream_t s) {
  f32_to_f64_kernel<<<kBlasBlocks, kBlasThreads, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

}  // namespace aao
