// Float-float arithmetic for the mixed-precision Arnoldi basis and the dot products fused into the
// matvec epilogue (shared by blas.cu and ntt.cu).
#pragma once
#include "common.cuh"

namespace aao {

// In the mixed path the Arnoldi basis v_0..v_m is stored as float-float pairs (hi, lo), hi + lo
// with |lo| <= ulp(hi) / 2 (about 48 significant bits), in the same 8 bytes per element as an FP64
// vector.  Error-free transformations (Dekker 1971; Knuth, TAOCP vol. 2, 4.2.2): two_sum and
// quick_two_sum for sums, fma for the exact product error.  This moves CGS2 from the FP64 pipe
// (1.6 FMA per clock per SM on this GPU) to the FP32 pipe; the basis and the Hessenberg
// coefficients keep ~1e-14 relative accuracy, far below the 1e-10 target of FGMRES.
__device__ __forceinline__ float2 ff_two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return float2{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ float2 ff_quick_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return float2{s, b - (s - a)};
}
__device__ __forceinline__ float2 ff_from_double(double x) {
  const float h = __double2float_rn(x);
  return float2{h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double ff_to_double(float2 x) { return (double)x.x + (double)x.y; }

// The conversions of ff_from_double out of line: a call is never evaluated speculatively, so the rare branch of
// ff_split costs the common one nothing on the FP64 pipe.
static __device__ __noinline__ float2 ff_from_double_call(double x) { return ff_from_double(x); }

// The same split with integer operations only (FP64<->FP32 conversions issue on the FP64 pipe, under 1 per
// clock per SM on this GPU): for 2^-74 <= |x| < 2^127, hi = x truncated to its 24 leading significant bits
// (exact in FP32) and lo = the remaining 29 bits correctly rounded to FP32 (|lo| < ulp(hi)), so
// |hi + lo - x| <= 2^-48 |x|.  Other x (zero, tiny, huge, non-finite) take the conversions, out of line.
__device__ __forceinline__ float2 ff_split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int hw = (unsigned int)(b >> 32), lw = (unsigned int)b;
  const int e = (int)((hw >> 20) & 0x7ffu);  // biased exponent of x
  if (e < 949 || e > 1150) return ff_from_double_call(x);
  const unsigned int sign = hw & 0x80000000u;
  const float hi = __uint_as_float(sign | ((unsigned int)(e - 896) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
  const unsigned int r = lw & 0x1fffffffu;  // lo = r 2^(e - 1075), r < 2^29
  // (float) r correctly rounded: r = a 2^15 + c with a, c < 2^15 converted exactly through the 2^23 bias
  const float fa = __uint_as_float(0x4b000000u | (r >> 15)) - 8388608.0f;
  const float fc = __uint_as_float(0x4b000000u | (r & 0x7fffu)) - 8388608.0f;
  const float lo = fmaf(fa, 32768.0f, fc) * __uint_as_float((unsigned int)(e - 948) << 23);
  return float2{hi, __uint_as_float(__float_as_uint(lo) ^ sign)};
}
__device__ __forceinline__ float2 ff_mul(float2 x, float2 y) {
  const float p = x.x * y.x;
  const float e = fmaf(x.x, y.y, fmaf(x.y, y.x, fmaf(x.x, y.x, -p)));
  return ff_quick_sum(p, e);
}
// x + y with error ~2^-46 (|x| + |y|)
__device__ __forceinline__ float2 ff_add(float2 x, float2 y) {
  float2 s = ff_two_sum(x.x, y.x);
  s.y += x.y + y.y;
  return ff_quick_sum(s.x, s.y);
}
__device__ __forceinline__ float2 ff_neg(float2 x) { return float2{-x.x, -x.y}; }


// Block partial sums of NVMAX per-thread accumulators (runtime nv <= NVMAX, NVMAX <= 65, a block of NTHREADS
// threads): writes out[i], i < nv, in a fixed order (deterministic).
template <int NVMAX, int NTHREADS>
__device__ __forceinline__ void block_partials_to(double (&acc)[NVMAX], int nv, double* out) {
  __shared__ double sred[NTHREADS / 32][NVMAX];
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
    double t = 0;
    for (int w = 0; w < NTHREADS / 32; ++w) t += sred[w][i];
    out[i] = t;
  }
}

}  // namespace aao
