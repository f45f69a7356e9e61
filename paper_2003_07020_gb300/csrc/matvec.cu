// All-at-once matvec, Sec. 3.2: calA v = vec(V C^T) - tau vec(K V), in FP64.
//
// One CTA per time row k.  The product c T v_k (c = tau kappa / h^alpha, so
// that -tau K = c T) is a linear convolution of the real row with the even
// FCD stencil, done by circulant embedding of length L = 2N: the real
// zero-padded row is packed as N complex points z_j = x_{2j} + i x_{2j+1},
// transformed with an N-point complex FFT in shared memory, split into the
// real-signal spectrum, multiplied by the (real, even) embedding spectrum,
// re-packed and transformed back.  The BDF band of C (Eq. 1.7) is added in
// the epilogue.
#include "common.cuh"
#include "kernels.h"

namespace aao {

template <typename TIn>
__device__ __forceinline__ double ld(const TIn* p) { return (double)__ldg(p); }

// In-place real-signal spectrum multiply on the bit-reversed N-point FFT of
// the packed signal: Z -> Z' such that backward(Z') packs c T x (see the
// derivation in the file comment).  Ehalf[m] = c * Ehat_m / N, m = 0..N.
__device__ __forceinline__ void r2c_mult_c2r(double2* sm, int logN, const double* __restrict__ Ehalf,
                                             const double2* q) {
  const int N = 1 << logN;
  for (int k = threadIdx.x; k <= N / 2; k += blockDim.x) {
    if (k == 0) {
      const int p0 = pad16(0);
      const double2 Z0 = sm[p0];
      const double Y0 = __ldg(&Ehalf[0]) * (Z0.x + Z0.y);
      const double YN = __ldg(&Ehalf[N]) * (Z0.x - Z0.y);
      sm[p0] = double2{0.5 * (Y0 + YN), 0.5 * (Y0 - YN)};
      continue;
    }
    const int kp = N - k;
    const int pk = pad16(bitrev(k, logN)), pkp = pad16(bitrev(kp, logN));
    const double2 Zk = sm[pk], Zkp = sm[pkp];
    // E_k = (Z_k + conj Z_{N-k})/2, O_k = -i (Z_k - conj Z_{N-k})/2
    const double2 Ek = double2{0.5 * (Zk.x + Zkp.x), 0.5 * (Zk.y - Zkp.y)};
    const double2 Ok = double2{0.5 * (Zk.y + Zkp.y), -0.5 * (Zk.x - Zkp.x)};
    const double ek = __ldg(&Ehalf[k]), ekp = __ldg(&Ehalf[kp]);
    {
      const double2 W = twiddle<-1>(q, k, logN + 1);
      const double2 WO = cmul(W, Ok);
      const double2 Y = cscale(cadd(Ek, WO), ek);    // Y_k
      const double2 YN = cscale(csub(Ek, WO), ekp);  // Y_{k+N}
      const double2 S = cadd(Y, YN), D = csub(Y, YN);
      const double2 iWcD = double2{-(W.x * D.y - W.y * D.x), W.x * D.x + W.y * D.y};  // i conj(W) D
      sm[pk] = double2{0.5 * (S.x + iWcD.x), 0.5 * (S.y + iWcD.y)};
    }
    if (kp != k) {
      const double2 Ekp = cconj(Ek), Okp = cconj(Ok);
      const double2 W = twiddle<-1>(q, kp, logN + 1);
      const double2 WO = cmul(W, Okp);
      const double2 Y = cscale(cadd(Ekp, WO), ekp);
      const double2 YN = cscale(csub(Ekp, WO), ek);
      const double2 S = cadd(Y, YN), D = csub(Y, YN);
      const double2 iWcD = double2{-(W.x * D.y - W.y * D.x), W.x * D.x + W.y * D.y};
      sm[pkp] = double2{0.5 * (S.x + iWcD.x), 0.5 * (S.y + iWcD.y)};
    }
  }
}

template <typename TIn>
__global__ void __launch_bounds__(256) matvec_f64_kernel(const TIn* __restrict__ v, const double* __restrict__ rhs,
                                                         double* __restrict__ w, double* __restrict__ sq_partial,
                                                         int M, int logN, const double* __restrict__ Ehalf,
                                                         const double2* __restrict__ twL) {
  extern __shared__ double2 sm[];
  __shared__ double red[32];
  const int N = 1 << logN;
  const int k = blockIdx.x;
  double2* q = sm + padded_size(N);  // quarter twiddle table of the length-2N embedding
  load_quarter(q, twL, N / 2);
  const TIn* vk = v + (size_t)k * M;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const int i0 = 2 * j;
    const double x0 = (i0 < M) ? ld(vk + i0) : 0.0;
    const double x1 = (i0 + 1 < M) ? ld(vk + i0 + 1) : 0.0;
    sm[pad16(j)] = double2{x0, x1};
  }
  fft_forward(sm, logN, 1, 0, q, logN + 1);
  r2c_mult_c2r(sm, logN, Ehalf, q);
  fft_backward(sm, logN, 1, 0, q, logN + 1);
  const TIn* vk1 = vk - M;
  const TIn* vk2 = vk - 2 * M;
  double* wk = w + (size_t)k * M;
  const double* rk = rhs ? rhs + (size_t)k * M : nullptr;
  double sq = 0.0;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    const double2 t = sm[pad16(i >> 1)];
    const double y = (i & 1) ? t.y : t.x;
    double band;
    if (k == 0) band = ld(vk + i);
    else if (k == 1) band = 1.5 * ld(vk + i) - 2.0 * ld(vk1 + i);
    else band = 1.5 * ld(vk + i) - 2.0 * ld(vk1 + i) + 0.5 * ld(vk2 + i);
    double out = band + y;
    if (rk) out = rk[i] - out;
    wk[i] = out;
    sq += out * out;
  }
  if (sq_partial) {
    double a[1] = {sq};
    block_sum<double, 1>(a, red);
    if (threadIdx.x == 0) sq_partial[k] = a[0];
  }
}

size_t matvec_smem_bytes(int logL) {
  return ((size_t)padded_size(1 << (logL - 1)) + (size_t)(1 << (logL - 2))) * sizeof(double2);
}

template <typename TIn>
static cudaError_t launch_mv(const TIn* v, const double* rhs, double* w, double* sq_partial, int M, int Nt,
                             int logL, const double* Ehalf, const double2* twL, cudaStream_t s) {
  const size_t smem = matvec_smem_bytes(logL);
  cudaError_t e = allow_max_dynamic_smem(matvec_f64_kernel<TIn>);
  if (e != cudaSuccess) return e;
  matvec_f64_kernel<TIn><<<Nt, 256, smem, s>>>(v, rhs, w, sq_partial, M, logL - 1, Ehalf, twL);
  return cudaGetLastError();
}

cudaError_t launch_matvec_f64(const double* v, const double* rhs, double* w, double* sq_partial, int M, int Nt,
                              int logL, const double* Ehalf, const double2* twL, cudaStream_t s) {
  return launch_mv<double>(v, rhs, w, sq_partial, M, Nt, logL, Ehalf, twL, s);
}
cudaError_t launch_matvec_f64_fin(const float* v, const double* rhs, double* w, double* sq_partial, int M,
                                  int Nt, int logL, const double* Ehalf, const double2* twL, cudaStream_t s) {
  return launch_mv<float>(v, rhs, w, sq_partial, M, Nt, logL, Ehalf, twL, s);
}

}  // namespace aao
