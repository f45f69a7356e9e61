// Step (b) of the block-circulant preconditioner (Sec. 3.1): for every
// frequency n = 0 .. Nt/2 solve the complex-shifted Toeplitz system
//     (lambda_n I - tau K) x = zhat_n,    -tau K = c T,
// by preconditioned COCG (conjugate-orthogonal CG: CG with the bilinear form
// u^T w, which is the right Krylov method for a complex SYMMETRIC matrix).
//
// One CTA solves one system with all iterations inside the kernel.  Products
// with T use the length-L circulant embedding (FFT in shared memory); the
// preconditioner is either
//   * the Strang circulant S of T: (lambda I + c S)^{-1} r = IDFT_M(DFT_M(r)
//     / (lambda + c s_hat)), each length-M DFT done by Bluestein's chirp-z
//     convolution with length-L FFTs; or
//   * the natural tau matrix tau(T) = T - H(T) (the tau-algebra approximation
//     of Sec. 3.2): (lambda I + c tau(T))^{-1} r = (2/(M+1)) S D S r with the
//     DST-I matrix S, each DST done as an FFT of length L = 2(M+1) of the odd
//     extension.
// Vectors r and p live in global memory (L2-resident per-system workspace);
// x accumulates in the output buffer.
#include "cocg_reg.cuh"

namespace aao {

template <typename R> struct Tabs;
template <> struct Tabs<float> { using type = CocgTables32; };
template <> struct Tabs<double> { using type = CocgTables64; };

// buf <- FFT-domain product: forward FFT, multiply by kernel, backward FFT.
// The multiply is a functor of the bit-reversed position p.
template <typename C, typename F>
__device__ __forceinline__ void convolve(C* buf, int logL, const C* q, F factor) {
  fft_convolve(buf, logL, q, logL, factor);
}

// z = P^{-1} r, written to buf[pad16(i)], i < M (natural order).
template <typename R, int KIND>
__device__ __forceinline__ void precond(typename cplx_t<R>::type* buf, const typename cplx_t<R>::type* r, int M,
                                        int logL, typename cplx_t<R>::type lam, const typename Tabs<R>::type& tb,
                                        const typename cplx_t<R>::type* q) {
  using C = typename cplx_t<R>::type;
  const int L = 1 << logL;
  if (KIND == 0) {
    // a_j = r_j w_j, zero-padded; c = a * conj-chirp filter; X_k = w_k c_k;
    // then a'_k = X_k conj(w_k) / (M (lambda + s_k)) = c_k / (M (lambda + s_k)); z_j = conj(w_j) (a' * chirp filter)_j
    for (int j = threadIdx.x; j < L; j += blockDim.x)
      buf[pad16(j)] = (j < M) ? cmul(r[j], __ldg(&tb.chirp[j])) : C{0, 0};
    convolve(buf, logL, q, [&](int p) { return __ldg(&tb.chat_br[p]); });
    const R invM = (R)1 / (R)M;
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
      if (k < M) {
        C d = lam;
        d.x += __ldg(&tb.seig[k]);
        buf[pad16(k)] = cscale(cdiv(buf[pad16(k)], d), invM);
      } else {
        buf[pad16(k)] = C{0, 0};
      }
    }
    convolve(buf, logL, q, [&](int p) { return cconj(__ldg(&tb.chat_br[p])); });
    for (int j = threadIdx.x; j < M; j += blockDim.x) buf[pad16(j)] = cmulc(buf[pad16(j)], __ldg(&tb.chirp[j]));
    __syncthreads();
  } else {
    // odd extension y (length L = 2(M+1)), DIF, multiply by 1/(L (lambda + c sigma_f)), DIT; z_{l-1} = buf[l]
    const int Mp1 = M + 1;
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
      C y{0, 0};
      if (l >= 1 && l <= M) y = r[l - 1];
      else if (l > Mp1) { const C t = r[L - l - 1]; y = C{-t.x, -t.y}; }
      buf[pad16(l)] = y;
    }
    const R invL = (R)1 / (R)L;
    convolve(buf, logL, q, [&](int p) {
      C d = lam;
      d.x += __ldg(&tb.taueig_br[p]);
      return cdiv(C{invL, 0}, d);
    });
    (void)Mp1;
    // z_i = buf[pad16(i + 1)], see z_at
  }
}

template <typename R, int KIND>
__device__ __forceinline__ typename cplx_t<R>::type z_at(const typename cplx_t<R>::type* buf, int i) {
  return KIND == 0 ? buf[pad16(i)] : buf[pad16(i + 1)];
}

template <typename R, int KIND, bool GBUF>
__global__ void __launch_bounds__(512) cocg_kernel(typename cplx_t<R>::type* __restrict__ xb,
                                                   typename cplx_t<R>::type* __restrict__ rws,
                                                   typename cplx_t<R>::type* __restrict__ pws,
                                                   typename cplx_t<R>::type* __restrict__ gbuf, int M, int logL,
                                                   int nsys, typename Tabs<R>::type tb, R tol, int maxit,
                                                   int* __restrict__ iters, int* __restrict__ flags) {
  using C = typename cplx_t<R>::type;
  extern __shared__ unsigned char smraw[];
  __shared__ R red[4 * 32];
  C* buf = GBUF ? gbuf + (size_t)blockIdx.x * padded_size(1 << logL) : reinterpret_cast<C*>(smraw);
  C* q = GBUF ? reinterpret_cast<C*>(smraw) : reinterpret_cast<C*>(smraw) + padded_size(1 << logL);
  const int L = 1 << logL;
  load_quarter(q, tb.twL, L / 4);
  for (int n = blockIdx.x; n < nsys; n += gridDim.x) {
    const double2 lamd = tb.lambda[n];
    const C lam = C{(R)lamd.x, (R)lamd.y};
    C* x = xb + (size_t)n * M;
    C* r = rws + (size_t)n * M;
    C* p = pws + (size_t)n * M;
    R nb2[1] = {0};
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
      const C b = x[i];
      r[i] = b;
      x[i] = C{0, 0};
      nb2[0] += b.x * b.x + b.y * b.y;
    }
    block_sum<R, 1>(nb2, red);
    if (nb2[0] == (R)0) {
      if (threadIdx.x == 0) { iters[n] = 0; flags[n] = 0; }
      continue;
    }
    const R thr = tol * tol * nb2[0];
    precond<R, KIND>(buf, r, M, logL, lam, tb, q);
    R rho2[3] = {0, 0, 0};  // r^T z, |z|^2
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
      const C z = z_at<R, KIND>(buf, i);
      const C ri = r[i];
      rho2[0] += ri.x * z.x - ri.y * z.y;
      rho2[1] += ri.x * z.y + ri.y * z.x;
      rho2[2] += z.x * z.x + z.y * z.y;
      p[i] = z;
    }
    block_sum<R, 3>(rho2, red);
    C rho{rho2[0], rho2[1]};
    int it = 0, flag = 1;
    const bool bd0 = near_breakdown(rho2[0], rho2[1], rho2[2], nb2[0]);  // z^T r of the first step
    if (bd0) flag = 2;
    while (!bd0 && it < maxit) {
      // q = (lambda I + c T) p
      for (int j = threadIdx.x; j < L; j += blockDim.x) buf[pad16(j)] = (j < M) ? p[j] : C{0, 0};
      convolve(buf, logL, q, [&](int q) { return C{__ldg(&tb.Ebr[q]), (R)0}; });
      R pq2[4] = {0, 0, 0, 0};  // p^T q, |p|^2, |q|^2
      for (int i = threadIdx.x; i < M; i += blockDim.x) {
        const C pi = p[i];
        const C q = cadd(buf[pad16(i)], cmul(lam, pi));
        buf[pad16(i)] = q;
        pq2[0] += pi.x * q.x - pi.y * q.y;
        pq2[1] += pi.x * q.y + pi.y * q.x;
        pq2[2] += pi.x * pi.x + pi.y * pi.y;
        pq2[3] += q.x * q.x + q.y * q.y;
      }
      block_sum<R, 4>(pq2, red);
      const C pq{pq2[0], pq2[1]};
      if (near_breakdown(pq2[0], pq2[1], pq2[2], pq2[3])) { flag = 2; break; }
      const C a = cdiv(rho, pq);
      R rr[1] = {0};
      for (int i = threadIdx.x; i < M; i += blockDim.x) {
        const C pi = p[i];
        const C q = buf[pad16(i)];
        C xi = x[i];
        xi = cadd(xi, cmul(a, pi));
        x[i] = xi;
        C ri = r[i];
        ri = csub(ri, cmul(a, q));
        r[i] = ri;
        rr[0] += ri.x * ri.x + ri.y * ri.y;
      }
      block_sum<R, 1>(rr, red);
      ++it;
      if (!(rr[0] == rr[0]) || rr[0] > (R)1e30 * nb2[0]) { flag = 3; break; }
      if (rr[0] <= thr) { flag = 0; break; }
      precond<R, KIND>(buf, r, M, logL, lam, tb, q);
      R rn2[3] = {0, 0, 0};  // r^T z, |z|^2
      for (int i = threadIdx.x; i < M; i += blockDim.x) {
        const C z = z_at<R, KIND>(buf, i);
        const C ri = r[i];
        rn2[0] += ri.x * z.x - ri.y * z.y;
        rn2[1] += ri.x * z.y + ri.y * z.x;
        rn2[2] += z.x * z.x + z.y * z.y;
      }
      block_sum<R, 3>(rn2, red);
      const C rho_new{rn2[0], rn2[1]};
      if (near_breakdown(rn2[0], rn2[1], rn2[2], rr[0])) { flag = 2; break; }
      const C beta = cdiv(rho_new, rho);
      rho = rho_new;
      for (int i = threadIdx.x; i < M; i += blockDim.x) p[i] = cadd(z_at<R, KIND>(buf, i), cmul(beta, p[i]));
      __syncthreads();
    }
    if (threadIdx.x == 0) { iters[n] = it; flags[n] = flag; }
    __syncthreads();
  }
  (void)L;
}


// The paper's own Step (b) (Sec. 3.2, Eq. 3.9; Example 2, Eq. 4.5): every shifted system solved
// directly with the tau-matrix approximation, x_n = (lambda_n I + c tau(T))^{-1} zhat_n, by one DST-I
// pair (the odd extension of length L = 2(M+1), one FFT convolution).  One CTA per system; no
// inner iterations (iters[n] = 0, flags[n] = 0).
template <typename R, bool GBUF>
__global__ void __launch_bounds__(512) tau_direct_kernel(typename cplx_t<R>::type* __restrict__ xb,
                                                         typename cplx_t<R>::type* __restrict__ gbuf, int M,
                                                         int logL, int nsys, typename Tabs<R>::type tb,
                                                         int* __restrict__ iters, int* __restrict__ flags) {
  using C = typename cplx_t<R>::type;
  extern __shared__ unsigned char smraw[];
  C* buf = GBUF ? gbuf + (size_t)blockIdx.x * padded_size(1 << logL) : reinterpret_cast<C*>(smraw);
  C* q = GBUF ? reinterpret_cast<C*>(smraw) : reinterpret_cast<C*>(smraw) + padded_size(1 << logL);
  const int L = 1 << logL;
  load_quarter(q, tb.twL, L / 4);
  for (int n = blockIdx.x; n < nsys; n += gridDim.x) {
    const double2 lamd = tb.lambda[n];
    const C lam = C{(R)lamd.x, (R)lamd.y};
    C* x = xb + (size_t)n * M;
    __syncthreads();  // the previous system's readers of buf are done
    precond<R, 1>(buf, x, M, logL, lam, tb, q);  // ends synchronised
    for (int i = threadIdx.x; i < M; i += blockDim.x) x[i] = z_at<R, 1>(buf, i);
    if (threadIdx.x == 0) { iters[n] = 0; flags[n] = 0; }
  }
}

static const size_t kSmemLimit = 200 * 1024;

size_t cocg_gbuf_elems_f64(int logL, int grid) {
  if (cocg_smem<double>(logL) <= kSmemLimit) return 0;
  return (size_t)padded_size(1 << logL) * (size_t)grid;
}

template <typename R, int KIND, bool GBUF>
static cudaError_t launch_k(typename cplx_t<R>::type* xb, typename cplx_t<R>::type* rws,
                            typename cplx_t<R>::type* pws, typename cplx_t<R>::type* gbuf, int M, int logL,
                            int nsys, const typename Tabs<R>::type& tb, R tol, int maxit, int* iters, int* flags,
                            int grid, cudaStream_t s) {
  const size_t smem = (GBUF ? 0 : cocg_smem<R>(logL)) + cocg_table_bytes<R>(logL);
  cudaError_t e = allow_max_dynamic_smem(cocg_kernel<R, KIND, GBUF>);
  if (e != cudaSuccess) return e;
  cocg_kernel<R, KIND, GBUF><<<grid, 512, smem, s>>>(xb, rws, pws, gbuf, M, logL, nsys, tb, tol, maxit, iters,
                                                     flags);
  return cudaGetLastError();
}

// Per-system spectra of the Strang inverse as an L-point circulant (see launch_strang_conv_setup).
__global__ void __launch_bounds__(kRegMaxThreads, 1)
    strang_conv_kernel(int M, int logL, int nsys, CocgTables32 tb, float2* __restrict__ out) {
  constexpr int NT = kRegMaxThreads;
  extern __shared__ unsigned char smraw[];
  float2* buf = reinterpret_cast<float2*>(smraw);
  float2* q = buf + padded_size(1 << logL);
  float2* pt = q + (1 << logL) / 4;
  const int L = 1 << logL;
  const int t = threadIdx.x;
  load_quarter(q, tb.twL, L / 4);
  __syncthreads();
  build_pass_tables(pt, q, logL, logL);
  const float invL = 1.0f / (float)L;
  for (int n = blockIdx.x; n < nsys; n += gridDim.x) {
    const double2 lamd = tb.lambda[n];
    const float2 lam{(float)lamd.x, (float)lamd.y};
    float2 r[kRegElems];
#pragma unroll
    for (int j = 0; j < kRegElems; ++j) r[j] = (t == 0 && j == 0) ? float2{1, 0} : float2{0, 0};
    precond_reg<0, NT>(buf, r, M, logL, lam, tb, q, pt, nullptr);  // h = (lambda I + c S)^{-1} e_0
    float2 h[kRegElems];
#pragma unroll
    for (int j = 0; j < kRegElems; ++j) {
      const int i = t + NT * j;
      h[j] = i < M ? zval<0>(buf, tb, i) : float2{0, 0};
    }
    __syncthreads();
    for (int i = t; i < L; i += NT) buf[pad16(i)] = float2{0, 0};
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kRegElems; ++j) {
      const int i = t + NT * j;
      if (i < M) {
        buf[pad16(i)] = h[j];                          // g_i = h_i
        if (i >= 1) buf[pad16(L - M + i)] = h[j];      // g_{L-d} = h_{M-d}, d = M - i
      }
    }
    fft_forward_fused(buf, logL, q, logL, pt);
    float2* o = out + ((size_t)n << logL);
    for (int p = t; p < L; p += NT) o[p] = cscale(buf[pad16(p)], invL);
    __syncthreads();
  }
}

cudaError_t launch_strang_conv_setup(int M, int logL, int nsys, const CocgTables32& tb, float2* out,
                                     cudaStream_t s) {
  if (M > kRegMaxThreads * kRegElems) return cudaErrorInvalidValue;
  const size_t smem = cocg_reg_smem(logL);
  cudaError_t e = allow_max_dynamic_smem(strang_conv_kernel);
  if (e != cudaSuccess) return e;
  strang_conv_kernel<<<nsys, kRegMaxThreads, smem, s>>>(M, logL, nsys, tb, out);
  return cudaGetLastError();
}

// Deterministic test right-hand sides in [-1, 1)^2 for the autotuner (a 32-bit integer hash).
__global__ void fill_test_rhs_kernel(float2* __restrict__ x, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    unsigned h = (unsigned)i * 2654435761u;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    const float a = (float)(h & 0xffffu) / 32768.0f - 1.0f, b = (float)(h >> 16) / 32768.0f - 1.0f;
    x[i] = float2{a, b};
  }
}

cudaError_t launch_fill_test_rhs(float2* x, size_t n, cudaStream_t s) {
  fill_test_rhs_kernel<<<152 * 4, 256, 0, s>>>(x, n);
  return cudaGetLastError();
}

int cocg_reg_min_threads(int M) {
  int nt = 64;
  while (nt * kRegElems < M) nt *= 2;
  return nt <= kRegMaxThreads ? nt : 0;
}

cudaError_t launch_cocg_f32(float2* xb, float2* rws, float2* pws, int M, int logL, int nsys, int inner,
                            const CocgTables32& tb, float tol, int maxit, int* iters, int* flags, int grid,
                            cudaStream_t s, const float2* x0, int threads) {
  const int nt_min = cocg_reg_min_threads(M);
  if (nt_min) {
    const int nt = threads ? threads : kRegMaxThreads;
    if (nt < nt_min || nt > kRegMaxThreads) return cudaErrorInvalidValue;
    if (inner == 1) return launch_cocg_reg_tau(xb, x0, M, logL, nsys, tb, tol, maxit, iters, flags, grid, nt, s);
    if (tb.sconv) return launch_cocg_reg_sconv(xb, x0, M, logL, nsys, tb, tol, maxit, iters, flags, grid, nt, s);
    // Strang by Bluestein (no precomputed spectra: calls without a plan): 512 threads, no initial guess
    if (nt != kRegMaxThreads || x0) return cudaErrorInvalidValue;
    return launch_reg_one<0, false, kRegMaxThreads>(xb, nullptr, M, logL, nsys, tb, tol, maxit, iters, flags, grid,
                                                    s);
  }
  if (x0) return cudaErrorInvalidValue;
  if (inner == 0)
    return launch_k<float, 0, false>(xb, rws, pws, nullptr, M, logL, nsys, tb, tol, maxit, iters, flags, grid, s);
  return launch_k<float, 1, false>(xb, rws, pws, nullptr, M, logL, nsys, tb, tol, maxit, iters, flags, grid, s);
}

cudaError_t launch_tau_direct_f32(float2* xb, int M, int logL, int nsys, const CocgTables32& tb, int* iters,
                                  int* flags, cudaStream_t s) {
  const size_t smem = cocg_smem<float>(logL) + cocg_table_bytes<float>(logL);
  cudaError_t e = allow_max_dynamic_smem(tau_direct_kernel<float, false>);
  if (e != cudaSuccess) return e;
  tau_direct_kernel<float, false><<<nsys, 512, smem, s>>>(xb, nullptr, M, logL, nsys, tb, iters, flags);
  return cudaGetLastError();
}

cudaError_t launch_tau_direct_f64(double2* xb, double2* gbuf, int M, int logL, int nsys, const CocgTables64& tb,
                                  int* iters, int* flags, int grid, cudaStream_t s) {
  const bool g = cocg_smem<double>(logL) > kSmemLimit;
  if (g && !gbuf) return cudaErrorInvalidValue;
  const size_t smem = (g ? 0 : cocg_smem<double>(logL)) + cocg_table_bytes<double>(logL);
  if (g) {
    cudaError_t e = allow_max_dynamic_smem(tau_direct_kernel<double, true>);
    if (e != cudaSuccess) return e;
    tau_direct_kernel<double, true><<<grid, 512, smem, s>>>(xb, gbuf, M, logL, nsys, tb, iters, flags);
  } else {
    cudaError_t e = allow_max_dynamic_smem(tau_direct_kernel<double, false>);
    if (e != cudaSuccess) return e;
    tau_direct_kernel<double, false><<<nsys, 512, smem, s>>>(xb, nullptr, M, logL, nsys, tb, iters, flags);
  }
  return cudaGetLastError();
}

cudaError_t launch_cocg_f64(double2* xb, double2* rws, double2* pws, double2* gbuf, int M, int logL, int nsys,
                            int inner, const CocgTables64& tb, double tol, int maxit, int* iters, int* flags,
                            int grid, cudaStream_t s) {
  const bool g = cocg_smem<double>(logL) > kSmemLimit;
  if (inner == 0) {
    if (g) return launch_k<double, 0, true>(xb, rws, pws, gbuf, M, logL, nsys, tb, tol, maxit, iters, flags, grid, s);
    return launch_k<double, 0, false>(xb, rws, pws, gbuf, M, logL, nsys, tb, tol, maxit, iters, flags, grid, s);
  }
  if (g) return launch_k<double, 1, true>(xb, rws, pws, gbuf, M, logL, nsys, tb, tol, maxit, iters, flags, grid, s);
  return launch_k<double, 1, false>(xb, rws, pws, gbuf, M, logL, nsys, tb, tol, maxit, iters, flags, grid, s);
}

}  // namespace aao
