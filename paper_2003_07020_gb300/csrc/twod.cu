// The 2D all-at-once system: K = I (x) K_x + K_y (x) I (x fastest), the
// Kronecker-sum Jacobian of Eq. 4.2, on (0,1)^2 with M_x x M_y interior
// points.  A time level is a "slab" [My][Mx]; a system of Step (b) is a
// complex slab.  Operators are separable, so every kernel here works on
// batches of lines: rows (x direction, contiguous) or columns (y direction,
// stride Mx, loaded as tiles of consecutive columns so that global accesses
// stay coalesced), each line transformed with the shared-memory FFT engine.
//
//  * matvec (FP64): c_x T_x along rows and c_y T_y along columns by
//    circulant-embedding convolutions; two real lines share one complex
//    transform (the embedding spectrum is real and even); the BDF band of
//    Eq. 1.7 is added in the column pass.
//  * Step (b): preconditioned COCG on all systems at once, with either the 2D
//    Strang (BCCB) circulant I (x) c_x S_x + c_y S_y (x) I (precomputed 2D
//    spectra, FFTs of the embedding) or the 2D tau
//    matrix tau(T_x) (x) I + I (x) tau(T_y) (Sec. 4, Ex. 2) as preconditioner:
//    P^{-1} = (2/(Mx+1)) S_x [ (2/(My+1)) S_y D S_y ] S_x with the DST-I
//    matrices S and D = 1/(lambda_n + c_x sigma^x_i + c_y sigma^y_j).
//    Per-system scalars (rho, a, beta) and convergence flags live on the
//    device; kernels skip converged systems.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace aao {

namespace {

template <typename R> using Cx = typename cplx_t<R>::type;

constexpr int kLineThreads = 256;
constexpr int kElemThreads = 256;

__host__ __device__ inline int lines_per_cta(int L, int csize) {
  const int b = 73728 / (padded_size(L) * csize);
  return b < 1 ? 1 : (b > 16 ? 16 : b);
}

template <typename TIn> __device__ __forceinline__ double ldd(const TIn* p) { return (double)__ldg(p); }

// Spectrum providers for the fused pass of the line convolutions (see fused_mid_pass_b): a real spectrum
// shared by all lines, and per-line complex spectra G[line][.] (zero beyond the lines); a thread's R
// contiguous factors come in 16-byte loads (FP32).
template <typename R> struct LineReal {
  const R* e;
  __device__ __forceinline__ Cx<R> operator()(int, int pf) const { return Cx<R>{__ldg(&e[pf]), (R)0}; }
  template <int RR> __device__ __forceinline__ void block(int, int s, Cx<R> (&f)[RR]) const {
    if constexpr (sizeof(R) == 4 && RR % 4 == 0) {
      const float4* e4 = reinterpret_cast<const float4*>(e + s);
#pragma unroll
      for (int m = 0; m < RR / 4; ++m) {
        const float4 a = __ldg(&e4[m]);
        f[4 * m] = Cx<R>{a.x, 0};
        f[4 * m + 1] = Cx<R>{a.y, 0};
        f[4 * m + 2] = Cx<R>{a.z, 0};
        f[4 * m + 3] = Cx<R>{a.w, 0};
      }
    } else {
#pragma unroll
      for (int m = 0; m < RR; ++m) f[m] = (*this)(0, s + m);
    }
  }
};
template <typename R> struct LineCplx {
  const Cx<R>* g;  // line b at g + (p0 + b) * stride
  int p0, nlines, stride;
  __device__ __forceinline__ Cx<R> operator()(int b, int pf) const {
    const int p = p0 + b;
    return p < nlines ? g[(size_t)p * stride + pf] : Cx<R>{0, 0};
  }
  template <int RR> __device__ __forceinline__ void block(int b, int s, Cx<R> (&f)[RR]) const {
    const int p = p0 + b;
    if constexpr (sizeof(R) == 4 && RR % 2 == 0) {
      if (p < nlines) {
        const float4* g4 = reinterpret_cast<const float4*>(g + (size_t)p * stride + s);
#pragma unroll
        for (int m = 0; m < RR / 2; ++m) {
          const float4 a = __ldg(&g4[m]);
          f[2 * m] = Cx<R>{a.x, a.y};
          f[2 * m + 1] = Cx<R>{a.z, a.w};
        }
      } else {
#pragma unroll
        for (int m = 0; m < RR; ++m) f[m] = Cx<R>{0, 0};
      }
    } else {
#pragma unroll
      for (int m = 0; m < RR; ++m) f[m] = (*this)(b, s + m);
    }
  }
};

// ---------------------------------------------------------------- matvec, FP64
// tmp[k][j][i] = c_x (T_x v[k][j][:])_i, rows j = 2q, 2q+1 packed as one complex line
template <typename TIn>
__global__ void __launch_bounds__(kLineThreads) mv2d_rows(const TIn* __restrict__ v, double* __restrict__ tmp, int Mx,
                                                          int My, int logLx, const double2* __restrict__ twx,
                                                          const double* __restrict__ Exf, int B) {
  extern __shared__ unsigned char smraw[];
  double2* buf = reinterpret_cast<double2*>(smraw);
  const int Lx = 1 << logLx, bs = padded_size(Lx);
  double2* q = buf + B * bs;
  load_quarter(q, twx, Lx / 4);
  const size_t slab = (size_t)blockIdx.y * Mx * My;
  const int pair0 = blockIdx.x * B, npairs = (My + 1) / 2;
  for (int idx = threadIdx.x; idx < B * Lx; idx += blockDim.x) {
    const int b = idx / Lx, i = idx - b * Lx, pr = pair0 + b;
    double x0 = 0, x1 = 0;
    if (pr < npairs && i < Mx) {
      x0 = ldd(v + slab + (size_t)(2 * pr) * Mx + i);
      if (2 * pr + 1 < My) x1 = ldd(v + slab + (size_t)(2 * pr + 1) * Mx + i);
    }
    buf[b * bs + pad16(i)] = double2{x0, x1};
  }
  fft_convolve_batched(buf, logLx, B, bs, q, logLx, [&](int, int pf) { return double2{__ldg(&Exf[pf]), 0.0}; });
  for (int idx = threadIdx.x; idx < B * Mx; idx += blockDim.x) {
    const int b = idx / Mx, i = idx - b * Mx, pr = pair0 + b;
    if (pr >= npairs) continue;
    const double2 t = buf[b * bs + pad16(i)];
    tmp[slab + (size_t)(2 * pr) * Mx + i] = t.x;
    if (2 * pr + 1 < My) tmp[slab + (size_t)(2 * pr + 1) * Mx + i] = t.y;
  }
}

// w = band(v) + tmp + c_y T_y v (columns; 2B columns per CTA, packed in pairs), or rhs - that;
// per-CTA sums of squares in sq_partial[k * gridDim.x + blockIdx.x]
template <typename TIn>
__global__ void __launch_bounds__(kLineThreads) mv2d_cols(const TIn* __restrict__ v, const double* __restrict__ tmp,
                                                          const double* __restrict__ rhs, double* __restrict__ w,
                                                          double* __restrict__ sq_partial, int Mx, int My, int logLy,
                                                          const double2* __restrict__ twy,
                                                          const double* __restrict__ Eyf, int B) {
  extern __shared__ unsigned char smraw[];
  __shared__ double red[32];
  double2* buf = reinterpret_cast<double2*>(smraw);
  double* bufr = reinterpret_cast<double*>(smraw);
  const int Ly = 1 << logLy, bs = padded_size(Ly);
  double2* q = buf + B * bs;
  load_quarter(q, twy, Ly / 4);
  const int k = blockIdx.y;
  const size_t Ms = (size_t)Mx * My, slab = (size_t)k * Ms;
  const int i0 = blockIdx.x * 2 * B, W = 2 * B;
  for (int idx = threadIdx.x; idx < Ly * W; idx += blockDim.x) {
    const int j = idx / W, cc = idx - j * W, i = i0 + cc;
    const double val = (j < My && i < Mx) ? ldd(v + slab + (size_t)j * Mx + i) : 0.0;
    bufr[2 * ((cc >> 1) * bs + pad16(j)) + (cc & 1)] = val;
  }
  fft_convolve_batched(buf, logLy, B, bs, q, logLy, [&](int, int pf) { return double2{__ldg(&Eyf[pf]), 0.0}; });
  double sq = 0;
  for (int idx = threadIdx.x; idx < My * W; idx += blockDim.x) {
    const int j = idx / W, cc = idx - j * W, i = i0 + cc;
    if (i >= Mx) continue;
    const size_t e = slab + (size_t)j * Mx + i;
    const double y = bufr[2 * ((cc >> 1) * bs + pad16(j)) + (cc & 1)];
    double band;
    if (k == 0) band = ldd(v + e);
    else if (k == 1) band = 1.5 * ldd(v + e) - 2.0 * ldd(v + e - Ms);
    else band = 1.5 * ldd(v + e) - 2.0 * ldd(v + e - Ms) + 0.5 * ldd(v + e - 2 * Ms);
    double out = band + tmp[e] + y;
    if (rhs) out = rhs[e] - out;
    w[e] = out;
    sq += out * out;
  }
  if (sq_partial) {
    double a[1] = {sq};
    block_sum<double, 1>(a, red);
    if (threadIdx.x == 0) sq_partial[(size_t)k * gridDim.x + blockIdx.x] = a[0];
  }
}

// ---------------------------------------------------------------- Step (b), 2D COCG
constexpr int kLU = 8;  // independent global loads in flight per thread in the line kernels

struct SysState {  // per system, FP64 scalars
  double2 rho, a, beta;
  double nb2, thr;
  int active, iters, flag, pad_;
};

__device__ __forceinline__ double2 cdivd(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return double2{(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}

template <typename R>
__device__ __forceinline__ Cx<R> to_c(double2 v) { return Cx<R>{(R)v.x, (R)v.y}; }

// partial sums of a complex value per CTA: part[n * P + blockIdx.x]
template <typename R>
__device__ __forceinline__ void write_partial(R re, R im, double2* part, int n, int P, R* red) {
  R a[2] = {re, im};
  block_sum<R, 2>(a, red);
  if (threadIdx.x == 0) part[(size_t)n * P + blockIdx.x] = double2{(double)a[0], (double)a[1]};
}

// r = b (taken from X), X = 0, partial |b|^2
template <typename R>
__global__ void __launch_bounds__(kElemThreads) c2d_init(Cx<R>* __restrict__ X, Cx<R>* __restrict__ Rr, size_t Ms,
                                                         double2* __restrict__ part) {
  __shared__ R red[64];
  const int n = blockIdx.y;
  R s = 0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < Ms; e += (size_t)gridDim.x * blockDim.x) {
    const size_t o = (size_t)n * Ms + e;
    const Cx<R> b = X[o];
    Rr[o] = b;
    X[o] = Cx<R>{0, 0};
    s += b.x * b.x + b.y * b.y;
  }
  write_partial<R>(s, 0, part, n, gridDim.x, red);
}

// out = scale * S_x in (rows, odd extension of length Lx = 2 (Mx+1)); MODE 1 also accumulates
// the bilinear partial sum_e r_e out_e (rho of COCG).
template <typename R, int MODE>
__global__ void __launch_bounds__(kLineThreads, sizeof(R) == 4 ? 3 : 1) c2d_rows_dst(const Cx<R>* __restrict__ in, Cx<R>* __restrict__ out,
                                                             const Cx<R>* __restrict__ rr, int Mx, int My, int logLx,
                                                             const Cx<R>* __restrict__ twx, R scale, int B,
                                                             const SysState* __restrict__ st,
                                                             double2* __restrict__ part) {
  using C = Cx<R>;
  extern __shared__ unsigned char smraw[];
  __shared__ R red[64];
  const int n = blockIdx.y;
  if (!st[n].active) return;
  C* buf = reinterpret_cast<C*>(smraw);
  const int Lx = 1 << logLx, bs = padded_size(Lx);
  C* q = buf + B * bs;
  load_quarter(q, twx, Lx / 4);
  const size_t slab = (size_t)n * Mx * My;
  const int j0 = blockIdx.x * B;
  for (int base = threadIdx.x; base < B * Lx; base += kLU * blockDim.x) {
    C y[kLU];
#pragma unroll
    for (int u = 0; u < kLU; ++u) {  // independent loads first (latency-bound otherwise)
      const int idx = base + u * blockDim.x;
      const int b = idx / Lx, l = idx - b * Lx, j = j0 + b;
      y[u] = C{0, 0};
      if (idx < B * Lx && j < My) {
        if (l >= 1 && l <= Mx) y[u] = in[slab + (size_t)j * Mx + (l - 1)];
        else if (l > Mx + 1) { const C t = in[slab + (size_t)j * Mx + (Lx - l - 1)]; y[u] = C{-t.x, -t.y}; }
      }
    }
#pragma unroll
    for (int u = 0; u < kLU; ++u) {
      const int idx = base + u * blockDim.x;
      if (idx >= B * Lx) break;
      const int b = idx / Lx, l = idx - b * Lx;
      buf[b * bs + pad16(l)] = y[u];
    }
  }
  fft_forward(buf, logLx, B, bs, q, logLx);
  R sre = 0, sim = 0;
  const R h = scale * (R)0.5;
  for (int idx = threadIdx.x; idx < B * Mx; idx += blockDim.x) {
    const int b = idx / Mx, i = idx - b * Mx, j = j0 + b;
    if (j >= My) continue;
    const C Y = buf[b * bs + pad16(bitrev(i + 1, logLx))];
    const C z = C{-h * Y.y, h * Y.x};  // scale * (i/2) * Y
    const size_t e = slab + (size_t)j * Mx + i;
    out[e] = z;
    if (MODE == 1) {
      const C r = rr[e];
      sre += r.x * z.x - r.y * z.y;
      sim += r.x * z.y + r.y * z.x;
    }
  }
  if (MODE == 1) write_partial<R>(sre, sim, part, n, gridDim.x, red);
}

// out = (2/(My+1)) S_y D S_y in along columns (B complex columns per CTA), D from lambda_n,
// c_x sigma^x_i (natural order) and c_y sigma^y (fused order, 1e30 where the DST multiplier vanishes)
template <typename R>
__global__ void __launch_bounds__(kLineThreads, sizeof(R) == 4 ? 3 : 1) c2d_cols_dst_div(const Cx<R>* __restrict__ in, Cx<R>* __restrict__ out,
                                                                 int Mx, int My, int logLy,
                                                                 const Cx<R>* __restrict__ twy,
                                                                 const R* __restrict__ sxn, const R* __restrict__ syf,
                                                                 const double2* __restrict__ lambda, int B,
                                                                 const SysState* __restrict__ st) {
  using C = Cx<R>;
  extern __shared__ unsigned char smraw[];
  const int n = blockIdx.y;
  if (!st[n].active) return;
  C* buf = reinterpret_cast<C*>(smraw);
  const int Ly = 1 << logLy, bs = padded_size(Ly);
  C* q = buf + B * bs;
  load_quarter(q, twy, Ly / 4);
  const size_t slab = (size_t)n * Mx * My;
  const int i0 = blockIdx.x * B;
  for (int base = threadIdx.x; base < Ly * B; base += kLU * blockDim.x) {
    C y[kLU];
#pragma unroll
    for (int u = 0; u < kLU; ++u) {
      const int idx = base + u * blockDim.x;
      const int l = idx / B, b = idx - l * B, i = i0 + b;
      y[u] = C{0, 0};
      if (idx < Ly * B && i < Mx) {
        if (l >= 1 && l <= My) y[u] = in[slab + (size_t)(l - 1) * Mx + i];
        else if (l > My + 1) { const C t = in[slab + (size_t)(Ly - l - 1) * Mx + i]; y[u] = C{-t.x, -t.y}; }
      }
    }
#pragma unroll
    for (int u = 0; u < kLU; ++u) {
      const int idx = base + u * blockDim.x;
      if (idx >= Ly * B) break;
      const int l = idx / B, b = idx - l * B;
      buf[b * bs + pad16(l)] = y[u];
    }
  }
  const C lam = to_c<R>(lambda[n]);
  const R invL = (R)1 / (R)Ly;
  fft_convolve_batched(buf, logLy, B, bs, q, logLy, [&](int b, int pf) {
    const int i = i0 + b;
    C d = lam;
    d.x += (i < Mx ? sxn[i] : (R)0) + __ldg(&syf[pf]);
    const R den = d.x * d.x + d.y * d.y;
    return C{invL * d.x / den, -invL * d.y / den};
  });
  for (int idx = threadIdx.x; idx < My * B; idx += blockDim.x) {
    const int j = idx / B, b = idx - j * B, i = i0 + b;
    if (i < Mx) out[slab + (size_t)j * Mx + i] = buf[b * bs + pad16(j + 1)];
  }
}

// p = z + beta p (written back), then tmp = c_x T_x p along rows
template <typename R>
__global__ void __launch_bounds__(kLineThreads, sizeof(R) == 4 ? 3 : 1) c2d_rows_conv(const Cx<R>* __restrict__ Z, Cx<R>* __restrict__ P,
                                                              Cx<R>* __restrict__ Tm, int Mx, int My, int logLx,
                                                              const Cx<R>* __restrict__ twx,
                                                              const R* __restrict__ Exf, int B,
                                                              const SysState* __restrict__ st) {
  using C = Cx<R>;
  extern __shared__ unsigned char smraw[];
  const int n = blockIdx.y;
  if (!st[n].active) return;
  C* buf = reinterpret_cast<C*>(smraw);
  const int Lx = 1 << logLx, bs = padded_size(Lx);
  C* q = buf + B * bs;
  load_quarter(q, twx, Lx / 4);
  const C beta = to_c<R>(st[n].beta);
  const size_t slab = (size_t)n * Mx * My;
  const int j0 = blockIdx.x * B;
  for (int base = threadIdx.x; base < B * Lx; base += kLU * blockDim.x) {
    C zv[kLU], pv[kLU];
#pragma unroll
    for (int u = 0; u < kLU; ++u) {
      const int idx = base + u * blockDim.x;
      const int b = idx / Lx, i = idx - b * Lx, j = j0 + b;
      zv[u] = C{0, 0};
      pv[u] = C{0, 0};
      if (idx < B * Lx && j < My && i < Mx) {
        const size_t e = slab + (size_t)j * Mx + i;
        zv[u] = Z[e];
        pv[u] = P[e];
      }
    }
#pragma unroll
    for (int u = 0; u < kLU; ++u) {
      const int idx = base + u * blockDim.x;
      if (idx >= B * Lx) break;
      const int b = idx / Lx, i = idx - b * Lx, j = j0 + b;
      const C p = cadd(zv[u], cmul(beta, pv[u]));
      if (j < My && i < Mx) P[slab + (size_t)j * Mx + i] = p;
      buf[b * bs + pad16(i)] = (j < My && i < Mx) ? p : C{0, 0};
    }
  }
  fft_convolve_batched(buf, logLx, B, bs, q, logLx, LineReal<R>{Exf});
  for (int idx = threadIdx.x; idx < B * Mx; idx += blockDim.x) {
    const int b = idx / Mx, i = idx - b * Mx, j = j0 + b;
    if (j < My) Tm[slab + (size_t)j * Mx + i] = buf[b * bs + pad16(i)];
  }
}

// q = tmp + lambda p + c_y T_y p along columns; partial p^T q
template <typename R>
__global__ void __launch_bounds__(kLineThreads, sizeof(R) == 4 ? 3 : 1) c2d_cols_conv(const Cx<R>* __restrict__ P, const Cx<R>* __restrict__ Tm,
                                                              Cx<R>* __restrict__ Q, int Mx, int My, int logLy,
                                                              const Cx<R>* __restrict__ twy,
                                                              const R* __restrict__ Eyf,
                                                              const double2* __restrict__ lambda, int B,
                                                              const SysState* __restrict__ st,
                                                              double2* __restrict__ part) {
  using C = Cx<R>;
  extern __shared__ unsigned char smraw[];
  __shared__ R red[64];
  const int n = blockIdx.y;
  if (!st[n].active) return;
  C* buf = reinterpret_cast<C*>(smraw);
  const int Ly = 1 << logLy, bs = padded_size(Ly);
  C* q = buf + B * bs;
  load_quarter(q, twy, Ly / 4);
  const size_t slab = (size_t)n * Mx * My;
  const int i0 = blockIdx.x * B;
  for (int base = threadIdx.x; base < Ly * B; base += kLU * blockDim.x) {
    C pv[kLU];
#pragma unroll
    for (int u = 0; u < kLU; ++u) {
      const int idx = base + u * blockDim.x;
      const int j = idx / B, b = idx - j * B, i = i0 + b;
      pv[u] = (idx < Ly * B && j < My && i < Mx) ? P[slab + (size_t)j * Mx + i] : C{0, 0};
    }
#pragma unroll
    for (int u = 0; u < kLU; ++u) {
      const int idx = base + u * blockDim.x;
      if (idx >= Ly * B) break;
      const int j = idx / B, b = idx - j * B;
      buf[b * bs + pad16(j)] = pv[u];
    }
  }
  fft_convolve_batched(buf, logLy, B, bs, q, logLy, LineReal<R>{Eyf});
  const C lam = to_c<R>(lambda[n]);
  R sre = 0, sim = 0;
  for (int idx = threadIdx.x; idx < My * B; idx += blockDim.x) {
    const int j = idx / B, b = idx - j * B, i = i0 + b;
    if (i >= Mx) continue;
    const size_t e = slab + (size_t)j * Mx + i;
    const C p = P[e];
    const C qv = cadd(cadd(buf[b * bs + pad16(j)], Tm[e]), cmul(lam, p));
    Q[e] = qv;
    sre += p.x * qv.x - p.y * qv.y;
    sim += p.x * qv.y + p.y * qv.x;
  }
  write_partial<R>(sre, sim, part, n, gridDim.x, red);
}

// x += a p, r -= a q, partial |r|^2
template <typename R>
__global__ void __launch_bounds__(kElemThreads) c2d_update(Cx<R>* __restrict__ X, Cx<R>* __restrict__ Rr,
                                                           const Cx<R>* __restrict__ P, const Cx<R>* __restrict__ Q,
                                                           size_t Ms, const SysState* __restrict__ st,
                                                           double2* __restrict__ part) {
  __shared__ R red[64];
  const int n = blockIdx.y;
  if (!st[n].active) return;
  const Cx<R> a = to_c<R>(st[n].a);
  R s = 0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < Ms; e += (size_t)gridDim.x * blockDim.x) {
    const size_t o = (size_t)n * Ms + e;
    X[o] = cadd(X[o], cmul(a, P[o]));
    const Cx<R> r = csub(Rr[o], cmul(a, Q[o]));
    Rr[o] = r;
    s += r.x * r.x + r.y * r.y;
  }
  write_partial<R>(s, 0, part, n, gridDim.x, red);
}

// ---- 2D Strang (BCCB) preconditioner (lambda_n I + I (x) c_x S_x + c_y S_y (x) I)^{-1} ------------------
// A BCCB inverse is a 2D cyclic convolution of period (Mx, My) with its first column h_n; it equals the
// first Mx x My outputs of a (Lx, Ly)-periodic convolution with the wrapped kernel (Lx >= 2 Mx - 1), done as
// a forward FFT along x of every zero-padded row, then per x-frequency a convolution along y with the
// precomputed spectrum G_n (fused order, 1/(Lx Ly) folded in), then an inverse FFT along x.

// W[n][j][p] = forward DIF FFT along x of the zero-padded row j of X[n] (position p holds frequency bitrev(p))
template <typename R>
__global__ void __launch_bounds__(kLineThreads, sizeof(R) == 4 ? 3 : 1) c2d_rows_fft_fwd(const Cx<R>* __restrict__ in, Cx<R>* __restrict__ W,
                                                                 int Mx, int My, int logLx,
                                                                 const Cx<R>* __restrict__ twx, int B,
                                                                 const SysState* __restrict__ st) {
  using C = Cx<R>;
  extern __shared__ unsigned char smraw[];
  const int n = blockIdx.y;
  if (st && !st[n].active) return;
  C* buf = reinterpret_cast<C*>(smraw);
  const int Lx = 1 << logLx, bs = padded_size(Lx);
  C* q = buf + B * bs;
  load_quarter(q, twx, Lx / 4);
  const size_t slab = (size_t)n * Mx * My;
  const int j0 = blockIdx.x * B;
  for (int base = threadIdx.x; base < B * Lx; base += kLU * blockDim.x) {
    C y[kLU];
#pragma unroll
    for (int u = 0; u < kLU; ++u) {
      const int idx = base + u * blockDim.x;
      const int b = idx / Lx, i = idx - b * Lx, j = j0 + b;
      y[u] = (idx < B * Lx && j < My && i < Mx) ? in[slab + (size_t)j * Mx + i] : C{0, 0};
    }
#pragma unroll
    for (int u = 0; u < kLU; ++u) {
      const int idx = base + u * blockDim.x;
      if (idx >= B * Lx) break;
      const int b = idx / Lx, i = idx - b * Lx;
      buf[b * bs + pad16(i)] = y[u];
    }
  }
  fft_forward(buf, logLx, B, bs, q, logLx);
  const size_t wslab = (size_t)n * My * Lx;
  for (int idx = threadIdx.x; idx < B * Lx; idx += blockDim.x) {
    const int b = idx / Lx, p = idx - b * Lx, j = j0 + b;
    if (j < My) W[wslab + (size_t)j * Lx + p] = buf[b * bs + pad16(p)];
  }
}

// Along y for every x-position p: W[n][:][p] <- first My outputs of the Ly-periodic convolution of the
// zero-padded column with the spectrum G[n][p][:] (fused order)
template <typename R>
__global__ void __launch_bounds__(kLineThreads, sizeof(R) == 4 ? 3 : 1) c2d_cols_conv_g(Cx<R>* __restrict__ W, int Lx, int My, int logLy,
                                                                const Cx<R>* __restrict__ twy,
                                                                const Cx<R>* __restrict__ G, int B,
                                                                const SysState* __restrict__ st) {
  using C = Cx<R>;
  extern __shared__ unsigned char smraw[];
  const int n = blockIdx.y;
  if (st && !st[n].active) return;
  C* buf = reinterpret_cast<C*>(smraw);
  const int Ly = 1 << logLy, bs = padded_size(Ly);
  C* q = buf + B * bs;
  load_quarter(q, twy, Ly / 4);
  const size_t wslab = (size_t)n * My * Lx;
  const int p0 = blockIdx.x * B;
  for (int base = threadIdx.x; base < Ly * B; base += kLU * blockDim.x) {
    C y[kLU];
#pragma unroll
    for (int u = 0; u < kLU; ++u) {
      const int idx = base + u * blockDim.x;
      const int j = idx / B, b = idx - j * B, p = p0 + b;
      y[u] = (idx < Ly * B && j < My && p < Lx) ? W[wslab + (size_t)j * Lx + p] : C{0, 0};
    }
#pragma unroll
    for (int u = 0; u < kLU; ++u) {
      const int idx = base + u * blockDim.x;
      if (idx >= Ly * B) break;
      const int j = idx / B, b = idx - j * B;
      buf[b * bs + pad16(j)] = y[u];
    }
  }
  const C* Gn = G + (size_t)n * Lx * Ly;
  fft_convolve_batched(buf, logLy, B, bs, q, logLy, LineCplx<R>{Gn, p0, Lx, Ly});
  for (int idx = threadIdx.x; idx < My * B; idx += blockDim.x) {
    const int j = idx / B, b = idx - j * B, p = p0 + b;
    if (p < Lx) W[wslab + (size_t)j * Lx + p] = buf[b * bs + pad16(j)];
  }
}

// out[n][j][i] = inverse DIT FFT along x of W[n][j][:] (bit-reversed in), first Mx outputs; MODE 1 also
// accumulates the bilinear partial sum_e r_e out_e (rho of COCG)
template <typename R, int MODE>
__global__ void __launch_bounds__(kLineThreads, sizeof(R) == 4 ? 3 : 1) c2d_rows_fft_inv(const Cx<R>* __restrict__ W, Cx<R>* __restrict__ out,
                                                                 const Cx<R>* __restrict__ rr, int Mx, int My,
                                                                 int logLx, const Cx<R>* __restrict__ twx, int B,
                                                                 const SysState* __restrict__ st,
                                                                 double2* __restrict__ part) {
  using C = Cx<R>;
  extern __shared__ unsigned char smraw[];
  __shared__ R red[64];
  const int n = blockIdx.y;
  if (!st[n].active) return;
  C* buf = reinterpret_cast<C*>(smraw);
  const int Lx = 1 << logLx, bs = padded_size(Lx);
  C* q = buf + B * bs;
  load_quarter(q, twx, Lx / 4);
  const size_t wslab = (size_t)n * My * Lx, slab = (size_t)n * Mx * My;
  const int j0 = blockIdx.x * B;
  for (int base = threadIdx.x; base < B * Lx; base += kLU * blockDim.x) {
    C y[kLU];
#pragma unroll
    for (int u = 0; u < kLU; ++u) {
      const int idx = base + u * blockDim.x;
      const int b = idx / Lx, p = idx - b * Lx, j = j0 + b;
      y[u] = (idx < B * Lx && j < My) ? W[wslab + (size_t)j * Lx + p] : C{0, 0};
    }
#pragma unroll
    for (int u = 0; u < kLU; ++u) {
      const int idx = base + u * blockDim.x;
      if (idx >= B * Lx) break;
      const int b = idx / Lx, p = idx - b * Lx;
      buf[b * bs + pad16(p)] = y[u];
    }
  }
  fft_backward(buf, logLx, B, bs, q, logLx);
  R sre = 0, sim = 0;
  for (int idx = threadIdx.x; idx < B * Mx; idx += blockDim.x) {
    const int b = idx / Mx, i = idx - b * Mx, j = j0 + b;
    if (j >= My) continue;
    const C z = buf[b * bs + pad16(i)];
    const size_t e = slab + (size_t)j * Mx + i;
    out[e] = z;
    if (MODE == 1) {
      const C r = rr[e];
      sre += r.x * z.x - r.y * z.y;
      sim += r.x * z.y + r.y * z.x;
    }
  }
  if (MODE == 1) write_partial<R>(sre, sim, part, n, gridDim.x, red);
}

// Spectra of the 2D Strang inverses, G[n][p][pf] = sum_{l,k} Qy[pf][l] Qx[p][k] / (lambda_n + sy[l] + sx[k]),
// in two tiled complex products: Bt[n][l][p] = sum_k Qx[p][k] / E_n[l][k] (pass 1), then
// G[n][p][pf] = sum_l Qy[pf][l] Bt[n][l][p] (pass 2).  Q* carry the wrap of the kernel, the DFT sizes and
// the orders the apply kernels read; computed in the plan's precision.
constexpr int kGT = 16;
template <typename R>
__global__ void __launch_bounds__(kGT * kGT) strang2d_spec_pass1(const Cx<R>* __restrict__ Qx, const R* __restrict__ sx,
                                                                 const R* __restrict__ sy,
                                                                 const double2* __restrict__ lambda, int Mx, int My,
                                                                 int Lx, Cx<R>* __restrict__ Bt) {
  using C = Cx<R>;
  __shared__ C sa[kGT][kGT + 1], sb[kGT][kGT + 1];
  const int n = blockIdx.z;
  const int l = blockIdx.y * kGT + threadIdx.y;   // row of Bt
  const int p = blockIdx.x * kGT + threadIdx.x;   // column of Bt
  const C lam{(R)lambda[n].x, (R)lambda[n].y};
  C acc{0, 0};
  for (int k0 = 0; k0 < Mx; k0 += kGT) {
    {  // sa[ty][tx] = 1 / E[l][k0 + tx]
      const int k = k0 + threadIdx.x;
      C v{0, 0};
      if (l < My && k < Mx) {
        const C d{lam.x + sy[l] + sx[k], lam.y};
        const R den = d.x * d.x + d.y * d.y;
        v = C{d.x / den, -d.y / den};
      }
      sa[threadIdx.y][threadIdx.x] = v;
    }
    {  // sb[ty][tx] = Qx[p' = blockIdx.x kGT + tx][k0 + ty]
      const int k = k0 + threadIdx.y, pp = blockIdx.x * kGT + threadIdx.x;
      sb[threadIdx.y][threadIdx.x] = (pp < Lx && k < Mx) ? Qx[(size_t)pp * Mx + k] : C{0, 0};
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < kGT; ++t) acc = cadd(acc, cmul(sa[threadIdx.y][t], sb[t][threadIdx.x]));
    __syncthreads();
  }
  if (l < My && p < Lx) Bt[((size_t)n * My + l) * Lx + p] = acc;
}

template <typename R>
__global__ void __launch_bounds__(kGT * kGT) strang2d_spec_pass2(const Cx<R>* __restrict__ Qy, const Cx<R>* __restrict__ Bt,
                                                                 int My, int Lx, int Ly, Cx<R>* __restrict__ G) {
  using C = Cx<R>;
  __shared__ C sa[kGT][kGT + 1], sb[kGT][kGT + 1];
  const int n = blockIdx.z;
  const int p = blockIdx.y * kGT + threadIdx.y;   // row of G_n
  const int f = blockIdx.x * kGT + threadIdx.x;   // column of G_n (fused y index)
  C acc{0, 0};
  for (int l0 = 0; l0 < My; l0 += kGT) {
    {  // sa[ty][tx] = Bt[n][l0 + tx][p]
      const int l = l0 + threadIdx.x;
      sa[threadIdx.y][threadIdx.x] = (p < Lx && l < My) ? Bt[((size_t)n * My + l) * Lx + p] : C{0, 0};
    }
    {  // sb[ty][tx] = Qy[f' = blockIdx.x kGT + tx][l0 + ty]
      const int l = l0 + threadIdx.y, ff = blockIdx.x * kGT + threadIdx.x;
      sb[threadIdx.y][threadIdx.x] = (ff < Ly && l < My) ? Qy[(size_t)ff * My + l] : C{0, 0};
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < kGT; ++t) acc = cadd(acc, cmul(sa[threadIdx.y][t], sb[t][threadIdx.x]));
    __syncthreads();
  }
  if (p < Lx && f < Ly) G[((size_t)n * Lx + p) * Ly + f] = acc;
}

enum { S_INIT = 0, S_RHO0 = 1, S_ALPHA = 2, S_CHECK = 3, S_BETA = 4 };

// one block per system: reduce the partials of the last kernel and update the scalars
__global__ void c2d_scalars(int step, SysState* __restrict__ st, const double2* __restrict__ part, int P, double tol,
                            int* __restrict__ active_count, int* __restrict__ iters, int* __restrict__ flags) {
  __shared__ double sr[256], si[256];
  const int n = blockIdx.x;
  SysState& s = st[n];
  if (step != S_INIT && !s.active) return;
  double a = 0, b = 0;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    a += part[(size_t)n * P + i].x;
    b += part[(size_t)n * P + i].y;
  }
  sr[threadIdx.x] = a;
  si[threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sr[threadIdx.x] += sr[threadIdx.x + o];
      si[threadIdx.x] += si[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x) return;
  const double2 v{sr[0], si[0]};
  switch (step) {
    case S_INIT:
      s.nb2 = v.x;
      s.thr = tol * tol * v.x;
      s.active = v.x > 0;
      s.iters = 0;
      s.flag = v.x > 0 ? 1 : 0;
      s.beta = double2{0, 0};
      break;
    case S_RHO0:
      s.rho = v;
      s.beta = double2{0, 0};
      break;
    case S_ALPHA:
      if (!(v.x * v.x + v.y * v.y > 0)) { s.flag = 2; s.active = 0; break; }
      s.a = cdivd(s.rho, v);
      break;
    case S_CHECK:
      s.iters++;
      if (!(v.x == v.x) || v.x > 1e30 * s.nb2) { s.flag = 3; s.active = 0; break; }
      if (v.x <= s.thr) { s.flag = 0; s.active = 0; break; }
      atomicAdd(active_count, 1);
      break;
    case S_BETA:
      if (!(s.rho.x * s.rho.x + s.rho.y * s.rho.y > 0)) { s.flag = 2; s.active = 0; break; }
      s.beta = cdivd(v, s.rho);
      s.rho = v;
      break;
  }
  if (step == S_CHECK || step == S_ALPHA || step == S_BETA) {
    iters[n] = s.iters;
    flags[n] = s.flag;
  }
}

template <typename R>
size_t line_smem(int L, int B) {
  return ((size_t)B * padded_size(L) + (size_t)(L / 4)) * sizeof(Cx<R>);
}

template <typename K>
cudaError_t allow_smem(K kern, size_t smem) {
  return allow_max_dynamic_smem(kern);
}

}  // namespace

size_t mv2d_partials(int Mx, int Nt, int logLy) {
  const int B = lines_per_cta(1 << logLy, (int)sizeof(double2));
  return (size_t)Nt * ((Mx + 2 * B - 1) / (2 * B));
}

template <typename TIn>
static cudaError_t mv2d(const TIn* v, const double* rhs, double* w, double* tmp, double* sq, int Mx, int My, int Nt,
                        int logLx, int logLy, const double2* twx, const double2* twy, const double* Exf,
                        const double* Eyf, cudaStream_t s) {
  const int Bx = lines_per_cta(1 << logLx, (int)sizeof(double2));
  const int By = lines_per_cta(1 << logLy, (int)sizeof(double2));
  const size_t smx = line_smem<double>(1 << logLx, Bx), smy = line_smem<double>(1 << logLy, By);
  cudaError_t e = allow_smem(mv2d_rows<TIn>, smx);
  if (e != cudaSuccess) return e;
  e = allow_smem(mv2d_cols<TIn>, smy);
  if (e != cudaSuccess) return e;
  const int npairs = (My + 1) / 2;
  mv2d_rows<TIn><<<dim3((npairs + Bx - 1) / Bx, Nt), kLineThreads, smx, s>>>(v, tmp, Mx, My, logLx, twx, Exf, Bx);
  mv2d_cols<TIn><<<dim3((Mx + 2 * By - 1) / (2 * By), Nt), kLineThreads, smy, s>>>(v, tmp, rhs, w, sq, Mx, My,
                                                                                    logLy, twy, Eyf, By);
  return cudaGetLastError();
}

cudaError_t launch_matvec2d_f64(const double* v, const double* rhs, double* w, double* tmp, double* sq, int Mx,
                                int My, int Nt, int logLx, int logLy, const double2* twx, const double2* twy,
                                const double* Exf, const double* Eyf, cudaStream_t s) {
  return mv2d<double>(v, rhs, w, tmp, sq, Mx, My, Nt, logLx, logLy, twx, twy, Exf, Eyf, s);
}
cudaError_t launch_matvec2d_f64_fin(const float* v, const double* rhs, double* w, double* tmp, double* sq, int Mx,
                                    int My, int Nt, int logLx, int logLy, const double2* twx, const double2* twy,
                                    const double* Exf, const double* Eyf, cudaStream_t s) {
  return mv2d<float>(v, rhs, w, tmp, sq, Mx, My, Nt, logLx, logLy, twx, twy, Exf, Eyf, s);
}

size_t cocg2d_state_bytes(int nsys) { return (size_t)nsys * sizeof(SysState); }

int cocg2d_max_partials(int Mx, int My, int logLx, int logLy, int csize) {
  const int Bx = lines_per_cta(1 << logLx, csize), By = lines_per_cta(1 << logLy, csize);
  const size_t Ms = (size_t)Mx * My;
  const int ne = (int)std::min<size_t>((Ms + kElemThreads - 1) / kElemThreads, 64);
  return std::max(ne, std::max((My + Bx - 1) / Bx, (Mx + By - 1) / By));
}

// The kernels of the 2D COCG: the start (r = b, x = 0, z = P^{-1} r, rho) and one iteration (q = A p, alpha,
// x and r updates, convergence check, z = P^{-1} r, beta and p).  Converged systems skip every kernel.
template <typename R>
struct Cocg2dRun {
  using C = Cx<R>;
  const Cocg2dArgs<R>& A;
  int Mx, My, nsys, Bx, By, ne;
  size_t Ms, smx, smy;
  dim3 g_rows, g_cols, g_elem;
  SysState* st;
  R sx;

  explicit Cocg2dRun(const Cocg2dArgs<R>& a) : A(a) {
    Mx = A.Mx; My = A.My; nsys = A.nsys;
    Ms = (size_t)Mx * My;
    const int Lx = 1 << A.logLx, Ly = 1 << A.logLy;
    Bx = lines_per_cta(Lx, (int)sizeof(C));
    By = lines_per_cta(Ly, (int)sizeof(C));
    smx = line_smem<R>(Lx, Bx);
    smy = line_smem<R>(Ly, By);
    st = reinterpret_cast<SysState*>(A.state);
    g_rows = dim3((My + Bx - 1) / Bx, nsys);
    g_cols = dim3((Mx + By - 1) / By, nsys);
    ne = (int)std::min<size_t>((Ms + kElemThreads - 1) / kElemThreads, 64);
    g_elem = dim3(ne, nsys);
    sx = (R)(2.0 / (Mx + 1));
  }
  cudaError_t prepare() const {
    cudaError_t e;
    if ((e = allow_smem(c2d_rows_dst<R, 0>, smx)) != cudaSuccess) return e;
    if ((e = allow_smem(c2d_rows_dst<R, 1>, smx)) != cudaSuccess) return e;
    if ((e = allow_smem(c2d_rows_conv<R>, smx)) != cudaSuccess) return e;
    if ((e = allow_smem(c2d_cols_dst_div<R>, smy)) != cudaSuccess) return e;
    if ((e = allow_smem(c2d_rows_fft_fwd<R>, smx)) != cudaSuccess) return e;
    if ((e = allow_smem(c2d_rows_fft_inv<R, 1>, smx)) != cudaSuccess) return e;
    if ((e = allow_smem(c2d_cols_conv_g<R>, smy)) != cudaSuccess) return e;
    return allow_smem(c2d_cols_conv<R>, smy);
  }
  void precond(cudaStream_t s) const {
    if (A.G2) {  // 2D Strang (BCCB): Z = P_n^{-1} Rr through W2, and rho's partials
      const int Lx = 1 << A.logLx;
      const dim3 g_colsg((Lx + By - 1) / By, nsys);
      c2d_rows_fft_fwd<R><<<g_rows, kLineThreads, smx, s>>>(A.Rr, A.W2, Mx, My, A.logLx, A.twx, Bx, st);
      c2d_cols_conv_g<R><<<g_colsg, kLineThreads, smy, s>>>(A.W2, Lx, My, A.logLy, A.twy, A.G2, By, st);
      c2d_rows_fft_inv<R, 1><<<g_rows, kLineThreads, smx, s>>>(A.W2, A.Z, A.Rr, Mx, My, A.logLx, A.twx, Bx, st,
                                                               A.part);
      return;
    }
    c2d_rows_dst<R, 0><<<g_rows, kLineThreads, smx, s>>>(A.Rr, A.Tm, nullptr, Mx, My, A.logLx, A.twx, (R)1, Bx, st,
                                                         A.part);
    c2d_cols_dst_div<R><<<g_cols, kLineThreads, smy, s>>>(A.Tm, A.Q, Mx, My, A.logLy, A.twy, A.sxn, A.syf, A.lambda,
                                                          By, st);
    c2d_rows_dst<R, 1><<<g_rows, kLineThreads, smx, s>>>(A.Q, A.Z, A.Rr, Mx, My, A.logLx, A.twx, sx, Bx, st, A.part);
  }
  void start(cudaStream_t s) const {  // 4 kernels + the preconditioner (3)
    c2d_init<R><<<g_elem, kElemThreads, 0, s>>>(A.X, A.Rr, Ms, A.part);
    c2d_scalars<<<nsys, 256, 0, s>>>(S_INIT, st, A.part, ne, A.tol, A.active_count, A.iters, A.flags);
    precond(s);
    c2d_scalars<<<nsys, 256, 0, s>>>(S_RHO0, st, A.part, g_rows.x, A.tol, A.active_count, A.iters, A.flags);
  }
  void iter_until_check(cudaStream_t s) const {  // 5 kernels
    c2d_rows_conv<R><<<g_rows, kLineThreads, smx, s>>>(A.Z, A.P, A.Tm, Mx, My, A.logLx, A.twx, A.Exf, Bx, st);
    c2d_cols_conv<R><<<g_cols, kLineThreads, smy, s>>>(A.P, A.Tm, A.Q, Mx, My, A.logLy, A.twy, A.Eyf, A.lambda, By,
                                                       st, A.part);
    c2d_scalars<<<nsys, 256, 0, s>>>(S_ALPHA, st, A.part, g_cols.x, A.tol, A.active_count, A.iters, A.flags);
    c2d_update<R><<<g_elem, kElemThreads, 0, s>>>(A.X, A.Rr, A.P, A.Q, Ms, st, A.part);
    c2d_scalars<<<nsys, 256, 0, s>>>(S_CHECK, st, A.part, ne, A.tol, A.active_count, A.iters, A.flags);
  }
  void iter_after_check(cudaStream_t s) const {  // 4 kernels
    precond(s);
    c2d_scalars<<<nsys, 256, 0, s>>>(S_BETA, st, A.part, g_rows.x, A.tol, A.active_count, A.iters, A.flags);
  }
};

// Before the loop: counters to zero, and the loop runs if any system is still active.
__global__ void c2d_loop_start(const SysState* __restrict__ st, int nsys, int* __restrict__ it_dev,
                               int* __restrict__ active_count, cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0) return;
  int any = 0;
  for (int n = 0; n < nsys; ++n) any |= st[n].active;
  *it_dev = 0;
  *active_count = 0;
  cudaGraphSetConditional(h, any ? 1u : 0u);
}

// End of one iteration: continue while some system was still active at its check and fewer than maxit
// iterations have run; the count of systems still active is reset for the next check.
__global__ void c2d_loop_next(int* __restrict__ it_dev, int* __restrict__ active_count, int maxit,
                              long long* __restrict__ loops_total, cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0) return;
  const int a = *active_count;
  *active_count = 0;
  const int it = ++*it_dev;
  ++*loops_total;
  cudaGraphSetConditional(h, (a > 0 && it < maxit) ? 1u : 0u);
}

// Host-driven loop (one host synchronisation per iteration); used while profiling each launch.
template <typename R>
static cudaError_t cocg2d(const Cocg2dArgs<R>& A, cudaStream_t s, int* inner_iters_out) {
  Cocg2dRun<R> run(A);
  cudaError_t e = run.prepare();
  if (e != cudaSuccess) return e;
  run.start(s);
  int it = 0;
  for (; it < A.maxit; ++it) {
    if ((e = cudaMemsetAsync(A.active_count, 0, sizeof(int), s)) != cudaSuccess) return e;
    run.iter_until_check(s);
    if ((e = cudaMemcpyAsync(A.host_count, A.active_count, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    if (*A.host_count == 0) { ++it; break; }
    run.iter_after_check(s);
  }
  if (inner_iters_out) *inner_iters_out = it;
  return cudaGetLastError();
}

// Records the whole 2D COCG into the graph that `s` is capturing: the start kernels, then a conditional
// WHILE node whose body (captured on body_stream) is one iteration followed by c2d_loop_next, so that the
// iterations run without any host synchronisation.
template <typename R>
static cudaError_t cocg2d_capture(const Cocg2dArgs<R>& A, cudaStream_t s, cudaStream_t body_stream) {
  Cocg2dRun<R> run(A);
  cudaError_t e = run.prepare();
  if (e != cudaSuccess) return e;
  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  if ((e = cudaStreamGetCaptureInfo(s, &cst, nullptr, &g)) != cudaSuccess) return e;
  if (cst != cudaStreamCaptureStatusActive || !g) return cudaErrorStreamCaptureUnsupported;
  cudaGraphConditionalHandle h;
  if ((e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault)) != cudaSuccess) return e;
  run.start(s);
  c2d_loop_start<<<1, 32, 0, s>>>(run.st, A.nsys, A.it_dev, A.active_count, h);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  if ((e = cudaStreamGetCaptureInfo(s, &cst, nullptr, nullptr, &deps, nullptr, &ndeps)) != cudaSuccess) return e;
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if ((e = cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &np)) != cudaSuccess) return e;
  if ((e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) != cudaSuccess)
    return e;
  cudaGraph_t body = np.conditional.phGraph_out[0];
  if ((e = cudaStreamBeginCaptureToGraph(body_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) !=
      cudaSuccess)
    return e;
  run.iter_until_check(body_stream);
  run.iter_after_check(body_stream);
  c2d_loop_next<<<1, 32, 0, body_stream>>>(A.it_dev, A.active_count, A.maxit, A.loops_total, h);
  cudaError_t e2 = cudaGetLastError();
  cudaGraph_t out = nullptr;
  e = cudaStreamEndCapture(body_stream, &out);
  return e2 != cudaSuccess ? e2 : e;
}

// every system active, no iterations: the state the line kernels test before the direct solve
__global__ void c2d_activate(SysState* __restrict__ st, int nsys, int* __restrict__ iters, int* __restrict__ flags) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nsys) return;
  st[n].active = 1;
  st[n].iters = 0;
  st[n].flag = 0;
  iters[n] = 0;
  flags[n] = 0;
}

// X[n] <- (lambda_n I + c_x tau(T_x) (x) I + I (x) c_y tau(T_y))^{-1} X[n]: the 2D DST diagonalisation of
// Example 2 (Eq. 4.5), i.e. the three line passes of the COCG preconditioner applied once to the rhs.
template <typename R>
static cudaError_t tau2d_direct(const Cocg2dArgs<R>& A, cudaStream_t s) {
  Cocg2dRun<R> run(A);
  cudaError_t e = run.prepare();
  if (e != cudaSuccess) return e;
  c2d_activate<<<(A.nsys + 255) / 256, 256, 0, s>>>(run.st, A.nsys, A.iters, A.flags);
  c2d_rows_dst<R, 0><<<run.g_rows, kLineThreads, run.smx, s>>>(A.X, A.Tm, nullptr, A.Mx, A.My, A.logLx, A.twx, (R)1,
                                                               run.Bx, run.st, A.part);
  c2d_cols_dst_div<R><<<run.g_cols, kLineThreads, run.smy, s>>>(A.Tm, A.Q, A.Mx, A.My, A.logLy, A.twy, A.sxn, A.syf,
                                                                A.lambda, run.By, run.st);
  c2d_rows_dst<R, 0><<<run.g_rows, kLineThreads, run.smx, s>>>(A.Q, A.X, nullptr, A.Mx, A.My, A.logLx, A.twx, run.sx,
                                                               run.Bx, run.st, A.part);
  return cudaGetLastError();
}

template <typename R>
static cudaError_t strang2d_setup(const Cx<R>* Qx, const Cx<R>* Qy, const R* sx, const R* sy, const double2* lambda,
                                  int Mx, int My, int logLx, int logLy, int nsys, Cx<R>* Bt, Cx<R>* G,
                                  cudaStream_t s) {
  const int Lx = 1 << logLx, Ly = 1 << logLy;
  const dim3 blk(kGT, kGT);
  strang2d_spec_pass1<R><<<dim3((Lx + kGT - 1) / kGT, (My + kGT - 1) / kGT, nsys), blk, 0, s>>>(Qx, sx, sy, lambda, Mx,
                                                                                               My, Lx, Bt);
  strang2d_spec_pass2<R><<<dim3((Ly + kGT - 1) / kGT, (Lx + kGT - 1) / kGT, nsys), blk, 0, s>>>(Qy, Bt, My, Lx, Ly, G);
  return cudaGetLastError();
}
cudaError_t launch_strang2d_setup_f32(const float2* Qx, const float2* Qy, const float* sx, const float* sy,
                                      const double2* lambda, int Mx, int My, int logLx, int logLy, int nsys,
                                      float2* Bt, float2* G, cudaStream_t s) {
  return strang2d_setup<float>(Qx, Qy, sx, sy, lambda, Mx, My, logLx, logLy, nsys, Bt, G, s);
}
cudaError_t launch_strang2d_setup_f64(const double2* Qx, const double2* Qy, const double* sx, const double* sy,
                                      const double2* lambda, int Mx, int My, int logLx, int logLy, int nsys,
                                      double2* Bt, double2* G, cudaStream_t s) {
  return strang2d_setup<double>(Qx, Qy, sx, sy, lambda, Mx, My, logLx, logLy, nsys, Bt, G, s);
}

cudaError_t launch_tau2d_direct_f32(const Cocg2dArgs<float>& a, cudaStream_t s) { return tau2d_direct<float>(a, s); }
cudaError_t launch_tau2d_direct_f64(const Cocg2dArgs<double>& a, cudaStream_t s) { return tau2d_direct<double>(a, s); }

cudaError_t launch_cocg2d_f32(const Cocg2dArgs<float>& a, cudaStream_t s, int* launches) {
  return cocg2d<float>(a, s, launches);
}
cudaError_t launch_cocg2d_f64(const Cocg2dArgs<double>& a, cudaStream_t s, int* launches) {
  return cocg2d<double>(a, s, launches);
}
cudaError_t capture_cocg2d_f32(const Cocg2dArgs<float>& a, cudaStream_t s, cudaStream_t body_stream) {
  return cocg2d_capture<float>(a, s, body_stream);
}
cudaError_t capture_cocg2d_f64(const Cocg2dArgs<double>& a, cudaStream_t s, cudaStream_t body_stream) {
  return cocg2d_capture<double>(a, s, body_stream);
}

}  // namespace aao
