// Device helpers shared by the sm_103a kernels: complex arithmetic, the
// in-shared-memory radix-16 FFT engine, and deterministic block reductions.
//
// FFT conventions (used by every kernel of the library):
//   * forward  = DIF, X_k = sum_j x_j exp(-2 pi i jk/N), natural order in,
//                bit-reversed order out;
//   * backward = DIT, x_j = sum_k X_k exp(+2 pi i jk/N) (no 1/N), bit-reversed
//                order in, natural order out.
// A convolution therefore never permutes: DIF, multiply by a kernel
// spectrum stored in bit-reversed order, DIT (see fft_convolve, which also
// fuses the multiply into the last forward / first backward pass).
//
// A pass handles 2^r consecutive radix-2 stages at once: each thread loads
// 2^r elements at stride S, does a 2^r-point DFT in registers, multiplies by
// the external twiddles W_{N'}^{j0 m} (N' = 2^r S, j0 the position of the
// group inside its block) and stores output m at offset bitrev_r(m) * S.
// This is exactly r radix-2 decimation-in-frequency stages, so the global
// order stays bit-reversed.
//
// Twiddles come from a quarter-circle table q[e] = exp(-2 pi i e / Nq),
// e < Nq/4, held in shared memory; exp(-2 pi i e/Nq) for any e < Nq follows
// by rotating with (-i)^(e div Nq/4).
//
// Shared-memory layout of the data: element i lives at pad16(i) = i + i/16,
// which keeps the unit-stride last pass free of bank conflicts.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

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

template <int r> __host__ __device__ constexpr int brev_c(int m) {
  int o = 0;
  for (int b = 0; b < r; ++b) o |= ((m >> b) & 1) << (r - 1 - b);
  return o;
}

// multiply by -i (DIR < 0) or +i (DIR > 0)
template <int DIR, typename T> __device__ __forceinline__ T rot90(T a) {
  return DIR < 0 ? T{a.y, -a.x} : T{-a.y, a.x};
}

// exp(DIR * 2 pi i e / Nq) from the quarter table q (Nq = 4 * quarter), 0 <= e < Nq
template <int DIR, typename T>
__device__ __forceinline__ T twiddle(const T* q, int e, int logNq) {
  const int quad = e >> (logNq - 2);
  const T w = q[e & ((1 << (logNq - 2)) - 1)];
  T r;
  switch (quad) {  // w * (-i)^quad
    case 0: r = w; break;
    case 1: r = T{w.y, -w.x}; break;
    case 2: r = T{-w.x, -w.y}; break;
    default: r = T{-w.y, w.x}; break;
  }
  return DIR < 0 ? r : cconj(r);
}

// ---- small DFTs in registers, natural order in and out -------------------------------------
template <int DIR, typename T> __device__ __forceinline__ void dft4(T& x0, T& x1, T& x2, T& x3) {
  const T a = cadd(x0, x2), c = csub(x0, x2), b = cadd(x1, x3), d = rot90<DIR>(csub(x1, x3));
  x0 = cadd(a, b);
  x2 = csub(a, b);
  x1 = cadd(c, d);
  x3 = csub(c, d);
}

template <typename T> struct Consts;
template <> struct Consts<float2> {
  static __device__ __forceinline__ float c8() { return 0.70710678118654752f; }
  static __device__ __forceinline__ float c16() { return 0.92387953251128676f; }
  static __device__ __forceinline__ float s16() { return 0.38268343236508977f; }
};
template <> struct Consts<double2> {
  static __device__ __forceinline__ double c8() { return 0.70710678118654752440; }
  static __device__ __forceinline__ double c16() { return 0.92387953251128675613; }
  static __device__ __forceinline__ double s16() { return 0.38268343236508977173; }
};

// multiply by W16^e (DIR < 0: exp(-2 pi i e/16)) for a compile-time e in 0..9
template <int DIR, int e, typename T> __device__ __forceinline__ T w16(T a) {
  using K = Consts<T>;
  const auto c8 = K::c8(), c = K::c16(), s = K::s16();
  T w;
  switch (e) {
    case 0: return a;
    case 1: w = T{c, -s}; break;
    case 2: w = T{c8, -c8}; break;
    case 3: w = T{s, -c}; break;
    case 4: return rot90<DIR>(a);
    case 6: w = T{-c8, -c8}; break;
    case 9: w = T{-c, s}; break;
    default: w = T{1, 0}; break;
  }
  if (DIR > 0) w = cconj(w);
  return cmul(a, w);
}

// In-place DFT of R = 2^r points, natural order in and out.
template <int DIR, int r, typename T> __device__ __forceinline__ void dft(T (&v)[1 << r]) {
  if (r == 1) {
    const T a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
  } else if (r == 2) {
    dft4<DIR>(v[0], v[1], v[2], v[3]);
  } else if (r == 3) {
    // 8 = 2 x 4: k = k1 + 2 k2; inner 4-point DFTs over k2, twiddle W8^{k1 m2}, outer radix 2
    T e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    dft4<DIR>(e[0], e[1], e[2], e[3]);
    dft4<DIR>(o[0], o[1], o[2], o[3]);
    o[1] = w16<DIR, 2>(o[1]);
    o[2] = rot90<DIR>(o[2]);
    o[3] = w16<DIR, 6>(o[3]);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      v[m] = cadd(e[m], o[m]);
      v[m + 4] = csub(e[m], o[m]);
    }
  } else if (r == 4) {
    // 16 = 4 x 4: k = k1 + 4 k2, m = 4 m1 + m2
    T y[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      T a = v[k1], b = v[k1 + 4], c = v[k1 + 8], d = v[k1 + 12];
      dft4<DIR>(a, b, c, d);  // over k2 -> m2
      y[4 * k1 + 0] = a;
      y[4 * k1 + 1] = b;
      y[4 * k1 + 2] = c;
      y[4 * k1 + 3] = d;
    }
    y[4 * 1 + 1] = w16<DIR, 1>(y[5]);
    y[4 * 1 + 2] = w16<DIR, 2>(y[6]);
    y[4 * 1 + 3] = w16<DIR, 3>(y[7]);
    y[4 * 2 + 1] = w16<DIR, 2>(y[9]);
    y[4 * 2 + 2] = w16<DIR, 4>(y[10]);
    y[4 * 2 + 3] = w16<DIR, 6>(y[11]);
    y[4 * 3 + 1] = w16<DIR, 3>(y[13]);
    y[4 * 3 + 2] = w16<DIR, 6>(y[14]);
    y[4 * 3 + 3] = w16<DIR, 9>(y[15]);
#pragma unroll
    for (int m2 = 0; m2 < 4; ++m2) {
      T a = y[m2], b = y[4 + m2], c = y[8 + m2], d = y[12 + m2];
      dft4<DIR>(a, b, c, d);  // over k1 -> m1
      v[m2] = a;
      v[4 + m2] = b;
      v[8 + m2] = c;
      v[12 + m2] = d;
    }
  }
}

// ---- passes ----------------------------------------------------------------------------------
// One DIF pass of r stages (global stages s0 .. s0+r-1) over `batch`
// transforms of length N = 2^logN at buf[b*bstride + pad16(i)].
template <typename T, int r>
__device__ __forceinline__ void dif_pass(T* buf, int logN, int s0, int batch, int bstride, const T* q, int logNq,
                                         const T* pt = nullptr) {
  constexpr int R = 1 << r;
  const int S = 1 << (logN - s0 - r);
  const int per = 1 << (logN - r);
  const int tshift = logNq - logN + s0;  // W_{N'}^{x} = W_{Nq}^{x << tshift}
  for (int g = threadIdx.x; g < batch * per; g += blockDim.x) {
    const int b = g >> (logN - r);
    const int gi = g & (per - 1);
    const int j0 = gi & (S - 1);
    const int start = (gi >> (logN - s0 - r)) << (logN - s0);
    T v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = buf[b * bstride + pad16(start + j0 + k * S)];
    dft<-1, r>(v);
    if (j0 != 0) {
      if (pt) {
#pragma unroll
        for (int m = 1; m < R; ++m) v[m] = cmul(v[m], pt[(m - 1) * S + j0]);
      } else {
#pragma unroll
        for (int m = 1; m < R; ++m) v[m] = cmul(v[m], twiddle<-1>(q, (j0 * m) << tshift, logNq));
      }
    }
#pragma unroll
    for (int m = 0; m < R; ++m) buf[b * bstride + pad16(start + j0 + brev_c<r>(m) * S)] = v[m];
  }
}

// The inverse of dif_pass (up to the factor 2^r): conjugate twiddles, backward DFT.
template <typename T, int r>
__device__ __forceinline__ void dit_pass(T* buf, int logN, int s0, int batch, int bstride, const T* q, int logNq,
                                         const T* pt = nullptr) {
  constexpr int R = 1 << r;
  const int S = 1 << (logN - s0 - r);
  const int per = 1 << (logN - r);
  const int tshift = logNq - logN + s0;
  for (int g = threadIdx.x; g < batch * per; g += blockDim.x) {
    const int b = g >> (logN - r);
    const int gi = g & (per - 1);
    const int j0 = gi & (S - 1);
    const int start = (gi >> (logN - s0 - r)) << (logN - s0);
    T v[R];
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = buf[b * bstride + pad16(start + j0 + brev_c<r>(m) * S)];
    if (j0 != 0) {
      if (pt) {
#pragma unroll
        for (int m = 1; m < R; ++m) v[m] = cmulc(v[m], pt[(m - 1) * S + j0]);
      } else {
#pragma unroll
        for (int m = 1; m < R; ++m) v[m] = cmul(v[m], twiddle<+1>(q, (j0 * m) << tshift, logNq));
      }
    }
    dft<+1, r>(v);
#pragma unroll
    for (int k = 0; k < R; ++k) buf[b * bstride + pad16(start + j0 + k * S)] = v[k];
  }
}

// The first pass takes the leftover logN mod 4 stages so that every later
// pass has 16 points; the last forward (first backward) pass has stride 1.
__device__ __forceinline__ int first_pass_stages(int logN) {
  const int rem = logN & 3;
  return rem ? rem : 4;
}

// Per-pass twiddle tables: every 16-point pass after the first and before the
// last (stride S = N >> (s0 + 4) >= 16) gets a table pt[(m-1) * S + j0] =
// W_{16 S}^{j0 m}, m = 1..15, so that consecutive threads (consecutive j0)
// read consecutive shared-memory words.  pass_table_size gives the total
// entry count; pass_table_offset the start of the pass that begins at s0.
__host__ __device__ inline int pass_table_size(int logN) {
  const int r0 = (logN & 3) ? (logN & 3) : 4;
  int tot = 0;
  for (int s0 = r0; s0 + 4 < logN; s0 += 4) tot += 15 * (1 << (logN - s0 - 4));
  return tot;
}
__device__ __forceinline__ int pass_table_offset(int logN, int s0) {
  const int r0 = first_pass_stages(logN);
  int off = 0;
  for (int t = r0; t < s0; t += 4) off += 15 * (1 << (logN - t - 4));
  return off;
}
template <typename T>
__device__ void build_pass_tables(T* pt, const T* q, int logN, int logNq) {
  const int r0 = first_pass_stages(logN);
  int off = 0;
  for (int s0 = r0; s0 + 4 < logN; s0 += 4) {
    const int S = 1 << (logN - s0 - 4), tshift = logNq - logN + s0;
    for (int idx = threadIdx.x; idx < 15 * S; idx += blockDim.x) {
      const int m = idx / S + 1, j0 = idx - (m - 1) * S;
      pt[off + idx] = twiddle<-1>(q, (j0 * m) << tshift, logNq);
    }
    off += 15 * S;
  }
}

template <typename T>
__device__ __forceinline__ void dif_pass_any(int r, T* buf, int logN, int s0, int batch, int bstride, const T* q,
                                             int logNq) {
  switch (r) {
    case 1: dif_pass<T, 1>(buf, logN, s0, batch, bstride, q, logNq); break;
    case 2: dif_pass<T, 2>(buf, logN, s0, batch, bstride, q, logNq); break;
    case 3: dif_pass<T, 3>(buf, logN, s0, batch, bstride, q, logNq); break;
    default: dif_pass<T, 4>(buf, logN, s0, batch, bstride, q, logNq); break;
  }
}
template <typename T>
__device__ __forceinline__ void dit_pass_any(int r, T* buf, int logN, int s0, int batch, int bstride, const T* q,
                                             int logNq) {
  switch (r) {
    case 1: dit_pass<T, 1>(buf, logN, s0, batch, bstride, q, logNq); break;
    case 2: dit_pass<T, 2>(buf, logN, s0, batch, bstride, q, logNq); break;
    case 3: dit_pass<T, 3>(buf, logN, s0, batch, bstride, q, logNq); break;
    default: dit_pass<T, 4>(buf, logN, s0, batch, bstride, q, logNq); break;
  }
}

// Forward FFT (DIF) of `batch` transforms; starts and ends with __syncthreads().
// q: quarter twiddle table of size Nq/4 (Nq >= N, both powers of two).
template <typename T>
__device__ void fft_forward(T* buf, int logN, int batch, int bstride, const T* q, int logNq,
                            const T* pt = nullptr) {
  __syncthreads();
  const int r0 = first_pass_stages(logN);
  dif_pass_any<T>(r0, buf, logN, 0, batch, bstride, q, logNq);
  __syncthreads();
  int off = 0;
  for (int s0 = r0; s0 < logN; s0 += 4) {
    const bool tab = pt && s0 + 4 < logN;
    dif_pass<T, 4>(buf, logN, s0, batch, bstride, q, logNq, tab ? pt + off : nullptr);
    if (s0 + 4 < logN) off += 15 * (1 << (logN - s0 - 4));
    __syncthreads();
  }
}

// Backward FFT (DIT, unnormalised) of `batch` transforms; starts and ends with __syncthreads().
template <typename T>
__device__ void fft_backward(T* buf, int logN, int batch, int bstride, const T* q, int logNq,
                             const T* pt = nullptr) {
  __syncthreads();
  const int r0 = first_pass_stages(logN);
  int s0 = logN - 4;
  while (s0 >= r0) {
    const bool tab = pt && s0 + 4 < logN;
    dit_pass<T, 4>(buf, logN, s0, batch, bstride, q, logNq, tab ? pt + pass_table_offset(logN, s0) : nullptr);
    __syncthreads();
    s0 -= 4;
  }
  dit_pass_any<T>(r0, buf, logN, 0, batch, bstride, q, logNq);
  __syncthreads();
}

// buf <- backward(factor .* forward(buf)) for one transform of length N: the
// last forward pass, the pointwise multiply and the first backward pass are
// fused into one register pass.  factor(pf) is called with the "fused-order"
// index pf = start + m of the 2^r-point group starting at `start` (m the
// natural DFT output index), i.e. the kernel spectrum for bit-reversed
// position start + bitrev_r(m); tables are stored in that order so that a
// thread reads its 2^r factors contiguously.
// A factor provider may also offer block<R>(start, f), filling f[m] = factor(start + m) for m < R in one
// go (vector loads of the R contiguous values a thread needs); fused_mid_pass uses it when present.
template <typename F, typename T, int R, typename = void> struct has_block : std::false_type {};
template <typename F, typename T, int R>
struct has_block<F, T, R,
                 std::void_t<decltype(std::declval<const F&>().template block<R>(0, std::declval<T (&)[R]>()))>>
    : std::true_type {};

template <typename T, int r, typename F>
__device__ __forceinline__ void fused_mid_pass(T* buf, int logN, F factor) {
  constexpr int R = 1 << r;
  const int per = 1 << (logN - r);
  for (int g = threadIdx.x; g < per; g += blockDim.x) {
    const int start = g << r;
    T v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = buf[pad16(start + k)];
    dft<-1, r>(v);
    if constexpr (has_block<F, T, R>::value) {
      T f[R];
      factor.template block<R>(start, f);
#pragma unroll
      for (int m = 0; m < R; ++m) v[m] = cmul(v[m], f[m]);
    } else {
#pragma unroll
      for (int m = 0; m < R; ++m) v[m] = cmul(v[m], factor(start + m));
    }
    dft<+1, r>(v);
#pragma unroll
    for (int k = 0; k < R; ++k) buf[pad16(start + k)] = v[k];
  }
}

// Batched form of fused_mid_pass: factor(b, pf) for transform b (and factor.block<R>(b, start, f) when
// the provider offers it).
template <typename F, typename T, int R, typename = void> struct has_block_b : std::false_type {};
template <typename F, typename T, int R>
struct has_block_b<
    F, T, R, std::void_t<decltype(std::declval<const F&>().template block<R>(0, 0, std::declval<T (&)[R]>()))>>
    : std::true_type {};

template <typename T, int r, typename F>
__device__ __forceinline__ void fused_mid_pass_b(T* buf, int logN, int batch, int bstride, F factor) {
  constexpr int R = 1 << r;
  const int per = 1 << (logN - r);
  for (int gg = threadIdx.x; gg < batch * per; gg += blockDim.x) {
    const int b = gg >> (logN - r);
    const int start = (gg & (per - 1)) << r;
    T* base = buf + b * bstride;
    T v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = base[pad16(start + k)];
    dft<-1, r>(v);
    if constexpr (has_block_b<F, T, R>::value) {
      T f[R];
      factor.template block<R>(b, start, f);
#pragma unroll
      for (int m = 0; m < R; ++m) v[m] = cmul(v[m], f[m]);
    } else {
#pragma unroll
      for (int m = 0; m < R; ++m) v[m] = cmul(v[m], factor(b, start + m));
    }
    dft<+1, r>(v);
#pragma unroll
    for (int k = 0; k < R; ++k) base[pad16(start + k)] = v[k];
  }
}

// fft_convolve over `batch` transforms at buf + b * bstride; factor(b, pf).
template <typename T, typename F>
__device__ void fft_convolve_batched(T* buf, int logN, int batch, int bstride, const T* q, int logNq, F factor,
                                     const T* pt = nullptr) {
  __syncthreads();
  const int r0 = first_pass_stages(logN);
  int s0 = 0, r = r0, off = 0;
  while (s0 + r < logN) {
    if (s0 == 0) {
      dif_pass_any<T>(r, buf, logN, 0, batch, bstride, q, logNq);
    } else {
      dif_pass<T, 4>(buf, logN, s0, batch, bstride, q, logNq, pt ? pt + off : nullptr);
      off += 15 * (1 << (logN - s0 - 4));
    }
    __syncthreads();
    s0 += r;
    r = 4;
  }
  switch (logN - s0) {
    case 1: fused_mid_pass_b<T, 1>(buf, logN, batch, bstride, factor); break;
    case 2: fused_mid_pass_b<T, 2>(buf, logN, batch, bstride, factor); break;
    case 3: fused_mid_pass_b<T, 3>(buf, logN, batch, bstride, factor); break;
    default: fused_mid_pass_b<T, 4>(buf, logN, batch, bstride, factor); break;
  }
  __syncthreads();
  if (s0 > 0) {
    int t0 = s0 - 4;
    while (t0 >= r0) {
      dit_pass<T, 4>(buf, logN, t0, batch, bstride, q, logNq, pt ? pt + pass_table_offset(logN, t0) : nullptr);
      __syncthreads();
      t0 -= 4;
    }
    dit_pass_any<T>(r0, buf, logN, 0, batch, bstride, q, logNq);
    __syncthreads();
  }
}

template <typename T, typename F>
__device__ void fft_convolve(T* buf, int logN, const T* q, int logNq, F factor, const T* pt = nullptr) {
  __syncthreads();
  const int r0 = first_pass_stages(logN);
  // forward passes except the last
  int s0 = 0, r = r0, off = 0;
  while (s0 + r < logN) {
    if (s0 == 0) {
      dif_pass_any<T>(r, buf, logN, 0, 1, 0, q, logNq);
    } else {
      dif_pass<T, 4>(buf, logN, s0, 1, 0, q, logNq, pt ? pt + off : nullptr);
      off += 15 * (1 << (logN - s0 - 4));
    }
    __syncthreads();
    s0 += r;
    r = 4;
  }
  // s0 is now the start of the last forward pass (stride 1, r stages)
  switch (logN - s0) {
    case 1: fused_mid_pass<T, 1>(buf, logN, factor); break;
    case 2: fused_mid_pass<T, 2>(buf, logN, factor); break;
    case 3: fused_mid_pass<T, 3>(buf, logN, factor); break;
    default: fused_mid_pass<T, 4>(buf, logN, factor); break;
  }
  __syncthreads();
  // backward passes except the first
  if (s0 > 0) {
    int t0 = s0 - 4;
    while (t0 >= r0) {
      dit_pass<T, 4>(buf, logN, t0, 1, 0, q, logNq, pt ? pt + pass_table_offset(logN, t0) : nullptr);
      __syncthreads();
      t0 -= 4;
    }
    dit_pass_any<T>(r0, buf, logN, 0, 1, 0, q, logNq);
    __syncthreads();
  }
}

// The passes of fft_convolve between its first forward and its last backward pass (both of
// r0 = first_pass_stages(logN) stages at stride N >> r0), for logN > r0: the remaining forward
// 16-point passes, the fused middle pass and the backward 16-point passes.  The caller has
// synchronised after the first pass; ends synchronised.
template <typename T, typename F>
__device__ void fft_convolve_inner(T* buf, int logN, const T* q, int logNq, F factor, const T* pt) {
  const int r0 = first_pass_stages(logN);
  int s0 = r0, off = 0;
  while (s0 + 4 < logN) {
    dif_pass<T, 4>(buf, logN, s0, 1, 0, q, logNq, pt ? pt + off : nullptr);
    off += 15 * (1 << (logN - s0 - 4));
    __syncthreads();
    s0 += 4;
  }
  switch (logN - s0) {
    case 1: fused_mid_pass<T, 1>(buf, logN, factor); break;
    case 2: fused_mid_pass<T, 2>(buf, logN, factor); break;
    case 3: fused_mid_pass<T, 3>(buf, logN, factor); break;
    default: fused_mid_pass<T, 4>(buf, logN, factor); break;
  }
  __syncthreads();
  for (int t0 = s0 - 4; t0 >= r0; t0 -= 4) {
    dit_pass<T, 4>(buf, logN, t0, 1, 0, q, logNq, pt ? pt + pass_table_offset(logN, t0) : nullptr);
    __syncthreads();
  }
}

// Last forward pass of fft_forward_fused: the 2^r-point DFT of each group, stored in fused order.
template <typename T, int r>
__device__ __forceinline__ void fused_last_pass(T* buf, int logN) {
  constexpr int R = 1 << r;
  const int per = 1 << (logN - r);
  for (int g = threadIdx.x; g < per; g += blockDim.x) {
    const int start = g << r;
    T v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = buf[pad16(start + k)];
    dft<-1, r>(v);
#pragma unroll
    for (int k = 0; k < R; ++k) buf[pad16(start + k)] = v[k];
  }
}

// Forward DFT (sign -1) of one transform with the output left in the fused order that
// fft_convolve's factor(pf) uses: buf[pad16(pf)] = spectrum at fused index pf.  Starts and
// ends with __syncthreads().
template <typename T>
__device__ void fft_forward_fused(T* buf, int logN, const T* q, int logNq, const T* pt = nullptr) {
  __syncthreads();
  const int r0 = first_pass_stages(logN);
  int s0 = 0, r = r0, off = 0;
  while (s0 + r < logN) {
    if (s0 == 0) {
      dif_pass_any<T>(r, buf, logN, 0, 1, 0, q, logNq);
    } else {
      dif_pass<T, 4>(buf, logN, s0, 1, 0, q, logNq, pt ? pt + off : nullptr);
      off += 15 * (1 << (logN - s0 - 4));
    }
    __syncthreads();
    s0 += r;
    r = 4;
  }
  switch (logN - s0) {
    case 1: fused_last_pass<T, 1>(buf, logN); break;
    case 2: fused_last_pass<T, 2>(buf, logN); break;
    case 3: fused_last_pass<T, 3>(buf, logN); break;
    default: fused_last_pass<T, 4>(buf, logN); break;
  }
  __syncthreads();
}

// (double) f * 2^d (d in {-1, 0, 1}) from the bits of f, exactly, with integer operations only: the FP64<->FP32
// conversions issue on the FP64 pipe of this GPU (under 1 per clock per SM), and a conversion kept for the rare
// cases would be evaluated for every element when the compiler turns the branch into a select.  Zero keeps its
// sign, a subnormal f is normalised (its leading one at bit p of the significand gives the exponent p - 149),
// infinities and NaNs keep their payload (the quiet bit moves to the FP64 quiet bit).
__device__ __forceinline__ double f2d_exact(float f, int d = 0) {
  const unsigned int u = __float_as_uint(f), ex = (u >> 23) & 0xffu, man = u & 0x7fffffu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  unsigned long long bits;
  if (ex == 255u) {
    bits = sign | (0x7ffull << 52) | ((unsigned long long)man << 29);
  } else if (ex != 0u) {
    bits = sign | ((unsigned long long)(ex + 896u + d) << 52) | ((unsigned long long)man << 29);
  } else if (man == 0u) {
    bits = sign;
  } else {
    const int p = 31 - __clz((int)man);  // 0 <= p <= 22
    bits = sign | ((unsigned long long)(p + 874 + d) << 52) |
           (((unsigned long long)man << (52 - p)) & 0xfffffffffffffull);
  }
  return __longlong_as_double((long long)bits);
}
__device__ __forceinline__ double f2d_bits(float f) { return f2d_exact(f, 0); }

// Copies the quarter twiddle table (n4 entries) from global to shared memory.
template <typename T>
__device__ __forceinline__ void load_quarter(T* dst, const T* __restrict__ src, int n4) {
  for (int i = threadIdx.x; i < n4; i += blockDim.x) dst[i] = __ldg(&src[i]);
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

// Lets `kern` use as much dynamic shared memory as the device allows.  The
// attribute is global per kernel function, so every launcher sets the same
// (maximal) value: a launch from one host thread can never see a smaller limit
// set by a concurrent launch of another problem size.
// Done once per (kernel, device); later calls only look the pair up.
cudaError_t allow_max_dynamic_smem_impl(const void* kern);
template <typename K>
inline cudaError_t allow_max_dynamic_smem(K kern) {
  return allow_max_dynamic_smem_impl(reinterpret_cast<const void*>(kern));
}

}  // namespace aao
