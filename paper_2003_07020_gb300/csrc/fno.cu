// Learned warm start for the shifted solves of Step (b): a Fourier neural
// operator (4 Fourier layers, width 32, 16 modes) that predicts the initial
// guess x0 of (lambda_n I + c T) x = b from (b / ||b||, lambda_n, alpha, x).
// The paper has no learned component; the true residual decides whether a
// prediction is used (the COCG kernel keeps x0 only if ||b - A x0|| < ||b||).
//
// Architecture (per sample, M grid points, channels last [M][32]):
//   features -> lift (6 -> 32) -> 4 x [ truncated DFT (16 modes), complex 32x32
//   mixing per mode, inverse, + pointwise 32x32 + bias, GELU (not after the
//   last) ] -> projection (32 -> 2) -> x0 = ||b|| (y0 + i y1).
// Weights are read as BF16 and every sum is accumulated in FP32; training
// keeps FP32 master weights, Adam moments and FP32 gradients.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "../../include/aao.h"
#include "kernels.h"

namespace aao {

namespace {

constexpr int FC = 32, FK = 16, FL = 4, FF = 6;
constexpr int LAYER_SIZE = FK * FC * FC * 2 + FC * FC + FC;
constexpr int OFF_LW = 0, OFF_LB = FC * FF;
__host__ __device__ constexpr int off_R(int l) { return FC * FF + FC + l * LAYER_SIZE; }
__host__ __device__ constexpr int off_W(int l) { return off_R(l) + FK * FC * FC * 2; }
__host__ __device__ constexpr int off_b(int l) { return off_W(l) + FC * FC; }
constexpr int OFF_PW = FC * FF + FC + FL * LAYER_SIZE;
constexpr int OFF_PB = OFF_PW + 2 * FC;
constexpr int NPARAM = OFF_PB + 2;

using bf16 = __nv_bfloat16;
__device__ __forceinline__ float wv(const bf16* P, int i) { return __bfloat162float(P[i]); }

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

__global__ void k_norms(const float2* __restrict__ b, int M, float* __restrict__ norms) {
  __shared__ float red[256];
  const int s = blockIdx.x;
  float a = 0;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    const float2 v = b[(size_t)s * M + i];
    a += v.x * v.x + v.y * v.y;
  }
  red[threadIdx.x] = a;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) norms[s] = sqrtf(red[0]);
}

// Truncated DFT, the first step of a Fourier layer, over tiles of TP = 64 points:
// part[s][chunk][k][c] = sum_{i in chunk} h[s][i][c] tw[i][k]  (tw[i][k] = e^{-2 pi i ik/M});
// the chunk partials are summed (in a fixed order) by k_mix.
constexpr int TP = 64;
constexpr int DT = TP;
constexpr int TILE_SMEM_FLOATS = 8 * FK * FC * 2;  // 32 KB: activation + twiddle tiles, then warp partials

// Loads the twiddles of the tile starting at point i0 (8 float4 = 16 complex per point, zero past M).
__device__ __forceinline__ void load_tile_twiddles(float2* ts, const float2* __restrict__ tw, int i0, int M) {
  for (int q = threadIdx.x; q < TP * FK / 2; q += blockDim.x) {
    const int r = q >> 3, i = i0 + r;
    float4 v{0, 0, 0, 0};
    if (i < M) v = __ldg(reinterpret_cast<const float4*>(tw) + (size_t)i * (FK / 2) + (q & 7));
    reinterpret_cast<float4*>(ts + r * FK)[q & 7] = v;
  }
}

// DFT partials of one tile: hs [TP][FC] activations, ts [TP][FK] twiddles (both in `raw`), 256
// threads; warp w takes the points r = w (mod 8) for all 16 modes, then the 8 warp partials are
// added in shared memory (overwriting the tiles).  Writes FK * FC values to out.
__device__ __forceinline__ void tile_dft(float* raw, float2* __restrict__ out) {
  const float* hs = raw;
  const float2* ts = reinterpret_cast<const float2*>(raw + TP * FC);
  const int t = threadIdx.x, w = t >> 5, c = t & 31;
  __syncthreads();
  float2 acc[FK];
#pragma unroll
  for (int k = 0; k < FK; ++k) acc[k] = float2{0, 0};
#pragma unroll 2
  for (int r = w; r < TP; r += 8) {
    const float v = hs[r * FC + c];
    const float4* t4 = reinterpret_cast<const float4*>(ts + r * FK);
#pragma unroll
    for (int k4 = 0; k4 < FK / 2; ++k4) {
      const float4 q = t4[k4];
      acc[2 * k4].x = fmaf(v, q.x, acc[2 * k4].x);
      acc[2 * k4].y = fmaf(v, q.y, acc[2 * k4].y);
      acc[2 * k4 + 1].x = fmaf(v, q.z, acc[2 * k4 + 1].x);
      acc[2 * k4 + 1].y = fmaf(v, q.w, acc[2 * k4 + 1].y);
    }
  }
  __syncthreads();
  float2* red = reinterpret_cast<float2*>(raw);  // [8 warps][FK][FC]
#pragma unroll
  for (int k = 0; k < FK; ++k) red[(w * FK + k) * FC + c] = acc[k];
  __syncthreads();
  for (int q = t; q < FK * FC; q += blockDim.x) {
    float2 a{0, 0};
#pragma unroll
    for (int ww = 0; ww < 8; ++ww) {
      const float2 v = red[ww * FK * FC + q];
      a.x += v.x;
      a.y += v.y;
    }
    out[q] = a;
  }
}

// grid (chunks, B), 256 threads: DFT partials of h (the backward's gradient transforms)
__global__ void __launch_bounds__(256) k_dft(const float* __restrict__ h, int M, const float2* __restrict__ tw,
                                             float2* __restrict__ part, int nch) {
  __shared__ __align__(16) float raw[TILE_SMEM_FLOATS];
  const int s = blockIdx.y, ch = blockIdx.x, i0 = ch * TP, t = threadIdx.x;
  for (int q = t; q < TP * FC / 4; q += blockDim.x) {
    const int r = q >> 3, c4 = q & 7, i = i0 + r;
    float4 v{0, 0, 0, 0};
    if (i < M) v = reinterpret_cast<const float4*>(h + ((size_t)s * M + i) * FC)[c4];
    reinterpret_cast<float4*>(raw + r * FC)[c4] = v;
  }
  load_tile_twiddles(reinterpret_cast<float2*>(raw + TP * FC), tw, i0, M);
  tile_dft(raw, part + ((size_t)s * nch + ch) * FK * FC);
}

// Features, lift and the first layer's DFT partials in one pass over a tile of points:
// f_i = [Re b_i / ||b||, Im b_i / ||b||, Re lambda, Im lambda, alpha, (i+1)/(M+1)],
// h0_i = W_lift f_i + b_lift (feat and h0 are kept for the backward).
__global__ void __launch_bounds__(256) k_lift_dft(const float2* __restrict__ b, const double2* __restrict__ lam,
                                                  const float* __restrict__ alpha, const float* __restrict__ norms,
                                                  const bf16* __restrict__ P, int M, const float2* __restrict__ tw,
                                                  float* __restrict__ feat, float* __restrict__ h0,
                                                  float2* __restrict__ part, int nch) {
  __shared__ __align__(16) float raw[TILE_SMEM_FLOATS];
  __shared__ float Wl[FC * FF + FC];  // lift W [32][6] then bias
  const int s = blockIdx.y, ch = blockIdx.x, i0 = ch * TP, t = threadIdx.x;
  for (int q = t; q < FC * FF + FC; q += blockDim.x) Wl[q] = wv(P, OFF_LW + q);
  load_tile_twiddles(reinterpret_cast<float2*>(raw + TP * FC), tw, i0, M);
  __syncthreads();
  const int o = t & 31, w = t >> 5;
  const float inv = norms[s] > 0 ? 1.0f / norms[s] : 0.0f;
  const float l0 = (float)lam[s].x, l1 = (float)lam[s].y, al = alpha[s];
  for (int il = w; il < TP; il += 8) {
    const int i = i0 + il;
    float hv = 0.0f;
    if (i < M) {
      const size_t n = (size_t)s * M + i;
      const float2 v = b[n];
      const float f[FF] = {v.x * inv, v.y * inv, l0, l1, al, (float)(i + 1) / (float)(M + 1)};
      if (o < FF) feat[n * FF + o] = f[o];
      hv = Wl[FC * FF + o];
#pragma unroll
      for (int q = 0; q < FF; ++q) hv = fmaf(Wl[o * FF + q], f[q], hv);
      h0[n * FC + o] = hv;
    }
    raw[il * FC + o] = hv;
  }
  tile_dft(raw, part + ((size_t)s * nch + ch) * FK * FC);
}

// Spectral mixing, one block per (mode k, group of MIX_S samples), R[k] staged in shared memory.
// First X[s][k][c] = sum over chunks of part (times c_k / M when grad_scale), stored to Xsum.
// forward: out[s][k][o] = sum_i R[k][o][i] X[s][k][i]
// adjoint: out[s][k][i] = sum_o conj(R[k][o][i]) X[s][k][o]
constexpr int MIX_S = 16;
__global__ void __launch_bounds__(512) k_mix(const float2* __restrict__ part, int nch, float2* __restrict__ Xsum,
                                             const bf16* __restrict__ P, int offR, int B, int M,
                                             float2* __restrict__ out, int adjoint, int grad_scale) {
  __shared__ float2 Rs[FC][FC + 1];
  __shared__ float2 xs[MIX_S][FC];
  const int k = blockIdx.x, s0 = blockIdx.y * MIX_S, t = threadIdx.x;
  for (int q = t; q < FC * FC; q += blockDim.x) {
    const int o = q >> 5, i = q & 31, idx = offR + ((k * FC + o) * FC + i) * 2;
    Rs[o][i] = float2{wv(P, idx), wv(P, idx + 1)};
  }
  {
    const int sl = t >> 5, c = t & 31, s = s0 + sl;
    float2 x{0, 0};
    if (s < B) {
      const float2* ps = part + (size_t)s * nch * FK * FC + k * FC + c;
      for (int ch = 0; ch < nch; ++ch) {
        const float2 v = ps[(size_t)ch * FK * FC];
        x.x += v.x;
        x.y += v.y;
      }
      if (grad_scale) {
        const float sc = (k == 0 ? 1.0f : 2.0f) / (float)M;
        x.x *= sc;
        x.y *= sc;
      }
      Xsum[((size_t)s * FK + k) * FC + c] = x;
    }
    xs[sl][c] = x;
  }
  __syncthreads();
  const int sl = t >> 5, a = t & 31, s = s0 + sl;
  if (s >= B) return;
  float re = 0, im = 0;
#pragma unroll 8
  for (int j = 0; j < FC; ++j) {
    const float2 x = xs[sl][j];
    if (adjoint) {  // conj(R[k][j][a]) x_j
      const float2 r = Rs[j][a];
      re += r.x * x.x + r.y * x.y;
      im += r.x * x.y - r.y * x.x;
    } else {        // R[k][a][j] x_j
      const float2 r = Rs[a][j];
      re += r.x * x.x - r.y * x.y;
      im += r.x * x.y + r.y * x.x;
    }
  }
  out[((size_t)s * FK + k) * FC + a] = float2{re, im};
}

// z = (1/M) Re sum_k c_k G_k e^{+i theta} + W h + b;  h_out = act(z); with part != null also the
// next layer's DFT partials of h_out for this tile (tile_dft).
// Thread o keeps G[.][o] (scaled by c_k / M) and row o of W in registers; per point it reads the
// activation row and the 16 twiddles as broadcast float4.
__global__ void __launch_bounds__(256) k_inv_pw(const float2* __restrict__ G, const float* __restrict__ hin,
                                                const bf16* __restrict__ P, int offW, int offb, int M,
                                                const float2* __restrict__ tw, float* __restrict__ z,
                                                float* __restrict__ hout, int act, float2* __restrict__ part,
                                                int nch) {
  __shared__ __align__(16) float raw[TILE_SMEM_FLOATS];
  __shared__ float Ws[FC][FC + 1];
  float* hs = raw;                                          // [TP][FC]
  float2* ts = reinterpret_cast<float2*>(raw + TP * FC);    // [TP][FK]
  const int s = blockIdx.y, ch = blockIdx.x, i0 = ch * TP, t = threadIdx.x;
  for (int q = t; q < FC * FC; q += blockDim.x) Ws[q >> 5][q & 31] = wv(P, offW + q);
  for (int q = t; q < TP * FC / 4; q += blockDim.x) {
    const int r = q >> 3, c4 = q & 7, i = i0 + r;
    float4 v{0, 0, 0, 0};
    if (i < M) v = reinterpret_cast<const float4*>(hin + ((size_t)s * M + i) * FC)[c4];
    reinterpret_cast<float4*>(hs + r * FC)[c4] = v;
  }
  load_tile_twiddles(ts, tw, i0, M);
  const int o = t & 31, w = t >> 5;
  const float invM = 1.0f / (float)M;
  float2 g[FK];
#pragma unroll
  for (int k = 0; k < FK; ++k) {
    const float2 v = G[((size_t)s * FK + k) * FC + o];
    const float sc = (k == 0 ? 1.0f : 2.0f) * invM;
    g[k] = float2{v.x * sc, v.y * sc};
  }
  const float bias = wv(P, offb + o);
  __syncthreads();
  float wr[FC];  // row o of W
#pragma unroll
  for (int c = 0; c < FC; ++c) wr[c] = Ws[o][c];
#pragma unroll 1
  for (int il = w; il < TP; il += 8) {
    const int i = i0 + il;
    if (i >= M) break;
    float sp = 0, u = bias;
    const float4* t4 = reinterpret_cast<const float4*>(ts + il * FK);
#pragma unroll
    for (int k4 = 0; k4 < FK / 2; ++k4) {  // Re(G e^{+i theta}) with e^{+i theta} = conj(tw)
      const float4 q = t4[k4];
      sp = fmaf(g[2 * k4].x, q.x, sp);
      sp = fmaf(g[2 * k4].y, q.y, sp);
      sp = fmaf(g[2 * k4 + 1].x, q.z, sp);
      sp = fmaf(g[2 * k4 + 1].y, q.w, sp);
    }
    const float4* h4 = reinterpret_cast<const float4*>(hs + il * FC);
#pragma unroll
    for (int c4 = 0; c4 < FC / 4; ++c4) {
      const float4 v = h4[c4];
      u = fmaf(wr[4 * c4], v.x, u);
      u = fmaf(wr[4 * c4 + 1], v.y, u);
      u = fmaf(wr[4 * c4 + 2], v.z, u);
      u = fmaf(wr[4 * c4 + 3], v.w, u);
    }
    const float zz = sp + u;
    const float hv = act ? gelu(zz) : zz;
    const size_t e = ((size_t)s * M + i) * FC + o;
    z[e] = zz;
    hout[e] = hv;
    __syncwarp();             // every lane has read row il
    hs[il * FC + o] = hv;     // the warp owns row il: the tile becomes h_out
  }
  if (part) tile_dft(raw, part + ((size_t)s * nch + ch) * FK * FC);
}

// y[n] = W_proj h[n] + b_proj, one thread per point (row read as float4)
__global__ void __launch_bounds__(256) k_proj(const float* __restrict__ h, const bf16* __restrict__ P, size_t N,
                                              float* __restrict__ y) {
  __shared__ float Wp[2 * FC + 2];
  for (int q = threadIdx.x; q < 2 * FC + 2; q += blockDim.x) Wp[q] = wv(P, OFF_PW + q);  // proj W then bias
  __syncthreads();
  const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const float4* h4 = reinterpret_cast<const float4*>(h + n * FC);
  float y0 = Wp[2 * FC], y1 = Wp[2 * FC + 1];
#pragma unroll
  for (int c4 = 0; c4 < FC / 4; ++c4) {
    const float4 v = h4[c4];
    y0 += Wp[4 * c4] * v.x + Wp[4 * c4 + 1] * v.y + Wp[4 * c4 + 2] * v.z + Wp[4 * c4 + 3] * v.w;
    y1 += Wp[FC + 4 * c4] * v.x + Wp[FC + 4 * c4 + 1] * v.y + Wp[FC + 4 * c4 + 2] * v.z + Wp[FC + 4 * c4 + 3] * v.w;
  }
  reinterpret_cast<float2*>(y)[n] = float2{y0, y1};
}

__global__ void k_output(const float* __restrict__ y, const float* __restrict__ norms, int M, size_t N,
                         float2* __restrict__ x0) {
  const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const float nb = norms[n / M];
  x0[n] = float2{nb * y[2 * n], nb * y[2 * n + 1]};
}

// per sample: t = x / ||b||, loss = sum|y - t|^2 / sum|t|^2, dy = 2 (y - t) / (sum|t|^2 B)
__global__ void k_loss(const float* __restrict__ y, const float2* __restrict__ xt, const float* __restrict__ norms,
                       int M, int B, float* __restrict__ dy, float* __restrict__ loss) {
  __shared__ float r1[256], r2[256];
  const int s = blockIdx.x;
  const float inv = norms[s] > 0 ? 1.0f / norms[s] : 0.0f;
  float a = 0, e = 0;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    const size_t n = (size_t)s * M + i;
    const float tx = xt[n].x * inv, ty = xt[n].y * inv;
    const float dx = y[2 * n] - tx, dyy = y[2 * n + 1] - ty;
    a += tx * tx + ty * ty;
    e += dx * dx + dyy * dyy;
  }
  r1[threadIdx.x] = a;
  r2[threadIdx.x] = e;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      r1[threadIdx.x] += r1[threadIdx.x + o];
      r2[threadIdx.x] += r2[threadIdx.x + o];
    }
    __syncthreads();
  }
  const float den = r1[0] > 0 ? r1[0] : 1.0f;
  if (threadIdx.x == 0) loss[s] = r2[0] / den;
  const float sc = 2.0f / (den * (float)B);
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    const size_t n = (size_t)s * M + i;
    dy[2 * n] = sc * (y[2 * n] - xt[n].x * inv);
    dy[2 * n + 1] = sc * (y[2 * n + 1] - xt[n].y * inv);
  }
}

// dh[n][c] = sum_o PW[o][c] dy[n][o]
__global__ void k_proj_back(const float* __restrict__ dy, const bf16* __restrict__ P, size_t N, float* __restrict__ dh) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * FC) return;
  const size_t n = t / FC;
  const int c = (int)(t % FC);
  dh[t] = wv(P, OFF_PW + c) * dy[2 * n] + wv(P, OFF_PW + FC + c) * dy[2 * n + 1];
}

__global__ void k_act_back(const float* __restrict__ dh, const float* __restrict__ z, float* __restrict__ dz, size_t n,
                           int act) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) dz[t] = act ? dh[t] * gelu_grad(z[t]) : dh[t];
}

// Weight gradients as sums of outer products over all points, in two
// deterministic stages.  Stage 1: block j reduces a contiguous range of points
// in tiles of 32 into part[j] = (sum_n A[n][a] B[n][b] for a, b < 32; then
// sum_n A[n][a]); thread (a = t / 8, 4 consecutive b) reads As as a broadcast
// and Bs as float4.  Stage 2 (k_outer_sum) adds the block partials in order.
constexpr int OUTER_PART = FC * FC + FC;
constexpr int OUTER_MAX_BLOCKS = 8 * 152;
__global__ void __launch_bounds__(256) k_outer(const float* __restrict__ A, int na, const float* __restrict__ Bm,
                                               int nb, size_t N, float* __restrict__ part) {
  __shared__ float As[32][33];
  __shared__ __align__(16) float Bs[32][36];
  const int t = threadIdx.x, a = t >> 3, b0 = (t & 7) * 4;
  float acc[4] = {0, 0, 0, 0}, accb = 0;
  const size_t chunk = (N + gridDim.x - 1) / gridDim.x;
  const size_t n0 = blockIdx.x * chunk, n1 = n0 + chunk < N ? n0 + chunk : N;
  for (size_t base = n0; base < n1; base += 32) {
    __syncthreads();
    for (int q = t; q < 32 * 32; q += blockDim.x) {
      const int r = q >> 5, col = q & 31;
      const size_t n = base + r;
      As[r][col] = (n < n1 && col < na) ? A[n * na + col] : 0.0f;
      Bs[r][col] = (n < n1 && col < nb) ? Bm[n * nb + col] : 0.0f;
    }
    __syncthreads();
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
      const float av = As[r][a];
      const float4 bv = *reinterpret_cast<const float4*>(&Bs[r][b0]);
      acc[0] = fmaf(av, bv.x, acc[0]);
      acc[1] = fmaf(av, bv.y, acc[1]);
      acc[2] = fmaf(av, bv.z, acc[2]);
      acc[3] = fmaf(av, bv.w, acc[3]);
    }
    if (t < 32)
      for (int r = 0; r < 32; ++r) accb += As[r][t];
  }
  float* o = part + (size_t)blockIdx.x * OUTER_PART;
  *reinterpret_cast<float4*>(o + a * FC + b0) = float4{acc[0], acc[1], acc[2], acc[3]};
  if (t < 32) o[FC * FC + t] = accb;
}

// gOut[a][b] = sum_j part[j][a][b] (a < na, b < nb), gBias[a] = sum_j part[j][1024 + a]
__global__ void __launch_bounds__(1024) k_outer_sum(const float* __restrict__ part, int nparts, int na, int nb,
                                                    float* __restrict__ gOut, float* __restrict__ gBias) {
  __shared__ float red[32][33];
  const int cw = threadIdx.x & 31, rr = threadIdx.x >> 5, col = blockIdx.x * 32 + cw;
  float a = 0;
  if (col < OUTER_PART)
    for (int j = rr; j < nparts; j += 32) a += part[(size_t)j * OUTER_PART + col];
  red[rr][cw] = a;
  __syncthreads();
  if (rr == 0 && col < OUTER_PART) {
    float v = 0;
    for (int q = 0; q < 32; ++q) v += red[q][cw];
    if (col < FC * FC) {
      const int ia = col >> 5, ib = col & 31;
      if (ia < na && ib < nb) gOut[ia * nb + ib] = v;
    } else if (gBias && col - FC * FC < na) {
      gBias[col - FC * FC] = v;
    }
  }
}

// gR[k][o][i] += sum_s gG[s][k][o] conj(H[s][k][i])  (re/im interleaved)
__global__ void __launch_bounds__(1024) k_gR(const float2* __restrict__ gG, const float2* __restrict__ H, int B,
                                             float* __restrict__ gR) {
  const int k = blockIdx.x, o = threadIdx.x >> 5, i = threadIdx.x & 31;
  float re = 0, im = 0;
#pragma unroll 8
  for (int s = 0; s < B; ++s) {
    const float2 g = gG[((size_t)s * FK + k) * FC + o], h = H[((size_t)s * FK + k) * FC + i];
    re += g.x * h.x + g.y * h.y;
    im += g.y * h.x - g.x * h.y;
  }
  float* d = gR + ((size_t)(k * FC + o) * FC + i) * 2;
  d[0] += re;
  d[1] += im;
}

// Back through the point-wise matrix and the inverse DFT of a Fourier layer:
// dh_prev[s][i][c] = sum_o W[o][c] dz[s][i][o] + sum_k Re(gH[s][k][c] e^{+i theta_ik}).
// Thread c keeps column c of W and gH[.][c] in registers (as k_inv_pw).
__global__ void __launch_bounds__(256) k_back_pw_idft(const float* __restrict__ dz, const float2* __restrict__ gH,
                                                      const bf16* __restrict__ P, int offW, int M,
                                                      const float2* __restrict__ tw, float* __restrict__ dhp) {
  __shared__ __align__(16) float ds[TP][FC];
  __shared__ __align__(16) float2 ts[TP][FK];
  __shared__ float Ws[FC][FC + 1];
  const int s = blockIdx.y, i0 = blockIdx.x * TP, t = threadIdx.x;
  for (int q = t; q < FC * FC; q += blockDim.x) Ws[q >> 5][q & 31] = wv(P, offW + q);
  for (int q = t; q < TP * FC / 4; q += blockDim.x) {
    const int r = q >> 3, c4 = q & 7, i = i0 + r;
    float4 v{0, 0, 0, 0};
    if (i < M) v = reinterpret_cast<const float4*>(dz + ((size_t)s * M + i) * FC)[c4];
    reinterpret_cast<float4*>(ds[r])[c4] = v;
  }
  for (int q = t; q < TP * FK / 2; q += blockDim.x) {
    const int r = q >> 3, i = i0 + r;
    float4 v{0, 0, 0, 0};
    if (i < M) v = __ldg(reinterpret_cast<const float4*>(tw) + (size_t)i * (FK / 2) + (q & 7));
    reinterpret_cast<float4*>(ts[r])[q & 7] = v;
  }
  const int c = t & 31, w = t >> 5;
  float2 g[FK];
#pragma unroll
  for (int k = 0; k < FK; ++k) g[k] = gH[((size_t)s * FK + k) * FC + c];
  __syncthreads();
  float wc[FC];  // column c of W
#pragma unroll
  for (int o = 0; o < FC; ++o) wc[o] = Ws[o][c];
#pragma unroll 1
  for (int il = w; il < TP; il += 8) {
    const int i = i0 + il;
    if (i >= M) break;
    float a = 0;
    const float4* t4 = reinterpret_cast<const float4*>(ts[il]);
#pragma unroll
    for (int k4 = 0; k4 < FK / 2; ++k4) {
      const float4 q = t4[k4];
      a = fmaf(g[2 * k4].x, q.x, a);
      a = fmaf(g[2 * k4].y, q.y, a);
      a = fmaf(g[2 * k4 + 1].x, q.z, a);
      a = fmaf(g[2 * k4 + 1].y, q.w, a);
    }
    const float4* d4 = reinterpret_cast<const float4*>(ds[il]);
#pragma unroll
    for (int o4 = 0; o4 < FC / 4; ++o4) {
      const float4 v = d4[o4];
      a = fmaf(wc[4 * o4], v.x, a);
      a = fmaf(wc[4 * o4 + 1], v.y, a);
      a = fmaf(wc[4 * o4 + 2], v.z, a);
      a = fmaf(wc[4 * o4 + 3], v.w, a);
    }
    dhp[((size_t)s * M + i) * FC + c] = a;
  }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       bf16* __restrict__ p16, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float gt = g[t];
  const float mt = b1 * m[t] + (1 - b1) * gt, vt = b2 * v[t] + (1 - b2) * gt * gt;
  m[t] = mt;
  v[t] = vt;
  const float pt = p[t] - lr * (mt / c1) / (sqrtf(vt / c2) + eps);
  p[t] = pt;
  p16[t] = __float2bfloat16(pt);
}

__global__ void k_to_bf16(const float* __restrict__ p, bf16* __restrict__ p16, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) p16[t] = __float2bfloat16(p[t]);
}

inline unsigned nblk(size_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// Batch gather for aao_fno_train: sample j of the batch is pair idx[j] of the training set.
__global__ void k_gather_pairs(const float2* __restrict__ b, const float2* __restrict__ x,
                               const double2* __restrict__ lam, const float* __restrict__ alpha,
                               const int64_t* __restrict__ idx, int M, int B, float2* __restrict__ gb,
                               float2* __restrict__ gx, double2* __restrict__ glam, float* __restrict__ galpha) {
  const int j = blockIdx.y;
  const int64_t src = idx[j];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    gb[(size_t)j * M + i] = b[(size_t)src * M + i];
    gx[(size_t)j * M + i] = x[(size_t)src * M + i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    glam[j] = lam[src];
    galpha[j] = alpha[src];
  }
}

}  // namespace

}  // namespace aao

using aao::bf16;

struct aao_fno {
  int M = 0, maxB = 0;
  int64_t steps = 0;
  float *P32 = nullptr, *G32 = nullptr, *Am = nullptr, *Av = nullptr;
  bf16* P16 = nullptr;
  float2* tw = nullptr;
  float *feat = nullptr, *h[aao::FL + 1] = {}, *z[aao::FL] = {}, *y = nullptr, *dy = nullptr, *dh = nullptr,
        *dz = nullptr, *dh2 = nullptr, *norms = nullptr, *loss = nullptr;
  float2 *H[aao::FL] = {}, *G = nullptr, *gG = nullptr, *gH = nullptr, *part = nullptr;
  float* opart = nullptr;  // weight-gradient block partials
  int nch = 0;  // DFT chunks of aao::DT points
  // batch gather buffers of aao_fno_train (allocated on its first shuffled call)
  float2 *gb = nullptr, *gx = nullptr;
  double2* glam = nullptr;
  float* galpha = nullptr;
  int64_t* gidx = nullptr;
  size_t gidx_cap = 0;
  std::vector<void*> allocs;
  std::string err;
};

namespace {

aao_status ffail(aao_fno* f, aao_status st, const std::string& m) {
  if (f) f->err = m;
  aao::set_planless_error(m);
  return st;
}

#define FCK(call)                                                                                 \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return ffail(f, AAO_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
aao_status falloc(aao_fno* f, T** p, size_t n) {
  void* q = nullptr;
  if (cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) return ffail(f, AAO_ENOMEM, "cudaMalloc failed");
  f->allocs.push_back(q);
  *p = (T*)q;
  return AAO_OK;
}

// forward pass on B samples; fills f->y (and every cached activation)
aao_status fno_forward(aao_fno* f, int B, const float2* b, const double2* lam, const float* alpha, cudaStream_t s) {
  using namespace aao;
  const int M = f->M;
  const size_t N = (size_t)B * M;
  const dim3 tiles(f->nch, B);
  k_norms<<<B, 256, 0, s>>>(b, M, f->norms);
  k_lift_dft<<<tiles, 256, 0, s>>>(b, lam, alpha, f->norms, f->P16, M, f->tw, f->feat, f->h[0], f->part, f->nch);
  for (int l = 0; l < FL; ++l) {
    k_mix<<<dim3(FK, (B + MIX_S - 1) / MIX_S), 512, 0, s>>>(f->part, f->nch, f->H[l], f->P16, off_R(l), B, M, f->G,
                                                            0, 0);
    const bool last = l == FL - 1;
    k_inv_pw<<<tiles, 256, 0, s>>>(f->G, f->h[l], f->P16, off_W(l), off_b(l), M, f->tw, f->z[l], f->h[l + 1],
                                   !last, last ? nullptr : f->part, f->nch);
  }
  k_proj<<<nblk(N), 256, 0, s>>>(f->h[FL], f->P16, N, f->y);
  FCK(cudaGetLastError());
  return AAO_OK;
}

aao_status fno_backward(aao_fno* f, int B, cudaStream_t s) {
  using namespace aao;
  const int M = f->M;
  const size_t N = (size_t)B * M;
  // about four 32-point tiles per block, at most OUTER_MAX_BLOCKS blocks
  const int go = (int)std::max<size_t>(1, std::min<size_t>(OUTER_MAX_BLOCKS, (N + 127) / 128));
  const int gs = (OUTER_PART + 31) / 32;
  auto outer = [&](const float* A, int na, const float* Bm, int nb, int offg, int offb) {
    k_outer<<<go, 256, 0, s>>>(A, na, Bm, nb, N, f->opart);
    k_outer_sum<<<gs, 1024, 0, s>>>(f->opart, go, na, nb, f->G32 + offg, f->G32 + offb);
  };
  FCK(cudaMemsetAsync(f->G32, 0, (size_t)NPARAM * sizeof(float), s));
  outer(f->dy, 2, f->h[FL], FC, OFF_PW, OFF_PB);
  k_proj_back<<<nblk(N * FC), 256, 0, s>>>(f->dy, f->P16, N, f->dh);
  for (int l = FL - 1; l >= 0; --l) {
    k_act_back<<<nblk(N * FC), 256, 0, s>>>(f->dh, f->z[l], f->dz, N * FC, l < FL - 1);
    outer(f->dz, FC, f->h[l], FC, off_W(l), off_b(l));
    k_dft<<<dim3(f->nch, B), 256, 0, s>>>(f->dz, M, f->tw, f->part, f->nch);
    k_mix<<<dim3(FK, (B + MIX_S - 1) / MIX_S), 512, 0, s>>>(f->part, f->nch, f->gG, f->P16, off_R(l), B, M, f->gH,
                                                            1, 1);
    k_gR<<<FK, 1024, 0, s>>>(f->gG, f->H[l], B, f->G32 + off_R(l));
    k_back_pw_idft<<<dim3((M + TP - 1) / TP, B), 256, 0, s>>>(f->dz, f->gH, f->P16, off_W(l), M, f->tw, f->dh2);
    std::swap(f->dh, f->dh2);
  }
  outer(f->dh, FC, f->feat, FF, OFF_LW, OFF_LB);
  FCK(cudaGetLastError());
  return AAO_OK;
}

aao_status check_batch(aao_fno* f, int B) {
  if (!f) return ffail(nullptr, AAO_EINVAL, "null FNO");
  if (B < 1 || B > f->maxB) return ffail(f, AAO_EINVAL, "batch size must be in [1, max_batch]");
  return AAO_OK;
}

}  // namespace

extern "C" {

int64_t aao_fno_num_params(void) { return aao::NPARAM; }

aao_status aao_fno_create(int64_t M, int max_batch, uint64_t seed, aao_fno** out) {
  using namespace aao;
  if (!out) return ffail(nullptr, AAO_EINVAL, "out is NULL");
  *out = nullptr;
  if (M < 2 * FK || M > 8191 || max_batch < 1) return ffail(nullptr, AAO_EINVAL, "need 32 <= M <= 8191, max_batch >= 1");
  aao_fno* f = new aao_fno();
  f->M = (int)M;
  f->maxB = max_batch;
  auto bail = [&](aao_status st) {
    aao_fno_destroy(f);
    return st;
  };
#define FTRY(x)                        \
  do {                                 \
    aao_status s_ = (x);               \
    if (s_ != AAO_OK) return bail(s_); \
  } while (0)
  const size_t N = (size_t)max_batch * M;
  FTRY(falloc(f, &f->P32, NPARAM));
  FTRY(falloc(f, &f->G32, NPARAM));
  FTRY(falloc(f, &f->Am, NPARAM));
  FTRY(falloc(f, &f->Av, NPARAM));
  FTRY(falloc(f, &f->P16, NPARAM));
  FTRY(falloc(f, &f->tw, (size_t)FK * M));
  FTRY(falloc(f, &f->feat, N * FF));
  for (int l = 0; l <= FL; ++l) FTRY(falloc(f, &f->h[l], N * FC));
  for (int l = 0; l < FL; ++l) {
    FTRY(falloc(f, &f->z[l], N * FC));
    FTRY(falloc(f, &f->H[l], (size_t)max_batch * FK * FC));
  }
  FTRY(falloc(f, &f->G, (size_t)max_batch * FK * FC));
  f->nch = (int)((M + DT - 1) / DT);
  FTRY(falloc(f, &f->part, (size_t)max_batch * f->nch * FK * FC));
  FTRY(falloc(f, &f->opart, (size_t)OUTER_MAX_BLOCKS * OUTER_PART));
  FTRY(falloc(f, &f->gG, (size_t)max_batch * FK * FC));
  FTRY(falloc(f, &f->gH, (size_t)max_batch * FK * FC));
  FTRY(falloc(f, &f->y, N * 2));
  FTRY(falloc(f, &f->dy, N * 2));
  FTRY(falloc(f, &f->dh, N * FC));
  FTRY(falloc(f, &f->dz, N * FC));
  FTRY(falloc(f, &f->dh2, N * FC));
  FTRY(falloc(f, &f->norms, (size_t)max_batch));
  FTRY(falloc(f, &f->loss, (size_t)max_batch));
  // tw[i][k] = exp(-2 pi i i k / M), point-major, in FP64 on the host
  std::vector<float2> tw((size_t)FK * M);
  for (int k = 0; k < FK; ++k)
    for (int i = 0; i < M; ++i) {
      const double a = -2.0 * 3.14159265358979323846 * (double)(((int64_t)i * k) % M) / (double)M;
      tw[(size_t)i * FK + k] = float2{(float)std::cos(a), (float)std::sin(a)};
    }
  if (cudaMemcpy(f->tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(ffail(f, AAO_ECUDA, "cudaMemcpy failed"));
  // scaled Gaussian initialisation (fan-in), biases zero; Box-Muller on a SplitMix64 stream
  std::vector<float> p(NPARAM, 0.0f);
  uint64_t st = seed;
  auto next_u = [&]() {
    uint64_t x = (st += 0x9E3779B97F4A7C15ull);
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    return ((x >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  };
  auto gauss = [&]() { return std::sqrt(-2.0 * std::log(next_u())) * std::cos(2.0 * 3.14159265358979323846 * next_u()); };
  for (int q = 0; q < FC * FF; ++q) p[OFF_LW + q] = (float)(gauss() / std::sqrt((double)FF));
  for (int l = 0; l < FL; ++l) {
    for (int q = 0; q < FK * FC * FC * 2; ++q) p[off_R(l) + q] = (float)(gauss() / (FC * std::sqrt(2.0)));
    for (int q = 0; q < FC * FC; ++q) p[off_W(l) + q] = (float)(gauss() / std::sqrt((double)FC));
  }
  for (int q = 0; q < 2 * FC; ++q) p[OFF_PW + q] = (float)(gauss() / std::sqrt((double)FC));
  aao_status s2 = aao_fno_set_params(f, p.data());
  if (s2 != AAO_OK) return bail(s2);
#undef FTRY
  *out = f;
  return AAO_OK;
}

aao_status aao_fno_destroy(aao_fno* f) {
  if (!f) return AAO_OK;
  for (void* q : f->allocs) cudaFree(q);
  delete f;
  return AAO_OK;
}

aao_status aao_fno_set_params(aao_fno* f, const float* host) {
  if (!f || !host) return ffail(f, AAO_EINVAL, "null argument");
  FCK(cudaMemcpy(f->P32, host, (size_t)aao::NPARAM * sizeof(float), cudaMemcpyHostToDevice));
  FCK(cudaMemset(f->Am, 0, (size_t)aao::NPARAM * sizeof(float)));
  FCK(cudaMemset(f->Av, 0, (size_t)aao::NPARAM * sizeof(float)));
  f->steps = 0;
  aao::k_to_bf16<<<aao::nblk(aao::NPARAM), 256>>>(f->P32, f->P16, aao::NPARAM);
  FCK(cudaGetLastError());
  FCK(cudaDeviceSynchronize());
  return AAO_OK;
}

aao_status aao_fno_get_params(aao_fno* f, float* host, int bf16_rounded) {
  if (!f || !host) return ffail(f, AAO_EINVAL, "null argument");
  FCK(cudaDeviceSynchronize());
  if (!bf16_rounded) {
    FCK(cudaMemcpy(host, f->P32, (size_t)aao::NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    return AAO_OK;
  }
  std::vector<bf16> t(aao::NPARAM);
  FCK(cudaMemcpy(t.data(), f->P16, t.size() * sizeof(bf16), cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < t.size(); ++i) host[i] = __bfloat162float(t[i]);
  return AAO_OK;
}

aao_status aao_fno_predict(aao_fno* f, int B, const void* b, const void* lambda, const float* alpha, void* x0,
                           void* stream) {
  aao_status st = check_batch(f, B);
  if (st != AAO_OK) return st;
  if (!b || !lambda || !alpha || !x0) return ffail(f, AAO_EINVAL, "null pointer");
  cudaStream_t s = (cudaStream_t)stream;
  st = fno_forward(f, B, (const float2*)b, (const double2*)lambda, alpha, s);
  if (st != AAO_OK) return st;
  const size_t N = (size_t)B * f->M;
  aao::k_output<<<aao::nblk(N), 256, 0, s>>>(f->y, f->norms, f->M, N, (float2*)x0);
  FCK(cudaGetLastError());
  return AAO_OK;
}

aao_status aao_fno_loss_grad(aao_fno* f, int B, const void* b, const void* lambda, const float* alpha,
                             const void* x_true, double* loss, float* grad_host, void* stream) {
  aao_status st = check_batch(f, B);
  if (st != AAO_OK) return st;
  if (!b || !lambda || !alpha || !x_true) return ffail(f, AAO_EINVAL, "null pointer");
  cudaStream_t s = (cudaStream_t)stream;
  st = fno_forward(f, B, (const float2*)b, (const double2*)lambda, alpha, s);
  if (st != AAO_OK) return st;
  aao::k_loss<<<B, 256, 0, s>>>(f->y, (const float2*)x_true, f->norms, f->M, B, f->dy, f->loss);
  st = fno_backward(f, B, s);
  if (st != AAO_OK) return st;
  if (loss) {
    std::vector<float> l(B);
    FCK(cudaMemcpyAsync(l.data(), f->loss, B * sizeof(float), cudaMemcpyDeviceToHost, s));
    FCK(cudaStreamSynchronize(s));
    double a = 0;
    for (float v : l) a += v;
    *loss = a / B;
  }
  if (grad_host) {
    FCK(cudaMemcpyAsync(grad_host, f->G32, (size_t)aao::NPARAM * sizeof(float), cudaMemcpyDeviceToHost, s));
    FCK(cudaStreamSynchronize(s));
  }
  return AAO_OK;
}

}  // extern "C"

namespace {
// One Adam step on B samples without host synchronisation; the per-sample losses of the batch
// (before the step) are copied to loss_out (device, B floats) when it is not NULL.
aao_status fno_train_step_dev(aao_fno* f, int B, const float2* b, const double2* lam, const float* alpha,
                              const float2* x_true, float lr, float* loss_out, cudaStream_t s) {
  aao_status st = fno_forward(f, B, b, lam, alpha, s);
  if (st != AAO_OK) return st;
  aao::k_loss<<<B, 256, 0, s>>>(f->y, x_true, f->norms, f->M, B, f->dy, f->loss);
  st = fno_backward(f, B, s);
  if (st != AAO_OK) return st;
  if (loss_out) FCK(cudaMemcpyAsync(loss_out, f->loss, (size_t)B * sizeof(float), cudaMemcpyDeviceToDevice, s));
  f->steps++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - std::pow(b1, (float)f->steps), c2 = 1.0f - std::pow(b2, (float)f->steps);
  aao::k_adam<<<aao::nblk(aao::NPARAM), 256, 0, s>>>(f->P32, f->G32, f->Am, f->Av, f->P16, aao::NPARAM, lr, b1, b2,
                                                     1e-8f, c1, c2);
  FCK(cudaGetLastError());
  return AAO_OK;
}
}  // namespace

extern "C" {

aao_status aao_fno_train_step(aao_fno* f, int B, const void* b, const void* lambda, const float* alpha,
                              const void* x_true, float lr, double* loss, void* stream) {
  aao_status st = aao_fno_loss_grad(f, B, b, lambda, alpha, x_true, loss, nullptr, stream);
  if (st != AAO_OK) return st;
  f->steps++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - std::pow(b1, (float)f->steps), c2 = 1.0f - std::pow(b2, (float)f->steps);
  aao::k_adam<<<aao::nblk(aao::NPARAM), 256, 0, (cudaStream_t)stream>>>(f->P32, f->G32, f->Am, f->Av, f->P16,
                                                                        aao::NPARAM, lr, b1, b2, 1e-8f, c1, c2);
  FCK(cudaGetLastError());
  return AAO_OK;
}

aao_status aao_fno_train(aao_fno* f, int64_t n_pairs, const void* b, const void* lambda, const float* alpha,
                         const void* x_true, int steps, int batch, float lr0, uint64_t seed, double* losses_host,
                         void* stream) {
  aao_status st = check_batch(f, batch);
  if (st != AAO_OK) return st;
  if (!b || !lambda || !alpha || !x_true) return ffail(f, AAO_EINVAL, "null pointer");
  if (steps < 0 || n_pairs < batch) return ffail(f, AAO_EINVAL, "need steps >= 0 and n_pairs >= batch");
  if (steps == 0) return AAO_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int M = f->M;
  const float2* bp = (const float2*)b;
  const float2* xp = (const float2*)x_true;
  const double2* lp = (const double2*)lambda;
  // per-sample losses of every step stay on the device until the end (no synchronisation per step)
  float* loss_dev = nullptr;
  if (losses_host && cudaMalloc(&loss_dev, (size_t)steps * batch * sizeof(float)) != cudaSuccess)
    return ffail(f, AAO_ENOMEM, "cudaMalloc failed");
  auto release = [&](aao_status r) {
    if (loss_dev) cudaFree(loss_dev);
    return r;
  };
  // seed != 0: batches are gathered through a per-epoch permutation (Fisher-Yates on SplitMix64)
  std::vector<int64_t> perm;
  const int64_t per_epoch = n_pairs / batch;
  if (seed != 0) {
    if (!f->gb) {
      const size_t N = (size_t)f->maxB * M;
      if (falloc(f, &f->gb, N) != AAO_OK || falloc(f, &f->gx, N) != AAO_OK ||
          falloc(f, &f->glam, (size_t)f->maxB) != AAO_OK || falloc(f, &f->galpha, (size_t)f->maxB) != AAO_OK)
        return release(ffail(f, AAO_ENOMEM, "cudaMalloc failed"));
    }
    if (f->gidx_cap < (size_t)n_pairs) {  // index buffers of earlier calls stay in f->allocs until destroy
      if (falloc(f, &f->gidx, (size_t)n_pairs) != AAO_OK) return release(ffail(f, AAO_ENOMEM, "cudaMalloc failed"));
      f->gidx_cap = (size_t)n_pairs;
    }
    perm.resize((size_t)n_pairs);
  }
  uint64_t rng = seed;
  auto next = [&]() {
    uint64_t z = (rng += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  const double pi = 3.14159265358979323846;
  for (int t = 0; t < steps; ++t) {
    const float lr = (float)(lr0 * 0.5 * (1.0 + std::cos(pi * t / steps)));
    float* lo = loss_dev ? loss_dev + (size_t)t * batch : nullptr;
    if (seed == 0) {
      const int64_t o = ((int64_t)t * batch) % (n_pairs - batch + (n_pairs == batch ? 1 : 0));
      st = fno_train_step_dev(f, batch, bp + (size_t)o * M, lp + o, alpha + o, xp + (size_t)o * M, lr, lo, s);
    } else {
      const int64_t k = t % per_epoch;
      if (k == 0) {  // a new epoch: a fresh permutation of all pairs
        for (int64_t i = 0; i < n_pairs; ++i) perm[(size_t)i] = i;
        for (int64_t i = n_pairs - 1; i > 0; --i) std::swap(perm[(size_t)i], perm[(size_t)(next() % (uint64_t)(i + 1))]);
        // pageable copy: staged before cudaMemcpyAsync returns, so perm may change afterwards
        if (cudaMemcpyAsync(f->gidx, perm.data(), (size_t)n_pairs * sizeof(int64_t), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
          return release(ffail(f, AAO_ECUDA, "cudaMemcpyAsync failed"));
      }
      aao::k_gather_pairs<<<dim3((M + 255) / 256, batch), 256, 0, s>>>(bp, xp, lp, alpha, f->gidx + k * batch, M,
                                                                       batch, f->gb, f->gx, f->glam, f->galpha);
      st = fno_train_step_dev(f, batch, f->gb, f->glam, f->galpha, f->gx, lr, lo, s);
    }
    if (st != AAO_OK) return release(st);
  }
  if (losses_host) {
    std::vector<float> l((size_t)steps * batch);
    if (cudaMemcpyAsync(l.data(), loss_dev, l.size() * sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return release(ffail(f, AAO_ECUDA, "loss readback failed"));
    for (int t = 0; t < steps; ++t) {  // the batch mean of aao_fno_loss_grad, summed in the same order
      double a = 0;
      for (int j = 0; j < batch; ++j) a += l[(size_t)t * batch + j];
      losses_host[t] = a / batch;
    }
  }
  return release(AAO_OK);
}

aao_status aao_fno_save(aao_fno* f, const char* path) {
  if (!f || !path) return ffail(f, AAO_EINVAL, "null argument");
  std::vector<float> p(aao::NPARAM);
  aao_status st = aao_fno_get_params(f, p.data(), 0);
  if (st != AAO_OK) return st;
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return ffail(f, AAO_EINVAL, std::string("cannot open ") + path);
  char head[256];
  std::snprintf(head, sizeof head,
                "{\"format\": \"aao-fno\", \"version\": 1, \"width\": %d, \"modes\": %d, \"layers\": %d, "
                "\"features\": %d, \"num_params\": %d, \"M\": %d, \"adam_steps\": %lld, \"dtype\": \"float32le\"}\n",
                aao::FC, aao::FK, aao::FL, aao::FF, aao::NPARAM, f->M, (long long)f->steps);
  bool ok = std::fputs(head, fp) >= 0;
  // little-endian float32 regardless of the host's byte order
  std::vector<unsigned char> raw((size_t)aao::NPARAM * 4);
  for (int i = 0; i < aao::NPARAM; ++i) {
    uint32_t u;
    std::memcpy(&u, &p[i], 4);
    for (int b = 0; b < 4; ++b) raw[(size_t)i * 4 + b] = (unsigned char)(u >> (8 * b));
  }
  ok = ok && std::fwrite(raw.data(), 1, raw.size(), fp) == raw.size();
  ok = (std::fclose(fp) == 0) && ok;
  if (!ok) return ffail(f, AAO_EINVAL, std::string("write failed: ") + path);
  return AAO_OK;
}

aao_status aao_fno_load(aao_fno* f, const char* path) {
  if (!f || !path) return ffail(f, AAO_EINVAL, "null argument");
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return ffail(f, AAO_EINVAL, std::string("cannot open ") + path);
  std::string head;
  int c;
  while ((c = std::fgetc(fp)) != EOF && c != '\n' && head.size() < 4096) head.push_back((char)c);
  auto field = [&](const char* key) -> long long {
    const std::string k = std::string("\"") + key + "\":";
    const size_t at = head.find(k);
    if (at == std::string::npos) return -1;
    return std::atoll(head.c_str() + at + k.size());
  };
  const bool hdr_ok = c == '\n' && head.find("\"aao-fno\"") != std::string::npos && field("version") == 1 &&
                      field("width") == aao::FC && field("modes") == aao::FK && field("layers") == aao::FL &&
                      field("features") == aao::FF && field("num_params") == aao::NPARAM;
  std::vector<unsigned char> raw((size_t)aao::NPARAM * 4);
  const bool body_ok = hdr_ok && std::fread(raw.data(), 1, raw.size(), fp) == raw.size() && std::fgetc(fp) == EOF;
  std::fclose(fp);
  if (!body_ok) return ffail(f, AAO_EINVAL, std::string("not an aao-fno weight file of this architecture: ") + path);
  std::vector<float> p(aao::NPARAM);
  for (int i = 0; i < aao::NPARAM; ++i) {
    uint32_t u = 0;
    for (int b = 0; b < 4; ++b) u |= (uint32_t)raw[(size_t)i * 4 + b] << (8 * b);
    std::memcpy(&p[i], &u, 4);
  }
  return aao_fno_set_params(f, p.data());
}

}  // extern "C"

namespace aao {
int fno_grid_size(const aao_fno* f) { return f ? f->M : 0; }
int fno_max_batch(const aao_fno* f) { return f ? f->maxB : 0; }
}  // namespace aao
