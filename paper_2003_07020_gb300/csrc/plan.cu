// The C ABI of include/aao.h: plan creation (host FP64 setup + device
// workspace), the three hot-path calls, and the restarted flexible GMRES
// driver (Sec. 4: right preconditioning, x0 = 0, stopping on the true
// relative residual).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <map>
#include <mutex>
#include <tuple>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/aao.h"
#include "kernels.h"
#include "setup.h"

extern "C" int aao_setup_coeffs_impl(double alpha, int64_t n, double* g);

namespace {

thread_local std::string g_create_error;

constexpr int kMaxRestart = 64;

__global__ void iter_stats_kernel(const int* __restrict__ iters, const int* __restrict__ flags, int n,
                                  int* __restrict__ out) {
  __shared__ int smax[256], fmax_[256], ssum[256], sacc[256];
  int a = 0, b = 0, c = 0, d = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    a = max(a, iters[i]);
    b = max(b, flags[i] & 3);
    c += iters[i];
    d += (flags[i] >> 2) & 1;  // warm start accepted
  }
  smax[threadIdx.x] = a;
  fmax_[threadIdx.x] = b;
  ssum[threadIdx.x] = c;
  sacc[threadIdx.x] = d;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      smax[threadIdx.x] = max(smax[threadIdx.x], smax[threadIdx.x + o]);
      fmax_[threadIdx.x] = max(fmax_[threadIdx.x], fmax_[threadIdx.x + o]);
      ssum[threadIdx.x] += ssum[threadIdx.x + o];
      sacc[threadIdx.x] += sacc[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { out[0] = smax[0]; out[1] = fmax_[0]; out[2] = ssum[0]; out[3] = sacc[0]; }
}

// ---- graph-captured restart cycles ---------------------------------------------------------
// Device copy of the FGMRES recurrences of one restart cycle (Givens rotations,
// residual estimate, least-squares solution), so that a whole cycle runs as one
// CUDA graph whose Arnoldi steps are conditional nodes.
struct GmresDevState {
  double H[(kMaxRestart + 1) * kMaxRestart];  // H[i * kMaxRestart + j]
  double cs[kMaxRestart], sn[kMaxRestart], g[kMaxRestart + 1], y[kMaxRestart];
  double thr;                                 // 0.5 * tol * ||F||: stop when |g[j+1]| <= thr
  double inv_beta, inv_hn;
  int jdone, active, status, outer_total;
  int inner_max, flag_max;
  long long inner_sum, accepted;
};

// Start of a cycle: g = (beta, 0, ...), beta^2 = *beta2 from the residual reduction; enables step 0.
__global__ void cycle_init_kernel(GmresDevState* d, const double* beta2, int m, cudaGraphConditionalHandle h,
                                  int set_cond) {
  if (threadIdx.x != 0) return;
  const double beta = sqrt(*beta2);
  for (int i = 0; i <= m; ++i) d->g[i] = 0.0;
  d->g[0] = beta;
  d->inv_beta = 1.0 / beta;
  d->jdone = 0;
  d->active = 1;
  d->status = 0;
  if (set_cond) cudaGraphSetConditional(h, 1u);
}

// Column j of H from the two Gram-Schmidt passes (hd[i] + hd[65 + i], norm^2 in hd[130]),
// the previous rotations, a new rotation and the residual estimate |g[j+1]|; enables step
// j + 1 (its conditional handle h_next, when has_next) unless the cycle stops here.
__global__ void givens_kernel(GmresDevState* d, const double* hd, int j, int m, cudaGraphConditionalHandle h_next,
                              int has_next) {
  if (threadIdx.x != 0) return;
  double* H = d->H;
  auto at = [&](int i, int k) -> double& { return H[i * kMaxRestart + k]; };
  for (int i = 0; i <= j; ++i) at(i, j) = hd[i] + hd[65 + i];
  const double hn = sqrt(hd[130]);
  at(j + 1, j) = hn;
  bool stop = false;
  if (!isfinite(hn)) {
    d->status = AAO_ENONFINITE;
    stop = true;
  } else {
    d->inv_hn = hn > 0 ? 1.0 / hn : 0.0;
    for (int i = 0; i < j; ++i) {
      const double t = d->cs[i] * at(i, j) + d->sn[i] * at(i + 1, j);
      at(i + 1, j) = -d->sn[i] * at(i, j) + d->cs[i] * at(i + 1, j);
      at(i, j) = t;
    }
    const double dd = hypot(at(j, j), at(j + 1, j));
    if (dd == 0.0) {
      d->status = AAO_EBREAKDOWN;
      stop = true;
    } else {
      d->cs[j] = at(j, j) / dd;
      d->sn[j] = at(j + 1, j) / dd;
      at(j, j) = dd;
      at(j + 1, j) = 0.0;
      d->g[j + 1] = -d->sn[j] * d->g[j];
      d->g[j] = d->cs[j] * d->g[j];
      d->outer_total++;
      d->jdone = j + 1;
      if (fabs(d->g[j + 1]) <= d->thr || hn == 0.0 || j + 1 == m) stop = true;
    }
  }
  if (stop) d->active = 0;
  if (has_next) cudaGraphSetConditional(h_next, stop ? 0u : 1u);
}

// y = H(0:jdone, 0:jdone)^{-1} g by back substitution (upper triangular after the rotations)
__global__ void lsq_kernel(GmresDevState* d) {
  if (threadIdx.x != 0 || d->status != 0) return;
  const int jd = d->jdone;
  for (int i = jd - 1; i >= 0; --i) {
    double s = d->g[i];
    for (int k = i + 1; k < jd; ++k) s -= d->H[i * kMaxRestart + k] * d->y[k];
    d->y[i] = s / d->H[i * kMaxRestart + i];
  }
}

// COCG iteration statistics of one preconditioner application, accumulated on the device
__global__ void iter_stats_accum_kernel(const int* __restrict__ iters, const int* __restrict__ flags, int n,
                                        GmresDevState* d) {
  __shared__ int smax[256], fmax_[256], ssum[256], sacc[256];
  int a = 0, b = 0, c = 0, e = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    a = max(a, iters[i]);
    b = max(b, flags[i] & 3);
    c += iters[i];
    e += (flags[i] >> 2) & 1;
  }
  smax[threadIdx.x] = a;
  fmax_[threadIdx.x] = b;
  ssum[threadIdx.x] = c;
  sacc[threadIdx.x] = e;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      smax[threadIdx.x] = max(smax[threadIdx.x], smax[threadIdx.x + o]);
      fmax_[threadIdx.x] = max(fmax_[threadIdx.x], fmax_[threadIdx.x + o]);
      ssum[threadIdx.x] += ssum[threadIdx.x + o];
      sacc[threadIdx.x] += sacc[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    d->inner_max = max(d->inner_max, smax[0]);
    if (d->flag_max == 0) d->flag_max = fmax_[0];
    d->inner_sum += ssum[0];
    d->accepted += sacc[0];
  }
}

}  // namespace

namespace aao {
// Error message for calls that have no plan (see aao_last_error(NULL)).
void set_planless_error(const std::string& msg) { g_create_error = msg; }
}  // namespace aao

struct aao_plan {
  aao_problem prob{};
  aao_opts opts{};
  cudaStream_t stream = nullptr;
  aao::HostTables ht;
  int M = 0, Nt = 0, logL = 0, nsys = 0, m = 0;
  size_t n = 0;
  // 2D (dim == 2): M is M_x; Msp = spatial unknowns per time level (M in 1D, M * My in 2D)
  int dim = 1, My = 1, logLy = 0;
  size_t Msp = 0;
  aao::HostTables hty;
  double2 *twy64 = nullptr, *Px = nullptr, *Zx = nullptr, *Qx = nullptr, *Tx = nullptr;
  float2* twy32 = nullptr;
  double *Exf64 = nullptr, *Eyf64 = nullptr, *sxn64 = nullptr, *syf64 = nullptr, *tmp2d = nullptr;
  float *Exf32 = nullptr, *Eyf32 = nullptr, *sxn32 = nullptr, *syf32 = nullptr;
  void* state2d = nullptr;
  double2* part2d = nullptr;
  int* active2d = nullptr;
  int* host_count = nullptr;
  // 2D Strang (BCCB) preconditioner: row spectra scratch [nsys][My][Lx] and the per-system spectra of
  // the BCCB inverses [nsys][Lx][Ly], complex in the plan's Step (b) precision
  void* W2d = nullptr;
  void* G2d = nullptr;
  // 2D COCG as a graph with a conditional WHILE loop (no host synchronisation per iteration)
  cudaStream_t cap3 = nullptr, c2d_cap = nullptr;
  cudaGraphExec_t c2d_exec = nullptr;
  int* c2d_it = nullptr;
  long long* c2d_loops = nullptr;  // device count of graph-driven COCG iterations
  long long c2d_loops_seen = 0;
  size_t nsq = 0;  // partial sums produced by the residual matvec
  bool mixed = true;
  std::vector<void*> allocs;
  size_t ws_bytes = 0;
  std::string err;
  // tables
  double* Ehalf = nullptr;
  double2* twL64 = nullptr;
  float2* twL32 = nullptr;
  double2* twNt64 = nullptr;
  float2* twNt32 = nullptr;
  double* Ebr64 = nullptr;
  float* Ebr32 = nullptr;
  double2* lambda = nullptr;
  double* sfwd64 = nullptr;
  double* sinv64 = nullptr;
  float* sfwd32 = nullptr;
  float* sinv32 = nullptr;
  double2* chirp64 = nullptr;
  float2* chirp32 = nullptr;
  double2* chat64 = nullptr;
  float2* chat32 = nullptr;
  double* seig64 = nullptr;
  float* seig32 = nullptr;
  double* tau64 = nullptr;
  float* tau32 = nullptr;
  // workspace
  double* V = nullptr;   // (m+1) x n; in the mixed path a float-float basis (float2 per element)
  double* W = nullptr;   // n: the new Arnoldi vector A z_j (and r_0) in FP64 before its CGS2 (mixed path)
  void* Z = nullptr;     // m x n, float (mixed) or double
  void* spec = nullptr;  // nsys x M complex
  void* rws = nullptr;
  void* pws = nullptr;
  double2* gbuf = nullptr;
  int cocg_grid = 0;
  int cocg_threads = 0;  // CTA size of the register-resident FP32 COCG kernel (0: not used)
  bool direct = false;     // Step (b) by the direct tau-matrix solve (AAO_INNER_TAU_DIRECT)
  double* polyw = nullptr; // n doubles: right-hand side of a Horner step of P_eps(m) (opts.poly_m > 0)
  float2* sconv = nullptr;  // mixed Strang: per-system spectra of (lambda_n I + c S)^{-1} as L-point circulants
  // Step (b) by the tensor-memory kernel (cocg_tm.cu): the spectra in the order of its fused pass
  bool tm = false;
  float2* sconv_tm = nullptr;
  float* Ebr_tm = nullptr;
  // exact-integer matvec (opts.matvec == AAO_MATVEC_NTT, 1D)
  bool ntt = false;
  aao::NttTables ntt_tab{};
  uint32_t* ntt_res = nullptr;  // 1D: 4 n residues + n int64 quantised entries; 2D: 2 x 4 n residues + n int64
  double* ntt_rowscale = nullptr;  // one scale per time row (1D) or per time level (2D)
  // exact-integer 2D matvec (opts.matvec == AAO_MATVEC_NTT, dim 2): ntt_tab holds the x stencil, this the y one
  bool ntt2d = false;
  aao::NttTables ntt_tab_y{};
  int* iters = nullptr;
  int* flags = nullptr;
  int* stats = nullptr;
  double* partial = nullptr;
  double* hdev = nullptr;   // 3 x kMaxVec doubles + y
  double* sq = nullptr;     // Nt row partials
  double* pinned = nullptr; // host pinned scratch
  double* Fh = nullptr;     // device copies for the host-buffer entry point
  double* Uh = nullptr;
  // tracing (aao_plan_set_profiling / aao_plan_get_profile)
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
  cudaEvent_t ev_open = nullptr;
  double prof_ms[AAO_NUM_STAGES] = {0};
  int64_t prof_launches[AAO_NUM_STAGES] = {0};
  // learned warm start (aao_plan_set_warm_start) and training-pair recording
  aao_fno* fno = nullptr;
  float2* x0buf = nullptr;
  float* fno_alpha = nullptr;
  float2 *rec_b = nullptr, *rec_x = nullptr;
  double2* rec_lam = nullptr;
  int64_t rec_cap = 0, rec_count = 0;
  // graph-captured restart cycles (opts.use_graphs)
  GmresDevState* gd = nullptr;
  GmresDevState* gd_host = nullptr;  // pinned mirror for the per-cycle readback
  cudaGraphExec_t cycle_exec = nullptr;
  cudaStream_t cap1 = nullptr, cap2 = nullptr;
  aao_fno* graph_fno = nullptr;      // warm-start model baked into cycle_exec
  int64_t step_launches[AAO_NUM_STAGES] = {0};
};

namespace {

aao_status fail(aao_plan* p, aao_status st, const std::string& msg) {
  if (p) p->err = msg;
  else g_create_error = msg;
  return st;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(p, AAO_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));          \
  } while (0)

enum { ST_MATVEC = 0, ST_TDFT_FWD = 1, ST_COCG = 2, ST_TDFT_INV = 3, ST_VEC = 4, ST_FNO = 5 };
constexpr int kFnoLaunches = 12;  // kernels of one aao_fno_predict

cudaEvent_t take_event(aao_plan* p) {
  if (!p->ev_pool.empty()) {
    cudaEvent_t e = p->ev_pool.back();
    p->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void prof_begin(aao_plan* p) {
  if (!p->prof_on) return;
  p->ev_open = take_event(p);
  cudaEventRecord(p->ev_open, p->stream);
}

void prof_end(aao_plan* p, int stage, int nkern) {
  p->prof_launches[stage] += nkern;
  if (!p->prof_on || !p->ev_open) return;
  cudaEvent_t e = take_event(p);
  cudaEventRecord(e, p->stream);
  p->ev_pending.push_back({stage, {p->ev_open, e}});
  p->ev_open = nullptr;
}

// Launch `call` (which enqueues nkern kernels) as part of stage `stage`.
#define LAUNCH(stage, nkern, call)       \
  do {                                   \
    prof_begin(p);                       \
    CK(call);                            \
    prof_end(p, stage, nkern);           \
  } while (0)

template <typename T>
aao_status dalloc(aao_plan* p, T** ptr, size_t count) {
  void* q = nullptr;
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) return fail(p, AAO_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  p->allocs.push_back(q);
  p->ws_bytes += bytes;
  *ptr = static_cast<T*>(q);
  return AAO_OK;
}

template <typename Td, typename Ts>
aao_status upload(aao_plan* p, Td** dst, const std::vector<Ts>& src) {
  std::vector<Td> tmp(src.size());
  for (size_t i = 0; i < src.size(); ++i) tmp[i] = (Td)src[i];
  aao_status st = dalloc(p, dst, tmp.size());
  if (st != AAO_OK) return st;
  CK(cudaMemcpy(*dst, tmp.data(), tmp.size() * sizeof(Td), cudaMemcpyHostToDevice));
  return AAO_OK;
}

template <typename Td>
aao_status upload_c(aao_plan* p, Td** dst, const std::vector<aao::cd>& src) {
  std::vector<Td> tmp(src.size());
  for (size_t i = 0; i < src.size(); ++i) {
    tmp[i].x = (decltype(tmp[i].x))src[i].real();
    tmp[i].y = (decltype(tmp[i].y))src[i].imag();
  }
  aao_status st = dalloc(p, dst, tmp.size());
  if (st != AAO_OK) return st;
  CK(cudaMemcpy(*dst, tmp.data(), tmp.size() * sizeof(Td), cudaMemcpyHostToDevice));
  return AAO_OK;
}

#define TRY(x)                         \
  do {                                 \
    aao_status s_ = (x);               \
    if (s_ != AAO_OK) return s_;       \
  } while (0)

// sum of the first cnt doubles of a device array of per-block partials -> host
aao_status reduce_to_host(aao_plan* p, const double* partials, int nblocks, int nv, double* host_out) {
  LAUNCH(ST_VEC, 1, aao::launch_reduce_partials(partials, nblocks, nv, p->hdev, p->stream));
  CK(cudaMemcpyAsync(p->pinned, p->hdev, nv * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  std::memcpy(host_out, p->pinned, nv * sizeof(double));
  return AAO_OK;
}

aao_status matvec_any(aao_plan* p, const void* v, bool v_is_f32, const double* rhs, double* w, double* sq) {
  if (p->dim == 2 && p->ntt2d) {
    if (v_is_f32)
      LAUNCH(ST_MATVEC, 4, aao::launch_matvec2d_ntt_fin((const float*)v, rhs, w, sq, p->M, p->My, p->Nt, p->logL,
                                                        p->logLy, p->ntt_tab, p->ntt_tab_y, p->ntt_res,
                                                        p->ntt_rowscale, p->stream));
    else
      LAUNCH(ST_MATVEC, 4, aao::launch_matvec2d_ntt((const double*)v, rhs, w, sq, p->M, p->My, p->Nt, p->logL,
                                                    p->logLy, p->ntt_tab, p->ntt_tab_y, p->ntt_res, p->ntt_rowscale,
                                                    p->stream));
    return AAO_OK;
  }
  if (p->dim == 2) {
    if (v_is_f32)
      LAUNCH(ST_MATVEC, 2, aao::launch_matvec2d_f64_fin((const float*)v, rhs, w, p->tmp2d, sq, p->M, p->My, p->Nt,
                                                        p->logL, p->logLy, p->twL64, p->twy64, p->Exf64, p->Eyf64,
                                                        p->stream));
    else
      LAUNCH(ST_MATVEC, 2, aao::launch_matvec2d_f64((const double*)v, rhs, w, p->tmp2d, sq, p->M, p->My, p->Nt,
                                                    p->logL, p->logLy, p->twL64, p->twy64, p->Exf64, p->Eyf64,
                                                    p->stream));
    return AAO_OK;
  }
  if (p->ntt) {
    if (v_is_f32)
      LAUNCH(ST_MATVEC, 3, aao::launch_matvec_ntt_fin((const float*)v, rhs, w, sq, p->M, p->Nt, p->logL, p->ntt_tab,
                                                      p->ntt_res, p->ntt_rowscale, p->stream));
    else
      LAUNCH(ST_MATVEC, 3, aao::launch_matvec_ntt((const double*)v, rhs, w, sq, p->M, p->Nt, p->logL, p->ntt_tab,
                                                  p->ntt_res, p->ntt_rowscale, p->stream));
    return AAO_OK;
  }
  if (v_is_f32)
    LAUNCH(ST_MATVEC, 1, aao::launch_matvec_f64_fin((const float*)v, rhs, w, sq, p->M, p->Nt, p->logL, p->Ehalf,
                                                    p->twL64, p->stream));
  else
    LAUNCH(ST_MATVEC, 1, aao::launch_matvec_f64((const double*)v, rhs, w, sq, p->M, p->Nt, p->logL, p->Ehalf,
                                                p->twL64, p->stream));
  return AAO_OK;
}

// out = P^{-1} v.  out_kind: 0 float (mixed Z basis), 1 double.
// Step (b) in 2D: all shifted systems by the batched COCG of twod.cu
template <typename R>
aao_status cocg2d_any(aao_plan* p, void* spec) {
  using C = typename aao::VecT<R>::c;
  aao::Cocg2dArgs<R> a{};
  a.X = (C*)spec;
  a.Rr = (C*)p->rws;
  a.P = (C*)p->Px;
  a.Z = (C*)p->Zx;
  a.Q = (C*)p->Qx;
  a.Tm = (C*)p->Tx;
  a.Mx = p->M;
  a.My = p->My;
  a.nsys = p->nsys;
  a.logLx = p->logL;
  a.logLy = p->logLy;
  if constexpr (sizeof(R) == 4) {
    a.twx = p->twL32; a.twy = p->twy32; a.Exf = p->Exf32; a.Eyf = p->Eyf32; a.sxn = p->sxn32; a.syf = p->syf32;
  } else {
    a.twx = p->twL64; a.twy = p->twy64; a.Exf = p->Exf64; a.Eyf = p->Eyf64; a.sxn = p->sxn64; a.syf = p->syf64;
  }
  a.lambda = p->lambda;
  a.state = p->state2d;
  a.part = p->part2d;
  a.active_count = p->active2d;
  a.host_count = p->host_count;
  a.iters = p->iters;
  a.flags = p->flags;
  a.tol = p->opts.inner_tol;
  a.maxit = p->opts.inner_maxit;
  a.it_dev = p->c2d_it;
  a.loops_total = p->c2d_loops;
  a.W2 = (C*)p->W2d;
  a.G2 = (const C*)p->G2d;
  if (p->direct) {
    prof_begin(p);
    cudaError_t e;
    if constexpr (sizeof(R) == 4) e = aao::launch_tau2d_direct_f32(a, p->stream);
    else e = aao::launch_tau2d_direct_f64(a, p->stream);
    if (e != cudaSuccess) return fail(p, AAO_ECUDA, std::string("tau2d direct: ") + cudaGetErrorString(e));
    prof_end(p, ST_COCG, 4);
    return AAO_OK;
  }
  auto capture = [&](cudaStream_t cs) {
    if constexpr (sizeof(R) == 4) return aao::capture_cocg2d_f32(a, cs, p->cap3);
    else return aao::capture_cocg2d_f64(a, cs, p->cap3);
  };
  if (p->prof_on) {  // host-driven iterations, so that every launch can be counted and timed
    int its = 0;
    prof_begin(p);
    cudaError_t e;
    if constexpr (sizeof(R) == 4) e = aao::launch_cocg2d_f32(a, p->stream, &its);
    else e = aao::launch_cocg2d_f64(a, p->stream, &its);
    if (e != cudaSuccess) return fail(p, AAO_ECUDA, std::string("cocg2d: ") + cudaGetErrorString(e));
    prof_end(p, ST_COCG, 7 + its * 9);
    return AAO_OK;
  }
  cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(p->stream, &cst));
  if (cst == cudaStreamCaptureStatusActive) {  // inside a restart-cycle graph: the loop becomes a WHILE node
    cudaError_t e = capture(p->stream);
    if (e != cudaSuccess) return fail(p, AAO_ECUDA, std::string("cocg2d capture: ") + cudaGetErrorString(e));
    prof_end(p, ST_COCG, 8);
    return AAO_OK;
  }
  if (!p->c2d_exec) {  // the standalone graph of the whole Step (b), built once per plan
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(p->c2d_cap, cudaStreamCaptureModeRelaxed));
    cudaError_t e = capture(p->c2d_cap);
    cudaError_t e2 = cudaStreamEndCapture(p->c2d_cap, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->c2d_exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      p->c2d_exec = nullptr;
      return fail(p, AAO_ECUDA, std::string("cocg2d graph: ") + cudaGetErrorString(e));
    }
  }
  LAUNCH(ST_COCG, 8, cudaGraphLaunch(p->c2d_exec, p->stream));
  return AAO_OK;
}

// out = P_eps^{-1} v (Steps (a)-(c)).  out_kind: 0 float (mixed Z basis), 1 double; v_ff: v is a
// float-float vector (the mixed Arnoldi basis).
aao_status precond_once(aao_plan* p, const double* v, void* out, int out_kind, bool v_ff) {
  const int Ms = (int)p->Msp;
  if (p->mixed) {
    float2* spec = (float2*)p->spec;
    if (v_ff)
      LAUNCH(ST_TDFT_FWD, 1, aao::launch_tdft_fwd_f32_ff((const float2*)(const void*)v, spec, Ms, p->Nt, p->sfwd32,
                                                         p->twNt32, p->stream));
    else
      LAUNCH(ST_TDFT_FWD, 1, aao::launch_tdft_fwd_f32(v, spec, Ms, p->Nt, p->sfwd32, p->twNt32, p->stream));
    if (p->dim == 2) {
      TRY(cocg2d_any<float>(p, spec));
    } else {
      aao::CocgTables32 tb{p->twL32, p->Ebr32, p->lambda, p->chirp32, p->chat32, p->seig32, p->tau32, p->sconv};
      const int64_t nrec = std::min<int64_t>(p->nsys, p->rec_cap - p->rec_count);
      if (nrec > 0) {
        CK(cudaMemcpyAsync(p->rec_b + p->rec_count * p->M, spec, nrec * p->M * sizeof(float2),
                           cudaMemcpyDeviceToDevice, p->stream));
        CK(cudaMemcpyAsync(p->rec_lam + p->rec_count, p->lambda, nrec * sizeof(double2), cudaMemcpyDeviceToDevice,
                           p->stream));
      }
      if (p->fno) {
        prof_begin(p);
        const aao_status fs = aao_fno_predict(p->fno, p->nsys, spec, p->lambda, p->fno_alpha, p->x0buf, p->stream);
        if (fs != AAO_OK) return fail(p, fs, std::string("warm start: ") + aao_last_error(nullptr));
        prof_end(p, ST_FNO, kFnoLaunches);
      }
      if (p->direct)
        LAUNCH(ST_COCG, 1, aao::launch_tau_direct_f32(spec, p->M, p->logL, p->nsys, tb, p->iters, p->flags,
                                                      p->stream));
      else if (p->tm && !p->fno)
        LAUNCH(ST_COCG, 1, aao::launch_cocg_tm(spec, p->M, p->logL, p->nsys,
                                               aao::CocgTmTables{p->twL32, p->Ebr_tm, p->sconv_tm, p->lambda},
                                               (float)p->opts.inner_tol, p->opts.inner_maxit, p->iters, p->flags,
                                               p->stream));
      else
        LAUNCH(ST_COCG, 1, aao::launch_cocg_f32(spec, (float2*)p->rws, (float2*)p->pws, p->M, p->logL, p->nsys,
                                                (int)p->opts.inner, tb, (float)p->opts.inner_tol,
                                                p->opts.inner_maxit, p->iters, p->flags, p->cocg_grid, p->stream,
                                                p->fno ? p->x0buf : nullptr, p->cocg_threads));
      if (nrec > 0) {
        CK(cudaMemcpyAsync(p->rec_x + p->rec_count * p->M, spec, nrec * p->M * sizeof(float2),
                           cudaMemcpyDeviceToDevice, p->stream));
        p->rec_count += nrec;
      }
    }
    if (out_kind == 0)
      LAUNCH(ST_TDFT_INV, 1, aao::launch_tdft_inv_f32(spec, (float*)out, Ms, p->Nt, p->sinv32, p->twNt32,
                                                      p->stream));
    else
      LAUNCH(ST_TDFT_INV, 1, aao::launch_tdft_inv_f32_to_f64(spec, (double*)out, Ms, p->Nt, p->sinv32,
                                                             p->twNt32, p->stream));
  } else {
    double2* spec = (double2*)p->spec;
    LAUNCH(ST_TDFT_FWD, 1, aao::launch_tdft_fwd_f64(v, spec, Ms, p->Nt, p->sfwd64, p->twNt64, p->stream));
    if (p->dim == 2) {
      TRY(cocg2d_any<double>(p, spec));
    } else {
      aao::CocgTables64 tb{p->twL64, p->Ebr64, p->lambda, p->chirp64, p->chat64, p->seig64, p->tau64};
      if (p->direct)
        LAUNCH(ST_COCG, 1, aao::launch_tau_direct_f64(spec, p->gbuf, p->M, p->logL, p->nsys, tb, p->iters, p->flags,
                                                      p->cocg_grid, p->stream));
      else
        LAUNCH(ST_COCG, 1, aao::launch_cocg_f64(spec, (double2*)p->rws, (double2*)p->pws, p->gbuf, p->M, p->logL,
                                                p->nsys, (int)p->opts.inner, tb, p->opts.inner_tol,
                                                p->opts.inner_maxit, p->iters, p->flags, p->cocg_grid, p->stream));
    }
    LAUNCH(ST_TDFT_INV, 1, aao::launch_tdft_inv_f64(spec, (double*)out, Ms, p->Nt, p->sinv64, p->twNt64,
                                                    p->stream));
  }
  return AAO_OK;
}

// out = P(m) v with P(m) = sum_{k<=m} (P_eps^{-1} S_eps)^k P_eps^{-1}, m = opts.poly_m, the polynomial
// preconditioner of Sec. 3.1 (the remark after Thm 3.1), by Horner's rule z <- P_eps^{-1} (v + S_eps z);
// S_eps = (C_eps - C) (x) I touches only time rows 0 and 1.  m = 0: out = P_eps^{-1} v.
aao_status precond_any(aao_plan* p, const double* v, void* out, int out_kind, bool v_ff = false) {
  TRY(precond_once(p, v, out, out_kind, v_ff));
  for (int k = 0; k < p->opts.poly_m; ++k) {
    LAUNCH(ST_VEC, 1, aao::launch_poly_rhs(p->polyw, v, v_ff, out, out_kind == 0, p->ht.eps, p->Msp, p->Nt,
                                           p->stream));
    TRY(precond_once(p, p->polyw, out, out_kind, false));
  }
  return AAO_OK;
}

aao_status arnoldi_orthogonalise(aao_plan* p, int j);

// One Arnoldi step j of FGMRES (Sec. 4): z_j = P^{-1} v_j (Steps (a)-(c)), COCG statistics
// (into p->stats, or accumulated into acc), w = calA z_j, and CGS2 against v_0..v_j:
// h1 = V^T w (p->hdev), w -= V h1, h2 = V^T w (p->hdev + 65), w -= V h2, ||w||^2 (p->hdev[130]).
aao_status arnoldi_step(aao_plan* p, int j, GmresDevState* acc) {
  const size_t n = p->n;
  double* vj = p->V + (size_t)j * n;
  void* zj = p->mixed ? (void*)((float*)p->Z + (size_t)j * n) : (void*)((double*)p->Z + (size_t)j * n);
  TRY(precond_any(p, vj, zj, p->mixed ? 0 : 1, p->mixed));
  if (acc)
    LAUNCH(ST_VEC, 1, (iter_stats_accum_kernel<<<1, 256, 0, p->stream>>>(p->iters, p->flags, p->nsys, acc),
                       cudaGetLastError()));
  else
    LAUNCH(ST_VEC, 1, (iter_stats_kernel<<<1, 256, 0, p->stream>>>(p->iters, p->flags, p->nsys, p->stats),
                       cudaGetLastError()));
  return arnoldi_orthogonalise(p, j);
}

// The rest of Arnoldi step j after z_j = P^{-1} v_j: w = calA z_j and CGS2 against v_0..v_j,
// h1 = V^T w (p->hdev), w -= V h1, h2 = V^T w (p->hdev + 65), w -= V h2, ||w||^2 (p->hdev[130]).
aao_status arnoldi_orthogonalise(aao_plan* p, int j) {
  const size_t n = p->n;
  const int nb = aao::blas_partial_blocks();
  double* w = p->V + (size_t)(j + 1) * n;
  void* zj = p->mixed ? (void*)((float*)p->Z + (size_t)j * n) : (void*)((double*)p->Z + (size_t)j * n);
  const int nv = j + 1;
  if (p->mixed) {  // float-float basis: w = A z_j into W (FP64), CGS2 writes v_{j+1} as float-float
    const float2* Vf = (const float2*)(const void*)p->V;
    float2* wf = (float2*)(void*)w;
    if (p->ntt) {  // 1D: pass-1 dots fused into the matvec epilogue (one read of w less)
      LAUNCH(ST_MATVEC, 3, aao::launch_matvec_ntt_fin_dots((const float*)zj, p->W, p->M, p->Nt, p->logL, p->ntt_tab,
                                                           p->ntt_res, p->ntt_rowscale, Vf, n, nv, p->partial,
                                                           p->stream));
      LAUNCH(ST_VEC, 1, aao::launch_reduce_partials(p->partial, (int)p->nsq, nv, p->hdev, p->stream));
    } else {
      TRY(matvec_any(p, zj, true, nullptr, p->W, nullptr));
      LAUNCH(ST_VEC, 1, aao::launch_dots_ff(p->W, Vf, n, nv, n, p->partial, p->stream));
      LAUNCH(ST_VEC, 1, aao::launch_reduce_partials(p->partial, nb, nv, p->hdev, p->stream));
    }
    LAUNCH(ST_VEC, 1, aao::launch_update_dots_ff(p->W, wf, Vf, n, nv, n, p->hdev, p->partial, p->stream));
    LAUNCH(ST_VEC, 1, aao::launch_reduce_partials(p->partial, nb, nv, p->hdev + 65, p->stream));
    LAUNCH(ST_VEC, 1, aao::launch_update_norm_ff(wf, Vf, n, nv, n, p->hdev + 65, p->partial, p->stream));
    LAUNCH(ST_VEC, 1, aao::launch_reduce_partials(p->partial, nb, 1, p->hdev + 130, p->stream));
    return AAO_OK;
  }
  TRY(matvec_any(p, zj, p->mixed, nullptr, w, nullptr));
  LAUNCH(ST_VEC, 1, aao::launch_dots(w, p->V, n, nv, n, p->partial, p->stream));
  LAUNCH(ST_VEC, 1, aao::launch_reduce_partials(p->partial, nb, nv, p->hdev, p->stream));
  LAUNCH(ST_VEC, 1, aao::launch_update_dots(w, p->V, n, nv, n, p->hdev, p->partial, p->stream));
  LAUNCH(ST_VEC, 1, aao::launch_reduce_partials(p->partial, nb, nv, p->hdev + 65, p->stream));
  LAUNCH(ST_VEC, 1, aao::launch_update_norm(w, p->V, n, nv, n, p->hdev + 65, p->partial, p->stream));
  LAUNCH(ST_VEC, 1, aao::launch_reduce_partials(p->partial, nb, 1, p->hdev + 130, p->stream));
  return AAO_OK;
}

void release_cycle_graph(aao_plan* p) {
  if (p->cycle_exec) cudaGraphExecDestroy(p->cycle_exec);
  p->cycle_exec = nullptr;
  p->graph_fno = nullptr;
}

// Captures one restart cycle as a graph: init (g = beta e_1, v_0 /= beta), then for j < m a
// conditional IF node whose body is Arnoldi step j + the device Givens update + v_{j+1} /= h,
// then the least-squares solve.  Each IF node has its own handle, reset to 0 at every launch;
// the init kernel enables step 0 and step j's Givens kernel enables step j + 1.  Kernels are
// recorded on plan-owned capture streams.
// The device FGMRES state (and its pinned host mirror) of the graph-driven and batched cycles.
aao_status ensure_dev_state(aao_plan* p) {
  if (!p->gd) {
    TRY(dalloc(p, &p->gd, 1));
    if (cudaMallocHost(&p->gd_host, sizeof(GmresDevState)) != cudaSuccess) {
      p->gd_host = nullptr;
      return fail(p, AAO_ENOMEM, "cudaMallocHost failed");
    }
  }
  return AAO_OK;
}

aao_status build_cycle_graph(aao_plan* p) {
  release_cycle_graph(p);
  TRY(ensure_dev_state(p));
  if (!p->cap1) {
    CK(cudaStreamCreateWithFlags(&p->cap1, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&p->cap2, cudaStreamNonBlocking));
  }
  const int m = p->m;
  const size_t n = p->n;
  cudaStream_t user = p->stream;
  int64_t saved[AAO_NUM_STAGES];
  std::memcpy(saved, p->prof_launches, sizeof saved);
  cudaGraph_t g = nullptr;
  std::string err;
  auto check = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && err.empty()) err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaSuccess;
  };
  p->stream = p->cap1;
  if (check(cudaStreamBeginCapture(p->cap1, cudaStreamCaptureModeRelaxed), "begin capture")) {
    cudaStreamCaptureStatus cst;
    std::vector<cudaGraphConditionalHandle> hs(m, 0);
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    bool ok = check(cudaStreamGetCaptureInfo(p->cap1, &cst, nullptr, &g), "capture info");
    for (int j = 0; ok && j < m; ++j)
      ok = check(cudaGraphConditionalHandleCreate(&hs[j], g, 0, cudaGraphCondAssignDefault), "conditional handle");
    if (ok) {
      cycle_init_kernel<<<1, 1, 0, p->cap1>>>(p->gd, p->hdev, m, hs[0], 1);
      ok = check(cudaGetLastError(), "cycle init") &&
           check(p->mixed ? aao::launch_scale_to_ff((float2*)(void*)p->V, p->W, &p->gd->inv_beta, 0.0, n, p->cap1)
                          : aao::launch_scale_dev(p->V, p->V, &p->gd->inv_beta, n, p->cap1),
                 "scale v0");
    }
    for (int j = 0; ok && j < m; ++j) {
      ok = check(cudaStreamGetCaptureInfo(p->cap1, &cst, nullptr, nullptr, &deps, nullptr, &ndeps), "capture info");
      if (!ok) break;
      cudaGraphNodeParams np{};
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = hs[j];
      np.conditional.type = cudaGraphCondTypeIf;
      np.conditional.size = 1;
      cudaGraphNode_t node;
      ok = check(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &np), "conditional node") &&
           check(cudaStreamUpdateCaptureDependencies(p->cap1, &node, nullptr, 1, cudaStreamSetCaptureDependencies),
                 "capture dependencies");
      if (!ok) break;
      cudaGraph_t body = np.conditional.phGraph_out[0];
      p->stream = p->cap2;
      if (!check(cudaStreamBeginCaptureToGraph(p->cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed),
                 "begin body capture")) {
        ok = false;
        break;
      }
      int64_t before[AAO_NUM_STAGES];
      std::memcpy(before, p->prof_launches, sizeof before);
      const aao_status st = arnoldi_step(p, j, p->gd);
      if (st == AAO_OK) {
        givens_kernel<<<1, 1, 0, p->cap2>>>(p->gd, p->hdev, j, m, j + 1 < m ? hs[j + 1] : hs[j], j + 1 < m);
        double* w = p->V + (size_t)(j + 1) * n;
        if (check(cudaGetLastError(), "givens"))
          check(p->mixed ? aao::launch_scale_ff((float2*)(void*)w, &p->gd->inv_hn, 0.0, n, p->cap2)
                         : aao::launch_scale_dev(w, w, &p->gd->inv_hn, n, p->cap2),
                "scale");
        if (j == 0)
          for (int q = 0; q < AAO_NUM_STAGES; ++q) p->step_launches[q] = p->prof_launches[q] - before[q];
      } else if (err.empty()) {
        err = p->err;
      }
      cudaGraph_t body_out = nullptr;
      check(cudaStreamEndCapture(p->cap2, &body_out), "end body capture");
      p->stream = p->cap1;
      ok = err.empty();
    }
    if (ok) {
      lsq_kernel<<<1, 1, 0, p->cap1>>>(p->gd);
      check(cudaGetLastError(), "lsq");
    }
    cudaGraph_t g_out = nullptr;
    check(cudaStreamEndCapture(p->cap1, &g_out), "end capture");
    if (err.empty()) check(cudaGraphInstantiate(&p->cycle_exec, g_out, 0), "instantiate");
    if (g_out) cudaGraphDestroy(g_out);
  }
  p->stream = user;
  std::memcpy(p->prof_launches, saved, sizeof saved);
  // givens + scale per step on top of the step's own kernels
  p->step_launches[ST_VEC] += 2;
  if (!err.empty()) {
    release_cycle_graph(p);
    return fail(p, AAO_ECUDA, "cycle graph: " + err);
  }
  p->graph_fno = p->fno;
  return AAO_OK;
}

// Autotuner of the Step (b) launch shape: times every admissible CTA size of the
// register-resident COCG kernel on the plan's own shifted systems (deterministic test
// right-hand sides, tol 0, a fixed 4 iterations, so every candidate does the same work)
// and keeps the fastest.  Results are cached per (device, M, L, inner, systems).
aao_status autotune_cocg_threads(aao_plan* p) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int, int>, int> cache;
  const int nt_min = aao::cocg_reg_min_threads(p->M);
  if (nt_min == 0) return AAO_OK;
  if (nt_min == 512) {
    p->cocg_threads = 512;
    return AAO_OK;
  }
  int dev = 0;
  CK(cudaGetDevice(&dev));
  const auto key = std::make_tuple(dev, p->M, p->logL, (int)p->opts.inner, p->nsys);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      p->cocg_threads = it->second;
      return AAO_OK;
    }
  }
  aao::CocgTables32 tb{p->twL32, p->Ebr32, p->lambda, p->chirp32, p->chat32, p->seig32, p->tau32, p->sconv};
  float2* spec = (float2*)p->spec;
  const size_t ns = (size_t)p->nsys * p->M;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(p, AAO_ECUDA, "cudaEventCreate failed");
  }
  int best = 512;
  float best_ms = 1e30f;
  cudaError_t e = cudaSuccess;
  for (int nt = nt_min; nt <= 512 && e == cudaSuccess; nt *= 2) {
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // rep 0 warms up
      e = aao::launch_fill_test_rhs(spec, ns, p->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e0, p->stream);
      if (e == cudaSuccess)
        e = aao::launch_cocg_f32(spec, (float2*)p->rws, (float2*)p->pws, p->M, p->logL, p->nsys, (int)p->opts.inner,
                                 tb, 0.0f, 4, p->iters, p->flags, p->cocg_grid, p->stream, nullptr, nt);
      if (e == cudaSuccess) e = cudaEventRecord(e1, p->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0;
      if (e == cudaSuccess && rep == 1 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best_ms) {
        best_ms = ms;
        best = nt;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(p, AAO_ECUDA, std::string("COCG autotuning: ") + cudaGetErrorString(e));
  p->cocg_threads = best;
  std::lock_guard<std::mutex> lock(mu);
  cache[key] = best;
  return AAO_OK;
}

aao_status check_problem(const aao_problem* prob, const aao_opts* o) {
  if (!prob || !o) return fail(nullptr, AAO_EINVAL, "null problem or options");
  if (prob->dim != 1 && prob->dim != 2) return fail(nullptr, AAO_EINVAL, "dim must be 1 or 2");
  if (prob->M < 1 || prob->M > 8191) return fail(nullptr, AAO_EINVAL, "M must be in [1, 8191]");
  if (prob->dim == 2) {
    if (prob->M > 2047 || prob->My < 1 || prob->My > 2047)
      return fail(nullptr, AAO_EINVAL, "2D: M and My must be in [1, 2047]");
    if (((prob->M + 1) & prob->M) || ((prob->My + 1) & prob->My))
      return fail(nullptr, AAO_EINVAL, "2D: M+1 and My+1 must be powers of two");

  }
  if (prob->Nt < 4 || prob->Nt > 65536 || (prob->Nt & (prob->Nt - 1)))
    return fail(nullptr, AAO_EINVAL, "Nt must be a power of two in [4, 65536]");
  {  // a time-DFT CTA holds all Nt rows of its column tile in shared memory
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess) {
      const int lim = aao::tdft_max_Nt(o->prec == AAO_PREC_MIXED, (size_t)optin);
      if (prob->Nt > lim)
        return fail(nullptr, AAO_EINVAL,
                    "Nt must be at most " + std::to_string(lim) + " in this precision on this device (the time-DFT "
                    "tile of Nt rows must fit in " + std::to_string(optin) + " bytes of shared memory)");
    }
  }
  if (o->restart < 1 || o->restart > kMaxRestart) return fail(nullptr, AAO_EINVAL, "restart must be in [1, 64]");
  if (o->max_cycles < 1) return fail(nullptr, AAO_EINVAL, "max_cycles must be >= 1");
  if (!(o->tol > 0) || !(o->inner_tol > 0)) return fail(nullptr, AAO_EINVAL, "tolerances must be > 0");
  if (o->inner_maxit < 1) return fail(nullptr, AAO_EINVAL, "inner_maxit must be >= 1");
  if (o->prec != AAO_PREC_FP64 && o->prec != AAO_PREC_MIXED) return fail(nullptr, AAO_EINVAL, "bad precision");
  if (o->inner != AAO_INNER_STRANG && o->inner != AAO_INNER_TAU && o->inner != AAO_INNER_TAU_DIRECT)
    return fail(nullptr, AAO_EINVAL, "bad inner");
  if (o->inner != AAO_INNER_STRANG && ((prob->M + 1) & prob->M))
    return fail(nullptr, AAO_EINVAL, "the tau preconditioner needs M+1 to be a power of two");
  if (o->poly_m < 0 || o->poly_m > 16) return fail(nullptr, AAO_EINVAL, "poly_m must be in [0, 16]");
  if (o->use_graphs != 0 && o->use_graphs != 1) return fail(nullptr, AAO_EINVAL, "use_graphs must be 0 or 1");
  if (o->matvec != AAO_MATVEC_FFT64 && o->matvec != AAO_MATVEC_NTT) return fail(nullptr, AAO_EINVAL, "bad matvec");
  if (o->cocg_threads != 0 && o->cocg_threads != 64 && o->cocg_threads != 128 && o->cocg_threads != 256 &&
      o->cocg_threads != 512 && o->cocg_threads != AAO_COCG_TMEM)
    return fail(nullptr, AAO_EINVAL, "cocg_threads must be 0, 64, 128, 256, 512 or AAO_COCG_TMEM");
  if (o->cocg_threads > 0 && o->prec == AAO_PREC_MIXED && prob->dim == 1 &&
      o->cocg_threads < aao::cocg_reg_min_threads((int)prob->M))
    return fail(nullptr, AAO_EINVAL, "cocg_threads must be at least M / 16");
  if (o->cocg_threads == AAO_COCG_TMEM &&
      (o->prec != AAO_PREC_MIXED || prob->dim != 1 || o->inner != AAO_INNER_STRANG || prob->M <= 4096))
    return fail(nullptr, AAO_EINVAL, "AAO_COCG_TMEM needs mixed precision, 1D, the Strang preconditioner and M > 4096");
  return AAO_OK;
}

// aao_gmres_solve with each restart cycle replayed as one CUDA graph (1D and 2D); nF = ||F|| > 0.
aao_status gmres_solve_graph(aao_plan* p, const double* F, double* U, aao_info* info, double nF,
                             bool zero_guess) {
  if (!p->cycle_exec || p->graph_fno != p->fno) TRY(build_cycle_graph(p));
  const size_t n = p->n;
  const size_t tail = sizeof(GmresDevState) - offsetof(GmresDevState, thr);
  GmresDevState& hs = *p->gd_host;
  std::memset(&hs.thr, 0, tail);
  hs.thr = 0.5 * p->opts.tol * nF;
  CK(cudaMemcpyAsync(&p->gd->thr, &hs.thr, tail, cudaMemcpyHostToDevice, p->stream));
  aao_info inf{};
  aao_status result = AAO_ENOCONV;
  int outer_prev = 0;
  for (int cycle = 0; cycle <= p->opts.max_cycles; ++cycle) {
    double beta2 = 0;
    double* r0 = p->mixed ? p->W : p->V;  // the graph scales r0 into v_0
    if (cycle == 0 && zero_guess) {  // r = F; beta^2 = ||F||^2 is already in p->hdev[0]
      CK(cudaMemcpyAsync(r0, F, n * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
      beta2 = nF * nF;
    } else {
      TRY(matvec_any(p, U, false, F, r0, p->sq));  // r = F - calA U, row sums of squares
      inf.matvecs++;
      TRY(reduce_to_host(p, p->sq, (int)p->nsq, 1, &beta2));  // leaves beta^2 in p->hdev[0]
    }
    const double beta = std::sqrt(beta2);
    if (!std::isfinite(beta)) { result = AAO_ENONFINITE; p->err = "non-finite residual"; break; }
    inf.true_rel_res = beta / nF;
    inf.cycles = cycle;
    if (inf.true_rel_res <= p->opts.tol) { result = AAO_OK; break; }
    if (cycle == p->opts.max_cycles) break;
    CK(cudaGraphLaunch(p->cycle_exec, p->stream));
    CK(cudaMemcpyAsync(&hs.thr, &p->gd->thr, tail, cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    const int steps = hs.outer_total - outer_prev + (hs.status != 0 ? 1 : 0);
    outer_prev = hs.outer_total;
    inf.matvecs += steps;
    for (int q = 0; q < AAO_NUM_STAGES; ++q) p->prof_launches[q] += steps * p->step_launches[q];
    p->prof_launches[ST_VEC] += 3;  // cycle init, v_0 scaling, least squares
    if (hs.status != 0) {
      result = (aao_status)hs.status;
      p->err = result == AAO_EBREAKDOWN ? "GMRES breakdown" : "non-finite Arnoldi vector";
      break;
    }
    if (hs.jdone > 0) {
      if (p->mixed)
        LAUNCH(ST_VEC, 1, aao::launch_zy_update_f32(U, (const float*)p->Z, n, hs.jdone, n, p->gd->y, p->stream));
      else
        LAUNCH(ST_VEC, 1, aao::launch_zy_update_f64(U, (const double*)p->Z, n, hs.jdone, n, p->gd->y, p->stream));
    }
  }
  CK(cudaStreamSynchronize(p->stream));
  inf.outer_iters = hs.outer_total;
  inf.inner_iters_max = hs.inner_max;
  inf.inner_iters_sum = hs.inner_sum;
  inf.warm_accepted = hs.accepted;
  if (hs.flag_max != 0)
    inf.status_detail = hs.flag_max == 1 ? AAO_ENOCONV : (hs.flag_max == 2 ? AAO_EBREAKDOWN : AAO_ENONFINITE);
  if (info) *info = inf;
  if (result == AAO_ENOCONV) p->err = "FGMRES did not reach the tolerance within max_cycles";
  return result;
}

}  // namespace

extern "C" {

void aao_default_opts(aao_opts* o, aao_precision prec) {
  if (!o) return;
  o->restart = 20;
  o->max_cycles = 50;
  o->tol = 1e-10;
  o->inner_tol = prec == AAO_PREC_MIXED ? 1e-6 : 1e-12;
  o->inner_maxit = 200;
  o->prec = prec;
  o->inner = AAO_INNER_STRANG;
  o->use_graphs = 1;
  o->matvec = AAO_MATVEC_NTT;
  o->cocg_threads = 0;
  o->poly_m = 0;
}

aao_status aao_setup_coeffs(double alpha, int64_t n, double* g_host) {
  if (aao_setup_coeffs_impl(alpha, n, g_host) != 0)
    return fail(nullptr, AAO_EINVAL, "aao_setup_coeffs: need n >= 1, g_host != NULL, 0 < alpha <= 2");
  return AAO_OK;
}

const char* aao_last_error(const aao_plan* plan) {
  return plan ? plan->err.c_str() : g_create_error.c_str();
}

size_t aao_plan_workspace_bytes(const aao_plan* plan) { return plan ? plan->ws_bytes : 0; }

aao_status aao_plan_destroy(aao_plan* p) {
  if (!p) return AAO_OK;
  for (auto& pr : p->ev_pending) {
    cudaEventDestroy(pr.second.first);
    cudaEventDestroy(pr.second.second);
  }
  for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
  release_cycle_graph(p);
  if (p->cap1) cudaStreamDestroy(p->cap1);
  if (p->cap2) cudaStreamDestroy(p->cap2);
  if (p->c2d_exec) cudaGraphExecDestroy(p->c2d_exec);
  if (p->cap3) cudaStreamDestroy(p->cap3);
  if (p->c2d_cap) cudaStreamDestroy(p->c2d_cap);
  if (p->gd_host) cudaFreeHost(p->gd_host);
  for (void* q : p->allocs) cudaFree(q);
  if (p->pinned) cudaFreeHost(p->pinned);
  if (p->host_count) cudaFreeHost(p->host_count);
  delete p;
  return AAO_OK;
}

aao_status aao_plan_create(const aao_problem* prob, const aao_opts* opts, void* cuda_stream, aao_plan** out) {
  if (!out) return fail(nullptr, AAO_EINVAL, "out is NULL");
  *out = nullptr;
  TRY(check_problem(prob, opts));
  aao_plan* p = new aao_plan();
  p->prob = *prob;
  p->opts = *opts;
  p->stream = (cudaStream_t)cuda_stream;
  p->mixed = opts->prec == AAO_PREC_MIXED;
  p->direct = opts->inner == AAO_INNER_TAU_DIRECT;
  const char* emsg = nullptr;
  const double eps = prob->eps > 0 ? prob->eps : aao::default_eps(prob->T / (double)prob->Nt, p->mixed);
  if (!aao::build_tables(prob->M, prob->Nt, prob->T, prob->alpha, prob->kappa, eps, p->ht, &emsg)) {
    delete p;
    return fail(nullptr, AAO_EINVAL, emsg);
  }
  p->dim = prob->dim;
  if (p->dim == 2 &&
      !aao::build_tables(prob->My, prob->Nt, prob->T, prob->alpha_y, prob->kappa_y, eps, p->hty, &emsg)) {
    delete p;
    return fail(nullptr, AAO_EINVAL, emsg);
  }
  p->M = (int)prob->M;
  p->My = p->dim == 2 ? (int)prob->My : 1;
  p->Msp = (size_t)p->M * p->My;
  p->Nt = (int)prob->Nt;
  p->logL = p->ht.logL;
  p->logLy = p->dim == 2 ? p->hty.logL : 0;
  p->nsys = p->Nt / 2 + 1;
  p->m = opts->restart;
  p->n = p->Msp * p->Nt;
  auto bail = [&](aao_status st) {
    g_create_error = p->err;
    aao_plan_destroy(p);
    return st;
  };
#define TRYP(x)                          \
  do {                                   \
    aao_status s_ = (x);                 \
    if (s_ != AAO_OK) return bail(s_);   \
  } while (0)
  const aao::HostTables& t = p->ht;
  TRYP(upload(p, &p->Ehalf, t.Ehat_half));
  TRYP(upload_c(p, &p->twL64, t.tw_L));
  TRYP(upload_c(p, &p->twL32, t.tw_L));
  TRYP(upload_c(p, &p->twNt64, t.tw_Nt));
  TRYP(upload_c(p, &p->twNt32, t.tw_Nt));
  TRYP(upload(p, &p->Ebr64, t.Ehat_f));
  TRYP(upload(p, &p->Ebr32, t.Ehat_f));
  TRYP(upload_c(p, &p->lambda, t.lambda));
  TRYP(upload(p, &p->sfwd64, t.scale_fwd));
  TRYP(upload(p, &p->sinv64, t.scale_inv));
  TRYP(upload(p, &p->sfwd32, t.scale_fwd));
  TRYP(upload(p, &p->sinv32, t.scale_inv));
  TRYP(upload_c(p, &p->chirp64, t.chirp));
  TRYP(upload_c(p, &p->chirp32, t.chirp));
  TRYP(upload_c(p, &p->chat64, t.chirp_hat_f));
  TRYP(upload_c(p, &p->chat32, t.chirp_hat_f));
  TRYP(upload(p, &p->seig64, t.strang_eig));
  TRYP(upload(p, &p->seig32, t.strang_eig));
  if (t.tau_ok) {
    TRYP(upload(p, &p->tau64, t.tau_eig_f));
    TRYP(upload(p, &p->tau32, t.tau_eig_f));
  }
  const size_t n = p->n;
  const size_t csz = p->mixed ? sizeof(float2) : sizeof(double2);
  if (p->dim == 1 && opts->matvec == AAO_MATVEC_NTT) {
    aao::build_ntt_tables(p->ht);
    uint32_t* q32;
    TRYP(upload(p, &q32, p->ht.ntt_twf));
    p->ntt_tab.twf = (const uint2*)q32;
    TRYP(upload(p, &q32, p->ht.ntt_twi));
    p->ntt_tab.twi = (const uint2*)q32;
    TRYP(upload(p, &q32, p->ht.ntt_ghat));
    p->ntt_tab.ghat = (const uint2*)q32;
    for (int i = 0; i < 6; ++i) p->ntt_tab.crt[i] = make_uint2(p->ht.ntt_crt[2 * i], p->ht.ntt_crt[2 * i + 1]);
    p->ntt_tab.c_gscale = p->ht.ntt_c_gscale;
    p->ntt_tab.gexp = p->ht.ntt_gexp;
    TRYP(dalloc(p, &p->ntt_res, (size_t)(aao::kNttPrimes + 2) * n));  // residues + int64 quantised rows
    TRYP(dalloc(p, &p->ntt_rowscale, (size_t)p->Nt));
    p->ntt = true;
  }
  TRYP(dalloc(p, &p->V, (size_t)(p->m + 1) * n));
  if (p->mixed) TRYP(dalloc(p, &p->W, n));
  {
    void* z = nullptr;
    TRYP(dalloc(p, reinterpret_cast<unsigned char**>(&z), (size_t)p->m * n * (p->mixed ? 4 : 8)));
    p->Z = z;
  }
  {
    unsigned char* q;
    TRYP(dalloc(p, &q, (size_t)p->nsys * p->Msp * csz));
    p->spec = q;
    TRYP(dalloc(p, &q, (size_t)p->nsys * p->Msp * csz));
    p->rws = q;
    TRYP(dalloc(p, &q, (size_t)p->nsys * p->Msp * csz));
    p->pws = q;
  }
  p->nsq = p->ntt ? (size_t)aao::ntt_partials(p->M, p->Nt) : (size_t)p->Nt;
  if (p->dim == 2) {
    const aao::HostTables& ty = p->hty;
    TRYP(upload_c(p, &p->twy64, ty.tw_L));
    TRYP(upload_c(p, &p->twy32, ty.tw_L));
    TRYP(upload(p, &p->Exf64, t.Ehat_f));
    TRYP(upload(p, &p->Exf32, t.Ehat_f));
    TRYP(upload(p, &p->Eyf64, ty.Ehat_f));
    TRYP(upload(p, &p->Eyf32, ty.Ehat_f));
    TRYP(upload(p, &p->sxn64, t.tau_eig_nat));
    TRYP(upload(p, &p->sxn32, t.tau_eig_nat));
    TRYP(upload(p, &p->syf64, ty.tau_eig_f));
    TRYP(upload(p, &p->syf32, ty.tau_eig_f));
    unsigned char* q;
    TRYP(dalloc(p, &q, (size_t)p->nsys * p->Msp * csz)); p->Px = (double2*)q;
    TRYP(dalloc(p, &q, (size_t)p->nsys * p->Msp * csz)); p->Zx = (double2*)q;
    TRYP(dalloc(p, &q, (size_t)p->nsys * p->Msp * csz)); p->Qx = (double2*)q;
    TRYP(dalloc(p, &q, (size_t)p->nsys * p->Msp * csz)); p->Tx = (double2*)q;
    TRYP(dalloc(p, &p->tmp2d, p->n));
    TRYP(dalloc(p, &q, aao::cocg2d_state_bytes(p->nsys))); p->state2d = q;
    const int np = aao::cocg2d_max_partials(p->M, p->My, p->logL, p->logLy, (int)csz);
    TRYP(dalloc(p, &p->part2d, (size_t)p->nsys * np));
    TRYP(dalloc(p, &p->active2d, 1));
    TRYP(dalloc(p, &p->c2d_it, 1));
    TRYP(dalloc(p, &p->c2d_loops, 1));
    if (cudaMemset(p->c2d_loops, 0, sizeof(long long)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->cap3, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->c2d_cap, cudaStreamNonBlocking) != cudaSuccess) {
      p->err = "2D COCG graph setup failed";
      return bail(AAO_ECUDA);
    }
    p->nsq = aao::mv2d_partials(p->M, p->Nt, p->logLy);
    if (opts->matvec == AAO_MATVEC_NTT) {
      // exact-integer line convolutions along x and y (Eq. 4.2), one quantisation scale per time level
      for (int d = 0; d < 2; ++d) {
        aao::HostTables& hd = d ? p->hty : p->ht;
        aao::NttTables& nt = d ? p->ntt_tab_y : p->ntt_tab;
        aao::build_ntt_tables(hd);
        uint32_t* q32;
        TRYP(upload(p, &q32, hd.ntt_twf));
        nt.twf = (const uint2*)q32;
        TRYP(upload(p, &q32, hd.ntt_twi));
        nt.twi = (const uint2*)q32;
        TRYP(upload(p, &q32, hd.ntt_ghat));
        nt.ghat = (const uint2*)q32;
        for (int i = 0; i < 6; ++i) nt.crt[i] = make_uint2(hd.ntt_crt[2 * i], hd.ntt_crt[2 * i + 1]);
        nt.c_gscale = hd.ntt_c_gscale;
        nt.gexp = hd.ntt_gexp;
      }
      TRYP(dalloc(p, &p->ntt_res, aao::ntt2d_scratch_words(p->M, p->My, p->Nt)));
      TRYP(dalloc(p, &p->ntt_rowscale, (size_t)p->Nt));
      p->nsq = (size_t)aao::ntt2d_partials(p->M, p->My, p->Nt);
      p->ntt2d = true;
    }
    if (opts->inner == AAO_INNER_STRANG) {
      // 2D Strang (BCCB): per-direction spectral maps on the host, the per-system spectra on the device
      std::vector<aao::cd> qx, qy;
      aao::build_strang2d_q(p->M, p->logL, false, qx);
      aao::build_strang2d_q(p->My, p->logLy, true, qy);
      const size_t Lx = (size_t)1 << p->logL, Ly = (size_t)1 << p->logLy;
      TRYP(dalloc(p, &q, (size_t)p->nsys * p->My * Lx * csz)); p->W2d = q;
      TRYP(dalloc(p, &q, (size_t)p->nsys * Lx * Ly * csz)); p->G2d = q;
      cudaError_t e;
      if (p->mixed) {
        float2 *Qx, *Qy;
        float *sx, *sy;
        TRYP(upload_c(p, &Qx, qx));
        TRYP(upload_c(p, &Qy, qy));
        TRYP(upload(p, &sx, t.strang_eig));
        TRYP(upload(p, &sy, ty.strang_eig));
        e = aao::launch_strang2d_setup_f32(Qx, Qy, sx, sy, p->lambda, p->M, p->My, p->logL, p->logLy, p->nsys,
                                           (float2*)p->W2d, (float2*)p->G2d, p->stream);
      } else {
        double2 *Qx, *Qy;
        double *sx, *sy;
        TRYP(upload_c(p, &Qx, qx));
        TRYP(upload_c(p, &Qy, qy));
        TRYP(upload(p, &sx, t.strang_eig));
        TRYP(upload(p, &sy, ty.strang_eig));
        e = aao::launch_strang2d_setup_f64(Qx, Qy, sx, sy, p->lambda, p->M, p->My, p->logL, p->logLy, p->nsys,
                                           (double2*)p->W2d, (double2*)p->G2d, p->stream);
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
      if (e != cudaSuccess) {
        p->err = std::string("2D Strang spectra: ") + cudaGetErrorString(e);
        return bail(AAO_ECUDA);
      }
    }
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  p->cocg_grid = std::min(p->nsys, std::max(1, sms));
  if (!p->mixed) {
    const size_t ge = aao::cocg_gbuf_elems_f64(p->logL, p->cocg_grid);
    if (ge) TRYP(dalloc(p, &p->gbuf, ge));
  } else {
    p->cocg_grid = p->nsys;  // shared-memory transforms: one CTA per system
  }
  if (!p->mixed) p->cocg_grid = p->gbuf ? p->cocg_grid : p->nsys;
  TRYP(dalloc(p, &p->iters, (size_t)p->nsys));
  TRYP(dalloc(p, &p->flags, (size_t)p->nsys));
  TRYP(dalloc(p, &p->stats, 4));
  if (cudaMemset(p->stats, 0, 4 * sizeof(int)) != cudaSuccess ||
      cudaMemset(p->iters, 0, (size_t)p->nsys * sizeof(int)) != cudaSuccess ||
      cudaMemset(p->flags, 0, (size_t)p->nsys * sizeof(int)) != cudaSuccess) {
    p->err = "cudaMemset failed";
    return bail(AAO_ECUDA);
  }
  TRYP(dalloc(p, &p->partial, std::max<size_t>((size_t)aao::blas_partial_blocks() * 65,
                                               std::max<size_t>(p->nsq * 65, (size_t)p->Nt))));
  TRYP(dalloc(p, &p->hdev, 4 * 65));
  TRYP(dalloc(p, &p->sq, p->nsq));
  if (cudaMallocHost(&p->pinned, 4 * 65 * sizeof(double)) != cudaSuccess) {
    p->pinned = nullptr;
    p->err = "cudaMallocHost failed";
    return bail(AAO_ENOMEM);
  }
  if (p->dim == 2 && cudaMallocHost(&p->host_count, sizeof(int)) != cudaSuccess) {
    p->host_count = nullptr;
    p->err = "cudaMallocHost failed";
    return bail(AAO_ENOMEM);
  }
  if (p->mixed && p->dim == 1 && opts->inner == AAO_INNER_STRANG && aao::cocg_reg_min_threads(p->M) > 0) {
    // the Strang preconditioner of every shifted system as one L-point circulant (2 FFTs per
    // application instead of Bluestein's 4), built once by the Bluestein form itself
    TRYP(dalloc(p, &p->sconv, (size_t)p->nsys << p->logL));
    aao::CocgTables32 tb{p->twL32, p->Ebr32, p->lambda, p->chirp32, p->chat32, p->seig32, p->tau32, nullptr};
    cudaError_t e = aao::launch_strang_conv_setup(p->M, p->logL, p->nsys, tb, p->sconv, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) {
      p->err = std::string("Strang spectra: ") + cudaGetErrorString(e);
      return bail(AAO_ECUDA);
    }
  }
  if (opts->poly_m > 0) TRYP(dalloc(p, &p->polyw, p->n));
  if (p->sconv && aao::cocg_tm_supported(p->M, p->logL) &&
      (opts->cocg_threads == AAO_COCG_TMEM || opts->cocg_threads == 0)) {
    // the spectra in the order of the tensor-memory kernel's fused pass: entry s holds L-frequency
    // tm_order_freq(s), read from the fused order of the register-resident kernel
    const int L = 1 << p->logL;
    std::vector<int> from_freq(L), perm(L);
    for (int f = 0; f < L; ++f) from_freq[aao::fused_to_freq(f, p->logL)] = f;
    for (int s2 = 0; s2 < L; ++s2) perm[s2] = from_freq[aao::tm_order_freq(s2)];
    int* dperm = nullptr;
    TRYP(upload(p, &dperm, perm));
    TRYP(dalloc(p, &p->sconv_tm, (size_t)p->nsys << p->logL));
    TRYP(dalloc(p, &p->Ebr_tm, (size_t)L));
    cudaError_t e = aao::launch_tm_gather(p->sconv, p->sconv_tm, p->Ebr32, p->Ebr_tm, dperm, p->nsys, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) {
      p->err = std::string("tensor-memory kernel spectra: ") + cudaGetErrorString(e);
      return bail(AAO_ECUDA);
    }
    p->tm = true;
  }
  if (p->mixed && p->dim == 1 && !p->direct && aao::cocg_reg_min_threads(p->M) > 0) {
    if (opts->cocg_threads > 0)
      p->cocg_threads = opts->cocg_threads;
    else if (p->tm)
      p->cocg_threads = 512;  // the register-resident kernel serves the learned warm start
    else
      TRYP(autotune_cocg_threads(p));
  }
#undef TRYP
  *out = p;
  return AAO_OK;
}

aao_status aao_plan_get_tuning(const aao_plan* p, int* cocg_threads) {
  if (!p || !cocg_threads) return fail(nullptr, AAO_EINVAL, "null argument");
  *cocg_threads = p->tm ? AAO_COCG_TMEM : p->cocg_threads;
  return AAO_OK;
}

aao_status aao_plan_get_inner_record(aao_plan* p, int n_sys, int* iters_host, int* flags_host) {
  if (!p) return fail(nullptr, AAO_EINVAL, "null plan");
  if (n_sys != p->nsys) return fail(p, AAO_EINVAL, "n_sys must be Nt/2 + 1");
  CK(cudaStreamSynchronize(p->stream));
  if (iters_host) CK(cudaMemcpy(iters_host, p->iters, sizeof(int) * n_sys, cudaMemcpyDeviceToHost));
  if (flags_host) CK(cudaMemcpy(flags_host, p->flags, sizeof(int) * n_sys, cudaMemcpyDeviceToHost));
  return AAO_OK;
}

aao_status aao_plan_set_profiling(aao_plan* p, int on) {
  if (!p) return fail(nullptr, AAO_EINVAL, "null plan");
  p->prof_on = on != 0;
  return AAO_OK;
}

aao_status aao_plan_get_profile(aao_plan* p, double* ms, int64_t* launches, int reset) {
  if (!p) return fail(nullptr, AAO_EINVAL, "null plan");
  CK(cudaStreamSynchronize(p->stream));
  for (auto& pr : p->ev_pending) {
    float t = 0;
    CK(cudaEventElapsedTime(&t, pr.second.first, pr.second.second));
    p->prof_ms[pr.first] += t;
    p->ev_pool.push_back(pr.second.first);
    p->ev_pool.push_back(pr.second.second);
  }
  p->ev_pending.clear();
  if (p->c2d_loops) {  // graph-driven 2D COCG iterations: 10 kernels each
    long long loops = 0;
    CK(cudaMemcpy(&loops, p->c2d_loops, sizeof loops, cudaMemcpyDeviceToHost));
    p->prof_launches[ST_COCG] += 10 * (loops - p->c2d_loops_seen);
    p->c2d_loops_seen = loops;
  }
  for (int i = 0; i < AAO_NUM_STAGES; ++i) {
    if (ms) ms[i] = p->prof_ms[i];
    if (launches) launches[i] = p->prof_launches[i];
    if (reset) { p->prof_ms[i] = 0; p->prof_launches[i] = 0; }
  }
  return AAO_OK;
}

aao_status aao_plan_set_warm_start(aao_plan* p, aao_fno* fno) {
  if (!p) return fail(nullptr, AAO_EINVAL, "null plan");
  release_cycle_graph(p);  // a captured cycle holds the previous model's buffers
  if (!fno) {
    p->fno = nullptr;
    return AAO_OK;
  }
  if (p->dim != 1 || !p->mixed || p->M > 8191 || p->direct)
    return fail(p, AAO_EINVAL, "the warm start needs a 1D AAO_PREC_MIXED plan with an iterative Step (b)");
  if (aao::fno_grid_size(fno) != p->M || aao::fno_max_batch(fno) < p->nsys)
    return fail(p, AAO_EINVAL, "the model's M must equal the plan's and its max_batch must be >= Nt/2 + 1");
  if (!p->x0buf) {
    TRY(dalloc(p, &p->x0buf, (size_t)p->nsys * p->M));
    TRY(dalloc(p, &p->fno_alpha, (size_t)p->nsys));
    std::vector<float> a(p->nsys, (float)p->prob.alpha);
    CK(cudaMemcpy(p->fno_alpha, a.data(), a.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  p->fno = fno;
  return AAO_OK;
}

aao_status aao_plan_record_pairs(aao_plan* p, int64_t capacity, void* b, void* x, void* lam) {
  if (!p) return fail(nullptr, AAO_EINVAL, "null plan");
  if (capacity < 0) return fail(p, AAO_EINVAL, "negative capacity");
  if (capacity > 0 && b && x && lam && (p->dim != 1 || !p->mixed))
    return fail(p, AAO_EINVAL, "pair recording needs a 1D AAO_PREC_MIXED plan");
  const bool on = capacity > 0 && b && x && lam;
  p->rec_b = on ? (float2*)b : nullptr;
  p->rec_x = on ? (float2*)x : nullptr;
  p->rec_lam = on ? (double2*)lam : nullptr;
  p->rec_cap = on ? capacity : 0;
  p->rec_count = 0;
  return AAO_OK;
}

aao_status aao_plan_recorded_pairs(const aao_plan* p, int64_t* count) {
  if (!p || !count) return fail(nullptr, AAO_EINVAL, "null argument");
  *count = p->rec_count;
  return AAO_OK;
}

aao_status aao_build_rhs(aao_plan* p, const double* u0, const double* f, double* F) {
  if (!p) return fail(nullptr, AAO_EINVAL, "null plan");
  if (!u0 || !f || !F) return fail(p, AAO_EINVAL, "null pointer");
  LAUNCH(ST_VEC, 1, aao::launch_build_rhs(u0, f, F, p->ht.tau, (int)p->Msp, p->Nt, p->stream));
  return AAO_OK;
}

aao_status aao_matvec(aao_plan* p, const double* v, double* w) {
  if (!p) return fail(nullptr, AAO_EINVAL, "null plan");
  if (!v || !w || v == w) return fail(p, AAO_EINVAL, "null or aliased pointers");
  return matvec_any(p, v, false, nullptr, w, nullptr);
}

aao_status aao_bc_precond_apply(aao_plan* p, const double* v, double* z) {
  if (!p) return fail(nullptr, AAO_EINVAL, "null plan");
  if (!v || !z) return fail(p, AAO_EINVAL, "null pointer");
  return precond_any(p, v, z, 1);
}

aao_status aao_gmres_solve(aao_plan* p, const double* F, double* U, aao_info* info) {
  if (!p) return fail(nullptr, AAO_EINVAL, "null plan");
  if (!F || !U) return fail(p, AAO_EINVAL, "null pointer");
  const size_t n = p->n;
  const int m = p->m;
  const int nb = aao::blas_partial_blocks();
  aao_info inf{};
  // ||F||^2 into p->hdev[0] and ||U||^2 into p->hdev[1]: with U = 0 the first residual is F itself
  LAUNCH(ST_VEC, 1, aao::launch_dots(F, F, 0, 1, n, p->partial, p->stream));
  LAUNCH(ST_VEC, 1, aao::launch_dots(U, U, 0, 1, n, p->partial + nb, p->stream));
  LAUNCH(ST_VEC, 1, aao::launch_reduce_partials(p->partial, nb, 1, p->hdev, p->stream));
  LAUNCH(ST_VEC, 1, aao::launch_reduce_partials(p->partial + nb, nb, 1, p->hdev + 1, p->stream));
  CK(cudaMemcpyAsync(p->pinned, p->hdev, 2 * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  const double nF2 = p->pinned[0];
  const bool zero_guess = p->pinned[1] == 0.0;
  const double nF = std::sqrt(nF2);
  if (!std::isfinite(nF)) return fail(p, AAO_ENONFINITE, "non-finite right-hand side");
  if (nF == 0.0) {
    CK(cudaMemsetAsync(U, 0, n * sizeof(double), p->stream));
    CK(cudaStreamSynchronize(p->stream));
    if (info) *info = inf;
    return AAO_OK;
  }
  if (p->opts.use_graphs && !p->prof_on && p->rec_cap <= p->rec_count)
    return gmres_solve_graph(p, F, U, info, nF, zero_guess);
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  auto Hij = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
  const double tol = p->opts.tol;
  aao_status result = AAO_ENOCONV;
  for (int cycle = 0; cycle <= p->opts.max_cycles; ++cycle) {
    // r = F - calA U  (into V_0) with row partial sums of squares
    double beta2 = 0;
    const double* r0 = p->V;
    if (cycle == 0 && zero_guess) {  // r = F
      if (p->mixed) r0 = F;
      else CK(cudaMemcpyAsync(p->V, F, n * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
      beta2 = nF2;
    } else {
      r0 = p->mixed ? p->W : p->V;
      TRY(matvec_any(p, U, false, F, const_cast<double*>(r0), p->sq));
      inf.matvecs++;
      TRY(reduce_to_host(p, p->sq, (int)p->nsq, 1, &beta2));
    }
    const double beta = std::sqrt(beta2);
    if (!std::isfinite(beta)) { result = AAO_ENONFINITE; p->err = "non-finite residual"; break; }
    inf.true_rel_res = beta / nF;
    inf.cycles = cycle;
    if (inf.true_rel_res <= tol) { result = AAO_OK; break; }
    if (cycle == p->opts.max_cycles) break;
    if (p->mixed)
      LAUNCH(ST_VEC, 1, aao::launch_scale_to_ff((float2*)(void*)p->V, r0, nullptr, 1.0 / beta, n, p->stream));
    else
      LAUNCH(ST_VEC, 1, aao::launch_scale(p->V, p->V, 1.0 / beta, n, p->stream));
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jdone = 0;
    bool stop = false;
    for (int j = 0; j < m && !stop; ++j) {
      double* w = p->V + (size_t)(j + 1) * n;
      TRY(arnoldi_step(p, j, nullptr));
      inf.matvecs++;
      CK(cudaMemcpyAsync(p->pinned, p->hdev, 131 * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
      int st[4] = {0, 0, 0, 0};
      CK(cudaMemcpyAsync(p->pinned + 200, p->stats, 4 * sizeof(int), cudaMemcpyDeviceToHost, p->stream));
      CK(cudaStreamSynchronize(p->stream));
      std::memcpy(st, p->pinned + 200, 4 * sizeof(int));
      inf.inner_iters_max = std::max(inf.inner_iters_max, st[0]);
      inf.inner_iters_sum += st[2];
      inf.warm_accepted += st[3];
      if (st[1] != 0 && inf.status_detail == 0)
        inf.status_detail = st[1] == 1 ? AAO_ENOCONV : (st[1] == 2 ? AAO_EBREAKDOWN : AAO_ENONFINITE);
      for (int i = 0; i <= j; ++i) Hij(i, j) = p->pinned[i] + p->pinned[65 + i];
      const double hn = std::sqrt(p->pinned[130]);
      Hij(j + 1, j) = hn;
      if (!std::isfinite(hn)) { result = AAO_ENONFINITE; p->err = "non-finite Arnoldi vector"; stop = true; break; }
      if (hn > 0) {
        if (p->mixed) LAUNCH(ST_VEC, 1, aao::launch_scale_ff((float2*)(void*)w, nullptr, 1.0 / hn, n, p->stream));
        else LAUNCH(ST_VEC, 1, aao::launch_scale(w, w, 1.0 / hn, n, p->stream));
      }
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * Hij(i, j) + sn[i] * Hij(i + 1, j);
        Hij(i + 1, j) = -sn[i] * Hij(i, j) + cs[i] * Hij(i + 1, j);
        Hij(i, j) = t;
      }
      const double d = std::hypot(Hij(j, j), Hij(j + 1, j));
      if (d == 0.0) { result = AAO_EBREAKDOWN; p->err = "GMRES breakdown"; stop = true; break; }
      cs[j] = Hij(j, j) / d;
      sn[j] = Hij(j + 1, j) / d;
      Hij(j, j) = d;
      Hij(j + 1, j) = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      inf.outer_iters++;
      jdone = j + 1;
      if (std::fabs(g[j + 1]) <= 0.5 * tol * nF || hn == 0.0) break;
    }
    if (result == AAO_ENONFINITE || result == AAO_EBREAKDOWN) break;
    for (int i = jdone - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < jdone; ++k) s -= Hij(i, k) * y[k];
      y[i] = s / Hij(i, i);
    }
    std::memcpy(p->pinned, y.data(), jdone * sizeof(double));
    CK(cudaMemcpyAsync(p->hdev + 195, p->pinned, jdone * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    if (p->mixed)
      LAUNCH(ST_VEC, 1, aao::launch_zy_update_f32(U, (const float*)p->Z, n, jdone, n, p->hdev + 195, p->stream));
    else
      LAUNCH(ST_VEC, 1, aao::launch_zy_update_f64(U, (const double*)p->Z, n, jdone, n, p->hdev + 195, p->stream));
  }
  CK(cudaStreamSynchronize(p->stream));
  if (info) *info = inf;
  if (result == AAO_ENOCONV) p->err = "FGMRES did not reach the tolerance within max_cycles";
  return result;
}

aao_status aao_gmres_solve_host(aao_plan* p, const double* F_host, double* U_host, aao_info* info) {
  if (!p) return fail(nullptr, AAO_EINVAL, "null plan");
  if (!F_host || !U_host) return fail(p, AAO_EINVAL, "null pointer");
  if (!p->Fh) {
    TRY(dalloc(p, &p->Fh, p->n));
    TRY(dalloc(p, &p->Uh, p->n));
  }
  CK(cudaMemcpyAsync(p->Fh, F_host, p->n * sizeof(double), cudaMemcpyHostToDevice, p->stream));
  CK(cudaMemsetAsync(p->Uh, 0, p->n * sizeof(double), p->stream));
  aao_status st = aao_gmres_solve(p, p->Fh, p->Uh, info);
  if (st != AAO_OK && st != AAO_ENOCONV) return st;
  CK(cudaMemcpyAsync(U_host, p->Uh, p->n * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return st;
}

namespace {
// Dot products of w with nv vectors V + i vstride, reduced on the device and read back to out (host).
aao_status dots_to_host(aao_plan* p, const double* w, const double* V, size_t vstride, int nv, double* out) {
  const int nb = aao::blas_partial_blocks();
  LAUNCH(ST_VEC, 1, aao::launch_dots(w, V, vstride, nv, p->n, p->partial, p->stream));
  return reduce_to_host(p, p->partial, nb, nv, out);
}

// COCG statistics of the last preconditioner application, accumulated into inf (synchronises).
aao_status add_inner_stats(aao_plan* p, aao_info& inf) {
  LAUNCH(ST_VEC, 1, (iter_stats_kernel<<<1, 256, 0, p->stream>>>(p->iters, p->flags, p->nsys, p->stats),
                     cudaGetLastError()));
  CK(cudaMemcpyAsync(p->pinned + 200, p->stats, 4 * sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  int st[4];
  std::memcpy(st, p->pinned + 200, sizeof st);
  inf.inner_iters_max = std::max(inf.inner_iters_max, st[0]);
  inf.inner_iters_sum += st[2];
  inf.warm_accepted += st[3];
  if (st[1] != 0 && inf.status_detail == 0)
    inf.status_detail = st[1] == 1 ? AAO_ENOCONV : (st[1] == 2 ? AAO_EBREAKDOWN : AAO_ENONFINITE);
  return AAO_OK;
}
}  // namespace

aao_status aao_bicgstab_solve(aao_plan* p, const double* F, double* U, aao_info* info) {
  if (!p) return fail(nullptr, AAO_EINVAL, "null plan");
  if (!F || !U || F == U) return fail(p, AAO_EINVAL, "null or aliased pointers");
  if (p->m < 7) return fail(p, AAO_EINVAL, "BiCGSTAB keeps 7 vectors in the Krylov workspace: restart must be >= 7");
  const size_t n = p->n;
  // FP64 views of the plan's Krylov workspace (V holds m + 1 >= 8 vectors of 8-byte elements)
  double* r = p->V;             // residual F - calA U; r and rh adjacent for one dots call
  double* rh = p->V + n;        // the shadow residual r0^
  double* pv = p->V + 2 * n;
  double* v = p->V + 3 * n;
  double* sv = p->V + 4 * n;    // s and t adjacent
  double* tv = p->V + 5 * n;
  double* y = p->V + 6 * n;     // P^{-1} p, then P^{-1} s
  aao_info inf{};
  double h[2];
  TRY(dots_to_host(p, F, F, 0, 1, h));
  const double nF = std::sqrt(h[0]);
  if (!std::isfinite(nF)) return fail(p, AAO_ENONFINITE, "non-finite right-hand side");
  if (nF == 0.0) {
    CK(cudaMemsetAsync(U, 0, n * sizeof(double), p->stream));
    CK(cudaStreamSynchronize(p->stream));
    if (info) *info = inf;
    return AAO_OK;
  }
  TRY(matvec_any(p, U, false, F, r, nullptr));  // r = F - calA U
  inf.matvecs++;
  CK(cudaMemcpyAsync(rh, r, n * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
  CK(cudaMemsetAsync(pv, 0, n * sizeof(double), p->stream));
  CK(cudaMemsetAsync(v, 0, n * sizeof(double), p->stream));
  TRY(dots_to_host(p, r, r, 0, 1, h));
  const double n0 = std::sqrt(h[0]);
  aao_status result = AAO_ENOCONV;
  if (!std::isfinite(n0)) { result = AAO_ENONFINITE; p->err = "non-finite residual"; }
  const double thr = p->opts.tol * n0;
  double rho = 1.0, alpha = 1.0, omega = 1.0;
  const long maxit = (long)p->opts.max_cycles * p->m;
  if (n0 <= thr) result = AAO_OK;
  for (long it = 0; result == AAO_ENOCONV && it < maxit; ++it) {
    TRY(dots_to_host(p, r, r, n, 2, h));  // (r, r), (r, r0^)
    const double rho_new = h[1];
    if (!std::isfinite(rho_new)) { result = AAO_ENONFINITE; p->err = "non-finite BiCGSTAB scalar"; break; }
    if (rho_new == 0.0 || omega == 0.0) { result = AAO_EBREAKDOWN; p->err = "BiCGSTAB breakdown (rho = 0)"; break; }
    const double beta = (rho_new / rho) * (alpha / omega);
    rho = rho_new;
    LAUNCH(ST_VEC, 1, aao::launch_lincomb3(pv, 1.0, r, beta, pv, -beta * omega, v, n, p->stream));  // p = r + beta (p - omega v)
    TRY(precond_any(p, pv, y, 1));  // y = P^{-1} p
    TRY(add_inner_stats(p, inf));
    TRY(matvec_any(p, y, false, nullptr, v, nullptr));  // v = calA y
    inf.matvecs++;
    inf.outer_iters++;
    TRY(dots_to_host(p, v, rh, 0, 1, h));
    if (h[0] == 0.0 || !std::isfinite(h[0])) {
      result = std::isfinite(h[0]) ? AAO_EBREAKDOWN : AAO_ENONFINITE;
      p->err = "BiCGSTAB breakdown ((r0^, v) = 0)";
      break;
    }
    alpha = rho / h[0];
    LAUNCH(ST_VEC, 1, aao::launch_lincomb3(U, 1.0, U, alpha, y, 0.0, nullptr, n, p->stream));   // U += alpha y
    LAUNCH(ST_VEC, 1, aao::launch_lincomb3(sv, 1.0, r, -alpha, v, 0.0, nullptr, n, p->stream));  // s = r - alpha v
    TRY(dots_to_host(p, sv, sv, 0, 1, h));
    if (std::sqrt(h[0]) <= thr) { result = AAO_OK; break; }  // converged at the half step
    TRY(precond_any(p, sv, y, 1));  // y = P^{-1} s
    TRY(add_inner_stats(p, inf));
    TRY(matvec_any(p, y, false, nullptr, tv, nullptr));  // t = calA y
    inf.matvecs++;
    inf.outer_iters++;
    TRY(dots_to_host(p, tv, sv, n, 2, h));  // (t, s), (t, t)
    if (!(h[1] > 0.0) || !std::isfinite(h[0])) {
      result = std::isfinite(h[1]) ? AAO_EBREAKDOWN : AAO_ENONFINITE;
      p->err = "BiCGSTAB breakdown ((t, t) = 0)";
      break;
    }
    omega = h[0] / h[1];
    LAUNCH(ST_VEC, 1, aao::launch_lincomb3(U, 1.0, U, omega, y, 0.0, nullptr, n, p->stream));    // U += omega y
    LAUNCH(ST_VEC, 1, aao::launch_lincomb3(r, 1.0, sv, -omega, tv, 0.0, nullptr, n, p->stream));  // r = s - omega t
    TRY(dots_to_host(p, r, r, 0, 1, h));
    inf.cycles = (int)it + 1;
    if (std::sqrt(h[0]) <= thr) result = AAO_OK;
  }
  // true relative residual in FP64
  TRY(matvec_any(p, U, false, F, y, p->sq));
  inf.matvecs++;
  double rr = 0;
  TRY(reduce_to_host(p, p->sq, (int)p->nsq, 1, &rr));
  inf.true_rel_res = std::sqrt(rr) / nF;
  if (info) *info = inf;
  if (result == AAO_ENOCONV) p->err = "BiCGSTAB did not reach the tolerance within max_cycles * restart iterations";
  return result;
}

aao_status aao_solve_windows(aao_plan* p, int n_windows, const double* u0, const double* f, double* U,
                             aao_info* info) {
  if (!p) return fail(nullptr, AAO_EINVAL, "null plan");
  if (n_windows < 1 || !u0 || !f || !U || f == U) return fail(p, AAO_EINVAL, "bad windowed-solve arguments");
  if (!p->Fh) {
    TRY(dalloc(p, &p->Fh, p->n));
    TRY(dalloc(p, &p->Uh, p->n));
  }
  aao_info tot{};
  const size_t n = p->n;
  for (int q = 0; q < n_windows; ++q) {
    const double* start = q == 0 ? u0 : U + (size_t)q * n - p->Msp;  // last level of window q - 1
    double* Uq = U + (size_t)q * n;
    LAUNCH(ST_VEC, 1, aao::launch_build_rhs(start, f + (size_t)q * n, p->Fh, p->ht.tau, (int)p->Msp, p->Nt,
                                            p->stream));
    CK(cudaMemsetAsync(Uq, 0, n * sizeof(double), p->stream));
    aao_info inf{};
    const aao_status st = aao_gmres_solve(p, p->Fh, Uq, &inf);
    tot.outer_iters += inf.outer_iters;
    tot.cycles += inf.cycles;
    tot.matvecs += inf.matvecs;
    tot.inner_iters_max = std::max(tot.inner_iters_max, inf.inner_iters_max);
    tot.inner_iters_sum += inf.inner_iters_sum;
    tot.warm_accepted += inf.warm_accepted;
    tot.true_rel_res = std::max(tot.true_rel_res, inf.true_rel_res);
    if (inf.status_detail && !tot.status_detail) tot.status_detail = inf.status_detail;
    if (st != AAO_OK) {
      if (info) *info = tot;
      p->err = "window " + std::to_string(q) + ": " + p->err;
      return st;
    }
  }
  if (info) *info = tot;
  return AAO_OK;
}

}  // extern "C"

// ---- many independent problems at once --------------------------------------------------
#include <atomic>
#include <thread>

namespace {

// The lockstep batched solver needs plans whose Step (b) is the register-resident COCG with the same kind
// (Strang spectra or tau), the same restart length and no per-plan extras (warm start, recording, P(m)).
int lockstep_kind(int n, aao_plan* const* plans) {
  int kind = 0;
  for (int i = 0; i < n; ++i) {
    const aao_plan* p = plans[i];
    const int k = (p->opts.inner == AAO_INNER_TAU) ? 1 : (p->opts.inner == AAO_INNER_STRANG && p->sconv ? 2 : 0);
    if (p->dim != 1 || !p->mixed || p->cocg_threads == 0 || p->tm || p->direct || p->fno || p->rec_cap > p->rec_count ||
        p->prof_on || p->opts.poly_m != 0 || p->m != plans[0]->m || k == 0 || (kind && k != kind))
      return 0;
    kind = k;
  }
  return kind;
}

struct LockstepInst {
  aao_plan* p;
  const double* F;
  double* U;
  cudaStream_t own, saved;
  cudaEvent_t ev;
  double nF = 0;
  bool zero_guess = false, done = false, in_cycle = false;
  aao_status st = AAO_ENOCONV;
  aao_info inf{};
};

// Restarted FGMRES of all instances in lockstep: every Arnoldi step runs Steps (a) and (c), the matvec and
// CGS2 of each active instance on its own stream, and Step (b) of all of them as ONE launch
// (launch_cocg_batched) on the first instance's stream, joined by events.  Givens rotations stay on the
// device (one FGMRES state per plan); the host reads every active instance's state once per step.
aao_status solve_lockstep(int n, aao_plan* const* plans, const double* const* F, double* const* U, aao_info* infos,
                          int kind) {
  std::vector<LockstepInst> L(n);
  aao_status result = AAO_OK;
  std::string err;
  auto cleanup = [&]() {
    for (auto& x : L) {
      if (x.own) {
        cudaStreamSynchronize(x.own);
        cudaStreamDestroy(x.own);
      }
      if (x.ev) cudaEventDestroy(x.ev);
      if (x.p) x.p->stream = x.saved;
    }
  };
  int nt = 64, max_logL = 0, total_sys = 0;
  for (int i = 0; i < n; ++i) {
    L[i].p = plans[i];
    L[i].F = F[i];
    L[i].U = U[i];
    L[i].saved = plans[i]->stream;
    cudaStreamSynchronize(L[i].saved);  // the caller's pending work on the plan's stream comes first
    if (cudaStreamCreateWithFlags(&L[i].own, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&L[i].ev, cudaEventDisableTiming) != cudaSuccess) {
      cleanup();
      return fail(nullptr, AAO_ECUDA, "stream or event creation failed");
    }
    plans[i]->stream = L[i].own;
    if (ensure_dev_state(plans[i]) != AAO_OK) {
      err = plans[i]->err;
      cleanup();
      return fail(nullptr, AAO_ENOMEM, err);
    }
    nt = std::max(nt, plans[i]->cocg_threads);
    max_logL = std::max(max_logL, plans[i]->logL);
    total_sys += plans[i]->nsys;
  }
  aao_plan* p0 = plans[0];
  cudaStream_t master = L[0].own;
  cudaEvent_t ev_cocg = nullptr;
  aao::CocgBatchInst* insts_d = nullptr;
  int2* work_d = nullptr;
  int2* work_h = nullptr;
  auto release = [&]() {
    if (ev_cocg) cudaEventDestroy(ev_cocg);
    if (insts_d) cudaFree(insts_d);
    if (work_d) cudaFree(work_d);
    if (work_h) cudaFreeHost(work_h);
    cleanup();
  };
#define LS_CK(call, what)                                                                      \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      release();                                                                               \
      return fail(nullptr, AAO_ECUDA, std::string(what) + ": " + cudaGetErrorString(e_));     \
    }                                                                                          \
  } while (0)
#define LS_TRY(i, call)                                                                        \
  do {                                                                                         \
    aao_status s_ = (call);                                                                    \
    if (s_ != AAO_OK) {                                                                        \
      err = "instance " + std::to_string(i) + ": " + L[i].p->err;                             \
      release();                                                                               \
      return fail(nullptr, s_, err);                                                           \
    }                                                                                          \
  } while (0)
  LS_CK(cudaEventCreateWithFlags(&ev_cocg, cudaEventDisableTiming), "event");
  LS_CK(cudaMalloc(&insts_d, (size_t)n * sizeof(aao::CocgBatchInst)), "cudaMalloc");
  LS_CK(cudaMalloc(&work_d, (size_t)std::max(total_sys, 1) * sizeof(int2)), "cudaMalloc");
  LS_CK(cudaMallocHost(&work_h, (size_t)std::max(total_sys, 1) * sizeof(int2)), "cudaMallocHost");
  {
    std::vector<aao::CocgBatchInst> h(n);
    for (int i = 0; i < n; ++i) {
      aao_plan* p = plans[i];
      h[i].xb = (float2*)p->spec;
      h[i].M = p->M;
      h[i].logL = p->logL;
      h[i].nsys = p->nsys;
      h[i].tb = aao::CocgTables32{p->twL32, p->Ebr32, p->lambda, p->chirp32, p->chat32, p->seig32, p->tau32, p->sconv};
      h[i].tol = (float)p->opts.inner_tol;
      h[i].maxit = p->opts.inner_maxit;
      h[i].iters = p->iters;
      h[i].flags = p->flags;
    }
    LS_CK(cudaMemcpyAsync(insts_d, h.data(), (size_t)n * sizeof(aao::CocgBatchInst), cudaMemcpyHostToDevice, master),
          "descriptor upload");
    LS_CK(cudaStreamSynchronize(master), "descriptor upload");
  }
  // ||F||^2 and ||U||^2 of every instance (as aao_gmres_solve)
  const int nb = aao::blas_partial_blocks();
  for (int i = 0; i < n; ++i) {
    aao_plan* p = L[i].p;
    LS_CK(aao::launch_dots(F[i], F[i], 0, 1, p->n, p->partial, p->stream), "norms");
    LS_CK(aao::launch_dots(U[i], U[i], 0, 1, p->n, p->partial + nb, p->stream), "norms");
    LS_CK(aao::launch_reduce_partials(p->partial, nb, 1, p->hdev, p->stream), "norms");
    LS_CK(aao::launch_reduce_partials(p->partial + nb, nb, 1, p->hdev + 1, p->stream), "norms");
    LS_CK(cudaMemcpyAsync(p->pinned, p->hdev, 2 * sizeof(double), cudaMemcpyDeviceToHost, p->stream), "norms");
    p->prof_launches[ST_VEC] += 4;
  }
  for (int i = 0; i < n; ++i) {
    aao_plan* p = L[i].p;
    LS_CK(cudaStreamSynchronize(p->stream), "norms");
    L[i].nF = std::sqrt(p->pinned[0]);
    L[i].zero_guess = p->pinned[1] == 0.0;
    if (!std::isfinite(L[i].nF)) {
      L[i].done = true;
      L[i].st = AAO_ENONFINITE;
      p->err = "non-finite right-hand side";
    } else if (L[i].nF == 0.0) {
      LS_CK(cudaMemsetAsync(U[i], 0, p->n * sizeof(double), p->stream), "memset");
      L[i].done = true;
      L[i].st = AAO_OK;
    } else {
      GmresDevState& hs = *p->gd_host;
      const size_t tail = sizeof(GmresDevState) - offsetof(GmresDevState, thr);
      std::memset(&hs.thr, 0, tail);
      hs.thr = 0.5 * p->opts.tol * L[i].nF;
      LS_CK(cudaMemcpyAsync(&p->gd->thr, &hs.thr, tail, cudaMemcpyHostToDevice, p->stream), "state upload");
    }
  }
  const size_t tail = sizeof(GmresDevState) - offsetof(GmresDevState, thr);
  const int m = p0->m;
  for (int cycle = 0; cycle <= p0->opts.max_cycles; ++cycle) {
    // residuals r0 = F - calA U (or F) and beta of every unfinished instance
    bool any = false;
    for (int i = 0; i < n; ++i) {
      if (L[i].done) continue;
      aao_plan* p = L[i].p;
      if (cycle == 0 && L[i].zero_guess) {
        LS_CK(cudaMemcpyAsync(p->W, F[i], p->n * sizeof(double), cudaMemcpyDeviceToDevice, p->stream), "copy");
        p->pinned[0] = L[i].nF * L[i].nF;
      } else {
        LS_TRY(i, matvec_any(p, U[i], false, F[i], p->W, p->sq));
        L[i].inf.matvecs++;
        p->prof_launches[ST_VEC] += 1;
        LS_CK(aao::launch_reduce_partials(p->sq, (int)p->nsq, 1, p->hdev, p->stream), "reduce");
        LS_CK(cudaMemcpyAsync(p->pinned, p->hdev, sizeof(double), cudaMemcpyDeviceToHost, p->stream), "readback");
      }
    }
    for (int i = 0; i < n; ++i) {
      if (L[i].done) continue;
      aao_plan* p = L[i].p;
      LS_CK(cudaStreamSynchronize(p->stream), "residual");
      const double beta = std::sqrt(p->pinned[0]);
      L[i].in_cycle = false;
      if (!std::isfinite(beta)) {
        L[i].done = true;
        L[i].st = AAO_ENONFINITE;
        p->err = "non-finite residual";
        continue;
      }
      L[i].inf.true_rel_res = beta / L[i].nF;
      L[i].inf.cycles = cycle;
      if (L[i].inf.true_rel_res <= p->opts.tol) {
        L[i].done = true;
        L[i].st = AAO_OK;
        continue;
      }
      if (cycle == p0->opts.max_cycles) {
        L[i].done = true;
        L[i].st = AAO_ENOCONV;
        p->err = "FGMRES did not reach the tolerance within max_cycles";
        continue;
      }
      L[i].in_cycle = true;
      any = true;
      cycle_init_kernel<<<1, 1, 0, p->stream>>>(p->gd, p->hdev, m, 0, 0);
      LS_CK(cudaGetLastError(), "cycle init");
      LS_CK(aao::launch_scale_to_ff((float2*)(void*)p->V, p->W, &p->gd->inv_beta, 0.0, p->n, p->stream), "scale");
      p->prof_launches[ST_VEC] += 2;
    }
    if (!any) break;
    for (int j = 0; j < m; ++j) {
      // Step (a) of every instance still in its cycle, then Step (b) of all of them in one launch
      int nwork = 0;
      for (int i = 0; i < n; ++i) {
        if (!L[i].in_cycle) continue;
        aao_plan* p = L[i].p;
        const float2* vj = (const float2*)(const void*)(p->V + (size_t)j * p->n);
        LS_CK(aao::launch_tdft_fwd_f32_ff(vj, (float2*)p->spec, p->M, p->Nt, p->sfwd32, p->twNt32, p->stream),
              "Step (a)");
        p->prof_launches[ST_TDFT_FWD] += 1;
        LS_CK(cudaEventRecord(L[i].ev, p->stream), "event");
        LS_CK(cudaStreamWaitEvent(master, L[i].ev, 0), "event wait");
        for (int q = 0; q < p->nsys; ++q) work_h[nwork++] = make_int2(i, q);
      }
      if (nwork == 0) break;
      LS_CK(cudaMemcpyAsync(work_d, work_h, (size_t)nwork * sizeof(int2), cudaMemcpyHostToDevice, master),
            "work upload");
      LS_CK(aao::launch_cocg_batched(insts_d, work_d, nwork, kind, nt, max_logL, master), "Step (b)");
      p0->prof_launches[ST_COCG] += 1;
      LS_CK(cudaEventRecord(ev_cocg, master), "event");
      // Step (c), the matvec and CGS2 of each, the Givens update on the device
      for (int i = 0; i < n; ++i) {
        if (!L[i].in_cycle) continue;
        aao_plan* p = L[i].p;
        LS_CK(cudaStreamWaitEvent(p->stream, ev_cocg, 0), "event wait");
        iter_stats_accum_kernel<<<1, 256, 0, p->stream>>>(p->iters, p->flags, p->nsys, p->gd);
        LS_CK(cudaGetLastError(), "stats");
        float* zj = (float*)p->Z + (size_t)j * p->n;
        LS_CK(aao::launch_tdft_inv_f32((const float2*)p->spec, zj, p->M, p->Nt, p->sinv32, p->twNt32, p->stream),
              "Step (c)");
        p->prof_launches[ST_TDFT_INV] += 1;
        p->prof_launches[ST_VEC] += 1;
        LS_TRY(i, arnoldi_orthogonalise(p, j));
        L[i].inf.matvecs++;
        givens_kernel<<<1, 1, 0, p->stream>>>(p->gd, p->hdev, j, m, 0, 0);
        LS_CK(cudaGetLastError(), "Givens");
        float2* w = (float2*)(void*)(p->V + (size_t)(j + 1) * p->n);
        LS_CK(aao::launch_scale_ff(w, &p->gd->inv_hn, 0.0, p->n, p->stream), "scale");
        p->prof_launches[ST_VEC] += 2;
        LS_CK(cudaMemcpyAsync(&p->gd_host->thr, &p->gd->thr, tail, cudaMemcpyDeviceToHost, p->stream), "readback");
      }
      if (j + 1 == m) break;
      for (int i = 0; i < n; ++i) {
        if (!L[i].in_cycle) continue;
        LS_CK(cudaStreamSynchronize(L[i].p->stream), "step");
        if (!L[i].p->gd_host->active) L[i].in_cycle = false;
      }
    }
    // end of the cycle: least squares and U += Z y for every instance that ran steps
    for (int i = 0; i < n; ++i) {
      if (L[i].done) continue;
      aao_plan* p = L[i].p;
      lsq_kernel<<<1, 1, 0, p->stream>>>(p->gd);
      LS_CK(cudaGetLastError(), "least squares");
      LS_CK(cudaMemcpyAsync(&p->gd_host->thr, &p->gd->thr, tail, cudaMemcpyDeviceToHost, p->stream), "readback");
      LS_CK(cudaStreamSynchronize(p->stream), "cycle");
      p->prof_launches[ST_VEC] += 1;
      GmresDevState& hs = *p->gd_host;
      if (hs.status != 0) {
        L[i].done = true;
        L[i].st = (aao_status)hs.status;
        p->err = L[i].st == AAO_EBREAKDOWN ? "GMRES breakdown" : "non-finite Arnoldi vector";
        continue;
      }
      if (hs.jdone > 0) {
        LS_CK(aao::launch_zy_update_f32(U[i], (const float*)p->Z, p->n, hs.jdone, p->n, p->gd->y, p->stream),
              "update");
        p->prof_launches[ST_VEC] += 1;
      }
    }
  }
  for (int i = 0; i < n; ++i) {
    aao_plan* p = L[i].p;
    LS_CK(cudaStreamSynchronize(p->stream), "final");
    GmresDevState& hs = *p->gd_host;
    aao_info& inf = L[i].inf;
    if (p->gd && L[i].nF > 0 && std::isfinite(L[i].nF)) {
      inf.outer_iters = hs.outer_total;
      inf.inner_iters_max = hs.inner_max;
      inf.inner_iters_sum = hs.inner_sum;
      inf.warm_accepted = hs.accepted;
      if (hs.flag_max != 0)
        inf.status_detail = hs.flag_max == 1 ? AAO_ENOCONV : (hs.flag_max == 2 ? AAO_EBREAKDOWN : AAO_ENONFINITE);
    }
    if (infos) infos[i] = inf;
    if (L[i].st != AAO_OK && result == AAO_OK) {
      result = L[i].st;
      err = "instance " + std::to_string(i) + ": " + p->err;
    }
  }
  release();
#undef LS_CK
#undef LS_TRY
  if (result != AAO_OK) return fail(nullptr, result, err);
  return AAO_OK;
}

}  // namespace

extern "C" aao_status aao_solve_batched(int n, aao_plan* const* plans, const double* const* F, double* const* U,
                                        aao_info* infos, int max_workers) {
  if (n < 0 || (n > 0 && (!plans || !F || !U))) return fail(nullptr, AAO_EINVAL, "bad batched arguments");
  if (n == 0) return AAO_OK;
  for (int i = 0; i < n; ++i)
    if (!plans[i] || !F[i] || !U[i]) return fail(nullptr, AAO_EINVAL, "null plan or vector in the batch");
  if (max_workers <= 0) {
    const int kind = lockstep_kind(n, plans);
    if (kind) return solve_lockstep(n, plans, F, U, infos, kind);
  }
  // one non-blocking stream per instance so that the instances' kernels overlap on the GPU
  std::vector<cudaStream_t> saved(n), own(n, nullptr);
  for (int i = 0; i < n; ++i) {
    saved[i] = plans[i]->stream;
    if (cudaStreamCreateWithFlags(&own[i], cudaStreamNonBlocking) != cudaSuccess) {
      for (int k = 0; k < i; ++k) cudaStreamDestroy(own[k]);
      return fail(nullptr, AAO_ECUDA, "cudaStreamCreateWithFlags failed");
    }
    // the caller's pending work on the plan's own stream comes first
    cudaStreamSynchronize(saved[i]);
    plans[i]->stream = own[i];
  }
  // largest instances first
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return plans[a]->n > plans[b]->n; });
  std::vector<aao_status> st(n, AAO_OK);
  std::vector<aao_info> inf(n);
  std::atomic<int> next(0);
  int dev = 0;
  cudaGetDevice(&dev);
  auto worker = [&]() {
    cudaSetDevice(dev);
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= n) break;
      const int i = order[k];
      st[i] = aao_gmres_solve(plans[i], F[i], U[i], &inf[i]);
    }
  };
  const int nw = std::max(1, std::min(n, max_workers > 0 ? max_workers : 32));
  std::vector<std::thread> pool;
  for (int w = 0; w < nw; ++w) pool.emplace_back(worker);
  for (auto& t : pool) t.join();
  aao_status result = AAO_OK;
  for (int i = 0; i < n; ++i) {
    cudaStreamSynchronize(own[i]);
    plans[i]->stream = saved[i];
    cudaStreamDestroy(own[i]);
    if (infos) infos[i] = inf[i];
    if (st[i] != AAO_OK && result == AAO_OK) {
      result = st[i];
      g_create_error = "instance " + std::to_string(i) + ": " + plans[i]->err;
    }
  }
  return result;
}
