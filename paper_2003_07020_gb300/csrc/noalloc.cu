// aao_bc_precond_apply_noalloc: the mixed-precision preconditioner apply
// (Steps (a)-(c), the same kernels as aao_bc_precond_apply) for callers that
// cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not safe,
// e.g. a host callback or a solver embedded in another library that owns
// all device memory through its own pool, or a caller that must not trigger
// the implicit device synchronisation and fragmentation of an allocation in
// the middle of its own pipeline.  Such callers cannot create an aao_plan
// (plan creation allocates the Krylov workspace), so this entry point needs
// no plan: it takes the problem, the options, the input and output buffers,
// and keeps its spectrum scratch and tables in one fixed file-scope device
// array.
//
// The array is kNoAllocScratchBytes (16 MiB) and is held by every GPU that
// loads the library until the process exits.  Every call looks up its
// address on the current device with cudaGetSymbolAddress (a cached address
// would go stale when the context is recreated, e.g. after cudaDeviceReset).
// Every call reuses the whole array and overwrites what the previous call
// left there; nothing in it has to start at zero (each region is fully
// written before it is read).  Two calls whose work overlaps on the GPU
// (different streams, or different host threads) race on the array.
//
// The tables (twiddles, spectra, shifts, scalings) are built on the host and
// written into the array by small kernels that carry them in their launch
// parameters (up to kChunkBytes per launch), so a call copies nothing from
// pageable host memory and does not wait for work already queued on the
// caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/aao.h"
#include "kernels.h"
#include "setup.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// One launch's worth of table bytes, passed by value as the kernel's parameter (the kernel
// parameter space holds up to 32764 bytes).
constexpr unsigned kChunkBytes = 32 * 1024 - 64;
struct __align__(16) TableChunk {
  unsigned char* dst;
  unsigned int bytes;
  alignas(16) unsigned char data[kChunkBytes];
};
static_assert(sizeof(TableChunk) <= 32764 && kChunkBytes % 16 == 0, "one chunk must fit the parameter space");

// dst[0 .. bytes) = data[0 .. bytes); dst and data are 16-byte aligned.
__global__ void write_chunk_kernel(const __grid_constant__ TableChunk c) {
  const unsigned n16 = c.bytes / 16;
  const uint4* src = reinterpret_cast<const uint4*>(c.data);
  uint4* dst = reinterpret_cast<uint4*>(c.dst);
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += gridDim.x * blockDim.x) dst[i] = src[i];
  for (unsigned i = 16 * n16 + blockIdx.x * blockDim.x + threadIdx.x; i < c.bytes; i += gridDim.x * blockDim.x)
    c.dst[i] = c.data[i];
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

aao_status noalloc_fail(aao_status st, const std::string& msg) {
  aao::set_planless_error(msg);  // reported by aao_last_error(NULL)
  return st;
}

// Device address of the scratch array on the current device, looked up on every call.
aao_status scratch_address(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    return noalloc_fail(AAO_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  *out = p;
  return AAO_OK;
}

template <typename Td, typename Ts>
std::vector<Td> to_real(const std::vector<Ts>& v) {
  std::vector<Td> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = (Td)v[i];
  return o;
}
std::vector<float2> to_f2(const std::vector<aao::cd>& v) {
  std::vector<float2> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = float2{(float)v[i].real(), (float)v[i].imag()};
  return o;
}
std::vector<double2> to_d2(const std::vector<aao::cd>& v) {
  std::vector<double2> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = double2{v[i].real(), v[i].imag()};
  return o;
}

}  // namespace

extern "C" aao_status aao_bc_precond_apply_noalloc(const aao_problem* prob, const aao_opts* opts,
                                                   const double* v_dev, double* z_dev, void* cuda_stream) {
  if (!prob || !opts || !v_dev || !z_dev) return noalloc_fail(AAO_EINVAL, "null argument");
  if (prob->dim != 1) return noalloc_fail(AAO_EINVAL, "only dim = 1 is supported");
  if (opts->prec != AAO_PREC_MIXED) return noalloc_fail(AAO_EINVAL, "the no-allocation apply is mixed precision only");
  if (prob->M < 1 || prob->M > 8191) return noalloc_fail(AAO_EINVAL, "M must be in [1, 8191]");
  if (prob->Nt < 4 || prob->Nt > 65536 || (prob->Nt & (prob->Nt - 1)))
    return noalloc_fail(AAO_EINVAL, "Nt must be a power of two in [4, 65536]");
  {  // a time-DFT CTA holds all Nt rows of its column tile in shared memory
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return noalloc_fail(AAO_ECUDA, std::string("device query: ") + cudaGetErrorString(e));
    const int lim = aao::tdft_max_Nt(true, (size_t)optin);
    if (prob->Nt > lim)
      return noalloc_fail(AAO_EINVAL, "Nt must be at most " + std::to_string(lim) +
                                          " on this device (the time-DFT tile of Nt rows must fit in shared memory)");
  }
  if (!(opts->inner_tol > 0) || opts->inner_maxit < 1) return noalloc_fail(AAO_EINVAL, "bad inner options");
  if (opts->inner != AAO_INNER_STRANG && opts->inner != AAO_INNER_TAU)
    return noalloc_fail(AAO_EINVAL, "bad inner preconditioner");
  if (opts->inner == AAO_INNER_TAU && ((prob->M + 1) & prob->M))
    return noalloc_fail(AAO_EINVAL, "the tau preconditioner needs M+1 to be a power of two");
  aao::HostTables t;
  const char* emsg = nullptr;
  const double eps = prob->eps > 0 ? prob->eps : aao::default_eps(prob->T / (double)prob->Nt, true);
  if (!aao::build_tables(prob->M, prob->Nt, prob->T, prob->alpha, prob->kappa, eps, t, &emsg))
    return noalloc_fail(AAO_EINVAL, emsg);
  const int M = (int)t.M, Nt = (int)t.Nt, L = (int)t.L, nsys = Nt / 2 + 1;

  // layout of the scratch array
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off = align256(off + bytes); return o; };
  const size_t o_spec = take((size_t)nsys * M * sizeof(float2));
  const size_t o_iters = take((size_t)nsys * sizeof(int));
  const size_t o_flags = take((size_t)nsys * sizeof(int));
  const size_t o_twL = take((size_t)(L / 2) * sizeof(float2));
  const size_t o_Ebr = take((size_t)L * sizeof(float));
  const size_t o_lam = take((size_t)nsys * sizeof(double2));
  const size_t o_sfwd = take((size_t)Nt * sizeof(float));
  const size_t o_sinv = take((size_t)Nt * sizeof(float));
  const size_t o_twNt = take((size_t)(Nt / 2) * sizeof(float2));
  const size_t o_chirp = take((size_t)M * sizeof(float2));
  const size_t o_chat = take((size_t)L * sizeof(float2));
  const size_t o_seig = take((size_t)M * sizeof(float));
  const size_t o_tau = take((size_t)L * sizeof(float));
  if (off > kNoAllocScratchBytes)
    return noalloc_fail(AAO_EINVAL, "problem too large for the fixed no-allocation scratch: needs " +
                                        std::to_string(off) + " bytes, limit " +
                                        std::to_string(kNoAllocScratchBytes) + " (16 MiB)");
  void* base = nullptr;
  aao_status st = scratch_address(&base);
  if (st != AAO_OK) return st;
  unsigned char* b = static_cast<unsigned char*>(base);
  cudaStream_t s = (cudaStream_t)cuda_stream;

  // region o of the array <- bytes of host memory, through kernel parameters (see the file comment)
  TableChunk chunk;
  auto put = [&](size_t o, const void* src, size_t bytes) -> cudaError_t {
    const unsigned char* h = static_cast<const unsigned char*>(src);
    for (size_t done = 0; done < bytes; done += kChunkBytes) {
      const unsigned nb = (unsigned)std::min<size_t>(kChunkBytes, bytes - done);
      chunk.dst = b + o + done;  // o is 256-aligned and kChunkBytes a multiple of 16
      chunk.bytes = nb;
      std::memcpy(chunk.data, h + done, nb);
      write_chunk_kernel<<<8, 256, 0, s>>>(chunk);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  const std::vector<float2> twL = to_f2(t.tw_L), twNt = to_f2(t.tw_Nt), chirp = to_f2(t.chirp),
                            chat = to_f2(t.chirp_hat_f);
  const std::vector<double2> lam = to_d2(t.lambda);
  const std::vector<float> Ebr = to_real<float>(t.Ehat_f), sfwd = to_real<float>(t.scale_fwd),
                           sinv = to_real<float>(t.scale_inv), seig = to_real<float>(t.strang_eig),
                           tau = t.tau_ok ? to_real<float>(t.tau_eig_f) : std::vector<float>((size_t)L, 0.0f);
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = put(o_twL, twL.data(), twL.size() * sizeof(float2));
  if (e == cudaSuccess) e = put(o_Ebr, Ebr.data(), Ebr.size() * sizeof(float));
  if (e == cudaSuccess) e = put(o_lam, lam.data(), lam.size() * sizeof(double2));
  if (e == cudaSuccess) e = put(o_sfwd, sfwd.data(), sfwd.size() * sizeof(float));
  if (e == cudaSuccess) e = put(o_sinv, sinv.data(), sinv.size() * sizeof(float));
  if (e == cudaSuccess) e = put(o_twNt, twNt.data(), twNt.size() * sizeof(float2));
  if (e == cudaSuccess) e = put(o_chirp, chirp.data(), chirp.size() * sizeof(float2));
  if (e == cudaSuccess) e = put(o_chat, chat.data(), chat.size() * sizeof(float2));
  if (e == cudaSuccess) e = put(o_seig, seig.data(), seig.size() * sizeof(float));
  if (e == cudaSuccess) e = put(o_tau, tau.data(), tau.size() * sizeof(float));
  if (e != cudaSuccess) return noalloc_fail(AAO_ECUDA, std::string("table upload: ") + cudaGetErrorString(e));

  float2* spec = reinterpret_cast<float2*>(b + o_spec);
  const float2* twNt_d = reinterpret_cast<const float2*>(b + o_twNt);
  e = aao::launch_tdft_fwd_f32(v_dev, spec, M, Nt, reinterpret_cast<const float*>(b + o_sfwd), twNt_d, s);
  if (e == cudaSuccess) {
    aao::CocgTables32 tb{reinterpret_cast<const float2*>(b + o_twL), reinterpret_cast<const float*>(b + o_Ebr),
                         reinterpret_cast<const double2*>(b + o_lam), reinterpret_cast<const float2*>(b + o_chirp),
                         reinterpret_cast<const float2*>(b + o_chat), reinterpret_cast<const float*>(b + o_seig),
                         reinterpret_cast<const float*>(b + o_tau)};
    e = aao::launch_cocg_f32(spec, nullptr, nullptr, M, t.logL, nsys, (int)opts->inner, tb, (float)opts->inner_tol,
                             opts->inner_maxit, reinterpret_cast<int*>(b + o_iters),
                             reinterpret_cast<int*>(b + o_flags), nsys, s);
  }
  if (e == cudaSuccess)
    e = aao::launch_tdft_inv_f32_to_f64(spec, z_dev, M, Nt, reinterpret_cast<const float*>(b + o_sinv), twNt_d, s);
  if (e != cudaSuccess) return noalloc_fail(AAO_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return AAO_OK;
}
