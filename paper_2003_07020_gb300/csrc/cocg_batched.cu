// Step (b) of several independent problems in one launch (the batched solver of aao_solve_batched):
// the register-resident COCG of cocg_reg.cuh over a work list of (instance, shifted system) pairs, for
// every CTA size and both preconditioner kinds that use the register kernel (tau matrix, Strang spectra).
#include "cocg_reg.cuh"

namespace aao {

namespace {
template <int KIND, int NT>
cudaError_t launch_batched_one(const CocgBatchInst* insts, const int2* work, int nwork, int smem_logL, cudaStream_t s) {
  auto kern = cocg_reg_batched_kernel<KIND, NT>;
  cudaError_t e = allow_max_dynamic_smem(kern);
  if (e != cudaSuccess) return e;
  kern<<<nwork, NT, cocg_reg_smem(smem_logL), s>>>(insts, work);
  return cudaGetLastError();
}
template <int KIND>
cudaError_t launch_batched_kind(const CocgBatchInst* insts, const int2* work, int nwork, int nt, int smem_logL,
                                cudaStream_t s) {
  switch (nt) {
    case 64: return launch_batched_one<KIND, 64>(insts, work, nwork, smem_logL, s);
    case 128: return launch_batched_one<KIND, 128>(insts, work, nwork, smem_logL, s);
    case 256: return launch_batched_one<KIND, 256>(insts, work, nwork, smem_logL, s);
    case 512: return launch_batched_one<KIND, 512>(insts, work, nwork, smem_logL, s);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace

cudaError_t launch_cocg_batched(const CocgBatchInst* insts, const int2* work, int nwork, int kind, int nt,
                                int smem_logL, cudaStream_t s) {
  if (nwork <= 0) return cudaSuccess;
  if (kind == 1) return launch_batched_kind<1>(insts, work, nwork, nt, smem_logL, s);
  if (kind == 2) return launch_batched_kind<2>(insts, work, nwork, nt, smem_logL, s);
  return cudaErrorInvalidValue;
}

}  // namespace aao
