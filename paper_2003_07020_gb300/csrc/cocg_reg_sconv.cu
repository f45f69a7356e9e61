// Register-resident FP32 COCG of Step (b) (Sec. 3.1) with the Strang circulant, applied
// through its precomputed per-system spectra, as the preconditioner: every CTA size, with and
// without a learned initial guess (templates in cocg_reg.cuh).
#include "cocg_reg.cuh"

namespace aao {

cudaError_t launch_cocg_reg_sconv(float2* xb, const float2* x0, int M, int logL, int nsys, const CocgTables32& tb,
                                  float tol, int maxit, int* iters, int* flags, int grid, int nt, cudaStream_t s) {
  return launch_reg_kind<2>(xb, x0, M, logL, nsys, tb, tol, maxit, iters, flags, grid, nt, s);
}

}  // namespace aao
