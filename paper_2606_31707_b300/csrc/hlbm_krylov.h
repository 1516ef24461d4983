// Krylov vector algebra of the adjoint GMRES solver (hlbm_krylov.cu); vectors
// of L elements of the adjoint arithmetic type, V holds nv consecutive vectors.
#pragma once

#include <cuda_runtime.h>

namespace hlbm {

constexpr int kKrylovBlocks = 1184;  // 8 blocks per SM on 148 SMs
// out[i] = w . V_i (fixed-order FP64 reduction through part[nv * kKrylovBlocks])
cudaError_t launch_mdot(const void* w, const void* V, int nv, long long L, bool dbl, double* part,
                        double* out, cudaStream_t s);
// w += sign * sum_i coef[i] V_i  (coef on the device)
cudaError_t launch_maxpy(void* w, const void* V, const double* coef, int nv, double sign,
                         long long L, bool dbl, cudaStream_t s);
// y = a x + b z (z may be null)
cudaError_t launch_lincomb(void* y, const void* x, double a, const void* z, double b, long long L,
                           bool dbl, cudaStream_t s);

}  // namespace hlbm
