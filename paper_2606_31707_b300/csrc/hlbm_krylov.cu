// Vector kernels of the restarted GMRES solver for the adjoint fixed point.
//
// The adjoint iteration of the paper (Eq. adjoint_steady / adjoint_unsteady)
// is a fixed-point iteration lambda <- A^T lambda + g_bar whose convergence
// rate is the spectral radius of A^T; on the mean flow of the Karman case it
// needs ~10^5 sweeps for a 1e-4 update.  The same fixed point solves a linear
// system, which a Krylov method reaches in far fewer operator applications.
// These kernels supply the vector algebra (dot products with fixed-order FP64
// reductions, multi-vector updates); the operator itself is two adjoint sweeps
// of hlbm_adjoint.cu.  Vectors are q planes of `pitch` elements of the adjoint
// arithmetic type, the layout of the adjoint state; padding entries stay zero.
#include <cuda_runtime.h>

#include "hlbm_internal.h"
#include "hlbm_krylov.h"

namespace hlbm {

constexpr int KB = 256;          // threads per block of the vector kernels
constexpr int KGROUP = 8;        // vectors dotted per pass over w

// part[i * nb + b] = sum over block b's share of w . V_i, i < nv.  Products and
// each thread's running sum (a few dozen elements) use the vector type; the
// sums across threads and blocks are FP64 (B300 issues FP64 at a small
// fraction of its FP32 rate, so FP64 stays out of the per-element path).
template <class R>
__global__ void __launch_bounds__(KB) k_mdot(const R* w, const R* V, int nv, long long L,
                                             double* part) {
  __shared__ double sh[KB / 32];
  const int nb = gridDim.x;
  for (int i0 = 0; i0 < nv; i0 += KGROUP) {
    const int ng = nv - i0 < KGROUP ? nv - i0 : KGROUP;
    R acc[KGROUP];
#pragma unroll
    for (int k = 0; k < KGROUP; ++k) acc[k] = R(0);
    for (long long e = blockIdx.x * (long long)KB + threadIdx.x; e < L;
         e += (long long)nb * KB) {
      const R we = w[e];
#pragma unroll
      for (int k = 0; k < KGROUP; ++k)
        if (k < ng) acc[k] += we * V[(long long)(i0 + k) * L + e];
    }
#pragma unroll
    for (int k = 0; k < KGROUP; ++k) {
      if (k >= ng) break;
      const double s = block_sum<KB>((double)acc[k], sh);
      if (threadIdx.x == 0) part[(long long)(i0 + k) * nb + blockIdx.x] = s;
    }
  }
}

// out[i] = sum_b part[i * nb + b] in a fixed order (one block per vector)
__global__ void k_mfinal(const double* part, int nb, double* out) {
  __shared__ double sh[KB / 32];
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += KB) acc += part[(long long)blockIdx.x * nb + b];
  const double s = block_sum<KB>(acc, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// w += sign * sum_i coef[i] V_i  (coefficients converted once per block)
template <class R>
__global__ void __launch_bounds__(KB) k_maxpy(R* w, const R* V, const double* coef, int nv,
                                              double sign, long long L) {
  __shared__ R cf[64];
  if (threadIdx.x < nv) cf[threadIdx.x] = (R)(sign * coef[threadIdx.x]);
  __syncthreads();
  for (long long e = blockIdx.x * (long long)KB + threadIdx.x; e < L;
       e += (long long)gridDim.x * KB) {
    R v = w[e];
    for (int i = 0; i < nv; ++i) v += cf[i] * V[(long long)i * L + e];
    w[e] = v;
  }
}

// y = a * x + b * z   (z may be null)
template <class R>
__global__ void __launch_bounds__(KB) k_lincomb(R* y, const R* x, double a, const R* z, double b,
                                                long long L) {
  const R ar = (R)a, br = (R)b;
  for (long long e = blockIdx.x * (long long)KB + threadIdx.x; e < L;
       e += (long long)gridDim.x * KB) {
    R v = ar * x[e];
    if (z) v += br * z[e];
    y[e] = v;
  }
}

static int vec_blocks(long long L) {
  long long b = (L + KB - 1) / KB;
  return (int)(b < 1 ? 1 : (b > kKrylovBlocks ? kKrylovBlocks : b));
}

cudaError_t launch_mdot(const void* w, const void* V, int nv, long long L, bool dbl, double* part,
                        double* out, cudaStream_t s) {
  const int nb = vec_blocks(L);
  if (dbl) k_mdot<double><<<nb, KB, 0, s>>>((const double*)w, (const double*)V, nv, L, part);
  else k_mdot<float><<<nb, KB, 0, s>>>((const float*)w, (const float*)V, nv, L, part);
  k_mfinal<<<nv, KB, 0, s>>>(part, nb, out);
  return cudaGetLastError();
}

cudaError_t launch_maxpy(void* w, const void* V, const double* coef, int nv, double sign,
                         long long L, bool dbl, cudaStream_t s) {
  const int nb = vec_blocks(L);
  if (dbl) k_maxpy<double><<<nb, KB, 0, s>>>((double*)w, (const double*)V, coef, nv, sign, L);
  else k_maxpy<float><<<nb, KB, 0, s>>>((float*)w, (const float*)V, coef, nv, sign, L);
  return cudaGetLastError();
}

cudaError_t launch_lincomb(void* y, const void* x, double a, const void* z, double b, long long L,
                           bool dbl, cudaStream_t s) {
  const int nb = vec_blocks(L);
  if (dbl) k_lincomb<double><<<nb, KB, 0, s>>>((double*)y, (const double*)x, a, (const double*)z, b, L);
  else k_lincomb<float><<<nb, KB, 0, s>>>((float*)y, (const float*)x, a, (const float*)z, b, L);
  return cudaGetLastError();
}

}  // namespace hlbm
