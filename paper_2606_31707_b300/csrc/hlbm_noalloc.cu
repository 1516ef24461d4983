// Objective evaluation that allocates nothing.
//
// Some callers cannot call cudaMalloc: code that runs while another
// component owns the device memory budget (a fixed arena or memory pool that
// must not grow), code on a latency-critical path where an allocation's
// implicit device synchronisation is not acceptable, and plug-in hosts that
// forbid their plug-ins to allocate.  For them this file provides
// hlbm_objective_noalloc: it evaluates J_FFA or J_DISS (and optionally
// dJ/df and dJ/dd) of a caller-held canonical population field without any
// context and without any allocation.  The caller passes every input and
// output; the only scratch -- the per-block partial sums of J -- lives in the
// fixed file-scope device array below, which every GPU that loads this
// library keeps until the process exits.
//
// Scratch rules:
//  * The array holds at most HLBM_NOALLOC_MAX_BLOCKS partial sums (512 KiB);
//    larger regions are rejected with HLBM_ESCRATCH.
//  * All calls on a device share the array and it keeps the last call's
//    contents.  Each call writes every slot it later reads, so no clearing is
//    needed; calls that overlap on the GPU (different streams or threads
//    without ordering between them) race on it.
//  * Host code cannot use the array's name as a device address.  Its address
//    is looked up once per device with cudaGetSymbolAddress (with that device
//    current) on the first call there; make that first call before any stream
//    capture.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/hlbm.h"
#include "hlbm_device.cuh"

namespace hlbm_noalloc {

using namespace hlbm;

constexpr int NTB = 128;

static __device__ __align__(256) double g_partials[HLBM_NOALLOC_MAX_BLOCKS];

struct EvalArgs {
  const double* f;  // q x N canonical populations
  const double* d;  // N porosity
  int nx, ny, nz;
  long long N;
  int box[6];
  int objective;
  double tau0, kles, nu0, u_in;
  double us[3];
  double* dJdf;     // q x N or null
  double* dJdd;     // N or null
  double* partials;
};

// J and its partials at one cell, same definitions as the averaging pass of
// the primal kernel (Sec. 4.2 for J_FFA, Sec. 4.3 for J_DISS).
template <int Q>
__global__ void __launch_bounds__(NTB) k_eval(EvalArgs a) {
  using L = Lat<Q>;
  using R = double;
  const int bx = a.box[1] - a.box[0];
  const int xl = blockIdx.x * NTB + threadIdx.x;
  double jp = 0.0;
  if (xl < bx) {
    const int x = a.box[0] + xl, y = a.box[2] + blockIdx.y, z = a.box[4] + blockIdx.z;
    const long long cell = (long long)x + (long long)a.nx * ((long long)y + (long long)a.ny * z);
    R f[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = a.f[(long long)i * a.N + cell];
    const R d = a.d[cell];
    R rho;
    Vec3<R> u;
    moments<Q>(f, rho, u);
    const R one_d = R(1) - d;
    const Vec3<R> ut{d * u.x + one_d * a.us[0], d * u.y + one_d * a.us[1], d * u.z + one_d * a.us[2]};
    const R uu = dot3(ut, ut);
    R fneq[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) fneq[i] = f[i] - feq_i<Q>(i, rho, ut, uu);
    const Sym<R> P = second_moment<Q, R>(fneq);
    const R nP = sqrt(sym_norm2(P));
    const R tau = a.kles > 0 ? tau_smagorinsky<R>(a.tau0, a.kles, nP) : a.tau0;
    if (a.objective == HLBM_OBJ_DRAG_FFA) {
      const R c0 = u.x * u.x - R(1.0 / 3.0);
      const R c1 = a.u_in - R(2) * u.x;
      if (a.dJdf) {
#pragma unroll
        for (int i = 0; i < Q; ++i)
          a.dJdf[(long long)i * a.N + cell] = c0 + (L::cx(i) > 0 ? c1 : (L::cx(i) < 0 ? -c1 : R(0)));
      }
      if (a.dJdd) a.dJdd[cell] = 0.0;
      jp = rho * u.x * (a.u_in - u.x) + R(1.0 / 3.0) * (R(1) - rho);
    } else {
      const R uu_raw = dot3(u, u);
      jp = R(4.5) * a.nu0 * nP * nP / (tau * tau) + one_d / a.tau0 * uu_raw;
      R fac = R(1) / (tau * tau);
      if (a.kles > 0) fac -= nP * a.kles / (tau * tau * tau * (R(2) * tau - a.tau0));
      fac *= R(9) * a.nu0;
      const Vec3<R> PU = sym_mul(P, ut);
      if (a.dJdf) {
        const R uPu = dot3(ut, PU);
        const R trP = P.xx + P.yy + P.zz;
        const R uPU = dot3(u, PU);
        const R c2 = one_d / a.tau0 * R(2) / rho;
#pragma unroll
        for (int j = 0; j < Q; ++j) {
          const R pdp = xi_P_xi<Q>(j, P) - trP * R(1.0 / 3.0) - uPu - R(2) * d * (xi_dot<Q>(j, PU) - uPU);
          a.dJdf[(long long)j * a.N + cell] = fac * pdp + c2 * (xi_dot<Q>(j, u) - uu_raw);
        }
      }
      if (a.dJdd) {
        const Vec3<R> v{u.x - a.us[0], u.y - a.us[1], u.z - a.us[2]};
        a.dJdd[cell] = fac * (-R(2) * rho * dot3(v, PU)) - uu_raw / a.tau0;
      }
    }
  }
  __shared__ double sh[NTB / 32];
  const double s = block_sum<NTB>(jp, sh);
  if (threadIdx.x == 0) a.partials[block_linear()] = s;
}

__global__ void k_sum(const double* part, long long n, double* out) {
  __shared__ double sh[256 / 32];
  double acc = 0.0;
  for (long long k = threadIdx.x; k < n; k += blockDim.x) acc += part[k];
  const double t = block_sum<256>(acc, sh);
  if (threadIdx.x == 0) *out = t;
}

// device address of g_partials, looked up once per device
constexpr int kMaxDevices = 256;
std::mutex g_mutex;
double* g_ptr[kMaxDevices] = {};

int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return HLBM_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) {
      cudaGetLastError();
      return HLBM_ECUDA;
    }
    g_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_ptr[dev];
  return HLBM_OK;
}

}  // namespace hlbm_noalloc

extern "C" int hlbm_objective_noalloc(int lattice, const int dims[3], double tau, double Cs,
                                      double u_in, const double u_solid[3], int objective,
                                      const int region[6], const double* f, const double* d,
                                      double* J, double* dJdf, double* dJdd, void* stream) {
  using namespace hlbm_noalloc;
  if ((lattice != 9 && lattice != 19) || !dims || !region || !f || !d || !J) return HLBM_EINVAL;
  if (dims[0] < 4 || dims[1] < 1 || dims[2] < 1 || (lattice == 9 && dims[2] != 1)) return HLBM_EINVAL;
  if (!(tau > 0.5) || !(Cs >= 0.0)) return HLBM_EINVAL;
  if (objective != HLBM_OBJ_DRAG_FFA && objective != HLBM_OBJ_DISSIPATION) return HLBM_EINVAL;
  const int* b = region;
  if (b[0] < 0 || b[1] > dims[0] || b[0] >= b[1] || b[2] < 0 || b[3] > dims[1] || b[2] >= b[3] ||
      b[4] < 0 || b[5] > dims[2] || b[4] >= b[5])
    return HLBM_EINVAL;
  if (objective == HLBM_OBJ_DRAG_FFA && b[1] != b[0] + 1) return HLBM_EINVAL;
  if (b[3] - b[2] > 65535 || b[5] - b[4] > 65535) return HLBM_EINVAL;
  const long long gx = (b[1] - b[0] + NTB - 1) / NTB;
  const long long nblocks = gx * (b[3] - b[2]) * (b[5] - b[4]);
  if (nblocks > HLBM_NOALLOC_MAX_BLOCKS) return HLBM_ESCRATCH;
  double* part = nullptr;
  int rc = scratch_address(&part);
  if (rc != HLBM_OK) return rc;
  EvalArgs a{};
  a.f = f;
  a.d = d;
  a.nx = dims[0]; a.ny = dims[1]; a.nz = dims[2];
  a.N = (long long)dims[0] * dims[1] * dims[2];
  for (int k = 0; k < 6; ++k) a.box[k] = b[k];
  a.objective = objective;
  a.tau0 = tau;
  a.kles = 4.5 * sqrt(2.0) * Cs * Cs;
  a.nu0 = (tau - 0.5) / 3.0;
  a.u_in = u_in;
  for (int k = 0; k < 3; ++k) a.us[k] = u_solid ? u_solid[k] : 0.0;
  a.dJdf = dJdf;
  a.dJdd = dJdd;
  a.partials = part;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  dim3 grid((unsigned)gx, b[3] - b[2], b[5] - b[4]);
  if (lattice == 9) k_eval<9><<<grid, NTB, 0, s>>>(a);
  else k_eval<19><<<grid, NTB, 0, s>>>(a);
  k_sum<<<1, 256, 0, s>>>(part, nblocks, J);
  if (cudaGetLastError() != cudaSuccess) return HLBM_ECUDA;
  return HLBM_OK;
}
