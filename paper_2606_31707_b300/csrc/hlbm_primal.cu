// Primal HLBM time step on sm_103a: fused collide + AA-pattern in-place
// streaming + inflow/outflow nodes, with the tracking averages of the
// mean-flow adjoint (Ito et al., Sec. 2.1-2.2 and Sec. 3.3) fused into the
// same pass.  One thread per cell; the thread of column nx-2 also owns the
// outflow cell nx-1 (whose canonical state f^eq(1, u(nx-2)) it derives from
// its own velocity), the thread of column 0 owns the inflow cell whose
// canonical state is the constant f^eq(1, u_in e_x).
//
// Memory traffic per cell and step (algorithmic): q loads + q stores of the
// population storage type + one porosity load; the averaging variant adds a
// read-modify-write of the FP64 sums it updates.
#include <cuda_runtime.h>

#include "hlbm_internal.h"

namespace hlbm {

template <int Q, class R>
__device__ __forceinline__ void equilibrium(R (&f)[Q], R rho, const Vec3<R>& u) {
  const R uu = dot3(u, u);
#pragma unroll
  for (int i = 0; i < Q; ++i) f[i] = feq_i<Q>(i, rho, u, uu);
}

// Collide the canonical state f of one cell, store it AA-style, and (ACC)
// add the cell's samples to the running averages.  Returns the velocity.
template <int Q, int S, bool ODD, bool LES, bool ACC>
__device__ __forceinline__ Vec3<typename Store<S>::real> cell_update(
    const PrimalArgs& a, typename Store<S>::mem* A, int x, int y, int z, long long cell,
    typename Store<S>::real (&f)[Q], typename Store<S>::real d, double (&jp)[2]) {
  using R = typename Store<S>::real;
  using L = Lat<Q>;
  const Grid& g = a.g;
  R rho;
  Vec3<R> u;
  moments<Q>(f, rho, u);
  if (!(rho > R(0)) || !(fabs((double)u.x) + fabs((double)u.y) + fabs((double)u.z) < 1e30))
    atomicOr(a.err, 1u);
  const R one_d = R(1) - d;
  const Vec3<R> ut{d * u.x + one_d * R(a.us[0]), d * u.y + one_d * R(a.us[1]),
                   d * u.z + one_d * R(a.us[2])};
  const R uu = dot3(ut, ut);
  R fneq[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) fneq[i] = f[i] - feq_i<Q>(i, rho, ut, uu);

  const R tau0 = R(a.tau0);
  R tau = tau0;
  Sym<R> P{0, 0, 0, 0, 0, 0};
  R nP = 0;
  const bool diss_here = ACC && (a.obj_mask & 2) && x >= a.db[0] && x < a.db[1] &&
                         y >= a.db[2] && y < a.db[3] && z >= a.db[4] && z < a.db[5];
  if (LES || diss_here) {
    P = second_moment<Q>(fneq);
    nP = sqrt_r<R>(sym_norm2(P));
  }
  if (LES) tau = tau_smagorinsky<R>(tau0, R(a.kles), nP);
  const R om = R(1) / tau;

  if (ACC) {
    const long long N = g.N;
#pragma unroll
    for (int i = 0; i < Q; ++i) a.fsum[(long long)i * N + cell] += (double)f[i];
    if (LES) a.tsum[cell] += (double)(tau - tau0);
    // far-field drag J_FFA on Gamma_J (Sec. 4.2): rho u_x (u0 - u_x) + c_s^2 (1 - rho)
    if ((a.obj_mask & 1) && x == a.ffa[0] && y >= a.ffa[1] && y < a.ffa[2] && z >= a.ffa[3] &&
        z < a.ffa[4]) {
      const R u0 = R(a.u_in);
      const R c0 = u.x * u.x - R(1.0 / 3.0);
      const R c1 = u0 - R(2) * u.x;
      double* gs = a.gsum[0];
#pragma unroll
      for (int i = 0; i < Q; ++i)
        gs[(long long)i * N + cell] += (double)(c0 + (L::cx(i) > 0 ? c1 : (L::cx(i) < 0 ? -c1 : R(0))));
      jp[0] += (double)(rho * u.x * (u0 - u.x) + R(1.0 / 3.0) * (R(1) - rho));
    }
    // dissipation J_DISS on Omega_J (Sec. 4.3): 2 nu S:S + (1-d)/tau0 u.u,
    // S = -3 Pi / (2 tau):  J = (9 nu / 2) |Pi|^2 / tau^2 + (1-d)/tau0 |u|^2
    if (diss_here) {
      const R nu = R(a.nu0);
      const R PP = nP * nP;
      const R uu_raw = dot3(u, u);
      const R J = R(4.5) * nu * PP / (tau * tau) + one_d / tau0 * uu_raw;
      // d/dq of |Pi|^2 / tau^2 with tau(|Pi|): 2 Pi:dPi [1/tau^2 - |Pi| k/(tau^3 (2 tau - tau0))]
      R fac = R(1) / (tau * tau);
      if (LES) fac -= nP * R(a.kles) / (tau * tau * tau * (R(2) * tau - tau0));
      fac *= R(9) * nu;
      const Vec3<R> PU = sym_mul(P, ut);
      const R uPu = dot3(ut, PU);
      const R trP = P.xx + P.yy + P.zz;
      const R uPU = dot3(u, PU);
      const R inv_rho = R(1) / rho;
      const R c2 = one_d / tau0 * R(2) * inv_rho;
      double* gs = a.gsum[1];
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        // Pi : dPi/df_j = xi P xi - tr P / 3 - u~ P u~ - 2 d (xi_j - u) . P u~
        const R pdp = xi_P_xi<Q>(j, P) - trP * R(1.0 / 3.0) - uPu - R(2) * d * (xi_dot<Q>(j, PU) - uPU);
        const R dJ = fac * pdp + c2 * (xi_dot<Q>(j, u) - uu_raw);
        gs[(long long)j * N + cell] += (double)dJ;
      }
      const Vec3<R> v{u.x - R(a.us[0]), u.y - R(a.us[1]), u.z - R(a.us[2])};
      const R dd = fac * (-R(2) * rho * dot3(v, PU)) - uu_raw / tau0;
      a.ddsum[1][cell] += (double)dd;
      jp[1] += (double)J;
    }
  }

#pragma unroll
  for (int i = 0; i < Q; ++i) f[i] -= om * fneq[i];
  aa_store<Q, S, ODD, +1>(A, g, x, y, z, cell, f);
  return u;
}

template <int Q, int S, bool ODD, bool LES, bool ACC>
__global__ void __launch_bounds__(NT) k_primal(PrimalArgs a) {
  using St = Store<S>;
  using R = typename St::real;
  const Grid& g = a.g;
  const int x = blockIdx.x * NT + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  auto* A = static_cast<typename St::mem*>(a.f);
  const R* dp = static_cast<const R*>(a.d);
  double jp[2] = {0.0, 0.0};
  if (x < g.nx - 1) {
    const long long cell = cell_of(g, x, y, z);
    R f[Q];
    if (x == 0) {
      equilibrium<Q, R>(f, R(1), Vec3<R>{R(a.u_in), R(0), R(0)});
    } else {
      aa_load<Q, S, ODD, +1>(A, g, x, y, z, cell, f);
    }
    const Vec3<R> u = cell_update<Q, S, ODD, LES, ACC>(a, A, x, y, z, cell, f, dp[cell], jp);
    if (x == g.nx - 2) {
      // outflow node: f^eq(1, u(nx-2)), then relaxed and streamed like any cell
      R fo[Q];
      equilibrium<Q, R>(fo, R(1), u);
      cell_update<Q, S, ODD, LES, ACC>(a, A, x + 1, y, z, cell + 1, fo, dp[cell + 1], jp);
    }
  }
  if (ACC) {
    __shared__ double sh[NT / 32];
#pragma unroll
    for (int o = 0; o < 2; ++o) {
      if (!(a.obj_mask & (1 << o))) continue;
      const double s = block_sum<NT>(jp[o], sh);
      if (threadIdx.x == 0) a.jblk[o][block_linear()] += s;
    }
  }
}

template <int Q, int S>
static cudaError_t launch_primal_qs(const PrimalArgs& a, bool odd, bool les, bool acc,
                                    cudaStream_t s) {
  dim3 grid((a.g.nx + NT - 1) / NT, a.g.ny, a.g.nz);
#define HLBM_L(O, L_, A_) k_primal<Q, S, O, L_, A_><<<grid, NT, 0, s>>>(a)
  if (!odd) {
    if (!les) { if (!acc) HLBM_L(false, false, false); else HLBM_L(false, false, true); }
    else      { if (!acc) HLBM_L(false, true, false);  else HLBM_L(false, true, true); }
  } else {
    if (!les) { if (!acc) HLBM_L(true, false, false);  else HLBM_L(true, false, true); }
    else      { if (!acc) HLBM_L(true, true, false);   else HLBM_L(true, true, true); }
  }
#undef HLBM_L
  return cudaGetLastError();
}

cudaError_t launch_primal(const PrimalArgs& a, int q, int storage, bool odd, bool les, bool acc,
                          cudaStream_t s) {
  if (q == 9) {
    switch (storage) {
      case ST_F64: return launch_primal_qs<9, ST_F64>(a, odd, les, acc, s);
      case ST_F32: return launch_primal_qs<9, ST_F32>(a, odd, les, acc, s);
      case ST_F16: return launch_primal_qs<9, ST_F16>(a, odd, les, acc, s);
      case ST_BF16: return launch_primal_qs<9, ST_BF16>(a, odd, les, acc, s);
    }
  } else if (q == 19) {
    switch (storage) {
      case ST_F64: return launch_primal_qs<19, ST_F64>(a, odd, les, acc, s);
      case ST_F32: return launch_primal_qs<19, ST_F32>(a, odd, les, acc, s);
      case ST_F16: return launch_primal_qs<19, ST_F16>(a, odd, les, acc, s);
      case ST_BF16: return launch_primal_qs<19, ST_BF16>(a, odd, les, acc, s);
    }
  }
  return cudaErrorInvalidValue;
}

// ----------------------------------------------------------------------------
// state readout / initialisation
// ----------------------------------------------------------------------------
template <int Q, int S, bool ODD>
__global__ void __launch_bounds__(NT) k_readout(const void* fv, Grid g, double u_in, double* fout,
                                                double* rho_out, double* u_out) {
  using St = Store<S>;
  using R = typename St::real;
  const int x = blockIdx.x * NT + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= g.nx) return;
  const auto* A = static_cast<const typename St::mem*>(fv);
  const long long cell = cell_of(g, x, y, z);
  R f[Q];
  if (x == 0) {
    equilibrium<Q, R>(f, R(1), Vec3<R>{R(u_in), R(0), R(0)});
  } else if (x == g.nx - 1) {
    R fi[Q];
    aa_load<Q, S, ODD, +1>(A, g, x - 1, y, z, cell - 1, fi);
    R r;
    Vec3<R> u;
    moments<Q>(fi, r, u);
    equilibrium<Q, R>(f, R(1), u);
  } else {
    aa_load<Q, S, ODD, +1>(A, g, x, y, z, cell, f);
  }
  if (fout) {
#pragma unroll
    for (int i = 0; i < Q; ++i) fout[(long long)i * g.N + cell] = (double)f[i];
  }
  if (rho_out || u_out) {
    R r;
    Vec3<R> u;
    moments<Q>(f, r, u);
    if (rho_out) rho_out[cell] = (double)r;
    if (u_out) {
      u_out[cell] = (double)u.x;
      u_out[g.N + cell] = (double)u.y;
      if (Lat<Q>::D == 3) u_out[2 * g.N + cell] = (double)u.z;
    }
  }
}

template <int Q, int S>
__global__ void __launch_bounds__(NT) k_set_state(void* fv, Grid g, const double* in) {
  using St = Store<S>;
  const int x = blockIdx.x * NT + threadIdx.x;
  if (x >= g.nx) return;
  const long long cell = cell_of(g, x, blockIdx.y, blockIdx.z);
  auto* A = static_cast<typename St::mem*>(fv);
#pragma unroll
  for (int i = 0; i < Q; ++i)
    St::st(A + (long long)i * g.pitch + cell, (typename St::real)in[(long long)i * g.N + cell],
           Lat<Q>::w(i));
}

template <int Q, int S>
__global__ void __launch_bounds__(NT) k_init_eq(void* fv, Grid g, const double* rho,
                                                const double* u, double u_in) {
  using St = Store<S>;
  using R = typename St::real;
  const int x = blockIdx.x * NT + threadIdx.x;
  if (x >= g.nx) return;
  const long long cell = cell_of(g, x, blockIdx.y, blockIdx.z);
  auto* A = static_cast<typename St::mem*>(fv);
  R r = rho ? (R)rho[cell] : R(1);
  Vec3<R> v{R(u_in), R(0), R(0)};
  if (u) {
    v.x = (R)u[cell];
    v.y = (R)u[g.N + cell];
    v.z = Lat<Q>::D == 3 ? (R)u[2 * g.N + cell] : R(0);
  }
  R f[Q];
  equilibrium<Q, R>(f, r, v);
#pragma unroll
  for (int i = 0; i < Q; ++i) St::st(A + (long long)i * g.pitch + cell, f[i], Lat<Q>::w(i));
}

#define HLBM_DISPATCH_QS(q, storage, CALL)                                  \
  do {                                                                      \
    if (q == 9) {                                                           \
      switch (storage) {                                                    \
        case ST_F64: { constexpr int Q_ = 9; constexpr int S_ = ST_F64; CALL; } break;  \
        case ST_F32: { constexpr int Q_ = 9; constexpr int S_ = ST_F32; CALL; } break;  \
        case ST_F16: { constexpr int Q_ = 9; constexpr int S_ = ST_F16; CALL; } break;  \
        case ST_BF16: { constexpr int Q_ = 9; constexpr int S_ = ST_BF16; CALL; } break; \
        default: return cudaErrorInvalidValue;                              \
      }                                                                     \
    } else if (q == 19) {                                                   \
      switch (storage) {                                                    \
        case ST_F64: { constexpr int Q_ = 19; constexpr int S_ = ST_F64; CALL; } break;  \
        case ST_F32: { constexpr int Q_ = 19; constexpr int S_ = ST_F32; CALL; } break;  \
        case ST_F16: { constexpr int Q_ = 19; constexpr int S_ = ST_F16; CALL; } break;  \
        case ST_BF16: { constexpr int Q_ = 19; constexpr int S_ = ST_BF16; CALL; } break; \
        default: return cudaErrorInvalidValue;                              \
      }                                                                     \
    } else {                                                                \
      return cudaErrorInvalidValue;                                         \
    }                                                                       \
  } while (0)

cudaError_t launch_readout(const void* f, const void*, const Grid& g, int q, int storage,
                           bool odd, double u_in, double* fout, double* rho, double* u,
                           cudaStream_t s) {
  dim3 grid((g.nx + NT - 1) / NT, g.ny, g.nz);
  if (odd) {
    HLBM_DISPATCH_QS(q, storage, (k_readout<Q_, S_, true><<<grid, NT, 0, s>>>(f, g, u_in, fout, rho, u)));
  } else {
    HLBM_DISPATCH_QS(q, storage, (k_readout<Q_, S_, false><<<grid, NT, 0, s>>>(f, g, u_in, fout, rho, u)));
  }
  return cudaGetLastError();
}

cudaError_t launch_set_state(void* f, const Grid& g, int q, int storage, const double* in,
                             cudaStream_t s) {
  dim3 grid((g.nx + NT - 1) / NT, g.ny, g.nz);
  HLBM_DISPATCH_QS(q, storage, (k_set_state<Q_, S_><<<grid, NT, 0, s>>>(f, g, in)));
  return cudaGetLastError();
}

cudaError_t launch_init_eq(void* f, const Grid& g, int q, int storage, const double* rho,
                           const double* u, double u_in, cudaStream_t s) {
  dim3 grid((g.nx + NT - 1) / NT, g.ny, g.nz);
  HLBM_DISPATCH_QS(q, storage, (k_init_eq<Q_, S_><<<grid, NT, 0, s>>>(f, g, rho, u, u_in)));
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// small utilities
// ----------------------------------------------------------------------------
template <class R>
__global__ void k_set_porosity(R* d, const double* in, long long n, unsigned* err) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const double v = in[k];
    if (!(v >= 0.0 && v <= 1.0)) atomicOr(err, 2u);
    d[k] = (R)v;
  }
}

cudaError_t launch_set_porosity(void* d, bool dbl, const double* in, long long n, unsigned* err,
                                cudaStream_t s) {
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  if (dbl) k_set_porosity<double><<<blocks, 256, 0, s>>>((double*)d, in, n, err);
  else k_set_porosity<float><<<blocks, 256, 0, s>>>((float*)d, in, n, err);
  return cudaGetLastError();
}

template <class A, class B>
__global__ void k_convert(const A* in, B* out, long long n) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    out[k] = (B)in[k];
}

static int util_blocks(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 8192 ? 8192 : b));
}

cudaError_t launch_convert_f32_to_f64(const float* in, double* out, long long n, cudaStream_t s) {
  k_convert<float, double><<<util_blocks(n), 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}
cudaError_t launch_convert_f64_to_f32(const double* in, float* out, long long n, cudaStream_t s) {
  k_convert<double, float><<<util_blocks(n), 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}
cudaError_t launch_real_to_f64(const void* in, bool dbl, double* out, long long n, cudaStream_t s) {
  if (dbl) k_convert<double, double><<<util_blocks(n), 256, 0, s>>>((const double*)in, out, n);
  else k_convert<float, double><<<util_blocks(n), 256, 0, s>>>((const float*)in, out, n);
  return cudaGetLastError();
}

__global__ void k_finalize_sum(const double* v, long long n, double* out) {
  __shared__ double sh[256 / 32];
  double acc = 0.0;
  for (long long k = threadIdx.x; k < n; k += blockDim.x) acc += v[k];
  const double t = block_sum<256>(acc, sh);
  if (threadIdx.x == 0) *out = t;
}

cudaError_t launch_finalize_sum(const double* v, long long n, double* out, cudaStream_t s) {
  k_finalize_sum<<<1, 256, 0, s>>>(v, n, out);
  return cudaGetLastError();
}

__global__ void k_scale(double* v, long long n, double s_) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    v[k] *= s_;
}
cudaError_t launch_scale(double* v, long long n, double s_, cudaStream_t s) {
  k_scale<<<util_blocks(n), 256, 0, s>>>(v, n, s_);
  return cudaGetLastError();
}

template <class R>
__global__ void k_fill(R* v, long long n, R value) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    v[k] = value;
}
cudaError_t launch_fill_real(void* v, bool dbl, long long n, double value, cudaStream_t s) {
  if (dbl) k_fill<double><<<util_blocks(n), 256, 0, s>>>((double*)v, n, value);
  else k_fill<float><<<util_blocks(n), 256, 0, s>>>((float*)v, n, (float)value);
  return cudaGetLastError();
}

}  // namespace hlbm
