// Tangent-linear (forward-mode) primal step on sm_103a.
//
// Advances the primal state g = f - w and its directional derivative
// gd = (df/dd) . delta together: g <- Phi(g; d), gd <- Phi_f gd + Phi_d delta,
// with the same fused collide + AA streaming + inflow/outflow nodes as the
// primal kernel.  This is the forward sensitivity whose growth along an
// unsteady trajectory the paper studies (App. C) to motivate the mean-flow
// adjoint; per step it also returns the directional derivative of the
// instantaneous objective, J' = dJ/df . gd + dJ/dd . delta.
//
// Forward derivative of the collision C_i = g_i - omega (g_i - g^eq_i):
//   rho' = sum gd,  (rho u)' = sum xi gd,  u' = ((rho u)' - u rho') / rho,
//   u~' = d u' + (u - u_s) delta,
//   g^eq_i' = w_i [rho' (1 + 3 xi.u~ + 9/2 (xi.u~)^2 - 3/2 u~.u~)
//                  + rho (3 xi.u~' + 9 (xi.u~)(xi.u~') - 3 u~.u~')],
//   C_i' = gd_i - omega (gd_i - g^eq_i') - omega' (g_i - g^eq_i),
//   omega' = -omega^2 tau_eff',  tau_eff' = k (Pi:Pi')/(|Pi| (2 tau_eff - tau0)) (LES).
// Outflow node: f^eq(1, u(nx-2)) gives g_i' = w_i (3 xi.u' + 9 (xi.u)(xi.u') - 3 u.u').
#include <cuda_runtime.h>

#include "hlbm_internal.h"
#include "hlbm_tangent.h"

namespace hlbm {

template <int Q, class R>
__device__ __forceinline__ void geq_dev_all(R (&ge)[Q], R drho, R rho, const Vec3<R>& u) {
  const R uu = dot3(u, u);
#pragma unroll
  for (int i = 0; i < Q; ++i) ge[i] = geq_i<Q>(i, drho, rho, u, uu);
}

// derivative of g^eq(rho, u~) for (rho', u~')
template <int Q, class R>
__device__ __forceinline__ R dgeq_i(int i, R rho, const Vec3<R>& ut, R uu, R rhod,
                                    const Vec3<R>& utd) {
  const R cu = xi_dot<Q>(i, ut);
  const R cud = xi_dot<Q>(i, utd);
  return R(Lat<Q>::w(i)) * (rhod * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu) +
                            rho * (R(3) * cud + R(9) * cu * cud - R(3) * dot3(ut, utd)));
}

template <int Q, class R>
__device__ __forceinline__ R pi_eps_t();
template <>
__device__ __forceinline__ double pi_eps_t<9, double>() { return 1e-30; }
template <>
__device__ __forceinline__ double pi_eps_t<19, double>() { return 1e-30; }
template <>
__device__ __forceinline__ float pi_eps_t<9, float>() { return 1e-20f; }
template <>
__device__ __forceinline__ float pi_eps_t<19, float>() { return 1e-20f; }

// One cell: collide (g, gd), store both AA-style, add J' of this cell to jp.
template <int Q, int S, bool ODD, bool LES>
__device__ __forceinline__ void tangent_cell(const TangentArgs& a, typename Store<S>::mem* A,
                                             typename Store<RealKind<S>::K>::mem* T,
                                             const Rows& rows, int x, int y, int z,
                                             long long cell,
                                             typename Store<S>::real (&g)[Q],
                                             typename Store<S>::real (&gd)[Q],
                                             typename Store<S>::real d,
                                             typename Store<S>::real dl,
                                             typename JAcc<typename Store<S>::real>::T& jp,
                                             Vec3<typename Store<S>::real>& u_out,
                                             Vec3<typename Store<S>::real>& ud_out) {
  using R = typename Store<S>::real;
  constexpr int D = Lat<Q>::D;
  const Grid& gr = a.g;
  R drho, rho;
  Vec3<R> m, u;
  moments_dev<Q>(g, drho, rho, m, u);
  R rhod, rhod_unused;
  Vec3<R> md, ud_raw;
  moments_dev<Q>(gd, rhod, rhod_unused, md, ud_raw);  // rhod = sum gd, md = sum xi gd
  const R inv = R(1) / rho;
  const Vec3<R> ud{(md.x - u.x * rhod) * inv, (md.y - u.y * rhod) * inv, (md.z - u.z * rhod) * inv};
  u_out = u;
  ud_out = ud;
  const Vec3<R> us{par<R>(a.us[0], a.us_f[0]), par<R>(a.us[1], a.us_f[1]),
                   par<R>(a.us[2], a.us_f[2])};
  const R one_d = R(1) - d;
  const Vec3<R> ut{d * u.x + one_d * us.x, d * u.y + one_d * us.y, d * u.z + one_d * us.z};
  const Vec3<R> v{u.x - us.x, u.y - us.y, u.z - us.z};
  const Vec3<R> utd{d * ud.x + v.x * dl, d * ud.y + v.y * dl, d * ud.z + v.z * dl};
  const R uu = dot3(ut, ut);
  R fneq[Q], fneqd[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    fneq[i] = g[i] - geq_i<Q>(i, drho, rho, ut, uu);
    fneqd[i] = gd[i] - dgeq_i<Q>(i, rho, ut, uu, rhod, utd);
  }
  const R tau0 = par<R>(a.tau0, a.tau0_f);
  const R kles = par<R>(a.kles, a.kles_f);
  R tau = tau0, taud = 0;
  Sym<R> P{0, 0, 0, 0, 0, 0}, Pd{0, 0, 0, 0, 0, 0};
  R nP = 0;
  const bool diss_here = (a.objective == 2) && x >= a.db[0] && x < a.db[1] && y >= a.db[2] &&
                         y < a.db[3] && z >= a.db[4] && z < a.db[5];
  if (LES || diss_here) {
    P = second_moment<Q>(fneq);
    Pd = second_moment<Q>(fneqd);
    nP = sqrt_r<R>(sym_norm2(P));
  }
  const R PPd = P.xx * Pd.xx + P.yy * Pd.yy + P.zz * Pd.zz +
                R(2) * (P.xy * Pd.xy + P.xz * Pd.xz + P.yz * Pd.yz);
  if (LES) {
    tau = tau_smagorinsky<R>(tau0, kles, nP);
    if (nP > pi_eps_t<Q, R>()) taud = kles * PPd / (nP * (R(2) * tau - tau0));
  }
  const R om = R(1) / tau;
  const R omd = -om * om * taud;

  // J' at the canonical state
  if (a.objective == 1 && x == a.ffa[0] && y >= a.ffa[1] && y < a.ffa[2] && z >= a.ffa[3] &&
      z < a.ffa[4]) {
    // J = (rho u_x)(u0 - u_x) - c_s^2 (rho - 1): dJ/df_j = (u_x^2 - c_s^2) + (u0 - 2 u_x) xi_jx
    const R u0 = par<R>(a.u_in, a.u_in_f);
    jadd(jp, (u.x * u.x - R(1.0 / 3.0)) * rhod + (u0 - R(2) * u.x) * md.x);
  }
  if (diss_here) {
    // J = (9 nu / 2) |Pi|^2 / tau^2 + (1-d)/tau0 |u|^2 with Pi, tau and u along gd and delta
    const R nu = par<R>(a.nu0, a.nu0_f);
    const R uu_raw = dot3(u, u);
    R jd = R(4.5) * nu * (R(2) * PPd / (tau * tau) - R(2) * nP * nP * taud / (tau * tau * tau));
    jd += one_d / tau0 * R(2) * dot3(u, ud) - dl / tau0 * uu_raw;
    jadd(jp, jd);
  }

  // collide and store
  R gn[Q], gdn[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    gn[i] = g[i] - om * fneq[i];
    gdn[i] = gd[i] - om * fneqd[i] - omd * fneq[i];
  }
  aa_store<Q, S, ODD, +1>(A, gr, rows, x, cell, gn);
  aa_store<Q, RealKind<S>::K, ODD, +1>(T, gr, rows, x, cell, gdn);
  (void)D;
}

template <int Q, int S, bool ODD, bool LES>
__global__ void __launch_bounds__(NT) k_tangent(TangentArgs a) {
  using St = Store<S>;
  using R = typename St::real;
  constexpr int SD = RealKind<S>::K;
  const Grid& gr = a.g;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  auto* A = static_cast<typename St::mem*>(a.f);
  auto* T = static_cast<typename Store<SD>::mem*>(a.fd);
  const R* dp = static_cast<const R*>(a.d);
  const R* dlp = static_cast<const R*>(a.delta);
  typename JAcc<R>::T jp{};  // this thread's dJ/dd . delta terms (FP64, or double-float)
  if (x < gr.nx - 1) {
    const long long cell = cell_of(gr, x, y, z);
    const Rows rows = make_rows<Lat<Q>::D>(gr, y, z);
    R g[Q], gd[Q];
    if (x == 0) {
      const R uin = a.inflow ? (R)a.inflow[y + (long long)gr.ny * z] : par<R>(a.u_in, a.u_in_f);
      geq_dev_all<Q, R>(g, R(0), R(1), Vec3<R>{uin, R(0), R(0)});
#pragma unroll
      for (int i = 0; i < Q; ++i) gd[i] = R(0);
    } else {
      aa_load<Q, S, ODD, +1>(A, gr, rows, x, cell, g);
      aa_load<Q, SD, ODD, +1>(T, gr, rows, x, cell, gd);
    }
    Vec3<R> u, ud;
    tangent_cell<Q, S, ODD, LES>(a, A, T, rows, x, y, z, cell, g, gd, dp[cell], dlp[cell], jp, u, ud);
    if (x == gr.nx - 2) {
      R go[Q], gdo[Q];
      geq_dev_all<Q, R>(go, R(0), R(1), u);
      const R uu = dot3(u, u);
#pragma unroll
      for (int i = 0; i < Q; ++i) gdo[i] = dgeq_i<Q>(i, R(1), u, uu, R(0), ud);
      Vec3<R> u2, ud2;
      tangent_cell<Q, S, ODD, LES>(a, A, T, rows, x + 1, y, z, cell + 1, go, gdo, dp[cell + 1],
                                   dlp[cell + 1], jp, u2, ud2);
    }
  }
  __shared__ double sh[NT / 32];
  const double s = block_sum<NT>(jp, sh);
  if (threadIdx.x == 0) a.jpart[block_linear()] = s;
}

template <int Q, int S>
static cudaError_t launch_tangent_qs(const TangentArgs& a, bool odd, bool les, cudaStream_t s) {
  const int bx = a.g.bx;
  dim3 grid((a.g.nx + bx - 1) / bx, a.g.ny, a.g.nz);
  if (!odd) {
    if (!les) k_tangent<Q, S, false, false><<<grid, bx, 0, s>>>(a);
    else k_tangent<Q, S, false, true><<<grid, bx, 0, s>>>(a);
  } else {
    if (!les) k_tangent<Q, S, true, false><<<grid, bx, 0, s>>>(a);
    else k_tangent<Q, S, true, true><<<grid, bx, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_tangent(const TangentArgs& a, int q, int storage, bool odd, bool les,
                           cudaStream_t s) {
  if (q == 9) {
    switch (storage) {
      case ST_F64: return launch_tangent_qs<9, ST_F64>(a, odd, les, s);
      case ST_F32: return launch_tangent_qs<9, ST_F32>(a, odd, les, s);
      case ST_F16: return launch_tangent_qs<9, ST_F16>(a, odd, les, s);
      case ST_BF16: return launch_tangent_qs<9, ST_BF16>(a, odd, les, s);
    }
  } else if (q == 19) {
    switch (storage) {
      case ST_F64: return launch_tangent_qs<19, ST_F64>(a, odd, les, s);
      case ST_F32: return launch_tangent_qs<19, ST_F32>(a, odd, les, s);
      case ST_F16: return launch_tangent_qs<19, ST_F16>(a, odd, les, s);
      case ST_BF16: return launch_tangent_qs<19, ST_BF16>(a, odd, les, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace hlbm
