// Mean-flow adjoint LBM and gradient contraction on sm_103a
// (Ito et al., Eq. adjoint_unsteady / adjoint_steady, Eq. gradients_unsteady
// / gradients_steady, Sec. 5.4 for the exact LES and frozen-turbulence
// variants).
//
// One iteration applies lambda <- A^T lambda + g_bar with A = B_f S C_f the
// Jacobian of one primal step at the averaged state.  Stored is
// theta = B_f^T lambda (zero on the inflow column, the outflow column folded
// into column nx-2); a kernel gathers mu = S^T theta by streaming against
// the lattice velocities (the AA pattern with s = -1), applies the transposed
// collision Jacobian C_f^T locally, adds the source and scatters theta.
//
// Transposed BGK collision of the porous equilibrium, omega = 1/tau:
//   (C_f^T mu)_j = (1 - omega) mu_j + omega [ m0 + d (xi_j - u) . (s - 3 u~ s0) ]
//   m0 = sum_i mu_i f_i^eq / rho,  s0 = sum_i w_i mu_i,
//   s  = sum_i w_i mu_i xi_i (3 + 9 xi_i . u~)
// Exact LES adds  E (Pi : dPi/df_j),  E = -omega^2 (sum_i mu_i (f^eq_i - f_i))
//   * k / ((2 tau - tau_b) |Pi|),  k = (9 sqrt 2 / 2) Cs^2, the derivative of
// tau_eff = (tau_b + sqrt(tau_b^2 + 4 k |Pi|)) / 2.
#include <cuda_runtime.h>

#include "hlbm_internal.h"

namespace hlbm {

template <class R> struct RealStore;
template <> struct RealStore<double> { static constexpr int S = ST_F64; };
template <> struct RealStore<float> { static constexpr int S = ST_F32; };

template <class R> __device__ __forceinline__ R pi_eps();
template <> __device__ __forceinline__ double pi_eps<double>() { return 1e-30; }
template <> __device__ __forceinline__ float pi_eps<float>() { return 1e-20f; }

// Linearisation point of one cell, derived from the record.
template <int Q, class R, bool EXACT> struct LinCell {
  R rho, om, d;
  Vec3<R> u, ut;
  // EXACT only
  R fneq[EXACT ? Q : 1];
  Sym<R> P;
  R nP, tau;
};

template <int Q, class R, bool EXACT>
__device__ __forceinline__ void load_lin(const AdjointArgs& a, long long cell, R d,
                                         LinCell<Q, R, EXACT>& c) {
  const R* rec = static_cast<const R*>(a.rec);
  const long long rp = a.rec_pitch;
  c.d = d;
  R drho = 0;
  if constexpr (!EXACT) {
    c.rho = rec[cell];
    c.u.x = rec[rp + cell];
    c.u.y = rec[2 * rp + cell];
    c.u.z = Lat<Q>::D == 3 ? rec[3 * rp + cell] : R(0);
    c.om = rec[(Lat<Q>::D + 1) * rp + cell];
  } else {
    // the record holds f_bar - w
    R gb[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) gb[i] = rec[(long long)i * rp + cell];
    Vec3<R> m;
    moments_dev<Q>(gb, drho, c.rho, m, c.u);
  }
  const R one_d = R(1) - d;
  const Vec3<R> us{par<R>(a.us[0], a.us_f[0]), par<R>(a.us[1], a.us_f[1]),
                   par<R>(a.us[2], a.us_f[2])};
  c.ut = Vec3<R>{d * c.u.x + one_d * us.x, d * c.u.y + one_d * us.y, d * c.u.z + one_d * us.z};
  if constexpr (EXACT) {
    const R uu = dot3(c.ut, c.ut);
#pragma unroll
    for (int i = 0; i < Q; ++i)
      c.fneq[i] = rec[(long long)i * rp + cell] - geq_i<Q>(i, drho, c.rho, c.ut, uu);
    c.P = second_moment<Q, R>(c.fneq);
    c.nP = sqrt_r<R>(sym_norm2(c.P));
    c.tau = tau_smagorinsky<R>(par<R>(a.tau_b, a.tau_b_f), par<R>(a.kles, a.kles_f), c.nP);
    c.om = R(1) / c.tau;
  }
}

// s0 = sum w_i mu_i, s = sum w_i mu_i xi_i (3 + 9 xi_i.u~), m0 = sum mu_i f^eq_i / rho
template <int Q, class R>
__device__ __forceinline__ void contract(const R (&mu)[Q], const Vec3<R>& ut, R& s0, Vec3<R>& s,
                                         R& m0) {
  using L = Lat<Q>;
  const R uu = dot3(ut, ut);
  s0 = 0;
  m0 = 0;
  s = Vec3<R>{0, 0, 0};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const R cu = xi_dot<Q>(i, ut);
    const R wm = R(L::w(i)) * mu[i];
    s0 += wm;
    m0 += wm * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu);
    const R t = wm * (R(3) + R(9) * cu);
    if (L::cx(i)) s.x += L::cx(i) > 0 ? t : -t;
    if (L::cy(i)) s.y += L::cy(i) > 0 ? t : -t;
    if (L::cz(i)) s.z += L::cz(i) > 0 ? t : -t;
  }
}

// lam = C_f^T mu + g at one cell (mu is overwritten with lam)
template <int Q, class R, bool EXACT>
__device__ __forceinline__ void transpose_collide(const LinCell<Q, R, EXACT>& c, R (&mu)[Q],
                                                  const AdjointArgs& a) {
  R s0, m0;
  Vec3<R> s;
  contract<Q, R>(mu, c.ut, s0, s, m0);
  const Vec3<R> gv{s.x - R(3) * c.ut.x * s0, s.y - R(3) * c.ut.y * s0, s.z - R(3) * c.ut.z * s0};
  const R ug = dot3(c.u, gv);
  const R om = c.om;
  R E = 0;
  Vec3<R> PU{0, 0, 0};
  R uPu = 0, trP = 0, uPU = 0;
  if constexpr (EXACT) {
    if (c.nP > pi_eps<R>()) {
      R sn = 0;
#pragma unroll
      for (int i = 0; i < Q; ++i) sn += mu[i] * c.fneq[i];
      // sum mu_i (f^eq_i - f_i) = -sn
      E = om * om * sn * par<R>(a.kles, a.kles_f) /
          ((R(2) * c.tau - par<R>(a.tau_b, a.tau_b_f)) * c.nP);
    }
    PU = sym_mul(c.P, c.ut);
    uPu = dot3(c.ut, PU);
    trP = c.P.xx + c.P.yy + c.P.zz;
    uPU = dot3(c.u, PU);
  }
#pragma unroll
  for (int j = 0; j < Q; ++j) {
    R v = (R(1) - om) * mu[j] + om * (m0 + c.d * (xi_dot<Q>(j, gv) - ug));
    if constexpr (EXACT) {
      const R pdp = xi_P_xi<Q>(j, c.P) - trP * R(1.0 / 3.0) - uPu -
                    R(2) * c.d * (xi_dot<Q>(j, PU) - uPU);
      v += E * pdp;
    }
    mu[j] = v;
  }
}

template <int Q, class R>
__device__ __forceinline__ void add_source(const AdjointArgs& a, int x, int y, int z, R (&v)[Q]) {
  if (x >= a.sb[0] && x < a.sb[1] && y >= a.sb[2] && y < a.sb[3] && z >= a.sb[4] && z < a.sb[5]) {
    const long long bc = (long long)(x - a.sb[0]) +
                         (long long)(a.sb[1] - a.sb[0]) *
                             ((long long)(y - a.sb[2]) + (long long)(a.sb[3] - a.sb[2]) * (z - a.sb[4]));
    const R* src = static_cast<const R*>(a.src);
#pragma unroll
    for (int i = 0; i < Q; ++i) v[i] += src[(long long)i * a.src_pitch + bc];
  }
}

// outflow node transposed: theta(nx-2) += (d f^eq(1,u)/d u . d u/d f)^T lam(nx-1),
// u, rho the averaged velocity and density of column nx-2.
template <int Q, class R>
__device__ __forceinline__ void outlet_transpose(R (&th)[Q], const R (&lo)[Q], R rho,
                                                 const Vec3<R>& u) {
  using L = Lat<Q>;
  R l0 = 0;
  Vec3<R> h{0, 0, 0};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const R wl = R(L::w(i)) * lo[i];
    l0 += wl;
    const R t = wl * (R(3) + R(9) * xi_dot<Q>(i, u));
    if (L::cx(i)) h.x += L::cx(i) > 0 ? t : -t;
    if (L::cy(i)) h.y += L::cy(i) > 0 ? t : -t;
    if (L::cz(i)) h.z += L::cz(i) > 0 ? t : -t;
  }
  h.x -= R(3) * u.x * l0;
  h.y -= R(3) * u.y * l0;
  h.z -= R(3) * u.z * l0;
  const R inv = R(1) / rho;
  const R uh = dot3(u, h);
#pragma unroll
  for (int j = 0; j < Q; ++j) th[j] += (xi_dot<Q>(j, h) - uh) * inv;
}

template <int Q, class R, int RES>
__device__ __forceinline__ void residual_io(const AdjointArgs& a, long long cell, const R (&v)[Q],
                                            double& rp) {
  if (RES == 0) return;
  R* sn = static_cast<R*>(a.snap);
  R acc = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    R* p = sn + (long long)i * a.g.pitch + cell;
    if (RES == 1) {
      *p = v[i];
    } else {
      const R dlt = v[i] - *p;
      acc += dlt * dlt;
    }
  }
  if (RES == 2) rp += (double)acc;
}

template <int Q, class R, bool ODD, bool EXACT, int RES>
__global__ void __launch_bounds__(NT) k_adjoint(AdjointArgs a) {
  constexpr int S = RealStore<R>::S;
  const Grid& g = a.g;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  R* A = static_cast<R*>(a.lam);
  const R* dp = static_cast<const R*>(a.d);
  double rp = 0.0;
  if (x < g.nx - 1) {
    const long long cell = cell_of(g, x, y, z);
    const Rows rows = make_rows<Lat<Q>::D>(g, y, z);
    R v[Q];
    aa_load<Q, S, ODD, -1>(A, g, rows, x, cell, v);
    LinCell<Q, R, EXACT> c;
    load_lin<Q, R, EXACT>(a, cell, dp[cell], c);
    transpose_collide<Q, R, EXACT>(c, v, a);
    add_source<Q, R>(a, x, y, z, v);
    residual_io<Q, R, RES>(a, cell, v, rp);
    if (x == g.nx - 2) {
      R vo[Q];
      aa_load<Q, S, ODD, -1>(A, g, rows, x + 1, cell + 1, vo);
      LinCell<Q, R, EXACT> co;
      load_lin<Q, R, EXACT>(a, cell + 1, dp[cell + 1], co);
      transpose_collide<Q, R, EXACT>(co, vo, a);
      add_source<Q, R>(a, x + 1, y, z, vo);
      residual_io<Q, R, RES>(a, cell + 1, vo, rp);
      outlet_transpose<Q, R>(v, vo, c.rho, c.u);
#pragma unroll
      for (int i = 0; i < Q; ++i) vo[i] = R(0);
      aa_store<Q, S, ODD, -1>(A, g, rows, x + 1, cell + 1, vo);
    }
    if (x == 0) {
#pragma unroll
      for (int i = 0; i < Q; ++i) v[i] = R(0);
    }
    aa_store<Q, S, ODD, -1>(A, g, rows, x, cell, v);
  }
  if (RES == 2) {
    __shared__ double sh[NT / 32];
    const double s = block_sum<NT>(rp, sh);
    if (threadIdx.x == 0) a.red[block_linear()] = s;
  }
}

int adjoint_blocks(const Grid& g) { return ((g.nx + g.bx - 1) / g.bx) * g.ny * g.nz; }

template <int Q, class R>
static cudaError_t launch_adj_qr(const AdjointArgs& a, bool odd, bool exact, int res,
                                 cudaStream_t s) {
  const int bx = a.g.bx;
  dim3 grid((a.g.nx + bx - 1) / bx, a.g.ny, a.g.nz);
#define HLBM_A(O, E, RS) k_adjoint<Q, R, O, E, RS><<<grid, bx, 0, s>>>(a)
#define HLBM_AR(O, E) \
  do { if (res == 0) HLBM_A(O, E, 0); else if (res == 1) HLBM_A(O, E, 1); else HLBM_A(O, E, 2); } while (0)
  if (!odd) { if (!exact) HLBM_AR(false, false); else HLBM_AR(false, true); }
  else      { if (!exact) HLBM_AR(true, false);  else HLBM_AR(true, true); }
#undef HLBM_AR
#undef HLBM_A
  return cudaGetLastError();
}

cudaError_t launch_adjoint(const AdjointArgs& a, int q, bool dbl, bool odd, bool exact, int res,
                           cudaStream_t s) {
  if (q == 9) return dbl ? launch_adj_qr<9, double>(a, odd, exact, res, s)
                         : launch_adj_qr<9, float>(a, odd, exact, res, s);
  if (q == 19) return dbl ? launch_adj_qr<19, double>(a, odd, exact, res, s)
                          : launch_adj_qr<19, float>(a, odd, exact, res, s);
  return cudaErrorInvalidValue;
}

// ----------------------------------------------------------------------------
// linearisation record from the running sums
// ----------------------------------------------------------------------------
template <int Q, class R>
__global__ void __launch_bounds__(NT) k_prep(PrepArgs a) {
  const Grid& g = a.g;
  const int x = blockIdx.x * NT + threadIdx.x;
  if (x >= g.nx) return;
  const long long cell = cell_of(g, x, blockIdx.y, blockIdx.z);
  R* rec = static_cast<R*>(a.rec);
  const long long rp = a.rec_pitch;
  if (a.exact) {
#pragma unroll
    for (int i = 0; i < Q; ++i)
      rec[(long long)i * rp + cell] = (R)(a.fsum[(long long)i * g.N + cell] * a.inv_n);
    return;
  }
  // density and velocity of f_bar from the averaged moments (rho - 1, rho u)
  const double rho = 1.0 + a.msum[cell] * a.inv_n;
  const double ir = 1.0 / rho;
  double tau = a.tau_b;
  if (a.tsum) tau += a.tsum[cell] * a.inv_n;
  rec[cell] = (R)rho;
  rec[rp + cell] = (R)(a.msum[g.N + cell] * a.inv_n * ir);
  rec[2 * rp + cell] = (R)(a.msum[2 * g.N + cell] * a.inv_n * ir);
  if (Lat<Q>::D == 3) rec[3 * rp + cell] = (R)(a.msum[3 * g.N + cell] * a.inv_n * ir);
  rec[(Lat<Q>::D + 1) * rp + cell] = (R)(1.0 / tau);
}

cudaError_t launch_prep(const PrepArgs& a, int q, bool dbl, cudaStream_t s) {
  dim3 grid((a.g.nx + NT - 1) / NT, a.g.ny, a.g.nz);
  if (q == 9) { if (dbl) k_prep<9, double><<<grid, NT, 0, s>>>(a); else k_prep<9, float><<<grid, NT, 0, s>>>(a); }
  else if (q == 19) { if (dbl) k_prep<19, double><<<grid, NT, 0, s>>>(a); else k_prep<19, float><<<grid, NT, 0, s>>>(a); }
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <int Q, class R>
__global__ void __launch_bounds__(NT) k_source(SourceArgs a) {
  constexpr int D = Lat<Q>::D;
  const int bx = a.box[1] - a.box[0], by = a.box[3] - a.box[2];
  const int xl = blockIdx.x * NT + threadIdx.x;
  const int yl = blockIdx.y, zl = blockIdx.z;
  double acc = 0.0;
  if (xl < bx) {
    const long long bc = (long long)xl + (long long)bx * ((long long)yl + (long long)by * zl);
    const long long vol = (long long)bx * by * (a.box[5] - a.box[4]);
    const long long cell = cell_of(a.g, a.box[0] + xl, a.box[2] + yl, a.box[4] + zl);
    const int nc = ncoef(a.obj_slot, D);
    double cf[10];
    for (int k = 0; k < nc; ++k) cf[k] = a.gsum[(long long)k * a.g.N + cell] * a.inv_n;
    R* src = static_cast<R*>(a.src);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      double gv = 0.0;
      for (int k = 0; k < nc; ++k)
        gv += cf[k] * coef_basis(a.obj_slot, D, k, Lat<Q>::cx(i), Lat<Q>::cy(i), Lat<Q>::cz(i));
      const R v = (R)gv;
      src[(long long)i * vol + bc] = v;
      acc += (double)v * (double)v;
    }
  }
  __shared__ double sh[NT / 32];
  const double s = block_sum<NT>(acc, sh);
  if (threadIdx.x == 0) a.red[block_linear()] = s;
}

cudaError_t launch_source(const SourceArgs& a, int q, bool dbl, int* nblocks, cudaStream_t s) {
  const int bx = a.box[1] - a.box[0], by = a.box[3] - a.box[2], bz = a.box[5] - a.box[4];
  dim3 grid((bx + NT - 1) / NT, by, bz);
  *nblocks = (int)(grid.x * grid.y * grid.z);
  if (q == 9) { if (dbl) k_source<9, double><<<grid, NT, 0, s>>>(a); else k_source<9, float><<<grid, NT, 0, s>>>(a); }
  else if (q == 19) { if (dbl) k_source<19, double><<<grid, NT, 0, s>>>(a); else k_source<19, float><<<grid, NT, 0, s>>>(a); }
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// gradient: G = dJ/dd_bar + sum_i mu_i dC_i/dd over the design box
//   dC_i/dd = omega w_i rho (3 xi_i.v + 9 (xi_i.u~)(xi_i.v) - 3 u~.v),  v = u - u_s
//   so sum_i mu_i dC_i/dd = omega rho (s - 3 u~ s0) . v;
//   exact LES adds (sum_i mu_i (f^eq_i - f_i)) d omega/dd with
//   Pi : dPi/dd = -2 rho v . Pi . u~.
// ----------------------------------------------------------------------------
template <int Q, class R, bool EXACT>
__global__ void __launch_bounds__(NT) k_gradient(GradArgs ga) {
  constexpr int S = RealStore<R>::S;
  const int bx = ga.box[1] - ga.box[0], by = ga.box[3] - ga.box[2];
  const int xl = blockIdx.x * NT + threadIdx.x;
  if (xl >= bx) return;
  const int x = ga.box[0] + xl, y = ga.box[2] + blockIdx.y, z = ga.box[4] + blockIdx.z;
  const Grid& g = ga.g;
  const long long cell = cell_of(g, x, y, z);
  R mu[Q];
  const Rows rows = make_rows<Lat<Q>::D>(g, y, z);
  aa_load<Q, S, false, -1>(static_cast<const R*>(ga.lam), g, rows, x, cell, mu);
  AdjointArgs a{};
  a.rec = ga.rec;
  a.rec_pitch = ga.rec_pitch;
  a.tau_b = ga.tau_b;
  a.kles = ga.kles;
  a.tau_b_f = ga.tau_b_f;
  a.kles_f = ga.kles_f;
  for (int k = 0; k < 3; ++k) { a.us[k] = ga.us[k]; a.us_f[k] = ga.us_f[k]; }
  LinCell<Q, R, EXACT> c;
  load_lin<Q, R, EXACT>(a, cell, static_cast<const R*>(ga.d)[cell], c);
  R s0, m0;
  Vec3<R> s;
  contract<Q, R>(mu, c.ut, s0, s, m0);
  const Vec3<R> v{c.u.x - par<R>(ga.us[0], ga.us_f[0]), c.u.y - par<R>(ga.us[1], ga.us_f[1]),
                  c.u.z - par<R>(ga.us[2], ga.us_f[2])};
  const Vec3<R> gv{s.x - R(3) * c.ut.x * s0, s.y - R(3) * c.ut.y * s0, s.z - R(3) * c.ut.z * s0};
  R val = c.om * c.rho * dot3(gv, v);
  if constexpr (EXACT) {
    if (c.nP > pi_eps<R>()) {
      R sn = 0;
#pragma unroll
      for (int i = 0; i < Q; ++i) sn += mu[i] * c.fneq[i];
      const R pdd = -R(2) * c.rho * dot3(v, sym_mul(c.P, c.ut));
      // (sum mu (feq - f)) * (-om^2) * k pdd / ((2 tau - tau_b) |Pi|)
      val += sn * c.om * c.om * par<R>(ga.kles, ga.kles_f) * pdd /
             ((R(2) * c.tau - par<R>(ga.tau_b, ga.tau_b_f)) * c.nP);
    }
  }
  double G = (double)val;
  if (ga.ddsum) G += ga.ddsum[cell] * ga.inv_n;
  const long long bc = (long long)xl + (long long)bx * ((long long)blockIdx.y + (long long)by * blockIdx.z);
  ga.out[bc] = G;
  if (ga.mu_out) {
#pragma unroll
    for (int i = 0; i < Q; ++i) ga.mu_out[(long long)i * g.N + cell] = (double)mu[i];
  }
}

cudaError_t launch_gradient(const GradArgs& a, int q, bool dbl, bool exact, cudaStream_t s) {
  const int bx = a.box[1] - a.box[0], by = a.box[3] - a.box[2], bz = a.box[5] - a.box[4];
  dim3 grid((bx + NT - 1) / NT, by, bz);
#define HLBM_G(QQ, RR) \
  do { if (exact) k_gradient<QQ, RR, true><<<grid, NT, 0, s>>>(a); else k_gradient<QQ, RR, false><<<grid, NT, 0, s>>>(a); } while (0)
  if (q == 9) { if (dbl) HLBM_G(9, double); else HLBM_G(9, float); }
  else if (q == 19) { if (dbl) HLBM_G(19, double); else HLBM_G(19, float); }
  else return cudaErrorInvalidValue;
#undef HLBM_G
  return cudaGetLastError();
}

}  // namespace hlbm
