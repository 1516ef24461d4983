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
  // EXACT only: rho - 1, the non-equilibrium stress of f_bar, its norm,
  // tau_eff, and sg = sum_i mu_i (f_bar_i - w_i) for the mu this cell is
  // processed with (f_bar itself is not kept through the transpose)
  R drho;
  Sym<R> P;
  R nP, tau, sg;
};

template <int Q, class R, bool EXACT>
__device__ __forceinline__ void load_lin(const AdjointArgs& a, long long cell, R d,
                                         LinCell<Q, R, EXACT>& c, const R (&mu)[Q]) {
  constexpr int D = Lat<Q>::D;
  const R* rec = static_cast<const R*>(a.rec);
  const long long rp = a.rec_pitch;
  c.d = d;
  R gb[EXACT ? Q : 1];
  Sym<R> M2;
  if constexpr (!EXACT) {
    c.rho = rec[cell];
    c.u.x = rec[rp + cell];
    c.u.y = rec[2 * rp + cell];
    c.u.z = D == 3 ? rec[3 * rp + cell] : R(0);
    c.om = rec[(D + 1) * rp + cell];
  } else {
    // the record holds g = f_bar - w: rho - 1 = sum g, rho u = sum xi g,
    // M2 = sum xi xi g
#pragma unroll
    for (int i = 0; i < Q; ++i) gb[i] = rec[(long long)i * rp + cell];
    Mom<R> ax, dg;
    class_moments<Q, R>(gb, ax, dg);
    c.drho = gb[0] + ax.m0 + dg.m0;
    c.rho = R(1) + c.drho;
    const R inv = R(1) / c.rho;
    c.u = Vec3<R>{(ax.m1.x + dg.m1.x) * inv, (ax.m1.y + dg.m1.y) * inv,
                  D == 3 ? (ax.m1.z + dg.m1.z) * inv : R(0)};
    M2 = Sym<R>{ax.m2.xx + dg.m2.xx, ax.m2.yy + dg.m2.yy, ax.m2.zz + dg.m2.zz, dg.m2.xy,
                dg.m2.xz, dg.m2.yz};
  }
  const R one_d = R(1) - d;
  const Vec3<R> us{par<R>(a.us[0], a.us_f[0]), par<R>(a.us[1], a.us_f[1]),
                   par<R>(a.us[2], a.us_f[2])};
  c.ut = Vec3<R>{d * c.u.x + one_d * us.x, d * c.u.y + one_d * us.y, d * c.u.z + one_d * us.z};
  if constexpr (EXACT) {
    // Pi = sum xi xi (f_bar - f^eq(rho, u~)) = M2 - (rho - 1)/3 I - rho u~ u~: the
    // lattice sums of f^eq - w are (rho - 1) c_s^2 I + rho u~ u~ on both lattices
    const R t = c.drho * R(1.0 / 3.0);
    const Vec3<R>& w = c.ut;
    c.P = Sym<R>{M2.xx - t - c.rho * w.x * w.x, M2.yy - t - c.rho * w.y * w.y,
                 D == 3 ? M2.zz - t - c.rho * w.z * w.z : R(0), M2.xy - c.rho * w.x * w.y,
                 D == 3 ? M2.xz - c.rho * w.x * w.z : R(0),
                 D == 3 ? M2.yz - c.rho * w.y * w.z : R(0)};
    R sg = mu[0] * gb[0];
#pragma unroll
    for (int i = 1; i < Q; ++i) sg += mu[i] * gb[i];
    c.sg = sg;
    c.nP = sqrt_r<R>(sym_norm2(c.P));
    c.tau = tau_smagorinsky<R>(par<R>(a.tau_b, a.tau_b_f), par<R>(a.kles, a.kles_f), c.nP);
    c.om = R(1) / c.tau;
  }
}

// Contractions of mu at the linearisation point, from the weighted moments
// a0 = sum w mu, a1 = sum w mu xi, A2 = sum w mu xi xi (c_i = xi_i . u~):
//   m0 = sum mu_i f^eq_i / rho = a0 (1 - 3/2 u~.u~) + 3 a1.u~ + 9/2 u~.A2.u~
//   qe = sum mu_i (f^eq_i - w_i) = (rho - 1) a0 + rho (m0 - a0)
//   gv = sum w mu (3 xi + 9 c xi) - 3 u~ a0 = 3 a1 + 9 A2 u~ - 3 u~ a0
template <class R> struct MuC { R m0, qe; Vec3<R> gv; };

template <int Q, class R>
__device__ __forceinline__ MuC<R> mu_contract(const R (&mu)[Q], const Vec3<R>& ut, R drho,
                                              R rho) {
  using L = Lat<Q>;
  constexpr int D = L::D;
  Mom<R> ax, dg;
  class_moments<Q, R>(mu, ax, dg);
  const R wa = R(L::w(1)), wd = R(L::w(Q - 1));
  const R a0 = R(L::w(0)) * mu[0] + wa * ax.m0 + wd * dg.m0;
  const Vec3<R> a1{wa * ax.m1.x + wd * dg.m1.x, wa * ax.m1.y + wd * dg.m1.y,
                   D == 3 ? wa * ax.m1.z + wd * dg.m1.z : R(0)};
  const Sym<R> A2{wa * ax.m2.xx + wd * dg.m2.xx, wa * ax.m2.yy + wd * dg.m2.yy,
                  D == 3 ? wa * ax.m2.zz + wd * dg.m2.zz : R(0), wd * dg.m2.xy,
                  D == 3 ? wd * dg.m2.xz : R(0), D == 3 ? wd * dg.m2.yz : R(0)};
  Vec3<R> A2u;
  if constexpr (D == 3) {
    A2u = sym_mul(A2, ut);
  } else {
    A2u = Vec3<R>{A2.xx * ut.x + A2.xy * ut.y, A2.xy * ut.x + A2.yy * ut.y, R(0)};
  }
  const R uu = dot3(ut, ut);
  const R a1u = D == 3 ? dot3(a1, ut) : a1.x * ut.x + a1.y * ut.y;
  const R uAu = D == 3 ? dot3(ut, A2u) : ut.x * A2u.x + ut.y * A2u.y;
  const R h = R(3) * a1u + R(4.5) * uAu - R(1.5) * uu * a0;
  MuC<R> r;
  r.m0 = a0 + h;
  r.qe = drho * a0 + rho * h;
  r.gv = Vec3<R>{R(3) * a1.x + R(9) * A2u.x - R(3) * ut.x * a0,
                 R(3) * a1.y + R(9) * A2u.y - R(3) * ut.y * a0,
                 R(3) * a1.z + R(9) * A2u.z - R(3) * ut.z * a0};
  return r;
}

// lam = C_f^T mu + g at one cell (mu is overwritten with lam).  The transposed
// collision is a quadratic polynomial in xi_j,
//   lam_j = (1 - omega) mu_j + K0 + xi_j . K1 + xi_j . K2 . xi_j,
//   K0 = omega (m0 - d u.gv) + E (2 d u.Pi u~ - u~.Pi u~ - tr Pi / 3),
//   K1 = omega d gv - 2 d E Pi u~,   K2 = E Pi,
// evaluated over opposite pairs (xi_opp = -xi: the K0 and K2 parts are shared,
// the K1 part changes sign).
template <int Q, class R, bool EXACT>
__device__ __forceinline__ void transpose_collide(const LinCell<Q, R, EXACT>& c, R (&mu)[Q],
                                                  const AdjointArgs& a) {
  const MuC<R> k = mu_contract<Q, R>(mu, c.ut, EXACT ? c.drho : c.rho - R(1), c.rho);
  const R om = c.om, d = c.d;
  const R ug = dot3(c.u, k.gv);
  R K0 = om * (k.m0 - d * ug);
  const R odg = om * d;
  Vec3<R> K1{odg * k.gv.x, odg * k.gv.y, odg * k.gv.z};
  Sym<R> K2{0, 0, 0, 0, 0, 0};
  if constexpr (EXACT) {
    if (c.nP > pi_eps<R>()) {
      // sum mu_i (f_bar_i - f^eq_i) = sg - qe
      const R E = om * om * (c.sg - k.qe) * par<R>(a.kles, a.kles_f) /
                  ((R(2) * c.tau - par<R>(a.tau_b, a.tau_b_f)) * c.nP);
      const Vec3<R> PU = sym_mul(c.P, c.ut);
      const R uPu = dot3(c.ut, PU), uPU = dot3(c.u, PU);
      const R trP = c.P.xx + c.P.yy + c.P.zz;
      K0 += E * (R(2) * d * uPU - uPu - trP * R(1.0 / 3.0));
      const R e2 = R(2) * d * E;
      K1 = Vec3<R>{K1.x - e2 * PU.x, K1.y - e2 * PU.y, K1.z - e2 * PU.z};
      K2 = Sym<R>{E * c.P.xx, E * c.P.yy, E * c.P.zz, E * c.P.xy, E * c.P.xz, E * c.P.yz};
    }
  }
  const R c1 = R(1) - om;
  mu[0] = c1 * mu[0] + K0;
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    R psi = K0;
    if constexpr (EXACT) psi += xi_P_xi<Q>(i, K2);
    const R phi = xi_dot<Q>(i, K1);
    mu[i] = c1 * mu[i] + (psi + phi);
    mu[i + 1] = c1 * mu[i + 1] + (psi - phi);
  }
}

// ----------------------------------------------------------------------------
// Recursive regularised collision (Sec. 2.2, Eq. HRRLBM) transposed.  The
// collision depends on f only through rho, j = sum xi f and M2 = sum xi xi f,
// so (C_f^T mu)_j = G_rho + G_j . xi_j + xi_j . G_M . xi_j, where G_* are the
// derivatives of L = sum_i mu_i C_i with respect to those moments.  They
// are taken by reverse-mode differentiation of L written in the variables
// (rho, u~, a1 = j - rho u~, Pi = M2 - rho u~ u~ - c_s^2 (rho - 1) I, omega):
//   L = rho (s0 + 3 s1.u~ + 9/2 C2 - 3/2 s0 u~.u~) + 9/2 rho (A3 - (s1.u~) u~.u~)
//       + (1 - omega) F,
//   F = 3 s1.a1 + 9/2 (CP - s0 tr Pi / 3) + 9/2 (3 B3 - (s1.u~) tr Pi - 2 s1.Pi u~),
// with the weighted sums of mu over the lattice (c = xi.u~, p = xi.Pi.xi)
//   s0 = sum w mu, s1 = sum w mu xi, C2 = sum w mu c^2, A3 = sum w mu c^3,
//   CP = sum w mu p, B3 = sum w mu c p,
// and their derivatives V1 = sum w mu c xi, T1 = sum w mu c^2 xi,
// T2 = sum w mu p xi, s2 = sum w mu xi xi, T3 = sum w mu c xi xi.
// The exact LES variant adds the dependence of omega on |Pi|.  The
// derivative with respect to u~ also gives the porosity gradient,
// dL/dd = (dL/du~) . (u - u_s).
// ----------------------------------------------------------------------------
template <class R, bool EXACT> struct RRCell {
  R rho, om, d;
  Vec3<R> u, ut;
  Sym<R> P;
  R nP, tau;  // EXACT only
};

template <int Q, class R, bool EXACT>
__device__ __forceinline__ void load_lin(const AdjointArgs& a, long long cell, R d,
                                         RRCell<R, EXACT>& c) {
  constexpr int D = Lat<Q>::D;
  const R* rec = static_cast<const R*>(a.rec);
  const long long rp = a.rec_pitch;
  c.d = d;
  c.rho = rec[cell];
  c.u.x = rec[rp + cell];
  c.u.y = rec[2 * rp + cell];
  c.u.z = D == 3 ? rec[3 * rp + cell] : R(0);
  c.om = rec[(D + 1) * rp + cell];
  const R* pp = rec + (D + 2) * rp + cell;
  if constexpr (D == 2) {
    c.P = Sym<R>{pp[0], pp[rp], R(0), pp[2 * rp], R(0), R(0)};
  } else {
    c.P = Sym<R>{pp[0], pp[rp], pp[2 * rp], pp[3 * rp], pp[4 * rp], pp[5 * rp]};
  }
  const R one_d = R(1) - d;
  const Vec3<R> us{par<R>(a.us[0], a.us_f[0]), par<R>(a.us[1], a.us_f[1]),
                   par<R>(a.us[2], a.us_f[2])};
  c.ut = Vec3<R>{d * c.u.x + one_d * us.x, d * c.u.y + one_d * us.y, d * c.u.z + one_d * us.z};
  if constexpr (EXACT) {
    c.nP = sqrt_r<R>(sym_norm2(c.P));
    c.tau = tau_smagorinsky<R>(par<R>(a.tau_b, a.tau_b_f), par<R>(a.kles, a.kles_f), c.nP);
    c.om = R(1) / c.tau;
  }
}

// the regularised record does not depend on mu (same call shapes as the BGK one)
template <int Q, class R, bool EXACT>
__device__ __forceinline__ void load_lin(const AdjointArgs& a, long long cell, R d,
                                         RRCell<R, EXACT>& c, const R (&)[Q]) {
  load_lin<Q, R, EXACT>(a, cell, d, c);
}

template <int Q, class R>
__device__ __forceinline__ void add_xi(Vec3<R>& v, int i, R s) {
  using L = Lat<Q>;
  if (L::cx(i)) v.x += L::cx(i) > 0 ? s : -s;
  if (L::cy(i)) v.y += L::cy(i) > 0 ? s : -s;
  if (L::cz(i)) v.z += L::cz(i) > 0 ? s : -s;
}

// mu <- C_f^T mu at one cell; gut (optional) receives dL/du~
template <int Q, class R, bool EXACT>
__device__ __forceinline__ void rr_transpose(const RRCell<R, EXACT>& c, R (&mu)[Q],
                                             const AdjointArgs& a, Vec3<R>* gut) {
  using L = Lat<Q>;
  constexpr bool D3 = L::D == 3;
  const Vec3<R>& ut = c.ut;
  const Sym<R>& P = c.P;
  const R uu = dot3(ut, ut);
  const R trP = P.xx + P.yy + P.zz;
  R s0 = 0, C2 = 0, A3 = 0, B3 = 0, CP = 0;
  Vec3<R> s1{0, 0, 0}, V1{0, 0, 0}, T1{0, 0, 0}, T2{0, 0, 0};
  Sym<R> s2{0, 0, 0, 0, 0, 0}, T3{0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const R wm = R(L::w(i)) * mu[i];
    const R cu = xi_dot<Q>(i, ut);
    const R xPx = xi_P_xi<Q>(i, P);
    s0 += wm;
    C2 += wm * cu * cu;
    A3 += wm * cu * cu * cu;
    B3 += wm * cu * xPx;
    CP += wm * xPx;
    add_xi<Q>(s1, i, wm);
    add_xi<Q>(V1, i, wm * cu);
    add_xi<Q>(T1, i, wm * cu * cu);
    add_xi<Q>(T2, i, wm * xPx);
    sym_add_xixi<Q>(s2, i, wm);
    sym_add_xixi<Q>(T3, i, wm * cu);
  }
  const R rho = c.rho, om = c.om, c1 = R(1) - om;
  const R su = dot3(s1, ut);
  const Vec3<R> a1{rho * (c.u.x - ut.x), rho * (c.u.y - ut.y), rho * (c.u.z - ut.z)};
  const Vec3<R> Ps1 = sym_mul(P, s1);
  const R sPu = dot3(Ps1, ut);
  const R F = R(3) * dot3(s1, a1) + R(4.5) * (CP - s0 * trP * R(1.0 / 3.0)) +
              R(4.5) * (R(3) * B3 - su * trP - R(2) * sPu);
  R Lrho = s0 + R(3) * su + R(4.5) * C2 - R(1.5) * s0 * uu + R(4.5) * (A3 - su * uu);
  const Vec3<R> La1{R(3) * c1 * s1.x, R(3) * c1 * s1.y, R(3) * c1 * s1.z};
  // dL/dPi (symmetric, dL = G : dPi)
  const R k45 = R(4.5) * c1;
  const R diag = -s0 * R(1.0 / 3.0) - su;
  Sym<R> G{k45 * (s2.xx + diag + R(3) * T3.xx - R(2) * s1.x * ut.x),
           k45 * (s2.yy + diag + R(3) * T3.yy - R(2) * s1.y * ut.y),
           D3 ? k45 * (s2.zz + diag + R(3) * T3.zz - R(2) * s1.z * ut.z) : R(0),
           k45 * (s2.xy + R(3) * T3.xy - (s1.x * ut.y + ut.x * s1.y)),
           k45 * (s2.xz + R(3) * T3.xz - (s1.x * ut.z + ut.x * s1.z)),
           k45 * (s2.yz + R(3) * T3.yz - (s1.y * ut.z + ut.y * s1.z))};
  if constexpr (EXACT) {
    if (c.nP > pi_eps<R>()) {
      // omega(|Pi|): dL/dPi += (-F)(-omega^2) k / ((2 tau - tau_b) |Pi|) Pi
      const R e = F * om * om * par<R>(a.kles, a.kles_f) /
                  ((R(2) * c.tau - par<R>(a.tau_b, a.tau_b_f)) * c.nP);
      G.xx += e * P.xx; G.yy += e * P.yy; G.zz += e * P.zz;
      G.xy += e * P.xy; G.xz += e * P.xz; G.yz += e * P.yz;
    }
  }
  // explicit dL/du~
  Vec3<R> Lu;
  Lu.x = rho * (R(3) * s1.x + R(9) * V1.x - R(3) * s0 * ut.x) +
         R(4.5) * rho * (R(3) * T1.x - s1.x * uu - R(2) * su * ut.x) +
         k45 * (R(3) * T2.x - trP * s1.x - R(2) * Ps1.x);
  Lu.y = rho * (R(3) * s1.y + R(9) * V1.y - R(3) * s0 * ut.y) +
         R(4.5) * rho * (R(3) * T1.y - s1.y * uu - R(2) * su * ut.y) +
         k45 * (R(3) * T2.y - trP * s1.y - R(2) * Ps1.y);
  Lu.z = rho * (R(3) * s1.z + R(9) * V1.z - R(3) * s0 * ut.z) +
         R(4.5) * rho * (R(3) * T1.z - s1.z * uu - R(2) * su * ut.z) +
         k45 * (R(3) * T2.z - trP * s1.z - R(2) * Ps1.z);
  // through a1 = j - rho u~ and Pi = M2 - rho u~ u~ - (rho - 1)/3 I
  const Vec3<R> Gu = sym_mul(G, ut);
  const Vec3<R> Gut{Lu.x - rho * La1.x - R(2) * rho * Gu.x, Lu.y - rho * La1.y - R(2) * rho * Gu.y,
                    Lu.z - rho * La1.z - R(2) * rho * Gu.z};
  Lrho += -dot3(La1, ut) - dot3(ut, Gu) - (G.xx + G.yy + G.zz) * R(1.0 / 3.0);
  // through u~ = d j / rho + (1 - d) u_s
  const R dr = c.d / rho;
  const Vec3<R> Gj{La1.x + dr * Gut.x, La1.y + dr * Gut.y, La1.z + dr * Gut.z};
  Lrho -= dr * dot3(Gut, c.u);
#pragma unroll
  for (int j = 0; j < Q; ++j) mu[j] = Lrho + xi_dot<Q>(j, Gj) + xi_P_xi<Q>(j, G);
  if (gut) *gut = Gut;
}

template <int Q, class R, bool EXACT>
__device__ __forceinline__ void transpose_collide(const RRCell<R, EXACT>& c, R (&mu)[Q],
                                                  const AdjointArgs& a) {
  rr_transpose<Q, R, EXACT>(c, mu, a, nullptr);
}

template <int Q, class R, bool EXACT, bool RR> struct CellOf { using T = LinCell<Q, R, EXACT>; };
template <int Q, class R, bool EXACT> struct CellOf<Q, R, EXACT, true> { using T = RRCell<R, EXACT>; };

// v += g_bar at one cell from the coefficients c of the objective's derivative
// polynomial in xi (nc = 2: J_FFA, c0 + c1 xi_x; otherwise J_DISS,
// c0 + c . xi + xi . C . xi with the squares, then the doubled cross terms, in
// the order of coef_basis)
template <int Q, class R>
__device__ __forceinline__ void expand_source(int nc, const R* c, R (&v)[Q]) {
  using L = Lat<Q>;
  constexpr int D = L::D;
  if (nc == 2) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      R t = c[0];
      if (L::cx(i)) t += L::cx(i) > 0 ? c[1] : -c[1];
      v[i] += t;
    }
    return;
  }
  constexpr int S0 = 1 + D;  // first square coefficient
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int ex = L::cx(i), ey = L::cy(i), ez = L::cz(i);
    R t = c[0];
    if (ex) t += ex > 0 ? c[1] : -c[1];
    if (ey) t += ey > 0 ? c[2] : -c[2];
    if constexpr (D == 3) {
      if (ez) t += ez > 0 ? c[3] : -c[3];
    }
    if (ex) t += c[S0];
    if (ey) t += c[S0 + 1];
    if constexpr (D == 2) {
      if (ex && ey) t += (ex * ey > 0) ? R(2) * c[S0 + 2] : -R(2) * c[S0 + 2];
    } else {
      if (ez) t += c[S0 + 2];
      if (ex && ey) t += (ex * ey > 0) ? R(2) * c[S0 + 3] : -R(2) * c[S0 + 3];
      if (ex && ez) t += (ex * ez > 0) ? R(2) * c[S0 + 4] : -R(2) * c[S0 + 4];
      if (ey && ez) t += (ey * ez > 0) ? R(2) * c[S0 + 5] : -R(2) * c[S0 + 5];
    }
    v[i] += t;
  }
}

// lam += g_bar in the source box.  J_FFA and J_DISS store g_bar as the
// coefficients of their derivative polynomials in xi (2 or 1 + D + D(D+1)/2 per
// cell instead of q values), expanded here; J_MEA stores the q values.
__device__ __forceinline__ AdjRhs rhs_of(const AdjointArgs& a) {
  AdjRhs r;
  r.lam = a.lam;
  r.src = a.src;
#pragma unroll
  for (int k = 0; k < 6; ++k) r.sb[k] = a.sb[k];
  r.src_pitch = a.src_pitch;
  r.src_nc = a.src_nc;
  r.snap = a.snap;
  r.red = a.red;
  return r;
}

template <int Q, class R>
__device__ __forceinline__ void add_source(const AdjRhs& a, int x, int y, int z, R (&v)[Q]) {
  if (x >= a.sb[0] && x < a.sb[1] && y >= a.sb[2] && y < a.sb[3] && z >= a.sb[4] && z < a.sb[5]) {
    constexpr int D = Lat<Q>::D;
    const long long bc = (long long)(x - a.sb[0]) +
                         (long long)(a.sb[1] - a.sb[0]) *
                             ((long long)(y - a.sb[2]) + (long long)(a.sb[3] - a.sb[2]) * (z - a.sb[4]));
    const R* src = static_cast<const R*>(a.src);
    const long long sp = a.src_pitch;
    if (a.src_nc == 0) {
#pragma unroll
      for (int i = 0; i < Q; ++i) v[i] += src[(long long)i * sp + bc];
    } else {
      R c[1 + D + D * (D + 1) / 2];
      const int nc = a.src_nc;
#pragma unroll
      for (int k = 0; k < 1 + D + D * (D + 1) / 2; ++k)
        if (k < nc) c[k] = src[(long long)k * sp + bc];
      expand_source<Q, R>(nc, c, v);
    }
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

// The squared update of every population is added to the thread's partial
// without rounding error: FP64 sweeps add in FP64; FP32 sweeps add each square
// to an unevaluated pair of floats (error-free TwoSum), which the block sums in
// pairs and converts to FP64 once per warp.  (Differences and squares in FP64
// made the comparing sweep FP64-bound: 3.5 ms against 1.1 ms for a plain sweep
// on the LES grid.)
template <int Q, class R, int RES>
__device__ __forceinline__ void residual_io(const AdjRhs& a, long long pitch, long long cell,
                                            const R (&v)[Q], typename JAcc<R>::T& rp) {
  if (RES == 0) return;
  R* sn = static_cast<R*>(a.snap);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    R* p = sn + (long long)i * pitch + cell;
    if (RES == 1) {
      *p = v[i];
    } else {
      const R dlt = v[i] - *p;
      jadd(rp, dlt * dlt);
    }
  }
}

// One block of an adjoint sweep: x-block bxi of row (y, z); blin is the
// block's slot in the residual partial sums.
template <int Q, class R, bool ODD, bool EXACT, int RES, bool RR>
__device__ __forceinline__ void adjoint_body(const AdjointArgs& a, int bxi, int y, int z,
                                             long long blin) {
  constexpr int S = RealStore<R>::S;
  const Grid& g = a.g;
  const int x = bxi * blockDim.x + threadIdx.x;
  R* A = static_cast<R*>(a.lam);
  const R* dp = static_cast<const R*>(a.d);
  typename JAcc<R>::T rp{};
  if (x < g.nx - 1) {
    const long long cell = cell_of(g, x, y, z);
    const Rows rows = make_rows<Lat<Q>::D>(g, y, z);
    R v[Q];
    aa_load<Q, S, ODD, -1>(A, g, rows, x, cell, v);
    typename CellOf<Q, R, EXACT, RR>::T c;
    const AdjRhs r0 = rhs_of(a);
    load_lin<Q, R, EXACT>(a, cell, dp[cell], c, v);
    transpose_collide<Q, R, EXACT>(c, v, a);
    add_source<Q, R>(r0, x, y, z, v);
    residual_io<Q, R, RES>(r0, g.pitch, cell, v, rp);
    if (x == g.nx - 2) {
      R vo[Q];
      aa_load<Q, S, ODD, -1>(A, g, rows, x + 1, cell + 1, vo);
      typename CellOf<Q, R, EXACT, RR>::T co;
      load_lin<Q, R, EXACT>(a, cell + 1, dp[cell + 1], co, vo);
      transpose_collide<Q, R, EXACT>(co, vo, a);
      add_source<Q, R>(r0, x + 1, y, z, vo);
      residual_io<Q, R, RES>(r0, g.pitch, cell + 1, vo, rp);
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
    if (threadIdx.x == 0) a.red[blin] = s;
  }
}

// Resident blocks per SM requested from ptxas for the FP32 D3Q19 sweeps
// (0 = no request, ptxas chooses); the exact variants otherwise take more than
// 120 registers.  Chosen by timing sweeps on the LES case (640x320x100):
//   BGK exact LES: none 1419 us, 4 blocks 1262, 5: 1270; again with the
//     slice of the benchmark (J_FFA / J_DISS sweeps, GLUPS): 3: 16.1 / 12.9,
//     4: 18.4 / 14.9, 5: 18.9 / 15.4, 6: 17.9 / 14.7; with the transposed
//     collision written through the weighted moments of mu: none 23.4 / 19.4,
//     4: 23.0 / 18.9, 5: 23.3 / 19.5, 6: 24.3 / 20.6
//   RR exact:      none 1265, 4: 1154, 5: 1091
//   RR frozen:     none 1167, 5: 1057, 6: 1043
#ifndef HLBM_AMINB_D3Q19
#define HLBM_AMINB_D3Q19 0
#endif
#ifndef HLBM_AMINB_D3Q19_EXACT
#define HLBM_AMINB_D3Q19_EXACT 6
#endif
#ifndef HLBM_AMINB_D3Q19_RR
#define HLBM_AMINB_D3Q19_RR 6
#endif
#ifndef HLBM_AMINB_D3Q19_RR_EXACT
#define HLBM_AMINB_D3Q19_RR_EXACT 5
#endif
template <int Q, class R, bool EXACT, bool RR>
constexpr int adjoint_min_blocks() {
  if (Q != 19 || sizeof(R) != 4) return 0;
  if (RR) return EXACT ? HLBM_AMINB_D3Q19_RR_EXACT : HLBM_AMINB_D3Q19_RR;
  return EXACT ? HLBM_AMINB_D3Q19_EXACT : HLBM_AMINB_D3Q19;
}

template <int Q, class R, bool ODD, bool EXACT, int RES, bool RR>
__global__ void __launch_bounds__(NT) k_adjoint(AdjointArgs a) {
  adjoint_body<Q, R, ODD, EXACT, RES, RR>(a, blockIdx.x, blockIdx.y, blockIdx.z, block_linear());
}

template <int Q, class R, bool ODD, bool EXACT, int RES, bool RR, int MB>
__global__ void __launch_bounds__(NT, MB) k_adjoint_mb(AdjointArgs a) {
  adjoint_body<Q, R, ODD, EXACT, RES, RR>(a, blockIdx.x, blockIdx.y, blockIdx.z, block_linear());
}

// Batched sweep over a work list (see k_primal_batch): block b processes tile
// tiles[b] = (context k, x-block, y, z) with the arguments tab[k].
template <int Q, bool ODD, int RES>
__global__ void __launch_bounds__(NT) k_adjoint_batch(const AdjointArgs* __restrict__ tab,
                                                      const int4* __restrict__ tiles) {
  const int4 t = tiles[blockIdx.x];
  const AdjointArgs& a = tab[t.x];
  const long long gx = (a.g.nx + NT - 1) / NT;
  adjoint_body<Q, float, ODD, false, RES, false>(
      a, t.y, t.z, t.w, t.y + gx * ((long long)t.z + (long long)a.g.ny * t.w));
}

template <int Q, bool ODD>
static cudaError_t launch_adj_batch_q(const AdjointArgs* tab, const int4* tiles, int ntiles,
                                      int res, cudaStream_t s) {
  if (res == 0) k_adjoint_batch<Q, ODD, 0><<<ntiles, NT, 0, s>>>(tab, tiles);
  else if (res == 1) k_adjoint_batch<Q, ODD, 1><<<ntiles, NT, 0, s>>>(tab, tiles);
  else k_adjoint_batch<Q, ODD, 2><<<ntiles, NT, 0, s>>>(tab, tiles);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_batch(const AdjointArgs* tab, const int4* tiles, int ntiles, int q,
                                 bool odd, int res, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  if (q == 9) return odd ? launch_adj_batch_q<9, true>(tab, tiles, ntiles, res, s)
                         : launch_adj_batch_q<9, false>(tab, tiles, ntiles, res, s);
  if (q == 19) return odd ? launch_adj_batch_q<19, true>(tab, tiles, ntiles, res, s)
                          : launch_adj_batch_q<19, false>(tab, tiles, ntiles, res, s);
  return cudaErrorInvalidValue;
}

template <int Q, class R, bool ODD, bool EXACT, int RES, bool RR>
static void launch_adj_one(const AdjointArgs& a, dim3 grid, int bx, cudaStream_t s) {
  constexpr int mb = adjoint_min_blocks<Q, R, EXACT, RR>();
  if constexpr (mb > 0) k_adjoint_mb<Q, R, ODD, EXACT, RES, RR, (mb > 0 ? mb : 1)><<<grid, bx, 0, s>>>(a);
  else k_adjoint<Q, R, ODD, EXACT, RES, RR><<<grid, bx, 0, s>>>(a);
}

int adjoint_blocks(const Grid& g) { return ((g.nx + g.bx - 1) / g.bx) * g.ny * g.nz; }

template <int Q, class R, bool RR>
static cudaError_t launch_adj_qr(const AdjointArgs& a, bool odd, bool exact, int res,
                                 cudaStream_t s) {
  const int bx = a.g.bx;
  dim3 grid((a.g.nx + bx - 1) / bx, a.g.ny, a.g.nz);
#define HLBM_A(O, E, RS) launch_adj_one<Q, R, O, E, RS, RR>(a, grid, bx, s)
#define HLBM_AR(O, E) \
  do { if (res == 0) HLBM_A(O, E, 0); else if (res == 1) HLBM_A(O, E, 1); else HLBM_A(O, E, 2); } while (0)
  if (!odd) { if (!exact) HLBM_AR(false, false); else HLBM_AR(false, true); }
  else      { if (!exact) HLBM_AR(true, false);  else HLBM_AR(true, true); }
#undef HLBM_AR
#undef HLBM_A
  return cudaGetLastError();
}

template <bool RR>
static cudaError_t launch_adj_c(const AdjointArgs& a, int q, bool dbl, bool odd, bool exact, int res,
                                cudaStream_t s) {
  if (q == 9) return dbl ? launch_adj_qr<9, double, RR>(a, odd, exact, res, s)
                         : launch_adj_qr<9, float, RR>(a, odd, exact, res, s);
  if (q == 19) return dbl ? launch_adj_qr<19, double, RR>(a, odd, exact, res, s)
                          : launch_adj_qr<19, float, RR>(a, odd, exact, res, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_adjoint(const AdjointArgs& a, int q, bool dbl, bool odd, bool exact, int res,
                           bool rr, cudaStream_t s) {
  return rr ? launch_adj_c<true>(a, q, dbl, odd, exact, res, s)
            : launch_adj_c<false>(a, q, dbl, odd, exact, res, s);
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
  if (a.exact && !a.rr) {
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
  if (a.rr) {
    // non-equilibrium stress of f_bar: Pi = M2 - rho u~ u~ - (rho - 1)/3 I
    constexpr int D = Lat<Q>::D;
    const double d = (double)static_cast<const R*>(a.d)[cell];
    double ut[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < D; ++k) ut[k] = d * a.msum[(1 + k) * g.N + cell] * a.inv_n * ir + (1.0 - d) * a.us[k];
    const double t = (rho - 1.0) / 3.0;
    const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
    // plane order of the sums and of the record: 2D xx, yy, xy; 3D xx, yy, zz, xy, xz, yz
    const int map2[3] = {0, 1, 3};
    const int np = D == 2 ? 3 : 6;
    for (int k = 0; k < np; ++k) {
      const int e = D == 2 ? map2[k] : k;
      double v = a.msum[(long long)(1 + D + k) * g.N + cell] * a.inv_n - rho * ut[ia[e]] * ut[ib[e]];
      if (e < 3) v -= t;
      rec[(long long)(D + 2 + k) * rp + cell] = (R)v;
    }
  }
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
    R cf[1 + D + D * (D + 1) / 2];
    R* src = static_cast<R*>(a.src);
#pragma unroll
    for (int k = 0; k < 1 + D + D * (D + 1) / 2; ++k) {
      if (k >= nc) break;
      cf[k] = (R)(a.gsum[(long long)k * a.g.N + cell] * a.inv_n);
      src[(long long)k * vol + bc] = cf[k];
    }
    // ||g_bar||^2 of the values the sweep forms from these coefficients
    R gv[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) gv[i] = R(0);
    expand_source<Q, R>(nc, cf, gv);
#pragma unroll
    for (int i = 0; i < Q; ++i) acc += (double)gv[i] * (double)gv[i];
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
// momentum-exchange drag J_MEA (Sec. 4.1, Eq. obj_mea), n = e_x:
//   J = (1/A) sum_{x in Gamma_s} sum_i xi_ix (f_i(x + xi_i) - f_ibar(x)),
// Gamma_s the fluid-side surface nodes (d >= 1/2 with a lattice neighbour of
// d < 1/2), A their number; terms whose neighbour leaves the domain in x are
// left out.  J is linear in f, so its time average is J(f_bar) and its
// derivative is the constant
//   dJ/df_j(y) = (xi_jx / A) [1(y - xi_j in Gamma_s) + 1(y in Gamma_s, y - xi_j in domain)].
// ----------------------------------------------------------------------------
template <int Q, class R>
__device__ __forceinline__ bool is_surface(const R* d, const Grid& g, const Rows& rows, int x,
                                           long long cell) {
  if (!(d[cell] >= R(0.5))) return false;
  using L = Lat<Q>;
  bool hit = false;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const int xn = x + L::cx(i);
    if (xn < 0 || xn >= g.nx) continue;
    hit |= d[rows.r[L::cy(i) + 1][L::cz(i) + 1] + xn] < R(0.5);
  }
  return hit;
}

template <int Q, class R>
__global__ void __launch_bounds__(NT) k_mea_eval(const double* fsum, double inv_n, const void* dv,
                                                 Grid g, double* part_j, double* part_n) {
  using L = Lat<Q>;
  const R* d = static_cast<const R*>(dv);
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  double jv = 0.0, nv = 0.0;
  if (x < g.nx) {
    const long long cell = cell_of(g, x, y, z);
    const Rows rows = make_rows<L::D>(g, y, z);
    if (is_surface<Q, R>(d, g, rows, x, cell)) {
      nv = 1.0;
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        if (L::cx(i) == 0) continue;
        const int xn = x + L::cx(i);
        if (xn < 0 || xn >= g.nx) continue;
        const long long nb = rows.r[L::cy(i) + 1][L::cz(i) + 1] + xn;
        // deviations suffice: w_i = w_ibar cancels
        const double t = fsum[(long long)i * g.N + nb] - fsum[(long long)L::opp(i) * g.N + cell];
        jv += (L::cx(i) > 0 ? t : -t) * inv_n;
      }
    }
  }
  __shared__ double sh[NT / 32];
  const double sj = block_sum<NT>(jv, sh);
  const double sn = block_sum<NT>(nv, sh);
  if (threadIdx.x == 0) {
    part_j[block_linear()] = sj;
    part_n[block_linear()] = sn;
  }
}

template <int Q, class R>
__global__ void __launch_bounds__(NT) k_mea_source(const void* dv, Grid g, double inv_area, void* srcv,
                                                   double* red) {
  using L = Lat<Q>;
  const R* d = static_cast<const R*>(dv);
  R* src = static_cast<R*>(srcv);
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  double acc = 0.0;
  if (x < g.nx) {
    const long long cell = cell_of(g, x, y, z);
    const Rows rows = make_rows<L::D>(g, y, z);
    const bool here = is_surface<Q, R>(d, g, rows, x, cell);
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      double gv = 0.0;
      if (L::cx(j) != 0) {
        const int xb = x - L::cx(j);
        if (xb >= 0 && xb < g.nx) {
          // rows of y - xi_j: the neighbour in direction opp(j)
          const int o = L::opp(j);
          const long long nb = rows.r[L::cy(o) + 1][L::cz(o) + 1] + xb;
          const int yb = y - L::cy(j), zb = z - L::cz(j);
          const int yw = yb < 0 ? yb + g.ny : (yb >= g.ny ? yb - g.ny : yb);
          const int zw = zb < 0 ? zb + g.nz : (zb >= g.nz ? zb - g.nz : zb);
          const Rows rb = make_rows<L::D>(g, yw, zw);
          const double cnt = (is_surface<Q, R>(d, g, rb, xb, nb) ? 1.0 : 0.0) + (here ? 1.0 : 0.0);
          gv = (L::cx(j) > 0 ? cnt : -cnt) * inv_area;
        }
      }
      src[(long long)j * g.N + cell] = (R)gv;
      acc += gv * gv;
    }
  }
  __shared__ double sh[NT / 32];
  const double sm = block_sum<NT>(acc, sh);
  if (threadIdx.x == 0) red[block_linear()] = sm;
}

cudaError_t launch_mea_eval(const double* fsum, double inv_n, const void* d, const Grid& g, int q,
                            bool dbl, double* part_j, double* part_n, int* nblocks, cudaStream_t s) {
  dim3 grid((g.nx + NT - 1) / NT, g.ny, g.nz);
  *nblocks = (int)(grid.x * grid.y * grid.z);
#define HLBM_ME(QQ, RR) k_mea_eval<QQ, RR><<<grid, NT, 0, s>>>(fsum, inv_n, d, g, part_j, part_n)
  if (q == 9) { if (dbl) HLBM_ME(9, double); else HLBM_ME(9, float); }
  else if (q == 19) { if (dbl) HLBM_ME(19, double); else HLBM_ME(19, float); }
  else return cudaErrorInvalidValue;
#undef HLBM_ME
  return cudaGetLastError();
}

cudaError_t launch_mea_source(const void* d, const Grid& g, int q, bool dbl, double inv_area,
                              void* src, double* red, int* nblocks, cudaStream_t s) {
  dim3 grid((g.nx + NT - 1) / NT, g.ny, g.nz);
  *nblocks = (int)(grid.x * grid.y * grid.z);
#define HLBM_MS(QQ, RR) k_mea_source<QQ, RR><<<grid, NT, 0, s>>>(d, g, inv_area, src, red)
  if (q == 9) { if (dbl) HLBM_MS(9, double); else HLBM_MS(9, float); }
  else if (q == 19) { if (dbl) HLBM_MS(19, double); else HLBM_MS(19, float); }
  else return cudaErrorInvalidValue;
#undef HLBM_MS
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// gradient: G = dJ/dd_bar + sum_i mu_i dC_i/dd over the design box
//   dC_i/dd = omega w_i rho (3 xi_i.v + 9 (xi_i.u~)(xi_i.v) - 3 u~.v),  v = u - u_s
//   so sum_i mu_i dC_i/dd = omega rho (s - 3 u~ s0) . v;
//   exact LES adds (sum_i mu_i (f^eq_i - f_i)) d omega/dd with
//   Pi : dPi/dd = -2 rho v . Pi . u~.
// ----------------------------------------------------------------------------
template <int Q, class R, bool EXACT, bool RR>
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
  R val;
  if constexpr (RR) {
    RRCell<R, EXACT> c;
    load_lin<Q, R, EXACT>(a, cell, static_cast<const R*>(ga.d)[cell], c);
    R mt[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) mt[i] = mu[i];
    Vec3<R> gut;
    rr_transpose<Q, R, EXACT>(c, mt, a, &gut);
    const Vec3<R> v{c.u.x - par<R>(ga.us[0], ga.us_f[0]), c.u.y - par<R>(ga.us[1], ga.us_f[1]),
                    c.u.z - par<R>(ga.us[2], ga.us_f[2])};
    val = dot3(gut, v);
  } else {
    LinCell<Q, R, EXACT> c;
    load_lin<Q, R, EXACT>(a, cell, static_cast<const R*>(ga.d)[cell], c, mu);
    const MuC<R> k = mu_contract<Q, R>(mu, c.ut, EXACT ? c.drho : c.rho - R(1), c.rho);
    const Vec3<R> v{c.u.x - par<R>(ga.us[0], ga.us_f[0]), c.u.y - par<R>(ga.us[1], ga.us_f[1]),
                    c.u.z - par<R>(ga.us[2], ga.us_f[2])};
    val = c.om * c.rho * dot3(k.gv, v);
    if constexpr (EXACT) {
      if (c.nP > pi_eps<R>()) {
        const R pdd = -R(2) * c.rho * dot3(v, sym_mul(c.P, c.ut));
        // (sum mu (feq - f)) * (-om^2) * k pdd / ((2 tau - tau_b) |Pi|)
        val += (c.sg - k.qe) * c.om * c.om * par<R>(ga.kles, ga.kles_f) * pdd /
               ((R(2) * c.tau - par<R>(ga.tau_b, ga.tau_b_f)) * c.nP);
      }
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

cudaError_t launch_gradient(const GradArgs& a, int q, bool dbl, bool exact, bool rr, cudaStream_t s) {
  const int bx = a.box[1] - a.box[0], by = a.box[3] - a.box[2], bz = a.box[5] - a.box[4];
  dim3 grid((bx + NT - 1) / NT, by, bz);
#define HLBM_G(QQ, RT)                                                              \
  do {                                                                              \
    if (rr) { if (exact) k_gradient<QQ, RT, true, true><<<grid, NT, 0, s>>>(a);        \
              else k_gradient<QQ, RT, false, true><<<grid, NT, 0, s>>>(a); }           \
    else { if (exact) k_gradient<QQ, RT, true, false><<<grid, NT, 0, s>>>(a);          \
           else k_gradient<QQ, RT, false, false><<<grid, NT, 0, s>>>(a); }             \
  } while (0)
  if (q == 9) { if (dbl) HLBM_G(9, double); else HLBM_G(9, float); }
  else if (q == 19) { if (dbl) HLBM_G(19, double); else HLBM_G(19, float); }
  else return cudaErrorInvalidValue;
#undef HLBM_G
  return cudaGetLastError();
}

}  // namespace hlbm
