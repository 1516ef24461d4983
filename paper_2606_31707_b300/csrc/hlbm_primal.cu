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

// deviation of the equilibrium g^eq_i = f^eq_i(rho, u) - w_i for all i
template <int Q, class R>
__device__ __forceinline__ void equilibrium_dev(R (&g)[Q], R drho, const Vec3<R>& u) {
  const R uu = dot3(u, u);
  const R rho = R(1) + drho;
#pragma unroll
  for (int i = 0; i < Q; ++i) g[i] = geq_i<Q>(i, drho, rho, u, uu);
}

// The same update split in two: the old values are loaded right after the
// populations (so that all loads of a cell are in flight together, before any
// store), the new values are written at the end.
template <class R, int ACC>
struct AccSlot {
  double s;   // FP64 sum (FP64 kernels, and the fold of FP32 kernels)
  float t;    // FP32 staging value (FP32 kernels)
  __device__ __forceinline__ void load(const double* sum, const float* stage, long long k) {
    if constexpr (sizeof(R) == 8) {
      s = sum[k];
    } else {
      t = stage[k];
      if constexpr ((ACC & ACC_FLUSH) != 0) s = sum[k];
    }
  }
  __device__ __forceinline__ void store(double* sum, float* stage, long long k, R v) const {
    if constexpr (sizeof(R) == 8) {
      sum[k] = s + (double)v;
    } else if constexpr ((ACC & ACC_FLUSH) == 0) {
      stage[k] = t + v;
    } else {
      sum[k] = s + (double)(t + v);
      stage[k] = 0.0f;
    }
  }
};

// A group of G running sums of one cell updated together.  FP64 kernels add to
// the FP64 sums directly.  FP32 kernels keep the staged values of the group in
// G / 4 float4 planes followed by G % 4 float planes (no unused lanes: one
// 16-byte access per four sums, one 4-byte access per remaining sum) and, in
// the flush variant, fold them into the FP64 sums.  addr(k) gives the FP64 sum
// of component k at this cell.
__device__ __forceinline__ float& comp4(float4& v, int c) {
  return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}

// Shared-memory slots of one thread's staged sums: float4 slot j of the thread
// at s4[j * NT + tid], float slot j at sr[j * NT + tid].
struct Slots {
  float4* s4;
  float* sr;
};

template <class R, int ACC, int G>
struct SumGroup {
  static constexpr bool PACKED = sizeof(R) == 4;
  static constexpr bool FLUSH = (ACC & ACC_FLUSH) != 0;
  static constexpr int C4 = G / 4, CR = G % 4;
  float4 t[PACKED && C4 > 0 ? C4 : 1];
  float r[PACKED && CR > 0 ? CR : 1];
  double s[(!PACKED || FLUSH) ? G : 1];
  __device__ __forceinline__ float& staged(int k) {
    return k < 4 * C4 ? comp4(t[k / 4], k % 4) : r[k - 4 * C4];
  }
  // FP32: start copying this cell's staged values into the thread's shared slots
  __device__ __forceinline__ static void prefetch(const float* stage, long long N, long long cell,
                                                  const Slots& sl) {
    const float4* st = reinterpret_cast<const float4*>(stage);
    const int tid = threadIdx.x;
#pragma unroll
    for (int j = 0; j < C4; ++j) cp_async16(sl.s4 + j * NT + tid, st + (long long)j * N + cell);
    const float* sr = stage + 4LL * C4 * N;
#pragma unroll
    for (int j = 0; j < CR; ++j) cp_async4(sl.sr + j * NT + tid, sr + (long long)j * N + cell);
  }
  // FP32: the prefetched values (after cp_async_wait_all)
  __device__ __forceinline__ void take(const Slots& sl) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int j = 0; j < C4; ++j) t[j] = sl.s4[j * NT + tid];
#pragma unroll
    for (int j = 0; j < CR; ++j) r[j] = sl.sr[j * NT + tid];
  }
  // the FP64 sums read by this variant (FP64 kernels, and the fold of FP32 ones)
  template <class Addr>
  __device__ __forceinline__ void load_sums(const Addr& addr) {
    if constexpr (!PACKED || FLUSH) {
#pragma unroll
      for (int k = 0; k < G; ++k) s[k] = *addr(k);
    }
  }
  template <class Addr>
  __device__ __forceinline__ void load(const Addr& addr, const float* stage, long long N,
                                       long long cell) {
    if constexpr (PACKED) {
      const float4* st = reinterpret_cast<const float4*>(stage);
#pragma unroll
      for (int j = 0; j < C4; ++j) t[j] = st[(long long)j * N + cell];
      const float* sr = stage + 4LL * C4 * N;
#pragma unroll
      for (int j = 0; j < CR; ++j) r[j] = sr[(long long)j * N + cell];
    }
    load_sums(addr);
  }
  template <class Addr>
  __device__ __forceinline__ void store(const Addr& addr, float* stage, long long N,
                                        long long cell, const R (&v)[G]) {
    if constexpr (!PACKED) {
#pragma unroll
      for (int k = 0; k < G; ++k) *addr(k) = s[k] + (double)v[k];
    } else {
#pragma unroll
      for (int k = 0; k < G; ++k) {
        float& c = staged(k);
        if constexpr (FLUSH) {
          *addr(k) = s[k] + (double)(c + v[k]);
          c = 0.0f;
        } else {
          c += v[k];
        }
      }
      float4* st = reinterpret_cast<float4*>(stage);
#pragma unroll
      for (int j = 0; j < C4; ++j) st[(long long)j * N + cell] = t[j];
      float* sr = stage + 4LL * C4 * N;
#pragma unroll
      for (int j = 0; j < CR; ++j) sr[(long long)j * N + cell] = r[j];
    }
  }
};

// group sizes of the averaging variant ACC (see cell_update)
template <int Q, bool LES, int ACC, bool RR>
struct AccGroups {
  static constexpr int D = Lat<Q>::D;
  static constexpr bool FULL = (ACC & ACC_FULL) != 0;
  static constexpr int NM = 1 + D + (RR ? D * (D + 1) / 2 : 0);  // moment sums
  static constexpr int NTT = LES ? 1 : 0;                        // tau_eff - tau0
  static constexpr int NCD = 1 + D + D * (D + 1) / 2;             // dissipation coefficients
  static constexpr int GM = FULL ? 1 : NM + NTT;
  static constexpr int GF = FULL ? Q + NTT : 1;
  static constexpr int GA = FULL ? GF : GM;                       // the state group in use
  static constexpr int GD = NCD + 1;                              // dissipation group
  static constexpr int S4 = GA / 4 + GD / 4, SR = GA % 4 + GD % 4;  // shared slots per thread
};

// Collide the canonical state of one cell (as deviations g = f - w), store it
// AA-style, and (ACC > 0) add the cell's samples to the running averages.
// Returns the velocity.
//
// Averages kept (Sec. 3.3 and App. A: what the mean-flow adjoint reads):
//   rho - 1 and rho u of f (the BGK / frozen-turbulence linearisation needs
//   only the density and velocity of f_bar), all of f - w when ACC == 2 (the
//   exact LES linearisation needs f_bar itself), tau_eff - tau0 (LES), and per
//   objective the coefficients of dJ/df in the basis of coef_basis(), dJ/dd
//   and J.  With the recursive regularised collision (RR) also the second
//   moments sum xi xi (f - w): its linearisation reads rho, u and the
//   non-equilibrium stress of f_bar, all functions of moments up to order 2.
//
// RR selects the third-order recursive regularised collision of the
// turbulent model (Sec. 2.2, Eq. HRRLBM) instead of BGK:
//   f*_i = f^eq3_i + (1 - omega) f1_i,
//   f^eq3_i = f^eq_i + w_i rho (9/2) c (c^2 - u~.u~),    c = xi_i . u~,
//   f1_i = w_i [3 xi_i.a1 + (9/2)(xi_i Pi xi_i - tr Pi / 3)
//               + (9/2)(3 c xi_i Pi xi_i - c tr Pi - 2 xi_i . Pi u~)],
// with a1 = rho (u - u~), Pi the non-equilibrium stress, the recursive
// third-order coefficient a1^(3) = u~ (x) Pi (symmetrised) contracted with
// the third Hermite polynomial (the xxx and xyz entries vanish on D2Q9 and
// D3Q19).
//
// PF: the staged (FP32) values of this cell's sums were prefetched into the
// thread's shared-memory slots sla (state group) and sld (dissipation group).
template <int Q, int S, bool ODD, bool LES, int ACC, bool RR, bool PF>
__device__ __forceinline__ Vec3<typename Store<S>::real> cell_update(
    const PrimalArgs& a, typename Store<S>::mem* A, const Rows& rows, int x, int y, int z,
    long long cell,
    typename Store<S>::real (&g)[Q], typename Store<S>::real d,
    typename JAcc<typename Store<S>::real>::T (&jp)[2], const Slots& sla, const Slots& sld) {
  using R = typename Store<S>::real;
  using L = Lat<Q>;
  constexpr int D = L::D;
  const Grid& gr = a.g;
  // rho - 1 = sum g, m = rho u = sum xi g, M2 = sum xi xi g over the opposite pairs
  Mom<R> ax, dg;
  class_moments<Q, R>(g, ax, dg);
  const R drho = g[0] + ax.m0 + dg.m0;
  const R rho = R(1) + drho;
  const Vec3<R> m{ax.m1.x + dg.m1.x, ax.m1.y + dg.m1.y, D == 3 ? ax.m1.z + dg.m1.z : R(0)};
  const R inv_rho = R(1) / rho;
  const Vec3<R> u{m.x * inv_rho, m.y * inv_rho, m.z * inv_rho};
  if (!(rho > R(0)) || !(fabs(u.x) + fabs(u.y) + fabs(u.z) < R(1e30))) atomicOr(a.err, 1u);
  const Vec3<R> us{par<R>(a.us[0], a.us_f[0]), par<R>(a.us[1], a.us_f[1]),
                   par<R>(a.us[2], a.us_f[2])};
  const R one_d = R(1) - d;
  const Vec3<R> ut{d * u.x + one_d * us.x, d * u.y + one_d * us.y, d * u.z + one_d * us.z};
  const R uu = dot3(ut, ut);

  const R tau0 = par<R>(a.tau0, a.tau0_f);
  R tau = tau0;
  Sym<R> P{0, 0, 0, 0, 0, 0};
  R nP = 0;
  const bool diss_here = ACC > 0 && (a.obj_mask & 2) && x >= a.db[0] && x < a.db[1] &&
                         y >= a.db[2] && y < a.db[3] && z >= a.db[4] && z < a.db[5];
  // The non-equilibrium stress from the second moment of f - w (the lattice
  // sums of f^eq - w are (rho - 1)/3 I + rho u~ u~ on both lattices):
  //   Pi = sum xi xi (f - w) - rho u~ u~ - (rho - 1)/3 I,
  // so no array of f - f^eq is formed.
  const Sym<R> M2{ax.m2.xx + dg.m2.xx, ax.m2.yy + dg.m2.yy, D == 3 ? ax.m2.zz + dg.m2.zz : R(0),
                  dg.m2.xy, D == 3 ? dg.m2.xz : R(0), D == 3 ? dg.m2.yz : R(0)};
  if (RR || LES || diss_here) {
    const R t = drho * R(1.0 / 3.0);
    P = Sym<R>{M2.xx - rho * ut.x * ut.x - t, M2.yy - rho * ut.y * ut.y - t,
               D == 3 ? M2.zz - rho * ut.z * ut.z - t : R(0), M2.xy - rho * ut.x * ut.y,
               D == 3 ? M2.xz - rho * ut.x * ut.z : R(0), D == 3 ? M2.yz - rho * ut.y * ut.z : R(0)};
  }
  if (LES || diss_here) nP = sqrt_r<R>(sym_norm2(P));
  const R kles = par<R>(a.kles, a.kles_f);
  if (LES) tau = tau_smagorinsky<R>(tau0, kles, nP);
  const R om = R(1) / tau;

  if constexpr (ACC > 0) {
    const long long N = gr.N;
    const bool ffa_here = (a.obj_mask & 1) && x == a.ffa[0] && y >= a.ffa[1] && y < a.ffa[2] &&
                          z >= a.ffa[3] && z < a.ffa[4];
    using AG = AccGroups<Q, LES, ACC, RR>;
    constexpr int NCD = AG::NCD;  // dissipation coefficients
    constexpr bool FULL = AG::FULL;
    // The averaged state is kept either as its moments (compact: rho - 1,
    // rho u[, xi xi (f - w)], which is all the BGK / frozen-turbulence / RR
    // linearisation reads) or, when f_bar itself is needed, as all q sums of
    // f - w (the moments are then derived from them once per window).  The
    // turbulent relaxation time rides in the same group.
    constexpr int NM = AG::NM;  // moment sums
    constexpr int GM = AG::GM;
    constexpr int GF = AG::GF;
    // old values of every sum this cell updates, loaded together
    const auto maddr = [&](int k) {
      return k < NM ? a.msum + (long long)k * N + cell : a.tsum + cell;
    };
    const auto faddr = [&](int k) {
      return k < Q ? a.fsum + (long long)k * N + cell : a.tsum + cell;
    };
    double* const g1 = a.gsum[1];
    double* const dd1 = a.ddsum[1];
    const auto daddr = [&](int k) { return k < NCD ? g1 + (long long)k * N + cell : dd1 + cell; };
    SumGroup<R, ACC, GM> sm;
    SumGroup<R, ACC, GF> sf;
    SumGroup<R, ACC, NCD + 1> sdiss;
    AccSlot<R, ACC> sg0[2];
    if constexpr (PF) {
      // the staged values are on their way to shared memory; a fold reads the FP64 sums
      if constexpr (FULL) sf.load_sums(faddr);
      else sm.load_sums(maddr);
      if (diss_here) sdiss.load_sums(daddr);
    } else {
      if constexpr (FULL) sf.load(faddr, a.fstage, N, cell);
      else sm.load(maddr, a.mstage, N, cell);
      if (diss_here) sdiss.load(daddr, a.gstage[1], N, cell);
    }
    if (ffa_here) {
      sg0[0].load(a.gsum[0], a.gstage[0], cell);
      sg0[1].load(a.gsum[0], a.gstage[0], N + cell);
    }

    // tau_eff - tau0 = kles |Pi| / tau_eff (the quadratic tau (tau - tau0) =
    // kles |Pi|), free of the cancellation of the difference in FP32
    const R tturb = LES ? kles * nP / tau : R(0);
    if constexpr (PF) {
      cp_async_wait_all();
      if constexpr (FULL) sf.take(sla);
      else sm.take(sla);
      if (diss_here) sdiss.take(sld);
    }
    if constexpr (FULL) {
      R fv[GF];
#pragma unroll
      for (int i = 0; i < Q; ++i) fv[i] = g[i];
      if constexpr (LES) fv[GF - 1] = tturb;
      sf.store(faddr, a.fstage, N, cell, fv);
    } else {
      R mv[GM];
      mv[0] = drho;
      mv[1] = m.x;
      mv[2] = m.y;
      if constexpr (D == 3) mv[3] = m.z;
      if constexpr (RR) {
        if constexpr (D == 2) {
          mv[3] = M2.xx;
          mv[4] = M2.yy;
          mv[5] = M2.xy;
        } else {
          mv[4] = M2.xx;
          mv[5] = M2.yy;
          mv[6] = M2.zz;
          mv[7] = M2.xy;
          mv[8] = M2.xz;
          mv[9] = M2.yz;
        }
      }
      if constexpr (LES) mv[GM - 1] = tturb;
      sm.store(maddr, a.mstage, N, cell, mv);
    }
    // far-field drag J_FFA on Gamma_J (Sec. 4.2): rho u_x (u0 - u_x) + c_s^2 (1 - rho);
    // dJ/df_j = (u_x^2 - c_s^2) + (u0 - 2 u_x) xi_jx
    if (ffa_here) {
      const R u0 = par<R>(a.u_in, a.u_in_f);
      sg0[0].store(a.gsum[0], a.gstage[0], cell, u.x * u.x - R(1.0 / 3.0));
      sg0[1].store(a.gsum[0], a.gstage[0], N + cell, u0 - R(2) * u.x);
      jadd(jp[0], m.x * (u0 - u.x) - R(1.0 / 3.0) * drho);
    }
    // dissipation J_DISS on Omega_J (Sec. 4.3): 2 nu S:S + (1-d)/tau0 u.u,
    // S = -3 Pi / (2 tau):  J = (9 nu / 2) |Pi|^2 / tau^2 + (1-d)/tau0 |u|^2.
    // dJ/df_j = fac Pi:dPi/df_j + c2 (xi_j.u - |u|^2) with
    // Pi:dPi/df_j = xi_j Pi xi_j - tr Pi / 3 - u~ Pi u~ - 2 d (xi_j - u) . Pi u~,
    // i.e. coefficients (1, xi, xi xi) = (A0, A, fac Pi).
    if (diss_here) {
      const R nu = par<R>(a.nu0, a.nu0_f);
      const R uu_raw = dot3(u, u);
      const R J = R(4.5) * nu * nP * nP / (tau * tau) + one_d / tau0 * uu_raw;
      // d(|Pi|^2 / tau^2) with tau(|Pi|): 2 Pi:dPi [1/tau^2 - |Pi| k/(tau^3 (2 tau - tau0))]
      R fac = R(1) / (tau * tau);
      if (LES) fac -= nP * kles / (tau * tau * tau * (R(2) * tau - tau0));
      fac *= R(9) * nu;
      const Vec3<R> PU = sym_mul(P, ut);
      const R uPu = dot3(ut, PU);
      const R trP = P.xx + P.yy + P.zz;
      const R uPU = dot3(u, PU);
      const R c2 = one_d / tau0 * R(2) / rho;
      R cf[NCD + 1];  // the dJ/df coefficients, then dJ/dd
      cf[0] = fac * (-trP * R(1.0 / 3.0) - uPu + R(2) * d * uPU) - c2 * uu_raw;
      cf[1] = -R(2) * d * fac * PU.x + c2 * u.x;
      cf[2] = -R(2) * d * fac * PU.y + c2 * u.y;
      if constexpr (D == 2) {
        cf[3] = fac * P.xx;
        cf[4] = fac * P.yy;
        cf[5] = fac * P.xy;
      } else {
        cf[3] = -R(2) * d * fac * PU.z + c2 * u.z;
        cf[4] = fac * P.xx;
        cf[5] = fac * P.yy;
        cf[6] = fac * P.zz;
        cf[7] = fac * P.xy;
        cf[8] = fac * P.xz;
        cf[9] = fac * P.yz;
      }
      const Vec3<R> v{u.x - us.x, u.y - us.y, u.z - us.z};
      cf[NCD] = fac * (-R(2) * rho * dot3(v, PU)) - uu_raw / tau0;
      sdiss.store(daddr, a.gstage[1], N, cell, cf);
      jadd(jp[1], J);
    }
  }

  if constexpr (RR) {
    // the sum f^eq3 + (1 - omega) f1 as a polynomial in xi_i:
    //   w_i [C0 + xi.V + (9/2)(rho c^2 + c1 p) + (9/2) c (rho c^2 + 3 c1 p)],
    //   c = xi.u~, p = xi.Pi.xi, c1 = 1 - omega,
    //   C0 = (rho - 1) - (3/2) rho u~.u~ - (3/2) c1 tr Pi,
    //   V = 3 rho u~ + 3 c1 a1 - (9/2) rho (u~.u~) u~ - (9/2) c1 (tr Pi u~ + 2 Pi u~)
    const R c1 = R(1) - om;
    const R trP = P.xx + P.yy + P.zz;
    const Vec3<R> PU = sym_mul(P, ut);
    const R C0 = drho - R(1.5) * rho * uu - R(1.5) * c1 * trP;
    const R kv = R(3) * rho - R(4.5) * rho * uu - R(4.5) * c1 * trP - R(3) * c1 * rho;
    const Vec3<R> V{kv * ut.x + R(3) * c1 * m.x - R(9) * c1 * PU.x,
                    kv * ut.y + R(3) * c1 * m.y - R(9) * c1 * PU.y,
                    kv * ut.z + R(3) * c1 * m.z - R(9) * c1 * PU.z};
    const R r45 = R(4.5) * rho, c45 = R(4.5) * c1;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const R cu = xi_dot<Q>(i, ut);
      const R xPx = xi_P_xi<Q>(i, P);
      const R rc2 = r45 * cu * cu;
      g[i] = R(Lat<Q>::w(i)) * (C0 + xi_dot<Q>(i, V) + rc2 + c45 * xPx + cu * (rc2 + R(3) * c45 * xPx));
    }
  } else {
    // BGK toward f^eq(rho, u~): g_i <- g_i - omega (g_i - (f^eq_i - w_i)), with
    // f^eq_i - w_i = w_i (A + B c^2) + w_i T c, c = xi_i . u~,
    // A = rho - 1 - 3/2 rho u~.u~, B = 9/2 rho, T = 3 rho, formed over the
    // opposite pairs (c changes sign, the rest is shared).  The update keeps
    // the form g - omega (g - g^eq), whose rounding is relative to the small
    // non-equilibrium part; (1 - omega) g + omega g^eq rounds relative to g and
    // g^eq themselves, which at omega near 1.5 is about twice as much.
    const R A_ = drho - R(1.5) * rho * uu, B_ = R(4.5) * rho, T_ = R(3) * rho;
    const R wa = R(L::w(1)), wd = R(L::w(Q - 1));
    const R aA = wa * A_, aB = wa * B_, aT = wa * T_;
    const R dA = wd * A_, dB = wd * B_, dT = wd * T_;
    g[0] -= om * (g[0] - R(L::w(0)) * A_);
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
      const bool axd = axis_dir<Q>(i);
      const R cu = xi_dot<Q>(i, ut);
      const R sym = (axd ? aA : dA) + (axd ? aB : dB) * (cu * cu);
      const R anti = (axd ? aT : dT) * cu;
      g[i] -= om * (g[i] - (sym + anti));
      g[i + 1] -= om * (g[i + 1] - (sym - anti));
    }
  }
  aa_store<Q, S, ODD, +1>(A, gr, rows, x, cell, g);
  return u;
}

// Resident blocks per SM requested from ptxas (which then caps registers at
// 65536 / (NT * blocks)); 0 = no request (ptxas chooses).  Chosen by timing
// each variant (CUDA events, 3 repeats) on the Karman case (D2Q9 1100x410)
// and the LES case (D3Q19 640x320x100), FP32:
//   D2Q9 BGK averaging:   none 18.5 us, 8 blocks 16.4 us (64 registers)
//   D3Q19 BGK averaging with the shared-memory prefetch of the staged sums and
//   no barrier (the exact-LES window, full f): none 1621 us (108 / 134
//   registers even / odd), 4: 1452, 5: 1447, 6: 1582 (spills); after the
//   collision was written over opposite pairs with the stress from the second
//   moment (GLUPS in the benchmark slice): 4: 14.46, 5: 14.71, 6: 15.06
//   D3Q19 RR averaging:   none 1800 us, 4: 1880, 5: 1687
//   D3Q19 RR plain:       none 712 us, 4: 796
#ifndef HLBM_MINB_ACC_D2Q9
#define HLBM_MINB_ACC_D2Q9 8
#endif
#ifndef HLBM_MINB_ACC_D3Q19
#define HLBM_MINB_ACC_D3Q19 6
#endif
#ifndef HLBM_MINB_ACC_RR_D2Q9
#define HLBM_MINB_ACC_RR_D2Q9 0
#endif
#ifndef HLBM_MINB_ACC_RR_D3Q19
#define HLBM_MINB_ACC_RR_D3Q19 5
#endif
#ifndef HLBM_MINB_RR_D2Q9
#define HLBM_MINB_RR_D2Q9 0
#endif
#ifndef HLBM_MINB_RR_D3Q19
#define HLBM_MINB_RR_D3Q19 0
#endif
template <int Q, int ACC, bool RR>
constexpr int primal_min_blocks() {
  if (ACC > 0 && !RR) return Q == 9 ? HLBM_MINB_ACC_D2Q9 : HLBM_MINB_ACC_D3Q19;
  if (ACC > 0) return Q == 9 ? HLBM_MINB_ACC_RR_D2Q9 : HLBM_MINB_ACC_RR_D3Q19;
  if (RR) return Q == 9 ? HLBM_MINB_RR_D2Q9 : HLBM_MINB_RR_D3Q19;
  return 0;
}

// One block of a primal step: x-block bxi of row (y, z); blin is the block's
// linear index (its warps' objective slots follow from it).
template <int Q, int S, bool ODD, bool LES, int ACC, bool RR>
__device__ __forceinline__ void primal_body(const PrimalArgs& a, int bxi, int y, int z,
                                            long long blin) {
  using St = Store<S>;
  using R = typename St::real;
  const Grid& gr = a.g;
  const int x = bxi * blockDim.x + threadIdx.x;
  auto* A = static_cast<typename St::mem*>(a.f);
  const R* dp = static_cast<const R*>(a.d);
  typename JAcc<R>::T jp[2] = {};  // this thread's J terms (FP64, or double-float)
  // FP32 averaging variants copy the staged values of the cell's sums into
  // shared memory before the populations are read (cp.async: no registers
  // held while they are in flight; they are needed only at the end)
  constexpr bool PF = ACC > 0 && sizeof(R) == 4;
  using AG = AccGroups<Q, LES, ACC, RR>;
  __shared__ float4 pf4[PF && AG::S4 > 0 ? AG::S4 * NT : 1];
  __shared__ float pfr[PF && AG::SR > 0 ? AG::SR * NT : 1];
  const Slots sla{pf4, pfr};
  const Slots sld{pf4 + (AG::GA / 4) * NT, pfr + (AG::GA % 4) * NT};
  if (x < gr.nx - 1) {
    const long long cell = cell_of(gr, x, y, z);
    if constexpr (PF) {
      const long long N = gr.N;
      if constexpr (AG::FULL) SumGroup<R, ACC, AG::GF>::prefetch(a.fstage, N, cell, sla);
      else SumGroup<R, ACC, AG::GM>::prefetch(a.mstage, N, cell, sla);
      const bool diss_here = (a.obj_mask & 2) && x >= a.db[0] && x < a.db[1] && y >= a.db[2] &&
                             y < a.db[3] && z >= a.db[4] && z < a.db[5];
      if (diss_here) SumGroup<R, ACC, AG::GD>::prefetch(a.gstage[1], N, cell, sld);
    }
    const Rows rows = make_rows<Lat<Q>::D>(gr, y, z);
    R g[Q];
    if (x == 0) {
      const R uin = a.inflow ? (R)a.inflow[y + (long long)gr.ny * z] : par<R>(a.u_in, a.u_in_f);
      equilibrium_dev<Q, R>(g, R(0), Vec3<R>{uin, R(0), R(0)});
    } else {
      aa_load<Q, S, ODD, +1>(A, gr, rows, x, cell, g);
    }
    const Vec3<R> u =
        cell_update<Q, S, ODD, LES, ACC, RR, PF>(a, A, rows, x, y, z, cell, g, dp[cell], jp, sla, sld);
    if (x == gr.nx - 2) {
      // outflow node: f^eq(1, u(nx-2)), then relaxed and streamed like any cell
      // (its sums read directly)
      R go[Q];
      equilibrium_dev<Q, R>(go, R(0), u);
      cell_update<Q, S, ODD, LES, ACC, RR, false>(a, A, rows, x + 1, y, z, cell + 1, go,
                                                   dp[cell + 1], jp, sla, sld);
    }
  }
  if constexpr (ACC > 0) {
    // J of this step: each cell's term (computed in the arithmetic type) is
    // summed over the warp in FP64 (FP64 kernels) or as a double-float pair
    // (FP32 kernels) and added by the warp's first lane to the warp's own FP64
    // running slot (blocks x warps per block slots): no FP32 rounding in the
    // reduction, no barrier, and a fixed summation order
    const long long slot = blin * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5);
#pragma unroll
    for (int o = 0; o < 2; ++o) {
      if (!(a.obj_mask & (1 << o))) continue;
      const double w = warp_sum_j(jp[o]);
      if ((threadIdx.x & 31) == 0) a.jblk[o][slot] += w;
    }
  }
}

template <int Q, int S, bool ODD, bool LES, int ACC, bool RR>
__global__ void __launch_bounds__(NT) k_primal(PrimalArgs a) {
  primal_body<Q, S, ODD, LES, ACC, RR>(a, blockIdx.x, blockIdx.y, blockIdx.z, block_linear());
}

template <int Q, int S, bool ODD, bool LES, int ACC, bool RR, int MB>
__global__ void __launch_bounds__(NT, MB) k_primal_mb(PrimalArgs a) {
  primal_body<Q, S, ODD, LES, ACC, RR>(a, blockIdx.x, blockIdx.y, blockIdx.z, block_linear());
}

// Batched step over a work list: block b processes tile tiles[b] = (context k,
// x-block, y, z) of context k, whose arguments are tab[k].  Every context has
// NT-wide blocks, so a tile is exactly one of the context's own blocks and its
// objective slot is the one the single-context kernel would use.
template <int Q, int S, bool ODD, bool LES, int ACC, bool RR>
__global__ void __launch_bounds__(NT) k_primal_batch(const PrimalArgs* __restrict__ tab,
                                                     const int4* __restrict__ tiles) {
  const int4 t = tiles[blockIdx.x];
  const PrimalArgs& a = tab[t.x];
  const long long gx = (a.g.nx + NT - 1) / NT;
  primal_body<Q, S, ODD, LES, ACC, RR>(a, t.y, t.z, t.w,
                                       t.y + gx * ((long long)t.z + (long long)a.g.ny * t.w));
}

// Batched steps are built for the serving form: FP32 populations, BGK without
// the Smagorinsky model, compact averages (ACC 0, ON, ON | FLUSH)
template <int Q, bool ODD>
static cudaError_t launch_batch_q(const PrimalArgs* tab, const int4* tiles, int ntiles, int acc,
                                  cudaStream_t s) {
  switch (acc) {
    case 0: k_primal_batch<Q, ST_F32, ODD, false, 0, false><<<ntiles, NT, 0, s>>>(tab, tiles); break;
    case ACC_ON:
      k_primal_batch<Q, ST_F32, ODD, false, ACC_ON, false><<<ntiles, NT, 0, s>>>(tab, tiles);
      break;
    case ACC_ON | ACC_FLUSH:
      k_primal_batch<Q, ST_F32, ODD, false, ACC_ON | ACC_FLUSH, false><<<ntiles, NT, 0, s>>>(tab, tiles);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_primal_batch(const PrimalArgs* tab, const int4* tiles, int ntiles, int q,
                                bool odd, int acc, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  if (q == 9) return odd ? launch_batch_q<9, true>(tab, tiles, ntiles, acc, s)
                         : launch_batch_q<9, false>(tab, tiles, ntiles, acc, s);
  if (q == 19) return odd ? launch_batch_q<19, true>(tab, tiles, ntiles, acc, s)
                          : launch_batch_q<19, false>(tab, tiles, ntiles, acc, s);
  return cudaErrorInvalidValue;
}

template <int Q, int S, bool ODD, bool LES, int ACC, bool RR>
static void launch_one(const PrimalArgs& a, dim3 grid, int bx, cudaStream_t s) {
  constexpr int mb = primal_min_blocks<Q, ACC, RR>();
  if constexpr (mb > 0) k_primal_mb<Q, S, ODD, LES, ACC, RR, (mb > 0 ? mb : 1)><<<grid, bx, 0, s>>>(a);
  else k_primal<Q, S, ODD, LES, ACC, RR><<<grid, bx, 0, s>>>(a);
}

template <int Q, int S, bool RR>
static cudaError_t launch_primal_qs(const PrimalArgs& a, bool odd, bool les, int acc,
                                    cudaStream_t s) {
  const int bx = a.g.bx;
  dim3 grid((a.g.nx + bx - 1) / bx, a.g.ny, a.g.nz);
#define HLBM_L(O, L_, A_) launch_one<Q, S, O, L_, A_, RR>(a, grid, bx, s)
#define HLBM_LA(O, L_)                                   \
  do {                                                   \
    switch (acc) {                                       \
      case 0: HLBM_L(O, L_, 0); break;                   \
      case ACC_ON: HLBM_L(O, L_, ACC_ON); break;         \
      case ACC_ON | ACC_FULL: HLBM_L(O, L_, ACC_ON | ACC_FULL); break; \
      case ACC_ON | ACC_FLUSH: HLBM_L(O, L_, ACC_ON | ACC_FLUSH); break; \
      case ACC_ON | ACC_FULL | ACC_FLUSH: HLBM_L(O, L_, ACC_ON | ACC_FULL | ACC_FLUSH); break; \
      default: return cudaErrorInvalidValue;             \
    }                                                    \
  } while (0)
  if (!odd) { if (!les) HLBM_LA(false, false); else HLBM_LA(false, true); }
  else      { if (!les) HLBM_LA(true, false);  else HLBM_LA(true, true); }
#undef HLBM_LA
#undef HLBM_L
  return cudaGetLastError();
}

template <bool RR>
static cudaError_t launch_primal_c(const PrimalArgs& a, int q, int storage, bool odd, bool les,
                                   int acc, cudaStream_t s) {
  if (q == 9) {
    switch (storage) {
      case ST_F64: return launch_primal_qs<9, ST_F64, RR>(a, odd, les, acc, s);
      case ST_F32: return launch_primal_qs<9, ST_F32, RR>(a, odd, les, acc, s);
      case ST_F16: return launch_primal_qs<9, ST_F16, RR>(a, odd, les, acc, s);
      case ST_BF16: return launch_primal_qs<9, ST_BF16, RR>(a, odd, les, acc, s);
    }
  } else if (q == 19) {
    switch (storage) {
      case ST_F64: return launch_primal_qs<19, ST_F64, RR>(a, odd, les, acc, s);
      case ST_F32: return launch_primal_qs<19, ST_F32, RR>(a, odd, les, acc, s);
      case ST_F16: return launch_primal_qs<19, ST_F16, RR>(a, odd, les, acc, s);
      case ST_BF16: return launch_primal_qs<19, ST_BF16, RR>(a, odd, les, acc, s);
    }
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_primal(const PrimalArgs& a, int q, int storage, bool odd, bool les, int acc,
                          bool rr, cudaStream_t s) {
  return rr ? launch_primal_c<true>(a, q, storage, odd, les, acc, s)
            : launch_primal_c<false>(a, q, storage, odd, les, acc, s);
}

// ----------------------------------------------------------------------------
// state readout / initialisation
// ----------------------------------------------------------------------------
template <int Q, int S, bool ODD>
__global__ void __launch_bounds__(NT) k_readout(const void* fv, Grid gr, double u_in,
                                                const double* inflow, double* fout,
                                                double* rho_out, double* u_out) {
  using St = Store<S>;
  using R = typename St::real;
  const int x = blockIdx.x * NT + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= gr.nx) return;
  const auto* A = static_cast<const typename St::mem*>(fv);
  const long long cell = cell_of(gr, x, y, z);
  const Rows rows = make_rows<Lat<Q>::D>(gr, y, z);
  R g[Q];
  if (x == 0) {
    const double uin = inflow ? inflow[y + (long long)gr.ny * z] : u_in;
    equilibrium_dev<Q, R>(g, R(0), Vec3<R>{R(uin), R(0), R(0)});
  } else if (x == gr.nx - 1) {
    R gi[Q];
    aa_load<Q, S, ODD, +1>(A, gr, rows, x - 1, cell - 1, gi);
    R dr, r;
    Vec3<R> m, u;
    moments_dev<Q>(gi, dr, r, m, u);
    equilibrium_dev<Q, R>(g, R(0), u);
  } else {
    aa_load<Q, S, ODD, +1>(A, gr, rows, x, cell, g);
  }
  if (fout) {
#pragma unroll
    for (int i = 0; i < Q; ++i) fout[(long long)i * gr.N + cell] = (double)g[i] + Lat<Q>::w(i);
  }
  if (rho_out || u_out) {
    R dr, r;
    Vec3<R> m, u;
    moments_dev<Q>(g, dr, r, m, u);
    if (rho_out) rho_out[cell] = 1.0 + (double)dr;
    if (u_out) {
      u_out[cell] = (double)u.x;
      u_out[gr.N + cell] = (double)u.y;
      if (Lat<Q>::D == 3) u_out[2 * gr.N + cell] = (double)u.z;
    }
  }
}

template <int Q, int S>
__global__ void __launch_bounds__(NT) k_set_state(void* fv, Grid gr, const double* in) {
  using St = Store<S>;
  const int x = blockIdx.x * NT + threadIdx.x;
  if (x >= gr.nx) return;
  const long long cell = cell_of(gr, x, blockIdx.y, blockIdx.z);
  auto* A = static_cast<typename St::mem*>(fv);
#pragma unroll
  for (int i = 0; i < Q; ++i)
    St::st(A + (long long)i * gr.pitch + cell,
           (typename St::real)(in[(long long)i * gr.N + cell] - Lat<Q>::w(i)));
}

template <int Q, int S>
__global__ void __launch_bounds__(NT) k_init_eq(void* fv, Grid gr, const double* rho,
                                                const double* u, double u_in) {
  using St = Store<S>;
  using R = typename St::real;
  const int x = blockIdx.x * NT + threadIdx.x;
  if (x >= gr.nx) return;
  const long long cell = cell_of(gr, x, blockIdx.y, blockIdx.z);
  auto* A = static_cast<typename St::mem*>(fv);
  R dr = rho ? (R)(rho[cell] - 1.0) : R(0);
  Vec3<R> v{R(u_in), R(0), R(0)};
  if (u) {
    v.x = (R)u[cell];
    v.y = (R)u[gr.N + cell];
    v.z = Lat<Q>::D == 3 ? (R)u[2 * gr.N + cell] : R(0);
  }
  R g[Q];
  equilibrium_dev<Q, R>(g, dr, v);
#pragma unroll
  for (int i = 0; i < Q; ++i) St::st(A + (long long)i * gr.pitch + cell, g[i]);
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
                           bool odd, double u_in, const double* inflow, double* fout, double* rho,
                           double* u, cudaStream_t s) {
  dim3 grid((g.nx + NT - 1) / NT, g.ny, g.nz);
  if (odd) {
    HLBM_DISPATCH_QS(q, storage, (k_readout<Q_, S_, true><<<grid, NT, 0, s>>>(f, g, u_in, inflow, fout, rho, u)));
  } else {
    HLBM_DISPATCH_QS(q, storage, (k_readout<Q_, S_, false><<<grid, NT, 0, s>>>(f, g, u_in, inflow, fout, rho, u)));
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

// Sum of v[0..n) in a fixed order: block b sums the contiguous range
// [b chunk, (b+1) chunk) (thread-strided, then the block tree) into part[b];
// the last block to finish (atomic ticket, taken after the partial is written
// and fenced) adds the partials in block order and resets the ticket for the
// next call.  No block waits for another.  (One block for the whole sum took
// 195 us for the 640 000 per-warp objective slots of the LES grid, bound by
// that one SM's FP64 pipe.)
__global__ void __launch_bounds__(256) k_finalize_sum(const double* v, long long n, long long chunk,
                                                      double* part, unsigned* ticket, double* out) {
  __shared__ double sh[256 / 32];
  __shared__ bool last;
  const long long lo = (long long)blockIdx.x * chunk;
  const long long hi = lo + chunk < n ? lo + chunk : n;
  double acc = 0.0;
  for (long long k = lo + threadIdx.x; k < hi; k += blockDim.x) acc += v[k];
  const double t = block_sum<256>(acc, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = t;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last) {
    double a2 = 0.0;
    for (unsigned k = threadIdx.x; k < gridDim.x; k += blockDim.x)
      a2 += static_cast<volatile double*>(part)[k];
    const double r = block_sum<256>(a2, sh);
    if (threadIdx.x == 0) {
      *out = r;
      *ticket = 0u;
    }
  }
}

cudaError_t launch_finalize_sum(const double* v, long long n, double* out, double* scratch,
                                cudaStream_t s) {
  long long nb = (n + 4095) / 4096;
  if (nb < 1) nb = 1;
  if (nb > kFinBlocks) nb = kFinBlocks;
  const long long chunk = (n + nb - 1) / nb;
  k_finalize_sum<<<(unsigned)nb, 256, 0, s>>>(v, n, chunk, scratch,
                                               reinterpret_cast<unsigned*>(scratch + kFinBlocks), out);
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

// out[k][cell] = scale * sum_c coef[c][cell] b_c(xi_k)
template <int Q>
__global__ void k_expand_coef(const double* coef, int obj_slot, long long N, double scale,
                              double* out) {
  constexpr int D = Lat<Q>::D;
  const int nc = ncoef(obj_slot, D);
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    double cf[10];
    for (int k = 0; k < nc; ++k) cf[k] = coef[(long long)k * N + c];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      double v = 0.0;
      for (int k = 0; k < nc; ++k)
        v += cf[k] * coef_basis(obj_slot, D, k, Lat<Q>::cx(i), Lat<Q>::cy(i), Lat<Q>::cz(i));
      out[(long long)i * N + c] = scale * v;
    }
  }
}

struct ProjMat { double p[10 * 19]; };

template <int Q>
__global__ void k_project_coef(const double* gin, ProjMat P, int obj_slot, long long N,
                               double* coef) {
  constexpr int D = Lat<Q>::D;
  const int nc = ncoef(obj_slot, D);
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    double gv[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) gv[i] = gin[(long long)i * N + c];
    for (int k = 0; k < nc; ++k) {
      double v = 0.0;
#pragma unroll
      for (int i = 0; i < Q; ++i) v += P.p[k * Q + i] * gv[i];
      coef[(long long)k * N + c] = v;
    }
  }
}

// FROM_SUMS = false: fsum = f - w and msum = its moments (a set f_bar);
// FROM_SUMS = true: msum = the moments of the sums fsum (f is fsum itself)
template <int Q, bool FROM_SUMS>
__global__ void k_set_fbar(const double* f, long long N, double* fsum, double* msum, bool rr) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    double gv[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if constexpr (FROM_SUMS) {
        gv[i] = f[(long long)i * N + c];
      } else {
        gv[i] = f[(long long)i * N + c] - Lat<Q>::w(i);
        fsum[(long long)i * N + c] = gv[i];
      }
    }
    double dr, r;
    Vec3<double> m, u;
    moments_dev<Q, double>(gv, dr, r, m, u);
    msum[c] = dr;
    msum[N + c] = m.x;
    msum[2 * N + c] = m.y;
    if (Lat<Q>::D == 3) msum[3 * N + c] = m.z;
    if (rr) {
      const Sym<double> M2 = second_moment<Q, double>(gv);
      if (Lat<Q>::D == 2) {
        msum[3 * N + c] = M2.xx;
        msum[4 * N + c] = M2.yy;
        msum[5 * N + c] = M2.xy;
      } else {
        const double v[6] = {M2.xx, M2.yy, M2.zz, M2.xy, M2.xz, M2.yz};
        for (int k = 0; k < 6; ++k) msum[(4 + k) * N + c] = v[k];
      }
    }
  }
}

template <int Q>
__global__ void k_fbar_out(const double* fsum, long long N, double scale, double* out) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int i = 0; i < Q; ++i) out[(long long)i * N + c] = fsum[(long long)i * N + c] * scale + Lat<Q>::w(i);
  }
}

template <class R>
__global__ void k_fill(R* v, long long n, R value) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    v[k] = value;
}
cudaError_t launch_expand_coef(const double* coef, int obj_slot, int q, long long N, double scale,
                               double* out, cudaStream_t s) {
  if (q == 9) k_expand_coef<9><<<util_blocks(N), 256, 0, s>>>(coef, obj_slot, N, scale, out);
  else if (q == 19) k_expand_coef<19><<<util_blocks(N), 256, 0, s>>>(coef, obj_slot, N, scale, out);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_project_coef(const double* g, const double* Pmat, int obj_slot, int q,
                                long long N, double* coef, cudaStream_t s) {
  ProjMat P{};
  const int nc = ncoef(obj_slot, q == 9 ? 2 : 3);
  for (int k = 0; k < nc * q; ++k) P.p[k] = Pmat[k];
  if (q == 9) k_project_coef<9><<<util_blocks(N), 256, 0, s>>>(g, P, obj_slot, N, coef);
  else if (q == 19) k_project_coef<19><<<util_blocks(N), 256, 0, s>>>(g, P, obj_slot, N, coef);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_set_fbar(const double* f, int q, long long N, double* fsum, double* msum,
                            bool rr, cudaStream_t s) {
  if (q == 9) k_set_fbar<9, false><<<util_blocks(N), 256, 0, s>>>(f, N, fsum, msum, rr);
  else if (q == 19) k_set_fbar<19, false><<<util_blocks(N), 256, 0, s>>>(f, N, fsum, msum, rr);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_moments_of_sums(const double* fsum, int q, long long N, double* msum, bool rr,
                                   cudaStream_t s) {
  if (q == 9) k_set_fbar<9, true><<<util_blocks(N), 256, 0, s>>>(fsum, N, nullptr, msum, rr);
  else if (q == 19) k_set_fbar<19, true><<<util_blocks(N), 256, 0, s>>>(fsum, N, nullptr, msum, rr);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_fbar_out(const double* fsum, int q, long long N, double scale, double* out,
                            cudaStream_t s) {
  if (q == 9) k_fbar_out<9><<<util_blocks(N), 256, 0, s>>>(fsum, N, scale, out);
  else if (q == 19) k_fbar_out<19><<<util_blocks(N), 256, 0, s>>>(fsum, N, scale, out);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_fill_real(void* v, bool dbl, long long n, double value, cudaStream_t s) {
  if (dbl) k_fill<double><<<util_blocks(n), 256, 0, s>>>((double*)v, n, value);
  else k_fill<float><<<util_blocks(n), 256, 0, s>>>((float*)v, n, (float)value);
  return cudaGetLastError();
}

}  // namespace hlbm
