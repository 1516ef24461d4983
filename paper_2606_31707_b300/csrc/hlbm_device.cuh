// Device-side building blocks of the HLBM hot path: velocity sets, population
// storage formats, per-cell moments / porous equilibrium / Smagorinsky
// relaxation time, the AA-pattern addressing, and block reductions.
//
// Method (Ito et al., Sec. 2): BGK relaxation towards the porous equilibrium
//   f_i^eq(rho, u~) = w_i rho (1 + 3 xi_i.u~ + 9/2 (xi_i.u~)^2 - 3/2 u~.u~),
//   u~ = d u + (1 - d) u_s                                        (Sec. 2.1)
// with the local relaxation time of the Smagorinsky model (Sec. 2.2)
//   tau_eff = (nu0 + nu_t)/c_s^2 + 1/2,  nu_t = Cs^2 |S|,
//   S = -Pi/(2 tau_eff c_s^2),  |S| = sqrt(2 S:S),  Pi = sum xi xi (f - f^eq),
// which is a quadratic in tau_eff with the positive root
//   tau_eff = (tau0 + sqrt(tau0^2 + 18 sqrt(2) Cs^2 |Pi|)) / 2.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace hlbm {

// ----------------------------------------------------------------------------
// velocity sets.  Direction order of the library (exported through
// hlbm_velocity_set): rest first, then opposite pairs (2k+1, 2k+2).
// ----------------------------------------------------------------------------
template <int Q> struct Lat;

template <> struct Lat<9> {
  static constexpr int D = 2;
  __host__ __device__ static constexpr int cx(int i) {
    return (i == 1 || i == 5 || i == 7) ? 1 : (i == 2 || i == 6 || i == 8) ? -1 : 0;
  }
  __host__ __device__ static constexpr int cy(int i) {
    return (i == 3 || i == 5 || i == 8) ? 1 : (i == 4 || i == 6 || i == 7) ? -1 : 0;
  }
  __host__ __device__ static constexpr int cz(int) { return 0; }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  __host__ __device__ static constexpr int opp(int i) {
    return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
  }
};

template <> struct Lat<19> {
  static constexpr int D = 3;
  // 1,2: +-x  3,4: +-y  5,6: +-z
  // 7..10:  (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0)
  // 11..14: (1,0,1) (-1,0,-1) (1,0,-1) (-1,0,1)
  // 15..18: (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1)
  __host__ __device__ static constexpr int cx(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
           : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
  }
  __host__ __device__ static constexpr int cy(int i) {
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
           : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
  }
  __host__ __device__ static constexpr int cz(int i) {
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
           : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
  __host__ __device__ static constexpr int opp(int i) {
    return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
  }
};

// ----------------------------------------------------------------------------
// population storage formats (the precision form of the populations).  Every format
// stores the deviation g_i = f_i - w_i from the rest-state equilibrium, and all
// arithmetic works on deviations: they are O(Ma) small, so FP32 keeps ~2 more
// significant digits than it would on f_i ~ w_i, and the 16-bit formats need
// no shift.  The arithmetic type R is double for FP64 storage, else float.
// ----------------------------------------------------------------------------
enum StorageKind { ST_F64 = 0, ST_F32 = 1, ST_F16 = 2, ST_BF16 = 3 };

template <int S> struct Store;
template <> struct Store<ST_F64> {
  using mem = double; using real = double;
  static __device__ __forceinline__ real ld(const mem* p) { return *p; }
  static __device__ __forceinline__ void st(mem* p, real v) { *p = v; }
};
template <> struct Store<ST_F32> {
  using mem = float; using real = float;
  static __device__ __forceinline__ real ld(const mem* p) { return *p; }
  static __device__ __forceinline__ void st(mem* p, real v) { *p = v; }
};
template <> struct Store<ST_F16> {
  using mem = __half; using real = float;
  static __device__ __forceinline__ real ld(const mem* p) { return __half2float(*p); }
  static __device__ __forceinline__ void st(mem* p, real v) { *p = __float2half_rn(v); }
};
template <> struct Store<ST_BF16> {
  using mem = __nv_bfloat16; using real = float;
  static __device__ __forceinline__ real ld(const mem* p) { return __bfloat162float(*p); }
  static __device__ __forceinline__ void st(mem* p, real v) { *p = __float2bfloat16_rn(v); }
};

// scalar kernel parameters are passed in both precisions; FP32 kernels read the
// float copy so that no FP64 instruction is issued per cell
template <class R> __device__ __forceinline__ R par(double d, float f);
template <> __device__ __forceinline__ double par<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float par<float>(double, float f) { return f; }

template <class R> __device__ __forceinline__ R sqrt_r(R v);
template <> __device__ __forceinline__ double sqrt_r(double v) { return sqrt(v); }
template <> __device__ __forceinline__ float sqrt_r(float v) { return sqrtf(v); }

// ----------------------------------------------------------------------------
// grid geometry and the AA access pattern
//
// One array A holds q planes of `pitch` elements.  Canonical ("natural")
// layout: A[i][cell] = f_i(cell).  Even kernels read A[i][x] and write the
// relaxed value of direction i to A[opp(i)][x]; odd kernels read
// A[opp(i)][x - s xi_i] and write to A[i][x + s xi_i].  s = +1 streams
// along xi (primal), s = -1 against it (adjoint).  After an odd kernel the
// array is back in natural layout.  Every slot is read and written by the
// same thread in a kernel, so the update is in place without races.
// Targets outside 0 <= x < nx are skipped (boundary columns are recomputed
// by their owner threads); y and z wrap periodically.
// ----------------------------------------------------------------------------
struct Grid {
  int nx, ny, nz;
  long long N;      // cells
  long long pitch;  // plane stride (elements) of population arrays
  int bx;           // threads per block along x of the step kernels (32, 64 or 128)
};

__device__ __forceinline__ long long cell_of(const Grid& g, int x, int y, int z) {
  return (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z);
}

// Row bases (y + ny z) * nx of the 3 x 3 neighbouring rows of (y, z), with the
// periodic wrap resolved once per cell; the cell index of (x + dx, y + dy,
// z + dz) is row[dy + 1][dz + 1] + x + dx.  32-bit: grids have fewer than
// 2^31 cells (hlbm_create checks), which keeps the nine bases in nine
// registers instead of eighteen.
struct Rows {
  int r[3][3];
};

template <int D>
__device__ __forceinline__ Rows make_rows(const Grid& g, int y, int z) {
  Rows R;
  const int ym = y == 0 ? g.ny - 1 : y - 1;
  const int yp = y == g.ny - 1 ? 0 : y + 1;
  const int yy[3] = {ym, y, yp};
  if (D == 2) {
#pragma unroll
    for (int a = 0; a < 3; ++a) R.r[a][1] = yy[a] * g.nx;
  } else {
    const int zm = z == 0 ? g.nz - 1 : z - 1;
    const int zp = z == g.nz - 1 ? 0 : z + 1;
    const int zz[3] = {zm, z, zp};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        R.r[a][b] = (yy[a] + g.ny * zz[b]) * g.nx;
  }
  return R;
}

template <int Q, int S, bool ODD, int SIGN>
__device__ __forceinline__ void aa_load(const typename Store<S>::mem* A, const Grid& g,
                                        const Rows& rows, int x, long long cell,
                                        typename Store<S>::real (&f)[Q]) {
  using L = Lat<Q>;
  using St = Store<S>;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (!ODD) {
      f[i] = St::ld(A + (long long)i * g.pitch + cell);
    } else {
      // read A[opp(i)][x - s xi_i]
      const int dx = -SIGN * L::cx(i), dy = -SIGN * L::cy(i), dz = -SIGN * L::cz(i);
      const int xn = x + dx;
      const bool in = (dx == 0) || (xn >= 0 && xn < g.nx);
      const long long c = rows.r[dy + 1][dz + 1] + xn;
      f[i] = in ? St::ld(A + (long long)L::opp(i) * g.pitch + c) : typename St::real(0);
    }
  }
}

template <int Q, int S, bool ODD, int SIGN>
__device__ __forceinline__ void aa_store(typename Store<S>::mem* A, const Grid& g, const Rows& rows,
                                         int x, long long cell,
                                         const typename Store<S>::real (&f)[Q]) {
  using L = Lat<Q>;
  using St = Store<S>;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (!ODD) {
      St::st(A + (long long)L::opp(i) * g.pitch + cell, f[i]);
    } else {
      // write A[i][x + s xi_i]
      const int dx = SIGN * L::cx(i), dy = SIGN * L::cy(i), dz = SIGN * L::cz(i);
      const int xn = x + dx;
      const bool in = (dx == 0) || (xn >= 0 && xn < g.nx);
      const long long c = rows.r[dy + 1][dz + 1] + xn;
      if (in) St::st(A + (long long)i * g.pitch + c, f[i]);
    }
  }
}

// ----------------------------------------------------------------------------
// per-cell physics
// ----------------------------------------------------------------------------
template <class R> struct Vec3 { R x, y, z; };

// moments of a deviation field g_i = f_i - w_i: rho - 1 = sum g, rho u = sum xi g
// (the weights carry unit mass and zero momentum)
template <int Q, class R>
__device__ __forceinline__ void moments_dev(const R (&g)[Q], R& drho, R& rho, Vec3<R>& m,
                                            Vec3<R>& u) {
  using L = Lat<Q>;
  R r = 0, mx = 0, my = 0, mz = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    r += g[i];
    if (L::cx(i)) mx += L::cx(i) > 0 ? g[i] : -g[i];
    if (L::cy(i)) my += L::cy(i) > 0 ? g[i] : -g[i];
    if (L::cz(i)) mz += L::cz(i) > 0 ? g[i] : -g[i];
  }
  drho = r;
  rho = R(1) + r;
  m = Vec3<R>{mx, my, mz};
  const R inv = R(1) / rho;
  u = Vec3<R>{mx * inv, my * inv, mz * inv};
}

// moments of a full population field f (used by the no-context entry points)
template <int Q, class R>
__device__ __forceinline__ void moments(const R (&f)[Q], R& rho, Vec3<R>& u) {
  using L = Lat<Q>;
  R r = 0, mx = 0, my = 0, mz = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    r += f[i];
    if (L::cx(i)) mx += L::cx(i) > 0 ? f[i] : -f[i];
    if (L::cy(i)) my += L::cy(i) > 0 ? f[i] : -f[i];
    if (L::cz(i)) mz += L::cz(i) > 0 ? f[i] : -f[i];
  }
  rho = r;
  R inv = R(1) / r;
  u.x = mx * inv;
  u.y = my * inv;
  u.z = mz * inv;
}

// Per-direction sums below start at -0: -0 + x is x for every x, so the
// compiler drops the first addition (+0 + x is not x when x is -0).
template <int Q, class R>
__device__ __forceinline__ R xi_dot(int i, const Vec3<R>& v) {
  using L = Lat<Q>;
  R s = R(-0.0);
  if (L::cx(i)) s += L::cx(i) > 0 ? v.x : -v.x;
  if (L::cy(i)) s += L::cy(i) > 0 ? v.y : -v.y;
  if (L::cz(i)) s += L::cz(i) > 0 ? v.z : -v.z;
  return s;
}

// f_i^eq(rho, u) (Sec. 2.1)
template <int Q, class R>
__device__ __forceinline__ R feq_i(int i, R rho, const Vec3<R>& u, R uu) {
  R cu = xi_dot<Q>(i, u);
  return R(Lat<Q>::w(i)) * rho * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu);
}

// f_i^eq(rho, u) - w_i = w_i [(rho - 1) + rho (3 xi.u + 9/2 (xi.u)^2 - 3/2 u.u)]
template <int Q, class R>
__device__ __forceinline__ R geq_i(int i, R drho, R rho, const Vec3<R>& u, R uu) {
  R cu = xi_dot<Q>(i, u);
  return R(Lat<Q>::w(i)) * (drho + rho * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu));
}

// symmetric 3x3 tensor (xx, yy, zz, xy, xz, yz)
template <class R> struct Sym { R xx, yy, zz, xy, xz, yz; };

template <int Q, class R>
__device__ __forceinline__ Sym<R> second_moment(const R (&g)[Q]) {
  using L = Lat<Q>;
  Sym<R> P{0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int a = L::cx(i), b = L::cy(i), c = L::cz(i);
    if (a) P.xx += g[i];
    if (b) P.yy += g[i];
    if (c) P.zz += g[i];
    if (a && b) P.xy += (a * b > 0) ? g[i] : -g[i];
    if (a && c) P.xz += (a * c > 0) ? g[i] : -g[i];
    if (b && c) P.yz += (b * c > 0) ? g[i] : -g[i];
  }
  return P;
}

// S += v xi_i xi_i (one direction's contribution to a second moment)
template <int Q, class R>
__device__ __forceinline__ void sym_add_xixi(Sym<R>& S, int i, R v) {
  using L = Lat<Q>;
  const int a = L::cx(i), b = L::cy(i), c = L::cz(i);
  if (a) S.xx += v;
  if (b) S.yy += v;
  if (c) S.zz += v;
  if (a && b) S.xy += (a * b > 0) ? v : -v;
  if (a && c) S.xz += (a * c > 0) ? v : -v;
  if (b && c) S.yz += (b * c > 0) ? v : -v;
}

template <class R> __device__ __forceinline__ R sym_norm2(const Sym<R>& P) {
  return P.xx * P.xx + P.yy * P.yy + P.zz * P.zz +
         R(2) * (P.xy * P.xy + P.xz * P.xz + P.yz * P.yz);
}
template <class R> __device__ __forceinline__ Vec3<R> sym_mul(const Sym<R>& P, const Vec3<R>& v) {
  return Vec3<R>{P.xx * v.x + P.xy * v.y + P.xz * v.z, P.xy * v.x + P.yy * v.y + P.yz * v.z,
                 P.xz * v.x + P.yz * v.y + P.zz * v.z};
}
template <class R> __device__ __forceinline__ R dot3(const Vec3<R>& a, const Vec3<R>& b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}
// xi_i . P . xi_i
template <int Q, class R> __device__ __forceinline__ R xi_P_xi(int i, const Sym<R>& P) {
  using L = Lat<Q>;
  const int a = L::cx(i), b = L::cy(i), c = L::cz(i);
  R s = R(-0.0);
  if (a) s += P.xx;
  if (b) s += P.yy;
  if (c) s += P.zz;
  if (a && b) s += (a * b > 0) ? R(2) * P.xy : -R(2) * P.xy;
  if (a && c) s += (a * c > 0) ? R(2) * P.xz : -R(2) * P.xz;
  if (b && c) s += (b * c > 0) ? R(2) * P.yz : -R(2) * P.yz;
  return s;
}

// Moments m0 = sum v, m1 = sum v xi, m2 = sum v xi xi of a per-direction field
// over one weight class of the lattice: the axis directions (|xi|^2 = 1) or the
// diagonal ones (|xi|^2 = 2).  Both lattices list opposite directions as pairs
// (2k+1, 2k+2), so the sums run over pairs: with s = v_i + v_opp and
// t = v_i - v_opp a pair adds s to m0 and m2 and xi_i t to m1.  Weighted moments
// (sum w v ...) are w_axis times the axis class plus w_diag times the diagonal
// class, plus w_0 v_0 in m0.
template <class R> struct Mom { R m0; Vec3<R> m1; Sym<R> m2; };

template <int Q> __host__ __device__ constexpr bool axis_dir(int i) {
  return (Lat<Q>::cx(i) != 0) + (Lat<Q>::cy(i) != 0) + (Lat<Q>::cz(i) != 0) == 1;
}
template <int Q> __host__ __device__ constexpr bool weight_classes_hold() {
  for (int i = 1; i < Q; ++i) {
    if (Lat<Q>::opp(i) != ((i & 1) ? i + 1 : i - 1)) return false;
    if (Lat<Q>::w(i) != (axis_dir<Q>(i) ? Lat<Q>::w(1) : Lat<Q>::w(Q - 1))) return false;
  }
  return true;
}
static_assert(weight_classes_hold<9>() && weight_classes_hold<19>(),
              "direction order: rest, then opposite pairs; one weight per class");

template <int Q, class R>
__device__ __forceinline__ void pair_add(Mom<R>& m, int i, R s, R t) {
  using L = Lat<Q>;
  const int a = L::cx(i), b = L::cy(i), c = L::cz(i);
  m.m0 += s;
  if (a) m.m1.x += a > 0 ? t : -t;
  if (b) m.m1.y += b > 0 ? t : -t;
  if (c) m.m1.z += c > 0 ? t : -t;
  if (a) m.m2.xx += s;
  if (b) m.m2.yy += s;
  if (c) m.m2.zz += s;
  if (a && b) m.m2.xy += (a * b > 0) ? s : -s;
  if (a && c) m.m2.xz += (a * c > 0) ? s : -s;
  if (b && c) m.m2.yz += (b * c > 0) ? s : -s;
}

template <int Q, class R>
__device__ __forceinline__ void class_moments(const R (&v)[Q], Mom<R>& ax, Mom<R>& dg) {
  const R z = R(-0.0);
  ax = Mom<R>{z, {z, z, z}, {z, z, z, z, z, z}};
  dg = ax;
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const R s = v[i] + v[i + 1], t = v[i] - v[i + 1];
    if (axis_dir<Q>(i)) pair_add<Q, R>(ax, i, s, t);
    else pair_add<Q, R>(dg, i, s, t);
  }
}

// positive root of tau^2 - tb tau - kles |Pi| = 0, kles = (9 sqrt 2 / 2) Cs^2
template <class R> __device__ __forceinline__ R tau_smagorinsky(R tb, R kles, R normPi) {
  return R(0.5) * (tb + sqrt_r<R>(tb * tb + R(4) * kles * normPi));
}

// ----------------------------------------------------------------------------
// reductions (FP64): warp shuffle, then shared memory across warps
// ----------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block sum over blockDim.x <= NT threads (valid in thread 0)
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0;
  if (threadIdx.x == 0) {
    const int nw = (int)(blockDim.x >> 5);
    for (int k = 0; k < nw; ++k) r += sh[k];
  }
  __syncthreads();
  return r;
}

// ----------------------------------------------------------------------------
// Asynchronous global -> shared copies (cp.async): the data in flight holds no
// registers; a thread that reads back only its own slots needs no barrier
// after cp.async.wait_all.
// ----------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(smem)), "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// ----------------------------------------------------------------------------
// Double-float sums for the FP32 kernels.  B300's FP64 pipe runs at a small
// fraction of its FP32 rate, so the FP32 kernels add their per-cell objective
// terms as an unevaluated pair hi + lo of floats with Knuth's error-free
// TwoSum (s + e == a + b exactly in round-to-nearest), which carries about
// twice the float precision, and convert to FP64 once per warp.
// ----------------------------------------------------------------------------
struct F2 {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// x += v (double-float)
__device__ __forceinline__ void jadd(F2& x, float v) {
  float s, e;
  two_sum(x.hi, v, s, e);
  x.hi = s;
  x.lo += e;
}
__device__ __forceinline__ void jadd(double& x, double v) { x += v; }

// block sum of per-thread double-float values, in FP64 across warps (valid in thread 0)
template <int NT>
__device__ __forceinline__ double block_sum(F2 v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h = __shfl_xor_sync(0xffffffffu, v.hi, o);
    const float l = __shfl_xor_sync(0xffffffffu, v.lo, o);
    float s, e;
    two_sum(v.hi, h, s, e);
    v.hi = s;
    v.lo = v.lo + l + e;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = (double)v.hi + (double)v.lo;
  __syncthreads();
  double r = 0;
  if (threadIdx.x == 0) {
    const int nw = (int)(blockDim.x >> 5);
    for (int k = 0; k < nw; ++k) r += sh[k];
  }
  __syncthreads();
  return r;
}

// warp sums of the objective accumulators as FP64 (valid in every lane)
__device__ __forceinline__ double warp_sum_j(double v) { return warp_sum(v); }
__device__ __forceinline__ double warp_sum_j(F2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h = __shfl_xor_sync(0xffffffffu, v.hi, o);
    const float l = __shfl_xor_sync(0xffffffffu, v.lo, o);
    float s, e;
    two_sum(v.hi, h, s, e);
    v.hi = s;
    v.lo = v.lo + l + e;
  }
  return (double)v.hi + (double)v.lo;
}

// the objective accumulator of an arithmetic type: FP64 itself, or a double-float pair
template <class R> struct JAcc { using T = F2; };
template <> struct JAcc<double> { using T = double; };

__device__ __forceinline__ long long block_linear() {
  return (long long)blockIdx.x + (long long)gridDim.x * ((long long)blockIdx.y + (long long)gridDim.y * blockIdx.z);
}

}  // namespace hlbm
