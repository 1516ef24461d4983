// Internal interface between the C ABI (hlbm_capi.cu) and the kernel
// translation units (hlbm_primal.cu, hlbm_adjoint.cu).  Not installed.
#pragma once

#include <cuda_runtime.h>

#include "hlbm_device.cuh"

namespace hlbm {

constexpr int NT = 128;  // threads per block along x for all cell kernels

// --------------------------------------------------------------------------
// primal
// --------------------------------------------------------------------------
struct PrimalArgs {
  void* f;            // population array (storage type), q planes of g.pitch
  const void* d;      // porosity, real type (double for FP64 storage, else float)
  Grid g;
  double tau0;        // molecular relaxation time
  double kles;        // (9 sqrt(2) / 2) Cs^2 ; 0 disables LES
  double u_in;        // inflow velocity
  double us[3];       // solid velocity u_s
  double nu0;         // molecular viscosity (tau0 - 1/2)/3
  float tau0_f, kles_f, u_in_f, us_f[3], nu0_f;  // the same in float for FP32 kernels
  // averaging (only read when the ACC variant runs)
  double* msum;       // (1 + D) x N running sums of rho - 1 and rho u (moments of f);
                      // RR adds D(D+1)/2 planes of sum xi xi (f - w): xx, yy[, zz], xy[, xz, yz]
  double* fsum;       // q x N running sum of f - w (only with the full-f variant, which
                      // then leaves msum alone)
  double* tsum;       // N running sum of tau_eff - tau0 (LES only)
  double* gsum[2];    // ncoef(obj) x N running sums of the coefficients of dJ/df
                      // in the basis of coef_basis() (FFA, DISS); may be null
  double* ddsum[2];   // N running sums of dJ/dd
  double* jblk[2];    // per-warp running sums of J (block linear index x warps per block + warp)
  // FP32 kernels add each sample to a float staging copy of every sum and fold
  // the staged value into the FP64 sum every kStage samples (flush variant),
  // so that the per-step path issues no FP64 instruction; FP64 kernels add to
  // the sums directly and leave these null.
  // A group of G staged sums is laid out as G / 4 float4 planes (sum k in
  // component k % 4 of plane k / 4) followed by G % 4 float planes, N cells
  // each.  Groups: the moment sums then tau_eff - tau0 (mstage, compact
  // averages) or the q sums of f - w then tau_eff - tau0 (fstage, full
  // averages: the moment sums are derived from them after the window); the
  // dissipation coefficients then dJ/dd (gstage[1]).
  float* mstage;
  float* fstage;
  float* gstage[2];   // [0]: FFA coefficients, plain planes; [1]: dissipation group
  float* ddstage[2];  // unused by the dissipation group
  int obj_mask;
  int ffa[5];         // x, y0, y1, z0, z1 of Gamma_J
  int db[6];          // Omega_J box
  unsigned* err;      // bit 0: non-finite or non-positive density
  const double* inflow;  // ny * nz values of u_x on the inflow column (y fastest), or null:
                         // uniform u_in
};

// Every objective's dJ/df_j is a polynomial of degree <= 2 in the lattice
// velocity xi_j: dJ/df_j = sum_k c_k b_k(xi_j) with the basis
//   FFA:  b = (1, x)                                  -> 2 coefficients
//   DISS: b = (1, x, y[, z], x^2, y^2[, z^2], 2xy[, 2xz, 2yz])  -> 6 (2D) / 10 (3D)
// Averaging the coefficients is averaging dJ/df (the map is linear).
__host__ __device__ constexpr int ncoef(int obj_slot, int D) {
  return obj_slot == 0 ? 2 : 1 + D + D * (D + 1) / 2;
}
__host__ __device__ inline double coef_basis(int obj_slot, int D, int k, int x, int y, int z) {
  if (obj_slot == 0) return k == 0 ? 1.0 : (double)x;
  if (k == 0) return 1.0;
  if (k <= D) return (double)(k == 1 ? x : (k == 2 ? y : z));
  k -= D + 1;
  if (k < D) return (double)(k == 0 ? x * x : (k == 1 ? y * y : z * z));
  k -= D;
  if (D == 2) return 2.0 * x * y;
  return 2.0 * (k == 0 ? x * y : (k == 1 ? x * z : y * z));
}

// averaging variant bits of the primal kernel
enum { ACC_ON = 1, ACC_FULL = 2, ACC_FLUSH = 4 };
// 64 measured fastest of 16 / 32 / 64 (averaging step: Karman 16.4 / 16.1 / 16.0 us,
// LES 2203 / 2096 / 2042 us); the staged value holds 64 FP32 samples at most
#ifndef HLBM_KSTAGE
#define HLBM_KSTAGE 64
#endif
constexpr int kStage = HLBM_KSTAGE;  // samples staged in FP32 before folding into FP64

// launch one primal step kernel; storage 0..3, odd/les select variants,
// acc: 0 no averaging, else ACC_ON | optional ACC_FULL (also average f) |
// optional ACC_FLUSH (fold the FP32 staging into the FP64 sums)
cudaError_t launch_primal(const PrimalArgs& a, int q, int storage, bool odd, bool les, int acc,
                          bool rr, cudaStream_t s);
// one step of several contexts in one launch (the serving form): tab holds each
// context's arguments on the device, tiles the (context, x-block, y, z) of every
// NT-wide block; FP32 storage, BGK without LES, acc 0, ACC_ON or ACC_ON | ACC_FLUSH
cudaError_t launch_primal_batch(const PrimalArgs* tab, const int4* tiles, int ntiles, int q,
                                bool odd, int acc, cudaStream_t s);
// out[k] (k < q, per cell) = scale * sum_c coef[c] b_c(xi_k): expand coefficient sums
cudaError_t launch_expand_coef(const double* coef, int obj_slot, int q, long long N, double scale,
                               double* out, cudaStream_t s);
// coef = P g with P (ncoef x q, row-major) the least-squares inverse of the basis
cudaError_t launch_project_coef(const double* g, const double* Pmat, int obj_slot, int q,
                                long long N, double* coef, cudaStream_t s);
// fsum = f - w and msum = (rho - 1, rho u) of the q x N field f (a set f_bar)
cudaError_t launch_set_fbar(const double* f, int q, long long N, double* fsum, double* msum,
                            bool rr, cudaStream_t s);
// msum = the moments (rho - 1, rho u[, xi xi (f - w) with rr]) of the q x N sums fsum
cudaError_t launch_moments_of_sums(const double* fsum, int q, long long N, double* msum, bool rr,
                                   cudaStream_t s);
// out = fsum * scale + w (readout of f_bar)
cudaError_t launch_fbar_out(const double* fsum, int q, long long N, double scale, double* out,
                            cudaStream_t s);

// readout of the canonical state: f (q x N), rho (N), u (3 x N); any may be null
cudaError_t launch_readout(const void* f, const void* d, const Grid& g, int q, int storage,
                           bool odd, double u_in, const double* inflow, double* fout, double* rho, double* u,
                           cudaStream_t s);
// write a canonical state (q x N doubles) in natural layout
cudaError_t launch_set_state(void* f, const Grid& g, int q, int storage, const double* in,
                             cudaStream_t s);
// f = f^eq(rho, u); rho / u may be null (1, u_in e_x)
cudaError_t launch_init_eq(void* f, const Grid& g, int q, int storage, const double* rho,
                           const double* u, double u_in, cudaStream_t s);
// d (real type) from doubles; sets err bit 1 when a value is outside [0, 1]
cudaError_t launch_set_porosity(void* d, bool dbl, const double* in, long long n,
                                unsigned* err, cudaStream_t s);
cudaError_t launch_convert_f32_to_f64(const float* in, double* out, long long n, cudaStream_t s);
cudaError_t launch_convert_f64_to_f32(const double* in, float* out, long long n, cudaStream_t s);
cudaError_t launch_real_to_f64(const void* in, bool dbl, double* out, long long n, cudaStream_t s);
// out = sum of v[0..n) in a fixed order (up to kFinBlocks blocks); scratch holds
// kFinBlocks partials and then a ticket word that must be zero at the first call
// (each call leaves it zero).  Calls sharing a scratch must not overlap.
constexpr int kFinBlocks = 296;
constexpr size_t kFinScratchBytes = (size_t)(kFinBlocks + 1) * 8;
cudaError_t launch_finalize_sum(const double* v, long long n, double* out, double* scratch,
                                cudaStream_t s);
cudaError_t launch_scale(double* v, long long n, double s_, cudaStream_t s);
cudaError_t launch_fill_real(void* v, bool dbl, long long n, double value, cudaStream_t s);

// --------------------------------------------------------------------------
// adjoint
// --------------------------------------------------------------------------
struct PrepArgs {
  const double* fsum;  // q x N sums of f - w (EXACT with LES)
  const double* msum;  // moment sums (see PrimalArgs::msum)
  const double* tsum;  // N (FTA with LES) or null
  double inv_n;        // 1 / number of samples
  void* rec;           // real planes: BGK/FTA (rho, ux, uy[, uz], omega); EXACT: q planes of
                       // f_bar - w; RR: (rho, ux, uy[, uz], omega, Pi xx, yy[, zz], xy[, xz, yz])
  long long rec_pitch;
  Grid g;
  double tau_b;        // tau0 or tau_adj
  int exact;           // 1: EXACT with LES (store f_bar), 0: compact record
  int rr;              // 1: recursive regularised collision (record with Pi)
  const void* d;       // porosity (real), RR only
  double us[3];        // solid velocity, RR only
};
cudaError_t launch_prep(const PrepArgs& a, int q, bool dbl, cudaStream_t s);

struct SourceArgs {
  const double* gsum;  // ncoef x N coefficient sums
  int obj_slot;        // 0 FFA, 1 DISS
  double inv_n;
  void* src;           // real, ncoef planes of box volume: the averaged coefficients
  int box[6];
  Grid g;
  double* red;         // per-block partial sums of src^2
};
cudaError_t launch_source(const SourceArgs& a, int q, bool dbl, int* nblocks, cudaStream_t s);

// The part of an adjoint sweep that belongs to its right-hand side (the
// fields of the same names in AdjointArgs), as the source and residual
// helpers of the sweep read it.
struct AdjRhs {
  void* lam;
  const void* src;
  int sb[6];
  long long src_pitch;
  int src_nc;
  void* snap;
  double* red;
};

struct AdjointArgs {
  void* lam;           // AA array of the adjoint (real), q planes of g.pitch
  Grid g;
  const void* d;       // porosity (real)
  const void* rec;     // linearisation record (see PrepArgs)
  long long rec_pitch;
  double tau_b, kles;
  double us[3];
  float tau_b_f, kles_f, us_f[3];
  const void* src;     // g_bar restricted to the source box (real): src_nc = 0: q planes of
                       // its values; src_nc > 0: the src_nc planes of its coefficients in the
                       // basis of coef_basis (the objective's derivative polynomial in xi)
  int sb[6];
  long long src_pitch;
  int src_nc;
  void* snap;          // residual snapshot (real, q planes of g.pitch)
  double* red;         // per-block partial of the residual
};
// res: 0 plain, 1 write the snapshot (even kernels), 2 compare (odd kernels)
cudaError_t launch_adjoint(const AdjointArgs& a, int q, bool dbl, bool odd, bool exact, int res,
                           bool rr, cudaStream_t s);
int adjoint_blocks(const Grid& g);
// one sweep of several contexts in one launch (see launch_primal_batch): FP32,
// compact linearisation record (BGK / frozen turbulence), res as launch_adjoint
cudaError_t launch_adjoint_batch(const AdjointArgs* tab, const int4* tiles, int ntiles, int q,
                                 bool odd, int res, cudaStream_t s);

// momentum-exchange drag: J(f_bar) per-block partials and surface-node counts
cudaError_t launch_mea_eval(const double* fsum, double inv_n, const void* d, const Grid& g, int q,
                            bool dbl, double* part_j, double* part_n, int* nblocks, cudaStream_t s);
// its constant dJ/df over the whole grid (src: q planes of N), ||.||^2 partials in red
cudaError_t launch_mea_source(const void* d, const Grid& g, int q, bool dbl, double inv_area,
                              void* src, double* red, int* nblocks, cudaStream_t s);

struct GradArgs {
  const void* lam;     // adjoint AA array in natural layout (next kernel even)
  Grid g;
  const void* d;
  const void* rec;
  long long rec_pitch;
  double tau_b, kles;
  double us[3];
  float tau_b_f, kles_f, us_f[3];
  const double* ddsum; // N, may be null
  double inv_n;
  int box[6];          // design box
  double* out;         // box volume, x fastest
  double* mu_out;      // optional q x N output of mu (whole grid when box is the domain)
};
cudaError_t launch_gradient(const GradArgs& a, int q, bool dbl, bool exact, bool rr, cudaStream_t s);

}  // namespace hlbm
