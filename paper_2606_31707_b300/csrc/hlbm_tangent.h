// Tangent-linear primal step (hlbm_tangent.cu).
#pragma once

#include <cuda_runtime.h>

#include "hlbm_device.cuh"

namespace hlbm {

// storage kind of the arithmetic type: the tangent is kept in full arithmetic precision
template <int S> struct RealKind { static constexpr int K = ST_F32; };
template <> struct RealKind<ST_F64> { static constexpr int K = ST_F64; };

struct TangentArgs {
  void* f;            // primal AA array (storage type)
  void* fd;           // tangent AA array (arithmetic type)
  const void* d;      // porosity (arithmetic type)
  const void* delta;  // porosity direction (arithmetic type)
  Grid g;
  double tau0, kles, u_in, us[3], nu0;
  float tau0_f, kles_f, u_in_f, us_f[3], nu0_f;
  int objective;      // 1 drag, 2 dissipation
  int ffa[5];
  int db[6];
  double* jpart;      // per-block partial sums of J' of this step
  const double* inflow;  // u_x on the inflow column (ny * nz), or null: uniform u_in
};

cudaError_t launch_tangent(const TangentArgs& a, int q, int storage, bool odd, bool les,
                           cudaStream_t s);

}  // namespace hlbm
