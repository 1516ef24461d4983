// C ABI of the HLBM mean-flow adjoint hot path (see include/hlbm.h).
//
// Host-side orchestration only: argument checks, device memory, the order of
// kernel launches that realises Algorithm 1 of Ito et al. (primal with
// tracking averages -> linearisation -> adjoint iteration -> gradient), and
// copies in and out.  Every arithmetic step of the method runs in the
// kernels of hlbm_primal.cu and hlbm_adjoint.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <utility>
#include <vector>
#include <algorithm>
#include <string>

#include "../../include/hlbm.h"
#include "hlbm_internal.h"
#include "hlbm_krylov.h"
#include "hlbm_tangent.h"

using namespace hlbm;

struct hlbm_ctx {
  int q = 9, D = 2, storage = HLBM_FP32;
  Grid g{};
  double tau0 = 0.6, Cs = 0, kles = 0, nu0 = 0;
  hlbm_options opt{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  // primal state
  void* f = nullptr;
  void* d = nullptr;
  double* inflow = nullptr;  // u_x on the inflow column (ny * nz), or null: uniform u_in
  int phase = 0;  // 0: natural layout, next primal kernel is even
  long steps_done = 0;
  // averages
  bool rr = false;          // recursive regularised collision (Sec. 2.2)
  int mplanes = 3;          // planes of msum: 1 + D, + D(D+1)/2 with rr
  double* msum = nullptr;   // mplanes x N sums of rho - 1, rho u[, xi xi (f - w)]
  double* fsum = nullptr;   // q x N sums of f (full_f only, or set by the caller)
  bool full_f = false;
  double pmat[2][10 * 19] = {};  // least-squares inverse of the dJ/df coefficient basis
  double* tsum = nullptr;
  double* gsum[2] = {nullptr, nullptr};
  double* ddsum[2] = {nullptr, nullptr};
  double* jblk[2] = {nullptr, nullptr};
  float* mstage = nullptr;  // FP32 staging of the sums (FP32 / 16-bit storage only)
  float* fstage = nullptr;
  float* gstage[2] = {nullptr, nullptr};
  float* ddstage[2] = {nullptr, nullptr};
  long long nblk = 0;
  long long njslot = 0;  // per-warp slots of the objective sums (nblk x warps per block)
  long nsamples = 0;
  int acc_mask = 0;
  long generation = 0;  // bumps whenever the averaged state changes
  // adjoint
  void* lam = nullptr;
  void* snap = nullptr;
  void* rec = nullptr;
  size_t rec_bytes = 0;
  void* src = nullptr;
  size_t src_bytes = 0;
  double* red = nullptr;
  long long red_n = 0;
  void* fd = nullptr;         // tangent state (AA array of the arithmetic type)
  void* delta = nullptr;      // porosity direction of the tangent
  double* jhist = nullptr;    // per-step J' of the last tangent run
  long jhist_n = 0;
  void* kry = nullptr;        // GMRES vectors: basis (restart + 1), w, x, c
  size_t kry_bytes = 0;
  double* kpart = nullptr;    // multi-dot partial sums
  double* kdev = nullptr;     // device copies of the Arnoldi coefficients
  double* khost = nullptr;    // pinned host copies
  int rec_mode = -1;
  double rec_taub = 0;
  long rec_generation = -1;
  int last_obj = 0;
  int src_obj = 0;  // objective whose g_bar the source buffer holds
  int last_mode = 0;
  bool have_adjoint = false;
  bool lam_set = false;  // the adjoint array holds a solve's result (warm start)
  // scalars
  unsigned* err_dev = nullptr;
  unsigned* err_host = nullptr;
  double* scal_dev = nullptr;
  double* fin = nullptr;     // partials and ticket of launch_finalize_sum
  double* scal_host = nullptr;
  // staging
  double* stage = nullptr;
  size_t stage_bytes = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // captured CUDA graphs of kGraphSteps consecutive primal steps, one per
  // (averaging variant, phase of the first step)
  struct PrimalGraph {
    cudaGraphExec_t exec = nullptr;
    PrimalArgs args{};
  } pgraph[2][2];  // [plain, averaging pattern][phase]
  // captured adjoint chunk: check_every iterations, the residual reduction
  // and its copy to pinned host memory
  struct AdjointGraph {
    cudaGraphExec_t exec = nullptr;
    AdjointArgs args{};
    long chunk = 0;
    bool exact = false;
  } agraph;
  bool graphs_ok = true;
  hlbm_stats stats{};
  std::string msg;
};

namespace {

// count a kernel launch of context c, then call the launcher
#define CNT(c, fn) ((c)->stats.kernels_total++, fn)

int set_err(hlbm_ctx* c, int code, const char* fmt, const char* extra = nullptr) {
  if (c) {
    char buf[512];
    std::snprintf(buf, sizeof buf, fmt, extra ? extra : "");
    c->msg = buf;
  }
  return code;
}

int cuda_check(hlbm_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return HLBM_OK;
  char buf[512];
  std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  if (c) c->msg = buf;
  return e == cudaErrorMemoryAllocation ? HLBM_ENOMEM : HLBM_ECUDA;
}

#define HLBM_TRY(c, expr, what)                          \
  do {                                                   \
    int rc__ = cuda_check((c), (expr), (what));          \
    if (rc__ != HLBM_OK) return rc__;                    \
  } while (0)

void* dalloc(hlbm_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (c->opt.dev_alloc) {
    p = c->opt.dev_alloc(bytes, c->opt.alloc_user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  return p;
}

void dfree(hlbm_ctx* c, void* p) {
  if (!p) return;
  if (c->opt.dev_free) c->opt.dev_free(p, c->opt.alloc_user);
  else cudaFree(p);
}

size_t pop_elem_bytes(int storage) {
  switch (storage) {
    case HLBM_FP64: return 8;
    case HLBM_FP32: return 4;
    default: return 2;
  }
}
bool real_is_double(const hlbm_ctx* c) { return c->storage == HLBM_FP64; }
size_t real_bytes(const hlbm_ctx* c) { return real_is_double(c) ? 8 : 4; }

int ensure_stage(hlbm_ctx* c, size_t bytes) {
  if (c->stage_bytes >= bytes) return HLBM_OK;
  dfree(c, c->stage);
  c->stage = static_cast<double*>(dalloc(c, bytes));
  c->stage_bytes = c->stage ? bytes : 0;
  return c->stage ? HLBM_OK : set_err(c, HLBM_ENOMEM, "staging allocation failed");
}

// caller data (dtype, host/device) -> c->stage as doubles (n values)
int stage_in(hlbm_ctx* c, const void* data, int dtype, int on_device, long long n) {
  if (dtype != HLBM_DTYPE_F64 && dtype != HLBM_DTYPE_F32) return set_err(c, HLBM_EINVAL, "bad dtype");
  int rc = ensure_stage(c, (size_t)n * 8 * (dtype == HLBM_DTYPE_F32 ? 2 : 1));
  if (rc) return rc;
  if (dtype == HLBM_DTYPE_F64) {
    HLBM_TRY(c, cudaMemcpyAsync(c->stage, data, (size_t)n * 8,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                c->stream), "copy in");
  } else {
    float* tmp = reinterpret_cast<float*>(c->stage + n);
    HLBM_TRY(c, cudaMemcpyAsync(tmp, data, (size_t)n * 4,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                c->stream), "copy in");
    HLBM_TRY(c, CNT(c, launch_convert_f32_to_f64)(tmp, c->stage, n, c->stream), "convert");
  }
  return HLBM_OK;
}

// c->stage (n doubles) -> caller buffer
int stage_out(hlbm_ctx* c, void* out, int dtype, int on_device, long long n) {
  if (dtype == HLBM_DTYPE_F64) {
    HLBM_TRY(c, cudaMemcpyAsync(out, c->stage, (size_t)n * 8,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                c->stream), "copy out");
  } else if (dtype == HLBM_DTYPE_F32) {
    int rc = ensure_stage(c, (size_t)n * 12);
    if (rc) return rc;
    float* tmp = reinterpret_cast<float*>(c->stage + n);
    HLBM_TRY(c, CNT(c, launch_convert_f64_to_f32)(c->stage, tmp, n, c->stream), "convert");
    HLBM_TRY(c, cudaMemcpyAsync(out, tmp, (size_t)n * 4,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                c->stream), "copy out");
  } else {
    return set_err(c, HLBM_EINVAL, "bad dtype");
  }
  HLBM_TRY(c, cudaStreamSynchronize(c->stream), "sync");
  return HLBM_OK;
}

int check_box(const hlbm_ctx* c, const int b[6]) {
  return b[0] >= 0 && b[1] <= c->g.nx && b[0] < b[1] && b[2] >= 0 && b[3] <= c->g.ny &&
         b[2] < b[3] && b[4] >= 0 && b[5] <= c->g.nz && b[4] < b[5];
}

void objective_box(const hlbm_ctx* c, int obj, int box[6]) {
  if (obj == HLBM_OBJ_DRAG_MEA) {
    const int b[6] = {0, c->g.nx, 0, c->g.ny, 0, c->g.nz};
    std::memcpy(box, b, sizeof b);
  } else if (obj == HLBM_OBJ_DRAG_FFA) {
    box[0] = c->opt.ffa_x; box[1] = c->opt.ffa_x + 1;
    box[2] = c->opt.ffa_y0; box[3] = c->opt.ffa_y1;
    box[4] = c->opt.ffa_z0; box[5] = c->opt.ffa_z1;
  } else {
    std::memcpy(box, c->opt.diss_box, sizeof(int) * 6);
  }
}

int obj_slot(int obj) {
  return obj == HLBM_OBJ_DRAG_FFA ? 0
         : obj == HLBM_OBJ_DISSIPATION ? 1
         : obj == HLBM_OBJ_DRAG_MEA ? 2 : -1;
}

size_t coef_bytes(const hlbm_ctx* c, int o) { return (size_t)ncoef(o, c->D) * c->g.N * 8; }

// FP32 staging, one float per sum and cell, each group laid out as float4
// planes then float planes: the moment sums and tau_eff - tau0 (compact
// averages), or the q sums of f - w and tau_eff - tau0 (full averages); the
// drag coefficients; the dissipation coefficients and dJ/dd
size_t mstage_bytes(const hlbm_ctx* c) { return (size_t)(c->mplanes + 1) * c->g.N * 4; }
size_t fstage_bytes(const hlbm_ctx* c) { return (size_t)(c->q + 1) * c->g.N * 4; }
size_t gstage_bytes(const hlbm_ctx* c, int o) {
  return (size_t)(o == 0 ? ncoef(0, c->D) : ncoef(1, c->D) + 1) * c->g.N * 4;
}

int ensure_averages(hlbm_ctx* c, int mask) {
  const long long N = c->g.N;
  const size_t qN = (size_t)c->q * N * 8;
  if (!c->msum && !(c->msum = (double*)dalloc(c, (size_t)c->mplanes * N * 8)))
    return set_err(c, HLBM_ENOMEM, "msum");
  if (c->full_f && !c->fsum && !(c->fsum = (double*)dalloc(c, qN))) return set_err(c, HLBM_ENOMEM, "fsum");
  if (!c->tsum && !(c->tsum = (double*)dalloc(c, (size_t)N * 8))) return set_err(c, HLBM_ENOMEM, "tsum");
  const bool stage = !real_is_double(c);
  if (stage) {
    if (!c->full_f && !c->mstage && !(c->mstage = (float*)dalloc(c, mstage_bytes(c))))
      return set_err(c, HLBM_ENOMEM, "mstage");
    if (c->full_f && !c->fstage && !(c->fstage = (float*)dalloc(c, fstage_bytes(c))))
      return set_err(c, HLBM_ENOMEM, "fstage");
  }
  for (int o = 0; o < 2; ++o) {
    if (!(mask & (1 << o))) continue;
    if (stage && !c->gstage[o] && !(c->gstage[o] = (float*)dalloc(c, gstage_bytes(c, o)))) return set_err(c, HLBM_ENOMEM, "gstage");
    if (!c->gsum[o] && !(c->gsum[o] = (double*)dalloc(c, coef_bytes(c, o)))) return set_err(c, HLBM_ENOMEM, "gsum");
    if (!c->ddsum[o] && !(c->ddsum[o] = (double*)dalloc(c, (size_t)N * 8))) return set_err(c, HLBM_ENOMEM, "ddsum");
    if (!c->jblk[o] && !(c->jblk[o] = (double*)dalloc(c, (size_t)c->njslot * 8))) return set_err(c, HLBM_ENOMEM, "jblk");
  }
  return HLBM_OK;
}

int reset_averages(hlbm_ctx* c, int mask) {
  int rc = ensure_averages(c, mask);
  if (rc) return rc;
  const long long N = c->g.N;
  HLBM_TRY(c, cudaMemsetAsync(c->msum, 0, (size_t)c->mplanes * N * 8, c->stream), "memset");
  if (c->fsum) HLBM_TRY(c, cudaMemsetAsync(c->fsum, 0, (size_t)c->q * N * 8, c->stream), "memset");
  HLBM_TRY(c, cudaMemsetAsync(c->tsum, 0, (size_t)N * 8, c->stream), "memset");
  if (c->mstage) HLBM_TRY(c, cudaMemsetAsync(c->mstage, 0, mstage_bytes(c), c->stream), "memset");
  if (c->fstage) HLBM_TRY(c, cudaMemsetAsync(c->fstage, 0, fstage_bytes(c), c->stream), "memset");
  for (int o = 0; o < 2; ++o) {
    if (!(mask & (1 << o))) continue;
    if (c->gstage[o]) HLBM_TRY(c, cudaMemsetAsync(c->gstage[o], 0, gstage_bytes(c, o), c->stream), "memset");
    HLBM_TRY(c, cudaMemsetAsync(c->gsum[o], 0, coef_bytes(c, o), c->stream), "memset");
    HLBM_TRY(c, cudaMemsetAsync(c->ddsum[o], 0, (size_t)N * 8, c->stream), "memset");
    HLBM_TRY(c, cudaMemsetAsync(c->jblk[o], 0, (size_t)c->njslot * 8, c->stream), "memset");
  }
  c->nsamples = 0;
  c->acc_mask = mask;
  c->generation++;
  return HLBM_OK;
}

int read_err(hlbm_ctx* c, unsigned* out) {
  HLBM_TRY(c, cudaMemcpyAsync(c->err_host, c->err_dev, sizeof(unsigned), cudaMemcpyDeviceToHost,
                              c->stream), "err readback");
  HLBM_TRY(c, cudaStreamSynchronize(c->stream), "sync");
  *out = *c->err_host;
  HLBM_TRY(c, cudaMemsetAsync(c->err_dev, 0, sizeof(unsigned), c->stream), "memset");
  return HLBM_OK;
}

PrimalArgs primal_args(hlbm_ctx* c) {
  PrimalArgs a{};
  a.f = c->f;
  a.d = c->d;
  a.g = c->g;
  a.tau0 = c->tau0;
  a.kles = c->kles;
  a.u_in = c->opt.u_in;
  for (int k = 0; k < 3; ++k) a.us[k] = c->opt.u_solid[k];
  a.nu0 = c->nu0;
  a.tau0_f = (float)a.tau0;
  a.kles_f = (float)a.kles;
  a.u_in_f = (float)a.u_in;
  for (int k = 0; k < 3; ++k) a.us_f[k] = (float)a.us[k];
  a.nu0_f = (float)a.nu0;
  a.msum = c->msum;
  a.fsum = c->fsum;
  a.tsum = c->tsum;
  for (int o = 0; o < 2; ++o) {
    a.gsum[o] = c->gsum[o];
    a.ddsum[o] = c->ddsum[o];
    a.jblk[o] = c->jblk[o];
    a.gstage[o] = c->gstage[o];
    a.ddstage[o] = c->ddstage[o];
  }
  a.mstage = c->mstage;
  a.fstage = c->fstage;
  a.obj_mask = c->acc_mask;
  a.ffa[0] = c->opt.ffa_x;
  a.ffa[1] = c->opt.ffa_y0;
  a.ffa[2] = c->opt.ffa_y1;
  a.ffa[3] = c->opt.ffa_z0;
  a.ffa[4] = c->opt.ffa_z1;
  std::memcpy(a.db, c->opt.diss_box, sizeof a.db);
  a.err = c->err_dev;
  a.inflow = c->inflow;
  return a;
}

double bytes_plain(const hlbm_ctx* c) {
  return 2.0 * c->q * pop_elem_bytes(c->storage) + real_bytes(c);
}

}  // namespace

extern "C" {

int hlbm_velocity_set(int lattice, int* xi, double* w) {
  if (lattice == 9) {
    for (int i = 0; i < 9; ++i) {
      if (xi) { xi[3 * i] = Lat<9>::cx(i); xi[3 * i + 1] = Lat<9>::cy(i); xi[3 * i + 2] = 0; }
      if (w) w[i] = Lat<9>::w(i);
    }
    return 9;
  }
  if (lattice == 19) {
    for (int i = 0; i < 19; ++i) {
      if (xi) { xi[3 * i] = Lat<19>::cx(i); xi[3 * i + 1] = Lat<19>::cy(i); xi[3 * i + 2] = Lat<19>::cz(i); }
      if (w) w[i] = Lat<19>::w(i);
    }
    return 19;
  }
  return HLBM_EINVAL;
}

// Copy a caller's inflow profile (u_x on the inflow column, ny * nz values,
// y fastest) to the device; null restores the uniform inflow u_in.
static int check_inflow(hlbm_ctx* c, const double* host) {
  const long long n = (long long)c->g.ny * c->g.nz;
  for (long long k = 0; k < n; ++k)
    if (!std::isfinite(host[k]) || std::fabs(host[k]) >= 0.5)
      return set_err(c, HLBM_EINVAL, "inflow profile: |u_x| < 0.5 and finite");
  return HLBM_OK;
}

// u_in (the inflow and J_FFA reference velocity) and tau_adj (0: tau0, else
// the adjoint relaxation time, which like tau must exceed 1/2)
static bool options_valid(const hlbm_options* o) {
  if (!std::isfinite(o->u_in) || std::fabs(o->u_in) >= 0.5) return false;
  if (!std::isfinite(o->tau_adj) || !(o->tau_adj == 0.0 || o->tau_adj > 0.5)) return false;
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(o->u_solid[k]) || std::fabs(o->u_solid[k]) >= 0.5) return false;
  return true;
}

static int set_inflow(hlbm_ctx* c, const double* host) {
  if (!host) {
    if (c->inflow) dfree(c, c->inflow);
    c->inflow = nullptr;
    return HLBM_OK;
  }
  const long long n = (long long)c->g.ny * c->g.nz;
  int rc = check_inflow(c, host);
  if (rc) return rc;
  if (!c->inflow && !(c->inflow = (double*)dalloc(c, (size_t)n * 8)))
    return set_err(c, HLBM_ENOMEM, "inflow profile");
  HLBM_TRY(c, cudaMemcpyAsync(c->inflow, host, (size_t)n * 8, cudaMemcpyHostToDevice, c->stream), "copy");
  HLBM_TRY(c, cudaStreamSynchronize(c->stream), "sync");
  return HLBM_OK;
}

void hlbm_default_options(hlbm_options* o, const int dims[3]) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->storage = HLBM_FP32;
  o->u_in = 0.05;
  o->objectives = HLBM_OBJ_DRAG_FFA | HLBM_OBJ_DISSIPATION;
  int nx = dims ? dims[0] : 1, ny = dims ? dims[1] : 1, nz = dims ? dims[2] : 1;
  o->ffa_x = nx / 2;
  o->ffa_y0 = 0; o->ffa_y1 = ny;
  o->ffa_z0 = 0; o->ffa_z1 = nz;
  int box[6] = {0, nx, 0, ny, 0, nz};
  std::memcpy(o->diss_box, box, sizeof box);
  std::memcpy(o->design_box, box, sizeof box);
  o->accum_stride = 1;
  o->check_every = 100;
  o->gmres_restart = 30;
  o->gmres_inner = 100;
}

int hlbm_create(hlbm_ctx** out, int lattice, const int dims[3], double tau, double Cs,
                const hlbm_options* opt) {
  if (!out) return HLBM_EINVAL;
  *out = nullptr;
  if ((lattice != 9 && lattice != 19) || !dims) return HLBM_EINVAL;
  if (dims[0] < 4 || dims[1] < 1 || dims[2] < 1) return HLBM_EINVAL;
  if (lattice == 9 && dims[2] != 1) return HLBM_EINVAL;
  if (dims[1] > 65535 || dims[2] > 65535) return HLBM_EINVAL;
  // cell indices (and the padded plane pitch) are held in 32 bits in the kernels
  if ((long long)dims[0] * dims[1] * dims[2] + 64 > 2147483647LL) return HLBM_EINVAL;
  if (!(tau > 0.5) || !(Cs >= 0.0) || !std::isfinite(tau) || !std::isfinite(Cs)) return HLBM_EINVAL;
  hlbm_ctx* c = new hlbm_ctx();
  if (opt) c->opt = *opt;
  else hlbm_default_options(&c->opt, dims);
  if (c->opt.storage < HLBM_FP64 || c->opt.storage > HLBM_BF16DEV) { delete c; return HLBM_EINVAL; }
  if (!options_valid(&c->opt)) { delete c; return HLBM_EINVAL; }
  if (c->opt.accum_stride < 1) c->opt.accum_stride = 1;
  if (c->opt.check_every < 2) c->opt.check_every = 100;
  if (c->opt.check_every & 1) c->opt.check_every += 1;
  c->q = lattice;
  c->D = lattice == 9 ? 2 : 3;
  c->storage = c->opt.storage;
  c->g.nx = dims[0]; c->g.ny = dims[1]; c->g.nz = dims[2];
  c->g.N = (long long)dims[0] * dims[1] * dims[2];
  c->g.pitch = (c->g.N + 63) / 64 * 64;
  c->tau0 = tau;
  c->Cs = Cs;
  c->kles = 4.5 * std::sqrt(2.0) * Cs * Cs;
  c->nu0 = (tau - 0.5) / 3.0;
  // threads per block along x of the step kernels: the widest of 128 / 64 / 32
  // that still gives enough blocks to fill the GPU (small grids get narrower
  // blocks so that every SM has warps to switch between)
  {
    int bx = c->opt.block_x;
    if (bx != 32 && bx != 64 && bx != 128) {
      int sms = 148, dev = 0;
      if (cudaGetDevice(&dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        sms = 148;
      }
      bx = 32;
      for (int cand : {128, 64}) {
        const long long blocks = (long long)((dims[0] + cand - 1) / cand) * dims[1] * dims[2];
        if (blocks >= 16LL * sms) { bx = cand; break; }
      }
    }
    c->g.bx = bx;
  }
  c->nblk = (long long)((dims[0] + c->g.bx - 1) / c->g.bx) * dims[1] * dims[2];
  c->njslot = c->nblk * (c->g.bx / 32);
  if (c->opt.collision != HLBM_COLL_BGK && c->opt.collision != HLBM_COLL_RR) { delete c; return HLBM_EINVAL; }
  c->rr = c->opt.collision == HLBM_COLL_RR;
  c->mplanes = 1 + c->D + (c->rr ? c->D * (c->D + 1) / 2 : 0);
  // the exact LES linearisation of BGK and J_MEA (linear in f: J_bar = J(f_bar))
  // need f_bar; the regularised collision reads only moments up to order 2
  c->full_f = c->opt.average_full_f != 0 || (Cs > 0.0 && !c->rr) ||
              (c->opt.objectives & HLBM_OBJ_DRAG_MEA);
  // least-squares inverse P = (V^T V)^-1 V^T of the coefficient basis V (q x nc)
  for (int o = 0; o < 2; ++o) {
    const int nc = ncoef(o, c->D), q = c->q;
    double V[19][10], M[10][20];
    for (int i = 0; i < q; ++i) {
      const int x = lattice == 9 ? Lat<9>::cx(i) : Lat<19>::cx(i);
      const int y = lattice == 9 ? Lat<9>::cy(i) : Lat<19>::cy(i);
      const int z = lattice == 9 ? 0 : Lat<19>::cz(i);
      for (int k = 0; k < nc; ++k) V[i][k] = coef_basis(o, c->D, k, x, y, z);
    }
    for (int a = 0; a < nc; ++a)
      for (int b = 0; b < 2 * nc; ++b) {
        double v = 0.0;
        if (b < nc) for (int i = 0; i < q; ++i) v += V[i][a] * V[i][b];
        else v = (b - nc == a) ? 1.0 : 0.0;
        M[a][b] = v;
      }
    for (int col = 0; col < nc; ++col) {  // Gauss-Jordan with partial pivoting
      int piv = col;
      for (int r = col + 1; r < nc; ++r) if (std::fabs(M[r][col]) > std::fabs(M[piv][col])) piv = r;
      for (int b = 0; b < 2 * nc; ++b) std::swap(M[col][b], M[piv][b]);
      const double inv = 1.0 / M[col][col];
      for (int b = 0; b < 2 * nc; ++b) M[col][b] *= inv;
      for (int r = 0; r < nc; ++r) {
        if (r == col) continue;
        const double fct = M[r][col];
        for (int b = 0; b < 2 * nc; ++b) M[r][b] -= fct * M[col][b];
      }
    }
    for (int k = 0; k < nc; ++k)
      for (int i = 0; i < q; ++i) {
        double v = 0.0;
        for (int a = 0; a < nc; ++a) v += M[k][nc + a] * V[i][a];
        c->pmat[o][k * q + i] = v;
      }
  }
  int ffa[6] = {c->opt.ffa_x, c->opt.ffa_x + 1, c->opt.ffa_y0, c->opt.ffa_y1, c->opt.ffa_z0, c->opt.ffa_z1};
  if (!check_box(c, ffa) || !check_box(c, c->opt.diss_box) || !check_box(c, c->opt.design_box)) {
    delete c;
    return HLBM_EINVAL;
  }
  if (cudaGetDevice(&c->device) != cudaSuccess) { cudaGetLastError(); delete c; return HLBM_ECUDA; }
  if (c->opt.stream) {
    c->stream = static_cast<cudaStream_t>(c->opt.stream);
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return HLBM_ECUDA;
    }
    c->own_stream = true;
  }
  const size_t popb = (size_t)c->q * c->g.pitch * pop_elem_bytes(c->storage);
  c->f = dalloc(c, popb);
  c->d = dalloc(c, (size_t)c->g.N * real_bytes(c));
  if (!c->f || !c->d) { hlbm_destroy(c); return HLBM_ENOMEM; }
  if (cudaMalloc(&c->err_dev, 64) != cudaSuccess || cudaMallocHost(&c->err_host, 64) != cudaSuccess ||
      cudaMalloc(&c->scal_dev, 64) != cudaSuccess || cudaMallocHost(&c->scal_host, 64) != cudaSuccess ||
      cudaMalloc(&c->fin, kFinScratchBytes) != cudaSuccess ||
      cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) {
    cudaGetLastError();
    hlbm_destroy(c);
    return HLBM_ENOMEM;
  }
  cudaMemsetAsync(c->err_dev, 0, 64, c->stream);
  cudaMemsetAsync(c->fin, 0, kFinScratchBytes, c->stream);
  // porosity 1 everywhere, uniform inflow equilibrium
  int rc = cuda_check(c, CNT(c, launch_fill_real)(c->d, real_is_double(c), c->g.N, 1.0, c->stream), "porosity");
  if (rc == HLBM_OK)
    rc = cuda_check(c, CNT(c, launch_init_eq)(c->f, c->g, c->q, c->storage, nullptr, nullptr, c->opt.u_in, c->stream), "init");
  if (rc == HLBM_OK) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "sync");
  if (rc != HLBM_OK) { hlbm_destroy(c); return rc; }
  if (rc == HLBM_OK) rc = set_inflow(c, c->opt.inflow_ux);
  c->opt.inflow_ux = nullptr;  // the context keeps its own copy
  if (rc != HLBM_OK) { hlbm_destroy(c); return rc; }
  c->stats.primal_bytes_per_lup_plain = bytes_plain(c);
  *out = c;
  return HLBM_OK;
}

int hlbm_configure(hlbm_ctx* c, double tau, double Cs, const hlbm_options* opt) {
  if (!c) return HLBM_EINVAL;
  if (!(tau > 0.5) || !(Cs >= 0.0) || !std::isfinite(tau) || !std::isfinite(Cs))
    return set_err(c, HLBM_EINVAL, "need tau > 0.5 and Cs >= 0");
  if (opt) {
    if (opt->collision != c->opt.collision)
      return set_err(c, HLBM_EINVAL, "the collision model is fixed when the context is created");
    int ffa[6] = {opt->ffa_x, opt->ffa_x + 1, opt->ffa_y0, opt->ffa_y1, opt->ffa_z0, opt->ffa_z1};
    if (!check_box(c, ffa) || !check_box(c, opt->diss_box) || !check_box(c, opt->design_box))
      return set_err(c, HLBM_EINVAL, "region outside the grid");
    if (!options_valid(opt))
      return set_err(c, HLBM_EINVAL, "need |u_in|, |u_solid| < 0.5 and tau_adj = 0 or > 0.5");
    // everything is checked, and the inflow profile's buffer allocated and
    // filled, before any option changes: a rejected call (HLBM_EINVAL,
    // HLBM_ENOMEM or HLBM_ECUDA from the profile) leaves the options as they were
    if (opt->inflow_ux) {
      int rc = check_inflow(c, opt->inflow_ux);
      if (rc) return rc;
    }
    int rc = set_inflow(c, opt->inflow_ux);
    if (rc) return rc;
    hlbm_options n = c->opt;
    n.u_in = opt->u_in;
    for (int k = 0; k < 3; ++k) n.u_solid[k] = opt->u_solid[k];
    n.tau_adj = opt->tau_adj;
    n.objectives = opt->objectives;
    n.ffa_x = opt->ffa_x;
    n.ffa_y0 = opt->ffa_y0; n.ffa_y1 = opt->ffa_y1;
    n.ffa_z0 = opt->ffa_z0; n.ffa_z1 = opt->ffa_z1;
    std::memcpy(n.diss_box, opt->diss_box, sizeof n.diss_box);
    std::memcpy(n.design_box, opt->design_box, sizeof n.design_box);
    n.accum_stride = opt->accum_stride < 1 ? 1 : opt->accum_stride;
    n.check_every = opt->check_every < 2 ? 100 : opt->check_every + (opt->check_every & 1);
    n.average_full_f = opt->average_full_f;
    n.adjoint_solver = opt->adjoint_solver;
    n.gmres_restart = opt->gmres_restart;
    n.gmres_inner = opt->gmres_inner;
    n.adjoint_warm_start = opt->adjoint_warm_start;
    n.inflow_ux = nullptr;  // the context keeps its own device copy
    c->opt = n;
  }
  c->tau0 = tau;
  c->Cs = Cs;
  c->kles = 4.5 * std::sqrt(2.0) * Cs * Cs;
  c->nu0 = (tau - 0.5) / 3.0;
  c->full_f = c->full_f || c->opt.average_full_f != 0 || (Cs > 0.0 && !c->rr) ||
              (c->opt.objectives & HLBM_OBJ_DRAG_MEA);
  c->nsamples = 0;
  c->acc_mask = 0;
  c->generation++;
  c->have_adjoint = false;
  return HLBM_OK;
}

int hlbm_set_porosity(hlbm_ctx* c, const void* d, int dtype, int on_device) {
  if (!c || !d) return HLBM_EINVAL;
  int rc = stage_in(c, d, dtype, on_device, c->g.N);
  if (rc) return rc;
  HLBM_TRY(c, CNT(c, launch_set_porosity)(c->d, real_is_double(c), c->stage, c->g.N, c->err_dev, c->stream), "porosity");
  unsigned e = 0;
  rc = read_err(c, &e);
  if (rc) return rc;
  c->generation++;
  if (e & 2u) return set_err(c, HLBM_EINVAL, "porosity outside [0, 1] or not finite");
  return HLBM_OK;
}

int hlbm_init_equilibrium(hlbm_ctx* c, const void* rho, const void* u, int dtype, int on_device) {
  if (!c) return HLBM_EINVAL;
  const long long N = c->g.N;
  double* rd = nullptr;
  double* ud = nullptr;
  int rc;
  if (rho || u) {
    rc = ensure_stage(c, (size_t)N * 8 * (1 + c->D) * 2);
    if (rc) return rc;
  }
  // stage layout: [rho (N)] [u (D N)] [f32 scratch]
  if (rho) {
    rc = stage_in(c, rho, dtype, on_device, N);
    if (rc) return rc;
    rd = c->stage;
  }
  if (u) {
    // place u after rho in the staging buffer
    double* dst = c->stage + N;
    if (dtype == HLBM_DTYPE_F64) {
      HLBM_TRY(c, cudaMemcpyAsync(dst, u, (size_t)N * c->D * 8,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  c->stream), "copy u");
    } else if (dtype == HLBM_DTYPE_F32) {
      float* tmp = reinterpret_cast<float*>(c->stage + N * (1 + c->D));
      HLBM_TRY(c, cudaMemcpyAsync(tmp, u, (size_t)N * c->D * 4,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  c->stream), "copy u");
      HLBM_TRY(c, CNT(c, launch_convert_f32_to_f64)(tmp, dst, N * c->D, c->stream), "convert");
    } else {
      return set_err(c, HLBM_EINVAL, "bad dtype");
    }
    ud = dst;
  }
  HLBM_TRY(c, CNT(c, launch_init_eq)(c->f, c->g, c->q, c->storage, rd, ud, c->opt.u_in, c->stream), "init");
  HLBM_TRY(c, cudaStreamSynchronize(c->stream), "sync");
  c->phase = 0;
  c->steps_done = 0;
  c->nsamples = 0;
  c->acc_mask = 0;
  c->generation++;
  c->have_adjoint = false;
  return HLBM_OK;
}

static constexpr long kGraphSteps = 64;  // a multiple of 2 (AA phase) and of kStage

// Variant of the k-th step of a run: plain (acc_base = 0) or, inside an
// averaging window of `nsamp` samples taken every step, the averaging variant
// that folds the FP32 staging into the FP64 sums every kStage samples and at
// the last sample.
static int step_variant(int acc_base, long k, long nsamp) {
  if (!acc_base) return 0;
  const bool flush = (k % kStage) == kStage - 1 || k == nsamp - 1;
  return acc_base | (flush ? ACC_FLUSH : 0);
}

// Run `count` consecutive steps (k = 0 .. count-1 of a plain stretch, or of an
// averaging window with one sample per step).  Whole blocks of kGraphSteps
// steps replay a captured CUDA graph -- every step of a block has the same
// arguments, only the AA phase alternates and the flush falls on fixed
// positions -- and the remaining steps are launched directly.
static int primal_steps(hlbm_ctx* c, const PrimalArgs& a, bool les, int acc_base, long count) {
  long done = 0;
  const long blocks = count / kGraphSteps;
  if (c->graphs_ok && blocks > 0) {
    auto& pg = c->pgraph[acc_base ? 1 : 0][c->phase];
    if (pg.exec && std::memcmp(&pg.args, &a, sizeof a) != 0) {
      cudaGraphExecDestroy(pg.exec);
      pg.exec = nullptr;
    }
    if (!pg.exec) {
      cudaGraph_t graph = nullptr;
      bool ok = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      int ph = c->phase;
      for (long k = 0; ok && k < kGraphSteps; ++k) {
        const int v = step_variant(acc_base, k, kGraphSteps + 1);  // interior block: flush on % kStage
        ok = launch_primal(a, c->q, c->storage, ph == 1, les, v, c->rr, c->stream) == cudaSuccess;
        ph ^= 1;
      }
      if (cudaStreamEndCapture(c->stream, &graph) != cudaSuccess) ok = false;
      if (ok && cudaGraphInstantiate(&pg.exec, graph, 0) != cudaSuccess) {
        ok = false;
        pg.exec = nullptr;
      }
      if (graph) cudaGraphDestroy(graph);
      if (!ok) {
        cudaGetLastError();
        c->graphs_ok = false;  // fall back to direct launches from now on
      } else {
        pg.args = a;
      }
    }
    if (pg.exec) {
      // kGraphSteps is a multiple of kStage, so a replayed block ends on a
      // flush; the window's own last sample must be a flush too, which holds
      // when it is the last step of a block
      for (; done + kGraphSteps <= count; done += kGraphSteps) {
        HLBM_TRY(c, cudaGraphLaunch(pg.exec, c->stream), "graph launch");
        c->stats.kernels_total += kGraphSteps;
      }
      // kGraphSteps is even: the phase is unchanged after each replay
    }
  }
  for (; done < count; ++done) {
    const int v = step_variant(acc_base, done, count);
    cudaError_t e = CNT(c, launch_primal)(a, c->q, c->storage, c->phase == 1, les, v, c->rr, c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "primal launch");
    c->phase ^= 1;
  }
  return HLBM_OK;
}

int hlbm_run_primal(hlbm_ctx* c, long steps, long W) {
  if (!c) return HLBM_EINVAL;
  if (steps < 0 || W < 0 || W > steps) return set_err(c, HLBM_EINVAL, "need 0 <= avg_window <= steps");
  int rc;
  const int mask = c->opt.objectives & 7;
  if (W > 0) {
    rc = reset_averages(c, mask);
    if (rc) return rc;
  }
  PrimalArgs a = primal_args(c);
  const bool les = c->Cs > 0.0;
  const long first = steps - W;
  const long stride = c->opt.accum_stride;
  HLBM_TRY(c, cudaEventRecord(c->ev0, c->stream), "event");
  long launches = 0, samples = 0;
  const int acc_base = ACC_ON | (c->full_f ? ACC_FULL : 0);
  // plain steps before the window
  rc = primal_steps(c, a, les, 0, first);
  if (rc) return rc;
  launches += first;
  if (W > 0 && stride == 1) {
    rc = primal_steps(c, a, les, acc_base, W);
    if (rc) return rc;
    launches += W;
    samples = W;
  } else if (W > 0) {
    const long nsamp = (W + stride - 1) / stride;
    for (long n = first; n < steps; ++n) {
      const bool acc = ((n - first) % stride) == 0;
      const int v = acc ? step_variant(acc_base, samples, nsamp) : 0;
      cudaError_t e = CNT(c, launch_primal)(a, c->q, c->storage, c->phase == 1, les, v, c->rr, c->stream);
      if (e != cudaSuccess) return cuda_check(c, e, "primal launch");
      c->phase ^= 1;
      ++launches;
      if (acc) ++samples;
    }
  }
  HLBM_TRY(c, cudaEventRecord(c->ev1, c->stream), "event");
  unsigned err = 0;
  rc = read_err(c, &err);
  if (rc) return rc;
  float ms = 0;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  c->stats.primal_ms = ms;
  c->stats.primal_launches = launches;
  c->stats.primal_steps += steps;
  c->steps_done += steps;
  if (W > 0) {
    c->nsamples = samples;
    c->generation++;
    c->have_adjoint = false;
    // a window that averaged f itself derives the moment sums from it
    if (c->full_f)
      HLBM_TRY(c, CNT(c, launch_moments_of_sums)(c->fsum, c->q, c->g.N, c->msum, c->rr, c->stream),
               "moments of the averages");
  }
  if (err & 1u) return set_err(c, HLBM_ENONFINITE, "primal state became non-finite");
  return HLBM_OK;
}

int hlbm_run_tangent(hlbm_ctx* c, long steps, const void* delta, int dtype, int on_device,
                     int objective, double* jdot_out) {
  if (!c || !delta || !jdot_out || steps < 1) return HLBM_EINVAL;
  const int o = obj_slot(objective);
  if (o < 0 || o > 1) return set_err(c, HLBM_EINVAL, "tangent: drag (far field) or dissipation");
  if (c->rr) return set_err(c, HLBM_EINVAL, "tangent: BGK collision only");
  const long long N = c->g.N;
  const size_t rb = real_bytes(c);
  const size_t fd_bytes = (size_t)c->q * c->g.pitch * rb;
  if (!c->fd && !(c->fd = dalloc(c, fd_bytes))) return set_err(c, HLBM_ENOMEM, "tangent state");
  if (!c->delta && !(c->delta = dalloc(c, (size_t)N * rb))) return set_err(c, HLBM_ENOMEM, "direction");
  if (c->jhist_n < steps) {
    dfree(c, c->jhist);
    c->jhist = (double*)dalloc(c, (size_t)steps * 8);
    c->jhist_n = c->jhist ? steps : 0;
    if (!c->jhist) return set_err(c, HLBM_ENOMEM, "history");
  }
  if (c->red_n < c->nblk) {
    dfree(c, c->red);
    c->red = (double*)dalloc(c, (size_t)c->nblk * 8);
    c->red_n = c->red ? c->nblk : 0;
    if (!c->red) return set_err(c, HLBM_ENOMEM, "reduction buffer");
  }
  int rc = stage_in(c, delta, dtype, on_device, N);
  if (rc) return rc;
  if (real_is_double(c)) {
    HLBM_TRY(c, cudaMemcpyAsync(c->delta, c->stage, (size_t)N * 8, cudaMemcpyDeviceToDevice, c->stream), "copy");
  } else {
    HLBM_TRY(c, CNT(c, launch_convert_f64_to_f32)(c->stage, (float*)c->delta, N, c->stream), "convert");
  }
  // the tangent starts from zero: the initial state does not depend on d
  HLBM_TRY(c, cudaMemsetAsync(c->fd, 0, fd_bytes, c->stream), "memset");
  TangentArgs a{};
  a.f = c->f;
  a.fd = c->fd;
  a.d = c->d;
  a.delta = c->delta;
  a.g = c->g;
  a.tau0 = c->tau0; a.kles = c->kles; a.u_in = c->opt.u_in; a.nu0 = c->nu0;
  for (int k = 0; k < 3; ++k) { a.us[k] = c->opt.u_solid[k]; a.us_f[k] = (float)a.us[k]; }
  a.tau0_f = (float)a.tau0; a.kles_f = (float)a.kles; a.u_in_f = (float)a.u_in; a.nu0_f = (float)a.nu0;
  a.objective = objective;
  a.ffa[0] = c->opt.ffa_x; a.ffa[1] = c->opt.ffa_y0; a.ffa[2] = c->opt.ffa_y1;
  a.ffa[3] = c->opt.ffa_z0; a.ffa[4] = c->opt.ffa_z1;
  std::memcpy(a.db, c->opt.diss_box, sizeof a.db);
  a.jpart = c->red;
  a.inflow = c->inflow;
  const bool les = c->Cs > 0.0;
  for (long n = 0; n < steps; ++n) {
    HLBM_TRY(c, CNT(c, launch_tangent)(a, c->q, c->storage, c->phase == 1, les, c->stream), "tangent");
    HLBM_TRY(c, CNT(c, launch_finalize_sum)(c->red, c->nblk, c->jhist + n, c->fin, c->stream), "reduce");
    c->phase ^= 1;
  }
  HLBM_TRY(c, cudaMemcpyAsync(jdot_out, c->jhist, (size_t)steps * 8, cudaMemcpyDeviceToHost, c->stream), "copy");
  unsigned err = 0;
  rc = read_err(c, &err);
  if (rc) return rc;
  c->steps_done += steps;
  c->stats.primal_steps += steps;
  c->nsamples = 0;
  c->acc_mask = 0;
  c->generation++;
  c->have_adjoint = false;
  return HLBM_OK;
}

int hlbm_objective(hlbm_ctx* c, int obj, double* J) {
  if (!c || !J) return HLBM_EINVAL;
  const int o = obj_slot(obj);
  if (o < 0) return set_err(c, HLBM_EINVAL, "unknown objective");
  if (c->nsamples < 1 || !(c->acc_mask & obj)) return set_err(c, HLBM_ESTATE, "objective not averaged");
  if (obj == HLBM_OBJ_DRAG_MEA) {
    if (!c->fsum) return set_err(c, HLBM_ESTATE, "J_MEA needs the averaged f");
    const long long nbm = (long long)((c->g.nx + NT - 1) / NT) * c->g.ny * c->g.nz;
    if (c->red_n < 2 * nbm) {
      dfree(c, c->red);
      c->red = (double*)dalloc(c, (size_t)(2 * nbm) * 8);
      c->red_n = c->red ? 2 * nbm : 0;
      if (!c->red) return set_err(c, HLBM_ENOMEM, "reduction buffer");
    }
    int nb = 0;
    HLBM_TRY(c, CNT(c, launch_mea_eval)(c->fsum, 1.0 / (double)c->nsamples, c->d, c->g, c->q,
                                        real_is_double(c), c->red, c->red + nbm, &nb, c->stream), "mea");
    HLBM_TRY(c, CNT(c, launch_finalize_sum)(c->red, nb, c->scal_dev, c->fin, c->stream), "reduce");
    HLBM_TRY(c, CNT(c, launch_finalize_sum)(c->red + nbm, nb, c->scal_dev + 1, c->fin, c->stream), "reduce");
    HLBM_TRY(c, cudaMemcpyAsync(c->scal_host, c->scal_dev, 16, cudaMemcpyDeviceToHost, c->stream), "copy");
    HLBM_TRY(c, cudaStreamSynchronize(c->stream), "sync");
    *J = c->scal_host[0] / (c->scal_host[1] > 0 ? c->scal_host[1] : 1.0);
    return HLBM_OK;
  }
  HLBM_TRY(c, CNT(c, launch_finalize_sum)(c->jblk[o], c->njslot, c->scal_dev, c->fin, c->stream), "reduce");
  HLBM_TRY(c, cudaMemcpyAsync(c->scal_host, c->scal_dev, 8, cudaMemcpyDeviceToHost, c->stream), "copy");
  HLBM_TRY(c, cudaStreamSynchronize(c->stream), "sync");
  *J = c->scal_host[0] / (double)c->nsamples;
  return HLBM_OK;
}

static int prepare_linearisation(hlbm_ctx* c, int mode) {
  const bool exact_les = (mode == HLBM_ADJ_EXACT) && c->Cs > 0.0;
  const double tau_b = c->opt.tau_adj > 0.0 ? c->opt.tau_adj : c->tau0;
  const int want = exact_les ? 1 : 0;
  // record kinds: 0 BGK, 1 BGK exact LES (f_bar), 2 BGK frozen turbulence,
  // 3 RR (rho, u, omega, Pi), 4 RR exact LES (omega from Pi in the kernels)
  int rec_mode_key = exact_les ? 1 : (mode == HLBM_ADJ_FTA && c->Cs > 0.0 ? 2 : 0);
  if (c->rr) rec_mode_key = exact_les ? 4 : 3;
  if (c->rec && c->rec_mode == rec_mode_key && c->rec_taub == tau_b && c->rec_generation == c->generation)
    return HLBM_OK;
  const int planes = c->rr ? c->D + 2 + c->D * (c->D + 1) / 2 : (want ? c->q : c->D + 2);
  const size_t bytes = (size_t)planes * c->g.N * real_bytes(c);
  if (c->rec_bytes < bytes) {
    dfree(c, c->rec);
    c->rec = dalloc(c, bytes);
    c->rec_bytes = c->rec ? bytes : 0;
    if (!c->rec) return set_err(c, HLBM_ENOMEM, "record");
  }
  if (want && !c->rr && !c->fsum) return set_err(c, HLBM_ESTATE, "exact LES linearisation needs the averaged f");
  PrepArgs p{};
  p.fsum = c->fsum;
  p.msum = c->msum;
  p.tsum = (mode == HLBM_ADJ_FTA && c->Cs > 0.0) ? c->tsum : nullptr;
  p.inv_n = 1.0 / (double)c->nsamples;
  p.rec = c->rec;
  p.rec_pitch = c->g.N;
  p.g = c->g;
  p.tau_b = tau_b;
  p.exact = want;
  p.rr = c->rr ? 1 : 0;
  p.d = c->d;
  for (int k = 0; k < 3; ++k) p.us[k] = c->opt.u_solid[k];
  HLBM_TRY(c, CNT(c, launch_prep)(p, c->q, real_is_double(c), c->stream), "prep");
  c->rec_mode = rec_mode_key;
  c->rec_taub = tau_b;
  c->rec_generation = c->generation;
  return HLBM_OK;
}

static AdjointArgs adjoint_args(hlbm_ctx* c, int mode, const int sb[6]) {
  AdjointArgs a{};
  a.lam = c->lam;
  a.g = c->g;
  a.d = c->d;
  a.rec = c->rec;
  a.rec_pitch = c->g.N;
  a.tau_b = c->rec_taub;
  a.kles = c->kles;
  for (int k = 0; k < 3; ++k) { a.us[k] = c->opt.u_solid[k]; a.us_f[k] = (float)a.us[k]; }
  a.tau_b_f = (float)a.tau_b;
  a.kles_f = (float)a.kles;
  a.src = c->src;
  std::memcpy(a.sb, sb, sizeof a.sb);
  a.src_pitch = (long long)(sb[1] - sb[0]) * (sb[3] - sb[2]) * (sb[5] - sb[4]);
  // J_MEA keeps its q values; the others their derivative-polynomial coefficients
  a.src_nc = c->src_obj == HLBM_OBJ_DRAG_MEA ? 0 : ncoef(obj_slot(c->src_obj), c->D);
  a.snap = c->snap;
  a.red = c->red;
  (void)mode;
  return a;
}

static constexpr int kMaxRestart = 64;

// Restarted GMRES on the fixed point of the adjoint sweeps.  In natural layout
// the stored adjoint state mu = S^T B_f^T lambda obeys, over one pair of
// sweeps, mu <- M^2 mu + c.  Its fixed point solves (I - M^2) mu = c with
// c = two sweeps from mu = 0; the operator is two sweeps without source.
// Arnoldi with classical Gram-Schmidt applied twice, Givens rotations, FP64
// small matrices on the host.  Returns the number of sweeps used; on exit the
// adjoint array holds the solution x.
static int adjoint_gmres(hlbm_ctx* c, const AdjointArgs& a, bool dbl, bool exact, double tol,
                         long max_sweeps, long* sweeps_out, bool warm) {
  const long long L = (long long)c->q * c->g.pitch;
  const size_t rb = real_bytes(c);
  int m = c->opt.gmres_restart;
  if (m < 2) m = 30;
  if (m > kMaxRestart) m = kMaxRestart;
  const size_t need = (size_t)(m + 4) * L * rb;
  if (c->kry_bytes < need) {
    dfree(c, c->kry);
    c->kry = dalloc(c, need);
    c->kry_bytes = c->kry ? need : 0;
    if (!c->kry) return set_err(c, HLBM_ENOMEM, "GMRES vectors");
  }
  if (!c->kpart && !(c->kpart = (double*)dalloc(c, (size_t)(kMaxRestart + 1) * kKrylovBlocks * 8)))
    return set_err(c, HLBM_ENOMEM, "GMRES partials");
  if (!c->kdev && !(c->kdev = (double*)dalloc(c, (size_t)3 * (kMaxRestart + 1) * 8)))
    return set_err(c, HLBM_ENOMEM, "GMRES coefficients");
  if (!c->khost && cudaMallocHost(&c->khost, (size_t)3 * (kMaxRestart + 1) * 8) != cudaSuccess) {
    cudaGetLastError();
    c->khost = nullptr;
    return set_err(c, HLBM_ENOMEM, "GMRES host buffer");
  }
  char* base = static_cast<char*>(c->kry);
  auto vec = [&](long long k) { return (void*)(base + (size_t)k * L * rb); };
  void* V = vec(0);
  void* w = vec(m + 1);
  void* x = vec(m + 2);
  void* cv = vec(m + 3);
  double* h1 = c->kdev;
  double* h2 = c->kdev + (kMaxRestart + 1);
  double* hn = c->kdev + 2 * (kMaxRestart + 1);
  cudaStream_t st = c->stream;
  AdjointArgs a0 = a;  // operator: no source
  for (int k = 0; k < 6; ++k) a0.sb[k] = 0;
  long sweeps = 0;
  // one operator application = `inner` pairs of sweeps (polynomial
  // preconditioning by the fixed-point iteration itself: the fast-decaying
  // modes are damped before the Krylov space has to resolve them)
  const int inner = c->opt.gmres_inner < 1 ? 1 : c->opt.gmres_inner;
  auto pair = [&](const AdjointArgs& aa) -> cudaError_t {
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < inner && e == cudaSuccess; ++k) {
      e = CNT(c, launch_adjoint)(aa, c->q, dbl, false, exact, 0, c->rr, st);
      if (e == cudaSuccess) e = CNT(c, launch_adjoint)(aa, c->q, dbl, true, exact, 0, c->rr, st);
      sweeps += 2;
    }
    return e;
  };
  auto fetch = [&](const double* dsrc, int n) -> int {
    HLBM_TRY(c, cudaMemcpyAsync(c->khost, dsrc, (size_t)n * 8, cudaMemcpyDeviceToHost, st), "copy");
    HLBM_TRY(c, cudaStreamSynchronize(st), "sync");
    return HLBM_OK;
  };
  // c = P(0); x = 0, or with a warm start the adjoint array's content
  if (warm) HLBM_TRY(c, CNT(c, launch_lincomb)(x, c->lam, 1.0, nullptr, 0.0, L, dbl, st), "copy");
  HLBM_TRY(c, cudaMemsetAsync(c->lam, 0, (size_t)L * rb, st), "memset");
  HLBM_TRY(c, pair(a), "adjoint");
  HLBM_TRY(c, CNT(c, launch_lincomb)(cv, c->lam, 1.0, nullptr, 0.0, L, dbl, st), "copy");
  if (!warm) HLBM_TRY(c, cudaMemsetAsync(x, 0, (size_t)L * rb, st), "memset");
  HLBM_TRY(c, CNT(c, launch_mdot)(cv, cv, 1, L, dbl, c->kpart, hn, st), "dot");
  int rc = fetch(hn, 1);
  if (rc) return rc;
  const double cnorm = std::sqrt(c->khost[0]) > 0 ? std::sqrt(c->khost[0]) : 1.0;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  bool first = !warm;  // from x = 0 the first residual is c itself
  // progress check of the restarts' true residuals over windows of kStallSweeps
  constexpr long kStallSweeps = 4000;
  double beta_ref = INFINITY;
  long sweeps_ref = 0;
  while (sweeps < max_sweeps) {
    // r = c - (I - M^2) x  into V_0
    if (first) {
      HLBM_TRY(c, CNT(c, launch_lincomb)(V, cv, 1.0, nullptr, 0.0, L, dbl, st), "copy");
      first = false;
    } else {
      HLBM_TRY(c, CNT(c, launch_lincomb)(c->lam, x, 1.0, nullptr, 0.0, L, dbl, st), "copy");
      HLBM_TRY(c, pair(a0), "adjoint");
      HLBM_TRY(c, CNT(c, launch_lincomb)(V, cv, 1.0, x, -1.0, L, dbl, st), "lincomb");
      HLBM_TRY(c, CNT(c, launch_lincomb)(V, V, 1.0, c->lam, 1.0, L, dbl, st), "lincomb");
    }
    HLBM_TRY(c, CNT(c, launch_mdot)(V, V, 1, L, dbl, c->kpart, hn, st), "dot");
    rc = fetch(hn, 1);
    if (rc) return rc;
    const double beta = std::sqrt(c->khost[0]);
    if (!std::isfinite(beta)) return set_err(c, HLBM_ENONFINITE, "adjoint became non-finite");
    if (beta / cnorm <= tol * 0.5) break;
    // less than 5 % off the true residual over kStallSweeps sweeps: the rounding
    // floor of the arithmetic is reached, more restarts would only spend sweeps
    if (sweeps - sweeps_ref >= kStallSweeps || beta_ref == INFINITY) {
      if (beta >= 0.95 * beta_ref) break;
      beta_ref = beta;
      sweeps_ref = sweeps;
    }
    HLBM_TRY(c, CNT(c, launch_lincomb)(V, V, 1.0 / beta, nullptr, 0.0, L, dbl, st), "scale");
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    for (int j = 0; j < m && sweeps < max_sweeps; ++j) {
      void* Vj = vec(j);
      // w = (I - M^2) V_j
      HLBM_TRY(c, CNT(c, launch_lincomb)(c->lam, Vj, 1.0, nullptr, 0.0, L, dbl, st), "copy");
      HLBM_TRY(c, pair(a0), "adjoint");
      HLBM_TRY(c, CNT(c, launch_lincomb)(w, Vj, 1.0, c->lam, -1.0, L, dbl, st), "lincomb");
      // classical Gram-Schmidt, twice
      HLBM_TRY(c, CNT(c, launch_mdot)(w, V, j + 1, L, dbl, c->kpart, h1, st), "dot");
      HLBM_TRY(c, CNT(c, launch_maxpy)(w, V, h1, j + 1, -1.0, L, dbl, st), "axpy");
      HLBM_TRY(c, CNT(c, launch_mdot)(w, V, j + 1, L, dbl, c->kpart, h2, st), "dot");
      HLBM_TRY(c, CNT(c, launch_maxpy)(w, V, h2, j + 1, -1.0, L, dbl, st), "axpy");
      HLBM_TRY(c, CNT(c, launch_mdot)(w, w, 1, L, dbl, c->kpart, hn, st), "dot");
      HLBM_TRY(c, cudaMemcpyAsync(c->khost, h1, (size_t)(j + 1) * 8, cudaMemcpyDeviceToHost, st), "copy");
      HLBM_TRY(c, cudaMemcpyAsync(c->khost + (kMaxRestart + 1), h2, (size_t)(j + 1) * 8,
                                  cudaMemcpyDeviceToHost, st), "copy");
      HLBM_TRY(c, cudaMemcpyAsync(c->khost + 2 * (kMaxRestart + 1), hn, 8, cudaMemcpyDeviceToHost, st), "copy");
      HLBM_TRY(c, cudaStreamSynchronize(st), "sync");
      double* col = &H[(size_t)j * (m + 1)];
      for (int i = 0; i <= j; ++i) col[i] = c->khost[i] + c->khost[(kMaxRestart + 1) + i];
      const double hnorm = std::sqrt(c->khost[2 * (kMaxRestart + 1)]);
      col[j + 1] = hnorm;
      if (!std::isfinite(hnorm)) return set_err(c, HLBM_ENONFINITE, "adjoint became non-finite");
      if (hnorm > 0) HLBM_TRY(c, CNT(c, launch_lincomb)(vec(j + 1), w, 1.0 / hnorm, nullptr, 0.0, L, dbl, st), "scale");
      // previous rotations, then a new one that zeroes col[j + 1]
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = t;
      }
      const double rr = std::hypot(col[j], col[j + 1]);
      cs[j] = rr > 0 ? col[j] / rr : 1.0;
      sn[j] = rr > 0 ? col[j + 1] / rr : 0.0;
      col[j] = rr;
      col[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      k = j + 1;
      if (std::fabs(g[j + 1]) / cnorm <= tol * 0.5 || hnorm <= 1e-300) break;
    }
    // y = H^-1 g (upper triangular k x k), x += V y
    for (int i = k - 1; i >= 0; --i) {
      double v = g[i];
      for (int l = i + 1; l < k; ++l) v -= H[(size_t)l * (m + 1) + i] * y[l];
      y[i] = v / H[(size_t)i * (m + 1) + i];
    }
    for (int i = 0; i < k; ++i) c->khost[i] = y[i];
    HLBM_TRY(c, cudaMemcpyAsync(h1, c->khost, (size_t)k * 8, cudaMemcpyHostToDevice, st), "copy");
    HLBM_TRY(c, CNT(c, launch_maxpy)(x, V, h1, k, 1.0, L, dbl, st), "axpy");
    HLBM_TRY(c, cudaStreamSynchronize(st), "sync");
  }
  // the adjoint array holds the solution
  HLBM_TRY(c, CNT(c, launch_lincomb)(c->lam, x, 1.0, nullptr, 0.0, L, dbl, st), "copy");
  *sweeps_out = sweeps;
  return HLBM_OK;
}

// Everything an adjoint solve does before its sweeps: the argument checks of
// the objective and mode, the buffers, the linearisation record at the
// averaged state, the source g_bar and its norm, lambda = 0; ev0 is recorded
// before the source.
struct AdjSetup {
  AdjointArgs a;
  bool exact;
  long long nb_adj;
  double gnorm;
  bool warm;  // the solve starts from the adjoint array's content
};

static int adjoint_setup(hlbm_ctx* c, int obj, int mode, AdjSetup* out) {
  const int o = obj_slot(obj);
  if (o < 0 || (mode != HLBM_ADJ_EXACT && mode != HLBM_ADJ_FTA))
    return set_err(c, HLBM_EINVAL, "bad objective or mode");
  if (c->nsamples < 1 || !(c->acc_mask & obj)) return set_err(c, HLBM_ESTATE, "run the primal with this objective averaged first");
  const bool dbl = real_is_double(c);
  const size_t lam_bytes = (size_t)c->q * c->g.pitch * real_bytes(c);
  if (!c->lam && !(c->lam = dalloc(c, lam_bytes))) return set_err(c, HLBM_ENOMEM, "lambda");
  if (!c->snap && !(c->snap = dalloc(c, lam_bytes))) return set_err(c, HLBM_ENOMEM, "snapshot");
  const long long nb_adj = adjoint_blocks(c->g);
  int sb[6];
  objective_box(c, obj, sb);
  const long long vol = (long long)(sb[1] - sb[0]) * (sb[3] - sb[2]) * (sb[5] - sb[4]);
  const long long nb_src = (long long)((sb[1] - sb[0] + NT - 1) / NT) * (sb[3] - sb[2]) * (sb[5] - sb[4]);
  long long need_red = nb_adj > nb_src ? nb_adj : nb_src;
  if (need_red < 2 * nb_src) need_red = 2 * nb_src;  // J_MEA: values and counts
  if (c->red_n < need_red) {
    dfree(c, c->red);
    c->red = (double*)dalloc(c, (size_t)need_red * 8);
    c->red_n = c->red ? need_red : 0;
    if (!c->red) return set_err(c, HLBM_ENOMEM, "reduction buffer");
  }
  const size_t src_bytes = (size_t)c->q * vol * real_bytes(c);
  if (c->src_bytes < src_bytes) {
    dfree(c, c->src);
    c->src = dalloc(c, src_bytes);
    c->src_bytes = c->src ? src_bytes : 0;
    if (!c->src) return set_err(c, HLBM_ENOMEM, "source");
  }
  int rc = prepare_linearisation(c, mode);
  if (rc) return rc;
  const bool exact = c->rec_mode == 1 || c->rec_mode == 4;

  HLBM_TRY(c, cudaEventRecord(c->ev0, c->stream), "event");
  int nbs = 0;
  if (obj == HLBM_OBJ_DRAG_MEA) {
    // constant dJ_MEA/df over the grid; first the number of surface nodes
    if (!c->fsum) return set_err(c, HLBM_ESTATE, "J_MEA needs the averaged f");
    HLBM_TRY(c, CNT(c, launch_mea_eval)(c->fsum, 1.0 / (double)c->nsamples, c->d, c->g, c->q, dbl,
                                        c->red, c->red + nb_src, &nbs, c->stream), "mea");
    HLBM_TRY(c, CNT(c, launch_finalize_sum)(c->red + nb_src, nbs, c->scal_dev, c->fin, c->stream), "reduce");
    HLBM_TRY(c, cudaMemcpyAsync(c->scal_host, c->scal_dev, 8, cudaMemcpyDeviceToHost, c->stream), "copy");
    HLBM_TRY(c, cudaStreamSynchronize(c->stream), "sync");
    const double area = c->scal_host[0] > 0 ? c->scal_host[0] : 1.0;
    HLBM_TRY(c, CNT(c, launch_mea_source)(c->d, c->g, c->q, dbl, 1.0 / area, c->src, c->red, &nbs,
                                          c->stream), "source");
  } else {
    SourceArgs sa{};
    sa.gsum = c->gsum[o];
    sa.obj_slot = o;
    sa.inv_n = 1.0 / (double)c->nsamples;
    sa.src = c->src;
    std::memcpy(sa.box, sb, sizeof sa.box);
    sa.g = c->g;
    sa.red = c->red;
    HLBM_TRY(c, CNT(c, launch_source)(sa, c->q, dbl, &nbs, c->stream), "source");
  }
  HLBM_TRY(c, CNT(c, launch_finalize_sum)(c->red, nbs, c->scal_dev, c->fin, c->stream), "reduce");
  HLBM_TRY(c, cudaMemcpyAsync(c->scal_host, c->scal_dev, 8, cudaMemcpyDeviceToHost, c->stream), "copy");
  const bool warm = c->opt.adjoint_warm_start != 0 && c->lam_set;
  if (!warm) HLBM_TRY(c, cudaMemsetAsync(c->lam, 0, lam_bytes, c->stream), "memset");
  HLBM_TRY(c, cudaStreamSynchronize(c->stream), "sync");
  double gnorm = std::sqrt(c->scal_host[0]);
  if (!(gnorm > 0.0)) gnorm = 1.0;

  c->src_obj = obj;
  out->a = adjoint_args(c, mode, sb);
  out->exact = exact;
  out->nb_adj = nb_adj;
  out->gnorm = gnorm;
  out->warm = warm;
  return HLBM_OK;
}

// Everything an adjoint solve does after its sweeps (ev1, statistics, the
// state flags, the message of the status); returns the status.
static int adjoint_finish(hlbm_ctx* c, int obj, int mode, int status, long k, long launches,
                          bool exact) {
  HLBM_TRY(c, cudaEventRecord(c->ev1, c->stream), "event");
  HLBM_TRY(c, cudaEventSynchronize(c->ev1), "sync");
  float ms = 0;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  c->stats.adjoint_ms = ms;
  c->stats.adjoint_iters = k;
  c->stats.adjoint_launches = launches;
  {
    const int recp = exact ? c->q : c->D + 2;
    const double rb = (double)real_bytes(c);
    c->stats.adjoint_bytes_per_lup = (2.0 * c->q + recp + 1) * rb;
  }
  c->last_obj = obj;
  c->last_mode = mode;
  c->have_adjoint = (status == HLBM_OK || status == HLBM_NOT_CONVERGED);
  c->lam_set = c->have_adjoint;
  if (status == HLBM_ENONFINITE) return set_err(c, status, "adjoint became non-finite");
  if (status == HLBM_EDIVERGED) return set_err(c, status, "adjoint residual diverged");
  if (status == HLBM_NOT_CONVERGED) set_err(c, status, "adjoint reached max_iter");
  return status;
}

int hlbm_solve_adjoint(hlbm_ctx* c, int obj, int mode, double tol, long max_iter, long* iters_out,
                       double* res_out) {
  if (!c) return HLBM_EINVAL;
  if (!(tol >= 0) || max_iter < 2) return set_err(c, HLBM_EINVAL, "bad tol or max_iter");
  AdjSetup su{};
  int rc = adjoint_setup(c, obj, mode, &su);
  if (rc) return rc;
  const bool dbl = real_is_double(c);
  const bool exact = su.exact;
  const long long nb_adj = su.nb_adj;
  const double gnorm = su.gnorm;
  AdjointArgs a = su.a;
  const long m = c->opt.check_every;
  long k = 0, launches = 0;
  double r = INFINITY, rmin = INFINITY;
  int status = HLBM_NOT_CONVERGED;
  auto enqueue_chunk = [&](long chunk) -> cudaError_t {
    for (long j = 0; j < chunk; ++j) {
      const bool odd = (j & 1) != 0;
      const int res = j == chunk - 2 ? 1 : (j == chunk - 1 ? 2 : 0);
      cudaError_t e = launch_adjoint(a, c->q, dbl, odd, exact, res, c->rr, c->stream);
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = launch_finalize_sum(c->red, nb_adj, c->scal_dev, c->fin, c->stream);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(c->scal_host, c->scal_dev, 8, cudaMemcpyDeviceToHost, c->stream);
  };
  if (c->opt.adjoint_solver == 1) {
    // Krylov passes on the fixed point, each result checked by the plain
    // iteration's update criterion (one more pair of sweeps).  GMRES stops on
    // its own residual, which is not that criterion: when the check misses
    // tol, the Krylov tolerance is tightened by the ratio seen and GMRES goes
    // on from the checked iterate, until the criterion holds, the sweeps run
    // out, or a pass no longer halves it (the rounding floor of the arithmetic).
    double tol_k = tol, r_prev = INFINITY;
    bool warm = su.warm;
    for (;;) {
      long left = max_iter - k - 2;
      if (k == 0 && left < 2) left = 2;
      // a further pass needs room for its source and one operator application
      const long pass_min = 4L * (c->opt.gmres_inner < 1 ? 1 : c->opt.gmres_inner);
      if (left < 2 || (k > 0 && left < pass_min)) break;
      long sweeps = 0;
      rc = adjoint_gmres(c, a, dbl, exact, tol_k, left, &sweeps, warm);
      if (rc) return rc;
      k += sweeps;
      launches += sweeps;
      HLBM_TRY(c, enqueue_chunk(2), "adjoint launch");
      c->stats.kernels_total += 3;
      launches += 2;
      k += 2;
      HLBM_TRY(c, cudaStreamSynchronize(c->stream), "sync");
      r = std::sqrt(c->scal_host[0]) / gnorm;
      if (!std::isfinite(r)) { status = HLBM_ENONFINITE; break; }
      if (r <= tol) { status = HLBM_OK; break; }
      if (!(r < 0.5 * r_prev)) break;
      r_prev = r;
      tol_k *= 0.5 * tol / r;
      warm = true;
    }
    if (iters_out) *iters_out = k;
    if (res_out) *res_out = r;
    return adjoint_finish(c, obj, mode, status, k, launches, exact);
  }
  auto& ag = c->agraph;
  if (ag.exec && (ag.chunk != m || ag.exact != exact || std::memcmp(&ag.args, &a, sizeof a) != 0)) {
    cudaGraphExecDestroy(ag.exec);
    ag.exec = nullptr;
  }
  while (k < max_iter) {
    long chunk = max_iter - k < m ? max_iter - k : m;
    if (chunk & 1) chunk += 1;
    if (chunk < 2) chunk = 2;
    if (chunk == m && c->graphs_ok && !ag.exec) {
      cudaGraph_t graph = nullptr;
      bool ok = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) ok = enqueue_chunk(chunk) == cudaSuccess;
      if (cudaStreamEndCapture(c->stream, &graph) != cudaSuccess) ok = false;
      if (ok && cudaGraphInstantiate(&ag.exec, graph, 0) != cudaSuccess) {
        ok = false;
        ag.exec = nullptr;
      }
      if (graph) cudaGraphDestroy(graph);
      if (!ok) {
        cudaGetLastError();
        c->graphs_ok = false;
      } else {
        ag.args = a;
        ag.chunk = m;
        ag.exact = exact;
      }
    }
    if (chunk == m && ag.exec) {
      HLBM_TRY(c, cudaGraphLaunch(ag.exec, c->stream), "graph launch");
    } else {
      HLBM_TRY(c, enqueue_chunk(chunk), "adjoint launch");
    }
    c->stats.kernels_total += chunk + 1;
    launches += chunk;
    k += chunk;
    HLBM_TRY(c, cudaStreamSynchronize(c->stream), "sync");
    r = std::sqrt(c->scal_host[0]) / gnorm;
    if (!std::isfinite(r)) { status = HLBM_ENONFINITE; break; }
    if (r < rmin) rmin = r;
    if (r <= tol) { status = HLBM_OK; break; }
    if (r > 1e6 * rmin && rmin > 0) { status = HLBM_EDIVERGED; break; }
  }
  if (iters_out) *iters_out = k;
  if (res_out) *res_out = r;
  return adjoint_finish(c, obj, mode, status, k, launches, exact);
}

static int run_gradient(hlbm_ctx* c, const int box[6], double* out, double* mu_out) {
  const int o = obj_slot(c->last_obj);
  GradArgs ga{};
  ga.lam = c->lam;
  ga.g = c->g;
  ga.d = c->d;
  ga.rec = c->rec;
  ga.rec_pitch = c->g.N;
  ga.tau_b = c->rec_taub;
  ga.kles = c->kles;
  for (int k = 0; k < 3; ++k) { ga.us[k] = c->opt.u_solid[k]; ga.us_f[k] = (float)ga.us[k]; }
  ga.tau_b_f = (float)ga.tau_b;
  ga.kles_f = (float)ga.kles;
  ga.ddsum = o < 2 ? c->ddsum[o] : nullptr;  // dJ_MEA/dd = 0
  ga.inv_n = 1.0 / (double)c->nsamples;
  std::memcpy(ga.box, box, sizeof ga.box);
  ga.out = out;
  ga.mu_out = mu_out;
  HLBM_TRY(c, CNT(c, launch_gradient)(ga, c->q, real_is_double(c), c->rec_mode == 1 || c->rec_mode == 4,
                                      c->rr, c->stream), "gradient");
  return HLBM_OK;
}

int hlbm_gradient(hlbm_ctx* c, void* out, int dtype, int on_device) {
  if (!c || !out) return HLBM_EINVAL;
  if (!c->have_adjoint || c->rec_generation != c->generation)
    return set_err(c, HLBM_ESTATE, "solve the adjoint first");
  const int* b = c->opt.design_box;
  const long long vol = (long long)(b[1] - b[0]) * (b[3] - b[2]) * (b[5] - b[4]);
  int rc = ensure_stage(c, (size_t)vol * 12);
  if (rc) return rc;
  rc = run_gradient(c, b, c->stage, nullptr);
  if (rc) return rc;
  return stage_out(c, out, dtype, on_device, vol);
}

int hlbm_get_field(hlbm_ctx* c, int which, void* out, int dtype, int on_device) {
  if (!c || !out) return HLBM_EINVAL;
  const long long N = c->g.N;
  const long long qN = (long long)c->q * N;
  long long n = 0;
  int rc;
  switch (which) {
    case HLBM_FIELD_RHO:
    case HLBM_FIELD_U:
    case HLBM_FIELD_F: {
      n = which == HLBM_FIELD_RHO ? N : (which == HLBM_FIELD_U ? (long long)c->D * N : qN);
      rc = ensure_stage(c, (size_t)n * 12);
      if (rc) return rc;
      HLBM_TRY(c, CNT(c, launch_readout)(c->f, c->d, c->g, c->q, c->storage, c->phase == 1, c->opt.u_in, c->inflow,
                                 which == HLBM_FIELD_F ? c->stage : nullptr,
                                 which == HLBM_FIELD_RHO ? c->stage : nullptr,
                                 which == HLBM_FIELD_U ? c->stage : nullptr, c->stream), "readout");
      break;
    }
    case HLBM_FIELD_GBAR_FFA:
    case HLBM_FIELD_GBAR_DISS: {
      if (c->nsamples < 1) return set_err(c, HLBM_ESTATE, "no averages");
      const int o = which == HLBM_FIELD_GBAR_FFA ? 0 : 1;
      if (!c->gsum[o] || !(c->acc_mask & (1 << o))) return set_err(c, HLBM_ESTATE, "field not averaged");
      n = qN;
      rc = ensure_stage(c, (size_t)n * 12);
      if (rc) return rc;
      HLBM_TRY(c, CNT(c, launch_expand_coef)(c->gsum[o], o, c->q, N, 1.0 / (double)c->nsamples,
                                             c->stage, c->stream), "expand");
      break;
    }
    case HLBM_FIELD_FBAR:
    case HLBM_FIELD_DJDD_FFA:
    case HLBM_FIELD_DJDD_DISS:
    case HLBM_FIELD_TAU_T: {
      if (c->nsamples < 1) return set_err(c, HLBM_ESTATE, "no averages");
      const double* src = nullptr;
      if (which == HLBM_FIELD_FBAR) {
        if (!c->fsum) return set_err(c, HLBM_ESTATE, "f_bar is not averaged (needs average_full_f or Cs > 0)");
        n = qN;
        rc = ensure_stage(c, (size_t)n * 12);
        if (rc) return rc;
        HLBM_TRY(c, CNT(c, launch_fbar_out)(c->fsum, c->q, N, 1.0 / (double)c->nsamples, c->stage,
                                            c->stream), "fbar");
        break;
      }
      if (which == HLBM_FIELD_DJDD_FFA) { src = c->ddsum[0]; n = N; }
      if (which == HLBM_FIELD_DJDD_DISS) { src = c->ddsum[1]; n = N; }
      if (which == HLBM_FIELD_TAU_T) { src = c->tsum; n = N; }
      if (!src) return set_err(c, HLBM_ESTATE, "field not averaged (f_bar needs average_full_f or Cs > 0)");
      rc = ensure_stage(c, (size_t)n * 12);
      if (rc) return rc;
      HLBM_TRY(c, cudaMemcpyAsync(c->stage, src, (size_t)n * 8, cudaMemcpyDeviceToDevice, c->stream), "copy");
      HLBM_TRY(c, CNT(c, launch_scale)(c->stage, n, 1.0 / (double)c->nsamples, c->stream), "scale");
      break;
    }
    case HLBM_FIELD_LAMBDA: {
      if (!c->have_adjoint) return set_err(c, HLBM_ESTATE, "no adjoint");
      n = qN;
      rc = ensure_stage(c, (size_t)(n + N) * 12);
      if (rc) return rc;
      int box[6] = {0, c->g.nx, 0, c->g.ny, 0, c->g.nz};
      rc = run_gradient(c, box, c->stage + n, c->stage);
      if (rc) return rc;
      break;
    }
    case HLBM_FIELD_POROSITY: {
      n = N;
      rc = ensure_stage(c, (size_t)n * 12);
      if (rc) return rc;
      HLBM_TRY(c, CNT(c, launch_real_to_f64)(c->d, real_is_double(c), c->stage, N, c->stream), "copy");
      break;
    }
    default:
      return set_err(c, HLBM_EINVAL, "unknown field");
  }
  return stage_out(c, out, dtype, on_device, n);
}

int hlbm_set_field(hlbm_ctx* c, int which, const void* data, int dtype, int on_device) {
  if (!c || !data) return HLBM_EINVAL;
  const long long N = c->g.N;
  const long long qN = (long long)c->q * N;
  int rc;
  if (which == HLBM_FIELD_F) {
    rc = stage_in(c, data, dtype, on_device, qN);
    if (rc) return rc;
    HLBM_TRY(c, CNT(c, launch_set_state)(c->f, c->g, c->q, c->storage, c->stage, c->stream), "set state");
    HLBM_TRY(c, cudaStreamSynchronize(c->stream), "sync");
    c->phase = 0;
    return HLBM_OK;
  }
  double* dst = nullptr;
  long long n = 0;
  int need_mask = 0;
  switch (which) {
    case HLBM_FIELD_FBAR: n = qN; break;
    case HLBM_FIELD_GBAR_FFA: n = qN; need_mask = 1; break;
    case HLBM_FIELD_GBAR_DISS: n = qN; need_mask = 2; break;
    case HLBM_FIELD_DJDD_FFA: n = N; need_mask = 1; break;
    case HLBM_FIELD_DJDD_DISS: n = N; need_mask = 2; break;
    case HLBM_FIELD_TAU_T: n = N; break;
    default: return set_err(c, HLBM_EINVAL, "field cannot be set");
  }
  rc = ensure_averages(c, need_mask | c->acc_mask);
  if (rc) return rc;
  if (which == HLBM_FIELD_FBAR && !c->fsum) {
    if (!(c->fsum = (double*)dalloc(c, (size_t)qN * 8))) return set_err(c, HLBM_ENOMEM, "fsum");
    HLBM_TRY(c, cudaMemsetAsync(c->fsum, 0, (size_t)qN * 8, c->stream), "memset");
  }
  // a set field defines a window of one sample: rescale existing sums
  if (c->nsamples > 1) {
    const double s = 1.0 / (double)c->nsamples;
    CNT(c, launch_scale)(c->msum, (long long)c->mplanes * N, s, c->stream);
    if (c->fsum) CNT(c, launch_scale)(c->fsum, qN, s, c->stream);
    CNT(c, launch_scale)(c->tsum, N, s, c->stream);
    for (int o = 0; o < 2; ++o) {
      if (!(c->acc_mask & (1 << o))) continue;
      CNT(c, launch_scale)(c->gsum[o], (long long)ncoef(o, c->D) * N, s, c->stream);
      CNT(c, launch_scale)(c->ddsum[o], N, s, c->stream);
      CNT(c, launch_scale)(c->jblk[o], c->njslot, s, c->stream);
    }
  }
  if (c->nsamples < 1) {
    // fresh window: clear everything first
    rc = reset_averages(c, need_mask | c->acc_mask);
    if (rc) return rc;
  }
  if (need_mask && !(c->acc_mask & need_mask)) {
    const int o = need_mask - 1;
    HLBM_TRY(c, cudaMemsetAsync(c->gsum[o], 0, coef_bytes(c, o), c->stream), "memset");
    HLBM_TRY(c, cudaMemsetAsync(c->ddsum[o], 0, (size_t)N * 8, c->stream), "memset");
    HLBM_TRY(c, cudaMemsetAsync(c->jblk[o], 0, (size_t)c->njslot * 8, c->stream), "memset");
    c->acc_mask |= need_mask;
  }
  rc = stage_in(c, data, dtype, on_device, n);
  if (rc) return rc;
  switch (which) {
    case HLBM_FIELD_FBAR:
      HLBM_TRY(c, CNT(c, launch_set_fbar)(c->stage, c->q, N, c->fsum, c->msum, c->rr, c->stream), "fbar");
      break;
    case HLBM_FIELD_GBAR_FFA:
    case HLBM_FIELD_GBAR_DISS: {
      const int o = which == HLBM_FIELD_GBAR_FFA ? 0 : 1;
      HLBM_TRY(c, CNT(c, launch_project_coef)(c->stage, c->pmat[o], o, c->q, N, c->gsum[o], c->stream), "project");
      break;
    }
    default:
      dst = which == HLBM_FIELD_DJDD_FFA ? c->ddsum[0]
            : which == HLBM_FIELD_DJDD_DISS ? c->ddsum[1] : c->tsum;
      HLBM_TRY(c, cudaMemcpyAsync(dst, c->stage, (size_t)n * 8, cudaMemcpyDeviceToDevice, c->stream), "copy");
  }
  HLBM_TRY(c, cudaStreamSynchronize(c->stream), "sync");
  c->nsamples = 1;
  c->generation++;
  c->have_adjoint = false;
  return HLBM_OK;
}

int hlbm_get_stats(const hlbm_ctx* c, hlbm_stats* out) {
  if (!c || !out) return HLBM_EINVAL;
  *out = c->stats;
  return HLBM_OK;
}

// checkpoint file: header, then the raw population array and the FP64 sums
struct CkptHeader {
  char magic[8];
  int q, storage, nx, ny, nz, phase, acc_mask, has_fsum, mplanes, pad;
  long long steps_done, nsamples;
};

int hlbm_save(hlbm_ctx* c, const char* path) {
  if (!c || !path) return HLBM_EINVAL;
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return set_err(c, HLBM_EINVAL, "cannot open %s", path);
  CkptHeader h{};
  std::memcpy(h.magic, "HLBMCK4", 8);
  h.has_fsum = c->fsum != nullptr;
  h.mplanes = c->mplanes;
  h.q = c->q; h.storage = c->storage; h.nx = c->g.nx; h.ny = c->g.ny; h.nz = c->g.nz;
  h.phase = c->phase; h.acc_mask = c->nsamples > 0 ? c->acc_mask : 0;
  h.steps_done = c->steps_done; h.nsamples = c->nsamples;
  std::fwrite(&h, sizeof h, 1, fp);
  auto dump = [&](const void* dptr, size_t bytes) -> int {
    const size_t chunk = 64u << 20;
    std::string buf;
    buf.resize(chunk);
    for (size_t off = 0; off < bytes; off += chunk) {
      size_t n = bytes - off < chunk ? bytes - off : chunk;
      if (cudaMemcpy(&buf[0], (const char*)dptr + off, n, cudaMemcpyDeviceToHost) != cudaSuccess) return HLBM_ECUDA;
      if (std::fwrite(buf.data(), 1, n, fp) != n) return HLBM_EINVAL;
    }
    return HLBM_OK;
  };
  cudaStreamSynchronize(c->stream);
  int rc = dump(c->f, (size_t)c->q * c->g.pitch * pop_elem_bytes(c->storage));
  if (!rc) rc = dump(c->d, (size_t)c->g.N * real_bytes(c));
  if (!rc && h.nsamples > 0) {
    rc = dump(c->msum, (size_t)c->mplanes * c->g.N * 8);
    if (!rc && h.has_fsum) rc = dump(c->fsum, (size_t)c->q * c->g.N * 8);
    if (!rc) rc = dump(c->tsum, (size_t)c->g.N * 8);
    for (int o = 0; o < 2 && !rc; ++o) {
      if (!(h.acc_mask & (1 << o))) continue;
      rc = dump(c->gsum[o], coef_bytes(c, o));
      if (!rc) rc = dump(c->ddsum[o], (size_t)c->g.N * 8);
      if (!rc) rc = dump(c->jblk[o], (size_t)c->njslot * 8);
    }
  }
  std::fclose(fp);
  if (rc) return set_err(c, rc, "checkpoint write failed");
  return HLBM_OK;
}

int hlbm_load(hlbm_ctx* c, const char* path) {
  if (!c || !path) return HLBM_EINVAL;
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return set_err(c, HLBM_EINVAL, "cannot open %s", path);
  CkptHeader h{};
  if (std::fread(&h, sizeof h, 1, fp) != 1 || std::memcmp(h.magic, "HLBMCK4", 8) != 0 ||
      h.q != c->q || h.storage != c->storage || h.nx != c->g.nx || h.ny != c->g.ny || h.nz != c->g.nz ||
      h.mplanes != c->mplanes) {
    std::fclose(fp);
    return set_err(c, HLBM_EINVAL, "checkpoint does not match this context");
  }
  auto load = [&](void* dptr, size_t bytes) -> int {
    const size_t chunk = 64u << 20;
    std::string buf;
    buf.resize(chunk);
    for (size_t off = 0; off < bytes; off += chunk) {
      size_t n = bytes - off < chunk ? bytes - off : chunk;
      if (std::fread(&buf[0], 1, n, fp) != n) return HLBM_EINVAL;
      if (cudaMemcpy((char*)dptr + off, buf.data(), n, cudaMemcpyHostToDevice) != cudaSuccess) return HLBM_ECUDA;
    }
    return HLBM_OK;
  };
  cudaStreamSynchronize(c->stream);
  int rc = load(c->f, (size_t)c->q * c->g.pitch * pop_elem_bytes(c->storage));
  if (!rc) rc = load(c->d, (size_t)c->g.N * real_bytes(c));
  if (!rc && h.nsamples > 0) {
    rc = ensure_averages(c, h.acc_mask);
    if (!rc) rc = load(c->msum, (size_t)c->mplanes * c->g.N * 8);
    if (!rc && h.has_fsum) {
      if (!c->fsum && !(c->fsum = (double*)dalloc(c, (size_t)c->q * c->g.N * 8))) rc = HLBM_ENOMEM;
      if (!rc) rc = load(c->fsum, (size_t)c->q * c->g.N * 8);
    }
    if (!rc) rc = load(c->tsum, (size_t)c->g.N * 8);
    for (int o = 0; o < 2 && !rc; ++o) {
      if (!(h.acc_mask & (1 << o))) continue;
      rc = load(c->gsum[o], coef_bytes(c, o));
      if (!rc) rc = load(c->ddsum[o], (size_t)c->g.N * 8);
      if (!rc) rc = load(c->jblk[o], (size_t)c->njslot * 8);
    }
  }
  std::fclose(fp);
  if (rc) return set_err(c, rc, "checkpoint read failed");
  c->phase = h.phase;
  c->steps_done = h.steps_done;
  c->nsamples = h.nsamples;
  c->acc_mask = h.acc_mask;
  c->generation++;
  c->have_adjoint = false;
  return HLBM_OK;
}

const char* hlbm_last_error(const hlbm_ctx* c) {
  if (!c) return "null context";
  return c->msg.c_str();
}

void hlbm_destroy(hlbm_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  dfree(c, c->f);
  dfree(c, c->d);
  if (c->inflow) dfree(c, c->inflow);
  dfree(c, c->msum);
  dfree(c, c->fsum);
  dfree(c, c->mstage);
  dfree(c, c->fstage);
  for (int o = 0; o < 2; ++o) {
    dfree(c, c->gstage[o]);
    dfree(c, c->ddstage[o]);
  }
  dfree(c, c->tsum);
  for (int o = 0; o < 2; ++o) {
    dfree(c, c->gsum[o]);
    dfree(c, c->ddsum[o]);
    dfree(c, c->jblk[o]);
  }
  dfree(c, c->lam);
  dfree(c, c->snap);
  dfree(c, c->rec);
  dfree(c, c->src);
  dfree(c, c->red);
  dfree(c, c->stage);
  dfree(c, c->fd);
  dfree(c, c->delta);
  dfree(c, c->jhist);
  dfree(c, c->kry);
  dfree(c, c->kpart);
  dfree(c, c->kdev);
  if (c->khost) cudaFreeHost(c->khost);
  if (c->err_dev) cudaFree(c->err_dev);
  if (c->err_host) cudaFreeHost(c->err_host);
  if (c->scal_dev) cudaFree(c->scal_dev);
  if (c->fin) cudaFree(c->fin);
  if (c->scal_host) cudaFreeHost(c->scal_host);
  for (auto& row : c->pgraph)
    for (auto& pg : row)
      if (pg.exec) cudaGraphExecDestroy(pg.exec);
  if (c->agraph.exec) cudaGraphExecDestroy(c->agraph.exec);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

// ---------------------------------------------------------------------------
// Batched stepping (the serving form)
// ---------------------------------------------------------------------------

struct hlbm_batch {
  int q = 9;
  cudaStream_t stream = nullptr;
  PrimalArgs* ptab = nullptr;   // device: one PrimalArgs per context
  AdjointArgs* atab = nullptr;  // device: one AdjointArgs per context
  int tab_n = 0;
  int4* tiles = nullptr;        // device work list: (context, x-block, y, z)
  long long tiles_n = 0;
  int4* tiles_host = nullptr;   // pinned copy
  long long tiles_host_n = 0;
  // captured graph of kGraphSteps batched primal steps, per (averaging pattern, phase)
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    int ntiles = 0;
  } pg[2][2];
  bool graphs_ok = true;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double last_ms = 0.0;
};

namespace {

void batch_drop_graphs(hlbm_batch* b) {
  // the captured graphs hold the pointers of the tables and the work list
  for (auto& row : b->pg)
    for (auto& g : row)
      if (g.exec) { cudaGraphExecDestroy(g.exec); g.exec = nullptr; }
}

int batch_tables(hlbm_batch* b, int n, long long ntiles) {
  if (b->tab_n < n) {
    batch_drop_graphs(b);
    if (b->ptab) cudaFree(b->ptab);
    if (b->atab) cudaFree(b->atab);
    b->ptab = nullptr;
    b->atab = nullptr;
    b->tab_n = 0;
    if (cudaMalloc(&b->ptab, sizeof(PrimalArgs) * n) != cudaSuccess ||
        cudaMalloc(&b->atab, sizeof(AdjointArgs) * n) != cudaSuccess) {
      cudaGetLastError();
      return HLBM_ENOMEM;
    }
    b->tab_n = n;
  }
  if (b->tiles_n < ntiles) {
    batch_drop_graphs(b);
    if (b->tiles) cudaFree(b->tiles);
    b->tiles = nullptr;
    b->tiles_n = 0;
    if (cudaMalloc(&b->tiles, sizeof(int4) * ntiles) != cudaSuccess) {
      cudaGetLastError();
      return HLBM_ENOMEM;
    }
    b->tiles_n = ntiles;
  }
  if (b->tiles_host_n < ntiles) {
    if (b->tiles_host) cudaFreeHost(b->tiles_host);
    b->tiles_host = nullptr;
    b->tiles_host_n = 0;
    if (cudaMallocHost(&b->tiles_host, sizeof(int4) * ntiles) != cudaSuccess) {
      cudaGetLastError();
      return HLBM_ENOMEM;
    }
    b->tiles_host_n = ntiles;
  }
  return HLBM_OK;
}

// the work list of contexts ctxs[idx[0..m)]: every NT-wide block of each
long long batch_tiles(hlbm_batch* b, hlbm_ctx* const* ctxs, const int* idx, int m) {
  long long t = 0;
  for (int j = 0; j < m; ++j) {
    const hlbm_ctx* c = ctxs[idx[j]];
    const int gx = (c->g.nx + NT - 1) / NT;
    for (int z = 0; z < c->g.nz; ++z)
      for (int y = 0; y < c->g.ny; ++y)
        for (int xb = 0; xb < gx; ++xb) b->tiles_host[t++] = make_int4(j, xb, y, z);
  }
  return t;
}

long long batch_count(hlbm_ctx* const* ctxs, int n) {
  long long t = 0;
  for (int k = 0; k < n; ++k) t += (long long)((ctxs[k]->g.nx + NT - 1) / NT) * ctxs[k]->g.ny * ctxs[k]->g.nz;
  return t;
}

// what a batch may hold: contexts of its lattice and stream, FP32 storage, BGK
// without the Smagorinsky model, NT-wide blocks, the same AA phase
int batch_check(hlbm_batch* b, hlbm_ctx* const* ctxs, int n) {
  if (!b || !ctxs || n < 1) return HLBM_EINVAL;
  for (int k = 0; k < n; ++k) {
    hlbm_ctx* c = ctxs[k];
    if (!c) return HLBM_EINVAL;
    if (c->q != b->q || c->stream != b->stream || c->storage != HLBM_FP32 || c->rr ||
        c->Cs != 0.0 || c->full_f || c->g.bx != NT || c->phase != ctxs[0]->phase ||
        c->opt.accum_stride != 1 || c->opt.adjoint_solver != 0)
      return set_err(c, HLBM_EINVAL,
                     "batched stepping needs contexts of the batch's lattice and stream, FP32 "
                     "storage, BGK with Cs = 0, compact averages, block_x 128, stride 1, the "
                     "fixed-point adjoint and the same AA phase");
  }
  return HLBM_OK;
}

}  // namespace

int hlbm_batch_create(hlbm_batch** out, int lattice, void* stream) {
  if (!out) return HLBM_EINVAL;
  *out = nullptr;
  if ((lattice != 9 && lattice != 19) || !stream) return HLBM_EINVAL;
  hlbm_batch* b = new hlbm_batch();
  b->q = lattice;
  b->stream = static_cast<cudaStream_t>(stream);
  if (cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess) {
    cudaGetLastError();
    hlbm_batch_destroy(b);
    return HLBM_ECUDA;
  }
  *out = b;
  return HLBM_OK;
}

int hlbm_batch_run_primal(hlbm_batch* b, hlbm_ctx* const* ctxs, int n, long steps, long W) {
  int rc = batch_check(b, ctxs, n);
  if (rc) return rc;
  if (steps < 0 || W < 0 || W > steps) return set_err(ctxs[0], HLBM_EINVAL, "need 0 <= avg_window <= steps");
  const long long ntiles = batch_count(ctxs, n);
  if (ntiles > 0x7fffffffLL) return set_err(ctxs[0], HLBM_EINVAL, "batch too large");
  rc = batch_tables(b, n, ntiles);
  if (rc) return set_err(ctxs[0], rc, "batch tables");
  for (int k = 0; k < n; ++k) {
    if (W > 0) {
      rc = reset_averages(ctxs[k], ctxs[k]->opt.objectives & 7);
      if (rc) return rc;
    }
  }
  std::vector<PrimalArgs> tab(n);
  std::vector<int> idx(n);
  for (int k = 0; k < n; ++k) {
    tab[k] = primal_args(ctxs[k]);
    idx[k] = k;
  }
  batch_tiles(b, ctxs, idx.data(), n);
  cudaStream_t s = b->stream;
  hlbm_ctx* c0 = ctxs[0];
  HLBM_TRY(c0, cudaMemcpyAsync(b->ptab, tab.data(), sizeof(PrimalArgs) * n, cudaMemcpyHostToDevice, s), "table");
  HLBM_TRY(c0, cudaMemcpyAsync(b->tiles, b->tiles_host, sizeof(int4) * ntiles, cudaMemcpyHostToDevice, s), "tiles");
  HLBM_TRY(c0, cudaEventRecord(b->ev0, s), "event");
  int phase = c0->phase;
  long launches = 0;
  const long first = steps - W;
  // a stretch of `count` steps of one pattern (plain, or averaging samples 0..count-1)
  auto stretch = [&](int acc_base, long count) -> int {
    long done = 0;
    auto& g = b->pg[acc_base ? 1 : 0][phase];
    if (b->graphs_ok && count >= kGraphSteps) {
      if (g.exec && g.ntiles != (int)ntiles) {
        cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
      }
      if (!g.exec) {
        cudaGraph_t graph = nullptr;
        bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        int ph = phase;
        for (long k = 0; ok && k < kGraphSteps; ++k) {
          ok = launch_primal_batch(b->ptab, b->tiles, (int)ntiles, b->q, ph == 1,
                                   step_variant(acc_base, k, kGraphSteps + 1), s) == cudaSuccess;
          ph ^= 1;
        }
        if (cudaStreamEndCapture(s, &graph) != cudaSuccess) ok = false;
        if (ok && cudaGraphInstantiate(&g.exec, graph, 0) != cudaSuccess) {
          ok = false;
          g.exec = nullptr;
        }
        if (graph) cudaGraphDestroy(graph);
        if (!ok) {
          cudaGetLastError();
          b->graphs_ok = false;
        } else {
          g.ntiles = (int)ntiles;
        }
      }
      if (g.exec) {
        for (; done + kGraphSteps <= count; done += kGraphSteps) {
          if (cudaGraphLaunch(g.exec, s) != cudaSuccess) return HLBM_ECUDA;
          launches += kGraphSteps;
        }
      }
    }
    for (; done < count; ++done) {
      if (launch_primal_batch(b->ptab, b->tiles, (int)ntiles, b->q, phase == 1,
                              step_variant(acc_base, done, count), s) != cudaSuccess)
        return HLBM_ECUDA;
      phase ^= 1;
      ++launches;
    }
    return HLBM_OK;
  };
  rc = stretch(0, first);
  if (rc == HLBM_OK && W > 0) rc = stretch(ACC_ON, W);
  if (rc) {
    cudaGetLastError();
    return set_err(c0, HLBM_ECUDA, "batched primal launch");
  }
  HLBM_TRY(c0, cudaEventRecord(b->ev1, s), "event");
  HLBM_TRY(c0, cudaEventSynchronize(b->ev1), "sync");
  float ms = 0;
  cudaEventElapsedTime(&ms, b->ev0, b->ev1);
  b->last_ms = ms;
  int status = HLBM_OK;
  for (int k = 0; k < n; ++k) {
    hlbm_ctx* c = ctxs[k];
    c->phase = phase;
    c->stats.primal_ms = ms;
    c->stats.primal_launches = launches;
    c->stats.primal_steps += steps;
    c->stats.kernels_total += launches;
    c->steps_done += steps;
    if (W > 0) {
      c->nsamples = W;
      c->generation++;
      c->have_adjoint = false;
    }
    unsigned err = 0;
    rc = read_err(c, &err);
    if (rc) return rc;
    if (err & 1u) status = set_err(c, HLBM_ENONFINITE, "primal state became non-finite");
  }
  return status;
}

int hlbm_batch_solve_adjoint(hlbm_batch* b, hlbm_ctx* const* ctxs, int n, const int* objectives,
                             int mode, double tol, long max_iter, long* iters_out,
                             double* residual_out, int* status_out) {
  int rc = batch_check(b, ctxs, n);
  if (rc) return rc;
  if (!objectives || !(tol >= 0) || max_iter < 2) return set_err(ctxs[0], HLBM_EINVAL, "bad tol, max_iter or objectives");
  const long long ntiles_all = batch_count(ctxs, n);
  if (ntiles_all > 0x7fffffffLL) return set_err(ctxs[0], HLBM_EINVAL, "batch too large");
  rc = batch_tables(b, n, ntiles_all);
  if (rc) return set_err(ctxs[0], rc, "batch tables");
  std::vector<AdjSetup> su(n);
  for (int k = 0; k < n; ++k) {
    hlbm_ctx* c = ctxs[k];
    if (c->nsamples < 1 || !(c->acc_mask & objectives[k]) || objectives[k] == HLBM_OBJ_DRAG_MEA)
      return set_err(c, HLBM_ESTATE, "run the primal with this objective averaged first (J_FFA or J_DISS)");
    rc = adjoint_setup(c, objectives[k], mode, &su[k]);
    if (rc) return rc;
    if (su[k].exact) return set_err(c, HLBM_EINVAL, "batched sweeps use the compact record");
  }
  std::vector<AdjointArgs> tab(n);
  for (int k = 0; k < n; ++k) tab[k] = su[k].a;
  cudaStream_t s = b->stream;
  hlbm_ctx* c0 = ctxs[0];
  HLBM_TRY(c0, cudaMemcpyAsync(b->atab, tab.data(), sizeof(AdjointArgs) * n, cudaMemcpyHostToDevice, s), "table");
  std::vector<int> active(n), status(n, HLBM_NOT_CONVERGED);
  std::vector<long> iters(n, 0);
  std::vector<double> r(n, INFINITY), rmin(n, INFINITY);
  for (int k = 0; k < n; ++k) active[k] = k;
  const long m = c0->opt.check_every;
  long k_done = 0, launches = 0;
  while (!active.empty() && k_done < max_iter) {
    // the work list of the contexts still iterating (table entries keep their index)
    long long t = 0;
    for (int k : active) {
      const hlbm_ctx* c = ctxs[k];
      const int gx = (c->g.nx + NT - 1) / NT;
      for (int z = 0; z < c->g.nz; ++z)
        for (int y = 0; y < c->g.ny; ++y)
          for (int xb = 0; xb < gx; ++xb) b->tiles_host[t++] = make_int4(k, xb, y, z);
    }
    HLBM_TRY(c0, cudaMemcpyAsync(b->tiles, b->tiles_host, sizeof(int4) * t, cudaMemcpyHostToDevice, s), "tiles");
    long chunk = max_iter - k_done < m ? max_iter - k_done : m;
    if (chunk & 1) chunk += 1;
    if (chunk < 2) chunk = 2;
    for (long j = 0; j < chunk; ++j) {
      const int res = j == chunk - 2 ? 1 : (j == chunk - 1 ? 2 : 0);
      if (launch_adjoint_batch(b->atab, b->tiles, (int)t, b->q, (j & 1) != 0, res, s) != cudaSuccess) {
        cudaGetLastError();
        return set_err(c0, HLBM_ECUDA, "batched adjoint launch");
      }
    }
    launches += chunk;
    k_done += chunk;
    for (int k : active) {
      hlbm_ctx* c = ctxs[k];
      HLBM_TRY(c, CNT(c, launch_finalize_sum)(c->red, su[k].nb_adj, c->scal_dev, c->fin, s), "reduce");
      HLBM_TRY(c, cudaMemcpyAsync(c->scal_host, c->scal_dev, 8, cudaMemcpyDeviceToHost, s), "copy");
    }
    HLBM_TRY(c0, cudaStreamSynchronize(s), "sync");
    std::vector<int> still;
    for (int k : active) {
      iters[k] = k_done;
      const double rk = std::sqrt(ctxs[k]->scal_host[0]) / su[k].gnorm;
      r[k] = rk;
      if (!std::isfinite(rk)) { status[k] = HLBM_ENONFINITE; continue; }
      if (rk < rmin[k]) rmin[k] = rk;
      if (rk <= tol) { status[k] = HLBM_OK; continue; }
      if (rk > 1e6 * rmin[k] && rmin[k] > 0) { status[k] = HLBM_EDIVERGED; continue; }
      still.push_back(k);
    }
    active.swap(still);
  }
  int worst = HLBM_OK;
  for (int k = 0; k < n; ++k) {
    hlbm_ctx* c = ctxs[k];
    c->stats.kernels_total += iters[k];
    const int st = adjoint_finish(c, objectives[k], mode, status[k], iters[k], iters[k], su[k].exact);
    if (iters_out) iters_out[k] = iters[k];
    if (residual_out) residual_out[k] = r[k];
    if (status_out) status_out[k] = st;
    if (st < 0 && worst >= 0) worst = st;
    else if (st == HLBM_NOT_CONVERGED && worst == HLBM_OK) worst = st;
  }
  (void)launches;
  return worst;
}

void hlbm_batch_destroy(hlbm_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->ptab) cudaFree(b->ptab);
  if (b->atab) cudaFree(b->atab);
  if (b->tiles) cudaFree(b->tiles);
  if (b->tiles_host) cudaFreeHost(b->tiles_host);
  for (auto& row : b->pg)
    for (auto& g : row)
      if (g.exec) cudaGraphExecDestroy(g.exec);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  delete b;
}

}  // extern "C"
