// C ABI of the coupled cathode step: domain lifetime, parameters, material
// palette, time stepping (with CUDA-graph replay) and read-outs.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <optional>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/pemlbm.h"
#include "lbm_core.cuh"
#include "lbm_launch.h"

using namespace pemlbm;

namespace {

thread_local std::string g_err;

lbm_status fail(lbm_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(LBM_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                          \
  } while (0)

// Host-side NVTX ranges around the library's calls and phases, for
// timelines (header-only NVTX: no cost without an attached tool).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// Host-side fault injection for tests of the ENOMEM paths: with
// PEMLBM_FAIL_ALLOC=n in the environment, the n-th allocation the library
// makes after the variable last changed fails as if memory were exhausted.
// Nothing reaches the device.
bool inject_alloc_failure() {
  static std::mutex mu;
  static std::string last;
  static long count = 0;
  const char *e = std::getenv("PEMLBM_FAIL_ALLOC");
  const std::string cur = e ? e : "";
  std::lock_guard<std::mutex> lock(mu);
  if (cur != last) {
    last = cur;
    count = 0;
  }
  if (cur.empty()) return false;
  return ++count == std::atol(cur.c_str());
}
template <typename T> cudaError_t dmalloc(T **p, size_t bytes) {
  if (inject_alloc_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc((void **)p, bytes);
}
template <typename T> cudaError_t hmalloc(T **p, size_t bytes) {
  if (inject_alloc_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocHost((void **)p, bytes);
}

constexpr int kGraphSteps = 64;   // even: a replay returns to the same buffer
constexpr int kMaxPalette = 65535;

size_t elem_size(int prec) {
  switch (prec) {
    case LBM_FP64: return 8;
    case LBM_FP32: return 4;
    default: return 2;
  }
}

}  // namespace

struct lbm_domain {
  lbm_domain_desc desc{};
  lbm_params prm{};
  bool have_params = false, have_fields = false, have_state = false;
  int nx = 0, ny = 0, nxp = 0;
  long long plane = 0;
  size_t esize = 4;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void *pop[2] = {nullptr, nullptr};
  int cur = 0;                 // buffer holding the latest state
  int64_t steps = 0;
  uint8_t *mask = nullptr;    // [2][ny][nxp]: node bits, then solid-neighbour bits
  uint16_t *mid = nullptr;
  void *pal = nullptr;
  MatRaw *raw = nullptr;
  int npal = 0;
  std::vector<MatRaw> hraw;    // host copy of the palette's raw tuples
  int ref_entry = 0;           // palette entry of the reference cell
  void *snap = nullptr;        // two residual snapshots [2][5][ny][nx], arithmetic precision
  int snap_cur = 0;            // the one the next lbm_residual compares with
  double *partial = nullptr;   // residual block partials [blocks][10]
  double *colsum = nullptr;    // catalyst column sums [2][nx]
  int variant = 0;             // launch shape of the step kernel (lbm_tune picks one)
  int64_t grad_mem_limit = -1; // device bytes lbm_grad may keep records in (-1: what is free)
  double tuned_ms[kStepVariants] = {};
  double *dsmall = nullptr;    // device results (16 doubles)
  int *dbad = nullptr;
  unsigned *dseed = nullptr;   // step counter seeding stochastic 16-bit rounding
  double *hsmall = nullptr;    // pinned host mirror
  double *scratch = nullptr;   // [24][ny][nx] doubles, lazily allocated
  void *pal_scratch = nullptr; // device palette build's work space, allocated at its first use
  float *dprofile = nullptr;   // [nx]
  // references of the deviation storage: part of the state's representation,
  // so they change only at reset (or with a loaded state)
  double Cref[3] = {0, 0, 0}, bref[3] = {0, 0, 0};
  double bref_next[3] = {0, 0, 0};   // reference b the next reset will use
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // observed stepping: per-step (J, heat) sums in device slots [2][64][2],
  // copied every step into pinned host slots of the same shape; one graph
  // per (starting buffer, slot half)
  double *dobs = nullptr, *hobs = nullptr;
  cudaGraphExec_t obs_graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  cudaEvent_t obs_done[2] = {nullptr, nullptr};
  cudaStream_t obs_side = nullptr;             // the reductions, beside the steps
  cudaEvent_t obs_fork = nullptr, obs_join = nullptr;
  // x-slab of a larger lattice: columns [x0, x0 + nx) of nxg; a side that
  // borders a neighbour slab reads the ghost column the exchange fills
  int x0 = 0, nxg = 0;
  bool halo_lo = false, halo_hi = false;
  std::vector<uint8_t> hsolid;                 // the whole lattice's solids (slabs)
  cudaEvent_t ev_halo = nullptr;
};

namespace {

bool fp64(const lbm_domain *d) { return d->desc.precision == LBM_FP64; }

KArgs make_args(const lbm_domain *d) {
  const lbm_params &p = d->prm;
  KArgs a{};
  a.nx = d->nx;
  a.ny = d->ny;
  a.nxp = d->nxp;
  a.periodic = d->desc.periodic_x;
  a.plane = d->plane;
  a.mode = d->desc.reaction_mode;
  a.ny_cl = d->desc.ny_cl;
  a.y_ch0 = d->desc.ny_cl + d->desc.ny_gdl;
  a.top_dirichlet = p.top_dirichlet;
  const double tau = 3.0 * p.nu + 0.5;
  a.s_nu = 1.0 / tau;
  a.s_q = 8.0 * (2.0 - 1.0 / tau) / (8.0 - 1.0 / tau);
  a.stochastic = d->desc.rounding == 1;
  a.seed_ctr = d->dseed;
  a.body_g = p.body_force_x;
  a.gam_x = p.buoy_gx;
  a.gam_y = p.buoy_gy;
  a.buoy_off = d->Cref[0] - p.T_buoy;
  a.closed_x = d->desc.closed_x;
  a.halo_lo = d->halo_lo;
  a.halo_hi = d->halo_hi;
  a.wall_dir = p.wall_dirichlet;
  a.npal = d->npal;
  for (int k = 0; k < 3; ++k)
    for (int s = 0; s < 3; ++s) a.Cwall[k][s] = p.C_wall[k][s];
  a.u_in_avg = p.inlet_mode == 0 ? p.u_in_avg : 0.0;
  a.inlet_pressure = p.inlet_mode == 1;
  a.dp_in = p.inlet_mode == 1 ? p.dp_in : 0.0;
  a.h_ch = d->ny - a.y_ch0;
  a.Q3 = 6.0 / (3.0 + 2.0 * std::sqrt(3.0));
  const double Cin[3] = {p.T_in, p.C_O2_in, p.C_H2O_in};
  const double Ctop[3] = {p.T_top, p.C_O2_top, p.C_H2O_top};
  for (int s = 0; s < 3; ++s) {
    a.Cref[s] = d->Cref[s];
    a.bref[s] = d->bref[s];
    a.wr0[s] = (1.0 - d->bref[s]) / 5.0;
    a.wr1[s] = (4.0 + d->bref[s]) / 20.0;
    a.Cin[s] = Cin[s];
    a.Ctop[s] = Ctop[s];
    a.adv_off[s] = d->Cref[s] - (p.scalar_advection ? Cin[s] : 0.0);
  }
  // Tafel rate (Eq. 13, 14, 16, 17) per unit O2 mole fraction:
  //   k(T) = A exp(-E (1/T - 1/T_ref) + alpha_c F (U0(T) - V)/(R T))
  //        = A exp(c0 + c1/T),  c0 = E/T_ref + alpha_c F dU0dT / R,
  //                             c1 = -E + alpha_c F (U0_0 - V)/R,
  // written around T_in: k = A exp(e_in - c1 (T - T_in)/(T T_in)).
  const double four_F_c = 4.0 * p.F * p.c_tot;
  a.kA_surf = p.aj0_ref * p.delta_cl_cm / (p.x_ref * four_F_c) * p.dt_s / p.dx_cm;
  a.kA_vol = p.aj0_ref / (p.x_ref * four_F_c) * p.dt_s;
  const double c0 = p.E_act / p.T_ref_kin + p.alpha_c * p.F * p.dU0dT / p.R;
  const double c1 = -p.E_act + p.alpha_c * p.F * (p.U0_0 - p.V_op) / p.R;
  a.k_ein = c0 + c1 / p.T_in;
  a.k_c1 = c1;
  // Butler-Volmer anodic branch (zero in the Tafel case): the O2 produced
  // per step, k_a(T) = A x_ref exp(e_in_a - c1_a (T - T_in)/(T T_in)) with
  //   c0_a = E/T_ref - alpha_a F dU0dT / R,  c1_a = -E + alpha_a F (V - U0_0)/R.
  if (p.alpha_a > 0.0) {
    const double c0a = p.E_act / p.T_ref_kin - p.alpha_a * p.F * p.dU0dT / p.R;
    const double c1a = -p.E_act + p.alpha_a * p.F * (p.V_op - p.U0_0) / p.R;
    a.kA_surf_a = a.kA_surf * p.x_ref;
    a.kA_vol_a = a.kA_vol * p.x_ref;
    a.k_ein_a = c0a + c1a / p.T_in;
    a.k_c1_a = c1a;
  } else {
    a.kA_surf_a = a.kA_vol_a = a.k_ein_a = a.k_c1_a = 0.0;
  }
  a.T_in = p.T_in;
  a.theta0 = d->Cref[0] - p.T_in;
  // Eq. 15 with Eq. 16: eta + T dU0/dT = V - U0_0, so the heat per O2
  // consumed does not depend on T.
  a.hpo = four_F_c * (p.V_op - p.U0_0) / p.rho_cp_f;
  return a;
}

DevGeom geom(const lbm_domain *d) { return DevGeom{d->mask, d->mid, d->pal}; }

template <typename F>
void dispatch(int prec, F &&f) {
  switch (prec) {
    case LBM_FP64: f((double *)nullptr); break;
    case LBM_FP32: f((float *)nullptr); break;
    case LBM_BF16: f((__nv_bfloat16 *)nullptr); break;
    default: f((__half *)nullptr); break;
  }
}

void drop_graphs(lbm_domain *d) {
  for (auto &g : d->graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  for (auto &row : d->obs_graph)
    for (auto &g : row)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
}

lbm_status launch_steps(lbm_domain *d, int64_t n) {
  const KArgs a = make_args(d);
  const DevGeom g = geom(d);
  for (int64_t k = 0; k < n; ++k) {
    dispatch(d->desc.precision, [&](auto *tag) {
      using S = std::remove_pointer_t<decltype(tag)>;
      launch_step<S>(d->pop[d->cur], d->pop[d->cur ^ 1], g, a, d->variant, d->stream);
    });
    if (a.stochastic) launch_seed_advance(d->dseed, d->stream);
    d->cur ^= 1;
  }
  CK(cudaGetLastError());
  return LBM_OK;
}

lbm_status ensure_graph(lbm_domain *d) {
  if (d->graph[d->cur]) return LBM_OK;
  const int start = d->cur;
  cudaGraph_t gr = nullptr;
  CK(cudaStreamBeginCapture(d->stream, cudaStreamCaptureModeThreadLocal));
  lbm_status s = launch_steps(d, kGraphSteps);
  cudaError_t e = cudaStreamEndCapture(d->stream, &gr);
  d->cur = start;
  if (s != LBM_OK) return s;
  if (e != cudaSuccess) return fail(LBM_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&d->graph[start], gr, 0);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) return fail(LBM_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  return LBM_OK;
}

// Observed steps: n steps (n <= kGraphSteps).  The reaction of a step is a
// function of the state it starts from, so its catalyst reduction (into
// device slot half `half`) and the asynchronous copy of its (J, heat) sums
// to the pinned host slots run on the side stream concurrently with the
// step itself; the next step, which overwrites that state, waits for them.
lbm_status launch_observed(lbm_domain *d, int64_t n, int half) {
  const KArgs a = make_args(d);
  const lbm_params &p = d->prm;
  const double i_scale = 4.0 * p.F * p.c_tot * p.dx_cm / p.dt_s;
  for (int64_t k = 0; k < n; ++k) {
    if (k > 0) CK(cudaStreamWaitEvent(d->stream, d->obs_join, 0));
    CK(cudaEventRecord(d->obs_fork, d->stream));
    CK(cudaStreamWaitEvent(d->obs_side, d->obs_fork, 0));
    const size_t slot = ((size_t)half * kGraphSteps + (size_t)k) * 2;
    dispatch(d->desc.precision, [&](auto *tag) {
      using S = std::remove_pointer_t<decltype(tag)>;
      launch_catalyst<S>(d->pop[d->cur], geom(d), a, i_scale, nullptr, d->colsum,
                         d->dobs + slot, d->obs_side);
    });
    CK(cudaMemcpyAsync(d->hobs + slot, d->dobs + slot, 2 * sizeof(double),
                       cudaMemcpyDeviceToHost, d->obs_side));
    CK(cudaEventRecord(d->obs_join, d->obs_side));
    lbm_status s = launch_steps(d, 1);
    if (s != LBM_OK) return s;
  }
  if (n > 0) CK(cudaStreamWaitEvent(d->stream, d->obs_join, 0));
  CK(cudaGetLastError());
  return LBM_OK;
}

lbm_status ensure_obs_graph(lbm_domain *d, int half) {
  cudaGraphExec_t &ge = d->obs_graph[d->cur][half];
  if (ge) return LBM_OK;
  const int start = d->cur;
  cudaGraph_t gr = nullptr;
  CK(cudaStreamBeginCapture(d->stream, cudaStreamCaptureModeThreadLocal));
  lbm_status s = launch_observed(d, kGraphSteps, half);
  cudaError_t e = cudaStreamEndCapture(d->stream, &gr);
  d->cur = start;
  if (s != LBM_OK) return s;
  if (e != cudaSuccess) return fail(LBM_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiateWithFlags(&ge, gr, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) return fail(LBM_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  return LBM_OK;
}

lbm_status ensure_scratch(lbm_domain *d) {
  if (!d->scratch && dmalloc(&d->scratch, sizeof(double) * 24 * (size_t)d->nx * d->ny) != cudaSuccess) {
    cudaGetLastError();
    return fail(LBM_ENOMEM, "read-out scratch of %.1f MB", 192.0 * d->nx * d->ny / 1e6);
  }
  return LBM_OK;
}

// Derives the palette coefficients for the current parameters and the
// deviation-storage reference b of each scalar.
lbm_status prep_palette(lbm_domain *d) {
  ScalarMode mode{};
  mode.fickian = d->prm.interface_mode == 1;
  for (const MatRaw &r : d->hraw)
    for (int s = 0; s < 3; ++s) mode.alpha_max[s] = std::fmax(mode.alpha_max[s], r.alpha[s]);
  launch_prep_palette(d->pal, d->raw, d->npal, d->prm.nu, d->prm.forchheimer, mode, fp64(d),
                      d->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(d->stream));
  const MatRaw &r = d->hraw[d->ref_entry];
  for (int s = 0; s < 3; ++s)
    d->bref_next[s] = 20.0 * std::sqrt(3.0) * (mode.fickian ? mode.alpha_max[s] : r.alpha[s]) - 4.0;
  return LBM_OK;
}

struct TupleHash {
  size_t operator()(const MatRaw &r) const {
    const double v[6] = {r.phi, r.K, r.alpha[0], r.alpha[1], r.alpha[2], r.sigma};
    size_t h = 1469598103934665603ull;
    for (double x : v) {
      uint64_t b;
      std::memcpy(&b, &x, 8);
      h = (h ^ b) * 1099511628211ull;
      h ^= h >> 29;
    }
    return h;
  }
};
struct TupleEq {
  bool operator()(const MatRaw &a, const MatRaw &b) const {
    return a.phi == b.phi && a.K == b.K && a.alpha[0] == b.alpha[0] && a.alpha[1] == b.alpha[1] &&
           a.alpha[2] == b.alpha[2] && a.sigma == b.sigma;
  }
};

lbm_status check_ready(lbm_domain *d) {
  if (!d) return fail(LBM_EINVAL, "null domain");
  if (!d->have_params || !d->have_fields || !d->have_state)
    return fail(LBM_ESTATE, "call lbm_set_params, lbm_set_fields and lbm_reset first");
  return LBM_OK;
}

}  // namespace

extern "C" {

const char *lbm_last_error(void) { return g_err.c_str(); }

lbm_status lbm_create_domain(const lbm_domain_desc *desc, lbm_domain **out) {
  if (!desc || !out) return fail(LBM_EINVAL, "null argument");
  *out = nullptr;
  const lbm_domain_desc &D = *desc;
  if (D.nx < 4 || D.ny < 3) return fail(LBM_EINVAL, "lattice must be at least 4 x 3 (got %d x %d)", D.nx, D.ny);
  if ((long long)D.nx * D.ny > (1LL << 31)) return fail(LBM_EINVAL, "lattice too large");
  if (D.rounding != 0 && D.rounding != 1) return fail(LBM_EINVAL, "rounding must be 0 or 1");
  if (D.rounding == 1 && D.precision != LBM_BF16 && D.precision != LBM_FP16)
    return fail(LBM_EINVAL, "stochastic rounding applies to BF16/FP16 storage only");
  if (D.precision < LBM_FP64 || D.precision > LBM_FP16) return fail(LBM_EINVAL, "bad precision %d", D.precision);
  if (D.reaction_mode != 0 && D.reaction_mode != 1) return fail(LBM_EINVAL, "reaction_mode must be 0 or 1");
  if (D.reaction_mode == 0 && D.ny_cl != 0) return fail(LBM_EINVAL, "thin-film mode takes ny_cl = 0");
  if (D.reaction_mode == 1 && D.ny_cl < 1) return fail(LBM_EINVAL, "volumetric mode needs ny_cl >= 1");
  if (D.periodic_x != 0 && D.periodic_x != 1) return fail(LBM_EINVAL, "periodic_x must be 0 or 1");
  if (D.closed_x != 0 && D.closed_x != 1) return fail(LBM_EINVAL, "closed_x must be 0 or 1");
  if (D.closed_x && D.periodic_x) return fail(LBM_EINVAL, "closed_x excludes periodic_x");
  if (D.ny_cl < 0 || D.ny_gdl < 0 ||
      D.ny_cl + D.ny_gdl > D.ny - ((D.periodic_x || D.closed_x) ? 0 : 1))
    return fail(LBM_EINVAL, "row split leaves no channel rows");
  if (D.solid && !D.periodic_x) {
    for (int y = 0; y < D.ny; ++y)
      for (int x : {0, D.nx - 2, D.nx - 1})
        if (D.solid[(size_t)y * D.nx + x]) return fail(LBM_EINVAL, "solid cell on an end column x=%d", x);
  }
  const bool slab = D.x_begin != 0 || D.x_end != 0;
  if (slab) {
    if (!(D.x_begin >= 0 && D.x_begin < D.x_end && D.x_end <= D.nx))
      return fail(LBM_EINVAL, "slab [%d, %d) outside the lattice of %d columns", D.x_begin, D.x_end, D.nx);
    if (D.x_end - D.x_begin < 4) return fail(LBM_EINVAL, "a slab needs at least 4 columns");
    if (D.periodic_x) return fail(LBM_EINVAL, "x-slabs of a periodic lattice are not supported");
  }
  lbm_domain *d = new lbm_domain();
  d->desc = D;
  d->desc.solid = nullptr;
  d->x0 = slab ? D.x_begin : 0;
  d->nxg = D.nx;
  d->nx = slab ? D.x_end - D.x_begin : D.nx;
  d->halo_lo = slab && D.x_begin > 0;
  d->halo_hi = slab && D.x_end < D.nx;
  if (slab && D.solid) d->hsolid.assign(D.solid, D.solid + (size_t)D.nx * D.ny);
  d->ny = D.ny;
  const int align = 64;   // 128-byte rows for every storage type
  // a slab side's ghost column lives in the row padding: x = nx on the high
  // side, x = nxp - 1 of the row below on the low side (two spare columns)
  const int need = d->nx + ((d->halo_lo || d->halo_hi) ? 2 : 0);
  d->nxp = (need + align - 1) / align * align;
  d->plane = (long long)d->nxp * D.ny;
  d->esize = elem_size(D.precision);
  // untuned default: 64 x 2 cells at 8 blocks per SM for FP32 storage (the
  // tuner's usual choice at large sizes), the uncapped 128 x 2 otherwise
  d->variant = D.precision == LBM_FP32 ? 7 : 0;
  auto cleanup = [&](lbm_status s) { lbm_destroy_domain(d); return s; };
  if (D.cuda_stream) {
    d->stream = (cudaStream_t)D.cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&d->stream, cudaStreamNonBlocking) != cudaSuccess)
      return cleanup(fail(LBM_ECUDA, "cudaStreamCreate failed"));
    d->own_stream = true;
  }
  // the step kernel loads every cell's interior pulls unconditionally; the
  // guard after the last plane keeps the top row's upward pulls in bounds
  const size_t pop_bytes = (24 * (size_t)d->plane + d->nxp + 64) * d->esize;
  const size_t cells = (size_t)d->plane;
  const size_t coef = fp64(d) ? sizeof(MatCoef<double>) : sizeof(MatCoef<float>);
  const size_t rsize = fp64(d) ? 8 : 4;
  if (dmalloc(&d->pop[0], pop_bytes) != cudaSuccess || dmalloc(&d->pop[1], pop_bytes) != cudaSuccess ||
      dmalloc(&d->mask, 2 * cells) != cudaSuccess || dmalloc(&d->mid, cells * 2) != cudaSuccess ||
      dmalloc(&d->pal, coef * kMaxPalette) != cudaSuccess ||
      dmalloc(&d->raw, sizeof(MatRaw) * kMaxPalette) != cudaSuccess ||
      dmalloc(&d->snap, 2 * rsize * 5 * (size_t)d->nx * D.ny) != cudaSuccess ||
      dmalloc(&d->partial, sizeof(double) * 10 * residual_blocks(d->nx, D.ny)) != cudaSuccess ||
      dmalloc(&d->colsum, sizeof(double) * 2 * d->nx) != cudaSuccess ||
      dmalloc(&d->dsmall, sizeof(double) * 16) != cudaSuccess || dmalloc(&d->dbad, sizeof(int)) != cudaSuccess ||
      dmalloc(&d->dseed, 256) != cudaSuccess ||
      dmalloc(&d->dprofile, sizeof(float) * d->nx) != cudaSuccess ||
      hmalloc(&d->hsmall, sizeof(double) * 16) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(fail(LBM_ENOMEM, "device allocation of %.1f MB failed", 2.0 * pop_bytes / 1e6));
  }
  if (cudaEventCreate(&d->ev0) != cudaSuccess || cudaEventCreate(&d->ev1) != cudaSuccess)
    return cleanup(fail(LBM_ECUDA, "cudaEventCreate failed"));
  uint8_t *dsolid = nullptr;
  if (D.solid) {
    if (dmalloc(&dsolid, (size_t)D.nx * D.ny) != cudaSuccess) return cleanup(fail(LBM_ENOMEM, "solid mask"));
    cudaMemcpyAsync(dsolid, D.solid, (size_t)D.nx * D.ny, cudaMemcpyHostToDevice, d->stream);
  }
  cudaMemsetAsync(d->mid, 0, cells * 2, d->stream);
  cudaMemsetAsync(d->pop[0], 0, pop_bytes, d->stream);
  cudaMemsetAsync(d->pop[1], 0, pop_bytes, d->stream);
  launch_build_mask(d->mask, dsolid, d->nx, D.ny, d->nxp, D.ny_cl, D.ny_gdl, D.reaction_mode,
                    D.periodic_x, D.closed_x, d->x0, D.nx, d->stream);
  cudaError_t e = cudaStreamSynchronize(d->stream);
  if (dsolid) cudaFree(dsolid);
  if (e != cudaSuccess) return cleanup(fail(LBM_ECUDA, "mask build: %s", cudaGetErrorString(e)));
  *out = d;
  return LBM_OK;
}

lbm_status lbm_destroy_domain(lbm_domain *d) {
  if (!d) return LBM_OK;
  if (d->stream) cudaStreamSynchronize(d->stream);
  drop_graphs(d);
  for (void *p : {d->pop[0], d->pop[1], (void *)d->mask, (void *)d->mid, d->pal, (void *)d->raw,
                  d->snap, (void *)d->partial, (void *)d->colsum, (void *)d->dsmall, (void *)d->dbad, (void *)d->dseed,
                  (void *)d->scratch, (void *)d->dprofile, (void *)d->dobs, d->pal_scratch})
    if (p) cudaFree(p);
  if (d->hsmall) cudaFreeHost(d->hsmall);
  if (d->hobs) cudaFreeHost(d->hobs);
  for (auto e : {d->obs_done[0], d->obs_done[1], d->obs_fork, d->obs_join})
    if (e) cudaEventDestroy(e);
  if (d->obs_side) cudaStreamDestroy(d->obs_side);
  if (d->ev0) cudaEventDestroy(d->ev0);
  if (d->ev1) cudaEventDestroy(d->ev1);
  if (d->ev_halo) cudaEventDestroy(d->ev_halo);
  if (d->own_stream && d->stream) cudaStreamDestroy(d->stream);
  delete d;
  return LBM_OK;
}

lbm_status lbm_set_params(lbm_domain *d, const lbm_params *p) {
  if (!d || !p) return fail(LBM_EINVAL, "null argument");
  if (!(p->nu > 0)) return fail(LBM_EINVAL, "nu must be > 0");
  if (p->inlet_mode != 0 && p->inlet_mode != 1) return fail(LBM_EINVAL, "inlet_mode must be 0 or 1");
  if (p->inlet_mode == 0 && !(std::sqrt(3.0) * 1.5 * std::fabs(p->u_in_avg) < 0.3))
    return fail(LBM_EINVAL, "inlet Mach number too high (u_in_avg = %g)", p->u_in_avg);
  if (!(p->alpha_a >= 0.0 && p->alpha_a <= 4.0))
    return fail(LBM_EINVAL, "anodic transfer coefficient alpha_a = %g outside [0, 4]", p->alpha_a);
  if (p->inlet_mode == 1 && !(std::fabs(p->dp_in) < 0.01))
    return fail(LBM_EINVAL, "inlet pressure excess |dp_in| = %g not below 0.01", p->dp_in);
  if (!(p->T_in > 0) || !(p->dx_cm > 0) || !(p->dt_s > 0) || !(p->c_tot > 0) || !(p->rho_cp_f > 0) ||
      !(p->x_ref > 0) || !(p->R > 0) || !(p->F > 0) || !(p->T_ref_kin > 0) || !(p->aj0_ref >= 0))
    return fail(LBM_EINVAL, "non-positive physical constant");
  if (p->interface_mode != 0 && p->interface_mode != 1) return fail(LBM_EINVAL, "interface_mode must be 0 or 1");
  if (p->scalar_advection != 0 && p->scalar_advection != 1)
    return fail(LBM_EINVAL, "scalar_advection must be 0 or 1");
  if (p->wall_dirichlet & ~0x1ff) return fail(LBM_EINVAL, "wall_dirichlet has bits beyond 8");
  if ((p->wall_dirichlet & 0x38) && !d->desc.closed_x)
    return fail(LBM_EINVAL, "fixed values on the x = nx - 1 wall need closed_x");
  if ((p->wall_dirichlet & 0x180) && d->desc.reaction_mode == 0)
    return fail(LBM_EINVAL, "the thin film owns the bottom's O2 and H2O links");
  if (!std::isfinite(p->buoy_gx) || !std::isfinite(p->buoy_gy) || !std::isfinite(p->T_buoy))
    return fail(LBM_EINVAL, "buoyancy must be finite");
  if (d->desc.rounding == 1 && (d->desc.closed_x || p->wall_dirichlet || p->buoy_gx != 0.0 ||
                                p->buoy_gy != 0.0))
    return fail(LBM_EINVAL, "stochastic rounding is not combined with closed_x, buoyancy or "
                "fixed wall values");
  const bool reprep = d->have_fields && (p->nu != d->prm.nu || p->forchheimer != d->prm.forchheimer ||
                                         p->interface_mode != d->prm.interface_mode);
  d->prm = *p;
  d->have_params = true;
  drop_graphs(d);
  if (reprep) return prep_palette(d);
  return LBM_OK;
}

// EINVAL with a message unless the material tuple of cell (x, y) lies in the
// ranges lbm_set_fields accepts.
lbm_status check_tuple(const MatRaw &t, int x, int y) {
  const double amax = 5.0 / (20.0 * std::sqrt(3.0));
  if (!(t.phi > 0 && t.phi <= 1)) return fail(LBM_EINVAL, "porosity %g at (%d,%d) outside (0,1]", t.phi, x, y);
  if (!(t.K > 0)) return fail(LBM_EINVAL, "permeability %g at (%d,%d) must be > 0", t.K, x, y);
  if (!(t.sigma >= 1e-6) || std::isinf(t.sigma))
    return fail(LBM_EINVAL, "heat-capacity ratio %g at (%d,%d) must be finite and >= 1e-6", t.sigma, x, y);
  for (int s = 0; s < 3; ++s)
    if (!(t.alpha[s] > 0 && t.alpha[s] <= amax))
      return fail(LBM_EINVAL, "diffusivity %g at (%d,%d) outside (0, %g]", t.alpha[s], x, y, amax);
  return LBM_OK;
}

// Palette of device-resident fields: built by the palette kernels into
// scratch first, so that a refused set leaves the domain's material as it
// was; only the palette itself (at most 65535 tuples) comes to the host.
lbm_status set_fields_device(lbm_domain *d, const double *phi, const double *K,
                             const double *alpha_T, const double *D_O2, const double *D_H2O,
                             const double *rho_cp_ratio) {
  const int nx = d->nx, ny = d->ny;
  const size_t mid_bytes = sizeof(uint16_t) * (size_t)d->plane;
  const size_t raw_bytes = sizeof(MatRaw) * kMaxPalette;
  const size_t work = palette_scratch_bytes(nx, ny);
  const size_t off_mid = (work + 255) / 256 * 256, off_raw = (off_mid + mid_bytes + 255) / 256 * 256,
               off_st = (off_raw + raw_bytes + 255) / 256 * 256;
  // kept for later calls (freeing it would synchronise the device each time)
  if (!d->pal_scratch && dmalloc(&d->pal_scratch, off_st + sizeof(PalStatus)) != cudaSuccess) {
    d->pal_scratch = nullptr;
    cudaGetLastError();
    return fail(LBM_ENOMEM, "palette scratch of %.1f MB", (off_st + 256) / 1e6);
  }
  char *base = (char *)d->pal_scratch;
  uint16_t *mid = (uint16_t *)(base + off_mid);
  MatRaw *raw = (MatRaw *)(base + off_raw);
  PalStatus *st = (PalStatus *)(base + off_st);
  const PalFields f{phi, K, alpha_T, D_O2, D_H2O, rho_cp_ratio};
  CK(launch_device_palette(f, d->mask, nx, ny, d->nxp, mid, raw, kMaxPalette, d->pal_scratch, st,
                           d->stream));
  PalStatus h{};
  CK(cudaMemcpyAsync(&h, st, sizeof h, cudaMemcpyDeviceToHost, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  if (h.flags & kPalInvalid) {
    // the first invalid cell in row-major order, for the message
    const int x = h.bad_cell % nx, y = h.bad_cell / nx;
    MatRaw t{};
    t.sigma = 1.0;
    const double *src[6] = {phi, K, alpha_T, D_O2, D_H2O, rho_cp_ratio};
    double *dst[6] = {&t.phi, &t.K, &t.alpha[0], &t.alpha[1], &t.alpha[2], &t.sigma};
    for (int k = 0; k < 6; ++k)
      if (src[k]) CK(cudaMemcpy(dst[k], src[k] + h.bad_cell, sizeof(double), cudaMemcpyDeviceToHost));
    lbm_status s = check_tuple(t, x, y);
    return s != LBM_OK ? s : fail(LBM_EINVAL, "invalid material at (%d,%d)", x, y);
  }
  if ((h.flags & kPalTooMany) || h.npal > kMaxPalette)
    return fail(LBM_EINVAL, "more than %d distinct materials", kMaxPalette);
  if (h.flags & kPalCollision) return fail(LBM_ECUDA, "material hash collision in the palette build");
  if (h.npal == 0) return fail(LBM_EINVAL, "no fluid cells");
  std::vector<MatRaw> hraw((size_t)h.npal);
  CK(cudaMemcpyAsync(hraw.data(), raw, sizeof(MatRaw) * hraw.size(), cudaMemcpyDeviceToHost, d->stream));
  // reference material: the top fluid cell of the inlet column, as the host build
  std::vector<uint8_t> col_mask((size_t)ny);
  std::vector<uint16_t> col_mid((size_t)ny);
  CK(cudaMemcpy2DAsync(col_mask.data(), 1, d->mask, d->nxp, 1, ny, cudaMemcpyDeviceToHost, d->stream));
  CK(cudaMemcpy2DAsync(col_mid.data(), 2, mid, 2 * (size_t)d->nxp, 2, ny, cudaMemcpyDeviceToHost, d->stream));
  CK(cudaMemcpyAsync(d->raw, raw, sizeof(MatRaw) * hraw.size(), cudaMemcpyDeviceToDevice, d->stream));
  CK(cudaMemcpyAsync(d->mid, mid, mid_bytes, cudaMemcpyDeviceToDevice, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  d->npal = h.npal;
  d->ref_entry = 0;
  for (int y = ny - 1; y >= 0; --y)
    if ((col_mask[y] & REG_MASK) != REG_SOLID) {
      d->ref_entry = col_mid[y];
      break;
    }
  d->hraw = std::move(hraw);
  lbm_status st2 = prep_palette(d);
  if (st2 != LBM_OK) return st2;
  d->have_fields = true;
  drop_graphs(d);
  return LBM_OK;
}

lbm_status lbm_set_fields(lbm_domain *d, const double *phi, const double *K, const double *alpha_T,
                          const double *D_O2, const double *D_H2O, const double *rho_cp_ratio,
                          int32_t on_device) {
  NvtxRange nvtx_("pemlbm.set_fields");
  if (!d || !phi || !K || !alpha_T || !D_O2 || !D_H2O) return fail(LBM_EINVAL, "null argument");
  if (!d->have_params) return fail(LBM_ESTATE, "call lbm_set_params before lbm_set_fields");
  if (on_device != 0 && on_device != 1) return fail(LBM_EINVAL, "on_device must be 0 or 1");
  const bool slab = d->nx != d->nxg;
  if (on_device && slab) return fail(LBM_EINVAL, "an x-slab takes its material from host arrays");
  if (on_device) return set_fields_device(d, phi, K, alpha_T, D_O2, D_H2O, rho_cp_ratio);
  // an x-slab takes the whole lattice's arrays: its palette is the whole
  // lattice's, so that every slab holds the same entries and the same
  // deviation references, and it keeps the indices of its own columns
  const int nx = d->nxg, ny = d->ny;
  std::vector<uint8_t> mask;
  if (!slab) {
    mask.resize((size_t)d->plane);
    CK(cudaMemcpyAsync(mask.data(), d->mask, mask.size(), cudaMemcpyDeviceToHost, d->stream));
    CK(cudaStreamSynchronize(d->stream));
  }
  auto solid_at = [&](int x, int y) {
    if (!slab) return (mask[(size_t)y * d->nxp + x] & REG_MASK) == REG_SOLID;
    return !d->hsolid.empty() && d->hsolid[(size_t)y * nx + x] != 0;
  };
  std::unordered_map<MatRaw, int, TupleHash, TupleEq> index;
  std::vector<MatRaw> raw;
  std::vector<uint16_t> mid((size_t)d->plane, 0);
  MatRaw prev{};
  int prev_k = -1;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const size_t o = (size_t)y * nx + x;
      if (solid_at(x, y)) continue;
      const MatRaw t{phi[o], K[o], {alpha_T[o], D_O2[o], D_H2O[o]},
                     rho_cp_ratio ? rho_cp_ratio[o] : 1.0};
      int k;
      if (prev_k >= 0 && TupleEq()(t, prev)) {
        k = prev_k;   // same material as the previous cell: the common case
      } else {
        lbm_status vs = check_tuple(t, x, y);
        if (vs != LBM_OK) return vs;
        auto it = index.find(t);
        if (it == index.end()) {
          k = (int)raw.size();
          if (k >= kMaxPalette) return fail(LBM_EINVAL, "more than %d distinct materials", kMaxPalette);
          index.emplace(t, k);
          raw.push_back(t);
        } else {
          k = it->second;
        }
        prev = t;
        prev_k = k;
      }
      const int lx = x - d->x0;
      if (lx >= 0 && lx < d->nx) mid[(size_t)y * d->nxp + lx] = (uint16_t)k;
    }
  if (raw.empty()) return fail(LBM_EINVAL, "no fluid cells");
  // cells that carry no material (solids, padding) point at entry 0
  CK(cudaMemcpyAsync(d->raw, raw.data(), sizeof(MatRaw) * raw.size(), cudaMemcpyHostToDevice, d->stream));
  CK(cudaMemcpyAsync(d->mid, mid.data(), mid.size() * 2, cudaMemcpyHostToDevice, d->stream));
  d->npal = (int)raw.size();
  // reference material of the deviation storage: the top fluid cell of the
  // inlet column (the channel gas), else entry 0
  d->ref_entry = 0;
  for (int y = ny - 1; y >= 0; --y)
    if (!solid_at(0, y)) {
      const size_t o = (size_t)y * nx;
      const MatRaw t{phi[o], K[o], {alpha_T[o], D_O2[o], D_H2O[o]},
                     rho_cp_ratio ? rho_cp_ratio[o] : 1.0};
      d->ref_entry = index.at(t);   // every fluid cell's tuple is in the index
      break;
    }
  d->hraw = std::move(raw);
  lbm_status st = prep_palette(d);
  if (st != LBM_OK) return st;
  d->have_fields = true;
  drop_graphs(d);
  return LBM_OK;
}

lbm_status lbm_reset(lbm_domain *d) {
  NvtxRange nvtx_("pemlbm.reset");
  if (!d) return fail(LBM_EINVAL, "null domain");
  if (!d->have_params || !d->have_fields) return fail(LBM_ESTATE, "call lbm_set_params and lbm_set_fields first");
  d->Cref[0] = d->prm.T_in;
  d->Cref[1] = d->prm.C_O2_in;
  d->Cref[2] = d->prm.C_H2O_in;
  for (int s = 0; s < 3; ++s) d->bref[s] = d->bref_next[s];
  const KArgs a = make_args(d);
  const DevGeom g = geom(d);
  dispatch(d->desc.precision, [&](auto *tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    launch_init<S>(d->pop[0], g, a, d->stream);
    launch_init<S>(d->pop[1], g, a, d->stream);
  });
  CK(cudaMemsetAsync(d->dseed, 0, sizeof(unsigned), d->stream));
  CK(cudaGetLastError());
  d->cur = 0;
  d->steps = 0;
  d->have_state = true;
  drop_graphs(d);
  // first residual snapshot: compare against zeros, keep only the snapshot
  CK(cudaMemsetAsync(d->snap, 0, 2 * (fp64(d) ? 8 : 4) * 5 * (size_t)d->nx * d->ny, d->stream));
  d->snap_cur = 0;
  double r;
  lbm_status s = lbm_residual(d, &r);
  if (s != LBM_OK && s != LBM_EDIVERGED) return s;
  return LBM_OK;
}

lbm_status lbm_step(lbm_domain *d, int64_t nsteps) {
  NvtxRange nvtx_("pemlbm.step");
  lbm_status s = check_ready(d);
  if (s != LBM_OK) return s;
  if (nsteps < 0) return fail(LBM_EINVAL, "nsteps < 0");
  int64_t left = nsteps;
  while (left >= 2 * kGraphSteps) {
    if ((s = ensure_graph(d)) != LBM_OK) return s;
    CK(cudaGraphLaunch(d->graph[d->cur], d->stream));
    left -= kGraphSteps;
  }
  if ((s = launch_steps(d, left)) != LBM_OK) return s;
  d->steps += nsteps;
  return LBM_OK;
}

lbm_status lbm_time_steps(lbm_domain *d, int64_t nsteps, double *elapsed_ms) {
  lbm_status s = check_ready(d);
  if (s != LBM_OK) return s;
  if (!elapsed_ms) return fail(LBM_EINVAL, "null argument");
  CK(cudaEventRecord(d->ev0, d->stream));
  if ((s = lbm_step(d, nsteps)) != LBM_OK) return s;
  CK(cudaEventRecord(d->ev1, d->stream));
  CK(cudaEventSynchronize(d->ev1));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, d->ev0, d->ev1));
  *elapsed_ms = ms;
  return LBM_OK;
}

lbm_status lbm_current_density(lbm_domain *d, double *i_avg, double *heat, float *profile) {
  NvtxRange nvtx_("pemlbm.current_density");
  lbm_status s = check_ready(d);
  if (s != LBM_OK) return s;
  if (d->steps < 1) return fail(LBM_ESTATE, "no step taken yet");
  const lbm_params &p = d->prm;
  const double i_scale = 4.0 * p.F * p.c_tot * p.dx_cm / p.dt_s;
  const double q_scale = p.rho_cp_f * p.dx_cm / p.dt_s;
  const KArgs a = make_args(d);
  dispatch(d->desc.precision, [&](auto *tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    launch_catalyst<S>(d->pop[d->cur ^ 1], geom(d), a, i_scale, profile ? d->dprofile : nullptr,
                       d->colsum, d->dsmall, d->stream);
  });
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(d->hsmall, d->dsmall, 2 * sizeof(double), cudaMemcpyDeviceToHost, d->stream));
  if (profile) CK(cudaMemcpyAsync(profile, d->dprofile, sizeof(float) * d->nx, cudaMemcpyDeviceToHost, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  if (i_avg) *i_avg = d->hsmall[0] * i_scale / d->nx;
  if (heat) *heat = d->hsmall[1] * q_scale / d->nx;
  return LBM_OK;
}

lbm_status lbm_step_observe(lbm_domain *d, int64_t nsteps, double *i_avg, double *heat) {
  NvtxRange nvtx_("pemlbm.step_observe");
  lbm_status s = check_ready(d);
  if (s != LBM_OK) return s;
  if (nsteps < 0) return fail(LBM_EINVAL, "nsteps < 0");
  if (nsteps > 0 && !i_avg && !heat) return fail(LBM_EINVAL, "nothing to observe (use lbm_step)");
  if (!d->dobs) {
    // the reductions run at the highest priority, so that their few blocks
    // are dispatched while the step's blocks are still being issued
    // instead of after them
    int lo_prio = 0, hi_prio = 0;
    const size_t bytes = 2 * kGraphSteps * 2 * sizeof(double);
    if (dmalloc(&d->dobs, bytes) != cudaSuccess || hmalloc(&d->hobs, bytes) != cudaSuccess ||
        cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio) != cudaSuccess ||
        cudaStreamCreateWithPriority(&d->obs_side, cudaStreamNonBlocking, hi_prio) != cudaSuccess ||
        cudaEventCreateWithFlags(&d->obs_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&d->obs_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&d->obs_done[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&d->obs_done[1], cudaEventDisableTiming) != cudaSuccess) {
      // release what was made, so that a later call starts over
      if (d->dobs) cudaFree(d->dobs);
      if (d->hobs) cudaFreeHost(d->hobs);
      if (d->obs_side) cudaStreamDestroy(d->obs_side);
      for (cudaEvent_t *e : {&d->obs_fork, &d->obs_join, &d->obs_done[0], &d->obs_done[1]})
        if (*e) {
          cudaEventDestroy(*e);
          *e = nullptr;
        }
      d->dobs = d->hobs = nullptr;
      d->obs_side = nullptr;
      cudaGetLastError();
      return fail(LBM_ENOMEM, "observation slots");
    }
  }
  const lbm_params &p = d->prm;
  const double i_scale = 4.0 * p.F * p.c_tot * p.dx_cm / p.dt_s;
  const double q_scale = p.rho_cp_f * p.dx_cm / p.dt_s;
  // chunks of up to kGraphSteps steps alternate between the two slot halves:
  // while chunk c runs, the host reads chunk c - 1's slots
  auto collect = [&](int half, int64_t first, int64_t n) -> lbm_status {
    CK(cudaEventSynchronize(d->obs_done[half]));
    for (int64_t k = 0; k < n; ++k) {
      const double *v = d->hobs + ((size_t)half * kGraphSteps + (size_t)k) * 2;
      if (i_avg) i_avg[first + k] = v[0] * i_scale / d->nx;
      if (heat) heat[first + k] = v[1] * q_scale / d->nx;
    }
    return LBM_OK;
  };
  int64_t done = 0, prev_first = -1, prev_n = 0;
  int half = 0;
  while (done < nsteps) {
    const int64_t n = std::min<int64_t>(kGraphSteps, nsteps - done);
    if (n == kGraphSteps) {
      if ((s = ensure_obs_graph(d, half)) != LBM_OK) return s;
      CK(cudaGraphLaunch(d->obs_graph[d->cur][half], d->stream));   // even: cur unchanged
    } else if ((s = launch_observed(d, n, half)) != LBM_OK) {
      return s;
    }
    CK(cudaEventRecord(d->obs_done[half], d->stream));
    if (prev_n > 0 && (s = collect(half ^ 1, prev_first, prev_n)) != LBM_OK) return s;
    prev_first = done;
    prev_n = n;
    done += n;
    d->steps += n;
    half ^= 1;
  }
  if (prev_n > 0 && (s = collect(half ^ 1, prev_first, prev_n)) != LBM_OK) return s;
  return LBM_OK;
}

lbm_status lbm_balances(lbm_domain *d, double *out) {
  NvtxRange nvtx_("pemlbm.balances");
  lbm_status s = check_ready(d);
  if (s != LBM_OK) return s;
  if (!out) return fail(LBM_EINVAL, "null argument");
  if (d->steps < 1) return fail(LBM_ESTATE, "no step taken yet");
  const KArgs a = make_args(d);
  dispatch(d->desc.precision, [&](auto *tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    launch_catalyst<S>(d->pop[d->cur ^ 1], geom(d), a, 1.0, nullptr, d->colsum, d->dsmall,
                       d->stream);
    launch_balances<S>(d->pop[d->cur ^ 1], geom(d), a, d->dsmall + 2, d->stream);
  });
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(d->hsmall, d->dsmall, 10 * sizeof(double), cudaMemcpyDeviceToHost, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  std::memcpy(out, d->hsmall, 10 * sizeof(double));
  return LBM_OK;
}

lbm_status lbm_residual(lbm_domain *d, double *res) {
  NvtxRange nvtx_("pemlbm.residual");
  if (!d || !res) return fail(LBM_EINVAL, "null argument");
  if (!d->have_state) return fail(LBM_ESTATE, "call lbm_reset first");
  const KArgs a = make_args(d);
  CK(cudaMemsetAsync(d->dbad, 0, sizeof(int), d->stream));
  // compare with one snapshot, write the other (an in-place update of one
  // buffer makes the kernel several times slower)
  const size_t half = (fp64(d) ? 8 : 4) * 5 * (size_t)d->nx * d->ny;
  char *snaps = (char *)d->snap;
  dispatch(d->desc.precision, [&](auto *tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    launch_residual<S>(d->pop[d->cur], geom(d), a, snaps + d->snap_cur * half,
                       snaps + (d->snap_cur ^ 1) * half, d->partial, d->dbad, d->dsmall,
                       d->stream);
  });
  CK(cudaGetLastError());
  d->snap_cur ^= 1;
  CK(cudaMemcpyAsync(d->hsmall, d->dsmall, 10 * sizeof(double), cudaMemcpyDeviceToHost, d->stream));
  CK(cudaMemcpyAsync(d->hsmall + 10, d->dbad, sizeof(int), cudaMemcpyDeviceToHost, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  int bad;
  std::memcpy(&bad, d->hsmall + 10, sizeof(int));
  double r = 0.0;
  for (int k = 0; k < 5; ++k) {
    const double num = d->hsmall[k], den = d->hsmall[5 + k];
    const double rk = den > 0 ? std::sqrt(num / den) : (num > 0 ? INFINITY : 0.0);
    r = std::fmax(r, rk);
  }
  *res = r;
  if (bad || !std::isfinite(r)) return fail(LBM_EDIVERGED, "non-finite values in the state");
  return LBM_OK;
}

lbm_status lbm_get_fields(lbm_domain *d, double *out, int32_t on_device) {
  NvtxRange nvtx_("pemlbm.get_fields");
  lbm_status s = check_ready(d);
  if (s != LBM_OK) return s;
  if (!out) return fail(LBM_EINVAL, "null argument");
  double *dst = out;
  if (!on_device) {
    if ((s = ensure_scratch(d)) != LBM_OK) return s;
    dst = d->scratch;
  }
  const KArgs a = make_args(d);
  dispatch(d->desc.precision, [&](auto *tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    launch_fields<S>(d->pop[d->cur ^ 1], geom(d), a, dst, d->stream);
  });
  CK(cudaGetLastError());
  if (!on_device) {
    CK(cudaMemcpyAsync(out, dst, sizeof(double) * 6 * (size_t)d->nx * d->ny, cudaMemcpyDeviceToHost, d->stream));
    CK(cudaStreamSynchronize(d->stream));
  }
  return LBM_OK;
}

lbm_status lbm_get_state(lbm_domain *d, double *out) {
  lbm_status s = check_ready(d);
  if (s != LBM_OK) return s;
  if (!out) return fail(LBM_EINVAL, "null argument");
  if ((s = ensure_scratch(d)) != LBM_OK) return s;
  const KArgs a = make_args(d);
  dispatch(d->desc.precision, [&](auto *tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    launch_get_state<S>(d->pop[d->cur], geom(d), a, d->scratch, d->stream);
  });
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(out, d->scratch, sizeof(double) * 24 * (size_t)d->nx * d->ny, cudaMemcpyDeviceToHost, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  return LBM_OK;
}

lbm_status lbm_set_state(lbm_domain *d, const double *in) {
  lbm_status s = check_ready(d);
  if (s != LBM_OK) return s;
  if (!in) return fail(LBM_EINVAL, "null argument");
  if ((s = ensure_scratch(d)) != LBM_OK) return s;
  CK(cudaMemcpyAsync(d->scratch, in, sizeof(double) * 24 * (size_t)d->nx * d->ny, cudaMemcpyHostToDevice, d->stream));
  const KArgs a = make_args(d);
  dispatch(d->desc.precision, [&](auto *tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    launch_set_state<S>(d->pop[0], geom(d), a, d->scratch, d->stream);
    launch_set_state<S>(d->pop[1], geom(d), a, d->scratch, d->stream);
  });
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(d->stream));
  return LBM_OK;
}

lbm_status lbm_get_mask(lbm_domain *d, uint8_t *mask_host) {
  if (!d || !mask_host) return fail(LBM_EINVAL, "null argument");
  CK(cudaMemcpy2DAsync(mask_host, d->nx, d->mask, d->nxp, d->nx, d->ny, cudaMemcpyDeviceToHost, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  return LBM_OK;
}

lbm_status lbm_get_step(lbm_domain *d, int64_t *steps) {
  if (!d || !steps) return fail(LBM_EINVAL, "null argument");
  *steps = d->steps;
  return LBM_OK;
}

struct StateHeader {
  char magic[8];
  int32_t nx, ny, precision, cur;
  int64_t steps;
  double Cref[3], bref[3];
};

lbm_status lbm_save_state(lbm_domain *d, void *buf, size_t *bytes) {
  NvtxRange nvtx_("pemlbm.save_state");
  lbm_status s = check_ready(d);
  if (s != LBM_OK) return s;
  if (!bytes) return fail(LBM_EINVAL, "null argument");
  const size_t pop_bytes = 24 * (size_t)d->plane * d->esize;   // the guard is not state
  const size_t need = sizeof(StateHeader) + 2 * pop_bytes;
  if (!buf) {
    *bytes = need;
    return LBM_OK;
  }
  if (*bytes < need) return fail(LBM_EINVAL, "buffer of %zu bytes, need %zu", *bytes, need);
  StateHeader h{};
  std::memcpy(h.magic, "PEMLBM2", 8);
  h.nx = d->nx; h.ny = d->ny; h.precision = d->desc.precision; h.cur = d->cur; h.steps = d->steps;
  for (int k = 0; k < 3; ++k) { h.Cref[k] = d->Cref[k]; h.bref[k] = d->bref[k]; }
  std::memcpy(buf, &h, sizeof h);
  char *p = (char *)buf + sizeof h;
  CK(cudaMemcpyAsync(p, d->pop[0], pop_bytes, cudaMemcpyDeviceToHost, d->stream));
  CK(cudaMemcpyAsync(p + pop_bytes, d->pop[1], pop_bytes, cudaMemcpyDeviceToHost, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  *bytes = need;
  return LBM_OK;
}

lbm_status lbm_load_state(lbm_domain *d, const void *buf, size_t bytes) {
  NvtxRange nvtx_("pemlbm.load_state");
  if (!d || !buf) return fail(LBM_EINVAL, "null argument");
  if (!d->have_params || !d->have_fields) return fail(LBM_ESTATE, "call lbm_set_params and lbm_set_fields first");
  const size_t pop_bytes = 24 * (size_t)d->plane * d->esize;
  StateHeader h;
  if (bytes != sizeof h + 2 * pop_bytes) return fail(LBM_EINVAL, "blob of %zu bytes does not match this domain", bytes);
  std::memcpy(&h, buf, sizeof h);
  if (std::memcmp(h.magic, "PEMLBM2", 8) || h.nx != d->nx || h.ny != d->ny || h.precision != d->desc.precision)
    return fail(LBM_EINVAL, "blob was taken from another geometry or precision");
  const char *p = (const char *)buf + sizeof h;
  CK(cudaMemcpyAsync(d->pop[0], p, pop_bytes, cudaMemcpyHostToDevice, d->stream));
  CK(cudaMemcpyAsync(d->pop[1], p + pop_bytes, pop_bytes, cudaMemcpyHostToDevice, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  d->cur = h.cur;
  d->steps = h.steps;
  for (int k = 0; k < 3; ++k) { d->Cref[k] = h.Cref[k]; d->bref[k] = h.bref[k]; }
  d->have_state = true;
  drop_graphs(d);
  return LBM_OK;
}

lbm_status lbm_set_variant(lbm_domain *d, int32_t variant) {
  if (!d) return fail(LBM_EINVAL, "null domain");
  if (variant < 0 || variant >= kStepVariants) return fail(LBM_EINVAL, "variant %d outside [0, %d)", variant, kStepVariants);
  d->variant = variant;
  drop_graphs(d);
  return LBM_OK;
}

lbm_status lbm_tune(lbm_domain *d, int32_t trial_steps, int32_t *variant, double *best_ms) {
  NvtxRange nvtx_("pemlbm.tune");
  lbm_status s = check_ready(d);
  if (s != LBM_OK) return s;
  if (d->steps != 0) return fail(LBM_ESTATE, "lbm_tune runs between lbm_reset and the first step");
  if (trial_steps < 1) return fail(LBM_EINVAL, "trial_steps < 1");
  const KArgs a = make_args(d);
  const DevGeom g = geom(d);
  int best = 0;
  for (int v = 0; v < kStepVariants; ++v) {
    auto run = [&](int n) {
      for (int k = 0; k < n; ++k)
        dispatch(d->desc.precision, [&](auto *tag) {
          using S = std::remove_pointer_t<decltype(tag)>;
          // the same step from the same state every time: the state is kept
          launch_step<S>(d->pop[d->cur], d->pop[d->cur ^ 1], g, a, v, d->stream);
        });
    };
    run(2);
    CK(cudaEventRecord(d->ev0, d->stream));
    run(trial_steps);
    CK(cudaEventRecord(d->ev1, d->stream));
    CK(cudaEventSynchronize(d->ev1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, d->ev0, d->ev1));
    d->tuned_ms[v] = ms / trial_steps;
    if (d->tuned_ms[v] < d->tuned_ms[best]) best = v;
  }
  // the trials wrote the next state into the other buffer: restore it
  dispatch(d->desc.precision, [&](auto *tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    launch_init<S>(d->pop[d->cur ^ 1], g, a, d->stream);
  });
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(d->stream));
  d->variant = best;
  drop_graphs(d);
  if (variant) *variant = best;
  if (best_ms) *best_ms = d->tuned_ms[best];
  return LBM_OK;
}

lbm_status lbm_bytes_per_cell(lbm_domain *d, double *bytes) {
  if (!d || !bytes) return fail(LBM_EINVAL, "null argument");
  *bytes = 48.0 * d->esize + 1.0;
  return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Discrete adjoint (gradients of the objectives w.r.t. phi, K, D_O2 and the
// inlet velocity).
namespace {

struct DevBuf {
  void *p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  lbm_status alloc(size_t bytes) {
    if (dmalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(LBM_ENOMEM, "device allocation of %.1f MB for the adjoint failed", bytes / 1e6);
    }
    return LBM_OK;
  }
};

// Reverse workspace of one domain.
struct AdjWork {
  DevBuf lam[2], O[2], V[2], gphi, gK, gD, gU, tphi, tK, tD, cells, pushed, slot;
  int n_edge = 0, n_own = 0;
  size_t rsize = 4;                             // bytes of the arithmetic type
  cudaStream_t side = nullptr;                  // edge-cell branch of each step
  cudaEvent_t fork = nullptr, join = nullptr;
  ~AdjWork() {
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    if (side) cudaStreamDestroy(side);
  }
  lbm_status alloc(lbm_domain *d) {
    const size_t r = fp64(d) ? 8 : 4, planes = 24 * (size_t)d->plane;
    lbm_status s;
    if (cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return fail(LBM_ECUDA, "stream or event creation for the adjoint failed");
    }
    for (auto *b : {&lam[0], &lam[1], &O[0], &O[1]})
      if ((s = b->alloc(planes * r)) != LBM_OK) return s;
    for (auto *b : {&V[0], &V[1]})   // [outlet, inlet][down, up][10][ny]
      if ((s = b->alloc(40 * (size_t)d->ny * r)) != LBM_OK) return s;
    // everything starts at zero: lambda^{n-1} of solid cells is zeroed by
    // every step, and the own-use parts of the first lambda are zero
    for (auto *b : {&lam[0], &lam[1], &O[0], &O[1]})
      CK(cudaMemsetAsync(b->p, 0, planes * r, d->stream));
    for (auto *b : {&V[0], &V[1]}) CK(cudaMemsetAsync(b->p, 0, 40 * (size_t)d->ny * r, d->stream));
    for (auto *b : {&gphi, &gK, &gD})
      if ((s = b->alloc(r * d->plane)) != LBM_OK) return s;
    for (auto *b : {&tphi, &tK, &tD})
      if ((s = b->alloc(sizeof(double) * d->plane)) != LBM_OK) return s;
    if ((s = gU.alloc(sizeof(double))) != LBM_OK) return s;
    // cell lists: fluid cells with edge bits, then fluid catalyst cells of
    // the volumetric mode without them (both use their own state)
    std::vector<uint8_t> m((size_t)d->plane);
    CK(cudaMemcpyAsync(m.data(), d->mask, m.size(), cudaMemcpyDeviceToHost, d->stream));
    CK(cudaStreamSynchronize(d->stream));
    std::vector<long long> list;
    for (int pass = 0; pass < 2; ++pass) {
      for (int y = 0; y < d->ny; ++y)
        for (int x = 0; x < d->nx; ++x) {
          const long long c = (long long)y * d->nxp + x;
          const uint8_t b = m[c];
          if ((b & REG_MASK) == REG_SOLID) continue;
          const bool edge = (b & M_EDGE) != 0;
          const bool vol = d->desc.reaction_mode == 1 && (b & REG_MASK) == REG_CATALYST;
          if (pass == 0 ? edge : (vol && !edge)) list.push_back(c);
        }
      if (pass == 0) {
        // edge cells grouped by node type, so that the threads of a warp take
        // the same boundary path (row-major order would mix inlet and outlet
        // cells in one warp and serialise both paths)
        std::stable_sort(list.begin(), list.end(),
                         [&](long long p1, long long p2) { return m[p1] < m[p2]; });
        n_edge = (int)list.size();
      }
    }
    n_own = (int)list.size();
    rsize = r;
    // listed index of every cell (reverse records of own states), -1 for others
    std::vector<int> slots((size_t)d->plane, -1);
    for (size_t t = 0; t < list.size(); ++t) slots[(size_t)list[t]] = (int)t;
    if ((s = slot.alloc(sizeof(int) * slots.size())) != LBM_OK) return s;
    CK(cudaMemcpyAsync(slot.p, slots.data(), sizeof(int) * slots.size(), cudaMemcpyHostToDevice,
                       d->stream));
    CK(cudaStreamSynchronize(d->stream));
    // per edge cell, the links q whose consumer y + e_q is a fluid cell
    // (periodic seam included): only those are pushed by a consumer
    std::vector<uint32_t> bits(n_edge);
    for (int t = 0; t < n_edge; ++t) {
      const int y = (int)(list[t] / d->nxp), x = (int)(list[t] - (long long)y * d->nxp);
      uint32_t b = 0;
      for (int q = 0; q < 24; ++q) {
        const int l = q < 9 ? q : (q - 9) % 5;
        const int ex[9] = EX9_TAB, ey[9] = EY9_TAB;
        int cx = x + ex[l];
        const int cy = y + ey[l];
        if (cy < 0 || cy >= d->ny) continue;
        if (d->desc.periodic_x) cx = cx < 0 ? cx + d->nx : (cx >= d->nx ? cx - d->nx : cx);
        if (cx < 0 || cx >= d->nx) continue;
        if ((m[(size_t)cy * d->nxp + cx] & REG_MASK) != REG_SOLID) b |= 1u << q;
      }
      bits[t] = b;
    }
    if (n_own > 0) {
      if ((s = cells.alloc(sizeof(long long) * list.size())) != LBM_OK) return s;
      CK(cudaMemcpyAsync(cells.p, list.data(), sizeof(long long) * list.size(),
                         cudaMemcpyHostToDevice, d->stream));
    }
    if (n_edge > 0) {
      if ((s = pushed.alloc(sizeof(uint32_t) * bits.size())) != LBM_OK) return s;
      CK(cudaMemcpyAsync(pushed.p, bits.data(), sizeof(uint32_t) * bits.size(),
                         cudaMemcpyHostToDevice, d->stream));
    }
    CK(cudaStreamSynchronize(d->stream));
    return LBM_OK;
  }
  // Reverse records of one step (RecPtrs): the cell records, then the own
  // records of the listed cells, then the pulled values of the edge cells,
  // each part starting on a 256-byte boundary.
  static size_t up256(size_t b) { return (b + 255) / 256 * 256; }
  size_t rec_cell_bytes(const lbm_domain *d) const { return up256(8 * rsize * (size_t)d->plane); }
  size_t rec_own_bytes() const { return up256(4 * rsize * (size_t)n_own); }
  size_t rec_bytes(const lbm_domain *d) const {
    return rec_cell_bytes(d) + rec_own_bytes() + up256(24 * rsize * (size_t)n_edge);
  }
  RecBufs recs(const lbm_domain *d, void *base) const {
    char *b = (char *)base;
    return RecBufs{b, b + rec_cell_bytes(d), b + rec_cell_bytes(d) + rec_own_bytes(),
                   (const int *)slot.p};
  }
  lbm_status zero_grads(const lbm_domain *d) {
    const size_t r = fp64(d) ? 8 : 4;
    for (auto *b : {&gphi, &gK, &gD}) CK(cudaMemsetAsync(b->p, 0, r * d->plane, d->stream));
    for (auto *b : {&tphi, &tK, &tD}) CK(cudaMemsetAsync(b->p, 0, sizeof(double) * d->plane, d->stream));
    CK(cudaMemsetAsync(gU.p, 0, sizeof(double), d->stream));
    return LBM_OK;
  }
  // A step reading lambda = lam[cur] (own-use parts in O[cur], V[cur])
  // writes lam[cur ^ 1], O[cur ^ 1], V[cur ^ 1].
  AdjPtrs ptrs(int cur) {
    return AdjPtrs{lam[cur].p, O[cur ^ 1].p, V[cur ^ 1].p, O[cur].p, V[cur].p,
                   gphi.p, gK.p, gD.p, (double *)gU.p, lam[cur ^ 1].p,
                   (double *)tphi.p, (double *)tK.p, (double *)tD.p,
                   (const long long *)cells.p, (const uint32_t *)pushed.p, n_edge, n_own};
  }
  // Completion of lam[cur] in place (its own-use parts are O[cur], V[cur]).
  AdjPtrs finish_ptrs(int cur) {
    AdjPtrs b = ptrs(cur ^ 1);
    b.lam = nullptr;
    b.O_in = b.V_in = nullptr;
    return b;   // lam_out = lam[cur], O = O[cur], V = V[cur]
  }
};

// Adds the segment gradients into the FP64 totals.
void fold_grads(lbm_domain *d, AdjWork &w) {
  const KArgs a = make_args(d);
  dispatch(d->desc.precision, [&](auto *tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    launch_adj_fold<S>(geom(d), a, w.ptrs(0), d->stream);
  });
}

// One reverse step: lambda^n (w.lam[cur]) at state src = s^{n-1} ->
// lambda^{n-1} (w.lam[cur ^ 1]), gradients accumulated.
// lam_complete: lambda^n = w.lam[cur] holds every link in full (uploaded or
// seeded) rather than the pushed part of a previous reverse step.
void reverse_step(lbm_domain *d, AdjWork &w, int cur, const RecBufs &rec, long long seed_cell,
                  bool lam_complete = false) {
  const KArgs a = make_args(d);
  const int fick = d->prm.interface_mode == 1;
  const AdjPtrs b = w.ptrs(cur);
  dispatch(d->desc.precision, [&](auto *tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    launch_adj_step<S>(rec, geom(d), a, fick, b, seed_cell, lam_complete ? 1 : 0, d->stream,
                       w.side, w.fork, w.join);
  });
}

// One forward step src -> dst on stream st that also writes its reverse
// records into `rec` (RecPtrs).
void step_with_records(lbm_domain *d, const void *src, void *dst, const RecBufs &rec,
                       cudaStream_t st) {
  const KArgs a = make_args(d);
  dispatch(d->desc.precision, [&](auto *tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    launch_step_rec<S>(src, dst, geom(d), a, rec, st);
  });
}

// Completes lambda = lam[cur] after the last reverse step.
void finish_lambda(lbm_domain *d, AdjWork &w, int cur) {
  const KArgs a = make_args(d);
  dispatch(d->desc.precision, [&](auto *tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    launch_adj_finish<S>(geom(d), a, w.finish_ptrs(cur), d->stream);
  });
}

lbm_status copy_grads_out(lbm_domain *d, AdjWork &w, double *dphi, double *dK, double *dD,
                          double *du, bool on_device = false) {
  const size_t row = sizeof(double) * d->nx, pitch = sizeof(double) * d->nxp;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  fold_grads(d, w);
  if (dphi) CK(cudaMemcpy2DAsync(dphi, row, w.tphi.p, pitch, row, d->ny, kind, d->stream));
  if (dK) CK(cudaMemcpy2DAsync(dK, row, w.tK.p, pitch, row, d->ny, kind, d->stream));
  if (dD) CK(cudaMemcpy2DAsync(dD, row, w.tD.p, pitch, row, d->ny, kind, d->stream));
  if (du) CK(cudaMemcpyAsync(du, w.gU.p, sizeof(double), cudaMemcpyDeviceToHost, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  return LBM_OK;
}

// Full-value planes [24][ny][nx] (host) <-> deviation-free device planes of
// type R [24][plane]: adjoints of deviations equal adjoints of full values.
lbm_status lam_upload(lbm_domain *d, const double *host, void *dev) {
  const size_t n = (size_t)d->nx * d->ny;
  std::vector<unsigned char> tmp(24 * (size_t)d->plane * (fp64(d) ? 8 : 4), 0);
  for (int q = 0; q < 24; ++q)
    for (int y = 0; y < d->ny; ++y)
      for (int x = 0; x < d->nx; ++x) {
        const double v = host[q * n + (size_t)y * d->nx + x];
        const size_t o = (size_t)q * d->plane + (size_t)y * d->nxp + x;
        if (fp64(d)) ((double *)tmp.data())[o] = v;
        else ((float *)tmp.data())[o] = (float)v;
      }
  CK(cudaMemcpyAsync(dev, tmp.data(), tmp.size(), cudaMemcpyHostToDevice, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  return LBM_OK;
}
// The adjoint differentiates the cathode's boundaries and forces; the
// closed ends, buoyancy and fixed wall values of the validation set-ups
// have no transpose here.
lbm_status adjoint_covers(const lbm_domain *d) {
  const lbm_params &p = d->prm;
  if (d->desc.closed_x || p.buoy_gx != 0.0 || p.buoy_gy != 0.0 || p.wall_dirichlet != 0)
    return fail(LBM_EINVAL, "the adjoint does not cover closed_x, buoyancy or fixed wall values");
  if (d->nx != d->nxg) return fail(LBM_EINVAL, "the adjoint does not cover x-slabs");
  return LBM_OK;
}
lbm_status lam_download(lbm_domain *d, const void *dev, double *host) {
  const size_t n = (size_t)d->nx * d->ny;
  std::vector<unsigned char> tmp(24 * (size_t)d->plane * (fp64(d) ? 8 : 4));
  CK(cudaMemcpyAsync(tmp.data(), dev, tmp.size(), cudaMemcpyDeviceToHost, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  for (int q = 0; q < 24; ++q)
    for (int y = 0; y < d->ny; ++y)
      for (int x = 0; x < d->nx; ++x) {
        const size_t o = (size_t)q * d->plane + (size_t)y * d->nxp + x;
        host[q * n + (size_t)y * d->nx + x] =
            fp64(d) ? ((const double *)tmp.data())[o] : (double)((const float *)tmp.data())[o];
      }
  return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_vjp(lbm_domain *d, const double *lam_next, double *lam_prev, double *dphi,
                   double *dK, double *dD_O2, double *du_in) {
  NvtxRange nvtx_("pemlbm.vjp");
  lbm_status s = check_ready(d);
  if (s != LBM_OK) return s;
  if (!lam_next || !lam_prev) return fail(LBM_EINVAL, "null argument");
  if (d->desc.rounding != 0) return fail(LBM_EINVAL, "the adjoint needs round-to-nearest storage");
  if ((s = adjoint_covers(d)) != LBM_OK) return s;
  AdjWork w;
  if ((s = w.alloc(d)) != LBM_OK) return s;
  if ((s = w.zero_grads(d)) != LBM_OK) return s;
  if ((s = lam_upload(d, lam_next, w.lam[0].p)) != LBM_OK) return s;
  // the step's reverse records (its new state is not kept)
  DevBuf rec, next;
  if ((s = rec.alloc(w.rec_bytes(d))) != LBM_OK) return s;
  if ((s = next.alloc((24 * (size_t)d->plane + d->nxp + 64) * d->esize)) != LBM_OK) return s;
  step_with_records(d, d->pop[d->cur], next.p, w.recs(d, rec.p), d->stream);
  reverse_step(d, w, 0, w.recs(d, rec.p), -1, true);
  finish_lambda(d, w, 1);
  CK(cudaGetLastError());
  if ((s = lam_download(d, w.lam[1].p, lam_prev)) != LBM_OK) return s;
  return copy_grads_out(d, w, dphi, dK, dD_O2, du_in);
}

lbm_status lbm_grad(lbm_domain *d, int32_t objective, int64_t nsteps, int32_t segment,
                    double *J, double *dphi, double *dK, double *dD_O2, double *du_in,
                    int32_t on_device) {
  NvtxRange nvtx_("pemlbm.grad");
  lbm_status s = check_ready(d);
  if (s != LBM_OK) return s;
  if (on_device != 0 && on_device != 1) return fail(LBM_EINVAL, "on_device must be 0 or 1");
  if (objective != 0 && objective != 1) return fail(LBM_EINVAL, "objective must be 0 or 1");
  if (d->desc.rounding != 0) return fail(LBM_EINVAL, "the adjoint needs round-to-nearest storage");
  if ((s = adjoint_covers(d)) != LBM_OK) return s;
  if (nsteps < 2 || nsteps > (1LL << 30)) return fail(LBM_EINVAL, "nsteps outside [2, 2^30]");
  const int64_t N = nsteps;
  // Reverse step n (lambda^n -> lambda^{n-1}) reads the records R^n of
  // forward step n (s^{n-1} -> s^n).  Objective 0 is a function of s^{N-1}
  // and seeds lambda^{N-1} directly; objective 1 reads the fields of step
  // N, whose reverse (step N) needs R^N.
  const int64_t nrec = objective == 1 ? N : N - 1;
  const int seg = segment > 0 ? segment : (int)std::ceil(std::sqrt((double)N));
  const int64_t nseg = (nrec + seg - 1) / seg;   // segment k: R^{k seg + 1} .. R^{min((k+1) seg, nrec)}
  const size_t sbytes = (24 * (size_t)d->plane + d->nxp + 64) * d->esize;   // guard as in the domain
  AdjWork w;
  if ((s = w.alloc(d)) != LBM_OK) return s;
  if ((s = w.zero_grads(d)) != LBM_OK) return s;
  const size_t rbytes = w.rec_bytes(d), segbytes = rbytes * (size_t)seg;
  DevBuf fs[2];   // forward states
  for (auto &b : fs)
    if ((s = b.alloc(sbytes)) != LBM_OK) return s;
  // The last L segments keep the records their forward steps write; the
  // others are recomputed from checkpoints (two record buffers, so that
  // segment k - 1 is recomputed on a stream of its own while segment k is
  // reversed).  L is as large as the memory limit allows.
  size_t free_b = 0, total_b = 0;
  CK(cudaMemGetInfo(&free_b, &total_b));
  const size_t reserve = std::max<size_t>(total_b / 64, (size_t)1 << 30);
  size_t budget = free_b > reserve ? free_b - reserve : 0;
  if (d->grad_mem_limit >= 0) budget = std::min(budget, (size_t)d->grad_mem_limit);
  int64_t L = 0;
  if ((size_t)nseg <= budget / segbytes) {
    L = nseg;
  } else {
    const size_t rec_overhead = 2 * segbytes + 2 * sbytes + (size_t)nseg * sbytes;
    if (budget > rec_overhead) L = std::min<int64_t>(nseg - 1, (budget - rec_overhead) / segbytes);
  }
  DevBuf store;
  while (L > 0 && dmalloc(&store.p, segbytes * (size_t)L) != cudaSuccess) {
    cudaGetLastError();
    L /= 2;
  }
  const int64_t k0 = nseg - L;            // segments k >= k0 are stored
  DevBuf ck, rb[2], rs[2];
  if (k0 > 0) {
    if ((s = ck.alloc(sbytes * (size_t)k0)) != LBM_OK) return s;
    for (auto *b : {&rb[0], &rb[1]})
      if ((s = b->alloc(segbytes)) != LBM_OK) return s;
    for (auto &b : rs)
      if ((s = b.alloc(sbytes)) != LBM_OK) return s;
  }
  struct Sync {   // recompute stream and its two buffer events
    cudaStream_t rs = nullptr;
    cudaEvent_t ready[2] = {nullptr, nullptr}, freed[2] = {nullptr, nullptr};
    ~Sync() {
      for (cudaEvent_t e : {ready[0], ready[1], freed[0], freed[1]})
        if (e) cudaEventDestroy(e);
      if (rs) cudaStreamDestroy(rs);
    }
  } sync;
  if (k0 > 0) {
    if (cudaStreamCreateWithFlags(&sync.rs, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return fail(LBM_ECUDA, "cudaStreamCreate failed");
    }
    for (cudaEvent_t *e : {&sync.ready[0], &sync.ready[1], &sync.freed[0], &sync.freed[1]})
      if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return fail(LBM_ECUDA, "cudaEventCreate failed");
      }
  }
  auto first_of = [&](int64_t k) { return k * seg; };                       // segment's start state
  auto last_of = [&](int64_t k) { return std::min<int64_t>((k + 1) * seg, nrec); };
  auto stored_recs = [&](int64_t k, int64_t n) {                            // R^n of a stored segment
    return w.recs(d, (char *)store.p + ((size_t)(k - k0) * seg + (size_t)(n - 1 - first_of(k))) * rbytes);
  };
  auto buffer_recs = [&](int b, int64_t k, int64_t n) {
    return w.recs(d, (char *)rb[b].p + (size_t)(n - 1 - first_of(k)) * rbytes);
  };
  const KArgs a = make_args(d);
  const DevGeom g = geom(d);
  // ---- forward sweep s^0 .. s^{nrec}
  // Every forward step, stored or not, runs the record kernel (the records
  // of a segment that is not stored go to a record buffer the recompute
  // overwrites later): the recompute then repeats exactly the steps of the
  // sweep, so the gradient does not depend on how many segments are
  // stored.  (A separately compiled kernel, like the plain step, need not
  // round every value the same way.)
  std::optional<NvtxRange> nvtx_fwd;
  nvtx_fwd.emplace("pemlbm.grad.forward");
  CK(cudaMemcpyAsync(fs[0].p, d->pop[d->cur], sbytes, cudaMemcpyDeviceToDevice, d->stream));
  int fc = 0;   // fs[fc] holds the latest state
  for (int64_t k = 0; k < nseg; ++k) {
    if (k < k0)
      CK(cudaMemcpyAsync((char *)ck.p + (size_t)k * sbytes, fs[fc].p, sbytes,
                         cudaMemcpyDeviceToDevice, d->stream));
    for (int64_t n = first_of(k) + 1; n <= last_of(k); ++n) {
      step_with_records(d, fs[fc].p, fs[fc ^ 1].p,
                        k >= k0 ? stored_recs(k, n) : buffer_recs(0, k, n), d->stream);
      fc ^= 1;
    }
  }
  CK(cudaGetLastError());
  nvtx_fwd.reset();
  const void *sN1 = objective == 1 ? fs[fc ^ 1].p : fs[fc].p;   // s^{N-1}
  // ---- segment recompute (rstream): R^n of segment k into buffer k & 1
  auto recompute = [&](int64_t k) -> lbm_status {
    const int b = (int)(k & 1);
    CK(cudaStreamWaitEvent(sync.rs, sync.freed[b], 0));
    CK(cudaMemcpyAsync(rs[0].p, (char *)ck.p + (size_t)k * sbytes, sbytes,
                       cudaMemcpyDeviceToDevice, sync.rs));
    int c = 0;
    for (int64_t n = first_of(k) + 1; n <= last_of(k); ++n) {
      step_with_records(d, rs[c].p, rs[c ^ 1].p, buffer_recs(b, k, n), sync.rs);
      c ^= 1;
    }
    CK(cudaEventRecord(sync.ready[b], sync.rs));
    CK(cudaGetLastError());
    return LBM_OK;
  };
  if (k0 > 0)
    for (int b = 0; b < 2; ++b) CK(cudaEventRecord(sync.freed[b], d->stream));
  // ---- objective and its seed
  NvtxRange nvtx_rev("pemlbm.grad.reverse");
  int cur = 0;
  long long seed_cell = -1;
  bool fresh = true;   // lam[cur] is the seed, held in full (see reverse_step)
  const lbm_params &p = d->prm;
  if (objective == 0) {
    const double i_scale = 4.0 * p.F * p.c_tot * p.dx_cm / p.dt_s;
    dispatch(d->desc.precision, [&](auto *tag) {
      using S = std::remove_pointer_t<decltype(tag)>;
      launch_catalyst<S>(sN1, g, a, i_scale, nullptr, d->colsum, d->dsmall, d->stream);
      launch_adj_seed_current<S>(sN1, g, a, d->prm.interface_mode == 1, i_scale / d->nx,
                                 w.ptrs(1), d->stream);   // writes lam[0]
    });
    CK(cudaMemcpyAsync(d->hsmall, d->dsmall, sizeof(double), cudaMemcpyDeviceToHost, d->stream));
    CK(cudaStreamSynchronize(d->stream));
    if (J) *J = d->hsmall[0] * i_scale / d->nx;
  } else {
    if ((s = ensure_scratch(d)) != LBM_OK) return s;
    dispatch(d->desc.precision, [&](auto *tag) {
      using S = std::remove_pointer_t<decltype(tag)>;
      launch_fields<S>(sN1, g, a, d->scratch, d->stream);
    });
    std::vector<double> Trow(d->nx);
    const size_t n = (size_t)d->nx * d->ny;
    CK(cudaMemcpyAsync(Trow.data(), d->scratch + 3 * n, sizeof(double) * d->nx,
                       cudaMemcpyDeviceToHost, d->stream));
    CK(cudaStreamSynchronize(d->stream));
    int xs = 0;
    for (int x = 1; x < d->nx; ++x)
      if (Trow[x] > Trow[xs]) xs = x;       // ties: the smallest x
    if (J) *J = Trow[xs];
    seed_cell = xs;                          // row 0
    // lambda^N = 0 with the seed added by the reverse of step N
    CK(cudaMemsetAsync(w.lam[0].p, 0, 24 * (size_t)d->plane * w.rsize, d->stream));
  }
  // ---- reverse sweep, last segment first
  if (nseg - 1 < k0 && nseg - 1 >= 0 && (s = recompute(nseg - 1)) != LBM_OK) return s;
  for (int64_t k = nseg - 1; k >= 0; --k) {
    if (k - 1 >= 0 && k - 1 < k0 && (s = recompute(k - 1)) != LBM_OK) return s;
    const bool stored = k >= k0;
    const int b = (int)(k & 1);
    if (!stored) CK(cudaStreamWaitEvent(d->stream, sync.ready[b], 0));
    for (int64_t n = last_of(k); n >= first_of(k) + 1; --n) {
      const RecBufs r = stored ? stored_recs(k, n) : buffer_recs(b, k, n);
      if (objective == 1 && n == N) {
        reverse_step(d, w, cur, r, seed_cell, true);   // lam[1] = lambda^{N-1}
      } else {
        reverse_step(d, w, cur, r, -1, fresh);
      }
      fresh = false;
      cur ^= 1;
    }
    fold_grads(d, w);
    if (!stored) CK(cudaEventRecord(sync.freed[b], d->stream));
    CK(cudaGetLastError());
  }
  finish_lambda(d, w, cur);   // adds the last step's outlet term to gphi
  return copy_grads_out(d, w, dphi, dK, dD_O2, du_in, on_device == 1);
}

lbm_status lbm_bounds_check(uint64_t *first_bad) {
  if (!first_bad) return fail(LBM_EINVAL, "null argument");
  *first_bad = 0;
#ifndef PEMLBM_BOUNDS_CHECK
  return fail(LBM_ESTATE, "this library was built without bounds checks");
#else
  CK(cudaDeviceSynchronize());
  const unsigned long long v[4] = {bounds_first_bad<float>(), bounds_first_bad<double>(),
                                   bounds_first_bad<__nv_bfloat16>(), bounds_first_bad<__half>()};
  for (unsigned long long x : v)
    if (x && !*first_bad) *first_bad = x;
  CK(cudaGetLastError());
  return LBM_OK;
#endif
}

lbm_status lbm_set_grad_memory(lbm_domain *d, int64_t bytes) {
  if (!d) return fail(LBM_EINVAL, "null domain");
  if (bytes < -1) return fail(LBM_EINVAL, "bytes must be -1 (automatic) or >= 0");
  d->grad_mem_limit = bytes;
  return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched stepping of many domains (operating-point sweeps).
struct lbm_batch {
  std::vector<lbm_domain *> doms;
  int precision = LBM_FP32;
  cudaStream_t stream = nullptr;
  BatchCase *dcases = nullptr;      // device case table
  BatchCase *hcases = nullptr;      // pinned host staging of the table
  int *dtile = nullptr;             // device tile prefix sums [ncases + 1]
  int tile_bx = 0, tile_by = 0;     // tile shape of the current prefix sums
  int total_tiles = 0;
  int schedule = 0;                 // 0 per-step launches, 1 persistent, 2 launch per case
  int variant = 6;
  long long spin_limit = 1LL << 24; // polls of the grid barrier before giving up
  unsigned *dbar = nullptr;         // barrier counter and generation
  int *dstatus = nullptr;
  cudaGraphExec_t graph = nullptr;
  std::vector<cudaEvent_t> ev;      // one per domain, for stream ordering
  cudaEvent_t ev_batch = nullptr, ev0 = nullptr, ev1 = nullptr;
  // schedule 3: one stream ("lane") per case, each case's steps a chain of
  // single-domain launches; the chains run concurrently, replayed from one
  // graph captured for the cases' current buffers (conc_cur)
  std::vector<cudaStream_t> lanes;
  std::vector<cudaEvent_t> lane_done;
  cudaEvent_t ev_fork = nullptr;
  cudaGraphExec_t conc_graph = nullptr;
  std::vector<int> conc_cur;
  std::vector<KArgs> conc_args;     // the arguments the graph's launches carry
};

namespace {

constexpr int kBatchGraphSteps = 64;

void drop_batch_graph(lbm_batch *b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  if (b->conc_graph) {
    cudaGraphExecDestroy(b->conc_graph);
    b->conc_graph = nullptr;
  }
}

// Schedule 3: n steps of every case, each case on its own lane stream,
// forked from and joined back into the batch stream.  fixed_parity: every
// step starts from the case's current state (tuner trials).
lbm_status batch_lanes(lbm_batch *b, int64_t n, bool fixed_parity) {
  const int nc = (int)b->doms.size();
  if ((int)b->lanes.size() != nc) {
    // all or nothing: a partial set is released, so a later call starts over
    auto release = [&] {
      for (auto st : b->lanes)
        if (st) cudaStreamDestroy(st);
      for (auto e : b->lane_done)
        if (e) cudaEventDestroy(e);
      if (b->ev_fork) cudaEventDestroy(b->ev_fork);
      b->lanes.clear();
      b->lane_done.clear();
      b->ev_fork = nullptr;
      cudaGetLastError();
    };
    b->lanes.assign(nc, nullptr);
    b->lane_done.assign(nc, nullptr);
    bool ok = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    for (int c = 0; c < nc && ok; ++c)
      ok = cudaStreamCreateWithFlags(&b->lanes[c], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&b->lane_done[c], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      release();
      return fail(LBM_ECUDA, "lane streams for the concurrent schedule");
    }
  }
  CK(cudaEventRecord(b->ev_fork, b->stream));
  for (int c = 0; c < nc; ++c) {
    lbm_domain *d = b->doms[c];
    const KArgs a = make_args(d);
    CK(cudaStreamWaitEvent(b->lanes[c], b->ev_fork, 0));
    for (int64_t k = 0; k < n; ++k) {
      const int src = fixed_parity ? d->cur : (int)(d->cur ^ (k & 1));
      dispatch(b->precision, [&](auto *tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        launch_step<S>(d->pop[src], d->pop[src ^ 1], geom(d), a, b->variant, b->lanes[c]);
      });
    }
    CK(cudaEventRecord(b->lane_done[c], b->lanes[c]));
    CK(cudaStreamWaitEvent(b->stream, b->lane_done[c], 0));
  }
  CK(cudaGetLastError());
  return LBM_OK;
}

// Tile prefix sums of all cases for a bx x by tile shape.
lbm_status batch_tiles(lbm_batch *b, int bx, int by) {
  if (b->tile_bx == bx && b->tile_by == by) return LBM_OK;
  const int n = (int)b->doms.size();
  std::vector<int> start(n + 1, 0);
  for (int c = 0; c < n; ++c) {
    const lbm_domain *d = b->doms[c];
    const long long t = (long long)((d->nx + bx - 1) / bx) * ((d->ny + by - 1) / by);
    if (start[c] + t > (1LL << 30)) return fail(LBM_EINVAL, "batch too large");
    start[c + 1] = start[c] + (int)t;
  }
  CK(cudaStreamSynchronize(b->stream));
  CK(cudaMemcpy(b->dtile, start.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice));
  b->tile_bx = bx;
  b->tile_by = by;
  b->total_tiles = start[n];
  drop_batch_graph(b);
  return LBM_OK;
}

// Uploads the case table (arguments, buffers, current parity of each case).
lbm_status batch_table(lbm_batch *b, int bx) {
  CK(cudaStreamSynchronize(b->stream));   // the staging buffer is reused
  std::vector<BatchCase> table(b->doms.size());
  for (size_t c = 0; c < b->doms.size(); ++c) {
    lbm_domain *d = b->doms[c];
    BatchCase &bc = table[c];
    bc.a = make_args(d);
    bc.pop[0] = d->pop[0];
    bc.pop[1] = d->pop[1];
    bc.mask = d->mask;
    bc.mid = d->mid;
    bc.pal = d->pal;
    bc.cur0 = d->cur;
    bc.tiles_x = (d->nx + bx - 1) / bx;
  }
  dispatch(b->precision, [&](auto *tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    batch_upload<S>(table.data(), (int)table.size(), b->hcases, b->dcases, b->stream);
  });
  CK(cudaGetLastError());
  return LBM_OK;
}

// Orders the batch stream after (before) the work of every domain's stream.
lbm_status batch_join_in(lbm_batch *b) {
  for (size_t c = 0; c < b->doms.size(); ++c) {
    CK(cudaEventRecord(b->ev[c], b->doms[c]->stream));
    CK(cudaStreamWaitEvent(b->stream, b->ev[c], 0));
  }
  return LBM_OK;
}
lbm_status batch_join_out(lbm_batch *b) {
  CK(cudaEventRecord(b->ev_batch, b->stream));
  for (lbm_domain *d : b->doms) CK(cudaStreamWaitEvent(d->stream, b->ev_batch, 0));
  return LBM_OK;
}

void batch_launch_steps(lbm_batch *b, int64_t n, int parity0) {
  for (int64_t k = 0; k < n; ++k)
    dispatch(b->precision, [&](auto *tag) {
      using S = std::remove_pointer_t<decltype(tag)>;
      launch_batch_step<S>(b->dcases, b->dtile, (int)b->doms.size(), b->total_tiles, b->variant,
                           (int)((parity0 + k) & 1), b->stream);
    });
}

lbm_status batch_run(lbm_batch *b, int64_t nsteps, bool fixed_parity) {
  const int n = (int)b->doms.size();
  if (b->schedule == 3) {              // concurrent chains of single-domain launches
    if (fixed_parity) return batch_lanes(b, nsteps, true);
    std::vector<int> cur(n);
    std::vector<KArgs> args(n);
    for (int c = 0; c < n; ++c) {
      cur[c] = b->doms[c]->cur;
      args[c] = make_args(b->doms[c]);
    }
    // the graph bakes in each case's buffers and arguments: recapture when
    // a case was stepped alone or its parameters changed
    if (b->conc_graph &&
        (cur != b->conc_cur ||
         std::memcmp(args.data(), b->conc_args.data(), sizeof(KArgs) * n) != 0))
      drop_batch_graph(b);
    int64_t left = nsteps;
    while (left >= 2 * kBatchGraphSteps) {
      if (!b->conc_graph) {
        cudaGraph_t gr = nullptr;
        CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        lbm_status s = batch_lanes(b, kBatchGraphSteps, false);
        cudaError_t e = cudaStreamEndCapture(b->stream, &gr);
        if (s != LBM_OK) return s;
        if (e != cudaSuccess) return fail(LBM_ECUDA, "lane graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->conc_graph, gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess) return fail(LBM_ECUDA, "lane graph instantiate: %s", cudaGetErrorString(e));
        b->conc_cur = cur;
        b->conc_args = args;
      }
      CK(cudaGraphLaunch(b->conc_graph, b->stream));   // even count: parities return
      left -= kBatchGraphSteps;
    }
    return left > 0 ? batch_lanes(b, left, false) : LBM_OK;
  }
  if (b->schedule == 2) {              // one launch per case and step, no graph
    for (int64_t k = 0; k < nsteps; ++k)
      for (lbm_domain *d : b->doms) {
        const KArgs a = make_args(d);
        const int src = fixed_parity ? d->cur : (int)(d->cur ^ (k & 1));
        dispatch(b->precision, [&](auto *tag) {
          using S = std::remove_pointer_t<decltype(tag)>;
          launch_step<S>(d->pop[src], d->pop[src ^ 1], geom(d), a, d->variant, b->stream);
        });
      }
    CK(cudaGetLastError());
    return LBM_OK;
  }
  if (b->schedule == 1) {              // persistent cooperative launch
    lbm_status s = batch_tiles(b, kPersistBX, kPersistBY * kBatchRows);
    if (s != LBM_OK) return s;
    if ((s = batch_table(b, kPersistBX)) != LBM_OK) return s;
    CK(cudaMemsetAsync(b->dbar, 0, 2 * sizeof(unsigned), b->stream));
    CK(cudaMemsetAsync(b->dstatus, 0, sizeof(int), b->stream));
    int steps_arg = (int)nsteps;
    if (fixed_parity) {
      // trials: the same step again and again from each case's current state
      for (int64_t k = 0; k < nsteps; ++k) {
        cudaError_t e = cudaSuccess;
        dispatch(b->precision, [&](auto *tag) {
          using S = std::remove_pointer_t<decltype(tag)>;
          e = launch_batch_persistent<S>(b->dcases, b->dtile, n, b->total_tiles, 1, b->dbar,
                                         b->dstatus, b->spin_limit, b->stream);
        });
        if (e != cudaSuccess) return fail(LBM_ECUDA, "persistent launch: %s", cudaGetErrorString(e));
        CK(cudaMemsetAsync(b->dbar, 0, 2 * sizeof(unsigned), b->stream));
      }
    } else {
      cudaError_t e = cudaSuccess;
      dispatch(b->precision, [&](auto *tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        e = launch_batch_persistent<S>(b->dcases, b->dtile, n, b->total_tiles, steps_arg, b->dbar,
                                       b->dstatus, b->spin_limit, b->stream);
      });
      if (e != cudaSuccess) return fail(LBM_ECUDA, "persistent launch: %s", cudaGetErrorString(e));
    }
    int status = 0;
    CK(cudaMemcpyAsync(&status, b->dstatus, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    if (status) {
      for (lbm_domain *d : b->doms) d->have_state = false;
      return fail(LBM_ETIMEOUT, "grid barrier gave up after %lld polls; states are undefined, "
                  "reset or load them", b->spin_limit);
    }
    return LBM_OK;
  }
  // schedule 0: one launch per step over all tiles, replayed from a graph
  const StepShape sh = kStepShapes[b->variant];
  lbm_status s = batch_tiles(b, sh.bx, sh.by * kBatchRows);
  if (s != LBM_OK) return s;
  if ((s = batch_table(b, sh.bx)) != LBM_OK) return s;
  if (fixed_parity) {
    for (int64_t k = 0; k < nsteps; ++k) batch_launch_steps(b, 1, 0);
    CK(cudaGetLastError());
    return LBM_OK;
  }
  int64_t left = nsteps;
  while (left >= 2 * kBatchGraphSteps) {
    if (!b->graph) {
      cudaGraph_t gr = nullptr;
      CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      batch_launch_steps(b, kBatchGraphSteps, 0);
      cudaError_t e = cudaStreamEndCapture(b->stream, &gr);
      if (e != cudaSuccess) return fail(LBM_ECUDA, "batch graph capture: %s", cudaGetErrorString(e));
      e = cudaGraphInstantiate(&b->graph, gr, 0);
      cudaGraphDestroy(gr);
      if (e != cudaSuccess) return fail(LBM_ECUDA, "batch graph instantiate: %s", cudaGetErrorString(e));
    }
    CK(cudaGraphLaunch(b->graph, b->stream));   // even count: parity returns to 0
    left -= kBatchGraphSteps;
  }
  batch_launch_steps(b, left, 0);
  CK(cudaGetLastError());
  return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_create_batch(lbm_domain *const *domains, int32_t ncases, lbm_batch **out) {
  if (!domains || !out || ncases < 1) return fail(LBM_EINVAL, "need at least one domain");
  *out = nullptr;
  for (int c = 0; c < ncases; ++c) {
    lbm_status s = check_ready(domains[c]);
    if (s != LBM_OK) return s;
    if (domains[c]->desc.precision != domains[0]->desc.precision)
      return fail(LBM_EINVAL, "batched domains must share one precision");
    if (domains[c]->desc.rounding != 0)
      return fail(LBM_EINVAL, "batched domains need round-to-nearest storage");
    if (needs_extended(make_args(domains[c])))
      return fail(LBM_EINVAL, "batched domains step the cathode set-up (no closed_x, buoyancy "
                  "or fixed wall values)");
    if (domains[c]->nx != domains[c]->nxg)
      return fail(LBM_EINVAL, "batched domains are whole lattices, not x-slabs");
    for (int k = 0; k < c; ++k)
      if (domains[k] == domains[c]) return fail(LBM_EINVAL, "domain %d appears twice", c);
  }
  lbm_batch *b = new lbm_batch();
  b->doms.assign(domains, domains + ncases);
  b->precision = domains[0]->desc.precision;
  b->stream = domains[0]->stream;
  b->ev.resize(ncases, nullptr);
  auto cleanup = [&](lbm_status s) { lbm_destroy_batch(b); return s; };
  if (dmalloc(&b->dcases, sizeof(BatchCase) * ncases) != cudaSuccess ||
      hmalloc(&b->hcases, sizeof(BatchCase) * ncases) != cudaSuccess ||
      dmalloc(&b->dtile, sizeof(int) * (ncases + 1)) != cudaSuccess ||
      dmalloc(&b->dbar, 2 * sizeof(unsigned)) != cudaSuccess ||
      dmalloc(&b->dstatus, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(fail(LBM_ENOMEM, "batch tables"));
  }
  for (auto &e : b->ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return cleanup(fail(LBM_ECUDA, "cudaEventCreate failed"));
  if (cudaEventCreateWithFlags(&b->ev_batch, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess)
    return cleanup(fail(LBM_ECUDA, "cudaEventCreate failed"));
  *out = b;
  return LBM_OK;
}

lbm_status lbm_destroy_batch(lbm_batch *b) {
  if (!b) return LBM_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_batch_graph(b);
  for (void *p : {(void *)b->dcases, (void *)b->dtile, (void *)b->dbar, (void *)b->dstatus})
    if (p) cudaFree(p);
  if (b->hcases) cudaFreeHost(b->hcases);
  for (auto e : b->ev)
    if (e) cudaEventDestroy(e);
  for (auto e : {b->ev_batch, b->ev0, b->ev1, b->ev_fork})
    if (e) cudaEventDestroy(e);
  for (auto e : b->lane_done)
    if (e) cudaEventDestroy(e);
  for (auto st : b->lanes)
    if (st) cudaStreamDestroy(st);
  delete b;
  return LBM_OK;
}

lbm_status lbm_batch_set_schedule(lbm_batch *b, int32_t schedule, int32_t variant,
                                  int64_t spin_limit) {
  if (!b) return fail(LBM_EINVAL, "null batch");
  if (schedule < 0 || schedule > 3) return fail(LBM_EINVAL, "schedule must be 0, 1, 2 or 3");
  if (variant < 0 || variant >= kStepVariants) return fail(LBM_EINVAL, "variant %d outside [0, %d)", variant, kStepVariants);
  b->schedule = schedule;
  if (b->variant != variant) drop_batch_graph(b);
  b->variant = variant;
  if (spin_limit > 0) b->spin_limit = spin_limit;
  return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch *b, int64_t nsteps) {
  NvtxRange nvtx_("pemlbm.batch_step");
  if (!b) return fail(LBM_EINVAL, "null batch");
  if (nsteps < 0 || nsteps > (1LL << 30)) return fail(LBM_EINVAL, "nsteps outside [0, 2^30]");
  for (lbm_domain *d : b->doms) {
    lbm_status s = check_ready(d);
    if (s != LBM_OK) return s;
  }
  if (nsteps == 0) return LBM_OK;
  lbm_status s = batch_join_in(b);
  if (s != LBM_OK) return s;
  if ((s = batch_run(b, nsteps, false)) != LBM_OK) return s;
  for (lbm_domain *d : b->doms) {
    d->cur ^= (int)(nsteps & 1);
    d->steps += nsteps;
  }
  return batch_join_out(b);
}

lbm_status lbm_batch_time_steps(lbm_batch *b, int64_t nsteps, double *elapsed_ms) {
  if (!b || !elapsed_ms) return fail(LBM_EINVAL, "null argument");
  lbm_status s = batch_join_in(b);
  if (s != LBM_OK) return s;
  CK(cudaEventRecord(b->ev0, b->stream));
  if ((s = lbm_batch_step(b, nsteps)) != LBM_OK) return s;
  CK(cudaEventRecord(b->ev1, b->stream));
  CK(cudaEventSynchronize(b->ev1));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
  *elapsed_ms = ms;
  return LBM_OK;
}

lbm_status lbm_batch_tune(lbm_batch *b, int32_t trial_steps, int32_t *schedule, int32_t *variant,
                          double *best_ms) {
  NvtxRange nvtx_("pemlbm.batch_tune");
  if (!b || trial_steps < 1) return fail(LBM_EINVAL, "bad argument");
  for (lbm_domain *d : b->doms) {
    lbm_status s = check_ready(d);
    if (s != LBM_OK) return s;
    if (d->steps != 0) return fail(LBM_ESTATE, "lbm_batch_tune runs between lbm_reset and the first step");
  }
  lbm_status s = batch_join_in(b);
  if (s != LBM_OK) return s;
  const int keep_sched = b->schedule, keep_var = b->variant;
  double best = 1e300;
  int best_sched = 0, best_var = 0;
  auto trial = [&](int sched, int var) -> lbm_status {
    b->schedule = sched;
    if (b->variant != var) drop_batch_graph(b);
    b->variant = var;
    lbm_status st = batch_run(b, 1, true);   // warm-up (tables, occupancy)
    if (st != LBM_OK) return st;
    CK(cudaEventRecord(b->ev0, b->stream));
    if ((st = batch_run(b, trial_steps, true)) != LBM_OK) return st;
    CK(cudaEventRecord(b->ev1, b->stream));
    CK(cudaEventSynchronize(b->ev1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
    if (ms / trial_steps < best) {
      best = ms / trial_steps;
      best_sched = sched;
      best_var = var;
    }
    return LBM_OK;
  };
  for (int v = 0; v < kStepVariants && s == LBM_OK; ++v) s = trial(0, v);
  if (s == LBM_OK) s = trial(1, 6);
  for (int v = 0; v < kStepVariants && s == LBM_OK; ++v) s = trial(3, v);
  // the trials wrote each case's next state into its other buffer: restore
  for (lbm_domain *d : b->doms) {
    const KArgs a = make_args(d);
    dispatch(b->precision, [&](auto *tag) {
      using S = std::remove_pointer_t<decltype(tag)>;
      launch_init<S>(d->pop[d->cur ^ 1], geom(d), a, b->stream);
    });
  }
  CK(cudaStreamSynchronize(b->stream));
  if (s != LBM_OK) {
    b->schedule = keep_sched;
    b->variant = keep_var;
    return s;
  }
  b->schedule = best_sched;
  if (b->variant != best_var) drop_batch_graph(b);
  b->variant = best_var;
  if (schedule) *schedule = best_sched;
  if (variant) *variant = best_var;
  if (best_ms) *best_ms = best;
  return batch_join_out(b);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// ------------------------------------------------------------- x-slabs
namespace {

lbm_status slab_pair_check(const lbm_domain *l, const lbm_domain *r) {
  if (!l || !r || l == r) return fail(LBM_EINVAL, "need two distinct slabs");
  if (!l->have_state || !r->have_state) return fail(LBM_ESTATE, "reset both slabs first");
  if (!l->halo_hi || !r->halo_lo || l->x0 + l->nx != r->x0 || l->nxg != r->nxg || l->ny != r->ny)
    return fail(LBM_EINVAL, "slabs [%d, %d) and [%d, %d) are not neighbours of one lattice", l->x0,
                l->x0 + l->nx, r->x0, r->x0 + r->nx);
  if (l->desc.precision != r->desc.precision) return fail(LBM_EINVAL, "slabs of different storage");
  for (int s = 0; s < 3; ++s)
    if (l->Cref[s] != r->Cref[s] || l->bref[s] != r->bref[s])
      return fail(LBM_EINVAL, "slabs with different deviation references (set both from the "
                  "same lattice arrays and parameters)");
  if (l->steps != r->steps) return fail(LBM_ESTATE, "slabs at different steps (%lld, %lld)",
                                        (long long)l->steps, (long long)r->steps);
  return LBM_OK;
}

HaloSide edge_of(lbm_domain *d, bool high) {   // the edge column a side sends from
  return HaloSide{d->pop[d->cur], d->plane, d->nxp, high ? (long long)d->nx - 1 : 0, 0};
}
HaloSide ghost_of(lbm_domain *d, bool high) {  // the ghost column a side receives into
  return HaloSide{d->pop[d->cur], d->plane, d->nxp, high ? (long long)d->nx : -1, 0};
}

lbm_status ensure_halo_event(lbm_domain *d) {
  if (!d->ev_halo && cudaEventCreateWithFlags(&d->ev_halo, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    d->ev_halo = nullptr;
    return fail(LBM_ECUDA, "cudaEventCreate failed");
  }
  return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_halo_exchange(lbm_domain *left, lbm_domain *right) {
  NvtxRange nvtx_("pemlbm.halo_exchange");
  lbm_status s = slab_pair_check(left, right);
  if (s != LBM_OK) return s;
  if ((s = ensure_halo_event(left)) != LBM_OK || (s = ensure_halo_event(right)) != LBM_OK) return s;
  // both slabs' last steps finish before the copies, which run on the left
  // slab's stream; the right slab's next step waits for them
  CK(cudaEventRecord(right->ev_halo, right->stream));
  CK(cudaStreamWaitEvent(left->stream, right->ev_halo, 0));
  const int es = (int)left->esize;
  launch_halo_copy(edge_of(left, true), ghost_of(right, false), left->ny, 1, es, left->stream);
  launch_halo_copy(edge_of(right, false), ghost_of(left, true), left->ny, 0, es, left->stream);
  CK(cudaGetLastError());
  CK(cudaEventRecord(left->ev_halo, left->stream));
  CK(cudaStreamWaitEvent(right->stream, left->ev_halo, 0));
  return LBM_OK;
}

extern "C" lbm_status lbm_halo_pack(lbm_domain *d, int32_t side, void *buf) {
  NvtxRange nvtx_("pemlbm.halo_pack");
  if (!d || !buf) return fail(LBM_EINVAL, "null argument");
  if (side != 0 && side != 1) return fail(LBM_EINVAL, "side must be 0 (low x) or 1 (high x)");
  if (!(side ? d->halo_hi : d->halo_lo)) return fail(LBM_EINVAL, "side %d borders no slab", side);
  if (!d->have_state) return fail(LBM_ESTATE, "call lbm_reset first");
  launch_halo_copy(edge_of(d, side == 1), HaloSide{buf, 0, 0, 0, 1}, d->ny, side == 1 ? 1 : 0,
                   (int)d->esize, d->stream);
  CK(cudaGetLastError());
  return LBM_OK;
}

extern "C" lbm_status lbm_halo_unpack(lbm_domain *d, int32_t side, const void *buf) {
  NvtxRange nvtx_("pemlbm.halo_unpack");
  if (!d || !buf) return fail(LBM_EINVAL, "null argument");
  if (side != 0 && side != 1) return fail(LBM_EINVAL, "side must be 0 (low x) or 1 (high x)");
  if (!(side ? d->halo_hi : d->halo_lo)) return fail(LBM_EINVAL, "side %d borders no slab", side);
  if (!d->have_state) return fail(LBM_ESTATE, "call lbm_reset first");
  // into the low ghost come the +x movers of the left neighbour, into the
  // high ghost the -x movers of the right neighbour
  launch_halo_copy(HaloSide{(void *)buf, 0, 0, 0, 1}, ghost_of(d, side == 1), d->ny,
                   side == 1 ? 0 : 1, (int)d->esize, d->stream);
  CK(cudaGetLastError());
  return LBM_OK;
}

// Residual without allocation.
//
// Some callers must not let the library allocate device memory once they are
// running: real-time loops, where a cudaMalloc can stall the device's streams
// for an unbounded time, and hosts whose device memory comes only from their
// own pool.  For them the block partial sums of the residual reduction live in
// this file-scope device array instead of in memory the library allocates.
// Every GPU that loads the library holds it (1.31 MB) until the process exits.
namespace {

constexpr int kNoAllocBlocks = 16384;    // residual blocks of 128 x 2 cells: 4.19 M cells
constexpr int kNoAllocSums = kNoAllocBlocks * 10;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocSums + 16];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
lbm_status noalloc_scratch(double **out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(LBM_EINVAL, "device %d beyond %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return fail(LBM_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_noalloc_ptr[dev] = (double *)p;
  }
  *out = g_noalloc_ptr[dev];
  return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_residual_noalloc(lbm_domain *d, void *snapshot, double *res) {
  NvtxRange nvtx_("pemlbm.residual_noalloc");
  if (!d || !snapshot || !res) return fail(LBM_EINVAL, "null argument");
  if (!d->have_state) return fail(LBM_ESTATE, "call lbm_reset first");
  const int nblocks = residual_blocks(d->nx, d->ny);
  if (nblocks > kNoAllocBlocks)
    return fail(LBM_EINVAL,
                "lattice of %d x %d cells needs %d residual blocks; lbm_residual_noalloc "
                "handles at most %d (about 4.19 M cells)",
                d->nx, d->ny, nblocks, kNoAllocBlocks);
  double *scratch = nullptr;
  lbm_status s = noalloc_scratch(&scratch);
  if (s != LBM_OK) return s;
  double *sums = scratch + kNoAllocSums;        // 10 sums
  int *bad = (int *)(scratch + kNoAllocSums + 10);
  // the flag must start at zero; the partials are fully rewritten each call
  CK(cudaMemsetAsync(bad, 0, sizeof(int), d->stream));
  const KArgs a = make_args(d);
  dispatch(d->desc.precision, [&](auto *tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    launch_residual<S>(d->pop[d->cur], geom(d), a, snapshot, snapshot, scratch, bad, sums,
                       d->stream);
  });
  CK(cudaGetLastError());
  double h[11];
  CK(cudaMemcpyAsync(h, sums, 11 * sizeof(double), cudaMemcpyDeviceToHost, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  int flag;
  std::memcpy(&flag, h + 10, sizeof(int));
  double r = 0.0;
  for (int k = 0; k < 5; ++k) {
    const double num = h[k], den = h[5 + k];
    r = std::fmax(r, den > 0 ? std::sqrt(num / den) : (num > 0 ? INFINITY : 0.0));
  }
  *res = r;
  if (flag || !std::isfinite(r)) return fail(LBM_EDIVERGED, "non-finite values in the state");
  return LBM_OK;
}
