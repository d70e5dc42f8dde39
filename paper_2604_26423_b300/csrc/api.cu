// api.cu -- C ABI of libqaoa.so (declared in include/qaoa.h).
//
// Host side of the LR-QAOA simulation: graph validation, the weight matrix,
// plans and their cost tables, phase tables, launches and result transfer.
// Every step of the simulation itself runs in the CUDA kernels included below.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <stdexcept>
#include <string>
#include <vector>

#include "qaoa.h"
#include "plan.h"
#include "desc.h"
#include "device.cuh"
#include "pass_kernel.cuh"
#include "aux_kernels.cuh"
#include "stats_kernels.cuh"
#include "noise_kernels.cuh"
#include "small_kernel.cuh"
#include "adj_kernel.cuh"
#include "spec.h"

using namespace qaoa;

namespace {

constexpr int kR = 5, kWB = 3;           // forward tile: 2^5 registers x 32 lanes x 8 warps

constexpr int kRAdj = 4, kWBAdj = 3;     // adjoint tile: psi and lambda, 2^4 registers each
constexpr int kSmaxAdj = 12;             // adjoint super-tile: one tile of psi and lambda
constexpr int kMinUnitsLog2 = 9;         // keep >= 512 super-tiles when n allows
// Largest sum of |w|: 2^20 where the cost phase comes from a table indexed by
// C(x) (complex128, and the whole-circuit kernels of n <= 12); 2^30 - 1 for
// complex64 passes, whose phase comes from 64-bit fixed-point turn products of
// the integer C(x) (the first pass's extremes keys hold C - C_min in 30 bits).
constexpr long long kMaxAbsWeightSum = 1 << 20;
constexpr long long kMaxAbsWeightSumTurns = (1ll << 30) - 1;
constexpr int kMaxGrid = 4096;           // persistent grid cap (partial-sum buffer size)
constexpr size_t kErrWordOffset = 32;    // the kernels' error word in the 64-byte result buffer
constexpr int kFuseSumsMinQubits = 26;   // final pass writes sampling block sums from here on
constexpr int kGroupOrder = ORDER_LOW_LAST;  // default group order of the pass plans
constexpr int kFloatLanes = PLAN_FLOAT_LANES;  // default: lane bits float to a plain pass
constexpr size_t kTileTableMaxBytes = size_t(1) << 30;  // per-context cap on per-tile constant tables

thread_local std::string g_init_error;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  cudaError_t ensure(size_t b) {
    if (bytes >= b && p) return cudaSuccess;
    if (p) cudaDeviceSynchronize();  // the old buffer may still be read by queued work
    release();
    cudaError_t e = cudaMalloc(&p, b);
    if (e == cudaSuccess) bytes = b; else p = nullptr;
    return e;
  }
};

}  // namespace

struct qaoa_ctx {
  int n = 0, m = 0, prec = QAOA_C64, cost_mode = QAOA_COST_RECOMPUTE;
  qaoa_opts opts{};  // kernel configuration (qaoa_set_opts; 0 = default)
  int shape_force = -1;  // forward tile id while the gradient runs its forward (the adjoint's tile)
  double scale = 0.1;
  std::vector<int32_t> u, v, w;
  std::vector<int32_t> wmat;  // n x n
  long long W = 0, c_lo = 0, c_hi = 0;
  cudaStream_t stream = nullptr;
  int sms = 0;
  void* state = nullptr;
  bool own_state = false;
  void* aux = nullptr;
  size_t aux_bytes = 0;
  DevBuf aux_own;
  DevBuf d_wmat, d_ctabs, d_phase, d_partial, d_result, d_ext, d_ext_part, d_ext_keys;
  DevBuf d_sums, d_pre, d_pre2, d_shots, d_uni, d_ang;
  DevBuf d_lambda, d_gacc;                                            // adjoint vector (if no aux), per-pass sums
  DevBuf d_ckpt;                                                      // the gradient's stored forward states
  DevBuf d_cutplanes, d_flag;                                         // weight bit planes (qaoa_sample_cuts), error flag
  int cut_planes = -1;                                                // planes in d_cutplanes (-1: not built)
  DevBuf d_noisy, d_ntraj;                                            // noisy trajectories: edges + angles, outputs
  TableStore tabs;                                                     // host copy of all cost tables
  std::map<std::vector<int8_t>, DevBuf> tct_tabs;                     // per-tile constant tables by sub-pass layout
  size_t tct_bytes = 0;
  std::map<std::pair<int, int>, std::unique_ptr<Plan>> plans;         // forward plans by (p, group order)
  std::map<std::pair<int, int>, std::unique_ptr<Plan>> bplans;        // adjoint plans by (p, group order)
  // per-kernel CUDA-event timing (qaoa_profile_enable / qaoa_profile_read)
  struct ProfRec { int kind; cudaEvent_t a, b; double bytes; };
  bool prof_on = false;
  std::vector<ProfRec> prof_pending;
  std::vector<cudaEvent_t> ev_pool;
  double prof_ms[5] = {0, 0, 0, 0, 0}, prof_bytes[5] = {0, 0, 0, 0, 0};
  long long prof_n[5] = {0, 0, 0, 0, 0};
  long long nlaunch = 0;  // every kernel launch while profiling is enabled
  Extreme ext{};
  bool ext_ready = false;    // ext holds C_min / C_max and their indices
  bool ext_pending = false;  // d_ext_keys holds them (written by a run's first pass)
  bool have_result = false;
  bool state_ready = false;
  bool sums_ready = false;  // d_sums holds the sampling block sums of the current state
  std::string err;
  int set_err(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    err = buf;
    return code;
  }
};

#define CUDA_TRY(ctx, expr)                                                               \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return (ctx)->set_err(QAOA_ECUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), \
                            __FILE__, __LINE__);                                          \
  } while (0)

namespace {

int amp_bytes(int prec) { return prec == QAOA_C128 ? 16 : 8; }

cudaEvent_t prof_event(qaoa_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one kernel launch with events on the context's stream (when enabled).
struct ProfScope {
  qaoa_ctx* c;
  int kind;
  double bytes;
  cudaEvent_t a = nullptr;
  ProfScope(qaoa_ctx* c_, int kind_, double bytes_) : c(c_), kind(kind_), bytes(bytes_) {
    if (c->prof_on) {
      a = prof_event(c);
      cudaEventRecord(a, c->stream);
    }
  }
  ~ProfScope() {
    if (a) {
      cudaEvent_t b = prof_event(c);
      cudaEventRecord(b, c->stream);
      c->prof_pending.push_back({kind, a, b, bytes});
    }
  }
};

// Forward tile shape ids (the kernels' instantiations):
//   0 "5x3": 2^5 registers x 8 warps, T = 13, 2 CTAs per SM
//   1 "4x4": 2^4 registers x 16 warps, T = 13
//   2 "5x2": 2^5 registers x 4 warps, T = 12, 4 CTAs per SM
//   3 "4x3": 2^4 registers x 8 warps, T = 12, 4 CTAs per SM (default: four
//      tiles in flight per SM keep HBM busier than two larger ones)
//   4 "5x4": 2^5 registers x 16 warps, T = 14, 1 CTA per SM (three mixer
//      groups at n = 33 with 128-byte runs: 7 passes for p = 3 instead of 10)
// complex128 accepts 5x3 (one CTA per SM, phase table in shared memory) and
// 4x3 (two CTAs per SM, phase table read through L1).
constexpr int kFwdShapeC64 = 3;
constexpr int kFwdShapeC128 = 3;  // measured 6% faster than 5x3 at K_32 (FP64-bound)
constexpr int kSmallMaxQubits = 12;  // n <= 12: whole circuit in one CTA (small_circuit_kernel)

// A configuration value: the context's option when set (nonzero), else the
// environment variable `env` when set and recognised, else the default.
// Options and variables use the qaoa_opts encodings (QAOA_ON / QAOA_OFF, ...).
int shape_from_name(const char* e) {
  if (!e) return -1;
  if (strcmp(e, "5x3") == 0) return 0;
  if (strcmp(e, "4x4") == 0) return 1;
  if (strcmp(e, "5x2") == 0) return 2;
  if (strcmp(e, "4x3") == 0) return 3;
  if (strcmp(e, "5x4") == 0) return 4;
  return -1;
}
// QAOA_SHAPE_* (qaoa.h) -> kernel shape id
int shape_from_opt(int o) {
  switch (o) {
    case QAOA_SHAPE_5x3: return 0;
    case QAOA_SHAPE_4x4: return 1;
    case QAOA_SHAPE_5x2: return 2;
    case QAOA_SHAPE_4x3: return 3;
    case QAOA_SHAPE_5x4: return 4;
    default: return -1;
  }
}
// The paired global layout in complex64 forward plans (QAOA_PAIRED=0 turns
// it off: 8-byte accesses only).
bool paired_layout_enabled() {
  const char* e = getenv("QAOA_PAIRED");
  return !(e && strcmp(e, "0") == 0);
}

int on_off(int opt, const char* env, int dflt) {
  if (opt == QAOA_ON) return 1;
  if (opt == QAOA_OFF) return 0;
  const char* e = getenv(env);
  if (e && strcmp(e, "0") == 0) return 0;
  if (e && strcmp(e, "1") == 0) return 1;
  return dflt;
}

// Forward tile of a shape id; complex64 forward plans may use the paired
// global layout (16-byte accesses of two adjacent amplitudes).
TileShape shape_of(int id, int prec) {
  static const int R[5] = {kR, 4, 5, 4, 5}, WB[5] = {kWB, 4, 2, 3, 4};
  TileShape s;
  s.R = R[id];
  s.WB = WB[id];
  s.amp_bytes = amp_bytes(prec);
  s.paired = prec == QAOA_C64 && paired_layout_enabled();
  // the 5x4 tile's passes load their tiles by tensor loads (QAOA_PAIRED_STORE=0
  // keeps the paired first round)
  s.paired_store_first = s.paired && id == 4 && on_off(0, "QAOA_PAIRED_STORE", 1);
  return s;
}

// Default complex64 forward tile for n qubits: 5x4 (one CTA per SM, its next
// tile prefetched into L2) from 27 qubits (its specialised kernels are
// compiled for n = 27..34) where it needs fewer mixer groups than 4x3 (n = 29
// .. 34: three instead of four, 7 passes instead of 10 at p = 3; measured 218
// against 227 ms per K_33 step and 24.4 against 27.9 ms at K_30), else 4x3
// (four CTAs per SM; equal pass counts favour it).
int default_shape_c64(int n) {
  static int cache[kMaxQubits + 1] = {};  // 0 unknown, else id + 1
  if (n < 27 || n > kMaxQubits) return kFwdShapeC64;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  if (!cache[n]) {
    int id = kFwdShapeC64;
    try {
      const int order = kGroupOrder | kFloatLanes;
      const TileShape a = shape_of(3, QAOA_C64), b = shape_of(4, QAOA_C64);
      const size_t ga = plan_forward(n, 1, a, a.T(), kMinUnitsLog2, order).groups.size();
      const size_t gb = plan_forward(n, 1, b, b.T(), kMinUnitsLog2, order).groups.size();
      if (gb < ga) id = 4;
    } catch (std::exception&) {
    }
    cache[n] = id + 1;
  }
  return cache[n] - 1;
}

int fwd_shape_id(const qaoa_ctx* c, int prec, int n) {
  const int o = c ? shape_from_opt(c->opts.fwd_shape) : -1;
  if (prec != QAOA_C64) {
    if (o == 0 || o == 3) return o;
    const int e = shape_from_name(getenv("QAOA_FWD_SHAPE_C128"));
    return (e == 0 || e == 3) ? e : kFwdShapeC128;
  }
  if (c && c->shape_force >= 0) return c->shape_force;
  if (o >= 0) return o;
  const int e = shape_from_name(getenv("QAOA_FWD_SHAPE"));
  return e >= 0 ? e : default_shape_c64(n);
}
int fwd_shape_id(const qaoa_ctx* c, int prec) { return fwd_shape_id(c, prec, c ? c->n : 0); }
TileShape fwd_shape(const qaoa_ctx* c, int prec) { return shape_of(fwd_shape_id(c, prec), prec); }

// L2 prefetch of the next tile: on by default with the one-CTA-per-SM 5x4 tile
// (measured faster), off with the others (measured slower).
int l2_prefetch_on(const qaoa_ctx* c, int shape_id) {
  return on_off(c->opts.l2_prefetch, "QAOA_L2PREFETCH", shape_id == 4 ? 1 : 0);
}

// Adjoint tile shape: two vectors per thread, 2^4 registers each x 8 warps (T = 12).
TileShape adj_shape(int prec) {
  TileShape s;
  s.R = kRAdj;
  s.WB = kWBAdj;
  s.amp_bytes = amp_bytes(prec);
  s.nvec = 2;
  return s;
}

int upload_ctabs(qaoa_ctx* c) {
  if (!c->tabs.dirty) return QAOA_OK;
  const size_t bytes = std::max<size_t>(4, c->tabs.h.size() * 4);
  CUDA_TRY(c, c->d_ctabs.ensure(bytes));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_ctabs.p, c->tabs.h.data(), c->tabs.h.size() * 4, cudaMemcpyHostToDevice,
                              c->stream));
  c->tabs.dirty = false;
  return QAOA_OK;
}

// Per-tile constant table of a forward sub-pass (tile_const_table_kernel),
// built on first use and kept per layout (tile bits, super-tile bits); nullptr
// (the kernel computes the constants per tile) when QAOA_TILE_TABLES=0 or the
// context's tables would pass kTileTableMaxBytes.
int tile_const_table(qaoa_ctx* c, const PassDev& pd, SubDev& sd) {
  sd.tct = nullptr;
  if (!on_off(c->opts.tile_tables, "QAOA_TILE_TABLES", 1)) return QAOA_OK;
  std::vector<int8_t> key(sd.pos, sd.pos + pd.T);
  key.push_back(-1);
  key.insert(key.end(), pd.outer, pd.outer + pd.nouter);
  key.push_back(-2);
  key.insert(key.end(), sd.inner, sd.inner + sd.ninner);
  auto it = c->tct_tabs.find(key);
  if (it != c->tct_tabs.end()) {
    sd.tct = (const int32_t*)it->second.p;
    return QAOA_OK;
  }
  const uint64_t ntiles = pd.n_units << sd.ninner;
  const size_t bytes = size_t(ntiles) * kTileConstInts * 4;
  if (c->tct_bytes + bytes > kTileTableMaxBytes) return QAOA_OK;
  DevBuf b;
  if (b.ensure(bytes) != cudaSuccess) {
    cudaGetLastError();  // out of memory: fall back to the in-kernel constants
    return QAOA_OK;
  }
  TileConstArgs a;
  memset(&a, 0, sizeof a);
  for (int j = 0; j < pd.T; ++j) a.pos[j] = sd.pos[j];
  a.outer = pd.outer_runs;
  a.inner = sd.inner_runs;
  a.T = pd.T;
  a.n = c->n;
  a.ninner = sd.ninner;
  a.ntiles = ntiles;
  a.wmat = (const int32_t*)c->d_wmat.p;
  a.out = (int32_t*)b.p;
  const uint64_t runs = (ntiles + (1ull << kTileConstRunBits) - 1) >> kTileConstRunBits;  // one per thread
  tile_const_table_kernel<<<(unsigned)((runs + 255) / 256), 256, 0, c->stream>>>(a);
  if (c->prof_on) ++c->nlaunch;
  const cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess) {
    b.release();
    return c->set_err(QAOA_ECUDA, "tile_const_table_kernel: %s", cudaGetErrorString(le));
  }
  c->tct_bytes += bytes;
  sd.tct = (const int32_t*)b.p;
  c->tct_tabs[key] = b;
  return QAOA_OK;
}

// Phase tables exp(-i gamma_k s (W - 2c)) for c in [c_lo, c_hi], FP64 on the
// host, rounded to the state precision (h(x) = W - 2 C(x), Eqs. H_C and UC).
// Whether any kernel of this context reads the phase table (see kMaxAbsWeightSum).
bool phase_table_needed(const qaoa_ctx* c) { return c->prec == QAOA_C128 || c->n <= kSmallMaxQubits; }

int upload_phases(qaoa_ctx* c, int p, const double* gamma) {
  if (!phase_table_needed(c)) return QAOA_OK;
  const long long nc = c->c_hi - c->c_lo + 1;
  const int ab = amp_bytes(c->prec);
  std::vector<unsigned char> host((size_t)std::max(1, p) * nc * ab);
  for (int k = 0; k < p; ++k)
    for (long long i = 0; i < nc; ++i) {
      const long long cc = c->c_lo + i;
      const double th = -gamma[k] * c->scale * double(c->W - 2 * cc);
      const double cr = cos(th), ci = sin(th);
      if (c->prec == QAOA_C128) {
        double* d = reinterpret_cast<double*>(host.data()) + 2 * (k * nc + i);
        d[0] = cr;
        d[1] = ci;
      } else {
        float* f = reinterpret_cast<float*>(host.data()) + 2 * (k * nc + i);
        f[0] = float(cr);
        f[1] = float(ci);
      }
    }
  CUDA_TRY(c, c->d_phase.ensure(host.size()));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_phase.p, host.data(), host.size(), cudaMemcpyHostToDevice, c->stream));
  return QAOA_OK;
}

// Largest super-tile (index bits kept together through L2 by one CTA) of the
// adjoint passes; QAOA_SMAX_ADJ overrides the default (one tile).
int smax_adj() {
  const char* e = getenv("QAOA_SMAX_ADJ");
  const int v = e ? atoi(e) : kSmaxAdj;
  return v >= 12 && v <= 20 ? v : kSmaxAdj;
}

// Floating lane bits in the forward plans (PLAN_FLOAT_LANES): option
// float_lanes, QAOA_FLOAT_LANES=0 or 1.
int float_lanes_flag(const qaoa_ctx* c) {
  return on_off(c ? c->opts.float_lanes : 0, "QAOA_FLOAT_LANES", kFloatLanes != 0) ? PLAN_FLOAT_LANES : 0;
}

int order_of(int opt, const char* env, int dflt) {
  if (opt == QAOA_ORDER_LOW_LAST) return ORDER_LOW_LAST;
  if (opt == QAOA_ORDER_LOW_MIDDLE) return ORDER_LOW_MIDDLE;
  const char* e = getenv(env);
  if (e && strcmp(e, "middle") == 0) return ORDER_LOW_MIDDLE;
  if (e && strcmp(e, "last") == 0) return ORDER_LOW_LAST;
  return dflt;
}

// Group order of the run's pass plans (plan.h): option group_order,
// QAOA_GROUP_ORDER=middle or last; with the floating-lane flag.
int group_order(const qaoa_ctx* c) {
  return order_of(c ? c->opts.group_order : 0, "QAOA_GROUP_ORDER", kGroupOrder) | float_lanes_flag(c);
}

// Specialised pass kernels (spec.h): option specialised, QAOA_SPEC=0 selects
// the generic ones.
bool spec_enabled(const qaoa_ctx* c) { return on_off(c->opts.specialised, "QAOA_SPEC", 1) != 0; }

// Asynchronous tile copies in the adjoint passes (QAOA_ADJ_PREFETCH=1 enables;
// measured slower than the register loads with the specialised kernels).
// Tensor loads of whole tiles into shared memory in the forward passes that
// have a tensor prefetch (option tma_load, QAOA_TMA_LOAD)
bool tma_load_on(const qaoa_ctx* c) { return on_off(c->opts.tma_load, "QAOA_TMA_LOAD", 1) != 0; }

// Tensor L2 prefetch of the adjoint's next tile (option adj_l2_prefetch,
// QAOA_ADJ_L2_PREFETCH)
bool adj_l2_prefetch(const qaoa_ctx* c) { return on_off(c->opts.adj_l2_prefetch, "QAOA_ADJ_L2_PREFETCH", 0) != 0; }

bool adj_prefetch() {
  const char* e = getenv("QAOA_ADJ_PREFETCH");
  return e && strcmp(e, "1") == 0;
}

// group orders of the gradient's forward and adjoint plans (option
// grad_order, QAOA_GRAD_ORDER)
int grad_base_order(const qaoa_ctx* c) { return order_of(c->opts.grad_order, "QAOA_GRAD_ORDER", ORDER_LOW_MIDDLE); }
int grad_fwd_order(const qaoa_ctx* c) { return grad_base_order(c) | float_lanes_flag(c); }
int grad_bwd_order(const qaoa_ctx* c) { return grad_base_order(c); }

// Stored forward states in the gradient (option grad_checkpoint,
// QAOA_GRAD_CHECKPOINT=0 disables).
bool grad_checkpoint(const qaoa_ctx* c) { return on_off(c->opts.grad_checkpoint, "QAOA_GRAD_CHECKPOINT", 1) != 0; }

// Largest forward super-tile: option super_tile, QAOA_SMAX; T (one tile) by default.
int smax_fwd(const qaoa_ctx* c, int T) {
  int v = c ? c->opts.super_tile : 0;
  if (v <= 0) {
    const char* e = getenv("QAOA_SMAX");
    v = e ? atoi(e) : T;
  }
  return v >= T && v <= 20 ? v : T;
}

const Plan* get_plan(qaoa_ctx* c, int p, int order) {
  const auto key = std::make_pair(p, order | fwd_shape_id(c, c->prec) << 8);
  auto it = c->plans.find(key);
  if (it != c->plans.end()) return it->second.get();
  const TileShape sh = fwd_shape(c, c->prec);
  auto pl = std::make_unique<Plan>(plan_forward(c->n, p, sh, smax_fwd(c, sh.T()), kMinUnitsLog2, order));
  const Plan* r = pl.get();
  c->plans[key] = std::move(pl);
  return r;
}

template <typename Real, bool FAST, bool CC, int R = kR, int WB = kWB>
int launch_pass(qaoa_ctx* c, const PassDev& pd, const PassArgs& pa, const PassTma& pt, size_t smem, int grid) {
  auto kern = fwd_pass_kernel<Real, R, WB, FAST, CC>;
  CUDA_TRY(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, 32 << WB, smem, c->stream>>>(pd, pa, pt);
  if (c->prof_on) ++c->nlaunch;
  CUDA_TRY(c, cudaGetLastError());
  return QAOA_OK;
}

template <typename Real, bool FAST, bool CC, int R = kR, int WB = kWB>
int blocks_per_sm(qaoa_ctx* c, size_t smem, int* nb) {
  auto kern = fwd_pass_kernel<Real, R, WB, FAST, CC>;
  CUDA_TRY(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, kern, 32 << WB, smem));
  if (*nb < 1) return c->set_err(QAOA_ECUDA, "pass kernel does not fit on an SM (smem %zu)", smem);
  return QAOA_OK;
}

// Instantiation for (precision, tile shape, mixer form, C(x) code): occupancy
// query when `launch` is false, else the launch.
template <bool FAST, bool CC>
int pass_dispatch(qaoa_ctx* c, int shape, bool launch, const PassDev& pd, const PassArgs& pa, const PassTma& pt,
                  size_t smem, int grid,
                  int* bps) {
  if (c->prec == QAOA_C128) {
    if (shape == 3)
      return launch ? launch_pass<double, FAST, CC, 4, 3>(c, pd, pa, pt, smem, grid)
                    : blocks_per_sm<double, FAST, CC, 4, 3>(c, smem, bps);
    return launch ? launch_pass<double, FAST, CC>(c, pd, pa, pt, smem, grid) : blocks_per_sm<double, FAST, CC>(c, smem, bps);
  }
  if (shape == 1)
    return launch ? launch_pass<float, FAST, CC, 4, 4>(c, pd, pa, pt, smem, grid)
                  : blocks_per_sm<float, FAST, CC, 4, 4>(c, smem, bps);
  if (shape == 2)
    return launch ? launch_pass<float, FAST, CC, 5, 2>(c, pd, pa, pt, smem, grid)
                  : blocks_per_sm<float, FAST, CC, 5, 2>(c, smem, bps);
  if (shape == 3)
    return launch ? launch_pass<float, FAST, CC, 4, 3>(c, pd, pa, pt, smem, grid)
                  : blocks_per_sm<float, FAST, CC, 4, 3>(c, smem, bps);
  if (shape == 4)
    return launch ? launch_pass<float, FAST, CC, 5, 4>(c, pd, pa, pt, smem, grid)
                  : blocks_per_sm<float, FAST, CC, 5, 4>(c, smem, bps);
  return launch ? launch_pass<float, FAST, CC>(c, pd, pa, pt, smem, grid) : blocks_per_sm<float, FAST, CC>(c, smem, bps);
}

int pass_any(qaoa_ctx* c, bool fast, bool cc, int wide, bool launch, const PassDev& pd, const PassArgs& pa,
             const PassTma& pt,
             size_t smem, int grid, int* bps) {
  if (fast) return cc ? pass_dispatch<true, true>(c, wide, launch, pd, pa, pt, smem, grid, bps)
                      : pass_dispatch<true, false>(c, wide, launch, pd, pa, pt, smem, grid, bps);
  return cc ? pass_dispatch<false, true>(c, wide, launch, pd, pa, pt, smem, grid, bps)
            : pass_dispatch<false, false>(c, wide, launch, pd, pa, pt, smem, grid, bps);
}

int run_small(qaoa_ctx* c, int p, const double* gamma, const double* beta) {
  const int n = c->n;
  CUDA_TRY(c, c->d_ang.ensure(sizeof(double) * 2 * std::max(1, p)));
  std::vector<double> ang(2 * std::max(1, p));
  for (int k = 0; k < p; ++k) { ang[2 * k] = gamma[k]; ang[2 * k + 1] = beta[k]; }
  CUDA_TRY(c, cudaMemcpyAsync(c->d_ang.p, ang.data(), ang.size() * 8, cudaMemcpyHostToDevice, c->stream));
  SmallArgs sa;
  sa.n = n;
  sa.p = p;
  sa.state = c->state;
  sa.wmat = (const int32_t*)c->d_wmat.p;
  sa.phase = c->d_phase.p;
  sa.c_lo = (int)c->c_lo;
  sa.ncost = (int)(c->c_hi - c->c_lo + 1);
  sa.betas = (const double*)c->d_ang.p;
  sa.result = (double*)c->d_result.p;
  const size_t smem = (size_t(1) << n) * amp_bytes(c->prec);
  ProfScope ps(c, 4, double(smem));
  if (c->prec == QAOA_C128) {
    CUDA_TRY(c, cudaFuncSetAttribute(small_circuit_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    small_circuit_kernel<double><<<1, 512, smem, c->stream>>>(sa);
    if (c->prof_on) ++c->nlaunch;
  } else {
    CUDA_TRY(c, cudaFuncSetAttribute(small_circuit_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    small_circuit_kernel<float><<<1, 512, smem, c->stream>>>(sa);
    if (c->prof_on) ++c->nlaunch;
  }
  CUDA_TRY(c, cudaGetLastError());
  return QAOA_OK;
}

// Tensor map for the L2 prefetch of a forward pass's tiles (PassArgs, prefetch
// mode 2): the input state as 8-byte elements over runs of index bits (tile
// runs cut into dimensions of at most 8 bits, the box extent; every outer run
// one dimension of box extent 1), at most five dimensions. False when the pass
// does not fit that form or the driver's encoder is unavailable.
using TensorMapEncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                       const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                       CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
TensorMapEncodeFn tensor_map_encoder() {
  static TensorMapEncodeFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f = nullptr;
    }
    return reinterpret_cast<TensorMapEncodeFn>(f);
  }();
  return fn;
}

// Whether a pass has the form the tensor tile loads need: one sub-pass of one
// tile per super-tile, at least two rounds, the first loading the state, the
// last reading shared memory and writing the state, none other writing it.
bool tma_load_form(const PassDev& pd) {
  if (pd.nsub != 1 || pd.sub[0].ninner != 0) return false;
  const SubDev& sd = pd.sub[0];
  const int nr = sd.nrounds;
  if (nr < 2 || sd.rd[0].src != SRC_GLOBAL_D || sd.rd[nr - 1].src != SRC_SMEM_D || sd.rd[nr - 1].dst != DST_GLOBAL_D)
    return false;
  for (int r = 0; r + 1 < nr; ++r)
    if (sd.rd[r].dst != DST_SMEM_D || (r > 0 && sd.rd[r].src != SRC_SMEM_D)) return false;
  return true;
}

// Whether a pass's shared-memory rounds can use dense tile-index slots: one
// sub-pass of one tile per super-tile and no round whose lanes lie above
// tile bit 5 (menu layout 2, which needs the padding against bank conflicts).
bool dense_form(const PassDev& pd) {
  if (pd.nsub != 1 || pd.sub[0].ninner != 0) return false;
  for (int r = 0; r < pd.sub[0].nrounds; ++r)
    if (pd.sub[0].rd[r].layout == 2) return false;
  return true;
}

bool prefetch_tensor_map(int n, const PassDev& pd, const void* base, PassTma& pt, CUtensorMap* map) {
  const TensorMapEncodeFn enc = tensor_map_encoder();
  if (!enc || pd.nsub != 1 || pd.sub[0].ninner != 0) return false;
  const SubDev& sd = pd.sub[0];
  uint64_t tmask = 0;
  for (int j = 0; j < pd.T; ++j) tmask |= 1ull << sd.pos[j];
  int dims = 0;
  int bit[8], len[8];
  bool tile[8];
  for (int b = 0; b < n;) {
    const bool t = (tmask >> b & 1ull) != 0;
    int e = b;
    while (e < n && ((tmask >> e & 1ull) != 0) == t) ++e;
    while (b < e) {
      const int l = t ? std::min(8, e - b) : e - b;
      if (dims == 8 || l > 31) return false;
      bit[dims] = b;
      len[dims] = l;
      tile[dims] = t;
      ++dims;
      b += l;
    }
  }
  if (dims > 5 || !tile[0] || bit[0] != 0 || len[0] < 1) return false;
  cuuint64_t gdim[5], gstride[4];
  cuuint32_t box[5], estr[5];
  for (int d = 0; d < dims; ++d) {
    gdim[d] = 1ull << len[d];
    box[d] = tile[d] ? (cuuint32_t)(1u << len[d]) : 1u;
    estr[d] = 1;
    if (d) gstride[d - 1] = 8ull << bit[d];
  }
  if ((box[0] * 8) % 16) return false;
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, (cuuint32_t)dims, const_cast<void*>(base), gdim,
                         gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return false;
  pt.tdims = dims;
  pt.ttile = 0;
  for (int d = 0; d < dims; ++d) {
    pt.tbit[d] = (int8_t)bit[d];
    pt.tlen[d] = (int8_t)len[d];
    if (tile[d]) pt.ttile |= uint8_t(1u << d);
  }
  return true;
}

// reduce = false: the final pass skips <C> and norm (the gradient takes <C>
// from the adjoint's first pass instead). outs: null (every pass in place on
// the state) or one output buffer per pass of the plan, the last being the
// state; pass k then reads outs[k-1] and writes outs[k].
int run_forward(qaoa_ctx* c, int p, const double* gamma, const double* beta, int order, bool reduce = true,
                void* const* outs = nullptr) {
  const int n = c->n;
  const TileShape sh = fwd_shape(c, c->prec);
  const int T = sh.T();
  const int ab = amp_bytes(c->prec);
  c->state_ready = false;
  c->have_result = false;
  c->sums_ready = false;
  int rc = upload_phases(c, p, gamma);
  if (rc) return rc;
  if (n < std::max(T, kSmallMaxQubits + 1)) {
    rc = run_small(c, p, gamma, beta);
    if (rc) return rc;
    c->have_result = c->state_ready = true;
    return QAOA_OK;
  }
  const Plan* plan;
  try {
    plan = get_plan(c, p, order);
  } catch (std::exception& ex) {
    return c->set_err(QAOA_EINVAL, "planner: %s", ex.what());
  }
  const bool stream = c->cost_mode == QAOA_COST_STREAM;
  const long long nc = c->c_hi - c->c_lo + 1;
  // shared memory: tile | weights + tile consts | phase table (if it fits)
  const size_t tile_amps = ab == 8 ? padded_size<8>(T) : padded_size<16>(T);
  const size_t base_smem = ((tile_amps * ab + kTconstSmemInts * 4 + 15) & ~size_t(15));
  const size_t with_tab = base_smem + size_t(nc) * ab;
  int dev = 0, max_smem = 0;
  CUDA_TRY(c, cudaGetDevice(&dev));
  CUDA_TRY(c, cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  // complex64 kernels compute the phase (phase_turns); complex128 reads the table
  const bool tab_smem = c->prec == QAOA_C128 && fwd_shape_id(c, c->prec) == 0 && with_tab + 1024 <= (size_t)max_smem;
  const size_t smem = tab_smem ? with_tab : base_smem;

  // build every pass descriptor (and its cost tables) before launching
  std::vector<PassDev> pds(plan->passes.size());
  std::vector<char> fasts(plan->passes.size());
  bool fused_sums = false;
  PassInputs in;
  in.n = n;
  in.beta = beta;
  in.gamma = gamma;
  in.scale = c->scale;
  in.c_lo = c->c_lo;
  in.ncost = nc;
  in.W = c->W;
  in.wmat = c->wmat.data();
  in.stream = stream;
  in.adjoint = false;
  std::vector<char> ccs(plan->passes.size());
  for (size_t pi = 0; pi < plan->passes.size(); ++pi) {
    bool fast = true;
    const std::string why = fill_pass_dev(plan->passes[pi], sh, in, c->tabs, pds[pi], fast);
    if (!why.empty()) return c->set_err(QAOA_EINVAL, "%s", why.c_str());
    fasts[pi] = fast;
    bool cc = false;
    for (int si = 0; si < pds[pi].nsub; ++si) {
      SubDev& sd = pds[pi].sub[si];
      bool need = false;
      for (int r = 0; r < sd.nrounds; ++r) {
        if (!reduce) sd.rd[r].reduce = 0;
        need = need || sd.rd[r].cost || sd.rd[r].reduce;
      }
      if (!reduce) sd.needs_c = need;
      cc = cc || sd.needs_c || sd.init;
      if (sd.needs_c && !stream) {
        rc = tile_const_table(c, pds[pi], sd);
        if (rc) return rc;
      }
    }
    ccs[pi] = cc;
  }
  rc = upload_ctabs(c);
  if (rc) return rc;
  for (size_t pi = 0; pi < plan->passes.size(); ++pi) {
    const PassPlan& pp = plan->passes[pi];
    const PassDev& pd = pds[pi];
    const bool fast = fasts[pi];
    PassArgs pa;
    PassTma pt;
    pa.state = outs && pi > 0 ? outs[pi - 1] : c->state;
    pa.out = outs ? outs[pi] : c->state;
    if (pa.out != pa.state && pd.nsub != 1)
      return c->set_err(QAOA_EINVAL, "a pass of several sub-passes cannot write to another buffer");
    pa.diag = stream ? (const int32_t*)((char*)c->aux + (c->aux_bytes - (size_t(4) << n))) : nullptr;
    pa.phase = pp.layer_c >= 0 && c->d_phase.p
                   ? (const void*)((const char*)c->d_phase.p + size_t(pp.layer_c) * nc * ab) : nullptr;
    pa.wmat = (const int32_t*)c->d_wmat.p;
    pa.ctabs = (const int32_t*)c->d_ctabs.p;
    pa.phase_in_smem = tab_smem ? 1 : 0;
    {
      const char* e = getenv("QAOA_L2HINT");
      pa.l2hint = (e && atoi(e) != 0) ? 1 : 0;
      // the next tile into L2: one tensor prefetch per tile where the pass has
      // a tensor form, else one line per 16-amplitude run
      pa.prefetch = l2_prefetch_on(c, fwd_shape_id(c, c->prec));
      memset(&pt, 0, sizeof pt);
      {
        const char* d = getenv("QAOA_PREFETCH_DIST");
        pt.pfdist = d ? std::max(0, std::min(4, atoi(d))) : 1;
      }
      if (pa.prefetch && !pp.init && prefetch_tensor_map(n, pd, pa.state, pt, &pt.tmap)) pa.prefetch = 2;
      // tensor stores of each tile from shared memory (complex64, one tile
      // per super-tile): option tma_store, QAOA_TMA_STORE
      pa.tma_store = 0;
      const char* ts = getenv("QAOA_TMA_STORE");  // 1: every eligible pass, 2: the write-only first pass
      const int tsm = ts ? atoi(ts) : 0;
      if (c->prec == QAOA_C64 && (tsm == 1 || (tsm == 2 && pp.init)) && pd.nsub == 1 && pd.sub[0].ninner == 0) {
        PassTma probe = pt;
        if (prefetch_tensor_map(n, pd, pa.out, probe, &pt.smap) &&
            (pa.prefetch != 2 || (probe.tdims == pt.tdims && probe.ttile == pt.ttile))) {
          pt.tdims = probe.tdims;
          pt.ttile = probe.ttile;
          for (int d = 0; d < 5; ++d) { pt.tbit[d] = probe.tbit[d]; pt.tlen[d] = probe.tlen[d]; }
          pa.tma_store = 1;
        }
      }
      // tensor loads of each tile into shared memory (complex64, one tile per
      // super-tile, the first round loads the state and only the last round,
      // which reads shared memory, writes it): QAOA_TMA_LOAD
      pa.tma_load = 0;
      if (c->prec == QAOA_C64 && pa.prefetch == 2 && !pa.tma_store && tma_load_on(c) && tma_load_form(pd))
        pa.tma_load = 1;
      // dense shared-memory slots (QAOA_DENSE)
      pa.dense = 0;
      // (only where they drop the tile's first barrier: with the 4x3 tile's
      // passes, which load through the load-store unit, they measured slower)
      if (c->prec == QAOA_C64 && on_off(0, "QAOA_DENSE", 1) && dense_form(pd)) {
        const RoundDev& r0 = pd.sub[0].rd[0];
        pa.dense = pa.tma_load && !r0.cost && !r0.reduce && !r0.lam && r0.src == SRC_GLOBAL_D ? 2 : 0;
      }
    }
    pa.err = (unsigned long long*)((char*)c->d_result.p + kErrWordOffset);
    {
      // limit of one tensor-load wait (QAOA_TMA_WAIT_NS; the tests shorten it)
      const char* w = getenv("QAOA_TMA_WAIT_NS");
      const unsigned long long wn = w ? strtoull(w, nullptr, 10) : 0ull;
      pa.tma_wait_ns = wn > 0 ? wn : kTmaWaitNs;
    }
    // the first pass visits every index once: the extremes come with it when
    // they are not known yet
    pa.ext_keys = nullptr;
    const RoundDev& r0 = pd.sub[0].rd[0];
    if (pp.init && !c->ext_ready && !c->ext_pending && (r0.cost || r0.reduce)) {
      CUDA_TRY(c, c->d_ext_keys.ensure(2 * sizeof(unsigned long long)));
      CUDA_TRY(c, cudaMemsetAsync(c->d_ext_keys.p, 0xff, 2 * sizeof(unsigned long long), c->stream));
      pa.ext_keys = (unsigned long long*)c->d_ext_keys.p;
    }
    int bps = 0;
    const int wide = fwd_shape_id(c, c->prec);
    const bool cc = ccs[pi];
    const bool red = pp.reduce && reduce;
    // a specialised kernel when one was compiled for this pass's rounds
    FwdPassKernel spec = nullptr;
    if (c->prec == QAOA_C64 && (wide == 3 || wide == 4) && fast && pd.nsub == 1 && pd.sub[0].ninner == 0 &&
        spec_enabled(c))
      spec = find_fwd_spec(pd.sub[0], sh.R, sh.WB);
    if (spec) {
      CUDA_TRY(c, cudaFuncSetAttribute((const void*)spec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, (const void*)spec, 32 << sh.WB, smem));
      if (bps < 1) return c->set_err(QAOA_ECUDA, "pass kernel does not fit on an SM (smem %zu)", smem);
    } else {
      rc = pass_any(c, fast, cc, wide, false, pd, pa, pt, smem, 0, &bps);
      if (rc) return rc;
    }
    const long long want = std::min<long long>((long long)bps * c->sms, kMaxGrid);
    const int grid = (int)std::min<long long>(want, (long long)pd.n_units);
    pa.partial = red ? (double*)c->d_partial.p : nullptr;
    // the final pass writes the sampling block sums when its tile is the 2^T
    // lowest index bits (T = 12..14, one sub-pass) and the state is large
    // enough for the separate block-sum read to matter (each thread's partial
    // over its register amplitudes is in the state precision, FP64 from there
    // on; block_sum_kernel sums every |psi|^2 in FP64, so shots whose
    // u * total lies within that rounding of a CDF step may differ in the
    // index between the two; both are valid draws)
    pa.bsum = nullptr;
    if (red && n >= kFuseSumsMinQubits && T >= 12 && T <= 14 && pp.subs.size() == 1) {
      bool contiguous = true;
      for (int j = 0; j < T; ++j) contiguous = contiguous && pp.subs[0].pos[j] == j;
      if (contiguous) {
        CUDA_TRY(c, c->d_sums.ensure(sizeof(double) * (size_t(1) << (n - 12))));
        pa.bsum = (double*)c->d_sums.p;
        fused_sums = true;
      }
    }
    {
      // algorithmic HBM bytes: one read (none for the |+> pass) and one write of
      // the state, plus one int32 diagonal read per sub-pass needing C(x)
      const double N = double(1ull << n);
      double bytes = (pp.init ? 0.0 : N * ab) + N * ab;
      if (stream)
        for (const SubPassPlan& sp : pp.subs) bytes += sp.needs_c ? 4.0 * N : 0.0;
      ProfScope ps(c, 0, bytes);
      if (spec) {
        spec<<<grid, 32 << sh.WB, smem, c->stream>>>(pd, pa, pt);
        if (c->prof_on) ++c->nlaunch;
        const cudaError_t le = cudaGetLastError();
        rc = le == cudaSuccess ? QAOA_OK : c->set_err(QAOA_ECUDA, "specialised pass kernel: %s", cudaGetErrorString(le));
      } else {
        rc = pass_any(c, fast, cc, wide, true, pd, pa, pt, smem, grid, nullptr);
      }
    }
    if (rc) return rc;
    if (pa.ext_keys) c->ext_pending = true;
    if (red) {
      sum_partials_kernel<<<1, 32, 0, c->stream>>>((const double*)c->d_partial.p, grid, 2, (double*)c->d_result.p);
      if (c->prof_on) ++c->nlaunch;
      CUDA_TRY(c, cudaGetLastError());
    }
  }
  c->have_result = reduce;
  c->state_ready = true;
  c->sums_ready = fused_sums;
  return QAOA_OK;
}

// ---------------------------------------------------------------- adjoint
const Plan* get_bplan(qaoa_ctx* c, int p, int order) {
  const auto key = std::make_pair(p, order);
  auto it = c->bplans.find(key);
  if (it != c->bplans.end()) return it->second.get();
  auto pl = std::make_unique<Plan>(plan_backward(c->n, p, adj_shape(c->prec), smax_adj(), kMinUnitsLog2, order));
  const Plan* r = pl.get();
  c->bplans[key] = std::move(pl);
  return r;
}

template <typename Real, bool FAST, bool CC, int R, int WB>
int adj_blocks_per_sm_rw(qaoa_ctx* c, size_t smem, int* nb) {
  auto kern = adj_pass_kernel<Real, R, WB, FAST, CC>;
  CUDA_TRY(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, kern, 32 << WB, smem));
  if (*nb < 1) return c->set_err(QAOA_ECUDA, "adjoint kernel does not fit on an SM (smem %zu)", smem);
  return QAOA_OK;
}

template <typename Real, bool FAST, bool CC, int R, int WB>
int launch_adj_rw(qaoa_ctx* c, const PassDev& pd, const AdjArgs& aa, const PassTma& pt, size_t smem, int grid) {
  auto kern = adj_pass_kernel<Real, R, WB, FAST, CC>;
  CUDA_TRY(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, 32 << WB, smem, c->stream>>>(pd, aa, pt);
  if (c->prof_on) ++c->nlaunch;
  CUDA_TRY(c, cudaGetLastError());
  return QAOA_OK;
}

template <typename Real, bool FAST, bool CC>
int adj_blocks_per_sm(qaoa_ctx* c, size_t smem, int* nb) {
  return adj_blocks_per_sm_rw<Real, FAST, CC, kRAdj, kWBAdj>(c, smem, nb);
}

template <typename Real, bool FAST, bool CC>
int launch_adj(qaoa_ctx* c, const PassDev& pd, const AdjArgs& aa, const PassTma& pt, size_t smem, int grid) {
  return launch_adj_rw<Real, FAST, CC, kRAdj, kWBAdj>(c, pd, aa, pt, smem, grid);
}

// Adjoint instantiation for (precision, mixer form, C(x) code): occupancy query
// when `launch` is false, else the launch. Plain inverse-mixer passes run the
// instantiation without the C(x) code.
template <typename Real>
int adj_any(qaoa_ctx* c, bool fast, bool cc, bool launch, const PassDev& pd, const AdjArgs& aa, const PassTma& pt,
            size_t smem, int grid, int* bps) {
  if (fast) {
    if (cc) return launch ? launch_adj<Real, true, true>(c, pd, aa, pt, smem, grid) : adj_blocks_per_sm<Real, true, true>(c, smem, bps);
    return launch ? launch_adj<Real, true, false>(c, pd, aa, pt, smem, grid) : adj_blocks_per_sm<Real, true, false>(c, smem, bps);
  }
  if (cc) return launch ? launch_adj<Real, false, true>(c, pd, aa, pt, smem, grid) : adj_blocks_per_sm<Real, false, true>(c, smem, bps);
  return launch ? launch_adj<Real, false, false>(c, pd, aa, pt, smem, grid) : adj_blocks_per_sm<Real, false, false>(c, smem, bps);
}

void* lambda_ptr(qaoa_ctx* c) {
  const size_t sb = qaoa_state_bytes(c->n, c->prec);
  const size_t need = qaoa_aux_bytes(c->n, c->prec, c->cost_mode, 1);
  if (c->aux && c->aux_bytes >= need) return c->aux;  // lambda is the first part of the aux buffer
  if (c->d_lambda.ensure(sb) != cudaSuccess) return nullptr;
  return c->d_lambda.p;
}

int run_gradient(qaoa_ctx* c, int p, const double* gamma, const double* beta, double* g_gamma, double* g_beta,
                 double* exp_c) {
  const int n = c->n;
  const int ab = amp_bytes(c->prec);
  const TileShape sh = adj_shape(c->prec);
  const int T = sh.T();
  std::vector<double> gg(p, 0.0), gbt(p, 0.0);
  if (n < T) {
    int rc = upload_phases(c, p, gamma);
    if (rc) return rc;
    CUDA_TRY(c, c->d_ang.ensure(sizeof(double) * 2 * p));
    std::vector<double> ang(2 * p);
    for (int k = 0; k < p; ++k) { ang[2 * k] = gamma[k]; ang[2 * k + 1] = beta[k]; }
    CUDA_TRY(c, cudaMemcpyAsync(c->d_ang.p, ang.data(), ang.size() * 8, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, c->d_gacc.ensure(sizeof(double) * (2 * p + 2)));
    SmallGradArgs ga;
    ga.base.n = n;
    ga.base.p = p;
    ga.base.state = c->state;
    ga.base.wmat = (const int32_t*)c->d_wmat.p;
    ga.base.phase = c->d_phase.p;
    ga.base.c_lo = (int)c->c_lo;
    ga.base.ncost = (int)(c->c_hi - c->c_lo + 1);
    ga.base.betas = (const double*)c->d_ang.p;
    ga.base.result = nullptr;
    ga.scale_s = c->scale;
    ga.wsum = (int)c->W;
    ga.grads = (double*)c->d_gacc.p;
    const size_t smem = (size_t(2) << n) * ab;
    {
      ProfScope ps(c, 4, 0.0);
      if (c->prec == QAOA_C128) {
        CUDA_TRY(c, cudaFuncSetAttribute(small_grad_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        small_grad_kernel<double><<<1, 512, smem, c->stream>>>(ga);
      } else {
        CUDA_TRY(c, cudaFuncSetAttribute(small_grad_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        small_grad_kernel<float><<<1, 512, smem, c->stream>>>(ga);
      }
      if (c->prof_on) ++c->nlaunch;
    }
    CUDA_TRY(c, cudaGetLastError());
    std::vector<double> h(2 * p + 2);
    CUDA_TRY(c, cudaMemcpyAsync(h.data(), c->d_gacc.p, h.size() * 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < p; ++k) { gg[k] = h[k]; gbt[k] = h[p + k]; }
    if (g_gamma) memcpy(g_gamma, gg.data(), sizeof(double) * p);
    if (g_beta) memcpy(g_beta, gbt.data(), sizeof(double) * p);
    if (exp_c) *exp_c = h[2 * p];
    c->state_ready = false;
    c->have_result = false;
    c->sums_ready = false;
    return QAOA_OK;
  }
  const Plan* plan;
  try {
    plan = get_bplan(c, p, grad_bwd_order(c));
  } catch (std::exception& ex) {
    return c->set_err(QAOA_EINVAL, "planner: %s", ex.what());
  }
  // the gradient's forward run samples nothing: the plan without the
  // block-sum constraint keeps the fused passes on the small groups
  int fwd_order = grad_fwd_order(c);
  // the gradient's complex64 forward runs the adjoint's tile (4x3), so that the
  // two plans can retrace each other pass by pass, unless a tile was asked for
  struct ShapeForce {
    qaoa_ctx* c;
    ~ShapeForce() { c->shape_force = -1; }
  } shape_guard{c};
  if (c->prec == QAOA_C64 && c->opts.fwd_shape == 0 && !getenv("QAOA_FWD_SHAPE")) c->shape_force = 3;
  // stored forward states: when the adjoint plan retraces the forward plan
  // pass by pass and half of the free device memory holds one state per
  // forward pass, the forward writes each pass's output to its own buffer and
  // adjoint pass j reads psi at its start from the output of forward pass
  // P-1-j instead of uncomputing it, which saves one state write per adjoint
  // pass (the in-tile uncompute of psi for the gradient terms stays)
  std::vector<void*> outs;
  if (grad_checkpoint(c) && n >= std::max(fwd_shape(c, c->prec).T(), kSmallMaxQubits + 1)) {
    try {
      const Plan* fp = get_plan(c, p, fwd_order);
      if (!plans_mirror(*fp, *plan) && fwd_order != grad_bwd_order(c)) {
        fwd_order = grad_bwd_order(c);
        fp = get_plan(c, p, fwd_order);
      }
      bool single = true;  // out-of-place passes have one sub-pass
      for (const PassPlan& pp : fp->passes) single = single && pp.subs.size() == 1;
      if (single && plans_mirror(*fp, *plan)) {
        const size_t sb = qaoa_state_bytes(n, c->prec);
        const size_t np = fp->passes.size();
        const size_t need = (np - 1) * sb;
        size_t fr = 0, tot = 0;
        bool ok = c->d_ckpt.p && c->d_ckpt.bytes >= need;
        if (!ok && cudaMemGetInfo(&fr, &tot) == cudaSuccess && need <= fr / 2) {
          ok = c->d_ckpt.ensure(need) == cudaSuccess;
          if (!ok) cudaGetLastError();  // out of memory: in-place forward, psi uncomputed
        }
        if (ok) {
          for (size_t k = 0; k + 1 < np; ++k) outs.push_back((char*)c->d_ckpt.p + k * sb);
          outs.push_back(c->state);
        }
      } else {
        fwd_order = grad_fwd_order(c);
      }
    } catch (std::exception& ex) {
      return c->set_err(QAOA_EINVAL, "planner: %s", ex.what());
    }
  }
  // two vectors: when the plans mirror each other, the forward's last pass
  // writes psi_p into the adjoint vector's buffer and leaves its input psi_{P-1}
  // in the state; the adjoint's first pass, which undoes exactly that pass,
  // reads psi_p there, creates lambda in place and need not write psi back
  // (one state write fewer; QAOA_GRAD_HYBRID=0 keeps the in-place forward)
  void* lam = lambda_ptr(c);
  if (!lam) return c->set_err(QAOA_ENOMEM, "allocation of the adjoint vector failed");
  bool hybrid = false;
  if (outs.empty() && n >= std::max(fwd_shape(c, c->prec).T(), kSmallMaxQubits + 1) &&
      on_off(0, "QAOA_GRAD_HYBRID", 1)) {
    try {
      const Plan* fp = get_plan(c, p, fwd_order);
      if (!plans_mirror(*fp, *plan) && fwd_order != grad_bwd_order(c)) {
        fwd_order = grad_bwd_order(c);
        fp = get_plan(c, p, fwd_order);
      }
      if (plans_mirror(*fp, *plan) && fp->passes.size() >= 2 && fp->passes.back().subs.size() == 1) {
        outs.assign(fp->passes.size(), c->state);
        outs.back() = lam;
        hybrid = true;
      } else {
        fwd_order = grad_fwd_order(c);
      }
    } catch (std::exception& ex) {
      return c->set_err(QAOA_EINVAL, "planner: %s", ex.what());
    }
  }
  // forward: psi_p (and the stored states)
  int rc = run_forward(c, p, gamma, beta, fwd_order, false, outs.empty() ? nullptr : outs.data());
  c->shape_force = -1;
  if (rc) return rc;
  const bool stream = c->cost_mode == QAOA_COST_STREAM;
  const long long nc = c->c_hi - c->c_lo + 1;
  const size_t tile_amps = ab == 8 ? padded_size<8>(T) : padded_size<16>(T);
  const size_t base_smem = ((2 * tile_amps * ab + kTconstSmemInts * 4 + 15) & ~size_t(15));
  const size_t with_tab = base_smem + size_t(nc) * ab;
  int dev = 0, max_smem = 0;
  CUDA_TRY(c, cudaGetDevice(&dev));
  CUDA_TRY(c, cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  // complex64 kernels compute the phase (phase_turns); complex128 reads the table
  const bool tab_smem = c->prec == QAOA_C128 && with_tab + 1024 <= (size_t)max_smem;
  const size_t smem = tab_smem ? with_tab : base_smem;
  const size_t npass = plan->passes.size();
  std::vector<PassDev> pds(npass);
  std::vector<char> fasts(npass);
  PassInputs in;
  in.n = n;
  in.beta = beta;
  in.gamma = gamma;
  in.scale = c->scale;
  in.c_lo = c->c_lo;
  in.ncost = nc;
  in.W = c->W;
  in.wmat = c->wmat.data();
  in.stream = stream;
  in.adjoint = true;
  for (size_t pi = 0; pi < npass; ++pi) {
    bool fast = true;
    const std::string why = fill_pass_dev(plan->passes[pi], sh, in, c->tabs, pds[pi], fast);
    if (!why.empty()) return c->set_err(QAOA_EINVAL, "%s", why.c_str());
    fasts[pi] = fast;
    for (int si = 0; si < pds[pi].nsub && !stream; ++si) {
      SubDev& sd = pds[pi].sub[si];
      if (!sd.needs_c) continue;
      rc = tile_const_table(c, pds[pi], sd);
      if (rc) return rc;
    }
    // complex64, one tile per super-tile: tiles are copied asynchronously,
    // the next one during the current one's last round
    if (c->prec == QAOA_C64 && pds[pi].nsub == 1 && pds[pi].sub[0].ninner == 0 && adj_prefetch())
      pds[pi].sub[0].cgtab = copy_geom_offset(c->tabs, sh, pds[pi].sub[0].pos);
  }
  rc = upload_ctabs(c);
  if (rc) return rc;
  CUDA_TRY(c, c->d_gacc.ensure(sizeof(double) * 4 * npass));
  for (size_t pi = 0; pi < npass; ++pi) {
    const PassPlan& pp = plan->passes[pi];
    const PassDev& pd = pds[pi];
    const bool fast = fasts[pi];
    AdjArgs aa;
    if (hybrid) {
      aa.psi = pi == 0 ? lam : c->state;
      aa.psi_store = pi == 0 ? 0 : 1;
    } else {
      aa.psi = outs.empty() ? c->state : outs[npass - 1 - pi];
      aa.psi_store = outs.empty() ? 1 : 0;
    }
    aa.lam = lam;
    aa.diag = stream ? (const int32_t*)((char*)c->aux + (c->aux_bytes - (size_t(4) << n))) : nullptr;
    aa.phase = pp.layer_c >= 0 && c->d_phase.p
                   ? (const void*)((const char*)c->d_phase.p + size_t(pp.layer_c) * nc * ab) : nullptr;
    aa.wmat = (const int32_t*)c->d_wmat.p;
    aa.ctabs = (const int32_t*)c->d_ctabs.p;
    aa.partial = (double*)c->d_partial.p;
    aa.phase_in_smem = tab_smem ? 1 : 0;
    // the next tile of both vectors into L2 by tensor prefetches (complex64,
    // one tile per super-tile, no shared-memory tile copies)
    PassTma pt;
    memset(&pt, 0, sizeof pt);
    aa.prefetch = 0;
    aa.tma_load = 0;
    {
      // tensor loads of each tile pair into shared memory (QAOA_ADJ_TMA_LOAD)
      const bool c64_single = c->prec == QAOA_C64 && pd.sub[0].cgtab < 0;
      const bool want_tma = c64_single && on_off(0, "QAOA_ADJ_TMA_LOAD", 1) && tma_load_form(pd);
      const bool want_pf = c64_single && adj_l2_prefetch(c);
      if ((want_tma || want_pf) && prefetch_tensor_map(n, pd, aa.psi, pt, &pt.tmap) &&
          prefetch_tensor_map(n, pd, aa.lam, pt, &pt.smap)) {
        if (want_pf) aa.prefetch = 2;
        if (want_tma) aa.tma_load = 1;
      }
    }
    aa.err = (unsigned long long*)((char*)c->d_result.p + kErrWordOffset);
    {
      const char* w = getenv("QAOA_TMA_WAIT_NS");
      const unsigned long long wn = w ? strtoull(w, nullptr, 10) : 0ull;
      aa.tma_wait_ns = wn > 0 ? wn : kTmaWaitNs;
    }
    int bps = 0;
    bool cc = false;
    for (const SubPassPlan& sp : pp.subs) cc = cc || sp.needs_c || sp.linit;
    // a specialised kernel when one was compiled for this pass's rounds
    AdjPassKernel spec = nullptr;
    if (c->prec == QAOA_C64 && fast && pd.nsub == 1 && pd.sub[0].ninner == 0 && spec_enabled(c))
      spec = find_adj_spec(pd.sub[0]);
    if (spec) {
      CUDA_TRY(c, cudaFuncSetAttribute((const void*)spec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, (const void*)spec, 32 << kWBAdj, smem));
      if (bps < 1) return c->set_err(QAOA_ECUDA, "adjoint kernel does not fit on an SM (smem %zu)", smem);
    } else {
      rc = c->prec == QAOA_C128 ? adj_any<double>(c, fast, cc, false, pd, aa, pt, smem, 0, &bps)
                                : adj_any<float>(c, fast, cc, false, pd, aa, pt, smem, 0, &bps);
      if (rc) return rc;
    }
    const long long want = std::min<long long>((long long)bps * c->sms, kMaxGrid);
    const int grid = (int)std::min<long long>(want, (long long)pd.n_units);
    {
      // algorithmic bytes: both vectors read (psi only when lambda is created)
      // and both written (lambda only with stored forward states; nothing in
      // the final pass)
      const double N = double(1ull << n);
      double bytes = (pp.linit ? 1.0 : 2.0) * N * ab + (pp.store ? (aa.psi_store ? 2.0 : 1.0) * N * ab : 0.0);
      if (stream)
        for (const SubPassPlan& sp : pp.subs) bytes += sp.needs_c ? 4.0 * N : 0.0;
      ProfScope ps(c, 1, bytes);
      if (spec) {
        spec<<<grid, 32 << kWBAdj, smem, c->stream>>>(pd, aa, pt);
        if (c->prof_on) ++c->nlaunch;
        const cudaError_t le = cudaGetLastError();
        rc = le == cudaSuccess ? QAOA_OK : c->set_err(QAOA_ECUDA, "specialised adjoint kernel: %s", cudaGetErrorString(le));
      } else {
        rc = c->prec == QAOA_C128 ? adj_any<double>(c, fast, cc, true, pd, aa, pt, smem, grid, nullptr)
                                  : adj_any<float>(c, fast, cc, true, pd, aa, pt, smem, grid, nullptr);
      }
    }
    if (rc) return rc;
    sum_partials_kernel<<<1, 32, 0, c->stream>>>((const double*)c->d_partial.p, grid, 4,
                                                 (double*)c->d_gacc.p + 4 * pi);
    if (c->prof_on) ++c->nlaunch;
    CUDA_TRY(c, cudaGetLastError());
  }
  std::vector<double> h(4 * npass);
  uint64_t errw = 0;
  CUDA_TRY(c, cudaMemcpyAsync(h.data(), c->d_gacc.p, h.size() * 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(&errw, (char*)c->d_result.p + kErrWordOffset, 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (errw) {
    CUDA_TRY(c, cudaMemsetAsync((char*)c->d_result.p + kErrWordOffset, 0, 8, c->stream));
    c->state_ready = false;
    c->sums_ready = false;
    return c->set_err(QAOA_ETIMEOUT, "a bounded wait for a tensor tile load gave up in a gradient pass");
  }
  for (size_t pi = 0; pi < npass; ++pi) {
    const PassPlan& pp = plan->passes[pi];
    if (pp.layer_a >= 0) gbt[pp.layer_a] += -2.0 * h[4 * pi];
    if (pp.layer_c >= 0) gg[pp.layer_c] += 2.0 * c->scale * h[4 * pi + 1];
    if (pp.layer_b >= 0) gbt[pp.layer_b] += -2.0 * h[4 * pi + 2];
  }
  if (g_gamma) memcpy(g_gamma, gg.data(), sizeof(double) * p);
  if (g_beta) memcpy(g_beta, gbt.data(), sizeof(double) * p);
  if (exp_c) *exp_c = h[3];  // <psi_p|C psi_p> from the first adjoint pass
  c->state_ready = false;  // psi walked back towards |+> (or psi_p, with stored forward states)
  c->sums_ready = false;
  return QAOA_OK;
}

// Exhaustive C_min / C_max with smallest argmin / argmax; optionally writes
// the full int32 diagonal. Without a diagonal only x with the top bit clear is
// scanned: C(x) = C(~x), so the smallest minimiser and maximiser lie there.
int compute_extremes(qaoa_ctx* c, int32_t* diag_out, bool restrict_half) {
  const int n = c->n;
  CUDA_TRY(c, c->d_ext.ensure(sizeof(Extreme)));
  ProfScope ps(c, 2, diag_out ? 4.0 * double(1ull << n) : 0.0);
  if (n < 16) {
    cost_small_kernel<<<1, 1024, 0, c->stream>>>(n, (const int32_t*)c->d_wmat.p, diag_out, (Extreme*)c->d_ext.p);
    if (c->prof_on) ++c->nlaunch;
    CUDA_TRY(c, cudaGetLastError());
    return QAOA_OK;
  }
  const int eff = restrict_half && !diag_out ? n - 1 : n;
  const long long blocks = 1ll << (eff - 15);
  CUDA_TRY(c, c->d_ext_part.ensure(sizeof(Extreme) * blocks));
  cost_block_kernel<15><<<(unsigned)blocks, 1024, 0, c->stream>>>(n, (const int32_t*)c->d_wmat.p, diag_out,
                                                                 (Extreme*)c->d_ext_part.p);
  if (c->prof_on) ++c->nlaunch;
  CUDA_TRY(c, cudaGetLastError());
  extreme_finalize_kernel<<<1, 1024, 0, c->stream>>>((const Extreme*)c->d_ext_part.p, blocks, (Extreme*)c->d_ext.p);
  if (c->prof_on) ++c->nlaunch;
  CUDA_TRY(c, cudaGetLastError());
  return QAOA_OK;
}

// C_min / C_max and their smallest indices on the host: from the keys of a
// run's first pass when it computed them, else from the exhaustive kernel.
int ensure_extremes(qaoa_ctx* c) {
  if (c->ext_ready) return QAOA_OK;
  if (c->ext_pending) {
    unsigned long long k[2];
    CUDA_TRY(c, cudaMemcpyAsync(k, c->d_ext_keys.p, sizeof k, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const unsigned long long mask = (1ull << 34) - 1;
    c->ext.vmin = c->c_lo + (long long)(k[0] >> 34);
    c->ext.amin = k[0] & mask;
    c->ext.vmax = c->c_hi - (long long)(k[1] >> 34);
    c->ext.amax = k[1] & mask;
  } else {
    int rc = compute_extremes(c, nullptr, true);
    if (rc) return rc;
    CUDA_TRY(c, cudaMemcpyAsync(&c->ext, c->d_ext.p, sizeof(Extreme), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  }
  c->ext_ready = true;
  c->ext_pending = false;
  return QAOA_OK;
}

}  // namespace

extern "C" {

size_t qaoa_state_bytes(int n, int precision) {
  if (precision != QAOA_C64 && precision != QAOA_C128) return 0;
  const int maxn = precision == QAOA_C64 ? QAOA_MAX_QUBITS_C64 : QAOA_MAX_QUBITS_C128;
  if (n < 1 || n > maxn) return 0;
  return (size_t(1) << n) * amp_bytes(precision);
}

int64_t qaoa_max_weight_sum(int n, int precision) {
  return precision == QAOA_C64 && n > kSmallMaxQubits ? kMaxAbsWeightSumTurns : kMaxAbsWeightSum;
}

int qaoa_quantize_weights(int m, const double* w, int64_t max_abs_sum, int32_t* w_int, double* unit) {
  if (m < 1 || !w || !w_int || !unit || max_abs_sum <= 2ll * m || max_abs_sum > INT32_MAX) return QAOA_EINVAL;
  double sum = 0.0;
  for (int e = 0; e < m; ++e) {
    if (!std::isfinite(w[e]) || w[e] == 0.0) return QAOA_EINVAL;
    sum += std::fabs(w[e]);
  }
  // rounding adds at most 1/2 per edge: sum |w_int| <= (max_abs_sum - m) + m / 2
  const double u = sum / double(max_abs_sum - m);
  for (int e = 0; e < m; ++e) {
    const long long q = std::llround(w[e] / u);
    if (q == 0) return QAOA_EINVAL;  // |w_e| below half a unit: the edge would vanish
    w_int[e] = (int32_t)q;
  }
  *unit = u;
  return QAOA_OK;
}

namespace {
// Cost modes recorded for QAOA_COST_AUTO per (n, precision) (qaoa_set_cost_choice).
std::mutex g_cost_mutex;
std::map<std::pair<int, int>, int> g_cost_choice;

int resolve_cost_mode(int n, int precision, int cost_mode) {
  if (cost_mode != QAOA_COST_AUTO) return cost_mode;
  std::lock_guard<std::mutex> lock(g_cost_mutex);
  auto it = g_cost_choice.find(std::make_pair(n, precision));
  return it != g_cost_choice.end() ? it->second : QAOA_COST_RECOMPUTE;
}
}  // namespace

int qaoa_set_cost_choice(int n, int precision, int cost_mode) {
  if (!qaoa_state_bytes(n, precision)) return QAOA_EINVAL;
  if (cost_mode < QAOA_COST_AUTO || cost_mode > QAOA_COST_STREAM) return QAOA_EINVAL;
  std::lock_guard<std::mutex> lock(g_cost_mutex);
  if (cost_mode == QAOA_COST_AUTO) g_cost_choice.erase(std::make_pair(n, precision));
  else g_cost_choice[std::make_pair(n, precision)] = cost_mode;
  return QAOA_OK;
}

size_t qaoa_aux_bytes(int n, int precision, int cost_mode, int with_grad) {
  const size_t sb = qaoa_state_bytes(n, precision);
  if (!sb) return 0;
  size_t b = with_grad ? sb : 0;
  if (resolve_cost_mode(n, precision, cost_mode) == QAOA_COST_STREAM) b += size_t(4) << n;
  return b;
}

int qaoa_set_opts(qaoa_ctx* c, const qaoa_opts* o) {
  if (!c) return QAOA_EINVAL;
  if (!o) return c->set_err(QAOA_EINVAL, "opts is NULL");
  auto onoff = [](int v) { return v == 0 || v == QAOA_ON || v == QAOA_OFF; };
  auto order = [](int v) { return v == 0 || v == QAOA_ORDER_LOW_LAST || v == QAOA_ORDER_LOW_MIDDLE; };
  if (o->fwd_shape != 0 && shape_from_opt(o->fwd_shape) < 0) return c->set_err(QAOA_EINVAL, "bad fwd_shape");
  if (c->prec == QAOA_C128 && o->fwd_shape != 0 && o->fwd_shape != QAOA_SHAPE_5x3 && o->fwd_shape != QAOA_SHAPE_4x3)
    return c->set_err(QAOA_EINVAL, "complex128 takes the 5x3 or 4x3 tile");
  if (o->super_tile != 0 && (o->super_tile < 12 || o->super_tile > 20))
    return c->set_err(QAOA_EINVAL, "super_tile outside 12..20");
  if (!order(o->group_order) || !order(o->grad_order)) return c->set_err(QAOA_EINVAL, "bad group order");
  if (!onoff(o->float_lanes) || !onoff(o->specialised) || !onoff(o->tile_tables) || !onoff(o->l2_prefetch) ||
      !onoff(o->grad_checkpoint) || !onoff(o->adj_l2_prefetch) || !onoff(o->tma_load))
    return c->set_err(QAOA_EINVAL, "on/off fields take 0, QAOA_ON or QAOA_OFF");
  cudaStreamSynchronize(c->stream);  // queued work may still read the old plans' tables
  c->opts = *o;
  c->plans.clear();
  c->bplans.clear();
  return QAOA_OK;
}

int qaoa_get_opts(const qaoa_ctx* c, qaoa_opts* o) {
  if (!c || !o) return QAOA_EINVAL;
  static const int kShapeOpt[5] = {QAOA_SHAPE_5x3, QAOA_SHAPE_4x4, QAOA_SHAPE_5x2, QAOA_SHAPE_4x3, QAOA_SHAPE_5x4};
  const int sid = fwd_shape_id(c, c->prec);
  qaoa_opts r{};
  r.fwd_shape = kShapeOpt[sid];
  r.super_tile = smax_fwd(c, shape_of(sid, c->prec).T());
  r.group_order = (group_order(c) & 3) == ORDER_LOW_MIDDLE ? QAOA_ORDER_LOW_MIDDLE : QAOA_ORDER_LOW_LAST;
  r.float_lanes = float_lanes_flag(c) ? QAOA_ON : QAOA_OFF;
  r.specialised = spec_enabled(c) ? QAOA_ON : QAOA_OFF;
  r.tile_tables = on_off(c->opts.tile_tables, "QAOA_TILE_TABLES", 1) ? QAOA_ON : QAOA_OFF;
  r.l2_prefetch = l2_prefetch_on(c, sid) ? QAOA_ON : QAOA_OFF;
  r.grad_order = grad_base_order(c) == ORDER_LOW_MIDDLE ? QAOA_ORDER_LOW_MIDDLE : QAOA_ORDER_LOW_LAST;
  r.grad_checkpoint = grad_checkpoint(c) ? QAOA_ON : QAOA_OFF;
  r.adj_l2_prefetch = adj_l2_prefetch(c) ? QAOA_ON : QAOA_OFF;
  r.tma_load = tma_load_on(c) ? QAOA_ON : QAOA_OFF;
  *o = r;
  return QAOA_OK;
}

int qaoa_init_graph(qaoa_ctx** out, int n, int m, const int32_t* u, const int32_t* v, const int32_t* w,
                    double weight_scale, int precision, int cost_mode, void* state_dev, size_t state_bytes,
                    void* aux_dev, size_t aux_bytes, void* cuda_stream) {
  g_init_error.clear();
  auto fail = [&](int code, const std::string& msg) {
    g_init_error = msg;
    if (out) *out = nullptr;
    return code;
  };
  if (!out) return fail(QAOA_EINVAL, "ctx output pointer is NULL");
  *out = nullptr;
  if (precision != QAOA_C64 && precision != QAOA_C128)
    return fail(QAOA_EINVAL, "precision must be QAOA_C64 or QAOA_C128");
  const size_t sb = qaoa_state_bytes(n, precision);
  if (!sb) return fail(QAOA_EINVAL, "n out of range for this precision");
  if (m < 0 || (m > 0 && (!u || !v || !w))) return fail(QAOA_EINVAL, "bad edge arrays");
  if (!(weight_scale > 0.0) || !std::isfinite(weight_scale)) return fail(QAOA_EINVAL, "weight_scale must be > 0");
  if (cost_mode < QAOA_COST_AUTO || cost_mode > QAOA_COST_STREAM) return fail(QAOA_EINVAL, "bad cost_mode");
  std::vector<int32_t> wmat;
  long long W = 0, pos = 0, neg = 0;
  {
    const std::string why = check_graph(n, m, u, v, w, qaoa_max_weight_sum(n, precision), wmat, W, neg, pos);
    if (!why.empty()) return fail(QAOA_EINVAL, why);
  }
  if (state_dev && state_bytes != sb)
    return fail(QAOA_ENOMEM, "state buffer size must equal qaoa_state_bytes(n, precision)");
  if (state_dev && (reinterpret_cast<uintptr_t>(state_dev) & 255))
    return fail(QAOA_EINVAL, "state buffer must be 256-byte aligned");
  const int mode = resolve_cost_mode(n, precision, cost_mode);
  if (aux_dev && aux_bytes < qaoa_aux_bytes(n, precision, mode, 0))
    return fail(QAOA_ENOMEM, "aux buffer smaller than qaoa_aux_bytes");
  if (aux_dev && (reinterpret_cast<uintptr_t>(aux_dev) & 255))
    return fail(QAOA_EINVAL, "aux buffer must be 256-byte aligned");

  std::unique_ptr<qaoa_ctx> c(new qaoa_ctx);
  c->n = n;
  c->m = m;
  c->prec = precision;
  c->cost_mode = mode;
  c->scale = weight_scale;
  c->u.assign(u, u + m);
  c->v.assign(v, v + m);
  c->w.assign(w, w + m);
  c->wmat = std::move(wmat);
  c->W = W;
  c->c_lo = neg;
  c->c_hi = pos;
  c->stream = (cudaStream_t)cuda_stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(QAOA_ECUDA, "no CUDA device");
  }
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
  if (state_dev) {
    c->state = state_dev;
  } else {
    if (cudaMalloc(&c->state, sb) != cudaSuccess) {
      cudaGetLastError();
      return fail(QAOA_ENOMEM, "cudaMalloc of the state failed");
    }
    c->own_state = true;
  }
  if (aux_dev) {
    c->aux = aux_dev;
    c->aux_bytes = aux_bytes;
  }
  if (c->d_wmat.ensure(sizeof(int32_t) * n * n) != cudaSuccess ||
      c->d_partial.ensure(sizeof(double) * 4 * kMaxGrid) != cudaSuccess || c->d_result.ensure(64) != cudaSuccess) {
    cudaGetLastError();
    qaoa_free(c.release());
    return fail(QAOA_ENOMEM, "cudaMalloc failed");
  }
  if (cudaMemsetAsync(c->d_result.p, 0, 64, c->stream) != cudaSuccess) {  // results and the error word
    qaoa_free(c.release());
    return fail(QAOA_ECUDA, "memset failed");
  }
  if (cudaMemcpyAsync(c->d_wmat.p, c->wmat.data(), sizeof(int32_t) * n * n, cudaMemcpyHostToDevice, c->stream) !=
      cudaSuccess) {
    qaoa_free(c.release());
    return fail(QAOA_ECUDA, "weight upload failed");
  }
  int32_t* diag = nullptr;
  if (mode == QAOA_COST_STREAM) {
    const size_t need = qaoa_aux_bytes(n, precision, mode, 0);
    if (!c->aux) {
      if (c->aux_own.ensure(need) != cudaSuccess) {
        cudaGetLastError();
        qaoa_free(c.release());
        return fail(QAOA_ENOMEM, "cudaMalloc of the cost diagonal failed");
      }
      c->aux = c->aux_own.p;
      c->aux_bytes = need;
    }
    diag = (int32_t*)((char*)c->aux + (c->aux_bytes - (size_t(4) << n)));
    // the diagonal is needed by every pass: it is written now, with the extremes
    int rc = compute_extremes(c.get(), diag, true);
    if (rc) {
      std::string msg = c->err;
      qaoa_free(c.release());
      return fail(rc, msg);
    }
    if (cudaMemcpyAsync(&c->ext, c->d_ext.p, sizeof(Extreme), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
      std::string msg = std::string("extremes transfer failed: ") + cudaGetErrorString(cudaGetLastError());
      qaoa_free(c.release());
      return fail(QAOA_ECUDA, msg);
    }
    c->ext_ready = true;
  }
  // recompute mode: the extremes come from the first run's |+> pass (every
  // index visited once), or from the exhaustive kernel when asked for first
  *out = c.release();
  return QAOA_OK;
}

int qaoa_run_angles(qaoa_ctx* c, int p, const double* gamma, const double* beta) {
  if (!c) return QAOA_EINVAL;
  if (p < 0 || (p > 0 && (!gamma || !beta))) return c->set_err(QAOA_EINVAL, "bad p or angle arrays");
  for (int k = 0; k < p; ++k)
    if (!std::isfinite(gamma[k]) || !std::isfinite(beta[k])) return c->set_err(QAOA_EINVAL, "non-finite angle");
  return run_forward(c, p, gamma, beta, group_order(c));
}

int qaoa_run(qaoa_ctx* c, int p, double dgamma, double dbeta) {
  if (!c) return QAOA_EINVAL;
  if (p < 0) return c->set_err(QAOA_EINVAL, "p must be >= 0");
  std::vector<double> g(p), b(p);
  for (int k = 0; k < p; ++k) {
    b[k] = (1.0 - double(k) / p) * dbeta;  // beta_k = (1 - k/p) dbeta
    g[k] = double(k + 1) / p * dgamma;      // gamma_k = (k+1)/p dgamma
  }
  return qaoa_run_angles(c, p, g.data(), b.data());
}

int qaoa_expect(qaoa_ctx* c, double* exp_c, double* r, double* norm, int64_t* c_min, int64_t* c_max,
                uint64_t* argmin, uint64_t* argmax) {
  if (!c) return QAOA_EINVAL;
  if (c_min || c_max || argmin || argmax || r) {
    const int rc = ensure_extremes(c);
    if (rc) return rc;
  }
  if (c_min) *c_min = c->ext.vmin;
  if (c_max) *c_max = c->ext.vmax;
  if (argmin) *argmin = c->ext.amin;
  if (argmax) *argmax = c->ext.amax;
  if (!exp_c && !r && !norm) return QAOA_OK;
  if (!c->have_result) return c->set_err(QAOA_ESTATE, "no run yet");
  // [norm, <C>, -, -, error word]
  double res[5];
  CUDA_TRY(c, cudaMemcpyAsync(res, c->d_result.p, sizeof res, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  uint64_t err;
  memcpy(&err, &res[kErrWordOffset / 8], 8);
  if (err) {
    CUDA_TRY(c, cudaMemsetAsync((char*)c->d_result.p + kErrWordOffset, 0, 8, c->stream));
    return c->set_err(QAOA_ETIMEOUT, "a bounded wait for a tensor tile load gave up in a forward pass");
  }
  if (norm) *norm = res[0];
  if (exp_c) *exp_c = res[1];
  if (r) {
    const double den = double(c->ext.vmax - c->ext.vmin);
    *r = den != 0.0 ? (res[1] - double(c->ext.vmin)) / den : 1.0;
  }
  return QAOA_OK;
}

int qaoa_sample(qaoa_ctx* c, int shots, const double* uniforms, uint64_t seed, uint64_t* out) {
  if (!c) return QAOA_EINVAL;
  if (shots < 0) return c->set_err(QAOA_EINVAL, "shots must be >= 0");
  if (shots > 0 && !out) return c->set_err(QAOA_EINVAL, "out is NULL");
  if (!c->state_ready) return c->set_err(QAOA_ESTATE, "no prepared state (call qaoa_run)");
  if (shots == 0) return QAOA_OK;
  if (uniforms)
    for (int i = 0; i < shots; ++i)
      if (!(uniforms[i] >= 0.0 && uniforms[i] < 1.0)) return c->set_err(QAOA_EINVAL, "uniforms must lie in [0, 1)");
  const int n = c->n;
  const int B = std::min(n, 12);
  const long long nb = 1ll << (n - B);
  CUDA_TRY(c, c->d_sums.ensure(sizeof(double) * nb));
  CUDA_TRY(c, c->d_pre.ensure(sizeof(double) * (nb + 1)));
  CUDA_TRY(c, c->d_shots.ensure(sizeof(unsigned long long) * shots));
  const double* d_uni = nullptr;
  if (uniforms) {
    CUDA_TRY(c, c->d_uni.ensure(sizeof(double) * shots));
    CUDA_TRY(c, cudaMemcpyAsync(c->d_uni.p, uniforms, sizeof(double) * shots, cudaMemcpyHostToDevice, c->stream));
    d_uni = (const double*)c->d_uni.p;
  }
  ProfScope ps(c, 3, c->sums_ready ? 0.0 : double(1ull << n) * amp_bytes(c->prec));
  if (!c->sums_ready) {  // else the final forward pass has written them
    if (c->prec == QAOA_C128)
      block_sum_kernel<double><<<(unsigned)nb, 256, 0, c->stream>>>((const double2*)c->state, B, (double*)c->d_sums.p);
    else
      block_sum_kernel<float><<<(unsigned)nb, 256, 0, c->stream>>>((const float2*)c->state, B, (double*)c->d_sums.p);
    if (c->prof_on) ++c->nlaunch;
    CUDA_TRY(c, cudaGetLastError());
  }
  if (nb <= kScanChunk) {
    scan_kernel<<<1, 1024, 0, c->stream>>>((const double*)c->d_sums.p, nb, (double*)c->d_pre.p);
    if (c->prof_on) ++c->nlaunch;
  } else {
    const long long nch = (nb + kScanChunk - 1) / kScanChunk;
    CUDA_TRY(c, c->d_pre2.ensure(sizeof(double) * (2 * nch + 1)));
    double* tot = (double*)c->d_pre2.p;
    double* pre2 = tot + nch;
    scan_chunk_kernel<<<(unsigned)nch, 512, 0, c->stream>>>((const double*)c->d_sums.p, nb, (double*)c->d_pre.p, tot);
    scan_kernel<<<1, 1024, 0, c->stream>>>(tot, nch, pre2);
    scan_offset_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, c->stream>>>((double*)c->d_pre.p, nb, pre2, nch);
    if (c->prof_on) c->nlaunch += 3;
  }
  CUDA_TRY(c, cudaGetLastError());
  const int wpb = 4, gb = (shots + wpb - 1) / wpb;
  if (c->prec == QAOA_C128)
    shot_warp_kernel<double><<<gb, 32 * wpb, 0, c->stream>>>((const double2*)c->state, B, (const double*)c->d_pre.p,
                                                              nb, shots, d_uni, seed, (unsigned long long*)c->d_shots.p);
  else
    shot_warp_kernel<float><<<gb, 32 * wpb, 0, c->stream>>>((const float2*)c->state, B, (const double*)c->d_pre.p,
                                                             nb, shots, d_uni, seed, (unsigned long long*)c->d_shots.p);
  if (c->prof_on) ++c->nlaunch;
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaMemcpyAsync(out, c->d_shots.p, sizeof(uint64_t) * shots, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return QAOA_OK;
}

int qaoa_sample_cuts(qaoa_ctx* c, int64_t count, const uint64_t* x_dev, uint64_t seed, uint64_t* x_out_dev,
                     int32_t* c_out_dev, double* r_out_dev) {
  if (!c) return QAOA_EINVAL;
  if (count < 0) return c->set_err(QAOA_EINVAL, "count must be >= 0");
  if (count == 0) return QAOA_OK;
  const int n = c->n;
  if (c->cut_planes < 0) {
    // weight bit planes of the upper triangle (j > i), by sign, non-empty only
    std::vector<unsigned long long> masks;
    std::vector<long long> coef;
    for (int sign = 1; sign >= -1; sign -= 2) {
      for (int t = 0; t < 31; ++t) {
        std::vector<unsigned long long> pl(n, 0ull);
        bool any = false;
        for (int i = 0; i < n; ++i)
          for (int j = i + 1; j < n; ++j) {
            const long long wij = c->wmat[size_t(i) * n + j];
            if (wij * sign > 0 && ((wij * sign) >> t & 1)) {
              pl[i] |= 1ull << j;
              any = true;
            }
          }
        if (!any) continue;
        masks.insert(masks.end(), pl.begin(), pl.end());
        coef.push_back(sign * (1ll << t));
      }
    }
    const int P = (int)coef.size();
    if (P > kMaxCutPlanes) return c->set_err(QAOA_EINVAL, "too many weight bit planes");
    std::vector<unsigned long long> tab(masks);
    for (long long cf : coef) tab.push_back((unsigned long long)cf);
    for (int i = 0; i < n; ++i) {
      long long d = 0;
      for (int j = 0; j < n; ++j) d += c->wmat[size_t(i) * n + j];
      tab.push_back((unsigned long long)d);
    }
    CUDA_TRY(c, c->d_cutplanes.ensure(tab.size() * 8));
    CUDA_TRY(c, cudaMemcpyAsync(c->d_cutplanes.p, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice, c->stream));
    c->cut_planes = P;
  }
  int rc = ensure_extremes(c);
  if (rc) return rc;
  CUDA_TRY(c, c->d_flag.ensure(sizeof(int)));
  CUDA_TRY(c, cudaMemsetAsync(c->d_flag.p, 0, sizeof(int), c->stream));
  SampleCutArgs a;
  a.n = n;
  a.planes = c->cut_planes;
  a.tab = (const unsigned long long*)c->d_cutplanes.p;
  a.count = count;
  a.x = (const unsigned long long*)x_dev;
  a.seed = seed;
  a.c_min = c->ext.vmin;
  a.c_max = c->ext.vmax;
  a.x_out = (unsigned long long*)x_out_dev;
  a.c_out = c_out_dev;
  a.r_out = r_out_dev;
  a.bad = (int*)c->d_flag.p;
  const size_t smem = size_t(a.planes * (n + 1) + n) * 8;
  const long long want = (long long)c->sms * 8;
  const int grid = (int)std::max<long long>(1, std::min<long long>(want, (count + 255) / 256));
  {
    const double per = (x_dev ? 8.0 : 0.0) + (x_out_dev ? 8.0 : 0.0) + (c_out_dev ? 4.0 : 0.0) + (r_out_dev ? 8.0 : 0.0);
    ProfScope ps(c, 3, per * double(count));
    sample_cut_kernel<<<grid, 256, smem, c->stream>>>(a);
    if (c->prof_on) ++c->nlaunch;
  }
  CUDA_TRY(c, cudaGetLastError());
  int bad = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&bad, c->d_flag.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (bad) return c->set_err(QAOA_EINVAL, "a bitstring has bits at or above n");
  return QAOA_OK;
}

int qaoa_noisy_expect(qaoa_ctx* c, int p, const double* gamma, const double* beta, double eps, int trajectories,
                      uint64_t seed, double* exp_c_dev, double* mean_exp_c, double* r_noisy) {
  if (!c) return QAOA_EINVAL;
  const int n = c->n, m = c->m;
  const int ab = amp_bytes(c->prec) / 2;  // bytes per real component
  if (n > kNoisyMaxQubits) return c->set_err(QAOA_EINVAL, "noisy trajectories need n <= %d", kNoisyMaxQubits);
  if (p < 0 || (p > 0 && (!gamma || !beta))) return c->set_err(QAOA_EINVAL, "p < 0 or missing angles");
  if (!(eps >= 0.0 && eps <= 1.0)) return c->set_err(QAOA_EINVAL, "eps must lie in [0, 1]");
  if (trajectories < 1) return c->set_err(QAOA_EINVAL, "trajectories must be >= 1");
  for (int k = 0; k < p; ++k)
    if (!std::isfinite(gamma[k]) || !std::isfinite(beta[k])) return c->set_err(QAOA_EINVAL, "angles must be finite");
  int rc = ensure_extremes(c);
  if (rc) return rc;
  // device block: u, v, w (int32, m each, padded to 8 bytes) | theta (p x m) | beta (p)
  const size_t ints = (3 * size_t(m) + 1) & ~size_t(1);
  std::vector<unsigned char> blk(ints * 4 + (size_t(p) * m + p) * 8 + 8);
  int32_t* hi = reinterpret_cast<int32_t*>(blk.data());
  for (int e = 0; e < m; ++e) { hi[e] = c->u[e]; hi[m + e] = c->v[e]; hi[2 * m + e] = c->w[e]; }
  double* hd = reinterpret_cast<double*>(blk.data() + ints * 4);
  for (int k = 0; k < p; ++k) {
    for (int e = 0; e < m; ++e) hd[size_t(k) * m + e] = gamma[k] * c->scale * double(c->w[e]);
    hd[size_t(p) * m + k] = beta[k];
  }
  CUDA_TRY(c, c->d_noisy.ensure(blk.size()));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_noisy.p, blk.data(), blk.size(), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, c->d_ntraj.ensure(sizeof(double) * (size_t(trajectories) + 1)));
  double* out = exp_c_dev ? exp_c_dev : (double*)c->d_ntraj.p;
  NoisyArgs a;
  a.n = n;
  a.m = m;
  a.p = p;
  a.trajectories = trajectories;
  a.u = (const int32_t*)c->d_noisy.p;
  a.v = a.u + m;
  a.w = a.u + 2 * m;
  a.theta = (const double*)((const unsigned char*)c->d_noisy.p + ints * 4);
  a.beta = a.theta + size_t(p) * m;
  a.eps = eps;
  a.seed = seed;
  a.exp_c = out;
  a.norm = nullptr;
  // complex64 contexts run the trajectories in FP32, complex128 in FP64
  const bool dbl = c->prec == QAOA_C128;
  const void* kern = dbl ? (const void*)noisy_trajectory_kernel<double> : (const void*)noisy_trajectory_kernel<float>;
  const size_t smem = (size_t(1) << n) * (size_t(2 * ab) + 4);
  CUDA_TRY(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int bps = 0;
  CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, kNoisyThreads, smem));
  const int grid = std::max(1, std::min(trajectories, std::max(1, bps) * c->sms));
  {
    ProfScope ps(c, 4, 0.0);
    if (dbl) noisy_trajectory_kernel<double><<<grid, kNoisyThreads, smem, c->stream>>>(a);
    else noisy_trajectory_kernel<float><<<grid, kNoisyThreads, smem, c->stream>>>(a);
    if (c->prof_on) ++c->nlaunch;
  }
  CUDA_TRY(c, cudaGetLastError());
  // mean over trajectories, summed in trajectory order
  double* sum_dev = (double*)c->d_ntraj.p + trajectories;
  sum_partials_kernel<<<1, 32, 0, c->stream>>>(out, trajectories, 1, sum_dev);
  if (c->prof_on) ++c->nlaunch;
  CUDA_TRY(c, cudaGetLastError());
  double sum = 0.0;
  CUDA_TRY(c, cudaMemcpyAsync(&sum, sum_dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const double mean = sum / trajectories;
  if (mean_exp_c) *mean_exp_c = mean;
  if (r_noisy) {
    const double span = double(c->ext.vmax - c->ext.vmin);
    *r_noisy = span != 0.0 ? (mean - double(c->ext.vmin)) / span : 1.0;
  }
  return QAOA_OK;
}

int qaoa_cost_diag(qaoa_ctx* c, int32_t* out_dev) {
  if (!c) return QAOA_EINVAL;
  if (!out_dev) return c->set_err(QAOA_EINVAL, "out_dev is NULL");
  if (reinterpret_cast<uintptr_t>(out_dev) & 15) return c->set_err(QAOA_EINVAL, "out_dev must be 16-byte aligned");
  return compute_extremes(c, out_dev, false);
}

void* qaoa_state_ptr(qaoa_ctx* c) { return c ? c->state : nullptr; }

int qaoa_describe_plan(int n, int precision, int p, int adjoint, char* out, int cap) {
  std::string s;
  try {
    const TileShape fsh = shape_of(fwd_shape_id(nullptr, precision, n), precision);
    Plan pl = adjoint ? plan_backward(n, p, adj_shape(precision), smax_adj(), kMinUnitsLog2, group_order(nullptr))
                      : plan_forward(n, p, fsh, smax_fwd(nullptr, fsh.T()), kMinUnitsLog2, group_order(nullptr));
    std::string e = validate(pl);
    s = pl.describe();
    if (!e.empty()) s += "INVALID: " + e + "\n";
  } catch (std::exception& ex) {
    s = std::string("error: ") + ex.what() + "\n";
  }
  if (out && cap > 0) {
    const int k = std::min<int>(cap - 1, (int)s.size());
    memcpy(out, s.data(), k);
    out[k] = 0;
  }
  return (int)s.size();
}

int qaoa_profile_enable(qaoa_ctx* c, int enable) {
  if (!c) return QAOA_EINVAL;
  if (enable) {
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    for (auto& r : c->prof_pending) { c->ev_pool.push_back(r.a); c->ev_pool.push_back(r.b); }
    c->prof_pending.clear();
    for (int k = 0; k < 5; ++k) { c->prof_ms[k] = 0; c->prof_bytes[k] = 0; c->prof_n[k] = 0; }
    c->nlaunch = 0;
  }
  c->prof_on = enable != 0;
  return QAOA_OK;
}

int qaoa_profile_read(qaoa_ctx* c, int kind, int64_t* launches, double* ms, double* bytes) {
  if (!c) return QAOA_EINVAL;
  if (kind < 0 || kind > 5) return c->set_err(QAOA_EINVAL, "profile kind must be 0..5");
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  for (auto& r : c->prof_pending) {
    float t = 0.f;
    CUDA_TRY(c, cudaEventElapsedTime(&t, r.a, r.b));
    c->prof_ms[r.kind] += t;
    c->prof_bytes[r.kind] += r.bytes;
    c->prof_n[r.kind] += 1;
    c->ev_pool.push_back(r.a);
    c->ev_pool.push_back(r.b);
  }
  c->prof_pending.clear();
  if (kind == 5) {
    if (launches) *launches = c->nlaunch;
    if (ms) *ms = 0.0;
    if (bytes) *bytes = 0.0;
    return QAOA_OK;
  }
  if (launches) *launches = c->prof_n[kind];
  if (ms) *ms = c->prof_ms[kind];
  if (bytes) *bytes = c->prof_bytes[kind];
  return QAOA_OK;
}

const char* qaoa_last_error(const qaoa_ctx* c) {
  if (!c) return g_init_error.c_str();
  return c->err.c_str();
}

void qaoa_free(qaoa_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  if (c->own_state && c->state) cudaFree(c->state);
  c->aux_own.release();
  DevBuf* bufs[] = {&c->d_wmat, &c->d_ctabs, &c->d_phase, &c->d_partial, &c->d_result, &c->d_ext,
                    &c->d_ext_part, &c->d_ext_keys, &c->d_sums, &c->d_pre, &c->d_pre2, &c->d_shots, &c->d_uni, &c->d_ang,
                    &c->d_lambda, &c->d_gacc, &c->d_ckpt, &c->d_cutplanes, &c->d_flag, &c->d_noisy, &c->d_ntraj};
  for (DevBuf* b : bufs) b->release();
  for (auto& kv : c->tct_tabs) kv.second.release();
  for (auto& r : c->prof_pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  delete c;
}

int qaoa_grad_angles(qaoa_ctx* c, int p, const double* gamma, const double* beta, double* g_gamma, double* g_beta,
                     double* exp_c) {
  if (!c) return QAOA_EINVAL;
  if (p < 1 || !gamma || !beta) return c->set_err(QAOA_EINVAL, "the gradient needs p >= 1 and angle arrays");
  for (int k = 0; k < p; ++k)
    if (!std::isfinite(gamma[k]) || !std::isfinite(beta[k])) return c->set_err(QAOA_EINVAL, "non-finite angle");
  return run_gradient(c, p, gamma, beta, g_gamma, g_beta, exp_c);
}

int qaoa_grad(qaoa_ctx* c, int p, double dgamma, double dbeta, double* g_gamma, double* g_beta, double* d_dgamma,
              double* d_dbeta, double* exp_c) {
  if (!c) return QAOA_EINVAL;
  if (p < 1) return c->set_err(QAOA_EINVAL, "the gradient needs p >= 1");
  std::vector<double> g(p), b(p), gg(p), gb(p);
  for (int k = 0; k < p; ++k) {
    b[k] = (1.0 - double(k) / p) * dbeta;
    g[k] = double(k + 1) / p * dgamma;
  }
  const int rc = qaoa_grad_angles(c, p, g.data(), b.data(), gg.data(), gb.data(), exp_c);
  if (rc) return rc;
  // chain rule through gamma_k = (k+1)/p dgamma and beta_k = (1 - k/p) dbeta
  double sg = 0.0, sb = 0.0;
  for (int k = 0; k < p; ++k) {
    sg += double(k + 1) / p * gg[k];
    sb += (1.0 - double(k) / p) * gb[k];
  }
  if (g_gamma) memcpy(g_gamma, gg.data(), sizeof(double) * p);
  if (g_beta) memcpy(g_beta, gb.data(), sizeof(double) * p);
  if (d_dgamma) *d_dgamma = sg;
  if (d_dbeta) *d_dbeta = sb;
  return QAOA_OK;
}

}  // extern "C"
