// batch.cu -- batched LR-QAOA instances (qaoa_batch_* in include/qaoa.h).
//
// Host side: validates and plans every instance, builds the work-item queue of
// the persistent kernel (batch_kernel.cuh), uploads all tables, and captures
// one run into a CUDA graph that qaoa_batch_run replays.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <numeric>
#include <stdexcept>
#include <string>
#include <vector>

#include "batch_kernel.cuh"
#include "desc.h"
#include "plan.h"
#include "qaoa.h"

using namespace qaoa;

namespace {

thread_local std::string g_batch_create_error;

constexpr long long kBatchMaxAbsWeight = 1 << 20;
constexpr int kBatchMaxP = 64;
constexpr unsigned long long kWaitNs = 2000000000ull;  // default limit of a dependency wait: 2 s

struct InstPlan {
  int n = 0, p = 0, mode = 0;
  long long W = 0, c_lo = 0, c_hi = 0;
  double dgamma = 0, dbeta = 0;
  std::vector<int32_t> wmat;
  std::vector<double> gamma, beta;
  TableStore tabs;
  std::vector<PassDev> fwd, adj;
  std::vector<PassPlan> fwd_pp, adj_pp;
  std::vector<char> fwd_fast, adj_fast;
  double work = 0;  // tiles x passes (scheduling weight)
};

}  // namespace

struct qaoa_batch {
  int count = 0, with_grad = 0;
  double scale = 0.1;
  cudaStream_t user_stream = nullptr, cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<void*> allocs;
  std::vector<size_t> state_off;  // byte offsets of the states
  std::vector<int> n, p;
  void* states = nullptr;
  BatchArgs args{}, args_adj{};
  double* d_out = nullptr;
  bool fast = true;
  bool stream = false;  // streamed int32 cost diagonals instead of the cost tables
  int fwd_r = kBatchR;  // register bits of the forward tile
  int nitems = 0, nitems_adj = 0, grid = 0, grid_adj = 0, ctas_per_sm = 0, nmode[3] = {0, 0, 0};
  size_t smem = 0, dev_bytes = 0, gtotal = 0;
  double bytes = 0;
  bool ran = false;
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
  ~qaoa_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (void* a : allocs) cudaFree(a);
  }
  void* dalloc(size_t bytes_) {
    void* p_ = nullptr;
    if (cudaMalloc(&p_, std::max<size_t>(bytes_, 256)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    allocs.push_back(p_);
    dev_bytes += bytes_;
    return p_;
  }
};

namespace {

template <typename T>
T* upload(qaoa_batch* b, const std::vector<T>& h) {
  T* d = (T*)b->dalloc(sizeof(T) * std::max<size_t>(1, h.size()));
  if (!d) return nullptr;
  if (!h.empty() && cudaMemcpy(d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return d;
}

int env_int(const char* name, int def) {
  const char* e = getenv(name);
  return e ? atoi(e) : def;
}

}  // namespace

extern "C" {

int qaoa_batch_create(qaoa_batch** out, int count, const int32_t* n, const int32_t* p, const int64_t* edge_off,
                      const int32_t* u, const int32_t* v, const int32_t* w, const double* dgamma, const double* dbeta,
                      double weight_scale, int with_grad, const qaoa_batch_opts* opts, void* cuda_stream) {
  g_batch_create_error.clear();
  auto fail = [&](int code, const std::string& msg) {
    g_batch_create_error = msg;
    if (out) *out = nullptr;
    return code;
  };
  if (!out) return fail(QAOA_EINVAL, "output pointer is NULL");
  *out = nullptr;
  if (count < 1 || !n || !p || !edge_off || !dgamma || !dbeta) return fail(QAOA_EINVAL, "bad instance arrays");
  if (!(weight_scale > 0.0) || !std::isfinite(weight_scale)) return fail(QAOA_EINVAL, "weight_scale must be > 0");
  qaoa_batch_opts o{};
  if (opts) o = *opts;
  const int solo_max_n = std::max(13, o.solo_max_n > 0 ? o.solo_max_n : env_int("QAOA_BATCH_SOLO", 16));
  const int max_units = std::max(1, o.max_units > 0 ? o.max_units : env_int("QAOA_BATCH_UNITS", 8));
  const int window_mb = std::max(1, o.window_mb > 0 ? o.window_mb : env_int("QAOA_BATCH_WINDOW_MB", 96));
  if (o.cost_mode < QAOA_COST_AUTO || o.cost_mode > QAOA_COST_STREAM) return fail(QAOA_EINVAL, "bad cost_mode");
  if (o.fwd_shape != 0 && o.fwd_shape != QAOA_SHAPE_5x3 && o.fwd_shape != QAOA_SHAPE_4x3)
    return fail(QAOA_EINVAL, "the batch's forward tile is QAOA_SHAPE_5x3 or QAOA_SHAPE_4x3");
  // streamed cost: C(x) of every instance precomputed once (int32 per amplitude)
  const bool stream = o.cost_mode == QAOA_COST_STREAM;
  const int fwd_r = o.fwd_shape == QAOA_SHAPE_4x3 ? 4 : kBatchR;

  std::unique_ptr<qaoa_batch> b(new qaoa_batch);
  b->count = count;
  b->with_grad = with_grad ? 1 : 0;
  b->scale = weight_scale;
  b->user_stream = (cudaStream_t)cuda_stream;

  // ------------------------------------------------------------ plan instances
  TileShape fsh;
  fsh.R = fwd_r;
  fsh.WB = kBatchWB;
  fsh.amp_bytes = 8;
  TileShape ash;
  ash.R = kBatchRAdj;
  ash.WB = kBatchWBAdj;
  ash.amp_bytes = 8;
  ash.nvec = 2;
  const int Tf = fsh.T(), Ta = ash.T();
  // one mixer form for the whole batch: the fast tan form unless some
  // beta_k has |tan beta_k| > 1
  bool all_fast = true;
  for (int i = 0; i < count; ++i) {
    if (p[i] < 1 || p[i] > kBatchMaxP || !std::isfinite(dbeta[i])) continue;
    for (int k = 0; k < p[i]; ++k) {
      const double bk = (1.0 - double(k) / p[i]) * dbeta[i];
      all_fast = all_fast && fabs(cos(bk)) >= fabs(sin(bk));
    }
  }
  b->fast = all_fast;
  b->stream = stream;
  b->fwd_r = fwd_r;
  std::vector<InstPlan> ip(count);
  for (int i = 0; i < count; ++i) {
    InstPlan& I = ip[i];
    I.n = n[i];
    I.p = p[i];
    if (I.n < 2 || I.n > kBatchMaxN) return fail(QAOA_EINVAL, "instance " + std::to_string(i) + ": n out of [2, 24]");
    if (I.p < 1 || I.p > kBatchMaxP) return fail(QAOA_EINVAL, "instance " + std::to_string(i) + ": p out of [1, 64]");
    if (!std::isfinite(dgamma[i]) || !std::isfinite(dbeta[i]))
      return fail(QAOA_EINVAL, "instance " + std::to_string(i) + ": angles must be finite");
    const long long e0 = edge_off[i], e1 = edge_off[i + 1];
    if (e0 < 0 || e1 < e0 || e1 - e0 > (long long)I.n * (I.n - 1) / 2)
      return fail(QAOA_EINVAL, "instance " + std::to_string(i) + ": bad edge offsets");
    if (e1 > e0 && (!u || !v || !w)) return fail(QAOA_EINVAL, "edge arrays are NULL");
    const std::string why = check_graph(I.n, int(e1 - e0), u ? u + e0 : nullptr, v ? v + e0 : nullptr,
                                        w ? w + e0 : nullptr, kBatchMaxAbsWeight, I.wmat, I.W, I.c_lo, I.c_hi);
    if (!why.empty()) return fail(QAOA_EINVAL, "instance " + std::to_string(i) + ": " + why);
    I.dgamma = dgamma[i];
    I.dbeta = dbeta[i];
    I.gamma.resize(I.p);
    I.beta.resize(I.p);
    for (int k = 0; k < I.p; ++k) {
      I.gamma[k] = double(k + 1) / I.p * I.dgamma;
      I.beta[k] = (1.0 - double(k) / I.p) * I.dbeta;
    }
    const bool small = with_grad ? I.n <= kBatchSmallGradMax : I.n <= kBatchSmallMax;
    I.mode = small ? BMODE_SMALL : (I.n < solo_max_n ? BMODE_SOLO : BMODE_MULTI);
    b->nmode[I.mode]++;
    PassInputs in;
    in.n = I.n;
    in.beta = I.beta.data();
    in.gamma = I.gamma.data();
    in.scale = weight_scale;
    in.c_lo = I.c_lo;
    in.ncost = I.c_hi - I.c_lo + 1;
    in.W = I.W;
    in.wmat = I.wmat.data();
    in.stream = stream;
    in.plain = !all_fast;
    try {
      if (!small && I.n >= Tf) {
        Plan pl = plan_forward(I.n, I.p, fsh, Tf, 0);
        I.fwd_pp = pl.passes;
        in.adjoint = false;
        for (const PassPlan& pp : pl.passes) {
          PassDev pd;
          bool fast = true;
          const std::string e = fill_pass_dev(pp, fsh, in, I.tabs, pd, fast);
          if (!e.empty()) return fail(QAOA_EINVAL, e);
          I.fwd.push_back(pd);
          I.fwd_fast.push_back(fast);
        }
      }
      if (!small && with_grad && I.n >= Ta) {
        Plan pl = plan_backward(I.n, I.p, ash, Ta, 0);
        I.adj_pp = pl.passes;
        in.adjoint = true;
        for (const PassPlan& pp : pl.passes) {
          PassDev pd;
          bool fast = true;
          const std::string e = fill_pass_dev(pp, ash, in, I.tabs, pd, fast);
          if (!e.empty()) return fail(QAOA_EINVAL, e);
          I.adj.push_back(pd);
          I.adj_fast.push_back(fast);
        }
      }
    } catch (std::exception& ex) {
      return fail(QAOA_EINVAL, std::string("planner: ") + ex.what());
    }
    for (const PassDev& pd : I.fwd) I.work += double(pd.n_units);
    for (const PassDev& pd : I.adj) I.work += 2.0 * double(pd.n_units);
    if (small) I.work = double(I.p) * I.n * (1 << I.n) / 8192.0;
  }

  // ------------------------------------------------------------ device layout
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(QAOA_ECUDA, "no CUDA device");
  }
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

  size_t state_total = 0;
  b->state_off.resize(count);
  b->n.resize(count);
  b->p.resize(count);
  for (int i = 0; i < count; ++i) {
    b->n[i] = ip[i].n;
    b->p[i] = ip[i].p;
    b->state_off[i] = state_total;
    state_total += ((size_t(8) << ip[i].n) + 255) & ~size_t(255);
  }
  b->states = b->dalloc(state_total);
  void* lams = with_grad ? b->dalloc(state_total) : nullptr;
  if (!b->states || (with_grad && !lams)) return fail(QAOA_ENOMEM, "cudaMalloc of the batch states failed");
  // streamed cost: one int32 diagonal per instance that runs HBM passes
  std::vector<size_t> diag_off(count, ~size_t(0));
  int32_t* diags = nullptr;
  if (stream) {
    size_t total = 0;
    for (int i = 0; i < count; ++i)
      if (!ip[i].fwd.empty() || !ip[i].adj.empty()) {
        diag_off[i] = total;
        total += ((size_t(4) << ip[i].n) + 255) & ~size_t(255);
      }
    diags = (int32_t*)b->dalloc(std::max<size_t>(total, 256));
    if (!diags) return fail(QAOA_ENOMEM, "cudaMalloc of the batch cost diagonals failed");
  }

  // per-instance tables: weights, cost tables, phase tables, angles
  std::vector<int32_t> h_w, h_ct;
  std::vector<float2> h_ph;
  std::vector<double> h_ang;
  std::vector<size_t> w_off(count), ct_off(count), ph_off(count), ang_off(count);
  for (int i = 0; i < count; ++i) {
    InstPlan& I = ip[i];
    w_off[i] = h_w.size();
    h_w.insert(h_w.end(), I.wmat.begin(), I.wmat.end());
    if (h_ct.size() & 1) h_ct.push_back(0);  // the geometry tables hold 64-bit words
    ct_off[i] = h_ct.size();
    h_ct.insert(h_ct.end(), I.tabs.h.begin(), I.tabs.h.end());
    ph_off[i] = h_ph.size();
    const long long nc = I.c_hi - I.c_lo + 1;
    for (int k = 0; k < I.p; ++k)
      for (long long c = 0; c < nc; ++c) {
        // exp(-i gamma_k s (W - 2 C)), FP64 then rounded (Eqs. H_C, UC)
        const double th = -I.gamma[k] * weight_scale * double(I.W - 2 * (I.c_lo + c));
        h_ph.push_back(make_float2(float(cos(th)), float(sin(th))));
      }
    ang_off[i] = h_ang.size();
    for (int k = 0; k < I.p; ++k) {
      h_ang.push_back(I.gamma[k]);
      h_ang.push_back(I.beta[k]);
    }
  }
  int32_t* d_w = upload(b.get(), h_w);
  int32_t* d_ct = upload(b.get(), h_ct);
  float2* d_ph = upload(b.get(), h_ph);
  double* d_ang = upload(b.get(), h_ang);
  if (!d_w || !d_ct || !d_ph || !d_ang) return fail(QAOA_ENOMEM, "upload of the batch tables failed");

  // ------------------------------------------------------------ passes, slots, items
  std::vector<BatchInst> h_inst(count);
  std::vector<PassDev> h_pass;
  std::vector<PassMeta> h_meta;
  int32_t nslots = 0, g_total = 0;
  std::vector<int> units_per_item;  // per global pass
  for (int i = 0; i < count; ++i) {
    InstPlan& I = ip[i];
    BatchInst& D = h_inst[i];
    memset(&D, 0, sizeof D);
    D.n = I.n;
    D.p = I.p;
    D.c_lo = (int32_t)I.c_lo;
    D.ncost = (int32_t)(I.c_hi - I.c_lo + 1);
    D.wsum = (int32_t)I.W;
    D.mode = I.mode;
    D.with_grad = with_grad ? 1 : 0;
    D.psi = (char*)b->states + b->state_off[i];
    D.lam = lams ? (char*)lams + b->state_off[i] : nullptr;
    D.wmat = d_w + w_off[i];
    D.ctabs = d_ct + ct_off[i];
    D.diag = diag_off[i] != ~size_t(0) ? (const int32_t*)((char*)diags + diag_off[i]) : nullptr;
    D.phase = d_ph + ph_off[i];
    D.ang = d_ang + ang_off[i];
    D.scale = weight_scale;
    D.g_off = g_total;
    g_total += 2 * I.p;
    D.slot0 = nslots;
    if (I.fwd.empty()) nslots += 2;  // [norm, <C>] of the shared-memory forward circuit
    auto add_passes = [&](const std::vector<PassDev>& pds, const std::vector<PassPlan>& pps,
                          const std::vector<char>& fasts, bool adjoint) {
      for (size_t j = 0; j < pds.size(); ++j) {
        const PassPlan& pp = pps[j];
        PassMeta M;
        memset(&M, 0, sizeof M);
        M.inst = i;
        M.layer_a = pp.layer_a;
        M.layer_c = pp.layer_c;
        M.layer_b = pp.layer_b;
        M.fast = fasts[j];
        M.reduce = pp.reduce;
        M.adjoint = adjoint;
        const long long units = (long long)pds[j].n_units;
        int upi = 1;
        if (I.mode == BMODE_MULTI) {
          upi = (int)std::max<long long>(1, std::min<long long>(max_units, units / 64));
          M.nitems = (int)((units + upi - 1) / upi);
        } else {
          upi = (int)units;
          M.nitems = 1;
        }
        M.slot0 = nslots;
        nslots += M.nitems * (adjoint ? 3 : (pp.reduce ? 2 : 0));
        h_pass.push_back(pds[j]);
        h_meta.push_back(M);
        units_per_item.push_back(upi);
        b->bytes += double(size_t(8) << I.n) * (adjoint ? ((pp.linit ? 1.0 : 2.0) + (pp.store ? 2.0 : 0.0))
                                                         : ((pp.init ? 1.0 : 2.0)));
        if (stream)  // the int32 diagonal read by each sub-pass that needs C(x)
          for (const SubPassPlan& sp : pp.subs) b->bytes += sp.needs_c ? double(size_t(4) << I.n) : 0.0;
      }
    };
    D.fwd_pass0 = (int32_t)h_pass.size();
    D.fwd_npass = (int32_t)I.fwd.size();
    add_passes(I.fwd, I.fwd_pp, I.fwd_fast, false);
    D.adj_pass0 = (int32_t)h_pass.size();
    D.adj_npass = (int32_t)I.adj.size();
    add_passes(I.adj, I.adj_pp, I.adj_fast, true);
    D.nslots = nslots - D.slot0;
    if (I.fwd.empty()) b->bytes += double(size_t(8) << I.n) * (with_grad ? 0.0 : 1.0);
  }
  b->gtotal = g_total;

  // items: interleaved passes of the MULTI instances (largest first, a window
  // of instances in flight), then SOLO and SMALL instances (largest first),
  // then the exhaustive-extremes blocks
  std::vector<BatchItem> items;
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return ip[a].work > ip[c].work; });
  auto item = [&](int inst, int kind, int pass, int slot, uint32_t u0, uint32_t u1, int need) {
    BatchItem it;
    it.inst = inst;
    it.kind = kind;
    it.pass = pass;
    it.slot = slot;
    it.u0 = u0;
    it.u1 = u1;
    it.need = need;
    it.pad = 0;
    items.push_back(it);
  };
  // occupancy of the persistent kernel
  b->smem = std::max<size_t>({size_t(padded_size<8>(Tf)) * 8, size_t(2 * padded_size<8>(Ta)) * 8,
                              (size_t(8) << kBatchSmallMax) + (size_t(4) << kBatchSmallMax),
                              (size_t(16) << kBatchSmallGradMax) + (size_t(4) << kBatchSmallGradMax)}) +
            32 * 4 + kBatchMaxN * kBatchMaxN * 4;
  auto fwd_kern = fwd_r == 4 ? (all_fast ? batch_kernel<true, false, 4> : batch_kernel<false, false, 4>)
                             : (all_fast ? batch_kernel<true, false, kBatchR> : batch_kernel<false, false, kBatchR>);
  auto adj_kern = all_fast ? batch_kernel<true, true, kBatchR> : batch_kernel<false, true, kBatchR>;
  int bps = 0;
  for (auto kern : {fwd_kern, adj_kern}) {
    int nb = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kBatchThreads, b->smem) != cudaSuccess || nb < 1) {
      cudaGetLastError();
      return fail(QAOA_ECUDA, "batch kernel does not fit on an SM");
    }
    bps = bps ? std::min(bps, nb) : nb;
  }
  const int want_cps = o.ctas_per_sm > 0 ? o.ctas_per_sm : env_int("QAOA_BATCH_CTAS", 0);
  b->ctas_per_sm = want_cps > 0 ? std::min(want_cps, bps) : std::min(bps, 2);
  const int ctas = b->ctas_per_sm * sms;
  const int window_items = o.window_items > 0 ? o.window_items : env_int("QAOA_BATCH_WINDOW_ITEMS", 2 * ctas);
  std::vector<BatchItem> items_adj;
  auto emit_window = [&](bool adjoint, std::vector<BatchItem>& q) {
    struct Act {
      int inst;
      int next;  // next pass of this phase
      int emitted;
    };
    std::vector<Act> act;
    size_t oi = 0;
    auto np_of = [&](int i) { return adjoint ? h_inst[i].adj_npass : h_inst[i].fwd_npass; };
    auto pass_at = [&](int i, int j) { return (adjoint ? h_inst[i].adj_pass0 : h_inst[i].fwd_pass0) + j; };
    auto next_multi = [&]() {
      while (oi < order.size() && (ip[order[oi]].mode != BMODE_MULTI || np_of(order[oi]) == 0)) ++oi;
      return oi < order.size() ? order[oi] : -1;
    };
    for (;;) {
      for (;;) {  // refill the window
        long long items_next = 0;
        double mb = 0;
        for (const Act& a : act) {
          items_next += h_meta[pass_at(a.inst, a.next)].nitems;
          mb += double(size_t(8) << ip[a.inst].n) * (with_grad ? 2 : 1) / 1048576.0;
        }
        if (act.size() >= 2 && (items_next >= window_items || mb >= window_mb)) break;
        const int c = next_multi();
        if (c < 0) break;
        ++oi;
        act.push_back({c, 0, 0});
      }
      if (act.empty()) break;
      for (Act& a : act) {
        const int pi = pass_at(a.inst, a.next);
        const PassMeta& M = h_meta[pi];
        const int upi = units_per_item[pi];
        const uint32_t units = (uint32_t)h_pass[pi].n_units;
        for (int k = 0; k < M.nitems; ++k) {
          const uint32_t u0 = (uint32_t)k * upi, u1 = std::min<uint32_t>(units, u0 + upi);
          const int slot = M.adjoint ? M.slot0 + 3 * k : (M.reduce ? M.slot0 + 2 * k : -1);
          BatchItem it;
          it.inst = a.inst;
          it.kind = BITEM_PASS;
          it.pass = pi;
          it.slot = slot;
          it.u0 = u0;
          it.u1 = u1;
          it.need = a.emitted;
          it.pad = 0;
          q.push_back(it);
        }
        a.emitted += M.nitems;
        ++a.next;
      }
      act.erase(std::remove_if(act.begin(), act.end(), [&](const Act& a) { return a.next >= np_of(a.inst); }),
                act.end());
    }
  };
  emit_window(false, items);
  emit_window(true, items_adj);
  for (int i : order)
    if (ip[i].mode == BMODE_SOLO) {
      item(i, BITEM_SOLO, -1, -1, 0, 0, 0);
      if (h_inst[i].adj_npass > 0) {
        BatchItem it = items.back();
        items_adj.push_back(it);
      }
    }
  for (int i : order)
    if (ip[i].mode == BMODE_SMALL) item(i, BITEM_SMALL, -1, -1, 0, 0, 0);
  for (int i : order) {
    // SMALL instances and the shared-memory forward of SOLO n = 12 find their
    // extremes themselves
    if (ip[i].mode == BMODE_SMALL || ip[i].fwd.empty()) continue;
    const uint32_t nb = (uint32_t)std::max<long long>(1, (1ll << (ip[i].n - 1)) >> kBatchExtBits);
    const uint32_t per = 8;
    for (uint32_t b0 = 0; b0 < nb; b0 += per) item(i, BITEM_EXT, -1, -1, b0, std::min(nb, b0 + per), 0);
  }
  b->nitems = (int)items.size();
  b->nitems_adj = (int)items_adj.size();
  // every wait is on earlier items of the same instance and phase
  for (const std::vector<BatchItem>* q : {&items, &items_adj}) {
    std::vector<int> seen(count, 0);
    for (const BatchItem& it : *q) {
      if (it.kind == BITEM_PASS) {
        if (it.need > seen[it.inst]) return fail(QAOA_EINVAL, "internal: item order violates a dependency");
        seen[it.inst]++;
      }
    }
  }

  BatchItem* d_items = upload(b.get(), items);
  BatchItem* d_items_adj = upload(b.get(), items_adj);
  BatchInst* d_inst = upload(b.get(), h_inst);
  PassDev* d_pass = upload(b.get(), h_pass);
  PassMeta* d_meta = upload(b.get(), h_meta);
  unsigned int* d_head = (unsigned int*)b->dalloc(256);  // [0] forward, [32] adjoint
  int32_t* d_done = (int32_t*)b->dalloc(sizeof(int32_t) * 2 * count);
  double* d_slots = (double*)b->dalloc(sizeof(double) * std::max(1, nslots));
  unsigned long long* d_emin = (unsigned long long*)b->dalloc(8ull * count);
  unsigned long long* d_emax = (unsigned long long*)b->dalloc(8ull * count);
  double* d_grads = (double*)b->dalloc(sizeof(double) * std::max(1, g_total));
  int32_t* d_err = (int32_t*)b->dalloc(256);
  b->d_out = (double*)b->dalloc(sizeof(double) * 9 * count);
  if (!d_items || !d_items_adj || !d_inst || !d_pass || !d_meta || !d_head || !d_done || !d_slots || !d_emin || !d_emax ||
      !d_grads || !d_err || !b->d_out)
    return fail(QAOA_ENOMEM, "cudaMalloc of the batch metadata failed");
  BatchArgs& A = b->args;
  A.items = d_items;
  A.nitems = b->nitems;
  A.insts = d_inst;
  A.passes = d_pass;
  A.pmeta = d_meta;
  A.head = d_head;
  A.done = d_done;
  A.slots = d_slots;
  A.ext_min = d_emin;
  A.ext_max = d_emax;
  A.grads = d_grads;
  A.error = d_err;
  A.wait_ns = o.wait_ns > 0 ? (unsigned long long)o.wait_ns : kWaitNs;
  b->grid = std::max(1, std::min(ctas, b->nitems));
  b->args_adj = A;
  b->args_adj.items = d_items_adj;
  b->args_adj.nitems = b->nitems_adj;
  b->args_adj.head = d_head + 32;
  b->args_adj.done = d_done + count;
  b->grid_adj = std::max(1, std::min(ctas, b->nitems_adj));

  // ------------------------------------------------------------ cost diagonals
  // (streamed cost) C(x) of each instance with HBM passes, once per batch: the
  // diagonal depends on the graph only, every run reads it
  if (stream) {
    Extreme* d_scratch = (Extreme*)b->dalloc(sizeof(Extreme) * (size_t(1) << (kBatchMaxN - 15)));
    if (!d_scratch) return fail(QAOA_ENOMEM, "cudaMalloc of the diagonal scratch failed");
    for (int i = 0; i < count; ++i) {
      if (diag_off[i] == ~size_t(0)) continue;
      int32_t* dg = (int32_t*)((char*)diags + diag_off[i]);
      const int32_t* wm = d_w + w_off[i];
      if (ip[i].n < 16) {
        cost_small_kernel<<<1, 1024>>>(ip[i].n, wm, dg, d_scratch);
      } else {
        cost_block_kernel<15><<<(unsigned)(1u << (ip[i].n - 15)), 1024>>>(ip[i].n, wm, dg, d_scratch);
      }
    }
    const cudaError_t de = cudaGetLastError();
    if (de != cudaSuccess) return fail(QAOA_ECUDA, std::string("cost diagonals: ") + cudaGetErrorString(de));
  }

  // ------------------------------------------------------------ graph
  if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return fail(QAOA_ECUDA, "cudaStreamCreate failed");
  }
  cudaStream_t s = b->cap_stream;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return fail(QAOA_ECUDA, "cudaStreamBeginCapture failed");
  }
  cudaMemsetAsync(d_head, 0, 256, s);
  cudaMemsetAsync(d_err, 0, 4, s);
  cudaMemsetAsync(d_done, 0, sizeof(int32_t) * 2 * count, s);
  cudaMemsetAsync(d_emin, 0xff, 8ull * count, s);
  cudaMemsetAsync(d_emax, 0, 8ull * count, s);
  fwd_kern<<<b->grid, kBatchThreads, b->smem, s>>>(A);
  if (b->nitems_adj > 0) adj_kern<<<b->grid_adj, kBatchThreads, b->smem, s>>>(b->args_adj);
  batch_finalize_kernel<<<(count + 127) / 128, 128, 0, s>>>(A, count, b->d_out);
  cudaError_t ce = cudaStreamEndCapture(s, &b->graph);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    return fail(QAOA_ECUDA, std::string("graph capture failed: ") + cudaGetErrorString(ce));
  }
  ce = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    return fail(QAOA_ECUDA, std::string("cudaGraphInstantiate failed: ") + cudaGetErrorString(ce));
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return fail(QAOA_ECUDA, "upload failed");
  }
  *out = b.release();
  return QAOA_OK;
}

int qaoa_batch_run(qaoa_batch* b) {
  if (!b) return QAOA_EINVAL;
  const cudaError_t e = cudaGraphLaunch(b->exec, b->user_stream);
  if (e != cudaSuccess) return b->set_err(QAOA_ECUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
  b->ran = true;
  return QAOA_OK;
}

int qaoa_batch_results(qaoa_batch* b, double* out, double* grads) {
  if (!b) return QAOA_EINVAL;
  if (!b->ran) return b->set_err(QAOA_ESTATE, "no run yet");
  int32_t errflag = 0;
  cudaError_t e = cudaMemcpyAsync(&errflag, b->args.error, 4, cudaMemcpyDeviceToHost, b->user_stream);
  if (e == cudaSuccess && out)
    e = cudaMemcpyAsync(out, b->d_out, sizeof(double) * 9 * b->count, cudaMemcpyDeviceToHost, b->user_stream);
  if (e == cudaSuccess && grads && b->with_grad)
    e = cudaMemcpyAsync(grads, b->args.grads, sizeof(double) * b->gtotal, cudaMemcpyDeviceToHost, b->user_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->user_stream);
  if (e != cudaSuccess) return b->set_err(QAOA_ECUDA, "result copy: %s", cudaGetErrorString(e));
  if (grads && !b->with_grad) memset(grads, 0, sizeof(double) * b->gtotal);
  if (errflag) return b->set_err(QAOA_ETIMEOUT, "a dependency wait of the batch kernel gave up");
  return QAOA_OK;
}

int qaoa_batch_state(qaoa_batch* b, int i, void** state_dev) {
  if (!b || !state_dev || i < 0 || i >= b->count) return b ? b->set_err(QAOA_EINVAL, "bad instance index") : QAOA_EINVAL;
  if (b->with_grad) return b->set_err(QAOA_ESTATE, "a gradient batch does not keep its final states");
  if (!b->ran) return b->set_err(QAOA_ESTATE, "no run yet");
  *state_dev = (char*)b->states + b->state_off[i];
  return QAOA_OK;
}

int qaoa_batch_describe(const qaoa_batch* b, char* out, size_t cap) {
  if (!b || !out || cap == 0) return QAOA_EINVAL;
  snprintf(out, cap,
           "instances=%d small=%d solo=%d multi=%d items=%d adjoint_items=%d grid=%d ctas_per_sm=%d smem=%zu "
           "device_bytes=%zu state_bytes=%.0f grad=%d fast=%d tile=%dx%d cost=%s",
           b->count, b->nmode[0], b->nmode[1], b->nmode[2], b->nitems, b->nitems_adj, b->grid, b->ctas_per_sm,
           b->smem, b->dev_bytes, b->bytes, b->with_grad, b->fast ? 1 : 0, b->fwd_r, kBatchWB,
           b->stream ? "stream" : "recompute");
  return QAOA_OK;
}

double qaoa_batch_bytes(const qaoa_batch* b) { return b ? b->bytes : 0.0; }

const char* qaoa_batch_last_error(const qaoa_batch* b) {
  return b ? b->err.c_str() : g_batch_create_error.c_str();
}

void qaoa_batch_free(qaoa_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->user_stream);
  delete b;
}

}  // extern "C"
