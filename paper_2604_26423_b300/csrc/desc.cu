// desc.cu -- pass descriptors and per-round cost tables (see desc.h).
#include "desc.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <set>

namespace qaoa {

namespace {

// Cost tables of one round (recompute mode), for tile bits at global
// positions pos[] and the round's register / lane / warp split:
//   CQ[q]     = sum_{k<l in Q} w [q_k != q_l]          (q: lane bits, then warp bits)
//   AJ[q][i]  = sum_{k in Q, q_k = 1} w[reg_i][k]
//   D[i]      = sum_{k in Q} w[reg_i][k]
//   CP[j]     = sum_{i<i'} w[reg_i][reg_i'] [j_i != j_i']
std::vector<int32_t> build_round_tables(const int32_t* wmat, int n, const TileShape& sh, const int8_t* pos,
                                        const RoundDev& rd) {
  const int R = sh.R, WB = sh.WB, QB = 5 + WB;
  const int QN = 1 << QB;
  auto W = [&](int tj, int tk) { return wmat[pos[tj] * n + pos[tk]]; };
  int qbits[16];
  for (int i = 0; i < 5; ++i) qbits[i] = rd.lane[i];
  for (int i = 0; i < WB; ++i) qbits[5 + i] = rd.warp[i];
  std::vector<int32_t> t(QN + QN * R + R + (1 << R));
  for (int q = 0; q < QN; ++q) {
    int cq = 0;
    for (int k = 0; k < QB; ++k)
      for (int l = k + 1; l < QB; ++l)
        if ((q >> k & 1) != (q >> l & 1)) cq += W(qbits[k], qbits[l]);
    t[q] = cq;
    for (int i = 0; i < R; ++i) {
      int a = 0;
      for (int k = 0; k < QB; ++k)
        if (q >> k & 1) a += W(rd.reg[i], qbits[k]);
      t[QN + q * R + i] = a;
    }
  }
  for (int i = 0; i < R; ++i) {
    int d = 0;
    for (int k = 0; k < QB; ++k) d += W(rd.reg[i], qbits[k]);
    t[QN + QN * R + i] = d;
  }
  for (int j = 0; j < (1 << R); ++j) {
    int cp = 0;
    for (int i = 0; i < R; ++i)
      for (int i2 = i + 1; i2 < R; ++i2)
        if ((j >> i & 1) != (j >> i2 & 1)) cp += W(rd.reg[i], rd.reg[i2]);
    t[QN + QN * R + R + j] = cp;
  }
  return t;
}

// Global index bits of a round's register / lane / warp tile bits.
void fill_round_globals(RoundDev& rd, const int8_t* pos) {
  for (int i = 0; i < 5; ++i) rd.greg[i] = pos[rd.reg[i]];
  for (int i = 0; i < 5; ++i) rd.glane[i] = pos[rd.lane[i]];
  for (int i = 0; i < 4; ++i) rd.gwarp[i] = pos[rd.warp[i]];
}

void to_round_dev(const RoundPlan& rp, RoundDev& rd) {
  memcpy(rd.reg, rp.reg, 5);
  memcpy(rd.lane, rp.lane, 5);
  memcpy(rd.warp, rp.warp, 4);
  rd.mixA = rp.mixA;
  rd.cost = rp.cost;
  rd.mixB = rp.mixB;
  rd.reduce = rp.reduce;
  rd.src = rp.src;
  rd.dst = rp.dst;
  rd.lam = rp.lam;
  rd.layout = rp.layout;
  rd.ctab = -1;
}

}  // namespace

int32_t TableStore::offset(const int32_t* wmat, int n, const TileShape& sh, const int8_t* pos, const RoundDev& rd) {
  std::vector<int8_t> key(pos, pos + sh.T());
  key.insert(key.end(), rd.reg, rd.reg + 5);
  key.insert(key.end(), rd.lane, rd.lane + 5);
  key.insert(key.end(), rd.warp, rd.warp + 4);
  auto k = std::make_pair(sh.R * 100 + sh.WB, key);
  auto it = index.find(k);
  if (it != index.end()) return it->second;
  std::vector<int32_t> t = build_round_tables(wmat, n, sh, pos, rd);
  const int32_t off = (int32_t)h.size();
  h.insert(h.end(), t.begin(), t.end());
  index[k] = off;
  dirty = true;
  return off;
}

std::string check_graph(int n, int m, const int32_t* u, const int32_t* v, const int32_t* w, long long max_abs,
                        std::vector<int32_t>& wmat, long long& W, long long& c_lo, long long& c_hi) {
  if (m < 0 || (m > 0 && (!u || !v || !w))) return "bad edge arrays";
  std::set<std::pair<int, int>> seen;
  W = 0;
  c_lo = 0;
  c_hi = 0;
  for (int e = 0; e < m; ++e) {
    if (u[e] < 0 || u[e] >= n || v[e] < 0 || v[e] >= n) return "edge vertex out of range";
    if (u[e] == v[e]) return "self loop";
    if (w[e] == 0) return "zero weight";
    auto key = std::make_pair(std::min(u[e], v[e]), std::max(u[e], v[e]));
    if (!seen.insert(key).second) return "repeated edge";
    W += w[e];
    if (w[e] > 0) c_hi += w[e]; else c_lo += w[e];
    if (c_hi - c_lo > max_abs) return "sum of |w| exceeds the limit " + std::to_string(max_abs);
  }
  wmat.assign((size_t)n * n, 0);
  for (int e = 0; e < m; ++e) {
    wmat[u[e] * n + v[e]] = w[e];
    wmat[v[e] * n + u[e]] = w[e];
  }
  return "";
}

int32_t TableStore::geom_offset(const TileShape& sh, const int8_t* pos, const RoundDev& rd) {
  std::vector<int8_t> key(pos, pos + sh.T());
  key.insert(key.end(), rd.lane, rd.lane + 5);
  key.insert(key.end(), rd.warp, rd.warp + 4);
  key.push_back(int8_t(sh.amp_bytes));
  auto k = std::make_pair(1000 + sh.R * 100 + sh.WB, key);
  auto it = index.find(k);
  if (it != index.end()) return it->second;
  const int NT = 32 << sh.WB;
  if (h.size() & 1) h.push_back(0);  // 8-byte alignment of the offsets part
  const int32_t off = (int32_t)h.size();
  h.resize(h.size() + 3 * NT, 0);
  for (int tid = 0; tid < NT; ++tid) {
    const int lane = tid & 31, warp = tid >> 5;
    uint32_t tb = 0;
    uint64_t g = 0;
    for (int i = 0; i < 5; ++i)
      if (lane >> i & 1) { tb |= 1u << rd.lane[i]; g |= 1ull << pos[rd.lane[i]]; }
    for (int i = 0; i < sh.WB; ++i)
      if (warp >> i & 1) { tb |= 1u << rd.warp[i]; g |= 1ull << pos[rd.warp[i]]; }
    const uint32_t sb = sh.amp_bytes == 8 ? padi<8>(tb) : padi<16>(tb);
    // bit 31: parity of the thread's global index offset (swapped storage)
    h[off + tid] = (int32_t)(sb | (uint32_t(__builtin_popcountll(g) & 1) << 31));
    h[off + NT + 2 * tid] = (int32_t)(uint32_t)(g & 0xffffffffull);
    h[off + NT + 2 * tid + 1] = (int32_t)(uint32_t)(g >> 32);
  }
  index[k] = off;
  dirty = true;
  return off;
}

int32_t copy_geom_offset(TableStore& tabs, const TileShape& sh, const int8_t* pos) {
  RoundDev rd;
  memset(&rd, 0, sizeof rd);
  for (int i = 0; i < 5; ++i) rd.lane[i] = int8_t(i);
  for (int i = 0; i < sh.WB; ++i) rd.warp[i] = int8_t(5 + i);
  return tabs.geom_offset(sh, pos, rd);
}

BitRuns make_runs(const std::vector<int>& bits) {
  BitRuns r;
  memset(&r, 0, sizeof r);
  int k = 0;
  for (size_t i = 0; i < bits.size();) {
    size_t j = i;
    while (j + 1 < bits.size() && bits[j + 1] == bits[j] + 1) ++j;
    r.src[k] = int8_t(i);
    r.dst[k] = int8_t(bits[i]);
    r.len[k] = int8_t(j - i + 1);
    ++k;
    i = j + 1;
  }
  r.n = int8_t(k);
  return r;
}

void mixer_coeffs(double beta, bool fast, double* tau, double* alpha) {
  if (fast) { *tau = tan(beta); *alpha = 1.0; }
  else { *tau = sin(beta); *alpha = cos(beta); }
}

namespace {

// frac(x) as a 64-bit fixed-point fraction (x in turns)
uint64_t turns_fixed(long double x) {
  x -= floorl(x);
  const long double f = x * 18446744073709551616.0L;
  return f >= 18446744073709551615.0L ? ~0ull : (uint64_t)f;
}

}  // namespace

std::string fill_pass_dev(const PassPlan& pp, const TileShape& sh, const PassInputs& in, TableStore& tabs,
                          PassDev& pd, bool& fast) {
  const int T = sh.T();
  memset(&pd, 0, sizeof pd);
  pd.n = in.n;
  pd.T = T;
  pd.nsub = (int)pp.subs.size();
  if (pd.nsub > kMaxSubDev) return "plan has too many sub-passes";
  pd.nouter = (int)pp.outer.size();
  for (int i = 0; i < pd.nouter; ++i) pd.outer[i] = (int8_t)pp.outer[i];
  pd.outer_runs = make_runs(pp.outer);
  pd.n_units = 1ull << pd.nouter;
  const double ba = pp.layer_a >= 0 ? in.beta[pp.layer_a] : 0.0;
  const double bb = pp.layer_b >= 0 ? in.beta[pp.layer_b] : 0.0;
  fast = !in.plain && fabs(cos(ba)) >= fabs(sin(ba)) && fabs(cos(bb)) >= fabs(sin(bb));
  mixer_coeffs(ba, fast, &pd.tauA, &pd.alphaA);
  mixer_coeffs(bb, fast, &pd.tauB, &pd.alphaB);
  pd.amp0 = in.adjoint ? 0.0 : pow(2.0, -0.5 * in.n);
  pd.c_lo = (int32_t)in.c_lo;
  pd.ncost = (int32_t)in.ncost;
  pd.wsum = (int32_t)in.W;
  pd.cA = cos(ba);
  pd.cB = cos(bb);
  pd.ftauA = float(pd.tauA);
  pd.falphaA = float(pd.alphaA);
  pd.ftauB = float(pd.tauB);
  pd.falphaB = float(pd.alphaB);
  pd.fcA = float(pd.cA);
  pd.fcB = float(pd.cB);
  if (pp.layer_c >= 0 && in.gamma) {
    // turns of exp(-i gamma s (W - 2c)) at c = c_lo + u: t0 + u d with
    // t0 = -gamma s (W - 2 c_lo) / (2 pi), d = gamma s / pi
    const long double pi = 3.141592653589793238462643383279502884L;
    const long double g = (long double)in.gamma[pp.layer_c] * (long double)in.scale;
    pd.ph0 = turns_fixed(-g * (long double)(in.W - 2 * in.c_lo) / (2 * pi));
    pd.ph1 = turns_fixed(g / pi);
  }
  pd.famp0 = float(pd.amp0);
  int cost_rounds = 0, c_rounds = 0;
  for (int s = 0; s < pd.nsub; ++s) {
    const SubPassPlan& sp = pp.subs[s];
    SubDev& sd = pd.sub[s];
    for (int j = 0; j < T; ++j) sd.pos[j] = sp.pos[j];
    std::vector<int> inner;
    for (int b : pp.sb) {
      bool in_tile = false;
      for (int j = 0; j < T; ++j) in_tile |= sp.pos[j] == b;
      if (!in_tile) inner.push_back(b);
    }
    sd.ninner = (int)inner.size();
    for (int i = 0; i < sd.ninner; ++i) sd.inner[i] = (int8_t)inner[i];
    sd.inner_runs = make_runs(inner);
    sd.cgtab = -1;
    // complex64 storage: a forward run ends in plain (re, im) amplitudes; the
    // adjoint starts from them (swapped storage in between, pass_kernel.cuh)
    sd.st_plain = !in.adjoint && pp.reduce && s + 1 == pd.nsub;
    sd.ld_plain = in.adjoint && pp.linit && s == 0;
    sd.nrounds = (int)sp.rounds.size();
    if (sd.nrounds > kMaxRoundsDev) return "plan has too many rounds";
    sd.needs_c = sp.needs_c;
    sd.store = sp.store;
    if (in.adjoint) {
      sd.scale = 1.0;
    } else {
      sd.init = sp.init;
      sd.keep = s + 1 < pd.nsub;
      sd.scale = fast ? pow(cos(ba), sp.nA) * pow(cos(bb), sp.nB) : 1.0;
    }
    sd.fscale = float(sd.scale);
    sd.rescale = sd.scale != 1.0;
    for (int r = 0; r < sd.nrounds; ++r) {
      RoundDev& rd = sd.rd[r];
      to_round_dev(sp.rounds[r], rd);
      fill_round_globals(rd, sd.pos);
      rd.gtab = tabs.geom_offset(sh, sd.pos, rd);
      const bool wants = in.adjoint ? (rd.cost || rd.lam) : (rd.cost || rd.reduce);
      if (wants && !in.stream) rd.ctab = tabs.offset(in.wmat, in.n, sh, sd.pos, rd);
      if (in.stream || rd.ctab < 0) continue;
      // the kernels take the register-pair part CP[j] of the pass's cost
      // round (cpc, cpt) and of its reduction round (forward) or
      // lambda-creation round (adjoint) (cpr) from the descriptor
      const int QN = 1 << (5 + sh.WB);
      const int32_t* cp = tabs.h.data() + rd.ctab + QN + QN * sh.R + sh.R;
      if (rd.cost) {
        if (cost_rounds++) return "plan has two cost rounds in one pass";
        for (int j = 0; j < (1 << sh.R); ++j) {
          pd.cpc[j] = cp[j];
          pd.cpt[j] = uint32_t(((uint64_t)(int64_t)cp[j] * pd.ph1) >> 32);
        }
      }
      if (in.adjoint ? rd.lam : rd.reduce) {
        if (c_rounds++) return "plan has two reduction rounds in one pass";
        for (int j = 0; j < (1 << sh.R); ++j) pd.cpr[j] = cp[j];
      }
    }
  }
  return "";
}

}  // namespace qaoa
