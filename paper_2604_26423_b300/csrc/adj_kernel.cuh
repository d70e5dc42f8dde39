// adj_kernel.cuh -- adjoint (reverse-mode) pass kernel for d<C>/d(gamma_k, beta_k).
//
// After the forward pass leaves psi_p = U_{p-1} ... U_0 |+>, the adjoint walks
// the layers backwards with two vectors, psi and lambda = U_{>k}^dag C psi_p,
// uncomputing both with the inverse gates (Sec. II-B: U_B(beta) = exp(+i beta
// H_B), U_C(gamma) = exp(-i gamma s H_C)), and accumulates
//   dbeta_k:  2 Re <lambda| i H_B |psi> = -2 sum_q Im <lambda| X_q |psi>
//   dgamma_k: 2 Re <lambda| -i s H_C |psi> = 2 s Im sum_x conj(lambda_x) psi_x h(x)
// with h(x) = W - 2 C(x). X_q commutes with every factor exp(+i beta X_q') of
// the mixer, so <lambda| X_q |psi> may be taken at any point of the mixer's
// uncomputation; a round evaluates the terms of all its bits first and then
// applies their inverse butterflies. In the fast (tan) form the vectors of a
// tile carry the pending factor cos(beta)^k of the butterflies applied so far;
// the bilinear terms are corrected by its square and the vectors by the factor
// itself when the tile is stored.
// Passes, sub-passes and rounds come from the adjoint plan (plan.h); one launch
// is one HBM pass reading and writing both vectors.
#pragma once
#include "device.cuh"
#include "pass_kernel.cuh"

namespace qaoa {

struct AdjArgs {
  void* psi;              // 2^n amplitudes (state)
  int psi_store;          // 1: write the uncomputed psi back; 0: psi is read from a
                          // stored forward state and only lambda is written
  void* lam;              // 2^n amplitudes (adjoint vector)
  const int32_t* diag;    // int32 C(x) (stream mode) or nullptr
  const void* phase;      // phase table of the cost layer (ncost entries)
  const int32_t* wmat;    // n x n weights
  const int32_t* ctabs;   // per-round cost tables
  double* partial;        // per-CTA [dA, dC, dB, <C> (first pass)] partial sums
  int phase_in_smem;
  int prefetch;           // 2: the CTA's next tile of psi (PassTma.tmap) and lambda
                          // (PassTma.smap) into L2 by tensor prefetches; 0: none
  int tma_load;           // complex64, one tile per super-tile: the CTA's next tiles of
                          // psi and lambda are loaded into shared memory by tensor loads
                          // (PassTma.tmap, .smap) issued by the last warp to read the
                          // current tile's last round; the first round reads them there
  unsigned long long* err;          // error word: bit 0 set when a tensor-load wait gave up
  unsigned long long tma_wait_ns;   // limit of one tensor-load wait (ns)
};

// Sum over the round's register pairs along bit i of Im(conj(l_a) v_b + conj(l_b) v_a).
template <int R, typename V, typename Real>
__device__ __forceinline__ Real pair_term(const V* v, const V* l, int i) {
  Real s = 0;
#pragma unroll
  for (int j = 0; j < (1 << R); ++j) {
    if (j >> i & 1) continue;
    const int k = j | (1 << i);
    s = fma(l[j].x, v[k].y, s);
    s = fma(-l[j].y, v[k].x, s);
    s = fma(l[k].x, v[j].y, s);
    s = fma(-l[k].y, v[j].x, s);
  }
  return s;
}

// inverse mixer exp(-i beta X) on both vectors for the bits in `mask`; the
// gradient terms of those bits are taken first. In the fast form the vectors
// carry a pending factor `sc` (the cos^k of the butterflies applied so far in
// this tile, restored at the store): the terms, bilinear in the two vectors,
// are added times sc^2, and sc takes this round's cos^k (`cpow`).
template <int R, typename V, typename Real>
__device__ __forceinline__ void inverse_mixer(V* v, V* l, uint8_t mask, Real tau, Real alpha, bool fast, Real cpow,
                                              Real& sc, Real& acc) {
  if (!mask) return;
  Real t = 0;
  if (mask == (1u << R) - 1) {
    // all register bits: straight-line code (no per-bit branches)
#pragma unroll
    for (int i = 0; i < R; ++i) t += pair_term<R, V, Real>(v, l, i);
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int j = 0; j < (1 << R); ++j)
        if (!(j >> i & 1)) {
          bfly<Real>(v[j], v[j | (1 << i)], -tau, alpha, fast);
          bfly<Real>(l[j], l[j | (1 << i)], -tau, alpha, fast);
        }
  } else {
#pragma unroll
    for (int i = 0; i < R; ++i)
      if (mask >> i & 1) t += pair_term<R, V, Real>(v, l, i);
#pragma unroll
    for (int i = 0; i < R; ++i) {
      if (mask >> i & 1) {
#pragma unroll
        for (int j = 0; j < (1 << R); ++j)
          if (!(j >> i & 1)) {
            bfly<Real>(v[j], v[j | (1 << i)], -tau, alpha, fast);
            bfly<Real>(l[j], l[j | (1 << i)], -tau, alpha, fast);
          }
      }
    }
  }
  acc = fma(sc * sc, t, acc);
  if (fast) sc *= cpow;
}

// Swapped storage (complex64, see pass_kernel.cuh): gradient terms of the bits
// in `mask`, then their inverse butterflies on both vectors. For a register
// pair (j, k = j | bit) with n its plain and w its swapped member,
//   Im conj(l_j) v_k + Im conj(l_k) v_j = (P.x - M.x) - (P.y - M.y)
// for the packed products P = l_n * v_w and M = l_w * v_n. The products are
// summed by the parity of j (pa: l_j v_k for even j, l_k v_j for odd j; pb the
// others), which gives (P, M) = (pa, pb) for s = 0 and (pb, pa) for s = 1.
template <int R>
// upd_v = false: psi is not needed after these butterflies (the pass's last
// mixer when psi is read from a stored forward state); only lambda is updated.
__device__ __forceinline__ void inverse_mixer_sw(float2* v, float2* l, uint8_t mask, float tau, float alpha,
                                                 bool fast, float cpow, float& sc, float& acc, int s,
                                                 bool upd_v = true) {
  if (!mask) return;
  float2 pa = make_float2(0.f, 0.f), pb = make_float2(0.f, 0.f);
  auto terms = [&](int i) {
#pragma unroll
    for (int j = 0; j < (1 << R); ++j) {
      if (j >> i & 1) continue;
      const int k = j | (1 << i);
      if (parity_c(j) == 0) {
        pa = __ffma2_rn(l[j], v[k], pa);
        pb = __ffma2_rn(l[k], v[j], pb);
      } else {
        pb = __ffma2_rn(l[j], v[k], pb);
        pa = __ffma2_rn(l[k], v[j], pa);
      }
    }
  };
  if (mask == (1u << R) - 1) {
#pragma unroll
    for (int i = 0; i < R; ++i) terms(i);
  } else {
#pragma unroll
    for (int i = 0; i < R; ++i)
      if (mask >> i & 1) terms(i);
  }
  const float t0 = (pa.x - pb.x) - (pa.y - pb.y);
  const float t = s ? -t0 : t0;
  if (upd_v) apply_mixer_sw<R>(v, mask, -tau, alpha, fast, s);
  apply_mixer_sw<R>(l, mask, -tau, alpha, fast, s);
  acc = fmaf(sc * sc, t, acc);
  if (fast) sc *= cpow;
}

template <typename Real>
__device__ __forceinline__ Real pow_bits(Real c, uint8_t mask) {
  Real r = 1;
  for (int i = 0; i < 8; ++i)
    if (mask >> i & 1) r *= c;
  return r;
}

// Asynchronous tile prefetch state of an adjoint pass (complex64, one tile per
// super-tile): the tile's vectors were copied into shared memory while the
// previous tile finished; the last round, once every thread has read its
// amplitudes, starts the copy of the next tile (super-tile gnext).
struct AdjPrefetch {
  bool on;      // this pass copies tiles asynchronously
  bool next;    // a next tile exists for this CTA
  uint64_t gnext;
};

template <typename Real, int R, int WB, bool FAST, bool CC = true, uint32_t SIG = 0>
__device__ __forceinline__ void adj_round(const PassDev& P, const AdjArgs& A, const SubDev& sp, const RoundDev& rd,
                                          typename Cx<Real>::T* tv, typename Cx<Real>::T* tl, uint64_t gbase,
                                          int gpar, const int* tconst, const typename Cx<Real>::T* phase, int lane,
                                          int warp,
                                          Real& ga, Real& gc, Real& gbv, Real& ge, Real& sc,
                                          typename Cx<Real>::T* v, typename Cx<Real>::T* l, const AdjPrefetch& pf,
                                          const PassTma* M = nullptr, uint32_t tbar = 0, uint64_t tnext = ~0ull) {
  using C2 = typename Cx<Real>::T;
  constexpr int NA = 1 << R;
  constexpr int AB = sizeof(C2);
  C2* gpsi = reinterpret_cast<C2*>(A.psi);
  C2* glam = reinterpret_cast<C2*>(A.lam);
  const bool stream = A.diag != nullptr;
  // the round's geometry is rebuilt where it is used instead of being kept
  // live across the butterflies (register pressure)
  using Geo = RoundGeo<R, WB, AB>;
  // complex64: swapped storage; s = parity of the thread's amplitude 0
  constexpr bool kSw = sizeof(Real) == 4;
  const uint32_t entry = Geo::entry_of(rd, lane, warp, A.ctabs);
  const uint32_t sb = entry & 0x7fffffffu;
  const int s = kSw ? int(entry >> 31) ^ gpar : 0;
  const RoundOps<SIG> op(rd);
  const bool need_c = CC && (op.cost || op.lam);
  RoundCost<R, WB> rcost;
  if (need_c && !stream) rcost.setup(A.ctabs + rd.ctab, tconst, rd.lane, rd.warp, rd.reg, lane, warp);
  // cp: the register-pair table CP[j] of the pass's cost round (P.cpc) or
  // lambda-creation round (P.cpr), from the descriptor
  auto for_costs = [&](const int32_t* cp, auto&& f) {
    if (stream) {
      const Geo geo(sp, rd, gbase, lane, warp, A.ctabs);
      gray_ptr_walk<R>(A.diag, geo.gb, geo.gstr, [&](int j, const int32_t* q) { f(j, __ldcg(q)); });
    } else {
      int lin = rcost.kappa;
#pragma unroll
      for (int k = 0; k < NA; ++k) {
        const int j = k ^ (k >> 1);
        if (k) {
          const int b = ctz_c(k);
          lin += (j >> b & 1) ? rcost.e[b] : -rcost.e[b];
        }
        f(j, lin + cp[j]);
      }
    }
  };

  // a global round's loads were issued by the caller before the tile barrier,
  // or copied into shared memory (prefetch)
  if (op.src == SRC_GLOBAL_D && pf.on) {
    smem_load<R, WB, AB>(op.layout, tv, sb, v);
    if (!(CC && op.lam)) smem_load<R, WB, AB>(op.layout, tl, sb, l);
  }
  if constexpr (kSw) {
    // the first sub-pass reads the forward run's plain amplitudes (psi only:
    // lambda is created from it)
    if (op.src == SRC_GLOBAL_D && sp.ld_plain) swap_odd<R>(reinterpret_cast<float2*>(v), s);
  }
  if (op.src == SRC_GLOBAL_D) {
    if (CC && op.lam) {
      // lambda = C(x) psi (the operator whose expectation is differentiated);
      // <psi|lambda> = <C> on the way
      for_costs(P.cpr, [&](int j, int c) {
        const Real cr = Real(c);
        l[j].x = cr * v[j].x;
        l[j].y = cr * v[j].y;
        ge = fma(cr, fma(v[j].x, v[j].x, v[j].y * v[j].y), ge);
      });
    }
  } else {
    smem_load<R, WB, AB>(op.layout, tv, sb, v);
    smem_load<R, WB, AB>(op.layout, tl, sb, l);
  }
  if constexpr (sizeof(Real) == 4) {
    if (A.tma_load && op.dstg && op.src == SRC_SMEM_D) {
      // once every warp has read the tile's last round, the tiles take the
      // CTA's next ones by tensor loads, issued by the last warp to finish
      // its reads (lambda is not loaded where the pass creates it)
      __syncwarp();
      if (lane == 0) {
        __threadfence_block();
        if (tile_read_count_add(tbar) == (1u << WB) - 1) {
          __threadfence_block();
          tile_read_count_reset(tbar);
          if (tnext < P.n_units && !tma_stopped(tbar)) {
            fence_proxy_async_smem();
            int32_t c[5];
            tile_coords(*M, P.outer_runs.scatter(tnext), c);
            const bool two = !(CC && sp.rd[0].lam);
            mbar_expect_tx(tbar, (uint32_t(AB) << (R + 5 + WB)) * (two ? 2u : 1u));
            tma_load_box(&M->tmap, M->tdims, c, (uint32_t)__cvta_generic_to_shared(dense_tile(tv)), tbar);
            if (two) tma_load_box(&M->smap, M->tdims, c, (uint32_t)__cvta_generic_to_shared(dense_tile(tl)), tbar);
          }
        }
      }
    }
  }

  if constexpr (sizeof(Real) == 4) {
    if (pf.on && op.dstg) {
      // every thread has read its amplitudes: the tiles are free for the next copy
      __syncthreads();
      if (pf.next) {
        const int tid = (warp << 5) | lane;
        tile_copy_async<R, WB>(tv, reinterpret_cast<const float2*>(A.psi), pf.gnext, sp, tid, A.ctabs);
        if (!(CC && sp.rd[0].lam))
          tile_copy_async<R, WB>(tl, reinterpret_cast<const float2*>(A.lam), pf.gnext, sp, tid, A.ctabs);
        cp_async_commit();
      }
    }
  }

  // psi read from a stored forward state is not written back: the pass's last
  // mixer need not update it (complex64)
  const bool v_dead = op.dstg && !A.psi_store;
  auto inv_mixer = [&](uint8_t mask, Real tau, Real alpha, Real cpow, Real& acc, bool upd_v) {
    if constexpr (kSw)
      inverse_mixer_sw<R>(reinterpret_cast<float2*>(v), reinterpret_cast<float2*>(l), mask, tau, alpha, FAST, cpow,
                          sc, acc, s, upd_v);
    else
      inverse_mixer<R>(v, l, mask, tau, alpha, FAST, cpow, sc, acc);
  };
  inv_mixer(op.mixA, pick<Real>(P.tauA, P.ftauA), pick<Real>(P.alphaA, P.falphaA),
            pow_bits(pick<Real>(P.cA, P.fcA), op.mixA), ga, !(v_dead && !op.mixB && !(CC && op.cost)));
  if (CC && op.cost) {
    // Im conj(l) v of a swapped pair of amplitudes has the opposite sign: the
    // terms are summed by the parity of j and combined with the thread's s;
    // a swapped amplitude takes the conjugate phase in the plain product
    // formula (angle scale k1 = -k0)
    Real tc0 = 0, tc1 = 0;
    const float k0 = s ? -kTurn32 : kTurn32, k1 = -k0;
    auto apply = [&](int j, Real h, C2 ph) {
      const Real q = fma(l[j].x, v[j].y, -l[j].y * v[j].x);
      if (parity_c(j)) tc1 = fma(q, h, tc1); else tc0 = fma(q, h, tc0);
      // multiply both vectors by the conjugate phase (inverse cost unitary)
      const Real vr = v[j].x, vi = v[j].y, lr = l[j].x, li = l[j].y;
      v[j].x = vr * ph.x + vi * ph.y;
      v[j].y = vi * ph.x - vr * ph.y;
      l[j].x = lr * ph.x + li * ph.y;
      l[j].y = li * ph.x - lr * ph.y;
    };
    bool walked = false;
    if constexpr (kSw) {
      if (!stream) {
        // complex64 from the tables: h(x) = W - 2 C(x) and the phase's 32-bit
        // turn count both follow the Gray walk (see fwd_round)
        walked = true;
        uint32_t E[R];
        uint32_t t = rcost.turns(P.ph0, P.ph1, P.c_lo, E);
        int lin = rcost.kappa;
#pragma unroll
        for (int k = 0; k < NA; ++k) {
          const int j = k ^ (k >> 1);
          if (k) {
            const int b = ctz_c(k);
            lin += (j >> b & 1) ? rcost.e[b] : -rcost.e[b];
            t += (j >> b & 1) ? E[b] : 0u - E[b];
          }
          const C2 ph = phase_turns32(t + P.cpt[j], parity_c(j) ? k1 : k0);
          apply(j, Real(P.wsum - 2 * (lin + P.cpc[j])), ph);
        }
      }
    }
    if (!walked) {
      for_costs(P.cpc, [&](int j, int c) {
        C2 ph;
        if constexpr (kSw) ph = phase_turns(P.ph0, P.ph1, uint32_t(c - P.c_lo), parity_c(j) ? k1 : k0);
        else ph = phase[min(unsigned(c - P.c_lo), unsigned(P.ncost - 1))];
        apply(j, Real(P.wsum - 2 * c), ph);
      });
    }
    const Real tc = !kSw ? tc0 + tc1 : s ? tc1 - tc0 : tc0 - tc1;
    gc = fma(sc * sc, tc, gc);
  }
  inv_mixer(op.mixB, pick<Real>(P.tauB, P.ftauB), pick<Real>(P.alphaB, P.falphaB),
            pow_bits(pick<Real>(P.cB, P.fcB), op.mixB), gbv, !v_dead);

  if (op.dstg) {
    if (sp.store) {
      const Geo geo(sp, rd, gbase, lane, warp, A.ctabs);
      if (A.psi_store) {
        if (FAST) {
#pragma unroll
          for (int j = 0; j < NA; ++j) { v[j].x *= sc; v[j].y *= sc; }
        }
        gray_ptr_walk<R>(gpsi, geo.gb, geo.gstr, [&](int j, C2* q) { __stcg(q, v[j]); });
      }
      if (FAST) {
#pragma unroll
        for (int j = 0; j < NA; ++j) { l[j].x *= sc; l[j].y *= sc; }
      }
      gray_ptr_walk<R>(glam, geo.gb, geo.gstr, [&](int j, C2* q) { __stcg(q, l[j]); });
    }
  } else {
    smem_store<R, WB, AB>(op.layout, tv, sb, v);
    smem_store<R, WB, AB>(op.layout, tl, sb, l);
  }
}

// One super-tile (unit) of an adjoint pass; the gradient terms of this
// thread's amplitudes are added to gA, gC, gB.
// tcount: the CTA's running tile count (tile-constant buffer when the
// constants come from a table); may be null when no sub-pass has a table.
// RS: the round signatures of a specialised kernel (one sub-pass of one tile
// per unit), empty for the generic kernel.
template <typename Real, int R, int WB, bool FAST, bool CC = true, uint32_t... RS>
__device__ __forceinline__ void adj_unit(const PassDev& P, const AdjArgs& A, uint64_t unit,
                                         typename Cx<Real>::T* tv, typename Cx<Real>::T* tl, int* tconst,
                                         const typename Cx<Real>::T* phase, double& gA, double& gC, double& gB,
                                         double& gE, uint32_t* tcount = nullptr, const PassTma* M = nullptr,
                                         uint32_t tbar = 0, uint32_t* tk = nullptr) {
  using C2 = typename Cx<Real>::T;
  constexpr int T = R + 5 + WB;
  constexpr int NT = 32 << WB;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = P.n;
  const bool stream = A.diag != nullptr;
  constexpr bool kSpec = sizeof...(RS) > 0;
  const uint64_t ubase = P.outer_runs.scatter(unit);
  for (int s = 0; s < (kSpec ? 1 : P.nsub); ++s) {
    const SubDev& sp = P.sub[s];
    const uint64_t ntiles = kSpec ? 1 : 1ull << sp.ninner;
    AdjPrefetch pf;
    pf.on = sizeof(Real) == 4 && sp.cgtab >= 0;  // one sub-pass of one tile per unit
    pf.next = pf.on && unit + gridDim.x < P.n_units;
    pf.gnext = pf.next ? P.outer_runs.scatter(unit + gridDim.x) : 0;
    for (uint64_t ti = 0; ti < ntiles; ++ti) {
      const uint64_t gbase = kSpec ? ubase : ubase | sp.inner_runs.scatter(ti);
      // issue the first round's global loads first: their latency overlaps the
      // barrier below and the tile constants
      C2 v[1 << R], l[1 << R];
      bool load0;
      if constexpr (kSpec) load0 = (first_sig<RS...>() >> 2 & 3u) == SRC_GLOBAL_D;
      else load0 = sp.rd[0].src == SRC_GLOBAL_D;
      if (load0 && A.prefetch == 2 && sp.ninner == 0 && tid == 0) {
        // the CTA's next tile of both vectors into L2 by tensor prefetches
        // (tensor memory accelerator; no load-store unit instructions)
        const uint64_t next = unit + gridDim.x;
        if (next < P.n_units) {
          int32_t c[5];
          tile_coords(*M, P.outer_runs.scatter(next), c);
          tma_prefetch_l2(&M->tmap, M->tdims, c);
          if (!(CC && sp.rd[0].lam)) tma_prefetch_l2(&M->smap, M->tdims, c);
        }
      }
      const bool tload = sizeof(Real) == 4 && load0 && A.tma_load;
      if (load0 && !pf.on && !tload) {
        const RoundGeo<R, WB, sizeof(C2)> g0(sp, sp.rd[0], gbase, lane, warp, A.ctabs);
        gray_ptr_walk<R>(reinterpret_cast<const C2*>(A.psi), g0.gb, g0.gstr,
                         [&](int j, const C2* q) { v[j] = __ldcg(q); });
        if (!(CC && sp.rd[0].lam))
          gray_ptr_walk<R>(reinterpret_cast<const C2*>(A.lam), g0.gb, g0.gstr,
                           [&](int j, const C2* q) { l[j] = __ldcg(q); });
      }
      int* tc = tconst;
      const bool tab = CC && sp.needs_c && !stream && sp.tct != nullptr;
      if (tab) {
        tc = tconst + 32 * (*tcount & 1u);
        *tcount += 1;
        if (tid < kTileConstInts)
          tc[tid == 15 ? 16 : tid] = __ldg(sp.tct + (((unit << sp.ninner) + ti) * kTileConstInts + tid));
      }
      if (pf.on) cp_async_wait_all();  // this tile's copies (issued by this thread)
      if constexpr (sizeof(Real) == 4) {
        if (tload) {
          // this tile's vectors arrived by tensor loads (the CTA's k-th,
          // mbarrier phase k & 1): the first round's amplitudes from the
          // dense boxes; the barrier below ends the reads before the first
          // round writes the padded tiles
          const uint32_t k = (*tk)++;
          if (!tma_stopped(tbar) && !mbar_wait_bounded(tbar, k & 1u, A.tma_wait_ns)) {
            tma_stop(tbar, k & 1u);
            if (lane == 0) atomicOr(A.err, 1ull);
          }
          constexpr uint32_t S0 = first_sig_or0<RS...>();
          const RoundDev& rd0 = sp.rd[0];
          uint32_t tb = 0;
#pragma unroll
          for (int i = 0; i < 5; ++i) tb |= uint32_t(lane >> i & 1) << tile_bit<R, WB, S0>(rd0, 1, i);
#pragma unroll
          for (int i = 0; i < WB; ++i) tb |= uint32_t(warp >> i & 1) << tile_bit<R, WB, S0>(rd0, 2, i);
          uint32_t toff[1 << R];
#pragma unroll
          for (int j = 0; j < (1 << R); ++j) {
            toff[j] = 0;
#pragma unroll
            for (int i = 0; i < R; ++i)
              if (j >> i & 1) toff[j] |= 1u << tile_bit<R, WB, S0>(rd0, 0, i);
          }
          const C2* dv = dense_tile(tv);
#pragma unroll
          for (int j = 0; j < (1 << R); ++j) v[j] = dv[tb + toff[j]];
          if (!(CC && rd0.lam)) {
            const C2* dl = dense_tile(tl);
#pragma unroll
            for (int j = 0; j < (1 << R); ++j) l[j] = dl[tb + toff[j]];
          }
        }
      }
      __syncthreads();
      if (CC && sp.needs_c && !stream && !tab) {
        if (tid == 0) tconst[16] = 0;
        __syncthreads();
        tile_consts<T>(sp.pos, gbase, A.wmat, n, tconst, lane, warp, NT / 32);
        __syncthreads();
      }
      Real sc = 1;  // pending fast-form factor of this tile's vectors
      const int gpar = __popcll(gbase) & 1;
      if constexpr (sizeof(Real) == 8) {
        for (int r = 0; r < sp.nrounds; ++r) {
          const RoundDev& rd = sp.rd[r];
          if (rd.src == SRC_SMEM_D) __syncthreads();
          adj_round<Real, R, WB, FAST, CC>(P, A, sp, rd, tv, tl, gbase, gpar, tc, phase, lane, warp, gA, gC, gB, gE,
                                           sc, v, l, pf, M, tbar, unit + gridDim.x);
        }
      } else {
        // fp32: the terms of one tile are summed in fp32, then added in FP64
        // (keeps fp64 conversions out of the rounds)
        Real ga = 0, gc = 0, gbv = 0, ge = 0;
        if constexpr (kSpec) {
          // rounds unrolled from the signatures
          int r = 0;
          auto run = [&](auto sigc) {
            constexpr uint32_t S = decltype(sigc)::value;
            if constexpr ((S >> 2 & 3u) == SRC_SMEM_D) __syncthreads();
            adj_round<Real, R, WB, FAST, CC, S>(P, A, sp, sp.rd[r], tv, tl, gbase, gpar, tc, phase, lane, warp, ga,
                                                gc, gbv, ge, sc, v, l, pf, M, tbar, unit + gridDim.x);
            ++r;
          };
          (run(std::integral_constant<uint32_t, RS>{}), ...);
        } else {
          for (int r = 0; r < sp.nrounds; ++r) {
            const RoundDev& rd = sp.rd[r];
            if (rd.src == SRC_SMEM_D) __syncthreads();
            adj_round<Real, R, WB, FAST, CC>(P, A, sp, rd, tv, tl, gbase, gpar, tc, phase, lane, warp, ga, gc, gbv,
                                             ge, sc, v, l, pf, M, tbar, unit + gridDim.x);
          }
        }
        gA += double(ga);
        gC += double(gc);
        gB += double(gbv);
        gE += double(ge);
      }
    }
    __syncthreads();
  }
}

// Body of the adjoint pass kernels.
// Shared memory: psi tile (padded 2^T) | lambda tile | tile consts (two buffers) | phase table
template <typename Real, int R, int WB, bool FAST, bool CC, uint32_t... RS>
__device__ __forceinline__ void adj_pass_body(const PassDev& P, const AdjArgs& A, const PassTma& M) {
  using C2 = typename Cx<Real>::T;
  constexpr int T = R + 5 + WB;
  constexpr int NT = 32 << WB;
  constexpr int AB = sizeof(C2);
  constexpr uint32_t TILE = padded_size<AB>(T);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* tv = reinterpret_cast<C2*>(smem_raw);
  C2* tl = tv + TILE;
  int* tconst = reinterpret_cast<int*>(tl + TILE);
  C2* ptab = reinterpret_cast<C2*>(smem_raw + ((size_t(2 * TILE) * AB + kTconstSmemInts * 4 + 15) & ~size_t(15)));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const C2* phase = reinterpret_cast<const C2*>(A.phase);
  if (A.phase_in_smem && A.phase) {
    for (int i = tid; i < P.ncost; i += NT) ptab[i] = phase[i];
    phase = ptab;
  }
  double gA = 0.0, gC = 0.0, gB = 0.0, gE = 0.0;

  uint32_t tcount = 0;
  if constexpr (sizeof(Real) == 4) {
    // asynchronous tile copies: the first tile's copy before the loop
    const SubDev& sp0 = P.sub[0];
    if (sp0.cgtab >= 0 && blockIdx.x < P.n_units) {
      const uint64_t g0 = P.outer_runs.scatter(blockIdx.x);
      tile_copy_async<R, WB>(tv, reinterpret_cast<const float2*>(A.psi), g0, sp0, tid, A.ctabs);
      if (!(CC && sp0.rd[0].lam)) tile_copy_async<R, WB>(tl, reinterpret_cast<const float2*>(A.lam), g0, sp0, tid, A.ctabs);
      cp_async_commit();
    }
  }
  // tensor tile loads: the mbarrier (then the stop word and the warps' read
  // count), and the CTA's first tiles
  __shared__ __align__(8) unsigned long long tma_bar[2];
  const uint32_t tbar = (uint32_t)__cvta_generic_to_shared(tma_bar);
  uint32_t tk = 0;
  if constexpr (sizeof(Real) == 4) {
    if (A.tma_load) {
      if (tid == 0) {
        tma_bar[1] = 0ull;
        mbar_init(tbar, 1);
      }
      __syncthreads();
      if (tid == 0 && blockIdx.x < P.n_units) {
        int32_t c[5];
        tile_coords(M, P.outer_runs.scatter(blockIdx.x), c);
        const bool two = !(CC && P.sub[0].rd[0].lam);
        mbar_expect_tx(tbar, (uint32_t(AB) << T) * (two ? 2u : 1u));
        tma_load_box(&M.tmap, M.tdims, c, (uint32_t)__cvta_generic_to_shared(dense_tile(tv)), tbar);
        if (two) tma_load_box(&M.smap, M.tdims, c, (uint32_t)__cvta_generic_to_shared(dense_tile(tl)), tbar);
      }
    }
  }
  for (uint64_t unit = blockIdx.x; unit < P.n_units; unit += gridDim.x)
    adj_unit<Real, R, WB, FAST, CC, RS...>(P, A, unit, tv, tl, tconst, phase, gA, gC, gB, gE, &tcount, &M, tbar, &tk);
  if constexpr (sizeof(Real) == 4) {
    if (A.tma_load) {
      // a CTA whose wait gave up ends only once the loads it gave up on have
      // landed (bounded)
      __syncthreads();
      const uint32_t f = tid == 0 ? tma_stop_word(tbar) : 0u;
      if (f) mbar_wait_bounded(tbar, f - 1u, kTmaWaitNs);
    }
  }

  __shared__ double red[4][32];
  for (int o = 16; o > 0; o >>= 1) {
    gA += __shfl_xor_sync(0xffffffffu, gA, o);
    gC += __shfl_xor_sync(0xffffffffu, gC, o);
    gB += __shfl_xor_sync(0xffffffffu, gB, o);
    gE += __shfl_xor_sync(0xffffffffu, gE, o);
  }
  if (lane == 0) { red[0][warp] = gA; red[1][warp] = gC; red[2][warp] = gB; red[3][warp] = gE; }
  __syncthreads();
  if (tid == 0) {
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    for (int w = 0; w < NT / 32; ++w) { s0 += red[0][w]; s1 += red[1][w]; s2 += red[2][w]; s3 += red[3][w]; }
    A.partial[4 * blockIdx.x] = s0;
    A.partial[4 * blockIdx.x + 1] = s1;
    A.partial[4 * blockIdx.x + 2] = s2;
    A.partial[4 * blockIdx.x + 3] = s3;
  }
}

// Generic adjoint pass: rounds decoded from the descriptor at run time.
template <typename Real, int R, int WB, bool FAST, bool CC>
__global__ void __launch_bounds__(32 << WB, sizeof(Real) == 4 ? 2 : 1)
adj_pass_kernel(const __grid_constant__ PassDev P, const AdjArgs A, const __grid_constant__ PassTma M) {
  adj_pass_body<Real, R, WB, FAST, CC>(P, A, M);
}

// Specialised complex64 adjoint pass for one round-signature sequence RS (one
// sub-pass of one tile per super-tile).
template <int R, int WB, bool FAST, uint32_t... RS>
__global__ void __launch_bounds__(32 << WB, 2)
adj_spec_kernel(const __grid_constant__ PassDev P, const AdjArgs A, const __grid_constant__ PassTma M) {
  adj_pass_body<float, R, WB, FAST, sigs_need_c<RS...>(), RS...>(P, A, M);
}

}  // namespace qaoa
