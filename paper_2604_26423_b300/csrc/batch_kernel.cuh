// batch_kernel.cuh -- many independent LR-QAOA instances in one persistent launch.
//
// A batch runs as two persistent launches, the forward phase and (with the
// gradient) the adjoint phase; each is a list of work items that its CTAs take
// in order from a global counter. Item kinds:
//   SMALL  the whole circuit of one instance in one CTA's shared memory
//          (forward, or forward and adjoint gradient), with its extremes;
//   SOLO   every pass of one phase of one instance run by one CTA over its
//          state in global memory (small enough to stay in L2);
//   PASS   a range of super-tiles of one forward or adjoint pass of a large
//          instance; it may start only when every item of the instance's
//          earlier passes has finished;
//   EXT    a range of 2^13-configuration blocks of one instance's exhaustive
//          C_min / C_max search (Sec. II-B, r uses C(x*)).
// The host orders the items so that an item only waits on items with smaller
// queue indices; those have been taken by running CTAs that never wait on later
// items, so every wait ends. Waits are bounded all the same (a time limit after
// which the batch's error flag is set and the item is skipped).
// The math of each pass is the single-instance kernels' (fwd_unit, adj_unit).
// Each launch is compiled for one mixer form (fast tan form, or plain cos/sin
// when some angle of the batch has |tan beta| > 1) and one phase, which keeps
// the register pressure of a single pass kernel.
#pragma once
#include <cstddef>
#include "adj_kernel.cuh"
#include "aux_kernels.cuh"
#include "device.cuh"
#include "pass_kernel.cuh"

namespace qaoa {

enum : int32_t { BITEM_SMALL = 0, BITEM_SOLO = 1, BITEM_PASS = 2, BITEM_EXT = 3 };
enum : int32_t { BMODE_SMALL = 0, BMODE_SOLO = 1, BMODE_MULTI = 2 };

constexpr int kBatchR = 5, kBatchWB = 3;        // default forward tile (T = 13); 4x3 (T = 12) selectable
constexpr int kBatchRAdj = 4, kBatchWBAdj = 3;  // adjoint tile (T = 12)
constexpr int kBatchThreads = 256;
constexpr int kBatchExtBits = 13;               // configurations per EXT block
constexpr int kBatchMaxN = 24;
constexpr int kBatchSmallMax = 12;              // forward in shared memory up to n = 12
constexpr int kBatchSmallGradMax = 11;          // forward + adjoint up to n = 11

struct BatchItem {
  int32_t inst;   // instance index
  int32_t kind;   // BITEM_*
  int32_t pass;   // global pass index (PASS)
  int32_t slot;   // partial-sum slot (PASS)
  uint32_t u0, u1;  // super-tile range (PASS) or block range (EXT)
  int32_t need;   // finished PASS items of this instance required first
  int32_t pad;
};

struct BatchInst {
  int32_t n, p, c_lo, ncost;
  int32_t wsum, mode;
  int32_t fwd_pass0, fwd_npass;   // forward passes (global indices), 0 for SMALL
  int32_t adj_pass0, adj_npass;   // adjoint passes, 0 without gradient or for SMALL
  int32_t slot0, nslots;          // FP64 slots: [norm, <C>] then 3 per adjoint item
  int32_t g_off, with_grad;       // offset of this instance's g_gamma / g_beta (p each)
  void* psi;
  void* lam;
  const int32_t* wmat;            // n x n
  const int32_t* ctabs;           // this instance's cost tables
  const int32_t* diag;            // int32 C(x) of all 2^n x (streamed cost), or nullptr
  const float2* phase;            // p tables of ncost entries
  const double* ang;              // (gamma_k, beta_k) interleaved
  double scale;                   // phase weight scale s
};

struct PassMeta {
  int32_t inst, layer_a, layer_c, layer_b;
  int32_t fast, reduce, adjoint, slot0;  // slot0: first slot of this pass's items
  int32_t nitems, pad[3];
};

struct BatchArgs {
  const BatchItem* items;         // this phase's queue
  int32_t nitems;
  const BatchInst* insts;
  const PassDev* passes;
  const PassMeta* pmeta;
  unsigned int* head;             // next item index
  int32_t* done;                  // finished PASS items per instance (this phase)
  double* slots;                  // FP64 partial sums
  unsigned long long* ext_min;    // packed (C + 2^31) << 32 | x, min
  unsigned long long* ext_max;    // packed (C + 2^31) << 32 | ~x, max
  double* grads;                  // g_gamma[p] | g_beta[p] per instance (SMALL grad)
  int32_t* error;                 // set when a wait gave up
  unsigned long long wait_ns;     // dependency wait limit
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acquire(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(int32_t* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ext_key_min(long long c, unsigned long long x) {
  return ((unsigned long long)(c + (1ll << 31)) << 32) | (x & 0xffffffffull);
}
__device__ __forceinline__ unsigned long long ext_key_max(long long c, unsigned long long x) {
  return ((unsigned long long)(c + (1ll << 31)) << 32) | (0xffffffffull - (x & 0xffffffffull));
}

__device__ __forceinline__ double block_sum(double x, double* red) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  double t = 0;
  for (int w = 0; w < kBatchThreads / 32; ++w) t += red[w];
  return t;
}

// Block min / max of C with the smallest index, merged into the instance's slots.
__device__ __forceinline__ void ext_commit(Extreme ex, Extreme* red, const BatchArgs& B, int inst) {
  ext_warp_merge(ex);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ex;
  __syncthreads();
  if (threadIdx.x == 0) {
    Extreme r = red[0];
    for (int i = 1; i < kBatchThreads / 32; ++i) ext_merge(r, red[i]);
    if (r.vmin != LLONG_MAX) {
      atomicMin(B.ext_min + inst, ext_key_min(r.vmin, r.amin));
      atomicMax(B.ext_max + inst, ext_key_max(r.vmax, r.amax));
    }
  }
}

// C(x) = sum_{k<l} w_kl [x_k != x_l] for every x < 2^n into cut[] (n <= 12).
__device__ __forceinline__ void small_cuts(const BatchInst& I, int* cut, Extreme& ex) {
  const int n = I.n, N = 1 << n;
  for (int x = threadIdx.x; x < N; x += kBatchThreads) {
    int c = 0;
    for (int g = 0; g < n; ++g)
      for (int h = g + 1; h < n; ++h)
        if ((x >> g & 1) != (x >> h & 1)) c += __ldg(I.wmat + g * n + h);
    cut[x] = c;
    if (c < ex.vmin) { ex.vmin = c; ex.amin = (unsigned long long)x; }
    if (c > ex.vmax) { ex.vmax = c; ex.amax = (unsigned long long)x; }
  }
}

// Forward circuit of a SMALL instance in shared memory: cost phase from the
// layer's phase table (Eqs. H_C, UC), then exp(+i beta_k X_q) for every qubit
// (Eq. UB). Leaves psi_p in s[] and the cuts in cut[].
__device__ __forceinline__ void small_forward(const BatchInst& I, float2* s, const int* cut) {
  const int n = I.n, N = 1 << n, tid = threadIdx.x;
  const float amp0 = float(rsqrt(double(N)));
  for (int x = tid; x < N; x += kBatchThreads) s[x] = make_float2(amp0, 0.f);
  for (int k = 0; k < I.p; ++k) {
    __syncthreads();
    const float2* ph = I.phase + (size_t)k * I.ncost;
    for (int x = tid; x < N; x += kBatchThreads) {
      const float2 f = ph[min(max(cut[x] - I.c_lo, 0), I.ncost - 1)];
      const float xr = s[x].x, xi = s[x].y;
      s[x] = make_float2(xr * f.x - xi * f.y, xr * f.y + xi * f.x);
    }
    const double beta = I.ang[2 * k + 1];
    const float cb = float(cos(beta)), sb = float(sin(beta));
    for (int q = 0; q < n; ++q) {
      __syncthreads();
      for (int i = tid; i < N / 2; i += kBatchThreads) {
        const int x0 = ((i >> q) << (q + 1)) | (i & ((1 << q) - 1));
        const int x1 = x0 | (1 << q);
        const float2 p0 = s[x0], p1 = s[x1];
        s[x0] = make_float2(fmaf(cb, p0.x, -sb * p1.y), fmaf(cb, p0.y, sb * p1.x));
        s[x1] = make_float2(fmaf(cb, p1.x, -sb * p0.y), fmaf(cb, p1.y, sb * p0.x));
      }
    }
  }
  __syncthreads();
}

// SMALL item: forward (and, with gradient, the adjoint sweep) in shared memory.
// Slots: [norm, <C>]; gradient terms go straight to grads[g_off ..].
__device__ __noinline__ void batch_small(const BatchArgs& B, const BatchInst& I, int inst, unsigned char* smem,
                                         double* red, Extreme* ered) {
  const int n = I.n, N = 1 << n, tid = threadIdx.x;
  float2* s = reinterpret_cast<float2*>(smem);
  float2* l = s + N;
  int* cut = reinterpret_cast<int*>(l + (I.with_grad ? N : 0));
  Extreme ex = ext_empty();
  small_cuts(I, cut, ex);
  ext_commit(ex, ered, B, inst);
  small_forward(I, s, cut);
  double nr = 0.0, ec = 0.0;
  for (int x = tid; x < N; x += kBatchThreads) {
    const float2 v = s[x];
    const double pr = double(v.x) * v.x + double(v.y) * v.y;
    nr += pr;
    ec += pr * double(cut[x]);
    if (I.with_grad) {
      const float c = float(cut[x]);
      l[x] = make_float2(c * v.x, c * v.y);
    } else {
      __stcg(reinterpret_cast<float2*>(I.psi) + x, v);
    }
  }
  nr = block_sum(nr, red);
  ec = block_sum(ec, red);
  if (tid == 0) {
    B.slots[I.slot0] = nr;
    B.slots[I.slot0 + 1] = ec;
  }
  if (!I.with_grad) return;
  double* gg = B.grads + I.g_off;
  for (int k = I.p - 1; k >= 0; --k) {
    const double beta = I.ang[2 * k + 1];
    const float cb = float(cos(beta)), sb = float(sin(beta));
    double tb = 0.0;
    for (int q = 0; q < n; ++q) {
      __syncthreads();
      for (int i = tid; i < N / 2; i += kBatchThreads) {
        const int x0 = ((i >> q) << (q + 1)) | (i & ((1 << q) - 1));
        const int x1 = x0 | (1 << q);
        const float2 p0 = s[x0], p1 = s[x1], m0 = l[x0], m1 = l[x1];
        // Im(conj(l0) p1 + conj(l1) p0), taken before the inverse rotation
        tb += double(m0.x) * p1.y - double(m0.y) * p1.x + double(m1.x) * p0.y - double(m1.y) * p0.x;
        s[x0] = make_float2(fmaf(cb, p0.x, sb * p1.y), fmaf(cb, p0.y, -sb * p1.x));
        s[x1] = make_float2(fmaf(cb, p1.x, sb * p0.y), fmaf(cb, p1.y, -sb * p0.x));
        l[x0] = make_float2(fmaf(cb, m0.x, sb * m1.y), fmaf(cb, m0.y, -sb * m1.x));
        l[x1] = make_float2(fmaf(cb, m1.x, sb * m0.y), fmaf(cb, m1.y, -sb * m0.x));
      }
    }
    __syncthreads();
    const float2* ph = I.phase + (size_t)k * I.ncost;
    double tg = 0.0;
    for (int x = tid; x < N; x += kBatchThreads) {
      const float2 f = ph[min(max(cut[x] - I.c_lo, 0), I.ncost - 1)];
      const float2 v = s[x], m = l[x];
      tg += (double(m.x) * v.y - double(m.y) * v.x) * double(I.wsum - 2 * cut[x]);
      s[x] = make_float2(v.x * f.x + v.y * f.y, v.y * f.x - v.x * f.y);
      l[x] = make_float2(m.x * f.x + m.y * f.y, m.y * f.x - m.x * f.y);
    }
    tb = block_sum(tb, red);
    tg = block_sum(tg, red);
    if (tid == 0) {
      gg[I.p + k] = -2.0 * tb;
      gg[k] = 2.0 * I.scale * tg;
    }
  }
}

// EXT item: blocks [b0, b1) of 2^13 consecutive configurations x < 2^(n-1)
// (C(x) = C(~x), so the lower half holds every value and the smallest index).
// Thread t covers x = block | t << 5 | j for j < 32, with C split as
//   C = C_hi + sum_{k<13} x_k delta_k + C_13(x mod 2^13),
//   delta_k = sum_{g>=13} w_kg (1 - 2 x_g),  C_hi over the pairs g<h>=13 plus
//   sum_{k<13, g>=13} w_kg x_g (weights of missing vertices are zero).
__device__ __noinline__ void batch_ext(const BatchArgs& B, const BatchInst& I, int inst, uint32_t b0, uint32_t b1,
                                       unsigned char* smem, Extreme* ered) {
  constexpr int LB = kBatchExtBits;
  const int n = I.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int* w = reinterpret_cast<int*>(smem);  // kBatchMaxN x kBatchMaxN, zero padded
  int* delta = w + kBatchMaxN * kBatchMaxN;
  int* misc = delta + 32;                 // [0] C_hi part
  for (int i = tid; i < kBatchMaxN * kBatchMaxN; i += kBatchThreads) {
    const int g = i / kBatchMaxN, h = i % kBatchMaxN;
    w[i] = (g < n && h < n) ? __ldg(I.wmat + g * n + h) : 0;
  }
  const unsigned long long limit = n >= 1 ? 1ull << (n - 1) : 1ull;
  Extreme ex = ext_empty();
  // thread-invariant parts over bits 0..12
  for (uint32_t b = b0; b < b1; ++b) {
    const unsigned long long hi = (unsigned long long)b << LB;
    __syncthreads();
    if (warp == 0) {
      int a = 0;
      if (lane < LB) {
        int d = 0;
        for (int g = LB; g < kBatchMaxN; ++g) {
          const int fg = int(hi >> g & 1ull), wg = w[lane * kBatchMaxN + g];
          d += fg ? -wg : wg;
          a += fg ? wg : 0;
        }
        delta[lane] = d;
      }
      int cf = 0;
      for (int g = LB + lane; g < kBatchMaxN; g += 32) {
        const int fg = int(hi >> g & 1ull);
        for (int h = g + 1; h < kBatchMaxN; ++h)
          if (fg != int(hi >> h & 1ull)) cf += w[g * kBatchMaxN + h];
      }
      int tot = a + cf;
      for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
      if (lane == 0) misc[0] = tot;
    }
    __syncthreads();
    const unsigned long long x0 = hi | ((unsigned long long)tid << 5);
    if (x0 >= limit) continue;
    // C at j = 0 and the change of C when each low bit i < 5 is set
    int c0 = misc[0];
    for (int k = 5; k < LB; ++k) {
      const int tk = tid >> (k - 5) & 1;
      if (tk) c0 += delta[k];
      for (int l = k + 1; l < LB; ++l)
        if (tk != (tid >> (l - 5) & 1)) c0 += w[k * kBatchMaxN + l];
    }
    int e[5];
    for (int i = 0; i < 5; ++i) {
      int ai = 0, di = 0;
      for (int k = 5; k < LB; ++k) {
        const int wk = w[i * kBatchMaxN + k];
        di += wk;
        if (tid >> (k - 5) & 1) ai += wk;
      }
      c0 += ai;
      e[i] = delta[i] + di - 2 * ai;
    }
    const int jn = limit - x0 < 32ull ? int(limit - x0) : 32;
    for (int j = 0; j < jn; ++j) {
      int c = c0;
      for (int i = 0; i < 5; ++i)
        if (j >> i & 1) c += e[i];
      for (int i = 0; i < 5; ++i)
        for (int i2 = i + 1; i2 < 5; ++i2)
          if ((j >> i & 1) != (j >> i2 & 1)) c += w[i * kBatchMaxN + i2];
      if (c < ex.vmin) { ex.vmin = c; ex.amin = x0 | j; }
      if (c > ex.vmax) { ex.vmax = c; ex.amax = x0 | j; }
    }
  }
  ext_commit(ex, ered, B, inst);
}

// Super-tiles [u0, u1) of one pass (descriptor staged in shared memory P);
// the pass's partial sums go to `slot`.
template <bool FAST, bool ADJ, int FR>
__device__ __forceinline__ void batch_pass(const BatchArgs& B, const BatchInst& I, int pass, int slot, uint32_t u0,
                                           uint32_t u1, unsigned char* smem, double* wacc, double* red, PassDev& P) {
  const PassMeta& M = B.pmeta[pass];
  const int tid = threadIdx.x;
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(B.passes + pass);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&P);
    const int words = int(offsetof(PassDev, sub) / 4) + B.passes[pass].nsub * int(sizeof(SubDev) / 4);
    for (int i = tid; i < words; i += kBatchThreads) dst[i] = __ldg(src + i);
    __syncthreads();
  }
  const float2* phase = M.layer_c >= 0 ? I.phase + (size_t)M.layer_c * I.ncost : nullptr;
  if constexpr (!ADJ) {
    PassArgs A;
    A.state = I.psi;
    A.out = I.psi;
    A.diag = I.diag;
    A.phase = phase;
    A.wmat = I.wmat;
    A.ctabs = I.ctabs;
    A.partial = nullptr;
    A.bsum = nullptr;
    A.phase_in_smem = 0;
    A.l2hint = 0;
    A.prefetch = 0;
    A.tma_store = 0;
    A.tma_load = 0;
    A.err = nullptr;
    A.dense = 0;
    A.tma_wait_ns = 0;
    A.ext_keys = nullptr;
    constexpr int TILE = padded_size<8>(FR + 5 + kBatchWB);
    float2* tile = reinterpret_cast<float2*>(smem);
    int* tconst = reinterpret_cast<int*>(tile + TILE);
    wacc[tid] = 0.0;
    wacc[kBatchThreads + tid] = 0.0;
    for (uint32_t u = u0; u < u1; ++u) fwd_unit<float, FR, kBatchWB, FAST>(P, A, u, tile, tconst, phase, wacc);
    if (M.reduce) {
      finish_thread_sums<float, kBatchThreads>(wacc, tid);
      __syncthreads();
      double sN, sC;
      reduce_thread_sums<kBatchThreads>(wacc, sN, sC);
      if (tid == 0) {
        B.slots[slot] = sN;
        B.slots[slot + 1] = sC;
      }
    }
  } else {
    AdjArgs A;
    A.psi = I.psi;
    A.psi_store = 1;
    A.lam = I.lam;
    A.diag = I.diag;
    A.phase = phase;
    A.wmat = I.wmat;
    A.ctabs = I.ctabs;
    A.partial = nullptr;
    A.phase_in_smem = 0;
    A.prefetch = 0;
    A.tma_load = 0;
    A.err = nullptr;
    A.tma_wait_ns = 0;
    constexpr int TILE = padded_size<8>(kBatchRAdj + 5 + kBatchWBAdj);
    float2* tv = reinterpret_cast<float2*>(smem);
    float2* tl = tv + TILE;
    int* tconst = reinterpret_cast<int*>(tl + TILE);
    double gA = 0.0, gC = 0.0, gB = 0.0, gE = 0.0;
    for (uint32_t u = u0; u < u1; ++u)
      adj_unit<float, kBatchRAdj, kBatchWBAdj, FAST>(P, A, u, tv, tl, tconst, phase, gA, gC, gB, gE);
    gA = block_sum(gA, red);
    gC = block_sum(gC, red);
    gB = block_sum(gB, red);
    if (tid == 0) {
      B.slots[slot] = gA;
      B.slots[slot + 1] = gC;
      B.slots[slot + 2] = gB;
    }
  }
  __syncthreads();
}

// Forward circuit of a SOLO n = 12 instance (gradient batches) in shared
// memory, written to its state for the adjoint passes; norm, <C> and extremes.
__device__ __noinline__ void batch_solo_small(const BatchArgs& B, const BatchInst& I, int inst, unsigned char* smem,
                                              double* red, Extreme* ered) {
  const int n = I.n, N = 1 << n;
  float2* s = reinterpret_cast<float2*>(smem);
  int* cut = reinterpret_cast<int*>(s + N);
  Extreme ex = ext_empty();
  small_cuts(I, cut, ex);
  ext_commit(ex, ered, B, inst);
  small_forward(I, s, cut);
  double nr = 0.0, ec = 0.0;
  for (int x = threadIdx.x; x < N; x += kBatchThreads) {
    const float2 v = s[x];
    const double pr = double(v.x) * v.x + double(v.y) * v.y;
    nr += pr;
    ec += pr * double(cut[x]);
    __stcg(reinterpret_cast<float2*>(I.psi) + x, v);
  }
  nr = block_sum(nr, red);
  ec = block_sum(ec, red);
  if (threadIdx.x == 0) {
    B.slots[I.slot0] = nr;
    B.slots[I.slot0 + 1] = ec;
  }
  __syncthreads();
}

// One phase of the batch (ADJ: the adjoint sweep). Dynamic shared memory:
// max(forward tile, two adjoint tiles, SMALL state + cuts, EXT weights) + the
// tile constants.
// FR: register bits of the forward tile (5: 5x3 tiles, T = 13; 4: 4x3, T = 12).
template <bool FAST, bool ADJ, int FR>
__global__ void __launch_bounds__(kBatchThreads, 2) batch_kernel(const BatchArgs B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double wacc[2 * kBatchThreads + 2 * kBatchThreads / 32];
  __shared__ double red[kBatchThreads / 32];
  __shared__ Extreme ered[kBatchThreads / 32];
  __shared__ PassDev sP;
  __shared__ unsigned int s_next;
  __shared__ int s_skip;
  const int tid = threadIdx.x;
  if (tid == 0) s_next = atomicAdd(B.head, 1u);
  __syncthreads();
  unsigned int idx = s_next;
  while (idx < (unsigned int)B.nitems) {
    const BatchItem it = B.items[idx];
    // take the following item now; its index is only needed at the end
    unsigned int nxt = 0;
    if (tid == 0) nxt = atomicAdd(B.head, 1u);
    if (tid == 0) {
      int skip = 0;
      if (it.need > 0) {
        const int32_t* d = B.done + it.inst;
        if (ld_acquire(d) < it.need) {
          const unsigned long long t0 = global_ns();
          while (ld_acquire(d) < it.need) {
            __nanosleep(200);
            if (global_ns() - t0 > B.wait_ns) {
              atomicExch(B.error, 1);
              skip = 1;
              break;
            }
          }
        }
      }
      s_skip = skip;
    }
    __syncthreads();
    const BatchInst& I = B.insts[it.inst];
    if (!s_skip) {
      if (it.kind == BITEM_PASS || it.kind == BITEM_SOLO) {
        // a PASS item is a unit range of one pass; a SOLO item is every pass of
        // this phase of its instance, in order (one call site for both)
        int p0 = it.pass, p1 = it.pass + 1;
        if (it.kind == BITEM_SOLO) {
          if (!ADJ && I.fwd_npass == 0) batch_solo_small(B, I, it.inst, smem_raw, red, ered);
          p0 = ADJ ? I.adj_pass0 : I.fwd_pass0;
          p1 = p0 + (ADJ ? I.adj_npass : I.fwd_npass);
        }
        for (int pi = p0; pi < p1; ++pi) {
          const bool whole = it.kind == BITEM_SOLO;
          batch_pass<FAST, ADJ, FR>(B, I, pi, whole ? B.pmeta[pi].slot0 : it.slot, whole ? 0u : it.u0,
                                whole ? (uint32_t)B.passes[pi].n_units : it.u1, smem_raw, wacc, red, sP);
        }
      } else if constexpr (!ADJ) {
        if (it.kind == BITEM_SMALL) batch_small(B, I, it.inst, smem_raw, red, ered);
        else batch_ext(B, I, it.inst, it.u0, it.u1, smem_raw, ered);
      }
    }
    __syncthreads();  // every thread's writes of this item precede the release below
    if (tid == 0) {
      if (it.kind == BITEM_PASS) red_release_add(B.done + it.inst, 1);
      s_next = nxt;
    }
    __syncthreads();
    idx = s_next;
  }
}

// Per instance: <C>, norm, r from the slots and extremes; layer gradients from
// the adjoint slots (g_beta: -2 sum Im <l|X|psi>; g_gamma: 2 s sum Im <l|h psi>)
// and the chain rule through gamma_k = (k+1)/p dgamma, beta_k = (1 - k/p) dbeta.
// out[i * 9 + ...] = {<C>, r, norm, C_min, C_max, argmin, argmax, d/d dgamma, d/d dbeta}.
__global__ void batch_finalize_kernel(const BatchArgs B, int count, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const BatchInst& I = B.insts[i];
  double nr = 0.0, ec = 0.0;
  if (I.fwd_npass == 0) {
    nr = B.slots[I.slot0];
    ec = B.slots[I.slot0 + 1];
  } else {
    const PassMeta& M = B.pmeta[I.fwd_pass0 + I.fwd_npass - 1];
    for (int k = 0; k < M.nitems; ++k) {
      nr += B.slots[M.slot0 + 2 * k];
      ec += B.slots[M.slot0 + 2 * k + 1];
    }
  }
  const unsigned long long km = B.ext_min[i], kx = B.ext_max[i];
  const long long cmin = (long long)(km >> 32) - (1ll << 31);
  const long long cmax = (long long)(kx >> 32) - (1ll << 31);
  const unsigned long long amin = km & 0xffffffffull, amax = 0xffffffffull - (kx & 0xffffffffull);
  const double den = double(cmax - cmin);
  double* o = out + (size_t)i * 9;
  o[0] = ec;
  o[1] = den != 0.0 ? (ec - double(cmin)) / den : 1.0;
  o[2] = nr;
  o[3] = double(cmin);
  o[4] = double(cmax);
  o[5] = double(amin);
  o[6] = double(amax);
  o[7] = 0.0;
  o[8] = 0.0;
  if (!I.with_grad) return;
  double* gg = B.grads + I.g_off;  // g_gamma[p] | g_beta[p]
  const int p = I.p;
  if (I.adj_npass > 0) {
    for (int k = 0; k < 2 * p; ++k) gg[k] = 0.0;
    for (int j = 0; j < I.adj_npass; ++j) {
      const PassMeta& M = B.pmeta[I.adj_pass0 + j];
      double a = 0.0, c = 0.0, b = 0.0;
      for (int k = 0; k < M.nitems; ++k) {
        a += B.slots[M.slot0 + 3 * k];
        c += B.slots[M.slot0 + 3 * k + 1];
        b += B.slots[M.slot0 + 3 * k + 2];
      }
      if (M.layer_a >= 0) gg[p + M.layer_a] += -2.0 * a;
      if (M.layer_c >= 0) gg[M.layer_c] += 2.0 * I.scale * c;
      if (M.layer_b >= 0) gg[p + M.layer_b] += -2.0 * b;
    }
  }
  double sg = 0.0, sb = 0.0;
  for (int k = 0; k < p; ++k) {
    sg += double(k + 1) / p * gg[k];
    sb += (1.0 - double(k) / p) * gg[p + k];
  }
  o[7] = sg;
  o[8] = sb;
}

}  // namespace qaoa
