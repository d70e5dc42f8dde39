// pass_kernel.cuh -- the fused forward pass kernel of the LR-QAOA simulation.
//
// One launch = one HBM pass over the state (see plan.h). For every super-tile
// the CTA runs the sub-passes of the pass; a sub-pass moves 2^T-amplitude
// tiles global -> registers -> (shared memory -> registers)* -> global, and in
// each round applies, on the thread's 2^R register amplitudes:
//   mixer of layer a   exp(+i beta_a X_q) on the round's target bits (Eq. UB)
//   cost phase         exp(-i gamma_c s h(x)), h = W - 2 C(x)  (Eqs. H_C, UC)
//   mixer of layer b   on the round's target bits
//   reduction          |psi_x|^2 and |psi_x|^2 C(x) (final pass)
// The mixer rotation [[c, i s], [i s, c]] is applied as c * [[1, i t], [i t, 1]]
// (t = tan beta) so each butterfly costs four FMAs; the accumulated factor c^k
// is folded into one multiply before the store ("fast" form). Angles with
// |tan beta| > 1 use the plain form.
//
// Rounds are compiled once per entry of the planner's layout menu
// (menu_layout in plan.h), so register bit positions are constants: shared
// memory offsets become immediates through the additive padded layout `padi`,
// and global offsets are walked in Gray-code order (one XOR per amplitude).
#pragma once
#include <cuda.h>

#include <type_traits>

#include "device.cuh"

namespace qaoa {

enum : uint8_t { SRC_SMEM_D = 0, SRC_GLOBAL_D = 1, SRC_INIT_D = 2 };
enum : uint8_t { DST_SMEM_D = 0, DST_GLOBAL_D = 1 };

struct PassArgs {
  void* state;            // 2^n amplitudes, interleaved (re, im): the pass's input
  void* out;              // where the pass writes its output: `state` (in place) or,
                          // for a pass of one sub-pass, another 2^n buffer (the
                          // gradient's stored forward states)
  const int32_t* diag;    // int32 C(x) for all x (stream mode) or nullptr
  const void* phase;      // phase table of the cost layer: ncost complex entries
  const int32_t* wmat;    // n x n symmetric integer weights
  const int32_t* ctabs;   // per-round cost tables (recompute mode)
  double* partial;        // per-CTA [norm, <C>] partial sums (final pass)
  double* bsum;           // sampling block sums (2^12 consecutive amplitudes) written by
                          // the final pass when its tiles are index-contiguous, or nullptr
  int phase_in_smem;      // copy the phase table into shared memory
  int l2hint;             // L2 priorities: keep sub-pass outputs that are read back
  int prefetch;           // prefetch the CTA's next tile into L2 while this one runs
                          // (passes of one tile per super-tile that load the state):
                          // 1 one line per 16-amplitude run from every thread, 2 one
                          // tensor prefetch of the whole tile (tmap) from one thread
  int tma_store;          // the final round writes the tile densely into shared memory
                          // and one thread stores it with a tensor store (PassTma)
  int tma_load;           // complex64, one tile per super-tile: the CTA's next tile is
                          // loaded into shared memory by one tensor load (PassTma.tmap),
                          // issued by the last warp to read the current tile's last
                          // round, and the first round reads it from there
  unsigned long long* err;  // error word: bit 0 set when a tensor-load wait gave up
  unsigned long long tma_wait_ns;  // limit of one tensor-load wait (ns)
  int dense;              // complex64, one tile per super-tile, no round in menu layout 2:
                          // shared-memory rounds use dense tile-index slots (1), and
                          // with tensor tile loads and a first round without tile
                          // constants the tile's first barrier is dropped (2)
  // exhaustive extremes in the |+> round (every index visited once): packed
  // keys [(C - c_lo) << 34 | x, (c_hi - C) << 34 | x], each the minimum over
  // all x (smallest C, resp. largest C, then smallest index); must hold ~0 on
  // entry; nullptr: not computed in this pass
  unsigned long long* ext_keys;
};

// Tensor maps of a pass kernel (a separate kernel parameter, so that the
// persistent batch kernel, which builds its PassArgs locally, carries none):
// the pass's input state (tmap: next-tile prefetch, PassArgs.prefetch == 2) and
// output state (smap: tensor stores, PassArgs.tma_store) as tensors of tdims <=
// 5 dimensions over runs of index bits (dimension d: bits tbit[d] .. tbit[d] +
// tlen[d] - 1, inside the tile when bit d of ttile is set), the box one tile;
// the coordinates of a tile are its outer index bits.
struct PassTma {
  CUtensorMap tmap;  // 128-byte aligned by its type
  CUtensorMap smap;
  int tdims;
  int pfdist;        // prefetch distance in the CTA's tiles (1..4; 0: no L2 prefetches,
                     // the map serving the tensor tile loads only)
  int8_t tbit[5], tlen[5];
  uint8_t ttile;
};

// Compile-time copy of the planner's layout menu (plan.cpp, menu_layout).
template <int R, int WB, int L>
struct Lay {
  static constexpr int T = R + 5 + WB;
  __host__ __device__ static constexpr int reg(int i) {
    return L == 0 ? 5 + i : L == 1 ? T - R + i : L == 2 ? i : L == 3 ? (i == 0 ? 4 : T - R + i)
                                                                      : (i == 0 ? 0 : T - R + i);
  }
  __host__ __device__ static constexpr int lane(int i) {
    return L == 2 ? R + i : L == 4 ? 1 + i : (L == 3 && i == 4) ? T - R : i;
  }
  __host__ __device__ static constexpr int warp(int i) {
    return L == 0 ? 5 + R + i : L == 2 ? R + 5 + i : L == 4 ? 6 + i : 5 + i;
  }
  // tile-index offset of register amplitude j
  __host__ __device__ static constexpr uint32_t toff(int j) {
    uint32_t o = 0;
    for (int i = 0; i < R; ++i)
      if (j >> i & 1) o |= 1u << reg(i);
    return o;
  }
};

// warps per CTA of a shape
template <int WB>
constexpr int NT32 = 1 << WB;

// Layout id of a round signature (plan.h, round_sig: bits 0-1 and 18).
__host__ __device__ constexpr int sig_layout(uint32_t sig) { return int(sig & 3u) | int(sig >> 18 & 1u) << 2; }

// Tile bits above the 2^12-amplitude sampling block (0 for T <= 12, at most 2).
template <int R, int WB>
constexpr int kBlkBits = R + 5 + WB > 12 ? R + 5 + WB - 12 : 0;

// Tile bit held by register (kind 0), lane (1) or warp (2) position i of a
// round: a compile-time constant of the layout for a specialised round
// (SIG != 0), else read from the round descriptor.
template <int R, int WB, uint32_t SIG>
__device__ __forceinline__ int tile_bit(const RoundDev& rd, int kind, int i) {
  if constexpr (SIG != 0) {
    constexpr int L = sig_layout(SIG);
    return kind == 0 ? Lay<R, WB, L>::reg(i) : kind == 1 ? Lay<R, WB, L>::lane(i) : Lay<R, WB, L>::warp(i);
  } else {
    return kind == 0 ? rd.reg[i] : kind == 1 ? rd.lane[i] : rd.warp[i];
  }
}

__host__ __device__ constexpr int ctz_c(int k) {
  int b = 0;
  while (!(k >> b & 1)) ++b;
  return b;
}

template <typename Real>
__device__ __forceinline__ void bfly(typename Cx<Real>::T& a, typename Cx<Real>::T& b, Real tau, Real alpha,
                                     bool fast) {
  const Real ar = a.x, ai = a.y, br = b.x, bi = b.y;
  if (fast) {
    a.x = fma(-tau, bi, ar);
    a.y = fma(tau, br, ai);
    b.x = fma(-tau, ai, br);
    b.y = fma(tau, ar, bi);
  } else {
    a.x = fma(alpha, ar, -tau * bi);
    a.y = fma(alpha, ai, tau * br);
    b.x = fma(alpha, br, -tau * ai);
    b.y = fma(alpha, bi, tau * ar);
  }
}

// Butterflies on the register bits in `mask`. The all-bits case is straight-line
// code: a branch per bit would make the compiler restore the registers' roles
// after every bit (a move per amplitude per bit).
template <int R, typename V, typename Real>
__device__ __forceinline__ void apply_mixer(V* v, uint8_t mask, Real tau, Real alpha, bool fast) {
  if (mask == (1u << R) - 1) {
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int j = 0; j < (1 << R); ++j)
        if (!(j >> i & 1)) bfly<Real>(v[j], v[j | (1 << i)], tau, alpha, fast);
    return;
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    if (mask >> i & 1) {
#pragma unroll
      for (int j = 0; j < (1 << R); ++j)
        if (!(j >> i & 1)) bfly<Real>(v[j], v[j | (1 << i)], tau, alpha, fast);
    }
  }
}

// ---------------------------------------------------------------------------
// Swapped storage (complex64). Between the passes of a run, the amplitude of
// index x is held as (re, im) when x has an even number of set bits and as
// (im, re) when it has an odd number. A butterfly on any bit pairs one plain
// amplitude a with one swapped amplitude b~ = (b.y, b.x), and the rotation
// a' = a + i t b, b' = b + i t a becomes two packed FMAs (fma.rn.f32x2, one
// issue slot for two FP32 FMAs) with no register moves:
//   a'  = a  + (-t,  t) * b~,      b~' = b~ + ( t, -t) * a
// (the same FP32 operations as the plain form, so the results are identical).
// In a round, register amplitude j of a thread is swapped when parity(j) xor s,
// s being the parity of the thread's amplitude 0 (tile base and the thread's
// lane / warp offset). The first forward pass writes this form; the last
// forward sub-pass writes plain amplitudes (st_plain); the adjoint's first
// sub-pass reads plain ones (ld_plain). complex128 kernels keep plain storage.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int parity_c(int j) { return __builtin_popcount(unsigned(j)) & 1; }

// Butterflies on the register bits in `mask` of swapped-storage amplitudes.
// kp = (-tau, tau) for a thread with s = 0, (tau, -tau) for s = 1 (the
// coefficient of the update of a parity-0 amplitude), kn = -kp; fast form
// a' = a + i tau b, else a' = alpha a + i tau b.
template <int R>
__device__ __forceinline__ void bfly_sw(float2& a, float2& b, float2 ca, float2 cb, float2 al, bool fast) {
  const float2 a0 = a, b0 = b;
  if (fast) {
    a = __ffma2_rn(ca, b0, a0);
    b = __ffma2_rn(cb, a0, b0);
  } else {
    a = __ffma2_rn(al, a0, __fmul2_rn(ca, b0));
    b = __ffma2_rn(al, b0, __fmul2_rn(cb, a0));
  }
}
template <int R>
__device__ __forceinline__ void apply_mixer_sw(float2* v, uint8_t mask, float tau, float alpha, bool fast, int s) {
  if (!mask) return;
  const float2 kp = s ? make_float2(tau, -tau) : make_float2(-tau, tau);
  const float2 kn = make_float2(-kp.x, -kp.y);
  const float2 al = make_float2(alpha, alpha);
  auto bit = [&](int i) {
#pragma unroll
    for (int j = 0; j < (1 << R); ++j)
      if (!(j >> i & 1)) {
        if (parity_c(j) == 0) bfly_sw<R>(v[j], v[j | (1 << i)], kp, kn, al, fast);
        else bfly_sw<R>(v[j], v[j | (1 << i)], kn, kp, al, fast);
      }
  };
  if (mask == (1u << R) - 1) {
#pragma unroll
    for (int i = 0; i < R; ++i) bit(i);
    return;
  }
#pragma unroll
  for (int i = 0; i < R; ++i)
    if (mask >> i & 1) bit(i);
}

// Exchanges the components of the register amplitudes stored swapped (plain
// <-> swapped storage at the edges of a run).
template <int R>
__device__ __forceinline__ void swap_odd(float2* v, int s) {
#pragma unroll
  for (int j = 0; j < (1 << R); ++j)
    if (parity_c(j) ^ s) v[j] = make_float2(v[j].y, v[j].x);
}

// L2 prefetch of one box of a tensor (cp.async.bulk.prefetch.tensor): tmap is a
// kernel parameter (grid constant) holding a tensor map, c the box's
// coordinates (innermost first); dims 1..5.
__device__ __forceinline__ void tma_prefetch_l2(const CUtensorMap* tmap, int dims, const int32_t* c) {
  const uint64_t t = reinterpret_cast<uint64_t>(tmap);
  switch (dims) {
    case 1:
      asm volatile("cp.async.bulk.prefetch.tensor.1d.L2.global.tile [%0, {%1}];" ::"l"(t), "r"(c[0]) : "memory");
      break;
    case 2:
      asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(t), "r"(c[0]), "r"(c[1])
                   : "memory");
      break;
    case 3:
      asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(t), "r"(c[0]),
                   "r"(c[1]), "r"(c[2])
                   : "memory");
      break;
    case 4:
      asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];" ::"l"(t), "r"(c[0]),
                   "r"(c[1]), "r"(c[2]), "r"(c[3])
                   : "memory");
      break;
    default:
      asm volatile("cp.async.bulk.prefetch.tensor.5d.L2.global.tile [%0, {%1, %2, %3, %4, %5}];" ::"l"(t),
                   "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4])
                   : "memory");
      break;
  }
}

// Tensor store of one box from shared memory (cp.async.bulk.tensor, bulk
// group): tmap a grid-constant tensor map, c the box's coordinates, smem the
// 128-byte aligned shared-memory address of the dense box.
__device__ __forceinline__ void tma_store_box(const CUtensorMap* tmap, int dims, const int32_t* c, uint32_t smem) {
  const uint64_t t = reinterpret_cast<uint64_t>(tmap);
  switch (dims) {
    case 1:
      asm volatile("cp.async.bulk.tensor.1d.global.shared::cta.bulk_group [%0, {%1}], [%2];" ::"l"(t), "r"(c[0]),
                   "r"(smem)
                   : "memory");
      break;
    case 2:
      asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(t), "r"(c[0]),
                   "r"(c[1]), "r"(smem)
                   : "memory");
      break;
    case 3:
      asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(t),
                   "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(smem)
                   : "memory");
      break;
    case 4:
      asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(t),
                   "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(smem)
                   : "memory");
      break;
    default:
      asm volatile("cp.async.bulk.tensor.5d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4, %5}], [%6];" ::"l"(t),
                   "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]), "r"(smem)
                   : "memory");
      break;
  }
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Waits until the committed tensor stores have read their shared memory
// (read) or completed (all).
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Makes this thread's shared-memory writes visible to the tensor engine.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Tensor loads of whole tiles into shared memory, completed on a shared-memory
// mbarrier (transaction bytes), and the named barrier that frees the tile
// buffer for them.
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for phase `parity` of the mbarrier, at most limit_ns: false when it
// gave up. A limit below 1 us means one non-blocking test (a suspended
// try_wait could outlast it).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, unsigned long long limit_ns) {
  if (mbar_test_wait(bar, parity)) return true;
  if (limit_ns < 1000ull) return false;
  const unsigned long long t0 = timer_ns();
  while (!mbar_try_wait(bar, parity))
    if (timer_ns() - t0 > limit_ns) return false;
  return true;
}
// Tensor load of one box (coordinates c, innermost first) into shared memory
// at smem (128-byte aligned); its bytes complete the mbarrier's transaction.
__device__ __forceinline__ void tma_load_box(const CUtensorMap* tmap, int dims, const int32_t* c, uint32_t smem,
                                             uint32_t bar) {
  const uint64_t t = reinterpret_cast<uint64_t>(tmap);
  switch (dims) {
    case 1:
      asm volatile(
          "cp.async.bulk.tensor.1d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2}], [%3];" ::"r"(
              smem),
          "l"(t), "r"(c[0]), "r"(bar)
          : "memory");
      break;
    case 2:
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
          "[%4];" ::"r"(smem),
          "l"(t), "r"(c[0]), "r"(c[1]), "r"(bar)
          : "memory");
      break;
    case 3:
      asm volatile(
          "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
          "[%5];" ::"r"(smem),
          "l"(t), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(bar)
          : "memory");
      break;
    case 4:
      asm volatile(
          "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
          "%5}], [%6];" ::"r"(smem),
          "l"(t), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(bar)
          : "memory");
      break;
    default:
      asm volatile(
          "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
          "%5, %6}], [%7];" ::"r"(smem),
          "l"(t), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]), "r"(bar)
          : "memory");
      break;
  }
}
// Count of the warps that have read the current tile's last round (the word
// at tbar + 12): returns the count before this warp's increment.
__device__ __forceinline__ uint32_t tile_read_count_add(uint32_t tbar) {
  uint32_t prev;
  asm volatile("atom.shared.add.u32 %0, [%1], 1;" : "=r"(prev) : "r"(tbar + 12) : "memory");
  return prev;
}
__device__ __forceinline__ void tile_read_count_reset(uint32_t tbar) {
  asm volatile("st.volatile.shared.u32 [%0], %1;" ::"r"(tbar + 12), "r"(0u) : "memory");
}
// Default limit of one wait for a tensor tile load (ns; PassArgs.tma_wait_ns).
// A wait that gives up sets the error word and the CTA's stop word (at tbar +
// 8, after the mbarrier: 1 + the parity of the phase it gave up on): the CTA
// then issues no further tensor loads and waits for none, and before it ends
// waits (bounded by this default) for the load it gave up on, so that no copy
// is left in flight into its shared memory; the pass's output is invalid.
constexpr unsigned long long kTmaWaitNs = 2000000000ull;
__device__ __forceinline__ uint32_t tma_stop_word(uint32_t tbar) {
  uint32_t f;
  asm volatile("ld.volatile.shared.u32 %0, [%1];" : "=r"(f) : "r"(tbar + 8) : "memory");
  return f;
}
__device__ __forceinline__ bool tma_stopped(uint32_t tbar) { return tma_stop_word(tbar) != 0; }
__device__ __forceinline__ void tma_stop(uint32_t tbar, uint32_t parity) {
  asm volatile("st.volatile.shared.u32 [%0], %1;" ::"r"(tbar + 8), "r"(1u + parity) : "memory");
}

// Dense (unpadded) view of a tile's shared memory, 128-byte aligned: the box
// of a tensor store. The padded tile is at least 127 bytes larger than the
// dense one for every shape, so the view fits inside it.
template <typename C2>
__device__ __forceinline__ C2* dense_tile(C2* tile) {
  return reinterpret_cast<C2*>((reinterpret_cast<uintptr_t>(tile) + 127) & ~uintptr_t(127));
}

// Tensor coordinates of the tile at global index base (outer dimensions from
// its bits, tile dimensions 0).
__device__ __forceinline__ void tile_coords(const PassTma& M, uint64_t base, int32_t* c) {
#pragma unroll
  for (int d = 0; d < 5; ++d)
    c[d] = (d < M.tdims && !(M.ttile >> d & 1)) ? int32_t(base >> M.tbit[d] & ((1ull << M.tlen[d]) - 1)) : 0;
}

// Per-round thread geometry: the padded shared-memory slot of the thread's
// amplitude 0 and its global index (tile base | the thread's lane and warp
// bits), both read from the round's host-built table (one entry per thread),
// and the global strides of the register bits.
template <int R, int WB, int AB>
struct RoundGeo {
  uint32_t sbase;
  uint64_t gb;
  uint64_t gstr[R];
  __device__ __forceinline__ RoundGeo(const SubDev& sp, const RoundDev& rd, uint64_t gbase, int lane, int warp,
                                      const int32_t* tabs) {
    const int tid = (warp << 5) | lane;
    sbase = (uint32_t)__ldg(tabs + rd.gtab + tid) & 0x7fffffffu;
    gb = gbase | __ldg(reinterpret_cast<const unsigned long long*>(tabs + rd.gtab + (32 << WB)) + tid);
#pragma unroll
    for (int i = 0; i < R; ++i) gstr[i] = 1ull << rd.greg[i];
  }
  __device__ __forceinline__ static uint32_t sbase_of(const RoundDev& rd, int lane, int warp, const int32_t* tabs) {
    return (uint32_t)__ldg(tabs + rd.gtab + ((warp << 5) | lane)) & 0x7fffffffu;
  }
  // slot and the parity of the thread's global index offset (bit 31 of the entry)
  __device__ __forceinline__ static uint32_t entry_of(const RoundDev& rd, int lane, int warp, const int32_t* tabs) {
    return (uint32_t)__ldg(tabs + rd.gtab + ((warp << 5) | lane));
  }
};

// Calls f(j, global index of register amplitude j) for j in Gray-code order.
template <int R, typename F>
__device__ __forceinline__ void gray_walk(uint64_t g0, const uint64_t* gstr, F&& f) {
  uint64_t g = g0;
#pragma unroll
  for (int k = 0; k < (1 << R); ++k) {
    if (k) g ^= gstr[ctz_c(k)];
    f(k ^ (k >> 1), g);
  }
}

// Calls f(j, pointer to register amplitude j) for j in Gray-code order. Step k
// flips bit ctz(k) of j; whether it turns on or off is known at compile time,
// so the pointer moves by +-stride with one 64-bit add.
template <int R, typename T, typename F>
__device__ __forceinline__ void gray_ptr_walk(T* base, uint64_t g0, const uint64_t* gstr, F&& f) {
  T* q = base + g0;
#pragma unroll
  for (int k = 0; k < (1 << R); ++k) {
    if (k) {
      const int b = ctz_c(k);
      const int j = k ^ (k >> 1);
      if (j >> b & 1) q += gstr[b]; else q -= gstr[b];
    }
    f(k ^ (k >> 1), q);
  }
}

// As gray_ptr_walk over register bits 1..R-1 only: f(j, pointer to register
// amplitude j) for the even j (register bit 0 clear), whose partner j | 1 is
// the next amplitude in memory (register bit 0 on index bit 0).
template <int R, typename T, typename F>
__device__ __forceinline__ void gray_ptr_walk_pairs(T* base, uint64_t g0, const uint64_t* gstr, F&& f) {
  T* q = base + g0;
#pragma unroll
  for (int k = 0; k < (1 << (R - 1)); ++k) {
    if (k) {
      const int b = ctz_c(k);
      const int j = k ^ (k >> 1);
      if (j >> b & 1) q += gstr[b + 1]; else q -= gstr[b + 1];
    }
    f((k ^ (k >> 1)) << 1, q);
  }
}

// Two adjacent complex64 amplitudes in one 16-byte access (the address is
// 16-byte aligned: the first has index bit 0 clear). The complex128 forms are
// never called (the paired layout is complex64 only).
__device__ __forceinline__ void load_pair(const float2* q, float2& a, float2& b) {
  const float4 t = __ldcg(reinterpret_cast<const float4*>(q));
  a = make_float2(t.x, t.y);
  b = make_float2(t.z, t.w);
}
__device__ __forceinline__ void store_pair(float2* q, const float2& a, const float2& b) {
  __stcg(reinterpret_cast<float4*>(q), make_float4(a.x, a.y, b.x, b.y));
}
__device__ __forceinline__ void load_pair(const double2* q, double2& a, double2& b) { a = __ldcg(q); b = __ldcg(q + 1); }
__device__ __forceinline__ void store_pair(double2* q, const double2& a, const double2& b) {
  __stcg(q, a);
  __stcg(q + 1, b);
}

// Issues the asynchronous copy of one vector's tile (complex64, global indices
// gbase | scatter(t) for tile index t) into its padded shared-memory tile:
// thread (lane, warp) copies the amplitudes at tile indices
// lane | warp << 5 | k << (5 + WB) for the 2^R values of k, 8 bytes each
// (lanes on tile bits 0..4, i.e. global bits 0..4: 256-byte runs per warp).
// Its slot and global offset come from the sub-pass's copy-geometry table.
template <int R, int WB>
__device__ __forceinline__ void tile_copy_async(float2* tile, const float2* g, uint64_t gbase, const SubDev& sp,
                                                int tid, const int32_t* tabs) {
  constexpr int NT = 32 << WB;
  const uint32_t sb = (uint32_t)__ldg(tabs + sp.cgtab + tid) & 0x7fffffffu;
  const uint64_t gb = gbase | __ldg(reinterpret_cast<const unsigned long long*>(tabs + sp.cgtab + NT) + tid);
  uint64_t gstr[R];
#pragma unroll
  for (int i = 0; i < R; ++i) gstr[i] = 1ull << sp.pos[5 + WB + i];
  gray_ptr_walk<R>(g, gb, gstr, [&](int k, const float2* q) {
    cp_async8(tile + sb + padi<8>(uint32_t(k) << (5 + WB)), q);
  });
}

// Shared-memory loads / stores of the register amplitudes: the only code that
// depends on the layout, compiled with constant offsets per menu entry.
template <int R, int WB, int L, int AB, typename C2>
__device__ __forceinline__ void smem_load_l(const C2* tile, uint32_t sbase, C2* v) {
#pragma unroll
  for (int j = 0; j < (1 << R); ++j) v[j] = tile[sbase + padi<AB>(Lay<R, WB, L>::toff(j))];
}
template <int R, int WB, int L, int AB, typename C2>
__device__ __forceinline__ void smem_store_l(C2* tile, uint32_t sbase, const C2* v) {
#pragma unroll
  for (int j = 0; j < (1 << R); ++j) tile[sbase + padi<AB>(Lay<R, WB, L>::toff(j))] = v[j];
}
// Dense variant (PassArgs.dense): slots in tile-index order without padding,
// the tensor box's order, for passes none of whose rounds puts its lanes above
// tile bit 5 (menu layout 2): with lanes on tile bits 0..3 (8-byte accesses)
// or 1..3 and register bit 0 on tile bit 0 (16-byte accesses of a pair) every
// access is bank-conflict free. dense: the 128-byte aligned tile.
template <int R, int WB, int L>
__device__ __forceinline__ uint32_t dense_base(int lane, int warp) {
  uint32_t b = 0;
#pragma unroll
  for (int i = 0; i < 5; ++i) b |= uint32_t(lane >> i & 1) << Lay<R, WB, L>::lane(i);
#pragma unroll
  for (int i = 0; i < WB; ++i) b |= uint32_t(warp >> i & 1) << Lay<R, WB, L>::warp(i);
  return b;
}
template <int R, int WB, int L>
__device__ __forceinline__ void smem_load_dense_l(const float2* dense, int lane, int warp, float2* v) {
  const uint32_t b = dense_base<R, WB, L>(lane, warp);
  if constexpr (L == 4) {
#pragma unroll
    for (int j = 0; j < (1 << R); j += 2) {
      const float4 q = *reinterpret_cast<const float4*>(dense + b + Lay<R, WB, L>::toff(j));
      v[j] = make_float2(q.x, q.y);
      v[j | 1] = make_float2(q.z, q.w);
    }
  } else {
#pragma unroll
    for (int j = 0; j < (1 << R); ++j) v[j] = dense[b + Lay<R, WB, L>::toff(j)];
  }
}
template <int R, int WB, int L>
__device__ __forceinline__ void smem_store_dense_l(float2* dense, int lane, int warp, const float2* v) {
  const uint32_t b = dense_base<R, WB, L>(lane, warp);
  if constexpr (L == 4) {
#pragma unroll
    for (int j = 0; j < (1 << R); j += 2)
      *reinterpret_cast<float4*>(dense + b + Lay<R, WB, L>::toff(j)) = make_float4(v[j].x, v[j].y, v[j | 1].x, v[j | 1].y);
  } else {
#pragma unroll
    for (int j = 0; j < (1 << R); ++j) dense[b + Lay<R, WB, L>::toff(j)] = v[j];
  }
}
template <int R, int WB>
__device__ __forceinline__ void smem_load_dense(int layout, const float2* dense, int lane, int warp, float2* v) {
  switch (layout) {
    case 0: smem_load_dense_l<R, WB, 0>(dense, lane, warp, v); break;
    case 1: smem_load_dense_l<R, WB, 1>(dense, lane, warp, v); break;
    case 2: smem_load_dense_l<R, WB, 2>(dense, lane, warp, v); break;
    case 3: smem_load_dense_l<R, WB, 3>(dense, lane, warp, v); break;
    default: smem_load_dense_l<R, WB, 4>(dense, lane, warp, v); break;
  }
}
template <int R, int WB>
__device__ __forceinline__ void smem_store_dense(int layout, float2* dense, int lane, int warp, const float2* v) {
  switch (layout) {
    case 0: smem_store_dense_l<R, WB, 0>(dense, lane, warp, v); break;
    case 1: smem_store_dense_l<R, WB, 1>(dense, lane, warp, v); break;
    case 2: smem_store_dense_l<R, WB, 2>(dense, lane, warp, v); break;
    case 3: smem_store_dense_l<R, WB, 3>(dense, lane, warp, v); break;
    default: smem_store_dense_l<R, WB, 4>(dense, lane, warp, v); break;
  }
}

template <int R, int WB, int AB, typename C2>
__device__ __forceinline__ void smem_load(int layout, const C2* tile, uint32_t sbase, C2* v) {
  switch (layout) {
    case 0: smem_load_l<R, WB, 0, AB>(tile, sbase, v); break;
    case 1: smem_load_l<R, WB, 1, AB>(tile, sbase, v); break;
    case 2: smem_load_l<R, WB, 2, AB>(tile, sbase, v); break;
    case 3: smem_load_l<R, WB, 3, AB>(tile, sbase, v); break;
    default: smem_load_l<R, WB, 4, AB>(tile, sbase, v); break;
  }
}
template <int R, int WB, int AB, typename C2>
__device__ __forceinline__ void smem_store(int layout, C2* tile, uint32_t sbase, const C2* v) {
  switch (layout) {
    case 0: smem_store_l<R, WB, 0, AB>(tile, sbase, v); break;
    case 1: smem_store_l<R, WB, 1, AB>(tile, sbase, v); break;
    case 2: smem_store_l<R, WB, 2, AB>(tile, sbase, v); break;
    case 3: smem_store_l<R, WB, 3, AB>(tile, sbase, v); break;
    default: smem_store_l<R, WB, 4, AB>(tile, sbase, v); break;
  }
}

// Double-float accumulation (complex64 reductions): a value is held as the
// unevaluated sum hi + lo of two floats, and a float is added with Knuth's
// TwoSum, which yields the rounded sum s and its exact rounding error e
// (s + e == a + b), so hi keeps the rounded running sum and lo collects the
// errors. This keeps about 48 bits of the sum on the FP32 pipe: the FP64 pipe
// issues two operations per SM per clock on this part, which made the final
// pass's per-tile FP64 sums a sixth of its time.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}
__device__ __forceinline__ void df_add(float2& acc, float x) {
  float s, e;
  two_sum(acc.x, x, s, e);
  acc.x = s;
  acc.y += e;
}
__device__ __forceinline__ void df_add(float2& acc, float2 y) {
  float s, e;
  two_sum(acc.x, y.x, s, e);
  acc.x = s;
  acc.y += e + y.y;
}
// complex64: thread tid's [norm, <C>] running sums are double-float pairs in
// the memory of wacc[tid], wacc[NT + tid] during the passes; this turns them
// into the FP64 values reduce_thread_sums reads (each thread its own).
template <typename Real, int NT>
__device__ __forceinline__ void finish_thread_sums(double* wacc, int tid) {
  if constexpr (sizeof(Real) == 4) {
    const float2 a = reinterpret_cast<const float2*>(wacc)[tid];
    const float2 b = reinterpret_cast<const float2*>(wacc)[NT + tid];
    wacc[tid] = double(a.x) + double(a.y);
    wacc[NT + tid] = double(b.x) + double(b.y);
  }
}

// CTA total of the per-thread FP64 [norm, <C>] sums in wacc (fixed order: each
// lane of warp 0 adds a strided set, then a shuffle tree); valid in thread 0.
// A barrier must precede the call.
template <int NT>
__device__ __forceinline__ void reduce_thread_sums(const double* wacc, double& sN, double& sC) {
  sN = 0.0;
  sC = 0.0;
  if (threadIdx.x < 32) {
    for (int t = threadIdx.x; t < NT; t += 32) { sN += wacc[t]; sC += wacc[NT + t]; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sN += __shfl_xor_sync(0xffffffffu, sN, o);
      sC += __shfl_xor_sync(0xffffffffu, sC, o);
    }
  }
}

// One round. For a round whose source is global memory, v already holds the
// loaded amplitudes (issued before the tile's barrier). Reduction partials:
// wacc[t], wacc[NT + t] hold thread t's running [norm, <C>] sums;
// wacc[(2 + h) NT + t] thread t's partial of sampling block h of the tile.
// CC: the kernel contains the C(x) code (cost phase, |+> initialisation and
// reductions); passes without any of them run an instantiation without it
// (smaller code, measured faster).
// Operations of a round: compile-time constants taken from a round signature
// (SIG != 0, plan.h round_sig: the specialised pass kernels) or the round
// descriptor's fields read at run time (SIG == 0, the generic kernels).
template <uint32_t SIG>
struct RoundOps {
  static constexpr bool kConst = SIG != 0;
  int layout, src;
  bool dstg, cost, reduce, lam;
  uint8_t mixA, mixB;
  __device__ __forceinline__ explicit RoundOps(const RoundDev& rd)
      : layout(kConst ? sig_layout(SIG) : int(rd.layout)),
        src(kConst ? int(SIG >> 2 & 3u) : int(rd.src)),
        dstg(kConst ? bool(SIG >> 4 & 1u) : rd.dst == DST_GLOBAL_D),
        cost(kConst ? bool(SIG >> 5 & 1u) : rd.cost != 0),
        reduce(kConst ? bool(SIG >> 6 & 1u) : rd.reduce != 0),
        lam(kConst ? bool(SIG >> 7 & 1u) : rd.lam != 0),
        mixA(kConst ? uint8_t(SIG >> 8 & 31u) : rd.mixA),
        mixB(kConst ? uint8_t(SIG >> 13 & 31u) : rd.mixB) {}
};

// Whether a signature sequence needs the C(x) code (cost, reduction, |+>,
// lambda creation).
template <uint32_t... RS>
constexpr bool sigs_need_c() {
  return ((((RS >> 5 & 1u) | (RS >> 6 & 1u) | (RS >> 7 & 1u)) != 0 || (RS >> 2 & 3u) == 2u) || ...);
}
template <uint32_t S0, uint32_t... RS>
constexpr uint32_t first_sig() { return S0; }
// The first signature, 0 for an empty sequence (generic kernels).
template <uint32_t... RS>
constexpr uint32_t first_sig_or0() {
  if constexpr (sizeof...(RS) == 0) return 0u;
  else return first_sig<RS...>();
}

template <typename Real, int R, int WB, bool FAST, bool CC = true, uint32_t SIG = 0>
__device__ __forceinline__ void fwd_round(const PassDev& P, const PassArgs& A, const SubDev& sp, const RoundDev& rd,
                                          typename Cx<Real>::T* tile, uint64_t gbase, int gpar, const int* tconst,
                                          const typename Cx<Real>::T* phase, int lane, int warp, double* wacc,
                                          typename Cx<Real>::T* v, unsigned long long* ext_s,
                                          const PassTma* M = nullptr, uint32_t tbar = 0, uint64_t tnext = ~0ull) {
  using C2 = typename Cx<Real>::T;
  constexpr int NA = 1 << R;
  constexpr int AB = sizeof(C2);
  // complex64: swapped storage (packed butterflies) and the cost phase from
  // 32-bit turn increments; complex128: plain storage, phase table
  constexpr bool kSw = sizeof(Real) == 4;
  C2* gstate = reinterpret_cast<C2*>(A.out);
  const bool stream = A.diag != nullptr;
  const RoundOps<SIG> op(rd);
  const bool init = CC && op.src == SRC_INIT_D;
  // the round's geometry is rebuilt where needed instead of being kept live
  // across the butterflies (register pressure); s: parity of the thread's
  // amplitude 0 (register amplitude j is stored swapped when parity(j) ^ s)
  const uint32_t entry = RoundGeo<R, WB, AB>::entry_of(rd, lane, warp, A.ctabs);
  const int s = kSw ? int(entry >> 31) ^ gpar : 0;
  if (init) {
    // |+>: every amplitude amp0; with the turn path the cost round writes
    // amp0 times the phase directly
    if (!kSw || stream || !op.cost) {
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        const bool sw = kSw && (parity_c(j) ^ s);
        v[j].x = sw ? Real(0) : Real(P.amp0);
        v[j].y = sw ? Real(P.amp0) : Real(0);
      }
    }
  } else if (op.src == SRC_SMEM_D) {
    bool dn = false;
    if constexpr (AB == 8) {
      if (A.dense) {
        smem_load_dense<R, WB>(op.layout, dense_tile(tile), lane, warp, v);
        dn = true;
      }
    }
    if (!dn) smem_load<R, WB, AB>(op.layout, tile, entry & 0x7fffffffu, v);
  }
  if constexpr (AB == 8) {
    if (A.tma_load && op.dstg && op.src == SRC_SMEM_D) {
      // once every warp has read the tile's last round, the buffer takes the
      // CTA's next tile by one tensor load, issued by the last warp to
      // finish its reads (no warp waits for the others)
      __syncwarp();
      if (lane == 0) {
        __threadfence_block();  // this warp's reads are performed before its count
        if (tile_read_count_add(tbar) == (1u << WB) - 1) {
          __threadfence_block();
          tile_read_count_reset(tbar);
          if (tnext < P.n_units && !tma_stopped(tbar)) {
            fence_proxy_async_smem();
            int32_t c[5];
            tile_coords(*M, P.outer_runs.scatter(tnext), c);
            mbar_expect_tx(tbar, uint32_t(AB) << (R + 5 + WB));
            tma_load_box(&M->tmap, M->tdims, c, (uint32_t)__cvta_generic_to_shared(dense_tile(tile)), tbar);
          }
        }
      }
    }
  }

  if (CC && init && A.ext_keys && (op.cost || op.reduce)) {
    // exhaustive extremes: packed keys of this thread's amplitudes (C(x) and
    // x along one Gray walk), warp minimum, shared-memory minimum per CTA.
    // C(x) = C(~x), so the smallest index of every value has bit n-1 clear:
    // a thread whose amplitudes all have it set skips the scan.
    const RoundGeo<R, WB, AB> geo(sp, rd, gbase, lane, warp, A.ctabs);
    unsigned long long kmin = ~0ull, kmax = ~0ull;
    const bool upper = (geo.gb >> (P.n - 1) & 1ull) != 0;
    const int c_top = P.ncost - 1;
    auto key = [&](int c, uint64_t x) {
      const unsigned long long a = (unsigned long long)(c - P.c_lo) << 34 | x;
      const unsigned long long b = (unsigned long long)(c_top - (c - P.c_lo)) << 34 | x;
      kmin = a < kmin ? a : kmin;
      kmax = b < kmax ? b : kmax;
    };
    if (upper) {
    } else if (stream) {
      gray_walk<R>(geo.gb, geo.gstr, [&](int j, uint64_t x) { key(__ldcg(A.diag + x), x); });
    } else {
      RoundCost<R, WB> rc;
      rc.setup(A.ctabs + rd.ctab, tconst, rd.lane, rd.warp, rd.reg, lane, warp);
      const int32_t* cp = op.cost ? P.cpc : P.cpr;
      // when the register bits' global positions increase with the register
      // index, x grows with j, and 32-bit keys (C - c_lo) << R | j per thread
      // order like the 64-bit ones; the thread's two minima are widened once
      bool ordered = c_top < (1 << 27);
#pragma unroll
      for (int i = 1; i < R; ++i) ordered = ordered && rd.greg[i - 1] < rd.greg[i];
      int lin = rc.kappa;
      if (ordered) {
        uint32_t m0 = ~0u, m1 = ~0u;
#pragma unroll
        for (int k = 0; k < NA; ++k) {
          const int j = k ^ (k >> 1);
          if (k) {
            const int b = ctz_c(k);
            lin += (j >> b & 1) ? rc.e[b] : -rc.e[b];
          }
          const uint32_t d = uint32_t(lin + cp[j] - P.c_lo);
          m0 = min(m0, d << R | uint32_t(j));
          m1 = min(m1, uint32_t(c_top - int(d)) << R | uint32_t(j));
        }
        auto x_of = [&](uint32_t j) {
          uint64_t x = geo.gb;
#pragma unroll
          for (int i = 0; i < R; ++i)
            if (j >> i & 1u) x |= geo.gstr[i];
          return x;
        };
        kmin = (unsigned long long)(m0 >> R) << 34 | x_of(m0 & uint32_t(NA - 1));
        kmax = (unsigned long long)(m1 >> R) << 34 | x_of(m1 & uint32_t(NA - 1));
      } else {
        uint64_t x = geo.gb;
#pragma unroll
        for (int k = 0; k < NA; ++k) {
          const int j = k ^ (k >> 1);
          if (k) {
            const int b = ctz_c(k);
            lin += (j >> b & 1) ? rc.e[b] : -rc.e[b];
            x ^= geo.gstr[b];
          }
          key(lin + cp[j], x);
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long a = __shfl_xor_sync(0xffffffffu, kmin, o);
      const unsigned long long b = __shfl_xor_sync(0xffffffffu, kmax, o);
      kmin = a < kmin ? a : kmin;
      kmax = b < kmax ? b : kmax;
    }
    if (lane == 0) {
      atomicMin(ext_s, kmin);
      atomicMin(ext_s + 1, kmax);
    }
  }

  auto mixer = [&](uint8_t mask, Real tau, Real alpha) {
    if constexpr (kSw) apply_mixer_sw<R>(v, mask, tau, alpha, FAST, s);
    else apply_mixer<R>(v, mask, tau, alpha, FAST);
  };
  mixer(op.mixA, pick<Real>(P.tauA, P.ftauA), pick<Real>(P.alphaA, P.falphaA));

  if (CC && (op.cost || op.reduce)) {
    // C(x) of each register amplitude (streamed, or kappa + CP[j] +
    // sum_{i: j_i = 1} e_i from the round's tables; cp: the round's
    // register-pair table CP[j], of the pass's cost or reduction round). The
    // tables are set up separately for the cost phase and for the reduction
    // so that neither keeps them live across the other.
    auto for_costs = [&](const int32_t* cp, auto&& f) {
      if (stream) {
        const RoundGeo<R, WB, AB> geo(sp, rd, gbase, lane, warp, A.ctabs);
        gray_ptr_walk<R>(A.diag, geo.gb, geo.gstr, [&](int j, const int32_t* q) { f(j, __ldcg(q)); });
      } else {
        RoundCost<R, WB> rc;
        rc.setup(A.ctabs + rd.ctab, tconst, rd.lane, rd.warp, rd.reg, lane, warp);
        int lin = rc.kappa;
#pragma unroll
        for (int k = 0; k < NA; ++k) {
          const int j = k ^ (k >> 1);
          if (k) {
            const int b = ctz_c(k);
            lin += (j >> b & 1) ? rc.e[b] : -rc.e[b];
          }
          f(j, lin + cp[j]);
        }
      }
    };
    if (op.cost) {
      // a swapped amplitude takes the conjugate phase in the plain product
      // formula: the angle scale is -2pi/2^32 for it (k1) and +2pi/2^32 for
      // a plain one (k0)
      const float k0 = s ? -kTurn32 : kTurn32, k1 = -k0;
      if (kSw && !stream) {
        // turn count of amplitude j: t0 + sum_{i: j_i} E_i + cpt[j] (Gray order)
        uint32_t E[R];
        uint32_t t;
        {
          RoundCost<R, WB> rc;
          rc.setup(A.ctabs + rd.ctab, tconst, rd.lane, rd.warp, rd.reg, lane, warp);
          t = rc.turns(P.ph0, P.ph1, P.c_lo, E);
        }
        // |+> round: a swapped amplitude is amp0 (sin, cos) = amp0 exp(i (pi/2 - angle)):
        // turn count 2^30 - t (quarter turn), i.e. t * m + q with (m, q) = (-1, 2^30)
        const uint32_t m0 = s ? 0xffffffffu : 1u, q0 = s ? (1u << 30) : 0u;
        const uint32_t m1 = s ? 1u : 0xffffffffu, q1 = s ? 0u : (1u << 30);
#pragma unroll
        for (int k = 0; k < NA; ++k) {
          const int j = k ^ (k >> 1);
          if (k) {
            const int b = ctz_c(k);
            t += (j >> b & 1) ? E[b] : 0u - E[b];
          }
          const uint32_t tj = t + P.cpt[j];
          if (init) {
            const float2 ph = parity_c(j) ? phase_turns32(tj * m1 + q1) : phase_turns32(tj * m0 + q0);
            v[j].x = P.famp0 * ph.x;
            v[j].y = P.famp0 * ph.y;
          } else {
            const float2 ph = phase_turns32(tj, parity_c(j) ? k1 : k0);
            const Real xr = v[j].x, xi = v[j].y;
            v[j].x = xr * ph.x - xi * ph.y;
            v[j].y = xr * ph.y + xi * ph.x;
          }
        }
      } else {
        for_costs(P.cpc, [&](int j, int c) {
          C2 ph;
          if constexpr (kSw) ph = phase_turns(P.ph0, P.ph1, uint32_t(c - P.c_lo), parity_c(j) ? k1 : k0);
          else ph = phase[min(unsigned(c - P.c_lo), unsigned(P.ncost - 1))];
          const Real xr = v[j].x, xi = v[j].y;
          v[j].x = xr * ph.x - xi * ph.y;
          v[j].y = xr * ph.y + xi * ph.x;
        });
      }
    }
    mixer(op.mixB, pick<Real>(P.tauB, P.ftauB), pick<Real>(P.alphaB, P.falphaB));
    if (op.dstg && sp.rescale) {
      const Real sc = pick<Real>(sp.scale, sp.fscale);
#pragma unroll
      for (int j = 0; j < NA; ++j) scale_amp(v[j], sc);
    }
    if (op.reduce) {
      // |psi|^2 and C(x) do not depend on the storage order of (re, im)
      Real sn = 0, scc = 0;
      if (A.bsum) {
        // also |psi|^2 per sampling block of 2^12 amplitudes: tile bits 12
        // and 13 (if any) select the block; hr[k]: the register position of
        // tile bit 12 + k, or -1 when a lane or warp bit holds it (hthr)
        int hr[2] = {-1, -1}, hthr = 0;
#pragma unroll
        for (int i = 0; i < R; ++i) {
          const int b = tile_bit<R, WB, SIG>(rd, 0, i);
          if (b >= 12 && b < 12 + kBlkBits<R, WB>) hr[b - 12] = i;
        }
#pragma unroll
        for (int i = 0; i < 5; ++i) {
          const int b = tile_bit<R, WB, SIG>(rd, 1, i);
          if (b >= 12 && b < 12 + kBlkBits<R, WB>) hthr |= (lane >> i & 1) << (b - 12);
        }
#pragma unroll
        for (int i = 0; i < WB; ++i) {
          const int b = tile_bit<R, WB, SIG>(rd, 2, i);
          if (b >= 12 && b < 12 + kBlkBits<R, WB>) hthr |= (warp >> i & 1) << (b - 12);
        }
        constexpr int NB = 1 << kBlkBits<R, WB>;
        Real sb[NB];
#pragma unroll
        for (int k = 0; k < NB; ++k) sb[k] = 0;
        for_costs(P.cpr, [&](int j, int c) {
          const Real pr = v[j].x * v[j].x + v[j].y * v[j].y;
          sn += pr;
          scc = fma(pr, Real(c), scc);
          int h = hthr;
          if (hr[0] >= 0) h |= j >> hr[0] & 1;
          if (NB > 2 && hr[1] >= 0) h |= (j >> hr[1] & 1) << 1;
#pragma unroll
          for (int k = 0; k < NB; ++k)
            if (h == k) sb[k] += pr;
        });
        // block sums: each thread's partial over its register amplitudes
        // (at most 2^R terms in the state precision), then FP64 (complex64:
        // double-float) from there on: the partials go to shared memory and
        // the caller adds them in a fixed order
        const int tid = (warp << 5) | lane;
        if constexpr (sizeof(Real) == 4) {
          float* wf = reinterpret_cast<float*>(wacc + 2 * (32 << WB));
#pragma unroll
          for (int k = 0; k < NB; ++k) wf[k * (32 << WB) + tid] = sb[k];
        } else {
#pragma unroll
          for (int k = 0; k < NB; ++k) wacc[(2 + k) * (32 << WB) + tid] = double(sb[k]);
        }
      } else {
        for_costs(P.cpr, [&](int j, int c) {
          const Real pr = v[j].x * v[j].x + v[j].y * v[j].y;
          sn += pr;
          scc = fma(pr, Real(c), scc);
        });
      }
      // <C> and norm: this thread's running sums (one add per tile; FP64, or
      // double-float for complex64), the cross-thread FP64 reduction runs once
      // at the end (finish_thread_sums, reduce_thread_sums)
      const int tid = (warp << 5) | lane;
      if constexpr (sizeof(Real) == 4) {
        df_add(reinterpret_cast<float2*>(wacc)[tid], sn);
        df_add(reinterpret_cast<float2*>(wacc)[(32 << WB) + tid], scc);
      } else {
        wacc[tid] += double(sn);
        wacc[(32 << WB) + tid] += double(scc);
      }
    }
  } else {
    mixer(op.mixB, pick<Real>(P.tauB, P.ftauB), pick<Real>(P.alphaB, P.falphaB));
    if (op.dstg && sp.rescale) {
      const Real sc = pick<Real>(sp.scale, sp.fscale);
#pragma unroll
      for (int j = 0; j < NA; ++j) scale_amp(v[j], sc);
    }
  }

  if (op.dstg) {
    if constexpr (kSw) {
      if (sp.st_plain) swap_odd<R>(reinterpret_cast<float2*>(v), s);  // a run's output: plain storage
    }
    if constexpr (AB == 8) {
     if (A.tma_store) {
      // the tile densely into shared memory (tile index order, the tensor
      // store's box) once every thread has read this round's amplitudes from
      // the padded tile; one thread stores the box after the round
      __syncthreads();
      C2* dense = dense_tile(tile);
      uint32_t tb = 0;
#pragma unroll
      for (int i = 0; i < 5; ++i) tb |= uint32_t(lane >> i & 1) << tile_bit<R, WB, SIG>(rd, 1, i);
#pragma unroll
      for (int i = 0; i < WB; ++i) tb |= uint32_t(warp >> i & 1) << tile_bit<R, WB, SIG>(rd, 2, i);
      auto toff = [&](int j) {
        uint32_t o = 0;
#pragma unroll
        for (int i = 0; i < R; ++i)
          if (j >> i & 1) o |= 1u << tile_bit<R, WB, SIG>(rd, 0, i);
        return o;
      };
      if (op.layout == 4) {
#pragma unroll
        for (int j = 0; j < (1 << R); j += 2)
          *reinterpret_cast<float4*>(dense + tb + toff(j)) = make_float4(v[j].x, v[j].y, v[j + 1].x, v[j + 1].y);
      } else {
#pragma unroll
        for (int j = 0; j < (1 << R); ++j) dense[tb + toff(j)] = v[j];
      }
      fence_proxy_async_smem();
      return;
     }
    }
    const RoundGeo<R, WB, AB> geo(sp, rd, gbase, lane, warp, A.ctabs);
    if (A.l2hint) {
      // outputs of a sub-pass that a later sub-pass reads back stay in L2
      const uint64_t pol = sp.keep ? l2_policy_evict_last() : l2_policy_evict_first();
      gray_ptr_walk<R>(gstate, geo.gb, geo.gstr, [&](int j, C2* q) { st_hint(q, v[j], pol); });
    } else {
      if (AB == 8 && op.layout == 4)  // paired layout: one 16-byte store per register pair
        gray_ptr_walk_pairs<R>(gstate, geo.gb, geo.gstr, [&](int j, C2* q) { store_pair(q, v[j], v[j | 1]); });
      else
        gray_ptr_walk<R>(gstate, geo.gb, geo.gstr, [&](int j, C2* q) { __stcg(q, v[j]); });
    }
  } else {
    bool dn = false;
    if constexpr (AB == 8) {
      if (A.dense) {
        smem_store_dense<R, WB>(op.layout, dense_tile(tile), lane, warp, v);
        dn = true;
      }
    }
    if (!dn) smem_store<R, WB, AB>(op.layout, tile, entry & 0x7fffffffu, v);
  }
}

// One super-tile (unit) of a forward pass: every tile of each of its sub-passes.
// All threads of the CTA take part; shared memory is free again on return.
// tcount: the CTA's running tile count (selects the tile-constant buffer when
// the constants come from a table); may be null when no sub-pass has a table.
// RS: the round signatures of a specialised kernel (one sub-pass of one tile
// per unit, rounds compiled from the signatures), empty for the generic kernel.
template <typename Real, int R, int WB, bool FAST, bool CC = true, uint32_t... RS>
__device__ __forceinline__ void fwd_unit(const PassDev& P, const PassArgs& A, uint64_t unit,
                                         typename Cx<Real>::T* tile, int* tconst,
                                         const typename Cx<Real>::T* phase, double* wacc,
                                         uint32_t* tcount = nullptr, unsigned long long* ext_s = nullptr,
                                         const PassTma* M = nullptr, uint32_t tbar = 0, uint32_t* tk = nullptr) {
  using C2 = typename Cx<Real>::T;
  constexpr int T = R + 5 + WB;
  constexpr int NT = 32 << WB;
  constexpr int AB = sizeof(C2);
  constexpr bool kSpec = sizeof...(RS) > 0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = P.n;
  const bool stream = A.diag != nullptr;
  C2 v[1 << R];
  const uint64_t ubase = P.outer_runs.scatter(unit);
  for (int s = 0; s < (kSpec ? 1 : P.nsub); ++s) {
    const SubDev& sp = P.sub[s];
    const uint64_t ntiles = kSpec ? 1 : 1ull << sp.ninner;
    for (uint64_t ti = 0; ti < ntiles; ++ti) {
      const uint64_t gbase = kSpec ? ubase : ubase | sp.inner_runs.scatter(ti);
      // issue the tile's global loads first: their latency overlaps the
      // barrier below and the tile constants
      bool load0;
      if constexpr (kSpec) load0 = (first_sig<RS...>() >> 2 & 3u) == SRC_GLOBAL_D;
      else load0 = sp.rd[0].src == SRC_GLOBAL_D;
      if (load0 && A.prefetch == 2 && sp.ninner == 0 && M->pfdist > 0) {
        // the CTA's next tile into L2 by one tensor prefetch (tensor memory
        // accelerator; no load-store unit instructions)
        // (pfdist tiles ahead; the CTA's first tile also issues the nearer ones)
        if (tid == 0) {
          for (int k = unit == blockIdx.x ? 1 : M->pfdist; k <= M->pfdist; ++k) {
            const uint64_t next = unit + uint64_t(k) * gridDim.x;
            if (next >= P.n_units) break;
            int32_t c[5];
            tile_coords(*M, P.outer_runs.scatter(next), c);
            tma_prefetch_l2(&M->tmap, M->tdims, c);
          }
        }
      } else if (load0 && A.prefetch == 1 && sp.ninner == 0) {
        // the CTA's next tile (unit + gridDim.x) into L2: its 2^(T-4) runs of
        // 16 consecutive amplitudes (tile bits 0..3 are global bits 0..3),
        // one 128-byte line each
        const uint64_t next = unit + gridDim.x;
        if (next < P.n_units) {
          const uint64_t nbase = P.outer_runs.scatter(next);
          const C2* gs = reinterpret_cast<const C2*>(A.state);
          for (int r = tid; r < (1 << (T - 4)); r += NT) {
            uint64_t g = nbase;
#pragma unroll
            for (int j = 4; j < T; ++j) g |= uint64_t(r >> (j - 4) & 1) << sp.pos[j];
            asm volatile("prefetch.global.L2 [%0];" ::"l"(gs + g));
          }
        }
      }
      const bool tload = AB == 8 && load0 && A.tma_load;
      if (load0 && !tload) {
        const RoundGeo<R, WB, AB> g0(sp, sp.rd[0], gbase, lane, warp, A.ctabs);
        const C2* gs = reinterpret_cast<const C2*>(A.state);
        if (A.l2hint) {
          const uint64_t pol = l2_policy_evict_first();
          gray_ptr_walk<R>(gs, g0.gb, g0.gstr, [&](int j, const C2* q) { v[j] = ld_hint(q, pol); });
        } else {
          bool paired = false;
          if constexpr (kSpec) paired = sig_layout(first_sig<RS...>()) == 4;
          else paired = sp.rd[0].layout == 4;
          if (AB == 8 && paired) {
            // paired layout: register bit 0 is index bit 0, one 16-byte load
            // brings amplitudes j and j | 1
            gray_ptr_walk_pairs<R>(gs, g0.gb, g0.gstr, [&](int j, const C2* q) { load_pair(q, v[j], v[j | 1]); });
          } else {
            gray_ptr_walk<R>(gs, g0.gb, g0.gstr, [&](int j, const C2* q) { v[j] = __ldcg(q); });
          }
        }
      }
      // tile constants from the table: into the buffer the previous tile did
      // not use, published by the barrier below. The specialised write-only
      // |+> pass, which has no state load to hide the table read behind,
      // copies them asynchronously one unit ahead (the CTA's next unit is
      // unit + gridDim.x). (Passes that load the state measured slower with
      // the early copy.)
      int* tc = tconst;
      const bool tab = CC && sp.needs_c && !stream && sp.tct != nullptr;
      bool ahead = false;
      if constexpr (kSpec) ahead = tab && (first_sig<RS...>() >> 2 & 3u) == SRC_INIT_D;
      if (tab) {
        tc = tconst + 32 * (*tcount & 1u);
        if (ahead && *tcount != 0) {
          cp_async_wait_all();  // this tile's constants, copied during the previous tile
        } else if (tid < kTileConstInts) {
          tc[tid == 15 ? 16 : tid] = __ldg(sp.tct + (((unit << sp.ninner) + ti) * kTileConstInts + tid));
        }
        *tcount += 1;
      }
      if (AB == 8 && A.tma_store && tid == 0) bulk_wait_read();  // the previous tile's store has read its box
      if constexpr (AB == 8) {
        if (tload) {
          // this tile arrived by a tensor load (the CTA's k-th, mbarrier
          // phase k & 1): the first round's amplitudes from the dense box
          // (tile index order); the barrier below ends the reads before the
          // first round writes the padded tile
          const uint32_t k = (*tk)++;
          if (!tma_stopped(tbar) && !mbar_wait_bounded(tbar, k & 1u, A.tma_wait_ns)) {
            tma_stop(tbar, k & 1u);
            if (lane == 0) atomicOr(A.err, 1ull);
          }
          constexpr uint32_t S0 = first_sig_or0<RS...>();
          const RoundDev& rd0 = sp.rd[0];
          const C2* dense = dense_tile(tile);
          uint32_t tb = 0;
#pragma unroll
          for (int i = 0; i < 5; ++i) tb |= uint32_t(lane >> i & 1) << tile_bit<R, WB, S0>(rd0, 1, i);
#pragma unroll
          for (int i = 0; i < WB; ++i) tb |= uint32_t(warp >> i & 1) << tile_bit<R, WB, S0>(rd0, 2, i);
          auto toff = [&](int j) {
            uint32_t o = 0;
#pragma unroll
            for (int i = 0; i < R; ++i)
              if (j >> i & 1) o |= 1u << tile_bit<R, WB, S0>(rd0, 0, i);
            return o;
          };
          bool paired;
          if constexpr (kSpec) paired = sig_layout(S0) == 4;
          else paired = rd0.layout == 4;
          if (paired) {
#pragma unroll
            for (int j = 0; j < (1 << R); j += 2) {
              const float4 q = *reinterpret_cast<const float4*>(dense + tb + toff(j));
              v[j] = make_float2(q.x, q.y);
              v[j | 1] = make_float2(q.z, q.w);
            }
          } else {
#pragma unroll
            for (int j = 0; j < (1 << R); ++j) v[j] = dense[tb + toff(j)];
          }
        }
      }
      // previous tile finished with shared memory. Not needed when the tile
      // came by a tensor load into dense slots and the first round reads no
      // tile constants: every warp read the previous tile's last round before
      // that load was issued, and the first round writes back only the slots
      // it read (dense == 2)
      if (!(AB == 8 && tload && A.dense == 2)) __syncthreads();
      if (ahead) {
        const uint64_t next = unit + gridDim.x;
        if (next < P.n_units && tid < kTileConstInts)
          cp_async4(tconst + 32 * (*tcount & 1u) + (tid == 15 ? 16 : tid), sp.tct + next * kTileConstInts + tid);
        cp_async_commit();
      }
      if (CC && sp.needs_c && !stream && !tab) {
        if (tid == 0) tconst[16] = 0;
        __syncthreads();
        tile_consts<T>(sp.pos, gbase, A.wmat, n, tconst, lane, warp, NT / 32);
        __syncthreads();
      }
      const int gpar = __popcll(gbase) & 1;
      bool red_last;
      if constexpr (kSpec) {
        // rounds unrolled from the signatures
        int r = 0;
        auto run = [&](auto sigc) {
          constexpr uint32_t S = decltype(sigc)::value;
          if constexpr ((S >> 2 & 3u) == SRC_SMEM_D) __syncthreads();
          fwd_round<Real, R, WB, FAST, CC, S>(P, A, sp, sp.rd[r], tile, gbase, gpar, tc, phase, lane, warp, wacc, v,
                                              ext_s, M, tbar, unit + gridDim.x);
          ++r;
        };
        (run(std::integral_constant<uint32_t, RS>{}), ...);
        red_last = ((RS >> 6 & 1u) | ...) != 0;  // the reduction is in the last round
      } else {
        for (int r = 0; r < sp.nrounds; ++r) {
          const RoundDev& rd = sp.rd[r];
          if (rd.src == SRC_SMEM_D) __syncthreads();
          fwd_round<Real, R, WB, FAST, CC>(P, A, sp, rd, tile, gbase, gpar, tc, phase, lane, warp, wacc, v, ext_s, M,
                                           tbar, unit + gridDim.x);
        }
        red_last = sp.rd[sp.nrounds - 1].reduce != 0;
      }
      if (AB == 8 && A.tma_store) {
        __syncthreads();  // the dense box is complete (each writer fenced its writes)
        if (tid == 0) {
          int32_t c[5];
          tile_coords(*M, gbase, c);
          tma_store_box(&M->smap, M->tdims, c, (uint32_t)__cvta_generic_to_shared(dense_tile(tile)));
        }
      }
      if (CC && A.bsum && red_last) {
        // this tile is 2^T consecutive amplitudes: its 2^(T-12) block sums;
        // warp k adds block k's per-thread partials (each lane a strided set
        // in two accumulators, then a shuffle tree: a fixed order), in FP64,
        // or for complex64 in double-float, converted to FP64 once per block
        constexpr int NB = 1 << kBlkBits<R, WB>;
        __syncthreads();
        if (warp < NB) {
          if constexpr (sizeof(Real) == 4) {
            const float* wf = reinterpret_cast<const float*>(wacc + 2 * NT) + warp * NT;
            float2 b0 = make_float2(0.f, 0.f), b1 = make_float2(0.f, 0.f);
            for (int t = lane; t < NT; t += 64) {
              df_add(b0, wf[t]);
              df_add(b1, wf[t + 32]);
            }
            df_add(b0, b1);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
              df_add(b0, make_float2(__shfl_xor_sync(0xffffffffu, b0.x, o), __shfl_xor_sync(0xffffffffu, b0.y, o)));
            if (lane == 0) A.bsum[(gbase >> 12) + warp] = double(b0.x) + double(b0.y);
          } else {
            double b = 0.0;
            for (int t = lane; t < NT; t += 32) b += wacc[(2 + warp) * NT + t];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
            if (lane == 0) A.bsum[(gbase >> 12) + warp] = b;
          }
        }
      }
    }
    __syncthreads();  // sub-pass boundary: this CTA's global writes are visible to it
  }
}

// Body of the forward pass kernels. Shared-memory layout of the dynamic buffer:
//   tile[padded 2^T] complex | tile consts (two buffers) | phase table
template <typename Real, int R, int WB, bool FAST, bool CC, uint32_t... RS>
__device__ __forceinline__ void fwd_pass_body(const PassDev& P, const PassArgs& A, const PassTma& M) {
  using C2 = typename Cx<Real>::T;
  constexpr int T = R + 5 + WB;
  constexpr int NT = 32 << WB;
  constexpr int AB = sizeof(C2);
  constexpr uint32_t TILE = padded_size<AB>(T);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* tile = reinterpret_cast<C2*>(smem_raw);
  int* tconst = reinterpret_cast<int*>(tile + TILE);  // 2 x (delta[0..15], base at [16])
  C2* ptab = reinterpret_cast<C2*>(smem_raw + ((size_t(TILE) * AB + kTconstSmemInts * 4 + 15) & ~size_t(15)));

  const int tid = threadIdx.x;
  const C2* phase = reinterpret_cast<const C2*>(A.phase);
  if (A.phase_in_smem && A.phase) {
    for (int i = tid; i < P.ncost; i += NT) ptab[i] = phase[i];
    phase = ptab;
  }
  // per-thread running sums [norm for all threads, <C> for all threads], then
  // per-thread block-sum partials (2^(T-12) blocks per tile)
  __shared__ double wacc[(2 + (1 << kBlkBits<R, WB>)) * NT];
  wacc[tid] = 0.0;
  wacc[NT + tid] = 0.0;

  // exhaustive extremes (optional): this CTA's minimum keys
  __shared__ unsigned long long ext_s[2];
  if (tid < 2) ext_s[tid] = ~0ull;  // published by the first tile's barrier

  // tensor tile loads: the mbarrier, and the CTA's first tile
  __shared__ __align__(8) unsigned long long tma_bar[2];  // mbarrier; stop flag, warps' read count
  const uint32_t tbar = (uint32_t)__cvta_generic_to_shared(tma_bar);
  if (AB == 8 && A.tma_load) {
    if (tid == 0) {
      tma_bar[1] = 0ull;
      mbar_init(tbar, 1);
    }
    __syncthreads();
    if (tid == 0 && blockIdx.x < P.n_units) {
      int32_t c[5];
      tile_coords(M, P.outer_runs.scatter(blockIdx.x), c);
      mbar_expect_tx(tbar, uint32_t(AB) << T);
      tma_load_box(&M.tmap, M.tdims, c, (uint32_t)__cvta_generic_to_shared(dense_tile(tile)), tbar);
    }
  }

  uint32_t tcount = 0, tk = 0;
  for (uint64_t unit = blockIdx.x; unit < P.n_units; unit += gridDim.x)
    fwd_unit<Real, R, WB, FAST, CC, RS...>(P, A, unit, tile, tconst, phase, wacc, &tcount, ext_s, &M, tbar, &tk);
  if (A.tma_store && tid == 0) bulk_wait_all();  // the last tensor store is complete before the CTA ends
  if (AB == 8 && A.tma_load) {
    // a CTA whose wait gave up ends only once the load it gave up on has
    // landed (bounded)
    __syncthreads();
    const uint32_t f = tid == 0 ? tma_stop_word(tbar) : 0u;
    if (f) mbar_wait_bounded(tbar, f - 1u, kTmaWaitNs);
  }

  if (CC && A.ext_keys) {
    __syncthreads();
    if (tid < 2) atomicMin(A.ext_keys + tid, ext_s[tid]);
  }

  if (A.partial) {
    finish_thread_sums<Real, NT>(wacc, tid);
    __syncthreads();
    double sN, sC;
    reduce_thread_sums<NT>(wacc, sN, sC);
    if (tid == 0) {
      A.partial[2 * blockIdx.x] = sN;
      A.partial[2 * blockIdx.x + 1] = sC;
    }
  }
}

// Generic forward pass: rounds decoded from the descriptor at run time.
template <typename Real, int R, int WB, bool FAST, bool CC>
__global__ void __launch_bounds__(32 << WB, sizeof(Real) == 4 ? (R + WB <= 7 ? 4 : R + WB <= 8 ? 2 : 1)
                                                              : (R + WB <= 7 ? 2 : 1))
fwd_pass_kernel(const __grid_constant__ PassDev P, const PassArgs A, const __grid_constant__ PassTma M) {
  fwd_pass_body<Real, R, WB, FAST, CC>(P, A, M);
}

// Specialised complex64 forward pass for one round-signature sequence RS
// (one sub-pass of one tile per super-tile): the rounds' operations, layouts
// and masks are compile-time constants.
template <int R, int WB, bool FAST, uint32_t... RS>
__global__ void __launch_bounds__(32 << WB, R + WB <= 7 ? 4 : R + WB <= 8 ? 2 : 1)
fwd_spec_kernel(const __grid_constant__ PassDev P, const PassArgs A, const __grid_constant__ PassTma M) {
  fwd_pass_body<float, R, WB, FAST, sigs_need_c<RS...>(), RS...>(P, A, M);
}

}  // namespace qaoa
