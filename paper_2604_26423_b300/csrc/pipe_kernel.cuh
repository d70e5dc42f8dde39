// pipe_kernel.cuh -- software-pipelined forward pass kernel (complex64).
//
// Same plan, rounds and arithmetic as fwd_pass_kernel (pass_kernel.cuh), but
// the tile a round 0 would read from global memory is instead prefetched into
// one of two shared-memory buffers with per-thread asynchronous copies
// (cp.async, 8 bytes per amplitude, written straight into the swizzled slots)
// while the previous tile is being processed. Round 0 then reads shared
// memory. One CTA per SM keeps the HBM read stream busy during compute.
//
// Work order: a CTA takes super-tiles in adjacent pairs and interleaves them
// sub-pass by sub-pass ([s0 of A][s0 of B][s1 of A][s1 of B]...), so the tile
// prefetched at a sub-pass boundary always belongs to a super-tile whose
// previous sub-pass finished at least one full sub-pass earlier.
#pragma once
#include "device.cuh"
#include "pass_kernel.cuh"

namespace qaoa {

__device__ __forceinline__ void cp_async8(uint32_t smem_addr, const void* gptr) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr), "l"(gptr) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

struct PipeItem {
  uint64_t pair;   // pair index
  int s;           // sub-pass
  int uu;          // 0 or 1 within the pair
  uint64_t ti;     // tile inside the super-tile
  bool valid;
};

template <int R, int WB, bool FAST>
__global__ void __launch_bounds__(32 << WB, 1)
fwd_pipe_kernel(const __grid_constant__ PassDev P, const PassArgs A) {
  using Real = float;
  using C2 = float2;
  constexpr int T = R + 5 + WB;
  constexpr int NT = 32 << WB;
  constexpr int NA = 1 << R;
  constexpr int AB = 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* buf0 = reinterpret_cast<C2*>(smem_raw);
  int* wsm = reinterpret_cast<int*>(buf0 + (2 << T));
  int* tconst = wsm + P.n * P.n;
  C2* ptab = reinterpret_cast<C2*>(smem_raw +
                                   (((size_t(2) << T) * AB + size_t(P.n * P.n + 32) * 4 + 15) & ~size_t(15)));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = P.n;
  for (int i = tid; i < n * n; i += NT) wsm[i] = A.wmat[i];
  const C2* phase = reinterpret_cast<const C2*>(A.phase);
  if (A.phase_in_smem && A.phase) {
    for (int i = tid; i < P.ncost; i += NT) ptab[i] = phase[i];
    phase = ptab;
  }
  C2* gstate = reinterpret_cast<C2*>(A.state);
  const bool stream = A.diag != nullptr;
  const uint64_t npairs = (P.n_units + 1) / 2;
  double accN = 0.0, accC = 0.0;

  auto unit_of = [&](const PipeItem& it) { return it.pair * 2 + it.uu; };
  auto advance = [&](PipeItem it) {
    const uint64_t ntiles = 1ull << P.sub[it.s].ninner;
    const int nuu = (it.pair * 2 + 1 < P.n_units) ? 2 : 1;
    if (++it.ti < ntiles) return it;
    it.ti = 0;
    if (++it.uu < nuu) return it;
    it.uu = 0;
    if (++it.s < P.nsub) return it;
    it.s = 0;
    it.pair += gridDim.x;
    it.valid = it.pair < npairs;
    return it;
  };
  auto tile_base = [&](const PipeItem& it) {
    const SubDev& sp = P.sub[it.s];
    return scatter_bits(unit_of(it), P.outer, P.nouter) | scatter_bits(it.ti, sp.inner, sp.ninner);
  };
  // copies the tile of `it` into buffer b in round 0's lane / warp / register split
  auto prefetch = [&](const PipeItem& it, int b) {
    const SubDev& sp = P.sub[it.s];
    const RoundDev& rd = sp.rd[0];
    if (rd.src != SRC_GLOBAL_D) return;
    const uint64_t gbase = tile_base(it);
    uint32_t tb = 0;
    uint64_t gb = gbase;
#pragma unroll
    for (int i = 0; i < 5; ++i)
      if (lane >> i & 1) { tb |= 1u << rd.lane[i]; gb |= 1ull << sp.pos[rd.lane[i]]; }
#pragma unroll
    for (int i = 0; i < WB; ++i)
      if (warp >> i & 1) { tb |= 1u << rd.warp[i]; gb |= 1ull << sp.pos[rd.warp[i]]; }
    const uint32_t sbase = static_cast<uint32_t>(__cvta_generic_to_shared(buf0 + (size_t(b) << T)));
    const uint32_t sb0 = swz<AB>(tb);
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      uint32_t so = sb0;
      uint64_t go = gb;
#pragma unroll
      for (int i = 0; i < R; ++i)
        if (j >> i & 1) { so ^= swz<AB>(1u << rd.reg[i]); go |= 1ull << sp.pos[rd.reg[i]]; }
      cp_async8(sbase + so * AB, gstate + go);
    }
  };

  PipeItem it{blockIdx.x, 0, 0, 0, blockIdx.x < npairs};
  if (it.valid) prefetch(it, 0);
  cp_async_commit();
  int k = 0;
  while (it.valid) {
    const PipeItem nx = advance(it);
    // a lone super-tile (odd count) crossing into its next sub-pass reads what
    // this tile is about to write: prefetch it only after this tile's stores
    const bool lone = it.pair * 2 + 1 >= P.n_units;
    const bool defer = nx.valid && nx.pair == it.pair && nx.s != it.s && lone;
    if (nx.valid && !defer) prefetch(nx, (k + 1) & 1);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();  // this tile's copies are visible to every thread
    const SubDev& sp = P.sub[it.s];
    const uint64_t gbase = tile_base(it);
    C2* tile = buf0 + (size_t(k & 1) << T);
    if (sp.needs_c && !stream) {
      if (warp == 0) tile_consts<T>(sp.pos, gbase, wsm, n, tconst, lane);
      __syncthreads();
    }
    for (int r = 0; r < sp.nrounds; ++r) {
      const RoundDev& rd = sp.rd[r];
      if (r > 0) __syncthreads();
      uint32_t tb = 0;
      uint64_t gb = gbase;
#pragma unroll
      for (int i = 0; i < 5; ++i)
        if (lane >> i & 1) { tb |= 1u << rd.lane[i]; gb |= 1ull << sp.pos[rd.lane[i]]; }
#pragma unroll
      for (int i = 0; i < WB; ++i)
        if (warp >> i & 1) { tb |= 1u << rd.warp[i]; gb |= 1ull << sp.pos[rd.warp[i]]; }
      uint32_t sstr[R];
      uint64_t gstr[R];
#pragma unroll
      for (int i = 0; i < R; ++i) {
        sstr[i] = swz<AB>(1u << rd.reg[i]);
        gstr[i] = 1ull << sp.pos[rd.reg[i]];
      }
      const uint32_t sb0 = swz<AB>(tb);
      auto soff = [&](int j) {
        uint32_t o = sb0;
#pragma unroll
        for (int i = 0; i < R; ++i)
          if (j >> i & 1) o ^= sstr[i];
        return o;
      };
      auto goff = [&](int j) {
        uint64_t o = gb;
#pragma unroll
        for (int i = 0; i < R; ++i)
          if (j >> i & 1) o |= gstr[i];
        return o;
      };
      C2 v[NA];
      if (rd.src == SRC_INIT_D) {
#pragma unroll
        for (int j = 0; j < NA; ++j) { v[j].x = Real(P.amp0); v[j].y = Real(0); }
      } else {
#pragma unroll
        for (int j = 0; j < NA; ++j) v[j] = tile[soff(j)];
      }
      apply_mixer<R>(v, rd.mixA, Real(P.tauA), Real(P.alphaA), FAST);
      if (rd.cost | rd.reduce) {
        RoundCost<R, WB> rc;
        if (!stream) rc.setup(A.ctabs + rd.ctab, tconst, rd.lane, rd.warp, rd.reg, lane, warp);
        auto cv = [&](int j) { return stream ? __ldcg(A.diag + goff(j)) : rc(j); };
        if (rd.cost) {
#pragma unroll
          for (int j = 0; j < NA; ++j) {
            const C2 ph = phase[min(max(cv(j) - P.c_lo, 0), P.ncost - 1)];
            const Real xr = v[j].x, xi = v[j].y;
            v[j].x = xr * ph.x - xi * ph.y;
            v[j].y = xr * ph.y + xi * ph.x;
          }
        }
        apply_mixer<R>(v, rd.mixB, Real(P.tauB), Real(P.alphaB), FAST);
        if (rd.dst == DST_GLOBAL_D && sp.scale != 1.0) {
          const Real sc = Real(sp.scale);
#pragma unroll
          for (int j = 0; j < NA; ++j) { v[j].x *= sc; v[j].y *= sc; }
        }
        if (rd.reduce) {
          Real sn = 0, sc = 0;
#pragma unroll
          for (int j = 0; j < NA; ++j) {
            const Real pr = v[j].x * v[j].x + v[j].y * v[j].y;
            sn += pr;
            sc = fma(pr, Real(cv(j)), sc);
          }
          accN += double(sn);
          accC += double(sc);
        }
      } else {
        apply_mixer<R>(v, rd.mixB, Real(P.tauB), Real(P.alphaB), FAST);
        if (rd.dst == DST_GLOBAL_D && sp.scale != 1.0) {
          const Real sc = Real(sp.scale);
#pragma unroll
          for (int j = 0; j < NA; ++j) { v[j].x *= sc; v[j].y *= sc; }
        }
      }
      if (rd.dst == DST_GLOBAL_D) {
#pragma unroll
        for (int j = 0; j < NA; ++j) __stcg(gstate + goff(j), v[j]);
      } else {
#pragma unroll
        for (int j = 0; j < NA; ++j) tile[soff(j)] = v[j];
      }
    }
    __syncthreads();  // buffer k&1 and the tile constants are free again
    if (defer) {
      prefetch(nx, (k + 1) & 1);
      cp_async_commit();
    }
    it = nx;
    ++k;
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");

  if (A.partial) {
    __shared__ double red[2][32];
    for (int o = 16; o > 0; o >>= 1) {
      accN += __shfl_xor_sync(0xffffffffu, accN, o);
      accC += __shfl_xor_sync(0xffffffffu, accC, o);
    }
    if (lane == 0) { red[0][warp] = accN; red[1][warp] = accC; }
    __syncthreads();
    if (tid == 0) {
      double sN = 0, sC = 0;
      for (int w = 0; w < NT / 32; ++w) { sN += red[0][w]; sC += red[1][w]; }
      A.partial[2 * blockIdx.x] = sN;
      A.partial[2 * blockIdx.x + 1] = sC;
    }
  }
}

}  // namespace qaoa
