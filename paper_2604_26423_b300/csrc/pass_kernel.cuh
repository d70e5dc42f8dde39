// pass_kernel.cuh -- the fused forward pass kernel of the LR-QAOA simulation.
//
// One launch = one HBM pass over the state (see plan.h). For every super-tile
// the CTA runs the sub-passes of the pass; a sub-pass moves 2^T-amplitude
// tiles global -> registers -> (shared memory -> registers)* -> global, and in
// each round applies, on the thread's 2^R register amplitudes:
//   mixer of layer a   exp(+i beta_a X_q) on the round's target bits (Eq. UB)
//   cost phase         exp(-i gamma_b s h(x)), h = W - 2 C(x)  (Eqs. H_C, UC)
//   mixer of layer b   on the round's target bits
//   reduction          |psi_x|^2 and |psi_x|^2 C(x) (final pass)
// The mixer rotation [[c, i s], [i s, c]] is applied as c * [[1, i t], [i t, 1]]
// (t = tan beta) so each butterfly costs four FMAs; the accumulated factor c^k
// is folded into one multiply before the store ("fast" form). Angles with
// |tan beta| > 1 use the plain form.
#pragma once
#include "device.cuh"

namespace qaoa {

enum : uint8_t { SRC_SMEM_D = 0, SRC_GLOBAL_D = 1, SRC_INIT_D = 2 };
enum : uint8_t { DST_SMEM_D = 0, DST_GLOBAL_D = 1 };

struct PassArgs {
  void* state;            // 2^n amplitudes, interleaved (re, im)
  const int32_t* diag;    // int32 C(x) for all x (stream mode) or nullptr
  const void* phase;      // phase table of layer b: ncost complex entries
  const int32_t* wmat;    // n x n symmetric integer weights
  const int32_t* ctabs;   // per-round cost tables (recompute mode)
  double* partial;        // per-CTA [norm, <C>] partial sums (final pass)
  int phase_in_smem;      // copy the phase table into shared memory
};

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

template <int R, typename V, typename Real>
__device__ __forceinline__ void apply_mixer(V* v, uint8_t mask, Real tau, Real alpha, bool fast) {
#pragma unroll
  for (int i = 0; i < R; ++i) {
    if (mask >> i & 1) {
#pragma unroll
      for (int j = 0; j < (1 << R); ++j)
        if (!(j >> i & 1)) bfly<Real>(v[j], v[j | (1 << i)], tau, alpha, fast);
    }
  }
}

// Shared-memory layout of the dynamic buffer:
//   tile[2^T] complex | wmat[n*n] int | tile consts [16] int + base | phase table
template <typename Real, int R, int WB, bool FAST>
__global__ void __launch_bounds__(32 << WB, sizeof(Real) == 4 ? 2 : 1)
fwd_pass_kernel(const __grid_constant__ PassDev P, const PassArgs A) {
  using C2 = typename Cx<Real>::T;
  constexpr int T = R + 5 + WB;
  constexpr int NT = 32 << WB;
  constexpr int NA = 1 << R;
  constexpr int AB = sizeof(C2);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* tile = reinterpret_cast<C2*>(smem_raw);
  int* wsm = reinterpret_cast<int*>(tile + (1 << T));
  int* tconst = wsm + P.n * P.n;  // delta[0..15], base at [16]
  C2* ptab = reinterpret_cast<C2*>(smem_raw +
                                   (((size_t(1) << T) * AB + size_t(P.n * P.n + 32) * 4 + 15) & ~size_t(15)));

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

  double accN = 0.0, accC = 0.0;

  for (uint64_t unit = blockIdx.x; unit < P.n_units; unit += gridDim.x) {
    const uint64_t ubase = scatter_bits(unit, P.outer, P.nouter);
    for (int s = 0; s < P.nsub; ++s) {
      const SubDev& sp = P.sub[s];
      const uint64_t ntiles = 1ull << sp.ninner;
      for (uint64_t ti = 0; ti < ntiles; ++ti) {
        const uint64_t gbase = ubase | scatter_bits(ti, sp.inner, sp.ninner);
        __syncthreads();  // previous tile finished with shared memory
        if (sp.needs_c && !stream && warp == 0) tile_consts<T>(sp.pos, gbase, wsm, n, tconst, lane);
        if (sp.needs_c && !stream) __syncthreads();

        for (int r = 0; r < sp.nrounds; ++r) {
          const RoundDev& rd = sp.rd[r];
          if (rd.src == SRC_SMEM_D) __syncthreads();
          // thread's tile index over its lane / warp bits, and the matching
          // global offset and shared-memory slot
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
          } else if (rd.src == SRC_GLOBAL_D) {
#pragma unroll
            for (int j = 0; j < NA; ++j) v[j] = __ldcg(gstate + goff(j));
          } else {
#pragma unroll
            for (int j = 0; j < NA; ++j) v[j] = tile[soff(j)];
          }

          apply_mixer<R>(v, rd.mixA, Real(P.tauA), Real(P.alphaA), FAST);

          if (rd.cost | rd.reduce) {
            // C(x) of register amplitude j: streamed from the diagonal, or
            // kappa + CP[j] + sum_{i: j_i = 1} e_i from the round's tables
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
      }
      __syncthreads();  // sub-pass boundary: this CTA's global writes are visible to it
    }
  }

  if (A.partial) {
    // block reduction of the FP64 partial sums
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
