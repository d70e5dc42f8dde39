// small_kernel.cuh -- whole LR-QAOA circuit in one CTA's shared memory (n < 13).
//
// The state (2^n amplitudes) and its cut values C(x) stay in shared memory for
// all p layers: cost phase exp(-i gamma_k s (W - 2 C(x))) from the layer's
// phase table (Eqs. H_C, UC), then exp(+i beta_k X_q) on every qubit (Eq. UB),
// then the FP64 norm and <C> reductions and one write of the final state.
#pragma once
#include "device.cuh"

namespace qaoa {

struct SmallArgs {
  int n, p;
  void* state;
  const int32_t* wmat;
  const void* phase;     // p tables of ncost entries
  int c_lo, ncost;
  const double* betas;   // (gamma_k, beta_k) interleaved
  double* result;        // [norm, <C>]
};

template <typename Real>
__global__ void __launch_bounds__(512) small_circuit_kernel(const SmallArgs a) {
  using C2 = typename Cx<Real>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* s = reinterpret_cast<C2*>(smem_raw);
  __shared__ int cut[1 << 12];
  __shared__ double red[2][16];
  const int n = a.n, N = 1 << n, tid = threadIdx.x;
  const Real amp0 = Real(rsqrt(double(N)));
  for (int x = tid; x < N; x += 512) {
    int c = 0;
    for (int g = 0; g < n; ++g)
      for (int h = g + 1; h < n; ++h)
        if ((x >> g & 1) != (x >> h & 1)) c += a.wmat[g * n + h];
    cut[x] = c;
    s[x].x = amp0;
    s[x].y = Real(0);
  }
  const C2* ph = reinterpret_cast<const C2*>(a.phase);
  for (int k = 0; k < a.p; ++k) {
    __syncthreads();
    for (int x = tid; x < N; x += 512) {
      const C2 f = ph[(size_t)k * a.ncost + min(max(cut[x] - a.c_lo, 0), a.ncost - 1)];
      const Real xr = s[x].x, xi = s[x].y;
      s[x].x = xr * f.x - xi * f.y;
      s[x].y = xr * f.y + xi * f.x;
    }
    const double beta = a.betas[2 * k + 1];
    const Real cb = Real(cos(beta)), sb = Real(sin(beta));
    for (int q = 0; q < n; ++q) {
      __syncthreads();
      for (int i = tid; i < N / 2; i += 512) {
        const int x0 = ((i >> q) << (q + 1)) | (i & ((1 << q) - 1));
        const int x1 = x0 | (1 << q);
        const C2 p0 = s[x0], p1 = s[x1];
        s[x0].x = fma(cb, p0.x, -sb * p1.y);
        s[x0].y = fma(cb, p0.y, sb * p1.x);
        s[x1].x = fma(cb, p1.x, -sb * p0.y);
        s[x1].y = fma(cb, p1.y, sb * p0.x);
      }
    }
  }
  __syncthreads();
  double sn = 0.0, sc = 0.0;
  C2* g = reinterpret_cast<C2*>(a.state);
  for (int x = tid; x < N; x += 512) {
    const C2 v = s[x];
    const double pr = double(v.x) * double(v.x) + double(v.y) * double(v.y);
    sn += pr;
    sc += pr * double(cut[x]);
    g[x] = v;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sn += __shfl_xor_sync(0xffffffffu, sn, o);
    sc += __shfl_xor_sync(0xffffffffu, sc, o);
  }
  if ((tid & 31) == 0) { red[0][tid >> 5] = sn; red[1][tid >> 5] = sc; }
  __syncthreads();
  if (tid == 0) {
    double t0 = 0, t1 = 0;
    for (int w = 0; w < 16; ++w) { t0 += red[0][w]; t1 += red[1][w]; }
    a.result[0] = t0;
    a.result[1] = t1;
  }
}

}  // namespace qaoa
