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

// Whole adjoint gradient for small n (< 12) in one CTA's shared memory: the
// forward circuit as above, lambda = C psi, then for k = p-1..0 the terms
// -2 Im <lambda| X_q |psi> (before each qubit's inverse rotation) and
// 2 s Im sum_x conj(lambda_x) psi_x h(x) (at the inverse cost phase).
// grads: [g_gamma[0..p-1], g_beta[0..p-1], <C>, norm]. Angles (gamma_k, beta_k)
// interleaved in a.betas; a.scale_s = s; a.wsum = W.
struct SmallGradArgs {
  SmallArgs base;
  double scale_s;
  int wsum;
  double* grads;
};

template <typename Real>
__device__ __forceinline__ double block_sum512(double x, double* red) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  double t = 0;
  for (int w = 0; w < 16; ++w) t += red[w];
  return t;
}

template <typename Real>
__global__ void __launch_bounds__(512) small_grad_kernel(const SmallGradArgs ga) {
  using C2 = typename Cx<Real>::T;
  const SmallArgs& a = ga.base;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = a.n, N = 1 << n, tid = threadIdx.x;
  C2* s = reinterpret_cast<C2*>(smem_raw);
  C2* l = s + N;
  __shared__ int cut[1 << 11];
  __shared__ double red[16];
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
  double ec = 0.0, nr = 0.0;
  for (int x = tid; x < N; x += 512) {
    const double pr = double(s[x].x) * double(s[x].x) + double(s[x].y) * double(s[x].y);
    nr += pr;
    ec += pr * double(cut[x]);
    const Real c = Real(cut[x]);
    l[x].x = c * s[x].x;
    l[x].y = c * s[x].y;
  }
  ec = block_sum512<Real>(ec, red);
  nr = block_sum512<Real>(nr, red);
  if (tid == 0) { ga.grads[2 * a.p] = ec; ga.grads[2 * a.p + 1] = nr; }
  for (int k = a.p - 1; k >= 0; --k) {
    const double beta = a.betas[2 * k + 1];
    const Real cb = Real(cos(beta)), sb = Real(sin(beta));
    double tb = 0.0;
    for (int q = 0; q < n; ++q) {
      __syncthreads();
      for (int i = tid; i < N / 2; i += 512) {
        const int x0 = ((i >> q) << (q + 1)) | (i & ((1 << q) - 1));
        const int x1 = x0 | (1 << q);
        const C2 p0 = s[x0], p1 = s[x1], m0 = l[x0], m1 = l[x1];
        // Im(conj(l0) p1 + conj(l1) p0)
        tb += double(m0.x) * p1.y - double(m0.y) * p1.x + double(m1.x) * p0.y - double(m1.y) * p0.x;
        s[x0].x = fma(cb, p0.x, sb * p1.y);
        s[x0].y = fma(cb, p0.y, -sb * p1.x);
        s[x1].x = fma(cb, p1.x, sb * p0.y);
        s[x1].y = fma(cb, p1.y, -sb * p0.x);
        l[x0].x = fma(cb, m0.x, sb * m1.y);
        l[x0].y = fma(cb, m0.y, -sb * m1.x);
        l[x1].x = fma(cb, m1.x, sb * m0.y);
        l[x1].y = fma(cb, m1.y, -sb * m0.x);
      }
    }
    __syncthreads();
    double tg = 0.0;
    for (int x = tid; x < N; x += 512) {
      const C2 f = ph[(size_t)k * a.ncost + min(max(cut[x] - a.c_lo, 0), a.ncost - 1)];
      const C2 v = s[x], m = l[x];
      tg += (double(m.x) * v.y - double(m.y) * v.x) * double(ga.wsum - 2 * cut[x]);
      s[x].x = v.x * f.x + v.y * f.y;
      s[x].y = v.y * f.x - v.x * f.y;
      l[x].x = m.x * f.x + m.y * f.y;
      l[x].y = m.y * f.x - m.x * f.y;
    }
    tb = block_sum512<Real>(tb, red);
    tg = block_sum512<Real>(tg, red);
    if (tid == 0) {
      ga.grads[a.p + k] = -2.0 * tb;
      ga.grads[k] = 2.0 * ga.scale_s * tg;
    }
  }
}

}  // namespace qaoa
