// noise_kernels.cuh -- noisy LR-QAOA (Sec. II-C): a two-qubit depolarizing
// channel after every ZZ gate, sampled as stochastic trajectories, one CTA per
// trajectory with the state of n <= 12 qubits in shared memory (complex128, or
// complex64 with FP32 phases and butterflies; <C>_t and the norm in FP64).
//
// A sampled Pauli error is not applied to the state: it is kept in a Pauli
// frame F (bit masks fx, fz; the state is F|phi> up to a global phase) and
// the later gates act on |phi> conjugated by the frame, F^dag U F:
//   exp(-i theta Z_i Z_j) -> exp(-i sigma theta Z_i Z_j), sigma = (-1)^(fx_i + fx_j),
//   exp(+i beta X_q)      -> exp(+i tau beta X_q),       tau   = (-1)^(fz_q),
// since X and Y anticommute with Z, and Z and Y with X. A measurement of
// F|phi> returns x with probability |phi(x ^ fx)|^2, so
//   <C>_t = sum_y |phi(y)|^2 C(y ^ fx).
// The error draws (channel and Pauli) follow the rule of the oracle: gate
// g = k m + e of trajectory t takes draw t (p m) + g of stream `seed`; an
// error when (draw >> 11) 2^-53 < eps, then Pauli (draw & 3) on qubit u_e and
// ((draw >> 2) & 3) on v_e (0 I, 1 X, 2 Y, 3 Z).
#pragma once
#include <cstdint>

#include "aux_kernels.cuh"

namespace qaoa {

constexpr int kNoisyMaxQubits = 12;
constexpr int kNoisyMaxEdges = kNoisyMaxQubits * (kNoisyMaxQubits - 1) / 2;
constexpr int kNoisyThreads = 256;
constexpr int kNoisyLowBits = kNoisyMaxQubits - 8;  // log2(2^12 / kNoisyThreads)

struct NoisyArgs {
  int n = 0, m = 0, p = 0, trajectories = 0;
  const int32_t* u = nullptr;        // m edges (device)
  const int32_t* v = nullptr;
  const int32_t* w = nullptr;
  const double* theta = nullptr;     // p x m: gamma_k s w_e
  const double* beta = nullptr;      // p
  double eps = 0.0;
  unsigned long long seed = 0;
  double* exp_c = nullptr;           // per trajectory <C>_t
  double* norm = nullptr;            // per trajectory |phi|^2 (1 up to rounding)
};

__device__ __forceinline__ void sincos_t(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ void sincos_t(float x, float* s, float* c) { sincosf(x, s, c); }

// Dynamic shared memory: 2^n complex state, 2^n int32 cut values.
template <typename Real>
__global__ void __launch_bounds__(kNoisyThreads) noisy_trajectory_kernel(const NoisyArgs a) {
  using C2 = typename Cx<Real>::T;
  extern __shared__ __align__(16) unsigned char nsm[];
  const int n = a.n, m = a.m, N = 1 << n;
  C2* phi = reinterpret_cast<C2*>(nsm);
  int* cut = reinterpret_cast<int*>(phi + N);
  __shared__ Real sig[kNoisyMaxEdges];
  __shared__ Real sgn[kNoisyMaxEdges];
  __shared__ Real all[1 << kNoisyLowBits];
  __shared__ Real tau[kNoisyMaxQubits];
  __shared__ unsigned fxs;
  __shared__ int su[kNoisyMaxEdges], sv[kNoisyMaxEdges];
  __shared__ double red[2 * kNoisyThreads / 32];
  const int tid = threadIdx.x;
  // low bits per thread: L = 2^lb consecutive amplitudes (16 at n = 12)
  const int lb = n > 8 ? n - 8 : 0, L = 1 << lb;
  for (int e = tid; e < m; e += kNoisyThreads) {
    su[e] = a.u[e];
    sv[e] = a.v[e];
  }
  __syncthreads();
  for (int x = tid; x < N; x += kNoisyThreads) {
    int c = 0;
    for (int e = 0; e < m; ++e) c += ((x >> su[e]) ^ (x >> sv[e])) & 1 ? a.w[e] : 0;
    cut[x] = c;
  }
  for (int t = blockIdx.x; t < a.trajectories; t += gridDim.x) {
    const Real amp0 = Real(exp2(-0.5 * n));
    for (int x = tid; x < N; x += kNoisyThreads) {
      phi[x].x = amp0;
      phi[x].y = Real(0);
    }
    unsigned fx = 0, fz = 0;  // the frame, kept by thread 0
    for (int k = 0; k < a.p; ++k) {
      if (tid == 0) {
        const unsigned long long base = (unsigned long long)t * (unsigned long long)(a.p * m) +
                                        (unsigned long long)(k * m);
        for (int e = 0; e < m; ++e) {
          sig[e] = (((fx >> su[e]) ^ (fx >> sv[e])) & 1u) ? Real(-1) : Real(1);
          const unsigned long long d = splitmix_draw(a.seed, base + (unsigned long long)e);
          if (double(d >> 11) * 0x1.0p-53 < a.eps) {
            const unsigned pi = unsigned(d & 3ull), pj = unsigned(d >> 2 & 3ull);
            // X (1) and Y (2) carry an X part, Z (3) and Y a Z part
            if (pi == 1 || pi == 2) fx ^= 1u << su[e];
            if (pi == 2 || pi == 3) fz ^= 1u << su[e];
            if (pj == 1 || pj == 2) fx ^= 1u << sv[e];
            if (pj == 2 || pj == 3) fz ^= 1u << sv[e];
          }
        }
        for (int q = 0; q < n; ++q) tau[q] = (fz >> q & 1u) ? Real(-1) : Real(1);
      }
      __syncthreads();
      // cost layer with the frame's signs: phi_x *= exp(-i sum_e s_e z_a z_b),
      // s_e = sigma_e theta_e. A thread owns L = 2^lb consecutive x = x0 + j:
      //   angle = A_hh(x0) + A_ll(j) + sum_{i < lb} z_i(j) h_i(x0)
      // with A_hh the edges among bits >= lb, A_ll (a table per layer) those
      // among bits < lb, and h_i the cross edges of low bit i.
      const double* th = a.theta + (size_t)k * m;
      for (int e = tid; e < m; e += kNoisyThreads) sgn[e] = sig[e] * Real(th[e]);
      __syncthreads();
      if (tid < L) {
        Real al = 0;
        for (int e = 0; e < m; ++e)
          if (su[e] < lb && sv[e] < lb) al += (((tid >> su[e]) ^ (tid >> sv[e])) & 1) ? -sgn[e] : sgn[e];
        all[tid] = al;
      }
      __syncthreads();
      const int x0 = tid * L;
      if (x0 < N) {
        Real ahh = 0, h[kNoisyLowBits] = {0, 0, 0, 0};
        for (int e = 0; e < m; ++e) {
          const int ea = su[e], eb = sv[e];
          const Real se = sgn[e];
          if (ea >= lb && eb >= lb) {
            ahh += (((x0 >> ea) ^ (x0 >> eb)) & 1) ? -se : se;
          } else if (ea >= lb || eb >= lb) {
            const int lo = ea < lb ? ea : eb, hi = ea < lb ? eb : ea;
#pragma unroll
            for (int i = 0; i < kNoisyLowBits; ++i)
              if (i == lo) h[i] += (x0 >> hi & 1) ? -se : se;
          }
        }
        for (int j = 0; j < L; ++j) {
          Real ang = ahh + all[j];
#pragma unroll
          for (int i = 0; i < kNoisyLowBits; ++i)
            if (i < lb) ang += (j >> i & 1) ? -h[i] : h[i];
          Real sn, cs;
          sincos_t(ang, &sn, &cs);
          const C2 f = phi[x0 + j];
          phi[x0 + j].x = f.x * cs + f.y * sn;
          phi[x0 + j].y = f.y * cs - f.x * sn;
        }
      }
      // mixer exp(+i tau_q beta_k X_q), qubit by qubit
      double sbd, cbd;
      sincos(a.beta[k], &sbd, &cbd);
      const Real sb = Real(sbd), cb = Real(cbd);
      for (int q = 0; q < n; ++q) {
        __syncthreads();
        const Real s = tau[q] * sb;
        for (int pr = tid; pr < N / 2; pr += kNoisyThreads) {
          const int lo = pr & ((1 << q) - 1);
          const int xa = ((pr >> q) << (q + 1)) | lo, xb = xa | (1 << q);
          const C2 pa = phi[xa], pb = phi[xb];
          // a' = c a + i s b, b' = i s a + c b
          phi[xa].x = cb * pa.x - s * pb.y;
          phi[xa].y = cb * pa.y + s * pb.x;
          phi[xb].x = cb * pb.x - s * pa.y;
          phi[xb].y = cb * pb.y + s * pa.x;
        }
      }
      if (tid == 0) fxs = fx;
      __syncthreads();
    }
    if (a.p == 0) {
      if (tid == 0) fxs = 0;
      __syncthreads();
    }
    // <C>_t = sum_y |phi(y)|^2 C(y ^ fx), and the norm
    const unsigned f = fxs;
    double ec = 0.0, nr = 0.0;
    for (int x = tid; x < N; x += kNoisyThreads) {
      const C2 z = phi[x];
      const double pr = double(z.x) * z.x + double(z.y) * z.y;
      nr += pr;
      ec += pr * double(cut[x ^ (int)f]);
    }
    for (int o = 16; o > 0; o >>= 1) {
      ec += __shfl_xor_sync(0xffffffffu, ec, o);
      nr += __shfl_xor_sync(0xffffffffu, nr, o);
    }
    if ((tid & 31) == 0) {
      red[2 * (tid >> 5)] = ec;
      red[2 * (tid >> 5) + 1] = nr;
    }
    __syncthreads();
    if (tid == 0) {
      double se = 0.0, sn = 0.0;
      for (int wi = 0; wi < kNoisyThreads / 32; ++wi) {
        se += red[2 * wi];
        sn += red[2 * wi + 1];
      }
      a.exp_c[t] = se;
      if (a.norm) a.norm[t] = sn;
    }
    __syncthreads();  // the next trajectory reuses phi, fxs and red
  }
}

}  // namespace qaoa
