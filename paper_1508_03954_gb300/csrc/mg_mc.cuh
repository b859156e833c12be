// mg_mc.cuh -- kernels of the coupled multichannel cycle (Section 7.5),
// sm_103a.
//
// Every vertex carries a tuple of C channels, stored interleaved (vertex
// major, channel fastest), so one thread reads and writes a vertex's whole
// tuple as C consecutive complex values.  The operator is
//     (A u)_i = K u_i - sum_j Phi_ij M u_j        (i, j = 0 .. C-1),
// H_ii = K - phi_i M on the diagonal blocks and A_ij = -kappa_ij M off them
// (Phi: phi_i on its diagonal, kappa_ij off it), with the complex-scaled
// d-linear stiffness K and mass M of the single-channel path (Section 4,
// Appendix B), taken per vertex type from 3^D-point rows.  The smoother is
// damped block Jacobi, du_v = omega D_t^{-1} r_v with the C x C diagonal
// block D_t = K_t,centre I - Phi M_t,centre of the vertex's type t, inverted
// on the host.  Transfers act channel by channel.
//
// What bounds it: per vertex the two stencils cost 2 * 3^D * C real x
// complex MACs and the coupling C^2 complex MACs, all FP64, against 16 C
// bytes per array touched; on GB300 (2 FP64 FMA per clock per SM) the
// residual is bound by the FP64 pipe for every C.
#pragma once
#include "mg_kernels.cuh"

namespace mg {

constexpr int kMcThreads = 256;

template <int D> struct McPow3 { static constexpr int v = 3 * McPow3<D - 1>::v; };
template <> struct McPow3<0> { static constexpr int v = 1; };

// per-block FP64 partial sums of |r|^2 (read back and summed in block order
// by the host)
__device__ __forceinline__ void mc_block_sum(double v, double* partial) {
  __shared__ double s[kMcThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kMcThreads / 32; ++w) t += s[w];
    partial[blockIdx.x] = t;
  }
}

template <int D>
__device__ __forceinline__ void mc_coords(long long v, int N, int q[3]) {
  for (int a = 0; a < D; ++a) {
    q[a] = (int)(v % N);
    v /= N;
  }
}

// out = b - A x at interior vertices (zero on the boundary).  With jac != 0
// the output is the damped block-Jacobi update omega D_t^{-1} r instead (and
// zero at c-points when hb).  partial: |r|^2 per block (nullable).
template <int D, int C>
__global__ void __launch_bounds__(kMcThreads) mc_residual_kernel(
    int n, const cplx<double>* __restrict__ x, const cplx<double>* __restrict__ b, cplx<double>* __restrict__ out,
    const uint8_t* __restrict__ typ, const cplx<double>* __restrict__ Krow, const cplx<double>* __restrict__ Mrow,
    const cplx<double>* __restrict__ Phi, const cplx<double>* __restrict__ Dinv, int jac, cplx<double> omega,
    int hb, double* __restrict__ partial) {
  constexpr int NS = McPow3<D>::v;
  const int N = n + 1;
  long long total = 1;
  for (int a = 0; a < D; ++a) total *= N;
  double nrm = 0.0;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < total;
       v += (long long)gridDim.x * blockDim.x) {
    int q[3] = {0, 0, 0};
    mc_coords<D>(v, N, q);
    bool inner = true, cp = true;
    int t = 0, tw = 1;
    for (int a = 0; a < D; ++a) {
      inner = inner && q[a] > 0 && q[a] < n;
      cp = cp && q[a] % 3 == 0;
      t += tw * (int)typ[q[a]];
      tw *= 4;
    }
    cplx<double> r[C];
#pragma unroll
    for (int i = 0; i < C; ++i) r[i] = cz<double>();
    if (inner) {
      cplx<double> kx[C], mx[C];
#pragma unroll
      for (int i = 0; i < C; ++i) kx[i] = mx[i] = cz<double>();
      for (int s = 0; s < NS; ++s) {
        long long w = v, st = 1;
        int ss = s;
        for (int a = 0; a < D; ++a) {
          w += (long long)(ss % 3 - 1) * st;
          ss /= 3;
          st *= N;
        }
        const cplx<double> k = Krow[t * NS + s], m = Mrow[t * NS + s];
        const cplx<double>* xw = x + w * C;
#pragma unroll
        for (int i = 0; i < C; ++i) {
          const cplx<double> xi = xw[i];
          kx[i] = cfma(k, xi, kx[i]);
          mx[i] = cfma(m, xi, mx[i]);
        }
      }
#pragma unroll
      for (int i = 0; i < C; ++i) {
        cplx<double> ri = b[v * C + i] - kx[i];
#pragma unroll
        for (int j = 0; j < C; ++j) ri = cfma(Phi[i * C + j], mx[j], ri);
        r[i] = ri;
        nrm = fma(ri.x, ri.x, fma(ri.y, ri.y, nrm));
      }
    }
    cplx<double>* o = out + v * C;
    if (!jac) {
#pragma unroll
      for (int i = 0; i < C; ++i) o[i] = r[i];
    } else {
      const cplx<double>* Dt = Dinv + (size_t)t * C * C;
#pragma unroll
      for (int i = 0; i < C; ++i) {
        cplx<double> du = cz<double>();
        if (inner && !(hb && cp)) {
#pragma unroll
          for (int j = 0; j < C; ++j) du = cfma(Dt[i * C + j], r[j], du);
          du = omega * du;
        }
        o[i] = du;
      }
    }
  }
  if (partial != nullptr) mc_block_sum(nrm, partial);
}

// b = M f at interior vertices (zero on the boundary), channel by channel
template <int D, int C>
__global__ void __launch_bounds__(kMcThreads) mc_mass_kernel(int n, const cplx<double>* __restrict__ f,
                                                              cplx<double>* __restrict__ b,
                                                              const uint8_t* __restrict__ typ,
                                                              const cplx<double>* __restrict__ Mrow) {
  constexpr int NS = McPow3<D>::v;
  const int N = n + 1;
  long long total = 1;
  for (int a = 0; a < D; ++a) total *= N;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < total;
       v += (long long)gridDim.x * blockDim.x) {
    int q[3] = {0, 0, 0};
    mc_coords<D>(v, N, q);
    bool inner = true;
    int t = 0, tw = 1;
    for (int a = 0; a < D; ++a) {
      inner = inner && q[a] > 0 && q[a] < n;
      t += tw * (int)typ[q[a]];
      tw *= 4;
    }
    cplx<double> acc[C];
#pragma unroll
    for (int i = 0; i < C; ++i) acc[i] = cz<double>();
    if (inner) {
      for (int s = 0; s < NS; ++s) {
        long long w = v, st = 1;
        int ss = s;
        for (int a = 0; a < D; ++a) {
          w += (long long)(ss % 3 - 1) * st;
          ss /= 3;
          st *= N;
        }
        const cplx<double> m = Mrow[t * NS + s];
#pragma unroll
        for (int i = 0; i < C; ++i) acc[i] = cfma(m, f[w * C + i], acc[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < C; ++i) b[v * C + i] = acc[i];
  }
}

// dst = src at interior vertices, zero on the Dirichlet ring
template <int D, int C>
__global__ void __launch_bounds__(kMcThreads) mc_interior_kernel(int n, const cplx<double>* __restrict__ src,
                                                                  cplx<double>* __restrict__ dst) {
  const int N = n + 1;
  long long total = 1;
  for (int a = 0; a < D; ++a) total *= N;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < total;
       v += (long long)gridDim.x * blockDim.x) {
    int q[3] = {0, 0, 0};
    mc_coords<D>(v, N, q);
    bool inner = true;
    for (int a = 0; a < D; ++a) inner = inner && q[a] > 0 && q[a] < n;
#pragma unroll
    for (int i = 0; i < C; ++i) dst[v * C + i] = inner ? src[v * C + i] : cz<double>();
  }
}

// coarse c-point copy: uc(c) = uf(3c)
template <int D, int C>
__global__ void __launch_bounds__(kMcThreads) mc_inject_kernel(int nf, const cplx<double>* __restrict__ uf,
                                                                cplx<double>* __restrict__ uc) {
  const int Nf = nf + 1, Nc = nf / 3 + 1;
  long long total = 1;
  for (int a = 0; a < D; ++a) total *= Nc;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < total;
       c += (long long)gridDim.x * blockDim.x) {
    int q[3] = {0, 0, 0};
    mc_coords<D>(c, Nc, q);
    long long f = 0, st = 1;
    for (int a = 0; a < D; ++a) {
      f += 3LL * q[a] * st;
      st *= Nf;
    }
#pragma unroll
    for (int i = 0; i < C; ++i) uc[c * C + i] = uf[f * C + i];
  }
}

// d-linear tripartite prolongation of a coarse tuple field at fine vertex q
template <int D, int C>
__device__ __forceinline__ void mc_interp(const int q[3], int Nc, const cplx<double>* __restrict__ xc,
                                          cplx<double> out[C]) {
#pragma unroll
  for (int i = 0; i < C; ++i) out[i] = cz<double>();
  for (int e = 0; e < (1 << D); ++e) {
    double w = 1.0;
    long long c = 0, st = 1;
    bool ok = true;
    for (int a = 0; a < D; ++a) {
      const int cb = q[a] / 3, o = q[a] - 3 * cb, bit = (e >> a) & 1;
      const double wa = bit ? o / 3.0 : 1.0 - o / 3.0;
      if (wa == 0.0) ok = false;
      w *= wa;
      c += (long long)(cb + bit) * st;
      st *= Nc;
    }
    if (!ok) continue;
#pragma unroll
    for (int i = 0; i < C; ++i) out[i] = rfma(w, xc[c * C + i], out[i]);
  }
}

// hierarchical surplus uh = u - P uc
template <int D, int C>
__global__ void __launch_bounds__(kMcThreads) mc_surplus_kernel(int nf, const cplx<double>* __restrict__ u,
                                                                 const cplx<double>* __restrict__ uc,
                                                                 cplx<double>* __restrict__ uh) {
  const int Nf = nf + 1, Nc = nf / 3 + 1;
  long long total = 1;
  for (int a = 0; a < D; ++a) total *= Nf;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < total;
       v += (long long)gridDim.x * blockDim.x) {
    int q[3] = {0, 0, 0};
    mc_coords<D>(v, Nf, q);
    cplx<double> p[C];
    mc_interp<D, C>(q, Nc, uc, p);
#pragma unroll
    for (int i = 0; i < C; ++i) uh[v * C + i] = u[v * C + i] - p[i];
  }
}

// restriction R = P^T at interior coarse vertices (zero on the boundary)
template <int D, int C>
__global__ void __launch_bounds__(kMcThreads) mc_restrict_kernel(int nf, const cplx<double>* __restrict__ rf,
                                                                  cplx<double>* __restrict__ bc) {
  const int Nf = nf + 1, nc = nf / 3, Nc = nc + 1;
  long long total = 1;
  for (int a = 0; a < D; ++a) total *= Nc;
  constexpr int NT = D == 2 ? 25 : 125;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < total;
       c += (long long)gridDim.x * blockDim.x) {
    int q[3] = {0, 0, 0};
    mc_coords<D>(c, Nc, q);
    bool inner = true;
    for (int a = 0; a < D; ++a) inner = inner && q[a] > 0 && q[a] < nc;
    cplx<double> acc[C];
#pragma unroll
    for (int i = 0; i < C; ++i) acc[i] = cz<double>();
    if (inner) {
      for (int s = 0; s < NT; ++s) {
        double w = 1.0;
        long long f = 0, st = 1;
        int ss = s;
        for (int a = 0; a < D; ++a) {
          const int o = ss % 5 - 2;
          ss /= 5;
          w *= 1.0 - (o < 0 ? -o : o) / 3.0;
          f += (long long)(3 * q[a] + o) * st;
          st *= Nf;
        }
#pragma unroll
        for (int i = 0; i < C; ++i) acc[i] = rfma(w, rf[f * C + i], acc[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < C; ++i) bc[c * C + i] = acc[i];
  }
}

// corr_l = T t + P corr_{l-1} (corr_c nullable on level 1); T: hb masks the
// c-points, BPX subtracts P I t (I t: t at this level's c-points).  With
// add_to != null the result is added to that field (the finest level's u)
// instead of being stored in out.
template <int D, int C>
__global__ void __launch_bounds__(kMcThreads) mc_correct_kernel(int n, const cplx<double>* __restrict__ t,
                                                                 const cplx<double>* __restrict__ corr_c, int hb,
                                                                 int bpx, cplx<double>* __restrict__ out,
                                                                 cplx<double>* __restrict__ add_to) {
  const int N = n + 1, Nc = n / 3 + 1;
  long long total = 1;
  for (int a = 0; a < D; ++a) total *= N;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < total;
       v += (long long)gridDim.x * blockDim.x) {
    int q[3] = {0, 0, 0};
    mc_coords<D>(v, N, q);
    bool cp = true;
    for (int a = 0; a < D; ++a) cp = cp && q[a] % 3 == 0;
    cplx<double> c[C];
#pragma unroll
    for (int i = 0; i < C; ++i) c[i] = (hb && cp) ? cz<double>() : t[v * C + i];
    if (bpx) {
      // P I t: interpolate t from this level's c-points (masked ones are zero)
#pragma unroll
      for (int i = 0; i < C; ++i) {
        cplx<double> p = cz<double>();
        for (int e = 0; e < (1 << D); ++e) {
          double w = 1.0;
          long long f = 0, st = 1;
          for (int a = 0; a < D; ++a) {
            const int cb = q[a] / 3, o = q[a] - 3 * cb, bit = (e >> a) & 1;
            w *= bit ? o / 3.0 : 1.0 - o / 3.0;
            f += 3LL * (cb + bit < Nc ? cb + bit : cb) * st;
            st *= N;
          }
          if (w != 0.0 && !hb) p = rfma(w, t[f * C + i], p);
        }
        c[i] = c[i] - p;
      }
    }
    if (corr_c != nullptr) {
      cplx<double> p[C];
      mc_interp<D, C>(q, Nc, corr_c, p);
#pragma unroll
      for (int i = 0; i < C; ++i) c[i] = c[i] + p[i];
    }
    if (add_to != nullptr) {
#pragma unroll
      for (int i = 0; i < C; ++i) add_to[v * C + i] = add_to[v * C + i] + c[i];
    } else {
#pragma unroll
      for (int i = 0; i < C; ++i) out[v * C + i] = c[i];
    }
  }
}

}  // namespace mg
