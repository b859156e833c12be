// mg_adjoint.cuh -- kernels of the adjoint (far-field functional) form.
//
// Forward: H(V) u = b = M f with k^2 = E - V per vertex, a cell using the mean
// of its vertex values.  Functional: s = sum_q g_q u(x_q) (d-linear samples),
// J = |s|^2.  With the adjoint H^T lambda = a (H is complex-symmetric, so
// this is H lambda = a, a_v = sum_q g_q psi_v(x_q)):
//   dJ/df_v = 2 Re( conj(s) (M lambda)_v )                      (f real)
//   dJ/dV_v = 2 Re( conj(s) * (-2^-d) sum_{c ni v} lambda_c^T M_c u_c )
// because dH/dV_v = +2^-d sum_{c ni v} M_c and ds/dp = lambda^T (db/dp - dH/dp u).
#pragma once
#include "mg_kernels.cuh"

namespace mg {

// Cell shift of a level from the fine k^2 field: phi_c = mean of k^2 at the
// cell's 2^D vertices, sampled on the level's own vertices (stride
// 3^(L - l) on the fine grid, fine row length NL).  The corners are summed in
// the same order as the host version, so both give the same values.
template <typename R, int D>
__global__ void cell_shift_kernel(int n, long long stride, long long NL, const double* __restrict__ k2,
                                  R* __restrict__ phic) {
  long long ncell = 1;
  for (int a = 0; a < D; ++a) ncell *= n;
  for (long long ci = blockIdx.x * (long long)blockDim.x + threadIdx.x; ci < ncell;
       ci += (long long)gridDim.x * blockDim.x) {
    long long q[3] = {0, 0, 0}, r = ci;
    for (int a = 0; a < D; ++a) { q[a] = r % n; r /= n; }
    double acc = 0.0;
    for (int e = 0; e < (1 << D); ++e) {
      long long gi = 0, st = 1;
      for (int a = 0; a < D; ++a) {
        gi += (q[a] + ((e >> a) & 1)) * stride * st;
        st *= NL;
      }
      acc += k2[gi];
    }
    phic[ci] = (R)(acc / (double)(1 << D));
  }
}

// q_c = lambda_c^T M_c u_c for every cell c of a 2D or 3D level (complex).
template <int D>
__global__ void cell_mass_form_kernel(int n, const cplx<double>* __restrict__ lam,
                                      const cplx<double>* __restrict__ u,
                                      const cplx<double>* __restrict__ hcell,
                                      cplx<double>* __restrict__ q) {
  const int N = n + 1;
  long long ncell = 1;
  for (int a = 0; a < D; ++a) ncell *= n;
  for (long long ci = blockIdx.x * (long long)blockDim.x + threadIdx.x; ci < ncell;
       ci += (long long)gridDim.x * blockDim.x) {
    int c[3];
    long long r = ci;
    for (int a = 0; a < D; ++a) { c[a] = (int)(r % n); r /= n; }
    cplx<double> acc = cz<double>();
    for (int ia = 0; ia < (1 << D); ++ia) {
      long long va = 0, st = 1;
      for (int a = 0; a < D; ++a) { va += (long long)(c[a] + ((ia >> a) & 1)) * st; st *= N; }
      cplx<double> row = cz<double>();
      for (int ib = 0; ib < (1 << D); ++ib) {
        long long vb = 0, sb = 1;
        cplx<double> w{1.0, 0.0};
        for (int a = 0; a < D; ++a) {
          const int ba = (ib >> a) & 1, aa = (ia >> a) & 1;
          vb += (long long)(c[a] + ba) * sb;
          sb *= N;
          w = w * rmul((aa == ba ? 2.0 : 1.0) / 6.0, hcell[c[a]]);
        }
        row = cfma(w, u[vb], row);
      }
      acc = cfma(lam[va], row, acc);
    }
    q[ci] = acc;
  }
}

// Per vertex: dJ/dV_v from the cell forms, dJ/df_v = 2 Re(conj(s) (M lam)_v).
template <int D>
__global__ void adjoint_grad_kernel(int n, const cplx<double>* __restrict__ lam,
                                    const cplx<double>* __restrict__ q,
                                    const cplx<double>* __restrict__ hcell, cplx<double> s,
                                    double* __restrict__ dJdV, double* __restrict__ dJdf) {
  const int N = n + 1;
  long long nv = 1;
  for (int a = 0; a < D; ++a) nv *= N;
  const cplx<double> sc{s.x, -s.y};  // conj(s)
  const double inv2d = 1.0 / (double)(1 << D);
  for (long long vi = blockIdx.x * (long long)blockDim.x + threadIdx.x; vi < nv;
       vi += (long long)gridDim.x * blockDim.x) {
    int g[3];
    unsigned r = (unsigned)vi;  // vertex counts stay below 2^32
    for (int a = 0; a < D; ++a) { g[a] = (int)(r % (unsigned)N); r /= (unsigned)N; }
    cplx<double> sq = cz<double>(), ml = cz<double>();
    for (int e = 0; e < (1 << D); ++e) {
      int c[3];
      bool in = true;
      long long ci = 0, cs = 1;
      for (int a = 0; a < D; ++a) {
        c[a] = g[a] - 1 + ((e >> a) & 1);
        in = in && c[a] >= 0 && c[a] < n;
        ci += (long long)c[a] * cs;
        cs *= n;
      }
      if (!in) continue;
      sq = sq + q[ci];
      // (M_c lam)(v): v is corner a = g - c of the cell
      for (int ib = 0; ib < (1 << D); ++ib) {
        long long vb = 0, sb = 1;
        cplx<double> w{1.0, 0.0};
        for (int a = 0; a < D; ++a) {
          const int ba = (ib >> a) & 1, aa = g[a] - c[a];
          vb += (long long)(c[a] + ba) * sb;
          sb *= N;
          w = w * rmul((aa == ba ? 2.0 : 1.0) / 6.0, hcell[c[a]]);
        }
        ml = cfma(w, lam[vb], ml);
      }
    }
    const cplx<double> gv = sc * rmul(-inv2d, sq);
    const cplx<double> gf = sc * ml;
    if (dJdV) dJdV[vi] = 2.0 * gv.x;
    if (dJdf) dJdf[vi] = 2.0 * gf.x;
  }
}

// s = sum_q w_q u(x_q), d-linear interpolation; deterministic block sum
// (one block, samples strided over threads, fixed-order reduction).
template <int D, int NTHR>
__global__ void sample_kernel(int n, int npts, const double* __restrict__ xyz,
                              const cplx<double>* __restrict__ w, const cplx<double>* __restrict__ u,
                              cplx<double>* __restrict__ out) {
  const int N = n + 1;
  __shared__ double sre[NTHR], sim[NTHR];
  cplx<double> acc = cz<double>();
  for (int p = threadIdx.x; p < npts; p += NTHR) {
    int i[3];
    double f[3];
    for (int a = 0; a < D; ++a) {
      double x = xyz[p * D + a] * n;
      int k = (int)floor(x);
      if (k < 0) k = 0;
      if (k > n - 1) k = n - 1;
      i[a] = k;
      f[a] = x - k;
    }
    cplx<double> v = cz<double>();
    for (int e = 0; e < (1 << D); ++e) {
      double wt = 1.0;
      long long vi = 0, st = 1;
      for (int a = 0; a < D; ++a) {
        const int b = (e >> a) & 1;
        wt *= b ? f[a] : 1.0 - f[a];
        vi += (long long)(i[a] + b) * st;
        st *= N;
      }
      v = rfma(wt, u[vi], v);
    }
    acc = cfma(w[p], v, acc);
  }
  sre[threadIdx.x] = acc.x;
  sim[threadIdx.x] = acc.y;
  __syncthreads();
  for (int o = NTHR / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sre[threadIdx.x] += sre[threadIdx.x + o];
      sim[threadIdx.x] += sim[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = cplx<double>{sre[0], sim[0]};
}

// b[idx[k]] = val[k] (indices distinct; the rest of b was cleared)
__global__ void scatter_kernel(int m, const long long* __restrict__ idx, const cplx<double>* __restrict__ val,
                               cplx<double>* __restrict__ b) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) b[idx[k]] = val[k];
}

}  // namespace mg
