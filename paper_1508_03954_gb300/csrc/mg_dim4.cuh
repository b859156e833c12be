// mg_dim4.cuh -- the cycle in four dimensions (p = 4 of Section 7.1), constant
// shift, sm_103a.  Templated on the arithmetic R: complex128 cycles, and the
// complex64 inner cycles of the defect-correction form.
//
// A d-linear 4D stencil row has 81 points and 256 vertex types, too many for
// the shared-memory tiles of the 2D/3D sweeps.  With coordinate-wise scaling
// and a constant shift the operator is a sum of tensor products of assembled
// 1D rows (Section 4 element matrices, one factor per axis):
//   H = M0 [M1 [M2 (K3 - phi M3) + K2 M3] + K1 M2 M3] + K0 M1 M2 M3,
// so H u is ten 3-tap passes along single axes; the Galerkin operator
// G = R H P of the coarse right-hand side has the same form with the 1D
// Galerkin rows, and R, P, I act axis by axis.  Every kernel here is one such
// pass over a 4D box (axis 0 fastest): coalesced, one thread per output
// vertex.  GB300 issues 2 FP64 FMA per clock per SM, about 3 per 32 bytes of
// HBM traffic, so the passes are bound by their FP64 work, not by memory:
// they count FP64 operations (real rows take real x complex products).  A
// pass zeroes its outputs on the two boundary planes of its own axis; the
// other coordinates carry through, so a chain of passes gives the interior
// rows of the product and zero Dirichlet rows.
#pragma once
#include "mg_kernels.cuh"

namespace mg {

struct Box4 {
  int n[4];  // extent per axis, axis 0 fastest
};

__device__ __forceinline__ unsigned box4_total(const Box4& B) {
  return (unsigned)B.n[0] * B.n[1] * B.n[2] * B.n[3];
}

__device__ __forceinline__ void box4_coords(unsigned i, const Box4& B, int* c) {
  c[0] = (int)(i % (unsigned)B.n[0]);
  i /= (unsigned)B.n[0];
  c[1] = (int)(i % (unsigned)B.n[1]);
  i /= (unsigned)B.n[1];
  c[2] = (int)(i % (unsigned)B.n[2]);
  c[3] = (int)(i / (unsigned)B.n[2]);
}

__device__ __forceinline__ unsigned box4_index(const Box4& B, const int* c) {
  return (((unsigned)c[3] * B.n[2] + c[2]) * B.n[1] + c[1]) * B.n[0] + c[0];
}

// True when the value is +0 or -0, tested on its bits: an FP64 comparison
// issues on the FP64 pipe, which the complex128 kernels are bound by
// (measured: a three-way imaginary-part test doubled the time of a pass).
__device__ __forceinline__ bool zero_bits(double v) {
  return (static_cast<unsigned long long>(__double_as_longlong(v)) << 1) == 0ull;
}
__device__ __forceinline__ bool zero_bits(float v) {
  return (static_cast<unsigned>(__float_as_int(v)) << 1) == 0u;
}

// y = b + (A x + z) or y = b - (A x + z) (neg), A the 3-tap rows along
// `axis` (rows[3 i + k] couples coordinate i with i - 1 + k); zero on the
// axis' boundary planes.  b and z may be null; y may alias b (element-wise
// update).  Real rows (cells outside the layer) take real x complex products,
// half the FMAs: REAL when every row of the table is real, else per row.
template <typename R, bool REAL>
__global__ void pass4_kernel(Box4 B, int axis, const cplx<R>* __restrict__ rows,
                             const cplx<R>* __restrict__ x, const cplx<R>* __restrict__ z,
                             const cplx<R>* b, cplx<R>* y, int neg) {
  const unsigned total = box4_total(B);
  unsigned s = 1;
  for (int a = 0; a < axis; ++a) s *= (unsigned)B.n[a];
  const int na = B.n[axis];
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int ca = (int)((i / s) % (unsigned)na);
    cplx<R> v = cz<R>();
    if (ca > 0 && ca < na - 1) {
      const cplx<R> r0 = rows[3 * ca], r1 = rows[3 * ca + 1], r2 = rows[3 * ca + 2];
      const cplx<R> xm = x[i - s], x0 = x[i], xp = x[i + s];
      if (REAL || (zero_bits(r0.y) && zero_bits(r1.y) && zero_bits(r2.y))) {
        v = rmul(r0.x, xm);
        v = rfma(r1.x, x0, v);
        v = rfma(r2.x, xp, v);
      } else {
        v = r0 * xm;
        v = cfma(r1, x0, v);
        v = cfma(r2, xp, v);
      }
      if (z != nullptr) v = v + z[i];
    }
    if (b != nullptr) {
      const cplx<R> bi = b[i];
      v = neg ? cplx<R>{bi.x - v.x, bi.y - v.y} : bi + v;
    } else if (neg) {
      v = cplx<R>{-v.x, -v.y};
    }
    y[i] = v;
  }
}

// Restriction R = P^T along `axis`: the output box is the input box with
// (n_f - 1)/3 + 1 points along the axis; coarse c collects fine 3c + o,
// o = -2..2, with weights 1 - |o|/3.  Zero on the axis' boundary planes.
template <typename R>
__global__ void restrict4_kernel(Box4 Bout, int axis, int nf, const cplx<R>* __restrict__ x,
                                 cplx<R>* __restrict__ y) {
  const unsigned total = box4_total(Bout);
  Box4 Bin = Bout;
  Bin.n[axis] = nf;
  unsigned s = 1;
  for (int a = 0; a < axis; ++a) s *= (unsigned)Bin.n[a];
  const int nc = Bout.n[axis];
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    int c[4];
    box4_coords(i, Bout, c);
    const int ca = c[axis];
    cplx<R> v = cz<R>();
    if (ca > 0 && ca < nc - 1) {
      c[axis] = 3 * ca;
      const unsigned j = box4_index(Bin, c);
      v = x[j];
      v = rfma(R(2.0 / 3.0), x[j - s], v);
      v = rfma(R(2.0 / 3.0), x[j + s], v);
      v = rfma(R(1.0 / 3.0), x[j - 2 * s], v);
      v = rfma(R(1.0 / 3.0), x[j + 2 * s], v);
    }
    y[i] = v;
  }
}

// d-linear interpolation along `axis`: the output box has n_f = 3 (n_c - 1) + 1
// points along the axis; fine 3c + o takes (1 - o/3) x[c] + (o/3) x[c+1].
// y = base + P x or base - P x (neg); base may be null, y may alias base.
template <typename R>
__global__ void prolong4_kernel(Box4 Bout, int axis, const cplx<R>* __restrict__ x, const cplx<R>* base,
                                cplx<R>* y, int neg) {
  const unsigned total = box4_total(Bout);
  Box4 Bin = Bout;
  Bin.n[axis] = (Bout.n[axis] - 1) / 3 + 1;
  unsigned s = 1;
  for (int a = 0; a < axis; ++a) s *= (unsigned)Bin.n[a];
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    int c[4];
    box4_coords(i, Bout, c);
    const int f = c[axis], o = f % 3;
    c[axis] = f / 3;
    const unsigned j = box4_index(Bin, c);
    cplx<R> v;
    if (o == 0) {
      v = x[j];
    } else {
      const R w0 = o == 1 ? R(2.0 / 3.0) : R(1.0 / 3.0), w1 = o == 1 ? R(1.0 / 3.0) : R(2.0 / 3.0);
      v = rmul(w0, x[j]);
      v = rfma(w1, x[j + s], v);
    }
    if (base != nullptr) {
      const cplx<R> bi = base[i];
      v = neg ? cplx<R>{bi.x - v.x, bi.y - v.y} : bi + v;
    } else if (neg) {
      v = cplx<R>{-v.x, -v.y};
    }
    y[i] = v;
  }
}

// Injection u_{l-1} = I u_l: coarse vertex C copies fine vertex 3C.
template <typename R>
__global__ void inject4_kernel(Box4 Bc, const cplx<R>* __restrict__ x, cplx<R>* __restrict__ y) {
  const unsigned total = box4_total(Bc);
  Box4 Bf;
  for (int a = 0; a < 4; ++a) Bf.n[a] = 3 * (Bc.n[a] - 1) + 1;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    int c[4];
    box4_coords(i, Bc, c);
    for (int a = 0; a < 4; ++a) c[a] *= 3;
    y[i] = x[box4_index(Bf, c)];
  }
}

// omd[t] = omega / D_t for the 256 vertex types of a level (one block).
template <typename R>
__global__ void omega_table4_kernel(const cplx<R>* __restrict__ invd, cplx<double> omega,
                                    cplx<R>* __restrict__ omd) {
  const int t = threadIdx.x;
  if (t < 256) omd[t] = cplx<R>{R(omega.x), R(omega.y)} * invd[t];
}

// du = omega D^{-1} r at interior vertices (omd: omega / D by vertex type),
// zero at c-points for the hierarchical basis variant and on the boundary;
// |r|^2 over the interior into *norm2 (deterministic last-block sum) when
// norm2 is not null.  REAL: every omega / D is real (real factor, no layer),
// two multiplies per vertex instead of a complex product -- the complex128
// step is bound by its FP64 operations, not by its 32 bytes per vertex.
template <typename R, bool REAL>
__global__ void __launch_bounds__(256) jacobi4_kernel(int n, const cplx<R>* __restrict__ r,
                                                      cplx<R>* __restrict__ t,
                                                      const uint8_t* __restrict__ typ,
                                                      const cplx<R>* __restrict__ omd, int hb,
                                                      double* partial, unsigned* ticket, double* norm2) {
  Box4 B;
  for (int a = 0; a < 4; ++a) B.n[a] = n + 1;
  const unsigned total = box4_total(B);
  double nrm = 0.0;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    int c[4];
    box4_coords(i, B, c);
    bool inner = true, cpt = true;
    int ty = 0;
#pragma unroll
    for (int a = 3; a >= 0; --a) {
      inner = inner && c[a] > 0 && c[a] < n;
      cpt = cpt && (c[a] % 3 == 0);
    }
    cplx<R> du = cz<R>();
    if (inner) {
#pragma unroll
      for (int a = 3; a >= 0; --a) ty = 4 * ty + (int)typ[c[a]];
      const cplx<R> ri = r[i];
      if (norm2 != nullptr) nrm = fma((double)ri.x, (double)ri.x, fma((double)ri.y, (double)ri.y, nrm));
      if (!(hb && cpt)) {
        const cplx<R> q = omd[ty];
        du = REAL ? rmul(q.x, ri) : q * ri;
      }
    }
    t[i] = du;
  }
  if (norm2 != nullptr) {
    __shared__ double s_red[8];
    block_norm_finish<256>(nrm, s_red, partial, ticket, norm2, gridDim.x);
  }
}

// |x|^2 over the interior of a level array (deterministic).
__global__ void __launch_bounds__(256) norm4_kernel(int n, const cplx<double>* __restrict__ x, double* partial,
                                                    unsigned* ticket, double* norm2) {
  Box4 B;
  for (int a = 0; a < 4; ++a) B.n[a] = n + 1;
  const unsigned total = box4_total(B);
  double nrm = 0.0;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const cplx<double> v = x[i];
    nrm = fma(v.x, v.x, fma(v.y, v.y, nrm));
  }
  __shared__ double s_red[8];
  block_norm_finish<256>(nrm, s_red, partial, ticket, norm2, gridDim.x);
}

// u += c at interior vertices (c in precision R, added in u's precision U);
// boundary vertices of u are set to zero.
template <typename U, typename R>
__global__ void update4_kernel(int n, cplx<U>* __restrict__ u, const cplx<R>* __restrict__ c) {
  Box4 B;
  for (int a = 0; a < 4; ++a) B.n[a] = n + 1;
  const unsigned total = box4_total(B);
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    int q[4];
    box4_coords(i, B, q);
    bool inner = true;
#pragma unroll
    for (int a = 0; a < 4; ++a) inner = inner && q[a] > 0 && q[a] < n;
    cplx<U> v = cz<U>();
    if (inner) {
      v = u[i];
      if (c != nullptr) {
        const cplx<R> ci = c[i];
        v = cplx<U>{v.x + U(ci.x), v.y + U(ci.y)};
      }
    }
    u[i] = v;
  }
}

// y = x converted to complex64 (the FP64 residual as the rhs of the inner
// complex64 problem of the defect-correction form).
__global__ void to_c64_kernel(long long n, const cplx<double>* __restrict__ x, cplx<float>* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const cplx<double> v = x[i];
    y[i] = cplx<float>{(float)v.x, (float)v.y};
  }
}

}  // namespace mg
