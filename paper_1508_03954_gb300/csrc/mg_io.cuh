// mg_io.cuh -- host <-> device transfers of level arrays through the SMs
// (sm_103a).  On a GB300 the GPU reads and writes page-locked host memory
// directly over the host link; for the 8-16 MB arrays of one solve this moves
// data faster than a staged cudaMemcpyAsync, and it lets a transfer carry
// work of its own (zeroing the Dirichlet ring on the way in).
#pragma once
#include "mg_kernels.cuh"

namespace mg {

// dst = src (n complex128 values, 16-byte loads and stores).
__global__ void copy_c128_kernel(long long n, const cplx<double>* __restrict__ src,
                                 cplx<double>* __restrict__ dst) {
  const double2* s = reinterpret_cast<const double2*>(src);
  double2* d = reinterpret_cast<double2*>(dst);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    d[i] = s[i];
}

// dst = src with the Dirichlet ring (vertices with a coordinate 0 or n) set
// to zero; a level array of (n + 1)^D values.
template <int D>
__global__ void copy_zero_ring_kernel(int n, const cplx<double>* __restrict__ src,
                                      cplx<double>* __restrict__ dst) {
  const unsigned N = (unsigned)n + 1;
  unsigned total = 1;
  for (int a = 0; a < D; ++a) total *= N;
  const double2* s = reinterpret_cast<const double2*>(src);
  double2* d = reinterpret_cast<double2*>(dst);
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    unsigned r = i;
    bool inner = true;
    for (int a = 0; a < D; ++a) {
      const unsigned g = r % N;
      r /= N;
      inner = inner && g > 0 && g < (unsigned)n;
    }
    d[i] = inner ? s[i] : make_double2(0.0, 0.0);
  }
}

// The 1D mass rows (h_l / 6, (h_l + h_r) / 3, h_r / 6) of the four axis
// classes (left / right cell in the scaling layer); bit t of `real`: class t
// has a real row.
struct MassRows3 {
  cplx<double> m[4][3];
  unsigned real;
};

// One pass of the assembled mass matrix along axis AX (0 = x, 1 = y, 2 = z) of
// a 3D level array with n + 1 points per axis: y = M_AX x at vertices inside
// along AX, zero on that axis's Dirichlet planes.  With coordinate-wise
// scaling every cell's mass matrix is the tensor product of 1D ones (Section
// 4: M_c = (x)_a M), so b = M f is three such passes, about 20 FP64 operations
// per vertex against 54-108 for the 27-point rows.  x is read at stride xs
// along every axis of an array with xs n + 1 points per axis (the fine f that
// a coarser level samples; xs = 1 for a level array).
template <int AX>
__global__ void mass_pass3_kernel(int n, int xs, const cplx<double>* __restrict__ x,
                                  cplx<double>* __restrict__ y, const uint8_t* __restrict__ typ,
                                  const MassRows3 rows) {
  const int N = n + 1;
  const long long total = (long long)N * N * N;
  const long long Nx = (long long)xs * n + 1;
  const long long st = (long long)xs * (AX == 0 ? 1 : (AX == 1 ? Nx : Nx * Nx));
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int g0 = (int)(i % N), g1 = (int)((i / N) % N), g2 = (int)(i / ((long long)N * N));
    const int ga = AX == 0 ? g0 : (AX == 1 ? g1 : g2);
    const bool in = ga > 0 && ga < n;
    const int t = in ? typ[ga] : 0;
    // one path per warp (the complex one gives real rows the same result):
    // along x a warp often holds both classes
    const bool wreal = __all_sync(__activemask(), ((rows.real >> t) & 1u) != 0u);
    cplx<double> v = cz<double>();
    if (in) {
      const long long j = (((long long)g2 * xs) * Nx + (long long)g1 * xs) * Nx + (long long)g0 * xs;
      const cplx<double> a = x[j - st], b = x[j], d = x[j + st];
      if (wreal)
        v = rfma(rows.m[t][2].x, d, rfma(rows.m[t][1].x, b, rmul(rows.m[t][0].x, a)));
      else
        v = cfma(rows.m[t][2], d, cfma(rows.m[t][1], b, rows.m[t][0] * a));
    }
    y[i] = v;
  }
}

// The z-pass of b = M f fused with the copy of f from page-locked host memory:
// one thread per (x, y) column marches along z, reads each value of f over
// the host link once, stores it into fcopy (the device copy later passes and
// FMG stages sample) and stores y = M_z f (zero on the z = 0 and z = n
// planes).  The z-pass arithmetic is that of mass_pass3_kernel<2>, so b is
// bit for bit the same as from a staged copy; the pass costs no time of its
// own, since the host link is the slower part.
__global__ void mass_z_copy_kernel(int n, const cplx<double>* __restrict__ f, cplx<double>* __restrict__ fcopy,
                                   cplx<double>* __restrict__ y, const uint8_t* __restrict__ typ,
                                   const MassRows3 rows) {
  const int N = n + 1;
  const long long NN = (long long)N * N;
  for (long long col = blockIdx.x * (long long)blockDim.x + threadIdx.x; col < NN;
       col += (long long)gridDim.x * blockDim.x) {
    cplx<double> fm = f[col], f0 = f[NN + col];
    fcopy[col] = fm;
    fcopy[NN + col] = f0;
    y[col] = cz<double>();
    for (int z = 1; z < n; ++z) {
      const cplx<double> fp = f[(long long)(z + 1) * NN + col];
      fcopy[(long long)(z + 1) * NN + col] = fp;
      const int t = typ[z];  // one class per plane: every lane takes the same path
      cplx<double> v;
      if ((rows.real >> t) & 1u)
        v = rfma(rows.m[t][2].x, fp, rfma(rows.m[t][1].x, f0, rmul(rows.m[t][0].x, fm)));
      else
        v = cfma(rows.m[t][2], fp, cfma(rows.m[t][1], f0, rows.m[t][0] * fm));
      y[(long long)z * NN + col] = v;
      fm = f0;
      f0 = fp;
    }
    y[(long long)n * NN + col] = cz<double>();
  }
}

}  // namespace mg
