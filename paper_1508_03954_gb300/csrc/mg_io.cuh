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

}  // namespace mg
