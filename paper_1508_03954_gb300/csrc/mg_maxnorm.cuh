// mg_maxnorm.cuh -- maximum modulus of a complex vector (sm_103a), the max
// norm of the residual reductions of the Section 7.4 table.
#pragma once
#include "mg_kernels.cuh"

namespace mg {

// ---------------------------------------------------------------------------
// Maximum modulus of n complex values into *out, held as the bit pattern of a
// non-negative double (the patterns of non-negative doubles order like their
// values, so an integer atomicMax reduces them).  *out starts at 0.  A value
// that is not finite counts as +infinity, so a diverged residual reads as
// infinite rather than being skipped.
// ---------------------------------------------------------------------------
__global__ void max_abs_kernel(const cplx<double>* __restrict__ y, long long n,
                               unsigned long long* out) {
  double m = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const cplx<double> v = y[i];
    double a = sqrt(v.x * v.x + v.y * v.y);
    if (!(a <= 1.7976931348623157e308)) a = __longlong_as_double(0x7ff0000000000000LL);
    m = fmax(m, a);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

}  // namespace mg
