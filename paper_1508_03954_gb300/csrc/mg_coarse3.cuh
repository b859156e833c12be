// mg_coarse3.cuh -- coarse 3D levels with a constant shift, one thread (or a
// small group of lanes) per vertex, and the separable 3D corrections (sm_103a).
//
// The step is the one of the level sweeps (Appendix A Algorithm 4 on a coarse
// level l: r_l = b_l - H_l u_l, du_l = omega_l D_l^{-1} r_l, the c-point mask
// of hb, u_{l-1} = I u_l), but the coarse right-hand side is formed by the
// next coarser level's kernel from the stored residual instead of inside a
// z-marching tile:
//     b_{l-1} = R r_l + G_{l-1} u_{l-1}     (G = R H P, Eq. HTMG by linearity)
// so a level is one launch over its (3^l + 1)^3 vertices with no halo, no
// plane pipeline and no warm-up: the small levels of a 3D hierarchy (at most a
// few hundred thousand vertices) are latency-bound in a marching sweep, whose
// blocks each walk several planes in series while most SMs idle.
//
// With the BPX transfer (and no hb mask) the kernel stores du_l and its
// c-point values I du_l on the coarser grid; the correction stage forms
// corr_l = du_l + P (corr_{l-1} - I du_l), which equals (id - P I) du_l +
// P corr_{l-1} by linearity of P (Section 5, BPX as the hierarchical
// transfer).
#pragma once
#include "mg_kernels.cuh"
#include "mg_sweep3d.cuh"
#include "mg_defect3.cuh"

namespace mg {

template <typename R>
struct Coarse3Args {
  int n;                     // level l: 3^l cells per axis
  int fused;                 // form b_l = R r_{l+1} + G_l u_l here (else read b)
  int has_coarse;            // l > 1: store r_l and u_{l-1} = I u_l
  int hb;                    // c-point mask of du
  unsigned long long realrow;  // bit t: H row of vertex type t is real
  unsigned greal;            // bit k: 1D Galerkin row class k is real
  const cplx<R>* u;          // u_l (the injected copy of the finer level)
  cplx<R>* b;                // b_l: read, or written when fused
  const cplx<R>* rf;         // r_{l+1} (fused)
  const uint8_t* gtyp;       // Galerkin row class per level-l index (fused)
  const cplx<R>* gcoef;      // [kMaxG3^3][27] rows of G_l (fused)
  const uint8_t* typ;        // vertex type per level-l index
  const cplx<R>* coef;       // [64][27] rows of H_l
  cplx<R> omd[64];           // omega_l / D_l per vertex type
  cplx<R>* r;                // r_l (has_coarse)
  cplx<R>* t;                // du_l, c-points zeroed for hb
  cplx<R>* idu;              // I du_l on level l-1 (BPX; may be null)
  cplx<R>* u_coarse;         // u_{l-1} (has_coarse)
};

// Partial sum of the 27-point row at vertex i (N points per axis) over the
// entries k = q, q + LPV, ...; neighbour k at offset (k % 3 - 1, k / 3 % 3 - 1,
// k / 9 - 1).
template <typename R, int LPV, bool REAL>
__device__ __forceinline__ cplx<R> row27_part(const cplx<R>* __restrict__ cf, const cplx<R>* __restrict__ v,
                                              long long i, int N, int q, cplx<R> acc) {
  const long long NN = (long long)N * N;
#pragma unroll
  for (int m = 0; m < (27 + LPV - 1) / LPV; ++m) {
    const int k = q + m * LPV;
    if (LPV == 1 || k < 27) {
      const long long j = i + (k % 3 - 1) + (long long)(k / 3 % 3 - 1) * N + (k / 9 - 1) * NN;
      const cplx<R> a = ldg_c(v + j);
      if (REAL) acc = rfma(__ldg(&cf[k].x), a, acc);
      else acc = cfma(ldg_c(cf + k), a, acc);
    }
  }
  return acc;
}

template <typename R>
__device__ __forceinline__ cplx<R> shfl_xor_c(cplx<R> v, int o) {
  return cplx<R>{__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o)};
}

// LPV lanes share a vertex: each sums a share of the restriction taps and of
// the row entries, and the shares are combined by shuffles.  A single
// thread's chain of ~400 dependent FP64 operations, at one FP64 warp
// instruction per 64 cycles of a sub-partition, makes the few-thousand-vertex
// levels latency-bound; the lane groups shorten it for the small levels
// (LPV = 1 on levels large enough to fill the GPU).
template <typename R, int LPV>
__global__ void __launch_bounds__(128) coarse3_kernel(const Coarse3Args<R> A) {
  using C = cplx<R>;
  constexpr int VPW = 32 / LPV;  // vertices per warp and pass
  const int n = A.n, N = n + 1, Nc = n / 3 + 1;
  const long long total = (long long)N * N * N;
  const int lane = threadIdx.x & 31, q = lane % LPV;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = warp * VPW; base < total; base += nwarps * VPW) {  // warp-uniform trip count
    const long long i = base + lane / LPV;
    const bool valid = i < total;
    const long long iv = valid ? i : 0;
    const int x = (int)(iv % N), y = (int)((iv / N) % N), z = (int)(iv / ((long long)N * N));
    const bool inner = valid && x > 0 && x < n && y > 0 && y < n && z > 0 && z < n;
    const int ty = inner ? (int)A.typ[x] + 4 * (int)A.typ[y] + 16 * (int)A.typ[z] : 0;
    int gt = 0;
    bool greal = true;
    if (inner && A.fused) {
      const int G = kMaxG3;
      const int gx = A.gtyp[x], gy = A.gtyp[y], gz = A.gtyp[z];
      gt = gx + G * (gy + G * gz);
      greal = (((A.greal >> gx) & (A.greal >> gy) & (A.greal >> gz)) & 1u) != 0u;
    }
    // one path per warp: a warp at a layer edge holds real and complex rows,
    // and the complex path gives real rows the same sums (zero imaginary
    // parts), so taking it for the whole warp avoids running both
    const bool hreal = __all_sync(0xffffffffu, !inner || ((A.realrow >> ty) & 1ull) != 0ull);
    const bool greal_w = __all_sync(0xffffffffu, greal);
    C pb = cz<R>(), ph = cz<R>();
    if (inner) {
      if (A.fused) {
        // R r_{l+1}: 5^3 taps of the tripartite weights (3 - |o|) / 3 per axis,
        // integer products summed, one division by 27 at the end; this lane's
        // share is the (z, y) rows q, q + LPV, ...
        const int Nf = 3 * n + 1;
        const C* rf = A.rf + ((long long)(3 * z - 2) * Nf + (3 * y - 2)) * Nf + (3 * x - 2);
#pragma unroll
        for (int m = 0; m < (25 + LPV - 1) / LPV; ++m) {
          const int rr = q + m * LPV;
          if (LPV == 1 || rr < 25) {
            const int oz = rr / 5, oy = rr % 5;
            const C* p = rf + ((long long)oz * Nf + oy) * Nf;
            C row = rfma(R(2), ldg_c(p + 1), ldg_c(p));
            row = rfma(R(3), ldg_c(p + 2), row);
            row = rfma(R(2), ldg_c(p + 3), row);
            row = row + ldg_c(p + 4);
            pb = rfma(R((3 - abs(oz - 2)) * (3 - abs(oy - 2))), row, pb);
          }
        }
        pb = rmul(R(1) / R(27), pb);
        // + G_l u_l: the Galerkin row of the vertex's three 1D classes
        const C* gc = A.gcoef + gt * 27;
        if (greal_w)
          pb = row27_part<R, LPV, true>(gc, A.u, i, N, q, pb);
        else
          pb = row27_part<R, LPV, false>(gc, A.u, i, N, q, pb);
      }
      const C* cf = A.coef + ty * 27;
      ph = hreal ? row27_part<R, LPV, true>(cf, A.u, i, N, q, ph) : row27_part<R, LPV, false>(cf, A.u, i, N, q, ph);
    }
#pragma unroll
    for (int o = LPV / 2; o > 0; o >>= 1) {
      pb = pb + shfl_xor_c(pb, o);
      ph = ph + shfl_xor_c(ph, o);
    }
    if (q != 0 || !valid) continue;
    const bool cpt = x % 3 == 0 && y % 3 == 0 && z % 3 == 0;
    C rv = cz<R>(), du = cz<R>();
    if (inner) {
      C bv;
      if (A.fused) {
        bv = pb;
        A.b[i] = bv;
      } else {
        bv = A.b[i];
      }
      rv = bv - ph;
      du = A.omd[ty] * rv;
      if (A.hb && cpt) du = cz<R>();
    } else if (A.fused) {
      A.b[i] = cz<R>();
    }
    if (A.has_coarse) {
      A.r[i] = rv;
      if (cpt) {
        const long long ci = ((long long)(z / 3) * Nc + y / 3) * Nc + x / 3;
        A.u_coarse[ci] = inner ? A.u[i] : cz<R>();
        if (A.idu != nullptr) A.idu[ci] = du;
      }
    }
    A.t[i] = du;
  }
}

// corr_l = t_l + P (c - sub_c) - sub_f on a 3D level (sub_c, sub_f may be
// null): the tensor-product prolongation taken one axis at a time on a tile
// of 9^3 fine vertices in shared memory (4^3 coarse corners -> x -> y -> z),
// with the integer weights 3 - o and o of the tripartite interpolation and
// one division by 27 at the end.  About 6 FP64 operations per fine vertex
// against 16-32 for the 2^3 corner products formed per vertex.
template <typename R>
__global__ void __launch_bounds__(256) prolong3_kernel(int n, const cplx<R>* __restrict__ t,
                                                       const cplx<R>* __restrict__ cc,
                                                       cplx<R>* __restrict__ out,
                                                       const cplx<R>* __restrict__ sub_c,
                                                       const cplx<R>* __restrict__ sub_f) {
  using C = cplx<R>;
  __shared__ C s_c[4][4][4];
  __shared__ C s_x[4][4][9];
  __shared__ C s_y[4][9][9];
  const int N = n + 1, nc = n / 3, Nc = nc + 1;
  const int tiles = (N + 8) / 9;
  int b = blockIdx.x;
  const int TX = b % tiles;
  b /= tiles;
  const int TY = b % tiles, TZ = b / tiles;
  for (int i = threadIdx.x; i < 64; i += blockDim.x) {
    const int cx = 3 * TX + (i & 3), cy = 3 * TY + ((i >> 2) & 3), cz_ = 3 * TZ + (i >> 4);
    C v = cz<R>();
    if (cx <= nc && cy <= nc && cz_ <= nc) {
      const long long ci = ((long long)cz_ * Nc + cy) * Nc + cx;
      v = cc[ci];
      if (sub_c != nullptr) v = v - sub_c[ci];
    }
    s_c[i >> 4][(i >> 2) & 3][i & 3] = v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 144; i += blockDim.x) {
    const int ox = i % 9, jy = (i / 9) & 3, jz = i / 36, j = ox / 3, o = ox % 3;
    s_x[jz][jy][ox] = rfma(R(o), s_c[jz][jy][j + 1], rmul(R(3 - o), s_c[jz][jy][j]));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 324; i += blockDim.x) {
    const int ox = i % 9, oy = (i / 9) % 9, jz = i / 81, j = oy / 3, o = oy % 3;
    s_y[jz][oy][ox] = rfma(R(o), s_x[jz][j + 1][ox], rmul(R(3 - o), s_x[jz][j][ox]));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 729; i += blockDim.x) {
    const int ox = i % 9, oy = (i / 9) % 9, oz = i / 81;
    const int gx = 9 * TX + ox, gy = 9 * TY + oy, gz = 9 * TZ + oz;
    if (gx > n || gy > n || gz > n) continue;
    const long long gi = ((long long)gz * N + gy) * N + gx;
    C v = cz<R>();
    if (gx > 0 && gx < n && gy > 0 && gy < n && gz > 0 && gz < n) {
      const int j = oz / 3, o = oz % 3;
      const C p = rfma(R(o), s_y[j + 1][oy][ox], rmul(R(3 - o), s_y[j][oy][ox]));
      v = rfma(R(1) / R(27), p, t[gi]);
      if (sub_f != nullptr) v = v - sub_f[gi];
    }
    out[gi] = v;
  }
}

}  // namespace mg
