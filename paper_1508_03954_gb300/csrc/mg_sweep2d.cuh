// mg_sweep2d.cuh -- FP64 fine-to-coarse sweep for 2D levels with a constant
// shift (sm_103a).
//
// Same step as sweep_kernel (Appendix A Algorithm 4 on one level, plus the
// single-touch pending correction of Algorithm 2), arranged to spend as few
// FP64 instructions as possible, because GB300 issues only 2 FP64 FMA per
// clock per SM:
//  * the coarse right-hand side uses b_{l-1} = R r_l + G_{l-1} u_{l-1} with
//    G_{l-1} = R H_l P (on interior unknowns).  Since uhat = u - P I u and
//    u_{l-1} = I u_l, R(b_l - H_l uhat_l) = R r_l + R H_l P u_{l-1}: the
//    same quantity as Eq. HTMG, without a second fine stencil.  G has a 3x3
//    row per coarse vertex that is a tensor product of 1D Galerkin rows; the
//    host tabulates it per pair of 1D row classes.
//  * stencil rows that are real (cells outside the scaling layer) use
//    real x complex products;
//  * interpolation (P c, P I du) and restriction are separable two-pass
//    operations in shared memory with the tripartite weights selected, not
//    multiplied.
#pragma once
#include "mg_kernels.cuh"

namespace mg {

constexpr int kMaxGTypes = 8;  // 1D Galerkin row classes per axis

template <typename R>
struct Sweep2Args {
  int n, fine, has_coarse, hb, hier, tiles_x;
  int first;              // fine: U is zero and nothing is pending (first inner cycle)
  int ntiles;             // tiles of this level (last-tile norm reduction)
  unsigned realrow;      // bit t: stencil row of vertex type t is real
  unsigned realjac;      // bit t: omega/D of type t is real
  const cplx<R>* u;
  const cplx<R>* c;       // pending correction on level l-1 (fine, may be null)
  const cplx<R>* b;
  cplx<R>* out;
  cplx<R>* b_coarse;
  cplx<R>* u_coarse;
  const uint8_t* typ;     // vertex type per fine index (n+1)
  const uint8_t* gtyp;    // Galerkin row class per coarse index (n/3+1)
  const cplx<R>* coef;    // [16][9]
  const cplx<R>* gcoef;   // [kMaxGTypes^2][9], index gx + kMaxGTypes*gy
  cplx<R> omd[16];
  double* partial;
  unsigned* ticket;
  double* norm2;
};

template <int TC, typename R = double>
struct Tile2 {
  static constexpr int F = 3 * TC;
  static constexpr int SU = F + 5;   // u box [x0-3, x0+F+1]
  static constexpr int SR = F + 3;   // r box [x0-2, x0+F]
  static constexpr int SC = TC + 3;  // pending-correction box [C0-1, C0+TC+1]
  static constexpr int SD = TC + 1;  // c-point du box [C0, C0+TC]
  // region A holds the pending correction (P0-P2), then the restriction and
  // P I du buffers (P4-P6)
  static constexpr size_t A1 = (size_t)SC * SC + (size_t)SC * SU;
  static constexpr size_t A2 = (size_t)(F + 2) * TC + (size_t)SD * SD + (size_t)SD * F;
  static constexpr size_t AR = A1 > A2 ? A1 : A2;
  static constexpr size_t smem_cplx = AR + (size_t)SU * SU + (size_t)SR * SR + 16 * 9 + 16;
  static constexpr size_t smem_bytes = smem_cplx * sizeof(cplx<R>) + 2 * SU;
};

template <typename R = double>
__device__ __forceinline__ R w0(int o) { return o == 0 ? R(1) : (o == 1 ? R(2) / R(3) : R(1) / R(3)); }
template <typename R = double>
__device__ __forceinline__ R w1(int o) { return o == 0 ? R(0) : (o == 1 ? R(1) / R(3) : R(2) / R(3)); }
// a*s0 + b*s1 (real weights)
template <typename R>
__device__ __forceinline__ cplx<R> lerp2(R s0, cplx<R> a, R s1, cplx<R> b) {
  return cplx<R>{fma(s1, b.x, s0 * a.x), fma(s1, b.y, s0 * a.y)};
}
// acc + a*s0 + b*s1
template <typename R>
__device__ __forceinline__ cplx<R> lerp2acc(cplx<R> acc, R s0, cplx<R> a, R s1, cplx<R> b) {
  return cplx<R>{fma(s1, b.x, fma(s0, a.x, acc.x)), fma(s1, b.y, fma(s0, a.y, acc.y))};
}
// 1D restriction of five values at offsets -2..2: weights 1/3, 2/3, 1, 2/3, 1/3
template <typename R>
__device__ __forceinline__ cplx<R> restrict5(cplx<R> m2, cplx<R> m1, cplx<R> z, cplx<R> p1, cplx<R> p2) {
  return cplx<R>{fma(m2.x + p2.x, R(1) / R(3), fma(m1.x + p1.x, R(2) / R(3), z.x)),
                 fma(m2.y + p2.y, R(1) / R(3), fma(m1.y + p1.y, R(2) / R(3), z.y))};
}

// Loads of arrays that other blocks of the same launch may have written
// (persistent launches) bypass L1.
template <typename T> __device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }
template <> __device__ __forceinline__ cplx<double> ldcg(const cplx<double>* p) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return cplx<double>{v.x, v.y};
}
template <> __device__ __forceinline__ cplx<float> ldcg(const cplx<float>* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return cplx<float>{v.x, v.y};
}

// One tile of the sweep; `tile` indexes the tiles of the level row by row.
template <int TC, int NTHR, typename R = double>
__device__ __forceinline__ void sweep2_tile(const Sweep2Args<R>& A, int tile, unsigned char* smem_raw,
                                            double* s_red) {
  using T = Tile2<TC, R>;
  constexpr int F = T::F, SU = T::SU, SR = T::SR, SC = T::SC, SD = T::SD;
  using C = cplx<R>;
  C* s_A = reinterpret_cast<C*>(smem_raw);
  C* s_c = s_A;                  // [SC][SC]  pending correction
  C* s_X = s_c + SC * SC;        // [SC][SU]  x-interpolated pending correction
  C* s_Y = s_A;                  // [F+2][TC] x-restricted residual (after P2)
  C* s_dc = s_Y + (F + 2) * TC;  // [SD][SD]  du at c-points
  C* s_Z = s_dc + SD * SD;       // [SD][F]   x-interpolated c-point du
  C* s_u = s_A + T::AR;          // [SU][SU]
  C* s_r = s_u + SU * SU;        // [SR][SR]
  C* s_coef = s_r + SR * SR;     // [16][9]
  C* s_omd = s_coef + 16 * 9;    // [16]
  uint8_t* s_tx = reinterpret_cast<uint8_t*>(s_omd + 16);  // [SU] types along x of the u box
  uint8_t* s_ty = s_tx + SU;                                  // [SU] types along y
  __syncthreads();  // a previous tile of this block may still read shared memory

  const int n = A.n, N = n + 1, nc = n / 3;
  const int tile_x = tile % A.tiles_x, tile_y = tile / A.tiles_x;
  const int C0x = tile_x * TC, C0y = tile_y * TC;
  const int x0 = 3 * C0x, y0 = 3 * C0y;
  const bool use_c = A.fine && !A.first && A.c != nullptr;

  // P0: tables, vertex types of the u box, pending correction
  for (int i = threadIdx.x; i < 16 * 9; i += NTHR) s_coef[i] = A.coef[i];
  for (int i = threadIdx.x; i < 16; i += NTHR) s_omd[i] = A.omd[i];
  for (int i = threadIdx.x; i < 2 * SU; i += NTHR) {
    const int q = i % SU;
    const int g = (i < SU ? x0 : y0) - 3 + q;
    (i < SU ? s_tx : s_ty)[q] = (g >= 0 && g <= n) ? A.typ[g] : (uint8_t)0;
  }
  if (use_c) {
    for (int i = threadIdx.x; i < SC * SC; i += NTHR) {
      const int qx = i % SC, qy = i / SC;
      const int cx = C0x - 1 + qx, cy = C0y - 1 + qy;
      const bool in = cx >= 0 && cx <= nc && cy >= 0 && cy <= nc;
      s_c[i] = in ? ldcg(A.c + (long long)cy * (nc + 1) + cx) : cz<R>();
    }
  }

  // b of this thread's P3 points, in flight together with the u loads below
  constexpr int KB = (SR * SR + NTHR - 1) / NTHR;
  C bpre[KB];
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    const int i = threadIdx.x + k * NTHR;
    const int gx = x0 - 2 + i % SR, gy = y0 - 2 + i / SR;
    bpre[k] = (i < SR * SR && gx > 0 && gx < n && gy > 0 && gy < n) ? ldcg(A.b + (long long)gy * N + gx)
                                                                      : cz<R>();
  }
  // P2: u = U + P c on the u box (zero outside the interior).  Without a
  // pending correction the u loads overlap those of P0 (one barrier less).
  auto load_u = [&](bool with_c) {
    for (int i = threadIdx.x; i < SU * SU; i += NTHR) {
      const int bx = i % SU, by = i / SU;
      const int gx = x0 - 3 + bx, gy = y0 - 3 + by;
      C v = cz<R>();
      if (gx > 0 && gx < n && gy > 0 && gy < n) {
        if (!(A.fine && A.first)) v = ldcg(A.u + (long long)gy * N + gx);
        if (with_c) {
          const int oy = by % 3, cy = by / 3;
          v = lerp2acc(v, w0<R>(oy), s_X[cy * SU + bx], w1<R>(oy), s_X[(cy + 1) * SU + bx]);
        }
      }
      s_u[i] = v;
    }
  };
  if (!use_c) load_u(false);
  __syncthreads();
  if (use_c) {
    // P1: pending correction interpolated along x for every coarse row of the box
    for (int i = threadIdx.x; i < SC * SU; i += NTHR) {
      const int bx = i % SU, cy = i / SU;
      const int ox = bx % 3, cx = bx / 3;  // box origin x0-3 is a c-point
      s_X[i] = lerp2(w0<R>(ox), s_c[cy * SC + cx], w1<R>(ox), s_c[cy * SC + cx + 1]);
    }
    __syncthreads();
    load_u(true);
    __syncthreads();
  }

  // P3: r = b - H u on the r box; |r|^2 over the owned interior
  double nrm = 0.0;
#pragma unroll
  for (int kb = 0; kb < KB; ++kb) {
    const int i = threadIdx.x + kb * NTHR;
    if (i >= SR * SR) break;
    const int qx = i % SR, qy = i / SR;
    const int gx = x0 - 2 + qx, gy = y0 - 2 + qy;
    C r = cz<R>();
    if (gx > 0 && gx < n && gy > 0 && gy < n) {
      const int bx = qx + 1, by = qy + 1;  // u-box coordinates
      const int t = s_tx[bx] + 4 * s_ty[by];
      const C* cf = s_coef + t * 9;
      const C* up = s_u + by * SU + bx;
      r = bpre[kb];
      if ((A.realrow >> t) & 1u) {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          const C uk = up[(k / 3 - 1) * SU + (k % 3 - 1)];
          const R a = cf[k].x;
          r.x = fma(-a, uk.x, r.x);
          r.y = fma(-a, uk.y, r.y);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          const C uk = up[(k / 3 - 1) * SU + (k % 3 - 1)];
          const C a = cf[k];
          r.x = fma(-a.x, uk.x, r.x);
          r.x = fma(a.y, uk.y, r.x);
          r.y = fma(-a.x, uk.y, r.y);
          r.y = fma(-a.y, uk.x, r.y);
        }
      }
      if (qx >= 2 && qx < F + 2 && qy >= 2 && qy < F + 2)
        nrm = fma((double)r.x, (double)r.x, fma((double)r.y, (double)r.y, nrm));
    }
    s_r[i] = r;
  }
  __syncthreads();

  // P4: restriction along x (rows of the r box, owned coarse columns); du at
  // the c-points [C0, C0+TC]^2
  if (A.has_coarse) {
    for (int i = threadIdx.x; i < (F + 2) * TC; i += NTHR) {
      const int j = i % TC, qy = i / TC;
      const C* rp = s_r + qy * SR + 3 * j + 2;
      s_Y[qy * TC + j] = restrict5(rp[-2], rp[-1], rp[0], rp[1], rp[2]);
    }
  }
  if (A.hier && !A.hb) {
    for (int i = threadIdx.x; i < SD * SD; i += NTHR) {
      const int jx = i % SD, jy = i / SD;
      const int qx = 3 * jx + 2, qy = 3 * jy + 2;  // r-box coordinates of the c-point
      const int t = s_tx[qx + 1] + 4 * s_ty[qy + 1];
      const C r = s_r[qy * SR + qx];
      const C w = s_omd[t];
      s_dc[i] = ((A.realjac >> t) & 1u) ? rmul(w.x, r) : w * r;
    }
  }
  __syncthreads();

  // P5: coarse outputs (b_{l-1} = R r + G u_{l-1}, u_{l-1} = I u) and the
  // x-pass of P I du
  if (A.has_coarse) {
    for (int i = threadIdx.x; i < TC * TC; i += NTHR) {
      const int jx = i % TC, jy = i / TC;
      const int cx = C0x + jx, cy = C0y + jy;
      if (cx > nc || cy > nc) continue;
      const long long ci = (long long)cy * (nc + 1) + cx;
      const bool inner = cx > 0 && cx < nc && cy > 0 && cy < nc;
      C bs = cz<R>(), uc = cz<R>();
      if (inner) {
        const C* yp = s_Y + (3 * jy + 2) * TC + jx;
        bs = restrict5(yp[-2 * TC], yp[-TC], yp[0], yp[TC], yp[2 * TC]);
        const int gt = A.gtyp[cx] + kMaxGTypes * A.gtyp[cy];
        const C* gc = A.gcoef + gt * 9;  // read-only table, shared by all tiles
        const C* up = s_u + (3 * jy + 3) * SU + (3 * jx + 3);
#pragma unroll
        for (int k = 0; k < 9; ++k) bs = cfma(gc[k], up[3 * (k / 3 - 1) * SU + 3 * (k % 3 - 1)], bs);
        uc = up[0];
      }
      A.b_coarse[ci] = bs;
      A.u_coarse[ci] = uc;
    }
  }
  if (A.hier && !A.hb) {
    for (int i = threadIdx.x; i < SD * F; i += NTHR) {
      const int qx = i % F, jy = i / F;
      const int ox = qx % 3, jx = qx / 3;
      s_Z[i] = lerp2(w0<R>(ox), s_dc[jy * SD + jx], w1<R>(ox), s_dc[jy * SD + jx + 1]);
    }
  }
  __syncthreads();

  // P6: T du and the output at the owned fine vertices
  for (int i = threadIdx.x; i < F * F; i += NTHR) {
    const int qx = i % F, qy = i / F;
    const int gx = x0 + qx, gy = y0 + qy;
    if (gx > n || gy > n) continue;
    C val = cz<R>();
    if (gx > 0 && gx < n && gy > 0 && gy < n) {
      const int t = s_tx[qx + 3] + 4 * s_ty[qy + 3];
      const C r = s_r[(qy + 2) * SR + (qx + 2)];
      const C w = s_omd[t];
      C du = ((A.realjac >> t) & 1u) ? rmul(w.x, r) : w * r;
      const int ox = qx % 3, oy = qy % 3;
      if (A.hb && ox == 0 && oy == 0) du = cz<R>();
      if (A.hier && !A.hb) {
        const int jy = qy / 3;
        const C pi = lerp2(w0<R>(oy), s_Z[jy * F + qx], w1<R>(oy), s_Z[(jy + 1) * F + qx]);
        du = du - pi;
      }
      val = A.fine ? s_u[(qy + 3) * SU + (qx + 3)] + du : du;
    }
    A.out[(long long)gy * N + gx] = val;
  }

  if (A.fine && A.norm2 != nullptr)
    block_norm_finish_tile<NTHR>(nrm, s_red, A.partial, A.ticket, A.norm2, tile, A.ntiles);
}

template <int TC, int NTHR, typename R = double>
__global__ void __launch_bounds__(NTHR) sweep2_kernel(const Sweep2Args<R> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double s_red[NTHR / 32];
  sweep2_tile<TC, NTHR, R>(A, blockIdx.x, smem_raw, s_red);
}

}  // namespace mg
