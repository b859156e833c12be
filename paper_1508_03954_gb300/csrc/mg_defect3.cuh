// mg_defect3.cuh -- FP64 defect of a 3D level with a constant shift, fused
// with the update that precedes it (sm_103a).
//
//   u' = u + e + P c        (e: fine correction, c: pending coarse correction,
//                            both optional, of precision RC; e + P c is formed
//                            in RC and added to u in FP64)
//   r  = b - H u'           (FP64, the separable form of mg_sweep3s.cuh:
//                            H = M_x [M_y (K_z - phi M_z) + K_y M_z] + K_x M_y M_z)
//   outputs: u' (optional), r as complex64 (optional), sum |r|^2 (FP64,
//   deterministic order).
//
// This is the outer step of the defect-correction form (complex64 cycles on
// H e = r inside an FP64 loop): one pass updates the iterate, forms the next
// right-hand side of the inner problem and the convergence norm.  With e and
// c null and no outputs but the norm it is the plain FP64 residual norm.
//
// Layout: blocks of 512 threads, lane = x and warp = y of a 32 x 16 box of
// fine columns; the block owns the inner 30 x 14 columns and marches a range
// of coarse planes (three fine planes each) along z.  u' is recomputed on the
// one-column halo by the neighbouring tiles, so no step reads data another
// block writes.  The (tile, coarse plane) units are split into ranges of
// equal FP64 cost, one block per SM: the host tabulates each unit's cost from
// how many of its axis passes take complex coefficients (scaling layer), and
// each block finds its range in the prefix sums.  The kernel is bound by the
// FP64 pipe (50-90 FP64 operations per vertex against 2 FP64 FMA per clock
// per SM).
#pragma once
#include "mg_kernels.cuh"
#include "mg_sweep3s.cuh"

namespace mg {

constexpr int kD3Threads = 512;

template <typename RC>
struct Defect3Args {
  int n;
  int tiles_x, tiles_y;     // 30-column by 14-row tiles
  long long nunits;         // tiles_x * tiles_y * (n / 3)
  const unsigned* upref;    // prefix sums of the unit costs, nunits + 1 entries
  const cplx<double>* u;
  const cplx<RC>* e;        // fine correction (nullable)
  const cplx<RC>* c;        // pending correction on level n/3 (nullable)
  const cplx<double>* b;
  cplx<double>* u_out;      // u' (nullable; must not alias u)
  cplx<float>* r32;         // r as complex64 (nullable)
  const uint8_t* typ;
  cplx<double> row[4][9];   // by axis class: mass, stiffness, stiffness - phi mass
  double* partial;
  unsigned* ticket;
  double* norm2;
};

template <typename RC>
struct Defect3Shared {
  cplx<double> za[2][16][32];
  cplx<double> zb[2][16][32];
  cplx<RC> cc[8][13];       // one coarse plane of c, coarse box from floor((x0-1)/3), floor((y0-1)/3)
  cplx<double> row[4][9];
};

__device__ __forceinline__ cplx<double> tap3d(double c0, double c1, double c2, cplx<double> a,
                                              cplx<double> b, cplx<double> d) {
  return cplx<double>{fma(c2, d.x, fma(c1, b.x, c0 * a.x)), fma(c2, d.y, fma(c1, b.y, c0 * a.y))};
}
__device__ __forceinline__ cplx<double> tap3d_acc(double c0, double c1, double c2, cplx<double> a,
                                                  cplx<double> b, cplx<double> d, cplx<double> acc) {
  return cplx<double>{fma(c2, d.x, fma(c1, b.x, fma(c0, a.x, acc.x))),
                      fma(c2, d.y, fma(c1, b.y, fma(c0, a.y, acc.y)))};
}
__device__ __forceinline__ cplx<double> tap3dc_acc(const cplx<double>* c, cplx<double> a, cplx<double> b,
                                                   cplx<double> d, cplx<double> acc) {
  return cfma(c[2], d, cfma(c[1], b, cfma(c[0], a, acc)));
}
__device__ __forceinline__ cplx<double> shfl_cd(cplx<double> v, int delta, bool up) {
  cplx<double> o;
  if (up) {
    o.x = __shfl_up_sync(0xffffffffu, v.x, delta);
    o.y = __shfl_up_sync(0xffffffffu, v.y, delta);
  } else {
    o.x = __shfl_down_sync(0xffffffffu, v.x, delta);
    o.y = __shfl_down_sync(0xffffffffu, v.y, delta);
  }
  return o;
}
template <typename R> __device__ __forceinline__ cplx<R> ldg_c(const cplx<R>* p) {
  if constexpr (sizeof(R) == 4) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return cplx<R>{v.x, v.y};
  } else {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    return cplx<R>{v.x, v.y};
  }
}

template <typename RC>
__global__ void __launch_bounds__(kD3Threads, 1) defect3_kernel(const Defect3Args<RC> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double s_red[kD3Threads / 32];
  Defect3Shared<RC>& S = *reinterpret_cast<Defect3Shared<RC>*>(smem_raw);
  using C = cplx<double>;
  using CR = cplx<RC>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n = A.n, N = n + 1, nc = n / 3;
  const long long NN = (long long)N * N, Nc = nc + 1, NNc = Nc * Nc;
  for (int i = threadIdx.x; i < 36; i += kD3Threads) S.row[i / 9][i % 9] = A.row[i / 9][i % 9];
  const double m0 = A.row[0][0].x, m1 = A.row[0][1].x, m2 = A.row[0][2].x;
  const double k0 = A.row[0][3].x, k1 = A.row[0][4].x, k2 = A.row[0][5].x;
  const double p0 = A.row[0][6].x, p1 = A.row[0][7].x, p2 = A.row[0][8].x;
  const bool has_e = A.e != nullptr, has_c = A.c != nullptr;
  const bool own_lane = lane >= 1 && lane <= 30, own_row = warp >= 1 && warp <= 14;
  double nrm = 0.0;

  // this block's units: those whose prefix cost lies in [W b / B, W (b+1) / B)
  const long long U = A.nunits;
  const unsigned long long W = A.upref[U];
  auto first_at = [&](unsigned long long target) -> long long {
    long long lo = 0, hi = U;  // first i in [0, U] with upref[i] >= target
    while (lo < hi) {
      const long long mid = (lo + hi) >> 1;
      if ((unsigned long long)__ldg(A.upref + mid) >= target) hi = mid; else lo = mid + 1;
    }
    return lo;
  };
  long long unit = first_at(W * blockIdx.x / gridDim.x);
  const long long uend = first_at(W * (blockIdx.x + 1) / gridDim.x);
  while (unit < uend) {
    const int tile = (int)(unit / nc), Z0 = (int)(unit % nc);
    const int Z1 = (int)min((long long)nc, (long long)Z0 + (uend - unit));
    unit += Z1 - Z0;
    const int x0 = (tile % A.tiles_x) * 30, y0 = (tile / A.tiles_x) * 14;
    const int gx = x0 - 1 + lane, gy = y0 - 1 + warp;
    const bool colin = gx > 0 && gx < n && gy > 0 && gy < n;
    const bool owncol = own_lane && own_row && gx <= n && gy <= n;
    const long long col = (long long)gy * N + gx;
    const int tx = (gx >= 0 && gx <= n) ? (int)A.typ[gx] : 0;
    const int ty = (gy >= 0 && gy <= n) ? (int)A.typ[gy] : 0;
    const bool xreal = __all_sync(0xffffffffu, tx == 0);
    const bool yreal = ty == 0;
    // coarse cell of this column inside the coarse box of S.cc
    const int cbx = (x0 + 2) / 3 - 1, cby = (y0 + 2) / 3 - 1;  // floor((x0-1)/3) for x0 >= 0
    const int ccx = gx >= 0 ? gx / 3 : -1, ccy = gy >= 0 ? gy / 3 : -1;
    const int jx = ccx - cbx, jy = ccy - cby;  // 0..11, 0..6 for interior columns
    const int ox = gx - 3 * ccx, oy = gy - 3 * ccy;
    const RC wx1 = ox == 1 ? RC(1) / RC(3) : (ox == 2 ? RC(2) / RC(3) : RC(0)), wx0 = RC(1) - wx1;
    const RC wy1 = oy == 1 ? RC(1) / RC(3) : (oy == 2 ? RC(2) / RC(3) : RC(0)), wy0 = RC(1) - wy1;

    auto ld_cc = [&](int Zc) -> CR {
      const int t = threadIdx.x;
      const int cx = cbx + t % 13, cy = cby + t / 13;
      return (has_c && t < 104 && Zc >= 0 && Zc <= nc && cx >= 0 && cx <= nc && cy >= 0 && cy <= nc)
                 ? ldg_c(A.c + Zc * NNc + (long long)cy * Nc + cx)
                 : CR{RC(0), RC(0)};
    };
    auto bil_cc = [&]() -> CR {
      if (!colin) return CR{RC(0), RC(0)};
      const CR a = S.cc[jy][jx], b2 = S.cc[jy][jx + 1], c2 = S.cc[jy + 1][jx], d2 = S.cc[jy + 1][jx + 1];
      return CR{wy0 * (wx0 * a.x + wx1 * b2.x) + wy1 * (wx0 * c2.x + wx1 * d2.x),
                wy0 * (wx0 * a.y + wx1 * b2.y) + wy1 * (wx0 * c2.y + wx1 * d2.y)};
    };
    auto in_plane = [&](int z) { return colin && z > 0 && z < n; };
    auto ldU = [&](int z) -> C { return in_plane(z) ? ldg_c(A.u + z * NN + col) : cz<double>(); };
    auto ldE = [&](int z) -> CR {
      return (has_e && in_plane(z)) ? ldg_c(A.e + z * NN + col) : CR{RC(0), RC(0)};
    };
    auto ldB = [&](int z) -> C { return in_plane(z) ? ldg_c(A.b + z * NN + col) : cz<double>(); };
    // u' = u + (e + w0 cA + w1 cB), the correction summed in RC
    auto form = [&](int z, C uu, CR ee, RC w0, CR cA, RC w1, CR cB) -> C {
      if (!in_plane(z)) return cz<double>();
      CR v = ee;
      if (has_c) {
        v.x += w0 * cA.x + w1 * cB.x;
        v.y += w0 * cA.y + w1 * cB.y;
      }
      return C{uu.x + (double)v.x, uu.y + (double)v.y};
    };

    __syncthreads();  // shared memory of the previous range is free
    CR cxyA{RC(0), RC(0)}, cxyB{RC(0), RC(0)}, cprev{RC(0), RC(0)}, ccpre{RC(0), RC(0)};
    if (has_c) {
      if (threadIdx.x < 104) S.cc[threadIdx.x / 13][threadIdx.x % 13] = ld_cc(Z0 - 1);
      __syncthreads();
      cprev = bil_cc();
      __syncthreads();
      if (threadIdx.x < 104) S.cc[threadIdx.x / 13][threadIdx.x % 13] = ld_cc(Z0);
      __syncthreads();
      cxyA = bil_cc();
      __syncthreads();
      if (threadIdx.x < 104) S.cc[threadIdx.x / 13][threadIdx.x % 13] = ld_cc(Z0 + 1);
      __syncthreads();
      cxyB = bil_cc();
      ccpre = ld_cc(Z0 + 2);
      __syncthreads();
    }
    C um = form(3 * Z0 - 1, ldU(3 * Z0 - 1), ldE(3 * Z0 - 1), RC(1) / RC(3), cprev, RC(2) / RC(3), cxyA);
    C u0 = form(3 * Z0, ldU(3 * Z0), ldE(3 * Z0), RC(1), cxyA, RC(0), cxyB);
    if (A.u_out != nullptr && owncol) A.u_out[3 * Z0 * NN + col] = u0;
    // prefetch: step z (slot z mod 3) uses u, e at z + 1 and b at z
    C pu[3], pb[3];
    CR pe[3];
    pu[0] = ldU(3 * Z0 + 1);
    pu[1] = ldU(3 * Z0 + 2);
    pu[2] = ldU(3 * Z0 + 3);
    pe[0] = ldE(3 * Z0 + 1);
    pe[1] = ldE(3 * Z0 + 2);
    pe[2] = ldE(3 * Z0 + 3);
    pb[0] = ldB(3 * Z0);
    pb[1] = ldB(3 * Z0 + 1);
    pb[2] = ldB(3 * Z0 + 2);

    auto step = [&](auto ozc, int z) {
      constexpr int OZ = decltype(ozc)::value;
      constexpr int OZP = (OZ + 1) % 3;
      const int zp = z + 1;
      const int buf = z & 1;
      if (OZP == 0) cxyA = cxyB;
      const RC w1 = OZP == 1 ? RC(1) / RC(3) : (OZP == 2 ? RC(2) / RC(3) : RC(0));
      const C up = form(zp, pu[OZ], pe[OZ], RC(1) - w1, cxyA, w1, cxyB);
      if (A.u_out != nullptr && owncol && zp < 3 * Z1) A.u_out[zp * NN + col] = up;
      if (OZP == 2 && has_c && threadIdx.x < 104) S.cc[threadIdx.x / 13][threadIdx.x % 13] = ccpre;
      pu[OZ] = ldU(z + 4);
      pe[OZ] = ldE(z + 4);
      const int tz = (z >= 0 && z <= n) ? (int)__ldg(A.typ + z) : 0;
      C za, zb;
      if (tz == 0) {
        za = tap3d(m0, m1, m2, um, u0, up);
        zb = tap3d(p0, p1, p2, um, u0, up);
      } else {
        za = tap3dc_acc(&S.row[tz][0], um, u0, up, cz<double>());
        zb = tap3dc_acc(&S.row[tz][6], um, u0, up, cz<double>());
      }
      S.za[buf][warp][lane] = za;
      S.zb[buf][warp][lane] = zb;
      __syncthreads();
      if (OZP == 0 && has_c) {
        cxyB = bil_cc();
        ccpre = ld_cc(zp / 3 + 2);
      }
      if (own_row) {
        const C am = S.za[buf][warp - 1][lane], ap = S.za[buf][warp + 1][lane];
        const C bm = S.zb[buf][warp - 1][lane], bp = S.zb[buf][warp + 1][lane];
        C cy, ey;
        if (yreal) {
          cy = tap3d_acc(k0, k1, k2, am, za, ap, tap3d(m0, m1, m2, bm, zb, bp));
          ey = tap3d(m0, m1, m2, am, za, ap);
        } else {
          const C* rw = &S.row[ty][0];
          cy = tap3dc_acc(rw + 3, am, za, ap, tap3dc_acc(rw, bm, zb, bp, cz<double>()));
          ey = tap3dc_acc(rw, am, za, ap, cz<double>());
        }
        const C cl = shfl_cd(cy, 1, true), cr = shfl_cd(cy, 1, false);
        const C el = shfl_cd(ey, 1, true), er = shfl_cd(ey, 1, false);
        C hu;
        if (xreal) {
          hu = tap3d_acc(k0, k1, k2, el, ey, er, tap3d(m0, m1, m2, cl, cy, cr));
        } else {
          const C* rw = &S.row[tx][0];
          hu = tap3dc_acc(rw + 3, el, ey, er, tap3dc_acc(rw, cl, cy, cr, cz<double>()));
        }
        C r = cz<double>();
        if (in_plane(z)) r = pb[OZ] - hu;
        if (owncol) {
          nrm = fma(r.x, r.x, fma(r.y, r.y, nrm));
          if (A.r32 != nullptr) A.r32[z * NN + col] = cplx<float>{(float)r.x, (float)r.y};
        }
      }
      pb[OZ] = ldB(z + 3);
      um = u0;
      u0 = up;
    };

    for (int Zc = Z0; Zc < Z1; ++Zc) {
      step(IC<0>{}, 3 * Zc);
      step(IC<1>{}, 3 * Zc + 1);
      step(IC<2>{}, 3 * Zc + 2);
    }
    // the boundary plane n belongs to the range that ends there
    if (Z1 == nc && owncol) {
      if (A.u_out != nullptr) A.u_out[n * NN + col] = cz<double>();
      if (A.r32 != nullptr) A.r32[n * NN + col] = cplx<float>{0.f, 0.f};
    }
  }
  if (A.norm2 != nullptr)
    block_norm_finish_tile<kD3Threads>(nrm, s_red, A.partial, A.ticket, A.norm2, blockIdx.x, gridDim.x);
}

}  // namespace mg
