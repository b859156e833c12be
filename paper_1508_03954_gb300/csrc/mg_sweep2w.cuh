// mg_sweep2w.cuh -- warp-strip sweep for large 2D levels with a constant
// shift, complex64 (sm_103a).
//
// The step is the one of mg_sweep2d.cuh (Appendix A Algorithm 4 on one level,
// the single-touch pending correction of Algorithm 2, coarse right-hand side
// b_{l-1} = R r_l + G_{l-1} u_{l-1}), laid out so that one warp does all of
// it for a strip of the level without shared memory or block barriers:
//
//  * lane = x: a warp owns 27 fine columns (9 coarse cells) of a strip,
//    [x0-3, x0+28] with a 3-column halo before and 2 after, and marches a
//    range of coarse rows along y holding u(y-1), u(y), u(y+1) in registers;
//  * operator: H u = M_x (K_y - phi M_y) u + K_x (M_y u) (Section 4, the 2D
//    element operator as a tensor product of 1D rows): the y-pass runs in
//    registers, the x-pass takes its neighbours by shuffles; interior rows
//    take real coefficients;
//  * restriction: along x by shuffles, along y by accumulating each fine
//    row into the two coarse rows it touches (weights 1 - |o|/3);
//  * BPX (id - P I): the c-row Jacobi updates are interpolated along x by
//    shuffles from the c-lanes and along y between consecutive c-rows; the
//    two fine rows between c-rows wait in registers;
//  * G_{l-1} u_{l-1}: the c-lanes keep u at the c-points of three c-rows
//    and take the neighbouring coarse columns by shuffles.
//
// Rows of U and b are loaded three rows ahead into registers.  A range whose
// rows all lie inside the level (the common case) runs a step without any
// boundary tests.
//
// Work split: (strip, coarse row) units, contiguous equal ranges per warp.
#pragma once
#include "mg_kernels.cuh"
#include "mg_sweep2d.cuh"
#include "mg_sweep3s.cuh"

namespace mg {

struct Sweep2wArgs {
  int n, fine, first, has_coarse, hb, hier;
  int scells;           // coarse cells per strip: 9 (a column per lane) or 18 (two)
  int strips;           // strips of scells coarse cells
  int nunits;           // strips * (n / 3)
  const cplx<float>* u;     // fine: pending U; coarse: u_l
  const cplx<float>* c;     // pending correction on level l-1 (fine, may be null)
  const cplx<float>* b;
  cplx<float>* out;         // fine: U'; coarse: T du
  cplx<float>* b_coarse;
  cplx<float>* u_coarse;
  const uint8_t* typ;       // axis class per fine index (n+1)
  const uint8_t* gtyp;      // Galerkin row class per coarse index (n/3+1)
  const cplx<float>* gcoef; // [kMaxGTypes^2][9], index gx + kMaxGTypes * gy
  cplx<float> row[4][9];    // by axis class: mass, stiffness, stiffness - phi mass
  cplx<float> omd[16];      // omega / D per vertex type tx + 4 ty
  double* partial;
  unsigned* ticket;
  double* norm2;
};

__device__ __forceinline__ cplx<float> shfl_idx(cplx<float> v, int src) {
  return cplx<float>{__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src)};
}

// One segment (strip, coarse rows [Y0, Y1)) of one warp.  INNER: every row
// the march touches, [3 Y0 - 3, 3 Y1 + 4], is an interior row.
template <bool INNER>
__device__ __forceinline__ void strip2w_segment(const Sweep2wArgs& A, int strip, int Y0, int Y1,
                                                const cplx<float>* srow, const cplx<float>* somd,
                                                float& nrm) {
  using C = cplx<float>;
  const int lane = threadIdx.x & 31;
  const int n = A.n, N = n + 1, nc = n / 3, Nc = nc + 1;
  const bool zero_u = A.fine && A.first;
  const bool use_c = A.fine && !A.first && A.c != nullptr;
  const bool bpx = A.hier && !A.hb;
  const int ox = lane % 3;
  const bool cpx = ox == 0;
  const float wx1 = ox == 0 ? 0.f : (ox == 1 ? 1.f / 3.f : 2.f / 3.f), wx0 = 1.f - wx1;
  const float M0 = A.row[0][0].x, M1 = A.row[0][1].x, M2 = A.row[0][2].x;
  const float K0 = A.row[0][3].x, K1 = A.row[0][4].x, K2 = A.row[0][5].x;
  const float P0 = A.row[0][6].x, P1 = A.row[0][7].x, P2 = A.row[0][8].x;
  const int C0 = 9 * strip, x0 = 27 * strip;
  const int gx = x0 - 3 + lane;
  const bool xin = gx > 0 && gx < n;
  const bool last = C0 + 9 >= nc;
  const bool ownx = lane >= 3 && (lane < 30 || (lane == 30 && last)) && gx <= n;
  const bool rlane = xin && lane >= 1 && lane <= 30;  // lanes of the r box
  const int tx = (gx >= 0 && gx <= n) ? (int)A.typ[gx] : 0;
  const bool xreal = __all_sync(0xffffffffu, tx == 0);
  const int cx = C0 - 1 + lane / 3;  // coarse column left of (or at) this lane
  const int ls = lane - ox, rs = min(lane - ox + 3, 31);
  const int l3 = lane < 3 ? 0 : lane - 3, r3 = min(lane + 3, 31);
  const int ccol = C0 + lane / 3 - 1;
  const bool cemit = cpx && lane >= 3 && (lane <= 27 || ccol == nc) && ccol <= nc;
  const C* pu_ = A.u + gx;  // column pointers; row y at + y * N
  const C* pb_ = A.b + gx;
  C* po_ = A.out + gx;
  auto rowok = [&](int y) { return INNER || (y > 0 && y < n); };
  auto ldU = [&](int y) -> C { return (!zero_u && xin && rowok(y)) ? ld_nc(pu_ + y * N) : cz<float>(); };
  auto ldB = [&](int y) -> C { return (xin && rowok(y)) ? ld_nc(pb_ + y * N) : cz<float>(); };
  auto ldc2 = [&](int Yc, C& a, C& b) {
    a = cz<float>();
    b = cz<float>();
    if (use_c && xin && Yc >= 0 && Yc <= nc) {
      const C* p = A.c + (Yc * Nc + cx);
      a = ld_nc(p);
      if (ox) b = ld_nc(p + 1);
    }
  };
  auto lerpx = [&](C a, C b) -> C {
    return cplx<float>{fmaf(wx1, b.x, wx0 * a.x), fmaf(wx1, b.y, wx0 * a.y)};
  };
  auto tyof = [&](int y) -> int { return (y >= 0 && y <= n) ? (int)__ldg(A.typ + y) : 0; };
  // pending correction interpolated along x on coarse rows (Ya, Ya + 1); the
  // raw values of the row after are in flight
  C cA, cB, cpa, cpb;
  {
    C a, b;
    ldc2(Y0 - 1, a, b);
    cA = lerpx(a, b);
    ldc2(Y0, a, b);
    cB = lerpx(a, b);
    ldc2(Y0 + 1, cpa, cpb);
  }
  C um = ldU(3 * Y0 - 3), u0 = ldU(3 * Y0 - 2);
  if (use_c && xin) {
    if (INNER || 3 * Y0 - 3 > 0) um = um + cA;
    if (INNER || 3 * Y0 - 2 > 0) {
      u0 = rfma(W0<1>(), cA, u0);
      u0 = rfma(W1<1>(), cB, u0);
    }
  }
  C pu[3], pb[3];
  pu[1] = ldU(3 * Y0 - 1);
  pu[2] = ldU(3 * Y0);
  pu[0] = ldU(3 * Y0 + 1);
  pb[1] = ldB(3 * Y0 - 2);
  pb[2] = ldB(3 * Y0 - 1);
  pb[0] = ldB(3 * Y0);
  int tyn = tyof(3 * Y0 - 2);
  // u at the c-points of c-rows (Ynew - 2, Ynew - 1, Ynew), c-lanes only
  C qa = cz<float>(), qb = cz<float>(), qc = um;
  C accA = cz<float>(), accB = cz<float>();
  C pv1 = cz<float>(), pv2 = cz<float>(), pidp = cz<float>();
  const int yo0 = 3 * Y0, yo1 = 3 * Y1;

  auto step = [&](auto ozc, int y) {
    constexpr int OZ = decltype(ozc)::value;
    constexpr int OZP = (OZ + 1) % 3;
    const int yp = y + 1;
    if (OZP == 0) cA = cB;
    C up = pu[OZ];
    if (use_c && xin && rowok(yp)) {
      up = rfma(W0<OZP>(), cA, up);
      if (OZP != 0) up = rfma(W1<OZP>(), cB, up);
    }
    if (OZP == 0) {
      if (use_c) {
        cB = lerpx(cpa, cpb);
        ldc2(yp / 3 + 2, cpa, cpb);
      }
      qa = qb;
      qb = qc;
      qc = up;
    }
    pu[OZ] = ldU(y + 4);
    const int ty = tyn;
    tyn = tyof(y + 1);
    // y-pass in registers (the class of row y is uniform over the warp)
    C ya, yb;
    if (ty == 0) {
      ya = tap3r(M0, M1, M2, um, u0, up);
      yb = tap3r(P0, P1, P2, um, u0, up);
    } else {
      ya = tap3c_acc(srow + ty * 9, um, u0, up, cz<float>());
      yb = tap3c_acc(srow + ty * 9 + 6, um, u0, up, cz<float>());
    }
    // x-pass by shuffles
    const C al = shfl_c(ya, 1, true), ar = shfl_c(ya, 1, false);
    const C bl = shfl_c(yb, 1, true), br = shfl_c(yb, 1, false);
    C hu;
    if (xreal) {
      hu = tap3r_acc(K0, K1, K2, al, ya, ar, tap3r(M0, M1, M2, bl, yb, br));
    } else {
      const C* rw = srow + tx * 9;
      hu = tap3c_acc(rw + 3, al, ya, ar, tap3c_acc(rw, bl, yb, br, cz<float>()));
    }
    const bool yown = INNER ? (y >= yo0 && y < yo1) : ((y >= yo0 && y < yo1) || y == n);
    C r = cz<float>();
    if (rlane && rowok(y)) r = pb[OZ] - hu;
    pb[OZ] = ldB(y + 3);
    if (ownx && yown) nrm = fmaf(r.x, r.x, fmaf(r.y, r.y, nrm));
    C du = somd[tx + 4 * ty] * r;
    if (A.hb && OZ == 0 && cpx) du = cz<float>();
    const C v = A.fine ? u0 + du : du;
    if (!bpx) {
      if (ownx && yown) po_[y * N] = v;
    } else if (OZ == 1) {
      pv1 = v;
    } else if (OZ == 2) {
      pv2 = v;
    } else {
      // c-row: P I du along x from the c-lanes, along y against the last c-row
      const C pid = lerpx(shfl_idx(du, ls), shfl_idx(du, rs));
      if (ownx) {
        if (y - 2 >= yo0) {
          po_[(y - 2) * N] = pv1 - (rmul(2.f / 3.f, pidp) + rmul(1.f / 3.f, pid));
          po_[(y - 1) * N] = pv2 - (rmul(1.f / 3.f, pidp) + rmul(2.f / 3.f, pid));
        }
        if (yown) po_[y * N] = v - pid;
      }
      pidp = pid;
    }
    if (A.has_coarse) {
      // restriction along x, then into the two coarse rows this row touches
      const C r1l = shfl_c(r, 1, true), r1r = shfl_c(r, 1, false);
      const C r2l = shfl_c(r, 2, true), r2r = shfl_c(r, 2, false);
      const C rx = restrict5f(r2l, r1l, r, r1r, r2r);
      if (OZ == 0) {
        accA = accB + rx;
        accB = cz<float>();
      } else {
        accA = rfma(W0<OZ>(), rx, accA);
        accB = rfma(W1<OZ>(), rx, accB);
      }
      if (OZ == 2) {
        // coarse row Yc = (y - 2) / 3 is complete: b_{l-1} = R r + G u_{l-1}
        const int Yc = (y - 2) / 3;
        const C qaL = shfl_idx(qa, l3), qaR = shfl_idx(qa, r3);
        const C qbL = shfl_idx(qb, l3), qbR = shfl_idx(qb, r3);
        const C qcL = shfl_idx(qc, l3), qcR = shfl_idx(qc, r3);
        if (cemit && Yc >= Y0 && Yc < Y1) {
          const bool inner = ccol > 0 && ccol < nc && Yc > 0 && Yc < nc;
          C bs = cz<float>(), uc = cz<float>();
          if (inner) {
            const C* gc = A.gcoef + (A.gtyp[ccol] + kMaxGTypes * A.gtyp[Yc]) * 9;
            bs = accA;
            bs = cfma(ld_nc(gc + 0), qaL, bs);
            bs = cfma(ld_nc(gc + 1), qa, bs);
            bs = cfma(ld_nc(gc + 2), qaR, bs);
            bs = cfma(ld_nc(gc + 3), qbL, bs);
            bs = cfma(ld_nc(gc + 4), qb, bs);
            bs = cfma(ld_nc(gc + 5), qbR, bs);
            bs = cfma(ld_nc(gc + 6), qcL, bs);
            bs = cfma(ld_nc(gc + 7), qc, bs);
            bs = cfma(ld_nc(gc + 8), qcR, bs);
            uc = qb;
          }
          A.b_coarse[Yc * Nc + ccol] = bs;
          A.u_coarse[Yc * Nc + ccol] = uc;
        }
      }
    }
    um = u0;
    u0 = up;
  };

  for (int Yc = Y0 - 1; Yc < Y1; ++Yc) {
    step(IC<1>{}, 3 * Yc + 1);
    step(IC<2>{}, 3 * Yc + 2);
    step(IC<0>{}, 3 * Yc + 3);
  }
  // the boundary coarse row nc belongs to the range that ends there
  if (A.has_coarse && Y1 == nc && cemit) {
    A.b_coarse[nc * Nc + ccol] = cz<float>();
    A.u_coarse[nc * Nc + ccol] = cz<float>();
  }
}

// Strips of 18 coarse cells with two columns per lane.  A warp owns 54 fine
// columns, box [x0 - 4, x0 + 60): lane L holds box columns 2L and 2L + 1, so a
// row comes in and goes out as one 16-byte access per lane (n + 1 is even and
// the box starts on an even column), the x-pass takes one neighbour per side
// by shuffle for two points, and the per-row control is shared by two points.
// Columns 3 apart are c-points, so a lane holds at most one: lanes L = 2 mod 3
// at their first column, L = 0 mod 3 at their second.  The c-point neighbours
// (Galerkin row, P I du) sit one or two lanes away.  Arithmetic per point is
// that of strip2w_segment.
template <bool INNER, bool BPX>
__device__ __forceinline__ void strip2w2_segment(const Sweep2wArgs& A, int strip, int Y0, int Y1,
                                                 const cplx<float>* srow, const cplx<float>* somd,
                                                 float& nrm) {
  using C = cplx<float>;
  const int lane = threadIdx.x & 31;
  const int n = A.n, N = n + 1, nc = n / 3, Nc = nc + 1;
  const bool zero_u = A.fine && A.first;
  const bool use_c = A.fine && !A.first && A.c != nullptr;
  const float M0 = A.row[0][0].x, M1 = A.row[0][1].x, M2 = A.row[0][2].x;
  const float K0 = A.row[0][3].x, K1 = A.row[0][4].x, K2 = A.row[0][5].x;
  const float P0 = A.row[0][6].x, P1 = A.row[0][7].x, P2 = A.row[0][8].x;
  const int C0 = 18 * strip, x0 = 54 * strip;
  const int g0 = x0 - 4 + 2 * lane;      // fine column of the lane's first point (even)
  const bool pin = g0 >= 0 && g0 < n;    // both points inside [0, n] (n is odd)
  const bool last = C0 + 18 >= nc;
  bool xin[2], ownx[2], rl[2];
  int tx[2], ox[2], srcl[2], srcr[2];
  float wx0[2], wx1[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int gx = g0 + s, bx = 2 * lane + s;
    xin[s] = gx > 0 && gx < n;
    ownx[s] = bx >= 4 && (bx < 58 || (bx == 58 && last)) && gx <= n;
    rl[s] = xin[s] && bx >= 2 && bx <= 58;  // the r box [x0 - 2, x0 + 54]
    tx[s] = (gx >= 0 && gx <= n) ? (int)A.typ[gx] : 0;
    ox[s] = ((bx - 4) % 3 + 3) % 3;         // offset from the c-column on the left
    wx1[s] = ox[s] == 0 ? 0.f : (ox[s] == 1 ? 1.f / 3.f : 2.f / 3.f);
    wx0[s] = 1.f - wx1[s];
    srcl[s] = max(0, (bx - ox[s]) >> 1);      // lanes holding the c-columns left / right
    srcr[s] = min(31, (bx - ox[s] + 3) >> 1);
  }
  const bool xreal = __all_sync(0xffffffffu, tx[0] == 0 && tx[1] == 0);
  const int m3 = lane % 3;
  const int csub = m3 == 2 ? 0 : (m3 == 0 ? 1 : -1);       // which point is a c-point
  const int jc = csub >= 0 ? (2 * lane + csub - 4) / 3 : -1;  // its coarse column C0 + jc
  const int ccol = C0 + jc;
  const bool cemit = csub >= 0 && lane >= 2 && (jc <= 17 || (jc == 18 && ccol == nc)) && ccol <= nc;
  const int gl = max(0, csub == 0 ? lane - 2 : lane - 1), gr = min(31, csub == 0 ? lane + 1 : lane + 2);
  const C* pu_ = A.u + g0;  // the pair's pointers; row y at + y * N
  const C* pb_ = A.b + g0;
  C* po_ = A.out + g0;
  auto rowok = [&](int y) { return INNER || (y > 0 && y < n); };
  // a row of the pair, zero outside the level (and on the Dirichlet ring)
  auto ld2 = [&](const C* base, int y, bool ok, C& a, C& b) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ok && pin && rowok(y)) v = __ldg(reinterpret_cast<const float4*>(base + (long long)y * N));
    a = xin[0] ? C{v.x, v.y} : cz<float>();
    b = xin[1] ? C{v.z, v.w} : cz<float>();
  };
  auto ldc1 = [&](int Yc, int s, C& a, C& b) {
    a = cz<float>();
    b = cz<float>();
    if (use_c && xin[s] && Yc >= 0 && Yc <= nc) {
      const C* p = A.c + (Yc * Nc + (g0 + s) / 3);
      a = ld_nc(p);
      if (ox[s]) b = ld_nc(p + 1);
    }
  };
  auto lerpx = [&](int s, C a, C b) -> C {
    return cplx<float>{fmaf(wx1[s], b.x, wx0[s] * a.x), fmaf(wx1[s], b.y, wx0[s] * a.y)};
  };
  auto tyof = [&](int y) -> int { return (y >= 0 && y <= n) ? (int)__ldg(A.typ + y) : 0; };
  auto pick = [&](const C* v) -> C { return csub == 1 ? v[1] : v[0]; };
  C cA[2], cB[2], cpa[2], cpb[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    C a, b;
    ldc1(Y0 - 1, s, a, b);
    cA[s] = lerpx(s, a, b);
    ldc1(Y0, s, a, b);
    cB[s] = lerpx(s, a, b);
    ldc1(Y0 + 1, s, cpa[s], cpb[s]);
  }
  C um[2], u0[2];
  ld2(pu_, 3 * Y0 - 3, !zero_u, um[0], um[1]);
  ld2(pu_, 3 * Y0 - 2, !zero_u, u0[0], u0[1]);
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    if (use_c && xin[s]) {
      if (INNER || 3 * Y0 - 3 > 0) um[s] = um[s] + cA[s];
      if (INNER || 3 * Y0 - 2 > 0) {
        u0[s] = rfma(W0<1>(), cA[s], u0[s]);
        u0[s] = rfma(W1<1>(), cB[s], u0[s]);
      }
    }
  }
  C pu[3][2], pb[3][2];
  ld2(pu_, 3 * Y0 - 1, !zero_u, pu[1][0], pu[1][1]);
  ld2(pu_, 3 * Y0, !zero_u, pu[2][0], pu[2][1]);
  ld2(pu_, 3 * Y0 + 1, !zero_u, pu[0][0], pu[0][1]);
  ld2(pb_, 3 * Y0 - 2, true, pb[1][0], pb[1][1]);
  ld2(pb_, 3 * Y0 - 1, true, pb[2][0], pb[2][1]);
  ld2(pb_, 3 * Y0, true, pb[0][0], pb[0][1]);
  int tyn = tyof(3 * Y0 - 2);
  // u at the lane's c-point on c-rows (Ynew - 2, Ynew - 1, Ynew)
  C qa = cz<float>(), qb = cz<float>(), qc = pick(um);
  C accA = cz<float>(), accB = cz<float>();
  C pv1[2] = {cz<float>(), cz<float>()}, pv2[2] = {cz<float>(), cz<float>()}, pidp[2] = {cz<float>(), cz<float>()};
  const int yo0 = 3 * Y0, yo1 = 3 * Y1;
  auto step = [&](auto ozc, int y) {
    constexpr int OZ = decltype(ozc)::value;
    constexpr int OZP = (OZ + 1) % 3;
    const int yp = y + 1;
    C up[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      if (OZP == 0) cA[s] = cB[s];
      up[s] = pu[OZ][s];
      if (use_c && xin[s] && rowok(yp)) {
        up[s] = rfma(W0<OZP>(), cA[s], up[s]);
        if (OZP != 0) up[s] = rfma(W1<OZP>(), cB[s], up[s]);
      }
    }
    if (OZP == 0) {
      if (use_c) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          cB[s] = lerpx(s, cpa[s], cpb[s]);
          ldc1(yp / 3 + 2, s, cpa[s], cpb[s]);
        }
      }
      qa = qb;
      qb = qc;
      qc = pick(up);
    }
    ld2(pu_, y + 4, !zero_u, pu[OZ][0], pu[OZ][1]);
    const int ty = tyn;
    tyn = tyof(y + 1);
    // y-pass in registers (the class of row y is uniform over the warp)
    C ya[2], yb[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      if (ty == 0) {
        ya[s] = tap3r(M0, M1, M2, um[s], u0[s], up[s]);
        yb[s] = tap3r(P0, P1, P2, um[s], u0[s], up[s]);
      } else {
        ya[s] = tap3c_acc(srow + ty * 9, um[s], u0[s], up[s], cz<float>());
        yb[s] = tap3c_acc(srow + ty * 9 + 6, um[s], u0[s], up[s], cz<float>());
      }
    }
    // x-pass: the outer neighbours of the pair from the lanes beside
    const C al = shfl_c(ya[1], 1, true), ar = shfl_c(ya[0], 1, false);
    const C bl = shfl_c(yb[1], 1, true), br = shfl_c(yb[0], 1, false);
    C hu[2];
    if (xreal) {
      hu[0] = tap3r_acc(K0, K1, K2, al, ya[0], ya[1], tap3r(M0, M1, M2, bl, yb[0], yb[1]));
      hu[1] = tap3r_acc(K0, K1, K2, ya[0], ya[1], ar, tap3r(M0, M1, M2, yb[0], yb[1], br));
    } else {
      const C* rw0 = srow + tx[0] * 9;
      const C* rw1 = srow + tx[1] * 9;
      hu[0] = tap3c_acc(rw0 + 3, al, ya[0], ya[1], tap3c_acc(rw0, bl, yb[0], yb[1], cz<float>()));
      hu[1] = tap3c_acc(rw1 + 3, ya[0], ya[1], ar, tap3c_acc(rw1, yb[0], yb[1], br, cz<float>()));
    }
    const bool yown = INNER ? (y >= yo0 && y < yo1) : ((y >= yo0 && y < yo1) || y == n);
    C r[2], du[2], v[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      r[s] = (rl[s] && rowok(y)) ? pb[OZ][s] - hu[s] : cz<float>();
      const C rn = (ownx[s] && yown) ? r[s] : cz<float>();
      nrm = fmaf(rn.x, rn.x, fmaf(rn.y, rn.y, nrm));
      du[s] = somd[tx[s] + 4 * ty] * r[s];
      if (A.hb && OZ == 0 && s == csub) du[s] = cz<float>();
      v[s] = A.fine ? u0[s] + du[s] : du[s];
    }
    ld2(pb_, y + 3, true, pb[OZ][0], pb[OZ][1]);
    if (!BPX) {
      if (ownx[0] && ownx[1] && yown) {
        *reinterpret_cast<float4*>(po_ + (long long)y * N) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
      } else {
        st_global_if(po_ + (long long)y * N, v[0], ownx[0] && yown);
        st_global_if(po_ + (long long)y * N + 1, v[1], ownx[1] && yown);
      }
    } else if (OZ == 1) {
      pv1[0] = v[0];
      pv1[1] = v[1];
    } else if (OZ == 2) {
      pv2[0] = v[0];
      pv2[1] = v[1];
    } else {
      // c-row: P I du along x from the lanes holding the c-points, along y
      // against the last c-row
      const C dc = pick(du);
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const C pid = lerpx(s, shfl_idx(dc, srcl[s]), shfl_idx(dc, srcr[s]));
        if (ownx[s]) {
          if (y - 2 >= yo0) {
            po_[(long long)(y - 2) * N + s] = pv1[s] - (rmul(2.f / 3.f, pidp[s]) + rmul(1.f / 3.f, pid));
            po_[(long long)(y - 1) * N + s] = pv2[s] - (rmul(1.f / 3.f, pidp[s]) + rmul(2.f / 3.f, pid));
          }
          if (yown) po_[(long long)y * N + s] = v[s] - pid;
        }
        pidp[s] = pid;
      }
    }
    if (A.has_coarse) {
      // restriction along x at the lane's c-point (five columns around it),
      // then into the two coarse rows this row touches
      const C l0 = shfl_c(r[0], 1, true), l1 = shfl_c(r[1], 1, true);
      const C r0 = shfl_c(r[0], 1, false), r1 = shfl_c(r[1], 1, false);
      const C rx = csub == 0 ? restrict5f(l0, l1, r[0], r[1], r0) : restrict5f(l1, r[0], r[1], r0, r1);
      if (OZ == 0) {
        accA = accB + rx;
        accB = cz<float>();
      } else {
        accA = rfma(W0<OZ>(), rx, accA);
        accB = rfma(W1<OZ>(), rx, accB);
      }
      if (OZ == 2) {
        // coarse row Yc = (y - 2) / 3 is complete: b_{l-1} = R r + G u_{l-1}
        const int Yc = (y - 2) / 3;
        const C qaL = shfl_idx(qa, gl), qaR = shfl_idx(qa, gr);
        const C qbL = shfl_idx(qb, gl), qbR = shfl_idx(qb, gr);
        const C qcL = shfl_idx(qc, gl), qcR = shfl_idx(qc, gr);
        if (cemit && Yc >= Y0 && Yc < Y1) {
          const bool inner = ccol > 0 && ccol < nc && Yc > 0 && Yc < nc;
          C bs = cz<float>(), uc = cz<float>();
          if (inner) {
            const C* gc = A.gcoef + (A.gtyp[ccol] + kMaxGTypes * A.gtyp[Yc]) * 9;
            bs = accA;
            bs = cfma(ld_nc(gc + 0), qaL, bs);
            bs = cfma(ld_nc(gc + 1), qa, bs);
            bs = cfma(ld_nc(gc + 2), qaR, bs);
            bs = cfma(ld_nc(gc + 3), qbL, bs);
            bs = cfma(ld_nc(gc + 4), qb, bs);
            bs = cfma(ld_nc(gc + 5), qbR, bs);
            bs = cfma(ld_nc(gc + 6), qcL, bs);
            bs = cfma(ld_nc(gc + 7), qc, bs);
            bs = cfma(ld_nc(gc + 8), qcR, bs);
            uc = qb;
          }
          A.b_coarse[Yc * Nc + ccol] = bs;
          A.u_coarse[Yc * Nc + ccol] = uc;
        }
      }
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      um[s] = u0[s];
      u0[s] = up[s];
    }
  };

  for (int Yc = Y0 - 1; Yc < Y1; ++Yc) {
    step(IC<1>{}, 3 * Yc + 1);
    step(IC<2>{}, 3 * Yc + 2);
    step(IC<0>{}, 3 * Yc + 3);
  }
  // the boundary coarse row nc belongs to the range that ends there
  if (A.has_coarse && Y1 == nc && cemit) {
    A.b_coarse[nc * Nc + ccol] = cz<float>();
    A.u_coarse[nc * Nc + ccol] = cz<float>();
  }
}

// One warp: units [ubeg, uend).  srow = row[4][9], somd = omd[16] (shared).
// Returns this lane's sum of |r|^2 over owned interior vertices.
__device__ __forceinline__ float strip2w_run(const Sweep2wArgs& A, int ubeg, int uend,
                                             const cplx<float>* srow, const cplx<float>* somd) {
  const int n = A.n, nc = n / 3;
  float nrm = 0.f;
  int unit = ubeg;
  while (unit < uend) {
    const int strip = unit / nc, Y0 = unit % nc;
    const int Y1 = min(nc, Y0 + (uend - unit));
    unit += Y1 - Y0;
    const bool inner = 3 * Y0 - 3 >= 1 && 3 * Y1 + 4 <= n - 1;
    if (A.scells == 9) {
      if (inner) strip2w_segment<true>(A, strip, Y0, Y1, srow, somd, nrm);
      else strip2w_segment<false>(A, strip, Y0, Y1, srow, somd, nrm);
    } else if (A.hier && !A.hb) {
      if (inner) strip2w2_segment<true, true>(A, strip, Y0, Y1, srow, somd, nrm);
      else strip2w2_segment<false, true>(A, strip, Y0, Y1, srow, somd, nrm);
    } else {
      if (inner) strip2w2_segment<true, false>(A, strip, Y0, Y1, srow, somd, nrm);
      else strip2w2_segment<false, false>(A, strip, Y0, Y1, srow, somd, nrm);
    }
  }
  return nrm;
}

constexpr int kS2wThreads = 256;
#ifndef MG_S2W_MINB
#define MG_S2W_MINB 2  // resident blocks per SM the register budget is sized for
#endif

__global__ void __launch_bounds__(kS2wThreads, MG_S2W_MINB) sweep2w_kernel(const Sweep2wArgs A) {
  __shared__ cplx<float> s_row[36];
  __shared__ cplx<float> s_omd[16];
  __shared__ double s_red[kS2wThreads / 32];
  for (int i = threadIdx.x; i < 36; i += kS2wThreads) s_row[i] = A.row[i / 9][i % 9];
  for (int i = threadIdx.x; i < 16; i += kS2wThreads) s_omd[i] = A.omd[i];
  __syncthreads();
  const long long W = (long long)gridDim.x * (kS2wThreads / 32);
  const long long gw = (long long)blockIdx.x * (kS2wThreads / 32) + (threadIdx.x >> 5);
  const int ub = (int)(A.nunits * gw / W), ue = (int)(A.nunits * (gw + 1) / W);
  const float nrm = strip2w_run(A, ub, ue, s_row, s_omd);
  if (A.fine && A.norm2 != nullptr)
    block_norm_finish_tile<kS2wThreads>((double)nrm, s_red, A.partial, A.ticket, A.norm2, blockIdx.x,
                                         gridDim.x);
}

}  // namespace mg
