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
  int strips;           // 27-column strips
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
    if (3 * Y0 - 3 >= 1 && 3 * Y1 + 4 <= n - 1)
      strip2w_segment<true>(A, strip, Y0, Y1, srow, somd, nrm);
    else
      strip2w_segment<false>(A, strip, Y0, Y1, srow, somd, nrm);
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
