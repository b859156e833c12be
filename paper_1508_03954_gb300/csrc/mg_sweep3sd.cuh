// mg_sweep3sd.cuh -- separable z-marching sweep for large 3D levels with a
// constant shift, complex128 (sm_103a).
//
// The step is the fused fine-to-coarse step of Appendix A Algorithm 4 on one
// level, with the single-touch pending correction of Algorithm 2 on the
// finest level (u = U + P corr_{l-1} formed on the fly, U' = u + T du written
// once) and the coarse right-hand side b_{l-1} = R r_l + G_{l-1} u_{l-1}
// (G = R H P, the Galerkin row of Eq. HTMG's R(b - H uhat) by linearity).
//
// Operator (Section 4, Appendix B, separable for a constant shift under
// coordinate-wise scaling):
//     H u = M_x [ M_y (K_z - phi M_z) u + K_y M_z u ] + K_x (M_y M_z u),
// seven 3-tap passes along single axes.  The 1D rows depend on the vertex's
// class along that axis (left / right cell rotated or not).
//
// What bounds it on GB300: the FP64 pipe (2 FMA per clock per SM; an FP64
// warp instruction holds a sub-partition's FP64 unit for 64 cycles whatever
// its active lanes).  Bytes are not the limit (about 50 B per vertex against
// ~80 FP64 operations), so the kernel spends integer, shuffle and shared
// memory work to save FP64 instructions:
//  * unscaled (real) rows are symmetric, so each real pass factors the sum of
//    the outer neighbours (5 instead of 6 operations per component for the
//    z-pass pair, 8 instead of 9 for the y-pass pair, 6 instead of 7 for the
//    x-pass with the subtraction from b folded in);
//  * the x-restriction of two rows is computed by 20 lanes at once (values
//    gathered by shuffles), not by every lane of each row;
//  * Jacobi and the Galerkin rows take real coefficients when every lane of
//    the warp has real ones;
//  * one plane of prefetch is enough: a plane step is ~20 us of FP64 work.
//
// Layout (the one of the complex64 sweep): a block of 512 threads owns an x-y
// tile of 9 x 9 coarse cells (27 x 27 fine columns) and a range of coarse
// planes; lane = x and warp w holds rows 2w, 2w+1 of the 32 x 32 box of fine
// columns [x0-3, x0+28] x [y0-3, y0+28], marching z with u(z-1), u(z), u(z+1)
// in registers.  The residual box is [x0-2, x0+27]^2.  One barrier per fine
// plane; the (tile, coarse plane) units are split into contiguous ranges of
// equal FP64 cost (tabulated on the host: units with scaled rows cost more),
// one block per SM.  Level sizes stay below 2^31 vertices.
#pragma once
#include "mg_kernels.cuh"
#include "mg_sweep3s.cuh"
#include "mg_defect3.cuh"

namespace mg {

struct Sweep3sdArgs {
  int n, fine, has_coarse, hb, hier;
  int tiles_x;              // x-y tiles per axis (9 coarse cells each)
  long long nunits;         // tiles_x^2 * (n / 3)
  const unsigned* upref;    // prefix sums of the unit costs, nunits + 1 entries
  const unsigned* usplit;   // block b takes units [usplit[b], usplit[b+1]) (null: by upref)
  const cplx<double>* u;    // fine: pending U; coarse: u_l
  const cplx<double>* c;    // pending correction on level l-1 (fine only; may be null)
  const cplx<double>* b;
  cplx<double>* out;        // fine: U'; coarse: T du
  cplx<double>* b_coarse;
  cplx<double>* u_coarse;
  cplx<double>* idu;        // BPX: du at the c-points (I du, level l-1 layout); the
                            // output then holds du, and the correction stage
                            // subtracts P I du (corr_l = du + P (corr_{l-1} - I du))
  const uint8_t* typ;       // axis class per fine index (n+1)
  const uint8_t* gtyp;      // Galerkin row class per coarse index (n/3+1)
  const cplx<double>* gcoef;  // [kMaxG3^3][27]
  unsigned greal;           // bit k: 1D Galerkin class k has real rows
  // by axis class: mass row (l, c, r), stiffness row, stiffness - phi * mass
  cplx<double> row[4][9];
  cplx<double> omd[64];     // omega / D per vertex type tx + 4 ty + 16 tz
  double* partial;
  unsigned* ticket;
  double* norm2;
};

struct Sweep3sdShared {
  cplx<double> za[2][32][32];  // M_z u of the plane (two planes in flight)
  cplx<double> zb[2][32][32];  // (K_z - phi M_z) u
  cplx<double> rx[2][32][10];  // r restricted along x at the c-columns C0 .. C0+9
  cplx<double> q[3][11][11];   // u at the c-points of three c-planes, C0-1 .. C0+9
  cplx<double> cc[12][12];     // one coarse plane of the pending correction, C0-1 .. C0+10
  cplx<double> ccx[12][32];    // that plane interpolated along x to the box's columns
  cplx<double> cxy[2][32][32]; // P c at this column on the two coarse planes bracketing z + 1
  cplx<double> pu[32][32];     // U(z + 1), copied asynchronously one step ahead
  cplx<double> pb[32][32];     // b(z), copied asynchronously one step ahead
  cplx<double> row[4][9];
  cplx<double> omd[64];
};

// weight of the left (D0) and right (D1) coarse vertex at fine offset O
template <int O> __device__ __forceinline__ constexpr double D0() {
  return O == 0 ? 1.0 : (O == 1 ? 2.0 / 3.0 : 1.0 / 3.0);
}
template <int O> __device__ __forceinline__ constexpr double D1() {
  return O == 0 ? 0.0 : (O == 1 ? 1.0 / 3.0 : 2.0 / 3.0);
}

// 1D restriction of five values at offsets -2..2: weights 1/3, 2/3, 1, 2/3, 1/3
__device__ __forceinline__ cplx<double> restrict5d(cplx<double> m2, cplx<double> m1, cplx<double> z,
                                                   cplx<double> p1, cplx<double> p2) {
  return cplx<double>{fma(m2.x + p2.x, 1.0 / 3.0, fma(m1.x + p1.x, 2.0 / 3.0, z.x)),
                      fma(m2.y + p2.y, 1.0 / 3.0, fma(m1.y + p1.y, 2.0 / 3.0, z.y))};
}
__device__ __forceinline__ cplx<double> shfl_idx_cd(cplx<double> v, int src) {
  return cplx<double>{__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src)};
}
// 16-byte asynchronous copy global -> shared; zero-filled when !valid (no
// global read then)
__device__ __forceinline__ void cp_async16_zfill(void* dst, const void* src, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// all but the most recent group complete
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

__global__ void __launch_bounds__(512, 1) sweep3sd_kernel(const Sweep3sdArgs A) {
  constexpr int NTHR = 512, NW = 16, RPT = 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double s_red[NTHR / 32];
  Sweep3sdShared& S = *reinterpret_cast<Sweep3sdShared*>(smem_raw);
  using C = cplx<double>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n = A.n, N = n + 1, nc = n / 3;
  const int NN = N * N, Nc = nc + 1, NNc = Nc * Nc;
  for (int i = threadIdx.x; i < 36; i += NTHR) S.row[i / 9][i % 9] = A.row[i / 9][i % 9];
  for (int i = threadIdx.x; i < 64; i += NTHR) S.omd[i] = A.omd[i];
  const bool use_c = A.fine && A.c != nullptr;
  const bool bpx = A.hier && !A.hb;
  // y/z-restriction and coarse outputs: 4 warps x 25 lanes take the 10 x 10
  // coarse columns C0 .. C0+9 (column 9 only matters on the last tile).  The
  // four are warps 0, 4 (sub-partition 0) and 3, 7 (sub-partition 3): those
  // sub-partitions also hold warps 0 and 15, whose box rows 0 and 31 need no
  // residual, so every sub-partition's FP64 unit gets about the same work
  // between two barriers
  const int wsel = warp == 0 ? 0 : (warp == 4 ? 1 : (warp == 3 ? 2 : (warp == 7 ? 3 : -1)));
  const int ek = (wsel >= 0 && lane < 25) ? wsel * 25 + lane : -1;
  const bool emit = ek >= 0 && A.has_coarse;
  const int ejx = emit ? ek % 10 : 0, ejy = emit ? ek / 10 : 0;
  // unscaled rows are symmetric: (outer sum) * c0 + centre * c1
  const double m0 = A.row[0][0].x, m1 = A.row[0][1].x;
  const double k0 = A.row[0][3].x, k1 = A.row[0][4].x;
  const double p0 = A.row[0][6].x, p1 = A.row[0][7].x;
  const int ox = lane % 3;
  const bool cpx = ox == 0;
  int by[RPT], oy[RPT];
  bool cpy[RPT], rrow[RPT];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    by[r] = RPT * warp + r;  // box row
    oy[r] = by[r] % 3;
    cpy[r] = oy[r] == 0;
    rrow[r] = by[r] >= 1 && by[r] <= 30;
  }
  // d-linear weights of the right / upper coarse vertex at fine offset o
  // (formed where used: they would otherwise hold registers all along)
  auto w1 = [](int o) { return o == 0 ? 0.0 : (o == 1 ? 1.0 / 3.0 : 2.0 / 3.0); };
  // x-restriction gather: lane = 10 * rr + jc (lanes 0..19) takes row rr of
  // the warp's pair at c-column jc, from box columns 3 jc + 1 .. 3 jc + 5
  const int xr_rr = lane / 10, xr_jc = lane % 10;
  const bool xr_act = lane < 20;
  double nrm = 0.0;

  // this block's units: those whose prefix cost lies in [W b / B, W (b+1) / B)
  const long long U = A.nunits;
  const unsigned long long Wt = A.upref[U];
  auto first_at = [&](unsigned long long target) -> int {
    long long lo = 0, hi = U;  // first i in [0, U] with upref[i] >= target
    while (lo < hi) {
      const long long mid = (lo + hi) >> 1;
      if ((unsigned long long)__ldg(A.upref + mid) >= target) hi = mid; else lo = mid + 1;
    }
    return (int)lo;
  };
  int unit = A.usplit != nullptr ? (int)A.usplit[blockIdx.x] : first_at(Wt * blockIdx.x / gridDim.x);
  const int uend = A.usplit != nullptr ? (int)A.usplit[blockIdx.x + 1] : first_at(Wt * (blockIdx.x + 1) / gridDim.x);
  while (unit < uend) {
    const int tile = unit / nc, Z0 = unit % nc;
    const int Z1 = min(nc, Z0 + (uend - unit));
    unit += Z1 - Z0;
    const int C0x = (tile % A.tiles_x) * 9, C0y = (tile / A.tiles_x) * 9;
    const int x0 = 3 * C0x, y0 = 3 * C0y;
    const int gx = x0 - 3 + lane;
    const bool lastx = C0x + 9 >= nc, lasty = C0y + 9 >= nc;
    const int tx = (gx >= 0 && gx <= n) ? (int)A.typ[gx] : 0;
    // only the residual box (lanes 1..30) takes x-rows
    const bool xreal = __all_sync(0xffffffffu, tx == 0 || lane == 0 || lane == 31);
    int gy[RPT], col[RPT], ty[RPT];
    bool colin[RPT], owncol[RPT], yreal[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      gy[r] = y0 - 3 + by[r];
      colin[r] = gx > 0 && gx < n && gy[r] > 0 && gy[r] < n;
      owncol[r] = lane >= 3 && (lane < 30 || (lane == 30 && lastx)) && by[r] >= 3 &&
                  (by[r] < 30 || (by[r] == 30 && lasty)) && gx <= n && gy[r] <= n;
      col[r] = gy[r] * N + gx;  // used only for owned or interior columns
      ty[r] = (gy[r] >= 0 && gy[r] <= n) ? (int)A.typ[gy[r]] : 0;
      yreal[r] = ty[r] == 0;
    }
    const int zs = 3 * Z0 - 2;
    auto qslot = [](int Zc) { return (Zc + 3) % 3; };
    auto ldU = [&](int z, int r) -> C {
      return (colin[r] && z > 0 && z < n) ? ldg_c(A.u + (z * NN + col[r])) : cz<double>();
    };
    // the thread's own slots of the staged planes (row r at +32)
    C* spu = &S.pu[by[0]][lane];
    C* spb = &S.pb[by[0]][lane];
    auto cpU = [&](int z, int r) {
      const bool v = colin[r] && z > 0 && z < n;
      cp_async16_zfill(spu + 32 * r, v ? (const void*)(A.u + (z * NN + col[r])) : (const void*)A.u, v);
    };
    auto cpB = [&](int z, int r) {
      const bool v = rrow[r] && colin[r] && z > 0 && z < n;
      cp_async16_zfill(spb + 32 * r, v ? (const void*)(A.b + (z * NN + col[r])) : (const void*)A.b, v);
    };
    auto ld_cc = [&](int Zc) -> C {
      const int t = threadIdx.x;
      const int cx = C0x - 1 + t % 12, cy = C0y - 1 + t / 12;
      return (use_c && t < 144 && Zc >= 0 && Zc <= nc && cx >= 0 && cx <= nc && cy >= 0 && cy <= nc)
                 ? ldg_c(A.c + (Zc * NNc + cy * Nc + cx))
                 : cz<double>();
    };
    // the coarse plane in S.cc interpolated separably: along x to the box's
    // lanes by 384 threads (S.ccx), then along y per column
    auto xint_cc = [&]() {
      if (threadIdx.x < 384) {
        const int jy = threadIdx.x >> 5, jx = lane / 3;
        const double wx1 = w1(ox), wx0 = 1.0 - wx1;
        const C a = S.cc[jy][jx], b2 = S.cc[jy][jx + 1];
        S.ccx[jy][lane] = C{fma(wx1, b2.x, wx0 * a.x), fma(wx1, b2.y, wx0 * a.y)};
      }
    };
    auto bil_cc = [&](int r) -> C {
      const int jy = by[r] / 3;
      const double wy1 = w1(oy[r]), wy0 = 1.0 - wy1;
      const C a = S.ccx[jy][lane], c2 = S.ccx[jy + 1][lane];
      return C{fma(wy1, c2.x, wy0 * a.x), fma(wy1, c2.y, wy0 * a.y)};
    };

    __syncthreads();  // the previous range's shared memory is free
    // per-column state kept in shared memory (private to the thread): the
    // coarse correction on the two planes bracketing z + 1
    C* cxy0 = &S.cxy[0][by[0]][lane];  // [r * 32]: row r
    C* cxy1 = &S.cxy[1][by[0]][lane];
    C ccpre = cz<double>();
#pragma unroll
    for (int r = 0; r < RPT; ++r) cxy0[32 * r] = cxy1[32 * r] = cz<double>();
    // one coarse plane of the pending correction through S.cc: threads < 144
    // load it
    if (use_c) {
      if (threadIdx.x < 144) S.cc[threadIdx.x / 12][threadIdx.x % 12] = ld_cc(Z0 - 1);
      __syncthreads();
      xint_cc();
      __syncthreads();
#pragma unroll
      for (int r = 0; r < RPT; ++r) cxy0[32 * r] = bil_cc(r);
      __syncthreads();
      if (threadIdx.x < 144) S.cc[threadIdx.x / 12][threadIdx.x % 12] = ld_cc(Z0);
      __syncthreads();
      xint_cc();
      __syncthreads();
#pragma unroll
      for (int r = 0; r < RPT; ++r) cxy1[32 * r] = bil_cc(r);
      ccpre = ld_cc(Z0 + 1);
      __syncthreads();
    }
    C um[RPT], u0[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      // u on planes 3 Z0 - 3 (c-plane Z0 - 1) and 3 Z0 - 2
      um[r] = ldU(3 * Z0 - 3, r);
      u0[r] = ldU(3 * Z0 - 2, r);
      if (use_c && colin[r]) {
        if (3 * Z0 - 3 > 0) um[r] = um[r] + cxy0[32 * r];
        if (3 * Z0 - 2 > 0) {
          u0[r] = rfma(D0<1>(), cxy0[32 * r], u0[r]);
          u0[r] = rfma(D1<1>(), cxy1[32 * r], u0[r]);
        }
      }
      if (cpx && cpy[r]) S.q[qslot(Z0 - 1)][by[r] / 3][lane / 3] = um[r];
    }
    // one plane staged ahead: step z takes U(z + 1) and b(z) from shared
    // memory; groups alternate U, b so that each wait leaves the newest
    // group in flight
#pragma unroll
    for (int r = 0; r < RPT; ++r) cpU(3 * Z0 - 1, r);
    cp_async_commit();
#pragma unroll
    for (int r = 0; r < RPT; ++r) cpB(3 * Z0 - 2, r);
    cp_async_commit();
    C accA = cz<double>(), accB = cz<double>();

    // deferred work of residual plane zd, after the barrier of the next step
    auto deferred = [&](auto ozc, int zd) {
      constexpr int OZD = decltype(ozc)::value;
      const int bufd = zd & 1;
      if (emit && ejx < 9 && ejy < 9) {
        const int ry_ = 3 + 3 * ejy;
        const C ry = restrict5d(S.rx[bufd][ry_ - 2][ejx], S.rx[bufd][ry_ - 1][ejx], S.rx[bufd][ry_][ejx],
                                S.rx[bufd][ry_ + 1][ejx], S.rx[bufd][ry_ + 2][ejx]);
        if (OZD == 0) {
          accA = accB + ry;
          accB = cz<double>();
        } else {
          accA = rfma(D0<OZD>(), ry, accA);
          accB = rfma(D1<OZD>(), ry, accB);
        }
      }
      if (OZD == 2 && A.has_coarse) {
        const int Zc = (zd - 2) / 3;
        const int cx = C0x + ejx, cy = C0y + ejy;
        const bool act = emit && Zc >= Z0 && Zc < Z1 && cx <= nc && cy <= nc && (ejx < 9 || cx == nc) &&
                         (ejy < 9 || cy == nc);
        const bool inner = act && cx > 0 && cx < nc && cy > 0 && cy < nc && Zc > 0 && Zc < nc;
        int gt = 0;
        bool gr = true;
        if (inner) {
          const int gxx = A.gtyp[cx], gyy = A.gtyp[cy], gzz = A.gtyp[Zc];
          gt = gxx + kMaxG3 * (gyy + kMaxG3 * gzz);
          gr = ((A.greal >> gxx) & (A.greal >> gyy) & (A.greal >> gzz) & 1u) != 0;
        }
        const bool allreal = __all_sync(0xffffffffu, gr);
        if (act) {
          C bs = cz<double>(), uc = cz<double>();
          if (inner) {
            bs = accA;
            const C* gc = A.gcoef + gt * 27;
            if (allreal) {
#pragma unroll
              for (int kz = 0; kz < 3; ++kz) {
                const int qs = qslot(Zc - 1 + kz);
#pragma unroll
                for (int k = 0; k < 9; ++k)
                  bs = rfma(__ldg(&gc[kz * 9 + k].x), S.q[qs][ejy + k / 3][ejx + k % 3], bs);
              }
            } else {
#pragma unroll
              for (int kz = 0; kz < 3; ++kz) {
                const int qs = qslot(Zc - 1 + kz);
#pragma unroll
                for (int k = 0; k < 9; ++k)
                  bs = cfma(ldg_c(gc + kz * 9 + k), S.q[qs][ejy + k / 3][ejx + k % 3], bs);
              }
            }
            uc = S.q[qslot(Zc)][ejy + 1][ejx + 1];
          }
          const int ci = Zc * NNc + cy * Nc + cx;
          A.b_coarse[ci] = bs;
          A.u_coarse[ci] = uc;
        }
      }
    };

    // one fine step: u plane z + 1 in, residual plane z, outputs
    auto step = [&](auto ozc, int z) {
      constexpr int OZ = decltype(ozc)::value;
      constexpr int OZP = (OZ + 1) % 3;
      const int zp = z + 1;
      const int buf = z & 1;
      const int tz = (z >= 0 && z <= n) ? (int)__ldg(A.typ + z) : 0;
      // phase 1: u on plane z + 1, z-pass of both rows
      C up[RPT], za[RPT], zb[RPT];
      cp_async_wait_1();  // U(z + 1) is in
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        if (OZP == 0 && use_c) cxy0[32 * r] = cxy1[32 * r];
        up[r] = spu[32 * r];
        if (use_c && colin[r] && zp > 0 && zp < n) {
          up[r] = rfma(D0<OZP>(), cxy0[32 * r], up[r]);
          if (OZP != 0) up[r] = rfma(D1<OZP>(), cxy1[32 * r], up[r]);
        }
        if (OZP == 0 && cpx && cpy[r]) S.q[qslot(zp / 3)][by[r] / 3][lane / 3] = up[r];
        if (tz == 0) {
          const C s = um[r] + up[r];
          za[r] = C{fma(m0, s.x, m1 * u0[r].x), fma(m0, s.y, m1 * u0[r].y)};
          zb[r] = C{fma(p0, s.x, p1 * u0[r].x), fma(p0, s.y, p1 * u0[r].y)};
        } else {
          za[r] = tap3dc_acc(&S.row[tz][0], um[r], u0[r], up[r], cz<double>());
          zb[r] = tap3dc_acc(&S.row[tz][6], um[r], u0[r], up[r], cz<double>());
        }
        S.za[buf][by[r]][lane] = za[r];
        S.zb[buf][by[r]][lane] = zb[r];
      }
      // the slots were read above (their values feed za, zb): refill them
#pragma unroll
      for (int r = 0; r < RPT; ++r) cpU(z + 2, r);
      cp_async_commit();
      if (OZP == 2 && use_c && threadIdx.x < 144) S.cc[threadIdx.x / 12][threadIdx.x % 12] = ccpre;
      if (OZP == 0 && use_c) ccpre = ld_cc(zp / 3 + 2);
      __syncthreads();
      // phase 2: deferred work of plane z - 1; coarse correction plane for the next steps
      if (z > zs) deferred(IC<(OZ + 2) % 3>{}, z - 1);
      if (OZP == 2 && use_c) xint_cc();  // S.cc was refilled before the barrier
      if (OZP == 0 && use_c) {
#pragma unroll
        for (int r = 0; r < RPT; ++r) cxy1[32 * r] = bil_cc(r);
      }
      // phase 3: residuals on plane z; the pair's outer neighbour rows from shared memory
      const bool zin = z > 0 && z < n;
      const bool zown = (z >= 3 * Z0 && z < 3 * Z1) || z == n;
      const C aU = warp > 0 ? S.za[buf][by[0] - 1][lane] : cz<double>();
      const C bU = warp > 0 ? S.zb[buf][by[0] - 1][lane] : cz<double>();
      const C aD = warp < NW - 1 ? S.za[buf][by[RPT - 1] + 1][lane] : cz<double>();
      const C bD = warp < NW - 1 ? S.zb[buf][by[RPT - 1] + 1][lane] : cz<double>();
      C res[RPT];
      cp_async_wait_1();  // b(z) is in
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        res[r] = cz<double>();
        if (!rrow[r]) continue;  // warp-uniform
        // neighbour rows: the thread's own rows, the pair's outer ones from shared memory
        const C am = r == 0 ? aU : za[r > 0 ? r - 1 : 0], ap = r == RPT - 1 ? aD : za[r < RPT - 1 ? r + 1 : r];
        const C bm = r == 0 ? bU : zb[r > 0 ? r - 1 : 0], bp = r == RPT - 1 ? bD : zb[r < RPT - 1 ? r + 1 : r];
        C cy, ey;
        if (yreal[r]) {
          const C sa = am + ap, sb = bm + bp;
          cy = C{fma(k0, sa.x, fma(k1, za[r].x, fma(m0, sb.x, m1 * zb[r].x))),
                 fma(k0, sa.y, fma(k1, za[r].y, fma(m0, sb.y, m1 * zb[r].y)))};
          ey = C{fma(m0, sa.x, m1 * za[r].x), fma(m0, sa.y, m1 * za[r].y)};
        } else {
          const C* rw = &S.row[ty[r]][0];
          cy = tap3dc_acc(rw + 3, am, za[r], ap, tap3dc_acc(rw, bm, zb[r], bp, cz<double>()));
          ey = tap3dc_acc(rw, am, za[r], ap, cz<double>());
        }
        const C cl = shfl_cd(cy, 1, true), cr = shfl_cd(cy, 1, false);
        const C el = shfl_cd(ey, 1, true), er = shfl_cd(ey, 1, false);
        const C bb = (colin[r] && zin) ? spb[32 * r] : cz<double>();
        C rv;
        if (xreal) {
          // r = b - (K_x e + M_x c), symmetric rows
          const C se = el + er, sc = cl + cr;
          rv = C{fma(-k0, se.x, fma(-k1, ey.x, fma(-m0, sc.x, fma(-m1, cy.x, bb.x)))),
                 fma(-k0, se.y, fma(-k1, ey.y, fma(-m0, sc.y, fma(-m1, cy.y, bb.y))))};
        } else {
          const C* rw = &S.row[tx][0];
          rv = bb - tap3dc_acc(rw + 3, el, ey, er, tap3dc_acc(rw, cl, cy, cr, cz<double>()));
        }
        if (colin[r] && zin && lane >= 1 && lane <= 30) res[r] = rv;
        if (owncol[r] && zown) nrm = fma(res[r].x, res[r].x, fma(res[r].y, res[r].y, nrm));
        // Jacobi update, c-point mask (hb), outputs; BPX: I du at the owned
        // c-points (the correction stage subtracts P I du)
        const C om = S.omd[tx + 4 * ty[r] + 16 * tz];
        C du;
        if (__all_sync(0xffffffffu, om.y == 0.0))
          du = rmul(om.x, res[r]);
        else
          du = om * res[r];
        if (A.hb && OZ == 0 && cpx && cpy[r]) du = cz<double>();
        const C v = A.fine ? u0[r] + du : du;
        if (owncol[r] && zown) {
          A.out[z * NN + col[r]] = v;
          if (bpx && OZ == 0 && cpx && cpy[r]) A.idu[((z / 3) * Nc + gy[r] / 3) * Nc + gx / 3] = du;
        }
      }
      // restriction along x to the c-columns, both rows by 20 lanes
      if (A.has_coarse) {
        // gathered as (t0 + t4), (t1 + t3), t2 to keep few values live
        auto gather = [&](int k) -> C {
          const int src = min(3 * xr_jc + 1 + k, 31);
          const C a0 = shfl_idx_cd(res[0], src), a1 = shfl_idx_cd(res[1], src);
          return xr_rr == 0 ? a0 : a1;
        };
        C s04 = gather(0);
        s04 = s04 + gather(4);
        C s13 = gather(1);
        s13 = s13 + gather(3);
        const C t2 = gather(2);
        const bool xr_row = xr_rr ? rrow[1] : rrow[0];
        const int xr_by = xr_rr ? by[1] : by[0];
        if (xr_act && xr_row && 3 * xr_jc + 3 <= 30)
          S.rx[buf][xr_by][xr_jc] =
              C{fma(s04.x, 1.0 / 3.0, fma(s13.x, 2.0 / 3.0, t2.x)), fma(s04.y, 1.0 / 3.0, fma(s13.y, 2.0 / 3.0, t2.y))};
      }
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        cpB(z + 1, r);
        um[r] = u0[r];
        u0[r] = up[r];
      }
      cp_async_commit();
    };

    for (int Zc = Z0 - 1; Zc < Z1; ++Zc) {
      step(IC<1>{}, 3 * Zc + 1);
      step(IC<2>{}, 3 * Zc + 2);
      step(IC<0>{}, 3 * Zc + 3);
    }
    __syncthreads();
    deferred(IC<0>{}, 3 * Z1);
    // the boundary coarse plane nc belongs to the range that ends there
    if (Z1 == nc && emit) {
      const int cx = C0x + ejx, cy = C0y + ejy;
      if (cx <= nc && cy <= nc && (ejx < 9 || cx == nc) && (ejy < 9 || cy == nc)) {
        const int ci = nc * NNc + cy * Nc + cx;
        A.b_coarse[ci] = cz<double>();
        A.u_coarse[ci] = cz<double>();
      }
    }
  }
  if (A.fine && A.norm2 != nullptr)
    block_norm_finish_tile<NTHR>(nrm, s_red, A.partial, A.ticket, A.norm2, blockIdx.x, gridDim.x);
}

}  // namespace mg
