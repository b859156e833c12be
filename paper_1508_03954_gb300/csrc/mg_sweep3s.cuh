// mg_sweep3s.cuh -- separable z-marching sweep for large 3D levels with a
// constant shift, complex64 (sm_103a).
//
// The step is the one of mg_sweep3d.cuh (Appendix A Algorithm 4 on one level,
// the single-touch pending correction of Algorithm 2, coarse right-hand side
// b_{l-1} = R r_l + G_{l-1} u_{l-1}); what changes is how the residual is
// evaluated and how the work is laid out.
//
// Operator.  With coordinate-wise exterior scaling every cell is a tensor
// product of 1D cells, so the assembled level operator with a constant shift
// phi is a sum of tensor products of assembled 1D tridiagonal rows
// (Section 3: K_c = sum_j (x)_a (K if a == j else M), M_c = (x)_a M):
//     H u = M_x [ M_y (K_z - phi M_z) u + K_y M_z u ] + K_x (M_y M_z u).
// The rows depend only on the vertex's scaling class along that axis (left
// and right cell plain or rotated), so seven 3-tap passes replace the
// 27-point row, and rows in the unscaled interior take real coefficients.
//
// Layout.  A block of 1024 threads owns an x-y tile of 9 x 9 coarse cells
// (27 x 27 fine vertices) and a range of coarse planes; lane = x and warp = y
// of a 32 x 32 box of fine columns [x0-3, x0+28] x [y0-3, y0+28].  Each
// thread marches its column along z holding u(z-1), u(z), u(z+1) in
// registers: the z-pass runs in registers, the y-pass reads the neighbouring
// rows from shared memory, the x-pass takes its neighbours by warp shuffles.
// The r box is [x0-2, x0+27]^2 (lanes/warps 1..30), enough for the
// restriction of the owned coarse vertices and for the c-point Jacobi update
// of the next tile's first c-point (BPX).  One barrier per fine plane.
//
// Work split.  The (tile, coarse plane) units of the level are split into
// gridDim.x contiguous ranges of equal size (one block per SM), so the load
// is balanced to one coarse plane; a range may continue into the next tile.
#pragma once
#include "mg_kernels.cuh"
#include "mg_sweep3d.cuh"

namespace mg {

constexpr int kS3sThreads = 1024;

struct Sweep3sArgs {
  int n, fine, first, has_coarse, hb, hier;
  int tiles_x;          // x-y tiles per axis (9 coarse cells each)
  long long nunits;     // tiles_x^2 * (n / 3)
  const cplx<float>* u;     // fine: pending U; coarse: u_l
  const cplx<float>* c;     // pending correction on level l-1 (fine, may be null)
  const cplx<float>* b;
  cplx<float>* out;         // fine: U'; coarse: T du
  cplx<float>* b_coarse;
  cplx<float>* u_coarse;
  const uint8_t* typ;       // axis class per fine index (n+1)
  const uint8_t* gtyp;      // Galerkin row class per coarse index (n/3+1)
  const cplx<float>* gcoef; // [kMaxG3^3][27]
  // by axis class: mass row (l, c, r), stiffness row, stiffness - phi * mass
  cplx<float> row[4][9];
  cplx<float> omd[64];      // omega / D per vertex type tx + 4 ty + 16 tz
  double* partial;
  unsigned* ticket;
  double* norm2;
};

struct Sweep3sShared {
  cplx<float> za[2][32][32];  // M_z u of the plane (two planes in flight)
  cplx<float> zb[2][32][32];  // (K_z - phi M_z) u
  cplx<float> pv[3][32][32];  // BPX: u + du of the fine planes waiting for P I du
  cplx<float> rx[2][32][10];  // r restricted along x at the c-columns of coarse C0 .. C0+9
  cplx<float> dc[10][10];     // du at the c-points of the last c-plane, coarse C0 .. C0+9
  cplx<float> q[3][11][11];   // u at the c-points of three c-planes, coarse C0-1 .. C0+9
  cplx<float> cc[12][12];     // one coarse plane of the pending correction, C0-1 .. C0+10
  cplx<float> row[4][9];
  cplx<float> omd[64];
};

template <int V> struct IC { static constexpr int value = V; };

__device__ __forceinline__ cplx<float> tap3r(float c0, float c1, float c2, cplx<float> a,
                                             cplx<float> b, cplx<float> d) {
  return cplx<float>{fmaf(c2, d.x, fmaf(c1, b.x, c0 * a.x)), fmaf(c2, d.y, fmaf(c1, b.y, c0 * a.y))};
}
__device__ __forceinline__ cplx<float> tap3r_acc(float c0, float c1, float c2, cplx<float> a,
                                                 cplx<float> b, cplx<float> d, cplx<float> acc) {
  return cplx<float>{fmaf(c2, d.x, fmaf(c1, b.x, fmaf(c0, a.x, acc.x))),
                     fmaf(c2, d.y, fmaf(c1, b.y, fmaf(c0, a.y, acc.y)))};
}
__device__ __forceinline__ cplx<float> tap3c_acc(const cplx<float>* c, cplx<float> a, cplx<float> b,
                                                 cplx<float> d, cplx<float> acc) {
  return cfma(c[2], d, cfma(c[1], b, cfma(c[0], a, acc)));
}
__device__ __forceinline__ cplx<float> shfl_c(cplx<float> v, int delta, bool up) {
  cplx<float> o;
  if (up) {
    o.x = __shfl_up_sync(0xffffffffu, v.x, delta);
    o.y = __shfl_up_sync(0xffffffffu, v.y, delta);
  } else {
    o.x = __shfl_down_sync(0xffffffffu, v.x, delta);
    o.y = __shfl_down_sync(0xffffffffu, v.y, delta);
  }
  return o;
}
__device__ __forceinline__ cplx<float> ld_nc(const cplx<float>* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return cplx<float>{v.x, v.y};
}

// 1D restriction of five values at offsets -2..2: weights 1/3, 2/3, 1, 2/3, 1/3
__device__ __forceinline__ cplx<float> restrict5f(cplx<float> m2, cplx<float> m1, cplx<float> z,
                                                  cplx<float> p1, cplx<float> p2) {
  return cplx<float>{fmaf(m2.x + p2.x, 1.f / 3.f, fmaf(m1.x + p1.x, 2.f / 3.f, z.x)),
                     fmaf(m2.y + p2.y, 1.f / 3.f, fmaf(m1.y + p1.y, 2.f / 3.f, z.y))};
}

// weight of the left (W0) and right (W1) coarse vertex at fine offset o
template <int O> __device__ __forceinline__ constexpr float W0() {
  return O == 0 ? 1.f : (O == 1 ? 2.f / 3.f : 1.f / 3.f);
}
template <int O> __device__ __forceinline__ constexpr float W1() {
  return O == 0 ? 0.f : (O == 1 ? 1.f / 3.f : 2.f / 3.f);
}

__global__ void __launch_bounds__(kS3sThreads, 1) sweep3s_kernel(const Sweep3sArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double s_red[32];
  Sweep3sShared& S = *reinterpret_cast<Sweep3sShared*>(smem_raw);
  using C = cplx<float>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n = A.n, N = n + 1, nc = n / 3;
  const long long NN = (long long)N * N, Nc = nc + 1, NNc = Nc * Nc;
  for (int i = threadIdx.x; i < 36; i += kS3sThreads) S.row[i / 9][i % 9] = A.row[i / 9][i % 9];
  for (int i = threadIdx.x; i < 64; i += kS3sThreads) S.omd[i] = A.omd[i];
  const bool zero_u = A.fine && A.first;
  const bool use_c = A.fine && !A.first && A.c != nullptr;
  const bool bpx = A.hier && !A.hb;
  // restriction and coarse outputs: 4 warps x 25 lanes take the 10 x 10
  // coarse columns C0 .. C0+9 (column 9 only matters on the last tile)
  const int ek = (warp < 4 && lane < 25) ? warp * 25 + lane : -1;
  const bool emit = ek >= 0 && A.has_coarse;
  const int ejx = emit ? ek % 10 : 0, ejy = emit ? ek / 10 : 0;
  // the real rows of the unscaled interior: mass h/6 (1, 4, 1), stiffness, shifted stiffness
  const float m0 = A.row[0][0].x, m1 = A.row[0][1].x, m2 = A.row[0][2].x;
  const float k0 = A.row[0][3].x, k1 = A.row[0][4].x, k2 = A.row[0][5].x;
  const float p0 = A.row[0][6].x, p1 = A.row[0][7].x, p2 = A.row[0][8].x;
  const int ox = lane % 3, oy = warp % 3;
  const float wx1 = ox == 0 ? 0.f : (ox == 1 ? 1.f / 3.f : 2.f / 3.f), wx0 = 1.f - wx1;
  const float wy1 = oy == 0 ? 0.f : (oy == 1 ? 1.f / 3.f : 2.f / 3.f), wy0 = 1.f - wy1;
  const bool cpx = ox == 0, cpy = oy == 0;  // c-point column (the box origin is a c-point)
  const bool rrow = warp >= 1 && warp <= 30;
  float nrm = 0.f;

  const long long U = A.nunits;
  long long unit = U * blockIdx.x / gridDim.x;
  const long long uend = U * (blockIdx.x + 1) / gridDim.x;
  while (unit < uend) {
    const int tile = (int)(unit / nc), Z0 = (int)(unit % nc);
    const int Z1 = (int)min((long long)nc, (long long)Z0 + (uend - unit));
    unit += Z1 - Z0;
    const int C0x = (tile % A.tiles_x) * 9, C0y = (tile / A.tiles_x) * 9;
    const int x0 = 3 * C0x, y0 = 3 * C0y;
    const int gx = x0 - 3 + lane, gy = y0 - 3 + warp;
    const bool colin = gx > 0 && gx < n && gy > 0 && gy < n;
    const bool lastx = C0x + 9 >= nc, lasty = C0y + 9 >= nc;
    const bool owncol = lane >= 3 && (lane < 30 || (lane == 30 && lastx)) && warp >= 3 &&
                        (warp < 30 || (warp == 30 && lasty)) && gx <= n && gy <= n;
    const long long col = (long long)gy * N + gx;  // used only for owned or interior columns
    const int tx = (gx >= 0 && gx <= n) ? (int)A.typ[gx] : 0;
    const int ty = (gy >= 0 && gy <= n) ? (int)A.typ[gy] : 0;
    const bool xreal = __all_sync(0xffffffffu, tx == 0);
    const bool yreal = ty == 0;
    const int zs = 3 * Z0 - 2;
    auto qslot = [](int Zc) { return (Zc + 3) % 3; };
    auto ldU = [&](int z) -> C {
      return (!zero_u && colin && z > 0 && z < n) ? ld_nc(A.u + z * NN + col) : cz<float>();
    };
    auto ldB = [&](int z) -> C {
      return (colin && z > 0 && z < n) ? ld_nc(A.b + z * NN + col) : cz<float>();
    };
    auto ld_cc = [&](int Zc) -> C {
      const int t = threadIdx.x;
      const int cx = C0x - 1 + t % 12, cy = C0y - 1 + t / 12;
      return (use_c && t < 144 && Zc >= 0 && Zc <= nc && cx >= 0 && cx <= nc && cy >= 0 && cy <= nc)
                 ? ld_nc(A.c + Zc * NNc + (long long)cy * Nc + cx)
                 : cz<float>();
    };
    // bilinear interpolation of the coarse plane in S.cc to this column
    auto bil_cc = [&]() -> C {
      const int jx = lane / 3, jy = warp / 3;
      const C a = S.cc[jy][jx], b2 = S.cc[jy][jx + 1], c2 = S.cc[jy + 1][jx], d2 = S.cc[jy + 1][jx + 1];
      return cplx<float>{wy0 * (wx0 * a.x + wx1 * b2.x) + wy1 * (wx0 * c2.x + wx1 * d2.x),
                         wy0 * (wx0 * a.y + wx1 * b2.y) + wy1 * (wx0 * c2.y + wx1 * d2.y)};
    };

    __syncthreads();  // the previous segment's shared-memory reads are done
    C cxy0 = cz<float>(), cxy1 = cz<float>(), ccpre = cz<float>();
    if (use_c) {
      if (threadIdx.x < 144) S.cc[threadIdx.x / 12][threadIdx.x % 12] = ld_cc(Z0 - 1);
      __syncthreads();
      cxy0 = bil_cc();
      __syncthreads();
      if (threadIdx.x < 144) S.cc[threadIdx.x / 12][threadIdx.x % 12] = ld_cc(Z0);
      __syncthreads();
      cxy1 = bil_cc();
      ccpre = ld_cc(Z0 + 1);
      __syncthreads();
    }
    // u on planes 3 Z0 - 3 (c-plane Z0 - 1) and 3 Z0 - 2
    C um = ldU(3 * Z0 - 3), u0 = ldU(3 * Z0 - 2);
    if (use_c && colin) {
      if (3 * Z0 - 3 > 0) um = um + cxy0;
      if (3 * Z0 - 2 > 0) {
        u0 = rfma(W0<1>(), cxy0, u0);
        u0 = rfma(W1<1>(), cxy1, u0);
      }
    }
    if (cpx && cpy) S.q[qslot(Z0 - 1)][warp / 3][lane / 3] = um;
    // prefetch: step z uses U(z + 1) and b(z), slot z mod 3
    C pu[3], pb[3];
    pu[1] = ldU(3 * Z0 - 1);
    pu[2] = ldU(3 * Z0);
    pu[0] = ldU(3 * Z0 + 1);
    pb[1] = ldB(3 * Z0 - 2);
    pb[2] = ldB(3 * Z0 - 1);
    pb[0] = ldB(3 * Z0);
    C accA = cz<float>(), accB = cz<float>(), pidp = cz<float>();

    // deferred work of residual plane zd, after the barrier of the next step
    auto deferred = [&](auto ozc, int zd) {
      constexpr int OZD = decltype(ozc)::value;
      const int bufd = zd & 1;
      if (emit && ejx < 9 && ejy < 9) {
        const int by = 3 + 3 * ejy;
        const C r0 = S.rx[bufd][by - 2][ejx], r1 = S.rx[bufd][by - 1][ejx], r2 = S.rx[bufd][by][ejx];
        const C r3 = S.rx[bufd][by + 1][ejx], r4 = S.rx[bufd][by + 2][ejx];
        const C ry = cplx<float>{fmaf(r0.x + r4.x, 1.f / 3.f, fmaf(r1.x + r3.x, 2.f / 3.f, r2.x)),
                                 fmaf(r0.y + r4.y, 1.f / 3.f, fmaf(r1.y + r3.y, 2.f / 3.f, r2.y))};
        if (OZD == 0) {
          accA = accB + ry;
          accB = cz<float>();
        } else {
          accA = rfma(W0<OZD>(), ry, accA);
          accB = rfma(W1<OZD>(), ry, accB);
        }
        if (OZD == 2) {
          const int Zc = (zd - 2) / 3;
          const int cx = C0x + ejx, cy = C0y + ejy;
          if (Zc >= Z0 && Zc < Z1 && cx <= nc && cy <= nc && (ejx < 9 || cx == nc) && (ejy < 9 || cy == nc)) {
            const bool inner = cx > 0 && cx < nc && cy > 0 && cy < nc && Zc > 0 && Zc < nc;
            C bs = cz<float>(), uc = cz<float>();
            if (inner) {
              bs = accA;
              const int gt = A.gtyp[cx] + kMaxG3 * (A.gtyp[cy] + kMaxG3 * A.gtyp[Zc]);
              const C* gc = A.gcoef + gt * 27;
#pragma unroll
              for (int kz = 0; kz < 3; ++kz) {
                const int qs = qslot(Zc - 1 + kz);
#pragma unroll
                for (int k = 0; k < 9; ++k)
                  bs = cfma(ld_nc(gc + kz * 9 + k), S.q[qs][ejy + k / 3][ejx + k % 3], bs);
              }
              uc = S.q[qslot(Zc)][ejy + 1][ejx + 1];
            }
            const long long ci = Zc * NNc + (long long)cy * Nc + cx;
            A.b_coarse[ci] = bs;
            A.u_coarse[ci] = uc;
          }
        }
      }
      if (bpx && OZD == 0 && owncol) {
        // P I du on this column from the c-points of c-plane zd / 3
        const int jx = lane / 3 - 1, jy = warp / 3 - 1;
        const C a = S.dc[jy][jx];
        const C b2 = ox ? S.dc[jy][jx + 1] : cz<float>();
        const C c2 = oy ? S.dc[jy + 1][jx] : cz<float>();
        const C d2 = (ox && oy) ? S.dc[jy + 1][jx + 1] : cz<float>();
        const C pid = cplx<float>{wy0 * (wx0 * a.x + wx1 * b2.x) + wy1 * (wx0 * c2.x + wx1 * d2.x),
                                  wy0 * (wx0 * a.y + wx1 * b2.y) + wy1 * (wx0 * c2.y + wx1 * d2.y)};
        if (zd - 2 >= 3 * Z0) {
          const C v1 = S.pv[0][warp][lane], v2 = S.pv[1][warp][lane];
          A.out[(zd - 2) * NN + col] = v1 - (rmul(2.f / 3.f, pidp) + rmul(1.f / 3.f, pid));
          A.out[(zd - 1) * NN + col] = v2 - (rmul(1.f / 3.f, pidp) + rmul(2.f / 3.f, pid));
        }
        if (zd < 3 * Z1 || zd == n) A.out[zd * NN + col] = S.pv[2][warp][lane] - pid;
        pidp = pid;
      }
    };

    // one fine step: u plane z + 1 in, residual plane z, outputs
    auto step = [&](auto ozc, int z) {
      constexpr int OZ = decltype(ozc)::value;
      constexpr int OZP = (OZ + 1) % 3;
      const int zp = z + 1;
      const int buf = z & 1;
      // phase 1: u on plane z + 1
      if (OZP == 0) cxy0 = cxy1;
      C up = pu[OZ];
      if (use_c && colin && zp > 0 && zp < n) {
        up = rfma(W0<OZP>(), cxy0, up);
        if (OZP != 0) up = rfma(W1<OZP>(), cxy1, up);
      }
      if (OZP == 0 && cpx && cpy) S.q[qslot(zp / 3)][warp / 3][lane / 3] = up;
      if (OZP == 2 && use_c && threadIdx.x < 144) S.cc[threadIdx.x / 12][threadIdx.x % 12] = ccpre;
      if (OZP == 0 && use_c) ccpre = ld_cc(zp / 3 + 2);
      pu[OZ] = ldU(z + 4);
      // z-pass (class of plane z is uniform over the block)
      const int tz = (z >= 0 && z <= n) ? (int)__ldg(A.typ + z) : 0;
      C za, zb;
      if (tz == 0) {
        za = tap3r(m0, m1, m2, um, u0, up);
        zb = tap3r(p0, p1, p2, um, u0, up);
      } else {
        za = tap3c_acc(&S.row[tz][0], um, u0, up, cz<float>());
        zb = tap3c_acc(&S.row[tz][6], um, u0, up, cz<float>());
      }
      S.za[buf][warp][lane] = za;
      S.zb[buf][warp][lane] = zb;
      __syncthreads();
      // phase 2: deferred work of plane z - 1; coarse correction plane for the next steps
      if (z > zs) deferred(IC<(OZ + 2) % 3>{}, z - 1);
      if (OZP == 0 && use_c) cxy1 = bil_cc();
      // phase 3: residual on plane z
      const bool zin = z > 0 && z < n;
      const bool zown = (z >= 3 * Z0 && z < 3 * Z1) || z == n;
      C r = cz<float>();
      if (rrow) {
        const C am = S.za[buf][warp - 1][lane], ap = S.za[buf][warp + 1][lane];
        const C bm = S.zb[buf][warp - 1][lane], bp = S.zb[buf][warp + 1][lane];
        C cy, ey;
        if (yreal) {
          cy = tap3r_acc(k0, k1, k2, am, za, ap, tap3r(m0, m1, m2, bm, zb, bp));
          ey = tap3r(m0, m1, m2, am, za, ap);
        } else {
          const C* rw = &S.row[ty][0];
          cy = tap3c_acc(rw + 3, am, za, ap, tap3c_acc(rw, bm, zb, bp, cz<float>()));
          ey = tap3c_acc(rw, am, za, ap, cz<float>());
        }
        const C cl = shfl_c(cy, 1, true), cr = shfl_c(cy, 1, false);
        const C el = shfl_c(ey, 1, true), er = shfl_c(ey, 1, false);
        C hu;
        if (xreal) {
          hu = tap3r_acc(k0, k1, k2, el, ey, er, tap3r(m0, m1, m2, cl, cy, cr));
        } else {
          const C* rw = &S.row[tx][0];
          hu = tap3c_acc(rw + 3, el, ey, er, tap3c_acc(rw, cl, cy, cr, cz<float>()));
        }
        if (colin && zin && lane >= 1 && lane <= 30) r = pb[OZ] - hu;
        if (owncol && zown) nrm = fmaf(r.x, r.x, fmaf(r.y, r.y, nrm));
        // Jacobi update, c-point mask (hb), outputs or BPX hold
        C du = S.omd[tx + 4 * ty + 16 * tz] * r;
        if (A.hb && OZ == 0 && cpx && cpy) du = cz<float>();
        const C v = A.fine ? u0 + du : du;
        if (!bpx) {
          if (owncol && zown) A.out[z * NN + col] = v;
        } else if (owncol) {
          S.pv[OZ == 1 ? 0 : (OZ == 2 ? 1 : 2)][warp][lane] = v;
        }
        if (bpx && OZ == 0 && cpx && cpy && lane >= 3 && warp >= 3) S.dc[warp / 3 - 1][lane / 3 - 1] = du;
        // restriction along x to the c-columns
        if (A.has_coarse) {
          const C r1l = shfl_c(r, 1, true), r1r = shfl_c(r, 1, false);
          const C r2l = shfl_c(r, 2, true), r2r = shfl_c(r, 2, false);
          const C rr = cplx<float>{fmaf(r2l.x + r2r.x, 1.f / 3.f, fmaf(r1l.x + r1r.x, 2.f / 3.f, r.x)),
                                   fmaf(r2l.y + r2r.y, 1.f / 3.f, fmaf(r1l.y + r1r.y, 2.f / 3.f, r.y))};
          if (cpx && lane >= 3 && lane <= 30) S.rx[buf][warp][lane / 3 - 1] = rr;
        }
      }
      pb[OZ] = ldB(z + 3);
      um = u0;
      u0 = up;
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
        const long long ci = nc * NNc + (long long)cy * Nc + cx;
        A.b_coarse[ci] = cz<float>();
        A.u_coarse[ci] = cz<float>();
      }
    }
  }
  if (A.fine && A.norm2 != nullptr)
    block_norm_finish_tile<kS3sThreads>((double)nrm, s_red, A.partial, A.ticket, A.norm2, blockIdx.x,
                                         gridDim.x);
}

}  // namespace mg
