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
// (Section 4: K_c = sum_j (x)_a (K if a == j else M), M_c = (x)_a M):
//     H u = M_x [ M_y (K_z - phi M_z) u + K_y M_z u ] + K_x (M_y M_z u).
// The rows depend only on the vertex's scaling class along that axis (left
// and right cell plain or rotated), so seven 3-tap passes replace the
// 27-point row, and rows in the unscaled interior take real coefficients.
//
// Layout.  A block of 512 threads owns an x-y tile of 9 x 9 coarse cells
// (27 x 27 fine vertices) and a range of coarse planes; lane = x and the two
// rows 2w, 2w+1 of warp w = y of a 32 x 32 box of fine columns
// [x0-3, x0+28] x [y0-3, y0+28].  Each thread marches its two columns along z
// holding u(z-1), u(z), u(z+1) in registers: the z-pass runs in registers,
// the y-pass takes the pair's outer neighbour rows from shared memory, the
// x-pass takes its neighbours by warp shuffles.
// The r box is [x0-2, x0+27]^2 (lanes/warps 1..30), enough for the
// restriction of the owned coarse vertices and for the c-point Jacobi update
// of the next tile's first c-point (BPX).  One barrier per fine plane.
//
// Plane staging by TMA.  The u and b planes of the box come into shared
// memory as tensor-map box loads (mg_tma.cuh): rings of four planes, each
// slot with an mbarrier that the load completes.  Thread 0 issues u(z + 3)
// and b(z + 2) at fine step z (the slots they overwrite were last read before
// the previous step's barrier); every thread waits (bounded) for u(z + 1)
// and b(z).  The hardware zero-fills what lies outside the level array, so
// the loads carry no per-thread address or bounds work.  A box starts on an
// even column (16-byte rule for the x coordinate), so it is 34 columns wide
// and the tile's columns sit at offset 0 or 1.
//
// Work split.  The (tile, coarse plane) units of the level are split into
// gridDim.x contiguous ranges of equal cost (tabulated on the host: units
// with scaled rows cost more; one block per SM); a range may continue into
// the next tile.
#pragma once
#include "mg_kernels.cuh"
#include "mg_sweep3d.cuh"
#include "mg_tma.cuh"

namespace mg {


struct Sweep3sArgs {
  int n, fine, first, has_coarse, hb, hier;
  int tiles_x;          // x-y tiles per axis (9 coarse cells each)
  long long nunits;     // tiles_x^2 * (n / 3)
  const unsigned* upref;    // prefix sums of the unit costs, nunits + 1 entries
  const unsigned* usplit;   // block b takes units [usplit[b], usplit[b+1]) (null: by upref)
  unsigned spin_limit;      // polls before a plane wait gives up
  unsigned* err;            // sticky error flag (bit 2: a plane wait gave up)
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

constexpr int kS3Ring = 4;   // planes of u and of b in flight
constexpr int kS3BoxW = 34;  // box columns (start rounded down to an even column)
constexpr unsigned kS3PlaneBytes = 32u * kS3BoxW * 8u;  // 8704 = 68 x 128

struct Sweep3sShared {
  cplx<float> ub[kS3Ring][32][kS3BoxW];  // TMA destinations (128-byte aligned)
  cplx<float> bb[kS3Ring][32][kS3BoxW];
  unsigned long long bar_u[kS3Ring], bar_b[kS3Ring];
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
// Stores taken by some lanes only, as predicated instructions: the other
// lanes skip them without a divergent branch and its reconvergence (the
// address is formed by every lane and used by none whose predicate is false).
__device__ __forceinline__ void st_global_if(cplx<float>* p, cplx<float> v, bool pred) {
  asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %3, 0;\n @q st.global.v2.f32 [%0], {%1, %2};\n}\n" ::"l"(p),
               "f"(v.x), "f"(v.y), "r"((unsigned)pred));
}
__device__ __forceinline__ void st_shared_if(cplx<float>* p, cplx<float> v, bool pred) {
  asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %3, 0;\n @q st.shared.v2.f32 [%0], {%1, %2};\n}\n" ::"r"(
                   smem_u32(p)),
               "f"(v.x), "f"(v.y), "r"((unsigned)pred)
               : "memory");
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

// Two vertically adjacent box rows per thread (512 threads, warp w holds rows
// 2w and 2w+1): the per-plane control, address and barrier work is shared by
// two columns, the y-pass of a row pair needs only the two outer neighbour
// rows from shared memory, and 128 registers hold both columns' state (one
// row per thread at 1024 threads was 15% slower and spilled at 64 registers).
// FINE, HB, BPX: the level's role and the variant, fixed at compile time so
// that each instantiation carries only its own branches (the kernel is
// issue-bound); A.fine, A.hb and A.hier must agree with them.
template <int RPT, bool FINE, bool HB, bool BPX>
__global__ void __launch_bounds__(32 * (32 / RPT), 1)
    sweep3s_kernel(const Sweep3sArgs A, const __grid_constant__ CUtensorMap tmU,
                   const __grid_constant__ CUtensorMap tmB) {
  constexpr int NTHR = 32 * (32 / RPT), NW = 32 / RPT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double s_red[NTHR / 32];
  // TMA destinations need 128-byte alignment: the launch adds 128 bytes
  Sweep3sShared& S = *reinterpret_cast<Sweep3sShared*>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
  using C = cplx<float>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n = A.n, N = n + 1, nc = n / 3;
  const int NN = N * N, Nc = nc + 1, NNc = Nc * Nc;  // level sizes stay below 2^31 vertices
  for (int i = threadIdx.x; i < 36; i += NTHR) S.row[i / 9][i % 9] = A.row[i / 9][i % 9];
  for (int i = threadIdx.x; i < 64; i += NTHR) S.omd[i] = A.omd[i];
  if (threadIdx.x == 0) {
    for (int k = 0; k < kS3Ring; ++k) {
      mbar_init(&S.bar_u[k], 1);
      mbar_init(&S.bar_b[k], 1);
    }
    fence_mbar_init();
  }
  __syncthreads();
  unsigned ph_u = 0, ph_b = 0;  // parity of the next wait, one bit per slot
  constexpr bool use_c = FINE;  // a finest level always has a pending correction level
  constexpr bool bpx = BPX;
  // restriction and coarse outputs: 4 warps x 25 lanes take the 10 x 10
  // coarse columns C0 .. C0+9 (column 9 only matters on the last tile)
  // (warps 0, 4, 3, 7: the sub-partitions that also hold the box rows 0 and
  // 31, which need no residual, so the issue work per sub-partition evens out)
  const int wsel = warp == 0 ? 0 : (warp == 4 ? 1 : (warp == 3 ? 2 : (warp == 7 ? 3 : -1)));
  const int ek = (wsel >= 0 && lane < 25) ? wsel * 25 + lane : -1;
  const bool emit = ek >= 0 && A.has_coarse;
  const int ejx = emit ? ek % 10 : 0, ejy = emit ? ek / 10 : 0;
  const float m0 = A.row[0][0].x, m1 = A.row[0][1].x, m2 = A.row[0][2].x;
  const float k0 = A.row[0][3].x, k1 = A.row[0][4].x, k2 = A.row[0][5].x;
  const float p0 = A.row[0][6].x, p1 = A.row[0][7].x, p2 = A.row[0][8].x;
  const int ox = lane % 3;
  const float wx1 = ox == 0 ? 0.f : (ox == 1 ? 1.f / 3.f : 2.f / 3.f), wx0 = 1.f - wx1;
  const bool cpx = ox == 0;
  int by[RPT], oy[RPT];
  float wy0[RPT], wy1[RPT];
  bool cpy[RPT], rrow[RPT];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    by[r] = RPT * warp + r;  // box row
    oy[r] = by[r] % 3;
    wy1[r] = oy[r] == 0 ? 0.f : (oy[r] == 1 ? 1.f / 3.f : 2.f / 3.f);
    wy0[r] = 1.f - wy1[r];
    cpy[r] = oy[r] == 0;
    rrow[r] = by[r] >= 1 && by[r] <= 30;
  }
  float nrm = 0.f;

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
    const bool xreal = __all_sync(0xffffffffu, tx == 0);
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
    auto ld_cc = [&](int Zc) -> C {
      const int t = threadIdx.x;
      const int cx = C0x - 1 + t % 12, cy = C0y - 1 + t / 12;
      return (use_c && t < 144 && Zc >= 0 && Zc <= nc && cx >= 0 && cx <= nc && cy >= 0 && cy <= nc)
                 ? ld_nc(A.c + (Zc * NNc + cy * Nc + cx))
                 : cz<float>();
    };
    // bilinear interpolation of the coarse plane in S.cc to column (lane, box row r)
    auto bil_cc = [&](int r) -> C {
      const int jx = lane / 3, jy = by[r] / 3;
      const C a = S.cc[jy][jx], b2 = S.cc[jy][jx + 1], c2 = S.cc[jy + 1][jx], d2 = S.cc[jy + 1][jx + 1];
      return cplx<float>{wy0[r] * (wx0 * a.x + wx1 * b2.x) + wy1[r] * (wx0 * c2.x + wx1 * d2.x),
                         wy0[r] * (wx0 * a.y + wx1 * b2.y) + wy1[r] * (wx0 * c2.y + wx1 * d2.y)};
    };

    // plane rings: box columns from the even column xs, the tile's box
    // column 0 (fine x0 - 3) at offset xsh
    const int xs = (x0 - 3) - ((x0 - 3) & 1), xsh = (x0 - 3) - xs;
    auto issueU = [&](int z) {  // thread 0
      const int k = (z + 8) & (kS3Ring - 1);
      mbar_arrive_expect_tx(&S.bar_u[k], kS3PlaneBytes);
      tma_load_plane(&S.ub[k][0][0], &tmU, &S.bar_u[k], 2 * xs, y0 - 3, z);
    };
    auto issueB = [&](int z) {
      const int k = (z + 8) & (kS3Ring - 1);
      mbar_arrive_expect_tx(&S.bar_b[k], kS3PlaneBytes);
      tma_load_plane(&S.bb[k][0][0], &tmB, &S.bar_b[k], 2 * xs, y0 - 3, z);
    };
    auto waitU = [&](int z) -> const C* {  // every thread; returns the plane's row 0 at the tile's column 0
      const int k = (z + 8) & (kS3Ring - 1);
      mbar_wait_bounded(&S.bar_u[k], (ph_u >> k) & 1u, A.spin_limit, A.err);
      ph_u ^= 1u << k;
      return &S.ub[k][0][xsh];
    };
    auto waitB = [&](int z) -> const C* {
      const int k = (z + 8) & (kS3Ring - 1);
      mbar_wait_bounded(&S.bar_b[k], (ph_b >> k) & 1u, A.spin_limit, A.err);
      ph_b ^= 1u << k;
      return &S.bb[k][0][xsh];
    };
    auto plane_val = [&](const C* pl, int r) -> C {
      return pl[by[r] * kS3BoxW + lane];
    };

    __syncthreads();  // the previous range's shared memory is free
    if (threadIdx.x == 0) {
      // the planes of the first steps: u(zs - 1 .. zs + 2), b(zs, zs + 1)
      fence_proxy_async_smem();
      issueU(3 * Z0 - 3);
      issueU(3 * Z0 - 2);
      issueU(3 * Z0 - 1);
      issueU(3 * Z0);
      issueB(3 * Z0 - 2);
      issueB(3 * Z0 - 1);
    }
    C cxy0[RPT], cxy1[RPT], ccpre = cz<float>();
#pragma unroll
    for (int r = 0; r < RPT; ++r) cxy0[r] = cxy1[r] = cz<float>();
    // one coarse plane of the pending correction through S.cc: threads < 144
    // load it (blocks have at least 256 threads)
    if (use_c) {
      if (threadIdx.x < 144) S.cc[threadIdx.x / 12][threadIdx.x % 12] = ld_cc(Z0 - 1);
      __syncthreads();
#pragma unroll
      for (int r = 0; r < RPT; ++r) cxy0[r] = bil_cc(r);
      __syncthreads();
      if (threadIdx.x < 144) S.cc[threadIdx.x / 12][threadIdx.x % 12] = ld_cc(Z0);
      __syncthreads();
#pragma unroll
      for (int r = 0; r < RPT; ++r) cxy1[r] = bil_cc(r);
      ccpre = ld_cc(Z0 + 1);
      __syncthreads();
    }
    C um[RPT], u0[RPT], pidp[RPT];
    const C* plm = waitU(3 * Z0 - 3);
    const C* pl0 = waitU(3 * Z0 - 2);
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      // u on planes 3 Z0 - 3 (c-plane Z0 - 1) and 3 Z0 - 2
      um[r] = plane_val(plm, r);
      u0[r] = plane_val(pl0, r);
      // P c is exactly zero on and beyond the Dirichlet ring (the coarse
      // correction's ring is zero and the coarse plane loads are zero outside
      // the grid), so it is added without tests
      if (use_c) {
        um[r] = um[r] + cxy0[r];
        u0[r] = rfma(W0<1>(), cxy0[r], u0[r]);
        u0[r] = rfma(W1<1>(), cxy1[r], u0[r]);
      }
      if (cpx && cpy[r]) S.q[qslot(Z0 - 1)][by[r] / 3][lane / 3] = um[r];
      pidp[r] = cz<float>();
    }
    C accA = cz<float>(), accB = cz<float>();

    // deferred work of residual plane zd, after the barrier of the next step
    auto deferred = [&](auto ozc, int zd) {
      constexpr int OZD = decltype(ozc)::value;
      const int bufd = zd & 1;
      if (emit && ejx < 9 && ejy < 9) {
        const int ry_ = 3 + 3 * ejy;
        const C ry = restrict5f(S.rx[bufd][ry_ - 2][ejx], S.rx[bufd][ry_ - 1][ejx], S.rx[bufd][ry_][ejx],
                                S.rx[bufd][ry_ + 1][ejx], S.rx[bufd][ry_ + 2][ejx]);
        if (OZD == 0) {
          accA = accB + ry;
          accB = cz<float>();
        } else {
          accA = rfma(W0<OZD>(), ry, accA);
          accB = rfma(W1<OZD>(), ry, accB);
        }
      }
      if (OZD == 2 && emit) {
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
          const int ci = Zc * NNc + cy * Nc + cx;
          A.b_coarse[ci] = bs;
          A.u_coarse[ci] = uc;
        }
      }
      if (bpx && OZD == 0) {
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          if (!owncol[r]) continue;
          // P I du on this column from the c-points of c-plane zd / 3
          const int jx = lane / 3 - 1, jy = by[r] / 3 - 1;
          const C a = S.dc[jy][jx];
          const C b2 = ox ? S.dc[jy][jx + 1] : cz<float>();
          const C c2 = oy[r] ? S.dc[jy + 1][jx] : cz<float>();
          const C d2 = (ox && oy[r]) ? S.dc[jy + 1][jx + 1] : cz<float>();
          const C pid = cplx<float>{wy0[r] * (wx0 * a.x + wx1 * b2.x) + wy1[r] * (wx0 * c2.x + wx1 * d2.x),
                                    wy0[r] * (wx0 * a.y + wx1 * b2.y) + wy1[r] * (wx0 * c2.y + wx1 * d2.y)};
          if (zd - 2 >= 3 * Z0) {
            const C v1 = S.pv[0][by[r]][lane], v2 = S.pv[1][by[r]][lane];
            A.out[(zd - 2) * NN + col[r]] = v1 - (rmul(2.f / 3.f, pidp[r]) + rmul(1.f / 3.f, pid));
            A.out[(zd - 1) * NN + col[r]] = v2 - (rmul(1.f / 3.f, pidp[r]) + rmul(2.f / 3.f, pid));
          }
          if (zd < 3 * Z1 || zd == n) A.out[zd * NN + col[r]] = S.pv[2][by[r]][lane] - pid;
          pidp[r] = pid;
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
      // staging: u(z + 3) and b(z + 2) into the slots of u(z - 1) and b(z - 2),
      // both last read before the previous step's barrier
      if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        if (z + 3 <= 3 * Z1 + 1) issueU(z + 3);
        if (z + 2 <= 3 * Z1) issueB(z + 2);
      }
      // phase 1: u on plane z + 1, z-pass of both rows
      C up[RPT], za[RPT], zb[RPT];
      const C* plp = waitU(z + 1);
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        if (OZP == 0) cxy0[r] = cxy1[r];
        up[r] = plane_val(plp, r);
        if (use_c) {  // zero on and beyond the ring (see the first planes)
          up[r] = rfma(W0<OZP>(), cxy0[r], up[r]);
          if (OZP != 0) up[r] = rfma(W1<OZP>(), cxy1[r], up[r]);
        }
        if (OZP == 0) st_shared_if(&S.q[qslot(zp / 3)][by[r] / 3][lane / 3], up[r], cpx && cpy[r]);
        if (tz == 0) {
          za[r] = tap3r(m0, m1, m2, um[r], u0[r], up[r]);
          zb[r] = tap3r(p0, p1, p2, um[r], u0[r], up[r]);
        } else {
          za[r] = tap3c_acc(&S.row[tz][0], um[r], u0[r], up[r], cz<float>());
          zb[r] = tap3c_acc(&S.row[tz][6], um[r], u0[r], up[r], cz<float>());
        }
        S.za[buf][by[r]][lane] = za[r];
        S.zb[buf][by[r]][lane] = zb[r];
      }
      if (OZP == 2 && use_c && threadIdx.x < 144) S.cc[threadIdx.x / 12][threadIdx.x % 12] = ccpre;
      if (OZP == 0 && use_c) ccpre = ld_cc(zp / 3 + 2);
      __syncthreads();
      // phase 2: deferred work of plane z - 1; coarse correction plane for the next steps
      if (z > zs) deferred(IC<(OZ + 2) % 3>{}, z - 1);
      if (OZP == 0 && use_c) {
#pragma unroll
        for (int r = 0; r < RPT; ++r) cxy1[r] = bil_cc(r);
      }
      // phase 3: residuals on plane z; the pair's outer neighbour rows from shared memory
      const bool zin = z > 0 && z < n;
      const bool zown = (z >= 3 * Z0 && z < 3 * Z1) || z == n;
      const C* plb = waitB(z);
      const C aU = warp > 0 ? S.za[buf][by[0] - 1][lane] : cz<float>();
      const C bU = warp > 0 ? S.zb[buf][by[0] - 1][lane] : cz<float>();
      const C aD = warp < NW - 1 ? S.za[buf][by[RPT - 1] + 1][lane] : cz<float>();
      const C bD = warp < NW - 1 ? S.zb[buf][by[RPT - 1] + 1][lane] : cz<float>();
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        if (!rrow[r]) continue;  // warp-uniform
        // neighbour rows: the thread's own rows, the pair's outer ones from shared memory
        const C am = r == 0 ? aU : za[r > 0 ? r - 1 : 0], ap = r == RPT - 1 ? aD : za[r < RPT - 1 ? r + 1 : r];
        const C bm = r == 0 ? bU : zb[r > 0 ? r - 1 : 0], bp = r == RPT - 1 ? bD : zb[r < RPT - 1 ? r + 1 : r];
        C cy, ey;
        if (yreal[r]) {
          cy = tap3r_acc(k0, k1, k2, am, za[r], ap, tap3r(m0, m1, m2, bm, zb[r], bp));
          ey = tap3r(m0, m1, m2, am, za[r], ap);
        } else {
          const C* rw = &S.row[ty[r]][0];
          cy = tap3c_acc(rw + 3, am, za[r], ap, tap3c_acc(rw, bm, zb[r], bp, cz<float>()));
          ey = tap3c_acc(rw, am, za[r], ap, cz<float>());
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
        C res = cz<float>();
        {
          const C rr = plb[by[r] * kS3BoxW + lane] - hu;
          res = (colin[r] && zin && lane >= 1 && lane <= 30) ? rr : cz<float>();
          const C rn = (owncol[r] && zown) ? res : cz<float>();
          nrm = fmaf(rn.x, rn.x, fmaf(rn.y, rn.y, nrm));
        }
        // Jacobi update, c-point mask (hb), outputs or BPX hold
        C du = S.omd[tx + 4 * ty[r] + 16 * tz] * res;
        if (HB && OZ == 0 && cpx && cpy[r]) du = cz<float>();
        const C v = FINE ? u0[r] + du : du;
        if (!bpx) {
          st_global_if(A.out + ((long long)z * NN + col[r]), v, owncol[r] && zown);
        } else if (owncol[r]) {
          S.pv[OZ == 1 ? 0 : (OZ == 2 ? 1 : 2)][by[r]][lane] = v;
        }
        if (bpx && OZ == 0 && cpx && cpy[r] && lane >= 3 && by[r] >= 3)
          S.dc[by[r] / 3 - 1][lane / 3 - 1] = du;
        // restriction along x to the c-columns
        if (A.has_coarse) {
          const C r1l = shfl_c(res, 1, true), r1r = shfl_c(res, 1, false);
          const C r2l = shfl_c(res, 2, true), r2r = shfl_c(res, 2, false);
          const C rxv = restrict5f(r2l, r1l, res, r1r, r2r);
          st_shared_if(&S.rx[buf][by[r]][lane >= 3 ? lane / 3 - 1 : 0], rxv, cpx && lane >= 3 && lane <= 30);
        }
      }
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        um[r] = u0[r];
        u0[r] = up[r];
      }
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
        A.b_coarse[ci] = cz<float>();
        A.u_coarse[ci] = cz<float>();
      }
    }
  }
  if (FINE && A.norm2 != nullptr)
    block_norm_finish_tile<NTHR>((double)nrm, s_red, A.partial, A.ticket, A.norm2, blockIdx.x,
                                         gridDim.x);
}

}  // namespace mg
