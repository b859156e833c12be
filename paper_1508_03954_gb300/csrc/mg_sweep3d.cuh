// mg_sweep3d.cuh -- fine-to-coarse sweep for 3D levels with a constant shift
// (sm_103a), marching along z.
//
// Same step as the 2D sweep (Appendix A Algorithm 4 on one level with the
// single-touch pending correction of Algorithm 2 and the coarse right-hand
// side b_{l-1} = R r_l + G_{l-1} u_{l-1}, G = R H P).  A block owns an x-y
// tile of TC x TC coarse cells (F = 3 TC fine vertices per edge) and a range
// of coarse z-planes [Z0, Z1).  It walks up the range one coarse plane at a
// time; fine planes of u, of the residual r and of the c-point Jacobi update
// live in ring buffers in shared memory, so every plane of U and b is read
// from global memory once per block and every residual plane is computed
// once (the x-y halo is recomputed by the neighbouring tiles; the z halo
// only at the ends of the range).
//
// Step Z (coarse plane) with the rings holding u on fine planes [3Z, 3Z+4]
// (plus the c-point values of the c-planes Z-1 .. Z+1), r on [3Z, 3Z+3] and
// the x-y restriction of r on [3Z-2, 3Z+3]:
//   a. load U (+ P c) on fine planes 3Z+2 .. 3Z+4          (u ring)
//   b. r = b - H u on fine planes 3Z+1 .. 3Z+3              (r ring); |r|^2
//      on owned points; x-y restriction of each new r plane (rxy ring)
//   c. du on the c-points of fine plane 3Z+3 (c-plane Z+1)  (dc ring)
//   d. coarse outputs of plane Z: b_{l-1} = R r + G u_{l-1}, u_{l-1} = I u
//   e. fine outputs of planes 3Z .. 3Z+2: U' = u + T du, or T du
#pragma once
#include "mg_kernels.cuh"

namespace mg {

constexpr int kMaxG3 = 6;  // 1D Galerkin row classes per axis (3D table kMaxG3^3 x 27)

template <typename R>
struct Sweep3Args {
  int n, fine, first, has_coarse, hb, hier;
  int tiles_x, ntiles_xy, zchunk, nzchunks, ntiles;  // tile = xy + ntiles_xy * zc
  unsigned long long realrow;  // bit t: stencil row of vertex type t (64 types) is real
  unsigned long long realjac;  // bit t: omega/D of type t is real
  const cplx<R>* u;
  const cplx<R>* c;        // pending correction on level l-1 (fine, may be null)
  const cplx<R>* b;
  cplx<R>* out;
  cplx<R>* b_coarse;
  cplx<R>* u_coarse;
  const uint8_t* typ;      // vertex type per fine index (n+1)
  const uint8_t* gtyp;     // Galerkin row class per coarse index (n/3+1)
  const cplx<R>* coef;     // [64][27]
  const cplx<R>* gcoef;    // [kMaxG3^3][27], index gx + G gy + G^2 gz
  cplx<R> omd[64];
  double* partial;
  unsigned* ticket;
  double* norm2;
};

template <typename R, int TC>
struct Tile3 {
  static constexpr int F = 3 * TC;
  static constexpr int SU = F + 5;   // u plane box [x0-3, x0+F+1]
  static constexpr int SR = F + 3;   // r plane box [x0-2, x0+F]
  static constexpr int SC = TC + 3;  // coarse c box [C0-1, C0+TC+1]
  static constexpr int SD = TC + 1;  // c-point du box [C0, C0+TC]
  static constexpr int SQ = TC + 2;  // c-point u box [C0-1, C0+TC]
  static constexpr int NU = 5, NRR = 4, NCR = 4, NDR = 2, NXY = 6, NQ = 3, NB = 3;  // ring depths
  static constexpr size_t cplx_count =
      (size_t)NU * SU * SU + (size_t)NRR * SR * SR + (size_t)NB * SR * SR + (size_t)NCR * SC * SC +
      (size_t)3 * SC * SU +
      (size_t)NDR * SD * SD + (size_t)NXY * TC * TC + (size_t)(F + 2) * TC + (size_t)SD * F +
      (size_t)NDR * F * F + (size_t)NQ * SQ * SQ + 64 * 27 + 64;
  static constexpr size_t smem_bytes = cplx_count * sizeof(cplx<R>) + 3 * SU + 16;
};

template <typename R> __device__ __forceinline__ R w0r(int o) {
  return o == 0 ? R(1) : (o == 1 ? R(2) / R(3) : R(1) / R(3));
}
template <typename R> __device__ __forceinline__ R w1r(int o) {
  return o == 0 ? R(0) : (o == 1 ? R(1) / R(3) : R(2) / R(3));
}
template <typename R>
__device__ __forceinline__ cplx<R> lerp2r(R s0, cplx<R> a, R s1, cplx<R> b) {
  return cplx<R>{fma(s1, b.x, s0 * a.x), fma(s1, b.y, s0 * a.y)};
}
template <typename R>
__device__ __forceinline__ cplx<R> restrict5r(cplx<R> m2, cplx<R> m1, cplx<R> z, cplx<R> p1, cplx<R> p2) {
  return cplx<R>{fma(m2.x + p2.x, R(1) / R(3), fma(m1.x + p1.x, R(2) / R(3), z.x)),
                 fma(m2.y + p2.y, R(1) / R(3), fma(m1.y + p1.y, R(2) / R(3), z.y))};
}

// Asynchronous global->shared copies of one complex value (8 or 16 bytes).
template <typename R>
__device__ __forceinline__ void cp_async_cplx(cplx<R>* dst, const cplx<R>* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(cplx<R>) == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
  }
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <typename R, int TC, int NTHR>
__device__ void sweep3_tile(const Sweep3Args<R>& A, int tile, unsigned char* smem_raw, double* s_red) {
  using T = Tile3<R, TC>;
  using C = cplx<R>;
  constexpr int F = T::F, SU = T::SU, SR = T::SR, SC = T::SC, SD = T::SD;
  C* s_u = reinterpret_cast<C*>(smem_raw);            // [NU][SU*SU]
  C* s_r = s_u + T::NU * SU * SU;                     // [NRR][SR*SR]
  C* s_b = s_r + T::NRR * SR * SR;                    // [NB][SR*SR] right-hand side planes
  C* s_c = s_b + T::NB * SR * SR;                     // [NCR][SC*SC]
  C* s_cx = s_c + T::NCR * SC * SC;                   // [3][SC*SU] x-interpolated c planes
  C* s_dc = s_cx + 3 * SC * SU;                       // [NDR][SD*SD]
  C* s_rxy = s_dc + T::NDR * SD * SD;                 // [NXY][TC*TC] x-y restricted r planes
  C* s_Y = s_rxy + T::NXY * TC * TC;                  // [F+2][TC] x-pass of one r plane
  C* s_Z = s_Y + (F + 2) * TC;                        // [SD][F] x-pass of one dc plane
  C* s_pi = s_Z + SD * F;                             // [NDR][F*F] P I du per c-plane
  C* s_q = s_pi + T::NDR * F * F;                     // [NQ][SQ*SQ] u at the c-points of c-planes
  C* s_coef = s_q + T::NQ * T::SQ * T::SQ;            // [64][27]
  C* s_omd = s_coef + 64 * 27;                        // [64]
  uint8_t* s_tx = reinterpret_cast<uint8_t*>(s_omd + 64);  // [SU] x types, then y, z? (z per plane)
  uint8_t* s_ty = s_tx + SU;
  __syncthreads();

  const int n = A.n, N = n + 1, nc = n / 3;
  const long long NN = (long long)N * N, Ncc = (long long)(nc + 1) * (nc + 1);
  const int txy = tile % A.ntiles_xy, zc = tile / A.ntiles_xy;
  const int C0x = (txy % A.tiles_x) * TC, C0y = (txy / A.tiles_x) * TC;
  const int x0 = 3 * C0x, y0 = 3 * C0y;
  const int Z0 = zc * A.zchunk;
  const int Z1 = min(Z0 + A.zchunk, nc + 1);
  const bool use_c = A.fine && !A.first && A.c != nullptr;

  for (int i = threadIdx.x; i < 64 * 27; i += NTHR) s_coef[i] = A.coef[i];
  for (int i = threadIdx.x; i < 64; i += NTHR) s_omd[i] = A.omd[i];
  for (int i = threadIdx.x; i < 2 * SU; i += NTHR) {
    const int q = i % SU;
    const int g = (i < SU ? x0 : y0) - 3 + q;
    (i < SU ? s_tx : s_ty)[q] = (g >= 0 && g <= n) ? A.typ[g] : (uint8_t)0;
  }
  auto ztype = [&](int z) -> int { return (z >= 0 && z <= n) ? (int)A.typ[z] : 0; };
  auto uslot = [](int z) { return ((z % 5) + 5) % 5; };
  auto rslot = [](int z) { return ((z % 4) + 4) % 4; };
  auto xslot = [](int z) { return ((z % 6) + 6) % 6; };
  auto qslot = [](int Zc) { return ((Zc % 3) + 3) % 3; };
  constexpr int SQ = T::SQ;
  auto cslot = [](int Z) { return ((Z % 4) + 4) % 4; };
  auto dslot = [](int Z) { return ((Z % 2) + 2) % 2; };

  const bool zero_u = A.fine && A.first;
  // issue the copies of coarse plane Zc of the pending correction
  auto issue_c = [&](int Zc) {
    C* dst = s_c + cslot(Zc) * SC * SC;
    for (int i = threadIdx.x; i < SC * SC; i += NTHR) {
      const int qx = i % SC, qy = i / SC;
      const int cx = C0x - 1 + qx, cy = C0y - 1 + qy;
      const bool in = use_c && Zc >= 0 && Zc <= nc && cx >= 0 && cx <= nc && cy >= 0 && cy <= nc;
      if (in) cp_async_cplx(dst + i, A.c + Zc * Ncc + (long long)cy * (nc + 1) + cx);
      else dst[i] = cz<R>();
    }
  };
  // x-interpolated coarse plane Zc (s_cx slot Zc % 3), after its copy landed
  auto cx_pass = [&](int Zc) {
    const C* src = s_c + cslot(Zc) * SC * SC;
    C* dst = s_cx + (((Zc % 3) + 3) % 3) * SC * SU;
    for (int i = threadIdx.x; i < SC * SU; i += NTHR) {
      const int bx = i % SU, cy = i / SU;
      const int ox = bx % 3, cxi = bx / 3;
      dst[i] = lerp2r(w0r<R>(ox), src[cy * SC + cxi], w1r<R>(ox), src[cy * SC + cxi + 1]);
    }
  };
  // issue the copies of U plane z (zero outside the interior)
  auto issue_u = [&](int z) {
    C* dst = s_u + uslot(z) * SU * SU;
    const bool zin = z > 0 && z < n;
    for (int i = threadIdx.x; i < SU * SU; i += NTHR) {
      const int bx = i % SU, by = i / SU;
      const int gx = x0 - 3 + bx, gy = y0 - 3 + by;
      if (!zero_u && zin && gx > 0 && gx < n && gy > 0 && gy < n)
        cp_async_cplx(dst + i, A.u + z * NN + (long long)gy * N + gx);
      else
        dst[i] = cz<R>();
    }
  };
  // issue the copies of the right-hand side on the r box of plane z
  auto issue_b = [&](int z) {
    C* dst = s_b + (((z % 3) + 3) % 3) * SR * SR;
    const bool zin = z > 0 && z < n;
    for (int i = threadIdx.x; i < SR * SR; i += NTHR) {
      const int qx = i % SR, qy = i / SR;
      const int gx = x0 - 2 + qx, gy = y0 - 2 + qy;
      if (zin && gx > 0 && gx < n && gy > 0 && gy < n)
        cp_async_cplx(dst + i, A.b + z * NN + (long long)gy * N + gx);
      else
        dst[i] = cz<R>();
    }
  };
  // u = U + P c on plane z, in place (after the c planes are x-interpolated)
  auto add_pc = [&](int z) {
    if (!use_c) return;
    C* dst = s_u + uslot(z) * SU * SU;
    if (!(z > 0 && z < n)) return;
    const int Zc = z / 3, oz = z % 3;
    const C* X0 = s_cx + (((Zc % 3) + 3) % 3) * SC * SU;
    const C* X1 = s_cx + ((((Zc + 1) % 3) + 3) % 3) * SC * SU;
    for (int i = threadIdx.x; i < SU * SU; i += NTHR) {
      const int bx = i % SU, by = i / SU;
      const int gx = x0 - 3 + bx, gy = y0 - 3 + by;
      if (!(gx > 0 && gx < n && gy > 0 && gy < n)) continue;
      const int oy = by % 3, cy = by / 3;
      C v = dst[i];
      const C a = lerp2r(w0r<R>(oy), X0[cy * SU + bx], w1r<R>(oy), X0[(cy + 1) * SU + bx]);
      v = v + rmul(w0r<R>(oz), a);
      if (oz != 0) {
        const C b2 = lerp2r(w0r<R>(oy), X1[cy * SU + bx], w1r<R>(oy), X1[(cy + 1) * SU + bx]);
        v = v + rmul(w1r<R>(oz), b2);
      }
      dst[i] = v;
    }
  };
  // c-point values of u plane z = 3 Zc into the q ring (after a sync)
  auto save_q = [&](int z) {
    const C* src = s_u + uslot(z) * SU * SU;
    C* dst = s_q + qslot(z >= 0 ? z / 3 : -1) * SQ * SQ;
    for (int i = threadIdx.x; i < SQ * SQ; i += NTHR) {
      const int jx = i % SQ, jy = i / SQ;
      dst[i] = src[(3 * jy) * SU + 3 * jx];  // box coordinate 3j is coarse C0-1+j
    }
  };
  // residual plane z into the r ring; returns this thread's |r|^2 on owned points
  auto comp_r = [&](int z) -> double {
    C* dst = s_r + rslot(z) * SR * SR;
    const bool zin = z > 0 && z < n;
    const bool zown = z >= 3 * Z0 && z < 3 * Z1;
    const int tz = ztype(z);
    const C* um = s_u + uslot(z - 1) * SU * SU;
    const C* u0 = s_u + uslot(z) * SU * SU;
    const C* up = s_u + uslot(z + 1) * SU * SU;
    double nrm = 0.0;
    for (int i = threadIdx.x; i < SR * SR; i += NTHR) {
      const int qx = i % SR, qy = i / SR;
      const int gx = x0 - 2 + qx, gy = y0 - 2 + qy;
      C r = cz<R>();
      if (zin && gx > 0 && gx < n && gy > 0 && gy < n) {
        const int bx = qx + 1, by = qy + 1;
        const int t = s_tx[bx] + 4 * s_ty[by] + 16 * tz;
        const C* cf = s_coef + t * 27;
        r = s_b[(((z % 3) + 3) % 3) * SR * SR + i];
        const int o = by * SU + bx;
        const bool real = (A.realrow >> t) & 1ull;
#pragma unroll
        for (int kz = 0; kz < 3; ++kz) {
          const C* pl = kz == 0 ? um : (kz == 1 ? u0 : up);
#pragma unroll
          for (int k = 0; k < 9; ++k) {
            const C uk = pl[o + (k / 3 - 1) * SU + (k % 3 - 1)];
            const C a = cf[kz * 9 + k];
            if (real) {
              r.x = fma(-a.x, uk.x, r.x);
              r.y = fma(-a.x, uk.y, r.y);
            } else {
              r.x = fma(-a.x, uk.x, r.x);
              r.x = fma(a.y, uk.y, r.x);
              r.y = fma(-a.x, uk.y, r.y);
              r.y = fma(-a.y, uk.x, r.y);
            }
          }
        }
        if (zown && qx >= 2 && qx < F + 2 && qy >= 2 && qy < F + 2 && gx <= n && gy <= n)
          nrm += (double)r.x * (double)r.x + (double)r.y * (double)r.y;
      }
      dst[i] = r;
    }
    return nrm;
  };
  // x-y restriction of r plane z into the rxy ring (two passes, two syncs)
  auto rxy_plane = [&](int z) {
    const C* rp = s_r + rslot(z) * SR * SR;
    for (int i = threadIdx.x; i < (F + 2) * TC; i += NTHR) {
      const int j = i % TC, qy = i / TC;
      const C* p = rp + qy * SR + 3 * j + 2;
      s_Y[qy * TC + j] = restrict5r(p[-2], p[-1], p[0], p[1], p[2]);
    }
    __syncthreads();
    C* dst = s_rxy + xslot(z) * TC * TC;
    for (int i = threadIdx.x; i < TC * TC; i += NTHR) {
      const int jx = i % TC, jy = i / TC;
      const C* yp = s_Y + (3 * jy + 2) * TC + jx;
      dst[i] = restrict5r(yp[-2 * TC], yp[-TC], yp[0], yp[TC], yp[2 * TC]);
    }
    __syncthreads();
  };
  // du at the c-points of fine plane 3*Zc, and its x-y interpolation to the owned points
  auto comp_dc = [&](int Zc) {
    const int z = 3 * Zc;
    const C* rp = s_r + rslot(z) * SR * SR;
    C* dst = s_dc + dslot(Zc) * SD * SD;
    const int tz = ztype(z);
    for (int i = threadIdx.x; i < SD * SD; i += NTHR) {
      const int jx = i % SD, jy = i / SD;
      const int qx = 3 * jx + 2, qy = 3 * jy + 2;
      const int t = s_tx[qx + 1] + 4 * s_ty[qy + 1] + 16 * tz;
      const C r = rp[qy * SR + qx];
      const C w = s_omd[t];
      dst[i] = ((A.realjac >> t) & 1ull) ? rmul(w.x, r) : w * r;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SD * F; i += NTHR) {
      const int qx = i % F, jy = i / F;
      const int ox = qx % 3, jx = qx / 3;
      s_Z[i] = lerp2r(w0r<R>(ox), dst[jy * SD + jx], w1r<R>(ox), dst[jy * SD + jx + 1]);
    }
    __syncthreads();
    C* pi = s_pi + dslot(Zc) * F * F;
    for (int i = threadIdx.x; i < F * F; i += NTHR) {
      const int qx = i % F, qy = i / F;
      const int oy = qy % 3, jy = qy / 3;
      pi[i] = lerp2r(w0r<R>(oy), s_Z[jy * F + qx], w1r<R>(oy), s_Z[(jy + 1) * F + qx]);
    }
  };

  const bool bpx = A.hier && !A.hb;
  double nrm = 0.0;
  // prologue: c planes Z0-1 .. Z0+1, u planes 3Z0-3 .. 3Z0+1, r planes 3Z0-2 .. 3Z0
  for (int Zc = Z0 - 1; Zc <= Z0 + 1; ++Zc) issue_c(Zc);
  for (int z = 3 * Z0 - 3; z <= 3 * Z0 + 1; ++z) issue_u(z);
  for (int z = 3 * Z0 - 2; z <= 3 * Z0; ++z) issue_b(z);
  cp_async_wait_all();
  __syncthreads();
  if (use_c) {
    for (int Zc = Z0 - 1; Zc <= Z0 + 1; ++Zc) cx_pass(Zc);
    __syncthreads();
    for (int z = 3 * Z0 - 3; z <= 3 * Z0 + 1; ++z) add_pc(z);
    __syncthreads();
  }
  save_q(3 * Z0 - 3);
  save_q(3 * Z0);
  for (int z = 3 * Z0 - 2; z <= 3 * Z0; ++z) nrm += comp_r(z);
  __syncthreads();
  if (A.has_coarse)
    for (int z = 3 * Z0 - 2; z <= 3 * Z0; ++z) rxy_plane(z);
  if (bpx) {
    comp_dc(Z0);
    __syncthreads();
  }

  for (int Z = Z0; Z < Z1; ++Z) {
    // a. c plane Z+2, U planes 3Z+2 .. 3Z+4 and b planes 3Z+1 .. 3Z+3, all in flight at once
    issue_c(Z + 2);
    for (int z = 3 * Z + 2; z <= 3 * Z + 4; ++z) issue_u(z);
    for (int z = 3 * Z + 1; z <= 3 * Z + 3; ++z) issue_b(z);
    cp_async_wait_all();
    __syncthreads();
    if (use_c) {
      cx_pass(Z + 2);
      __syncthreads();
      for (int z = 3 * Z + 2; z <= 3 * Z + 4; ++z) add_pc(z);
      __syncthreads();
    }
    save_q(3 * Z + 3);
    // b. residual planes 3Z+1 .. 3Z+3 and their x-y restriction
    for (int z = 3 * Z + 1; z <= 3 * Z + 3; ++z) nrm += comp_r(z);
    __syncthreads();
    if (A.has_coarse)
      for (int z = 3 * Z + 1; z <= 3 * Z + 3; ++z) rxy_plane(z);
    // c. du on c-plane Z+1
    if (bpx) {
      comp_dc(Z + 1);
      __syncthreads();
    }
    // d. coarse outputs of plane Z
    if (A.has_coarse && Z <= nc) {
      for (int i = threadIdx.x; i < TC * TC; i += NTHR) {
        const int jx = i % TC, jy = i / TC;
        const int cx = C0x + jx, cy = C0y + jy;
        if (cx > nc || cy > nc) continue;
        const long long ci = Z * Ncc + (long long)cy * (nc + 1) + cx;
        const bool inner = cx > 0 && cx < nc && cy > 0 && cy < nc && Z > 0 && Z < nc;
        C bs = cz<R>(), uc = cz<R>();
        if (inner) {
          const int t = i;
          const C* r0 = s_rxy + xslot(3 * Z - 2) * TC * TC;
          const C* r1 = s_rxy + xslot(3 * Z - 1) * TC * TC;
          const C* r2 = s_rxy + xslot(3 * Z) * TC * TC;
          const C* r3 = s_rxy + xslot(3 * Z + 1) * TC * TC;
          const C* r4 = s_rxy + xslot(3 * Z + 2) * TC * TC;
          bs = restrict5r(r0[t], r1[t], r2[t], r3[t], r4[t]);
          const int gt = A.gtyp[cx] + kMaxG3 * (A.gtyp[cy] + kMaxG3 * A.gtyp[Z]);
          const C* gc = A.gcoef + gt * 27;
          const int o = (jy + 1) * SQ + (jx + 1);
#pragma unroll
          for (int kz = 0; kz < 3; ++kz) {
            const C* pl = s_q + qslot(Z + kz - 1) * SQ * SQ;
#pragma unroll
            for (int k = 0; k < 9; ++k) bs = cfma(gc[kz * 9 + k], pl[o + (k / 3 - 1) * SQ + (k % 3 - 1)], bs);
          }
          uc = s_q[qslot(Z) * SQ * SQ + o];
        }
        A.b_coarse[ci] = bs;
        A.u_coarse[ci] = uc;
      }
    }
    // e. fine outputs of planes 3Z .. 3Z+2
    for (int oz = 0; oz < 3; ++oz) {
      const int z = 3 * Z + oz;
      if (z > n) break;
      const bool zin = z > 0 && z < n;
      const int tz = ztype(z);
      const C* rp = s_r + rslot(z) * SR * SR;
      const C* u0 = s_u + uslot(z) * SU * SU;
      const C* p0 = s_pi + dslot(Z) * F * F;
      const C* p1 = s_pi + dslot(Z + 1) * F * F;
      for (int i = threadIdx.x; i < F * F; i += NTHR) {
        const int qx = i % F, qy = i / F;
        const int gx = x0 + qx, gy = y0 + qy;
        if (gx > n || gy > n) continue;
        C val = cz<R>();
        if (zin && gx > 0 && gx < n && gy > 0 && gy < n) {
          const int t = s_tx[qx + 3] + 4 * s_ty[qy + 3] + 16 * tz;
          const C r = rp[(qy + 2) * SR + (qx + 2)];
          const C w = s_omd[t];
          C du = ((A.realjac >> t) & 1ull) ? rmul(w.x, r) : w * r;
          if (A.hb && oz == 0 && qx % 3 == 0 && qy % 3 == 0) du = cz<R>();
          if (bpx) du = du - (oz == 0 ? p0[i] : lerp2r(w0r<R>(oz), p0[i], w1r<R>(oz), p1[i]));
          val = A.fine ? u0[(qy + 3) * SU + (qx + 3)] + du : du;
        }
        A.out[z * NN + (long long)gy * N + gx] = val;
      }
    }
    __syncthreads();
  }
  if (A.fine && A.norm2 != nullptr)
    block_norm_finish_tile<NTHR>(nrm, s_red, A.partial, A.ticket, A.norm2, tile, A.ntiles);
}

template <typename R, int TC, int NTHR>
__global__ void __launch_bounds__(NTHR) sweep3_kernel(const Sweep3Args<R> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double s_red[NTHR / 32];
  sweep3_tile<R, TC, NTHR>(A, blockIdx.x, smem_raw, s_red);
}

}  // namespace mg
