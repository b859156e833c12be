// mg_kernels.cuh -- device code of the additive multilevel cycle (sm_103a).
//
// One cycle on levels 1..s (s = finest active level) is
//   sweep(s, fine) -> sweep(s-1) -> ... -> sweep(1) -> prolong(2) -> ... -> prolong(s-1)
// where sweep(l) is the fused fine-to-coarse step of Appendix A Algorithm 4
// on level l (residual r_l = b_l - H_l u_l, Jacobi du_l = omega_l D_l^{-1}
// r_l, surplus uhat_l = u_l - P I u_l, hierarchical residual
// rhat_l = b_l - H_l uhat_l, restriction b_{l-1} = R rhat_l, injection
// u_{l-1} = I u_l) and prolong(l) is corr_l = T_l du_l + P corr_{l-1}.
//
// Single touch on the finest level (Section 5, Algorithm 2 pipelining): the
// fine solution is stored as U = u - P corr_{s-1}, the part of the last
// cycle's update that did not depend on the coarse levels.  The fine sweep
// forms u = U + P corr_{s-1} in shared memory, runs the fused step and
// writes U' = u + T_s du_s once; corr_{s-1} of the new cycle stays pending
// until the next sweep.  So the fine level reads U and b once and writes U'
// once per cycle.
//
// Operator: H_l = sum over cells of K_c - phi_c M_c (Section 4, Appendix B).
// With coordinate-wise exterior scaling every vertex has one of 4^d
// "types" (the scaling class of its left/right cell along each axis), and
// its 3^d stencil row is a table entry of that type, assembled on the host
// from the 1D element matrices.  With a per-cell shift the table holds K
// only and the kernel adds -sum_c phi_c M_c u cell by cell.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mg {

template <typename R>
struct __align__(2 * sizeof(R)) cplx {
  R x, y;
};

template <typename R> __device__ __forceinline__ cplx<R> cz() { return cplx<R>{R(0), R(0)}; }
template <typename R> __device__ __forceinline__ cplx<R> operator+(cplx<R> a, cplx<R> b) {
  return cplx<R>{a.x + b.x, a.y + b.y};
}
template <typename R> __device__ __forceinline__ cplx<R> operator-(cplx<R> a, cplx<R> b) {
  return cplx<R>{a.x - b.x, a.y - b.y};
}
template <typename R> __device__ __forceinline__ cplx<R> operator*(cplx<R> a, cplx<R> b) {
  return cplx<R>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename R> __device__ __forceinline__ cplx<R> rmul(R s, cplx<R> a) {
  return cplx<R>{s * a.x, s * a.y};
}
// acc + a * b
template <typename R> __device__ __forceinline__ cplx<R> cfma(cplx<R> a, cplx<R> b, cplx<R> acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
// acc + s * a (real s)
template <typename R> __device__ __forceinline__ cplx<R> rfma(R s, cplx<R> a, cplx<R> acc) {
  return cplx<R>{fma(s, a.x, acc.x), fma(s, a.y, acc.y)};
}
template <typename R> __device__ __forceinline__ cplx<R> cdiv(cplx<R> a, cplx<R> b) {
  R den = b.x * b.x + b.y * b.y;
  return cplx<R>{(a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den};
}

template <int D> struct P3 { static constexpr int v = 3 * P3<D - 1>::v; };
template <> struct P3<0> { static constexpr int v = 1; };
template <int S, int D> struct IPow { static constexpr int v = S * IPow<S, D - 1>::v; };
template <int S> struct IPow<S, 0> { static constexpr int v = 1; };

constexpr int kMaxTypes = 64;  // 4^3

// Interpolation weights of the tripartite d-linear prolongation: fine
// offset o in {0,1,2} inside a coarse cell takes (1-o/3, o/3).
template <typename R> __device__ __forceinline__ R pw(int o, int b) {
  return o == 0 ? (b == 0 ? R(1) : R(0))
                : (o == 1 ? (b == 0 ? R(2) / R(3) : R(1) / R(3))
                          : (b == 0 ? R(1) / R(3) : R(2) / R(3)));
}
// Restriction weight 1 - |o|/3, o in -2..2.
template <typename R> __device__ __forceinline__ R rw(int o) {
  int a = o < 0 ? -o : o;
  return a == 0 ? R(1) : (a == 1 ? R(2) / R(3) : R(1) / R(3));
}

enum : int { kVariantAdd = 0, kVariantHB = 1 };
enum : int { kTransferDLinear = 0, kTransferHier = 1 };

template <typename R>
struct SweepArgs {
  int n;            // cells per axis of this level (n = 3^l)
  int fine;         // 1: u = U + P c and write U' = u + T du; 0: write T du
  int has_coarse;   // level > 1: restriction and injection outputs
  int hb;           // variant hierarchical basis (mask c-points)
  int hier;         // transfer (id - P I)
  int varphi;       // per-cell shift (table holds K only)
  int first;        // fine: U is zero and nothing is pending (first inner cycle)
  int ntiles;       // tiles of the level (last-tile norm reduction)
  int tiles[3];     // tiles per axis
  const cplx<R>* u;       // fine: pending U; coarse: materialised u_l
  const cplx<R>* c;       // fine: pending corr on level l-1 (nullptr = none)
  const cplx<R>* b;       // rhs b_l
  cplx<R>* out;           // fine: U'; coarse: T du
  cplx<R>* b_coarse;      // b_{l-1}
  cplx<R>* u_coarse;      // u_{l-1} = I u_l
  const uint8_t* typ;     // vertex type per axis index, n+1 entries
  const cplx<R>* coef;    // [4^d][3^d] stencil rows
  const R* phic;          // per-cell shift, n^d (varphi)
  const cplx<R>* hcell;   // complex cell width per axis index, n (varphi)
  cplx<R> omega;          // relaxation factor of this level (varphi)
  cplx<R> omd[kMaxTypes]; // omega / D per vertex type (constant shift)
  double* partial;        // per-block sum |r|^2 (fine)
  unsigned* ticket;       // last-block counter (fine)
  double* norm2;          // |r|^2 over the fine interior (fine)
};

// ---------------------------------------------------------------------------
// Block-wide FP64 sum; the last block to finish sums all block partials in a
// fixed order, so the result is deterministic.
// ---------------------------------------------------------------------------
template <int NTHR>
__device__ __forceinline__ void block_norm_finish(double v, double* s_red, double* partial,
                                                  unsigned* ticket, double* norm2,
                                                  int nblocks) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < NTHR / 32; ++w) t += s_red[w];
    partial[blockIdx.x] = t;
    __threadfence();
    unsigned k = atomicAdd(ticket, 1u);
    s_last = (k == (unsigned)(nblocks - 1));
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    double t = 0;
    for (int i = threadIdx.x; i < nblocks; i += NTHR) t += ((volatile double*)partial)[i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) s_red[warp] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0;
      for (int w = 0; w < NTHR / 32; ++w) s += s_red[w];
      *norm2 = s;
      *ticket = 0u;
    }
  }
}

// Same reduction for tiles processed by any block: partial slot `tile`, the
// last of `ntiles` tiles to finish sums all partials in a fixed order.
template <int NTHR>
__device__ __forceinline__ void block_norm_finish_tile(double v, double* s_red, double* partial,
                                                       unsigned* ticket, double* norm2, int tile,
                                                       int ntiles) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();  // s_red may still be read by a previous item
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  __shared__ int s_last_t;
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < NTHR / 32; ++w) t += s_red[w];
    __stcg(partial + tile, t);
    __threadfence();
    unsigned k = atomicAdd(ticket, 1u);
    s_last_t = (k == (unsigned)(ntiles - 1));
  }
  __syncthreads();
  if (s_last_t) {
    __threadfence();
    double t = 0;
    for (int i = threadIdx.x; i < ntiles; i += NTHR) t += __ldcg(partial + i);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    __syncthreads();
    if (lane == 0) s_red[warp] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0;
      for (int w = 0; w < NTHR / 32; ++w) s += s_red[w];
      __stcg(norm2, s);
      atomicExch(ticket, 0u);
    }
  }
}

// ---------------------------------------------------------------------------
// Shared-memory tile of one sweep.  The block owns coarse vertices
// [C0, C0+TC) per axis, i.e. fine vertices [x0, x0+F), x0 = 3 C0, F = 3 TC.
//   u box   [x0-3, x0+F+1]  (SU = F+5): u, and uhat on [x0-3, x0+F]
//   r box   [x0,   x0+F  ]  (SR = F+1): du; the extra c-point feeds P I du
//   rh box  [x0-2, x0+F-1]  (SH = F+2): rhat, what R of the owned coarse
//                                        vertices reads
//   c box   [C0-1, C0+TC+1] (SC = TC+3): pending coarse correction
// ---------------------------------------------------------------------------
template <int D, int TC>
struct TileGeom {
  static constexpr int F = 3 * TC;
  static constexpr int SU = F + 5;
  static constexpr int SR = F + 1;
  static constexpr int SH = F + 2;
  static constexpr int SC = TC + 3;
  static constexpr int NU = IPow<SU, D>::v;
  static constexpr int NR = IPow<SR, D>::v;
  static constexpr int NH = IPow<SH, D>::v;
  static constexpr int NC = IPow<SC, D>::v;
  static constexpr int NS = P3<D>::v;        // stencil points
  static constexpr int NT = IPow<4, D>::v;   // vertex types
  static constexpr int NCELL = SU - 1;       // cells per axis covered by the u box
};

template <int D>
__device__ __forceinline__ void decode(int t, int S, int* c) {
  c[0] = t % S;
  if (D > 1) c[1] = (t / S) % S;
  if (D > 2) c[2] = t / (S * S);
}

template <typename R, int D, int TC>
size_t sweep_smem_bytes(int varphi) {
  using G = TileGeom<D, TC>;
  size_t b = sizeof(cplx<R>) * (size_t)(2 * G::NU + G::NR + G::NH + G::NC + G::NT * G::NS);
  if (varphi) b += sizeof(R) * (size_t)IPow<G::NCELL, D>::v + sizeof(cplx<R>) * D * G::NCELL;
  return b;
}

// 6^D and 3^D: the mass of a d-linear cell is prod_a h_a / 6^D times the
// integer weight prod_a (2 if the two corners agree along a, else 1); its
// diagonal entry is prod_a h_a / 3^D.
template <int D> struct MassScale {
  static constexpr double inv6 = D == 1 ? 1.0 / 6.0 : (D == 2 ? 1.0 / 36.0 : 1.0 / 216.0);
  static constexpr double inv3 = D == 1 ? 1.0 / 3.0 : (D == 2 ? 1.0 / 9.0 : 1.0 / 27.0);
};

// Integer mass weight of corner q in the row of corner g (bit a of each is
// the local coordinate along axis a).
template <int D>
__host__ __device__ constexpr int mass_weight(int g, int q) {
  int w = 1;
  for (int a = 0; a < D; ++a) w *= (((g >> a) & 1) == ((q >> a) & 1)) ? 2 : 1;
  return w;
}

// Per-cell shift term: sum over the 2^d cells c around vertex g of
// phi_c (M_c u)(g), with M_c the tensor product of 1D masses h/6 [[2,1],[1,2]]:
// per cell one product of the d complex widths and 2^d real-weighted adds.
template <typename R, int D, int TC>
__device__ __forceinline__ cplx<R> mass_phi(const cplx<R>* s, int pbox /*index in u box*/,
                                            const int* bc /*u-box coords of g*/,
                                            const R* s_phi, const cplx<R>* s_h) {
  using G = TileGeom<D, TC>;
  cplx<R> acc = cz<R>();
#pragma unroll
  for (int e = 0; e < (1 << D); ++e) {
    // cell = g - 1 + bit along each axis; its u-box cell index = bc - 1 + bit;
    // g sits at local coordinate 1 - bit along each axis
    int cidx = 0, cstride = 1;
    cplx<R> hp{R(1), R(0)};
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int ca = bc[a] - 1 + ((e >> a) & 1);
      cidx += ca * cstride;
      cstride *= G::NCELL;
      hp = a == 0 ? s_h[ca] : hp * s_h[a * G::NCELL + ca];
    }
    const int gl = ((1 << D) - 1) ^ e;
    cplx<R> loc = cz<R>();
#pragma unroll
    for (int q = 0; q < (1 << D); ++q) {
      int off = 0, ostride = 1;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        off += (((q >> a) & 1) - ((gl >> a) & 1)) * ostride;
        ostride *= G::SU;
      }
      loc = rfma(R(mass_weight<D>(gl, q)), s[pbox + off], loc);
    }
    acc = cfma(rmul(s_phi[cidx], hp), loc, acc);
  }
  return rmul(R(MassScale<D>::inv6), acc);
}

template <typename R, int D, int TC>
__device__ __forceinline__ cplx<R> diag_phi(const int* bc, const R* s_phi, const cplx<R>* s_h) {
  using G = TileGeom<D, TC>;
  cplx<R> acc = cz<R>();
#pragma unroll
  for (int e = 0; e < (1 << D); ++e) {
    cplx<R> hp{R(1), R(0)};
    int cidx = 0, cstride = 1;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int ca = bc[a] - 1 + ((e >> a) & 1);
      hp = a == 0 ? s_h[ca] : hp * s_h[a * G::NCELL + ca];
      cidx += ca * cstride;
      cstride *= G::NCELL;
    }
    acc = acc + rmul(s_phi[cidx], hp);
  }
  return rmul(R(MassScale<D>::inv3), acc);
}

// Loads of arrays that other blocks of the same launch may have written
// (persistent launches) bypass L1.
template <typename T> __device__ __forceinline__ T ldcg_(const T* p) { return __ldcg(p); }
template <> __device__ __forceinline__ cplx<double> ldcg_(const cplx<double>* p) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return cplx<double>{v.x, v.y};
}
template <> __device__ __forceinline__ cplx<float> ldcg_(const cplx<float>* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return cplx<float>{v.x, v.y};
}

// One tile of the sweep (see TileGeom); `tile` indexes the tiles of the
// level with x fastest.
template <typename R, int D, int TC, int NTHR>
__device__ __forceinline__ void sweep_tile(const SweepArgs<R>& A, int tile_index,
                                           unsigned char* smem_raw, double* s_red) {
  using G = TileGeom<D, TC>;
  __syncthreads();  // a previous tile of this block may still read shared memory
  cplx<R>* s_u = reinterpret_cast<cplx<R>*>(smem_raw);
  cplx<R>* s_h = s_u + G::NU;       // uhat
  cplx<R>* s_du = s_h + G::NU;
  cplx<R>* s_rh = s_du + G::NR;
  cplx<R>* s_c = s_rh + G::NH;
  cplx<R>* s_coef = s_c + G::NC;
  R* s_phi = reinterpret_cast<R*>(s_coef + G::NT * G::NS);
  cplx<R>* s_hc = reinterpret_cast<cplx<R>*>(s_phi + IPow<G::NCELL, D>::v);

  const int n = A.n, N = n + 1, nc = n / 3;
  int tile[3] = {0, 0, 0};
  {
    int t = tile_index;
    tile[0] = t % A.tiles[0];
    t /= A.tiles[0];
    if (D > 1) { tile[1] = t % A.tiles[1]; t /= A.tiles[1]; }
    if (D > 2) tile[2] = t;
  }
  int C0[3], x0[3];
#pragma unroll
  for (int a = 0; a < D; ++a) { C0[a] = tile[a] * TC; x0[a] = 3 * C0[a]; }

  // stencil rows
  for (int i = threadIdx.x; i < G::NT * G::NS; i += NTHR) s_coef[i] = A.coef[i];
  // pending coarse correction
  const bool use_c = A.fine && !A.first && A.c != nullptr;
  if (use_c) {
    for (int t = threadIdx.x; t < G::NC; t += NTHR) {
      int q[3];
      decode<D>(t, G::SC, q);
      bool in = true;
      long long gi = 0, st = 1;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        int cc = C0[a] - 1 + q[a];
        in = in && cc >= 0 && cc <= nc;
        gi += (long long)cc * st;
        st *= (nc + 1);
      }
      s_c[t] = in ? ldcg_(A.c + gi) : cz<R>();
    }
  }
  if (A.varphi) {
    for (int t = threadIdx.x; t < IPow<G::NCELL, D>::v; t += NTHR) {
      int q[3];
      decode<D>(t, G::NCELL, q);
      bool in = true;
      long long gi = 0, st = 1;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        int cc = x0[a] - 3 + q[a];
        in = in && cc >= 0 && cc < n;
        gi += (long long)cc * st;
        st *= n;
      }
      s_phi[t] = in ? A.phic[gi] : R(0);
    }
    for (int t = threadIdx.x; t < D * G::NCELL; t += NTHR) {
      int a = t / G::NCELL, q = t % G::NCELL;
      int cc = x0[a] - 3 + q;
      s_hc[t] = (cc >= 0 && cc < n) ? A.hcell[cc] : cplx<R>{R(1), R(0)};
    }
  }
  __syncthreads();

  // u = U (+ P c) on the u box; zero outside the domain and on the boundary
  for (int t = threadIdx.x; t < G::NU; t += NTHR) {
    int q[3];
    decode<D>(t, G::SU, q);
    bool inner = true;
    long long gi = 0, st = 1;
    int g[3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      g[a] = x0[a] - 3 + q[a];
      inner = inner && g[a] > 0 && g[a] < n;
      gi += (long long)g[a] * st;
      st *= N;
    }
    cplx<R> v = cz<R>();
    if (inner && !(A.fine && A.first)) {
      v = ldcg_(A.u + gi);
      if (use_c) {
        // P c: corners of the coarse cell containing g
#pragma unroll
        for (int e = 0; e < (1 << D); ++e) {
          R w = R(1);
          int ci = 0, cs = 1;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            int bit = (e >> a) & 1;
            int o = g[a] % 3;
            w *= pw<R>(o, bit);
            ci += (g[a] / 3 + bit - (C0[a] - 1)) * cs;
            cs *= G::SC;
          }
          if (w != R(0)) v = rfma(w, s_c[ci], v);
        }
      }
    }
    s_u[t] = v;
  }
  __syncthreads();

  // uhat = u - P I u on [x0-3, x0+F] (zero at c-points and outside)
  for (int t = threadIdx.x; t < G::NU; t += NTHR) {
    int q[3];
    decode<D>(t, G::SU, q);
    bool ok = true;
#pragma unroll
    for (int a = 0; a < D; ++a) ok = ok && q[a] <= G::F + 3;
    cplx<R> v = cz<R>();
    if (ok && A.has_coarse) {
      cplx<R> pi = cz<R>();
#pragma unroll
      for (int e = 0; e < (1 << D); ++e) {
        R w = R(1);
        int bi = 0, bs = 1;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          int bit = (e >> a) & 1;
          int o = q[a] % 3;  // box origin x0-3 is a c-point
          w *= pw<R>(o, bit);
          bi += (q[a] - o + 3 * bit) * bs;
          bs *= G::SU;
        }
        if (w != R(0)) pi = rfma(w, s_u[bi], pi);
      }
      v = s_u[t] - pi;
    }
    s_h[t] = v;
  }
  __syncthreads();

  // stencil offsets in the u box
  int soff[G::NS];
#pragma unroll
  for (int k = 0; k < G::NS; ++k) {
    int kk = k, o = 0, st = 1;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      o += (kk % 3 - 1) * st;
      kk /= 3;
      st *= G::SU;
    }
    soff[k] = o;
  }

  // residual r and Jacobi du on the r box; |r|^2 over owned interior
  double nrm = 0.0;
  for (int t = threadIdx.x; t < G::NR; t += NTHR) {
    int q[3];
    decode<D>(t, G::SR, q);
    bool inner = true, owned = true;
    long long gi = 0, st = 1;
    int g[3], bc[3], ty = 0, ts = 1, pb = 0, ps = 1;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      g[a] = x0[a] + q[a];
      inner = inner && g[a] > 0 && g[a] < n;
      owned = owned && q[a] < G::F;
      gi += (long long)g[a] * st;
      st *= N;
      bc[a] = q[a] + 3;
      pb += bc[a] * ps;
      ps *= G::SU;
    }
    cplx<R> du = cz<R>();
    if (inner) {
#pragma unroll
      for (int a = 0; a < D; ++a) { ty += (int)A.typ[g[a]] * ts; ts *= 4; }
      const cplx<R>* cf = s_coef + ty * G::NS;
      cplx<R> hu = cz<R>();
#pragma unroll
      for (int k = 0; k < G::NS; ++k) hu = cfma(cf[k], s_u[pb + soff[k]], hu);
      cplx<R> dg = cf[G::NS / 2];
      if (A.varphi) {
        hu = hu - mass_phi<R, D, TC>(s_u, pb, bc, s_phi, s_hc);
        dg = dg - diag_phi<R, D, TC>(bc, s_phi, s_hc);
      }
      cplx<R> r = ldcg_(A.b + gi) - hu;
      du = A.varphi ? cdiv(A.omega * r, dg) : A.omd[ty] * r;
      if (A.fine && owned) nrm += (double)r.x * (double)r.x + (double)r.y * (double)r.y;
    }
    s_du[t] = du;
  }
  // hierarchical residual on the rh box
  if (A.has_coarse) {
    for (int t = threadIdx.x; t < G::NH; t += NTHR) {
      int q[3];
      decode<D>(t, G::SH, q);
      bool inner = true;
      long long gi = 0, st = 1;
      int g[3], bc[3], ty = 0, ts = 1, pb = 0, ps = 1;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        g[a] = x0[a] - 2 + q[a];
        inner = inner && g[a] > 0 && g[a] < n;
        gi += (long long)g[a] * st;
        st *= N;
        bc[a] = q[a] + 1;
        pb += bc[a] * ps;
        ps *= G::SU;
      }
      cplx<R> rh = cz<R>();
      if (inner) {
#pragma unroll
        for (int a = 0; a < D; ++a) { ty += (int)A.typ[g[a]] * ts; ts *= 4; }
        const cplx<R>* cf = s_coef + ty * G::NS;
        cplx<R> hu = cz<R>();
#pragma unroll
        for (int k = 0; k < G::NS; ++k) hu = cfma(cf[k], s_h[pb + soff[k]], hu);
        if (A.varphi) hu = hu - mass_phi<R, D, TC>(s_h, pb, bc, s_phi, s_hc);
        rh = ldcg_(A.b + gi) - hu;
      }
      s_rh[t] = rh;
    }
  }
  __syncthreads();

  // restriction and injection at the owned coarse vertices
  if (A.has_coarse) {
    const int NCo = IPow<TC, D>::v;
    for (int t = threadIdx.x; t < NCo; t += NTHR) {
      int q[3];
      decode<D>(t, TC, q);
      bool in = true, inner = true;
      long long gi = 0, st = 1;
      int cc[3];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        cc[a] = C0[a] + q[a];
        in = in && cc[a] <= nc;
        inner = inner && cc[a] > 0 && cc[a] < nc;
        gi += (long long)cc[a] * st;
        st *= (nc + 1);
      }
      if (!in) continue;
      cplx<R> bsum = cz<R>();
      if (inner) {
        // rh box index of fine 3C + o is 3 q + o + 2
        for (int k = 0; k < IPow<5, D>::v; ++k) {
          int kk = k, bi = 0, bs = 1;
          R w = R(1);
#pragma unroll
          for (int a = 0; a < D; ++a) {
            int o = kk % 5 - 2;
            kk /= 5;
            w *= rw<R>(o);
            bi += (3 * q[a] + o + 2) * bs;
            bs *= G::SH;
          }
          bsum = rfma(w, s_rh[bi], bsum);
        }
      }
      A.b_coarse[gi] = bsum;
      // u box index of fine 3C is 3 q + 3
      int ui = 0, us = 1;
#pragma unroll
      for (int a = 0; a < D; ++a) { ui += (3 * q[a] + 3) * us; us *= G::SU; }
      A.u_coarse[gi] = inner ? s_u[ui] : cz<R>();
    }
  }

  // transfer T du and output at the owned fine vertices
  {
    const int NF = IPow<G::F, D>::v;
    for (int t = threadIdx.x; t < NF; t += NTHR) {
      int q[3];
      decode<D>(t, G::F, q);
      bool in = true, inner = true, cpt = true;
      long long gi = 0, st = 1;
      int g[3];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        g[a] = x0[a] + q[a];
        in = in && g[a] <= n;
        inner = inner && g[a] > 0 && g[a] < n;
        cpt = cpt && (g[a] % 3 == 0);
        gi += (long long)g[a] * st;
        st *= N;
      }
      if (!in) continue;
      cplx<R> val = cz<R>();
      if (inner) {
        int ri = 0, rs = 1;
#pragma unroll
        for (int a = 0; a < D; ++a) { ri += q[a] * rs; rs *= G::SR; }
        cplx<R> tdu = s_du[ri];
        if (A.hb && cpt) tdu = cz<R>();
        if (A.hier && !A.hb) {
          // t = du - P I du, c-points of the r box (origin x0 is a c-point)
          cplx<R> pi = cz<R>();
#pragma unroll
          for (int e = 0; e < (1 << D); ++e) {
            R w = R(1);
            int bi = 0, bs = 1;
#pragma unroll
            for (int a = 0; a < D; ++a) {
              int bit = (e >> a) & 1;
              int o = q[a] % 3;
              w *= pw<R>(o, bit);
              bi += (q[a] - o + 3 * bit) * bs;
              bs *= G::SR;
            }
            if (w != R(0)) pi = rfma(w, s_du[bi], pi);
          }
          tdu = tdu - pi;
        }
        if (A.fine) {
          int ui = 0, us = 1;
#pragma unroll
          for (int a = 0; a < D; ++a) { ui += (q[a] + 3) * us; us *= G::SU; }
          val = s_u[ui] + tdu;
        } else {
          val = tdu;
        }
      }
      A.out[gi] = val;
    }
  }

  if (A.fine && A.norm2 != nullptr) {
    block_norm_finish_tile<NTHR>(nrm, s_red, A.partial, A.ticket, A.norm2, tile_index, A.ntiles);
  }
}

template <typename R, int D, int TC, int NTHR>
__global__ void __launch_bounds__(NTHR) sweep_kernel(const SweepArgs<R> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double s_red[NTHR / 32];
  sweep_tile<R, D, TC, NTHR>(A, blockIdx.x, smem_raw, s_red);
}

// ---------------------------------------------------------------------------
// Zeroes the Dirichlet ring of a level array (n cells per axis).  2D: 4n
// vertices (rows 0 and n, then columns 0 and n of rows 1..n-1); 3D: the six
// faces as (n+1)^2-vertex sheets (edges written more than once).
// ---------------------------------------------------------------------------
template <int D>
__global__ void zero_ring_kernel(int n, cplx<double>* u) {
  const int N = n + 1;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (D == 2) {
    if (i >= 4 * n) return;
    int x, y;
    if (i < 2 * N) {
      x = i % N;
      y = (i / N) ? n : 0;
    } else {
      const int k = i - 2 * N;  // 0 .. 2(n-1)-1
      y = 1 + k / 2;
      x = (k & 1) ? n : 0;
    }
    u[(size_t)y * N + x] = cz<double>();
  } else {
    const int F = N * N;
    if (i >= 6 * F) return;
    const int face = i / F, a = (i % F) % N, b = (i % F) / N;
    const int v = (face & 1) ? n : 0;
    int x, y, z;
    if (face < 2) { x = v; y = a; z = b; }
    else if (face < 4) { x = a; y = v; z = b; }
    else { x = a; y = b; z = v; }
    u[((size_t)z * N + y) * N + x] = cz<double>();
  }
}

// ---------------------------------------------------------------------------
// corr_l = t_l + P (corr_{l-1} - sub_c) - sub_f on all vertices of level l
// (boundary stays 0).  sub_c (on level l-1) and sub_f (on level l) may be
// null.  With sub_c = I du_l this is the BPX correction
// du_l - P I du_l + P corr_{l-1} of a level that stored t_l = du_l; sub_f =
// I du_{l+1} takes the finer level's P I du into the pending correction.
// ---------------------------------------------------------------------------
template <typename R, int D>
__global__ void prolong_add_kernel(int n, const cplx<R>* __restrict__ t,
                                   const cplx<R>* __restrict__ cc, cplx<R>* __restrict__ out,
                                   const cplx<R>* __restrict__ sub_c = nullptr,
                                   const cplx<R>* __restrict__ sub_f = nullptr) {
  const int N = n + 1, Nc = n / 3 + 1;
  long long total = 1;
  for (int a = 0; a < D; ++a) total *= N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int g[3];
    unsigned r = (unsigned)i;  // vertex counts stay below 2^32
    bool inner = true;
    for (int a = 0; a < D; ++a) {
      g[a] = (int)(r % (unsigned)N);
      r /= (unsigned)N;
      inner = inner && g[a] > 0 && g[a] < n;
    }
    cplx<R> v = cz<R>();
    if (inner) {
      // P with integer weights: the tripartite weights are k/3 per axis, so a
      // corner's weight is an integer product over 3^D, applied once at the end
      cplx<R> acc = cz<R>();
      for (int e = 0; e < (1 << D); ++e) {
        int iw = 1;
        long long ci = 0, cs = 1;
        for (int a = 0; a < D; ++a) {
          const int bit = (e >> a) & 1, o = g[a] % 3;
          iw *= bit ? o : 3 - o;
          ci += (long long)(g[a] / 3 + bit) * cs;
          cs *= Nc;
        }
        if (iw != 0) acc = rfma((R)iw, sub_c != nullptr ? cc[ci] - sub_c[ci] : cc[ci], acc);
      }
      v = rfma(R(1) / R(D == 2 ? 9 : 27), acc, t[i]);
      if (sub_f != nullptr) v = v - sub_f[i];
    }
    out[i] = v;
  }
}

// out = U + P c (c may be null; U null counts as zero): the materialised
// fine solution, or the plain interpolation P c.
template <typename R, int D>
__global__ void materialize_kernel(int n, const cplx<R>* __restrict__ U,
                                   const cplx<R>* __restrict__ c, cplx<R>* __restrict__ out) {
  const int N = n + 1, Nc = n / 3 + 1;
  long long total = 1;
  for (int a = 0; a < D; ++a) total *= N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int g[3];
    unsigned r = (unsigned)i;  // vertex counts stay below 2^32
    bool inner = true;
    for (int a = 0; a < D; ++a) {
      g[a] = (int)(r % (unsigned)N);
      r /= (unsigned)N;
      inner = inner && g[a] > 0 && g[a] < n;
    }
    cplx<R> v = cz<R>();
    if (inner) {
      if (U != nullptr) v = U[i];
      if (c != nullptr) {
        // d-linear weights as integers over 3^D: corner e weighs
        // prod_a (bit ? o_a : 3 - o_a), o_a the offset in the coarse cell
        cplx<R> s = cz<R>();
        for (int e = 0; e < (1 << D); ++e) {
          int iw = 1;
          long long ci = 0, cs = 1;
          for (int a = 0; a < D; ++a) {
            const int bit = (e >> a) & 1, o = g[a] % 3;
            iw *= bit ? o : 3 - o;
            ci += (long long)(g[a] / 3 + bit) * cs;
            cs *= Nc;
          }
          if (iw != 0) s = rfma((R)iw, c[ci], s);
        }
        v = rfma(R(1) / R(D == 2 ? 9 : 27), s, v);
      }
    }
    out[i] = v;
  }
}

// Generic stencil product y = b - A x (or y = A x when b is null) on the
// interior of level n, with x read at stride `xs` from a finer array of
// (xs*n+1)^d vertices (xs = 1: same level).  A is the type table `coef`,
// plus the per-cell shift term when phic != null.  Optional |y|^2 reduction.
// Used for b = M f (rhs set-up) and for the FP64 residual of the
// defect-correction form.
template <typename R, typename RO, int D>
__global__ void stencil_kernel(int n, int xs, const cplx<R>* __restrict__ x,
                               const cplx<R>* __restrict__ b, const uint8_t* __restrict__ typ,
                               const cplx<R>* __restrict__ coef, unsigned long long realmask,
                               const R* __restrict__ phic, const cplx<R>* __restrict__ hcell,
                               cplx<RO>* __restrict__ y, double* partial, unsigned* ticket,
                               double* norm2) {
  constexpr int NS = P3<D>::v;
  const int N = n + 1;
  const long long Nx = (long long)xs * n + 1;
  long long total = 1;
  for (int a = 0; a < D; ++a) total *= N;
  double nrm = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int g[3];
    unsigned r = (unsigned)i;  // vertex counts stay below 2^32
    bool inner = true;
    int ty = 0, ts = 1;
    for (int a = 0; a < D; ++a) {
      g[a] = (int)(r % (unsigned)N);
      r /= (unsigned)N;
      inner = inner && g[a] > 0 && g[a] < n;
    }
    cplx<R> v = cz<R>();
    if (inner) {
      for (int a = 0; a < D; ++a) { ty += (int)typ[g[a]] * ts; ts *= 4; }
      const cplx<R>* cf = coef + ty * NS;
      cplx<R> acc = cz<R>();
      // neighbour k at offset (k % 3 - 1, k / 3 % 3 - 1, k / 9 - 1), stride xs
      auto nbr = [&](int k) -> long long {
        long long xi = 0, st = 1;
        for (int a = 0; a < D; ++a) {
          xi += (long long)(g[a] + k % 3 - 1) * xs * st;
          k /= 3;
          st *= Nx;
        }
        return xi;
      };
      if ((realmask >> ty) & 1ull) {  // row of an unscaled vertex: real x complex
#pragma unroll
        for (int k = 0; k < NS; ++k) acc = rfma(cf[k].x, x[nbr(k)], acc);
      } else {
#pragma unroll
        for (int k = 0; k < NS; ++k) acc = cfma(cf[k], x[nbr(k)], acc);
      }
      if (phic != nullptr) {
        // - sum_c phi_c (M_c x)(g), M_c = prod_a h_a / 6^D x integer weights
        cplx<R> m = cz<R>();
#pragma unroll
        for (int e = 0; e < (1 << D); ++e) {
          int cell[3];
          long long cidx = 0, cst = 1;
          cplx<R> hp{R(1), R(0)};
#pragma unroll
          for (int a = 0; a < D; ++a) {
            cell[a] = g[a] - 1 + ((e >> a) & 1);
            cidx += (long long)cell[a] * cst;
            cst *= n;
            hp = a == 0 ? hcell[cell[a]] : hp * hcell[cell[a]];
          }
          const int gl = ((1 << D) - 1) ^ e;
          cplx<R> loc = cz<R>();
#pragma unroll
          for (int q = 0; q < (1 << D); ++q) {
            long long xi = 0, st = 1;
#pragma unroll
            for (int a = 0; a < D; ++a) {
              xi += (long long)(cell[a] + ((q >> a) & 1)) * xs * st;
              st *= Nx;
            }
            loc = rfma(R(mass_weight<D>(gl, q)), x[xi], loc);
          }
          m = cfma(rmul(phic[cidx], hp), loc, m);
        }
        acc = acc - rmul(R(MassScale<D>::inv6), m);
      }
      v = (b != nullptr) ? b[i] - acc : acc;
      nrm += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
    }
    if (y != nullptr) y[i] = cplx<RO>{(RO)v.x, (RO)v.y};
  }
  if (norm2 != nullptr) {
    __shared__ double s_red[8];
    block_norm_finish<256>(nrm, s_red, partial, ticket, norm2, gridDim.x);
  }
}

// u (FP64) += e (materialised E + P c in precision R); boundary untouched.
template <typename R, int D>
__global__ void update_kernel(int n, cplx<double>* __restrict__ u, const cplx<R>* __restrict__ E,
                              const cplx<R>* __restrict__ c) {
  const int N = n + 1, Nc = n / 3 + 1;
  long long total = 1;
  for (int a = 0; a < D; ++a) total *= N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int g[3];
    unsigned r = (unsigned)i;  // vertex counts stay below 2^32
    bool inner = true;
    for (int a = 0; a < D; ++a) {
      g[a] = (int)(r % (unsigned)N);
      r /= (unsigned)N;
      inner = inner && g[a] > 0 && g[a] < n;
    }
    if (!inner) continue;
    cplx<R> v = E[i];
    if (c != nullptr) {
      for (int e = 0; e < (1 << D); ++e) {
        R w = R(1);
        long long ci = 0, cs = 1;
        for (int a = 0; a < D; ++a) {
          int bit = (e >> a) & 1;
          w *= pw<R>(g[a] % 3, bit);
          ci += (long long)(g[a] / 3 + bit) * cs;
          cs *= Nc;
        }
        if (w != R(0)) v = rfma(w, c[ci], v);
      }
    }
    cplx<double> o = u[i];
    o.x += (double)v.x;
    o.y += (double)v.y;
    u[i] = o;
  }
}

}  // namespace mg
