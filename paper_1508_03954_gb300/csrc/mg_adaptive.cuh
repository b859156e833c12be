// mg_adaptive.cuh -- the additive cycle on an adaptive spacetree with hanging
// vertices (adaptive Cartesian grids of Section 3, hanging vertices and FAS
// injection of Section 4, relaxation factors of Section 5.1),
// FP64, d = 2 or 3, sm_103a.
//
// Every level keeps dense arrays over its full grid plus a flag per cell
// (bit 0: the cell exists, bit 1: it is refined) and a class per vertex
// (0: no existing cell around it, 1: hanging or Dirichlet, 2: unknown = all
// 2^d cells exist).  The cycle kernels run over the bounding box of each
// level's existing vertices, read from device memory, and skip what does
// not exist, so their work follows the adaptive grid.
//
// The cycle is the additive correction scheme on the hierarchical
// generating system of the adaptive grid (Lemma 2 / Theorem 2 form):
//   r_l = sum over the level-l leaves around v of (M_c f - H_c u)_v + R r_{l+1}
// (the restriction carries the partial residuals of hanging vertices),
//   du_l = omega_l r_l / H_l[v, v] at unknowns, hb mask / BPX (id - P I),
//   corr_l = T du_l + P corr_{l-1},  u_l += corr_l on every level,
// then hanging values := P u_{l-1} (coarse to fine) and coarse values at
// vertices with an unknown on the next finer level := that value (fine to
// coarse).  A cycle is three passes: the residuals fine to coarse (norm
// fused), one fused kernel per level coarse to fine, the injection fine to
// coarse -- 3L - 1 launches in one CUDA graph.
//
// Relaxation factors are per vertex (the Section 5.1 table): omega(v) is
// looked up by succ(v), 0 unless all 2^d cells of v's level are refined,
// else 1 + the minimum over v's children that carry unknowns.
//
// Feature-based dynamic refinement (Section 5.3) runs on the device too: the
// indicator s(v) = max over the axes of the undivided second difference at
// the fine-grid vertices, its global span, a histogram over equal bins and
// the choice of how many top / bottom bins to refine / erase, marks on cells
// and vertices (with the residual veto, absolute or relative to |u(v)|), the
// new cell flags (fine to coarse, then existence coarse to fine), the new
// vertex classes with zero hierarchical surplus on new vertices, the new
// bounding boxes, diagonals and succ -- each over the region of its level
// that a step can change.
#pragma once
#include "mg_kernels.cuh"

namespace mg {

enum : uint8_t { kCellExists = 1, kCellRefined = 2 };
enum : uint8_t { kVertNone = 0, kVertBound = 1, kVertUnknown = 2 };

// Bounding box of a level's vertices of existing cells: the cycle kernels
// run over it instead of the level's full grid.
struct AdaBox {
  int lo[3], ext[3];
};

// omega by succ: w[s] is the factor of a vertex with succ(v) = s.
constexpr int kAdaMaxLevels = 16;
struct AdaOmega {
  cplx<double> w[kAdaMaxLevels];
};

enum : uint8_t { kCellNewRef = 4 };  // scratch bit: refined after the step

// Coordinates g and level-grid index of the t-th vertex of the box.
template <int D>
__device__ __forceinline__ unsigned box_vertex(unsigned t, const AdaBox& B, int N, int* g) {
  unsigned i = 0, s = 1;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    g[a] = B.lo[a] + (int)(t % (unsigned)B.ext[a]);
    t /= (unsigned)B.ext[a];
    i += (unsigned)g[a] * s;
    s *= (unsigned)N;
  }
  return i;
}

template <int D>
__device__ __forceinline__ unsigned box_volume(const AdaBox& B) {
  unsigned v = 1;
#pragma unroll
  for (int a = 0; a < D; ++a) v *= (unsigned)B.ext[a];
  return v;
}

template <int D>
__device__ __forceinline__ void ada_coords(unsigned i, int N, int* g) {
#pragma unroll
  for (int a = 0; a < D; ++a) {
    g[a] = (int)(i % (unsigned)N);
    i /= (unsigned)N;
  }
}

// Regions of a level that a refinement step can change, from bounding
// boxes of vertices (null: the level's whole grid).  Iterated like boxes,
// with box_vertex over n cells or n + 1 vertices per axis.
template <int D>
__device__ __forceinline__ AdaBox region_full(int m) {
  AdaBox R;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    R.lo[a] = 0;
    R.ext[a] = a < D ? m : 1;
  }
  return R;
}
// the cells among the vertices of vb
template <int D>
__device__ __forceinline__ AdaBox cell_region(const AdaBox* vb, int n) {
  if (vb == nullptr) return region_full<D>(n);
  AdaBox R = *vb;
#pragma unroll
  for (int a = 0; a < D; ++a) R.ext[a] = R.ext[a] > 0 ? R.ext[a] - 1 : 0;
  return R;
}
// the children of the cells among the vertices of pvb (next coarser level)
template <int D>
__device__ __forceinline__ AdaBox child_cell_region(const AdaBox* pvb, int n) {
  if (pvb == nullptr) return region_full<D>(n);
  AdaBox R = *pvb;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    R.lo[a] *= 3;
    R.ext[a] = R.ext[a] > 0 ? 3 * (R.ext[a] - 1) : 0;
  }
  return R;
}
// the vertices of those children
template <int D>
__device__ __forceinline__ AdaBox child_vertex_region(const AdaBox* pvb, int n) {
  if (pvb == nullptr) return region_full<D>(n + 1);
  AdaBox R = *pvb;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    R.lo[a] *= 3;
    R.ext[a] = R.ext[a] > 0 ? 3 * (R.ext[a] - 1) + 1 : 0;
  }
  return R;
}
// the vertices of vb itself
template <int D>
__device__ __forceinline__ AdaBox vertex_region(const AdaBox* vb, int n) {
  return vb == nullptr ? region_full<D>(n + 1) : *vb;
}

// Entry [a][b] of the element matrices of a cell with per-axis widths h and
// inverse widths hi (corner bits a, b): M = prod h/6 (2 or 1), K = sum_j of
// the same product with axis j's factor replaced by (+1 or -1)/h.
template <int D>
__device__ __forceinline__ void element_entry(const cplx<double>* h, const cplx<double>* hi, int a, int b,
                                              cplx<double>& m, cplx<double>& k) {
  cplx<double> mf[3], kf[3];
#pragma unroll
  for (int ax = 0; ax < D; ++ax) {
    const bool same = ((a >> ax) & 1) == ((b >> ax) & 1);
    mf[ax] = rmul(same ? 1.0 / 3.0 : 1.0 / 6.0, h[ax]);
    kf[ax] = rmul(same ? 1.0 : -1.0, hi[ax]);
  }
  m = mf[0];
#pragma unroll
  for (int ax = 1; ax < D; ++ax) m = m * mf[ax];
  k = cz<double>();
#pragma unroll
  for (int j = 0; j < D; ++j) {
    cplx<double> p = j == 0 ? kf[0] : mf[0];
#pragma unroll
    for (int ax = 1; ax < D; ++ax) p = p * (ax == j ? kf[ax] : mf[ax]);
    k = k + p;
  }
}

// r_l(v) = sum over the leaves around v of (M_c f - H_c u)_v, plus R r_{l+1}
// (rf, the finer level's residual, may be null), zero where no cell exists
// and on the Dirichlet boundary.
// The level's fine-grid unknowns (unknown here, none on the next finer
// level at the same point; vcls_f null on the finest level) add |r|^2 into
// *norm2 (deterministic last-block sum) when norm2 is not null.
template <int D>
__global__ void __launch_bounds__(256) ada_residual_kernel(
    int n, const cplx<double>* __restrict__ u, const cplx<double>* __restrict__ f,
    const uint8_t* __restrict__ cellf, const uint8_t* __restrict__ vcls, const cplx<double>* __restrict__ hcell,
    const cplx<double>* __restrict__ hinv, const double* __restrict__ phic, double phi0,
    const cplx<double>* __restrict__ rf, cplx<double>* __restrict__ r, const uint8_t* __restrict__ vcls_f,
    double* partial, unsigned* ticket, double* norm2, const AdaBox* __restrict__ boxp,
    const uint8_t* __restrict__ rotf, const cplx<double>* __restrict__ emat, unsigned long long* maxabs) {
  const AdaBox box = *boxp;
  const int N = n + 1, Nf = 3 * n + 1;
  const unsigned vol = box_volume<D>(box);
  double nrm = 0.0, mx = 0.0;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < vol; t += gridDim.x * blockDim.x) {
    int g[3];
    const unsigned i = box_vertex<D>(t, box, N, g);
    bool inner = true;
#pragma unroll
    for (int a = 0; a < D; ++a) inner = inner && g[a] > 0 && g[a] < n;
    cplx<double> acc = cz<double>();
    if (inner && vcls[i] != kVertNone) {
#pragma unroll
      for (int e = 0; e < (1 << D); ++e) {
        int c[3];
        unsigned ci = 0, cs = 1;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          c[a] = g[a] - 1 + ((e >> a) & 1);
          ci += (unsigned)c[a] * cs;
          cs *= (unsigned)n;
        }
        if ((cellf[ci] & (kCellExists | kCellRefined)) != kCellExists) continue;  // leaves only
        // the cell's element matrices from the table of its width class
        // (which axes lie in the layer): rows of M and of K - phi0 M
        int cls = 0;
#pragma unroll
        for (int a = 0; a < D; ++a) cls |= (int)rotf[c[a]] << a;
        const int av = ((1 << D) - 1) ^ e;  // v's corner in the cell
        const cplx<double>* Mrow = emat + ((size_t)(2 * cls) << (2 * D)) + (av << D);
        const cplx<double>* Hrow = Mrow + (1 << (2 * D));
        const double dphi = phic != nullptr ? phic[ci] - phi0 : 0.0;
#pragma unroll
        for (int b = 0; b < (1 << D); ++b) {
          unsigned vi = 0, vs = 1;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            vi += (unsigned)(c[a] + ((b >> a) & 1)) * vs;
            vs *= (unsigned)N;
          }
          const cplx<double> m = Mrow[b];
          acc = cfma(m, f[vi], acc);
          cplx<double> hm = Hrow[b];
          if (phic != nullptr) hm = hm - rmul(dphi, m);
          acc = acc - hm * u[vi];
        }
      }
      if (rf != nullptr) {
        // R = P^T: fine 3v + o, o in [-2, 2]^D, weight prod (1 - |o|/3);
        // unrolled so that the loads are in flight together
#pragma unroll
        for (int o = 0; o < (D == 2 ? 25 : 125); ++o) {
          int q = o;
          double w = 1.0;
          unsigned fi = 0, fs = 1;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            const int oa = q % 5 - 2;
            q /= 5;
            const int x = 3 * g[a] + oa;
            w *= oa == 0 ? 1.0 : (oa == -1 || oa == 1 ? 2.0 / 3.0 : 1.0 / 3.0);
            fi += (unsigned)x * fs;
            fs *= (unsigned)Nf;
          }
          acc = rfma(w, rf[fi], acc);
        }
      }
      if (vcls[i] == kVertUnknown) {
        bool own = true;
        if (vcls_f != nullptr) {
          unsigned fi = 0, fs = 1;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            fi += (unsigned)(3 * g[a]) * fs;
            fs *= (unsigned)Nf;
          }
          own = vcls_f[fi] != kVertUnknown;
        }
        if (own) {
          nrm = fma(acc.x, acc.x, fma(acc.y, acc.y, nrm));
          if (maxabs != nullptr) {
            const double m = sqrt(fma(acc.x, acc.x, acc.y * acc.y));
            mx = m == m ? fmax(mx, m) : __longlong_as_double(0x7ff0000000000000LL);  // NaN counts as +inf
          }
        }
      }
    }
    r[i] = acc;
  }
  if (maxabs != nullptr) {
    // non-negative doubles order like their bit patterns
    unsigned long long b = (unsigned long long)__double_as_longlong(mx);
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long q = __shfl_xor_sync(0xffffffffu, b, o);
      b = q > b ? q : b;
    }
    if ((threadIdx.x & 31) == 0 && b != 0ull) atomicMax(maxabs, b);
  }
  if (norm2 != nullptr) {
    __shared__ double s_red[8];
    block_norm_finish<256>(nrm, s_red, partial, ticket, norm2, gridDim.x);
  }
}

// invd(v) = 1 / H_l[v, v] at unknowns (the diagonal summed over the 2^D
// cells), zero elsewhere; formed once per level.
template <int D>
__global__ void ada_diag_kernel(int n, const uint8_t* __restrict__ vcls, const cplx<double>* __restrict__ hcell,
                                const cplx<double>* __restrict__ hinv, const double* __restrict__ phic,
                                double phi0, cplx<double>* __restrict__ invd, const AdaBox* vb) {
  const int N = n + 1;
  const AdaBox R = vertex_region<D>(vb, n);
  const unsigned total = box_volume<D>(R);
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    int g[3];
    const unsigned i = box_vertex<D>(t, R, N, g);
    cplx<double> v = cz<double>();
    if (vcls[i] == kVertUnknown) {
      cplx<double> dg = cz<double>();
#pragma unroll
      for (int e = 0; e < (1 << D); ++e) {
        cplx<double> h[3], hi[3];
        unsigned ci = 0, cs = 1;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const int ca = g[a] - 1 + ((e >> a) & 1);
          h[a] = hcell[ca];
          hi[a] = hinv[ca];
          ci += (unsigned)ca * cs;
          cs *= (unsigned)n;
        }
        const int av = ((1 << D) - 1) ^ e;
        cplx<double> m, k;
        element_entry<D>(h, hi, av, av, m, k);
        dg = dg + (k - rmul(phic != nullptr ? phic[ci] : phi0, m));
      }
      v = cdiv(cplx<double>{1.0, 0.0}, dg);
    }
    invd[i] = v;
  }
}

// One level of the coarse-to-fine half of the cycle, fused: at every vertex
// of an existing cell
//   t = omega r invd at unknowns (zero at c-points for hb),
//   corr = t - [BPX] P I t + P corr_{l-1}     (corr_{l-1} null on level 1),
//   u += corr at unknowns, u = P u_{l-1} at hanging vertices,
// with I t read at the c-points of this level (their t recomputed locally)
// and u_{l-1}, corr_{l-1} already final (levels run coarse to fine).
template <int D>
__global__ void ada_down_kernel(int n, const cplx<double>* __restrict__ r, const cplx<double>* __restrict__ invd,
                                const uint8_t* __restrict__ vcls, const uint8_t* __restrict__ succ, AdaOmega om,
                                int hb, int hier,
                                const cplx<double>* __restrict__ corr_c, const cplx<double>* __restrict__ u_c,
                                cplx<double>* __restrict__ corr, cplx<double>* __restrict__ u,
                                const AdaBox* __restrict__ boxp) {
  const AdaBox box = *boxp;
  const int N = n + 1, Nc = n / 3 + 1;
  const unsigned vol = box_volume<D>(box);
  const double inv = D == 2 ? 1.0 / 9.0 : 1.0 / 27.0;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < vol; t += gridDim.x * blockDim.x) {
    int g[3];
    const unsigned i = box_vertex<D>(t, box, N, g);
    const uint8_t cls = vcls[i];
    if (cls == kVertNone) continue;
    bool inner = true, cpt = true;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      inner = inner && g[a] > 0 && g[a] < n;
      cpt = cpt && (g[a] % 3 == 0);
    }
    if (!inner) {
      corr[i] = cz<double>();
      u[i] = cz<double>();
      continue;
    }
    cplx<double> c = cz<double>();
    if (cls == kVertUnknown && !(hb && cpt)) c = om.w[succ[i]] * (r[i] * invd[i]);
    cplx<double> pc = cz<double>(), pt = cz<double>(), pu = cz<double>();
    if (corr_c != nullptr) {
#pragma unroll
      for (int e = 0; e < (1 << D); ++e) {
        int iw = 1;
        unsigned ci = 0, cs = 1, fi = 0, fs = 1;
        bool ok = true;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const int bit = (e >> a) & 1, o = g[a] % 3;
          iw *= bit ? o : 3 - o;
          const int cc = g[a] / 3 + bit;
          ok = ok && cc < Nc;
          ci += (unsigned)(ok ? cc : 0) * cs;
          cs *= (unsigned)Nc;
          fi += (unsigned)(ok ? 3 * cc : 0) * fs;
          fs *= (unsigned)N;
        }
        if (iw == 0 || !ok) continue;
        const double w = (double)iw;
        pc = rfma(w, corr_c[ci], pc);
        pu = rfma(w, u_c[ci], pu);
        if (hier && !hb && vcls[fi] == kVertUnknown) pt = rfma(w, om.w[succ[fi]] * (r[fi] * invd[fi]), pt);
      }
    }
    c = c - rmul(inv, pt) + rmul(inv, pc);
    corr[i] = c;
    u[i] = cls == kVertUnknown ? u[i] + c : rmul(inv, pu);
  }
}

// y[C] = x[3C] (injection to the next coarser level, n_c cells per axis).
template <int D>
__global__ void ada_inject_kernel(int nc, const cplx<double>* __restrict__ x, cplx<double>* __restrict__ y) {
  const int Nc = nc + 1, Nf = 3 * nc + 1;
  unsigned total = 1;
  for (int a = 0; a < D; ++a) total *= (unsigned)Nc;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    int g[3];
    ada_coords<D>(i, Nc, g);
    unsigned fi = 0, fs = 1;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      fi += (unsigned)(3 * g[a]) * fs;
      fs *= (unsigned)Nf;
    }
    y[i] = x[fi];
  }
}

// y = base + P x or base - P x (neg) on a level with n cells per axis, x on
// the next coarser level; base may be null.  Integer d-linear weights over 3^D.
template <int D>
__global__ void ada_prolong_kernel(int n, const cplx<double>* __restrict__ x, const cplx<double>* base,
                                   cplx<double>* y, int neg) {
  const int N = n + 1, Nc = n / 3 + 1;
  unsigned total = 1;
  for (int a = 0; a < D; ++a) total *= (unsigned)N;
  const double inv = D == 2 ? 1.0 / 9.0 : 1.0 / 27.0;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    int g[3];
    ada_coords<D>(i, N, g);
    cplx<double> s = cz<double>();
#pragma unroll
    for (int e = 0; e < (1 << D); ++e) {
      int iw = 1;
      unsigned ci = 0, cs = 1;
      bool ok = true;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int bit = (e >> a) & 1, o = g[a] % 3;
        iw *= bit ? o : 3 - o;
        const int cc = g[a] / 3 + bit;
        ok = ok && cc < Nc;
        ci += (unsigned)(ok ? cc : 0) * cs;
        cs *= (unsigned)Nc;
      }
      if (iw != 0 && ok) s = rfma((double)iw, x[ci], s);
    }
    s = rmul(inv, s);
    cplx<double> v = s;
    if (base != nullptr) {
      const cplx<double> bi = base[i];
      v = neg ? cplx<double>{bi.x - s.x, bi.y - s.y} : bi + s;
    } else if (neg) {
      v = cplx<double>{-s.x, -s.y};
    }
    y[i] = v;
  }
}

// Hanging values: u(w) = (P u_c)(w) at interior vertices of existing cells
// that carry no unknown (pu: P u_c on this level).
template <int D>
__global__ void ada_set_hanging_kernel(int n, const uint8_t* __restrict__ vcls, const cplx<double>* __restrict__ pu,
                                       cplx<double>* __restrict__ u) {
  const int N = n + 1;
  unsigned total = 1;
  for (int a = 0; a < D; ++a) total *= (unsigned)N;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    if (vcls[i] != kVertBound) continue;
    int g[3];
    ada_coords<D>(i, N, g);
    bool inner = true;
#pragma unroll
    for (int a = 0; a < D; ++a) inner = inner && g[a] > 0 && g[a] < n;
    if (inner) u[i] = pu[i];
  }
}

// Coarse values at vertices carrying an unknown on the finer level take the
// finer value (Eq. injection).
template <int D>
__global__ void ada_inject_unknown_kernel(int nc, const uint8_t* __restrict__ vcls_f,
                                          const cplx<double>* __restrict__ uf, cplx<double>* __restrict__ uc,
                                          const AdaBox* __restrict__ boxp) {
  const AdaBox box = *boxp;
  const int Nc = nc + 1, Nf = 3 * nc + 1;
  const unsigned vol = box_volume<D>(box);
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < vol; t += gridDim.x * blockDim.x) {
    int g[3];
    const unsigned i = box_vertex<D>(t, box, Nc, g);
    unsigned fi = 0, fs = 1;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      fi += (unsigned)(3 * g[a]) * fs;
      fs *= (unsigned)Nf;
    }
    if (vcls_f[fi] == kVertUnknown) uc[i] = uf[fi];
  }
}

// y = x where the level's cells exist around the vertex (vcls != 0), else
// keep y (assembling the fine-grid function level by level).
template <int D>
__global__ void ada_overwrite_kernel(int n, const uint8_t* __restrict__ vcls, const cplx<double>* __restrict__ x,
                                     cplx<double>* __restrict__ y) {
  const int N = n + 1;
  unsigned total = 1;
  for (int a = 0; a < D; ++a) total *= (unsigned)N;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x)
    if (vcls[i] != kVertNone) y[i] = x[i];
}

// ---------------------------------------------------------------------------
// Feature-based dynamic refinement (Section 5.3)

// Fine-grid vertex: an unknown with no unknown at the same point on the
// next finer level (vcls_f null: this is the finest level).
template <int D>
__device__ __forceinline__ bool ada_fine_grid(const uint8_t* vcls, const uint8_t* vcls_f, unsigned i, const int* g,
                                              int Nf) {
  if (vcls[i] != kVertUnknown) return false;
  if (vcls_f == nullptr) return true;
  unsigned fi = 0, fs = 1;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    fi += (unsigned)(3 * g[a]) * fs;
    fs *= (unsigned)Nf;
  }
  return vcls_f[fi] != kVertUnknown;
}

// The bin of s among `bins` equal subranges of [lo, hi], rounded as written
// (no contraction), the top value in the last bin.
__device__ __forceinline__ int ada_bin(double s, double lo, double hi, int bins) {
  if (!(hi > lo)) return 0;
  const double q = __dmul_rn(__ddiv_rn(__dsub_rn(s, lo), __dsub_rn(hi, lo)), (double)bins);
  if (!(q >= 0.0)) return 0;
  if (q >= (double)(bins - 1)) return bins - 1;
  return (int)floor(q);
}

__device__ __forceinline__ void warp_minmax_atomic(unsigned long long lo, unsigned long long hi,
                                                   unsigned long long* mm) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long a = __shfl_xor_sync(0xffffffffu, lo, o);
    const unsigned long long b = __shfl_xor_sync(0xffffffffu, hi, o);
    lo = a < lo ? a : lo;
    hi = b > hi ? b : hi;
  }
  if ((threadIdx.x & 31) == 0) {
    if (lo != ~0ull) atomicMin(mm, lo);
    if (hi != 0ull) atomicMax(mm + 1, hi);
  }
}

// s(v) = max over the axes of |u(v - e) - 2 u(v) + u(v + e)| at the
// fine-grid vertices of the level's box (sums rounded as written), -1
// elsewhere; the span over all levels into mm (bit patterns of non-negative
// doubles: min in mm[0], max in mm[1]) and the number of fine-grid vertices
// into *cnt.  One thread per box vertex: every lane reaches the warp
// reductions.
template <int D>
__global__ void ada_indicator_kernel(int n, const cplx<double>* __restrict__ u, const uint8_t* __restrict__ vcls,
                                     const uint8_t* __restrict__ vcls_f, double* __restrict__ s_out,
                                     const AdaBox* __restrict__ boxp, unsigned long long* mm,
                                     unsigned long long* cnt) {
  const AdaBox box = *boxp;
  const int N = n + 1, Nf = 3 * n + 1;
  const unsigned vol = box_volume<D>(box);
  unsigned long long lo = ~0ull, hi = 0ull;
  unsigned mine = 0;
  for (unsigned t0 = blockIdx.x * blockDim.x; t0 < vol; t0 += gridDim.x * blockDim.x) {
    const unsigned t = t0 + threadIdx.x;
    if (t < vol) {
      int g[3];
      const unsigned i = box_vertex<D>(t, box, N, g);
      double sv = -1.0;
      if (ada_fine_grid<D>(vcls, vcls_f, i, g, Nf)) {
        sv = 0.0;
        unsigned st = 1;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const cplx<double> um = u[i - st], up = u[i + st], u0 = u[i];
          const double sx = __dsub_rn(__dadd_rn(um.x, up.x), __dmul_rn(2.0, u0.x));
          const double sy = __dsub_rn(__dadd_rn(um.y, up.y), __dmul_rn(2.0, u0.y));
          sv = fmax(sv, sqrt(__dadd_rn(__dmul_rn(sx, sx), __dmul_rn(sy, sy))));
          st *= (unsigned)N;
        }
        const unsigned long long b = (unsigned long long)__double_as_longlong(sv);
        lo = b < lo ? b : lo;
        hi = b > hi ? b : hi;
        ++mine;
      }
      s_out[i] = sv;
    }
  }
  warp_minmax_atomic(lo, hi, mm);
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0 && mine != 0u) atomicAdd(cnt, (unsigned long long)mine);
}

// Histogram of the fine-grid vertices over the bins (bins <= 64).
template <int D>
__global__ void ada_hist_kernel(int n, const double* __restrict__ s, const AdaBox* __restrict__ boxp,
                                const unsigned long long* mm, int bins, unsigned long long* counts) {
  const AdaBox box = *boxp;
  __shared__ unsigned h[64];
  for (int k = threadIdx.x; k < 64; k += blockDim.x) h[k] = 0u;
  __syncthreads();
  const int N = n + 1;
  const double lo = __longlong_as_double((long long)mm[0]), hi = __longlong_as_double((long long)mm[1]);
  const unsigned vol = box_volume<D>(box);
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < vol; t += gridDim.x * blockDim.x) {
    int g[3];
    const unsigned i = box_vertex<D>(t, box, N, g);
    const double sv = s[i];
    if (sv >= 0.0) atomicAdd(&h[ada_bin(sv, lo, hi, bins)], 1u);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < bins; k += blockDim.x)
    if (h[k] != 0u) atomicAdd(counts + k, (unsigned long long)h[k]);
}

// The numbers of top and bottom bins to refine and erase: for each, the
// smallest k whose vertex total is closest to frac x (fine-grid vertices),
// written to kb[0] (first refined bin: bins - k) and kb[1] (bins below k are
// erased).  A non-finite indicator span selects nothing.  One thread.
__global__ void ada_choose_bins_kernel(const unsigned long long* counts, const unsigned long long* nfine,
                                       const unsigned long long* mm, int bins, double refine_frac,
                                       double erase_frac, int* kb) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (!isfinite(__longlong_as_double((long long)mm[1]))) {
    kb[0] = bins;
    kb[1] = 0;
    return;
  }
  const double n = (double)*nfine;
  for (int side = 0; side < 2; ++side) {
    const double goal = (side == 0 ? refine_frac : erase_frac) * n;
    int best_k = 0;
    double best = fabs(goal);
    unsigned long long acc = 0;
    for (int k = 1; k <= bins; ++k) {
      acc += counts[side == 0 ? bins - k : k - 1];
      const double dist = fabs((double)acc - goal);
      if (dist < best) {
        best = dist;
        best_k = k;
      }
    }
    kb[side] = side == 0 ? bins - best_k : best_k;
  }
}

// Selection: a fine-grid vertex in the top bins (bin >= kb[0]) that is
// not vetoed (|r / H[v, v]| <= veto, or <= veto |u(v)| with veto_relative)
// is refined -- its 2^D cells get
// rmark -- when can_refine; one in the bottom bins (bin < kb[1]), not in
// the top ones and not vetoed gets emark when can_erase.  sel[0], sel[1]
// count them.  The marks start at zero (the kernels that consume them
// clear them).
template <int D>
__global__ void ada_mark_kernel(int n, const double* __restrict__ s, const cplx<double>* __restrict__ r,
                                const cplx<double>* __restrict__ invd, const AdaBox* __restrict__ boxp,
                                const unsigned long long* mm, const cplx<double>* __restrict__ u,
                                int bins, const int* kb, double veto, int veto_relative, int can_refine, int can_erase,
                                uint8_t* __restrict__ rmark, uint8_t* __restrict__ emark,
                                unsigned long long* sel) {
  const AdaBox box = *boxp;
  const int N = n + 1;
  const double lo = __longlong_as_double((long long)mm[0]), hi = __longlong_as_double((long long)mm[1]);
  const int ref_from = kb[0], er_below = kb[1];
  const unsigned vol = box_volume<D>(box);
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < vol; t += gridDim.x * blockDim.x) {
    int g[3];
    const unsigned i = box_vertex<D>(t, box, N, g);
    const double sv = s[i];
    if (!(sv >= 0.0)) continue;
    const int b = ada_bin(sv, lo, hi, bins);
    const cplx<double> q = r[i] * invd[i];
    double bound = veto;
    if (veto_relative) {
      const cplx<double> uv = u[i];
      bound = veto * sqrt(fma(uv.x, uv.x, uv.y * uv.y));
    }
    const bool vetoed = sqrt(fma(q.x, q.x, q.y * q.y)) > bound;
    const bool top = b >= ref_from && !vetoed;
    if (top && can_refine) {
#pragma unroll
      for (int e = 0; e < (1 << D); ++e) {
        unsigned ci = 0, cs = 1;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          ci += (unsigned)(g[a] - 1 + ((e >> a) & 1)) * cs;
          cs *= (unsigned)n;
        }
        rmark[ci] = 1;
      }
      atomicAdd(sel, 1ull);
    } else if (!top && b < er_below && !vetoed && can_erase) {
      emark[i] = 1;
      atomicAdd(sel + 1, 1ull);
    }
  }
}

// New refine bit (kCellNewRef) of the level's cells, levels fine to coarse:
// refined after the step when marked, or refined before and not coarsened.
// A cell is coarsened (allow: its level is at least the h_max level) when it
// is refined, none of its 3^D children is refined or marked, and every
// fine-grid vertex of the next level on the closed cell carries emark.
// rmark_f, vcls_ff may be null (the next level is the finest).
template <int D>
__global__ void ada_coarsen_kernel(int n, uint8_t* __restrict__ cellf, const uint8_t* __restrict__ rmark,
                                   const uint8_t* __restrict__ cellf_f, const uint8_t* __restrict__ rmark_f,
                                   const uint8_t* __restrict__ vcls_f, const uint8_t* __restrict__ vcls_ff,
                                   const uint8_t* __restrict__ emark_f, int allow, const AdaBox* vb) {
  const AdaBox R = cell_region<D>(vb, n);  // cells that exist or carry marks lie among the old box's vertices
  const unsigned total = box_volume<D>(R);
  const int nf = 3 * n, Nf = nf + 1, Nff = 3 * nf + 1;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    int c[3];
    const unsigned ci = box_vertex<D>(t, R, n, c);
    const uint8_t old = cellf[ci] & (kCellExists | kCellRefined);
    bool coarsen = false;
    if (allow && (old & kCellRefined)) {
      coarsen = true;
      for (int o = 0; o < (D == 2 ? 9 : 27) && coarsen; ++o) {
        unsigned k = 0, ks = 1;
        int q = o;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          k += (unsigned)(3 * c[a] + q % 3) * ks;
          q /= 3;
          ks *= (unsigned)nf;
        }
        if ((cellf_f[k] & kCellRefined) || (rmark_f != nullptr && rmark_f[k])) coarsen = false;
      }
      for (int o = 0; o < (D == 2 ? 16 : 64) && coarsen; ++o) {
        int w[3];
        unsigned wi = 0, ws = 1;
        int q = o;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          w[a] = 3 * c[a] + q % 4;
          q /= 4;
          wi += (unsigned)w[a] * ws;
          ws *= (unsigned)Nf;
        }
        if (ada_fine_grid<D>(vcls_f, vcls_ff, wi, w, Nff) && !emark_f[wi]) coarsen = false;
      }
    }
    const bool nr = (old & kCellExists) && (rmark[ci] || ((old & kCellRefined) && !coarsen));
    cellf[ci] = old | (nr ? kCellNewRef : 0);
  }
}

// Final flags, levels coarse to fine: a cell exists on level 1 or when its
// parent (final) is refined; it is refined when it exists and carries
// kCellNewRef.  Clears the level's refine marks.
template <int D>
__global__ void ada_finalize_cells_kernel(int n, uint8_t* __restrict__ cellf, const uint8_t* __restrict__ cellf_p,
                                          uint8_t* __restrict__ rmark, const AdaBox* pvb) {
  // the level's cells before and after the step are children of cells that
  // existed on the next coarser level (old box pvb; null on level 1)
  const AdaBox R = child_cell_region<D>(pvb, n);
  const unsigned total = box_volume<D>(R);
  const int np = n / 3;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    int c[3];
    const unsigned ci = box_vertex<D>(t, R, n, c);
    bool ex = true;
    if (cellf_p != nullptr) {
      unsigned pi = 0, ps = 1;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        pi += (unsigned)(c[a] / 3) * ps;
        ps *= (unsigned)np;
      }
      ex = (cellf_p[pi] & kCellRefined) != 0;
    }
    const bool rf = ex && (cellf[ci] & kCellNewRef);
    cellf[ci] = (uint8_t)((ex ? kCellExists : 0) | (rf ? kCellRefined : 0));
    rmark[ci] = 0;
  }
}

// New vertex classes of a level from its final cells (levels coarse to
// fine), with zero hierarchical surplus on vertices that exist after the
// step and did not carry an unknown both before and after it: u = P u_c
// (u_c final; null on level 1), zero on the Dirichlet boundary.  The bounding
// box of the vertices of existing cells goes to box6 (min x, y, z, max x, y, z).
// Clears the level's erase marks and the residual of vertices that vanish
// (the restriction of the next coarser level reads it).
template <int D>
__global__ void ada_reclass_kernel(int n, const uint8_t* __restrict__ cellf, uint8_t* __restrict__ vcls,
                                   cplx<double>* __restrict__ u, const cplx<double>* __restrict__ u_c, int* box6,
                                   uint8_t* __restrict__ emark, cplx<double>* __restrict__ r, const AdaBox* pvb) {
  // vertices of the level's cells before and after the step: those of the
  // children of the cells that existed on the next coarser level (old box
  // pvb; null on level 1)
  const AdaBox R = child_vertex_region<D>(pvb, n);
  const int N = n + 1, Nc = n / 3 + 1;
  const unsigned total = box_volume<D>(R);
  const double inv = D == 2 ? 1.0 / 9.0 : 1.0 / 27.0;
  int lo[3] = {N, N, N}, hi[3] = {-1, -1, -1};
  for (unsigned t0 = blockIdx.x * blockDim.x; t0 < total; t0 += gridDim.x * blockDim.x) {
    const unsigned t = t0 + threadIdx.x;
    if (t < total) {
      int g[3];
      const unsigned i = box_vertex<D>(t, R, N, g);
      int cnt = 0;
      bool inner = true;
#pragma unroll
      for (int e = 0; e < (1 << D); ++e) {
        unsigned ci = 0, cs = 1;
        bool in = true;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const int ca = g[a] - 1 + ((e >> a) & 1);
          in = in && ca >= 0 && ca < n;
          ci += (unsigned)(in ? ca : 0) * cs;
          cs *= (unsigned)n;
        }
        if (in && (cellf[ci] & kCellExists)) ++cnt;
      }
#pragma unroll
      for (int a = 0; a < D; ++a) inner = inner && g[a] > 0 && g[a] < n;
      const uint8_t nc = cnt == 0 ? kVertNone : ((inner && cnt == (1 << D)) ? kVertUnknown : kVertBound);
      const uint8_t oc = vcls[i];
      if (nc != kVertNone) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
          lo[a] = min(lo[a], g[a]);
          hi[a] = max(hi[a], g[a]);
        }
        if (u_c != nullptr && !(nc == kVertUnknown && oc == kVertUnknown)) {
          cplx<double> pu = cz<double>();
          if (inner) {
#pragma unroll
            for (int e = 0; e < (1 << D); ++e) {
              int iw = 1;
              unsigned ci = 0, cs = 1;
              bool ok = true;
#pragma unroll
              for (int a = 0; a < D; ++a) {
                const int bit = (e >> a) & 1, o = g[a] % 3;
                iw *= bit ? o : 3 - o;
                const int cc = g[a] / 3 + bit;
                ok = ok && cc < Nc;
                ci += (unsigned)(ok ? cc : 0) * cs;
                cs *= (unsigned)Nc;
              }
              if (iw != 0 && ok) pu = rfma((double)iw, u_c[ci], pu);
            }
            pu = rmul(inv, pu);
          }
          u[i] = pu;
        }
      }
      vcls[i] = nc;
      emark[i] = 0;
      if (nc == kVertNone && oc != kVertNone) r[i] = cz<double>();  // no stale residual outside the boxes
    }
  }
  for (int a = 0; a < D; ++a) {
    int l = lo[a], h = hi[a];
    for (int o = 16; o > 0; o >>= 1) {
      l = min(l, __shfl_xor_sync(0xffffffffu, l, o));
      h = max(h, __shfl_xor_sync(0xffffffffu, h, o));
    }
    if ((threadIdx.x & 31) == 0 && h >= 0) {
      atomicMin(box6 + a, l);
      atomicMax(box6 + 3 + a, h);
    }
  }
}

// box6 of levels 0..nlev-1 before the reclass passes: min = large, max = -1.
__global__ void ada_box_init_kernel(int* box6, int nlev) {
  for (int k = threadIdx.x; k < 6 * nlev; k += blockDim.x) box6[k] = k % 6 < 3 ? (1 << 30) : -1;
}

// The bounding boxes of levels 1..L from box6 (an empty level gets a box of
// zero volume).  One thread.
template <int D>
__global__ void ada_boxes_kernel(const int* __restrict__ box6, int L, AdaBox* __restrict__ boxes) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int l = 1; l <= L; ++l) {
    const int* b = box6 + 6 * l;
    const bool empty = b[3] < 0;
    AdaBox B;
    for (int a = 0; a < 3; ++a) {
      B.lo[a] = a < D && !empty ? b[a] : 0;
      B.ext[a] = empty ? 0 : (a < D ? b[3 + a] - b[a] + 1 : 1);
    }
    boxes[l] = B;
  }
}

// succ(v) at the unknowns of a level (levels fine to coarse; succ_f null on
// the finest level): 0 unless all 2^D cells around v are refined, else 1 +
// the minimum of succ over the unknowns of the next level at 3v + o,
// o in [-3, 3]^D.  The level's fine-grid vertices are counted into *nfine.
template <int D>
__global__ void ada_succ_kernel(int n, const uint8_t* __restrict__ cellf, const uint8_t* __restrict__ vcls,
                                const uint8_t* __restrict__ vcls_f, const uint8_t* __restrict__ succ_f,
                                uint8_t* __restrict__ succ, unsigned long long* nfine, const AdaBox* vb) {
  const int N = n + 1, Nf = 3 * n + 1;
  const AdaBox R = vertex_region<D>(vb, n);  // the unknowns lie in the level's (new) box
  const unsigned total = box_volume<D>(R);
  unsigned mine = 0;
  for (unsigned t0 = blockIdx.x * blockDim.x; t0 < total; t0 += gridDim.x * blockDim.x) {
    const unsigned t = t0 + threadIdx.x;
    if (t < total) {
      int g[3];
      const unsigned i = box_vertex<D>(t, R, N, g);
      uint8_t sv = 0;
      if (vcls[i] == kVertUnknown) {
        if (ada_fine_grid<D>(vcls, vcls_f, i, g, Nf)) ++mine;
        bool refined = succ_f != nullptr;
#pragma unroll
        for (int e = 0; e < (1 << D); ++e) {
          unsigned ci = 0, cs = 1;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            ci += (unsigned)(g[a] - 1 + ((e >> a) & 1)) * cs;
            cs *= (unsigned)n;
          }
          refined = refined && (cellf[ci] & kCellRefined);
        }
        if (refined) {
          int m = 255;
          for (int o = 0; o < (D == 2 ? 49 : 343); ++o) {
            unsigned fi = 0, fs = 1;
            int q = o;
#pragma unroll
            for (int a = 0; a < D; ++a) {
              fi += (unsigned)(3 * g[a] + q % 7 - 3) * fs;
              q /= 7;
              fs *= (unsigned)Nf;
            }
            if (vcls_f[fi] == kVertUnknown) m = min(m, (int)succ_f[fi]);
          }
          sv = (uint8_t)(m + 1);
        }
      }
      succ[i] = sv;
    }
  }
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0 && mine != 0u) atomicAdd(nfine, (unsigned long long)mine);
}

}  // namespace mg
