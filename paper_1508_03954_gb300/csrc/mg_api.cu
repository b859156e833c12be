// mg_api.cu -- C ABI of the GB300 additive multilevel Helmholtz solver
// (declarations and argument contracts in include/mg.h).
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <type_traits>
#include <string>
#include <vector>

#include "mg.h"
#include "mg_kernels.cuh"
#include "mg_sweep2d.cuh"
#include "mg_sweep3d.cuh"
#include "mg_sweep3s.cuh"
#include "mg_defect3.cuh"
#include "mg_sweep3sd.cuh"
#include "mg_coarse3.cuh"
#include "mg_sweep2w.cuh"
#include "mg_persist.cuh"
#include "mg_adjoint.cuh"
#include "mg_maxnorm.cuh"
#include "mg_dim4.cuh"
#include "mg_io.cuh"
#include "mg_adaptive.cuh"
#include <map>

using mg::cplx;
using cd = std::complex<double>;

namespace {

constexpr int kMaxDepth2 = 9;  // (3^9+1)^2 vertices: 387 M
constexpr int kMaxDepth3 = 6;  // (3^6+1)^3 vertices: 389 M
constexpr int kMaxDepth4 = 4;  // (3^4+1)^4 vertices: 45 M (five fine-size temporaries)
constexpr int kThreads = 256;
constexpr int kTC2 = 8;        // coarse cells per tile edge, 2D
constexpr int kTC3 = 2;        // coarse cells per tile edge, 3D
// 2D levels whose 8-cell tiles would not give every SM a block take 2-cell
// tiles (a latency-bound level gains more from spreading than it loses to
// the wider halo).
inline int tc2_for(int n) {
  const int t8 = (n / 3 + 1 + kTC2 - 1) / kTC2;
  return t8 * t8 < 152 ? 2 : kTC2;
}

// resident blocks per SM of the persistent launches
#ifndef MG_FINE_BPSM
#define MG_FINE_BPSM 4
#endif
#ifndef MG_CHAIN_BPSM
#define MG_CHAIN_BPSM 4
#endif
constexpr int kTraceFine = 1 << 16;   // trace slots of the fine sweep
constexpr int kTraceChain = 1 << 16;  // trace slots of the chain

long long ipow(long long b, int e) {
  long long r = 1;
  while (e-- > 0) r *= b;
  return r;
}

// Per-level operator data and arrays of one precision.
template <typename R>
struct Hier {
  struct Lev {
    int n = 0;
    size_t nv = 0;
    cplx<R>* u[2] = {nullptr, nullptr};
    cplx<R>* b = nullptr;
    cplx<R>* t = nullptr;
    cplx<R>* corr = nullptr;  // level 1 aliases t
    uint8_t* typ = nullptr;
    cplx<R>* coefH = nullptr;
    cplx<R>* coefM = nullptr;
    R* phic = nullptr;
    cplx<R>* hcell = nullptr;
    std::vector<cd> diag;     // D per vertex type (constant shift)
    unsigned realrow = 0;     // bit t: stencil row of type t is real (2D types)
    unsigned long long realrow3 = 0;  // same for the 64 3D types
    unsigned long long realM = 0;     // bit t: mass row of type t is real
    bool g3ok = false;        // 3D Galerkin-row tables available
    unsigned greal = 0;       // bit k: 1D Galerkin row class k is real (3D)
    unsigned* s3pref = nullptr; // 3D FP64 separable sweep: prefix sums of the unit costs
    cplx<R>* idu = nullptr;     // 3D BPX with stored du (separable FP64 sweep, point levels): du at the c-points (level l-1 layout)
    cplx<R>* r = nullptr;       // 3D point levels (mg_coarse3.cuh): r_l for the next coarser level's restriction
    unsigned* s3split_f = nullptr;  // 3D separable sweeps: balanced unit ranges, finest-level grid
    unsigned* s3split_c = nullptr;  //   and coarse-level grid
    int s3grid_f = 0, s3grid_c = 0;
    // 2D FP64 path: Galerkin rows of G_{l-1} = R H_l P per coarse row class
    bool gok = false;
    int* order8 = nullptr;      // fine tiles (8 coarse cells) by decreasing cost
    unsigned* tflags = nullptr; // per such tile: generation + 1 once written (chain overlap)
    unsigned* d3pref = nullptr; // 3D FP64 defect: prefix sums of the unit costs
    uint8_t* gtyp = nullptr;
    cplx<R>* gcoef = nullptr;
  };
  int d = 0, L = 0;
  bool varphi = false;
  bool ready = false;
  std::vector<Lev> lev;
  int cur = 0;               // active fine U buffer
  // captured cycles: key -> (fine sweep graph, coarse chain graph)
  struct GraphEntry {
    std::vector<double> key;
    cudaGraphExec_t fine = nullptr, coarse = nullptr;
    int nfine = 0, ncoarse = 0;  // kernel nodes
  };
  std::vector<GraphEntry> graphs;
  // persistent coarse-chain plans: key -> device item list and argument tables
  struct ChainPlan {
    std::vector<double> key;
    mg::ChainItem* items = nullptr;
    mg::Sweep2Args<R>* s2 = nullptr;
    mg::ProlongArgs<R>* pr = nullptr;
    mg::CorrArgs<R>* co = nullptr;
    int nitems = 0, grid = 0;
  };
  std::vector<ChainPlan> chains;
  double* partial = nullptr;
  unsigned* ticket = nullptr;
  double* norm2 = nullptr;   // [0] cycle norm, [1] standalone norm, [2] max modulus (bits)
  std::vector<void*> allocs;
};

// Four-dimensional hierarchy (mg_dim4.cuh) in precision R: per level the
// solution (coarse: the injected copy), b, T du, the correction, and the
// separable operator as per-index 1D rows; fine-size temporaries for the
// pass chains.
template <typename R>
struct Lev4 {
  int n = 0;
  size_t nv = 0;
  cplx<R>* u = nullptr;
  cplx<R>* b = nullptr;
  cplx<R>* t = nullptr;
  cplx<R>* corr = nullptr;   // level 1: aliases t
  uint8_t* typ = nullptr;    // vertex type per axis index
  cplx<R>* rows = nullptr;   // [M, K, K - phi M][n + 1][3] of this level's operator
  cplx<R>* grows = nullptr;  // same for G = R H P on level l - 1 (l > 1)
  cplx<R>* invd = nullptr;   // [256] inverse diagonal by vertex type
  cplx<R>* omd = nullptr;    // [256] omega / D of the current cycle
  bool real = false;         // every row of `rows` is real
  bool greal = false;        // every row of `grows` is real
  bool dreal = false;        // every entry of `invd` is real
};

template <typename R>
struct Hier4 {
  std::vector<Lev4<R>> lev;   // 1..L
  cplx<R>* T[5] = {};         // fine-size temporaries; T[4] holds the residual
  double* partial = nullptr;  // block partials of the norms
  unsigned* ticket = nullptr;
  double* norm2 = nullptr;    // [0] cycle norm, [1] standalone norm, [2] max modulus (bits)
  std::vector<void*> allocs;
  cudaGraphExec_t exec = nullptr;  // the last captured cycle
  std::vector<double> key;
  long long nkern = 0;
};

// Adaptive spacetree (mg_adaptive.cuh): dense arrays over each level's full
// grid with a flag per cell and a class per vertex.
struct LevA {
  int n = 0;
  size_t nv = 0;
  cplx<double>* u = nullptr;
  cplx<double>* f = nullptr;     // nodal f sampled on this level
  cplx<double>* r = nullptr;     // generating-system residual
  cplx<double>* t = nullptr;     // T du
  cplx<double>* corr = nullptr;  // level 1: aliases t
  uint8_t* cellf = nullptr;      // kCellExists | kCellRefined per cell
  uint8_t* vcls = nullptr;       // kVertNone / kVertBound / kVertUnknown per vertex
  cplx<double>* hcell = nullptr; // complex width per axis index
  cplx<double>* hinv = nullptr;  // its inverse
  double* phic = nullptr;        // per-cell shift (null: constant)
  cplx<double>* invd = nullptr;  // 1 / H_l[v, v] at unknowns
  mg::AdaBox box{};              // bounding box of the vertices of existing cells
  size_t boxvol = 0;
  uint8_t* rotf = nullptr;       // per axis index: the cell lies in the layer
  cplx<double>* emat = nullptr;  // per width class: M, then K - phi0 M (2^d x 2^d each)
  uint8_t* succ = nullptr;       // succ(v) at unknowns (Section 5.1)
  double* s = nullptr;           // refinement indicator (-1: not a fine-grid vertex)
  uint8_t* rmark = nullptr;      // per cell: refined by this step's selection
  uint8_t* emark = nullptr;      // per vertex: selected for erasing
};

// Device scratch of the adaptive context (unsigned long long slots).
enum : int {
  kAbMinMax = 0,   // [2] span of the indicator (bit patterns)
  kAbCount = 2,    // fine-grid vertices seen by the indicator
  kAbSel = 3,      // [2] vertices selected for refining, erasing
  kAbFine = 5,     // fine-grid vertices after the step
  kAbBins = 6,     // [2] (as 4 ints) first refined bin, bins erased below
  kAbMax = 8,      // [kAdaMaxSlots] per-level max |r| (bit patterns)
  kAbCounts = 32,  // [64] histogram
  kAbSlots = 96,
  kAdaMaxSlots = 16
};

struct HierA {
  std::vector<LevA> lev;       // 1..L
  int Lf = 1;                  // finest level with cells
  unsigned long long* abuf = nullptr;  // kAb* slots
  int* box6 = nullptr;                 // per level: min x, y, z, max x, y, z
  mg::AdaBox* boxes = nullptr;         // per level: the bounding box, read by the kernels
  std::vector<int> gcap;               // per level: grid of the box kernels (grows, never shrinks)
  void* hbuf = nullptr;                // page-locked host mirror (4 KB)
  cudaGraphExec_t aexec = nullptr;     // the last captured refinement step
  std::vector<double> akey, aseen;
  long long ankern = 0;
  cplx<double>* T[2] = {};     // fine-size temporaries
  double* partial = nullptr;
  unsigned* ticket = nullptr;
  double* norm2 = nullptr;     // [l]: |r_l|^2 over the level's fine-grid unknowns
  std::vector<void*> allocs;
  cudaGraphExec_t exec = nullptr;  // the last captured cycle
  std::vector<double> key;
  std::vector<double> seen;    // a key run once without a graph (captured when it repeats)
  long long nkern = 0;
};

}  // namespace

struct mg_ctx {
  int d = 0, L = 0;
  double theta = 0, theta_in = 0;      // layer / interior rotation of the cell widths
  double wlo = 0, whi = 0;             // layer widths at the low / high face of every axis
  cudaStream_t stream = 0;
  Hier<double> h64;
  Hier<float> h32;
  Hier4<double>* h4 = nullptr;         // d = 4
  Hier4<float>* h4f = nullptr;         // d = 4, complex64 inner cycles
  HierA* ada = nullptr;                // adaptive spacetree (mg_create_adaptive)
  int precision = MG_C128;
  int inner_cycles = 4;
  double r0 = -1.0;                    // reference residual norm
  std::vector<double> k2;              // fine k^2 (host copy)
  cplx<double>* f_dev = nullptr;       // nodal f (fine)
  cplx<double>* scratch = nullptr;     // fine-size FP64 scratch
  double* k2dev = nullptr;             // fine k^2 field set from device memory (mg_set_k2)
  int device = -1;                     // CUDA device current at creation
  bool k2_host_stale = false;          // k2 (host copy) older than k2dev
  cplx<double>* rvec = nullptr;        // fine residual vector (allocated on first use)
  double* host_norm = nullptr;         // pinned
  std::string err;
  cudaStream_t cap_stream = nullptr;   // private stream the cycle graphs are captured on
  unsigned* chain_ctr = nullptr;       // [0] queue head, [1..] completion counters
  unsigned* dev_err = nullptr;         // bounded-wait timeout flag (sticky until read)
  unsigned spin_limit = 1u << 22;
  bool debug_stall = false;            // next chain launches wait on a counter nothing sets
  int chain_bpsm = 0;                  // resident chain blocks per SM
  int fine_bpsm = MG_FINE_BPSM;        // persistent fine-sweep blocks per SM
  // optional per-item trace of the persistent launches (last cycle only)
  unsigned long long* trace = nullptr; // [0, 4*kTraceFine): fine sweep; then chain
  bool tracing = false;
  bool use_graphs = true;
  // instrumentation
  long long launches = 0;
  bool timing = false;
  std::vector<cudaEvent_t> ev;         // pairs around fine sweeps
  size_t ev_used = 0;
};

namespace {

thread_local std::string g_create_err;

int fail(mg_ctx* c, int code, const std::string& m) {
  if (c) c->err = m; else g_create_err = m;
  return code;
}

#define MG_CUDA(ctx, call)                                                              \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      return fail((ctx), e_ == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA,   \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                 \
    }                                                                                   \
  } while (0)

// ------------------------------------------------------------------ geometry
// Along one axis a cell of level l lies in the scaling layer when its centre
// (i + 1/2)/n is closer than wlo to the low face or closer than whi to the
// high face: 2i+1 < 2 wlo n or 2n-2i-1 < 2 whi n (integer form); layers that
// cover the axis (wlo + whi >= 1) scale every cell (complex scaled grid).
std::vector<uint8_t> layer_flags(int n, double wlo, double whi) {
  std::vector<uint8_t> rot(n);
  for (int i = 0; i < n; ++i) {
    long long a = 2LL * i + 1, b = 2LL * n - 2LL * i - 1;
    rot[i] = (wlo + whi >= 1.0) || ((double)a < 2.0 * wlo * (double)n) || ((double)b < 2.0 * whi * (double)n);
  }
  return rot;
}

std::vector<uint8_t> layer_flags(const mg_ctx* c, int n) { return layer_flags(n, c->wlo, c->whi); }

// The two complex cell widths of a level with n cells per axis: h e^{i theta}
// in the scaling layer, h e^{i theta_in} elsewhere (theta_in = 0 gives the
// real h exactly).
struct Widths {
  cd in, rot;
};
Widths widths(const mg_ctx* c, int n) {
  const double h = 1.0 / n;
  return {h * cd(std::cos(c->theta_in), std::sin(c->theta_in)), h * cd(std::cos(c->theta), std::sin(c->theta))};
}

// The fast separable kernels (warp-strip 2D, z-marching 3D, fused 3D defect)
// take the rows of cells outside the layer as real; a rotated interior makes
// them complex and sends every level to the kernels with complex rows.
bool interior_real(const mg_ctx* c) { return c->theta_in == 0.0; }

// Coarse 3D levels up to 81 cells per axis with a constant shift run the
// one-thread-per-vertex kernel (mg_coarse3.cuh) within a cycle.
constexpr int kPoint3MaxN = 81;

// Stencil rows of the d-linear element operator for every vertex type.  A
// vertex of type t has left/right cell widths hl, hr along each axis; its
// assembled 1D stiffness row is (-1/hl, 1/hl + 1/hr, -1/hr) and its 1D mass
// row (hl/6, (hl+hr)/3, hr/6).  The d-dimensional rows are the tensor
// products K = sum_j (x)_a (K if a == j else M), M = (x)_a M (Section 4).
void type_tables(int d, const Widths& wd, std::vector<cd>& K, std::vector<cd>& M) {
  cd KX[4][3], MX[4][3];
  for (int t = 0; t < 4; ++t) {
    cd hl = (t & 1) ? wd.rot : wd.in, hr = (t & 2) ? wd.rot : wd.in;
    KX[t][0] = -1.0 / hl;
    KX[t][1] = 1.0 / hl + 1.0 / hr;
    KX[t][2] = -1.0 / hr;
    MX[t][0] = hl / 6.0;
    MX[t][1] = (hl + hr) / 3.0;
    MX[t][2] = hr / 6.0;
  }
  const int NT = (int)ipow(4, d), NS = (int)ipow(3, d);
  K.assign((size_t)NT * NS, cd(0));
  M.assign((size_t)NT * NS, cd(0));
  for (int t = 0; t < NT; ++t) {
    int ta[3] = {t % 4, (t / 4) % 4, t / 16};
    for (int k = 0; k < NS; ++k) {
      int ka[3] = {k % 3, (k / 3) % 3, k / 9};
      cd m(1);
      for (int a = 0; a < d; ++a) m *= MX[ta[a]][ka[a]];
      cd kk(0);
      for (int j = 0; j < d; ++j) {
        cd p(1);
        for (int a = 0; a < d; ++a) p *= (a == j ? KX[ta[a]][ka[a]] : MX[ta[a]][ka[a]]);
        kk += p;
      }
      K[(size_t)t * NS + k] = kk;
      M[(size_t)t * NS + k] = m;
    }
  }
}

// 1D Galerkin rows P1^T A P1 of level l's assembled 1D stiffness (A = K) and
// mass (A = M) on the coarse indices of level l-1, with P1 the tripartite
// interpolation (weights 1 - |o|/3).  Entry [C][0..2] is the coupling of
// coarse C with C-1, C, C+1 (interior C only; the rest stays zero).
// The coarse hat of C rises by 1/3 per fine cell over the three cells
// 3C-3..3C-1 (left, widths l0..l2) and falls by 1/3 over 3C..3C+2 (right,
// r0..r2), so with the linear element integrals of each fine cell
//   K: (-sum 1/l / 9, (sum 1/l + sum 1/r) / 9, -sum 1/r / 9)
//   M: ((7 l0 + 13 l1 + 7 l2) / 54,
//       (l0 + 7 l1 + 19 l2 + 19 r0 + 7 r1 + r2) / 27,
//       (7 r0 + 13 r1 + 7 r2) / 54).
// Written this way the stiffness row sums to zero up to one rounding per
// entry (exactly, for real widths h = 3^-l), which keeps the rounding of
// G u_{l-1} -- a sum that cancels to O(h^2) for smooth u -- near that of
// the fine stencil.  Couplings to boundary neighbours are formed like the
// others (they multiply Dirichlet zeros), so they do not split row classes.
void galerkin_rows_1d(int n, const std::vector<uint8_t>& rot, const Widths& wd,
                      std::vector<std::array<cd, 6>>& rows) {
  auto hw = [&](int cell) { return rot[cell] ? wd.rot : wd.in; };
  const int nc = n / 3;
  rows.assign(nc + 1, std::array<cd, 6>{});
  for (int c = 1; c < nc; ++c) {
    const cd l0 = hw(3 * c - 3), l1 = hw(3 * c - 2), l2 = hw(3 * c - 1);
    const cd r0 = hw(3 * c), r1 = hw(3 * c + 1), r2 = hw(3 * c + 2);
    const cd aL = 1.0 / l0 + 1.0 / l1 + 1.0 / l2, aR = 1.0 / r0 + 1.0 / r1 + 1.0 / r2;
    auto& row = rows[c];
    row[0] = -aL / 9.0;
    row[1] = (aL + aR) / 9.0;
    row[2] = -aR / 9.0;
    row[3] = (7.0 * l0 + 13.0 * l1 + 7.0 * l2) / 54.0;
    row[4] = (l0 + 7.0 * l1 + 19.0 * l2 + 19.0 * r0 + 7.0 * r1 + r2) / 27.0;
    row[5] = (7.0 * r0 + 13.0 * r1 + 7.0 * r2) / 54.0;
  }
}

template <typename R>
std::vector<cplx<R>> to_dev_type(const std::vector<cd>& v) {
  std::vector<cplx<R>> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = cplx<R>{(R)v[i].real(), (R)v[i].imag()};
  return o;
}

template <typename R>
int dalloc(mg_ctx* c, Hier<R>& H, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(c, MG_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  H.allocs.push_back(*p);
  e = cudaMemset(*p, 0, bytes);
  if (e != cudaSuccess) return fail(c, MG_ERR_CUDA, cudaGetErrorString(e));
  return MG_OK;
}

template <typename R>
void drop_graphs(Hier<R>& H) {
  for (auto& g : H.graphs) {
    if (g.fine) cudaGraphExecDestroy(g.fine);
    if (g.coarse) cudaGraphExecDestroy(g.coarse);
  }
  H.graphs.clear();
}

template <typename R>
void free_hier(Hier<R>& H) {
  drop_graphs(H);
  for (auto& cp : H.chains) {
    cudaFree(cp.items);
    cudaFree(cp.s2);
    cudaFree(cp.pr);
    cudaFree(cp.co);
  }
  H.chains.clear();
  for (void* p : H.allocs) cudaFree(p);
  H.allocs.clear();
  H.lev.clear();
  H.ready = false;
}

// Cell shift of level l: mean of the 2^d vertex values of k^2 sampled on the
// level's own vertices (injection of the fine field).
template <typename R>
std::vector<R> cell_shift(const mg_ctx* c, int l) {
  const int d = c->d, n = (int)ipow(3, l);
  const long long stride = ipow(3, c->L - l), NL = ipow(3, c->L) + 1;
  const size_t ncell = (size_t)ipow(n, d);
  std::vector<R> phic(ncell);
  for (size_t ci = 0; ci < ncell; ++ci) {
    long long q[3] = {0, 0, 0}, r = (long long)ci;
    for (int a = 0; a < d; ++a) { q[a] = r % n; r /= n; }
    double acc = 0;
    for (int e = 0; e < (1 << d); ++e) {
      long long gi = 0, st = 1;
      for (int a = 0; a < d; ++a) {
        gi += (q[a] + ((e >> a) & 1)) * stride * st;
        st *= NL;
      }
      acc += c->k2[(size_t)gi];
    }
    phic[ci] = (R)(acc / (double)(1 << d));
  }
  return phic;
}

int grid_for(size_t nv);

// Cell shift of level l formed on the device from the device copy of the fine
// field (the values of cell_shift), enqueued on the context's stream.
template <typename R>
cudaError_t cell_shift_dev(mg_ctx* c, int l, R* phic) {
  const int n = (int)ipow(3, l);
  const long long stride = ipow(3, c->L - l), NL = ipow(3, c->L) + 1;
  const size_t ncell = (size_t)ipow(n, c->d);
  ++c->launches;
  if (c->d == 2)
    mg::cell_shift_kernel<R, 2><<<grid_for(ncell), kThreads, 0, c->stream>>>(n, stride, NL, c->k2dev, phic);
  else
    mg::cell_shift_kernel<R, 3><<<grid_for(ncell), kThreads, 0, c->stream>>>(n, stride, NL, c->k2dev, phic);
  return cudaGetLastError();
}

// Contiguous ranges of (tile, coarse plane) units for G blocks of the 3D
// separable sweeps, minimising the largest range cost (binary search on the
// bound, greedy fill).  A range pays its units' costs plus a warm-up of two
// fine planes (2/3 of a unit) where it starts and wherever it enters a new
// tile (each tile's z-march starts two planes early for the restriction).
// Returns G + 1 unit indices (block b takes [r[b], r[b+1])).
std::vector<unsigned> balanced_ranges(const std::vector<unsigned>& pref, int nc, int G) {
  const size_t U = pref.size() - 1;
  auto cost = [&](size_t u) { return (double)(pref[u + 1] - pref[u]); };
  auto fill = [&](double T, std::vector<unsigned>* split) -> bool {
    int b = 0;
    double acc = 0.0;
    long long tile = -1;
    if (split) split->assign(1, 0u);
    for (size_t u = 0; u < U; ++u) {
      const long long t = (long long)(u / (size_t)nc);
      const double add = cost(u) * (t != tile ? 5.0 / 3.0 : 1.0);
      if (acc > 0.0 && acc + add > T) {
        if (++b >= G) return false;
        if (split) split->push_back((unsigned)u);
        acc = cost(u) * 5.0 / 3.0;
      } else {
        acc += add;
      }
      tile = t;
    }
    if (split) {
      while ((int)split->size() < G) split->push_back((unsigned)U);
      split->push_back((unsigned)U);
    }
    return true;
  };
  double lo = 0.0, hi = 2.0 * (double)pref[U] + 1.0;
  for (int it = 0; it < 60; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (fill(mid, nullptr)) hi = mid; else lo = mid;
  }
  std::vector<unsigned> split;
  fill(hi, &split);
  return split;
}

// Builds the arrays and tables of one precision.
template <typename R>
int build_hier(mg_ctx* c, Hier<R>& H) {
  const int d = c->d, L = c->L;
  H.d = d;
  H.L = L;
  H.lev.assign(L + 1, typename Hier<R>::Lev());
  const int nL = (int)ipow(3, L);
  // constant or varying shift
  bool constant = true;
  for (size_t i = 1; i < c->k2.size(); ++i)
    if (c->k2[i] != c->k2[0]) { constant = false; break; }
  H.varphi = !constant;
  const double phi0 = c->k2[0];
  size_t max_blocks = 1;
  int rc;
  for (int l = 1; l <= L; ++l) {
    auto& V = H.lev[l];
    V.n = (int)ipow(3, l);
    V.nv = (size_t)ipow(V.n + 1, d);
    const size_t bytes = V.nv * sizeof(cplx<R>);
    for (int k = 0; k < 2; ++k)
      if ((rc = dalloc(c, H, (void**)&V.u[k], bytes)) != MG_OK) return rc;
    if ((rc = dalloc(c, H, (void**)&V.b, bytes)) != MG_OK) return rc;
    if ((rc = dalloc(c, H, (void**)&V.t, bytes)) != MG_OK) return rc;
    if (l == 1) {
      V.corr = V.t;
    } else if ((rc = dalloc(c, H, (void**)&V.corr, bytes)) != MG_OK) {
      return rc;
    }
    // vertex types
    std::vector<uint8_t> rot = layer_flags(c, V.n), typ(V.n + 1);
    const Widths wd = widths(c, V.n);
    for (int i = 0; i <= V.n; ++i) {
      int left = rot[std::max(i - 1, 0)], right = rot[std::min(i, V.n - 1)];
      typ[i] = (uint8_t)(left + 2 * right);
    }
    if ((rc = dalloc(c, H, (void**)&V.typ, typ.size())) != MG_OK) return rc;
    MG_CUDA(c, cudaMemcpy(V.typ, typ.data(), typ.size(), cudaMemcpyHostToDevice));
    std::vector<cd> K, M;
    type_tables(d, wd, K, M);
    std::vector<cd> Hh(K.size());
    for (size_t i = 0; i < K.size(); ++i) Hh[i] = H.varphi ? K[i] : K[i] - phi0 * M[i];
    const int NT = (int)ipow(4, d), NS = (int)ipow(3, d);
    V.diag.resize(NT);
    for (int t = 0; t < NT; ++t) V.diag[t] = Hh[(size_t)t * NS + NS / 2];
    V.realrow = 0;
    V.realrow3 = 0;
    for (int t = 0; t < NT; ++t) {
      bool re = true, rm = true;
      for (int k = 0; k < NS; ++k) re = re && Hh[(size_t)t * NS + k].imag() == 0.0;
      for (int k = 0; k < NS; ++k) rm = rm && M[(size_t)t * NS + k].imag() == 0.0;
      if (re && t < 32) V.realrow |= 1u << t;
      if (re) V.realrow3 |= 1ull << t;
      if (rm) V.realM |= 1ull << t;
    }
    if (d == 3 && !H.varphi && l > 1) {
      std::vector<std::array<cd, 6>> rows;
      galerkin_rows_1d(V.n, rot, wd, rows);
      std::vector<std::array<cd, 6>> cls;
      std::vector<uint8_t> gt(rows.size(), 0);
      bool ok = true;
      for (size_t ci = 1; ci + 1 < rows.size() && ok; ++ci) {
        size_t k = 0;
        while (k < cls.size() && cls[k] != rows[ci]) ++k;
        if (k == cls.size()) {
          if ((int)cls.size() == mg::kMaxG3) { ok = false; break; }
          cls.push_back(rows[ci]);
        }
        gt[ci] = (uint8_t)k;
      }
      for (size_t k = 0; k < cls.size() && ok; ++k) {
        bool re = true;
        for (int j = 0; j < 6; ++j) re = re && cls[k][j].imag() == 0.0;
        if (re) V.greal |= 1u << k;
      }
      if (ok) {
        const int G = mg::kMaxG3;
        std::vector<cd> gc((size_t)G * G * G * 27, cd(0));
        for (size_t gz = 0; gz < cls.size(); ++gz)
          for (size_t gy = 0; gy < cls.size(); ++gy)
            for (size_t gx = 0; gx < cls.size(); ++gx)
              for (int k = 0; k < 27; ++k) {
                const int dx = k % 3, dy = (k / 3) % 3, dz = k / 9;
                const auto& X = cls[gx];
                const auto& Y = cls[gy];
                const auto& Zr = cls[gz];
                gc[(gx + G * (gy + G * gz)) * 27 + k] =
                    X[dx] * Y[3 + dy] * Zr[3 + dz] + X[3 + dx] * Y[dy] * Zr[3 + dz] +
                    X[3 + dx] * Y[3 + dy] * Zr[dz] - phi0 * X[3 + dx] * Y[3 + dy] * Zr[3 + dz];
              }
        auto gcd = to_dev_type<R>(gc);
        if ((rc = dalloc(c, H, (void**)&V.gtyp, gt.size())) != MG_OK) return rc;
        if ((rc = dalloc(c, H, (void**)&V.gcoef, gcd.size() * sizeof(cplx<R>))) != MG_OK) return rc;
        MG_CUDA(c, cudaMemcpy(V.gtyp, gt.data(), gt.size(), cudaMemcpyHostToDevice));
        MG_CUDA(c, cudaMemcpy(V.gcoef, gcd.data(), gcd.size() * sizeof(cplx<R>), cudaMemcpyHostToDevice));
        V.g3ok = true;
      }
    }
    if (d == 3 && !H.varphi && l > 1 && V.n >= 27 && V.g3ok) {
      // cost of each (9 x 9 coarse-cell tile, coarse plane) unit of the
      // separable sweeps: complex128 is bound by the FP64 pipe, so its weights
      // are FP64 operations per lane -- z-pair on the 32 box rows (10 real,
      // 24 complex), y-pair (16 / 36), x-pass (12 / 26) and the rest (~30) on
      // the 30 residual rows; complex64 is bound by instruction issue, where
      // the complex passes add less than a third as much relative to a row's
      // other work (weights 4 / 4 / 6 measured fastest; 7 / 7 / 10 and
      // 10 / 10 / 14 left the slowest blocks 1-5% further behind).  Blocks
      // take ranges of equal cost.
      const unsigned cz_ = std::is_same<R, double>::value ? 14u : 4u;
      const unsigned cx_ = std::is_same<R, double>::value ? 14u : 4u;
      const unsigned cy_ = std::is_same<R, double>::value ? 20u : 6u;
      const int n = V.n, nc = n / 3, tl = (nc + 8) / 9;
      std::vector<unsigned> pref((size_t)tl * tl * nc + 1, 0u);
      size_t u = 0;
      for (int t = 0; t < tl * tl; ++t) {
        const int x0 = (t % tl) * 27, y0 = (t / tl) * 27;
        bool xc = false;
        for (int g = x0 - 2; g <= x0 + 27; ++g) xc = xc || (g >= 0 && g <= n && typ[g] != 0);
        int yc = 0;
        for (int g = y0 - 2; g <= y0 + 27; ++g) yc += (g >= 0 && g <= n && typ[g] != 0) ? 1 : 0;
        for (int Z = 0; Z < nc; ++Z, ++u) {
          unsigned cost = 0;
          for (int z = 3 * Z; z < 3 * Z + 3; ++z)
            cost += 32u * (10u + (typ[z] != 0 ? cz_ : 0u)) + 30u * (58u + (xc ? cx_ : 0u)) + cy_ * (unsigned)yc;
          pref[u + 1] = pref[u] + cost;
        }
      }
      if ((rc = dalloc(c, H, (void**)&V.s3pref, pref.size() * sizeof(unsigned))) != MG_OK) return rc;
      MG_CUDA(c, cudaMemcpy(V.s3pref, pref.data(), pref.size() * sizeof(unsigned), cudaMemcpyHostToDevice));
      // ranges for the launch grids of the finest-level and coarse-level sweeps
      for (int k = 0; k < 2; ++k) {
        const long long U = (long long)tl * tl * nc;
        const long long upb = k == 0 ? 4 : (std::is_same<R, double>::value ? 2 : 1);
        const int G = (int)std::min<long long>(152, std::max<long long>(1, (U + upb - 1) / upb));
        const std::vector<unsigned> sp = balanced_ranges(pref, nc, G);
        unsigned*& dst = k == 0 ? V.s3split_f : V.s3split_c;
        if ((rc = dalloc(c, H, (void**)&dst, sp.size() * sizeof(unsigned))) != MG_OK) return rc;
        MG_CUDA(c, cudaMemcpy(dst, sp.data(), sp.size() * sizeof(unsigned), cudaMemcpyHostToDevice));
        (k == 0 ? V.s3grid_f : V.s3grid_c) = G;
      }
      if (std::is_same<R, double>::value &&
          (rc = dalloc(c, H, (void**)&V.idu, (size_t)ipow(nc + 1, 3) * sizeof(cplx<R>))) != MG_OK)
        return rc;
    }
    if (d == 3 && !H.varphi && l > 1 && V.g3ok && V.n <= kPoint3MaxN) {
      // a coarse level of the point kernel: its residual (read by the next
      // coarser level's restriction) and, for BPX, du at its c-points
      if ((rc = dalloc(c, H, (void**)&V.r, bytes)) != MG_OK) return rc;
      if (V.idu == nullptr &&
          (rc = dalloc(c, H, (void**)&V.idu, (size_t)ipow(V.n / 3 + 1, 3) * sizeof(cplx<R>))) != MG_OK)
        return rc;
    }
    if (d == 2 && !H.varphi && V.n / 3 + 1 >= 200) {
      // LPT order of the 8-coarse-cell tiles: interior vertices weighted by
      // the cost of their stencil row (complex rows cost about twice)
      const int nc = V.n / 3, tl = (nc + 8) / 8;
      std::vector<std::pair<double, int>> cost;
      for (int ty = 0; ty < tl; ++ty)
        for (int tx = 0; tx < tl; ++tx) {
          double w = 0;
          for (int gy = 24 * ty; gy < std::min(24 * ty + 24, V.n); ++gy)
            for (int gx = 24 * tx; gx < std::min(24 * tx + 24, V.n); ++gx) {
              if (gx == 0 || gy == 0) continue;
              const bool cpx = typ[gx] != 0 || typ[gy] != 0;
              w += cpx ? 2.0 : 1.0;
            }
          cost.push_back({-(w + 50.0), ty * tl + tx});
        }
      std::stable_sort(cost.begin(), cost.end());
      std::vector<int> order;
      for (auto& pr : cost) order.push_back(pr.second);
      if ((rc = dalloc(c, H, (void**)&V.order8, order.size() * sizeof(int))) != MG_OK) return rc;
      MG_CUDA(c, cudaMemcpy(V.order8, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice));
      if ((rc = dalloc(c, H, (void**)&V.tflags, order.size() * sizeof(unsigned))) != MG_OK) return rc;
    }
    if (d == 2 && !H.varphi && l > 1) {
      // classes of 1D Galerkin rows along an axis (same on both axes)
      std::vector<std::array<cd, 6>> rows;
      galerkin_rows_1d(V.n, rot, wd, rows);
      std::vector<std::array<cd, 6>> cls;
      std::vector<uint8_t> gt(rows.size(), 0);
      bool ok = true;
      for (size_t ci = 1; ci + 1 < rows.size() && ok; ++ci) {
        size_t k = 0;
        while (k < cls.size() && cls[k] != rows[ci]) ++k;
        if (k == cls.size()) {
          if ((int)cls.size() == mg::kMaxGTypes) { ok = false; break; }
          cls.push_back(rows[ci]);
        }
        gt[ci] = (uint8_t)k;
      }
      if (ok) {
        const int G = mg::kMaxGTypes;
        std::vector<cd> gc((size_t)G * G * 9, cd(0));
        for (size_t gy = 0; gy < cls.size(); ++gy)
          for (size_t gx = 0; gx < cls.size(); ++gx)
            for (int k = 0; k < 9; ++k) {
              const int dx = k % 3, dy = k / 3;
              const auto& X = cls[gx];
              const auto& Y = cls[gy];
              gc[(gx + G * gy) * 9 + k] = X[dx] * Y[3 + dy] + X[3 + dx] * Y[dy] - phi0 * X[3 + dx] * Y[3 + dy];
            }
        auto gcd = to_dev_type<R>(gc);
        if ((rc = dalloc(c, H, (void**)&V.gtyp, gt.size())) != MG_OK) return rc;
        if ((rc = dalloc(c, H, (void**)&V.gcoef, gcd.size() * sizeof(cplx<R>))) != MG_OK) return rc;
        MG_CUDA(c, cudaMemcpy(V.gtyp, gt.data(), gt.size(), cudaMemcpyHostToDevice));
        MG_CUDA(c, cudaMemcpy(V.gcoef, gcd.data(), gcd.size() * sizeof(cplx<R>), cudaMemcpyHostToDevice));
        V.gok = true;
      }
    }
    auto hH = to_dev_type<R>(Hh), hM = to_dev_type<R>(M);
    if ((rc = dalloc(c, H, (void**)&V.coefH, hH.size() * sizeof(cplx<R>))) != MG_OK) return rc;
    if ((rc = dalloc(c, H, (void**)&V.coefM, hM.size() * sizeof(cplx<R>))) != MG_OK) return rc;
    MG_CUDA(c, cudaMemcpy(V.coefH, hH.data(), hH.size() * sizeof(cplx<R>), cudaMemcpyHostToDevice));
    MG_CUDA(c, cudaMemcpy(V.coefM, hM.data(), hM.size() * sizeof(cplx<R>), cudaMemcpyHostToDevice));
    if (H.varphi) {
      const size_t ncell = (size_t)ipow(V.n, d);
      if ((rc = dalloc(c, H, (void**)&V.phic, ncell * sizeof(R))) != MG_OK) return rc;
      if (c->k2_host_stale) {
        // the field was last set from device memory
        MG_CUDA(c, cell_shift_dev<R>(c, l, V.phic));
        MG_CUDA(c, cudaStreamSynchronize(c->stream));
      } else {
        std::vector<R> phic = cell_shift<R>(c, l);
        MG_CUDA(c, cudaMemcpy(V.phic, phic.data(), ncell * sizeof(R), cudaMemcpyHostToDevice));
      }
    }
    {
      // complex cell width per axis index (per-cell shift and adjoint kernels)
      std::vector<cd> hc(V.n);
      for (int i = 0; i < V.n; ++i) hc[i] = rot[i] ? wd.rot : wd.in;
      auto hcd = to_dev_type<R>(hc);
      if ((rc = dalloc(c, H, (void**)&V.hcell, hcd.size() * sizeof(cplx<R>))) != MG_OK) return rc;
      MG_CUDA(c, cudaMemcpy(V.hcell, hcd.data(), hcd.size() * sizeof(cplx<R>), cudaMemcpyHostToDevice));
    }
    const int TC = d == 2 ? tc2_for(V.n) : kTC3;
    size_t nb = (size_t)ipow((V.n / 3 + 1 + TC - 1) / TC, d);
    max_blocks = std::max(max_blocks, nb);
  }
  max_blocks = std::max<size_t>(max_blocks, 152 * 16);
  if ((rc = dalloc(c, H, (void**)&H.partial, max_blocks * sizeof(double))) != MG_OK) return rc;
  if ((rc = dalloc(c, H, (void**)&H.ticket, 4 * sizeof(unsigned))) != MG_OK) return rc;
  if ((rc = dalloc(c, H, (void**)&H.norm2, 4 * sizeof(double))) != MG_OK) return rc;
  H.cur = 0;
  H.ready = true;
  return MG_OK;
}

// ------------------------------------------------------------------ launches
template <typename R, int D, int TC>
cudaError_t launch_sweep_tc(cudaStream_t s, mg::SweepArgs<R>& A) {
  const int nc = A.n / 3;
  const int tiles = (nc + 1 + TC - 1) / TC;
  int nblk = 1;
  for (int a = 0; a < 3; ++a) A.tiles[a] = a < D ? tiles : 1;
  for (int a = 0; a < D; ++a) nblk *= tiles;
  A.ntiles = nblk;
  const size_t smem = mg::sweep_smem_bytes<R, D, TC>(A.varphi);
  auto kern = mg::sweep_kernel<R, D, TC, kThreads>;
  kern<<<nblk, kThreads, smem, s>>>(A);
  return cudaGetLastError();
}

template <typename R, int D>
cudaError_t launch_sweep(cudaStream_t s, mg::SweepArgs<R>& A) {
  if constexpr (D == 2) {
    if (tc2_for(A.n) == 2) return launch_sweep_tc<R, 2, 2>(s, A);
    return launch_sweep_tc<R, 2, kTC2>(s, A);
  } else {
    return launch_sweep_tc<R, D, kTC3>(s, A);
  }
}

template <int TC, int NTHR, typename R>
cudaError_t launch_sweep2(cudaStream_t s, mg::Sweep2Args<R>& A) {
  const int nc = A.n / 3;
  const int tiles = (nc + 1 + TC - 1) / TC;
  A.tiles_x = tiles;
  constexpr size_t smem = mg::Tile2<TC, R>::smem_bytes;
  auto kern = mg::sweep2_kernel<TC, NTHR, R>;
  kern<<<tiles * tiles, NTHR, smem, s>>>(A);
  return cudaGetLastError();
}

// Shared-memory opt-in of the sweep kernels; done once per device before any
// launch or stream capture.
cudaError_t configure_kernels() {
  static std::mutex mu;
  static unsigned long long done = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (dev < 64 && (done >> dev) & 1ull) return cudaSuccess;
  auto set = [&](const void* f, size_t bytes) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  };
  set((const void*)mg::sweep_kernel<double, 2, kTC2, kThreads>, mg::sweep_smem_bytes<double, 2, kTC2>(1));
  set((const void*)mg::sweep_kernel<double, 3, kTC3, kThreads>, mg::sweep_smem_bytes<double, 3, kTC3>(1));
  set((const void*)mg::sweep_kernel<float, 2, kTC2, kThreads>, mg::sweep_smem_bytes<float, 2, kTC2>(1));
  set((const void*)mg::sweep_kernel<float, 3, kTC3, kThreads>, mg::sweep_smem_bytes<float, 3, kTC3>(1));
  set((const void*)mg::sweep2_kernel<12, 256>, mg::Tile2<12>::smem_bytes);
  set((const void*)mg::sweep2_kernel<4, 128>, mg::Tile2<4>::smem_bytes);
  set((const void*)mg::sweep2_kernel<15, 256>, mg::Tile2<15>::smem_bytes);
  set((const void*)mg::sweep2p_kernel<8, 256>, mg::Tile2<8>::smem_bytes);
  set((const void*)mg::sweep2p_kernel<8, 256, float>, mg::Tile2<8, float>::smem_bytes);
  set((const void*)mg::sweep2_kernel<4, 128, float>, mg::Tile2<4, float>::smem_bytes);
  set((const void*)mg::chain2_kernel<256, float>, mg::Tile2<4, float>::smem_bytes);
  set((const void*)mg::sweep3_kernel<double, 6, 512>, mg::Tile3<double, 6>::smem_bytes);
  set((const void*)mg::sweep3_kernel<double, 4, 256>, mg::Tile3<double, 4>::smem_bytes);
  set((const void*)mg::sweep3_kernel<float, 7, 512>, mg::Tile3<float, 7>::smem_bytes);
  set((const void*)mg::sweep3_kernel<float, 4, 256>, mg::Tile3<float, 4>::smem_bytes);
  set((const void*)mg::sweep3s_kernel<2, true, false, false>, sizeof(mg::Sweep3sShared) + 128);
  set((const void*)mg::sweep3s_kernel<2, true, true, false>, sizeof(mg::Sweep3sShared) + 128);
  set((const void*)mg::sweep3s_kernel<2, true, false, true>, sizeof(mg::Sweep3sShared) + 128);
  set((const void*)mg::sweep3s_kernel<2, false, false, false>, sizeof(mg::Sweep3sShared) + 128);
  set((const void*)mg::sweep3s_kernel<2, false, true, false>, sizeof(mg::Sweep3sShared) + 128);
  set((const void*)mg::sweep3s_kernel<2, false, false, true>, sizeof(mg::Sweep3sShared) + 128);
  set((const void*)mg::sweep3sd_kernel, sizeof(mg::Sweep3sdShared));
  set((const void*)mg::defect3_kernel<float>, sizeof(mg::Defect3Shared<float>));
  set((const void*)mg::defect3_kernel<double>, sizeof(mg::Defect3Shared<double>));
  set((const void*)mg::chain2_kernel<256>, mg::Tile2<4>::smem_bytes);
  static_assert(mg::Tile2<2>::smem_bytes <= mg::Tile2<4>::smem_bytes, "chain smem");
  if (e == cudaSuccess && dev < 64) done |= 1ull << dev;
  return e;
}

// 2D levels with a constant shift: the Galerkin-row sweep (level 1 has
// no coarser level and uses the same kernel with has_coarse = 0).
template <typename R>
cudaError_t sweep2(mg_ctx* c, Hier<R>& H, int l, bool fine, int hb, int hier, const cd& om) {
  auto& V = H.lev[l];
  mg::Sweep2Args<R> A;
  std::memset(&A, 0, sizeof(A));
  A.n = V.n;
  A.fine = fine ? 1 : 0;
  A.has_coarse = l > 1 ? 1 : 0;
  A.hb = hb;
  A.hier = hier;
  A.realrow = V.realrow;
  A.u = fine ? V.u[H.cur] : V.u[0];
  A.c = (fine && l > 1) ? H.lev[l - 1].corr : nullptr;
  A.b = V.b;
  A.out = fine ? V.u[1 - H.cur] : V.t;
  if (l > 1) {
    A.b_coarse = H.lev[l - 1].b;
    A.u_coarse = H.lev[l - 1].u[0];
    A.gtyp = V.gtyp;
    A.gcoef = V.gcoef;
  }
  A.typ = V.typ;
  A.coef = V.coefH;
  A.realjac = 0;
  for (size_t t = 0; t < V.diag.size() && t < 16; ++t) {
    const cd q = om / V.diag[t];
    A.omd[t] = cplx<R>{(R)q.real(), (R)q.imag()};
    if (q.imag() == 0.0) A.realjac |= 1u << t;
  }
  A.partial = H.partial;
  A.ticket = H.ticket;
  A.norm2 = H.norm2;
  const int nc = V.n / 3;
  if (nc + 1 >= 200 && V.order8 != nullptr) {
    const int tl = (nc + 8) / 8;
    A.tiles_x = tl;
    A.ntiles = tl * tl;
    // queue head chain_ctr[32] and exit counter [33] are zero between launches
    const int grid = std::min(A.ntiles, 152 * std::max(1, c->fine_bpsm));
    mg::sweep2p_kernel<8, 256, R><<<grid, 256, mg::Tile2<8, R>::smem_bytes, c->stream>>>(
        A, V.order8, c->chain_ctr + 32, c->tracing ? c->trace : nullptr, fine ? V.tflags : nullptr,
        c->chain_ctr + 34);
    return cudaGetLastError();
  }
  A.ntiles = ((nc + 4) / 4) * ((nc + 4) / 4);
  return launch_sweep2<4, 128, R>(c->stream, A);
}

// Arguments of a coarse level's sweep tile in the persistent chain (TC = 4).
template <typename R>
mg::Sweep2Args<R> sweep2_args(Hier<R>& H, int l, int hb, int hier, const cd& om, int TC) {
  auto& V = H.lev[l];
  mg::Sweep2Args<R> A;
  std::memset(&A, 0, sizeof(A));
  A.n = V.n;
  A.fine = 0;
  A.has_coarse = l > 1 ? 1 : 0;
  A.hb = hb;
  A.hier = hier;
  A.realrow = V.realrow;
  A.u = V.u[0];
  A.b = V.b;
  A.out = V.t;
  if (l > 1) {
    A.b_coarse = H.lev[l - 1].b;
    A.u_coarse = H.lev[l - 1].u[0];
    A.gtyp = V.gtyp;
    A.gcoef = V.gcoef;
  }
  A.typ = V.typ;
  A.coef = V.coefH;
  for (size_t t = 0; t < V.diag.size() && t < 16; ++t) {
    const cd q = om / V.diag[t];
    A.omd[t] = cplx<R>{(R)q.real(), (R)q.imag()};
    if (q.imag() == 0.0) A.realjac |= 1u << t;
  }
  const int nc = V.n / 3;
  A.tiles_x = (nc + TC) / TC;
  A.ntiles = A.tiles_x * A.tiles_x;
  return A;
}

// Item list of the coarse chain of one cycle on levels 1..s-1 of a 2D FP64
// hierarchy: sweeps of levels s-1 .. 1, then prolongations of levels 2 .. s-1.
template <typename R>
int build_chain2(mg_ctx* c, Hier<R>& H, int s, int hb, int hier, const cplx<double>* omega,
                 const std::vector<double>& key, typename Hier<R>::ChainPlan** out) {
  for (auto& cp : H.chains)
    if (cp.key == key) { *out = &cp; return MG_OK; }
  std::vector<mg::ChainItem> items;
  std::vector<mg::Sweep2Args<R>> s2;
  std::vector<mg::ProlongArgs<R>> pr;
  unsigned need = 0;
  for (int l = s - 1; l >= 1; --l) {
    const cplx<double> w = omega[l - 1 + (H.L - s)];
    // small levels take 2-coarse-cell tiles, and 1-cell tiles once those
    // still fit one per SM, so that a stage spreads over many SMs (its
    // latency is set by one tile's FP64 work)
    const int ncv = H.lev[l].n / 3 + 1;
    const int TC = ncv >= 60 ? 4 : (ncv * ncv <= 152 ? 1 : 2);
    s2.push_back(sweep2_args(H, l, hb, hier, cd(w.x, w.y), TC));
    const int nt = s2.back().ntiles;
    const int kind = TC == 4 ? mg::kItemSweep2 : (TC == 2 ? mg::kItemSweep2s : mg::kItemSweep2t);
    for (int t = 0; t < nt; ++t) items.push_back({kind, 0, (int)s2.size() - 1, t, need});
    need += nt;
  }
  // corr_{s-1} = sum_l P^{s-1-l} t_l in two stages: corr_{s-2} directly from
  // levels 1..s-2, then corr_{s-1} = t_{s-1} + P corr_{s-2}
  std::vector<mg::CorrArgs<R>> co;
  const int top = s - 1;
  if (top >= mg::kMaxChainLevels) return fail(c, MG_ERR_INVALID, "hierarchy too deep for the chain");
  auto add_corr = [&](int tgt, int lo, const cplx<R>* base) {
    mg::CorrArgs<R> ca;
    std::memset(&ca, 0, sizeof(ca));
    ca.s = tgt;
    ca.lo = lo;
    for (int l = lo; l <= tgt; ++l) ca.t[l] = H.lev[l].t;
    ca.base = base;
    ca.out = H.lev[tgt].corr;
    // about two items per SM, 64 .. 256 vertices each (one per thread at most)
    ca.chunk = (int)std::min<size_t>(256, std::max<size_t>(64, (H.lev[tgt].nv / 304 + 63) / 64 * 64));
    co.push_back(ca);
    const int nch = (int)((H.lev[tgt].nv + ca.chunk - 1) / ca.chunk);
    for (int t = 0; t < nch; ++t) items.push_back({mg::kItemCorr2, 0, (int)co.size() - 1, t, need});
    need += nch;
  };
  if (top >= 3) {
    add_corr(top - 1, 1, nullptr);
    add_corr(top, top, H.lev[top - 1].corr);
  } else if (top == 2) {
    add_corr(2, 1, nullptr);
  }
  typename Hier<R>::ChainPlan cp;
  cp.key = key;
  cp.nitems = (int)items.size();
  MG_CUDA(c, cudaMalloc(&cp.items, std::max<size_t>(1, items.size()) * sizeof(mg::ChainItem)));
  MG_CUDA(c, cudaMalloc(&cp.s2, std::max<size_t>(1, s2.size()) * sizeof(mg::Sweep2Args<R>)));
  MG_CUDA(c, cudaMalloc(&cp.pr, std::max<size_t>(1, pr.size()) * sizeof(mg::ProlongArgs<R>)));
  MG_CUDA(c, cudaMalloc(&cp.co, std::max<size_t>(1, co.size()) * sizeof(mg::CorrArgs<R>)));
  if (!co.empty())
    MG_CUDA(c, cudaMemcpy(cp.co, co.data(), co.size() * sizeof(mg::CorrArgs<R>), cudaMemcpyHostToDevice));
  if (!items.empty())
    MG_CUDA(c, cudaMemcpy(cp.items, items.data(), items.size() * sizeof(mg::ChainItem), cudaMemcpyHostToDevice));
  if (!s2.empty())
    MG_CUDA(c, cudaMemcpy(cp.s2, s2.data(), s2.size() * sizeof(mg::Sweep2Args<R>), cudaMemcpyHostToDevice));
  if (!pr.empty())
    MG_CUDA(c, cudaMemcpy(cp.pr, pr.data(), pr.size() * sizeof(mg::ProlongArgs<R>), cudaMemcpyHostToDevice));
  cp.grid = std::max(1, std::min(cp.nitems, 152 * std::min(MG_CHAIN_BPSM, std::max(1, c->chain_bpsm))));
  if (H.chains.size() >= 32) {
    // cached cycle graphs may launch the plan about to be freed
    drop_graphs(H);
    cudaFree(H.chains.front().items);
    cudaFree(H.chains.front().s2);
    cudaFree(H.chains.front().pr);
    cudaFree(H.chains.front().co);
    H.chains.erase(H.chains.begin());
  }
  H.chains.push_back(cp);
  *out = &H.chains.back();
  return MG_OK;
}

template <typename R>
cudaError_t launch_chain2(mg_ctx* c, Hier<R>& H, int s, const typename Hier<R>::ChainPlan& cp) {
  mg::ChainArgs<R> A;
  // the first stage waits for single fine tiles when the fine sweep was the
  // persistent LPT sweep that publishes them (levels s-1 in 4-cell tiles)
  auto& VF = H.lev[s];
  const int ncf = VF.n / 3;
  // (complex64 2D levels of this size take the warp-strip sweep instead)
  const bool tiled = std::is_same<R, double>::value && VF.tflags != nullptr && ncf + 1 >= 200 &&
                     VF.order8 != nullptr && (H.lev[s - 1].n / 3 + 1) >= 60;
  A.fine_flags = tiled ? VF.tflags : nullptr;
  A.gen = c->chain_ctr + 34;
  A.fine_tiles_x = (ncf + 8) / 8;
  A.first_tiles_x = (H.lev[s - 1].n / 3 + 4) / 4;
  A.items = cp.items;
  A.nitems = cp.nitems;
  A.s2 = cp.s2;
  A.pr = cp.pr;
  A.co = cp.co;
  A.head = c->chain_ctr;  // [0] head, [1] completions, [2] exits: zero between launches
  A.done = c->chain_ctr + 1;
  A.exitc = c->chain_ctr + 2;
  A.err = c->dev_err;
  A.spin_limit = c->spin_limit;
  A.trace = c->tracing ? c->trace + 4 * kTraceFine : nullptr;
  A.stall = c->debug_stall ? c->chain_ctr + 48 : nullptr;  // stays zero
  // programmatic dependent launch: the chain's blocks are scheduled while the
  // fine sweep drains and wait in the kernel until its writes are visible
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cp.grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = mg::Tile2<4, R>::smem_bytes;
  cfg.stream = c->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, mg::chain2_kernel<256, R>, A);
}

// 3D levels with a constant shift: the z-marching Galerkin-row sweep.
template <typename R, int TC, int NTHR>
cudaError_t launch_sweep3(cudaStream_t s, mg::Sweep3Args<R>& A) {
  const int nc = A.n / 3;
  const int tl = (nc + 1 + TC - 1) / TC;
  A.tiles_x = tl;
  A.ntiles_xy = tl * tl;
  // enough z-chunks for about four resident blocks per SM
  const int nz = std::max(1, std::min(nc + 1, (2 * 152 + A.ntiles_xy - 1) / A.ntiles_xy));
  A.zchunk = (nc + 1 + nz - 1) / nz;
  A.nzchunks = (nc + 1 + A.zchunk - 1) / A.zchunk;
  A.ntiles = A.ntiles_xy * A.nzchunks;
  mg::sweep3_kernel<R, TC, NTHR><<<A.ntiles, NTHR, mg::Tile3<R, TC>::smem_bytes, s>>>(A);
  return cudaGetLastError();
}

// 1D rows by axis class (left / right cell rotated): mass (hl/6, (hl+hr)/3,
// hr/6), stiffness (-1/hl, 1/hl + 1/hr, -1/hr), stiffness - phi mass
template <typename T>
void axis_rows(const mg_ctx* c, int n, T row[4][9]) {
  const double phi = c->k2[0];
  const Widths wd = widths(c, n);
  for (int t = 0; t < 4; ++t) {
    const cd hl = (t & 1) ? wd.rot : wd.in, hr = (t & 2) ? wd.rot : wd.in;
    const cd m[3] = {hl / 6.0, (hl + hr) / 3.0, hr / 6.0};
    const cd k[3] = {-1.0 / hl, 1.0 / hl + 1.0 / hr, -1.0 / hr};
    for (int j = 0; j < 3; ++j) {
      const cd kp = k[j] - phi * m[j];
      row[t][j] = T{(decltype(row[0][0].x))m[j].real(), (decltype(row[0][0].x))m[j].imag()};
      row[t][3 + j] = T{(decltype(row[0][0].x))k[j].real(), (decltype(row[0][0].x))k[j].imag()};
      row[t][6 + j] = T{(decltype(row[0][0].x))kp.real(), (decltype(row[0][0].x))kp.imag()};
    }
  }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); null when the driver does not provide it.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Tensor map of a 3D level array ((n+1)^3 complex values of T, x fastest) as
// 2(n+1) x (n+1) x (n+1) reals, with boxes of bw complex columns, 32 rows and
// one plane; elements outside the array read as zero.  Row and plane strides
// are multiples of 16 bytes because n + 1 is even (n = 3^l).
template <typename T>
bool plane_map(CUtensorMap* m, const void* base, int n, int bw) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (enc == nullptr) return false;
  const cuuint64_t N = (cuuint64_t)n + 1;
  const cuuint64_t dims[3] = {2 * N, N, N};
  const cuuint64_t strides[2] = {2 * N * sizeof(T), 2 * N * N * sizeof(T)};
  const cuuint32_t box[3] = {(cuuint32_t)(2 * bw), 32u, 1u};
  const cuuint32_t es[3] = {1u, 1u, 1u};
  const CUtensorMapDataType ty = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  return enc(m, ty, 3, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Large complex64 3D levels: the separable z-marching sweep, one block per SM
// over ranges of (tile, coarse plane) units of equal cost.
cudaError_t launch_sweep3s(mg_ctx* c, Hier<float>& H, int l, bool fine, int hb, int hier, const cd& om) {
  auto& V = H.lev[l];
  mg::Sweep3sArgs A;
  std::memset(&A, 0, sizeof(A));
  A.n = V.n;
  A.fine = fine ? 1 : 0;
  A.has_coarse = 1;
  A.hb = hb;
  A.hier = hier;
  const int nc = V.n / 3;
  A.tiles_x = (nc + 8) / 9;
  A.nunits = (long long)A.tiles_x * A.tiles_x * nc;
  A.u = fine ? V.u[H.cur] : V.u[0];
  A.c = fine ? H.lev[l - 1].corr : nullptr;
  A.b = V.b;
  A.out = fine ? V.u[1 - H.cur] : V.t;
  A.b_coarse = H.lev[l - 1].b;
  A.u_coarse = H.lev[l - 1].u[0];
  A.typ = V.typ;
  A.gtyp = V.gtyp;
  A.gcoef = V.gcoef;
  axis_rows(c, V.n, A.row);
  for (size_t t = 0; t < V.diag.size() && t < 64; ++t) {
    const cd q = om / V.diag[t];
    A.omd[t] = cplx<float>{(float)q.real(), (float)q.imag()};
  }
  A.partial = H.partial;
  A.ticket = H.ticket;
  A.norm2 = fine ? H.norm2 : nullptr;
  A.upref = V.s3pref;
  A.usplit = fine ? V.s3split_f : V.s3split_c;
  A.spin_limit = c->spin_limit;
  A.err = c->dev_err;
  // the u and b planes come in by TMA: 34-column boxes of 32 rows
  CUtensorMap tmU, tmB;
  if (!plane_map<float>(&tmU, A.u, V.n, mg::kS3BoxW) || !plane_map<float>(&tmB, A.b, V.n, mg::kS3BoxW))
    return cudaErrorNotSupported;
  // fine levels: about four coarse planes per block at least (a range's first
  // coarse step is overhead); coarse levels: every SM that has a unit; the
  // ranges were balanced for this grid at set-up
  const int grid = fine ? V.s3grid_f : V.s3grid_c;
  // two box rows per thread (four: 255 registers, 8 warps per SM, 17% slower);
  // one instantiation per level role and variant
  const size_t sm = sizeof(mg::Sweep3sShared) + 128;
  const bool bpx = hier && !hb;
  if (fine) {
    if (hb) mg::sweep3s_kernel<2, true, true, false><<<grid, 512, sm, c->stream>>>(A, tmU, tmB);
    else if (bpx) mg::sweep3s_kernel<2, true, false, true><<<grid, 512, sm, c->stream>>>(A, tmU, tmB);
    else mg::sweep3s_kernel<2, true, false, false><<<grid, 512, sm, c->stream>>>(A, tmU, tmB);
  } else {
    if (hb) mg::sweep3s_kernel<2, false, true, false><<<grid, 512, sm, c->stream>>>(A, tmU, tmB);
    else if (bpx) mg::sweep3s_kernel<2, false, false, true><<<grid, 512, sm, c->stream>>>(A, tmU, tmB);
    else mg::sweep3s_kernel<2, false, false, false><<<grid, 512, sm, c->stream>>>(A, tmU, tmB);
  }
  return cudaGetLastError();
}

// Large complex128 3D levels: the separable z-marching sweep in FP64, one
// block per SM over equal ranges of (tile, coarse plane) units.
cudaError_t launch_sweep3sd(mg_ctx* c, Hier<double>& H, int l, bool fine, int hb, int hier, const cd& om) {
  auto& V = H.lev[l];
  mg::Sweep3sdArgs A;
  std::memset(&A, 0, sizeof(A));
  A.n = V.n;
  A.fine = fine ? 1 : 0;
  A.has_coarse = 1;
  A.hb = hb;
  A.hier = hier;
  const int nc = V.n / 3;
  A.tiles_x = (nc + 8) / 9;
  A.nunits = (long long)A.tiles_x * A.tiles_x * nc;
  A.u = fine ? V.u[H.cur] : V.u[0];
  A.c = fine ? H.lev[l - 1].corr : nullptr;
  A.b = V.b;
  A.out = fine ? V.u[1 - H.cur] : V.t;
  A.b_coarse = H.lev[l - 1].b;
  A.u_coarse = H.lev[l - 1].u[0];
  A.typ = V.typ;
  A.gtyp = V.gtyp;
  A.gcoef = V.gcoef;
  A.greal = V.greal;
  A.upref = V.s3pref;
  A.usplit = fine ? V.s3split_f : V.s3split_c;
  A.idu = (hier && !hb) ? V.idu : nullptr;
  axis_rows(c, V.n, A.row);
  for (size_t t = 0; t < V.diag.size() && t < 64; ++t) {
    const cd q = om / V.diag[t];
    A.omd[t] = cplx<double>{q.real(), q.imag()};
  }
  A.partial = H.partial;
  A.ticket = H.ticket;
  A.norm2 = fine ? H.norm2 : nullptr;
  // at least two coarse planes per block: a range starts with two fine
  // planes of overhead (the restriction's lower halo); the ranges were
  // balanced for this grid at set-up
  const int grid = fine ? V.s3grid_f : V.s3grid_c;
  mg::sweep3sd_kernel<<<(int)grid, 512, sizeof(mg::Sweep3sdShared), c->stream>>>(A);
  return cudaGetLastError();
}

// Large complex64 2D levels: the warp-strip sweep.
cudaError_t launch_sweep2w(mg_ctx* c, Hier<float>& H, int l, bool fine, int hb, int hier, const cd& om) {
  auto& V = H.lev[l];
  mg::Sweep2wArgs A;
  std::memset(&A, 0, sizeof(A));
  A.n = V.n;
  A.fine = fine ? 1 : 0;
  A.has_coarse = 1;
  A.hb = hb;
  A.hier = hier;
  const int nc = V.n / 3;
  // two columns per lane (18-cell strips) where their grid still fills four
  // waves of warps at six coarse rows each (2D depth 8: 0.508 -> 0.445 ms); a
  // smaller level keeps one column per lane, whose twice as many warps hide
  // more of the level's latency (depth 7: 0.069 ms against 0.073 ms)
  const int s18 = (nc + 17) / 18;
  A.scells = (long long)s18 * nc / 6 >= 4LL * 152 * MG_S2W_MINB * 8 ? 18 : 9;
  A.strips = (nc + A.scells - 1) / A.scells;
  A.nunits = A.strips * nc;
  A.u = fine ? V.u[H.cur] : V.u[0];
  A.c = fine ? H.lev[l - 1].corr : nullptr;
  A.b = V.b;
  A.out = fine ? V.u[1 - H.cur] : V.t;
  A.b_coarse = H.lev[l - 1].b;
  A.u_coarse = H.lev[l - 1].u[0];
  A.typ = V.typ;
  A.gtyp = V.gtyp;
  A.gcoef = V.gcoef;
  axis_rows(c, V.n, A.row);
  for (size_t t = 0; t < V.diag.size() && t < 16; ++t) {
    const cd q = om / V.diag[t];
    A.omd[t] = cplx<float>{(float)q.real(), (float)q.imag()};
  }
  A.partial = H.partial;
  A.ticket = H.ticket;
  A.norm2 = fine ? H.norm2 : nullptr;
  // about six coarse rows per warp (three where that gives less than one
  // wave: more warps to hide a small level's latency), one wave of resident
  // blocks at most
  const int upw = A.nunits / 6 < 152 * MG_S2W_MINB * 8 ? 3 : 6;
  const int warps = std::max(1, std::min(A.nunits / upw, 152 * MG_S2W_MINB * 8));
  const int grid = (warps + 7) / 8;
  mg::sweep2w_kernel<<<grid, mg::kS2wThreads, 0, c->stream>>>(A);
  return cudaGetLastError();
}

template <typename R>
cudaError_t sweep3(mg_ctx* c, Hier<R>& H, int l, bool fine, int hb, int hier, const cd& om) {
  if (l > 1 && H.lev[l].g3ok && interior_real(c)) {
    // complex64: the separable sweep from 27 cells per axis; complex128: from
    // 27 on the finest level, from 81 on coarse levels (a 27-cell level has
    // nine units of the separable layout, too few for the FP64 pipes of the
    // GPU).  Within a cycle, coarse levels of up to 81 cells per axis run the
    // point kernel instead (sweep() dispatches them before this function).
    if constexpr (std::is_same<R, float>::value) {
      if (H.lev[l].n >= 27) return launch_sweep3s(c, H, l, fine, hb, hier, om);
    } else {
      if (H.lev[l].n >= (fine ? 27 : 81)) return launch_sweep3sd(c, H, l, fine, hb, hier, om);
    }
  }
  auto& V = H.lev[l];
  mg::Sweep3Args<R> A;
  std::memset(&A, 0, sizeof(A));
  A.n = V.n;
  A.fine = fine ? 1 : 0;
  A.first = 0;
  A.has_coarse = l > 1 ? 1 : 0;
  A.hb = hb;
  A.hier = hier;
  A.realrow = V.realrow3;
  A.u = fine ? V.u[H.cur] : V.u[0];
  A.c = (fine && l > 1) ? H.lev[l - 1].corr : nullptr;
  A.b = V.b;
  A.out = fine ? V.u[1 - H.cur] : V.t;
  if (l > 1) {
    A.b_coarse = H.lev[l - 1].b;
    A.u_coarse = H.lev[l - 1].u[0];
    A.gtyp = V.gtyp;
    A.gcoef = V.gcoef;
  }
  A.typ = V.typ;
  A.coef = V.coefH;
  A.realjac = 0;
  for (size_t t = 0; t < V.diag.size() && t < 64; ++t) {
    const cd q = om / V.diag[t];
    A.omd[t] = cplx<R>{(R)q.real(), (R)q.imag()};
    if (q.imag() == 0.0) A.realjac |= 1ull << t;
  }
  A.partial = H.partial;
  A.ticket = H.ticket;
  A.norm2 = fine ? H.norm2 : nullptr;
  const int nc = V.n / 3;
  if constexpr (std::is_same<R, double>::value) {
    if (nc + 1 >= 25) return launch_sweep3<double, 6, 512>(c->stream, A);
    return launch_sweep3<double, 4, 256>(c->stream, A);
  } else {
    if (nc + 1 >= 25) return launch_sweep3<float, 7, 512>(c->stream, A);
    return launch_sweep3<float, 4, 256>(c->stream, A);
  }
}

// Level l < s of a cycle on levels 1..s runs the point kernel (mg_coarse3.cuh):
// 3D, constant shift, at most kPoint3MaxN cells per axis, and every coarser
// level a point level too (a point level leaves its coarse right-hand side to
// the next coarser level's launch, which must therefore be one).
template <typename R>
bool point3_level(const mg_ctx* c, const Hier<R>& H, int l, int s) {
  if (c->d != 3 || H.varphi || l < 1 || l >= s || H.lev[l].n > kPoint3MaxN) return false;
  for (int k = 2; k <= l; ++k) {
    const auto& V = H.lev[k];
    if (!V.g3ok || V.r == nullptr || V.idu == nullptr) return false;
  }
  return true;
}

// A coarse level of the point kernel: its right-hand side is formed here from
// the finer level's stored residual when that level was a point level too.
template <typename R>
cudaError_t launch_coarse3(mg_ctx* c, Hier<R>& H, int l, int s, int hb, int hier, const cd& om) {
  auto& V = H.lev[l];
  mg::Coarse3Args<R> A;
  std::memset(&A, 0, sizeof(A));
  A.n = V.n;
  A.fused = point3_level(c, H, l + 1, s) ? 1 : 0;
  A.has_coarse = l > 1 ? 1 : 0;
  A.hb = hb;
  A.realrow = V.realrow3;
  A.u = V.u[0];
  A.b = V.b;
  if (A.fused) {
    const auto& F = H.lev[l + 1];
    A.rf = F.r;
    A.gtyp = F.gtyp;
    A.gcoef = F.gcoef;
    A.greal = F.greal;
  }
  A.typ = V.typ;
  A.coef = V.coefH;
  for (size_t t = 0; t < V.diag.size() && t < 64; ++t) {
    const cd q = om / V.diag[t];
    A.omd[t] = cplx<R>{(R)q.real(), (R)q.imag()};
  }
  A.r = V.r;
  A.t = V.t;
  A.idu = (l > 1 && hier && !hb) ? V.idu : nullptr;
  A.u_coarse = l > 1 ? H.lev[l - 1].u[0] : nullptr;
  // lanes per vertex: one where the level fills the GPU, more on the small,
  // FP64-latency-bound levels (blocks of 128 threads spread them over the SMs)
  const int lpv = V.nv > 200000 ? 1 : (V.nv > 8000 ? 8 : 32);
  const long long blocks = std::min<long long>(((long long)V.nv * lpv + 127) / 128, 152 * 16);
  if (lpv == 1) mg::coarse3_kernel<R, 1><<<(int)blocks, 128, 0, c->stream>>>(A);
  else if (lpv == 8) mg::coarse3_kernel<R, 8><<<(int)blocks, 128, 0, c->stream>>>(A);
  else mg::coarse3_kernel<R, 32><<<(int)blocks, 128, 0, c->stream>>>(A);
  return cudaGetLastError();
}

template <typename R>
cudaError_t sweep(mg_ctx* c, Hier<R>& H, int l, bool fine, int s_active, int hb, int hier,
                  const cplx<double>* omega) {
  auto& V = H.lev[l];
  ++c->launches;
  if (c->d == 3 && !H.varphi && (l == 1 || V.g3ok)) {
    const cplx<double> w = omega[l - 1 + (H.L - s_active)];
    if (!fine && point3_level(c, H, l, s_active)) return launch_coarse3(c, H, l, s_active, hb, hier, cd(w.x, w.y));
    return sweep3(c, H, l, fine, hb, hier, cd(w.x, w.y));
  }
  if constexpr (std::is_same<R, float>::value) {
    if (c->d == 2 && !H.varphi && l > 1 && V.n >= 27 && V.gok && interior_real(c)) {
      const cplx<double> w = omega[l - 1 + (H.L - s_active)];
      return launch_sweep2w(c, H, l, fine, hb, hier, cd(w.x, w.y));
    }
  }
  if (c->d == 2 && !H.varphi && (l == 1 || V.gok)) {
    const cplx<double> w = omega[l - 1 + (H.L - s_active)];
    return sweep2<R>(c, H, l, fine, hb, hier, cd(w.x, w.y));
  }
  mg::SweepArgs<R> A;
  std::memset(&A, 0, sizeof(A));
  A.n = V.n;
  A.fine = fine ? 1 : 0;
  A.has_coarse = l > 1 ? 1 : 0;
  A.hb = hb;
  A.hier = hier;
  A.varphi = H.varphi ? 1 : 0;
  A.u = fine ? V.u[H.cur] : V.u[0];
  A.c = (fine && l > 1) ? H.lev[l - 1].corr : nullptr;
  A.b = V.b;
  A.out = fine ? V.u[1 - H.cur] : V.t;
  if (l > 1) {
    A.b_coarse = H.lev[l - 1].b;
    A.u_coarse = H.lev[l - 1].u[0];
  }
  A.typ = V.typ;
  A.coef = V.coefH;
  A.phic = V.phic;
  A.hcell = V.hcell;
  // the factor of level l in stage s_active is the one of level l + (L - s)
  const cd om(omega[l - 1 + (H.L - s_active)].x, omega[l - 1 + (H.L - s_active)].y);
  A.omega = cplx<R>{(R)om.real(), (R)om.imag()};
  if (!H.varphi) {
    for (size_t t = 0; t < V.diag.size(); ++t) {
      cd q = om / V.diag[t];
      A.omd[t] = cplx<R>{(R)q.real(), (R)q.imag()};
    }
  }
  A.partial = H.partial;
  A.ticket = H.ticket;
  A.norm2 = H.norm2;
  return c->d == 2 ? launch_sweep<R, 2>(c->stream, A) : launch_sweep<R, 3>(c->stream, A);
}

int grid_for(size_t nv) {
  size_t b = (nv + kThreads - 1) / kThreads;
  return (int)std::min<size_t>(std::max<size_t>(b, 1), 152 * 16);
}

// Device address of a page-locked host buffer (cudaHostAlloc, or registered
// with cudaHostRegister), or null for pageable memory.  Kernels read and
// write such a buffer directly over the host link (mg_io.cuh).
template <typename T>
T* pinned_view(T* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, (const void*)p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || a.devicePointer == nullptr) return nullptr;
  return reinterpret_cast<T*>(a.devicePointer);
}

// Level l of a cycle on levels 1..s runs the complex128 separable 3D sweep
// with the BPX transfer: it then stores t_l = du_l and I du_l, and the
// correction stage forms du_l - P I du_l (the same test as the dispatch in
// sweep3/sweep).
template <typename R>
bool sd_bpx_level(const mg_ctx* c, const Hier<R>& H, int l, int s, int hb, int hier) {
  return std::is_same<R, double>::value && c->d == 3 && !H.varphi && l > 1 && H.lev[l].g3ok &&
         interior_real(c) && hier && !hb && H.lev[l].idu != nullptr && H.lev[l].n >= (l == s ? 27 : 81);
}

// corr_l = T_l du_l + P corr_{l-1}.  Levels whose sweep stored t_l = du_l
// and I du_l (BPX on the separable complex128 sweep) use
// corr_l = du_l + P (corr_{l-1} - I du_l); when the finest level s did so,
// corr_{s-1} (the pending correction) also takes - I du_s, so that
// U + P corr_{s-1} = u + du_s - P I du_s + P corr_{s-1}.
template <typename R>
cudaError_t prolong(mg_ctx* c, Hier<R>& H, int l, int s, int hb, int hier) {
  auto& V = H.lev[l];
  const bool stored_du = point3_level(c, H, l, s) ? (l > 1 && hier && !hb) : sd_bpx_level(c, H, l, s, hb, hier);
  const cplx<R>* sub_c = stored_du ? V.idu : nullptr;
  const cplx<R>* sub_f = (l == s - 1 && sd_bpx_level(c, H, s, s, hb, hier)) ? H.lev[s].idu : nullptr;
  ++c->launches;
  if (c->d == 2)
    mg::prolong_add_kernel<R, 2><<<grid_for(V.nv), kThreads, 0, c->stream>>>(
        V.n, V.t, H.lev[l - 1].corr, V.corr, sub_c, sub_f);
  else
    mg::prolong3_kernel<R><<<(int)ipow((V.n + 1 + 8) / 9, 3), 256, 0, c->stream>>>(
        V.n, V.t, H.lev[l - 1].corr, V.corr, sub_c, sub_f);
  return cudaGetLastError();
}

// Kernels of one cycle on levels 1..s (s = active finest level), enqueued on
// c->stream: the fine sweep (part 0) or the coarse chain (part 1).
template <typename R>
cudaError_t enqueue_cycle_part(mg_ctx* c, Hier<R>& H, int s, int hb, int hier,
                               const cplx<double>* omega, int part, int* nkern) {
  cudaError_t e = cudaSuccess;
  *nkern = 0;
  if (part == 2) {
    int k0 = 0, k1 = 0;
    e = enqueue_cycle_part(c, H, s, hb, hier, omega, 0, &k0);
    if (e == cudaSuccess && s > 1) e = enqueue_cycle_part(c, H, s, hb, hier, omega, 1, &k1);
    *nkern = k0 + k1;
    return e;
  }
  if (part == 0) {
    e = sweep(c, H, s, true, s, hb, hier, omega);
    *nkern = 1;
    return e;
  }
  {
    bool chain_ok = c->d == 2 && !H.varphi;
    for (int l = 2; l < s && chain_ok; ++l) chain_ok = H.lev[l].gok;
    if (chain_ok) {
      std::vector<double> key = {(double)s, (double)hb, (double)hier};
      for (int l = 0; l < H.L; ++l) {
        key.push_back(omega[l].x);
        key.push_back(omega[l].y);
      }
      typename Hier<R>::ChainPlan* cp = nullptr;
      if (build_chain2<R>(c, H, s, hb, hier, omega, key, &cp) != MG_OK) return cudaErrorUnknown;
      *nkern = 1;
      ++c->launches;
      return launch_chain2<R>(c, H, s, *cp);
    }
  }
  for (int l = s - 1; l >= 1 && e == cudaSuccess; --l, ++*nkern) e = sweep(c, H, l, false, s, hb, hier, omega);
  for (int l = 2; l <= s - 1 && e == cudaSuccess; ++l, ++*nkern) e = prolong(c, H, l, s, hb, hier);
  return e;
}

// Captures one part of the cycle as a graph on the private capture stream.
template <typename R>
cudaError_t capture_part(mg_ctx* c, Hier<R>& H, int s, int hb, int hier, const cplx<double>* omega,
                         int part, cudaGraph_t* graph, int* nkern) {
  *graph = nullptr;
  cudaStream_t user = c->stream;
  c->stream = c->cap_stream;
  const long long before = c->launches;
  cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
  cudaError_t ek = cudaSuccess;
  if (e == cudaSuccess) ek = enqueue_cycle_part(c, H, s, hb, hier, omega, part, nkern);
  cudaGraph_t g = nullptr;
  cudaError_t ee = e == cudaSuccess ? cudaStreamEndCapture(c->cap_stream, &g) : e;
  c->stream = user;
  c->launches = before;  // kernels count when the graph runs
  if (e == cudaSuccess) e = ek != cudaSuccess ? ek : ee;
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return e;
  }
  *graph = g;
  return cudaSuccess;
}

// An executable whole-cycle graph of the same stage, variant, transfer and
// buffer parity whose factors differ, once four such graphs are cached:
// alternating schedules keep their graphs, a schedule whose factors change
// every cycle (transition damping) updates the oldest one in place.
template <typename R>
int reusable_graph(Hier<R>& H, const std::vector<double>& key) {
  int first = -1, same = 0;
  for (size_t i = 0; i < H.graphs.size(); ++i) {
    const auto& g = H.graphs[i];
    if (g.coarse == nullptr && std::equal(key.begin(), key.begin() + 5, g.key.begin())) {
      if (first < 0) first = (int)i;
      ++same;
    }
  }
  return same >= 4 ? first : -1;
}

// One cycle on levels 1..s (s = active finest level).  The two parts run as
// captured CUDA graphs (captured on first use per stage, variant, transfer,
// relaxation factors and buffer parity); with timing on, an event pair
// brackets the fine-sweep graph.
template <typename R>
int run_cycle(mg_ctx* c, Hier<R>& H, int s, int hb, int hier, const cplx<double>* omega) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->timing) {
    if (c->ev_used + 2 > c->ev.size()) {
      for (int k = 0; k < 64; ++k) {
        cudaEvent_t ev;
        if (cudaEventCreate(&ev) != cudaSuccess) return fail(c, MG_ERR_CUDA, "cudaEventCreate failed");
        c->ev.push_back(ev);
      }
    }
    e0 = c->ev[c->ev_used];
    e1 = c->ev[c->ev_used + 1];
    c->ev_used += 2;
  }
  typename Hier<R>::GraphEntry* ge = nullptr;
  if (c->use_graphs) {
    std::vector<double> key = {(double)s, (double)hb, (double)hier, (double)H.cur, c->timing ? 1.0 : 0.0};
    for (int l = 0; l < H.L; ++l) {
      key.push_back(omega[l].x);
      key.push_back(omega[l].y);
    }
    for (auto& g : H.graphs)
      if (g.key == key) { ge = &g; break; }
    if (ge == nullptr) {
      {
        // plans allocate device tables: build them before capturing
        if (c->d == 2 && !H.varphi && s > 1) {
          std::vector<double> ck = {(double)s, (double)hb, (double)hier};
          for (int l = 0; l < H.L; ++l) {
            ck.push_back(omega[l].x);
            ck.push_back(omega[l].y);
          }
          bool ok = true;
          for (int l = 2; l < s && ok; ++l) ok = H.lev[l].gok;
          typename Hier<R>::ChainPlan* cp = nullptr;
          if (ok && build_chain2<R>(c, H, s, hb, hier, omega, ck, &cp) != MG_OK) return MG_ERR_OOM;
        }
      }
      typename Hier<R>::GraphEntry ne;
      ne.key = key;
      cudaGraph_t gf = nullptr, gc = nullptr;
      cudaError_t e;
      if (c->timing) {
        e = capture_part(c, H, s, hb, hier, omega, 0, &gf, &ne.nfine);
        if (e == cudaSuccess && s > 1) e = capture_part(c, H, s, hb, hier, omega, 1, &gc, &ne.ncoarse);
      } else {
        e = capture_part(c, H, s, hb, hier, omega, 2, &gf, &ne.nfine);  // whole cycle
      }
      const int reuse = (e == cudaSuccess && gc == nullptr) ? reusable_graph(H, key) : -1;
      if (reuse >= 0) {
        // same kernels with other arguments: update the executable in place;
        // an executable whose update fails is dropped and a new one built
        auto& old = H.graphs[reuse];
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(old.fine, gf, &info) == cudaSuccess) {
          old.key = key;
          old.nfine = ne.nfine;
          // most recently used last: the next reuse takes the oldest
          std::rotate(H.graphs.begin() + reuse, H.graphs.begin() + reuse + 1, H.graphs.end());
          ge = &H.graphs.back();
        } else {
          cudaGetLastError();
          cudaGraphExecDestroy(old.fine);
          H.graphs.erase(H.graphs.begin() + reuse);
        }
      }
      if (ge == nullptr && e == cudaSuccess) {
        e = cudaGraphInstantiate(&ne.fine, gf, 0);
        if (e == cudaSuccess && gc) e = cudaGraphInstantiate(&ne.coarse, gc, 0);
      }
      if (gf) cudaGraphDestroy(gf);
      if (gc) cudaGraphDestroy(gc);
      if (ge != nullptr) {
        // updated in place
      } else if (e != cudaSuccess) {
        if (ne.fine) cudaGraphExecDestroy(ne.fine);
        if (ne.coarse) cudaGraphExecDestroy(ne.coarse);
        cudaGetLastError();
        c->use_graphs = false;  // run this context's cycles as plain launches
      } else {
        if (H.graphs.size() >= 32) {
          cudaGraphExecDestroy(H.graphs.front().fine);
          if (H.graphs.front().coarse) cudaGraphExecDestroy(H.graphs.front().coarse);
          H.graphs.erase(H.graphs.begin());
        }
        H.graphs.push_back(ne);
        ge = &H.graphs.back();
      }
    }
  }
  cudaError_t e = cudaSuccess;
  int nk = 0;
  if (e0) e = cudaEventRecord(e0, c->stream);
  if (e == cudaSuccess) {
    if (ge) {
      e = cudaGraphLaunch(ge->fine, c->stream);
      c->launches += ge->nfine;
    } else {
      e = enqueue_cycle_part(c, H, s, hb, hier, omega, 0, &nk);
    }
  }
  if (e == cudaSuccess && e1) e = cudaEventRecord(e1, c->stream);
  if (e == cudaSuccess && s > 1 && !(ge && ge->coarse == nullptr)) {
    if (ge) {
      e = cudaGraphLaunch(ge->coarse, c->stream);
      c->launches += ge->ncoarse;
    } else {
      e = enqueue_cycle_part(c, H, s, hb, hier, omega, 1, &nk);
    }
  }
  if (e != cudaSuccess) return fail(c, MG_ERR_CUDA, std::string("cycle launch: ") + cudaGetErrorString(e));
  H.cur = 1 - H.cur;
  return MG_OK;
}

// materialised fine solution of level s into out (same precision)
template <typename R>
cudaError_t materialize(mg_ctx* c, Hier<R>& H, int s, cplx<R>* out) {
  auto& V = H.lev[s];
  ++c->launches;
  const cplx<R>* cc = s > 1 ? H.lev[s - 1].corr : nullptr;
  if (c->d == 2)
    mg::materialize_kernel<R, 2><<<grid_for(V.nv), kThreads, 0, c->stream>>>(V.n, V.u[H.cur], cc, out);
  else
    mg::materialize_kernel<R, 3><<<grid_for(V.nv), kThreads, 0, c->stream>>>(V.n, V.u[H.cur], cc, out);
  return cudaGetLastError();
}

// y = b - H_l x or y = A x with a chosen table, optional norm into norm2[slot]
template <typename R, typename RO>
cudaError_t stencil(mg_ctx* c, Hier<R>& H, int l, int xs, const cplx<R>* x, const cplx<R>* b,
                    const cplx<R>* coef, bool with_phi, cplx<RO>* y, int slot) {
  auto& V = H.lev[l];
  ++c->launches;
  const int g = grid_for(V.nv);
  double* nrm = slot >= 0 ? H.norm2 + slot : nullptr;
  const unsigned long long realmask = coef == V.coefH ? V.realrow3 : (coef == V.coefM ? V.realM : 0ull);
  if (c->d == 2)
    mg::stencil_kernel<R, RO, 2><<<g, kThreads, 0, c->stream>>>(
        V.n, xs, x, b, V.typ, coef, realmask, with_phi ? V.phic : nullptr, V.hcell, y, H.partial,
        H.ticket + 1, nrm);
  else
    mg::stencil_kernel<R, RO, 3><<<g, kThreads, 0, c->stream>>>(
        V.n, xs, x, b, V.typ, coef, realmask, with_phi ? V.phic : nullptr, V.hcell, y, H.partial,
        H.ticket + 1, nrm);
  return cudaGetLastError();
}

// 3D fine level, constant shift: u' = u + e + P cc (optional, into u_out),
// r = b - H u' in FP64 (optional complex64 copy into r32), |r|^2 into
// H.norm2[slot] -- the fused outer step of the defect-correction form and
// the plain FP64 residual norm.
// Cost of each (tile, coarse plane) unit of the 3D FP64 defect in FP64
// operations per vertex: the real passes (z 12, y 18, x 12, update and
// residual 12) plus what a complex coefficient row adds to each pass (z 12
// on planes in the layer, y 18 on rows in the layer, x 12 on tiles whose
// columns reach into it), summed over the unit's three fine planes.
int defect3_costs(mg_ctx* c, Hier<double>& H, int l) {
  auto& V = H.lev[l];
  if (V.d3pref != nullptr) return MG_OK;
  const int n = V.n, nc = n / 3;
  std::vector<uint8_t> rot = layer_flags(c, n), typ(n + 1);
  for (int i = 0; i <= n; ++i) typ[i] = (uint8_t)(rot[std::max(i - 1, 0)] + 2 * rot[std::min(i, n - 1)]);
  const int tx_n = (n + 1 + 29) / 30, ty_n = (n + 1 + 13) / 14;
  std::vector<unsigned> pref((size_t)tx_n * ty_n * nc + 1, 0u);
  size_t u = 0;
  for (int t = 0; t < tx_n * ty_n; ++t) {
    const int x0 = (t % tx_n) * 30, y0 = (t / tx_n) * 14;
    bool xc = false;
    for (int g = x0 - 1; g <= x0 + 30; ++g) xc = xc || (g >= 0 && g <= n && typ[g] != 0);
    int yc = 0, rows = 0;
    for (int g = y0; g < y0 + 14 && g <= n; ++g, ++rows) yc += typ[g] != 0;
    const double yfrac = rows ? (double)yc / rows : 0.0;
    for (int Z = 0; Z < nc; ++Z, ++u) {
      double cost = 0;
      for (int z = 3 * Z; z < 3 * Z + 3; ++z)
        cost += 54.0 + 12.0 * (typ[z] != 0) + 18.0 * yfrac + 12.0 * xc;
      pref[u + 1] = pref[u] + (unsigned)std::lround(cost);
    }
  }
  int rc = dalloc(c, H, (void**)&V.d3pref, pref.size() * sizeof(unsigned));
  if (rc != MG_OK) return rc;
  MG_CUDA(c, cudaMemcpy(V.d3pref, pref.data(), pref.size() * sizeof(unsigned), cudaMemcpyHostToDevice));
  return MG_OK;
}

template <typename RC>
cudaError_t defect3(mg_ctx* c, int l, const cplx<double>* u, const cplx<RC>* e, const cplx<RC>* cc,
                    cplx<double>* u_out, cplx<float>* r32, int slot) {
  auto& H = c->h64;
  auto& V = H.lev[l];
  if (defect3_costs(c, H, l) != MG_OK) return cudaErrorMemoryAllocation;
  mg::Defect3Args<RC> A;
  std::memset(&A, 0, sizeof(A));
  A.n = V.n;
  A.tiles_x = (V.n + 1 + 29) / 30;
  A.tiles_y = (V.n + 1 + 13) / 14;
  A.nunits = (long long)A.tiles_x * A.tiles_y * (V.n / 3);
  A.upref = V.d3pref;
  A.u = u;
  A.e = e;
  A.c = cc;
  A.b = V.b;
  A.u_out = u_out;
  A.r32 = r32;
  A.typ = V.typ;
  axis_rows(c, V.n, A.row);
  A.partial = H.partial;
  A.ticket = H.ticket + 3;
  A.norm2 = slot >= 0 ? H.norm2 + slot : nullptr;
  ++c->launches;
  const long long grid = std::min<long long>(152, std::max<long long>(1, (A.nunits + 3) / 4));
  mg::defect3_kernel<RC><<<(int)grid, mg::kD3Threads, sizeof(mg::Defect3Shared<RC>), c->stream>>>(A);
  return cudaGetLastError();
}

bool use_defect3(const mg_ctx* c) { return c->d == 3 && !c->h64.varphi && c->L >= 1 && interior_real(c); }

// The pending correction corr_{s-1} is the only coarse array a cycle reads
// before writing it (the fine sweep forms u = U + P corr_{s-1}; every t_l and
// the other corr_l are written by the cycle before they are read).
int zero_pending(mg_ctx* c, Hier<double>& H, int s) {
  if (s > 1)
    MG_CUDA(c, cudaMemsetAsync(H.lev[s - 1].corr, 0, H.lev[s - 1].nv * sizeof(cplx<double>), c->stream));
  return MG_OK;
}

int check_ctx(mg_ctx* c) { return c == nullptr ? MG_ERR_INVALID : MG_OK; }

int decode_variant(mg_ctx* c, int variant, int transfer, int* hb, int* hier) {
  if (variant < MG_ADD || variant > MG_BPX) return fail(c, MG_ERR_INVALID, "variant must be MG_ADD, MG_HB or MG_BPX");
  if (transfer != MG_DLINEAR && transfer != MG_HIERARCHICAL)
    return fail(c, MG_ERR_INVALID, "transfer must be MG_DLINEAR or MG_HIERARCHICAL");
  *hb = variant == MG_HB;
  *hier = (transfer == MG_HIERARCHICAL) || (variant == MG_BPX);
  return MG_OK;
}

// Reads and clears the sticky timeout flag of the bounded device waits
// (synchronising).
int check_timeout(mg_ctx* c) {
  unsigned f = 0;
  MG_CUDA(c, cudaMemcpyAsync(c->host_norm + 2, c->dev_err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  std::memcpy(&f, c->host_norm + 2, sizeof(unsigned));
  if (f != 0) {
    MG_CUDA(c, cudaMemsetAsync(c->dev_err, 0, sizeof(unsigned), c->stream));
    return fail(c, MG_ERR_TIMEOUT, "a bounded device-side wait gave up; results of the affected cycles are invalid");
  }
  return MG_OK;
}

// ||b_s - H_s u_s|| of the materialised fine solution of level s (FP64),
// synchronising.
cudaError_t d4_residual(mg_ctx* c, int slot);

int ada_residual_norm(mg_ctx* c, double* out);

int fine_residual(mg_ctx* c, int s, double* out) {
  if (c->ada != nullptr) return ada_residual_norm(c, out);
  if (c->d == 4) {
    cudaError_t e4 = d4_residual(c, 1);
    if (e4 == cudaSuccess)
      e4 = cudaMemcpyAsync(c->host_norm, c->h4->norm2 + 1, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e4 == cudaSuccess) e4 = cudaStreamSynchronize(c->stream);
    if (e4 != cudaSuccess) return fail(c, MG_ERR_CUDA, std::string("residual: ") + cudaGetErrorString(e4));
    *out = std::sqrt(*c->host_norm);
    return MG_OK;
  }
  auto& H = c->h64;
  cudaError_t e;
  if (use_defect3(c)) {
    // u = U + P corr_{s-1} formed in the same pass
    const cplx<double>* nul = nullptr;
    e = defect3<double>(c, s, H.lev[s].u[H.cur], nul, s > 1 ? H.lev[s - 1].corr : nul,
                        (cplx<double>*)nullptr, (cplx<float>*)nullptr, 1);
  } else {
    e = materialize(c, H, s, c->scratch);
    if (e == cudaSuccess)
      e = stencil<double, double>(c, H, s, 1, c->scratch, H.lev[s].b, H.lev[s].coefH, true,
                                  (cplx<double>*)nullptr, 1);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->host_norm, H.norm2 + 1, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(c, MG_ERR_CUDA, std::string("residual: ") + cudaGetErrorString(e));
  *out = std::sqrt(*c->host_norm);
  return check_timeout(c);
}

int ensure_r0(mg_ctx* c) {
  if (c->r0 >= 0) return MG_OK;
  double r;
  int rc = fine_residual(c, c->L, &r);
  if (rc != MG_OK) return rc;
  c->r0 = r;
  return MG_OK;
}

// rhs of level s from the stored nodal f: b_s = M_s (f sampled on level s)
// b_s = M_s f.  fhost (3D, s = L only): a device view of page-locked host
// memory holding f, copied into f_dev by the z-pass itself.
int set_level_rhs(mg_ctx* c, int s, const cplx<double>* fhost = nullptr) {
  auto& H = c->h64;
  cudaError_t e;
  if (c->d == 3) {
    // b = M_x M_y M_z f: z-pass from the (strided) fine f into b, y-pass into
    // the scratch array, x-pass back into b
    auto& V = H.lev[s];
    mg::MassRows3 mr;
    cplx<double> row[4][9];
    axis_rows(c, V.n, row);
    mr.real = 0;
    for (int t = 0; t < 4; ++t) {
      bool re = true;
      for (int j = 0; j < 3; ++j) {
        mr.m[t][j] = row[t][j];
        re = re && row[t][j].y == 0.0;
      }
      if (re) mr.real |= 1u << t;
    }
    const int g = grid_for(V.nv);
    c->launches += 3;
    if (fhost != nullptr && s == c->L)
      mg::mass_z_copy_kernel<<<grid_for((size_t)(V.n + 1) * (V.n + 1)), kThreads, 0, c->stream>>>(
          V.n, fhost, c->f_dev, V.b, V.typ, mr);
    else
      mg::mass_pass3_kernel<2><<<g, kThreads, 0, c->stream>>>(V.n, (int)ipow(3, c->L - s), c->f_dev, V.b, V.typ, mr);
    mg::mass_pass3_kernel<1><<<g, kThreads, 0, c->stream>>>(V.n, 1, V.b, c->scratch, V.typ, mr);
    mg::mass_pass3_kernel<0><<<g, kThreads, 0, c->stream>>>(V.n, 1, c->scratch, V.b, V.typ, mr);
    e = cudaGetLastError();
  } else {
    e = stencil<double, double>(c, H, s, (int)ipow(3, c->L - s), c->f_dev, nullptr, H.lev[s].coefM, false,
                                H.lev[s].b, -1);
  }
  if (e != cudaSuccess) return fail(c, MG_ERR_CUDA, cudaGetErrorString(e));
  return MG_OK;
}

// ------------------------------------------------------------------ d = 4
template <typename H>
int d4_alloc(mg_ctx* c, H& h, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(c, e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA,
                std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  h.allocs.push_back(*p);
  MG_CUDA(c, cudaMemset(*p, 0, bytes));
  return MG_OK;
}

template <typename R>
void d4_free(Hier4<R>* H) {
  if (H == nullptr) return;
  if (H->exec) cudaGraphExecDestroy(H->exec);
  for (void* p : H->allocs) cudaFree(p);
  delete H;
}

template <typename H, typename T>
int d4_upload(mg_ctx* c, H& h, T** dst, const std::vector<T>& v) {
  int rc = d4_alloc(c, h, (void**)dst, v.size() * sizeof(T));
  if (rc != MG_OK) return rc;
  MG_CUDA(c, cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return MG_OK;
}

template <typename R>
cplx<R> to_r(const cd& v) {
  return cplx<R>{(R)v.real(), (R)v.imag()};
}

// Per-level arrays and the separable operator tables, formed in FP64 and
// stored in R: the rows of each axis index are those of its vertex type
// (left / right cell in the layer), the Galerkin rows those of
// galerkin_rows_1d, the diagonal of vertex type (t0, t1, t2, t3) is
// sum_j prod_a (K if a == j else M)[t_a] centre entries minus
// phi prod_a M[t_a] centre (the tensor-product form of Section 4).
template <typename R>
int d4_build(mg_ctx* c, Hier4<R>*& out) {
  Hier4<R>* H = new (std::nothrow) Hier4<R>();
  if (H == nullptr) return fail(c, MG_ERR_OOM, "host allocation failed");
  out = H;
  const int L = c->L;
  const double phi = c->k2[0];
  H->lev.resize(L + 1);
  int rc;
  for (int l = 1; l <= L; ++l) {
    Lev4<R>& V = H->lev[l];
    V.n = (int)ipow(3, l);
    V.nv = (size_t)ipow(V.n + 1, 4);
    const size_t bytes = V.nv * sizeof(cplx<R>);
    if ((rc = d4_alloc(c, *H, (void**)&V.u, bytes)) != MG_OK) return rc;
    if ((rc = d4_alloc(c, *H, (void**)&V.b, bytes)) != MG_OK) return rc;
    if ((rc = d4_alloc(c, *H, (void**)&V.t, bytes)) != MG_OK) return rc;
    if (l == 1) {
      V.corr = V.t;
    } else if ((rc = d4_alloc(c, *H, (void**)&V.corr, bytes)) != MG_OK) {
      return rc;
    }
    std::vector<uint8_t> rot = layer_flags(c, V.n), typ(V.n + 1);
    for (int i = 0; i <= V.n; ++i) typ[i] = (uint8_t)(rot[std::max(i - 1, 0)] + 2 * rot[std::min(i, V.n - 1)]);
    if ((rc = d4_upload(c, *H, &V.typ, typ)) != MG_OK) return rc;
    cplx<double> row[4][9];
    axis_rows(c, V.n, row);
    std::vector<cplx<R>> rows((size_t)3 * (V.n + 1) * 3);
    for (int k = 0; k < 3; ++k)
      for (int i = 0; i <= V.n; ++i)
        for (int j = 0; j < 3; ++j) {
          const cplx<double>& v = row[typ[i]][3 * k + j];
          rows[((size_t)k * (V.n + 1) + i) * 3 + j] = cplx<R>{(R)v.x, (R)v.y};
        }
    if ((rc = d4_upload(c, *H, &V.rows, rows)) != MG_OK) return rc;
    V.real = std::all_of(rows.begin(), rows.end(), [](const cplx<R>& v) { return v.y == R(0); });
    std::vector<cplx<R>> invd(256);
    for (int ty = 0; ty < 256; ++ty) {
      cd mprod(1.0), kterm(0.0);
      for (int j = 0; j < 4; ++j) {
        cd p(1.0);
        for (int a = 0; a < 4; ++a) {
          const auto& r = row[(ty >> (2 * a)) & 3];
          p *= a == j ? cd(r[4].x, r[4].y) : cd(r[1].x, r[1].y);
        }
        kterm += p;
      }
      for (int a = 0; a < 4; ++a) {
        const auto& r = row[(ty >> (2 * a)) & 3];
        mprod *= cd(r[1].x, r[1].y);
      }
      invd[ty] = to_r<R>(1.0 / (kterm - phi * mprod));
    }
    if ((rc = d4_upload(c, *H, &V.invd, invd)) != MG_OK) return rc;
    V.dreal = std::all_of(invd.begin(), invd.end(), [](const cplx<R>& v) { return v.y == R(0); });
    if ((rc = d4_alloc(c, *H, (void**)&V.omd, 256 * sizeof(cplx<R>))) != MG_OK) return rc;
    if (l > 1) {
      std::vector<std::array<cd, 6>> g;
      galerkin_rows_1d(V.n, rot, widths(c, V.n), g);
      const int nc = V.n / 3;
      std::vector<cplx<R>> gr((size_t)3 * (nc + 1) * 3);
      for (int i = 0; i <= nc; ++i)
        for (int j = 0; j < 3; ++j) {
          const cd m = g[i][3 + j], k = g[i][j], kp = k - phi * m;
          gr[((size_t)0 * (nc + 1) + i) * 3 + j] = to_r<R>(m);
          gr[((size_t)1 * (nc + 1) + i) * 3 + j] = to_r<R>(k);
          gr[((size_t)2 * (nc + 1) + i) * 3 + j] = to_r<R>(kp);
        }
      if ((rc = d4_upload(c, *H, &V.grows, gr)) != MG_OK) return rc;
      V.greal = std::all_of(gr.begin(), gr.end(), [](const cplx<R>& v) { return v.y == R(0); });
    }
  }
  const size_t fb = H->lev[L].nv * sizeof(cplx<R>);
  for (int k = 0; k < 5; ++k)
    if ((rc = d4_alloc(c, *H, (void**)&H->T[k], fb)) != MG_OK) return rc;
  if ((rc = d4_alloc(c, *H, (void**)&H->partial, 152 * 16 * sizeof(double))) != MG_OK) return rc;
  if ((rc = d4_alloc(c, *H, (void**)&H->ticket, 4 * sizeof(unsigned))) != MG_OK) return rc;
  if ((rc = d4_alloc(c, *H, (void**)&H->norm2, 4 * sizeof(double))) != MG_OK) return rc;
  return MG_OK;
}

mg::Box4 box4(int n0, int n1, int n2, int n3) { return mg::Box4{{n0, n1, n2, n3}}; }

size_t box4_size(const mg::Box4& B) { return (size_t)B.n[0] * B.n[1] * B.n[2] * B.n[3]; }

template <typename R>
void pass4(mg_ctx* c, const mg::Box4& B, int axis, bool real, const cplx<R>* rows, const cplx<R>* x,
           const cplx<R>* z, const cplx<R>* b, cplx<R>* y, int neg) {
  ++c->launches;
  const int g = grid_for(box4_size(B));
  if (real)
    mg::pass4_kernel<R, true><<<g, kThreads, 0, c->stream>>>(B, axis, rows, x, z, b, y, neg);
  else
    mg::pass4_kernel<R, false><<<g, kThreads, 0, c->stream>>>(B, axis, rows, x, z, b, y, neg);
}

// y = b + A x or b - A x (neg): A the separable operator with rows
// [M, K, K - phi M] per index on a grid of n cells per axis (ten passes
// through T[0..3]).
template <typename R>
cudaError_t d4_apply(mg_ctx* c, Hier4<R>& H, int n, const cplx<R>* rows, bool real, const cplx<R>* x,
                     const cplx<R>* b, cplx<R>* y, int neg) {
  const int N = n + 1;
  const mg::Box4 B = box4(N, N, N, N);
  const cplx<R>* M = rows;
  const cplx<R>* K = rows + 3 * N;
  const cplx<R>* KP = rows + 6 * N;
  cplx<R>** T = H.T;
  const cplx<R>* nul = nullptr;
  pass4(c, B, 3, real, M, x, nul, nul, T[0], 0);       // A = M3 x
  pass4(c, B, 3, real, KP, x, nul, nul, T[1], 0);      // B = (K3 - phi M3) x
  pass4(c, B, 2, real, M, T[0], nul, nul, T[2], 0);    // C = M2 A
  pass4(c, B, 2, real, M, T[1], nul, nul, T[3], 0);    // M2 B
  pass4(c, B, 2, real, K, T[0], T[3], nul, T[1], 0);   // D = K2 A + M2 B
  pass4(c, B, 1, real, M, T[1], nul, nul, T[3], 0);    // M1 D
  pass4(c, B, 1, real, K, T[2], T[3], nul, T[0], 0);   // E = K1 C + M1 D
  pass4(c, B, 1, real, M, T[2], nul, nul, T[1], 0);    // F = M1 C
  pass4(c, B, 0, real, K, T[1], nul, nul, T[2], 0);    // K0 F
  pass4(c, B, 0, real, M, T[0], T[2], b, y, neg);      // y = b -+ (M0 E + K0 F)
  return cudaGetLastError();
}

// b = M f on the finest level (four mass passes).
cudaError_t d4_mass(mg_ctx* c, const cplx<double>* f, cplx<double>* b) {
  Hier4<double>& H = *c->h4;
  const Lev4<double>& V = H.lev[c->L];
  const int N = V.n + 1;
  const mg::Box4 B = box4(N, N, N, N);
  const cplx<double>* nul = nullptr;
  const cplx<double>* in[4] = {f, H.T[0], H.T[1], H.T[0]};
  cplx<double>* out[4] = {H.T[0], H.T[1], H.T[0], b};
  for (int k = 0; k < 4; ++k) pass4(c, B, 3 - k, V.real, V.rows, in[k], nul, nul, out[k], 0);
  return cudaGetLastError();
}

// Restriction of a level-l array (n fine cells per axis) to level l - 1,
// axis by axis through T[0], T[1].
template <typename R>
cudaError_t d4_restrict(mg_ctx* c, Hier4<R>& H, int n, const cplx<R>* x, cplx<R>* y) {
  const int N = n + 1, Nc = n / 3 + 1;
  int ext[4] = {N, N, N, N};
  const cplx<R>* src = x;
  cplx<R>* dst[4] = {H.T[0], H.T[1], H.T[0], y};
  for (int a = 0; a < 4; ++a) {
    ext[a] = Nc;
    const mg::Box4 B = box4(ext[0], ext[1], ext[2], ext[3]);
    ++c->launches;
    mg::restrict4_kernel<R><<<grid_for(box4_size(B)), kThreads, 0, c->stream>>>(B, a, N, src, dst[a]);
    src = dst[a];
  }
  return cudaGetLastError();
}

// y = base + P x (or base - P x with neg) for x on level l - 1 (n fine cells
// per axis), through T[1], T[2].
template <typename R>
cudaError_t d4_prolong(mg_ctx* c, Hier4<R>& H, int n, const cplx<R>* x, const cplx<R>* base, cplx<R>* y,
                       int neg) {
  const int N = n + 1, Nc = n / 3 + 1;
  int ext[4] = {Nc, Nc, Nc, Nc};
  const cplx<R>* src = x;
  cplx<R>* dst[4] = {H.T[1], H.T[2], H.T[1], y};
  for (int a = 0; a < 4; ++a) {
    ext[a] = N;
    const mg::Box4 B = box4(ext[0], ext[1], ext[2], ext[3]);
    const bool last = a == 3;
    ++c->launches;
    mg::prolong4_kernel<R><<<grid_for(box4_size(B)), kThreads, 0, c->stream>>>(
        B, a, src, last ? base : nullptr, dst[a], last ? neg : 0);
    src = dst[a];
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t d4_inject(mg_ctx* c, int n, const cplx<R>* x, cplx<R>* y) {
  const int Nc = n / 3 + 1;
  const mg::Box4 B = box4(Nc, Nc, Nc, Nc);
  ++c->launches;
  mg::inject4_kernel<R><<<grid_for(box4_size(B)), kThreads, 0, c->stream>>>(B, x, y);
  return cudaGetLastError();
}

// One additive FAS cycle in four dimensions (Appendix A, Algorithm 4 with the
// coarse right-hand side b_{l-1} = R r_l + G u_{l-1}): residual, Jacobi and
// restriction from the finest level down, then the corrections
// corr_l = T_l du_l + P corr_{l-1} and u_L += corr_L.  The fine level is
// read by the residual and updated at the end (no pending correction).  The
// fine residual norm is fused into the Jacobi step (complex128 only).
template <typename R>
cudaError_t d4_enqueue_cycle(mg_ctx* c, Hier4<R>& H, int hb, int hier, const cplx<double>* omega) {
  const int L = c->L;
  const bool f64 = std::is_same<R, double>::value;
  cudaError_t e = cudaSuccess;
  for (int l = L; l >= 1 && e == cudaSuccess; --l) {
    Lev4<R>& V = H.lev[l];
    if (l == L && c->timing) e = cudaEventRecord(c->ev[c->ev_used], c->stream);
    if (e == cudaSuccess) e = d4_apply(c, H, V.n, V.rows, V.real, V.u, V.b, H.T[4], 1);  // r_l
    if (l == L && c->timing && e == cudaSuccess) e = cudaEventRecord(c->ev[c->ev_used + 1], c->stream);
    if (e != cudaSuccess) break;
    c->launches += 2;
    mg::omega_table4_kernel<R><<<1, 256, 0, c->stream>>>(V.invd, omega[l - 1], V.omd);
    double* nrm = (l == L && f64) ? H.norm2 : nullptr;
    if (V.dreal && omega[l - 1].y == 0.0)
      mg::jacobi4_kernel<R, true><<<grid_for(V.nv), kThreads, 0, c->stream>>>(V.n, H.T[4], V.t, V.typ, V.omd, hb,
                                                                             H.partial, H.ticket, nrm);
    else
      mg::jacobi4_kernel<R, false><<<grid_for(V.nv), kThreads, 0, c->stream>>>(V.n, H.T[4], V.t, V.typ, V.omd, hb,
                                                                              H.partial, H.ticket, nrm);
    if (l > 1) {
      Lev4<R>& W = H.lev[l - 1];
      e = d4_inject(c, V.n, V.u, W.u);
      if (e == cudaSuccess) e = d4_restrict(c, H, V.n, H.T[4], W.b);
      if (e == cudaSuccess) e = d4_apply(c, H, W.n, V.grows, V.greal, W.u, W.b, W.b, 0);  // + G u_{l-1}
      if (hier && e == cudaSuccess) {
        // BPX transfer: T du = du - P I du
        e = d4_inject(c, V.n, V.t, H.T[0]);
        if (e == cudaSuccess) e = d4_prolong(c, H, V.n, H.T[0], V.t, V.t, 1);
      }
    }
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  for (int l = 2; l <= L && e == cudaSuccess; ++l)
    e = d4_prolong(c, H, H.lev[l].n, H.lev[l - 1].corr, H.lev[l].t, H.lev[l].corr, 0);
  if (e == cudaSuccess) {
    const Lev4<R>& F = H.lev[L];
    ++c->launches;
    mg::update4_kernel<R, R><<<grid_for(F.nv), kThreads, 0, c->stream>>>(F.n, F.u, F.corr);
    e = cudaGetLastError();
  }
  return e;
}

// One cycle as a CUDA graph: captured on first use and updated in place when
// the variant, transfer or factors change; with timing on, plain launches
// with an event pair around the finest level's residual.
template <typename R>
int d4_cycle(mg_ctx* c, Hier4<R>& H, int hb, int hier, const cplx<double>* omega) {
  cudaError_t e = cudaSuccess;
  if (c->timing) {
    if (c->ev_used + 2 > c->ev.size()) {
      for (int k = 0; k < 64; ++k) {
        cudaEvent_t ev;
        if (cudaEventCreate(&ev) != cudaSuccess) return fail(c, MG_ERR_CUDA, "cudaEventCreate failed");
        c->ev.push_back(ev);
      }
    }
    e = d4_enqueue_cycle(c, H, hb, hier, omega);
    c->ev_used += 2;
    if (e != cudaSuccess) return fail(c, MG_ERR_CUDA, std::string("cycle launch: ") + cudaGetErrorString(e));
    return MG_OK;
  }
  if (c->use_graphs) {
    std::vector<double> key = {(double)hb, (double)hier};
    for (int l = 0; l < c->L; ++l) {
      key.push_back(omega[l].x);
      key.push_back(omega[l].y);
    }
    if (H.exec == nullptr || H.key != key) {
      cudaStream_t user = c->stream;
      c->stream = c->cap_stream;
      const long long before = c->launches;
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
      cudaError_t ek = e == cudaSuccess ? d4_enqueue_cycle(c, H, hb, hier, omega) : e;
      cudaError_t ee = e == cudaSuccess ? cudaStreamEndCapture(c->cap_stream, &g) : e;
      c->stream = user;
      const long long nk = c->launches - before;
      c->launches = before;
      e = ek != cudaSuccess ? ek : ee;
      if (e == cudaSuccess) {
        cudaGraphExecUpdateResultInfo info;
        if (H.exec == nullptr || cudaGraphExecUpdate(H.exec, g, &info) != cudaSuccess) {
          cudaGetLastError();
          if (H.exec) cudaGraphExecDestroy(H.exec);
          H.exec = nullptr;
          e = cudaGraphInstantiate(&H.exec, g, 0);
        }
      }
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        cudaGetLastError();
        if (H.exec) cudaGraphExecDestroy(H.exec);
        H.exec = nullptr;
        c->use_graphs = false;
      } else {
        H.key = key;
        H.nkern = nk;
      }
    }
    if (H.exec != nullptr) {
      e = cudaGraphLaunch(H.exec, c->stream);
      c->launches += H.nkern;
      if (e != cudaSuccess) return fail(c, MG_ERR_CUDA, std::string("cycle launch: ") + cudaGetErrorString(e));
      return MG_OK;
    }
  }
  e = d4_enqueue_cycle(c, H, hb, hier, omega);
  if (e != cudaSuccess) return fail(c, MG_ERR_CUDA, std::string("cycle launch: ") + cudaGetErrorString(e));
  return MG_OK;
}

// Fine residual r = b - H u into T[4]; |r|^2 into norm2[slot] when slot >= 0.
cudaError_t d4_residual(mg_ctx* c, int slot) {
  Hier4<double>& H = *c->h4;
  const Lev4<double>& V = H.lev[c->L];
  cudaError_t e = d4_apply(c, H, V.n, V.rows, V.real, V.u, V.b, H.T[4], 1);
  if (e == cudaSuccess && slot >= 0) {
    ++c->launches;
    mg::norm4_kernel<<<grid_for(V.nv), kThreads, 0, c->stream>>>(V.n, H.T[4], H.partial, H.ticket + 1,
                                                                   H.norm2 + slot);
    e = cudaGetLastError();
  }
  return e;
}

// The defect-correction form in four dimensions: per outer step the FP64
// residual (norm fused) becomes the complex64 rhs of H e = r, `inner` complex64
// cycles from e = 0 follow, and u += e in FP64.
int d4_refine(mg_ctx* c, int hb, int hier, const cplx<double>* omega, double tol, int max_cycles, int* done,
              double* rel) {
  Hier4<double>& H = *c->h4;
  Hier4<float>& E = *c->h4f;
  const int L = c->L;
  Lev4<double>& F = H.lev[L];
  Lev4<float>& EF = E.lev[L];
  auto diverged = [&](double x) { return !std::isfinite(x) || x > 1e6; };
  // r = b - H u and its norm
  MG_CUDA(c, d4_residual(c, 1));
  while (true) {
    MG_CUDA(c, cudaMemcpyAsync(c->host_norm, H.norm2 + 1, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    MG_CUDA(c, cudaStreamSynchronize(c->stream));
    *rel = c->r0 > 0 ? std::sqrt(*c->host_norm) / c->r0 : 0.0;
    if (diverged(*rel)) return MG_DIVERGED;
    if (*rel <= tol) return MG_OK;
    if (*done >= max_cycles) return MG_NOT_CONVERGED;
    ++c->launches;
    mg::to_c64_kernel<<<grid_for(F.nv), kThreads, 0, c->stream>>>((long long)F.nv, H.T[4], EF.b);
    MG_CUDA(c, cudaMemsetAsync(EF.u, 0, EF.nv * sizeof(cplx<float>), c->stream));
    const int m = std::min(c->inner_cycles, std::max(1, max_cycles - *done));
    for (int k = 0; k < m; ++k) {
      int rc = d4_cycle(c, E, hb, hier, omega);
      if (rc != MG_OK) return rc;
      ++*done;
    }
    ++c->launches;
    mg::update4_kernel<double, float><<<grid_for(F.nv), kThreads, 0, c->stream>>>(F.n, F.u, EF.u);
    MG_CUDA(c, cudaGetLastError());
    MG_CUDA(c, d4_residual(c, 1));
  }
}

// ------------------------------------------------------------------ adaptive
// succ of every level, fine to coarse (Section 5.1); the fine-grid
// vertices are counted into *nfine when it is not null.
template <int D>
cudaError_t ada_succ_all(mg_ctx* c, unsigned long long* nfine) {
  HierA& H = *c->ada;
  const int L = c->L;
  for (int l = L; l >= 1; --l) {
    LevA& V = H.lev[l];
    const LevA* F = l < L ? &H.lev[l + 1] : nullptr;
    ++c->launches;
    mg::ada_succ_kernel<D><<<grid_for(V.nv), kThreads, 0, c->stream>>>(
        V.n, V.cellf, V.vcls, F ? F->vcls : nullptr, F ? F->succ : nullptr, V.succ,
        nfine != nullptr ? nfine : H.abuf + kAbFine, H.boxes + l);
  }
  return cudaGetLastError();
}

void ada_free(HierA* H) {
  if (H == nullptr) return;
  if (H->exec) cudaGraphExecDestroy(H->exec);
  if (H->aexec) cudaGraphExecDestroy(H->aexec);
  if (H->hbuf) cudaFreeHost(H->hbuf);
  for (void* p : H->allocs) cudaFree(p);
  delete H;
}

// Cells, vertex classes and operator data of every level of the adaptive
// tree.  refine: the flags of levels 1..L-1, level l's (3^l)^d cells x fastest,
// concatenated; flags of cells that do not exist are ignored.
int ada_build(mg_ctx* c, const unsigned char* refine) {
  HierA* H = new (std::nothrow) HierA();
  if (H == nullptr) return fail(c, MG_ERR_OOM, "host allocation failed");
  c->ada = H;
  const int d = c->d, L = c->L;
  bool varphi = false;
  for (size_t i = 1; i < c->k2.size() && !varphi; ++i) varphi = c->k2[i] != c->k2[0];
  H->lev.resize(L + 1);
  std::vector<uint8_t> cells(ipow(3, d), 1);  // level 1: every cell
  size_t off = 0;
  int rc;
  for (int l = 1; l <= L; ++l) {
    LevA& V = H->lev[l];
    V.n = (int)ipow(3, l);
    const int n = V.n, N = n + 1;
    V.nv = (size_t)ipow(N, d);
    const size_t ncell = (size_t)ipow(n, d);
    std::vector<uint8_t> cellf(ncell, 0);
    for (size_t ci = 0; ci < ncell; ++ci) {
      const bool ex = cells[ci] != 0;
      const bool rf = l < L && ex && refine[off + ci] != 0;
      cellf[ci] = (uint8_t)((ex ? mg::kCellExists : 0) | (rf ? mg::kCellRefined : 0));
    }
    if (l < L) off += ncell;
    // vertex classes from the number of existing cells around each vertex
    std::vector<uint8_t> vcls(V.nv, 0);
    for (size_t vi = 0; vi < V.nv; ++vi) {
      int g[3] = {0, 0, 0};
      size_t r = vi;
      bool inner = true;
      for (int a = 0; a < d; ++a) {
        g[a] = (int)(r % N);
        r /= N;
        inner = inner && g[a] > 0 && g[a] < n;
      }
      int cnt = 0, tot = 0;
      for (int e = 0; e < (1 << d); ++e) {
        size_t ci = 0, cs = 1;
        bool in = true;
        for (int a = 0; a < d; ++a) {
          const int ca = g[a] - 1 + ((e >> a) & 1);
          in = in && ca >= 0 && ca < n;
          ci += (size_t)(in ? ca : 0) * cs;
          cs *= (size_t)n;
        }
        if (!in) continue;
        ++tot;
        cnt += (cellf[ci] & mg::kCellExists) ? 1 : 0;
      }
      vcls[vi] = cnt == 0 ? mg::kVertNone : ((inner && cnt == (1 << d)) ? mg::kVertUnknown : mg::kVertBound);
      (void)tot;
    }
    {
      int lo[3] = {N, N, N}, hi[3] = {-1, -1, -1};
      for (size_t vi = 0; vi < V.nv; ++vi) {
        if (vcls[vi] == mg::kVertNone) continue;
        size_t r = vi;
        for (int a = 0; a < d; ++a) {
          const int g = (int)(r % N);
          r /= N;
          lo[a] = std::min(lo[a], g);
          hi[a] = std::max(hi[a], g);
        }
      }
      const bool empty = hi[0] < 0;
      V.boxvol = 1;
      for (int a = 0; a < 3; ++a) {
        V.box.lo[a] = a < d && !empty ? lo[a] : 0;
        V.box.ext[a] = empty ? 0 : (a < d ? hi[a] - lo[a] + 1 : 1);
        V.boxvol *= (size_t)V.box.ext[a];
      }
      if (!empty) H->Lf = l;
    }
    const size_t bytes = V.nv * sizeof(cplx<double>);
    for (cplx<double>** p : {&V.u, &V.f, &V.r, &V.t, &V.invd}) {
      if ((rc = d4_alloc(c, *H, (void**)p, bytes)) != MG_OK) return rc;
    }
    if (l == 1) {
      V.corr = V.t;
    } else if ((rc = d4_alloc(c, *H, (void**)&V.corr, bytes)) != MG_OK) {
      return rc;
    }
    if ((rc = d4_upload(c, *H, &V.cellf, cellf)) != MG_OK) return rc;
    if ((rc = d4_upload(c, *H, &V.vcls, vcls)) != MG_OK) return rc;
    if ((rc = d4_alloc(c, *H, (void**)&V.succ, V.nv)) != MG_OK) return rc;
    if ((rc = d4_alloc(c, *H, (void**)&V.s, V.nv * sizeof(double))) != MG_OK) return rc;
    if ((rc = d4_alloc(c, *H, (void**)&V.rmark, ncell)) != MG_OK) return rc;
    if ((rc = d4_alloc(c, *H, (void**)&V.emark, V.nv)) != MG_OK) return rc;
    const std::vector<uint8_t> rot = layer_flags(c, n);
    const Widths wd = widths(c, n);
    std::vector<cplx<double>> hc(n), hi(n);
    for (int k = 0; k < n; ++k) {
      const cd h = rot[k] ? wd.rot : wd.in;
      hc[k] = cplx<double>{h.real(), h.imag()};
      const cd q = 1.0 / h;
      hi[k] = cplx<double>{q.real(), q.imag()};
    }
    if ((rc = d4_upload(c, *H, &V.hcell, hc)) != MG_OK) return rc;
    if ((rc = d4_upload(c, *H, &V.hinv, hi)) != MG_OK) return rc;
    if ((rc = d4_upload(c, *H, &V.rotf, rot)) != MG_OK) return rc;
    {
      // element matrices of the 2^d width classes (Section 4): M = prod_a m1,
      // K = sum_j prod_a (k1 if a == j else m1), m1(h) = h/6 [2 1; 1 2],
      // k1(h) = 1/h [1 -1; -1 1]; stored as M and K - phi0 M
      const int nc = 1 << d, ne = nc * nc;
      std::vector<cplx<double>> em((size_t)(1 << d) * 2 * ne);
      for (int cls = 0; cls < (1 << d); ++cls)
        for (int a = 0; a < nc; ++a)
          for (int b = 0; b < nc; ++b) {
            cd m(1.0), k(0.0);
            for (int ax = 0; ax < d; ++ax) {
              const cd h = ((cls >> ax) & 1) ? wd.rot : wd.in;
              m *= h * ((((a >> ax) & 1) == ((b >> ax) & 1)) ? 1.0 / 3.0 : 1.0 / 6.0);
            }
            for (int j = 0; j < d; ++j) {
              cd p(1.0);
              for (int ax = 0; ax < d; ++ax) {
                const cd h = ((cls >> ax) & 1) ? wd.rot : wd.in;
                const bool same = ((a >> ax) & 1) == ((b >> ax) & 1);
                p *= ax == j ? (same ? 1.0 : -1.0) / h : h * (same ? 1.0 / 3.0 : 1.0 / 6.0);
              }
              k += p;
            }
            const cd hm = k - c->k2[0] * m;
            em[(size_t)(2 * cls) * ne + a * nc + b] = cplx<double>{m.real(), m.imag()};
            em[(size_t)(2 * cls + 1) * ne + a * nc + b] = cplx<double>{hm.real(), hm.imag()};
          }
      if ((rc = d4_upload(c, *H, &V.emat, em)) != MG_OK) return rc;
    }
    if (varphi) {
      std::vector<double> ph = cell_shift<double>(c, l);
      if ((rc = d4_upload(c, *H, &V.phic, ph)) != MG_OK) return rc;
    }
    if (d == 2)
      mg::ada_diag_kernel<2><<<grid_for(V.nv), kThreads>>>(n, V.vcls, V.hcell, V.hinv, V.phic, c->k2[0], V.invd,
                                                           nullptr);
    else
      mg::ada_diag_kernel<3><<<grid_for(V.nv), kThreads>>>(n, V.vcls, V.hcell, V.hinv, V.phic, c->k2[0], V.invd,
                                                           nullptr);
    MG_CUDA(c, cudaGetLastError());
    MG_CUDA(c, cudaDeviceSynchronize());
    // children of refined cells exist on the next level
    if (l < L) {
      const int nf = 3 * n;
      std::vector<uint8_t> next((size_t)ipow(nf, d), 0);
      for (size_t fi = 0; fi < next.size(); ++fi) {
        size_t r = fi, ci = 0, cs = 1;
        for (int a = 0; a < d; ++a) {
          ci += (r % nf) / 3 * cs;
          r /= nf;
          cs *= (size_t)n;
        }
        next[fi] = (cellf[ci] & mg::kCellRefined) ? 1 : 0;
      }
      cells.swap(next);
    }
  }
  const size_t fb = H->lev[L].nv * sizeof(cplx<double>);
  for (int k = 0; k < 2; ++k)
    if ((rc = d4_alloc(c, *H, (void**)&H->T[k], fb)) != MG_OK) return rc;
  if ((rc = d4_alloc(c, *H, (void**)&H->partial, 152 * 16 * sizeof(double))) != MG_OK) return rc;
  if ((rc = d4_alloc(c, *H, (void**)&H->ticket, 4 * sizeof(unsigned))) != MG_OK) return rc;
  if ((rc = d4_alloc(c, *H, (void**)&H->norm2, 32 * sizeof(double))) != MG_OK) return rc;
  if ((rc = d4_alloc(c, *H, (void**)&H->abuf, kAbSlots * sizeof(unsigned long long))) != MG_OK) return rc;
  if ((rc = d4_alloc(c, *H, (void**)&H->box6, 6 * (L + 1) * sizeof(int))) != MG_OK) return rc;
  {
    std::vector<mg::AdaBox> bx(L + 1);
    H->gcap.assign(L + 1, 1);
    for (int l = 1; l <= L; ++l) {
      bx[l] = H->lev[l].box;
      H->gcap[l] = grid_for(H->lev[l].boxvol);
    }
    if ((rc = d4_upload(c, *H, &H->boxes, bx)) != MG_OK) return rc;
  }
  MG_CUDA(c, cudaMallocHost(&H->hbuf, 4096));
  MG_CUDA(c, d == 2 ? ada_succ_all<2>(c, nullptr) : ada_succ_all<3>(c, nullptr));
  MG_CUDA(c, cudaDeviceSynchronize());
  return MG_OK;
}

// The residuals of levels Lf..1 (levels above Lf hold no cells), their
// fused norms and, when maxabs is requested, per-level max |r| into
// abuf[kAbMax + l].
template <int D>
cudaError_t ada_residuals(mg_ctx* c, bool maxabs = false) {
  HierA& H = *c->ada;
  const int Lf = H.Lf;
  const double phi0 = c->k2[0];
  for (int l = Lf; l >= 1; --l) {
    LevA& V = H.lev[l];
    ++c->launches;
    mg::ada_residual_kernel<D><<<H.gcap[l], kThreads, 0, c->stream>>>(
        V.n, V.u, V.f, V.cellf, V.vcls, V.hcell, V.hinv, V.phic, phi0, l < Lf ? H.lev[l + 1].r : nullptr, V.r,
        l < Lf ? H.lev[l + 1].vcls : nullptr, H.partial, H.ticket, H.norm2 + l, H.boxes + l, V.rotf, V.emat,
        maxabs ? H.abuf + kAbMax + l : nullptr);
  }
  return cudaGetLastError();
}

// Hanging values from the coarser level (coarse to fine), then injection of
// values that carry an unknown on the finer level (fine to coarse).
template <int D>
cudaError_t ada_invariants(mg_ctx* c) {
  HierA& H = *c->ada;
  const int L = c->L;
  for (int l = 2; l <= L; ++l) {
    LevA& V = H.lev[l];
    c->launches += 2;
    mg::ada_prolong_kernel<D><<<grid_for(V.nv), kThreads, 0, c->stream>>>(V.n, H.lev[l - 1].u, nullptr, H.T[0], 0);
    mg::ada_set_hanging_kernel<D><<<grid_for(V.nv), kThreads, 0, c->stream>>>(V.n, V.vcls, H.T[0], V.u);
  }
  for (int l = L - 1; l >= 1; --l) {
    LevA& V = H.lev[l];
    ++c->launches;
    mg::ada_inject_unknown_kernel<D><<<H.gcap[l], kThreads, 0, c->stream>>>(V.n, H.lev[l + 1].vcls,
                                                                           H.lev[l + 1].u, V.u, H.boxes + l);
  }
  return cudaGetLastError();
}

// One cycle: the residuals bottom-up (norm fused), the fused coarse-to-fine
// pass (Jacobi, transfer, correction, update, hanging values) and the
// injection bottom-up: 3L - 1 launches.
template <int D>
cudaError_t ada_enqueue_cycle(mg_ctx* c, int hb, int hier, const cplx<double>* omega) {
  HierA& H = *c->ada;
  const int L = c->L, Lf = H.Lf;
  // omega by succ (Section 5.1): the per-level array's entry for the
  // distance L - l to the finest level serves succ = L - l
  mg::AdaOmega om{};
  for (int s = 0; s < L; ++s) om.w[s] = omega[L - 1 - s];
  cudaError_t e = ada_residuals<D>(c);
  for (int l = 1; l <= Lf && e == cudaSuccess; ++l) {
    LevA& V = H.lev[l];
    const LevA* W = l > 1 ? &H.lev[l - 1] : nullptr;
    ++c->launches;
    mg::ada_down_kernel<D><<<H.gcap[l], kThreads, 0, c->stream>>>(
        V.n, V.r, V.invd, V.vcls, V.succ, om, hb, hier, W ? W->corr : nullptr, W ? W->u : nullptr, V.corr, V.u,
        H.boxes + l);
    e = cudaGetLastError();
  }
  for (int l = Lf - 1; l >= 1 && e == cudaSuccess; --l) {
    LevA& V = H.lev[l];
    ++c->launches;
    mg::ada_inject_unknown_kernel<D><<<H.gcap[l], kThreads, 0, c->stream>>>(V.n, H.lev[l + 1].vcls,
                                                                           H.lev[l + 1].u, V.u, H.boxes + l);
    e = cudaGetLastError();
  }
  return e;
}

int ada_norm_host(mg_ctx* c, double* out) {
  HierA& H = *c->ada;
  // the pinned buffer holds 4 doubles: copy the level norms in groups
  double tot = 0.0;
  for (int l0 = 1; l0 <= H.Lf; l0 += 4) {
    const int cnt = std::min(4, H.Lf - l0 + 1);
    MG_CUDA(c, cudaMemcpyAsync(c->host_norm, H.norm2 + l0, sizeof(double) * cnt, cudaMemcpyDeviceToHost,
                               c->stream));
    MG_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < cnt; ++k) tot += c->host_norm[k];
  }
  *out = std::sqrt(tot);
  return MG_OK;
}

int ada_residual_norm(mg_ctx* c, double* out) {
  cudaError_t e = c->d == 2 ? ada_residuals<2>(c) : ada_residuals<3>(c);
  if (e != cudaSuccess) return fail(c, MG_ERR_CUDA, std::string("residual: ") + cudaGetErrorString(e));
  return ada_norm_host(c, out);
}

// One cycle as a CUDA graph of one launch per pass, captured when the same
// cycle repeats and updated in place when the factors or the grid change.
int ada_cycle(mg_ctx* c, int hb, int hier, const cplx<double>* omega) {
  HierA& H = *c->ada;
  auto enqueue = [&]() {
    return c->d == 2 ? ada_enqueue_cycle<2>(c, hb, hier, omega) : ada_enqueue_cycle<3>(c, hb, hier, omega);
  };
  cudaError_t e = cudaSuccess;
  if (c->use_graphs && !c->timing) {
    // the boxes live on the device: a captured cycle stays valid while the
    // finest level and the grid capacities stay
    std::vector<double> key = {(double)hb, (double)hier, (double)H.Lf};
    for (int l = 1; l <= c->L; ++l) key.push_back((double)H.gcap[l]);
    for (int l = 0; l < c->L; ++l) {
      key.push_back(omega[l].x);
      key.push_back(omega[l].y);
    }
    const bool fresh = H.exec == nullptr || H.key != key;
    if (fresh && H.seen != key) {
      // a new grid or new factors runs once without a graph: capturing pays
      // off only when the same cycle repeats (a dynamically refined grid
      // changes every step)
      H.seen = key;
    } else if (fresh) {
      cudaStream_t user = c->stream;
      c->stream = c->cap_stream;
      const long long before = c->launches;
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
      cudaError_t ek = e == cudaSuccess ? enqueue() : e;
      cudaError_t ee = e == cudaSuccess ? cudaStreamEndCapture(c->cap_stream, &g) : e;
      c->stream = user;
      const long long nk = c->launches - before;
      c->launches = before;
      e = ek != cudaSuccess ? ek : ee;
      if (e == cudaSuccess) {
        cudaGraphExecUpdateResultInfo info;
        if (H.exec == nullptr || cudaGraphExecUpdate(H.exec, g, &info) != cudaSuccess) {
          cudaGetLastError();
          if (H.exec) cudaGraphExecDestroy(H.exec);
          H.exec = nullptr;
          e = cudaGraphInstantiate(&H.exec, g, 0);
        }
      }
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        cudaGetLastError();
        if (H.exec) cudaGraphExecDestroy(H.exec);
        H.exec = nullptr;
        c->use_graphs = false;
      } else {
        H.key = key;
        H.nkern = nk;
      }
    }
    if (H.exec != nullptr && H.key == key) {
      e = cudaGraphLaunch(H.exec, c->stream);
      c->launches += H.nkern;
      if (e != cudaSuccess) return fail(c, MG_ERR_CUDA, std::string("cycle launch: ") + cudaGetErrorString(e));
      return MG_OK;
    }
  }
  e = enqueue();
  if (e != cudaSuccess) return fail(c, MG_ERR_CUDA, std::string("cycle launch: ") + cudaGetErrorString(e));
  return MG_OK;
}

// The fine-grid function on the uniform finest grid: level 1 interpolated
// up, each level's values written where its cells exist.
template <int D>
cudaError_t ada_composite(mg_ctx* c, cplx<double>* out) {
  HierA& H = *c->ada;
  const int L = c->L;
  cudaError_t e = cudaMemcpyAsync(H.T[0], H.lev[1].u, H.lev[1].nv * sizeof(cplx<double>), cudaMemcpyDeviceToDevice,
                                  c->stream);
  int cur = 0;
  for (int l = 2; l <= L && e == cudaSuccess; ++l) {
    LevA& V = H.lev[l];
    cplx<double>* dst = l == L ? out : H.T[1 - cur];
    c->launches += 2;
    mg::ada_prolong_kernel<D><<<grid_for(V.nv), kThreads, 0, c->stream>>>(V.n, H.T[cur], nullptr, dst, 0);
    mg::ada_overwrite_kernel<D><<<grid_for(V.nv), kThreads, 0, c->stream>>>(V.n, V.vcls, V.u, dst);
    cur = 1 - cur;
    e = cudaGetLastError();
  }
  if (L == 1 && e == cudaSuccess)
    e = cudaMemcpyAsync(out, H.T[0], H.lev[1].nv * sizeof(cplx<double>), cudaMemcpyDeviceToDevice, c->stream);
  return e;
}

// One step of feature-based refinement (Section 5.3), all on the device:
// indicator, span, histogram and bin choice, marks, new cell flags, vertex
// classes with zero-surplus values, diagonals, succ, the new boxes and the
// injection; the counts and boxes are copied to the page-locked mirror.
// Every launch reads its box on the device, so the sequence replays as a
// graph while the finest level and the grid capacities stay.
template <int D>
cudaError_t ada_enqueue_adapt(mg_ctx* c, double refine_frac, double erase_frac, int bins, double veto,
                              int veto_relative, int min_level) {
  HierA& H = *c->ada;
  const int L = c->L, Lf = H.Lf;
  cudaStream_t st = c->stream;
  cudaError_t e;
  // 1. residuals (the veto), indicator, span, histogram, bin choice
  if ((e = cudaMemsetAsync(H.abuf, 0, kAbSlots * sizeof(unsigned long long), st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(H.abuf + kAbMinMax, 0xff, sizeof(unsigned long long), st)) != cudaSuccess) return e;
  if ((e = ada_residuals<D>(c)) != cudaSuccess) return e;
  for (int l = 1; l <= Lf; ++l) {
    LevA& V = H.lev[l];
    ++c->launches;
    mg::ada_indicator_kernel<D><<<H.gcap[l], kThreads, 0, st>>>(V.n, V.u, V.vcls,
                                                                l < Lf ? H.lev[l + 1].vcls : nullptr, V.s,
                                                                H.boxes + l, H.abuf + kAbMinMax, H.abuf + kAbCount);
  }
  for (int l = 1; l <= Lf; ++l) {
    LevA& V = H.lev[l];
    ++c->launches;
    mg::ada_hist_kernel<D><<<H.gcap[l], kThreads, 0, st>>>(V.n, V.s, H.boxes + l, H.abuf + kAbMinMax, bins,
                                                           H.abuf + kAbCounts);
  }
  int* kb = reinterpret_cast<int*>(H.abuf + kAbBins);
  ++c->launches;
  mg::ada_choose_bins_kernel<<<1, 32, 0, st>>>(H.abuf + kAbCounts, H.abuf + kAbCount, H.abuf + kAbMinMax, bins,
                                               refine_frac, erase_frac, kb);
  // 2. marks (zero on entry: the kernels that consume them clear them)
  for (int l = 1; l <= Lf; ++l) {
    LevA& V = H.lev[l];
    ++c->launches;
    mg::ada_mark_kernel<D><<<H.gcap[l], kThreads, 0, st>>>(V.n, V.s, V.r, V.invd, H.boxes + l, H.abuf + kAbMinMax,
                                                           V.u, bins, kb, veto, veto_relative, l < L ? 1 : 0,
                                                           l >= min_level + 1 ? 1 : 0, V.rmark, V.emark,
                                                           H.abuf + kAbSel);
  }
  // 3. new refine bits fine to coarse, then existence coarse to fine
  for (int l = std::min(Lf, L - 1); l >= 1; --l) {
    LevA& V = H.lev[l];
    const LevA& F = H.lev[l + 1];
    ++c->launches;
    mg::ada_coarsen_kernel<D><<<grid_for((size_t)ipow(V.n, D)), kThreads, 0, st>>>(
        V.n, V.cellf, V.rmark, F.cellf, l + 1 < L ? F.rmark : nullptr, F.vcls,
        l + 2 <= L ? H.lev[l + 2].vcls : nullptr, F.emark, l >= min_level ? 1 : 0, H.boxes + l);
  }
  const int Lt = std::min(Lf + 1, L);  // levels that may hold cells after the step
  for (int l = 1; l <= Lt; ++l) {
    LevA& V = H.lev[l];
    ++c->launches;
    mg::ada_finalize_cells_kernel<D><<<grid_for((size_t)ipow(V.n, D)), kThreads, 0, st>>>(
        V.n, V.cellf, l > 1 ? H.lev[l - 1].cellf : nullptr, V.rmark, l > 1 ? H.boxes + (l - 1) : nullptr);
  }
  // 4. vertex classes and zero-surplus values coarse to fine, boxes
  ++c->launches;
  mg::ada_box_init_kernel<<<1, 128, 0, st>>>(H.box6, L + 1);
  // (the old boxes are read until ada_boxes_kernel replaces them)
  for (int l = 1; l <= Lt; ++l) {
    LevA& V = H.lev[l];
    ++c->launches;
    mg::ada_reclass_kernel<D><<<grid_for(V.nv), kThreads, 0, st>>>(
        V.n, V.cellf, V.vcls, V.u, l > 1 ? H.lev[l - 1].u : nullptr, H.box6 + 6 * l, V.emark, V.r,
        l > 1 ? H.boxes + (l - 1) : nullptr);
  }
  ++c->launches;
  mg::ada_boxes_kernel<D><<<1, 32, 0, st>>>(H.box6, L, H.boxes);
  for (int l = 1; l <= Lt; ++l) {
    LevA& V = H.lev[l];
    ++c->launches;
    mg::ada_diag_kernel<D><<<grid_for(V.nv), kThreads, 0, st>>>(V.n, V.vcls, V.hcell, V.hinv, V.phic, c->k2[0],
                                                                V.invd, H.boxes + l);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = ada_succ_all<D>(c, H.abuf + kAbFine)) != cudaSuccess) return e;
  // 5. coarse copies of finer unknowns (fine to coarse) over the new boxes
  for (int l = Lt - 1; l >= 1; --l) {
    LevA& V = H.lev[l];
    ++c->launches;
    mg::ada_inject_unknown_kernel<D><<<grid_for(V.nv), kThreads, 0, st>>>(V.n, H.lev[l + 1].vcls,
                                                                          H.lev[l + 1].u, V.u, H.boxes + l);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(H.hbuf, H.abuf, kAbSlots * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st)) !=
      cudaSuccess)
    return e;
  return cudaMemcpyAsync(static_cast<char*>(H.hbuf) + 2048, H.box6, 6 * (L + 1) * sizeof(int),
                         cudaMemcpyDeviceToHost, st);
}

// Runs one step (directly the first time, then as a graph while the same
// step repeats on the same finest level and capacities), synchronises, and
// takes the new boxes: finest level, grid capacities (grown when a box
// outgrows its grid).  stats: vertices selected for refining and erasing,
// fine-grid vertices after the step, finest level with cells.
template <int D>
int ada_adapt(mg_ctx* c, double refine_frac, double erase_frac, int bins, double veto, int veto_relative,
              int min_level, long long* stats) {
  HierA& H = *c->ada;
  const int L = c->L;
  auto enqueue = [&]() {
    return ada_enqueue_adapt<D>(c, refine_frac, erase_frac, bins, veto, veto_relative, min_level);
  };
  std::vector<double> key = {refine_frac, erase_frac, (double)bins, veto, (double)veto_relative,
                             (double)min_level, (double)H.Lf};
  for (int l = 1; l <= L; ++l) key.push_back((double)H.gcap[l]);
  bool launched = false;
  if (c->use_graphs) {
    const bool fresh = H.aexec == nullptr || H.akey != key;
    if (fresh && H.aseen != key) {
      H.aseen = key;  // first time: run directly
    } else if (fresh) {
      cudaStream_t user = c->stream;
      c->stream = c->cap_stream;
      const long long before = c->launches;
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
      cudaError_t ek = e == cudaSuccess ? enqueue() : e;
      cudaError_t ee = e == cudaSuccess ? cudaStreamEndCapture(c->cap_stream, &g) : e;
      c->stream = user;
      const long long nk = c->launches - before;
      c->launches = before;
      e = ek != cudaSuccess ? ek : ee;
      if (e == cudaSuccess) {
        cudaGraphExecUpdateResultInfo info;
        if (H.aexec == nullptr || cudaGraphExecUpdate(H.aexec, g, &info) != cudaSuccess) {
          cudaGetLastError();
          if (H.aexec) cudaGraphExecDestroy(H.aexec);
          H.aexec = nullptr;
          e = cudaGraphInstantiate(&H.aexec, g, 0);
        }
      }
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        cudaGetLastError();
        if (H.aexec) cudaGraphExecDestroy(H.aexec);
        H.aexec = nullptr;
      } else {
        H.akey = key;
        H.ankern = nk;
      }
    }
    if (H.aexec != nullptr && H.akey == key) {
      MG_CUDA(c, cudaGraphLaunch(H.aexec, c->stream));
      c->launches += H.ankern;
      launched = true;
    }
  }
  if (!launched) MG_CUDA(c, enqueue());
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  const unsigned long long* hb = static_cast<const unsigned long long*>(H.hbuf);
  const int* bx = reinterpret_cast<const int*>(static_cast<const char*>(H.hbuf) + 2048);
  H.Lf = 1;
  for (int l = 1; l <= L; ++l) {
    LevA& V = H.lev[l];
    const bool empty = bx[6 * l + 3] < 0;
    V.boxvol = 1;
    for (int a = 0; a < 3; ++a) {
      V.box.lo[a] = a < D && !empty ? bx[6 * l + a] : 0;
      V.box.ext[a] = empty ? 0 : (a < D ? bx[6 * l + 3 + a] - bx[6 * l + a] + 1 : 1);
      V.boxvol *= (size_t)V.box.ext[a];
    }
    if (!empty) H.Lf = l;
    const int need = grid_for(V.boxvol);
    if (need > H.gcap[l]) H.gcap[l] = std::min(152 * 16, std::max(need, 2 * H.gcap[l]));
  }
  double hi;
  std::memcpy(&hi, hb + kAbMinMax + 1, sizeof hi);
  stats[0] = (long long)hb[kAbSel];
  stats[1] = (long long)hb[kAbSel + 1];
  stats[2] = (long long)hb[kAbFine];
  stats[3] = H.Lf;
  return hb[kAbCount] != 0 && !std::isfinite(hi) ? MG_DIVERGED : MG_OK;  // a non-finite span selects nothing
}

const char* kNot4 = " is not available for d = 4 (the four-dimensional path runs complex128 cycles)";
const char* kNotA = " is not available for an adaptive grid (mg_create_adaptive contexts run complex128 cycles)";

}  // namespace

// =========================================================================
extern "C" {

int mg_create(int d, int depth, const double* k2_field, double theta, double layer_width,
              mg_ctx** out) {
  g_create_err.clear();
  if (!(layer_width >= 0.0 && layer_width <= 0.5)) {
    if (out != nullptr) *out = nullptr;
    return fail(nullptr, MG_ERR_INVALID, "layer_width must be in [0, 0.5]");
  }
  return mg_create_ecs(d, depth, k2_field, theta, 0.0, layer_width, layer_width, out);
}

static int create_ctx(int d, int depth, const double* k2_field, double theta_layer, double theta_interior,
                      double width_lo, double width_hi, const unsigned char* refine, mg_ctx** out) {
  g_create_err.clear();
  if (out == nullptr) return fail(nullptr, MG_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (d != 2 && d != 3 && d != 4) return fail(nullptr, MG_ERR_INVALID, "d must be 2, 3 or 4");
  if (depth < 1 || depth > (d == 2 ? kMaxDepth2 : (d == 3 ? kMaxDepth3 : kMaxDepth4)))
    return fail(nullptr, MG_ERR_INVALID, "depth out of range");
  if (k2_field == nullptr) return fail(nullptr, MG_ERR_INVALID, "k2_field is NULL");
  if (!(theta_layer >= 0.0 && theta_layer < M_PI / 2))
    return fail(nullptr, MG_ERR_INVALID, "theta must be in [0, pi/2)");
  if (!(theta_interior >= 0.0 && theta_interior < M_PI / 2))
    return fail(nullptr, MG_ERR_INVALID, "theta_interior must be in [0, pi/2)");
  if (!(width_lo >= 0.0 && width_lo <= 1.0 && width_hi >= 0.0 && width_hi <= 1.0))
    return fail(nullptr, MG_ERR_INVALID, "layer widths must be in [0, 1]");
  const size_t nvf = (size_t)ipow(ipow(3, depth) + 1, d);
  for (size_t i = 0; i < nvf; ++i)
    if (!std::isfinite(k2_field[i])) return fail(nullptr, MG_ERR_INVALID, "k2_field holds a non-finite value");
  if (d == 4)
    for (size_t i = 1; i < nvf; ++i)
      if (k2_field[i] != k2_field[0])
        return fail(nullptr, MG_ERR_INVALID, "d = 4 takes a constant k2_field (separable operator)");
  // memory estimate: 5 fine-size c128 arrays per level plus scratch and f
  // (d = 4: 4 level arrays and 5 temporaries)
  {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return fail(nullptr, MG_ERR_CUDA, "cudaMemGetInfo failed");
    const double need = (double)nvf * 16.0 * (d == 4 ? 9.0 : 5.0) * 1.2 + (double)nvf * 32.0;
    if (need > (double)fr) return fail(nullptr, MG_ERR_OOM, "grid too large for free device memory");
  }
  mg_ctx* c = new (std::nothrow) mg_ctx();
  if (c != nullptr && cudaGetDevice(&c->device) != cudaSuccess) c->device = -1;
  if (c == nullptr) return fail(nullptr, MG_ERR_OOM, "host allocation failed");
  c->d = d;
  c->L = depth;
  c->theta = theta_layer;
  c->theta_in = theta_interior;
  c->wlo = width_lo;
  c->whi = width_hi;
  c->k2.assign(k2_field, k2_field + nvf);
  int rc = refine != nullptr ? ada_build(c, refine)
                              : (d == 4 ? d4_build<double>(c, c->h4) : build_hier<double>(c, c->h64));
  if (rc == MG_OK) {
    cudaError_t e = cudaMalloc(&c->f_dev, nvf * sizeof(cplx<double>));
    if (e == cudaSuccess) e = cudaMemset(c->f_dev, 0, nvf * sizeof(cplx<double>));
    if (e == cudaSuccess && d != 4) e = cudaMalloc(&c->scratch, nvf * sizeof(cplx<double>));  // d = 4 uses its own temporaries
    if (e == cudaSuccess) e = cudaMallocHost(&c->host_norm, 4 * sizeof(double));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = configure_kernels();
    if (e == cudaSuccess) e = cudaMalloc(&c->chain_ctr, 64 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(c->chain_ctr, 0, 64 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&c->dev_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(c->dev_err, 0, sizeof(unsigned));
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->chain_bpsm, mg::chain2_kernel<256>, 256,
                                                         mg::Tile2<4>::smem_bytes);
    if (e != cudaSuccess) rc = fail(c, MG_ERR_OOM, cudaGetErrorString(e));
  }
  if (rc != MG_OK) {
    g_create_err = c->err;
    mg_destroy(c);
    return rc;
  }
  *out = c;
  return MG_OK;
}

int mg_create_ecs(int d, int depth, const double* k2_field, double theta_layer, double theta_interior,
                  double width_lo, double width_hi, mg_ctx** out) {
  return create_ctx(d, depth, k2_field, theta_layer, theta_interior, width_lo, width_hi, nullptr, out);
}

int mg_create_adaptive(int d, int depth, const double* k2_field, double theta_layer, double theta_interior,
                       double width_lo, double width_hi, const unsigned char* refine, mg_ctx** out) {
  g_create_err.clear();
  if (out != nullptr) *out = nullptr;
  if (refine == nullptr) return fail(nullptr, MG_ERR_INVALID, "refine is NULL");
  if (d != 2 && d != 3) return fail(nullptr, MG_ERR_INVALID, "an adaptive grid takes d = 2 or 3");
  return create_ctx(d, depth, k2_field, theta_layer, theta_interior, width_lo, width_hi, refine, out);
}

int mg_adapt(mg_ctx* c, double refine_frac, double erase_frac, int bins, double veto, int veto_relative,
             int min_level, long long* stats) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  if (c->ada == nullptr) return fail(c, MG_ERR_INVALID, "mg_adapt takes an adaptive context (mg_create_adaptive)");
  if (!(refine_frac >= 0.0 && refine_frac <= 1.0 && erase_frac >= 0.0 && erase_frac <= 1.0))
    return fail(c, MG_ERR_INVALID, "refine_frac and erase_frac must be in [0, 1]");
  if (bins < 1 || bins > 64) return fail(c, MG_ERR_INVALID, "bins must be in [1, 64]");
  if (!(veto > 0.0)) return fail(c, MG_ERR_INVALID, "veto must be > 0");
  if (min_level < 1 || min_level > c->L) return fail(c, MG_ERR_INVALID, "min_level must be in [1, depth]");
  long long st[4] = {0, 0, 0, 0};
  const int rc = c->d == 2 ? ada_adapt<2>(c, refine_frac, erase_frac, bins, veto, veto_relative != 0, min_level, st)
                           : ada_adapt<3>(c, refine_frac, erase_frac, bins, veto, veto_relative != 0, min_level, st);
  if (rc != MG_OK && rc != MG_DIVERGED) return rc;
  if (stats != nullptr) std::memcpy(stats, st, sizeof st);
  return rc;
}

int mg_get_refinement(mg_ctx* c, unsigned char* refine) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  if (c->ada == nullptr) return fail(c, MG_ERR_INVALID, "mg_get_refinement takes an adaptive context");
  if (refine == nullptr) return fail(c, MG_ERR_INVALID, "refine is NULL");
  HierA& H = *c->ada;
  size_t off = 0;
  std::vector<uint8_t> fl;
  for (int l = 1; l < c->L; ++l) {
    const size_t ncell = (size_t)ipow(H.lev[l].n, c->d);
    fl.resize(ncell);
    MG_CUDA(c, cudaMemcpyAsync(fl.data(), H.lev[l].cellf, ncell, cudaMemcpyDeviceToHost, c->stream));
    MG_CUDA(c, cudaStreamSynchronize(c->stream));
    for (size_t i = 0; i < ncell; ++i) refine[off + i] = (fl[i] & mg::kCellRefined) ? 1 : 0;
    off += ncell;
  }
  return MG_OK;
}

void mg_destroy(mg_ctx* c) {
  if (c == nullptr) return;
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->trace) cudaFree(c->trace);
  if (c->chain_ctr) cudaFree(c->chain_ctr);
  if (c->dev_err) cudaFree(c->dev_err);
  free_hier(c->h64);
  free_hier(c->h32);
  d4_free(c->h4);
  d4_free(c->h4f);
  ada_free(c->ada);
  if (c->f_dev) cudaFree(c->f_dev);
  if (c->scratch) cudaFree(c->scratch);
  if (c->k2dev) cudaFree(c->k2dev);
  if (c->rvec) cudaFree(c->rvec);
  if (c->host_norm) cudaFreeHost(c->host_norm);
  delete c;
}

int mg_set_stream(mg_ctx* c, void* s) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  c->stream = (cudaStream_t)s;
  return MG_OK;
}

int mg_set_rhs(mg_ctx* c, const mg_c128* f, int on_device) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  if (f == nullptr) return fail(c, MG_ERR_INVALID, "f is NULL");
  if (c->ada != nullptr) {
    HierA& H = *c->ada;
    const LevA& F = H.lev[c->L];
    MG_CUDA(c, cudaMemcpyAsync(F.f, f, F.nv * sizeof(mg_c128),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    for (int l = c->L - 1; l >= 1; --l) {
      ++c->launches;
      if (c->d == 2)
        mg::ada_inject_kernel<2><<<grid_for(H.lev[l].nv), kThreads, 0, c->stream>>>(H.lev[l].n, H.lev[l + 1].f,
                                                                                   H.lev[l].f);
      else
        mg::ada_inject_kernel<3><<<grid_for(H.lev[l].nv), kThreads, 0, c->stream>>>(H.lev[l].n, H.lev[l + 1].f,
                                                                                   H.lev[l].f);
    }
    MG_CUDA(c, cudaGetLastError());
    c->r0 = -1.0;
    return MG_OK;
  }
  const size_t nv = c->d == 4 ? c->h4->lev[c->L].nv : c->h64.lev[c->L].nv;
  const cplx<double>* fv = on_device ? nullptr : pinned_view(reinterpret_cast<const cplx<double>*>(f));
  if (fv != nullptr && c->d == 3) {
    // the z-pass of b = M f copies f on its way (one pass over the host link)
    int rc = set_level_rhs(c, c->L, fv);
    if (rc != MG_OK) return rc;
    c->r0 = -1.0;
    return MG_OK;
  }
  if (fv != nullptr) {
    ++c->launches;
    mg::copy_c128_kernel<<<grid_for(nv), kThreads, 0, c->stream>>>((long long)nv, fv, c->f_dev);
    MG_CUDA(c, cudaGetLastError());
  } else {
    MG_CUDA(c, cudaMemcpyAsync(c->f_dev, f, nv * sizeof(mg_c128),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  }
  if (c->d == 4) {
    MG_CUDA(c, d4_mass(c, c->f_dev, c->h4->lev[c->L].b));
    c->r0 = -1.0;
    return MG_OK;
  }
  int rc = set_level_rhs(c, c->L);
  if (rc != MG_OK) return rc;
  c->r0 = -1.0;
  return MG_OK;
}

int mg_set_solution(mg_ctx* c, const mg_c128* u, int on_device) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  if (u == nullptr) return fail(c, MG_ERR_INVALID, "u is NULL");
  if (c->ada != nullptr) {
    // the uniform fine-grid samples on every level, then the invariants
    HierA& H = *c->ada;
    const LevA& F = H.lev[c->L];
    MG_CUDA(c, cudaMemcpyAsync(F.u, u, F.nv * sizeof(mg_c128),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    for (int l = c->L; l >= 1; --l) {
      const LevA& V = H.lev[l];
      if (l < c->L) {
        ++c->launches;
        if (c->d == 2)
          mg::ada_inject_kernel<2><<<grid_for(V.nv), kThreads, 0, c->stream>>>(V.n, H.lev[l + 1].u, V.u);
        else
          mg::ada_inject_kernel<3><<<grid_for(V.nv), kThreads, 0, c->stream>>>(V.n, H.lev[l + 1].u, V.u);
      }
    }
    for (int l = 1; l <= c->L; ++l) {
      const LevA& V = H.lev[l];
      const int ring = c->d == 2 ? 4 * V.n : 6 * (V.n + 1) * (V.n + 1);
      ++c->launches;
      if (c->d == 2)
        mg::zero_ring_kernel<2><<<(ring + 255) / 256, 256, 0, c->stream>>>(V.n, V.u);
      else
        mg::zero_ring_kernel<3><<<(ring + 255) / 256, 256, 0, c->stream>>>(V.n, V.u);
    }
    MG_CUDA(c, c->d == 2 ? ada_invariants<2>(c) : ada_invariants<3>(c));
    c->r0 = -1.0;
    return MG_OK;
  }
  if (c->d == 4) {
    const Lev4<double>& V = c->h4->lev[c->L];
    MG_CUDA(c, cudaMemcpyAsync(V.u, u, V.nv * sizeof(mg_c128),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    ++c->launches;
    mg::update4_kernel<double, double><<<grid_for(V.nv), kThreads, 0, c->stream>>>(V.n, V.u, (const cplx<double>*)nullptr);  // zero boundary
    MG_CUDA(c, cudaGetLastError());
    c->r0 = -1.0;
    return MG_OK;
  }
  auto& H = c->h64;
  auto& V = H.lev[c->L];
  const cplx<double>* uv = on_device ? nullptr : pinned_view(reinterpret_cast<const cplx<double>*>(u));
  ++c->launches;
  if (uv != nullptr) {
    // page-locked host buffer: read over the host link, ring zeroed on the way
    if (c->d == 2)
      mg::copy_zero_ring_kernel<2><<<grid_for(V.nv), kThreads, 0, c->stream>>>(V.n, uv, V.u[H.cur]);
    else
      mg::copy_zero_ring_kernel<3><<<grid_for(V.nv), kThreads, 0, c->stream>>>(V.n, uv, V.u[H.cur]);
  } else {
    // copy into the active fine array, then zero its Dirichlet ring
    MG_CUDA(c, cudaMemcpyAsync(V.u[H.cur], u, V.nv * sizeof(mg_c128),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    const int ring = c->d == 2 ? 4 * V.n : 6 * (V.n + 1) * (V.n + 1);
    if (c->d == 2)
      mg::zero_ring_kernel<2><<<(ring + 255) / 256, 256, 0, c->stream>>>(V.n, V.u[H.cur]);
    else
      mg::zero_ring_kernel<3><<<(ring + 255) / 256, 256, 0, c->stream>>>(V.n, V.u[H.cur]);
  }
  MG_CUDA(c, cudaGetLastError());
  int rc = zero_pending(c, H, c->L);
  if (rc != MG_OK) return rc;
  c->r0 = -1.0;
  return MG_OK;
}

int mg_get_solution(mg_ctx* c, mg_c128* out, int on_device) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  if (out == nullptr) return fail(c, MG_ERR_INVALID, "out is NULL");
  if (c->ada != nullptr) {
    const size_t nv = c->ada->lev[c->L].nv;
    if (on_device) {
      MG_CUDA(c, c->d == 2 ? ada_composite<2>(c, (cplx<double>*)out) : ada_composite<3>(c, (cplx<double>*)out));
      return MG_OK;
    }
    MG_CUDA(c, c->d == 2 ? ada_composite<2>(c, c->scratch) : ada_composite<3>(c, c->scratch));
    MG_CUDA(c, cudaMemcpyAsync(out, c->scratch, nv * sizeof(mg_c128), cudaMemcpyDeviceToHost, c->stream));
    MG_CUDA(c, cudaStreamSynchronize(c->stream));
    return MG_OK;
  }
  if (c->d == 4) {
    const Lev4<double>& V = c->h4->lev[c->L];
    MG_CUDA(c, cudaMemcpyAsync(out, V.u, V.nv * sizeof(mg_c128),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (!on_device) MG_CUDA(c, cudaStreamSynchronize(c->stream));
    return MG_OK;
  }
  auto& H = c->h64;
  const size_t nv = H.lev[c->L].nv;
  if (on_device) {
    MG_CUDA(c, materialize(c, H, c->L, (cplx<double>*)out));
    return MG_OK;
  }
  if (cplx<double>* ov = pinned_view(reinterpret_cast<cplx<double>*>(out))) {
    // page-locked host buffer: U + P corr written straight over the host link
    MG_CUDA(c, materialize(c, H, c->L, ov));
    MG_CUDA(c, cudaStreamSynchronize(c->stream));
    return MG_OK;
  }
  MG_CUDA(c, materialize(c, H, c->L, c->scratch));
  MG_CUDA(c, cudaMemcpyAsync(out, c->scratch, nv * sizeof(mg_c128), cudaMemcpyDeviceToHost, c->stream));
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  return MG_OK;
}

int mg_get_level(mg_ctx* c, int level, int which, mg_c128* out, int on_device) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  if (out == nullptr || level < 1 || level > c->L || (which != 0 && which != 1))
    return fail(c, MG_ERR_INVALID, "bad level/which/out");
  if (c->ada != nullptr) {
    // which = 0: the level's values, 1: its generating-system residual
    const LevA& V = c->ada->lev[level];
    MG_CUDA(c, cudaMemcpyAsync(out, which == 0 ? V.u : V.r, V.nv * sizeof(mg_c128),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (!on_device) MG_CUDA(c, cudaStreamSynchronize(c->stream));
    return MG_OK;
  }
  if (level == c->L && which == 0) return mg_get_solution(c, out, on_device);
  if (c->d == 4) {
    const Lev4<double>& V = c->h4->lev[level];
    MG_CUDA(c, cudaMemcpyAsync(out, which == 0 ? V.u : V.b, V.nv * sizeof(mg_c128),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (!on_device) MG_CUDA(c, cudaStreamSynchronize(c->stream));
    return MG_OK;
  }
  auto& V = c->h64.lev[level];
  const void* src = which == 0 ? (const void*)V.u[0] : (const void*)V.b;
  MG_CUDA(c, cudaMemcpyAsync(out, src, V.nv * sizeof(mg_c128),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  if (!on_device) MG_CUDA(c, cudaStreamSynchronize(c->stream));
  return MG_OK;
}

int mg_cycle(mg_ctx* c, int variant, const mg_c128* omega, int transfer) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  if (omega == nullptr) return fail(c, MG_ERR_INVALID, "omega is NULL");
  int hb, hier;
  if (decode_variant(c, variant, transfer, &hb, &hier)) return MG_ERR_INVALID;
  if (c->ada != nullptr) return ada_cycle(c, hb, hier, reinterpret_cast<const cplx<double>*>(omega));
  if (c->d == 4) return d4_cycle(c, *c->h4, hb, hier, reinterpret_cast<const cplx<double>*>(omega));
  return run_cycle(c, c->h64, c->L, hb, hier, reinterpret_cast<const cplx<double>*>(omega));
}

int mg_residual_norm(mg_ctx* c, double* abs_l2, double* rel_l2) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  int rc = ensure_r0(c);
  if (rc != MG_OK) return rc;
  double r;
  if ((rc = fine_residual(c, c->L, &r)) != MG_OK) return rc;
  if (abs_l2) *abs_l2 = r;
  if (rel_l2) *rel_l2 = c->r0 > 0 ? r / c->r0 : 0.0;
  return MG_OK;
}

int mg_residual_max(mg_ctx* c, double* abs_max) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  if (abs_max == nullptr) return fail(c, MG_ERR_INVALID, "abs_max is NULL");
  if (c->ada != nullptr) {
    // max |r| over the fine-grid vertices, fused into the residual pass
    HierA& H = *c->ada;
    MG_CUDA(c, cudaMemsetAsync(H.abuf + kAbMax, 0, kAdaMaxSlots * sizeof(unsigned long long), c->stream));
    MG_CUDA(c, c->d == 2 ? ada_residuals<2>(c, true) : ada_residuals<3>(c, true));
    MG_CUDA(c, cudaMemcpyAsync(H.hbuf, H.abuf + kAbMax, kAdaMaxSlots * sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, c->stream));
    MG_CUDA(c, cudaStreamSynchronize(c->stream));
    const unsigned long long* b = static_cast<const unsigned long long*>(H.hbuf);
    unsigned long long m = 0;
    for (int l = 1; l <= H.Lf; ++l) m = std::max(m, b[l]);
    double v;
    std::memcpy(&v, &m, sizeof v);
    *abs_max = v;
    return MG_OK;
  }
  if (c->d == 4) {
    Hier4<double>& H4 = *c->h4;
    unsigned long long* mx = reinterpret_cast<unsigned long long*>(H4.norm2 + 2);
    MG_CUDA(c, d4_residual(c, -1));
    MG_CUDA(c, cudaMemsetAsync(mx, 0, sizeof(unsigned long long), c->stream));
    ++c->launches;
    const size_t nv = H4.lev[c->L].nv;
    mg::max_abs_kernel<<<grid_for(nv), kThreads, 0, c->stream>>>(H4.T[4], (long long)nv, mx);
    MG_CUDA(c, cudaGetLastError());
    MG_CUDA(c, cudaMemcpyAsync(c->host_norm, mx, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    MG_CUDA(c, cudaStreamSynchronize(c->stream));
    *abs_max = *c->host_norm;
    return MG_OK;
  }
  auto& H = c->h64;
  auto& V = H.lev[c->L];
  if (c->rvec == nullptr) MG_CUDA(c, cudaMalloc(&c->rvec, V.nv * sizeof(cplx<double>)));
  unsigned long long* mx = reinterpret_cast<unsigned long long*>(H.norm2 + 2);
  MG_CUDA(c, materialize(c, H, c->L, c->scratch));
  MG_CUDA(c, (stencil<double, double>(c, H, c->L, 1, c->scratch, V.b, V.coefH, true, c->rvec, -1)));
  MG_CUDA(c, cudaMemsetAsync(mx, 0, sizeof(unsigned long long), c->stream));
  ++c->launches;
  mg::max_abs_kernel<<<grid_for(V.nv), kThreads, 0, c->stream>>>(c->rvec, (long long)V.nv, mx);
  MG_CUDA(c, cudaGetLastError());
  MG_CUDA(c, cudaMemcpyAsync(c->host_norm, mx, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  *abs_max = *c->host_norm;
  return check_timeout(c);
}

int mg_set_precision(mg_ctx* c, int precision, int inner_cycles) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  if (precision != MG_C128 && precision != MG_C64_REFINE) return fail(c, MG_ERR_INVALID, "bad precision");
  if (inner_cycles < 1 || inner_cycles > 1000) return fail(c, MG_ERR_INVALID, "inner_cycles out of range");
  if (c->ada != nullptr && precision != MG_C128) return fail(c, MG_ERR_INVALID, std::string("MG_C64_REFINE") + kNotA);
  c->precision = precision;
  c->inner_cycles = inner_cycles;
  if (c->d == 4) {
    if (precision == MG_C64_REFINE && c->h4f == nullptr) {
      int rc = d4_build<float>(c, c->h4f);
      if (rc != MG_OK) {
        d4_free(c->h4f);
        c->h4f = nullptr;
        c->precision = MG_C128;
        return rc;
      }
    }
    return MG_OK;
  }
  if (precision == MG_C64_REFINE && !c->h32.ready) {
    int rc = build_hier<float>(c, c->h32);
    if (rc != MG_OK) { free_hier(c->h32); return rc; }
  }
  return MG_OK;
}

int mg_solve(mg_ctx* c, int variant, const mg_c128* omega, int transfer, double tol, int max_cycles,
             int* cycles_done, double* rel_res) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  if (omega == nullptr) return fail(c, MG_ERR_INVALID, "omega is NULL");
  if (!(tol > 0) || max_cycles < 0) return fail(c, MG_ERR_INVALID, "tol must be > 0 and max_cycles >= 0");
  int hb, hier;
  if (decode_variant(c, variant, transfer, &hb, &hier)) return MG_ERR_INVALID;
  const cplx<double>* om = reinterpret_cast<const cplx<double>*>(omega);
  int rc = ensure_r0(c);
  if (rc != MG_OK) return rc;
  const int L = c->L;
  int done = 0;
  double rel = 0;
  {
    double r;
    if ((rc = fine_residual(c, L, &r)) != MG_OK) return rc;
    rel = c->r0 > 0 ? r / c->r0 : 0.0;
  }
  auto finish = [&](int status) {
    if (cycles_done) *cycles_done = done;
    if (rel_res) *rel_res = rel;
    return status;
  };
  auto diverged = [&](double x) { return !std::isfinite(x) || x > 1e6; };
  if (c->precision == MG_C128) {
    // fused norm of the iterate entering each cycle, read every few cycles
    const int check = std::max(1, std::min(8, max_cycles / 8));
    while (true) {
      if (diverged(rel)) return finish(MG_DIVERGED);
      if (rel <= tol) return finish(MG_OK);
      if (done >= max_cycles) return finish(MG_NOT_CONVERGED);
      const int m = std::min(check, max_cycles - done);
      for (int k = 0; k < m; ++k) {
        rc = c->ada != nullptr ? ada_cycle(c, hb, hier, om)
                               : (c->d == 4 ? d4_cycle(c, *c->h4, hb, hier, om) : run_cycle(c, c->h64, L, hb, hier, om));
        if (rc != MG_OK) return rc;
        ++done;
      }
      if (c->ada != nullptr) {
        // the residual of the iterate that entered the last cycle
        double r;
        if ((rc = ada_norm_host(c, &r)) != MG_OK) return rc;
        const double prev = r / (c->r0 > 0 ? c->r0 : 1.0);
        if (diverged(prev) || prev <= tol || done >= max_cycles) {
          if ((rc = fine_residual(c, L, &r)) != MG_OK) return rc;
          rel = c->r0 > 0 ? r / c->r0 : 0.0;
        } else {
          rel = prev;
        }
        continue;
      }
      MG_CUDA(c, cudaMemcpyAsync(c->host_norm, c->d == 4 ? c->h4->norm2 : c->h64.norm2, sizeof(double),
                                 cudaMemcpyDeviceToHost, c->stream));
      MG_CUDA(c, cudaStreamSynchronize(c->stream));
      if ((rc = check_timeout(c)) != MG_OK) return finish(rc);
      const double prev = std::sqrt(*c->host_norm) / (c->r0 > 0 ? c->r0 : 1.0);
      if (diverged(prev) || prev <= tol || done >= max_cycles) {
        double r;
        if ((rc = fine_residual(c, L, &r)) != MG_OK) return rc;
        rel = c->r0 > 0 ? r / c->r0 : 0.0;
      } else {
        rel = prev;  // residual of the iterate that entered the last cycle
      }
    }
  }
  // complex64 cycles inside FP64 defect correction
  if (c->d == 4) {
    const int st = d4_refine(c, hb, hier, om, tol, max_cycles, &done, &rel);
    if (st == MG_OK || st == MG_DIVERGED || st == MG_NOT_CONVERGED) return finish(st);
    return st;
  }
  auto& H = c->h64;
  auto& E = c->h32;
  auto& VF = H.lev[L];
  auto& EF = E.lev[L];
  cplx<double>* u = VF.u[H.cur];
  // u must be materialised: fold any pending correction into U
  MG_CUDA(c, materialize(c, H, L, c->scratch));
  MG_CUDA(c, cudaMemcpyAsync(u, c->scratch, VF.nv * sizeof(cplx<double>), cudaMemcpyDeviceToDevice, c->stream));
  if ((rc = zero_pending(c, H, L)) != MG_OK) return rc;
  const bool fused = use_defect3(c);
  if (fused) {
    // r = b - H u in FP64 as the complex64 rhs of the first inner problem
    MG_CUDA(c, (defect3<float>(c, L, u, nullptr, nullptr, nullptr, EF.b, -1)));
  }
  while (true) {
    if (diverged(rel)) return finish(MG_DIVERGED);
    if (rel <= tol) return finish(MG_OK);
    if (done >= max_cycles) return finish(MG_NOT_CONVERGED);
    // r = b - H u in FP64, stored as complex64 rhs of the inner problem
    if (!fused) MG_CUDA(c, (stencil<double, float>(c, H, L, 1, u, VF.b, VF.coefH, true, EF.b, -1)));
    MG_CUDA(c, cudaMemsetAsync(EF.u[E.cur], 0, EF.nv * sizeof(cplx<float>), c->stream));
    for (int l = 1; l < L; ++l) {
      MG_CUDA(c, cudaMemsetAsync(E.lev[l].corr, 0, E.lev[l].nv * sizeof(cplx<float>), c->stream));
      MG_CUDA(c, cudaMemsetAsync(E.lev[l].t, 0, E.lev[l].nv * sizeof(cplx<float>), c->stream));
    }
    const int m = std::min(c->inner_cycles, std::max(1, max_cycles - done));
    for (int k = 0; k < m; ++k) {
      if ((rc = run_cycle(c, E, L, hb, hier, om)) != MG_OK) return rc;
      ++done;
    }
    // u += E + P corr (FP64 update)
    const cplx<float>* cc = L > 1 ? E.lev[L - 1].corr : nullptr;
    if (fused) {
      // u' = u + E + P corr, the next inner rhs r = b - H u' and |r|^2 in one pass
      cplx<double>* u2 = VF.u[1 - H.cur];
      MG_CUDA(c, (defect3<float>(c, L, u, EF.u[E.cur], cc, u2, EF.b, 1)));
      H.cur = 1 - H.cur;
      u = u2;
      MG_CUDA(c, cudaMemcpyAsync(c->host_norm, H.norm2 + 1, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      MG_CUDA(c, cudaStreamSynchronize(c->stream));
      rel = c->r0 > 0 ? std::sqrt(*c->host_norm) / c->r0 : 0.0;
      continue;
    }
    ++c->launches;
    if (c->d == 2)
      mg::update_kernel<float, 2><<<grid_for(VF.nv), kThreads, 0, c->stream>>>(VF.n, u, EF.u[E.cur], cc);
    else
      mg::update_kernel<float, 3><<<grid_for(VF.nv), kThreads, 0, c->stream>>>(VF.n, u, EF.u[E.cur], cc);
    MG_CUDA(c, cudaGetLastError());
    double r;
    MG_CUDA(c, (stencil<double, double>(c, H, L, 1, u, VF.b, VF.coefH, true, (cplx<double>*)nullptr, 1)));
    MG_CUDA(c, cudaMemcpyAsync(c->host_norm, H.norm2 + 1, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    MG_CUDA(c, cudaStreamSynchronize(c->stream));
    r = std::sqrt(*c->host_norm);
    rel = c->r0 > 0 ? r / c->r0 : 0.0;
  }
}

int mg_fmg(mg_ctx* c, int variant, const mg_c128* omega, int transfer, int cycles_per_stage) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  if (c->d == 4) return fail(c, MG_ERR_INVALID, std::string("mg_fmg") + kNot4);
  if (c->ada != nullptr) return fail(c, MG_ERR_INVALID, std::string("mg_fmg") + kNotA);
  if (omega == nullptr || cycles_per_stage < 0) return fail(c, MG_ERR_INVALID, "bad omega/cycles_per_stage");
  int hb, hier;
  if (decode_variant(c, variant, transfer, &hb, &hier)) return MG_ERR_INVALID;
  const cplx<double>* om = reinterpret_cast<const cplx<double>*>(omega);
  auto& H = c->h64;
  const int L = c->L;
  int rc;
  for (int s = 1; s <= L; ++s) {
    auto& V = H.lev[s];
    if (s < L && (rc = set_level_rhs(c, s)) != MG_OK) return rc;
    if (s == 1) {
      MG_CUDA(c, cudaMemsetAsync(V.u[H.cur], 0, V.nv * sizeof(cplx<double>), c->stream));
    } else {
      // u_s = P u_{s-1}: materialised previous stage, interpolated
      MG_CUDA(c, materialize(c, H, s - 1, c->scratch));
      const cplx<double>* nul = nullptr;
      if (c->d == 2)
        mg::materialize_kernel<double, 2><<<grid_for(V.nv), kThreads, 0, c->stream>>>(
            V.n, nul, c->scratch, V.u[H.cur]);
      else
        mg::materialize_kernel<double, 3><<<grid_for(V.nv), kThreads, 0, c->stream>>>(
            V.n, nul, c->scratch, V.u[H.cur]);
      MG_CUDA(c, cudaGetLastError());
    }
    if ((rc = zero_pending(c, H, s)) != MG_OK) return rc;
    if (s == L) break;
    for (int k = 0; k < cycles_per_stage; ++k)
      if ((rc = run_cycle(c, H, s, hb, hier, om)) != MG_OK) return rc;
  }
  // coarse right-hand sides of later cycles are restricted from b_L again
  c->r0 = -1.0;
  return MG_OK;
}

int mg_omega_scheme(int scheme, mg_c128 omega_s, int depth, int iter_n, int l_grid, mg_c128* out) {
  if (out == nullptr || depth < 1) return MG_ERR_INVALID;
  if (scheme == MG_OMEGA_TRANSITION && iter_n < 1) return MG_ERR_INVALID;
  const cd w(omega_s.re, omega_s.im);
  for (int l = 1; l <= depth; ++l) {
    const int succ = depth - l;
    cd v;
    switch (scheme) {
      case MG_OMEGA_JACOBI: v = succ == 0 ? w : cd(0); break;
      case MG_OMEGA_UCG: v = w; break;
      case MG_OMEGA_LGRID: v = succ <= l_grid ? w : cd(0); break;
      case MG_OMEGA_EXP: v = std::pow(w, (double)(succ + 1)); break;
      case MG_OMEGA_TRANSITION: v = std::pow(w, (1.0 - 1.0 / iter_n) * (succ + 1)); break;
      default: return MG_ERR_INVALID;
    }
    out[l - 1].re = v.real();
    out[l - 1].im = v.imag();
  }
  return MG_OK;
}

namespace {
// Captured graphs hold the kernel arguments of their launches (the wait bound,
// the diagnostic counter), so a change of either recaptures them.
void drop_graphs(mg_ctx* c) {
  drop_graphs(c->h64);
  drop_graphs(c->h32);
}
}  // namespace

int mg_set_spin_limit(mg_ctx* c, unsigned polls) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  if (polls == 0) return fail(c, MG_ERR_INVALID, "the wait bound must be at least one poll");
  if (polls != c->spin_limit) drop_graphs(c);  // captured launches bake the bound
  c->spin_limit = polls;
  return MG_OK;
}

int mg_debug_unsatisfiable_wait(mg_ctx* c, int enable) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  if ((enable != 0) != c->debug_stall) drop_graphs(c);
  c->debug_stall = enable != 0;
  MG_CUDA(c, cudaMemsetAsync(c->chain_ctr + 48, 0, sizeof(unsigned), c->stream));
  return MG_OK;
}

int mg_set_trace(mg_ctx* c, int enable) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  if (c->d == 4) return fail(c, MG_ERR_INVALID, std::string("mg_set_trace") + kNot4);
  if (c->ada != nullptr) return fail(c, MG_ERR_INVALID, std::string("mg_set_trace") + kNotA);
  if (enable && c->trace == nullptr)
    MG_CUDA(c, cudaMalloc(&c->trace, 4ull * (kTraceFine + kTraceChain) * sizeof(unsigned long long)));
  if (enable) MG_CUDA(c, cudaMemset(c->trace, 0, 4ull * (kTraceFine + kTraceChain) * sizeof(unsigned long long)));
  // captured cycles (both precisions) bake the trace pointer: drop them when the switch flips
  if ((enable != 0) != c->tracing) drop_graphs(c);
  c->tracing = enable != 0;
  return MG_OK;
}

int mg_get_trace(mg_ctx* c, unsigned long long* out, int fine_slots, int chain_slots) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  if (out == nullptr || c->trace == nullptr || fine_slots < 0 || chain_slots < 0 ||
      fine_slots > kTraceFine || chain_slots > kTraceChain)
    return fail(c, MG_ERR_INVALID, "tracing is off or slot counts out of range");
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  MG_CUDA(c, cudaMemcpy(out, c->trace, 4ull * fine_slots * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
  MG_CUDA(c, cudaMemcpy(out + 4ull * fine_slots, c->trace + 4ull * kTraceFine,
                        4ull * chain_slots * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
  return MG_OK;
}

int mg_last_cycle_norm(mg_ctx* c, double* abs_l2, double* rel_l2) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  if (c->ada != nullptr) {
    double r;
    int rc = ada_norm_host(c, &r);
    if (rc != MG_OK) return rc;
    if (abs_l2) *abs_l2 = r;
    if (rel_l2) *rel_l2 = c->r0 > 0 ? r / c->r0 : -1.0;
    return MG_OK;
  }
  MG_CUDA(c, cudaMemcpyAsync(c->host_norm, c->d == 4 ? c->h4->norm2 : c->h64.norm2, sizeof(double),
                             cudaMemcpyDeviceToHost, c->stream));
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  const double r = std::sqrt(*c->host_norm);
  if (abs_l2) *abs_l2 = r;
  if (rel_l2) *rel_l2 = c->r0 > 0 ? r / c->r0 : -1.0;
  return check_timeout(c);
}

int mg_set_timing(mg_ctx* c, int enable) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  c->timing = enable != 0;
  return MG_OK;
}

int mg_get_stats(mg_ctx* c, long long* launches, int* fine_sweeps, double* fine_ms) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  double ms = 0;
  for (size_t i = 0; i + 1 < c->ev_used; i += 2) {
    float t = 0;
    MG_CUDA(c, cudaEventElapsedTime(&t, c->ev[i], c->ev[i + 1]));
    ms += t;
  }
  int trc = check_timeout(c);
  if (trc != MG_OK) return trc;
  if (launches) *launches = c->launches;
  if (fine_sweeps) *fine_sweeps = (int)(c->ev_used / 2);
  if (fine_ms) *fine_ms = ms;
  c->launches = 0;
  c->ev_used = 0;
  return MG_OK;
}

int mg_set_k2(mg_ctx* c, const double* k2, int on_device) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  if (c->d == 4) return fail(c, MG_ERR_INVALID, std::string("mg_set_k2") + kNot4);
  if (c->ada != nullptr) return fail(c, MG_ERR_INVALID, std::string("mg_set_k2") + kNotA);
  if (k2 == nullptr) return fail(c, MG_ERR_INVALID, "k2 is NULL");
  if (!c->h64.varphi)
    return fail(c, MG_ERR_INVALID, "the context was created with a constant k^2; create a new context");
  const size_t nv = c->k2.size();
  if (on_device) {
    // copied on the context's stream, cell shifts formed there: no host round trip
    if (c->k2dev == nullptr) MG_CUDA(c, cudaMalloc(&c->k2dev, nv * sizeof(double)));
    MG_CUDA(c, cudaMemcpyAsync(c->k2dev, k2, nv * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    for (int l = 1; l <= c->L; ++l) {
      MG_CUDA(c, cell_shift_dev<double>(c, l, c->h64.lev[l].phic));
      if (c->h32.ready) MG_CUDA(c, cell_shift_dev<float>(c, l, c->h32.lev[l].phic));
    }
    c->k2_host_stale = true;
    c->r0 = -1.0;
    return MG_OK;
  }
  for (size_t i = 0; i < nv; ++i)
    if (!std::isfinite(k2[i])) return fail(c, MG_ERR_INVALID, "k2 holds a non-finite value");
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  c->k2.assign(k2, k2 + nv);
  c->k2_host_stale = false;
  for (int l = 1; l <= c->L; ++l) {
    auto p64 = cell_shift<double>(c, l);
    MG_CUDA(c, cudaMemcpy(c->h64.lev[l].phic, p64.data(), p64.size() * sizeof(double), cudaMemcpyHostToDevice));
    if (c->h32.ready) {
      auto p32 = cell_shift<float>(c, l);
      MG_CUDA(c, cudaMemcpy(c->h32.lev[l].phic, p32.data(), p32.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
  }
  c->r0 = -1.0;
  return MG_OK;
}

int mg_set_rhs_vector(mg_ctx* c, const mg_c128* b, int on_device) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  if (c->ada != nullptr) return fail(c, MG_ERR_INVALID, std::string("mg_set_rhs_vector") + kNotA);
  if (b == nullptr) return fail(c, MG_ERR_INVALID, "b is NULL");
  if (c->d == 4) {
    const Lev4<double>& V = c->h4->lev[c->L];
    MG_CUDA(c, cudaMemcpyAsync(V.b, b, V.nv * sizeof(mg_c128),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    ++c->launches;
    mg::update4_kernel<double, double><<<grid_for(V.nv), kThreads, 0, c->stream>>>(V.n, V.b, (const cplx<double>*)nullptr);  // zero boundary
    MG_CUDA(c, cudaGetLastError());
    c->r0 = -1.0;
    return MG_OK;
  }
  auto& V = c->h64.lev[c->L];
  MG_CUDA(c, cudaMemcpyAsync(c->scratch, b, V.nv * sizeof(mg_c128),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  ++c->launches;
  if (c->d == 2)
    mg::materialize_kernel<double, 2><<<grid_for(V.nv), kThreads, 0, c->stream>>>(V.n, c->scratch, nullptr, V.b);
  else
    mg::materialize_kernel<double, 3><<<grid_for(V.nv), kThreads, 0, c->stream>>>(V.n, c->scratch, nullptr, V.b);
  MG_CUDA(c, cudaGetLastError());
  c->r0 = -1.0;
  return MG_OK;
}

namespace {
// host list of (vertex, weight) of the d-linear samples at npts points
int sample_stencil(mg_ctx* c, int npts, const double* xyz, const mg_c128* w,
                   std::map<long long, cd>& acc) {
  const int d = c->d, n = (int)ipow(3, c->L), N = n + 1;
  for (int p = 0; p < npts; ++p) {
    int i[3];
    double f[3];
    for (int a = 0; a < d; ++a) {
      const double x = xyz[(size_t)p * d + a];
      if (!(x >= 0.0 && x <= 1.0)) return fail(c, MG_ERR_INVALID, "sample points must lie in [0,1]^d");
      const double xs = x * n;
      int k = (int)std::floor(xs);
      k = std::min(std::max(k, 0), n - 1);
      i[a] = k;
      f[a] = xs - k;
    }
    for (int e = 0; e < (1 << d); ++e) {
      double wt = 1.0;
      long long vi = 0, st = 1;
      bool inner = true;
      for (int a = 0; a < d; ++a) {
        const int bb = (e >> a) & 1;
        wt *= bb ? f[a] : 1.0 - f[a];
        const int g = i[a] + bb;
        inner = inner && g > 0 && g < n;
        vi += (long long)g * st;
        st *= N;
      }
      if (inner) acc[vi] += wt * cd(w[p].re, w[p].im);
    }
  }
  return MG_OK;
}
}  // namespace

int mg_sample(mg_ctx* c, int npts, const double* xyz, const mg_c128* w, mg_c128* out) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  if (c->d == 4) return fail(c, MG_ERR_INVALID, std::string("mg_sample") + kNot4);
  if (c->ada != nullptr) return fail(c, MG_ERR_INVALID, std::string("mg_sample") + kNotA);
  if (npts < 1 || xyz == nullptr || w == nullptr || out == nullptr)
    return fail(c, MG_ERR_INVALID, "bad sample arguments");
  std::map<long long, cd> acc;
  int rc = sample_stencil(c, npts, xyz, w, acc);
  if (rc != MG_OK) return rc;
  // s = sum over the stencil of weight * u (materialised, copied back per vertex)
  auto& H = c->h64;
  MG_CUDA(c, materialize(c, H, c->L, c->scratch));
  std::vector<long long> idx;
  for (auto& kv : acc) idx.push_back(kv.first);
  std::vector<mg_c128> vals(idx.size());
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  cd s(0);
  for (size_t k = 0; k < idx.size(); ++k) {
    MG_CUDA(c, cudaMemcpy(&vals[k], c->scratch + idx[k], sizeof(mg_c128), cudaMemcpyDeviceToHost));
    s += acc[idx[k]] * cd(vals[k].re, vals[k].im);
  }
  out->re = s.real();
  out->im = s.imag();
  return check_timeout(c);
}

int mg_set_rhs_samples(mg_ctx* c, int npts, const double* xyz, const mg_c128* w) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  if (c->d == 4) return fail(c, MG_ERR_INVALID, std::string("mg_set_rhs_samples") + kNot4);
  if (c->ada != nullptr) return fail(c, MG_ERR_INVALID, std::string("mg_set_rhs_samples") + kNotA);
  if (npts < 1 || xyz == nullptr || w == nullptr) return fail(c, MG_ERR_INVALID, "bad sample arguments");
  std::map<long long, cd> acc;
  int rc = sample_stencil(c, npts, xyz, w, acc);
  if (rc != MG_OK) return rc;
  std::vector<mg_c128> b(c->h64.lev[c->L].nv, mg_c128{0.0, 0.0});
  for (auto& kv : acc) b[(size_t)kv.first] = mg_c128{kv.second.real(), kv.second.imag()};
  return mg_set_rhs_vector(c, b.data(), 0);
}

int mg_adjoint_grad(mg_ctx* c, const mg_c128* u, const mg_c128* lambda, mg_c128 s, double* dJdV,
                    double* dJdf) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  if (c->d == 4) return fail(c, MG_ERR_INVALID, std::string("mg_adjoint_grad") + kNot4);
  if (c->ada != nullptr) return fail(c, MG_ERR_INVALID, std::string("mg_adjoint_grad") + kNotA);
  if (u == nullptr || lambda == nullptr || (dJdV == nullptr && dJdf == nullptr))
    return fail(c, MG_ERR_INVALID, "u, lambda and at least one output are required");
  auto& V = c->h64.lev[c->L];
  const size_t ncell = (size_t)ipow(V.n, c->d);
  const auto* uu = reinterpret_cast<const cplx<double>*>(u);
  const auto* ll = reinterpret_cast<const cplx<double>*>(lambda);
  c->launches += 2;
  if (c->d == 2) {
    mg::cell_mass_form_kernel<2><<<grid_for(ncell), kThreads, 0, c->stream>>>(V.n, ll, uu, V.hcell, c->scratch);
    mg::adjoint_grad_kernel<2><<<grid_for(V.nv), kThreads, 0, c->stream>>>(
        V.n, ll, c->scratch, V.hcell, cplx<double>{s.re, s.im}, dJdV, dJdf);
  } else {
    mg::cell_mass_form_kernel<3><<<grid_for(ncell), kThreads, 0, c->stream>>>(V.n, ll, uu, V.hcell, c->scratch);
    mg::adjoint_grad_kernel<3><<<grid_for(V.nv), kThreads, 0, c->stream>>>(
        V.n, ll, c->scratch, V.hcell, cplx<double>{s.re, s.im}, dJdV, dJdf);
  }
  MG_CUDA(c, cudaGetLastError());
  return MG_OK;
}

const char* mg_last_error(const mg_ctx* c) { return c ? c->err.c_str() : g_create_err.c_str(); }

}  // extern "C"

// =========================================================================
// Allocation-free fine residual.
//
// Some callers cannot allocate device memory when they need a residual:
// frameworks that reserve the whole device up front for their own memory
// pool, and time-critical loops that cannot afford the implicit
// synchronisation a cudaMalloc/cudaFree may cause.  This entry point gives
// them r = b - H_L u and |r|^2 without allocating: the per-block partial sums
// and the completion ticket of the deterministic two-pass reduction live in a
// file-scope device array, not in memory obtained from cudaMalloc.
//
// Limit: one 256-thread block per 256 fine vertices and one partial per
// block, so the array (kNoAllocMaxBlocks doubles + the ticket) bounds the fine
// grid at kNoAllocMaxBlocks * 256 = 4,194,304 vertices.  Every call on a
// device shares the array and it keeps the last call's contents; calls whose
// kernels overlap on the GPU race on it.
// =========================================================================
#include <mutex>

namespace {
constexpr int kNoAllocMaxBlocks = 16384;
constexpr size_t kNoAllocTicketOffset = (size_t)kNoAllocMaxBlocks * sizeof(double);
constexpr size_t kNoAllocBytes = kNoAllocTicketOffset + 256;
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};
}  // namespace

// host code must not use this name as an address; see noalloc_scratch()
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
// Device address of the scratch array on the context's device, which must be
// the current one.  Looked up (with that device current) by the first call on
// the device and again by every call made outside stream capture, so an
// address that changed with a device reset is picked up; calls during
// capture use the cached address.
int noalloc_scratch(mg_ctx* c, unsigned char** out) {
  int dev = -1;
  MG_CUDA(c, cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(c, MG_ERR_INVALID, "device ordinal out of range");
  if (c->device >= 0 && dev != c->device)
    return fail(c, MG_ERR_INVALID, "mg_residual_noalloc: the current device is " + std::to_string(dev) +
                                       ", the context was created on device " + std::to_string(c->device));
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess) {
    cudaGetLastError();
    cs = cudaStreamCaptureStatusNone;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_addr[dev] == nullptr || cs == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return fail(c, MG_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_noalloc_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_noalloc_addr[dev]);
  return MG_OK;
}
}  // namespace

extern "C" int mg_residual_noalloc(mg_ctx* c, const mg_c128* u, const mg_c128* b, mg_c128* r,
                                   double* norm2) {
  if (check_ctx(c)) return MG_ERR_INVALID;
  if (c->d == 4) return fail(c, MG_ERR_INVALID, std::string("mg_residual_noalloc") + kNot4);
  if (c->ada != nullptr) return fail(c, MG_ERR_INVALID, std::string("mg_residual_noalloc") + kNotA);
  if (u == nullptr || b == nullptr || norm2 == nullptr)
    return fail(c, MG_ERR_INVALID, "u, b and norm2 must be device pointers");
  auto& H = c->h64;
  auto& V = H.lev[c->L];
  const size_t nblocks = (V.nv + kThreads - 1) / kThreads;
  if (nblocks > (size_t)kNoAllocMaxBlocks)
    return fail(c, MG_ERR_INVALID,
                "mg_residual_noalloc: the fine grid has " + std::to_string(V.nv) +
                    " vertices; the allocation-free residual handles at most " +
                    std::to_string((size_t)kNoAllocMaxBlocks * kThreads));
  unsigned char* scratch = nullptr;
  int rc = noalloc_scratch(c, &scratch);
  if (rc != MG_OK) return rc;
  double* partial = reinterpret_cast<double*>(scratch);
  unsigned* ticket = reinterpret_cast<unsigned*>(scratch + kNoAllocTicketOffset);
  // the ticket must start at zero; the partials are written before they are read
  MG_CUDA(c, cudaMemsetAsync(ticket, 0, sizeof(unsigned), c->stream));
  ++c->launches;
  const cplx<double>* x = reinterpret_cast<const cplx<double>*>(u);
  const cplx<double>* bb = reinterpret_cast<const cplx<double>*>(b);
  cplx<double>* y = reinterpret_cast<cplx<double>*>(r);
  if (c->d == 2)
    mg::stencil_kernel<double, double, 2><<<(unsigned)nblocks, kThreads, 0, c->stream>>>(
        V.n, 1, x, bb, V.typ, V.coefH, V.realrow3, V.phic, V.hcell, y, partial, ticket, norm2);
  else
    mg::stencil_kernel<double, double, 3><<<(unsigned)nblocks, kThreads, 0, c->stream>>>(
        V.n, 1, x, bb, V.typ, V.coefH, V.realrow3, V.phic, V.hcell, y, partial, ticket, norm2);
  MG_CUDA(c, cudaGetLastError());
  return MG_OK;
}

// =========================================================================
// Batched form: many independent 2D problems, one persistent launch per
// outer defect-correction iteration (mg_batch.cuh).
// =========================================================================
#include "mg_batch.cuh"

struct mg_batch {
  std::vector<mg_ctx*> ctx;
  cudaStream_t stream = 0;
  // plan (item list and argument tables) of the last solve configuration
  std::vector<double> key;
  mg::ChainItem* items = nullptr;
  mg::Sweep2Args<float>* sw = nullptr;
  mg::Sweep2wArgs* st = nullptr;
  mg::ResArgs* res = nullptr;
  mg::UpdArgs* upd = nullptr;
  mg::CorrArgsF* co = nullptr;
  int nitems = 0;
  int* active_dev = nullptr;
  int* active_host = nullptr;       // pinned
  unsigned* ctr = nullptr;          // [0] head, [1 + p] problem counters
  unsigned* err = nullptr;
  double* norm_dev = nullptr;
  double* norm_host = nullptr;      // pinned
  int tc = 8, bpsm = 4;             // fine tile and residency (autotuned)
  cudaGraphExec_t graph = nullptr;
  std::vector<double> graph_key;
  long long launches = 0;
  std::string errmsg;
};

namespace {
int bfail(mg_batch* b, int code, const std::string& m) {
  if (b) b->errmsg = m;
  return code;
}
#define MG_BCUDA(b, call)                                                               \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return bfail((b), MG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <int TC>
size_t batch_smem() {
  size_t a = mg::Tile2<TC, float>::smem_bytes, b2 = mg::Tile2<2, float>::smem_bytes;
  return std::max(a, b2);
}

void free_plan(mg_batch* b) {
  cudaFree(b->items);
  cudaFree(b->sw);
  cudaFree(b->st);
  cudaFree(b->res);
  cudaFree(b->upd);
  cudaFree(b->co);
  b->items = nullptr;
  b->sw = nullptr;
  b->st = nullptr;
  b->res = nullptr;
  b->upd = nullptr;
  b->co = nullptr;
  b->nitems = 0;
  b->key.clear();
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_key.clear();
}

// complex64 sweep arguments of level l of problem c (inner hierarchy): the
// Galerkin-row 2D tile; inner cycle k of an outer step (k = 0 starts from 0)
mg::Sweep2Args<float> fsweep_args(mg_ctx* c, int l, bool fine, int k, int hb, int hier, const cd& om, int tc) {
  auto& E = c->h32;
  mg::Sweep2Args<float> A = sweep2_args<float>(E, l, hb, hier, om, tc);
  auto& V = E.lev[l];
  A.fine = fine ? 1 : 0;
  A.first = (fine && k == 0) ? 1 : 0;
  A.u = fine ? V.u[k % 2] : V.u[0];
  A.c = (fine && l > 1) ? E.lev[l - 1].corr : nullptr;
  A.out = fine ? V.u[(k + 1) % 2] : V.t;
  A.norm2 = nullptr;
  return A;
}

// warp-strip arguments of level l of problem c in inner cycle k
mg::Sweep2wArgs fstrip_args(mg_ctx* c, int l, bool fine, int k, int hb, int hier, const cd& om) {
  auto& E = c->h32;
  auto& V = E.lev[l];
  mg::Sweep2wArgs A;
  std::memset(&A, 0, sizeof(A));
  A.n = V.n;
  A.fine = fine ? 1 : 0;
  A.first = (fine && k == 0) ? 1 : 0;
  A.has_coarse = 1;
  A.hb = hb;
  A.hier = hier;
  const int nc = V.n / 3;
  A.scells = 18;  // two columns per lane: a batch has parallelism to spare
  A.strips = (nc + A.scells - 1) / A.scells;
  A.nunits = A.strips * nc;
  A.u = fine ? V.u[k % 2] : V.u[0];
  A.c = fine ? E.lev[l - 1].corr : nullptr;
  A.b = V.b;
  A.out = fine ? V.u[(k + 1) % 2] : V.t;
  A.b_coarse = E.lev[l - 1].b;
  A.u_coarse = E.lev[l - 1].u[0];
  A.typ = V.typ;
  A.gtyp = V.gtyp;
  A.gcoef = V.gcoef;
  axis_rows(c, V.n, A.row);
  for (size_t t = 0; t < V.diag.size() && t < 16; ++t) {
    const cd q = om / V.diag[t];
    A.omd[t] = cplx<float>{(float)q.real(), (float)q.imag()};
  }
  return A;
}

int build_batch_plan(mg_batch* b, int hb, int hier, const cplx<double>* const* omega, int m,
                     const std::vector<double>& key) {
  if (b->key == key && b->items) return MG_OK;
  free_plan(b);
  const int np = (int)b->ctx.size();
  std::vector<mg::Sweep2Args<float>> sw;
  std::vector<mg::Sweep2wArgs> stp;
  std::vector<mg::ResArgs> res;
  std::vector<mg::UpdArgs> upd;
  std::vector<mg::CorrArgsF> co;
  // per problem: list of stages, each a list of items (need filled later)
  std::vector<std::vector<std::vector<mg::ChainItem>>> stages(np);
  for (int p = 0; p < np; ++p) {
    mg_ctx* c = b->ctx[p];
    const int L = c->L;
    auto& H = c->h64;
    auto& E = c->h32;
    auto& S = stages[p];
    auto V = [&](int l) -> int { return E.lev[l].n / 3 + 1; };
    // residual stage
    {
      mg::ResArgs r;
      std::memset(&r, 0, sizeof(r));
      r.n = H.lev[L].n;
      r.nchunks = (int)((H.lev[L].nv + mg::kBatchChunk - 1) / mg::kBatchChunk);
      r.u = H.lev[L].u[H.cur];
      r.b = H.lev[L].b;
      r.out = E.lev[L].b;
      r.typ = H.lev[L].typ;
      r.coef = H.lev[L].coefH;
      r.partial = H.partial;
      r.ticket = H.ticket + 2;
      r.norm2 = b->norm_dev + p;
      res.push_back(r);
      std::vector<mg::ChainItem> st;
      for (int t = 0; t < r.nchunks; ++t) st.push_back({mg::kBRes, p, (int)res.size() - 1, t, 0});
      S.push_back(st);
    }
    for (int l = 2; l <= L; ++l)
      if (!E.lev[l].gok) return bfail(b, MG_ERR_INVALID, "a level has too many Galerkin row classes for the batch");
    for (int k = 0; k < m; ++k) {
      for (int l = L; l >= 1; --l) {
        const cplx<double> w = omega[p][l - 1];
        const bool fine = l == L;
        if (l > 1 && E.lev[l].n >= 27) {
          stp.push_back(fstrip_args(c, l, fine, k, hb, hier, cd(w.x, w.y)));
          std::vector<mg::ChainItem> st;
          const int ni = (stp.back().nunits + mg::kStripUnits - 1) / mg::kStripUnits;
          for (int t = 0; t < ni; ++t) st.push_back({mg::kBStrip, p, (int)stp.size() - 1, t, 0});
          S.push_back(st);
          continue;
        }
        const int tc = (fine || V(l) >= 40) ? b->tc : 2;
        const int kind = tc == 2 ? mg::kBSweepS : mg::kBSweep;
        sw.push_back(fsweep_args(c, l, fine, k, hb, hier, cd(w.x, w.y), tc));
        std::vector<mg::ChainItem> st;
        for (int t = 0; t < sw.back().ntiles; ++t) st.push_back({kind, p, (int)sw.size() - 1, t, 0});
        S.push_back(st);
      }
      const int top = L - 1;
      auto add_corr = [&](int tgt, int lo, const cplx<float>* base) {
        mg::CorrArgsF ca;
        std::memset(&ca, 0, sizeof(ca));
        ca.s = tgt;
        ca.lo = lo;
        for (int l = lo; l <= tgt; ++l) ca.t[l] = E.lev[l].t;
        ca.base = base;
        ca.out = E.lev[tgt].corr;
        co.push_back(ca);
        std::vector<mg::ChainItem> st;
        const int nch = (int)((E.lev[tgt].nv + mg::kBatchChunk - 1) / mg::kBatchChunk);
        for (int t = 0; t < nch; ++t) st.push_back({mg::kBCorr, p, (int)co.size() - 1, t, 0});
        S.push_back(st);
      };
      if (top >= 3) {
        add_corr(top - 1, 1, nullptr);
        add_corr(top, top, E.lev[top - 1].corr);
      } else if (top == 2) {
        add_corr(2, 1, nullptr);
      }
    }
    {
      mg::UpdArgs u;
      u.n = H.lev[L].n;
      u.u = H.lev[L].u[H.cur];
      u.e = E.lev[L].u[m % 2];
      u.c = L > 1 ? E.lev[L - 1].corr : nullptr;
      upd.push_back(u);
      std::vector<mg::ChainItem> st;
      const int nch = (int)((H.lev[L].nv + mg::kBatchChunk - 1) / mg::kBatchChunk);
      for (int t = 0; t < nch; ++t) st.push_back({mg::kBUpd, p, (int)upd.size() - 1, t, 0});
      S.push_back(st);
    }
    unsigned need = 0;
    for (auto& st : S) {
      for (auto& it : st) it.need = need;
      need += (unsigned)st.size();
    }
  }
  // stage-major order across problems
  std::vector<mg::ChainItem> items;
  size_t maxst = 0;
  for (auto& S : stages) maxst = std::max(maxst, S.size());
  for (size_t j = 0; j < maxst; ++j)
    for (int p = 0; p < np; ++p)
      if (j < stages[p].size()) items.insert(items.end(), stages[p][j].begin(), stages[p][j].end());
  b->nitems = (int)items.size();
  auto up = [&](void** dst, const void* src, size_t bytes) -> cudaError_t {
    cudaError_t e = cudaMalloc(dst, std::max<size_t>(bytes, 16));
    if (e == cudaSuccess && bytes) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    return e;
  };
  MG_BCUDA(b, up((void**)&b->items, items.data(), items.size() * sizeof(mg::ChainItem)));
  MG_BCUDA(b, up((void**)&b->sw, sw.data(), sw.size() * sizeof(mg::Sweep2Args<float>)));
  MG_BCUDA(b, up((void**)&b->st, stp.data(), stp.size() * sizeof(mg::Sweep2wArgs)));
  MG_BCUDA(b, up((void**)&b->res, res.data(), res.size() * sizeof(mg::ResArgs)));
  MG_BCUDA(b, up((void**)&b->upd, upd.data(), upd.size() * sizeof(mg::UpdArgs)));
  MG_BCUDA(b, up((void**)&b->co, co.data(), co.size() * sizeof(mg::CorrArgsF)));
  b->key = key;
  return MG_OK;
}

// enqueue one outer iteration (counters, flags, kernel, norms) on b->stream
cudaError_t enqueue_batch(mg_batch* b) {
  const int np = (int)b->ctx.size();
  cudaError_t e = cudaMemcpyAsync(b->active_dev, b->active_host, np * sizeof(int), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->ctr, 0, (np + 1) * sizeof(unsigned), b->stream);
  mg::BatchArgs A;
  A.items = b->items;
  A.nitems = b->nitems;
  A.sw = b->sw;
  A.st = b->st;
  A.res = b->res;
  A.upd = b->upd;
  A.co = b->co;
  A.active = b->active_dev;
  A.head = b->ctr;
  A.done = b->ctr + 1;
  A.err = b->err;
  A.spin_limit = 1u << 22;
  const int grid = 152 * b->bpsm;
  if (e == cudaSuccess) {
    if (b->tc == 8)
      mg::batch2_kernel<8, 256><<<grid, 256, batch_smem<8>(), b->stream>>>(A);
    else
      mg::batch2_kernel<4, 256><<<grid, 256, batch_smem<4>(), b->stream>>>(A);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->norm_host, b->norm_dev, np * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
  return e;
}

// one outer iteration as a captured graph (captured once per plan and tuning)
int run_batch(mg_batch* b) {
  std::vector<double> gk = b->key;
  gk.push_back(b->tc);
  gk.push_back(b->bpsm);
  if (b->graph == nullptr || b->graph_key != gk) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    cudaStream_t cs;
    MG_BCUDA(b, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaStream_t user = b->stream;
    b->stream = cs;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    cudaError_t ek = e == cudaSuccess ? enqueue_batch(b) : e;
    cudaError_t ee = e == cudaSuccess ? cudaStreamEndCapture(cs, &g) : e;
    b->stream = user;
    if (e == cudaSuccess) e = ek != cudaSuccess ? ek : ee;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      b->graph = nullptr;
      return bfail(b, MG_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    }
    b->graph_key = gk;
  }
  MG_BCUDA(b, cudaGraphLaunch(b->graph, b->stream));
  ++b->launches;
  return MG_OK;
}

int batch_prepare(mg_batch* b, int variant, const mg_c128* const* omega, int transfer, int inner, int* hbp,
                  int* hierp) {
  if (omega == nullptr) return bfail(b, MG_ERR_INVALID, "omega is NULL");
  if (inner < 1 || inner > 64) return bfail(b, MG_ERR_INVALID, "inner_cycles must be in 1..64");
  int hb, hier;
  if (variant < MG_ADD || variant > MG_BPX || (transfer != MG_DLINEAR && transfer != MG_HIERARCHICAL))
    return bfail(b, MG_ERR_INVALID, "bad variant/transfer");
  hb = variant == MG_HB;
  hier = (transfer == MG_HIERARCHICAL) || (variant == MG_BPX);
  std::vector<double> key = {(double)hb, (double)hier, (double)inner, (double)b->tc};
  for (size_t p = 0; p < b->ctx.size(); ++p) {
    if (omega[p] == nullptr) return bfail(b, MG_ERR_INVALID, "omega[p] is NULL");
    for (int l = 0; l < b->ctx[p]->L; ++l) {
      key.push_back(omega[p][l].re);
      key.push_back(omega[p][l].im);
    }
  }
  std::vector<const cplx<double>*> om(b->ctx.size());
  for (size_t p = 0; p < b->ctx.size(); ++p) om[p] = reinterpret_cast<const cplx<double>*>(omega[p]);
  int rc = build_batch_plan(b, hb, hier, om.data(), inner, key);
  *hbp = hb;
  *hierp = hier;
  return rc;
}

// fold pending corrections of the FP64 fine solutions (the batch updates u in place)
int batch_materialize(mg_batch* b) {
  for (mg_ctx* c : b->ctx) {
    auto& H = c->h64;
    cudaStream_t keep = c->stream;
    c->stream = b->stream;
    cudaError_t e = materialize(c, H, c->L, c->scratch);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(H.lev[c->L].u[H.cur], c->scratch, H.lev[c->L].nv * sizeof(cplx<double>),
                          cudaMemcpyDeviceToDevice, b->stream);
    c->stream = keep;
    if (e != cudaSuccess) return bfail(b, MG_ERR_CUDA, cudaGetErrorString(e));
    if (zero_pending(c, H, c->L) != MG_OK) return bfail(b, MG_ERR_CUDA, c->err);
  }
  return MG_OK;
}
}  // namespace

extern "C" {

int mg_batch_create(int n, const int* d, const int* depth, const double* const* k2, const double* theta,
                    const double* layer_width, mg_batch** out) {
  if (out == nullptr || n < 1 || d == nullptr || depth == nullptr || k2 == nullptr || theta == nullptr ||
      layer_width == nullptr)
    return MG_ERR_INVALID;
  *out = nullptr;
  for (int p = 0; p < n; ++p)
    if (d[p] != 2) return fail(nullptr, MG_ERR_INVALID, "batched problems must be 2D");
  mg_batch* b = new (std::nothrow) mg_batch();
  if (b == nullptr) return MG_ERR_OOM;
  auto cleanup = [&](int rc) {
    mg_batch_destroy(b);
    return rc;
  };
  for (int p = 0; p < n; ++p) {
    mg_ctx* c = nullptr;
    int rc = mg_create(d[p], depth[p], k2[p], theta[p], layer_width[p], &c);
    if (rc != MG_OK) return cleanup(rc);
    b->ctx.push_back(c);
    if (c->h64.varphi) return cleanup(fail(nullptr, MG_ERR_INVALID, "batched problems need a constant k^2"));
    rc = mg_set_precision(c, MG_C64_REFINE, 4);
    if (rc != MG_OK) return cleanup(rc);
  }
  cudaError_t e = cudaMalloc(&b->active_dev, n * sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&b->active_host, n * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->ctr, (n + 1) * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc(&b->err, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(b->err, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc(&b->norm_dev, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&b->norm_host, n * sizeof(double));
  auto setsm = [&](const void* f, size_t bytes) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  };
  setsm((const void*)mg::batch2_kernel<8, 256>, batch_smem<8>());
  setsm((const void*)mg::batch2_kernel<4, 256>, batch_smem<4>());
  if (e != cudaSuccess) return cleanup(fail(nullptr, MG_ERR_CUDA, cudaGetErrorString(e)));
  for (int p = 0; p < n; ++p) b->active_host[p] = 1;
  *out = b;
  return MG_OK;
}

void mg_batch_destroy(mg_batch* b) {
  if (b == nullptr) return;
  free_plan(b);
  for (mg_ctx* c : b->ctx) mg_destroy(c);
  cudaFree(b->active_dev);
  if (b->active_host) cudaFreeHost(b->active_host);
  cudaFree(b->ctr);
  cudaFree(b->err);
  cudaFree(b->norm_dev);
  if (b->norm_host) cudaFreeHost(b->norm_host);
  delete b;
}

int mg_batch_get_ctx(mg_batch* b, int p, mg_ctx** out) {
  if (b == nullptr || out == nullptr || p < 0 || p >= (int)b->ctx.size()) return MG_ERR_INVALID;
  *out = b->ctx[p];
  return MG_OK;
}

int mg_batch_set_stream(mg_batch* b, void* stream) {
  if (b == nullptr) return MG_ERR_INVALID;
  b->stream = (cudaStream_t)stream;
  for (mg_ctx* c : b->ctx) c->stream = b->stream;
  return MG_OK;
}

int mg_batch_solve(mg_batch* b, int variant, const mg_c128* const* omega, int transfer, double tol,
                   int max_outer, int inner_cycles, int* status, int* cycles, double* rel_res) {
  if (b == nullptr) return MG_ERR_INVALID;
  if (!(tol > 0) || max_outer < 0) return bfail(b, MG_ERR_INVALID, "tol must be > 0 and max_outer >= 0");
  int hb, hier;
  int rc = batch_prepare(b, variant, omega, transfer, inner_cycles, &hb, &hier);
  if (rc != MG_OK) return rc;
  if ((rc = batch_materialize(b)) != MG_OK) return rc;
  const int np = (int)b->ctx.size();
  std::vector<double> r0(np, -1.0), rel(np, 1.0);
  std::vector<int> st(np, MG_NOT_CONVERGED), outer(np, 0);
  for (int p = 0; p < np; ++p) b->active_host[p] = 1;
  int live = np;
  // Each launch measures the residual of the iterate entering it and applies
  // one outer step to every active problem.  A problem whose entering
  // residual is below tol (or diverged) leaves the batch after that launch;
  // the step the launch applied to it anyway only refines a converged
  // iterate.  At most max_outer launches; the final residual below decides
  // the status of problems still active then.
  for (int it = 0; it < max_outer && live > 0; ++it) {
    if ((rc = run_batch(b)) != MG_OK) return rc;
    MG_BCUDA(b, cudaStreamSynchronize(b->stream));
    for (int p = 0; p < np; ++p) {
      if (!b->active_host[p]) continue;
      ++outer[p];
      const double r = std::sqrt(b->norm_host[p]);
      if (r0[p] < 0) r0[p] = r;
      rel[p] = r0[p] > 0 ? r / r0[p] : 0.0;
      if (!std::isfinite(rel[p]) || rel[p] > 1e6) {
        st[p] = MG_DIVERGED;
      } else if (rel[p] <= tol) {
        st[p] = MG_OK;
      } else {
        continue;  // stays active
      }
      b->active_host[p] = 0;
      --live;
    }
  }
  unsigned f = 0;
  MG_BCUDA(b, cudaMemcpy(&f, b->err, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (f) {
    cudaMemset(b->err, 0, sizeof(unsigned));
    return bfail(b, MG_ERR_TIMEOUT, "a bounded device-side wait gave up");
  }
  // final FP64 residual of every solution relative to its starting residual
  for (int p = 0; p < np; ++p) {
    mg_ctx* c = b->ctx[p];
    double r;
    if ((rc = fine_residual(c, c->L, &r)) != MG_OK) return bfail(b, rc, c->err);
    if (r0[p] < 0) r0[p] = r;  // no launch ran (max_outer = 0)
    const double relp = r0[p] > 0 ? r / r0[p] : 0.0;
    if (st[p] != MG_DIVERGED) st[p] = relp <= tol ? MG_OK : MG_NOT_CONVERGED;
    if (status) status[p] = st[p];
    if (cycles) cycles[p] = outer[p] * inner_cycles;  // every outer step applied
    if (rel_res) rel_res[p] = relp;
    c->r0 = r0[p];
  }
  return MG_OK;
}

int mg_batch_autotune(mg_batch* b, int variant, const mg_c128* const* omega, int transfer, int inner_cycles,
                      int* tc_out, int* bpsm_out, double* best_ms) {
  if (b == nullptr) return MG_ERR_INVALID;
  int rc = batch_materialize(b);
  if (rc != MG_OK) return rc;
  const int np = (int)b->ctx.size();
  // the trial launches update the solutions: save and restore them
  std::vector<cplx<double>*> saved(np, nullptr);
  for (int p = 0; p < np; ++p) {
    auto& V = b->ctx[p]->h64.lev[b->ctx[p]->L];
    MG_BCUDA(b, cudaMalloc(&saved[p], V.nv * sizeof(cplx<double>)));
    MG_BCUDA(b, cudaMemcpyAsync(saved[p], V.u[b->ctx[p]->h64.cur], V.nv * sizeof(cplx<double>),
                                cudaMemcpyDeviceToDevice, b->stream));
  }
  for (int p = 0; p < np; ++p) b->active_host[p] = 1;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  double best = 1e30;
  int btc = b->tc, bb = b->bpsm;
  cudaEvent_t e0, e1;
  MG_BCUDA(b, cudaEventCreate(&e0));
  MG_BCUDA(b, cudaEventCreate(&e1));
  for (int tc : {4, 8}) {
    int occ = 0;
    if (tc == 8)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, mg::batch2_kernel<8, 256>, 256, batch_smem<8>());
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, mg::batch2_kernel<4, 256>, 256, batch_smem<4>());
    for (int bp : {2, 4, 8}) {
      if (bp > occ) continue;
      b->tc = tc;
      b->bpsm = bp;
      int hb, hier;
      if ((rc = batch_prepare(b, variant, omega, transfer, inner_cycles, &hb, &hier)) != MG_OK) break;
      if ((rc = run_batch(b)) != MG_OK) break;  // warm-up
      MG_BCUDA(b, cudaEventRecord(e0, b->stream));
      for (int r = 0; r < 3 && rc == MG_OK; ++r) rc = run_batch(b);
      MG_BCUDA(b, cudaEventRecord(e1, b->stream));
      MG_BCUDA(b, cudaEventSynchronize(e1));
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rc == MG_OK && ms / 3 < best) {
        best = ms / 3;
        btc = tc;
        bb = bp;
      }
    }
    if (rc != MG_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int p = 0; p < np; ++p) {
    auto& V = b->ctx[p]->h64.lev[b->ctx[p]->L];
    cudaMemcpyAsync(V.u[b->ctx[p]->h64.cur], saved[p], V.nv * sizeof(cplx<double>), cudaMemcpyDeviceToDevice,
                    b->stream);
  }
  cudaStreamSynchronize(b->stream);
  for (auto* s : saved) cudaFree(s);
  if (rc != MG_OK) return rc;
  b->tc = btc;
  b->bpsm = bb;
  if (tc_out) *tc_out = btc;
  if (bpsm_out) *bpsm_out = bb;
  if (best_ms) *best_ms = best;
  (void)sms;
  return MG_OK;
}

long long mg_batch_launches(const mg_batch* b) { return b ? b->launches : -1; }

const char* mg_batch_last_error(const mg_batch* b) { return b ? b->errmsg.c_str() : ""; }

}  // extern "C"
