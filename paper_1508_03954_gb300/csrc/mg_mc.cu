// mg_mc.cu -- C ABI of the coupled multichannel form (Section 7.5): the
// additive cycle (Appendix A Algorithm 4) on c-channel tuples with the block
// operator A = I (x) K - Phi (x) M and damped block-Jacobi smoothing.
// Declarations and argument contracts in include/mg.h.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <cstring>
#include <string>
#include <vector>

#include "mg.h"
#include "mg_mc.cuh"

using mg::cplx;
using cd = std::complex<double>;

struct McLevel {
  int n = 0;
  size_t nv = 0;
  cplx<double>* u = nullptr;     // solution (coarse: injected copy)
  cplx<double>* b = nullptr;     // right-hand side
  cplx<double>* t = nullptr;     // block-Jacobi update
  cplx<double>* corr = nullptr;  // correction corr_l
  uint8_t* typ = nullptr;        // axis class per index (left / right cell rotated)
  cplx<double>* K = nullptr;     // [4^d][3^d] stiffness rows per vertex type
  cplx<double>* M = nullptr;     // [4^d][3^d] mass rows
  cplx<double>* Dinv = nullptr;  // [4^d][c][c] inverse diagonal blocks
};

struct mg_mc_ctx {
  int d = 0, L = 0, c = 0;
  double theta = 0, width = 0;
  cudaStream_t stream = 0;
  std::vector<McLevel> lev;
  cplx<double>* Phi = nullptr;   // c x c, device
  cplx<double>* uh = nullptr;    // fine-size scratch: surplus
  cplx<double>* rh = nullptr;    // fine-size scratch: hierarchical residual
  double* partial = nullptr;     // per-block |r|^2
  std::vector<double> hpart;
  std::vector<void*> allocs;
  double r0 = -1.0;
  std::string err;
};

namespace {

constexpr int kMaxBlocks = 152 * 16;

int fail(mg_mc_ctx* c, int code, const std::string& msg) {
  if (c != nullptr) c->err = msg;
  return code;
}

#define MC_CUDA(c, call)                                                       \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) return fail((c), MG_ERR_CUDA, cudaGetErrorString(e_)); \
  } while (0)

long long ipow(long long b, int e) {
  long long r = 1;
  while (e-- > 0) r *= b;
  return r;
}

int blocks_for(size_t n) {
  size_t b = (n + mg::kMcThreads - 1) / mg::kMcThreads;
  return (int)std::min<size_t>(std::max<size_t>(b, 1), kMaxBlocks);
}

int dalloc(mg_mc_ctx* c, void** p, size_t bytes) {
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(c, MG_ERR_OOM, "cudaMalloc failed");
  }
  c->allocs.push_back(*p);
  MC_CUDA(c, cudaMemset(*p, 0, bytes));
  return MG_OK;
}

// Layer membership of the cells of a level by their centre (the reading of
// the single-channel form): min(2i+1, 2n-2i-1) < 2 w n, every cell for w >= 0.5.
std::vector<uint8_t> cell_rotated(int n, double w) {
  std::vector<uint8_t> rot(n);
  for (int i = 0; i < n; ++i) {
    const long long a = 2LL * i + 1, b = 2LL * n - 2LL * i - 1;
    rot[i] = (w >= 0.5) || ((double)std::min(a, b) < 2.0 * w * (double)n);
  }
  return rot;
}

// In-place inverse of a c x c complex matrix (Gauss-Jordan, partial
// pivoting); false when singular.
bool invert(std::vector<cd>& A, int c) {
  std::vector<cd> I(c * c, cd(0));
  for (int i = 0; i < c; ++i) I[i * c + i] = 1;
  for (int col = 0; col < c; ++col) {
    int p = col;
    for (int r = col + 1; r < c; ++r)
      if (std::abs(A[r * c + col]) > std::abs(A[p * c + col])) p = r;
    if (std::abs(A[p * c + col]) == 0.0) return false;
    if (p != col)
      for (int k = 0; k < c; ++k) {
        std::swap(A[p * c + k], A[col * c + k]);
        std::swap(I[p * c + k], I[col * c + k]);
      }
    const cd inv = 1.0 / A[col * c + col];
    for (int k = 0; k < c; ++k) {
      A[col * c + k] *= inv;
      I[col * c + k] *= inv;
    }
    for (int r = 0; r < c; ++r) {
      if (r == col) continue;
      const cd f = A[r * c + col];
      if (f == cd(0)) continue;
      for (int k = 0; k < c; ++k) {
        A[r * c + k] -= f * A[col * c + k];
        I[r * c + k] -= f * I[col * c + k];
      }
    }
  }
  A = I;
  return true;
}

// Per-level tables: axis classes, K and M rows of every vertex type (tensor
// products of the assembled 1D rows, Section 4), inverse diagonal blocks.
int build_level(mg_mc_ctx* c, int l, const std::vector<cd>& phi) {
  McLevel& V = c->lev[l];
  const int d = c->d, C = c->c;
  V.n = (int)ipow(3, l);
  V.nv = (size_t)ipow(V.n + 1, d);
  const size_t bytes = V.nv * C * sizeof(cplx<double>);
  int rc;
  if ((rc = dalloc(c, (void**)&V.u, bytes)) != MG_OK) return rc;
  if ((rc = dalloc(c, (void**)&V.b, bytes)) != MG_OK) return rc;
  if ((rc = dalloc(c, (void**)&V.t, bytes)) != MG_OK) return rc;
  if ((rc = dalloc(c, (void**)&V.corr, bytes)) != MG_OK) return rc;
  const std::vector<uint8_t> rot = cell_rotated(V.n, c->width);
  std::vector<uint8_t> typ(V.n + 1);
  for (int i = 0; i <= V.n; ++i) typ[i] = (uint8_t)(rot[std::max(i - 1, 0)] + 2 * rot[std::min(i, V.n - 1)]);
  const double h = 1.0 / V.n;
  const cd hin(h, 0.0), hrot = h * cd(std::cos(c->theta), std::sin(c->theta));
  cd K1[4][3], M1[4][3];
  for (int t = 0; t < 4; ++t) {
    const cd hl = (t & 1) ? hrot : hin, hr = (t & 2) ? hrot : hin;
    K1[t][0] = -1.0 / hl;
    K1[t][1] = 1.0 / hl + 1.0 / hr;
    K1[t][2] = -1.0 / hr;
    M1[t][0] = hl / 6.0;
    M1[t][1] = (hl + hr) / 3.0;
    M1[t][2] = hr / 6.0;
  }
  const int NT = (int)ipow(4, d), NS = (int)ipow(3, d);
  std::vector<cplx<double>> K(NT * NS), M(NT * NS), Dinv((size_t)NT * C * C);
  for (int t = 0; t < NT; ++t) {
    int ta[3] = {t % 4, (t / 4) % 4, t / 16};
    cd kc(0), mc(0);
    for (int s = 0; s < NS; ++s) {
      int ka[3] = {s % 3, (s / 3) % 3, s / 9};
      cd m(1), k(0);
      for (int a = 0; a < d; ++a) m *= M1[ta[a]][ka[a]];
      for (int j = 0; j < d; ++j) {
        cd p(1);
        for (int a = 0; a < d; ++a) p *= (a == j ? K1 : M1)[ta[a]][ka[a]];
        k += p;
      }
      K[t * NS + s] = {k.real(), k.imag()};
      M[t * NS + s] = {m.real(), m.imag()};
      if (s == NS / 2) {
        kc = k;
        mc = m;
      }
    }
    std::vector<cd> D(C * C);
    for (int i = 0; i < C; ++i)
      for (int j = 0; j < C; ++j) D[i * C + j] = (i == j ? kc : cd(0)) - phi[i * C + j] * mc;
    if (!invert(D, C)) return fail(c, MG_ERR_INVALID, "a diagonal block K I - Phi M of the coupled operator is singular");
    for (int k = 0; k < C * C; ++k) Dinv[(size_t)t * C * C + k] = {D[k].real(), D[k].imag()};
  }
  if ((rc = dalloc(c, (void**)&V.typ, typ.size())) != MG_OK) return rc;
  if ((rc = dalloc(c, (void**)&V.K, K.size() * sizeof(cplx<double>))) != MG_OK) return rc;
  if ((rc = dalloc(c, (void**)&V.M, M.size() * sizeof(cplx<double>))) != MG_OK) return rc;
  if ((rc = dalloc(c, (void**)&V.Dinv, Dinv.size() * sizeof(cplx<double>))) != MG_OK) return rc;
  MC_CUDA(c, cudaMemcpy(V.typ, typ.data(), typ.size(), cudaMemcpyHostToDevice));
  MC_CUDA(c, cudaMemcpy(V.K, K.data(), K.size() * sizeof(cplx<double>), cudaMemcpyHostToDevice));
  MC_CUDA(c, cudaMemcpy(V.M, M.data(), M.size() * sizeof(cplx<double>), cudaMemcpyHostToDevice));
  MC_CUDA(c, cudaMemcpy(V.Dinv, Dinv.data(), Dinv.size() * sizeof(cplx<double>), cudaMemcpyHostToDevice));
  return MG_OK;
}

// kernels of one (d, c) pair
template <int D, int C>
struct McOps {
  static cudaError_t residual(mg_mc_ctx* c, const McLevel& V, const cplx<double>* x, cplx<double>* out, bool jac,
                              cplx<double> om, int hb, double* partial) {
    mg::mc_residual_kernel<D, C><<<blocks_for(V.nv), mg::kMcThreads, 0, c->stream>>>(
        V.n, x, V.b, out, V.typ, V.K, V.M, c->Phi, V.Dinv, jac ? 1 : 0, om, hb, partial);
    return cudaGetLastError();
  }
  static cudaError_t mass(mg_mc_ctx* c, const McLevel& V, const cplx<double>* f) {
    mg::mc_mass_kernel<D, C><<<blocks_for(V.nv), mg::kMcThreads, 0, c->stream>>>(V.n, f, V.b, V.typ, V.M);
    return cudaGetLastError();
  }
  // Algorithm 4 on tuples: fine to coarse (block-Jacobi update, injection,
  // surplus, hierarchical residual, restriction), then coarse to fine
  // (corr_l = T t_l + P corr_{l-1}; the finest level adds to u)
  static cudaError_t cycle(mg_mc_ctx* c, int hb, int bpx, const cplx<double>* om) {
    cudaError_t e = cudaSuccess;
    for (int l = c->L; l >= 1 && e == cudaSuccess; --l) {
      McLevel& V = c->lev[l];
      e = residual(c, V, V.u, V.t, true, om[l - 1], hb, nullptr);
      if (e != cudaSuccess || l == 1) continue;
      McLevel& W = c->lev[l - 1];
      mg::mc_inject_kernel<D, C><<<blocks_for(W.nv), mg::kMcThreads, 0, c->stream>>>(V.n, V.u, W.u);
      mg::mc_surplus_kernel<D, C><<<blocks_for(V.nv), mg::kMcThreads, 0, c->stream>>>(V.n, V.u, W.u, c->uh);
      e = residual(c, V, c->uh, c->rh, false, om[l - 1], 0, nullptr);
      if (e != cudaSuccess) break;
      mg::mc_restrict_kernel<D, C><<<blocks_for(W.nv), mg::kMcThreads, 0, c->stream>>>(V.n, c->rh, W.b);
      e = cudaGetLastError();
    }
    for (int l = 1; l <= c->L && e == cudaSuccess; ++l) {
      McLevel& V = c->lev[l];
      const cplx<double>* cc = l > 1 ? c->lev[l - 1].corr : nullptr;
      mg::mc_correct_kernel<D, C><<<blocks_for(V.nv), mg::kMcThreads, 0, c->stream>>>(
          V.n, V.t, cc, hb, bpx, V.corr, l == c->L ? V.u : nullptr);
      e = cudaGetLastError();
    }
    return e;
  }
};

template <int D>
cudaError_t dispatch_cycle(mg_mc_ctx* c, int hb, int bpx, const cplx<double>* om) {
  switch (c->c) {
    case 1: return McOps<D, 1>::cycle(c, hb, bpx, om);
    case 2: return McOps<D, 2>::cycle(c, hb, bpx, om);
    case 3: return McOps<D, 3>::cycle(c, hb, bpx, om);
    case 4: return McOps<D, 4>::cycle(c, hb, bpx, om);
    case 8: return McOps<D, 8>::cycle(c, hb, bpx, om);
    default: return McOps<D, 16>::cycle(c, hb, bpx, om);
  }
}

template <int D>
cudaError_t dispatch_residual(mg_mc_ctx* c, double* partial) {
  const McLevel& V = c->lev[c->L];
  const cplx<double> z{0, 0};
  switch (c->c) {
    case 1: return McOps<D, 1>::residual(c, V, V.u, c->rh, false, z, 0, partial);
    case 2: return McOps<D, 2>::residual(c, V, V.u, c->rh, false, z, 0, partial);
    case 3: return McOps<D, 3>::residual(c, V, V.u, c->rh, false, z, 0, partial);
    case 4: return McOps<D, 4>::residual(c, V, V.u, c->rh, false, z, 0, partial);
    case 8: return McOps<D, 8>::residual(c, V, V.u, c->rh, false, z, 0, partial);
    default: return McOps<D, 16>::residual(c, V, V.u, c->rh, false, z, 0, partial);
  }
}

template <int D>
cudaError_t dispatch_mass(mg_mc_ctx* c, const cplx<double>* f) {
  const McLevel& V = c->lev[c->L];
  switch (c->c) {
    case 1: return McOps<D, 1>::mass(c, V, f);
    case 2: return McOps<D, 2>::mass(c, V, f);
    case 3: return McOps<D, 3>::mass(c, V, f);
    case 4: return McOps<D, 4>::mass(c, V, f);
    case 8: return McOps<D, 8>::mass(c, V, f);
    default: return McOps<D, 16>::mass(c, V, f);
  }
}

template <int D>
cudaError_t dispatch_interior(mg_mc_ctx* c, const cplx<double>* src, cplx<double>* dst) {
  const McLevel& F = c->lev[c->L];
  const int g = blocks_for(F.nv);
  switch (c->c) {
    case 1: mg::mc_interior_kernel<D, 1><<<g, mg::kMcThreads, 0, c->stream>>>(F.n, src, dst); break;
    case 2: mg::mc_interior_kernel<D, 2><<<g, mg::kMcThreads, 0, c->stream>>>(F.n, src, dst); break;
    case 3: mg::mc_interior_kernel<D, 3><<<g, mg::kMcThreads, 0, c->stream>>>(F.n, src, dst); break;
    case 4: mg::mc_interior_kernel<D, 4><<<g, mg::kMcThreads, 0, c->stream>>>(F.n, src, dst); break;
    case 8: mg::mc_interior_kernel<D, 8><<<g, mg::kMcThreads, 0, c->stream>>>(F.n, src, dst); break;
    default: mg::mc_interior_kernel<D, 16><<<g, mg::kMcThreads, 0, c->stream>>>(F.n, src, dst); break;
  }
  return cudaGetLastError();
}

bool valid_channels(int ch) { return ch == 1 || ch == 2 || ch == 3 || ch == 4 || ch == 8 || ch == 16; }

// fine tuple array in from host or device, Dirichlet ring zeroed
int load_fine(mg_mc_ctx* c, const mg_c128* src, int on_device, cplx<double>* dst) {
  const McLevel& F = c->lev[c->L];
  const size_t bytes = F.nv * c->c * sizeof(cplx<double>);
  MC_CUDA(c, cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             c->stream));
  if (!on_device) MC_CUDA(c, cudaStreamSynchronize(c->stream));  // the host buffer may go away
  return MG_OK;
}

}  // namespace

extern "C" {

int mg_mc_create(int d, int depth, int channels, const mg_c128* phi, double theta, double layer_width,
                 mg_mc_ctx** out) {
  if (out == nullptr) return MG_ERR_INVALID;
  *out = nullptr;
  if ((d != 2 && d != 3) || depth < 1 || !valid_channels(channels) || phi == nullptr) return MG_ERR_INVALID;
  if (!(theta >= 0.0 && theta < M_PI / 2) || !(layer_width >= 0.0 && layer_width <= 0.5)) return MG_ERR_INVALID;
  if (d == 2 && depth > 8) return MG_ERR_INVALID;
  if (d == 3 && depth > 6) return MG_ERR_INVALID;
  std::vector<cd> ph((size_t)channels * channels);
  for (size_t k = 0; k < ph.size(); ++k) {
    if (!std::isfinite(phi[k].re) || !std::isfinite(phi[k].im)) return MG_ERR_INVALID;
    ph[k] = cd(phi[k].re, phi[k].im);
  }
  mg_mc_ctx* c = new (std::nothrow) mg_mc_ctx;
  if (c == nullptr) return MG_ERR_OOM;
  c->d = d;
  c->L = depth;
  c->c = channels;
  c->theta = theta;
  c->width = layer_width;
  c->lev.assign(depth + 1, McLevel());
  int rc = MG_OK;
  for (int l = 1; l <= depth && rc == MG_OK; ++l) rc = build_level(c, l, ph);
  const size_t fine = c->lev[depth].nv * channels * sizeof(cplx<double>);
  if (rc == MG_OK) rc = dalloc(c, (void**)&c->uh, fine);
  if (rc == MG_OK) rc = dalloc(c, (void**)&c->rh, fine);
  if (rc == MG_OK) rc = dalloc(c, (void**)&c->partial, kMaxBlocks * sizeof(double));
  if (rc == MG_OK) rc = dalloc(c, (void**)&c->Phi, ph.size() * sizeof(cplx<double>));
  if (rc == MG_OK) {
    std::vector<cplx<double>> p(ph.size());
    for (size_t k = 0; k < ph.size(); ++k) p[k] = {ph[k].real(), ph[k].imag()};
    if (cudaMemcpy(c->Phi, p.data(), p.size() * sizeof(cplx<double>), cudaMemcpyHostToDevice) != cudaSuccess)
      rc = MG_ERR_CUDA;
  }
  if (rc != MG_OK) {
    mg_mc_destroy(c);
    return rc;
  }
  *out = c;
  return MG_OK;
}

int mg_mc_set_stream(mg_mc_ctx* c, void* s) {
  if (c == nullptr) return MG_ERR_INVALID;
  c->stream = (cudaStream_t)s;
  return MG_OK;
}

int mg_mc_set_rhs(mg_mc_ctx* c, const mg_c128* f, int on_device) {
  if (c == nullptr) return MG_ERR_INVALID;
  if (f == nullptr) return fail(c, MG_ERR_INVALID, "f is NULL");
  int rc = load_fine(c, f, on_device, c->uh);
  if (rc != MG_OK) return rc;
  MC_CUDA(c, c->d == 2 ? dispatch_mass<2>(c, c->uh) : dispatch_mass<3>(c, c->uh));
  c->r0 = -1.0;
  return MG_OK;
}

int mg_mc_set_solution(mg_mc_ctx* c, const mg_c128* u, int on_device) {
  if (c == nullptr) return MG_ERR_INVALID;
  if (u == nullptr) return fail(c, MG_ERR_INVALID, "u is NULL");
  McLevel& F = c->lev[c->L];
  int rc = load_fine(c, u, on_device, c->uh);
  if (rc != MG_OK) return rc;
  MC_CUDA(c, c->d == 2 ? dispatch_interior<2>(c, c->uh, F.u) : dispatch_interior<3>(c, c->uh, F.u));
  c->r0 = -1.0;
  return MG_OK;
}

int mg_mc_get_solution(mg_mc_ctx* c, mg_c128* out, int on_device) {
  if (c == nullptr) return MG_ERR_INVALID;
  if (out == nullptr) return fail(c, MG_ERR_INVALID, "out is NULL");
  const McLevel& F = c->lev[c->L];
  MC_CUDA(c, cudaMemcpyAsync(out, F.u, F.nv * c->c * sizeof(cplx<double>),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  if (!on_device) MC_CUDA(c, cudaStreamSynchronize(c->stream));
  return MG_OK;
}

int mg_mc_cycle(mg_mc_ctx* c, int variant, const mg_c128* omega, int transfer) {
  if (c == nullptr) return MG_ERR_INVALID;
  if (omega == nullptr) return fail(c, MG_ERR_INVALID, "omega is NULL");
  if (variant < MG_ADD || variant > MG_BPX || (transfer != MG_DLINEAR && transfer != MG_HIERARCHICAL))
    return fail(c, MG_ERR_INVALID, "variant or transfer out of range");
  std::vector<cplx<double>> om(c->L);
  for (int l = 0; l < c->L; ++l) {
    if (!std::isfinite(omega[l].re) || !std::isfinite(omega[l].im)) return fail(c, MG_ERR_INVALID, "omega is not finite");
    om[l] = {omega[l].re, omega[l].im};
  }
  const int hb = variant == MG_HB ? 1 : 0;
  const int bpx = (variant == MG_BPX || transfer == MG_HIERARCHICAL) && !hb ? 1 : 0;
  MC_CUDA(c, c->d == 2 ? dispatch_cycle<2>(c, hb, bpx, om.data()) : dispatch_cycle<3>(c, hb, bpx, om.data()));
  return MG_OK;
}

int mg_mc_residual_norm(mg_mc_ctx* c, double* abs_l2, double* rel_l2) {
  if (c == nullptr) return MG_ERR_INVALID;
  if (abs_l2 == nullptr) return fail(c, MG_ERR_INVALID, "abs_l2 is NULL");
  const McLevel& F = c->lev[c->L];
  const int nb = blocks_for(F.nv);
  MC_CUDA(c, c->d == 2 ? dispatch_residual<2>(c, c->partial) : dispatch_residual<3>(c, c->partial));
  c->hpart.resize(nb);
  MC_CUDA(c, cudaMemcpyAsync(c->hpart.data(), c->partial, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  MC_CUDA(c, cudaStreamSynchronize(c->stream));
  double s = 0.0;
  for (int k = 0; k < nb; ++k) s += c->hpart[k];  // fixed order: deterministic
  const double a = std::sqrt(s);
  if (!std::isfinite(a)) return fail(c, MG_DIVERGED, "the residual norm is not finite");
  if (c->r0 < 0) c->r0 = a;
  *abs_l2 = a;
  if (rel_l2 != nullptr) *rel_l2 = c->r0 > 0 ? a / c->r0 : 0.0;
  return MG_OK;
}

const char* mg_mc_last_error(const mg_mc_ctx* c) { return c == nullptr ? "" : c->err.c_str(); }

void mg_mc_destroy(mg_mc_ctx* c) {
  if (c == nullptr) return;
  for (void* p : c->allocs) cudaFree(p);
  delete c;
}

}  // extern "C"
