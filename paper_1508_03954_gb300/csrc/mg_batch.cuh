// mg_batch.cuh -- batched persistent launch: one outer defect-correction
// iteration for many independent 2D problems of uneven depth (sm_103a).
//
// Per problem p one launch runs, in order:
//   R   FP64 residual r = b - H u of the fine level into the complex64
//       right-hand side of the inner problem, with |r|^2 (the norm of the
//       iterate entering this outer step);
//   m inner complex64 cycles on H e = r from e = 0: fine sweep items (warp
//       strips of mg_sweep2w.cuh on levels with n >= 27, tiles below),
//       coarse sweep items of levels L-1 .. 1, then the correction stages
//       (corr_{L-2} from levels 1..L-2, corr_{L-1} = t_{L-1} + P corr_{L-2});
//   U   FP64 update u += e (e = E + P corr_{L-1}).
// The items of all problems form one queue in stage-major order; a block
// takes the next item and waits (bounded) until its problem's counter shows
// that the earlier stages of that problem are complete (see mg_persist.cuh
// for why this cannot deadlock).  Problems already converged are marked
// inactive and their items complete at once, so the same item list, and the
// CUDA graph that launches it, serve every outer iteration.
#pragma once
#include "mg_persist.cuh"
#include "mg_sweep2w.cuh"

namespace mg {

enum : int { kBRes = 0, kBSweep = 1, kBSweepS = 2, kBCorr = 3, kBUpd = 4, kBStrip = 5 };

// strip items: coarse rows per item (8 warps of about 6 rows each)
constexpr int kStripUnits = 48;

struct ResArgs {
  int n, nchunks;
  const cplx<double>* u;
  const cplx<double>* b;
  cplx<float>* out;
  const uint8_t* typ;
  const cplx<double>* coef;  // [16][9]
  double* partial;
  unsigned* ticket;
  double* norm2;
};

struct UpdArgs {
  int n;
  cplx<double>* u;
  const cplx<float>* e;  // fine E
  const cplx<float>* c;  // pending corr on level L-1 (may be null)
};

using CorrArgsF = CorrArgs<float>;

constexpr int kBatchChunk = 1024;

struct BatchArgs {
  const ChainItem* items;
  int nitems;
  const Sweep2Args<float>* sw;
  const Sweep2wArgs* st;
  const ResArgs* res;
  const UpdArgs* upd;
  const CorrArgsF* co;
  const int* active;      // per problem
  unsigned* head;
  unsigned* done;         // per problem
  unsigned* err;
  unsigned spin_limit;
};

template <int NTHR>
__device__ __forceinline__ void res_chunk(const ResArgs& A, int chunk, double* s_red) {
  const int n = A.n, N = n + 1;
  const long long total = (long long)N * N;
  double nrm = 0.0;
  for (long long i = (long long)chunk * kBatchChunk + threadIdx.x;
       i < (long long)(chunk + 1) * kBatchChunk && i < total; i += NTHR) {
    const int gx = (int)((unsigned)i % (unsigned)N), gy = (int)((unsigned)i / (unsigned)N);
    cplx<double> r = cz<double>();
    if (gx > 0 && gx < n && gy > 0 && gy < n) {
      const int t = A.typ[gx] + 4 * A.typ[gy];
      const cplx<double>* cf = A.coef + t * 9;
      r = ldcg_(A.b + i);
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const long long j = i + (long long)(k / 3 - 1) * N + (k % 3 - 1);
        const cplx<double> uk = ldcg_(A.u + j);
        const cplx<double> a = cf[k];
        r.x = fma(-a.x, uk.x, r.x);
        r.x = fma(a.y, uk.y, r.x);
        r.y = fma(-a.x, uk.y, r.y);
        r.y = fma(-a.y, uk.x, r.y);
      }
      nrm = fma(r.x, r.x, fma(r.y, r.y, nrm));
    }
    A.out[i] = cplx<float>{(float)r.x, (float)r.y};
  }
  block_norm_finish_tile<NTHR>(nrm, s_red, A.partial, A.ticket, A.norm2, chunk, A.nchunks);
}

template <int NTHR>
__device__ __forceinline__ void upd_chunk(const UpdArgs& A, int chunk) {
  const int n = A.n, N = n + 1, Nc = n / 3 + 1;
  const long long total = (long long)N * N;
  for (long long i = (long long)chunk * kBatchChunk + threadIdx.x;
       i < (long long)(chunk + 1) * kBatchChunk && i < total; i += NTHR) {
    const int gx = (int)((unsigned)i % (unsigned)N), gy = (int)((unsigned)i / (unsigned)N);
    if (!(gx > 0 && gx < n && gy > 0 && gy < n)) continue;
    cplx<float> v = ldcg_(A.e + i);
    if (A.c != nullptr) {
      const int cx = gx / 3, cy = gy / 3, ox = gx % 3, oy = gy % 3;
      const cplx<float>* cp = A.c + (long long)cy * Nc + cx;
      const float wx0 = ox == 0 ? 1.f : (ox == 1 ? 2.f / 3.f : 1.f / 3.f), wx1 = 1.f - wx0;
      const float wy0 = oy == 0 ? 1.f : (oy == 1 ? 2.f / 3.f : 1.f / 3.f), wy1 = 1.f - wy0;
      const cplx<float> a0 = ldcg_(cp), a1 = ox ? ldcg_(cp + 1) : cz<float>();
      const cplx<float> b0 = oy ? ldcg_(cp + Nc) : cz<float>();
      const cplx<float> b1 = (ox && oy) ? ldcg_(cp + Nc + 1) : cz<float>();
      v.x += wy0 * (wx0 * a0.x + wx1 * a1.x) + wy1 * (wx0 * b0.x + wx1 * b1.x);
      v.y += wy0 * (wx0 * a0.y + wx1 * a1.y) + wy1 * (wx0 * b0.y + wx1 * b1.y);
    }
    cplx<double> o = ldcg_(A.u + i);
    o.x += (double)v.x;
    o.y += (double)v.y;
    A.u[i] = o;
  }
}

template <int NTHR>
__device__ __forceinline__ void corrf_chunk(const CorrArgsF& A, int chunk) {
  const int s = A.s;
  int n = 1;
  for (int k = 0; k < s; ++k) n *= 3;
  const int N = n + 1;
  const long long total = (long long)N * N;
  for (long long i = (long long)chunk * kBatchChunk + threadIdx.x;
       i < (long long)(chunk + 1) * kBatchChunk && i < total; i += NTHR) {
    const int gx = (int)((unsigned)i % (unsigned)N), gy = (int)((unsigned)i / (unsigned)N);
    cplx<float> v = cz<float>();
    if (gx > 0 && gx < n && gy > 0 && gy < n) {
      v = ldcg_(A.t[s] + i);
      int f = 1;
      float ik = 1.f;
      for (int l = s - 1; l >= A.lo - 1 && l >= 0; --l) {
        f *= 3;
        ik *= 1.f / 3.f;
        const cplx<float>* src = l >= A.lo ? A.t[l] : A.base;
        if (src == nullptr) break;
        const int Nl = n / f + 1;
        const int cx = gx / f, cy = gy / f, ox = gx - cx * f, oy = gy - cy * f;
        const float wx1 = (float)ox * ik, wy1 = (float)oy * ik, wx0 = 1.f - wx1, wy0 = 1.f - wy1;
        const cplx<float>* tp = src + (long long)cy * Nl + cx;
        const cplx<float> a0 = ldcg_(tp), a1 = ox ? ldcg_(tp + 1) : cz<float>();
        const cplx<float> b0 = oy ? ldcg_(tp + Nl) : cz<float>();
        const cplx<float> b1 = (ox && oy) ? ldcg_(tp + Nl + 1) : cz<float>();
        v.x += wy0 * (wx0 * a0.x + wx1 * a1.x) + wy1 * (wx0 * b0.x + wx1 * b1.x);
        v.y += wy0 * (wx0 * a0.y + wx1 * a1.y) + wy1 * (wx0 * b0.y + wx1 * b1.y);
      }
    }
    A.out[i] = v;
  }
}

// TC: tile of the fine sweeps (autotuned); coarse levels below a size use 2.
template <int TC, int NTHR>
__global__ void __launch_bounds__(NTHR, 2) batch2_kernel(const BatchArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double s_red[NTHR / 32];
  __shared__ int s_item;
  __shared__ __align__(16) union U {
    Sweep2Args<float> sw;
    ResArgs res;
    UpdArgs upd;
    CorrArgsF co;
    Sweep2wArgs st;
  } s_a;
  while (true) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(A.head, 1u);
    __syncthreads();
    const int i = s_item;
    if (i >= A.nitems) break;
    const ChainItem it = A.items[i];
    const bool act = A.active[it.prob] != 0;
    if (act) {
      switch (it.kind) {
        case kBRes: copy_args<ResArgs, NTHR>(&s_a.res, A.res + it.args); break;
        case kBUpd: copy_args<UpdArgs, NTHR>(&s_a.upd, A.upd + it.args); break;
        case kBCorr: copy_args<CorrArgsF, NTHR>(&s_a.co, A.co + it.args); break;
        case kBStrip: copy_args<Sweep2wArgs, NTHR>(&s_a.st, A.st + it.args); break;
        default: copy_args<Sweep2Args<float>, NTHR>(&s_a.sw, A.sw + it.args); break;
      }
      if (threadIdx.x == 0 && it.need > 0) wait_counter(A.done + it.prob, it.need, A.spin_limit, A.err);
    }
    __syncthreads();
    if (act) {
      switch (it.kind) {
        case kBRes: res_chunk<NTHR>(s_a.res, it.tile, s_red); break;
        case kBUpd: upd_chunk<NTHR>(s_a.upd, it.tile); break;
        case kBCorr: corrf_chunk<NTHR>(s_a.co, it.tile); break;
        case kBSweep: sweep2_tile<TC, NTHR, float>(s_a.sw, it.tile, smem_raw, s_red); break;
        case kBStrip: {
          // each warp takes an equal share of the item's coarse rows
          const int ub = it.tile * kStripUnits, ue = min(s_a.st.nunits, ub + kStripUnits);
          const int w = threadIdx.x >> 5, nw = NTHR / 32;
          strip2w_run(s_a.st, ub + (ue - ub) * w / nw, ub + (ue - ub) * (w + 1) / nw, &s_a.st.row[0][0],
                      s_a.st.omd);
        } break;
        default: sweep2_tile<2, NTHR, float>(s_a.sw, it.tile, smem_raw, s_red); break;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(A.done + it.prob, 1u);
    }
  }
}

}  // namespace mg
