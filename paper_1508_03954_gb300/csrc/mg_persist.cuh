// mg_persist.cuh -- persistent dataflow launch for the coarse part of a
// cycle (sm_103a).
//
// After the fine sweep, a cycle is a chain of small steps: the sweeps of
// levels L-1 .. 1 (each needs the whole finer level's restriction) and the
// prolongations corr_l = T_l du_l + P corr_{l-1} for l = 2 .. L-1 (each needs
// the coarser one).  On GB300 each of these is far too small to fill the
// machine and one launch per step costs more than the step.  Here one launch
// runs the whole chain (and, for batches, the chains of many problems): every
// block repeatedly takes the next work item (stage, tile) from a queue in
// topological order and, before working on it, waits until its problem's
// completion counter shows that every item of the earlier stages is done.
// Items are taken in index order and only wait on items with smaller
// indices, which running blocks already hold, so the scheme cannot deadlock
// and needs no cooperative launch.  Every wait is bounded: when the bound
// runs out the block sets an error flag and carries on, so a launch always
// ends and the host reports MG_ERR_TIMEOUT.
#pragma once
#include "mg_sweep2d.cuh"

#ifndef MG_BACKOFF_MAX_NS
#define MG_BACKOFF_MAX_NS 256
#endif

namespace mg {

enum : int { kItemSweep2 = 0, kItemProlong2 = 1, kItemCorr2 = 2, kItemSweep2s = 3, kItemSweep2t = 4 };

struct ChainItem {
  int kind;       // kItemSweep2 / kItemProlong2
  int prob;       // problem index (completion counter)
  int args;       // index into the argument table of its kind
  int tile;       // tile (sweep) or chunk (prolongation)
  unsigned need;  // items of this problem that must be complete first
};

template <typename R>
struct ProlongArgs {
  int n;                  // cells per axis of the level
  const cplx<R>* t;       // T du of the level
  const cplx<R>* cc;      // corr of the next coarser level
  cplx<R>* out;           // corr of the level
};

constexpr int kProlongChunk = 2048;  // vertices per prolongation item

// corr_s = t_s + sum_{l=lo..s-1} P^{s-l} t_l + P^{s-lo+1} base on level s,
// evaluated at every vertex by direct d-linear interpolation from each
// coarser level: on nested d-linear spaces P^k is exactly the interpolation
// over the 3^k-refined cell.  base is corr_{lo-1} (or null).
constexpr int kMaxChainLevels = 12;
template <typename R>
struct CorrArgs {
  int s, lo;                          // target level (3^s cells), first level summed
  int chunk;                          // vertices per item (chain); 0: kCorrChunk
  const cplx<R>* t[kMaxChainLevels];  // t[l] for l = lo..s (index l)
  const cplx<R>* base;                // corr_{lo-1} or null
  cplx<R>* out;                       // corr_s
};
constexpr int kCorrChunk = 256;          // vertices per item unless the plan sets one

template <typename R>
struct ChainArgs {
  const ChainItem* items;
  int nitems;
  const Sweep2Args<R>* s2;
  const ProlongArgs<R>* pr;
  const CorrArgs<R>* co;
  unsigned* head;        // queue head, zero at launch
  unsigned* exitc;       // blocks that left the queue; the last one zeroes the counters
  // first-stage items may wait for single fine tiles instead of the whole
  // fine sweep: fine_flags[t] >= *gen + 1 once fine tile t is written (null:
  // wait for the whole fine grid); the chain's last block advances *gen
  const unsigned* fine_flags;
  unsigned* gen;
  int fine_tiles_x;      // fine tiles (8 coarse cells) per axis
  int first_tiles_x;     // tiles (4 cells) per axis of the first chain level
  unsigned* done;        // per-problem completion counters, zero at launch
  unsigned* err;         // set when a bounded wait gave up
  unsigned spin_limit;   // polls before giving up
  unsigned long long* trace;  // optional: per item {taken, ready, done, sm} (ns, globaltimer)
  const unsigned* stall;      // diagnostic: the first item also waits for *stall >= 1 (nothing sets it)
};

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned smid() {
  unsigned r;
  asm volatile("mov.u32 %0, %smid;" : "=r"(r));
  return r;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// corr_l = t_l + P corr_{l-1} on vertices [chunk*kProlongChunk, ...) of a 2D level
template <int NTHR, typename R>
__device__ __forceinline__ void prolong2_chunk(const ProlongArgs<R>& A, int chunk) {
  const int n = A.n, N = n + 1, Nc = n / 3 + 1;
  const long long total = (long long)N * N;
  const long long beg = (long long)chunk * kProlongChunk;
  for (long long i = beg + threadIdx.x; i < beg + kProlongChunk && i < total; i += NTHR) {
    const int gx = (int)((unsigned)i % (unsigned)N), gy = (int)((unsigned)i / (unsigned)N);
    cplx<R> v = cz<R>();
    if (gx > 0 && gx < n && gy > 0 && gy < n) {
      v = ldcg(A.t + i);
      const int cx = gx / 3, cy = gy / 3, ox = gx % 3, oy = gy % 3;
      const cplx<R>* cp = A.cc + (long long)cy * Nc + cx;
      const cplx<R> a = lerp2(w0<R>(ox), ldcg(cp), w1<R>(ox), ldcg(cp + (ox ? 1 : 0)));
      const cplx<R> b = oy ? lerp2(w0<R>(ox), ldcg(cp + Nc), w1<R>(ox), ldcg(cp + Nc + (ox ? 1 : 0)))
                                : cz<R>();
      v = lerp2acc(v, w0<R>(oy), a, w1<R>(oy), b);
    }
    A.out[i] = v;
  }
}

// 1/3^k for k = 0..12 (interpolation weights without division)
template <typename R>
__device__ __forceinline__ R inv_pow3(int k) {
  R r = R(1);
  for (int i = 0; i < k; ++i) r *= (R(1) / R(3));
  return r;
}

template <int NTHR, typename R>
__device__ __forceinline__ void corr2_chunk(const CorrArgs<R>& A, int chunk) {
  const int s = A.s;
  int n = 1;
  for (int k = 0; k < s; ++k) n *= 3;
  const int N = n + 1;
  const long long total = (long long)N * N;
  const int csz = A.chunk > 0 ? A.chunk : kCorrChunk;
  for (long long i = (long long)chunk * csz + threadIdx.x; i < (long long)(chunk + 1) * csz && i < total;
       i += NTHR) {
    const int gx = (int)((unsigned)i % (unsigned)N), gy = (int)((unsigned)i / (unsigned)N);
    cplx<R> v = cz<R>();
    if (gx > 0 && gx < n && gy > 0 && gy < n) {
      v = ldcg(A.t[s] + i);
      int f = 1, k = 0;  // f = 3^(s-l)
      for (int l = s - 1; l >= A.lo - 1 && l >= 0; --l) {
        f *= 3;
        ++k;
        const cplx<R>* src = l >= A.lo ? A.t[l] : A.base;
        if (src == nullptr) break;
        const int nl = n / f, Nl = nl + 1;
        const int cx = gx / f, cy = gy / f, ox = gx - cx * f, oy = gy - cy * f;
        const R ik = inv_pow3<R>(k);
        const R wx1 = (R)ox * ik, wy1 = (R)oy * ik;
        const R wx0 = R(1) - wx1, wy0 = R(1) - wy1;
        const cplx<R>* tp = src + (long long)cy * Nl + cx;
        const cplx<R> a = lerp2(wx0, ldcg(tp), wx1, ldcg(tp + (ox ? 1 : 0)));
        const cplx<R> b = oy ? lerp2(wx0, ldcg(tp + Nl), wx1, ldcg(tp + Nl + (ox ? 1 : 0)))
                                  : cz<R>();
        v = lerp2acc(v, wy0, a, wy1, b);
      }
    }
    A.out[i] = v;
  }
}

// Copies a small argument struct from global to shared memory (the tile code
// then reads its fields with shared loads instead of re-reading global
// memory after every store).
template <typename T, int NTHR>
__device__ __forceinline__ void copy_args(T* dst, const T* src) {
  static_assert(sizeof(T) % 4 == 0, "4-byte granularity");
  const unsigned* s = reinterpret_cast<const unsigned*>(src);
  unsigned* d = reinterpret_cast<unsigned*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(T) / 4); i += NTHR) d[i] = __ldcg(s + i);
}

// Bounded wait of thread 0 until *ctr >= need, polling with exponential
// backoff (64 .. 256 ns) so that waiting blocks do not crowd the L2 slice
// that holds the counter.
__device__ __forceinline__ void wait_counter(const unsigned* ctr, unsigned need, unsigned spin_limit,
                                             unsigned* err) {
  unsigned spins = 0, ns = 64;
  while (ld_acquire_u32(ctr) < need) {
    if (++spins > spin_limit) {
      atomicOr(err, 1u);
      return;
    }
    __nanosleep(ns);
    if (ns < MG_BACKOFF_MAX_NS) ns <<= 1;
  }
}

// Programmatic dependent launch: a dependent grid may start before the grid it
// follows has finished; it waits here until that grid's writes are visible.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
// Lets the dependent grid be scheduled once every block has passed this point.
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
// The last block to leave a persistent queue zeroes its counters for the
// next launch (no memset node between launches).
__device__ __forceinline__ void queue_exit(unsigned* exitc, unsigned* a, unsigned* b,
                                           unsigned* gen = nullptr) {
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(exitc, 1u) == gridDim.x - 1) {
      *a = 0u;
      if (b != nullptr) *b = 0u;
      if (gen != nullptr) atomicAdd(gen, 1u);
      *exitc = 0u;
      __threadfence();
    }
  }
}

template <int NTHR, typename R = double>
__global__ void __launch_bounds__(NTHR) chain2_kernel(const ChainArgs<R> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double s_red[NTHR / 32];
  __shared__ int s_item;
  __shared__ __align__(16) Sweep2Args<R> s_a;
  __shared__ __align__(16) ProlongArgs<R> s_p;
  __shared__ __align__(16) CorrArgs<R> s_co;
  const bool tdep = A.fine_flags != nullptr;
  if (!tdep) pdl_wait();
  // generation of this cycle (the fine sweep read the same value)
  const unsigned gen = (tdep && threadIdx.x == 0) ? ld_acquire_u32(A.gen) : 0u;
  while (true) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(A.head, 1u);
    __syncthreads();
    const int i = s_item;
    if (i >= A.nitems) {
      queue_exit(A.exitc, A.head, A.done, A.gen);
      break;
    }
    const ChainItem it = A.items[i];
    unsigned long long t0 = 0, t1 = 0;
    if (A.trace != nullptr && threadIdx.x == 0) t0 = gtimer();
    if (it.kind == kItemSweep2 || it.kind == kItemSweep2s || it.kind == kItemSweep2t)
      copy_args<Sweep2Args<R>, NTHR>(&s_a, A.s2 + it.args);
    else if (it.kind == kItemProlong2) copy_args<ProlongArgs<R>, NTHR>(&s_p, A.pr + it.args);
    else copy_args<CorrArgs<R>, NTHR>(&s_co, A.co + it.args);
    if (threadIdx.x == 0 && it.need > 0) wait_counter(A.done + it.prob, it.need, A.spin_limit, A.err);
    if (threadIdx.x == 0 && tdep && it.need == 0 && it.kind == kItemSweep2) {
      // the fine tiles (8 cells) that wrote u and b on this tile's box, fine
      // vertices [12 t - 3, 12 t + 13] per axis of the first chain level
      const int tx = it.tile % A.first_tiles_x, ty = it.tile / A.first_tiles_x;
      const int fx0 = max(0, (12 * tx - 3) / 8), fx1 = min(A.fine_tiles_x - 1, (12 * tx + 13) / 8);
      const int fy0 = max(0, (12 * ty - 3) / 8), fy1 = min(A.fine_tiles_x - 1, (12 * ty + 13) / 8);
      for (int fy = fy0; fy <= fy1; ++fy)
        for (int fx = fx0; fx <= fx1; ++fx)
          wait_counter(A.fine_flags + fy * A.fine_tiles_x + fx, gen + 1u, A.spin_limit, A.err);
    }
    if (threadIdx.x == 0 && i == 0 && A.stall != nullptr) wait_counter(A.stall, 1u, A.spin_limit, A.err);
    if (A.trace != nullptr && threadIdx.x == 0) t1 = gtimer();
    __syncthreads();
    if (it.kind == kItemSweep2) {
      sweep2_tile<4, NTHR, R>(s_a, it.tile, smem_raw, s_red);
    } else if (it.kind == kItemSweep2s) {
      sweep2_tile<2, NTHR, R>(s_a, it.tile, smem_raw, s_red);
    } else if (it.kind == kItemSweep2t) {
      sweep2_tile<1, NTHR, R>(s_a, it.tile, smem_raw, s_red);
    } else if (it.kind == kItemProlong2) {
      prolong2_chunk<NTHR, R>(s_p, it.tile);
    } else {
      corr2_chunk<NTHR, R>(s_co, it.tile);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(A.done + it.prob, 1u);
      if (A.trace != nullptr) {
        unsigned long long* tr = A.trace + 4ull * i;
        tr[0] = t0;
        tr[1] = t1;
        tr[2] = gtimer();
        tr[3] = smid();
      }
    }
  }
}

// Finest-level sweep as a persistent launch: blocks take tiles from a queue
// ordered by decreasing cost (tiles with complex rows first), so that the
// uneven cost of scaling-layer tiles evens out over the SMs.
template <int TC, int NTHR, typename R = double>
__global__ void __launch_bounds__(NTHR) sweep2p_kernel(const Sweep2Args<R> A, const int* order,
                                                       unsigned* head, unsigned long long* trace,
                                                       unsigned* tflags, const unsigned* gen) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double s_red[NTHR / 32];
  __shared__ int s_k;
  // every block of this grid is resident from the start (one wave), so the
  // coarse chain may be scheduled on SMs as soon as they free up; it waits
  // for this grid's writes before it reads anything
  pdl_launch_dependents();
  const unsigned g = (tflags != nullptr && threadIdx.x == 0) ? ld_acquire_u32(gen) : 0u;
  while (true) {
    if (threadIdx.x == 0) s_k = (int)atomicAdd(head, 1u);
    __syncthreads();
    const int k = s_k;
    if (k >= A.ntiles) {
      queue_exit(head + 1, head, nullptr);
      break;
    }
    const unsigned long long t0 = (trace != nullptr && threadIdx.x == 0) ? gtimer() : 0ull;
    sweep2_tile<TC, NTHR, R>(A, order[k], smem_raw, s_red);
    __syncthreads();
    if (tflags != nullptr && threadIdx.x == 0) {
      // publish this tile's coarse outputs to the chain's first stage
      __threadfence();
      atomicExch(tflags + order[k], g + 1u);
    }
    if (trace != nullptr && threadIdx.x == 0) {
      unsigned long long* tr = trace + 4ull * k;
      tr[0] = t0;
      tr[1] = t0;
      tr[2] = gtimer();
      tr[3] = smid();
    }
  }
}

}  // namespace mg
