// lb_tile.cuh -- one tile of pairs through the whole path, in one thread block.
//
// The paper sorts all pairs by expression before launching one thread per
// pair (Sec. 4.3), so that warps do not diverge.  Here the grouping happens
// on chip, per tile of NT * LB_ITEMS pairs (NT threads per block):
//   tile_bin   loads the tile (coalesced, two pairs per load instruction),
//              handles domain edges, classifies the rest (Table "input
//              ranges") and sorts the pairs into one shared-memory list by
//              key: the region, and for mu_20 and the power series the
//              estimated term count too, so each region's pairs form one
//              contiguous range of the list, ordered by term count;
//   tile_eval  evaluates the per-thread expressions: warps take 32-pair
//              chunks of the list from shared counters, region by region,
//              so every warp runs a single expression at a time, on lanes
//              that need about the same number of terms; then stores the
//              tile's results coalesced (two per store instruction).
// The per-call kernels (logbessel.cu) and the persistent serving kernel
// (lb_serve.cu) are both built from these two steps; K pairs of the
// fallback region are left in the list for the K integral.
#pragma once

#include "lb_expr.cuh"
#include "lb_expr32.cuh"
#include "lb_kint.cuh"

// Threads per block of the serving kernel and of the K-integral and
// auxiliary kernels; the per-call tile kernel takes its own block size
// (LB_TILE_THREADS in logbessel.cu).  A tile holds LB_ITEMS pairs per thread.
#ifndef LB_THREADS
#define LB_THREADS 256
#endif
#ifndef LB_ITEMS
#define LB_ITEMS 4
#endif
#define LB_TILE (LB_THREADS * LB_ITEMS)            // tile of the serving kernel

namespace lb {

// Checked build (-DLB_CHECKS, liblogbessel_checks.so): every index into the
// tile's shared list, into the K-integral queue, and every pair offset read
// back from the queue is checked against its bound before use; a failed
// check sets a bit of lb_check_status (1 list write, 2 list read, 4 queue
// write, 8 queue count above the capacity, 16 pair offset beyond the chunk,
// 32 rule class out of range) and the access is skipped or clamped.  It
// stands in for a memory checker: the kernels record where an index left
// its buffer instead of faulting.  Release builds compile the checks out.
#ifdef LB_CHECKS
static __device__ unsigned int lb_check_status;
#define LB_CHECK(cond, bit) ((cond) || (atomicOr(&lb_check_status, (unsigned)(bit)), false))
#else
#define LB_CHECK(cond, bit) true
#endif

// List keys.  mu_20 (FP64 values) takes one key per term count n = 1..20,
// found while binning (an unrolled single-precision pass); the power series
// one key per band of x, log-spaced, 3 log2(1 + x) (its term count grows with
// x: rank correlation 0.98), because its exact count is a loop of up to 90
// steps that is cheaper once per 32-pair chunk than once per item round.  So
// each region's pairs come ordered by the number of terms their lanes sum.
// Keys of a region are adjacent; regions come in the order of their list
// ranges.
enum TileKey {
  KEY_MU20 = 0,                  // .. KEY_MU20 + 19
  KEY_U13 = 20,
  KEY_FB = 21,                   // .. KEY_FB + 14: power series (I), K integral (K)
  KEY_MU3 = 36,
  KEY_U4 = 37,
  KEY_U6 = 38,
  KEY_U9 = 39,
  NKEYS = 40
};

__host__ __device__ constexpr int region_key_first(int r) {
  return r == R_MU20 ? KEY_MU20 : r == R_U13 ? KEY_U13 : r == R_FALLBACK ? KEY_FB : r == R_MU3 ? KEY_MU3
       : r == R_U4 ? KEY_U4 : r == R_U6 ? KEY_U6 : KEY_U9;
}
__host__ __device__ constexpr int region_key_end(int r) {
  return r == R_MU20 ? KEY_MU20 + 20 : r == R_FALLBACK ? KEY_FB + 15 : region_key_first(r) + 1;
}

// One tile of NT * LB_ITEMS pairs in the shared memory of a block of NT threads.
template <typename T, int NT>
struct TileShared {
  static constexpr int kThreads = NT;
  static constexpr int kTile = NT * LB_ITEMS;
  T sv[kTile];
  union {                                          // a pair's result replaces its argument
    T sx[kTile];
    T sres[kTile];                                 // results, stored coalesced at the end of the tile
  };
  uint16_t list[kTile];                            // tile offsets of the pairs to evaluate, sorted by key
  uint8_t nt[kTile];                               // estimated term count (mu_20; FP64 values)
  uint8_t keep[kTile];                             // 1: sres holds this pair's result
  uint16_t wcount[LB_ITEMS][NT / 32][NKEYS];       // pairs per (item round, warp, key), then offsets
  int kbeg[NKEYS + 1];                             // start of each key's range in list
  int next_chunk[8];                               // per region: next chunk of 32 pairs to hand out (tile_eval)
  unsigned int qbase;
  // the range of region r in list
  __device__ __forceinline__ int rbeg(int r) const { return kbeg[region_key_first(r)]; }
  __device__ __forceinline__ int rend(int r) const { return kbeg[region_key_end(r)]; }
  __device__ __forceinline__ int rcount(int r) const { return rend(r) - rbeg(r); }
};

template <int KIND, bool DX, typename T>
__device__ __forceinline__ bool tile_special(T v, T x, T* r) {
  if constexpr (sizeof(T) == 8) {
    return DX ? special_dx<KIND>(v, x, r) : special_value<KIND>(v, x, r);
  } else {
    return special_value32<KIND>(v, x, r);
  }
}

template <int KIND, bool DX, typename T>
__device__ __forceinline__ int tile_classify(T v, T x, int mode) {
  if constexpr (sizeof(T) == 8) return classify(v, x, mode, DX ? WIDE_NONE : (KIND == KIND_K ? WIDE_K : WIDE_I));
  else return classify32(v, x, mode, DX ? WIDE_NONE : (KIND == KIND_K ? WIDE_K : WIDE_I));
}

// FP64 values with the lane's term count n (mu_20, series) given.
template <int KIND, bool DX, typename T>
__device__ __forceinline__ T tile_expr(int r, T v, T x, int n) {
  if constexpr (sizeof(T) == 4) {
    switch (r) {
      case R_MU20: return mu_expr32<KIND, 20>(v, x);
      case R_U13: return u_expr32<KIND, 13>(v, x);
      case R_MU3: return mu_expr32<KIND, 3>(v, x);
      case R_U4: return u_expr32<KIND, 4>(v, x);
      case R_U6: return u_expr32<KIND, 6>(v, x);
      case R_U9: return u_expr32<KIND, 9>(v, x);
      default: return (KIND == KIND_I) ? series_log_i32(v, x) : __int_as_float(0x7fc00000);
    }
  } else if constexpr (DX) {
    switch (r) {
      case R_MU20: return mu_dx_n<KIND, 20>(v, x, n);
      case R_U13: return u_dx<KIND, 13>(v, x);
      case R_MU3: return mu_dx<KIND, 3>(v, x);
      case R_U4: return u_dx<KIND, 4>(v, x);
      case R_U6: return u_dx<KIND, 6>(v, x);
      case R_U9: return u_dx<KIND, 9>(v, x);
      default: return (KIND == KIND_I) ? series_dx_n(v, x, n) : __longlong_as_double(0x7ff8000000000000LL);
    }
  } else {
    switch (r) {
      case R_MU20: return mu_expr_n<KIND, 20>(v, x, n);
      case R_U13: return u_expr<KIND, 13>(v, x);
      case R_MU3: return mu_expr<KIND, 3>(v, x);
      case R_U4: return u_expr<KIND, 4>(v, x);
      case R_U6: return u_expr<KIND, 6>(v, x);
      case R_U9: return u_expr<KIND, 9>(v, x);
      default: return (KIND == KIND_I) ? series_log_i_n(v, x, n) : __longlong_as_double(0x7ff8000000000000LL);
    }
  }
}

// List key of a classified pair, and the term count of mu_20 in *n (FP64
// values and x-derivatives; 0 otherwise).
template <int KIND, bool DX, typename T>
__device__ __forceinline__ int tile_key(int r, T v, T x, int* n) {
  *n = 0;
  if constexpr (sizeof(T) == 8) {
    if (r == R_MU20) {
      *n = mu_terms<20>(f32_cut(v), f32_cut(x));
      return KEY_MU20 + *n - 1;
    }
  }
  if (KIND == KIND_I && r == R_FALLBACK)
    return KEY_FB + min(14, (int)(3.0f * __log2f(1.0f + (sizeof(T) == 8 ? f32_cut((double)x) : (float)x))));
  return region_key_first(r);
}

// Tile offset of item round `it` of thread `tid`: each thread handles two
// adjacent pairs per pair of rounds, so it loads and stores them with one
// 16-byte (FP64) or 8-byte (FP32) instruction.
template <int NT>
__device__ __forceinline__ int tile_offset(int it, int tid) {
  return (it >> 1) * (2 * NT) + 2 * tid + (it & 1);
}

template <typename T>
struct Vec2;
template <>
struct Vec2<double> { typedef double2 type; };
template <>
struct Vec2<float> { typedef float2 type; };

// Load, edge-handle, classify and sort pairs [t0, min(t0 + NT * LB_ITEMS, n)).
// All threads of the block call it; it ends with a barrier.  The list is
// ordered by (key, item round, warp, lane), from one warp match per item
// and a per-key prefix over (item round, warp): the order, and so the warp
// mates of every pair, do not depend on scheduling.
template <int KIND, bool DX, typename T, int NT>
__device__ __forceinline__ void tile_bin(TileShared<T, NT>& S, const T* __restrict__ v, int64_t v_stride,
                                         const T* __restrict__ x, int64_t t0, int64_t n, int mode,
                                         int forced_region) {
  typedef typename Vec2<T>::type T2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned int lt = (1u << lane) - 1u;
  // the pair offsets t0 are multiples of the tile size, so aligned bases keep every pair of loads aligned
  const bool vec = ((reinterpret_cast<uintptr_t>(x) | (v_stride ? reinterpret_cast<uintptr_t>(v) : 0)) &
                    (2 * sizeof(T) - 1)) == 0;
  const T v0 = v_stride ? T(0) : v[0];
  T vv[LB_ITEMS], xx[LB_ITEMS];
#pragma unroll
  for (int h = 0; h < LB_ITEMS / 2; ++h) {
    const int li = tile_offset<NT>(2 * h, tid);
    const int64_t i = t0 + li;
    if (vec && i + 1 < n) {
      const T2 xv = *reinterpret_cast<const T2*>(x + i);
      xx[2 * h] = xv.x;
      xx[2 * h + 1] = xv.y;
      if (v_stride) {
        const T2 vw = *reinterpret_cast<const T2*>(v + i);
        vv[2 * h] = vw.x;
        vv[2 * h + 1] = vw.y;
      } else {
        vv[2 * h] = vv[2 * h + 1] = v0;
      }
    } else {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        xx[2 * h + e] = (i + e < n) ? x[i + e] : T(1);
        vv[2 * h + e] = (i + e < n) ? (v_stride ? v[i + e] : v0) : T(0);
      }
    }
  }
  int key[LB_ITEMS], rank[LB_ITEMS];
#pragma unroll
  for (int it = 0; it < LB_ITEMS; ++it) {
    const int li = tile_offset<NT>(it, tid);
    const int64_t i = t0 + li;
    int k = NKEYS;                                 // NKEYS: no list entry
    uint8_t keep = 0;
    if (i < n) {
      T vi = vv[it];
      const T xi = xx[it];
      if constexpr (KIND == KIND_K) {
        if constexpr (sizeof(T) == 8) vi = __longlong_as_double(__double_as_longlong(vi) & 0x7fffffffffffffffLL);
        else vi = fabsf(vi);
      }
      T sp;
      if (tile_special<KIND, DX, T>(vi, xi, &sp)) {
        S.sres[li] = sp;
        keep = 1;
      } else {
        S.sv[li] = vi;
        S.sx[li] = xi;
        const int r = forced_region >= 0 ? forced_region : tile_classify<KIND, DX, T>(vi, xi, mode);
        int nterm;
        k = tile_key<KIND, DX, T>(r, vi, xi, &nterm);
        S.nt[li] = (uint8_t)nterm;
        keep = (KIND == KIND_K && r == R_FALLBACK) ? 0 : 1;   // K integral pairs are stored later
      }
    }
    S.keep[li] = keep;
    // pairs of the same key in this warp: count and rank by lane
    for (int kk = lane; kk < NKEYS; kk += 32) S.wcount[it][warp][kk] = 0;
    __syncwarp();
    const unsigned int m = __match_any_sync(0xffffffffu, k);
    rank[it] = __popc(m & lt);
    if (k < NKEYS && rank[it] == 0) S.wcount[it][warp][k] = (uint16_t)__popc(m);
    key[it] = k;
  }
  __syncthreads();
  // exclusive prefix per key over (item round, warp); the key's total to kbeg
  if (tid < NKEYS) {
    int acc = 0;
    for (int it = 0; it < LB_ITEMS; ++it)
      for (int w = 0; w < NT / 32; ++w) {
        const int c = S.wcount[it][w][tid];
        S.wcount[it][w][tid] = (uint16_t)acc;
        acc += c;
      }
    S.kbeg[tid + 1] = acc;
  }
  __syncthreads();
  // exclusive scan of the key totals (one warp)
  if (warp == 0) {
    int a = S.kbeg[lane + 1], b = lane + 33 <= NKEYS ? S.kbeg[lane + 33] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int ua = __shfl_up_sync(0xffffffffu, a, o), ub = __shfl_up_sync(0xffffffffu, b, o);
      if (lane >= o) { a += ua; b += ub; }
    }
    const int tot_a = __shfl_sync(0xffffffffu, a, 31);
    __syncwarp();
    S.kbeg[lane + 1] = a;
    if (lane + 33 <= NKEYS) S.kbeg[lane + 33] = b + tot_a;
    if (lane == 0) S.kbeg[0] = 0;
  }
  if (tid < 8) S.next_chunk[tid] = 0;
  __syncthreads();
#pragma unroll
  for (int it = 0; it < LB_ITEMS; ++it)
    if (key[it] < NKEYS) {
      const int pos = S.kbeg[key[it]] + S.wcount[it][warp][key[it]] + rank[it];
      if (LB_CHECK(pos >= 0 && pos < (NT * LB_ITEMS), 1u)) S.list[pos] = (uint16_t)tile_offset<NT>(it, tid);
    }
  __syncthreads();
}

// The FP64 expressions with the order's constants of a ScalarOrder block.
template <int KIND>
__device__ __forceinline__ double tile_expr_so(int r, const ScalarOrder& so, double x, int n) {
  switch (r) {
    case R_MU20: return mu_expr_so<KIND>(so, x, n);
    case R_U13: return u_expr_so<KIND, 13>(so, x);
    case R_MU3: return mu_expr<KIND, 3>(so.v, x);
    case R_U4: return u_expr_so<KIND, 4>(so, x);
    case R_U6: return u_expr_so<KIND, 6>(so, x);
    case R_U9: return u_expr_so<KIND, 9>(so, x);
    default: return (KIND == KIND_I) ? series_so(so, x, n) : __longlong_as_double(0x7ff8000000000000LL);
  }
}

// The chunks (32 pairs, one warp each) of region R's range of the list,
// handed out from a shared counter: a warp that runs out moves on to the
// next region while the others finish this one.  Lanes past the end of the
// range recompute the chunk's first entry and do not keep it.  `so` (FP64
// values only) holds the constants of a call whose pairs all have one
// order, or is NULL.
template <int KIND, bool DX, typename T, int R, int NT>
__device__ __forceinline__ void tile_eval_region(TileShared<T, NT>& S, int lane, const ScalarOrder* so) {
  const int b0 = S.rbeg(R), c = S.rend(R) - b0;
  const int nch = (c + 31) >> 5;
  for (;;) {
    int id = 0;
    if (lane == 0) id = atomicAdd(&S.next_chunk[R], 1);
    id = __shfl_sync(0xffffffffu, id, 0);
    if (id >= nch) break;
    const int j0 = id << 5, j = j0 + lane;
    bool ok = j < c;
    int jl = b0 + (ok ? j : j0);
    if (!LB_CHECK(jl >= 0 && jl < (NT * LB_ITEMS), 2u)) {
      jl = 0;                                      // clamped: the warp still runs the expression together
      ok = false;
    }
    const int li = S.list[jl];
    int nterm = S.nt[li];
    if constexpr (sizeof(T) == 8 && KIND == KIND_I && R == R_FALLBACK)
      nterm = series_terms(f32_cut(so ? so->v : (double)S.sv[li]), f32_cut((double)S.sx[li]));
    T val;
    if constexpr (sizeof(T) == 8 && !DX) {
      if (so) val = tile_expr_so<KIND>(R, *so, S.sx[li], nterm);
      else val = tile_expr<KIND, DX, T>(R, S.sv[li], S.sx[li], nterm);
    } else {
      val = tile_expr<KIND, DX, T>(R, S.sv[li], S.sx[li], nterm);
    }
    __syncwarp();                                  // every lane has read its arguments (sres is sx)
    if (ok) S.sres[li] = val;
  }
}

// Per-thread expressions, region by region, costliest first (so that the
// last chunks of a tile are cheap and the warps reach the closing barrier
// close together); every warp runs a single expression at a time, and the
// result of a pair does not depend on which warp takes its chunk.  Then the
// tile's results (domain edges included) are stored, two pairs per
// instruction where both are kept and the buffer is aligned.  The K fallback
// pairs are left to the K integral: neither evaluated nor stored (so out may
// equal x: their arguments stay in place for it).  Ends with a barrier.
template <int KIND, bool DX, typename T, int NT>
__device__ __forceinline__ void tile_eval(TileShared<T, NT>& S, T* __restrict__ out, int64_t t0, int64_t n,
                                          const ScalarOrder* so = nullptr) {
  typedef typename Vec2<T>::type T2;
  const int tid = threadIdx.x, lane = tid & 31;
  if (KIND == KIND_I) tile_eval_region<KIND, DX, T, R_FALLBACK, NT>(S, lane, so);
  tile_eval_region<KIND, DX, T, R_U13, NT>(S, lane, so);
  tile_eval_region<KIND, DX, T, R_U9, NT>(S, lane, so);
  tile_eval_region<KIND, DX, T, R_MU20, NT>(S, lane, so);
  tile_eval_region<KIND, DX, T, R_U6, NT>(S, lane, so);
  tile_eval_region<KIND, DX, T, R_MU3, NT>(S, lane, so);
  tile_eval_region<KIND, DX, T, R_U4, NT>(S, lane, so);
  __syncthreads();
  const bool vec = (reinterpret_cast<uintptr_t>(out) & (2 * sizeof(T) - 1)) == 0;
#pragma unroll
  for (int h = 0; h < LB_ITEMS / 2; ++h) {
    const int li = tile_offset<NT>(2 * h, tid);
    const int64_t i = t0 + li;
    const bool k0 = i < n && S.keep[li], k1 = i + 1 < n && S.keep[li + 1];
    if (vec && k0 && k1) {
      T2 r;
      r.x = S.sres[li];
      r.y = S.sres[li + 1];
      *reinterpret_cast<T2*>(out + i) = r;
    } else {
      if (k0) out[i] = S.sres[li];
      if (k1) out[i + 1] = S.sres[li + 1];
    }
  }
  __syncthreads();
}

// K integral of a batch of up to 32 pairs by one warp: lane e holds pair e;
// each lane computes its pair's prefactor, then the warp evaluates the
// integrals one pair at a time with the nodes spread over the lanes.
// CLS >= 0: every pair is of that rule class (FP64 Gauss values; see
// kint_batch_gauss).
template <bool DX, typename T, int CLS = -1>
__device__ __forceinline__ T kint_warp_batch(T vi, T xi, int m, int lane, bool gauss,
                                            const KintScalar* ks = nullptr, const KintScalar32* ks32 = nullptr) {
  if constexpr (sizeof(T) == 8) {
    if (gauss) return kint_batch_gauss<DX, CLS>(vi, xi, m, lane, ks);
  }
  T pre;
  if constexpr (sizeof(T) == 8) pre = DX ? -(vi / xi + 1.0) : kint_prefactor(vi, xi);
  else pre = kint_prefactor32(vi, xi);
  float beta_i = 0.0f, logbeta_i = 0.0f;
  if constexpr (sizeof(T) == 4) {
    beta_i = 16.0f / (2.0f * vi + 1.0f);
    logbeta_i = logf(beta_i);
  }
  T mine = 0;
  for (int e = 0; e < m; ++e) {
    const T ve = __shfl_sync(0xffffffffu, vi, e);
    const T xe = __shfl_sync(0xffffffffu, xi, e);
    T li;
    if constexpr (sizeof(T) == 8) {
      li = kint_log_simpson(ve, xe, lane);
    } else {
      const float be = __shfl_sync(0xffffffffu, beta_i, e);
      const float lbe = __shfl_sync(0xffffffffu, logbeta_i, e);
      li = kint_gauss32(ve, xe, be, lbe, lane, ks32);
    }
    if (lane == e) mine = li;
  }
  return pre + mine;
}

}  // namespace lb
