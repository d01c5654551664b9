// lb_tile.cuh -- one tile of pairs through the whole path, in one thread block.
//
// The paper sorts all pairs by expression before launching one thread per
// pair (Sec. 4.3), so that warps do not diverge.  Here the grouping happens
// on chip, per tile of LB_TILE pairs:
//   tile_bin   loads the tile (coalesced), writes domain-edge results,
//              classifies the rest (Table "input ranges") and appends each
//              pair's index to a shared-memory list per region;
//   tile_eval  evaluates the per-thread expressions: warps take 32-pair
//              chunks of the lists from shared counters, region by region,
//              so every warp runs a single expression at a time;
//   tile_kint  evaluates the K integral of the tile's fallback pairs, one
//              warp per pair, 32 pairs per warp batch.
// The per-call kernels (logbessel.cu) and the persistent serving kernel
// (lb_serve.cu) are both built from these three steps.
#pragma once

#include "lb_expr.cuh"
#include "lb_expr32.cuh"
#include "lb_kint.cuh"

#define LB_THREADS 256
#define LB_ITEMS 4
#define LB_TILE (LB_THREADS * LB_ITEMS)

namespace lb {

template <typename T>
struct TileShared {
  T sv[LB_TILE];
  T sx[LB_TILE];
  uint16_t lists[8][LB_TILE];
  int counts[8];
  unsigned int qbase;
  uint16_t wcount[LB_ITEMS][LB_THREADS / 32][8];   // pairs per (item round, warp, region), then offsets
  int next_chunk[8];                               // per region: next chunk of 32 pairs to hand out (tile_eval)
};

template <int KIND, bool DX, typename T>
__device__ __forceinline__ bool tile_special(T v, T x, T* r) {
  if constexpr (sizeof(T) == 8) {
    return DX ? special_dx<KIND>(v, x, r) : special_value<KIND>(v, x, r);
  } else {
    return special_value32<KIND>(v, x, r);
  }
}

template <typename T>
__device__ __forceinline__ int tile_classify(T v, T x, int mode) {
  if constexpr (sizeof(T) == 8) return classify(v, x, mode);
  else return classify32(v, x, mode);
}

template <int KIND, bool DX, typename T>
__device__ __forceinline__ T tile_expr(int r, T v, T x) {
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
      case R_MU20: return mu_dx<KIND, 20>(v, x);
      case R_U13: return u_dx<KIND, 13>(v, x);
      case R_MU3: return mu_dx<KIND, 3>(v, x);
      case R_U4: return u_dx<KIND, 4>(v, x);
      case R_U6: return u_dx<KIND, 6>(v, x);
      case R_U9: return u_dx<KIND, 9>(v, x);
      default: return (KIND == KIND_I) ? series_dx(v, x) : __longlong_as_double(0x7ff8000000000000LL);
    }
  } else {
    switch (r) {
      case R_MU20: return mu_expr<KIND, 20>(v, x);
      case R_U13: return u_expr<KIND, 13>(v, x);
      case R_MU3: return mu_expr<KIND, 3>(v, x);
      case R_U4: return u_expr<KIND, 4>(v, x);
      case R_U6: return u_expr<KIND, 6>(v, x);
      case R_U9: return u_expr<KIND, 9>(v, x);
      default: return (KIND == KIND_I) ? series_log_i(v, x) : __longlong_as_double(0x7ff8000000000000LL);
    }
  }
}

// Load, edge-handle, classify and bin pairs [t0, min(t0 + LB_TILE, n)).
// All threads of the block call it; it ends with a barrier.  Binning is by
// warp ballots and a per-region prefix over (item round, warp), so every
// region list comes out in increasing pair order: the result of a pair does
// not depend on scheduling (the warp-uniform term counts see the same warp
// mates on every run) and the stores of a list are as contiguous as possible.
template <int KIND, bool DX, typename T>
__device__ __forceinline__ void tile_bin(TileShared<T>& S, const T* __restrict__ v, int64_t v_stride,
                                         const T* __restrict__ x, T* __restrict__ out, int64_t t0,
                                         int64_t n, int mode, int forced_region) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned int lt = (1u << lane) - 1u;
  int reg[LB_ITEMS];
  int rank[LB_ITEMS];
#pragma unroll
  for (int it = 0; it < LB_ITEMS; ++it) {
    const int li = it * LB_THREADS + tid;
    const int64_t i = t0 + li;
    int r = -1;
    if (i < n) {
      T vi = v[i * v_stride];
      const T xi = x[i];
      if (KIND == KIND_K) vi = fabs(vi);
      T sp;
      if (tile_special<KIND, DX, T>(vi, xi, &sp)) {
        out[i] = sp;
      } else {
        S.sv[li] = vi;
        S.sx[li] = xi;
        r = forced_region >= 0 ? forced_region : tile_classify<T>(vi, xi, mode);
      }
    }
    reg[it] = r;
    rank[it] = 0;
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) {
      const unsigned int m = __ballot_sync(0xffffffffu, r == rr);
      if (r == rr) rank[it] = __popc(m & lt);
      if (lane == rr) S.wcount[it][warp][rr] = (uint16_t)__popc(m);
    }
  }
  __syncthreads();
  // exclusive prefix per region over (item round, warp), in pair order; the
  // region's total goes to counts[]
  if (tid < 8) {
    int acc = 0;
    for (int it = 0; it < LB_ITEMS; ++it)
      for (int w = 0; w < LB_THREADS / 32; ++w) {
        const int c = S.wcount[it][w][tid];
        S.wcount[it][w][tid] = (uint16_t)acc;
        acc += c;
      }
    S.counts[tid] = acc;
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < LB_ITEMS; ++it)
    if (reg[it] >= 0) S.lists[reg[it]][S.wcount[it][warp][reg[it]] + rank[it]] = (uint16_t)(it * LB_THREADS + tid);
  if (tid < 8) S.next_chunk[tid] = 0;
  __syncthreads();
}

// The FP64 expressions with the order's constants of a ScalarOrder block.
template <int KIND>
__device__ __forceinline__ double tile_expr_so(int r, const ScalarOrder& so, double x) {
  switch (r) {
    case R_MU20: return mu_expr_so<KIND>(so, x);
    case R_U13: return u_expr_so<KIND, 13>(so, x);
    case R_MU3: return mu_expr<KIND, 3>(so.v, x);
    case R_U4: return u_expr_so<KIND, 4>(so, x);
    case R_U6: return u_expr_so<KIND, 6>(so, x);
    case R_U9: return u_expr_so<KIND, 9>(so, x);
    default: return (KIND == KIND_I) ? series_so(so, x) : __longlong_as_double(0x7ff8000000000000LL);
  }
}

// The chunks (32 pairs, one warp each) of region R's list, handed out from a
// shared counter: a warp that runs out moves on to the next region while the
// others finish this one.  Lanes past the end of the list recompute the
// chunk's first entry and do not store.  `so` (FP64 values only) holds the
// constants of a call whose pairs all have one order, or is NULL.
template <int KIND, bool DX, typename T, int R>
__device__ __forceinline__ void tile_eval_region(TileShared<T>& S, T* __restrict__ out, int64_t t0, int lane,
                                                 const ScalarOrder* so) {
  const int c = S.counts[R];
  const int nch = (c + 31) >> 5;
  for (;;) {
    int id = 0;
    if (lane == 0) id = atomicAdd(&S.next_chunk[R], 1);
    id = __shfl_sync(0xffffffffu, id, 0);
    if (id >= nch) break;
    const int j0 = id << 5, j = j0 + lane;
    const bool ok = j < c;
    const int li = S.lists[R][ok ? j : j0];
    T val;
    if constexpr (sizeof(T) == 8 && !DX) {
      if (so) val = tile_expr_so<KIND>(R, *so, S.sx[li]);
      else val = tile_expr<KIND, DX, T>(R, S.sv[li], S.sx[li]);
    } else {
      val = tile_expr<KIND, DX, T>(R, S.sv[li], S.sx[li]);
    }
    if (ok) out[t0 + li] = val;
  }
}

// Per-thread expressions, region by region, costliest first (so that the
// last chunks of a tile are cheap and the warps reach the closing barrier
// close together); every warp runs a single expression at a time, and the
// result of a pair does not depend on which warp takes its chunk.  The K
// fallback list is left for tile_kint or a queue.
template <int KIND, bool DX, typename T>
__device__ __forceinline__ void tile_eval(TileShared<T>& S, T* __restrict__ out, int64_t t0,
                                          const ScalarOrder* so = nullptr) {
  const int lane = threadIdx.x & 31;
  if (KIND == KIND_I) tile_eval_region<KIND, DX, T, R_FALLBACK>(S, out, t0, lane, so);
  tile_eval_region<KIND, DX, T, R_U13>(S, out, t0, lane, so);
  tile_eval_region<KIND, DX, T, R_U9>(S, out, t0, lane, so);
  tile_eval_region<KIND, DX, T, R_MU20>(S, out, t0, lane, so);
  tile_eval_region<KIND, DX, T, R_U6>(S, out, t0, lane, so);
  tile_eval_region<KIND, DX, T, R_MU3>(S, out, t0, lane, so);
  tile_eval_region<KIND, DX, T, R_U4>(S, out, t0, lane, so);
}

// K integral of a batch of up to 32 pairs by one warp: lane e holds pair e;
// each lane computes its pair's prefactor, then the warp evaluates the
// integrals one pair at a time with the nodes spread over the lanes.
template <bool DX, typename T>
__device__ __forceinline__ T kint_warp_batch(T vi, T xi, int m, int lane, bool gauss,
                                            const KintScalar* ks = nullptr, const KintScalar32* ks32 = nullptr) {
  if constexpr (sizeof(T) == 8) {
    if (gauss) return kint_batch_gauss<DX>(vi, xi, m, lane, ks);
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

// The tile's K fallback pairs, in block: warp w takes pairs 32w.., 32(w+W)...
template <bool DX, typename T>
__device__ __forceinline__ void tile_kint(TileShared<T>& S, T* __restrict__ out, int64_t t0, bool gauss) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int c = S.counts[R_FALLBACK];
  for (int b = warp * 32; b < c; b += nw * 32) {
    const int j = b + lane;
    const bool ok = j < c;
    const int li = S.lists[R_FALLBACK][ok ? j : b];
    const T val = kint_warp_batch<DX, T>(S.sv[li], S.sx[li], min(32, c - b), lane, gauss);
    if (ok) out[t0 + li] = val;
  }
}

}  // namespace lb
