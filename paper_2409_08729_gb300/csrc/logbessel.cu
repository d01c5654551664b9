// logbessel.cu -- kernels and C ABI of the GB300 log-Bessel library.
//
// Pipeline for one call (paper Sec. 4.3 sorts the pairs by expression before
// launch so that warps do not diverge; here the grouping is done on chip):
//
//   1. lb_tiles_kernel: persistent CTAs walk tiles of kTile pairs.  Each
//      thread loads LB_ITEMS pairs (coalesced), handles domain edges, and
//      classifies the rest (Table "input ranges").  The tile's pairs are
//      binned per region into shared-memory index lists; the warps take
//      32-pair chunks of the lists from shared counters, so every warp runs
//      one expression (mu_20, U_K, power series) at a time.  K pairs of the
//      fallback region are appended to a global queue instead.
//   2. lb_kint_kernel: one warp per queued K pair evaluates the integral with
//      the nodes spread over the lanes (lb_kint.cuh).
// A call with one order for all pairs (v_stride 0) has its order's
// constants computed once per block (ScalarOrder, KintScalar).
//
// The plain form computes in FP64; its exps and logs are evaluated in
// integer arithmetic where that is faster (lb_intmath.cuh).
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <utility>
#include <vector>
#include <stdio.h>
#include <string.h>
#include <string>

#include "logbessel.h"
#include "lb_tile.cuh"
#include "lb_fastmath.cuh"

#define LB_VERSION "0.2.0"

using namespace lb;

namespace {

// Resident CTAs per SM the two kernels are built and launched for (launch
// bounds and persistent grid sizes: a multiple of the SM count).
// The tile kernel runs blocks of LB_TILE_THREADS threads, so a tile holds
// LB_TILE_THREADS * LB_ITEMS pairs: 2048 at 512 threads.  Larger tiles leave
// fewer partly filled 32-pair chunks at the end of each region's range of a
// tile (lanes that idle through an expression); at 512 threads and 3 CTAs
// per SM the SM keeps its 48 resident warps and 40 registers a thread, and
// the sweep's tile kernel time fell 4 % against 1024-pair tiles (256
// threads, 6 CTAs per SM).
#ifndef LB_TILE_THREADS
#define LB_TILE_THREADS 512
#endif
#ifndef LB_TILES_CTAS_PER_SM
#define LB_TILES_CTAS_PER_SM 3
#endif
#ifndef LB_KINT_CTAS_PER_SM
#define LB_KINT_CTAS_PER_SM 4
#endif
// The class-specialized K-integral kernels (FP64 Gauss values, one per rule
// class of kint_class: split, one-slot s0 = 8, one-slot s0 = 3, packed,
// fixed 32 and 64 g nodes) each hold only their own rule's registers, so the
// short rules run with more resident warps (budgets measured on the sweep and
// the robustness sweep: 4, 8, 8, 6, 6, 6 CTAs per SM beat 4 everywhere by
// 1-2 %; the split rule keeps 4).
#ifndef LB_KINT_CTAS_C0
#define LB_KINT_CTAS_C0 4
#endif
#ifndef LB_KINT_CTAS_C12
#define LB_KINT_CTAS_C12 8
#endif
#ifndef LB_KINT_CTAS_C3
#define LB_KINT_CTAS_C3 6
#endif
#ifndef LB_KINT_CTAS_C45
#define LB_KINT_CTAS_C45 6
#endif
constexpr int kKintCtasCls[6] = {LB_KINT_CTAS_C0, LB_KINT_CTAS_C12, LB_KINT_CTAS_C12,
                                 LB_KINT_CTAS_C3, LB_KINT_CTAS_C45, LB_KINT_CTAS_C45};
// The x-derivative's class kernels carry the weighted sum besides the
// integer one and keep the general kernel's budget (64 registers).
__host__ __device__ constexpr int kint_ctas_per_sm(int cls, bool dx = false) {
  return (cls < 0 || dx) ? LB_KINT_CTAS_PER_SM : kKintCtasCls[cls];
}

// K-integral queue entries: the pair's offset within its chunk (chunks hold
// at most 2^26 pairs) in the low 26 bits, the quadrature rule class of the
// FP64 Gauss rules (kint_class; 0 otherwise) above them, so that a kernel
// that takes one class finds its pairs by reading the queue alone.
constexpr int kTileThreads = LB_TILE_THREADS;
constexpr int kTile = kTileThreads * LB_ITEMS;     // pairs per tile of the tile kernel
static_assert((1 << 26) % kTile == 0, "chunks of 2^26 pairs hold whole tiles");
constexpr int kQueueOffsetBits = 26;
constexpr uint32_t kQueueOffsetMask = (1u << kQueueOffsetBits) - 1u;

// Tile kernel: classify, bin per region in shared memory, evaluate the
// per-thread expressions (lb_tile.cuh); K fallback pairs go to a global queue
// for lb_kint_kernel.  T = double (FP64) or float (FP32-mixed).
// SO: one order for every argument (FP64 values, v_stride 0, no forced
// region): the order's constants once per block, and only the per-order
// forms of the expressions compiled in (each kernel carries one form's
// code, half the instruction footprint).
template <int KIND, bool DX, typename T, bool SO>
__global__ void __launch_bounds__(kTileThreads, LB_TILES_CTAS_PER_SM)
lb_tiles_kernel(const T* __restrict__ v, int64_t v_stride, const T* __restrict__ x, T* __restrict__ out,
                int64_t n, int mode, int forced_region, unsigned int* __restrict__ qcount,
                uint32_t* __restrict__ queue, int64_t qcap) {
  static_assert(!SO || (sizeof(T) == 8 && !DX), "per-order constants are built for FP64 values");
  __shared__ TileShared<T, kTileThreads> S;
  const int tid = threadIdx.x;
  const int64_t ntiles = (n + kTile - 1) / kTile;
  const ScalarOrder* so = nullptr;
  if constexpr (SO) {
    __shared__ ScalarOrder SOC;
    scalar_order_setup<KIND>(SOC, KIND == KIND_K ? fabs((double)v[0]) : (double)v[0]);
    so = &SOC;
  }
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t t0 = tile * kTile;
    tile_bin<KIND, DX, T>(S, v, v_stride, x, t0, n, mode, forced_region);
    tile_eval<KIND, DX, T>(S, out, t0, n, so);
    if (KIND == KIND_K) {
      const int c = S.rcount(R_FALLBACK), f0 = S.rbeg(R_FALLBACK);
      if (c > 0) {
        if (tid == 0) S.qbase = atomicAdd(qcount, (unsigned int)c);
        __syncthreads();
        const unsigned int b = S.qbase;
        unsigned cls = 0;                          // quadrature rule classes of the queued pairs
        for (int j = tid; j < c; j += kTileThreads) {
          const int li = S.list[f0 + j];
          uint32_t cl = 0;
          if constexpr (sizeof(T) == 8) {
            if (mode == MODE_TIGHT) {
              cl = (uint32_t)kint_class((double)S.sv[li], (double)S.sx[li], DX);   // sv holds |v|
              cls |= 1u << cl;
            }
          }
          // the pair's offset in the chunk (< 2^26) and its rule class above it
          if (LB_CHECK(b + j < qcap, 4u)) queue[b + j] = (uint32_t)(t0 + li) | (cl << kQueueOffsetBits);
        }
        if constexpr (sizeof(T) == 8) {
          cls = __reduce_or_sync(0xffffffffu, cls);
          if ((tid & 31) == 0 && cls) atomicOr(qcount + 1, cls);
        }
      }
    }
    __syncthreads();
  }
}

// K integral: one warp per queued pair, 32 pairs per warp batch.  CLS = -1:
// every queued pair; CLS = c (FP64 Gauss values): the pairs of rule class c
// only, with that class's code alone compiled in (the kernel returns at once
// when the queue holds none of them).
template <bool GAUSS, bool DX, typename T, int CLS = -1>
__global__ void __launch_bounds__(LB_THREADS, kint_ctas_per_sm(CLS, DX))
lb_kint_kernel(const T* __restrict__ v, int64_t v_stride, const T* __restrict__ x, T* __restrict__ out,
               const unsigned int* __restrict__ qcount, const uint32_t* __restrict__ queue, int64_t n,
               int64_t qcap) {
  unsigned int cnt = *qcount;
  if (!LB_CHECK(cnt <= qcap, 8u)) cnt = (unsigned int)qcap;
  const unsigned present = (GAUSS && sizeof(T) == 8) ? qcount[1] : 0u;
  if (CLS >= 0 && !(present & (1u << CLS))) return;     // the same for every thread of the grid
  const int lane = threadIdx.x & 31;
  const KintScalar* ks = nullptr;
  const KintScalar32* ks32 = nullptr;
  if constexpr (GAUSS && sizeof(T) == 8) {
    // one order for every pair: its node positions once per block
    __shared__ KintScalar KS;
    if (v_stride == 0 && cnt > 0) {
      kint_scalar_setup(KS, fabs((double)v[0]));
      ks = &KS;
    }
  } else if constexpr (GAUSS && sizeof(T) == 4) {
    __shared__ KintScalar32 KS32;
    if (v_stride == 0 && cnt > 0) {
      kint_scalar_setup32(KS32, fabsf((float)v[0]));
      ks32 = &KS32;
    }
  }
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  // FP64 Gauss rules with pairs of several quadrature rule classes queued
  // (split, 64 and 32 g nodes, packed, the two one-slot rules; the tile
  // kernel marks the classes it queues): the queue is processed in phases,
  // one present class each, costliest first: in phase c a warp scans its
  // windows of the queue (256 pairs when the queue gives every warp a full
  // window, else 32) for the pairs of class c, collects them in a ring in
  // its slice of shared memory and evaluates them 32 at a time.  So the
  // warps of an SM run one rule's code at a time; with the classes mixed,
  // every warp switching between up to six code paths, the instruction
  // cache thrashed (the K call of the robustness sweep took 2.2x the time of
  // its rule classes evaluated one after another).  A phase re-reads the
  // queue only, 4 bytes per pair: each entry carries its pair's class.  A pair's result
  // does not depend on its batch.  A queue of one class, and the other
  // kernels, take the queue in order, 32 pairs at a time.  A class kernel
  // is one phase of this: the host launches the six, costliest first.
  __shared__ uint32_t ring[LB_THREADS / 32][512];
  uint32_t* my = ring[threadIdx.x >> 5];
  const bool phased = __popc(present) > 1;
  const int P = phased && (int64_t)cnt >= nwarps * 256 ? 256 : 32;
  const int nphase = (phased && CLS < 0) ? 6 : 1;
  const unsigned lt = (1u << lane) - 1u;
  unsigned head = 0, nb = 0;                       // ring: first entry, entries held (warp-uniform)
  for (int ph = 0; ph < nphase; ++ph) {
    // costliest class first; -1: every pair
    const int c = !phased ? -1 : (CLS >= 0 ? CLS : (ph == 0 ? 0 : 6 - ph));
    if (phased && !(present & (1u << c))) continue;
    for (int64_t b = warp * P;; b += nwarps * P) {
      const bool last = b >= (int64_t)cnt;
      if (!last) {
        const int m = (int)min((int64_t)P, (int64_t)cnt - b);
        for (int j = 0; 32 * j < m; ++j) {
          const int t = 32 * j + lane;
          uint32_t id = 0;
          int cl = -1;
          if (t < m) {
            const uint32_t e = queue[b + t];       // offset and rule class: no gather of v and x to scan
            id = e & kQueueOffsetMask;
            cl = (int)(e >> kQueueOffsetBits);
            if (!LB_CHECK(cl <= 5, 32u)) cl = 0;
          }
          const bool take = t < m && (c < 0 || cl == c) && LB_CHECK((int64_t)id < n, 16u);
          const unsigned mk = __ballot_sync(0xffffffffu, take);
          if (take) my[(head + nb + __popc(mk & lt)) & 511u] = id;   // nb <= 31 + 256 < 512: no overrun
          nb += __popc(mk);
        }
        __syncwarp();
      }
      while (nb >= 32 || (last && nb > 0)) {
        const int k = nb < 32 ? (int)nb : 32;
        const int64_t idx = (int64_t)my[(head + (lane < k ? lane : 0)) & 511u];
        const T vi = fabs(v[idx * v_stride]);
        const T xi = x[idx];
        const T val = kint_warp_batch<DX, T, CLS>(vi, xi, k, lane, GAUSS, ks, ks32);
        if (lane < k) out[idx] = val;
        head += k;
        nb -= k;
      }
      __syncwarp();
      if (last) break;
    }
  }
}

template <int KIND>
__global__ void lb_classify_kernel32(const float* __restrict__ v, int64_t v_stride,
                                     const float* __restrict__ x, uint8_t* __restrict__ reg,
                                     int64_t n, int mode) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float vi = v[i * v_stride];
    const float xi = x[i];
    if (KIND == KIND_K) vi = fabsf(vi);
    float sp;
    reg[i] = special_value32<KIND>(vi, xi, &sp) ? (uint8_t)R_SPECIAL : (uint8_t)classify32(vi, xi, mode, KIND == KIND_K ? WIDE_K : WIDE_I);
  }
}

template <int KIND>
__global__ void lb_classify_kernel(const double* __restrict__ v, int64_t v_stride,
                                   const double* __restrict__ x, uint8_t* __restrict__ reg,
                                   int64_t n, int mode) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double vi = v[i * v_stride];
    const double xi = x[i];
    if (KIND == KIND_K) vi = fabs(vi);
    double sp;
    reg[i] = special_value<KIND>(vi, xi, &sp) ? (uint8_t)R_SPECIAL : (uint8_t)classify(vi, xi, mode, KIND == KIND_K ? WIDE_K : WIDE_I);
  }
}

// von Mises-Fisher log-normaliser (paper Sec. 6.3):
//   log C_d(k) = (d/2 - 1) log k - (d/2) log(2 pi) - log I_{d/2-1}(k),
// applied in place to out[i] = log I_{d/2-1}(kappa[i]) (or, for DX, to
// out[i] = d/dk log I_{d/2-1}, giving d/dk log C_d = (d/2-1)/k - I'/I).
// At k = 0: log C_d(0) = lgamma(d/2) - log 2 - (d/2) log pi, the limit of
// I_nu(k) ~ (k/2)^nu / Gamma(nu + 1).
template <bool DX>
__global__ void lb_vmf_finish_kernel(const double* __restrict__ kappa, double* __restrict__ out, int64_t n,
                                     double d) {
  const double nu = 0.5 * d - 1.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double k = kappa[i];
    if (DX) {
      out[i] = (k == 0.0) ? 0.0 : nu / k - out[i];
    } else if (k == 0.0) {
      out[i] = lgamma(0.5 * d) - 0.6931471805599453 - 0.5 * d * 1.1447298858494002;
    } else {
      out[i] = fma(nu, log(k), -0.5 * d * 1.8378770664093453) - out[i];
    }
  }
}

__global__ void lb_set_scalar_kernel(double* p, double value) { *p = value; }

// Elementwise exp/log for checking the table-driven implementations against
// the libm ones: which = 0 fm_exp, 1 fm_log, 2 exp, 3 log; and CUDA's
// special-purpose Bessel functions of orders 0 and 1 (the comparison system
// of paper Sec. 6.1): 4 log(cyl_bessel_i0), 5 log(cyl_bessel_i1).
__global__ void lb_math_kernel(int which, const double* __restrict__ in, double* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double a = in[i];
    double r;
    switch (which) {
      case 0: r = fm_exp(a); break;
      case 1: r = fm_log(a); break;
      case 2: r = exp(a); break;
      case 3: r = log(a); break;
      case 4: r = log(cyl_bessel_i0(a)); break;
      case 5: r = log(cyl_bessel_i1(a)); break;
      case 6: r = fm_exp_term(a); break;
      case 7: r = ix_exp(a); break;
      case 8: r = ix_log(a); break;
      case 9: r = ix_rcp(a); break;
      case 10: r = ix_rsqrt(a); break;
      case 11: r = __longlong_as_double(ix_log_q53(a)); break;          // the Q53 integer's bits
      default: r = __longlong_as_double((long long)ix_exp_q58_fx(__double_as_longlong(a))); break;
    }
    out[i] = r;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
thread_local std::string g_last_error;

lb_status fail(lb_status st, const char* fmt, const char* a = "", long long b = 0) {
  char buf[512];
  snprintf(buf, sizeof buf, fmt, a, b);
  g_last_error = buf;
  return st;
}

lb_status check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return LB_ECUDA;
  }
  return LB_OK;
}

int sm_count() {
  static std::mutex mu;
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  std::lock_guard<std::mutex> lk(mu);
  if (cache[dev] == 0) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
    cache[dev] = sms;
  }
  return cache[dev];
}

// ---------------------------------------------------------------------------
// launch accounting and optional per-kernel CUDA-event timing
// ---------------------------------------------------------------------------
enum ProfSlotId { PS_TILES = 0, PS_KINT = 1, PS_CLASSIFY = 2, PS_AUX = 3, PS_NSLOTS = 4 };
const char* const kSlotNames[PS_NSLOTS] = {"lb_tiles_kernel", "lb_kint_kernel", "lb_classify_kernel",
                                           "lb_aux_kernels"};

struct ProfState {
  std::mutex mu;
  bool on = false;
  long long launches[PS_NSLOTS] = {0, 0, 0, 0};
  long long timed[PS_NSLOTS] = {0, 0, 0, 0};
  double ms[PS_NSLOTS] = {0, 0, 0, 0};
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
};
ProfState& prof() {
  static ProfState p;
  return p;
}
std::atomic<long long> g_total_launches{0};

void prof_drain_locked(ProfState& P) {
  for (auto& e : P.pending) {
    float t = 0.f;
    if (cudaEventSynchronize(e.second.second) == cudaSuccess &&
        cudaEventElapsedTime(&t, e.second.first, e.second.second) == cudaSuccess) {
      P.ms[e.first] += t;
      P.timed[e.first] += 1;
    }
    cudaEventDestroy(e.second.first);
    cudaEventDestroy(e.second.second);
  }
  P.pending.clear();
}

// Launch `body` (one kernel launch) on stream st under slot `slot`.
template <typename F>
lb_status launch(int slot, cudaStream_t st, F&& body) {
  ProfState& P = prof();
  cudaEvent_t a = nullptr, b = nullptr;
  bool timed = false;
  {
    std::lock_guard<std::mutex> lk(P.mu);
    timed = P.on;
  }
  if (timed && (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)) timed = false;
  if (timed) cudaEventRecord(a, st);
  body();
  lb_status s = check_launch(kSlotNames[slot]);
  g_total_launches.fetch_add(1);
  {
    std::lock_guard<std::mutex> lk(P.mu);
    P.launches[slot] += 1;
    if (timed) {
      cudaEventRecord(b, st);
      P.pending.push_back({slot, {a, b}});
    }
  }
  return s;
}

lb_status validate(lb_dtype dtype, const void* v, int64_t v_stride, const void* x, const void* out,
                   int64_t n, int mode) {
  if (n < 0) return fail(LB_EINVAL, "n must be >= 0 (got %s%lld)", "", (long long)n);
  if (dtype != LB_F64 && dtype != LB_F32) return fail(LB_EINVAL, "unknown dtype %s%lld", "", (long long)dtype);
  if (mode < 0 || mode > 2) return fail(LB_EINVAL, "unknown mode %s%lld", "", (long long)mode);
  if (v_stride != 0 && v_stride != 1) return fail(LB_EINVAL, "v_stride must be 0 or 1 (got %s%lld)", "", (long long)v_stride);
  if (n > 0 && (!v || !x || !out)) return fail(LB_EINVAL, "NULL %s pointer with n = %lld", !v ? "v" : (!x ? "x" : "out"), (long long)n);
  return LB_OK;
}

template <bool DX, typename T, int CLS>
lb_status launch_kint_class(int sms, cudaStream_t st, const T* v, int64_t v_stride, const T* x, T* out,
                            const unsigned int* qcount, const uint32_t* queue, int64_t n, int64_t qcap) {
  const int grid = sms * 2 * kint_ctas_per_sm(CLS, DX);
  return launch(PS_KINT, st, [&] {
    lb_kint_kernel<true, DX, T, CLS><<<grid, LB_THREADS, 0, st>>>(v, v_stride, x, out, qcount, queue, n, qcap);
  });
}

// The six class kernels of the FP64 Gauss rules (values or x-derivatives),
// in the order of the phases.
template <bool DX, typename T>
lb_status launch_kint_classes(int sms, cudaStream_t st, const T* v, int64_t v_stride, const T* x, T* out,
                              const unsigned int* qcount, const uint32_t* queue, int64_t n, int64_t qcap) {
  lb_status s = launch_kint_class<DX, T, 0>(sms, st, v, v_stride, x, out, qcount, queue, n, qcap);
  if (s == LB_OK) s = launch_kint_class<DX, T, 5>(sms, st, v, v_stride, x, out, qcount, queue, n, qcap);
  if (s == LB_OK) s = launch_kint_class<DX, T, 4>(sms, st, v, v_stride, x, out, qcount, queue, n, qcap);
  if (s == LB_OK) s = launch_kint_class<DX, T, 3>(sms, st, v, v_stride, x, out, qcount, queue, n, qcap);
  if (s == LB_OK) s = launch_kint_class<DX, T, 2>(sms, st, v, v_stride, x, out, qcount, queue, n, qcap);
  if (s == LB_OK) s = launch_kint_class<DX, T, 1>(sms, st, v, v_stride, x, out, qcount, queue, n, qcap);
  return s;
}

// Largest chunk handled with one queue: the queue entries hold 26-bit offsets.
const int64_t kChunk = (int64_t)1 << kQueueOffsetBits;
// Smallest caller workspace: the counters and the queue of one tile.
const int64_t kWsMin = 256 + 4 * kTile;
static_assert(256 + 4 * kTile == 8448, "the documented smallest workspace");

// Enqueue the evaluation of n pairs.  The K fallback goes through a queue
// of 32-bit pair offsets in scratch memory (qcount: the counter and the
// mask of the quadrature rule classes queued, queue:
// min(n, chunk) entries), processed chunk by chunk; `scratch` supplies it,
// or, when NULL, it comes from the stream-ordered allocator.
template <int KIND, bool DX, typename T>
lb_status run_impl(const T* v, int64_t v_stride, const T* x, T* out, int64_t n, int mode, int forced_region,
                   cudaStream_t st, void* scratch, int64_t chunk) {
  const int sms = sm_count();
  const int64_t ntiles_all = (n + kTile - 1) / kTile;
  const bool per_order = sizeof(T) == 8 && !DX && v_stride == 0 && forced_region < 0;
  if (KIND == KIND_I || (forced_region >= 0 && forced_region != R_FALLBACK)) {
    const int grid = (int)(ntiles_all < (int64_t)sms * LB_TILES_CTAS_PER_SM ? ntiles_all : (int64_t)sms * LB_TILES_CTAS_PER_SM);
    return launch(PS_TILES, st, [&] {
      if (per_order)
        lb_tiles_kernel<KIND, DX, T, !DX && sizeof(T) == 8><<<grid, kTileThreads, 0, st>>>(
            v, v_stride, x, out, n, mode, forced_region, nullptr, nullptr, 0);
      else
        lb_tiles_kernel<KIND, DX, T, false><<<grid, kTileThreads, 0, st>>>(v, v_stride, x, out, n, mode,
                                                                          forced_region, nullptr, nullptr, 0);
    });
  }
  if (sizeof(T) == 4 && mode != MODE_TIGHT)
    return fail(LB_ENOTSUP, "%sthe FP32 K integral is implemented for LB_TIGHT only", "", 0);
  // queue entries a pass can write: every workspace holds at least this many
  const int64_t cap = n < chunk ? n : chunk;
  void* ws = scratch;
  if (!ws) {
    const size_t bytes = 256 + (size_t)cap * sizeof(uint32_t);
    if (cudaMallocAsync(&ws, bytes, st) != cudaSuccess) {
      cudaGetLastError();
      return fail(LB_ENOMEM, "cudaMallocAsync of %s%lld bytes failed", "", (long long)bytes);
    }
  }
  unsigned int* qcount = (unsigned int*)ws;
  uint32_t* queue = (uint32_t*)((char*)ws + 256);
  lb_status status = LB_OK;
  for (int64_t c0 = 0; c0 < n && status == LB_OK; c0 += chunk) {
    const int64_t cn = (n - c0) < chunk ? (n - c0) : chunk;
    if (cudaMemsetAsync(qcount, 0, 2 * sizeof(unsigned int), st) != cudaSuccess) { status = check_launch("cudaMemsetAsync"); break; }
    const T* vc = v + c0 * v_stride;
    const T* xc = x + c0;
    T* oc = out + c0;
    const int64_t ntiles = (cn + kTile - 1) / kTile;
    const int grid = (int)(ntiles < (int64_t)sms * LB_TILES_CTAS_PER_SM ? ntiles : (int64_t)sms * LB_TILES_CTAS_PER_SM);
    status = launch(PS_TILES, st, [&] {
      if (per_order)
        lb_tiles_kernel<KIND, DX, T, !DX && sizeof(T) == 8><<<grid, kTileThreads, 0, st>>>(
            vc, v_stride, xc, oc, cn, mode, forced_region, qcount, queue, cap);
      else
        lb_tiles_kernel<KIND, DX, T, false><<<grid, kTileThreads, 0, st>>>(vc, v_stride, xc, oc, cn, mode,
                                                                          forced_region, qcount, queue, cap);
    });
    if (status != LB_OK) break;
    bool done = false;
    if constexpr (sizeof(T) == 8) {
      if (mode == MODE_TIGHT) {
        // one kernel per rule class, costliest first (the phases of a mixed queue)
        status = launch_kint_classes<DX, T>(sms, st, vc, v_stride, xc, oc, qcount, queue, cn, cap);
        done = true;
      }
    }
    if (!done) {
      const int kgrid = sms * 2 * LB_KINT_CTAS_PER_SM;
      status = launch(PS_KINT, st, [&] {
        if (mode == MODE_TIGHT)
          lb_kint_kernel<true, DX, T><<<kgrid, LB_THREADS, 0, st>>>(vc, v_stride, xc, oc, qcount, queue, cn, cap);
        else
          lb_kint_kernel<false, DX, T><<<kgrid, LB_THREADS, 0, st>>>(vc, v_stride, xc, oc, qcount, queue, cn, cap);
      });
    }
  }
  if (!scratch) cudaFreeAsync(ws, st);
  return status;
}

template <int KIND, bool DX>
lb_status run(const double* v, int64_t v_stride, const double* x, double* out, int64_t n, int mode,
              int forced_region, cudaStream_t st) {
  return run_impl<KIND, DX, double>(v, v_stride, x, out, n, mode, forced_region, st, nullptr, kChunk);
}

lb_status run32(int kind, const float* v, int64_t v_stride, const float* x, float* out, int64_t n, int mode,
                int forced_region, cudaStream_t st) {
  if (kind == KIND_I) return run_impl<KIND_I, false, float>(v, v_stride, x, out, n, mode, forced_region, st, nullptr, kChunk);
  return run_impl<KIND_K, false, float>(v, v_stride, x, out, n, mode, forced_region, st, nullptr, kChunk);
}

// Fixed scratch for logbessel_k_noalloc: the queue counter (first 256
// bytes) and the queue of the K fallback pairs, for at most
// LB_NOALLOC_MAX_PAIRS pairs per call.  It lives in the module's global
// memory for as long as the library is loaded, on every device that loads it.
#define LB_NOALLOC_MAX_PAIRS (1 << 20)
static __device__ __align__(256) uint32_t lb_noalloc_scratch[64 + LB_NOALLOC_MAX_PAIRS];

// Device address of lb_noalloc_scratch in the current context, looked up on
// every call: cudaGetSymbolAddress allocates nothing, and a cached address
// would go stale when the device's primary context is torn down and made
// again (cudaDeviceReset), since the module then reloads elsewhere.
void* noalloc_scratch_address() {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, lb_noalloc_scratch);
  if (e != cudaSuccess) {
    cudaGetLastError();
    g_last_error = std::string("logbessel_k_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
    return nullptr;
  }
  return p;
}

}  // namespace

extern "C" {

lb_status logbessel_i(lb_dtype dtype, const void* v, int64_t v_stride, const void* x, void* out,
                      int64_t n, lb_mode mode, void* cuda_stream) {
  lb_status s = validate(dtype, v, v_stride, x, out, n, (int)mode);
  if (s != LB_OK || n == 0) return s;
  if (dtype == LB_F32)
    return run32(KIND_I, (const float*)v, v_stride, (const float*)x, (float*)out, n, (int)mode, -1,
                 (cudaStream_t)cuda_stream);
  return run<KIND_I, false>((const double*)v, v_stride, (const double*)x, (double*)out, n, (int)mode, -1,
                            (cudaStream_t)cuda_stream);
}

lb_status logbessel_k(lb_dtype dtype, const void* v, int64_t v_stride, const void* x, void* out,
                      int64_t n, lb_mode mode, void* cuda_stream) {
  lb_status s = validate(dtype, v, v_stride, x, out, n, (int)mode);
  if (s != LB_OK || n == 0) return s;
  if (dtype == LB_F32)
    return run32(KIND_K, (const float*)v, v_stride, (const float*)x, (float*)out, n, (int)mode, -1,
                 (cudaStream_t)cuda_stream);
  return run<KIND_K, false>((const double*)v, v_stride, (const double*)x, (double*)out, n, (int)mode, -1,
                            (cudaStream_t)cuda_stream);
}

lb_status logbessel_i_dx(lb_dtype dtype, const void* v, int64_t v_stride, const void* x, void* out,
                         int64_t n, lb_mode mode, void* cuda_stream) {
  lb_status s = validate(dtype, v, v_stride, x, out, n, (int)mode);
  if (s != LB_OK || n == 0) return s;
  if (dtype != LB_F64) return fail(LB_ENOTSUP, "%sthe derivatives are implemented for LB_F64 only", "", 0);
  return run<KIND_I, true>((const double*)v, v_stride, (const double*)x, (double*)out, n, (int)mode, -1,
                           (cudaStream_t)cuda_stream);
}

lb_status logbessel_k_dx(lb_dtype dtype, const void* v, int64_t v_stride, const void* x, void* out,
                         int64_t n, lb_mode mode, void* cuda_stream) {
  lb_status s = validate(dtype, v, v_stride, x, out, n, (int)mode);
  if (s != LB_OK || n == 0) return s;
  if (dtype != LB_F64) return fail(LB_ENOTSUP, "%sthe derivatives are implemented for LB_F64 only", "", 0);
  if (mode != LB_TIGHT) return fail(LB_ENOTSUP, "%sd/dx log K is implemented for LB_TIGHT only", "", 0);
  return run<KIND_K, true>((const double*)v, v_stride, (const double*)x, (double*)out, n, (int)mode, -1,
                           (cudaStream_t)cuda_stream);
}

lb_status logbessel_k_noalloc(lb_dtype dtype, const void* v, int64_t v_stride, const void* x, void* out,
                              int64_t n, lb_mode mode, void* cuda_stream) {
  lb_status s = validate(dtype, v, v_stride, x, out, n, (int)mode);
  if (s != LB_OK || n == 0) return s;
  if (dtype != LB_F64) return fail(LB_ENOTSUP, "%slogbessel_k_noalloc supports LB_F64 only", "", 0);
  if (n > LB_NOALLOC_MAX_PAIRS)
    return fail(LB_EINVAL, "%slogbessel_k_noalloc takes at most 1048576 pairs per call (got %lld)", "", (long long)n);
  void* scratch = noalloc_scratch_address();
  if (!scratch) return LB_ECUDA;
  return run_impl<KIND_K, false, double>((const double*)v, v_stride, (const double*)x, (double*)out, n, (int)mode,
                                         -1, (cudaStream_t)cuda_stream, scratch, LB_NOALLOC_MAX_PAIRS);
}

int64_t logbessel_workspace_bytes(int64_t n) {
  if (n < 0) return 0;
  const int64_t m = (n + kTile - 1) / kTile * kTile;        // passes hold whole tiles
  return 256 + 4 * (m < kTile ? kTile : (m < kChunk ? m : kChunk));
}

lb_status logbessel_k_ws(lb_dtype dtype, const void* v, int64_t v_stride, const void* x, void* out, int64_t n,
                         lb_mode mode, void* workspace, int64_t ws_bytes, void* cuda_stream) {
  lb_status s = validate(dtype, v, v_stride, x, out, n, (int)mode);
  if (s != LB_OK) return s;
  if (!workspace || ((uintptr_t)workspace & 255) || ws_bytes < kWsMin)
    return fail(LB_EINVAL, "%sworkspace must be non-NULL, 256-byte aligned and at least 8448 bytes (got %lld)", "",
                (long long)ws_bytes);
  if (n == 0) return LB_OK;
  // passes start on tile boundaries, so the results equal those of one pass
  const int64_t cap0 = (ws_bytes - 256) / 4;
  const int64_t cap = ((cap0 < kChunk ? cap0 : kChunk) / kTile) * kTile;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (dtype == LB_F32)
    return run_impl<KIND_K, false, float>((const float*)v, v_stride, (const float*)x, (float*)out, n, (int)mode, -1,
                                          st, workspace, cap);
  return run_impl<KIND_K, false, double>((const double*)v, v_stride, (const double*)x, (double*)out, n, (int)mode,
                                         -1, st, workspace, cap);
}

lb_status logbessel_k_dx_ws(lb_dtype dtype, const void* v, int64_t v_stride, const void* x, void* out, int64_t n,
                            lb_mode mode, void* workspace, int64_t ws_bytes, void* cuda_stream) {
  lb_status s = validate(dtype, v, v_stride, x, out, n, (int)mode);
  if (s != LB_OK) return s;
  if (!workspace || ((uintptr_t)workspace & 255) || ws_bytes < kWsMin)
    return fail(LB_EINVAL, "%sworkspace must be non-NULL, 256-byte aligned and at least 8448 bytes (got %lld)", "",
                (long long)ws_bytes);
  if (n == 0) return LB_OK;
  if (dtype != LB_F64) return fail(LB_ENOTSUP, "%sthe derivatives are implemented for LB_F64 only", "", 0);
  if (mode != LB_TIGHT) return fail(LB_ENOTSUP, "%sd/dx log K is implemented for LB_TIGHT only", "", 0);
  // passes start on tile boundaries, so the results equal those of one pass
  const int64_t cap0 = (ws_bytes - 256) / 4;
  const int64_t cap = ((cap0 < kChunk ? cap0 : kChunk) / kTile) * kTile;
  return run_impl<KIND_K, true, double>((const double*)v, v_stride, (const double*)x, (double*)out, n, (int)mode, -1,
                                        (cudaStream_t)cuda_stream, workspace, cap);
}

lb_status logbessel_classify(int kind, lb_dtype dtype, const void* v, int64_t v_stride,
                             const void* x, uint8_t* region_out, int64_t n, lb_mode mode,
                             void* cuda_stream) {
  if (kind != 0 && kind != 1) return fail(LB_EINVAL, "kind must be 0 (I) or 1 (K), got %s%lld", "", (long long)kind);
  lb_status s = validate(dtype, v, v_stride, x, region_out, n, (int)mode);
  if (s != LB_OK || n == 0) return s;
  const int grid = sm_count() * 4;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (dtype == LB_F32)
    return launch(PS_CLASSIFY, st, [&] {
      if (kind == 0)
        lb_classify_kernel32<KIND_I><<<grid, LB_THREADS, 0, st>>>((const float*)v, v_stride, (const float*)x, region_out, n, (int)mode);
      else
        lb_classify_kernel32<KIND_K><<<grid, LB_THREADS, 0, st>>>((const float*)v, v_stride, (const float*)x, region_out, n, (int)mode);
    });
  return launch(PS_CLASSIFY, st, [&] {
    if (kind == 0)
      lb_classify_kernel<KIND_I><<<grid, LB_THREADS, 0, st>>>((const double*)v, v_stride, (const double*)x, region_out, n, (int)mode);
    else
      lb_classify_kernel<KIND_K><<<grid, LB_THREADS, 0, st>>>((const double*)v, v_stride, (const double*)x, region_out, n, (int)mode);
  });
}

lb_status logbessel_eval_region(int kind, lb_dtype dtype, const void* v, int64_t v_stride,
                                const void* x, void* out, int64_t n, int region, lb_mode mode,
                                void* cuda_stream) {
  if (kind != 0 && kind != 1) return fail(LB_EINVAL, "kind must be 0 (I) or 1 (K), got %s%lld", "", (long long)kind);
  if (region < 0 || region > R_U9 || region == R_SPECIAL)
    return fail(LB_EINVAL, "region %s%lld is not an expression", "", (long long)region);
  lb_status s = validate(dtype, v, v_stride, x, out, n, (int)mode);
  if (s != LB_OK || n == 0) return s;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (dtype == LB_F32)
    return run32(kind, (const float*)v, v_stride, (const float*)x, (float*)out, n, (int)mode, region, st);
  if (kind == 0)
    return run<KIND_I, false>((const double*)v, v_stride, (const double*)x, (double*)out, n, (int)mode, region, st);
  return run<KIND_K, false>((const double*)v, v_stride, (const double*)x, (double*)out, n, (int)mode, region, st);
}

lb_status logbessel_vmf_log_c(lb_dtype dtype, double d, const void* kappa, void* out, int64_t n, int deriv,
                              void* cuda_stream) {
  if (!(d >= 2.0) || !isfinite(d)) return fail(LB_EINVAL, "dimension d must be finite and >= 2 (got %s%lld)", "", (long long)d);
  if (deriv != 0 && deriv != 1) return fail(LB_EINVAL, "deriv must be 0 or 1 (got %s%lld)", "", (long long)deriv);
  lb_status s = validate(dtype, kappa, 0, kappa, out, n, 0);
  if (s != LB_OK || n == 0) return s;
  if (dtype != LB_F64) return fail(LB_ENOTSUP, "%sthe vMF log-normaliser is implemented for LB_F64 only", "", 0);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double* nu = nullptr;
  if (cudaMallocAsync(&nu, sizeof(double), st) != cudaSuccess) {
    cudaGetLastError();
    return fail(LB_ENOMEM, "cudaMallocAsync of %s%lld bytes failed", "", 8);
  }
  s = launch(PS_AUX, st, [&] { lb_set_scalar_kernel<<<1, 1, 0, st>>>(nu, 0.5 * d - 1.0); });
  if (s == LB_OK)
    s = deriv ? run<KIND_I, true>(nu, 0, (const double*)kappa, (double*)out, n, MODE_TIGHT, -1, st)
              : run<KIND_I, false>(nu, 0, (const double*)kappa, (double*)out, n, MODE_TIGHT, -1, st);
  if (s == LB_OK) {
    const int grid = sm_count() * 4;
    s = launch(PS_AUX, st, [&] {
      if (deriv)
        lb_vmf_finish_kernel<true><<<grid, LB_THREADS, 0, st>>>((const double*)kappa, (double*)out, n, d);
      else
        lb_vmf_finish_kernel<false><<<grid, LB_THREADS, 0, st>>>((const double*)kappa, (double*)out, n, d);
    });
  }
  cudaFreeAsync(nu, st);
  return s;
}

lb_status logbessel_math_eval(int which, const double* in, double* out, int64_t n, void* cuda_stream) {
  if (which < 0 || which > 12) return fail(LB_EINVAL, "which must be 0..12 (got %s%lld)", "", (long long)which);
  if (n < 0 || (n > 0 && (!in || !out))) return fail(LB_EINVAL, "bad buffer or size %s%lld", "", (long long)n);
  if (n == 0) return LB_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int grid = sm_count() * 4;
  return launch(PS_AUX, st, [&] { lb_math_kernel<<<grid, LB_THREADS, 0, st>>>(which, in, out, n); });
}

// Chunk slots of the pipeline: one more than the three stages, so that a
// copy that stalls for a while (the host memory is shared) does not stop
// the evaluation of the next chunk.
constexpr int kHostSlots = 4;

// Streams, events and the device buffer of logbessel_host, kept per device
// from one call to the next: allocating and releasing the few hundred MB of
// chunk buffers on every call (the stream-ordered pool returns them to the
// driver at each synchronization) costs more than a short call's evaluation.
// A call holds its device's lock from start to end.
struct HostPipe {
  std::mutex mu;
  bool init = false;
  cudaStream_t st[4] = {};                      // copy-in, compute (even pieces), copy-out, compute (odd)
  cudaEvent_t ev_in[kHostSlots] = {}, ev_comp[kHostSlots] = {}, ev_out[kHostSlots] = {};
  char* dbuf = nullptr;
  size_t bytes = 0;
};
constexpr int kMaxDevices = 64;

HostPipe& host_pipe(int dev) {
  static HostPipe pipes[kMaxDevices];
  return pipes[dev];
}

void host_pipe_destroy(HostPipe& P) {
  if (P.dbuf) cudaFree(P.dbuf);
  for (int i = 0; i < kHostSlots; ++i) {
    if (P.ev_in[i]) cudaEventDestroy(P.ev_in[i]);
    if (P.ev_comp[i]) cudaEventDestroy(P.ev_comp[i]);
    if (P.ev_out[i]) cudaEventDestroy(P.ev_out[i]);
    P.ev_in[i] = P.ev_comp[i] = P.ev_out[i] = nullptr;
  }
  for (int i = 0; i < 4; ++i) {
    if (P.st[i]) cudaStreamDestroy(P.st[i]);
    P.st[i] = nullptr;
  }
  P.dbuf = nullptr;
  P.bytes = 0;
  P.init = false;
}

bool host_pipe_init(HostPipe& P) {
  bool ok = true;
  for (int i = 0; i < 4 && ok; ++i) ok = cudaStreamCreateWithFlags(&P.st[i], cudaStreamNonBlocking) == cudaSuccess;
  for (int i = 0; i < kHostSlots && ok; ++i)
    ok = cudaEventCreateWithFlags(&P.ev_in[i], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&P.ev_comp[i], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&P.ev_out[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    host_pipe_destroy(P);
    return false;
  }
  P.init = true;
  return true;
}

lb_status logbessel_host(int fn, lb_dtype dtype, const void* v, int64_t v_stride, const void* x, void* out,
                         int64_t n, lb_mode mode, int64_t chunk) {
  if (fn < 0 || fn > 3) return fail(LB_EINVAL, "fn must be 0..3 (got %s%lld)", "", (long long)fn);
  lb_status s = validate(dtype, v, v_stride, x, out, n, (int)mode);
  if (s != LB_OK || n == 0) return s;
  // default pieces of up to 16M pairs: on the sweep's 24 calls per step 2^24
  // measured 7.35 Gevals/s end to end against 7.17 (2^23), 6.88 (2^25) and
  // 6.62 (2^26): smaller pieces cost more kernel ends, larger ones longer
  // unoverlapped first and last copies
  if (chunk <= 0) chunk = (int64_t)1 << 24;
  if (chunk > kChunk) chunk = kChunk;
  if ((fn >= 2 && dtype != LB_F64) || (fn == 3 && mode != LB_TIGHT))
    return fail(LB_ENOTSUP, "%sthe derivatives are implemented for LB_F64 (and LB_TIGHT for K) only", "", 0);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return check_launch("cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(LB_EINVAL, "device %s%lld out of range", "", (long long)dev);
  HostPipe& P = host_pipe(dev);
  std::lock_guard<std::mutex> lk(P.mu);
  if (!P.init && !host_pipe_init(P))
    return fail(LB_ENOMEM, "%slogbessel_host: stream or event creation failed", "", 0);
  const size_t es = dtype == LB_F64 ? 8 : 4;
  const int64_t nbuf = kHostSlots;                // copy-in, compute and copy-out of successive chunks overlap
  const int64_t cap = n < chunk ? n : chunk;
  const size_t vbytes = (size_t)(v_stride ? cap : 1) * es, xbytes = (size_t)cap * es;
  const size_t slot = ((vbytes + 255) & ~(size_t)255) + 2 * ((xbytes + 255) & ~(size_t)255);
  const size_t qbytes = (256 + 4 * (size_t)cap + 255) & ~(size_t)255;
  const size_t need = slot * nbuf + 2 * qbytes;   // + a K fallback queue per compute stream
  if (P.bytes < need) {
    if (P.dbuf) cudaFree(P.dbuf);
    P.dbuf = nullptr;
    P.bytes = 0;
    if (cudaMalloc((void**)&P.dbuf, need) != cudaSuccess) {
      cudaGetLastError();
      P.dbuf = nullptr;
      return fail(LB_ENOMEM, "%slogbessel_host: cudaMalloc of %lld bytes failed", "", (long long)need);
    }
    P.bytes = need;
  }
  cudaStream_t* st = P.st;
  // Pieces: chunk/8, chunk/4, chunk/2, then whole chunks, and at the end
  // halves of what remains down to chunk/8, so that the first copy-in and
  // the last copy-out, which nothing overlaps, are short; piece edges stay
  // on tile boundaries (chunk a multiple of 8 tiles), so the results equal
  // those of one pass.
  const bool ramp = chunk % (8 * kTile) == 0;
  int64_t cn = 0;
  for (int64_t c0 = 0, i = 0; s == LB_OK && c0 < n; c0 += cn, ++i) {
    const int64_t r = n - c0;
    cn = chunk;
    if (ramp) {
      if (i < 3) cn = chunk >> (3 - i);
      if (r <= chunk) {
        const int64_t half = (r / 2) / kTile * kTile;
        cn = half > chunk / 8 ? half : chunk / 8;
      }
    }
    if (cn > r) cn = r;
    const int b = (int)(i % nbuf);
    char* dv = P.dbuf + b * slot;
    char* dx = dv + ((vbytes + 255) & ~(size_t)255);
    char* dout = dx + ((xbytes + 255) & ~(size_t)255);
    const char* hv = (const char*)v + (v_stride ? c0 * (int64_t)es : 0);
    if ((i >= nbuf && cudaStreamWaitEvent(st[0], P.ev_out[b], 0) != cudaSuccess) ||   // slot b's results are out
        cudaMemcpyAsync(dv, hv, (size_t)(v_stride ? cn : 1) * es, cudaMemcpyHostToDevice, st[0]) != cudaSuccess ||
        cudaMemcpyAsync(dx, (const char*)x + c0 * (int64_t)es, (size_t)cn * es, cudaMemcpyHostToDevice, st[0]) != cudaSuccess ||
        cudaEventRecord(P.ev_in[b], st[0]) != cudaSuccess) {
      s = check_launch("logbessel_host: copy-in");
      break;
    }
    // one pass per chunk (cn <= cap <= kChunk), the K queue in ws.  Even and
    // odd pieces run on two compute streams with a queue each, so a piece's
    // kernels start while the previous piece's last kernels drain (the K
    // integral's class kernels leave the GPU partly idle at their ends).
    cudaStream_t sc = st[(i & 1) ? 3 : 1];
    void* ws = P.dbuf + slot * nbuf + (size_t)(i & 1) * qbytes;
    if (cudaStreamWaitEvent(sc, P.ev_in[b], 0) != cudaSuccess) {
      s = check_launch("logbessel_host: copy-in");
      break;
    }
    if (dtype == LB_F32) {
      const float *fv = (const float*)dv, *fx = (const float*)dx;
      float* fo = (float*)dout;
      s = fn == 0 ? run_impl<KIND_I, false, float>(fv, v_stride, fx, fo, cn, (int)mode, -1, sc, nullptr, kChunk)
                  : run_impl<KIND_K, false, float>(fv, v_stride, fx, fo, cn, (int)mode, -1, sc, ws, kChunk);
    } else {
      const double *dvv = (const double*)dv, *dxx = (const double*)dx;
      double* dd = (double*)dout;
      switch (fn) {
        case 0: s = run_impl<KIND_I, false, double>(dvv, v_stride, dxx, dd, cn, (int)mode, -1, sc, nullptr, kChunk); break;
        case 1: s = run_impl<KIND_K, false, double>(dvv, v_stride, dxx, dd, cn, (int)mode, -1, sc, ws, kChunk); break;
        case 2: s = run_impl<KIND_I, true, double>(dvv, v_stride, dxx, dd, cn, (int)mode, -1, sc, nullptr, kChunk); break;
        default: s = run_impl<KIND_K, true, double>(dvv, v_stride, dxx, dd, cn, (int)mode, -1, sc, ws, kChunk); break;
      }
    }
    if (s != LB_OK) break;
    if (cudaEventRecord(P.ev_comp[b], sc) != cudaSuccess || cudaStreamWaitEvent(st[2], P.ev_comp[b], 0) != cudaSuccess ||
        cudaMemcpyAsync((char*)out + c0 * (int64_t)es, dout, (size_t)cn * es, cudaMemcpyDeviceToHost, st[2]) != cudaSuccess ||
        cudaEventRecord(P.ev_out[b], st[2]) != cudaSuccess) {
      s = check_launch("logbessel_host: copy-out");
      break;
    }
  }
  for (int i = 0; i < 4; ++i)
    if (cudaStreamSynchronize(st[i]) != cudaSuccess && s == LB_OK) s = check_launch("logbessel_host");
  // an asynchronous error of the last copies surfaces here, not in a later call
  if (s == LB_OK) s = check_launch("logbessel_host");
  return s;
}

lb_status logbessel_host_release(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return check_launch("cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(LB_EINVAL, "device %s%lld out of range", "", (long long)dev);
  HostPipe& P = host_pipe(dev);
  std::lock_guard<std::mutex> lk(P.mu);
  if (P.init) {
    for (int i = 0; i < 4; ++i) cudaStreamSynchronize(P.st[i]);
    host_pipe_destroy(P);
  }
  return LB_OK;
}

lb_status logbessel_check_status(unsigned int* bits, int clear) {
  if (!bits) return fail(LB_EINVAL, "%sNULL bits", "", 0);
  *bits = 0;
#ifdef LB_CHECKS
  unsigned int v = 0;
  if (cudaMemcpyFromSymbol(&v, lb_check_status, sizeof v) != cudaSuccess) return check_launch("logbessel_check_status");
  if (clear) {
    const unsigned int z = 0;
    if (cudaMemcpyToSymbol(lb_check_status, &z, sizeof z) != cudaSuccess) return check_launch("logbessel_check_status");
  }
  *bits = v;
  return LB_OK;
#else
  (void)clear;
  return fail(LB_ENOTSUP, "%sthis build has no index checks (build with LB_CHECKS)", "", 0);
#endif
}

const char* logbessel_last_error(void) { return g_last_error.c_str(); }

void logbessel_profile_enable(int on) {
  ProfState& P = prof();
  std::lock_guard<std::mutex> lk(P.mu);
  prof_drain_locked(P);
  if (on) {
    for (int i = 0; i < PS_NSLOTS; ++i) { P.ms[i] = 0.0; P.timed[i] = 0; }
  }
  P.on = on != 0;
}

int logbessel_profile_slots(void) { return PS_NSLOTS; }

lb_status logbessel_profile_get(int slot, const char** name, long long* launches, long long* timed_launches,
                                double* total_ms) {
  if (slot < 0 || slot >= PS_NSLOTS) return fail(LB_EINVAL, "profile slot %s%lld out of range", "", (long long)slot);
  ProfState& P = prof();
  std::lock_guard<std::mutex> lk(P.mu);
  prof_drain_locked(P);
  if (name) *name = kSlotNames[slot];
  if (launches) *launches = P.launches[slot];
  if (timed_launches) *timed_launches = P.timed[slot];
  if (total_ms) *total_ms = P.ms[slot];
  return LB_OK;
}

long long logbessel_launch_count(void) { return g_total_launches.load(); }

const char* logbessel_version(void) { return LB_VERSION; }

}  // extern "C"
