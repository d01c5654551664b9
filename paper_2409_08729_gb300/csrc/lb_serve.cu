// lb_serve.cu -- continuous-batching evaluation server.
//
// Requests (log I or log K, FP64 or FP32-mixed, 1 .. millions of pairs)
// arrive from host threads at any time, on host buffers (copied in and out
// by the server) or on device buffers (evaluated in place).  A host
// scheduler thread admits them as request slots and device memory (a fixed
// arena) free up, and publishes their work as items in a ring in mapped host
// memory.  A persistent kernel (one loop per CTA, several CTAs per SM)
// claims items with a compare-and-swap on a device counter.  Requests that
// arrive while others run are interleaved item by item, so their work
// overlaps on the device.
//
// A request runs in at most two stages, the same two as a direct library
// call (lb_tiles_kernel, then lb_kint_kernel):
//   stage A, tile items: each tile goes through classify, bin and the
//     per-thread expressions (lb_tile.cuh); the K pairs of the fallback
//     region are appended to per-class queues in the arena, one queue per
//     quadrature rule class of the K integral (the six code paths of
//     lb_kint.cuh for the FP64 Gauss rules; one queue otherwise);
//   stage B, K-window items: when a request's last tile is done, the device
//     posts the per-class queue lengths to mapped host memory and the
//     scheduler publishes windows of each class's queue, costliest class
//     first; a CTA evaluates a window 32 pairs per warp with the K-integral
//     code of lb_kint_kernel.  Every window holds pairs of one rule class, so
//     the warps that run it never switch code paths (mixed rules thrashed the
//     instruction cache of the direct kernel before it was phased by class).
// A request is done when its last item is; the scheduler then copies the
// results of a host request back and frees the slot and memory.
//
// Every device wait is bounded: a CTA that finds no work for idle_ms exits,
// and the scheduler relaunches the kernel when work appears.  Stopping sets
// a flag the CTAs poll.
#include <cuda/atomic>
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "logbessel.h"
#include "lb_tile.cuh"

using namespace lb;

// Resident CTAs per SM the persistent kernel is built for (its register budget).
#ifndef LB_SERVE_CTAS_PER_SM
#define LB_SERVE_CTAS_PER_SM 4
#endif

namespace {

constexpr int kItemsPerRequest = 64;   // stage A: a request is split into at most this many tile items
constexpr int kKClasses = 6;           // quadrature rule classes of the FP64 Gauss K integral (kint_class)
constexpr int kKItemsPerClass = 64;    // stage B: at most this many windows per class
constexpr int kKWindowMin = 512;       // smallest window of a class queue (pairs)
// Costliest class first, as the phases of lb_kint_kernel: the split rule,
// the 64- and 32-node fixed rules, the packed rule, the one-slot rules.
constexpr int kKClassOrder[kKClasses] = {0, 5, 4, 3, 2, 1};
// Item families of the device time accounts (lb_server_device_stats): FP64
// tiles of log I and log K, FP32 tiles of log I and log K, FP64 K windows of
// each rule class (or the one queue of the paper modes, as class 0), FP32 K
// windows.
constexpr int kFamilies = LB_SERVER_FAMILIES;
static_assert(kFamilies == 4 + kKClasses + 1, "item families");

struct SlotDesc {          // mapped host memory: written by the host, read by the device
  int kind;                // 0 = I, 1 = K
  int dtype;               // LB_F64 or LB_F32
  int mode;
  int nclass;              // K: queues (kKClasses for the FP64 Gauss rules, else 1); I: 0
  long long n;
  long long v_stride;
  unsigned long long v, x, out;   // device addresses (arena, or the caller's for device requests)
  unsigned long long queue;       // K: nclass queues of n uint32 pair offsets each (arena)
  long long ntiles;
  long long kitems;        // stage B items published for the request (written before they are)
};

struct WorkItem {          // 16 bytes
  int slot;
  int begin;               // tiles [begin, end), or a window [begin, end) of a class queue
  int end;
  int type;                // 0: tiles; 1 + c: a window of class c's queue
};

struct Ctl {               // mapped host memory shared by host and device
  int stop;
  int pad0;
  long long tail;          // number of published work items
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Shared memory of the persistent kernel: one tile, or the node table of a
// K window with one order for all pairs.
union ServeShared {
  TileShared<double, LB_THREADS> d;
  TileShared<float, LB_THREADS> f;
  KintScalar ks;
  KintScalar32 ks32;
};

struct ServeAux {          // per-tile class counts and queue bases of the K pairs
  int kc[8];
  unsigned kb[8];
};

// Stage A: one tile of a request.  K pairs of the fallback region go to the
// queue of their rule class (class 0 when the request has one queue); their
// order within a queue does not change any result.
template <int KIND, typename T>
__device__ __forceinline__ void serve_tile(TileShared<T, LB_THREADS>& S, ServeAux& A, const SlotDesc& d, int64_t tile,
                                           unsigned* qc) {
  const T* v = reinterpret_cast<const T*>(d.v);
  const T* x = reinterpret_cast<const T*>(d.x);
  T* out = reinterpret_cast<T*>(d.out);
  const int64_t t0 = tile * LB_TILE;
  const int tid = threadIdx.x;
  tile_bin<KIND, false, T>(S, v, d.v_stride, x, t0, d.n, d.mode, -1);
  tile_eval<KIND, false, T>(S, out, t0, d.n);
  if (KIND == KIND_K) {
    const int c = S.rcount(R_FALLBACK), f0 = S.rbeg(R_FALLBACK);
    if (c > 0) {                                   // block-uniform
      if (tid < 8) A.kc[tid] = 0;
      __syncthreads();
      int cl[LB_ITEMS], rk[LB_ITEMS], li[LB_ITEMS];
#pragma unroll
      for (int q = 0; q < LB_ITEMS; ++q) {
        const int j = tid + q * LB_THREADS;
        cl[q] = -1;
        rk[q] = 0;
        li[q] = 0;
        if (j < c) {
          li[q] = S.list[f0 + j];
          int k = 0;
          if constexpr (sizeof(T) == 8) {
            if (d.nclass > 1) k = kint_class((double)S.sv[li[q]], (double)S.sx[li[q]], false);   // sv holds |v|
          }
          cl[q] = k;
          rk[q] = atomicAdd(&A.kc[k], 1);
        }
      }
      __syncthreads();
      if (tid < d.nclass && A.kc[tid] > 0) A.kb[tid] = atomicAdd(qc + tid, (unsigned)A.kc[tid]);
      __syncthreads();
      uint32_t* queue = reinterpret_cast<uint32_t*>(d.queue);
#pragma unroll
      for (int q = 0; q < LB_ITEMS; ++q)
        if (cl[q] >= 0) queue[(int64_t)cl[q] * d.n + A.kb[cl[q]] + rk[q]] = (uint32_t)(t0 + li[q]);
    }
  }
  __syncthreads();
}

// Stage B: a window [q0, q1) of one class queue, 32 pairs per warp batch.
template <typename T>
__device__ __forceinline__ void serve_kwindow(ServeShared& U, const SlotDesc& d, int cls, int q0, int q1) {
  const T* v = reinterpret_cast<const T*>(d.v);
  const T* x = reinterpret_cast<const T*>(d.x);
  T* out = reinterpret_cast<T*>(d.out);
  const uint32_t* queue = reinterpret_cast<const uint32_t*>(d.queue) + (int64_t)cls * d.n;
  const bool gauss = d.mode == MODE_TIGHT;
  const KintScalar* ks = nullptr;
  const KintScalar32* ks32 = nullptr;
  if (d.v_stride == 0 && gauss) {                  // one order for all pairs: its node table once
    if constexpr (sizeof(T) == 8) {
      kint_scalar_setup(U.ks, fabs((double)v[0]));
      ks = &U.ks;
    } else {
      kint_scalar_setup32(U.ks32, fabsf((float)v[0]));
      ks32 = &U.ks32;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int b = q0 + 32 * warp; b < q1; b += LB_THREADS) {
    const int k = min(32, q1 - b);
    const int64_t idx = (int64_t)queue[b + (lane < k ? lane : 0)];
    const T vi = fabs(v[idx * d.v_stride]);
    const T xi = x[idx];
    const T val = kint_warp_batch<false, T>(vi, xi, k, lane, gauss, ks, ks32);
    if (lane < k) out[idx] = val;
  }
  __syncthreads();                                 // U is reused by the next item
}

__device__ __forceinline__ void signal_system(int* flag) {
  __threadfence_system();
  cuda::atomic_ref<int, cuda::thread_scope_system> r(*flag);
  r.store(1, cuda::memory_order_release);
}

__global__ void __launch_bounds__(LB_THREADS, LB_SERVE_CTAS_PER_SM)
lb_serve_kernel(Ctl* ctl, const SlotDesc* slots, const WorkItem* ring, int ring_cap, unsigned long long* head,
                long long* tiles_done, long long* kdone, unsigned* qcount, int* slot_done, int* stage_done,
                unsigned* kcount, long long idle_ns, unsigned long long* dstat,
                unsigned long long* claim_pos) {
  __shared__ ServeShared U;
  __shared__ ServeAux A;
  __shared__ long long claimed;
  __shared__ SlotDesc desc;
  __shared__ WorkItem item;
  cuda::atomic_ref<long long, cuda::thread_scope_system> tail_ref(ctl->tail);
  cuda::atomic_ref<int, cuda::thread_scope_system> stop_ref(ctl->stop);
  // thread 0: the family of the item in hand and when it was claimed
  int fam = -1;
  unsigned long long t_item = 0;
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned long long t_free = global_ns();
      if (fam >= 0) {                              // device time of the item just finished
        atomicAdd(dstat + 1 + fam, t_free - t_item);
        atomicAdd(dstat + 1 + kFamilies + fam, 1ull);
      }
      long long got = -1;
      const unsigned long long deadline = t_free + (unsigned long long)idle_ns;
      for (;;) {
        if (stop_ref.load(cuda::memory_order_relaxed)) break;
        const long long t = tail_ref.load(cuda::memory_order_acquire);
        const unsigned long long h = *(volatile unsigned long long*)head;
        if ((long long)h < t) {
          if (atomicCAS(head, h, h + 1) == h) { got = (long long)h; break; }
          continue;
        }
        if (global_ns() > deadline) break;
        __nanosleep(2000);
      }
      claimed = got;
      fam = -1;
      if (got >= 0) {
        // the ring position past this claim, for the host's count of items not yet taken
        cuda::atomic_ref<unsigned long long, cuda::thread_scope_system> pos(claim_pos[blockIdx.x]);
        pos.store((unsigned long long)got + 1ull, cuda::memory_order_relaxed);
        item = ring[got % ring_cap];
        desc = slots[item.slot];
        fam = item.type == 0 ? (desc.dtype == LB_F64 ? 0 : 2) + desc.kind
                             : (desc.dtype == LB_F64 ? 4 + (item.type - 1) : 4 + kKClasses);
      }
      t_item = global_ns();
      atomicAdd(dstat, t_item - t_free);           // claiming, and waiting for work
    }
    __syncthreads();
    if (claimed < 0) return;
    const SlotDesc d = desc;
    const WorkItem it = item;
    unsigned* qc = qcount + 8 * it.slot;
    if (it.type == 0) {
      for (int64_t tile = it.begin; tile < it.end; ++tile) {
        if (d.dtype == LB_F64) {
          if (d.kind == 0) serve_tile<KIND_I, double>(U.d, A, d, tile, qc);
          else serve_tile<KIND_K, double>(U.d, A, d, tile, qc);
        } else {
          if (d.kind == 0) serve_tile<KIND_I, float>(U.f, A, d, tile, qc);
          else serve_tile<KIND_K, float>(U.f, A, d, tile, qc);
        }
      }
      if (threadIdx.x == 0) {
        __threadfence();
        const long long nt = it.end - it.begin;
        const long long old = atomicAdd((unsigned long long*)&tiles_done[it.slot], (unsigned long long)nt);
        if (old + nt == d.ntiles) {                // the request's last tile
          tiles_done[it.slot] = 0;                 // ready for the slot's next request
          bool more = false;
          if (d.kind == 1) {
            __threadfence();
            for (int c = 0; c < d.nclass; ++c) {
              const unsigned m = *(volatile unsigned*)(qc + c);
              kcount[8 * it.slot + c] = m;
              qc[c] = 0;
              more = more || m > 0;
            }
          }
          signal_system(more ? &stage_done[it.slot] : &slot_done[it.slot]);
        }
      }
    } else {
      if (d.dtype == LB_F64) serve_kwindow<double>(U, d, it.type - 1, it.begin, it.end);
      else serve_kwindow<float>(U, d, it.type - 1, it.begin, it.end);
      if (threadIdx.x == 0) {
        __threadfence();
        const long long old = atomicAdd((unsigned long long*)&kdone[it.slot], 1ull);
        if (old + 1 == d.kitems) {                 // the request's last window
          kdone[it.slot] = 0;
          signal_system(&slot_done[it.slot]);
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Arena {           // first-fit allocator over one device buffer
  char* base = nullptr;
  size_t size = 0;
  std::map<size_t, size_t> free_;   // offset -> length
  void init(char* b, size_t s) { base = b; size = s; free_.clear(); free_[0] = s; }
  bool alloc(size_t n, size_t* off) {
    n = (n + 255) & ~(size_t)255;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const size_t rest = it->second - n, o = it->first + n;
        free_.erase(it);
        if (rest) free_[o] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = (n + 255) & ~(size_t)255;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) { it->second += nx->second; free_.erase(nx); }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) { pv->second += it->second; free_.erase(it); }
    }
  }
};

enum ReqState { RS_PENDING = 0, RS_COPY_IN = 1, RS_READY_WAIT = 2, RS_RUNNING = 3, RS_RUNNING_K = 4,
                RS_COPY_OUT = 5, RS_DONE = 6 };

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Request {
  long long ticket;
  int kind, dtype, mode, nclass;
  long long n, v_stride;
  bool device = false;             // buffers on the device: nothing is copied
  const void* hv;                  // caller's v, x, out (host or device)
  const void* hx;
  void* hout;
  cudaEvent_t ready = nullptr;     // device request: inputs ready once it completes (NULL: at once)
  size_t elem, off = 0, bytes = 0;
  int slot = -1;
  // scheduler state; RS_DONE is set under the server lock (waiters read it there)
  std::atomic<int> state{RS_PENDING};
  double t_submit = 0, t_admit = 0, t_done = 0;    // t_admit and t_done published with RS_DONE
  double t_admit_s = 0;                            // the scheduler's copy of t_admit

  size_t data_bytes() const {      // v, x, out in the arena (host requests)
    if (device) return 0;
    return round256((size_t)(v_stride ? n : 1) * elem) + 2 * round256((size_t)n * elem);
  }
  size_t queue_bytes() const { return kind == 1 ? round256((size_t)nclass * (size_t)n * 4) : 0; }
};

}  // namespace

// Threads: callers submit and wait; one scheduler thread owns everything
// between admission and completion (slots, arena, ring, copy events) and
// takes the lock only to collect new requests and to mark finished ones.
struct lb_server {
  int device = 0;
  int max_slots = 0, ring_cap = 0, ctas_per_sm = 4;
  long long idle_ns = 0;
  Ctl* ctl = nullptr;               // mapped host memory
  SlotDesc* slots = nullptr;        // mapped host memory
  WorkItem* ring = nullptr;         // mapped host memory
  int* slot_done = nullptr;         // mapped host memory [max_slots]: request finished
  int* stage_done = nullptr;        // mapped host memory [max_slots]: stage A finished, K queues posted
  unsigned* kcount = nullptr;       // mapped host memory [max_slots][8]: class queue lengths
  Ctl* d_ctl = nullptr;
  SlotDesc* d_slots = nullptr;
  WorkItem* d_ring = nullptr;
  int* d_slot_done = nullptr;
  int* d_stage_done = nullptr;
  unsigned* d_kcount = nullptr;
  unsigned long long* d_head = nullptr;
  long long* d_tiles_done = nullptr;
  long long* d_kdone = nullptr;
  unsigned* d_qcount = nullptr;     // device [max_slots][8]: class queue counters (reset by the device)
  unsigned long long* claim_pos = nullptr;     // mapped host memory [ctas]: ring position after each CTA's last claim
  unsigned long long* d_claim_pos = nullptr;
  int ctas = 0;                                  // CTAs of the persistent kernel
  unsigned long long* d_dstat = nullptr;   // device [1 + 2 kFamilies]: claim ns, busy ns and items per family
  unsigned long long* h_dstat = nullptr;   // pinned copy of d_dstat (lb_server_device_stats)
  cudaStream_t s_stats = nullptr;
  std::mutex stats_mu;
  char* d_arena = nullptr;
  cudaStream_t s_compute = nullptr, s_copy = nullptr;
  cudaEvent_t kernel_done = nullptr;

  // scheduler thread only
  Arena arena;
  bool kernel_live = false;
  long long tail = 0;               // host copy of the published count
  std::deque<Request*> waiting;     // submitted, not yet admitted (arrival order)
  std::vector<Request*> running;    // work published to the device
  std::vector<Request*> ready_wait; // device requests admitted, their ready event not yet complete
  std::deque<std::pair<Request*, cudaEvent_t>> copy_fifo;   // copies on s_copy, in stream order
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> free_slots;
  std::atomic<long long> kernel_launches{0};
  // items ready but not yet published, per item family, with the time each became ready
  std::deque<std::pair<WorkItem, double>> pend[kFamilies];
  long long pend_count = 0;

  // shared, under mu
  std::mutex mu;
  std::condition_variable cv;       // wakes the scheduler (submissions) and waiters (completions)
  std::deque<Request*> pending;
  std::map<long long, Request*> all;
  long long next_ticket = 1;
  bool stopping = false;
  std::string error;
  long long completed = 0;
  long long evals_done = 0;
  long long submitted = 0;
  std::thread sched;

  void loop();
  bool step(std::vector<Request*>& finished);
  void publish_tiles(Request* r);
  void publish_k(Request* r);
  void hold(int fam, const WorkItem& w, double t);
  bool publish_runs();
  void finish(Request* r, std::vector<Request*>& finished);
  cudaEvent_t take_event();
  lb_status submit(Request* r, long long* ticket);
};

namespace {
thread_local std::string g_serve_error;
lb_status serve_fail(lb_status s, const std::string& m) {
  g_serve_error = m;
  return s;
}
}  // namespace

cudaEvent_t lb_server::take_event() {
  if (!ev_pool.empty()) {
    cudaEvent_t e = ev_pool.back();
    ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  return e;
}

void lb_server::hold(int fam, const WorkItem& w, double t) {
  pend[fam].push_back({w, t});
  ++pend_count;
}

// Publishing.  Items of different families that run at the same time on an
// SM slow each other down (measured with lb_server_device_stats on a mix of
// the four request classes: the K-integral windows took 1.3x their time
// served alone, the FP32 items 2.2-2.6x; the kernels share the SMs'
// instruction caches).  So ready items wait in per-family lists and go to
// the ring in runs of one family: whenever fewer than one item per CTA is
// left untaken, a family publishes up to four items per CTA -- the family
// with the most items waiting, unless one has waited more than 1 ms (then
// the one that has waited longest).  The CTAs work through a run of one
// family before the next; families mix only at the ends of runs.  On the
// serving benchmark's mix (100,000 requests from 1024 slots) the capacity
// rose from 0.77 to 0.94 of large direct calls; runs of sixteen items per
// CTA gave the same capacity and a p99 latency of 79 ms at 80 % load
// (10 ms with four).
bool lb_server::publish_runs() {
  if (pend_count == 0) return false;
  unsigned long long head = 0;
  for (int i = 0; i < ctas; ++i) {
    const unsigned long long p = __atomic_load_n(&claim_pos[i], __ATOMIC_RELAXED);
    head = p > head ? p : head;
  }
  long long ahead = tail - (long long)head;
  bool progress = false;
  const double t_now = now_s();
  while (ahead < ctas && pend_count > 0) {
    int f = -1;
    for (int g = 0; g < kFamilies; ++g)
      if (!pend[g].empty() && t_now - pend[g].front().second > 1e-3 &&
          (f < 0 || pend[g].front().second < pend[f].front().second))
        f = g;
    if (f < 0)
      for (int g = 0; g < kFamilies; ++g)
        if (!pend[g].empty() && (f < 0 || pend[g].size() > pend[f].size())) f = g;
    const long long m = std::min<long long>((long long)pend[f].size(), 4ll * ctas);
    for (long long i = 0; i < m; ++i) {
      ring[tail % ring_cap] = pend[f].front().first;
      pend[f].pop_front();
      ++tail;
    }
    pend_count -= m;
    ahead += m;
    progress = true;
  }
  return progress;
}

// Stage A of a request: its tiles, in at most kItemsPerRequest items; FP32
// tiles are cheap, so an FP32 item holds at least four of them.
void lb_server::publish_tiles(Request* r) {
  const long long nt = slots[r->slot].ntiles;
  long long per = (nt + kItemsPerRequest - 1) / kItemsPerRequest;
  const long long min_tiles = r->dtype == LB_F64 ? 1 : 4;
  if (per < min_tiles) per = min_tiles;
  const int fam = (r->dtype == LB_F64 ? 0 : 2) + r->kind;
  const double t = now_s();
  for (long long b = 0; b < nt; b += per) {
    WorkItem w;
    w.slot = r->slot;
    w.begin = (int)b;
    w.end = (int)(b + per < nt ? b + per : nt);
    w.type = 0;
    hold(fam, w, t);
  }
  r->state.store(RS_RUNNING, std::memory_order_relaxed);
  running.push_back(r);
}

// Stage B of a K request: windows of each class queue, costliest class first.
void lb_server::publish_k(Request* r) {
  const unsigned* kc = kcount + 8 * r->slot;
  const double t = now_s();
  long long items = 0;
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) slots[r->slot].kitems = items;            // read by the device with the items
    for (int o = 0; o < kKClasses; ++o) {
      const int c = r->nclass == 1 ? (o == 0 ? 0 : -1) : kKClassOrder[o];
      if (c < 0) continue;
      const long long m = kc[c];
      if (m == 0) continue;
      long long w = (m + kKItemsPerClass - 1) / kKItemsPerClass;
      if (w < kKWindowMin) w = kKWindowMin;
      for (long long b = 0; b < m; b += w) {
        if (pass == 0) {
          ++items;
          continue;
        }
        WorkItem it;
        it.slot = r->slot;
        it.begin = (int)b;
        it.end = (int)(b + w < m ? b + w : m);
        it.type = 1 + c;
        hold(r->dtype == LB_F64 ? 4 + c : 4 + kKClasses, it, t);
      }
    }
  }
  r->state.store(RS_RUNNING_K, std::memory_order_relaxed);
}

// The request's work and copies are complete: free its slot and memory.
void lb_server::finish(Request* r, std::vector<Request*>& finished) {
  if (r->bytes) arena.release(r->off, r->bytes);
  free_slots.push_back(r->slot);
  r->t_done = now_s();
  finished.push_back(r);
}

// One pass of the scheduler; returns true if it made progress.
bool lb_server::step(std::vector<Request*>& finished) {
  {
    std::lock_guard<std::mutex> lk(mu);
    while (!pending.empty()) {
      waiting.push_back(pending.front());
      pending.pop_front();
    }
  }
  bool progress = false;
  const long long tail0 = tail;
  // admit: free slot and arena space, in arrival order (head of line blocks: no starvation)
  while (!waiting.empty() && !free_slots.empty()) {
    Request* r = waiting.front();
    const size_t vbytes = (size_t)(r->v_stride ? r->n : 1) * r->elem;
    const size_t xbytes = (size_t)r->n * r->elem;
    const size_t dbytes = r->data_bytes(), qbytes = r->queue_bytes();
    const size_t need = dbytes + qbytes;
    size_t off = 0;
    if (need > 0 && !arena.alloc(need, &off)) break;
    waiting.pop_front();
    r->off = off;
    r->bytes = need;
    r->slot = free_slots.back();
    free_slots.pop_back();
    char* base = d_arena + off;
    const char *dv, *dx;
    char* dout;
    if (r->device) {
      dv = (const char*)r->hv;
      dx = (const char*)r->hx;
      dout = (char*)r->hout;
    } else {
      dv = base;
      dx = base + round256(vbytes);
      dout = (char*)dx + round256(xbytes);
    }
    SlotDesc& sd = slots[r->slot];
    sd.kind = r->kind;
    sd.dtype = r->dtype;
    sd.mode = r->mode;
    sd.nclass = r->kind == 1 ? r->nclass : 0;
    sd.n = r->n;
    sd.v_stride = r->v_stride;
    sd.v = (unsigned long long)dv;
    sd.x = (unsigned long long)dx;
    sd.out = (unsigned long long)dout;
    sd.queue = (unsigned long long)(base + dbytes);
    sd.ntiles = (r->n + LB_TILE - 1) / LB_TILE;
    sd.kitems = 0;
    slot_done[r->slot] = 0;
    stage_done[r->slot] = 0;
    r->t_admit_s = now_s();
    if (!r->device) {
      cudaMemcpyAsync((void*)dv, r->hv, vbytes, cudaMemcpyHostToDevice, s_copy);
      cudaMemcpyAsync((void*)dx, r->hx, xbytes, cudaMemcpyHostToDevice, s_copy);
      cudaEvent_t e = take_event();
      cudaEventRecord(e, s_copy);
      r->state.store(RS_COPY_IN, std::memory_order_relaxed);
      copy_fifo.push_back({r, e});
    } else if (r->ready) {
      r->state.store(RS_READY_WAIT, std::memory_order_relaxed);
      ready_wait.push_back(r);
    } else {
      publish_tiles(r);
    }
    progress = true;
  }
  // copies complete in stream order: query from the oldest
  while (!copy_fifo.empty() && cudaEventQuery(copy_fifo.front().second) == cudaSuccess) {
    Request* r = copy_fifo.front().first;
    ev_pool.push_back(copy_fifo.front().second);
    copy_fifo.pop_front();
    if (r->state.load(std::memory_order_relaxed) == RS_COPY_IN) publish_tiles(r);
    else finish(r, finished);
    progress = true;
  }
  for (size_t i = 0; i < ready_wait.size();) {
    if (cudaEventQuery(ready_wait[i]->ready) == cudaSuccess) {
      publish_tiles(ready_wait[i]);
      ready_wait[i] = ready_wait.back();
      ready_wait.pop_back();
      progress = true;
    } else {
      ++i;
    }
  }
  for (size_t i = 0; i < running.size();) {
    Request* r = running[i];
    const int st = r->state.load(std::memory_order_relaxed);
    if (st == RS_RUNNING && __atomic_load_n(&stage_done[r->slot], __ATOMIC_ACQUIRE)) {
      publish_k(r);
      progress = true;
      ++i;
    } else if (__atomic_load_n(&slot_done[r->slot], __ATOMIC_ACQUIRE)) {
      if (r->device) {
        finish(r, finished);
      } else {
        cudaMemcpyAsync(r->hout, (const void*)slots[r->slot].out, (size_t)r->n * r->elem, cudaMemcpyDeviceToHost,
                        s_copy);
        cudaEvent_t e = take_event();
        cudaEventRecord(e, s_copy);
        r->state.store(RS_COPY_OUT, std::memory_order_relaxed);
        copy_fifo.push_back({r, e});
      }
      running[i] = running.back();
      running.pop_back();
      progress = true;
    } else {
      ++i;
    }
  }
  if (publish_runs()) progress = true;
  if (tail != tail0) __atomic_store_n(&ctl->tail, tail, __ATOMIC_RELEASE);
  // keep the persistent kernel running while work is published
  if (kernel_live && cudaEventQuery(kernel_done) == cudaSuccess) kernel_live = false;
  if (!running.empty() && !kernel_live) {
    lb_serve_kernel<<<ctas, LB_THREADS, 0, s_compute>>>(
        d_ctl, d_slots, d_ring, ring_cap, d_head, d_tiles_done, d_kdone, d_qcount, d_slot_done, d_stage_done,
        d_kcount, idle_ns, d_dstat, d_claim_pos);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      std::lock_guard<std::mutex> lk(mu);
      error = std::string("lb_serve_kernel launch: ") + cudaGetErrorString(e);
    }
    cudaEventRecord(kernel_done, s_compute);
    kernel_live = true;
    kernel_launches.fetch_add(1);
    progress = true;
  }
  return progress;
}

void lb_server::loop() {
  cudaSetDevice(device);
  std::vector<Request*> finished;
  for (;;) {
    const bool progress = step(finished);
    std::unique_lock<std::mutex> lk(mu);
    if (!finished.empty()) {
      for (Request* r : finished) {
        r->t_admit = r->t_admit_s;
        r->state.store(RS_DONE, std::memory_order_release);
        ++completed;
        evals_done += r->n;
      }
      finished.clear();
      cv.notify_all();
    }
    if (stopping) break;
    if (progress || !pending.empty()) continue;
    if (running.empty() && copy_fifo.empty() && ready_wait.empty() && waiting.empty()) {
      cv.wait_for(lk, std::chrono::milliseconds(2));         // idle: wait for a submission
    } else {
      lk.unlock();
      std::this_thread::yield();                             // work in flight: poll again
    }
  }
}

lb_status lb_server::submit(Request* r, long long* ticket) {
  r->elem = r->dtype == LB_F64 ? 8 : 4;
  r->nclass = (r->kind == 1 && r->dtype == LB_F64 && r->mode == LB_TIGHT) ? kKClasses : 1;
  const size_t need = r->data_bytes() + r->queue_bytes();
  if (need > arena.size) {                         // arena.size is fixed after creation
    delete r;
    return serve_fail(LB_ENOMEM, "request larger than the server arena");
  }
  {
    std::lock_guard<std::mutex> lk(mu);
    r->ticket = next_ticket++;
    r->t_submit = now_s();
    pending.push_back(r);
    all[r->ticket] = r;
    ++submitted;
    *ticket = r->ticket;
  }
  cv.notify_all();
  return LB_OK;
}

namespace {
lb_status check_request(lb_server* s, int kind, lb_dtype dtype, const void* v, int64_t v_stride, const void* x,
                        void* out, int64_t n, lb_mode mode, long long* ticket) {
  if (!s || !ticket) return serve_fail(LB_EINVAL, "NULL server or ticket");
  if (kind != 0 && kind != 1) return serve_fail(LB_EINVAL, "kind must be 0 (I) or 1 (K)");
  if (dtype != LB_F64 && dtype != LB_F32) return serve_fail(LB_EINVAL, "unknown dtype");
  if (mode < 0 || mode > 2) return serve_fail(LB_EINVAL, "unknown mode");
  if (dtype == LB_F32 && kind == 1 && mode != LB_TIGHT) return serve_fail(LB_ENOTSUP, "FP32 K needs LB_TIGHT");
  if (n < 1 || !v || !x || !out || (v_stride != 0 && v_stride != 1)) return serve_fail(LB_EINVAL, "bad request buffers");
  if (n > ((int64_t)1 << 31) - LB_TILE) return serve_fail(LB_EINVAL, "request larger than 2^31 - 1024 pairs");
  return LB_OK;
}

Request* new_request(int kind, lb_dtype dtype, const void* v, int64_t v_stride, const void* x, void* out, int64_t n,
                     lb_mode mode) {
  Request* r = new Request();
  r->kind = kind;
  r->dtype = dtype;
  r->mode = mode;
  r->n = n;
  r->v_stride = v_stride;
  r->hv = v;
  r->hx = x;
  r->hout = out;
  return r;
}
}  // namespace

extern "C" {

lb_status lb_server_create(const lb_server_config* cfg, lb_server** out) {
  if (!cfg || !out) return serve_fail(LB_EINVAL, "NULL config or out");
  if (cfg->arena_bytes < (1 << 20) || cfg->max_slots < 1 || cfg->max_slots > 4096 || cfg->ctas_per_sm < 1 ||
      cfg->ctas_per_sm > 8 || !(cfg->idle_ms > 0))
    return serve_fail(LB_EINVAL, "bad server configuration");
  lb_server* s = new lb_server();
  cudaGetDevice(&s->device);
  s->max_slots = cfg->max_slots;
  // every admitted request has at most kItemsPerRequest + kKClasses * kKItemsPerClass items
  // outstanding; twice that per slot, so the ring never wraps onto an item not yet read
  s->ring_cap = cfg->max_slots * 2 * (kItemsPerRequest + kKClasses * kKItemsPerClass);
  s->ctas_per_sm = cfg->ctas_per_sm;
  s->idle_ns = (long long)(cfg->idle_ms * 1e6);
  {
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    s->ctas = sms * cfg->ctas_per_sm;
  }
  const size_t ms = (size_t)cfg->max_slots;
  bool ok = cudaHostAlloc((void**)&s->ctl, sizeof(Ctl), cudaHostAllocMapped) == cudaSuccess &&
            cudaHostAlloc((void**)&s->slots, sizeof(SlotDesc) * ms, cudaHostAllocMapped) == cudaSuccess &&
            cudaHostAlloc((void**)&s->ring, sizeof(WorkItem) * s->ring_cap, cudaHostAllocMapped) == cudaSuccess &&
            cudaHostAlloc((void**)&s->slot_done, sizeof(int) * ms, cudaHostAllocMapped) == cudaSuccess &&
            cudaHostAlloc((void**)&s->stage_done, sizeof(int) * ms, cudaHostAllocMapped) == cudaSuccess &&
            cudaHostAlloc((void**)&s->kcount, sizeof(unsigned) * 8 * ms, cudaHostAllocMapped) == cudaSuccess &&
            cudaHostAlloc((void**)&s->claim_pos, sizeof(unsigned long long) * s->ctas, cudaHostAllocMapped) ==
                cudaSuccess;
  if (ok) {
    memset(s->ctl, 0, sizeof(Ctl));
    memset(s->slot_done, 0, sizeof(int) * ms);
    memset(s->stage_done, 0, sizeof(int) * ms);
    memset(s->kcount, 0, sizeof(unsigned) * 8 * ms);
    memset(s->claim_pos, 0, sizeof(unsigned long long) * s->ctas);
    ok = cudaHostGetDevicePointer((void**)&s->d_ctl, s->ctl, 0) == cudaSuccess &&
         cudaHostGetDevicePointer((void**)&s->d_slots, s->slots, 0) == cudaSuccess &&
         cudaHostGetDevicePointer((void**)&s->d_ring, s->ring, 0) == cudaSuccess &&
         cudaHostGetDevicePointer((void**)&s->d_slot_done, s->slot_done, 0) == cudaSuccess &&
         cudaHostGetDevicePointer((void**)&s->d_stage_done, s->stage_done, 0) == cudaSuccess &&
         cudaHostGetDevicePointer((void**)&s->d_kcount, s->kcount, 0) == cudaSuccess &&
         cudaHostGetDevicePointer((void**)&s->d_claim_pos, s->claim_pos, 0) == cudaSuccess &&
         cudaMalloc((void**)&s->d_head, sizeof(unsigned long long)) == cudaSuccess &&
         cudaMalloc((void**)&s->d_tiles_done, sizeof(long long) * ms) == cudaSuccess &&
         cudaMalloc((void**)&s->d_kdone, sizeof(long long) * ms) == cudaSuccess &&
         cudaMalloc((void**)&s->d_qcount, sizeof(unsigned) * 8 * ms) == cudaSuccess &&
         cudaMalloc((void**)&s->d_arena, (size_t)cfg->arena_bytes) == cudaSuccess &&
         cudaMalloc((void**)&s->d_dstat, sizeof(unsigned long long) * (1 + 2 * kFamilies)) == cudaSuccess &&
         cudaHostAlloc((void**)&s->h_dstat, sizeof(unsigned long long) * (1 + 2 * kFamilies),
                       cudaHostAllocDefault) == cudaSuccess &&
         cudaMemset(s->d_dstat, 0, sizeof(unsigned long long) * (1 + 2 * kFamilies)) == cudaSuccess &&
         cudaMemset(s->d_head, 0, sizeof(unsigned long long)) == cudaSuccess &&
         cudaMemset(s->d_tiles_done, 0, sizeof(long long) * ms) == cudaSuccess &&
         cudaMemset(s->d_kdone, 0, sizeof(long long) * ms) == cudaSuccess &&
         cudaMemset(s->d_qcount, 0, sizeof(unsigned) * 8 * ms) == cudaSuccess &&
         cudaStreamCreateWithFlags(&s->s_compute, cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithFlags(&s->s_copy, cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithFlags(&s->s_stats, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&s->kernel_done, cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    lb_server_destroy(s);
    return serve_fail(LB_ENOMEM, "server allocation failed");
  }
  s->arena.init(s->d_arena, (size_t)cfg->arena_bytes);
  for (int i = cfg->max_slots - 1; i >= 0; --i) s->free_slots.push_back(i);
  s->sched = std::thread([s] { s->loop(); });
  *out = s;
  return LB_OK;
}

lb_status lb_server_submit(lb_server* s, int kind, lb_dtype dtype, const void* v, int64_t v_stride, const void* x,
                           void* out, int64_t n, lb_mode mode, long long* ticket) {
  lb_status st = check_request(s, kind, dtype, v, v_stride, x, out, n, mode, ticket);
  if (st != LB_OK) return st;
  return s->submit(new_request(kind, dtype, v, v_stride, x, out, n, mode), ticket);
}

lb_status lb_server_submit_device(lb_server* s, int kind, lb_dtype dtype, const void* v, int64_t v_stride,
                                  const void* x, void* out, int64_t n, lb_mode mode, void* ready_event,
                                  long long* ticket) {
  lb_status st = check_request(s, kind, dtype, v, v_stride, x, out, n, mode, ticket);
  if (st != LB_OK) return st;
  Request* r = new_request(kind, dtype, v, v_stride, x, out, n, mode);
  r->device = true;
  r->ready = (cudaEvent_t)ready_event;
  return s->submit(r, ticket);
}

lb_status lb_server_wait(lb_server* s, long long ticket, double timeout_s) {
  if (!s) return serve_fail(LB_EINVAL, "NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return serve_fail(LB_EINVAL, "unknown ticket");
  Request* r = it->second;
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  while (r->state.load(std::memory_order_acquire) != RS_DONE) {
    if (!s->error.empty()) return serve_fail(LB_ECUDA, s->error);
    if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout &&
        r->state.load(std::memory_order_acquire) != RS_DONE)
      return serve_fail(LB_ETIMEOUT, "request not finished before the timeout");
  }
  return LB_OK;
}

lb_status lb_server_ticket_info(lb_server* s, long long ticket, int* done, double* t_submit, double* t_admit,
                                double* t_done) {
  if (!s) return serve_fail(LB_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return serve_fail(LB_EINVAL, "unknown ticket");
  Request* r = it->second;
  if (done) *done = r->state.load(std::memory_order_acquire) == RS_DONE;
  if (t_submit) *t_submit = r->t_submit;
  if (t_admit) *t_admit = r->t_admit;
  if (t_done) *t_done = r->t_done;
  return LB_OK;
}

lb_status lb_server_release(lb_server* s, long long ticket) {
  if (!s) return serve_fail(LB_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return serve_fail(LB_EINVAL, "unknown ticket");
  if (it->second->state.load(std::memory_order_acquire) != RS_DONE)
    return serve_fail(LB_EINVAL, "request still in flight");
  delete it->second;
  s->all.erase(it);
  return LB_OK;
}

lb_status lb_server_stats(lb_server* s, long long* completed, long long* evals, long long* kernel_launches,
                          long long* in_flight) {
  if (!s) return serve_fail(LB_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (completed) *completed = s->completed;
  if (evals) *evals = s->evals_done;
  if (kernel_launches) *kernel_launches = s->kernel_launches.load();
  if (in_flight) *in_flight = s->submitted - s->completed;
  return LB_OK;
}

lb_status lb_server_device_stats(lb_server* s, long long* claim_ns, long long* busy_ns, long long* items) {
  if (!s) return serve_fail(LB_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lk(s->stats_mu);
  const size_t nb = sizeof(unsigned long long) * (1 + 2 * kFamilies);
  // a copy engine reads the counters while the persistent kernel runs (its own non-blocking stream)
  if (cudaMemcpyAsync(s->h_dstat, s->d_dstat, nb, cudaMemcpyDeviceToHost, s->s_stats) != cudaSuccess ||
      cudaStreamSynchronize(s->s_stats) != cudaSuccess) {
    cudaGetLastError();
    return serve_fail(LB_ECUDA, "reading the device counters failed");
  }
  if (claim_ns) *claim_ns = (long long)s->h_dstat[0];
  for (int f = 0; f < kFamilies; ++f) {
    if (busy_ns) busy_ns[f] = (long long)s->h_dstat[1 + f];
    if (items) items[f] = (long long)s->h_dstat[1 + kFamilies + f];
  }
  return LB_OK;
}

lb_status lb_server_destroy(lb_server* s) {
  if (!s) return LB_OK;
  if (s->sched.joinable()) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stopping = true;
    }
    s->cv.notify_all();
    s->sched.join();
  }
  if (s->ctl) __atomic_store_n(&s->ctl->stop, 1, __ATOMIC_RELEASE);
  if (s->s_compute) cudaStreamSynchronize(s->s_compute);     // CTAs see the stop flag and return
  if (s->s_copy) cudaStreamSynchronize(s->s_copy);
  for (auto& kv : s->all) delete kv.second;      // every request not yet released, wherever it was
  for (auto& f : s->copy_fifo) cudaEventDestroy(f.second);
  for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
  if (s->kernel_done) cudaEventDestroy(s->kernel_done);
  if (s->s_compute) cudaStreamDestroy(s->s_compute);
  if (s->s_copy) cudaStreamDestroy(s->s_copy);
  if (s->s_stats) cudaStreamDestroy(s->s_stats);
  cudaFree(s->d_dstat);
  if (s->h_dstat) cudaFreeHost(s->h_dstat);
  cudaFree(s->d_arena);
  cudaFree(s->d_qcount);
  cudaFree(s->d_kdone);
  cudaFree(s->d_tiles_done);
  cudaFree(s->d_head);
  if (s->kcount) cudaFreeHost(s->kcount);
  if (s->claim_pos) cudaFreeHost(s->claim_pos);
  if (s->stage_done) cudaFreeHost(s->stage_done);
  if (s->slot_done) cudaFreeHost(s->slot_done);
  if (s->ring) cudaFreeHost(s->ring);
  if (s->slots) cudaFreeHost(s->slots);
  if (s->ctl) cudaFreeHost(s->ctl);
  delete s;
  return LB_OK;
}

const char* lb_server_last_error(void) { return g_serve_error.c_str(); }

}  // extern "C"
