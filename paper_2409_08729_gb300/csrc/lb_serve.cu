// lb_serve.cu -- continuous-batching evaluation server.
//
// Requests (log I or log K, FP64 or FP32-mixed, 1 .. millions of pairs)
// arrive from host threads at any time.  A host scheduler thread admits
// them as slots and device memory free up (admission by memory), copies
// their inputs into a device arena, and publishes their tiles as work items
// in a ring in mapped host memory.  A persistent kernel (one loop per CTA,
// several CTAs per SM) claims work items with a compare-and-swap on a
// device counter, runs each tile through the whole path of lb_tile.cuh
// (classify, bin, expressions, K integral in block), and flags a request
// done when its last tile finishes.  Requests that arrive while others run
// are interleaved tile by tile, so their work overlaps on the device.  The
// scheduler then copies results back and frees the slot and memory.
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

namespace {

constexpr int kItemsPerRequest = 64;   // a request is split into at most this many work items

struct SlotDesc {          // mapped host memory: written by the host, read by the device
  int kind;                // 0 = I, 1 = K
  int dtype;               // LB_F64 or LB_F32
  int mode;
  int pad;
  long long n;
  long long v_stride;
  unsigned long long v, x, out;   // device addresses in the arena
  long long ntiles;
};

struct WorkItem {          // 16 bytes
  int slot;
  int tile_begin;
  int tile_end;
  int pad;
};

struct Ctl {               // mapped host memory shared by host and device
  int stop;
  int pad0;
  long long tail;          // number of published work items
  int slot_done[1];        // [max_slots], set to 1 by the device
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <int KIND, typename T>
__device__ __forceinline__ void serve_tile(TileShared<T>& S, const SlotDesc& d, int64_t tile) {
  const T* v = reinterpret_cast<const T*>(d.v);
  const T* x = reinterpret_cast<const T*>(d.x);
  T* out = reinterpret_cast<T*>(d.out);
  const int64_t t0 = tile * LB_TILE;
  tile_bin<KIND, false, T>(S, v, d.v_stride, x, out, t0, d.n, d.mode, -1);
  tile_eval<KIND, false, T>(S, out, t0);
  if (KIND == KIND_K) tile_kint<false, T>(S, out, t0, d.mode == MODE_TIGHT);
  __syncthreads();
}

union ServeShared {
  TileShared<double> d;
  TileShared<float> f;
};

__global__ void __launch_bounds__(LB_THREADS)
lb_serve_kernel(Ctl* ctl, const SlotDesc* slots, const WorkItem* ring, int ring_cap,
                unsigned long long* head, long long* tiles_done, long long idle_ns) {
  __shared__ ServeShared U;
  __shared__ long long claimed;
  __shared__ SlotDesc desc;
  __shared__ WorkItem item;
  cuda::atomic_ref<long long, cuda::thread_scope_system> tail_ref(ctl->tail);
  cuda::atomic_ref<int, cuda::thread_scope_system> stop_ref(ctl->stop);
  for (;;) {
    if (threadIdx.x == 0) {
      long long got = -1;
      const unsigned long long deadline = global_ns() + (unsigned long long)idle_ns;
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
      if (got >= 0) {
        item = ring[got % ring_cap];
        desc = slots[item.slot];
      }
    }
    __syncthreads();
    if (claimed < 0) return;
    const SlotDesc d = desc;
    const WorkItem it = item;
    for (int64_t tile = it.tile_begin; tile < it.tile_end; ++tile) {
      if (d.dtype == LB_F64) {
        if (d.kind == 0) serve_tile<KIND_I, double>(U.d, d, tile);
        else serve_tile<KIND_K, double>(U.d, d, tile);
      } else {
        if (d.kind == 0) serve_tile<KIND_I, float>(U.f, d, tile);
        else serve_tile<KIND_K, float>(U.f, d, tile);
      }
    }
    if (threadIdx.x == 0) {
      __threadfence();
      const long long nt = it.tile_end - it.tile_begin;
      const long long old = atomicAdd((unsigned long long*)&tiles_done[it.slot], (unsigned long long)nt);
      if (old + nt == d.ntiles) {
        tiles_done[it.slot] = 0;                  // ready for the slot's next request
        __threadfence_system();
        cuda::atomic_ref<int, cuda::thread_scope_system> done_ref(ctl->slot_done[it.slot]);
        done_ref.store(1, cuda::memory_order_release);
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

enum ReqState { RS_PENDING = 0, RS_COPY_IN = 1, RS_RUNNING = 2, RS_COPY_OUT = 3, RS_DONE = 4, RS_FAILED = 5 };

struct Request {
  long long ticket;
  int kind, dtype, mode;
  long long n, v_stride;
  const void* hv;
  const void* hx;
  void* hout;
  size_t elem, off = 0, bytes = 0;
  int slot = -1;
  ReqState state = RS_PENDING;
  cudaEvent_t ev = nullptr;
  double t_submit = 0, t_admit = 0, t_done = 0;
};

}  // namespace

struct lb_server {
  int device = 0;
  int max_slots = 0, ring_cap = 0, ctas_per_sm = 4;
  long long idle_ns = 0;
  Ctl* ctl = nullptr;               // mapped host memory
  SlotDesc* slots = nullptr;        // mapped host memory
  WorkItem* ring = nullptr;         // mapped host memory
  Ctl* d_ctl = nullptr;
  SlotDesc* d_slots = nullptr;
  WorkItem* d_ring = nullptr;
  unsigned long long* d_head = nullptr;
  long long* d_tiles_done = nullptr;
  char* d_arena = nullptr;
  Arena arena;
  cudaStream_t s_compute = nullptr, s_copy = nullptr;
  cudaEvent_t kernel_done = nullptr;
  bool kernel_live = false;
  long long kernel_launches = 0;
  long long tail = 0;               // host copy of the published count

  std::mutex mu;
  std::condition_variable cv;       // wakes the scheduler and waiters
  std::deque<Request*> pending;
  std::vector<Request*> active;
  std::map<long long, Request*> all;
  std::vector<int> free_slots;
  long long next_ticket = 1;
  bool stopping = false;
  std::thread sched;
  std::string error;
  long long completed = 0;
  long long evals_done = 0;

  void loop();
  bool step_locked();
};

namespace {
thread_local std::string g_serve_error;
lb_status serve_fail(lb_status s, const std::string& m) {
  g_serve_error = m;
  return s;
}
}  // namespace

// One pass of the scheduler over the request states; returns true if it made progress.
bool lb_server::step_locked() {
  bool progress = false;
  // admit: free slot and arena space, in arrival order (head of line blocks: no starvation)
  while (!pending.empty() && !free_slots.empty()) {
    Request* r = pending.front();
    const size_t vbytes = (size_t)(r->v_stride ? r->n : 1) * r->elem;
    const size_t xbytes = (size_t)r->n * r->elem;
    const size_t need = ((vbytes + 255) & ~(size_t)255) + ((xbytes + 255) & ~(size_t)255) + ((xbytes + 255) & ~(size_t)255);
    size_t off;
    if (!arena.alloc(need, &off)) break;
    pending.pop_front();
    r->off = off;
    r->bytes = need;
    r->slot = free_slots.back();
    free_slots.pop_back();
    char* base = d_arena + off;
    char* dv = base;
    char* dx = dv + ((vbytes + 255) & ~(size_t)255);
    char* dout = dx + ((xbytes + 255) & ~(size_t)255);
    SlotDesc& sd = slots[r->slot];
    sd.kind = r->kind;
    sd.dtype = r->dtype;
    sd.mode = r->mode;
    sd.n = r->n;
    sd.v_stride = r->v_stride;
    sd.v = (unsigned long long)dv;
    sd.x = (unsigned long long)dx;
    sd.out = (unsigned long long)dout;
    sd.ntiles = (r->n + LB_TILE - 1) / LB_TILE;
    ctl->slot_done[r->slot] = 0;
    cudaMemcpyAsync(dv, r->hv, vbytes, cudaMemcpyHostToDevice, s_copy);
    cudaMemcpyAsync(dx, r->hx, xbytes, cudaMemcpyHostToDevice, s_copy);
    cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming);
    cudaEventRecord(r->ev, s_copy);
    r->state = RS_COPY_IN;
    r->t_admit = now_s();
    active.push_back(r);
    progress = true;
  }
  bool published = false;
  for (Request* r : active) {
    if (r->state == RS_COPY_IN && cudaEventQuery(r->ev) == cudaSuccess) {
      const long long nt = slots[r->slot].ntiles;
      const long long per = (nt + kItemsPerRequest - 1) / kItemsPerRequest;
      for (long long b = 0; b < nt; b += per) {
        WorkItem& w = ring[tail % ring_cap];
        w.slot = r->slot;
        w.tile_begin = (int)b;
        w.tile_end = (int)(b + per < nt ? b + per : nt);
        ++tail;
      }
      r->state = RS_RUNNING;
      published = true;
      progress = true;
    } else if (r->state == RS_RUNNING && __atomic_load_n(&ctl->slot_done[r->slot], __ATOMIC_ACQUIRE)) {
      const SlotDesc& sd = slots[r->slot];
      cudaMemcpyAsync(r->hout, (const void*)sd.out, (size_t)r->n * r->elem, cudaMemcpyDeviceToHost, s_copy);
      cudaEventRecord(r->ev, s_copy);
      r->state = RS_COPY_OUT;
      progress = true;
    } else if (r->state == RS_COPY_OUT && cudaEventQuery(r->ev) == cudaSuccess) {
      r->state = RS_DONE;
      r->t_done = now_s();
      arena.release(r->off, r->bytes);
      free_slots.push_back(r->slot);
      cudaEventDestroy(r->ev);
      r->ev = nullptr;
      ++completed;
      evals_done += r->n;
      progress = true;
    }
  }
  if (published) __atomic_store_n(&ctl->tail, tail, __ATOMIC_RELEASE);
  // drop finished requests from the active list
  std::vector<Request*> keep;
  keep.reserve(active.size());
  for (Request* r : active)
    if (r->state != RS_DONE) keep.push_back(r);
  if (keep.size() != active.size()) cv.notify_all();
  active.swap(keep);
  // keep the persistent kernel running while work is published
  bool want = false;
  for (Request* r : active)
    if (r->state == RS_RUNNING) want = true;
  if (kernel_live && cudaEventQuery(kernel_done) == cudaSuccess) kernel_live = false;
  if (want && !kernel_live) {
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    lb_serve_kernel<<<sms * ctas_per_sm, LB_THREADS, 0, s_compute>>>(d_ctl, d_slots, d_ring, ring_cap, d_head,
                                                                     d_tiles_done, idle_ns);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) error = std::string("lb_serve_kernel launch: ") + cudaGetErrorString(e);
    cudaEventRecord(kernel_done, s_compute);
    kernel_live = true;
    ++kernel_launches;
    progress = true;
  }
  return progress;
}

void lb_server::loop() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  while (!stopping) {
    const bool progress = step_locked();
    if (!progress) {
      // nothing moved: wait briefly for new submissions or device progress
      cv.wait_for(lk, std::chrono::microseconds(active.empty() ? 2000 : 20));
    }
  }
}

extern "C" {

lb_status lb_server_create(const lb_server_config* cfg, lb_server** out) {
  if (!cfg || !out) return serve_fail(LB_EINVAL, "NULL config or out");
  if (cfg->arena_bytes < (1 << 20) || cfg->max_slots < 1 || cfg->max_slots > 4096 || cfg->ctas_per_sm < 1 ||
      cfg->ctas_per_sm > 8 || !(cfg->idle_ms > 0))
    return serve_fail(LB_EINVAL, "bad server configuration");
  lb_server* s = new lb_server();
  cudaGetDevice(&s->device);
  s->max_slots = cfg->max_slots;
  s->ring_cap = cfg->max_slots * kItemsPerRequest;
  s->ctas_per_sm = cfg->ctas_per_sm;
  s->idle_ns = (long long)(cfg->idle_ms * 1e6);
  const size_t ctl_bytes = sizeof(Ctl) + sizeof(int) * (size_t)cfg->max_slots;
  bool ok = cudaHostAlloc((void**)&s->ctl, ctl_bytes, cudaHostAllocMapped) == cudaSuccess &&
            cudaHostAlloc((void**)&s->slots, sizeof(SlotDesc) * cfg->max_slots, cudaHostAllocMapped) == cudaSuccess &&
            cudaHostAlloc((void**)&s->ring, sizeof(WorkItem) * s->ring_cap, cudaHostAllocMapped) == cudaSuccess;
  if (ok) {
    memset(s->ctl, 0, ctl_bytes);
    ok = cudaHostGetDevicePointer((void**)&s->d_ctl, s->ctl, 0) == cudaSuccess &&
         cudaHostGetDevicePointer((void**)&s->d_slots, s->slots, 0) == cudaSuccess &&
         cudaHostGetDevicePointer((void**)&s->d_ring, s->ring, 0) == cudaSuccess &&
         cudaMalloc((void**)&s->d_head, sizeof(unsigned long long)) == cudaSuccess &&
         cudaMalloc((void**)&s->d_tiles_done, sizeof(long long) * cfg->max_slots) == cudaSuccess &&
         cudaMalloc((void**)&s->d_arena, (size_t)cfg->arena_bytes) == cudaSuccess &&
         cudaMemset(s->d_head, 0, sizeof(unsigned long long)) == cudaSuccess &&
         cudaMemset(s->d_tiles_done, 0, sizeof(long long) * cfg->max_slots) == cudaSuccess &&
         cudaStreamCreateWithFlags(&s->s_compute, cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithFlags(&s->s_copy, cudaStreamNonBlocking) == cudaSuccess &&
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
  if (!s || !ticket) return serve_fail(LB_EINVAL, "NULL server or ticket");
  if (kind != 0 && kind != 1) return serve_fail(LB_EINVAL, "kind must be 0 (I) or 1 (K)");
  if (dtype != LB_F64 && dtype != LB_F32) return serve_fail(LB_EINVAL, "unknown dtype");
  if (mode < 0 || mode > 2) return serve_fail(LB_EINVAL, "unknown mode");
  if (dtype == LB_F32 && kind == 1 && mode != LB_TIGHT) return serve_fail(LB_ENOTSUP, "FP32 K needs LB_TIGHT");
  if (n < 1 || !v || !x || !out || (v_stride != 0 && v_stride != 1)) return serve_fail(LB_EINVAL, "bad request buffers");
  Request* r = new Request();
  r->kind = kind;
  r->dtype = dtype;
  r->mode = mode;
  r->n = n;
  r->v_stride = v_stride;
  r->hv = v;
  r->hx = x;
  r->hout = out;
  r->elem = dtype == LB_F64 ? 8 : 4;
  const size_t need = 3 * (((size_t)n * r->elem + 255) & ~(size_t)255);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (need > s->arena.size) {
      delete r;
      return serve_fail(LB_ENOMEM, "request larger than the server arena");
    }
    r->ticket = s->next_ticket++;
    r->t_submit = now_s();
    s->pending.push_back(r);
    s->all[r->ticket] = r;
    *ticket = r->ticket;
  }
  s->cv.notify_all();
  return LB_OK;
}

lb_status lb_server_wait(lb_server* s, long long ticket, double timeout_s) {
  if (!s) return serve_fail(LB_EINVAL, "NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return serve_fail(LB_EINVAL, "unknown ticket");
  Request* r = it->second;
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  while (r->state != RS_DONE) {
    if (!s->error.empty()) return serve_fail(LB_ECUDA, s->error);
    if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout && r->state != RS_DONE)
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
  if (done) *done = r->state == RS_DONE;
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
  if (it->second->state != RS_DONE) return serve_fail(LB_EINVAL, "request still in flight");
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
  if (kernel_launches) *kernel_launches = s->kernel_launches;
  if (in_flight) *in_flight = (long long)(s->active.size() + s->pending.size());
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
  for (auto& kv : s->all) {
    if (kv.second->ev) cudaEventDestroy(kv.second->ev);
    delete kv.second;
  }
  for (Request* r : s->pending)
    if (s->all.find(r->ticket) == s->all.end()) delete r;
  if (s->kernel_done) cudaEventDestroy(s->kernel_done);
  if (s->s_compute) cudaStreamDestroy(s->s_compute);
  if (s->s_copy) cudaStreamDestroy(s->s_copy);
  cudaFree(s->d_arena);
  cudaFree(s->d_tiles_done);
  cudaFree(s->d_head);
  if (s->ring) cudaFreeHost(s->ring);
  if (s->slots) cudaFreeHost(s->slots);
  if (s->ctl) cudaFreeHost(s->ctl);
  delete s;
  return LB_OK;
}

const char* lb_server_last_error(void) { return g_serve_error.c_str(); }

}  // extern "C"
