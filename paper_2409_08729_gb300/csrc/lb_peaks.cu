// lb_peaks.cu -- throughput microbenchmarks of the FP64 pipe on the current GPU.
//
// The log-Bessel kernels are bound by double-precision arithmetic, so their
// roofline is the FP64 pipe.  These kernels measure, with every SM busy:
//   - DFMA throughput: 8 independent fma chains per thread;
//   - the throughput of the library calls the kernels use (exp, log, lgamma,
//     division, sqrt), 4 independent chains per thread.
// The ratio DFMA rate / call rate is the number of DFMA issue slots one call
// occupies, which the roofline accounting uses as the cost of a call.  The
// table-driven exp (also without its low table part) and log of
// lb_fastmath.cuh, and the integer-pipe exp, log, reciprocal and 1/sqrt of
// lb_intmath.cuh, are measured the same way.
#include <cuda_runtime.h>
#include <stdint.h>

#include "logbessel.h"
#include "lb_fastmath.cuh"
#include "lb_intmath.cuh"

namespace {

__global__ void peak_dfma(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <int OP>
__device__ __forceinline__ double call_op(double a) {
  if (OP == 0) return exp(a) * 0.1;
  if (OP == 1) return log(a) + 2.0;
  if (OP == 2) return 3.0 / a + 1.0;
  if (OP == 3) return sqrt(a) + 1.0;
  if (OP == 5) return lb::fm_exp(a) * 0.1;
  if (OP == 6) return lb::fm_log(a) + 2.0;
  if (OP == 7) return lb::fm_exp_term(a) * 0.1;
  if (OP == 8) return lb::ix_exp(a) * 0.1;
  if (OP == 9) return lb::ix_log(a) + 2.0;
  if (OP == 10) return lb::ix_rcp(a) + 2.0;
  if (OP == 11) return lb::ix_rsqrt(a) + 2.0;
  return lgamma(a) + 2.0;
}

template <int OP>
__global__ void peak_call(double* out, int iters) {
  double a = (OP == 0 || OP == 5 || OP == 7 || OP == 8 ? 0.1 : 2.1) + threadIdx.x * 1e-6, b = a + 0.2, c = a + 0.3, d = a + 0.4;
  for (int i = 0; i < iters; ++i) {
    a = call_op<OP>(a); b = call_op<OP>(b); c = call_op<OP>(c); d = call_op<OP>(d);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a + b + c + d;
}

}  // namespace

extern "C" lb_status logbessel_measure_fp64(double* rates, void* cuda_stream) {
  if (!rates) return LB_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return LB_ECUDA;
  const int threads = 256, blocks = sms * 8;
  double* buf = nullptr;
  if (cudaMallocAsync(&buf, sizeof(double) * blocks * threads, st) != cudaSuccess) return LB_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  lb_status status = LB_OK;
  for (int which = 0; which < 13 && status == LB_OK; ++which) {
    const int iters = which == 0 ? 1000 : (which == 5 ? 40 : 160);
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, st);
      switch (which) {
        case 0: peak_dfma<<<blocks, threads, 0, st>>>(buf, iters, 0.999999, 1e-7); break;
        case 1: peak_call<0><<<blocks, threads, 0, st>>>(buf, iters); break;
        case 2: peak_call<1><<<blocks, threads, 0, st>>>(buf, iters); break;
        case 3: peak_call<2><<<blocks, threads, 0, st>>>(buf, iters); break;
        case 4: peak_call<3><<<blocks, threads, 0, st>>>(buf, iters); break;
        case 5: peak_call<4><<<blocks, threads, 0, st>>>(buf, iters); break;
        case 6: peak_call<5><<<blocks, threads, 0, st>>>(buf, iters); break;
        case 7: peak_call<6><<<blocks, threads, 0, st>>>(buf, iters); break;
        case 8: peak_call<7><<<blocks, threads, 0, st>>>(buf, iters); break;
        case 9: peak_call<8><<<blocks, threads, 0, st>>>(buf, iters); break;
        case 10: peak_call<9><<<blocks, threads, 0, st>>>(buf, iters); break;
        case 11: peak_call<10><<<blocks, threads, 0, st>>>(buf, iters); break;
        default: peak_call<11><<<blocks, threads, 0, st>>>(buf, iters); break;
      }
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) { status = LB_ECUDA; break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) best = ms;
    }
    const double ops = (double)blocks * threads * iters * (which == 0 ? 64.0 : 4.0);
    rates[which] = ops / (best * 1e-3);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(buf, st);
  return status;
}
