// tpmc_measure_ceilings: the two throughput ceilings of the trace kernel's
// roofline, measured on the context's own device rather than taken from a
// datasheet.
//
// The trace kernel's per-particle work is FP32 arithmetic (box slabs, the
// watertight triangle test, the seeding solves) on node and triangle data
// that stays in L1/L2, so its two ceilings are:
//   - the FP32 FMA rate: a loop of independent dependent-FMA chains over
//     every SM, counted at 2 flops per FMA;
//   - the L2 read bandwidth: a buffer well inside L2, streamed repeatedly
//     with loads that bypass L1 (ld.global.cg), 16 bytes per load.
// A particle rate is bounded by min(fp32 / flops per particle,
// l2 / bytes per particle), with the per-particle work counted by the trace
// kernel's counters.
#include "runtime.h"

namespace tpmc {
namespace {

constexpr int kFmaChains = 8;
constexpr int kFmaIters = 8192;
constexpr size_t kL2Bytes = 32ull << 20;  // a quarter of the L2
constexpr int kL2Passes = 64;

// Every thread runs kFmaChains independent chains a <- a * b + c.  The
// result is stored only when it equals a value no chain reaches, so the
// compiler keeps the loop and the kernel writes nothing in practice.
__global__ void __launch_bounds__(256) fma_loop_kernel(float b, float c, float never, float* sink) {
  float a[kFmaChains];
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) a[k] = (float)(threadIdx.x + k);
#pragma unroll 1
  for (int it = 0; it < kFmaIters; it += 4) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int k = 0; k < kFmaChains; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) s += a[k];
  if (s == never) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Each pass reads the whole buffer once, grid-stride, four 16-byte loads in
// flight per thread; n4 counts float4 elements.  Blocks start their passes
// at different offsets so that all L2 slices serve every pass.
__global__ void __launch_bounds__(256) l2_read_kernel(const float4* __restrict__ buf, size_t n4, int passes,
                                                      float never, float* sink) {
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  float s = 0.0f;
#pragma unroll 1
  for (int p = 0; p < passes; ++p) {
    size_t i = tid;
#pragma unroll 1
    for (; i + 3 * stride < n4; i += 4 * stride) {
      const float4 v0 = __ldcg(&buf[i]);
      const float4 v1 = __ldcg(&buf[i + stride]);
      const float4 v2 = __ldcg(&buf[i + 2 * stride]);
      const float4 v3 = __ldcg(&buf[i + 3 * stride]);
      s += (v0.x + v1.y) + (v2.z + v3.w);
    }
    for (; i < n4; i += stride) s += __ldcg(&buf[i]).x;
  }
  if (s == never) sink[tid] = s;
}

// Best of `reps` timed launches after one warm-up launch, in milliseconds.
template <typename F>
cudaError_t time_best(cudaStream_t s, int reps, F launch, float* best_ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = launch();
  float best = 1e30f;
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms < best) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  *best_ms = best;
  return e;
}

}  // namespace
}  // namespace tpmc

using namespace tpmc;

extern "C" tpmc_status tpmc_measure_ceilings(tpmc_ctx* ctx, double* fp32_tflops, double* l2_read_gbs) {
  if (!ctx || !fp32_tflops || !l2_read_gbs) return fail(TPMC_EINVAL, "NULL argument");
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  const int threads = 256, blocks = c->num_sms * 4;
  void* buf = nullptr;
  tpmc_status st = c->alloc(&buf, kL2Bytes + (size_t)blocks * threads * sizeof(float), "ceiling buffers");
  if (st != TPMC_OK) return st;
  float* sink = reinterpret_cast<float*>(static_cast<char*>(buf) + kL2Bytes);
  cudaStream_t s = c->stream;
  float fma_ms = 0.0f, l2_ms = 0.0f;
  e = cudaMemsetAsync(buf, 0, kL2Bytes, s);
  if (e == cudaSuccess)
    e = time_best(s, 5, [&] {
      fma_loop_kernel<<<blocks, threads, 0, s>>>(0.999999f, 1e-6f, -1.0f, sink);
      return cudaGetLastError();
    }, &fma_ms);
  const size_t n4 = kL2Bytes / sizeof(float4);
  if (e == cudaSuccess)
    e = time_best(s, 5, [&] {
      l2_read_kernel<<<blocks, threads, 0, s>>>(static_cast<const float4*>(buf), n4, kL2Passes, -1.0f, sink);
      return cudaGetLastError();
    }, &l2_ms);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  c->release(buf);
  if (e != cudaSuccess) return cuda_fail(e, "tpmc_measure_ceilings");
  const double flops = 2.0 * kFmaChains * kFmaIters * (double)blocks * threads;
  *fp32_tflops = flops / (fma_ms * 1e-3) / 1e12;
  *l2_read_gbs = (double)kL2Bytes * kL2Passes / (l2_ms * 1e-3) / 1e9;
  return TPMC_OK;
}
