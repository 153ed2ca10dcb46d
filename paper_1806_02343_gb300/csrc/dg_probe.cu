// Throughput probes of the arithmetic the hot path uses (measurement support;
// the paper has no counterpart): packed FP32 FMA, FP64 FMA, the TF32 tensor
// core, and a device-memory copy, each timed with CUDA events on the caller's
// stream. They give the roofline denominators of the benchmark in the same job.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/dg_mhd.h"
#include "dg_tc.cuh"

namespace dgmhd {
namespace {

constexpr int kChains = 8;  // independent FMA chains per thread

// 8 packed FP32 FMA chains (fma.rn.f32x2: two FMAs per instruction)
__global__ void k_probe_f32(int iters, float seed, float* out) {
  float x[2 * kChains], y = 1.0000001f, z = 1e-7f;
#pragma unroll
  for (int i = 0; i < 2 * kChains; ++i) x[i] = seed + 0.001f * (threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i)
      asm volatile("{\n\t.reg .b64 ra, rb, rc;\n\tmov.b64 ra, {%0, %1};\n\tmov.b64 rb, {%2, %2};\n\t"
                   "mov.b64 rc, {%3, %3};\n\tfma.rn.f32x2 ra, ra, rb, rc;\n\tmov.b64 {%0, %1}, ra;\n\t}"
                   : "+f"(x[2 * i]), "+f"(x[2 * i + 1])
                   : "f"(y), "f"(z));
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 2 * kChains; ++i) s += x[i];
  if (s == 12345.f) out[0] = s;  // keeps the chains live
}

__global__ void k_probe_f64(int iters, double seed, double* out) {
  double x[kChains];
  const double y = 1.0000000001, z = 1e-12;
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = seed + 0.001 * (threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = __fma_rn(x[i], y, z);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == 12345.0) out[0] = s;
}

// One block per SM: one thread issues `iters` M = 128, N = 256, K = 8
// kind::tf32 MMAs alternating between two accumulators (columns 0..255 and
// 256..511), operands in shared memory; one commit, then a bounded wait.
__global__ void k_probe_tf32(int iters, int* status) {
  __shared__ __align__(1024) float A[128 * 8];
  __shared__ __align__(1024) float B[256 * 8];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t slot;
  const int t = threadIdx.x, warp = t >> 5;
  for (int i = t; i < 128 * 8; i += blockDim.x) A[i] = 0.01f * (i % 7);
  for (int i = t; i < 256 * 8; i += blockDim.x) B[i] = 0.01f * (i % 5);
  if (t == 0) {
    tc::mbar_init(&bar, 1);
    tc::mbar_fence_init();
  }
  if (warp == 0) tc::tmem_alloc(&slot, 512);
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tm = slot;
  bool ok = true;
  if (t == 0) {
    const uint32_t id = tc::idesc_tf32_f32(128, 256);
    // K-major [rows][8]: two 16-byte core matrices per 8-row group
    const uint64_t ad = tc::smem_desc(tc::smem_u32(A), 128, 256);
    const uint64_t bd = tc::smem_desc(tc::smem_u32(B), 128, 256);
    for (int i = 0; i < iters; ++i) {
      const uint32_t d = tm + (uint32_t)((i & 1) * 256);
      asm volatile(
          "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
          "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
          "l"(ad), "l"(bd), "r"(id), "r"(i >= 2 ? 1 : 0)
          : "memory");
    }
    tc::commit(&bar);
    ok = tc::mbar_wait_bounded(&bar, 0, 4000000000ll);
    if (!ok) atomicOr(status, 1);
  }
  __syncthreads();
  if (!ok && t == 0) tc::mbar_wait_bounded(&bar, 0, 4000000000ll);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tm, 512);
}

__global__ void k_probe_copy(const float4* __restrict__ src, float4* __restrict__ dst, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

}  // namespace
}  // namespace dgmhd

using namespace dgmhd;

extern "C" int dg_mhd_probe(int kind, const void* src, void* dst, int64_t bytes, double* rate, double* ms,
                            void* stream) {
  if (!rate || !ms || kind < 0 || kind > 3) return DG_E_ARG;
  if (kind == 3 && (!src || !dst || bytes <= 0 || bytes % 16 != 0)) return DG_E_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
    return DG_E_CUDA;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return DG_E_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return DG_E_CUDA;
  }
  void* scratch = nullptr;
  int code = DG_OK;
  double work = 0.0;
  if (cudaMalloc(&scratch, 64) != cudaSuccess || cudaMemsetAsync(scratch, 0, 64, st) != cudaSuccess) {
    code = DG_E_CUDA;
  } else {
    const unsigned blocks = (unsigned)nsm * 8, threads = 256;
    auto run = [&](auto launch) {
      launch();  // warm-up
      cudaEventRecord(e0, st);
      launch();
      cudaEventRecord(e1, st);
    };
    if (kind == 0) {
      const int iters = 4096;
      run([&] { k_probe_f32<<<blocks, threads, 0, st>>>(iters, 0.5f, (float*)scratch); });
      work = 2.0 * 2.0 * kChains * iters * (double)blocks * threads;
    } else if (kind == 1) {
      const int iters = 256;
      run([&] { k_probe_f64<<<blocks, threads, 0, st>>>(iters, 0.5, (double*)scratch); });
      work = 2.0 * kChains * iters * (double)blocks * threads;
    } else if (kind == 2) {
      const int iters = 8192;
      run([&] { k_probe_tf32<<<(unsigned)nsm, 128, 0, st>>>(iters, (int*)scratch); });
      work = 2.0 * 128.0 * 256.0 * 8.0 * iters * nsm;
    } else {
      const int64_t n = bytes / 16;
      run([&] { k_probe_copy<<<(unsigned)nsm * 8, 512, 0, st>>>((const float4*)src, (float4*)dst, n); });
      work = 2.0 * (double)bytes;
    }
    float t = 0.f;
    int flag = 0;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess ||
        cudaMemcpy(&flag, scratch, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      code = DG_E_CUDA;
    } else if (kind == 2 && flag) {
      code = DG_E_TIMEOUT;
    } else {
      *ms = t;
      *rate = t > 0.f ? work / (t * 1e-3) : 0.0;
    }
  }
  if (scratch) cudaFree(scratch);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return code;
}
