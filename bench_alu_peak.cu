// Arithmetic peaks of one GPU, for the ALU roofline of the bench: FP32 FMA
// (scalar and packed f32x2, the form the DG contractions use), FP64 FMA, and
// the SM clock while the FP32 loop runs (clock64 against the global timer).
// Each thread runs 8 independent FMA chains; the grid is 8 blocks of 256
// threads per SM. Timed with CUDA events after one warm-up launch.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o bench_alu_peak bench_alu_peak.cu && ./bench_alu_peak
// Prints one JSON line (TFLOP/s counts an FMA as 2 flop).
#include <cuda_runtime.h>

#include <cstdio>

namespace {

constexpr int K = 8;  // independent chains per thread

__global__ void k_ffma(float* out, int iters, float a, float b) {
  float x[K];
#pragma unroll
  for (int k = 0; k < K; ++k) x[k] = threadIdx.x * 1e-3f + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < K; ++k) x[k] = __fmaf_rn(x[k], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) s += x[k];
  if (s == 1234.5f) out[blockIdx.x] = s;  // keeps the chains live
}

__global__ void k_ffma2(float* out, int iters, float a, float b) {
  float x[2 * K];
#pragma unroll
  for (int k = 0; k < 2 * K; ++k) x[k] = threadIdx.x * 1e-3f + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < K; ++k)
      asm("{\n\t.reg .b64 ra, rb, rc;\n\t"
          "mov.b64 ra, {%0, %1};\n\t"
          "mov.b64 rb, {%2, %2};\n\t"
          "mov.b64 rc, {%3, %3};\n\t"
          "fma.rn.f32x2 ra, ra, rb, rc;\n\t"
          "mov.b64 {%0, %1}, ra;\n\t}"
          : "+f"(x[2 * k]), "+f"(x[2 * k + 1])
          : "f"(a), "f"(b));
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 2 * K; ++k) s += x[k];
  if (s == 1234.5f) out[blockIdx.x] = s;
}

__global__ void k_dfma(double* out, int iters, double a, double b) {
  double x[K];
#pragma unroll
  for (int k = 0; k < K; ++k) x[k] = threadIdx.x * 1e-3 + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < K; ++k) x[k] = __fma_rn(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) s += x[k];
  if (s == 1234.5) out[blockIdx.x] = s;
}

// SM clock: cycles against nanoseconds of the global timer over a busy loop
__global__ void k_clock(unsigned long long* out, int iters, float a, float b) {
  unsigned long long t0, t1;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  const long long c0 = clock64();
  float x = threadIdx.x * 1e-3f;
  for (int i = 0; i < iters; ++i) x = __fmaf_rn(x, a, b);
  const long long c1 = clock64();
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = (unsigned long long)(c1 - c0);
    out[2 * blockIdx.x + 1] = t1 - t0;
  }
  if (x == 1234.5f) out[2 * blockIdx.x] = 0;
}

template <typename F>
float time_ms(F launch) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  launch();  // warm-up
  cudaDeviceSynchronize();
  cudaEventRecord(e0);
  launch();
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms;
}

}  // namespace

int main() {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, 0) != cudaSuccess) return 1;
  const int sms = prop.multiProcessorCount, nthr = 256, nblk = 8 * sms;
  float* of = nullptr;
  double* od = nullptr;
  unsigned long long* oc = nullptr;
  if (cudaMalloc(&of, nblk * sizeof(float)) != cudaSuccess || cudaMalloc(&od, nblk * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&oc, 2 * nblk * sizeof(unsigned long long)) != cudaSuccess)
    return 1;
  const double thr = (double)nblk * nthr;
  const int it32 = 1 << 18, it64 = 1 << 12;
  const float ms1 = time_ms([&] { k_ffma<<<nblk, nthr>>>(of, it32, 0.999f, 1e-3f); });
  const float ms2 = time_ms([&] { k_ffma2<<<nblk, nthr>>>(of, it32, 0.999f, 1e-3f); });
  const float ms3 = time_ms([&] { k_dfma<<<nblk, nthr>>>(od, it64, 0.999, 1e-3); });
  k_clock<<<nblk, nthr>>>(oc, 1 << 20, 0.999f, 1e-3f);
  if (cudaDeviceSynchronize() != cudaSuccess) return 1;
  unsigned long long h[2];
  cudaMemcpy(h, oc, sizeof(h), cudaMemcpyDeviceToHost);
  const double f32 = 2.0 * K * it32 * thr / (ms1 * 1e-3) / 1e12;
  const double f32x2 = 2.0 * 2 * K * it32 * thr / (ms2 * 1e-3) / 1e12;
  const double f64 = 2.0 * K * it64 * thr / (ms3 * 1e-3) / 1e12;
  printf("{\"device\": \"%s\", \"sms\": %d, \"fp32_fma_tflops\": %.2f, \"fp32x2_fma_tflops\": %.2f, "
         "\"fp64_fma_tflops\": %.3f, \"sm_mhz_under_load\": %.0f, \"ms\": [%.3f, %.3f, %.3f]}\n",
         prop.name, sms, f32, f32x2, f64, h[1] ? 1e3 * (double)h[0] / (double)h[1] : 0.0, ms1, ms2, ms3);
  cudaFree(of);
  cudaFree(od);
  cudaFree(oc);
  return 0;
}
