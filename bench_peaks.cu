// bench_peaks.cu -- microbenchmark of the non-tensor peaks of one GPU that the
// rooflines in bench.py use: FP32 FMA (scalar and packed f32x2), MUFU ex2 /
// sin, FP64 FMA, INT32 add (8 independent dependency chains per thread,
// the grid fills every SM), and the shared-memory bandwidth of conflict-free
// 128-bit loads.  Prints one JSON object per measurement.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 bench_peaks.cu -o bench_peaks && ./bench_peaks
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#define ITERS 4096
constexpr int CH = 8;

__global__ void k_ffma(float *out, float a, float b) {
  float x[CH];
  for (int c = 0; c < CH; ++c) x[c] = threadIdx.x * 1e-7f + c;
  for (int i = 0; i < ITERS; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0; for (int c = 0; c < CH; ++c) s += x[c];
  if (s == 1234.5f) out[0] = s;
}
__global__ void k_ffma2(float *out, float a, float b) {
  unsigned long long x[CH];
  unsigned long long A, B;
  { float2 t = make_float2(a, a); A = *reinterpret_cast<unsigned long long*>(&t); }
  { float2 t = make_float2(b, b); B = *reinterpret_cast<unsigned long long*>(&t); }
  for (int c = 0; c < CH; ++c) { float2 t = make_float2(threadIdx.x * 1e-7f + c, c); x[c] = *reinterpret_cast<unsigned long long*>(&t); }
  for (int i = 0; i < ITERS; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(A), "l"(B));
  }
  float s = 0; for (int c = 0; c < CH; ++c) { float2 t = *reinterpret_cast<float2*>(&x[c]); s += t.x + t.y; }
  if (s == 1234.5f) out[0] = s;
}
__global__ void k_ex2(float *out, float a) {
  float x[CH];
  for (int c = 0; c < CH; ++c) x[c] = threadIdx.x * 1e-7f + c * a;
  for (int i = 0; i < ITERS; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(x[c]));
  }
  float s = 0; for (int c = 0; c < CH; ++c) s += x[c];
  if (s == 1234.5f) out[0] = s;
}
__global__ void k_sin(float *out, float a) {
  float x[CH];
  for (int c = 0; c < CH; ++c) x[c] = threadIdx.x * 1e-7f + c * a;
  for (int i = 0; i < ITERS; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) asm volatile("sin.approx.ftz.f32 %0, %0;" : "+f"(x[c]));
  }
  float s = 0; for (int c = 0; c < CH; ++c) s += x[c];
  if (s == 1234.5f) out[0] = s;
}
__global__ void k_dfma(double *out, double a, double b) {
  double x[CH];
  for (int c = 0; c < CH; ++c) x[c] = threadIdx.x * 1e-7 + c;
  for (int i = 0; i < ITERS / 16; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0; for (int c = 0; c < CH; ++c) s += x[c];
  if (s == 1234.5) out[0] = s;
}
__global__ void k_iadd(int *out, int a) {
  int x[CH];
  for (int c = 0; c < CH; ++c) x[c] = threadIdx.x + c;
  for (int i = 0; i < ITERS; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) asm volatile("add.s32 %0, %0, %1;" : "+r"(x[c]) : "r"(a));
  }
  int s = 0; for (int c = 0; c < CH; ++c) s += x[c];
  if (s == 12345) out[0] = s;
}

// shared-memory reads: every thread streams 128-bit loads over a 48 KB buffer,
// a quarter-warp reading 128 contiguous bytes (conflict-free); 4 CTAs of 256
// threads per SM
constexpr int kSmemF4 = 3072;   // 48 KB
__global__ void k_lds128(int *out, int iters)
{
  __shared__ float4 buf[kSmemF4];
  for (int q = threadIdx.x; q < kSmemF4; q += blockDim.x) buf[q] = make_float4(q, q + 1, q + 2, q + 3);
  __syncthreads();
  const unsigned base = (unsigned)__cvta_generic_to_shared(buf);
  unsigned acc = 0;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      // float4 index (threadIdx.x + 256 c + 8 (i mod 4)) mod 3072: 12 loads per iteration
      // + 8 (i mod 4): the addresses move every iteration, by whole 128-byte rows
      const unsigned a = base + ((threadIdx.x + 256u * c + 8u * (i & 3)) % kSmemF4) * 16u;
      unsigned x, y, z, w;
      asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(x), "=r"(y), "=r"(z), "=r"(w) : "r"(a));
      acc ^= x ^ y ^ z ^ w;
    }
  }
  if (acc == 0x12345678u) out[0] = (int)acc;
}

template <typename F> float timeit(F f, int reps) {
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  f(); cudaDeviceSynchronize();
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0); f(); cudaEventRecord(e1); cudaEventSynchronize(e1);
    float ms; cudaEventElapsedTime(&ms, e0, e1); if (ms < best) best = ms;
  }
  return best;
}

int main() {
  int dev = 0, nsm = 0; cudaSetDevice(dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  float *fo; double *dd; int *io;
  cudaMalloc(&fo, 64); cudaMalloc(&dd, 64); cudaMalloc(&io, 64);
  const int threads = 256, blocks = nsm * 8;   // 2048 threads per SM
  const double nthr = (double)threads * blocks;
  double ops = nthr * ITERS * CH;
  float t;
  t = timeit([&] { k_ffma<<<blocks, threads>>>(fo, 0.999f, 0.001f); }, 5);
  printf("{\"kind\": \"fp32_fma\", \"tflops\": %.2f, \"ms\": %.3f}\n", 2 * ops / (t * 1e-3) / 1e12, t);
  t = timeit([&] { k_ffma2<<<blocks, threads>>>(fo, 0.999f, 0.001f); }, 5);
  printf("{\"kind\": \"fp32x2_fma\", \"tflops\": %.2f, \"ms\": %.3f}\n", 4 * ops / (t * 1e-3) / 1e12, t);
  t = timeit([&] { k_ex2<<<blocks, threads>>>(fo, -0.5f); }, 5);
  printf("{\"kind\": \"mufu_ex2\", \"gops\": %.1f, \"per_sm_per_clk_at_2070\": %.2f, \"ms\": %.3f}\n", ops / (t * 1e-3) / 1e9, ops / (t * 1e-3) / nsm / 2.07e9, t);
  t = timeit([&] { k_sin<<<blocks, threads>>>(fo, 0.5f); }, 5);
  printf("{\"kind\": \"mufu_sin\", \"gops\": %.1f, \"per_sm_per_clk_at_2070\": %.2f, \"ms\": %.3f}\n", ops / (t * 1e-3) / 1e9, ops / (t * 1e-3) / nsm / 2.07e9, t);
  t = timeit([&] { k_dfma<<<blocks, threads>>>(dd, 0.999, 0.001); }, 3);
  printf("{\"kind\": \"fp64_fma\", \"tflops\": %.3f, \"ms\": %.3f}\n", 2 * ops / 16 / (t * 1e-3) / 1e12, t);
  t = timeit([&] { k_iadd<<<blocks, threads>>>(io, 3); }, 5);
  printf("{\"kind\": \"int32_add\", \"tops\": %.2f, \"ms\": %.3f}\n", ops / (t * 1e-3) / 1e12, t);
  {
    const int lblocks = nsm * 4, liters = 4096;
    t = timeit([&] { k_lds128<<<lblocks, 256>>>(io, liters); }, 5);
    const double bytes = (double)lblocks * 256 * liters * 12 * 16;
    printf("{\"kind\": \"smem_lds128\", \"gbs\": %.1f, \"bytes_per_sm_per_clk_at_2070\": %.2f, \"ms\": %.3f}\n",
           bytes / (t * 1e-3) / 1e9, bytes / (t * 1e-3) / nsm / 2.07e9, t);
  }
  printf("{\"kind\": \"config\", \"sms\": %d, \"blocks\": %d, \"threads\": %d, \"chains\": %d, \"iters\": %d}\n", nsm, blocks, threads, CH, ITERS);
  cudaError_t e = cudaGetLastError();
  printf("{\"kind\": \"status\", \"err\": \"%s\"}\n", cudaGetErrorString(e));
  return e == cudaSuccess ? 0 : 1;
}
