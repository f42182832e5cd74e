// Arithmetic issue rates of the GPU this runs on: float64 and float32 FMA,
// float64 and float32 division, float32 <-> float64 conversion. Each kernel
// runs 152*16 blocks x 256 threads, NCH independent chains of ITER operations
// per thread, and folds its results into one 64-bit word per thread, so that
// nothing is elided; the time of the second of two launches (CUDA events)
// gives operations per second. Prints one "name rate" line per kernel, rates
// in G operations/s. Test infrastructure: it measures the hardware the
// design choices of the float kernels rest on.
#include <cstdio>
#include <cuda_runtime.h>

constexpr int ITER = 2048, NCH = 8;

__global__ void k_dfma(const float* in, unsigned long long* out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  double x[NCH];
  for (int c = 0; c < NCH; ++c) x[c] = in[t % 1024] + c;
  for (int i = 0; i < ITER; ++i)
#pragma unroll
    for (int c = 0; c < NCH; ++c) x[c] = fma(x[c], 0.999999, 1e-7);
  double s = 0;
  for (int c = 0; c < NCH; ++c) s += x[c];
  out[t] = __double_as_longlong(s);
}
__global__ void k_ffma(const float* in, unsigned long long* out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  float x[NCH];
  for (int c = 0; c < NCH; ++c) x[c] = in[t % 1024] + c;
  for (int i = 0; i < ITER; ++i)
#pragma unroll
    for (int c = 0; c < NCH; ++c) x[c] = fmaf(x[c], 0.999999f, 1e-7f);
  float s = 0;
  for (int c = 0; c < NCH; ++c) s += x[c];
  out[t] = __float_as_uint(s);
}
__global__ void k_ddiv(const float* in, unsigned long long* out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  double x[NCH];
  for (int c = 0; c < NCH; ++c) x[c] = in[t % 1024] + c + 1.0;
  for (int i = 0; i < ITER / 8; ++i)
#pragma unroll
    for (int c = 0; c < NCH; ++c) x[c] = 1.0000001 / x[c] + 0.5;
  double s = 0;
  for (int c = 0; c < NCH; ++c) s += x[c];
  out[t] = __double_as_longlong(s);
}
__global__ void k_fdiv(const float* in, unsigned long long* out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  float x[NCH];
  for (int c = 0; c < NCH; ++c) x[c] = in[t % 1024] + c + 1.0f;
  for (int i = 0; i < ITER / 8; ++i)
#pragma unroll
    for (int c = 0; c < NCH; ++c) x[c] = 1.0000001f / x[c] + 0.5f;
  float s = 0;
  for (int c = 0; c < NCH; ++c) s += x[c];
  out[t] = __float_as_uint(s);
}
__global__ void k_f2d(const float* in, unsigned long long* out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned x[NCH];
  unsigned long long acc = 0;
  for (int c = 0; c < NCH; ++c) x[c] = __float_as_uint(in[t % 1024] + c + 1.0f);
  for (int i = 0; i < ITER; ++i)
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      unsigned long long b = __double_as_longlong((double)__uint_as_float(x[c]));
      acc ^= b;
      x[c] += (unsigned)(b >> 29) | 1u;
    }
  out[t] = acc;
}
__global__ void k_d2f(const float* in, unsigned long long* out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long x[NCH];
  unsigned acc = 0;
  for (int c = 0; c < NCH; ++c) x[c] = __double_as_longlong((double)in[t % 1024] + c + 1.0);
  for (int i = 0; i < ITER; ++i)
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      unsigned b = __float_as_uint((float)__longlong_as_double(x[c]));
      acc ^= b;
      x[c] += ((unsigned long long)(b & 7u) << 20) | 1ull;
    }
  out[t] = acc;
}

int main() {
  const int blocks = 152 * 16, threads = 256, n = blocks * threads;
  float* in = nullptr;
  unsigned long long* out = nullptr;
  if (cudaMalloc(&in, 1024 * sizeof(float)) || cudaMalloc(&out, (size_t)n * sizeof(unsigned long long))) return 1;
  cudaMemset(in, 0, 1024 * sizeof(float));
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  struct K {
    const char* name;
    void (*k)(const float*, unsigned long long*);
    double ops_per_thread;
  } ks[] = {{"fp64_fma", k_dfma, (double)ITER * NCH},   {"fp32_fma", k_ffma, (double)ITER * NCH},
            {"fp64_div", k_ddiv, (double)ITER / 8 * NCH}, {"fp32_div", k_fdiv, (double)ITER / 8 * NCH},
            {"cvt_f32_f64", k_f2d, (double)ITER * NCH},  {"cvt_f64_f32", k_d2f, (double)ITER * NCH}};
  for (const K& k : ks) {
    k.k<<<blocks, threads>>>(in, out);
    cudaEventRecord(a);
    k.k<<<blocks, threads>>>(in, out);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    printf("%s %.1f\n", k.name, (double)n * k.ops_per_thread / (ms * 1e-3) / 1e9);
  }
  cudaError_t e = cudaGetLastError();
  cudaFree(in);
  cudaFree(out);
  if (e != cudaSuccess) {
    printf("error %s\n", cudaGetErrorString(e));
    return 1;
  }
  return 0;
}
