// Learned per-column closure (an extension: the paper has no learned part).
//
// A dense MLP y = W_L^T relu(... relu(W_1^T x + b_1) ...) + b_L with float32
// master weights, bfloat16 weights and layer inputs on the tensor cores and
// float32 accumulation; trained with a mean-squared-error loss and Adam
// (Kingma and Ba 2015). The GEMMs run on the fifth-generation tensor cores:
// tcgen05.mma kind::f16 with bfloat16 operands in shared memory and the
// float32 accumulator in tensor memory, the operands brought in by TMA in
// the 128-byte swizzled layout (k_gemm_tma; transposed copies of the
// weights, layer inputs and gradients make every product read both operands
// along its contraction) or, for widths that are not multiples of 8, staged
// by threads (k_gemm_tc); the warp-level mma.sync m16n8k16 kernel
// (k_gemm_bf16) is kept as a switchable reference path (thor_mlp_tune).
//
// Closure: per column, the inputs are 5 fields (rho', M_x, M_y, M_z, Th') at
// all levels and the neighbour means of the same (as anomalies); the
// outputs are correction tendencies of the same 5 fields at all levels,
// added as field += dt * tendency after every large step. Training data come
// from high-resolution runs area-averaged onto the coarse grid
// (thor_coarse_grain).
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/thor.h"
#include "thor_state.h"

namespace thor {
namespace {

constexpr int BM = 64, BN = 64, BK = 16;   // block tile, 4 warps of 32 x 32

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[M][N] = op(A)[M][K] op(B)[K][N]; op(A)(m,k) = transA ? A[k*lda+m] : A[m*lda+k],
// op(B)(k,n) = transB ? B[n*ldb+k] : B[k*ldb+n]. Epilogue: + bias[n], relu,
// float32 store to C (ldc) and / or bfloat16 store to Cb (ldcb).
__global__ void __launch_bounds__(128) k_gemm_bf16(int M, int N, int K, const __nv_bfloat16* A, int lda,
                                                   int transA, const __nv_bfloat16* B, int ldb, int transB,
                                                   float* C, int ldc, const float* bias, int relu,
                                                   __nv_bfloat16* Cb, int ldcb) {
  __shared__ __align__(16) __nv_bfloat16 As[BM][BK + 8];
  __shared__ __align__(16) __nv_bfloat16 Bs[BK][BN + 8];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t = lane & 3;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const __nv_bfloat16 zero = __float2bfloat16(0.0f);
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int e = tid; e < BM * BK; e += 128) {
      const int r = e / BK, kk = e % BK, m = m0 + r, k = k0 + kk;
      __nv_bfloat16 v = zero;
      if (m < M && k < K) v = transA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k];
      As[r][kk] = v;
    }
    for (int e = tid; e < BK * BN; e += 128) {
      const int kk = e / BN, c = e % BN, k = k0 + kk, n = n0 + c;
      __nv_bfloat16 v = zero;
      if (k < K && n < N) v = transB ? B[(size_t)n * ldb + k] : B[(size_t)k * ldb + n];
      Bs[kk][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
      const int r = wm + mi * 16;
      uint32_t a[4];
      a[0] = pack_bf16(As[r + g][2 * t], As[r + g][2 * t + 1]);
      a[1] = pack_bf16(As[r + g + 8][2 * t], As[r + g + 8][2 * t + 1]);
      a[2] = pack_bf16(As[r + g][2 * t + 8], As[r + g][2 * t + 9]);
      a[3] = pack_bf16(As[r + g + 8][2 * t + 8], As[r + g + 8][2 * t + 9]);
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int c = wn + ni * 8;
        uint32_t b[2];
        b[0] = pack_bf16(Bs[2 * t][c + g], Bs[2 * t + 1][c + g]);
        b[1] = pack_bf16(Bs[2 * t + 8][c + g], Bs[2 * t + 9][c + g]);
        mma_bf16(acc[mi][ni], a, b);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + wm + mi * 16 + g + (q >= 2 ? 8 : 0);
        const int n = n0 + wn + ni * 8 + 2 * t + (q & 1);
        if (m >= M || n >= N) continue;
        float v = acc[mi][ni][q];
        if (bias) v += bias[n];
        if (relu) v = v > 0.0f ? v : 0.0f;
        if (C) C[(size_t)m * ldc + n] = v;
        if (Cb) Cb[(size_t)m * ldcb + n] = __float2bfloat16(v);
      }
}

__global__ void k_to_bf16(const float* x, __nv_bfloat16* y, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

// g <- g * (h > 0), then gb = bf16(g)
__global__ void k_relu_back(float* g, const __nv_bfloat16* h, __nv_bfloat16* gb, size_t n, int mask) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float v = g[i];
    if (mask && !(__bfloat162float(h[i]) > 0.0f)) v = 0.0f;
    g[i] = v;
    gb[i] = __float2bfloat16(v);
  }
}

// column sums of g [M][N] in two deterministic passes: partial sums over
// row blocks of 128 (k_colsum_part: 32 columns x 8 row lanes per block,
// lanes added in a fixed order), then one warp per column adds the R
// partials part[R][N] in a fixed order (k_colsum_final)
__global__ void __launch_bounds__(256) k_colsum_part(const float* g, int M, int N, float* part) {
  __shared__ float s[8][33];
  const int tx = threadIdx.x, ty = threadIdx.y, n = blockIdx.x * 32 + tx, r0 = blockIdx.y * 128;
  const int r1 = min(r0 + 128, M);
  float a = 0.0f;
  if (n < N) {
#pragma unroll 4
    for (int r = r0 + ty; r < r1; r += 8) a += g[(size_t)r * N + n];
  }
  s[ty][tx] = a;
  __syncthreads();
  if (ty == 0 && n < N) {
    float t = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) t += s[j][tx];
    part[(size_t)blockIdx.y * N + n] = t;
  }
}
__global__ void k_colsum_final(const float* part, int R, int N, float* out) {
  const int col = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (col >= N) return;
  float t = 0.0f;
  for (int j = lane; j < R; j += 32) t += part[(size_t)j * N + col];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) out[col] = t;
}

// dY = 2 (Y - T) / (M N); per-block partial sums of (Y - T)^2
__global__ void k_mse(const float* y, const float* t, float* dy, size_t n, float inv_n, float* part) {
  __shared__ float sh[256];
  float s = 0.0f;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float d = y[i] - t[i];
    dy[i] = 2.0f * d * inv_n;
    s += d * d;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// scale * (sum of part[0..n)), one block of 1024 threads, fixed-order tree
__global__ void __launch_bounds__(1024) k_sum_parts(const float* part, int n, float scale, float* out) {
  __shared__ float sh[1024];
  const int t = threadIdx.x;
  float a = 0.0f;
  for (int i = t; i < n; i += 1024) a += part[i];
  sh[t] = a;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if (t < w) sh[t] += sh[t + w];
    __syncthreads();
  }
  if (t == 0) *out = sh[0] * scale;
}

// Adam on float32 master weights, refreshing the bfloat16 copy of weights
__global__ void k_adam(float* p, const float* g, float* m, float* v, __nv_bfloat16* pb, size_t n, float lr,
                       float b1, float b2, float c1, float c2, float eps) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (pb) pb[i] = __float2bfloat16(pi);
  }
}

inline int blocks_for(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 4096); }

uint64_t splitmix(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}


// ------------------------------------------------------------ tcgen05 GEMM
//
// One CTA of 4 warps computes a 128 x NT tile of C (NT <= 256, a multiple of
// 16): row r of the tile is tensor-memory lane r, column n is tensor-memory
// column n of a float32 accumulator. Per chunk of 64 k, all threads stage the
// bfloat16 operand tiles (128 x 64 of op(A), NT x 64 of op(B)^T) into shared
// memory in the canonical K-major layout without swizzle: 8 x 8 core
// matrices of 16-byte rows, core matrices adjacent in k 128 B apart (leading
// byte offset), groups of 8 rows 1024 B apart (stride byte offset). One
// thread then issues four 128 x NT x 16 MMAs and commits them to an
// mbarrier, which every thread waits on (bounded) before the tiles are
// overwritten. The epilogue reads the accumulator with tcgen05.ld (warp w
// owns lanes 32w..32w+31), adds the bias, applies the ReLU and stores.

constexpr int TC_M = 128, TC_KC = 64;

__device__ __forceinline__ uint32_t tc_core_off(int r, int k) {
  return (uint32_t)((((r >> 3) * (TC_KC / 8) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

// shared-memory matrix descriptor: start address, leading and stride byte
// offsets (all >> 4), the fixed version bits 46-48 = 0b001, no swizzle
__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: float32 D (bits 4-5 = 1), bfloat16 A
// and B (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at 24
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__host__ __device__ constexpr int tc_cols(int nt) { return nt <= 32 ? 32 : nt <= 64 ? 64 : nt <= 128 ? 128 : 256; }

// Stages rows [r0, r0 + R) x k [k0, k0 + 64) of op(X) into core-matrix order
// at dst; op(X)(r, k) = X[r * ld + k] if kcontig, else X[k * ld + r]; zero
// outside rows_total x K. vec: ld a multiple of 8 and X 16-byte aligned, so
// full 8-element groups move as 16-byte vectors (transposed in registers when
// the source runs along r).
__device__ __forceinline__ void tc_stage(unsigned char* dst, const __nv_bfloat16* X, int ld, bool kcontig, int r0,
                                         int R, int rows_total, int k0, int K, bool vec, int tid) {
  const unsigned short* Xs = reinterpret_cast<const unsigned short*>(X);
  auto at = [&](int r, int k) -> uint32_t {
    if (r >= rows_total || k >= K) return 0u;
    return kcontig ? Xs[(size_t)r * ld + k] : Xs[(size_t)k * ld + r];
  };
  if (kcontig) {
    for (int u = tid; u < R * 8; u += 128) {
      const int r = u >> 3, kg = u & 7, row = r0 + r, k = k0 + kg * 8;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (row < rows_total) {
        if (vec && k + 8 <= K) {
          v = *reinterpret_cast<const uint4*>(Xs + (size_t)row * ld + k);
        } else {
          v.x = at(row, k) | (at(row, k + 1) << 16);
          v.y = at(row, k + 2) | (at(row, k + 3) << 16);
          v.z = at(row, k + 4) | (at(row, k + 5) << 16);
          v.w = at(row, k + 6) | (at(row, k + 7) << 16);
        }
      }
      *reinterpret_cast<uint4*>(dst + tc_core_off(r, kg * 8)) = v;
    }
  } else {
    const int G = R >> 3;
    for (int u = tid; u < G * 8; u += 128) {
      const int rg = u % G, kg = u / G, row = r0 + rg * 8, kb = k0 + kg * 8;
      uint32_t w[8][4];               // w[kk][j]: rows 2j, 2j+1 at k = kb + kk
      if (vec && row + 8 <= rows_total && kb + 8 <= K) {
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const uint4 v = *reinterpret_cast<const uint4*>(Xs + (size_t)(kb + kk) * ld + row);
          w[kk][0] = v.x;
          w[kk][1] = v.y;
          w[kk][2] = v.z;
          w[kk][3] = v.w;
        }
      } else {
#pragma unroll
        for (int kk = 0; kk < 8; ++kk)
#pragma unroll
          for (int j = 0; j < 4; ++j) w[kk][j] = at(row + 2 * j, kb + kk) | (at(row + 2 * j + 1, kb + kk) << 16);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        uint4 lo, hi;                 // core rows 2j (low halves) and 2j + 1 (high halves), k = kb..kb+7
        lo.x = __byte_perm(w[0][j], w[1][j], 0x5410);
        lo.y = __byte_perm(w[2][j], w[3][j], 0x5410);
        lo.z = __byte_perm(w[4][j], w[5][j], 0x5410);
        lo.w = __byte_perm(w[6][j], w[7][j], 0x5410);
        hi.x = __byte_perm(w[0][j], w[1][j], 0x7632);
        hi.y = __byte_perm(w[2][j], w[3][j], 0x7632);
        hi.z = __byte_perm(w[4][j], w[5][j], 0x7632);
        hi.w = __byte_perm(w[6][j], w[7][j], 0x7632);
        *reinterpret_cast<uint4*>(dst + tc_core_off(rg * 8 + 2 * j, kg * 8)) = lo;
        *reinterpret_cast<uint4*>(dst + tc_core_off(rg * 8 + 2 * j + 1, kg * 8)) = hi;
      }
    }
  }
}

// same contract as k_gemm_bf16; NT = tile width; err: device flag set when
// an MMA completion is not seen within the wait bound. Two shared-memory
// stages: chunk c + 1 is staged while the MMAs of chunk c run.
__global__ void __launch_bounds__(128, 1) k_gemm_tc(int M, int N, int K, const __nv_bfloat16* A, int lda,
                                                    int transA, const __nv_bfloat16* B, int ldb, int transB,
                                                    float* C, int ldc, const float* bias, int relu,
                                                    __nv_bfloat16* Cb, int ldcb, int NT, int* err) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  __shared__ uint64_t bar[2];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * TC_M, n0 = blockIdx.x * NT;
  const uint32_t ncols = (uint32_t)tc_cols(NT);
  const int stage_bytes = (TC_M + NT) * TC_KC * 2;
  const bool vecA = (lda % 8 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
  const bool vecB = (ldb % 8 == 0) && ((reinterpret_cast<uintptr_t>(B) & 15) == 0);
  if (warp == 0) tc_alloc(&tmem_base, ncols);
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = tc_idesc(TC_M, NT);
  const int nchunks = (K + TC_KC - 1) / TC_KC;
  uint32_t uses[2] = {0u, 0u};          // commits issued on each barrier
  bool ok = true;
  for (int c = 0; c < nchunks && ok; ++c) {
    const int b = c & 1;
    unsigned char* As = tsm + b * stage_bytes;
    unsigned char* Bs = As + TC_M * TC_KC * 2;
    if (c >= 2) ok = mbar_wait(&bar[b], (uses[b] - 1) & 1u);   // the MMAs that read this stage are done
    if (!__syncthreads_and(ok)) break;
    tc_stage(As, A, lda, !transA, m0, TC_M, M, c * TC_KC, K, vecA, tid);
    tc_stage(Bs, B, ldb, transB != 0, n0, NT, N, c * TC_KC, K, vecB, tid);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic-proxy writes -> tensor cores
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a_addr = smem_u32(As), b_addr = smem_u32(Bs);
#pragma unroll
      for (int kk = 0; kk < TC_KC / 16; ++kk) {
        const uint64_t ad = tc_smem_desc(a_addr + kk * 256, 128, 1024);
        const uint64_t bd = tc_smem_desc(b_addr + kk * 256, 128, 1024);
        tc_mma(tmem, ad, bd, idesc, (c > 0 || kk > 0) ? 1u : 0u);
      }
      tc_commit(&bar[b]);
    }
    uses[b] += 1u;
  }
  // the last commit covers every MMA issued before it
  const int last = (nchunks - 1) & 1;
  if (ok) ok = __syncthreads_and(mbar_wait(&bar[last], (uses[last] - 1) & 1u));
  tc_fence_after();
  if (ok) {
    // 64-column slabs: tensor memory -> shared memory (row r at stride 65
    // floats), then coalesced rows to global memory
    float* slab = reinterpret_cast<float*>(tsm);
    for (int s0 = 0; s0 < NT; s0 += 64) {
      const int w = NT - s0 < 64 ? NT - s0 : 64;
      for (int c = 0; c < w; c += 16) {
        uint32_t v[16];
        tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(s0 + c), v);
#pragma unroll
        for (int j = 0; j < 16; ++j) slab[(warp * 32 + lane) * 65 + c + j] = __uint_as_float(v[j]);
      }
      __syncthreads();
      for (int e = tid; e < TC_M * w; e += 128) {
        const int r = e / w, cc = e % w, row = m0 + r, n = n0 + s0 + cc;
        if (row < M && n < N) {
          float x = slab[r * 65 + cc];
          if (bias) x += bias[n];
          if (relu) x = x > 0.0f ? x : 0.0f;
          if (C) C[(size_t)row * ldc + n] = x;
          if (Cb) Cb[(size_t)row * ldcb + n] = __float2bfloat16(x);
        }
      }
      __syncthreads();
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
    for (int q = 0; q < 2; ++q)          // bounded: let outstanding MMAs finish before freeing
      if (uses[q]) mbar_wait(&bar[q], (uses[q] - 1) & 1u);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, ncols);
}

// dynamic shared memory of k_gemm_tc: the two tiles, and enough on top that
// no more CTAs share an SM than its 512 tensor-memory columns can hold
size_t tc_smem_bytes(int nt) {
  const size_t tiles = 2 * (size_t)(TC_M + nt) * TC_KC * 2;
  const int ctas = 512 / tc_cols(nt);
  const size_t cap = (size_t)(228 * 1024) / ctas - 2048;
  return std::max(tiles, std::min(cap, (size_t)200 * 1024));
}

// ------------------------------------------------ TMA-fed tcgen05 GEMM
//
// C[M][N] = A B^T for operands that both run along k in global memory
// (A [M][lda], B [N][ldb], ld a multiple of 8 elements, 16-byte aligned).
// The copy engine brings 128 x 64 and NT x 64 bfloat16 boxes into shared
// memory in the 128-byte swizzled K-major layout: one 128-byte row per
// matrix row, its eight 16-byte chunks permuted by XOR with (row mod 8),
// groups of 8 rows 1024 B apart (the stride byte offset); the four MMAs of
// a 64-deep chunk start 32 B apart inside those rows. Rows and k outside
// the operands arrive as zeros (tensor-map bounds). Stages form a ring of
// S <= TMA_STAGES with a full barrier (copies landed, by transaction bytes) and
// an empty barrier (the MMAs that read the stage are done, by
// tcgen05.commit). One thread issues copies and MMAs; all four warps run
// the epilogue, which can also store the bfloat16 result transposed (CbT,
// [N][ldt]) for a later product that contracts over the rows.

constexpr int TMA_STAGES = 4, TMA_KC = 64, kMaxSplit = 8;

// shared-memory matrix descriptor of the 128-byte swizzled K-major layout:
// stride byte offset 1024 (8-row atoms), leading byte offset unused within
// one swizzle row (encoded 1), version bits 46-47 = 1, layout type 2
// (SWIZZLE_128B) at bits 61-63
__device__ __forceinline__ uint64_t tc_desc_sw128(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
         (2ull << 61);
}

__device__ __forceinline__ void tma_load_box(uint32_t dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__global__ void __launch_bounds__(128, 1) k_gemm_tma(const __grid_constant__ CUtensorMap ma,
                                                     const __grid_constant__ CUtensorMap mb, int M, int N, int K,
                                                     float* C, int ldc, const float* bias, int relu,
                                                     __nv_bfloat16* Cb, int ldcb, __nv_bfloat16* CbT, int ldt,
                                                     int NT, int S, int kc_per, size_t c_split, int* err) {
  extern __shared__ unsigned char tma_raw[];
  __shared__ uint64_t full[TMA_STAGES], empty[TMA_STAGES], done;   // the first S in use
  __shared__ uint32_t tmem_base;
  __shared__ int all_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * TC_M, n0 = blockIdx.x * NT;
  const uint32_t ncols = (uint32_t)tc_cols(NT);
  const uint32_t raw = smem_u32(tma_raw), base = (raw + 1023u) & ~1023u;   // swizzle atoms need 1024 B alignment
  const uint32_t a_bytes = TC_M * TMA_KC * 2, stage_bytes = (uint32_t)(TC_M + NT) * TMA_KC * 2;
  if (warp == 0) tc_alloc(&tmem_base, ncols);
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    mbar_init_fence();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  // split-K: blockIdx.z takes chunks [c0, c0 + nchunks) and stores its
  // partial product at C + blockIdx.z * c_split
  const int c0 = blockIdx.z * kc_per;
  const int nchunks = min(kc_per, (K + TMA_KC - 1) / TMA_KC - c0);
  C += blockIdx.z * c_split;
  if (tid == 0) {
    const uint32_t idesc = tc_idesc(TC_M, NT);
    auto load = [&](int c) {
      const int s = c % S;
      const uint32_t a = base + (uint32_t)s * stage_bytes;
      mbar_arrive_expect_tx(&full[s], stage_bytes);
      tma_load_box(a, &ma, (c0 + c) * TMA_KC, m0, &full[s]);
      tma_load_box(a + a_bytes, &mb, (c0 + c) * TMA_KC, n0, &full[s]);
    };
    int issued = 0, c = 0;
    bool ok = true;
    for (; issued < nchunks && issued < S; ++issued) load(issued);
    for (; c < nchunks; ++c) {
      const int s = c % S;
      if (!mbar_wait(&full[s], (uint32_t)(c / S) & 1u)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t a = base + (uint32_t)s * stage_bytes, b = a + a_bytes;
#pragma unroll
      for (int kk = 0; kk < TMA_KC / 16; ++kk)
        tc_mma(tmem, tc_desc_sw128(a + kk * 32), tc_desc_sw128(b + kk * 32), idesc, (c > 0 || kk > 0) ? 1u : 0u);
      tc_commit(&empty[s]);
      // refill the stage of the previous chunk (issued == c - 1 + S)
      if (c >= 1 && issued < nchunks) {
        const int p = c - 1;
        if (!mbar_wait(&empty[p % S], (uint32_t)(p / S) & 1u)) {
          ok = false;
          ++c;
          break;
        }
        load(issued++);
      }
    }
    // on a timed-out wait, let the copies still in flight (chunks c .. issued - 1) land first (bounded)
    for (int q = c; q < issued; ++q) mbar_wait(&full[q % S], (uint32_t)(q / S) & 1u);
    tc_commit(&done);                                   // completes when every MMA issued above has
    const bool fin = mbar_wait(&done, 0u);
    all_ok = ok && fin;
    if (!(ok && fin)) atomicExch(err, 1);
  }
  __syncthreads();
  __syncwarp();
  tc_fence_after();
  if (all_ok) {
    // straight from the accumulator: lane r of warp w holds row 32w + r, 16
    // columns per tcgen05.ld; row-major stores move 16-byte vectors (N and
    // the leading dimensions are multiples of 8), the transposed store is
    // coalesced across the warp's 32 consecutive rows
    const int row = m0 + warp * 32 + lane;
    for (int c = 0; c < NT; c += 16) {
      uint32_t v[16];
      tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
      const int n = n0 + c;
      if (n >= N) break;                                 // warp-uniform
      float x[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        x[j] = __uint_as_float(v[j]);
        if (bias && n + j < N) x[j] += bias[n + j];
        if (relu) x[j] = x[j] > 0.0f ? x[j] : 0.0f;
      }
      if (row < M) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (n + 8 * h >= N) break;
          const float* y = x + 8 * h;
          if (C) {
            float4* o = reinterpret_cast<float4*>(C + (size_t)row * ldc + n + 8 * h);
            o[0] = make_float4(y[0], y[1], y[2], y[3]);
            o[1] = make_float4(y[4], y[5], y[6], y[7]);
          }
          if (Cb) {
            uint4 q;
            q.x = pack_bf16(__float2bfloat16(y[0]), __float2bfloat16(y[1]));
            q.y = pack_bf16(__float2bfloat16(y[2]), __float2bfloat16(y[3]));
            q.z = pack_bf16(__float2bfloat16(y[4]), __float2bfloat16(y[5]));
            q.w = pack_bf16(__float2bfloat16(y[6]), __float2bfloat16(y[7]));
            *reinterpret_cast<uint4*>(Cb + (size_t)row * ldcb + n + 8 * h) = q;
          }
        }
        if (CbT) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (n + j < N) CbT[(size_t)(n + j) * ldt + row] = __float2bfloat16(x[j]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  __syncwarp();
  if (warp == 0) tc_dealloc(tmem, ncols);
}

size_t tma_smem_bytes(int nt, int stages = TMA_STAGES) {
  return 1024 + (size_t)stages * (TC_M + nt) * TMA_KC * 2;
}

// C[M][N] (ldc) = sum over z < splits of W[z][M][N] (row length N), in z
// order; N a multiple of 4
__global__ void k_split_sum(const float* W, int splits, int M, int N, float* C, int ldc) {
  const size_t n4 = (size_t)M * (N / 4);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
    const size_t r = i / (N / 4), c = (i % (N / 4)) * 4;
    float4 a = *reinterpret_cast<const float4*>(W + r * N + c);
    for (int z = 1; z < splits; ++z) {
      const float4 b = *reinterpret_cast<const float4*>(W + (size_t)z * M * N + r * N + c);
      a.x += b.x;
      a.y += b.y;
      a.z += b.z;
      a.w += b.w;
    }
    *reinterpret_cast<float4*>(C + r * ldc + c) = a;
  }
}

// x (float32 [m][K]) -> h (bfloat16 [m][K]) and its transpose hT ([K][ldt])
// through a 32 x 32 shared-memory tile (both stores coalesced)
__global__ void k_to_bf16_t(const float* x, __nv_bfloat16* h, __nv_bfloat16* hT, int m, int K, int ldt) {
  __shared__ float t[32][33];
  const int k0 = blockIdx.x * 32, r0 = blockIdx.y * 32, tx = threadIdx.x;
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int r = r0 + j, k = k0 + tx;
    float v = 0.0f;
    if (r < m && k < K) {
      v = x[(size_t)r * K + k];
      h[(size_t)r * K + k] = __float2bfloat16(v);
    }
    t[j][tx] = v;
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int k = k0 + j, r = r0 + tx;
    if (k < K && r < m) hT[(size_t)k * ldt + r] = __float2bfloat16(t[tx][j]);
  }
}

// k_relu_back with the bfloat16 gradient also stored transposed (gbT
// [N][ldt]) and the column sums of the masked float32 gradient over each
// 32-row tile in part[row tile][N] (fixed order; k_colsum_final adds them)
__global__ void k_relu_back_t(float* g, const __nv_bfloat16* h, __nv_bfloat16* gb, __nv_bfloat16* gbT, int m, int N,
                              int ldt, int mask, float* part) {
  __shared__ float t[32][33];
  const int n0 = blockIdx.x * 32, r0 = blockIdx.y * 32, tx = threadIdx.x;
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int r = r0 + j, n = n0 + tx;
    float v = 0.0f;
    if (r < m && n < N) {
      const size_t i = (size_t)r * N + n;
      v = g[i];
      if (mask && !(__bfloat162float(h[i]) > 0.0f)) v = 0.0f;
      g[i] = v;
      gb[i] = __float2bfloat16(v);
    }
    t[j][tx] = v;
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int n = n0 + j, r = r0 + tx;
    if (n < N && r < m) gbT[(size_t)n * ldt + r] = __float2bfloat16(t[tx][j]);
  }
  if (threadIdx.y == 0 && n0 + tx < N) {
    float a = 0.0f;
#pragma unroll 8
    for (int j = 0; j < 32; ++j) a += t[j][tx];
    part[(size_t)blockIdx.y * N + n0 + tx] = a;
  }
}

// bfloat16 weights W_l [K][N] -> their transposes [N][K] at wtoff[l], every
// layer in one launch (blockIdx.z = layer)
struct WTable {
  int K[16], N[16];
  unsigned long long woff[16], wtoff[16];
};
__global__ void k_weights_t(const __nv_bfloat16* pb, __nv_bfloat16* pbt, WTable T) {
  __shared__ __nv_bfloat16 t[32][34];
  const int l = blockIdx.z, K = T.K[l], N = T.N[l];
  const int n0 = blockIdx.x * 32, k0 = blockIdx.y * 32, tx = threadIdx.x;
  if (n0 >= N || k0 >= K) return;
  const __nv_bfloat16* W = pb + T.woff[l];
  __nv_bfloat16* Wt = pbt + T.wtoff[l];
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int k = k0 + j, n = n0 + tx;
    if (k < K && n < N) t[j][tx] = W[(size_t)k * N + n];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int n = n0 + j, k = k0 + tx;
    if (n < N && k < K) Wt[(size_t)n * K + k] = t[tx][j];
  }
}
}  // namespace
}  // namespace thor

// ================================================================== MLP

struct thor_mlp {
  std::vector<int> sizes;              // layer widths, n_layers + 1 entries
  int use_tc = 1;                      // tcgen05 TMA-fed (1) or thread-staged (2), mma.sync reference path (0)
  bool tma_ok = false;                 // every width a multiple of 8 and the tensor-map encoder found
  bool fwd_tma = false;                // the last forward kept the transposed layer inputs
  int sms = 148;                       // streaming multiprocessors of the device
  int ldt = 0;                         // row length of the transposed buffers (max_batch rounded up to 64)
  int* err = nullptr;                  // device flag of the tcgen05 kernels
  int max_batch = 0;
  cudaStream_t stream = nullptr;
  size_t nparam = 0;
  std::vector<size_t> woff, boff;      // offsets of W_l and b_l in the flat parameter vector
  void* arena = nullptr;
  float *p = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;   // flat float32 [nparam]
  __nv_bfloat16* pb = nullptr;         // bf16 copy of all parameters (weights used)
  __nv_bfloat16* pbt = nullptr;        // bf16 transposed weights, W_l^T [N][K] at wtoff[l]
  std::vector<size_t> wtoff;
  std::vector<__nv_bfloat16*> h;       // layer inputs (bf16) [max_batch][sizes[l]]
  std::vector<__nv_bfloat16*> hT;      // their transposes [sizes[l]][ldt] (TMA-fed backward)
  __nv_bfloat16* gbT = nullptr;        // transposed bf16 gradient scratch [max width][ldt]
  std::vector<float*> z;               // hidden outputs / gradients (float32) [max_batch][sizes[l+1]]
  __nv_bfloat16* gb = nullptr;         // bf16 gradient scratch [max_batch][max width]
  float* y = nullptr;                  // network output [max_batch][n_out]
  float* dy = nullptr;                 // output gradient
  float* part = nullptr;               // reduction partials
  float* cpart = nullptr;              // column-sum partials [row blocks][max width]
  float* ws = nullptr;                 // split-K partial products [splits][M][N]
  size_t ws_elems = 0;
  int last_m = 0;
  long long step_count = 0;
  int n_layers() const { return (int)sizes.size() - 1; }
};

namespace thor {
namespace {

void gemm(const thor_mlp* net, int M, int N, int K, const __nv_bfloat16* A, int lda, int transA,
          const __nv_bfloat16* B, int ldb, int transB, float* C, int ldc, const float* bias, int relu,
          __nv_bfloat16* Cb, int ldcb) {
  cudaStream_t st = net->stream;
  if (net->use_tc) {
    // the widest tile (fewest re-stagings of A) that still gives about one
    // CTA per SM, else 64 columns
    const int mtiles = (M + TC_M - 1) / TC_M;
    int width = 64;
    for (int w : {256, 128})
      if (mtiles * ((N + w - 1) / w) >= 148) {
        width = w;
        break;
      }
    const int ntiles = (N + width - 1) / width;
    const int nt = ((N + ntiles - 1) / ntiles + 15) / 16 * 16;
    dim3 grid(ntiles, (M + TC_M - 1) / TC_M);
    k_gemm_tc<<<grid, 128, tc_smem_bytes(nt), st>>>(M, N, K, A, lda, transA, B, ldb, transB, C, ldc, bias, relu,
                                                    Cb, ldcb, nt, net->err);
    return;
  }
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
  k_gemm_bf16<<<grid, 128, 0, st>>>(M, N, K, A, lda, transA, B, ldb, transB, C, ldc, bias, relu, Cb, ldcb);
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_tiled() {
  static void* fn = nullptr;
  static bool looked = false;
  if (!looked) {
    looked = true;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
  }
  return reinterpret_cast<EncodeTiled>(fn);
}

// tensor map of a bfloat16 operand X [rows][ld] read along k (k < kext):
// boxes of 64 k x box_rows rows, 128-byte swizzle, zeros outside
bool encode_operand(CUtensorMap* map, const __nv_bfloat16* X, int kext, int rows, int ld, int box_rows) {
  EncodeTiled enc = encode_tiled();
  if (!enc || (reinterpret_cast<uintptr_t>(X) & 15) || ld % 8) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)kext, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)TMA_KC, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(X), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// C = A B^T, A [M][lda] and B [N][ldb] both along k, on k_gemm_tma: the
// widest tile (fewest re-reads of A) that still gives a CTA per SM, else
// 16 columns
int gemm_tma(const thor_mlp* net, int M, int N, int K, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B,
             int ldb, float* C, int ldc, const float* bias, int relu, __nv_bfloat16* Cb, int ldcb,
             __nv_bfloat16* CbT, int ldt) {
  const int mtiles = (M + TC_M - 1) / TC_M;
  int width = 16;
  for (int w : {256, 128, 64, 32})
    if (mtiles * ((N + w - 1) / w) >= net->sms) {
      width = w;
      break;
    }
  const int ntiles = (N + width - 1) / width;
  const int nt = ((N + ntiles - 1) / ntiles + 15) / 16 * 16;
  // a long contraction on too few tiles (the weight gradients: K = batch)
  // is split along k over the idle SMs; the float32 partials are added in
  // a fixed order afterwards
  const int nchunks = (K + TMA_KC - 1) / TMA_KC, ctas = mtiles * ntiles;
  int splits = 1;
  if (C && !Cb && !CbT && !bias && !relu && 2 * ctas <= net->sms && nchunks >= 8) {
    splits = std::min({(net->sms + ctas - 1) / ctas, nchunks / 4, kMaxSplit});
    while (splits > 1 && (size_t)splits * M * N > net->ws_elems) --splits;
  }
  const int kc_per = (nchunks + splits - 1) / splits;
  splits = (nchunks + kc_per - 1) / kc_per;
  // the deepest ring that still lets every CTA of the grid be resident at
  // once (a second, partial wave would double the time of a short product)
  const int per_sm = (ctas * splits + net->sms - 1) / net->sms;
  int stages = 2;
  for (int st = TMA_STAGES; st > 2; --st)
    if ((size_t)per_sm * (tma_smem_bytes(nt, st) + 2048) <= (size_t)227 * 1024 && per_sm * tc_cols(nt) <= 512) {
      stages = st;
      break;
    }
  CUtensorMap ma, mb;
  if (!encode_operand(&ma, A, K, M, lda, TC_M) || !encode_operand(&mb, B, K, N, ldb, nt)) return THOR_ECUDA;
  dim3 grid(ntiles, mtiles, splits);
  const size_t smem = tma_smem_bytes(nt, stages);
  if (splits == 1) {
    k_gemm_tma<<<grid, 128, smem, net->stream>>>(ma, mb, M, N, K, C, ldc, bias, relu, Cb, ldcb, CbT, ldt, nt, stages,
                                                  kc_per, 0, net->err);
  } else {
    k_gemm_tma<<<grid, 128, smem, net->stream>>>(ma, mb, M, N, K, net->ws, N, nullptr, 0, nullptr, 0, nullptr, 0, nt,
                                                  stages, kc_per, (size_t)M * N, net->err);
    const size_t n4 = (size_t)M * N / 4;
    k_split_sum<<<(int)std::min<size_t>((n4 + 255) / 256, 2048), 256, 0, net->stream>>>(net->ws, splits, M, N, C,
                                                                                          ldc);
  }
  return THOR_OK;
}

// forward for m rows of x (float32 [m][n_in] on the device); keep_t: also
// store the transposed layer inputs the TMA-fed backward contracts over
int mlp_forward(thor_mlp* net, const float* x, int m, bool keep_t = true) {
  cudaStream_t st = net->stream;
  const int L = net->n_layers();
  const bool tma = net->use_tc == 1 && net->tma_ok;
  net->fwd_tma = tma && keep_t;
  if (net->fwd_tma) {
    dim3 g((net->sizes[0] + 31) / 32, (m + 31) / 32);
    k_to_bf16_t<<<g, dim3(32, 8), 0, st>>>(x, net->h[0], net->hT[0], m, net->sizes[0], net->ldt);
  } else {
    k_to_bf16<<<blocks_for((size_t)m * net->sizes[0]), 256, 0, st>>>(x, net->h[0], (size_t)m * net->sizes[0]);
  }
  for (int l = 0; l < L; ++l) {
    const int K = net->sizes[l], N = net->sizes[l + 1];
    const float* b = net->p + net->boff[l];
    const bool last = l + 1 == L;
    if (tma) {
      // op(B) = W_l read along k from its transposed copy [N][K]
      int rc = gemm_tma(net, m, N, K, net->h[l], K, net->pbt + net->wtoff[l], K, last ? net->y : nullptr, N, b,
                        !last, last ? nullptr : net->h[l + 1], N,
                        last || !net->fwd_tma ? nullptr : net->hT[l + 1], net->ldt);
      if (rc) return rc;
      continue;
    }
    const __nv_bfloat16* W = net->pb + net->woff[l];
    if (!last)
      gemm(net, m, N, K, net->h[l], K, 0, W, N, 0, nullptr, 0, b, 1, net->h[l + 1], N);
    else
      gemm(net, m, N, K, net->h[l], K, 0, W, N, 0, net->y, N, b, 0, nullptr, 0);
  }
  net->last_m = m;
  return cudaGetLastError() == cudaSuccess ? THOR_OK : THOR_ECUDA;
}

// gradients of sum(y * dy) after a forward of the same batch; dy float32 [m][n_out]
int mlp_backward(thor_mlp* net, const float* dy, int m) {
  cudaStream_t st = net->stream;
  const int L = net->n_layers();
  // g (float32) lives in z[l] buffers: z[L-1] holds the output gradient
  float* g = net->z[L - 1];
  if (cudaMemcpyAsync(g, dy, (size_t)m * net->sizes[L] * sizeof(float), cudaMemcpyDeviceToDevice, st))
    return THOR_ECUDA;
  // the TMA-fed products need the transposed inputs of a TMA-fed forward
  const bool tma = net->fwd_tma && net->use_tc == 1;
  for (int l = L - 1; l >= 0; --l) {
    const int K = net->sizes[l], N = net->sizes[l + 1];
    float* gl = net->z[l];
    const size_t cnt = (size_t)m * N;
    const __nv_bfloat16* W = net->pb + net->woff[l];
    // relu mask of this layer's output (hidden layers), then bf16 copy
    if (tma) {
      dim3 g((N + 31) / 32, (m + 31) / 32);
      k_relu_back_t<<<g, dim3(32, 8), 0, st>>>(gl, l + 1 < L ? net->h[l + 1] : nullptr, net->gb, net->gbT, m, N,
                                               net->ldt, l + 1 < L, net->cpart);
      // db_l = column sums of g
      k_colsum_final<<<(N * 32 + 255) / 256, 256, 0, st>>>(net->cpart, (m + 31) / 32, N, net->grad + net->boff[l]);
      // dW_l = h_l^T gb ([K][N]) from the transposes, both along the batch
      int rc = gemm_tma(net, K, N, m, net->hT[l], net->ldt, net->gbT, net->ldt, net->grad + net->woff[l], N,
                        nullptr, 0, nullptr, 0, nullptr, 0);
      if (rc) return rc;
    } else {
      k_relu_back<<<blocks_for(cnt), 256, 0, st>>>(gl, l + 1 < L ? net->h[l + 1] : nullptr, net->gb, cnt,
                                                   l + 1 < L);
      // dW_l = h_l^T gb  ([K][N])
      gemm(net, K, N, m, net->h[l], K, 1, net->gb, N, 0, net->grad + net->woff[l], N, nullptr, 0, nullptr, 0);
      // db_l = column sums of g
      k_colsum_part<<<dim3((N + 31) / 32, (m + 127) / 128), dim3(32, 8), 0, st>>>(gl, m, N, net->cpart);
      k_colsum_final<<<(N * 32 + 255) / 256, 256, 0, st>>>(net->cpart, (m + 127) / 128, N, net->grad + net->boff[l]);
    }
    if (l > 0) {
      // g_{l-1} = gb W_l^T ([m][K]) into z[l-1]; W_l [K][N] runs along N, the contraction
      if (tma) {
        int rc = gemm_tma(net, m, K, N, net->gb, N, W, N, net->z[l - 1], K, nullptr, 0, nullptr, 0, nullptr, 0);
        if (rc) return rc;
      } else {
        gemm(net, m, K, N, net->gb, N, 0, W, N, 1, net->z[l - 1], K, nullptr, 0, nullptr, 0);
      }
    }
  }
  return cudaGetLastError() == cudaSuccess ? THOR_OK : THOR_ECUDA;
}

// refreshes the transposed bfloat16 weights from pb (TMA-fed forward)
void weights_t(const thor_mlp* net) {
  if (!net->tma_ok) return;
  WTable T{};
  int kmax = 0, nmax = 0;
  const int L = net->n_layers();
  for (int l = 0; l < L; ++l) {
    T.K[l] = net->sizes[l];
    T.N[l] = net->sizes[l + 1];
    T.woff[l] = net->woff[l];
    T.wtoff[l] = net->wtoff[l];
    kmax = std::max(kmax, T.K[l]);
    nmax = std::max(nmax, T.N[l]);
  }
  dim3 g((nmax + 31) / 32, (kmax + 31) / 32, L);
  k_weights_t<<<g, dim3(32, 8), 0, net->stream>>>(net->pb, net->pbt, T);
}

}  // namespace
}  // namespace thor

extern "C" {

int thor_mlp_create(const int* sizes, int n_sizes, int max_batch, unsigned long long seed, void* stream,
                    thor_mlp** out) {
  using namespace thor;
  if (!sizes || !out || n_sizes < 2 || n_sizes > 16 || max_batch < 1) return THOR_EINVAL;
  for (int i = 0; i < n_sizes; ++i)
    if (sizes[i] < 1 || sizes[i] > 8192) return THOR_EINVAL;
  thor_mlp* net = new (std::nothrow) thor_mlp;
  if (!net) return THOR_ENOMEM;
  net->sizes.assign(sizes, sizes + n_sizes);
  net->max_batch = max_batch;
  net->stream = static_cast<cudaStream_t>(stream);
  const int L = n_sizes - 1;
  int wmax = 0;
  for (int l = 0; l < L; ++l) {
    net->woff.push_back(net->nparam);
    net->nparam += (size_t)sizes[l] * sizes[l + 1];
    net->boff.push_back(net->nparam);
    net->nparam += sizes[l + 1];
  }
  for (int i = 0; i < n_sizes; ++i) wmax = std::max(wmax, sizes[i]);
  // the TMA-fed products read rows of 16-byte multiples
  net->tma_ok = encode_tiled() != nullptr;
  for (int i = 0; i < n_sizes; ++i) net->tma_ok = net->tma_ok && sizes[i] % 8 == 0;
  net->ldt = (max_batch + 63) / 64 * 64;
  size_t nwt = 0;
  for (int l = 0; l < L; ++l) {
    net->wtoff.push_back(nwt);
    nwt += ((size_t)sizes[l] * sizes[l + 1] + 63) / 64 * 64;
  }
  {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
      net->sms = sms;
  }
  // one arena: params, grads, Adam moments, bf16 params, activations
  size_t bytes = 0;
  auto take = [&](size_t b) { size_t o = bytes; bytes += (b + 255) / 256 * 256; return o; };
  size_t o_p = take(net->nparam * 4), o_g = take(net->nparam * 4), o_m = take(net->nparam * 4),
         o_v = take(net->nparam * 4), o_pb = take(net->nparam * 2);
  std::vector<size_t> o_h, o_z, o_ht;
  for (int l = 0; l < L; ++l) o_h.push_back(take((size_t)max_batch * sizes[l] * 2));
  for (int l = 0; l < L; ++l) o_z.push_back(take((size_t)max_batch * sizes[l + 1] * 4));
  size_t o_gb = take((size_t)max_batch * wmax * 2), o_y = take((size_t)max_batch * sizes[L] * 4),
         o_dy = take((size_t)max_batch * sizes[L] * 4), o_part = take(4096 * 4 + 64), o_err = take(64),
         o_cpart = take((size_t)((max_batch + 31) / 32) * wmax * 4);
  size_t o_pbt = 0, o_gbt = 0, o_ws = 0;
  if (net->tma_ok) {
    size_t wmn = 0;
    for (int l = 0; l < L; ++l) wmn = std::max(wmn, (size_t)sizes[l] * sizes[l + 1]);
    net->ws_elems = (size_t)kMaxSplit * wmn;
    o_ws = take(net->ws_elems * 4);
    o_pbt = take(nwt * 2);
    for (int l = 0; l < L; ++l) o_ht.push_back(take((size_t)sizes[l] * net->ldt * 2));
    o_gbt = take((size_t)wmax * net->ldt * 2);
  }
  if (cudaMalloc(&net->arena, bytes) != cudaSuccess) {
    delete net;
    return THOR_ENOMEM;
  }
  char* base = static_cast<char*>(net->arena);
  net->p = (float*)(base + o_p);
  net->grad = (float*)(base + o_g);
  net->m = (float*)(base + o_m);
  net->v = (float*)(base + o_v);
  net->pb = (__nv_bfloat16*)(base + o_pb);
  for (int l = 0; l < L; ++l) {
    net->h.push_back((__nv_bfloat16*)(base + o_h[l]));
    net->z.push_back((float*)(base + o_z[l]));
  }
  net->gb = (__nv_bfloat16*)(base + o_gb);
  net->y = (float*)(base + o_y);
  net->err = (int*)(base + o_err);
  if (net->tma_ok) {
    net->pbt = (__nv_bfloat16*)(base + o_pbt);
    for (int l = 0; l < L; ++l) net->hT.push_back((__nv_bfloat16*)(base + o_ht[l]));
    net->gbT = (__nv_bfloat16*)(base + o_gbt);
    net->ws = (float*)(base + o_ws);
  }
  if (cudaMemsetAsync(net->err, 0, 64, net->stream) ||
      cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024) ||
      cudaFuncSetAttribute(k_gemm_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma_smem_bytes(256))) {
    cudaFree(net->arena);
    delete net;
    return THOR_ECUDA;
  }
  net->dy = (float*)(base + o_dy);
  net->part = (float*)(base + o_part);
  net->cpart = (float*)(base + o_cpart);
  // He-uniform initial weights from SplitMix64, zero biases
  std::vector<float> host(net->nparam, 0.0f);
  for (int l = 0; l < L; ++l) {
    const double a = std::sqrt(6.0 / sizes[l]);
    const size_t nw = (size_t)sizes[l] * sizes[l + 1];
    for (size_t i = 0; i < nw; ++i) {
      uint64_t r = splitmix(seed ^ (net->woff[l] + i));
      double u = (double)(r >> 11) * (1.0 / 9007199254740992.0);
      host[net->woff[l] + i] = (float)((2.0 * u - 1.0) * a);
    }
  }
  cudaStream_t st = net->stream;
  if (cudaMemsetAsync(net->arena, 0, bytes, st) ||
      cudaMemcpyAsync(net->p, host.data(), net->nparam * 4, cudaMemcpyHostToDevice, st)) {
    cudaFree(net->arena);
    delete net;
    return THOR_ECUDA;
  }
  k_to_bf16<<<blocks_for(net->nparam), 256, 0, st>>>(net->p, net->pb, net->nparam);
  weights_t(net);
  if (cudaStreamSynchronize(st)) {
    cudaFree(net->arena);
    delete net;
    return THOR_ECUDA;
  }
  *out = net;
  return THOR_OK;
}

int thor_mlp_info(const thor_mlp* net, size_t* nparam) {
  if (!net || !nparam) return THOR_EINVAL;
  *nparam = net->nparam;
  return THOR_OK;
}

int thor_mlp_get_params(thor_mlp* net, float* host, size_t n) {
  if (!net || !host || n != net->nparam) return THOR_EINVAL;
  int flag = 0;
  if (cudaMemcpyAsync(host, net->p, n * 4, cudaMemcpyDeviceToHost, net->stream)) return THOR_ECUDA;
  if (cudaMemcpyAsync(&flag, net->err, sizeof(int), cudaMemcpyDeviceToHost, net->stream)) return THOR_ECUDA;
  if (cudaStreamSynchronize(net->stream)) return THOR_ECUDA;
  return flag ? THOR_ETIMEOUT : THOR_OK;
}

int thor_mlp_tune(thor_mlp* net, int knob, int value) {
  if (!net) return THOR_EINVAL;
  if (knob == THOR_MLP_TUNE_TCGEN05) {
    if (value < 0 || value > 2) return THOR_EINVAL;
    net->use_tc = value;
    return THOR_OK;
  }
  return THOR_EINVAL;
}

int thor_mlp_set_params(thor_mlp* net, const float* host, size_t n) {
  using namespace thor;
  if (!net || !host || n != net->nparam) return THOR_EINVAL;
  if (cudaMemcpyAsync(net->p, host, n * 4, cudaMemcpyHostToDevice, net->stream)) return THOR_ECUDA;
  k_to_bf16<<<blocks_for(n), 256, 0, net->stream>>>(net->p, net->pb, n);
  weights_t(net);
  if (cudaMemsetAsync(net->m, 0, n * 4, net->stream) || cudaMemsetAsync(net->v, 0, n * 4, net->stream))
    return THOR_ECUDA;
  net->step_count = 0;
  return cudaStreamSynchronize(net->stream) ? THOR_ECUDA : THOR_OK;
}

int thor_mlp_forward(thor_mlp* net, const float* x, int m, float* y) {
  using namespace thor;
  if (!net || !x || !y || m < 1 || m > net->max_batch) return THOR_EINVAL;
  int rc = mlp_forward(net, x, m);
  if (rc) return rc;
  const size_t cnt = (size_t)m * net->sizes.back() * sizeof(float);
  return cudaMemcpyAsync(y, net->y, cnt, cudaMemcpyDeviceToDevice, net->stream) ? THOR_ECUDA : THOR_OK;
}

int thor_mlp_backward(thor_mlp* net, const float* dy, int m, float* grad) {
  using namespace thor;
  if (!net || !dy || !grad || m != net->last_m || m < 1) return THOR_EINVAL;
  int rc = mlp_backward(net, dy, m);
  if (rc) return rc;
  return cudaMemcpyAsync(grad, net->grad, net->nparam * 4, cudaMemcpyDeviceToDevice, net->stream) ? THOR_ECUDA
                                                                                              : THOR_OK;
}

int thor_mlp_train_step(thor_mlp* net, const float* x, const float* target, int m, float lr, float* loss) {
  using namespace thor;
  if (!net || !x || !target || m < 1 || m > net->max_batch || !(lr > 0)) return THOR_EINVAL;
  cudaStream_t st = net->stream;
  int rc = mlp_forward(net, x, m);
  if (rc) return rc;
  const size_t cnt = (size_t)m * net->sizes.back();
  const int nb = std::min(blocks_for(cnt), 1024);
  k_mse<<<nb, 256, 0, st>>>(net->y, target, net->dy, cnt, 1.0f / (float)cnt, net->part);
  if (loss) k_sum_parts<<<1, 1024, 0, st>>>(net->part, nb, 1.0f / (float)cnt, loss);
  rc = mlp_backward(net, net->dy, m);
  if (rc) return rc;
  net->step_count += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)net->step_count), c2 = 1.0f - powf(b2, (float)net->step_count);
  k_adam<<<blocks_for(net->nparam), 256, 0, st>>>(net->p, net->grad, net->m, net->v, net->pb, net->nparam, lr,
                                                  b1, b2, c1, c2, 1e-8f);
  weights_t(net);
  return cudaGetLastError() == cudaSuccess ? THOR_OK : THOR_ECUDA;
}

void thor_mlp_destroy(thor_mlp* net) {
  if (!net) return;
  if (net->arena) cudaFree(net->arena);
  delete net;
}

}  // extern "C"

// ================================================================ closure

namespace thor {
namespace {

constexpr int kClosureFields = 5;   // rho', M_x, M_y, M_z, Th'

template <typename R>
__device__ __forceinline__ const R* closure_field(const Xf<R>& X, int f) {
  return f == 0 ? X.rho : f == 1 ? X.mx : f == 2 ? X.my : f == 3 ? X.mz : X.th;
}
template <typename R>
__device__ __forceinline__ R* closure_field_rw(const Xf<R>& X, int f) {
  return f == 0 ? X.rho : f == 1 ? X.mx : f == 2 ? X.my : f == 3 ? X.mz : X.th;
}

// x[c][f nv + k] = field f at level k; x[c][5 nv + f nv + k] = the mean of
// that field over the neighbours of c minus its value at c (the neighbour
// anomaly carries the horizontal-curvature signal without the cancellation
// that bfloat16 inputs would suffer if centre and mean were given apart);
// normalised by (x - mean) / std per feature
template <typename R>
__global__ void k_features(Geo<R> G, Xf<R> X, const float* mean, const float* std, float* x) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (c >= G.ncol) return;
  const int S = G.colp, nv = G.nv, F = 2 * kClosureFields * nv;
  int nb[6], nn = 0;
  for (int j = 0; j < 6; ++j) {
    const int q = G.nbr[j * S + c];
    if (q != c) nb[nn++] = q;
  }
  for (int f = 0; f < kClosureFields; ++f) {
    const R* a = closure_field(X, f) + (size_t)k * S;
    const int j0 = f * nv + k, j1 = kClosureFields * nv + f * nv + k;
    double s = 0.0;
    for (int j = 0; j < nn; ++j) s += (double)a[nb[j]];
    x[(size_t)c * F + j0] = ((float)a[c] - mean[j0]) / std[j0];
    x[(size_t)c * F + j1] = ((float)(s / nn - (double)a[c]) - mean[j1]) / std[j1];
  }
}

// field += span (y * out_std + out_mean); the momentum correction is projected
// onto the tangent plane like every horizontal-momentum update
template <typename R>
__global__ void k_apply(Geo<R> G, Xf<R> X, const float* y, const float* omean, const float* ostd, float span) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (c >= G.ncol) return;
  const int S = G.colp, nv = G.nv, F = kClosureFields * nv;
  const size_t i = (size_t)k * S + c;
  float t[kClosureFields];
  for (int f = 0; f < kClosureFields; ++f) {
    const int j = f * nv + k;
    t[f] = y[(size_t)c * F + j] * ostd[j] + omean[j];
  }
  const float rx = (float)G.rhat[c], ry = (float)G.rhat[S + c], rz = (float)G.rhat[2 * S + c];
  const float d = t[1] * rx + t[2] * ry + t[3] * rz;
  t[1] -= d * rx;
  t[2] -= d * ry;
  t[3] -= d * rz;
  for (int f = 0; f < kClosureFields; ++f) {
    R* a = closure_field_rw(X, f);
    a[i] = a[i] + (R)(span * t[f]);
  }
}

// tau_hat = MLP(features of the current state), kept in the binding's y buffer
template <typename R>
int closure_evaluate_t(thor_state* s) {
  Impl<R>* I = static_cast<Impl<R>*>(s->impl.get());
  ClosureBinding& cb = s->closure;
  thor_mlp* net = cb.net;
  cudaStream_t st = I->stream;
  const int ncol = I->G.ncol, nv = I->G.nv;
  dim3 grid((ncol + 127) / 128, nv);
  k_features<R><<<grid, 128, 0, st>>>(I->G, I->Xt, cb.in_mean, cb.in_std, cb.x);
  const int Fin = 2 * kClosureFields * nv, Fout = kClosureFields * nv;
  for (int c0 = 0; c0 < ncol; c0 += net->max_batch) {
    const int m = std::min(net->max_batch, ncol - c0);
    int rc = mlp_forward(net, cb.x + (size_t)c0 * Fin, m, false);
    if (rc) return rc;
    if (cudaMemcpyAsync(cb.y + (size_t)c0 * Fout, net->y, (size_t)m * Fout * 4, cudaMemcpyDeviceToDevice, st))
      return THOR_ECUDA;
  }
  I->launches += 1 + 4 * ((ncol + net->max_batch - 1) / net->max_batch);
  return cudaGetLastError() == cudaSuccess ? THOR_OK : THOR_ECUDA;
}

template <typename R>
int closure_correct_t(thor_state* s, double span) {
  Impl<R>* I = static_cast<Impl<R>*>(s->impl.get());
  ClosureBinding& cb = s->closure;
  dim3 grid((I->G.ncol + 127) / 128, I->G.nv);
  k_apply<R><<<grid, 128, 0, I->stream>>>(I->G, I->Xt, cb.y, cb.out_mean, cb.out_std, (float)span);
  I->launches += 1;
  return cudaGetLastError() == cudaSuccess ? THOR_OK : THOR_ECUDA;
}

// One large step with the closure. The network sees the state at the start
// of each window of `period` large steps and its correction, period * dt *
// tau_hat, is added when the window closes: the coarse solution after n
// steps plus n dt tau, which is how the training target is defined.
template <typename R>
int closure_large_step_t(thor_state* s, int n_small, double dt) {
  ClosureBinding& cb = s->closure;
  int rc = THOR_OK;
  if (cb.counter % cb.period == 0) rc = closure_evaluate_t<R>(s);
  if (!rc) rc = s->impl->step(1, n_small, dt);
  if (rc) return rc;
  cb.counter += 1;
  if (cb.counter % cb.period == 0) rc = closure_correct_t<R>(s, cb.period * dt);
  return rc;
}

// fine -> coarse area-weighted averages (CSR over the fine columns of each
// coarse column, weights normalised per coarse column)
template <typename R>
__global__ void k_coarse_grain(Geo<R> Gc, Xf<R> Xf_, int Sf, Xf<R> Xc, const int* start, const int* member,
                               const double* weight) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;               // 0..nv (interfaces use all nv+1)
  if (c >= Gc.ncol) return;
  const int Sc = Gc.colp, nv = Gc.nv;
  double a[6] = {0, 0, 0, 0, 0, 0};
  for (int e = start[c]; e < start[c + 1]; ++e) {
    const size_t i = (size_t)k * Sf + member[e];
    const double w = weight[e];
    if (k < nv) {
      a[0] += w * (double)Xf_.rho[i];
      a[1] += w * (double)Xf_.mx[i];
      a[2] += w * (double)Xf_.my[i];
      a[3] += w * (double)Xf_.mz[i];
      a[4] += w * (double)Xf_.th[i];
    }
    a[5] += w * (double)Xf_.w[i];
  }
  const size_t o = (size_t)k * Sc + c;
  if (k < nv) {
    const double rx = Gc.rhat[c], ry = Gc.rhat[Sc + c], rz = Gc.rhat[2 * Sc + c];
    const double d = a[1] * rx + a[2] * ry + a[3] * rz;
    Xc.rho[o] = (R)a[0];
    Xc.mx[o] = (R)(a[1] - d * rx);
    Xc.my[o] = (R)(a[2] - d * ry);
    Xc.mz[o] = (R)(a[3] - d * rz);
    Xc.th[o] = (R)a[4];
  }
  Xc.w[o] = (k == 0 || k == nv) ? (R)0 : (R)a[5];
}

}  // namespace

int closure_large_step(thor_state* s, int n_small, double dt) {
  return s->precision == THOR_FP64 ? closure_large_step_t<double>(s, n_small, dt)
                                   : closure_large_step_t<float>(s, n_small, dt);
}

void closure_release(thor_state* s) {
  if (s->closure.x) cudaFree(s->closure.x);
  if (s->closure.y) cudaFree(s->closure.y);
  s->closure = ClosureBinding();
}

}  // namespace thor

namespace {
template <typename R>
int features_t(thor_state* s, const float* mean, const float* std, float* x) {
  using namespace thor;
  Impl<R>* I = static_cast<Impl<R>*>(s->impl.get());
  dim3 grid((I->G.ncol + 127) / 128, I->G.nv);
  k_features<R><<<grid, 128, 0, I->stream>>>(I->G, I->Xt, mean, std, x);
  I->launches += 1;
  return cudaGetLastError() == cudaSuccess ? THOR_OK : THOR_ECUDA;
}

template <typename R>
int coarse_t(thor_state* fine, thor_state* coarse, const std::vector<int>& start, const std::vector<int>& member,
             const std::vector<double>& weight) {
  using namespace thor;
  Impl<R>* F = static_cast<Impl<R>*>(fine->impl.get());
  Impl<R>* C = static_cast<Impl<R>*>(coarse->impl.get());
  cudaStream_t st = C->stream;
  int *d_start = nullptr, *d_member = nullptr;
  double* d_weight = nullptr;
  if (cudaMalloc(&d_start, start.size() * 4) || cudaMalloc(&d_member, member.size() * 4) ||
      cudaMalloc(&d_weight, weight.size() * 8)) {
    cudaFree(d_start);
    cudaFree(d_member);
    cudaFree(d_weight);
    return THOR_ENOMEM;
  }
  int rc = THOR_OK;
  if (cudaStreamSynchronize(F->stream) ||
      cudaMemcpyAsync(d_start, start.data(), start.size() * 4, cudaMemcpyHostToDevice, st) ||
      cudaMemcpyAsync(d_member, member.data(), member.size() * 4, cudaMemcpyHostToDevice, st) ||
      cudaMemcpyAsync(d_weight, weight.data(), weight.size() * 8, cudaMemcpyHostToDevice, st)) {
    rc = THOR_ECUDA;
  } else {
    dim3 grid((C->G.ncol + 127) / 128, C->G.nv + 1);
    // the coarse state's fields are replaced: a compensated one's low parts restart at zero
    if (C->lo_buf)
      cudaMemsetAsync(C->lo_buf, 0, (size_t)(6 * C->G.nv + 1) * C->G.colp * sizeof(R), st);
    k_coarse_grain<R><<<grid, 128, 0, st>>>(C->G, F->Xt, F->G.colp, C->Xt, d_start, d_member, d_weight);
    C->launches += 1;
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st)) rc = THOR_ECUDA;
  }
  cudaFree(d_start);
  cudaFree(d_member);
  cudaFree(d_weight);
  return rc;
}
}  // namespace

extern "C" {

int thor_closure_features(thor_state* s, const float* mean, const float* std, float* x) {
  if (!s || !mean || !std || !x) return THOR_EINVAL;
  return s->precision == THOR_FP64 ? features_t<double>(s, mean, std, x) : features_t<float>(s, mean, std, x);
}

int thor_closure_attach(thor_state* s, thor_mlp* net, const float* in_mean, const float* in_std,
                        const float* out_mean, const float* out_std, int period) {
  using namespace thor;
  if (!s) return THOR_EINVAL;
  closure_release(s);
  if (!net) return THOR_OK;                 // detached: plain method
  if (!in_mean || !in_std || !out_mean || !out_std || period < 1) return THOR_EINVAL;
  const int ncol = s->grid->h.ncol, nv = s->grid->h.nv;
  if (net->sizes.front() != 2 * kClosureFields * nv || net->sizes.back() != kClosureFields * nv)
    return THOR_EINVAL;
  ClosureBinding cb;
  cb.net = net;
  cb.in_mean = in_mean;
  cb.in_std = in_std;
  cb.out_mean = out_mean;
  cb.out_std = out_std;
  cb.period = period;
  if (cudaMalloc(&cb.x, (size_t)ncol * 2 * kClosureFields * nv * 4) ||
      cudaMalloc(&cb.y, (size_t)ncol * kClosureFields * nv * 4)) {
    if (cb.x) cudaFree(cb.x);
    return THOR_ENOMEM;
  }
  net->stream = s->impl->stream;            // the closure runs on the state's stream
  s->closure = cb;
  return THOR_OK;
}

int thor_coarse_grain(thor_state* fine, thor_state* coarse, const int* fine_to_coarse, size_t nfine) {
  if (!fine || !coarse || !fine_to_coarse || fine->precision != coarse->precision) return THOR_EINVAL;
  const thor::HostGrid& gf = fine->grid->h;
  const thor::HostGrid& gc = coarse->grid->h;
  if (nfine != (size_t)gf.ncol || gf.nv != gc.nv) return THOR_EINVAL;
  std::vector<int> count(gc.ncol + 1, 0);
  std::vector<double> asum(gc.ncol, 0.0);
  for (size_t f = 0; f < nfine; ++f) {
    const int c = fine_to_coarse[f];
    if (c < 0 || c >= gc.ncol) return THOR_EINVAL;
    count[c + 1]++;
    asum[c] += gf.area[f];
  }
  for (int c = 0; c < gc.ncol; ++c) {
    if (count[c + 1] == 0) return THOR_EINVAL;   // every coarse column needs fine members
    count[c + 1] += count[c];
  }
  std::vector<int> member(nfine), fill(count.begin(), count.end() - 1);
  std::vector<double> weight(nfine);
  for (size_t f = 0; f < nfine; ++f) {
    const int c = fine_to_coarse[f];
    member[fill[c]] = (int)f;
    weight[fill[c]] = gf.area[f] / asum[c];
    fill[c]++;
  }
  return fine->precision == THOR_FP64 ? coarse_t<double>(fine, coarse, count, member, weight)
                                      : coarse_t<float>(fine, coarse, count, member, weight);
}

}  // extern "C"
