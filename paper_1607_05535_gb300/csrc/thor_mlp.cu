// Learned per-column closure (an extension: the paper has no learned part).
//
// A dense MLP y = W_L^T relu(... relu(W_1^T x + b_1) ...) + b_L with float32
// master weights, bfloat16 weights and layer inputs on the tensor cores and
// float32 accumulation; trained with a mean-squared-error loss and Adam
// (Kingma and Ba 2015). The GEMMs run on the fifth-generation tensor cores:
// tcgen05.mma kind::f16 with bfloat16 operands staged in shared memory and
// the float32 accumulator in tensor memory (k_gemm_tc); the warp-level
// mma.sync m16n8k16 kernel (k_gemm_bf16) is kept as a switchable reference
// path (thor_mlp_tune).
//
// Closure: per column, the inputs are 5 fields (rho', M_x, M_y, M_z, Th') at
// all levels and the neighbour means of the same (as anomalies); the
// outputs are correction tendencies of the same 5 fields at all levels,
// added as field += dt * tendency after every large step. Training data come
// from high-resolution runs area-averaged onto the coarse grid
// (thor_coarse_grain).
#include <cuda_bf16.h>

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

// column sums of g [M][N] (deterministic: one thread per column, fixed order)
// out[n] = sum over m of g[m][n]: a block sums 32 columns, its 32 x 32
// threads each take every 32nd row, then the 32 partials of a column are
// added in a fixed order
__global__ void __launch_bounds__(1024) k_colsum(const float* g, int M, int N, float* out) {
  __shared__ float part[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, n = blockIdx.x * 32 + tx;
  float s = 0.0f;
  if (n < N) {
#pragma unroll 4
    for (int m = ty; m < M; m += 32) s += g[(size_t)m * N + n];
  }
  part[ty][tx] = s;
  __syncthreads();
  if (ty == 0 && n < N) {
    float t = 0.0f;
    for (int j = 0; j < 32; ++j) t += part[j][tx];
    out[n] = t;
  }
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

__global__ void k_sum_parts(const float* part, int n, float scale, float* out) {
  if (threadIdx.x || blockIdx.x) return;
  float s = 0.0f;
  for (int i = 0; i < n; ++i) s += part[i];
  *out = s * scale;
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
}  // namespace
}  // namespace thor

// ================================================================== MLP

struct thor_mlp {
  std::vector<int> sizes;              // layer widths, n_layers + 1 entries
  int use_tc = 1;                      // tcgen05 GEMMs (1) or the mma.sync reference path (0)
  int* err = nullptr;                  // device flag of the tcgen05 kernel
  int max_batch = 0;
  cudaStream_t stream = nullptr;
  size_t nparam = 0;
  std::vector<size_t> woff, boff;      // offsets of W_l and b_l in the flat parameter vector
  void* arena = nullptr;
  float *p = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;   // flat float32 [nparam]
  __nv_bfloat16* pb = nullptr;         // bf16 copy of all parameters (weights used)
  std::vector<__nv_bfloat16*> h;       // layer inputs (bf16) [max_batch][sizes[l]]
  std::vector<float*> z;               // hidden outputs / gradients (float32) [max_batch][sizes[l+1]]
  __nv_bfloat16* gb = nullptr;         // bf16 gradient scratch [max_batch][max width]
  float* y = nullptr;                  // network output [max_batch][n_out]
  float* dy = nullptr;                 // output gradient
  float* part = nullptr;               // reduction partials
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

// forward for m rows of x (float32 [m][n_in] on the device)
int mlp_forward(thor_mlp* net, const float* x, int m) {
  cudaStream_t st = net->stream;
  const int L = net->n_layers();
  k_to_bf16<<<blocks_for((size_t)m * net->sizes[0]), 256, 0, st>>>(x, net->h[0], (size_t)m * net->sizes[0]);
  for (int l = 0; l < L; ++l) {
    const int K = net->sizes[l], N = net->sizes[l + 1];
    const __nv_bfloat16* W = net->pb + net->woff[l];
    const float* b = net->p + net->boff[l];
    if (l + 1 < L)
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
  for (int l = L - 1; l >= 0; --l) {
    const int K = net->sizes[l], N = net->sizes[l + 1];
    float* gl = net->z[l];
    const size_t cnt = (size_t)m * N;
    // relu mask of this layer's output (hidden layers), then bf16 copy
    k_relu_back<<<blocks_for(cnt), 256, 0, st>>>(gl, l + 1 < L ? net->h[l + 1] : nullptr, net->gb, cnt,
                                                 l + 1 < L);
    // dW_l = h_l^T gb  ([K][N]), db_l = column sums of g
    gemm(net, K, N, m, net->h[l], K, 1, net->gb, N, 0, net->grad + net->woff[l], N, nullptr, 0, nullptr, 0);
    k_colsum<<<(N + 31) / 32, 1024, 0, st>>>(gl, m, N, net->grad + net->boff[l]);
    if (l > 0) {
      // g_{l-1} = gb W_l^T ([m][K]) into z[l-1]
      const __nv_bfloat16* W = net->pb + net->woff[l];
      gemm(net, m, K, N, net->gb, N, 0, W, N, 1, net->z[l - 1], K, nullptr, 0, nullptr, 0);
    }
  }
  return cudaGetLastError() == cudaSuccess ? THOR_OK : THOR_ECUDA;
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
  // one arena: params, grads, Adam moments, bf16 params, activations
  size_t bytes = 0;
  auto take = [&](size_t b) { size_t o = bytes; bytes += (b + 255) / 256 * 256; return o; };
  size_t o_p = take(net->nparam * 4), o_g = take(net->nparam * 4), o_m = take(net->nparam * 4),
         o_v = take(net->nparam * 4), o_pb = take(net->nparam * 2);
  std::vector<size_t> o_h, o_z;
  for (int l = 0; l < L; ++l) o_h.push_back(take((size_t)max_batch * sizes[l] * 2));
  for (int l = 0; l < L; ++l) o_z.push_back(take((size_t)max_batch * sizes[l + 1] * 4));
  size_t o_gb = take((size_t)max_batch * wmax * 2), o_y = take((size_t)max_batch * sizes[L] * 4),
         o_dy = take((size_t)max_batch * sizes[L] * 4), o_part = take(4096 * 4 + 64), o_err = take(64);
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
  if (cudaMemsetAsync(net->err, 0, 64, net->stream) ||
      cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024)) {
    cudaFree(net->arena);
    delete net;
    return THOR_ECUDA;
  }
  net->dy = (float*)(base + o_dy);
  net->part = (float*)(base + o_part);
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
    net->use_tc = value != 0;
    return THOR_OK;
  }
  return THOR_EINVAL;
}

int thor_mlp_set_params(thor_mlp* net, const float* host, size_t n) {
  using namespace thor;
  if (!net || !host || n != net->nparam) return THOR_EINVAL;
  if (cudaMemcpyAsync(net->p, host, n * 4, cudaMemcpyHostToDevice, net->stream)) return THOR_ECUDA;
  k_to_bf16<<<blocks_for(n), 256, 0, net->stream>>>(net->p, net->pb, n);
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
  if (loss) k_sum_parts<<<1, 32, 0, st>>>(net->part, nb, 1.0f / (float)cnt, loss);
  rc = mlp_backward(net, net->dy, m);
  if (rc) return rc;
  net->step_count += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)net->step_count), c2 = 1.0f - powf(b2, (float)net->step_count);
  k_adam<<<blocks_for(net->nparam), 256, 0, st>>>(net->p, net->grad, net->m, net->v, net->pb, net->nparam, lr,
                                                  b1, b2, c1, c2, 1e-8f);
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
    int rc = mlp_forward(net, cb.x + (size_t)c0 * Fin, m);
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
