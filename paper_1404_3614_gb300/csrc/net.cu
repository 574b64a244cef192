// Learned CG warm start: a 2D or 3D Fourier-layer network (lift, L spectral layers,
// projection) trained and run with a BF16 tensor-core GEMM (tcgen05.mma, FP32 accumulation
// in tensor memory).
//
// Every operation is a GEMM or an elementwise kernel:
//   spectral layer  s = E_x [ H_y ( R_k ( G_y ( F_x v ) ) ) ]   (truncated DFTs as GEMMs
//                   against DFT bases, per-mode complex channel mixing R_k; in 3D a
//                   G_z / H_z pair sits inside G_y / H_y), then
//   z = s + v W + b, v' = GELU(z) (no activation after the last layer);
//   lift v0 = x W_l + b_l, projection out = GELU(v_L P1 + b1) P2 + b2.
// The network output is a real field on the N grid; its DFT, projected by Gamma^E /
// Gamma^J inside the solver, is a conforming starting field, so the bounds stay
// guaranteed whatever the network predicts (Lemma bounds; Krylov iterates stay in E_N,
// the remark after Eq. linear_system_dual).
#include <cuda_bf16.h>
#include <math.h>

#include <cmath>
#include <vector>

#include "attr.cuh"
#include "net.cuh"

namespace homb {

// ---------------------------------------------------------------------------------
// BF16 tensor-core GEMM on the 5th-generation tensor cores (tcgen05.mma, FP32 accumulators
// in tensor memory)
//
// One CTA of 128 threads computes a 128 x 64 tile of C. Per K chunk of 64, all threads read
// the FP32 operands, round them to BF16 and store them in shared memory in the canonical
// K-major, non-swizzled layout: 8-row x 16-byte core matrices, the M (or N) groups of a
// core column 128 bytes apart, the K core columns 16 (or 8) core matrices apart. One thread
// then issues four tcgen05.mma (K = 16 each) into a 128-lane x 64-column FP32 accumulator in
// tensor memory and commits them to an mbarrier; the CTA waits on it (bounded) before the
// next chunk overwrites the tiles. The epilogue reads the accumulator with tcgen05.ld
// (warp w owns lanes 32w..32w+31 = rows) and applies alpha / beta, or writes split-K partials.
// ---------------------------------------------------------------------------------
constexpr int TBM = 128, TBN = 64, TBK = 64;
constexpr int kTmemCols = 64;                       // power of two >= 32
constexpr int kTileABytes = TBM * TBK * 2, kTileBBytes = TBN * TBK * 2;
// 26 KB of dynamic shared memory: at most 8 CTAs per SM (228 KB), 8 x 64 = 512 TMEM columns,
// so an allocation never waits on a CTA that is not running
constexpr int kGemmSmem = 26 * 1024;
static_assert(kTileABytes + kTileBBytes + 16 <= kGemmSmem, "GEMM tiles exceed the shared-memory request");
static_assert(TBM * 36 * 4 <= kTileABytes + kTileBBytes, "the result staging must fit in the operand tiles");
static_assert(TBN % 32 == 0, "the staged epilogue works in 32-column halves");
constexpr long long kMbarSpinLimit = 1LL << 22;

__device__ int g_gemm_timeout[kGemmFlagSlots];   // per context: set when an mbarrier wait gave up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start address, leading (K-direction core) and stride
// (M/N-direction core) byte offsets, fixed 0b001 at bits 46-48, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor, kind::f16: D F32, A and B BF16, both K-major, N >> 3, M >> 4
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// Bounded wait for the phase `phase` of an mbarrier: at most `limit` polls. A limit below
// the default uses the non-blocking test (a test aid: the wait then gives up at once);
// otherwise the potentially blocking try_wait.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase, long long limit = kMbarSpinLimit) {
  const bool quick = limit < kMbarSpinLimit;
  for (long long it = 0; it < limit; ++it) {
    uint32_t done;
    if (quick)
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(mbar), "r"(phase)
          : "memory");
    else
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(mbar), "r"(phase)
          : "memory");
    if (done) return true;
  }
  return false;
}

__global__ void __launch_bounds__(128) k_gemm(GemmArgs g, int ksplit, float* partial) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;                                 // [TBK/8][TBM/8][8][16 B]
  unsigned char* sB = smem + kTileABytes;                   // [TBK/8][TBN/8][8][16 B]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + kTileABytes + kTileBBytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int bz = blockIdx.z / ksplit;
  const int ks = blockIdx.z - bz * ksplit;
  const float* A = g.A + (long long)bz * g.sA;
  const float* B = g.B + (long long)bz * g.sB;
  const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
  const int kchunk = ((g.K + ksplit - 1) / ksplit + TBK - 1) / TBK * TBK;
  const int kbeg = ks * kchunk;
  const int kend = min(g.K, kbeg + kchunk);
  const uint32_t mbar_a = smem_u32(mbar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar_a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = mma_idesc(TBM, TBN);
  uint32_t phase = 0;
  bool ok = true;
  for (int k0 = kbeg; k0 < kend && ok; k0 += TBK) {
    // A tile: 8-element K runs of one row per store (16 bytes = one core-matrix row)
    for (int c = tid; c < TBM * (TBK / 8); c += 128) {
      int r, kc;
      if (!g.ta) { r = c >> 3; kc = c & 7; }
      else { r = c & (TBM - 1); kc = c / TBM; }
      const int gm = m0 + r;
      float v[8];
      const int gk0 = k0 + kc * 8;
      if (g.vecA && gm < g.M && gk0 + 8 <= kend) {   // two 16-byte loads along K
        const float4* p = reinterpret_cast<const float4*>(A + (long long)gm * g.lda + gk0);
        const float4 lo = __ldg(p), hi = __ldg(p + 1);
        v[0] = lo.x; v[1] = lo.y; v[2] = lo.z; v[3] = lo.w; v[4] = hi.x; v[5] = hi.y; v[6] = hi.z; v[7] = hi.w;
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int gk = gk0 + j;
          v[j] = 0.f;
          if (gm < g.M && gk < kend) v[j] = g.ta ? A[(long long)gk * g.lda + gm] : A[(long long)gm * g.lda + gk];
        }
      }
      const uint4 q = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                                 pack_bf16(v[6], v[7]));
      *reinterpret_cast<uint4*>(sA + ((kc * (TBM / 8) + (r >> 3)) * 8 + (r & 7)) * 16) = q;
    }
    // B tile, stored N x K (K-major)
    for (int c = tid; c < TBN * (TBK / 8); c += 128) {
      int n, kc;
      if (g.tb) { n = c >> 3; kc = c & 7; }
      else { n = c & (TBN - 1); kc = c / TBN; }
      const int gn = n0 + n;
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int gk = k0 + kc * 8 + j;
        v[j] = 0.f;
        if (gn < g.N && gk < kend) v[j] = g.tb ? B[(long long)gn * g.ldb + gk] : B[(long long)gk * g.ldb + gn];
      }
      const uint4 q = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                                 pack_bf16(v[6], v[7]));
      *reinterpret_cast<uint4*>(sB + ((kc * (TBN / 8) + (n >> 3)) * 8 + (n & 7)) * 16) = q;
    }
    // make the generic-proxy stores visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int s = 0; s < TBK / 16; ++s) {
        const uint64_t ad = smem_desc(smem_u32(sA) + s * 2 * (TBM / 8) * 128, (TBM / 8) * 128, 128);
        const uint64_t bd = smem_desc(smem_u32(sB) + s * 2 * (TBN / 8) * 128, (TBN / 8) * 128, 128);
        const uint32_t acc = (k0 > kbeg || s > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_a)
                   : "memory");
    }
    ok = __syncthreads_and(mbar_wait(mbar_a, phase, g.spin) ? 1 : 0) != 0;   // one verdict for the CTA
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (!ok) {
    // drain: wait (with the default bound, whatever the first limit was) for the committed
    // MMAs before the accumulator is freed
    if (tid == 0) atomicExch(&g_gemm_timeout[g.slot], 1);
    mbar_wait(mbar_a, phase ^ 1u);
  } else if (ksplit == 1 && g.vecC) {
    // epilogue through shared memory (the operand tiles are free: the MMAs have completed):
    // per 32-column half, each warp writes its 32 accumulator rows, then the CTA stores whole
    // 128-byte row segments (8 threads per row, 16-byte accesses); row stride 36 floats keeps
    // both phases free of bank conflicts
    const bool have = kend > kbeg;
    float* Cs = reinterpret_cast<float*>(smem);
    const int lrow = warp * 32 + lane;
    for (int h = 0; h < TBN / 32; ++h) {
#pragma unroll
      for (int c = 0; c < 32; c += 16) {
        uint32_t r[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) r[j] = 0u;
        if (have) asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(h * 32 + c)));
        if (have) asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float4* dst = reinterpret_cast<float4*>(Cs + lrow * 36 + c);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          dst[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                               __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
      }
      __syncthreads();
      for (int idx = tid; idx < TBM * 8; idx += 128) {
        const int rr = idx >> 3, q = idx & 7;
        const int row = m0 + rr, col = n0 + h * 32 + 4 * q;
        if (row >= g.M || col >= g.N) continue;
        const float4 v = *reinterpret_cast<const float4*>(Cs + rr * 36 + 4 * q);
        float* C = g.C + (long long)bz * g.sC + (long long)row * g.ldc + col;
        if (col + 4 <= g.N) {
          float4 o = make_float4(g.alpha * v.x, g.alpha * v.y, g.alpha * v.z, g.alpha * v.w);
          if (g.beta != 0.f) {
            const float4 c4 = *reinterpret_cast<const float4*>(C);
            o.x += g.beta * c4.x; o.y += g.beta * c4.y; o.z += g.beta * c4.z; o.w += g.beta * c4.w;
          }
          *reinterpret_cast<float4*>(C) = o;
        } else {
          const float vv[4] = {v.x, v.y, v.z, v.w};
          for (int e = 0; e < 4 && col + e < g.N; ++e)
            C[e] = g.beta == 0.f ? g.alpha * vv[e] : g.alpha * vv[e] + g.beta * C[e];
        }
      }
      __syncthreads();
    }
  } else {
    // epilogue: warp w reads rows 32w + lane, 16 columns per tcgen05.ld (zeros when this
    // split has no K range: nothing was accumulated)
    const bool have = kend > kbeg;
    const int row = m0 + warp * 32 + lane;
#pragma unroll
    for (int c0 = 0; c0 < TBN; c0 += 16) {
      uint32_t r[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) r[j] = 0u;
      if (have) asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
      if (have) asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < g.M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = n0 + c0 + j;
          if (col >= g.N) continue;
          const float v = __uint_as_float(r[j]);
          if (ksplit == 1) {
            float* C = g.C + (long long)bz * g.sC + (long long)row * g.ldc + col;
            *C = g.beta == 0.f ? g.alpha * v : g.alpha * v + g.beta * *C;
          } else {
            partial[(((long long)ks * g.batch + bz) * g.M + row) * g.N + col] = v;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

__global__ void k_gemm_reduce(GemmArgs g, int ksplit, const float* partial) {
  const long long per = (long long)g.M * g.N;
  const long long total = per * g.batch;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < ksplit; ++k) s += partial[(long long)k * total + i];
    const int bz = (int)(i / per);
    const long long rc = i - bz * per;
    const int row = (int)(rc / g.N), col = (int)(rc - (long long)row * g.N);
    float* C = g.C + (long long)bz * g.sC + (long long)row * g.ldc + col;
    *C = g.beta == 0.f ? g.alpha * s : g.alpha * s + g.beta * *C;
  }
}

static thread_local int g_ctx_slot = 0;
static thread_local long long g_ctx_spin = 0;

void gemm_set_context(int slot, long long spin) {
  g_ctx_slot = ((slot % kGemmFlagSlots) + kGemmFlagSlots) % kGemmFlagSlots;
  g_ctx_spin = spin;
}

cudaError_t gemm_timeout_clear(int slot, cudaStream_t s) {
  int* base = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void**)&base, g_gemm_timeout);
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(base + (slot % kGemmFlagSlots), 0, sizeof(int), s);
}

cudaError_t gemm_timeout_read(int slot, int* host_flag, cudaStream_t s) {
  int* base = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void**)&base, g_gemm_timeout);
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(host_flag, base + (slot % kGemmFlagSlots), sizeof(int), cudaMemcpyDeviceToHost, s);
}

// split-K scratch, owned by the caller through net_workspace: set per call
static thread_local float* g_split_ws = nullptr;
static thread_local long long g_split_floats = 0;

cudaError_t gemm_bf16(const GemmArgs& g0, cudaStream_t s) {
  if (g0.M <= 0 || g0.N <= 0 || g0.batch <= 0) return cudaSuccess;
  GemmArgs g = g0;
  g.slot = g_ctx_slot;
  g.spin = g_ctx_spin > 0 ? g_ctx_spin : kMbarSpinLimit;
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  g.vecA = !g.ta && g.lda % 4 == 0 && g.sA % 4 == 0 && al16(g.A);
  g.vecC = g.ldc % 4 == 0 && g.sC % 4 == 0 && al16(g.C);
  if ((g.M + TBM - 1) / TBM > 65535) {   // grid y is limited to 65535 tiles: chunks of rows
    const int rows = 65535 * TBM;
    for (int r0 = 0; r0 < g.M; r0 += rows) {
      GemmArgs h = g;
      h.M = std::min(rows, g.M - r0);
      h.A = g.ta ? g.A + r0 : g.A + (long long)r0 * g.lda;
      h.C = g.C + (long long)r0 * g.ldc;
      const cudaError_t e = gemm_bf16(h, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  const int gm = (g.M + TBM - 1) / TBM, gn = (g.N + TBN - 1) / TBN;
  int ksplit = 1;
  const long long tiles = (long long)gm * gn * g.batch;
  if (tiles < 152 && g.K > 2048 && g_split_ws) {
    ksplit = (int)std::min<long long>(256, std::max<long long>(1, (304 + tiles - 1) / tiles));
    ksplit = std::min(ksplit, (g.K + 1023) / 1024);
    while (ksplit > 1 && (long long)ksplit * g.M * g.N * g.batch > g_split_floats) --ksplit;
  }
  if (ksplit == 1 && g.batch > 65535) {   // grid z is limited to 65535: chunks of batches
    for (int b0 = 0; b0 < g.batch; b0 += 65535) {
      GemmArgs h = g;
      h.batch = std::min(65535, g.batch - b0);
      h.A = g.A + (long long)b0 * g.sA;
      h.B = g.B + (long long)b0 * g.sB;
      h.C = g.C + (long long)b0 * g.sC;
      k_gemm<<<dim3(gn, gm, h.batch), 128, kGemmSmem, s>>>(h, 1, nullptr);
    }
    return cudaGetLastError();
  }
  dim3 grid(gn, gm, g.batch * ksplit);
  k_gemm<<<grid, 128, kGemmSmem, s>>>(g, ksplit, g_split_ws);
  if (ksplit > 1) {
    const long long total = (long long)g.M * g.N * g.batch;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 8);
    k_gemm_reduce<<<blocks, 256, 0, s>>>(g, ksplit, g_split_ws);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// elementwise kernels
// ---------------------------------------------------------------------------------
__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// z += b (per column); v = act(z)
__global__ void k_bias_act(float* z, const float* b, float* v, long long rows, int cols, int act) {
  const long long n = rows * cols;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float t = z[i] + b[i % cols];
    z[i] = t;
    v[i] = act ? gelu(t) : t;
  }
}

__global__ void k_gelu_back(const float* dv, const float* z, float* dz, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dz[i] = dv[i] * gelu_d(z[i]);
}

// deterministic column sums: stage 1 per row block, stage 2 over blocks
__global__ void k_colsum1(const float* x, long long rows, int cols, int rows_per, float* part) {
  const long long r0 = (long long)blockIdx.x * rows_per;
  const long long r1 = min(rows, r0 + rows_per);
  for (int c = threadIdx.x; c < cols; c += blockDim.x) {
    float s = 0.f;
    for (long long r = r0; r < r1; ++r) s += x[r * cols + c];
    part[(long long)blockIdx.x * cols + c] = s;
  }
}
__global__ void k_colsum2(const float* part, int nblk, int cols, float* out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += part[(long long)b * cols + c];
    out[c] = s;
  }
}

__global__ void k_mse(const float* out, const float* t, float* dout, long long n, float* part) {
  __shared__ float red[32];
  float acc = 0.f;
  const float sc = 2.f / (float)n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float d = out[i] - t[i];
    acc += d * d;
    dout[i] = sc * d;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}
__global__ void k_mse_final(const float* part, int nblk, long long n, float* loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[b];
    *loss = (float)(s / (double)n);
  }
}

__global__ void k_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// deterministic uniform numbers from a counter hash (SplitMix64 finaliser)
__device__ __forceinline__ float hash_uniform(unsigned long long seed, long long i) {
  unsigned long long z = seed + 0x9E3779B97F4A7C15ULL * (unsigned long long)(i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return (float)((z >> 40) * (1.0 / 16777216.0));   // [0, 1)
}
__global__ void k_init(float* p, long long n, float lo, float hi, unsigned long long seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = lo + (hi - lo) * hash_uniform(seed, i);
}
__global__ void k_fill(float* p, long long n, float v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = v;
}

static int eblocks(long long n) { return (int)std::min<long long>((n + 255) / 256, 152 * 16); }

// ---------------------------------------------------------------------------------
// layout
// ---------------------------------------------------------------------------------
// kept modes of one spectral layer: K1^(d-1) * K
static long long spectral_modes(const NetConfig& c) {
  const long long K1 = 2 * c.modes;
  return (c.d == 3 ? K1 * K1 : K1) * c.modes;
}
static long long ipow(long long b, int e) {
  long long r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

NetOffsets net_offsets(const NetConfig& c) {
  NetOffsets o{};
  long long off = 0;
  auto take = [&](long long n) { const long long r = off; off += n; return r; };
  o.lift_w = take((long long)c.cin * c.width);
  o.lift_b = take(c.width);
  for (int l = 0; l < c.layers; ++l) {
    o.R[l] = take(2LL * spectral_modes(c) * c.width * c.width);
    o.W[l] = take((long long)c.width * c.width);
    o.b[l] = take(c.width);
  }
  o.p1_w = take((long long)c.width * c.proj);
  o.p1_b = take(c.proj);
  o.p2_w = take((long long)c.proj * c.cout);
  o.p2_b = take(c.cout);
  o.total = off;
  return o;
}

long long bases_floats(const NetConfig& c) {
  const long long N = c.N, K = c.modes, K1 = 2 * c.modes;
  return 2 * K * N + 2 * K1 * N + 2 * N * K1 + 2 * N * K;
}

// Fr, Fi [K x N]: e^{-2 pi i kx x / N}; Gc, Gs [K1 x N]: cos, sin of 2 pi ky y / N (ky in
// 0..K-1, -K..-1); Hc, Hs [N x K1]: cos, sin of 2 pi ky y / N; Er, Ei [N x K]: the
// half-spectrum inverse along x with weights c_kx (1, then 2) and 1/N^d. The z axis of the
// 3D network uses the y bases (cubic grid).
void fill_bases(const NetConfig& c, float* h) {
  const int N = c.N, K = c.modes, K1 = 2 * c.modes;
  const double tp = 6.283185307179586476925286766559;
  float* Fr = h;
  float* Fi = Fr + (long long)K * N;
  float* Gc = Fi + (long long)K * N;
  float* Gs = Gc + (long long)K1 * N;
  float* Hc = Gs + (long long)K1 * N;
  float* Hs = Hc + (long long)N * K1;
  float* Er = Hs + (long long)N * K1;
  float* Ei = Er + (long long)N * K;
  auto ky_of = [&](int i) { return i < K ? i : i - K1; };
  for (int k = 0; k < K; ++k)
    for (int x = 0; x < N; ++x) {
      const double a = tp * k * x / N;
      Fr[k * N + x] = (float)std::cos(a);
      Fi[k * N + x] = (float)-std::sin(a);
      const double w = (k == 0 ? 1.0 : 2.0) / (double)ipow(N, c.d == 3 ? 3 : 2);
      Er[x * K + k] = (float)(w * std::cos(a));
      Ei[x * K + k] = (float)(-w * std::sin(a));
    }
  for (int i = 0; i < K1; ++i)
    for (int y = 0; y < N; ++y) {
      const double a = tp * ky_of(i) * y / N;
      Gc[i * N + y] = (float)std::cos(a);
      Gs[i * N + y] = (float)std::sin(a);
      Hc[y * K1 + i] = (float)std::cos(a);
      Hs[y * K1 + i] = (float)std::sin(a);
    }
}

// Activations: v, z [P x W] per layer (P = B N^d grid points); x1 / z1 after the x DFT
// [B][(z)][y][kx][W]; mr / mi (3D) after the y DFT [B][z][ky][kx][W]; x2[l] the kept
// spectrum of layer l [B][(kz)][ky][kx][W] (saved for the weight gradient), y the mixed one.
struct NetWs {
  float *v[9], *z[8], *x1r, *x1i, *x2r[8], *x2i[8], *yr, *yi, *z1r, *z1i, *mr, *mi, *pz, *ph;
  float *dv, *dz, *dx1r, *dx1i, *dx2r, *dx2i, *dyr, *dyi, *dz1r, *dz1i, *dmr, *dmi, *dh, *colpart, *lpart, *split;
  long long split_floats;
};

// Carves the workspace; returns the number of floats used (pointers set when ws != null).
static long long carve_n(const NetConfig& c, int B, float* ws, NetWs& w) {
  w = NetWs{};
  const int d = c.d == 3 ? 3 : 2;
  const long long P = (long long)B * ipow(c.N, d), W = c.width, K = c.modes, K1 = 2 * c.modes;
  const long long x1 = (long long)B * ipow(c.N, d - 1) * K * W, x2 = (long long)B * spectral_modes(c) * W;
  const long long xm = d == 3 ? (long long)B * c.N * K1 * K * W : 0;
  long long off = 0;
  auto take = [&](long long n) {
    float* r = ws ? ws + off : nullptr;
    off += (n + 63) & ~63LL;
    return r;
  };
  for (int l = 0; l <= c.layers; ++l) w.v[l] = take(P * W);
  for (int l = 0; l < c.layers; ++l) w.z[l] = take(P * W);
  w.x1r = take(x1); w.x1i = take(x1);
  for (int l = 0; l < c.layers; ++l) { w.x2r[l] = take(x2); w.x2i[l] = take(x2); }
  w.yr = take(x2); w.yi = take(x2); w.z1r = take(x1); w.z1i = take(x1);
  if (xm) { w.mr = take(xm); w.mi = take(xm); }
  w.pz = take(P * c.proj); w.ph = take(P * c.proj);
  w.dv = take(P * W); w.dz = take(P * W);
  w.dx1r = take(x1); w.dx1i = take(x1); w.dx2r = take(x2); w.dx2i = take(x2);
  w.dyr = take(x2); w.dyi = take(x2); w.dz1r = take(x1); w.dz1i = take(x1);
  if (xm) { w.dmr = take(xm); w.dmi = take(xm); }
  w.dh = take(P * c.proj);
  w.colpart = take(1024LL * std::max<long long>(c.proj, W));
  w.lpart = take(4096);
  w.split_floats = 4LL * 1024 * 1024;
  w.split = take(w.split_floats);
  return off;
}

static NetWs carve(const NetConfig& c, int B, float* ws) {
  NetWs w;
  carve_n(c, B, ws, w);
  return w;
}

long long net_workspace_floats(const NetConfig& c, int B) {
  NetWs w;
  return carve_n(c, B, nullptr, w);
}

static GemmArgs gemm(const float* A, const float* B, float* C, int M, int N, int K, int lda, int ldb, int ldc,
                     int ta, int tb, long long sA, long long sB, long long sC, int batch, float alpha, float beta) {
  GemmArgs g;
  g.A = A; g.B = B; g.C = C; g.M = M; g.N = N; g.K = K; g.lda = lda; g.ldb = ldb; g.ldc = ldc;
  g.ta = ta; g.tb = tb; g.sA = sA; g.sB = sB; g.sC = sC; g.batch = batch; g.alpha = alpha; g.beta = beta;
  return g;
}

#define NCK(x)                                \
  do {                                        \
    cudaError_t _e = (x);                     \
    if (_e != cudaSuccess) return _e;         \
  } while (0)

static cudaError_t colsum(const float* x, long long rows, int cols, float* out, float* part, cudaStream_t s) {
  const int nblk = (int)std::min<long long>(1024, std::max<long long>(1, rows / 256));
  const int rows_per = (int)((rows + nblk - 1) / nblk);
  k_colsum1<<<nblk, 128, 0, s>>>(x, rows, cols, rows_per, part);
  k_colsum2<<<(cols + 127) / 128, 128, 0, s>>>(part, nblk, cols, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// forward / backward
// ---------------------------------------------------------------------------------
struct Bases {
  const float *Fr, *Fi, *Gc, *Gs, *Hc, *Hs, *Er, *Ei;
};
static Bases bases_of(const NetConfig& c, const float* b) {
  const long long N = c.N, K = c.modes, K1 = 2 * c.modes;
  Bases r;
  r.Fr = b; r.Fi = r.Fr + K * N; r.Gc = r.Fi + K * N; r.Gs = r.Gc + K1 * N;
  r.Hc = r.Gs + K1 * N; r.Hs = r.Hc + N * K1; r.Er = r.Hs + N * K1; r.Ei = r.Er + N * K;
  return r;
}

// Complex DFT along one axis on the kept modes, as four real GEMMs per batch item, with
// bases Gc, Gs [K1 x Nn] and Hc, Hs [Nn x K1]; C columns per row, batch strides in floats.
//   forward  O = G I:  Or = Gc Ir + Gs Ii,  Oi = Gc Ii - Gs Ir   (e^{-2 pi i k y / N})
//   inverse  O = H I:  Or = Hc Ir - Hs Ii,  Oi = Hc Ii + Hs Ir   (e^{+2 pi i k y / N})
struct Axis {
  const Bases& bs;
  int Nn, K1;
  cudaStream_t s;
  cudaError_t fwd(const float* ir, const float* ii, float* orr, float* oi, int C, long long sI, long long sO,
                  int batch) const {
    NCK(gemm_bf16(gemm(bs.Gc, ir, orr, K1, C, Nn, Nn, C, C, 0, 0, 0, sI, sO, batch, 1.f, 0.f), s));
    NCK(gemm_bf16(gemm(bs.Gs, ii, orr, K1, C, Nn, Nn, C, C, 0, 0, 0, sI, sO, batch, 1.f, 1.f), s));
    NCK(gemm_bf16(gemm(bs.Gc, ii, oi, K1, C, Nn, Nn, C, C, 0, 0, 0, sI, sO, batch, 1.f, 0.f), s));
    return gemm_bf16(gemm(bs.Gs, ir, oi, K1, C, Nn, Nn, C, C, 0, 0, 0, sI, sO, batch, -1.f, 1.f), s);
  }
  cudaError_t inv(const float* ir, const float* ii, float* orr, float* oi, int C, long long sI, long long sO,
                  int batch) const {
    NCK(gemm_bf16(gemm(bs.Hc, ir, orr, Nn, C, K1, K1, C, C, 0, 0, 0, sI, sO, batch, 1.f, 0.f), s));
    NCK(gemm_bf16(gemm(bs.Hs, ii, orr, Nn, C, K1, K1, C, C, 0, 0, 0, sI, sO, batch, -1.f, 1.f), s));
    NCK(gemm_bf16(gemm(bs.Hc, ii, oi, Nn, C, K1, K1, C, C, 0, 0, 0, sI, sO, batch, 1.f, 0.f), s));
    return gemm_bf16(gemm(bs.Hs, ir, oi, Nn, C, K1, K1, C, C, 0, 0, 0, sI, sO, batch, 1.f, 1.f), s);
  }
  // adjoints: dI = G^T dO (of fwd), dI = H^T dO (of inv); dO has stride sO, dI stride sI
  cudaError_t fwd_adj(const float* dor, const float* doi, float* dir, float* dii, int C, long long sO,
                      long long sI, int batch) const {
    NCK(gemm_bf16(gemm(bs.Gc, dor, dir, Nn, C, K1, Nn, C, C, 1, 0, 0, sO, sI, batch, 1.f, 0.f), s));
    NCK(gemm_bf16(gemm(bs.Gs, doi, dir, Nn, C, K1, Nn, C, C, 1, 0, 0, sO, sI, batch, -1.f, 1.f), s));
    NCK(gemm_bf16(gemm(bs.Gs, dor, dii, Nn, C, K1, Nn, C, C, 1, 0, 0, sO, sI, batch, 1.f, 0.f), s));
    return gemm_bf16(gemm(bs.Gc, doi, dii, Nn, C, K1, Nn, C, C, 1, 0, 0, sO, sI, batch, 1.f, 1.f), s);
  }
  cudaError_t inv_adj(const float* dor, const float* doi, float* dir, float* dii, int C, long long sO,
                      long long sI, int batch) const {
    NCK(gemm_bf16(gemm(bs.Hc, dor, dir, K1, C, Nn, K1, C, C, 1, 0, 0, sO, sI, batch, 1.f, 0.f), s));
    NCK(gemm_bf16(gemm(bs.Hs, doi, dir, K1, C, Nn, K1, C, C, 1, 0, 0, sO, sI, batch, 1.f, 1.f), s));
    NCK(gemm_bf16(gemm(bs.Hc, doi, dii, K1, C, Nn, K1, C, C, 1, 0, 0, sO, sI, batch, 1.f, 0.f), s));
    return gemm_bf16(gemm(bs.Hs, dor, dii, K1, C, Nn, K1, C, C, 1, 0, 0, sO, sI, batch, -1.f, 1.f), s);
  }
};

cudaError_t net_forward(const NetConfig& c, const float* prm, const float* bases, int B, const float* in, float* out,
                        float* ws, int train, cudaStream_t s) {
  (void)train;
  const NetOffsets o = net_offsets(c);
  NetWs w = carve(c, B, ws);
  g_split_ws = w.split;
  g_split_floats = w.split_floats;
  const Bases bs = bases_of(c, bases);
  const Axis ax{bs, c.N, 2 * c.modes, s};
  const int d = c.d == 3 ? 3 : 2;
  const int N = c.N, W = c.width, K = c.modes, K1 = 2 * c.modes, KW = K * W;
  const long long P = (long long)B * ipow(N, d);
  const int BN = (int)(B * ipow(N, d - 1));   // rows of x transforms: (b, (z,) y)
  const long long nmodes = spectral_modes(c);
  // lift
  NCK(gemm_bf16(gemm(in, prm + o.lift_w, w.v[0], (int)P, W, c.cin, c.cin, W, W, 0, 0, 0, 0, 0, 1, 1.f, 0.f), s));
  k_bias_act<<<eblocks(P * W), 256, 0, s>>>(w.v[0], prm + o.lift_b, w.v[0], P, W, 0);
  for (int l = 0; l < c.layers; ++l) {
    const float* v = w.v[l];
    const float* Rr = prm + o.R[l];
    const float* Ri = Rr + nmodes * W * W;
    // (1) x DFT, per (b, (z,) y): [K x N] x [N x W]
    NCK(gemm_bf16(gemm(bs.Fr, v, w.x1r, K, W, N, N, W, W, 0, 0, 0, (long long)N * W, (long long)K * W, BN, 1.f, 0.f), s));
    NCK(gemm_bf16(gemm(bs.Fi, v, w.x1i, K, W, N, N, W, W, 0, 0, 0, (long long)N * W, (long long)K * W, BN, 1.f, 0.f), s));
    // (2) y DFT per (b, (z)): [K1 x N] x [N x KW]; (2z) z DFT per b: [K1 x N] x [N x K1 KW]
    const long long sx1 = (long long)N * KW, sx2 = (long long)K1 * KW;
    if (d == 2) {
      NCK(ax.fwd(w.x1r, w.x1i, w.x2r[l], w.x2i[l], KW, sx1, sx2, B));
    } else {
      NCK(ax.fwd(w.x1r, w.x1i, w.mr, w.mi, KW, sx1, sx2, B * N));
      NCK(ax.fwd(w.mr, w.mi, w.x2r[l], w.x2i[l], K1 * KW, (long long)N * K1 * KW, (long long)K1 * K1 * KW, B));
    }
    // (3) per mode m: Y = X2 R (complex), rows b (stride nmodes*W), batch over modes
    const int nm = (int)nmodes;
    const int ldm = nm * W;
    NCK(gemm_bf16(gemm(w.x2r[l], Rr, w.yr, B, W, W, ldm, W, ldm, 0, 0, W, (long long)W * W, W, nm, 1.f, 0.f), s));
    NCK(gemm_bf16(gemm(w.x2i[l], Ri, w.yr, B, W, W, ldm, W, ldm, 0, 0, W, (long long)W * W, W, nm, -1.f, 1.f), s));
    NCK(gemm_bf16(gemm(w.x2r[l], Ri, w.yi, B, W, W, ldm, W, ldm, 0, 0, W, (long long)W * W, W, nm, 1.f, 0.f), s));
    NCK(gemm_bf16(gemm(w.x2i[l], Rr, w.yi, B, W, W, ldm, W, ldm, 0, 0, W, (long long)W * W, W, nm, 1.f, 1.f), s));
    // (4) inverse (z then) y
    if (d == 2) {
      NCK(ax.inv(w.yr, w.yi, w.z1r, w.z1i, KW, sx2, sx1, B));
    } else {
      NCK(ax.inv(w.yr, w.yi, w.mr, w.mi, K1 * KW, (long long)K1 * K1 * KW, (long long)N * K1 * KW, B));
      NCK(ax.inv(w.mr, w.mi, w.z1r, w.z1i, KW, sx2, sx1, B * N));
    }
    // (5) inverse x (half spectrum), per (b, (z,) y): s = Er Z1r + Ei Z1i   ([N x K] x [K x W]) into z
    NCK(gemm_bf16(gemm(bs.Er, w.z1r, w.z[l], N, W, K, K, W, W, 0, 0, 0, (long long)K * W, (long long)N * W, BN, 1.f, 0.f), s));
    NCK(gemm_bf16(gemm(bs.Ei, w.z1i, w.z[l], N, W, K, K, W, W, 0, 0, 0, (long long)K * W, (long long)N * W, BN, 1.f, 1.f), s));
    // (6) z += v W ; (7) bias + activation
    NCK(gemm_bf16(gemm(v, prm + o.W[l], w.z[l], (int)P, W, W, W, W, W, 0, 0, 0, 0, 0, 1, 1.f, 1.f), s));
    k_bias_act<<<eblocks(P * W), 256, 0, s>>>(w.z[l], prm + o.b[l], w.v[l + 1], P, W, l + 1 < c.layers ? 1 : 0);
  }
  // projection
  NCK(gemm_bf16(gemm(w.v[c.layers], prm + o.p1_w, w.pz, (int)P, c.proj, W, W, c.proj, c.proj, 0, 0, 0, 0, 0, 1, 1.f, 0.f), s));
  k_bias_act<<<eblocks(P * c.proj), 256, 0, s>>>(w.pz, prm + o.p1_b, w.ph, P, c.proj, 1);
  NCK(gemm_bf16(gemm(w.ph, prm + o.p2_w, out, (int)P, c.cout, c.proj, c.proj, c.cout, c.cout, 0, 0, 0, 0, 0, 1, 1.f, 0.f), s));
  k_bias_act<<<eblocks(P * c.cout), 256, 0, s>>>(out, prm + o.p2_b, out, P, c.cout, 0);
  g_split_ws = nullptr;
  g_split_floats = 0;
  return cudaGetLastError();
}

cudaError_t net_backward(const NetConfig& c, const float* prm, const float* bases, int B, const float* in,
                         const float* target, float* grad, float* loss_dev, float* ws, cudaStream_t s) {
  const NetOffsets o = net_offsets(c);
  NetWs w = carve(c, B, ws);
  const Bases bs = bases_of(c, bases);
  const Axis ax{bs, c.N, 2 * c.modes, s};
  const int d = c.d == 3 ? 3 : 2;
  const int N = c.N, W = c.width, K = c.modes, K1 = 2 * c.modes, KW = K * W;
  const long long P = (long long)B * ipow(N, d);
  const int BN = (int)(B * ipow(N, d - 1));
  const long long nmodes = spectral_modes(c);
  // forward with the activations kept; output into dh's tail (reuse of pz for out is not possible)
  float* out = w.dh;   // [P x cout] fits in [P x proj]
  NCK(net_forward(c, prm, bases, B, in, out, ws, 1, s));
  g_split_ws = w.split;
  g_split_floats = w.split_floats;
  // loss and d out (in place in out)
  const long long nout = P * c.cout;
  const int lb = (int)std::min<long long>(1024, (nout + 255) / 256);
  k_mse<<<lb, 256, 0, s>>>(out, target, out, nout, w.lpart);
  k_mse_final<<<1, 32, 0, s>>>(w.lpart, lb, nout, loss_dev);
  // projection backward
  NCK(colsum(out, P, c.cout, grad + o.p2_b, w.colpart, s));
  NCK(gemm_bf16(gemm(w.ph, out, grad + o.p2_w, c.proj, c.cout, (int)P, c.proj, c.cout, c.cout, 1, 0, 0, 0, 0, 1, 1.f, 0.f), s));
  // dh = dout P2^T into pz's buffer after using pz for gelu'
  float* dh = w.ph;   // ph no longer needed after dP2
  NCK(gemm_bf16(gemm(out, prm + o.p2_w, dh, (int)P, c.proj, c.cout, c.cout, c.cout, c.proj, 0, 1, 0, 0, 0, 1, 1.f, 0.f), s));
  k_gelu_back<<<eblocks(P * c.proj), 256, 0, s>>>(dh, w.pz, dh, P * c.proj);
  NCK(colsum(dh, P, c.proj, grad + o.p1_b, w.colpart, s));
  NCK(gemm_bf16(gemm(w.v[c.layers], dh, grad + o.p1_w, W, c.proj, (int)P, W, c.proj, c.proj, 1, 0, 0, 0, 0, 1, 1.f, 0.f), s));
  NCK(gemm_bf16(gemm(dh, prm + o.p1_w, w.dv, (int)P, W, c.proj, c.proj, c.proj, W, 0, 1, 0, 0, 0, 1, 1.f, 0.f), s));
  // layers, last to first; w.dv holds d v_{l+1}
  for (int l = c.layers - 1; l >= 0; --l) {
    const float* v = w.v[l];
    const float* Rr = prm + o.R[l];
    const float* Ri = Rr + nmodes * W * W;
    float* dRr = grad + o.R[l];
    float* dRi = dRr + nmodes * W * W;
    if (l + 1 < c.layers) k_gelu_back<<<eblocks(P * W), 256, 0, s>>>(w.dv, w.z[l], w.dz, P * W);
    else NCK(cudaMemcpyAsync(w.dz, w.dv, P * W * sizeof(float), cudaMemcpyDeviceToDevice, s));
    NCK(colsum(w.dz, P, W, grad + o.b[l], w.colpart, s));
    NCK(gemm_bf16(gemm(v, w.dz, grad + o.W[l], W, W, (int)P, W, W, W, 1, 0, 0, 0, 0, 1, 1.f, 0.f), s));
    NCK(gemm_bf16(gemm(w.dz, prm + o.W[l], w.dv, (int)P, W, W, W, W, W, 0, 1, 0, 0, 0, 1, 1.f, 0.f), s));
    // (5') dZ1 = E^T dz, per (b, (z,) y): [K x N] x [N x W]
    NCK(gemm_bf16(gemm(bs.Er, w.dz, w.dz1r, K, W, N, K, W, W, 1, 0, 0, (long long)N * W, (long long)K * W, BN, 1.f, 0.f), s));
    NCK(gemm_bf16(gemm(bs.Ei, w.dz, w.dz1i, K, W, N, K, W, W, 1, 0, 0, (long long)N * W, (long long)K * W, BN, 1.f, 0.f), s));
    // (4') adjoint of the inverse y (and then z) transform: dY = H^T dZ1
    const long long sx1 = (long long)N * KW, sx2 = (long long)K1 * KW;
    if (d == 2) {
      NCK(ax.inv_adj(w.dz1r, w.dz1i, w.dyr, w.dyi, KW, sx1, sx2, B));
    } else {
      NCK(ax.inv_adj(w.dz1r, w.dz1i, w.dmr, w.dmi, KW, sx1, sx2, B * N));
      NCK(ax.inv_adj(w.dmr, w.dmi, w.dyr, w.dyi, K1 * KW, (long long)N * K1 * KW, (long long)K1 * K1 * KW, B));
    }
    // (3') per mode: dRr = X2r^T dYr + X2i^T dYi ; dRi = X2r^T dYi - X2i^T dYr   ([W x B] x [B x W])
    const int nm = (int)nmodes;
    const int ldm = nm * W;
    const long long WW = (long long)W * W;
    NCK(gemm_bf16(gemm(w.x2r[l], w.dyr, dRr, W, W, B, ldm, ldm, W, 1, 0, W, W, WW, nm, 1.f, 0.f), s));
    NCK(gemm_bf16(gemm(w.x2i[l], w.dyi, dRr, W, W, B, ldm, ldm, W, 1, 0, W, W, WW, nm, 1.f, 1.f), s));
    NCK(gemm_bf16(gemm(w.x2r[l], w.dyi, dRi, W, W, B, ldm, ldm, W, 1, 0, W, W, WW, nm, 1.f, 0.f), s));
    NCK(gemm_bf16(gemm(w.x2i[l], w.dyr, dRi, W, W, B, ldm, ldm, W, 1, 0, W, W, WW, nm, -1.f, 1.f), s));
    //      dX2r = dYr Rr^T + dYi Ri^T ; dX2i = dYi Rr^T - dYr Ri^T   ([B x W] x [W x W]^T)
    NCK(gemm_bf16(gemm(w.dyr, Rr, w.dx2r, B, W, W, ldm, W, ldm, 0, 1, W, WW, W, nm, 1.f, 0.f), s));
    NCK(gemm_bf16(gemm(w.dyi, Ri, w.dx2r, B, W, W, ldm, W, ldm, 0, 1, W, WW, W, nm, 1.f, 1.f), s));
    NCK(gemm_bf16(gemm(w.dyi, Rr, w.dx2i, B, W, W, ldm, W, ldm, 0, 1, W, WW, W, nm, 1.f, 0.f), s));
    NCK(gemm_bf16(gemm(w.dyr, Ri, w.dx2i, B, W, W, ldm, W, ldm, 0, 1, W, WW, W, nm, -1.f, 1.f), s));
    // (2') adjoint of the forward (z then) y transform: dX1 = G^T dX2
    if (d == 2) {
      NCK(ax.fwd_adj(w.dx2r, w.dx2i, w.dx1r, w.dx1i, KW, sx2, sx1, B));
    } else {
      NCK(ax.fwd_adj(w.dx2r, w.dx2i, w.dmr, w.dmi, K1 * KW, (long long)K1 * K1 * KW, (long long)N * K1 * KW, B));
      NCK(ax.fwd_adj(w.dmr, w.dmi, w.dx1r, w.dx1i, KW, sx2, sx1, B * N));
    }
    // (1') dv += Fr^T dX1r + Fi^T dX1i, per (b, (z,) y): [N x K] x [K x W]
    NCK(gemm_bf16(gemm(bs.Fr, w.dx1r, w.dv, N, W, K, N, W, W, 1, 0, 0, (long long)K * W, (long long)N * W, BN, 1.f, 1.f), s));
    NCK(gemm_bf16(gemm(bs.Fi, w.dx1i, w.dv, N, W, K, N, W, W, 1, 0, 0, (long long)K * W, (long long)N * W, BN, 1.f, 1.f), s));
  }
  // lift
  NCK(colsum(w.dv, P, W, grad + o.lift_b, w.colpart, s));
  NCK(gemm_bf16(gemm(in, w.dv, grad + o.lift_w, c.cin, W, (int)P, c.cin, W, W, 1, 0, 0, 0, 0, 1, 1.f, 0.f), s));
  g_split_ws = nullptr;
  g_split_floats = 0;
  return cudaGetLastError();
}

// Training targets: each group of `group` consecutive channels of one sample scaled to unit
// RMS over all its grid points and channels (the RMS clamped below at 1e-12). One CTA per
// (sample, group): an FP64 block sum of squares, then the scaling.
__global__ void k_normalise_groups(float* grid, long long pts, int ch, int group) {
  const int ngroups = ch / group;
  const int sample = blockIdx.x / ngroups;
  const int gi = blockIdx.x - sample * ngroups;
  float* base = grid + (long long)sample * pts * ch + (long long)gi * group;
  const long long total = pts * group;
  double acc = 0.0;
  for (long long t = threadIdx.x; t < total; t += blockDim.x) {
    const long long pt = t / group;
    const float v = base[pt * ch + (t - pt * group)];
    acc += (double)v * v;
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  const double rms = fmax(sqrt(red[0] / (double)total), 1e-12);
  const float inv = (float)(1.0 / rms);
  for (long long t = threadIdx.x; t < total; t += blockDim.x) {
    const long long pt = t / group;
    base[pt * ch + (t - pt * group)] *= inv;
  }
}

cudaError_t normalise_groups(float* grid, int n, long long pts, int ch, int group, cudaStream_t s) {
  if (n < 1 || group < 1 || ch % group) return cudaErrorInvalidValue;
  const long long blocks = (long long)n * (ch / group);
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  k_normalise_groups<<<(unsigned)blocks, 256, 0, s>>>(grid, pts, ch, group);
  return cudaGetLastError();
}

cudaError_t adam_step(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                      float eps, int step, cudaStream_t s) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam<<<eblocks(n), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t init_params(const NetConfig& c, float* prm, unsigned long long seed, cudaStream_t s) {
  const NetOffsets o = net_offsets(c);
  auto uni = [&](long long off, long long n, float a, unsigned long long sd) {
    k_init<<<eblocks(n), 256, 0, s>>>(prm + off, n, -a, a, seed * 1315423911ULL + sd);
  };
  auto zero = [&](long long off, long long n) { k_fill<<<eblocks(n), 256, 0, s>>>(prm + off, n, 0.f); };
  uni(o.lift_w, (long long)c.cin * c.width, 1.f / sqrtf((float)c.cin), 1);
  zero(o.lift_b, c.width);
  for (int l = 0; l < c.layers; ++l) {
    const float sc = 1.f / (float)(c.width * c.width);
    const long long nR = 2LL * spectral_modes(c) * c.width * c.width;
    k_init<<<eblocks(nR), 256, 0, s>>>(prm + o.R[l], nR, 0.f, sc, seed * 2654435761ULL + 100 + l);
    uni(o.W[l], (long long)c.width * c.width, 1.f / sqrtf((float)c.width), 200 + l);
    zero(o.b[l], c.width);
  }
  uni(o.p1_w, (long long)c.width * c.proj, 1.f / sqrtf((float)c.width), 300);
  zero(o.p1_b, c.proj);
  uni(o.p2_w, (long long)c.proj * c.cout, 1.f / sqrtf((float)c.proj), 301);
  zero(o.p2_b, c.cout);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// real N-grid fields <-> half spectra (direct DFT, one CTA per (sample, channel))
// ---------------------------------------------------------------------------------
// One CTA per (slab, channel): the 2D DFT of an N x N slab by direct sums (rows, then
// columns in FFT order). Slab s = b * Nz + z of grid [B][(Nz)][N][N][ch]; output at
// [b][ch][z][ky][kx] of the half spectrum, times `scale`.
__global__ void k_grid_to_half(int N, int ch, int Nz, const float* grid, void* half, int fp64, double scale) {
  extern __shared__ __align__(16) unsigned char sm[];
  float* u = reinterpret_cast<float*>(sm);                 // N*N
  float2* tw = reinterpret_cast<float2*>(u + N * N + (N * N & 1));   // N
  float2* R = tw + N;                                      // N * Nh
  const int Nh = (N + 1) / 2;
  const int sl = blockIdx.x / ch, c = blockIdx.x - (blockIdx.x / ch) * ch;
  const int b = sl / Nz, z = sl - (sl / Nz) * Nz;
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) u[i] = grid[((long long)sl * N * N + i) * ch + c];
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    float sn, cs;
    sincospif(2.f * i / N, &sn, &cs);
    tw[i] = make_float2(cs, sn);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < N * Nh; t += blockDim.x) {   // rows: R[y][kx] = sum_x u e^{-2 pi i kx x/N}
    const int y = t / Nh, kx = t - y * Nh;
    float re = 0.f, im = 0.f;
    int idx = 0;
    for (int x = 0; x < N; ++x) {
      const float2 w = tw[idx];
      re += u[y * N + x] * w.x;
      im -= u[y * N + x] * w.y;
      idx += kx;
      if (idx >= N) idx -= N;
    }
    R[t] = make_float2(re, im);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < N * Nh; t += blockDim.x) {   // columns, FFT order ky
    const int i = t / Nh, kx = t - i * Nh;
    float re = 0.f, im = 0.f;
    int idx = 0;
    for (int y = 0; y < N; ++y) {
      const float2 w = tw[idx];
      const float2 r = R[y * Nh + kx];
      re += r.x * w.x + r.y * w.y;
      im += r.y * w.x - r.x * w.y;
      idx += i;
      if (idx >= N) idx -= N;
    }
    const long long o = (((long long)(b * ch + c) * Nz + z) * N + i) * Nh + kx;
    if (fp64) reinterpret_cast<double2*>(half)[o] = make_double2(re * scale, im * scale);
    else reinterpret_cast<float2*>(half)[o] = make_float2((float)(re * scale), (float)(im * scale));
  }
}

// One CTA per (slab, channel): the real N x N slab of a half spectrum [b][ch][z][ky][kx]
// (columns inverse, then the Hermitian-weighted real inverse along x), no scaling.
__global__ void k_half_to_grid(int N, int ch, int Nz, const void* half, float* grid, int fp64) {
  extern __shared__ __align__(16) unsigned char sm[];
  float2* H = reinterpret_cast<float2*>(sm);   // N * Nh
  const int Nh = (N + 1) / 2;
  float2* S = H + N * Nh;                       // N * Nh
  float2* tw = S + N * Nh;                      // N
  const int sl = blockIdx.x / ch, c = blockIdx.x - (blockIdx.x / ch) * ch;
  const int b = sl / Nz, z = sl - (sl / Nz) * Nz;
  for (int i = threadIdx.x; i < N * Nh; i += blockDim.x) {
    const long long o = ((long long)(b * ch + c) * Nz + z) * N * Nh + i;
    if (fp64) {
      const double2 v = reinterpret_cast<const double2*>(half)[o];
      H[i] = make_float2((float)v.x, (float)v.y);
    } else {
      H[i] = reinterpret_cast<const float2*>(half)[o];
    }
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    float sn, cs;
    sincospif(2.f * i / N, &sn, &cs);
    tw[i] = make_float2(cs, sn);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < N * Nh; t += blockDim.x) {   // S[y][kx] = sum_i H[i][kx] e^{2 pi i i y/N}
    const int y = t / Nh, kx = t - y * Nh;
    float re = 0.f, im = 0.f;
    int idx = 0;
    for (int i = 0; i < N; ++i) {
      const float2 w = tw[idx];
      const float2 h = H[i * Nh + kx];
      re += h.x * w.x - h.y * w.y;
      im += h.x * w.y + h.y * w.x;
      idx += y;
      if (idx >= N) idx -= N;
    }
    S[t] = make_float2(re, im);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < N * N; t += blockDim.x) {   // u[y][x] = Re S[y][0] + 2 sum Re(S e^{...})
    const int y = t / N, x = t - y * N;
    float acc = S[y * Nh].x;
    int idx = x;
    for (int kx = 1; kx < Nh; ++kx) {
      const float2 w = tw[idx];
      const float2 sv = S[y * Nh + kx];
      acc += 2.f * (sv.x * w.x - sv.y * w.y);
      idx += x;
      if (idx >= N) idx -= N;
    }
    grid[((long long)sl * N * N + t) * ch + c] = acc;
  }
}

// DFT along z of columns of [bc][z][ky][kx] (N x N x Nh per bc): one CTA per (bc, ky,
// block of kZB kx); the N x kZB block is staged in shared memory, so in == out is allowed.
// sign -1: forward e^{-2 pi i kz z / N}; +1: inverse. Sums in FP32.
constexpr int kZB = 32;
__global__ void k_zdft(int N, const void* in, int fp64_in, void* out, int fp64_out, int sign) {
  extern __shared__ __align__(16) unsigned char sm[];
  float2* col = reinterpret_cast<float2*>(sm);   // N * kZB
  float2* tw = col + N * kZB;                      // N
  const int Nh = (N + 1) / 2;
  const int nkb = (Nh + kZB - 1) / kZB;
  const int kb = blockIdx.x % nkb;
  const int ky = (blockIdx.x / nkb) % N;
  const long long bc = blockIdx.x / ((long long)nkb * N);
  const int kx0 = kb * kZB, nk = min(kZB, Nh - kx0);
  const long long base = bc * N * N * Nh + (long long)ky * Nh + kx0;   // + z * N * Nh + j
  for (int t = threadIdx.x; t < N * kZB; t += blockDim.x) {
    const int z = t / kZB, j = t - z * kZB;
    float2 v = make_float2(0.f, 0.f);
    if (j < nk) {
      const long long o = base + (long long)z * N * Nh + j;
      if (fp64_in) {
        const double2 dv = reinterpret_cast<const double2*>(in)[o];
        v = make_float2((float)dv.x, (float)dv.y);
      } else {
        v = reinterpret_cast<const float2*>(in)[o];
      }
    }
    col[t] = v;
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    float sn, cs;
    sincospif(2.f * i / N, &sn, &cs);
    tw[i] = make_float2(cs, (float)sign * sn);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < N * kZB; t += blockDim.x) {
    const int kz = t / kZB, j = t - kz * kZB;
    if (j >= nk) continue;
    float re = 0.f, im = 0.f;
    int idx = 0;
    for (int z = 0; z < N; ++z) {
      const float2 w = tw[idx];
      const float2 v = col[z * kZB + j];
      re += v.x * w.x - v.y * w.y;
      im += v.x * w.y + v.y * w.x;
      idx += kz;
      if (idx >= N) idx -= N;
    }
    const long long o = base + (long long)kz * N * Nh + j;
    if (fp64_out) reinterpret_cast<double2*>(out)[o] = make_double2(re, im);
    else reinterpret_cast<float2*>(out)[o] = make_float2(re, im);
  }
}

static size_t g2h_smem(int N) {
  const int Nh = (N + 1) / 2;
  return (size_t)N * N * 4 + 8 + (size_t)N * 8 + (size_t)N * Nh * 8;
}
static size_t h2g_smem(int N) {
  const int Nh = (N + 1) / 2;
  return 2 * (size_t)N * Nh * 8 + (size_t)N * 8;
}
static size_t zdft_smem(int N) { return (size_t)N * kZB * 8 + (size_t)N * 8; }
constexpr size_t kMaxSmem = 227 * 1024;

static cudaError_t launch_zdft(int N, long long nbc, const void* in, int fp64_in, void* out, int fp64_out, int sign,
                               cudaStream_t s) {
  const size_t smem = zdft_smem(N);
  {
    static std::atomic<int> cache[kAttrDevices] = {};
    const cudaError_t ea = smem_attr(k_zdft, smem, cache);
    if (ea != cudaSuccess) return ea;
  }
  const int Nh = (N + 1) / 2;
  const long long blocks = nbc * N * ((Nh + kZB - 1) / kZB);
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  k_zdft<<<(unsigned)blocks, 256, smem, s>>>(N, in, fp64_in, out, fp64_out, sign);
  return cudaGetLastError();
}

cudaError_t grid_to_half(int d, int N, int B, int ch, const float* grid, void* half, int fp64, cudaStream_t s) {
  const size_t smem = g2h_smem(N);
  if (smem > kMaxSmem || zdft_smem(N) > kMaxSmem) return cudaErrorInvalidValue;
  {
    static std::atomic<int> cache[kAttrDevices] = {};
    const cudaError_t ea = smem_attr(k_grid_to_half, smem, cache);
    if (ea != cudaSuccess) return ea;
  }
  const int Nz = d == 3 ? N : 1;
  const double scale = 1.0 / ((double)ipow(N, d == 3 ? 3 : 2));
  k_grid_to_half<<<B * Nz * ch, 256, smem, s>>>(N, ch, Nz, grid, half, fp64, scale);
  NCK(cudaGetLastError());
  if (d == 3) return launch_zdft(N, (long long)B * ch, half, fp64, half, fp64, -1, s);
  return cudaSuccess;
}

size_t half3d_tmp_bytes(int N, int B, int ch) { return (size_t)B * ch * N * N * ((N + 1) / 2) * 8; }

cudaError_t half_to_grid(int d, int N, int B, int ch, const void* half, float* grid, int fp64, void* tmp,
                         cudaStream_t s) {
  const size_t smem = h2g_smem(N);
  if (smem > kMaxSmem || zdft_smem(N) > kMaxSmem) return cudaErrorInvalidValue;
  {
    static std::atomic<int> cache[kAttrDevices] = {};
    const cudaError_t ea = smem_attr(k_half_to_grid, smem, cache);
    if (ea != cudaSuccess) return ea;
  }
  if (d == 3) {
    if (!tmp) return cudaErrorInvalidValue;
    NCK(launch_zdft(N, (long long)B * ch, half, fp64, tmp, 0, +1, s));
    k_half_to_grid<<<B * N * ch, 256, smem, s>>>(N, ch, N, tmp, grid, 0);
  } else {
    k_half_to_grid<<<B * ch, 256, smem, s>>>(N, ch, 1, half, grid, fp64);
  }
  return cudaGetLastError();
}

}  // namespace homb
