// Block project / promote (Sec. 2.5.1, "Transfer between grids") for
// complex64 on the tensor cores (tcgen05): one small complex GEMM per coarse
// block x,
//   promote:  F(x) = B(x) C(x)          (v_block x nrhs)
//   project:  C(x) = B(x)^dagger F(x)   (n_basis x nrhs)
// with the basis B [n_blocks][v_block][n_basis], fine vectors
// [n_blocks][v_block][nrhs] and coarse vectors [n_blocks][n_basis][nrhs].
//
// Every FP32 value is split exactly into three bf16 terms (bf16x3.cuh) and
// the six products down to order 2^-16 are summed in FP32 tensor memory:
// FP32-class products, as the FMA kernels of blocking.cu give.
//
// Real forms as in blas_tc.cu: a complex64 row of r columns is 2r
// interleaved reals.  Promote multiplies each fine row of B(x) (K = 2
// n_basis reals) by the 2 n_basis x 2 nrhs real form of C(x); project forms
// P = Bre^T Fre over the block's fine rows (K = v_block) and reads
// C[a][r] = (P[2a][2r] + P[2a+1][2r+1]) + i (P[2a][2r+1] - P[2a+1][2r]).
// The MMAs (M = 128, bf16, FP32 accumulation), with the small operand's
// terms stacked along N as [h; m; l] (Nn = round16(2 nrhs) rows each):
//   A_h x [h; m; l],  A_m x [h; m],  A_l x [h]
// so the accumulator's three column blocks sum to the six wanted products.
//
// The blocks are many and small, so a CTA runs one block at a time without
// an internal pipeline (convert, one thread issues the MMAs and commits,
// everyone waits) and two or three CTAs per SM overlap one another.  Every
// wait is bounded (1 s); on expiry the CTA records an error bit in the word
// of mrhs_device_error (1024), stops and frees its tensor memory.
#include "bf16x3.cuh"
#include "internal.cuh"
#include "tc_ptx.cuh"

namespace mrhs {

__device__ unsigned int g_bltc_error = 0;

namespace {

constexpr int kBlThreads = 256;
constexpr uint32_t kErrBlocking = 1024u;

// the small operand's terms: Op[t Nn + j][k] = term t of W(k, j) (zero
// outside kreal x jreal), K-major with row groups `sbo` apart
template <typename Val>
__device__ inline void build_small_terms(uint8_t* dst, int Nn, int K16, int kreal, int jreal,
                                         uint32_t sbo, Val W) {
  for (int e = threadIdx.x; e < Nn * K16; e += blockDim.x) {
    const int j = e / K16, k = e - j * K16;
    const float v = (j < jreal && k < kreal) ? W(k, j) : 0.f;
    uint32_t h, m, l;
    split3(v, h, m, l);
    const uint32_t terms[3] = {h, m, l};
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const int n = t * Nn + j;
      const uint32_t off = (uint32_t)(n >> 3) * sbo + (uint32_t)(k >> 3) * 128u +
                           (uint32_t)(n & 7) * 16u + (uint32_t)(k & 7) * 2u;
      *reinterpret_cast<uint16_t*>(dst + off) = (uint16_t)(terms[t] >> 16);
    }
  }
}

// three MMAs of one K step into the accumulator d: A terms at a_h, a_h + dA,
// a_h + 2 dA (M = 128), the small operand's stacked terms at b (N = 3Nn, 2Nn,
// Nn); `first` starts the accumulation
__device__ __forceinline__ void mma3(uint32_t d, uint32_t a_h, uint32_t dA, uint32_t a_lbo,
                                     uint32_t a_sbo, uint32_t b, uint32_t b_sbo, int Nn,
                                     bool first) {
  const uint64_t bd = ptx::smem_desc(b, 128u, b_sbo);
  ptx::mma_f16(d, ptx::smem_desc(a_h, a_lbo, a_sbo), bd, ptx::idesc_f16(128, 3 * Nn, true),
               first ? 0u : 1u);
  ptx::mma_f16(d, ptx::smem_desc(a_h + dA, a_lbo, a_sbo), bd, ptx::idesc_f16(128, 2 * Nn, true),
               1u);
  ptx::mma_f16(d, ptx::smem_desc(a_h + 2 * dA, a_lbo, a_sbo), bd, ptx::idesc_f16(128, Nn, true),
               1u);
}

// thread 0 commits the MMAs issued so far to bar; everyone waits (bounded)
__device__ __forceinline__ bool commit_wait(uint64_t* bar, uint32_t& phase, volatile int* abort) {
  if (threadIdx.x == 0) ptx::mma_commit(bar);
  const bool ok = ptx::mbar_wait(bar, phase, abort);
  phase ^= 1u;
  ptx::tc_fence_after();
  return ok;
}

// ============================================================ promote
// F(x) = B(x) C(x).  Row tiles of 128 fine rows; K = 2 n_basis reals in
// halves of 64 (32 basis columns), each half's A terms (3 x 128 x 64 bf16 =
// 48 KB) converted from global memory and multiplied before the next.
constexpr uint32_t kPrA = 3 * 128 * 64 * 2;           // A terms of one K half
// smem: [small terms: 3 Nn x K16 bf16][A terms]
__global__ void __launch_bounds__(kBlThreads, 3)
    k_promote_tc(const float2* __restrict__ basis, const float2* __restrict__ Cc,
                 float2* __restrict__ F, int64_t nblk, int vb, int nbasis, int R) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t bar, done;
  __shared__ uint32_t tslot;
  __shared__ volatile int s_abort;
  const int kreal = 2 * nbasis, jreal = 2 * R;
  const int K16 = (kreal + 15) & ~15, Nn = (jreal + 15) & ~15;
  const uint32_t bsbo = (uint32_t)K16 * 16u;
  const uint32_t bbytes = (uint32_t)(3 * Nn) * (uint32_t)K16 * 2u;
  uint8_t* sB = smem;
  uint8_t* sA = smem + ((bbytes + 1023u) & ~1023u);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t tcols = 3 * Nn <= 128 ? 128u : 256u;
  if (threadIdx.x == 0) {
    ptx::mbar_init(&bar, 1);
    ptx::mbar_init(&done, 1);
    ptx::fence_mbar_init();
    s_abort = 0;
  }
  if (warp == 0) {
    ptx::tmem_alloc(&tslot, tcols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = tslot;
  uint32_t phase = 0;
  const int nkh = (kreal + 63) / 64;                    // K halves
  const int ntile = (vb + 127) / 128;
  for (int64_t x = blockIdx.x; x < nblk && !s_abort; x += gridDim.x) {
    // the three terms of C(x)'s real 2 nb x 2R form,
    // Wre[2c + p][2d + q]: (0,0) Re, (1,0) -Im, (0,1) Im, (1,1) Re
    const float2* Cx = Cc + x * (int64_t)nbasis * R;
    const float* Bx = reinterpret_cast<const float*>(basis + x * (int64_t)vb * nbasis);
    float2* Fx = F + x * (int64_t)vb * R;
    // unit u = (row tile u / nkh, K half u % nkh): its A terms, task = (row,
    // 8-real piece), lanes = 8 rows x 4 pieces, so loads cover whole
    // 128-byte row segments and stores whole core matrices.  The next
    // unit's loads are issued while the current unit's MMAs run.
    float v[4][8];
    auto load = [&](int u) {
      const int t = u / nkh, h = u - (u / nkh) * nkh;
#pragma unroll
      for (int it = 0; it < 4; ++it) {
        const int w = it * 8 + warp;         // 0..31
        const int row = 8 * (w & 15) + (lane & 7), pc = (lane >> 3) + 4 * (w >> 4);
        const int grow = 128 * t + row, k0 = 64 * h + 8 * pc;
        if (grow < vb && k0 < kreal) {
          const float4* p = reinterpret_cast<const float4*>(Bx + (int64_t)grow * kreal + k0);
          const float4 a = __ldg(p), b = __ldg(p + 1);
          v[it][0] = a.x; v[it][1] = a.y; v[it][2] = a.z; v[it][3] = a.w;
          v[it][4] = b.x; v[it][5] = b.y; v[it][6] = b.z; v[it][7] = b.w;
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) v[it][e] = 0.f;
        }
      }
    };
    load(0);
    // the three terms of C(x)'s real 2 nb x 2R form,
    // Wre[2c + p][2d + q]: (0,0) Re, (1,0) -Im, (0,1) Im, (1,1) Re
    build_small_terms(sB, Nn, K16, kreal, jreal, bsbo, [&](int k, int j) {
      const float2 z = __ldg(&Cx[(k >> 1) * R + (j >> 1)]);
      const int p = k & 1, q = j & 1;
      return p == q ? z.x : (p ? -z.y : z.y);
    });
    const int nunit = ntile * nkh;
    for (int u = 0; u < nunit; ++u) {
      const int t = u / nkh, h = u - t * nkh;
#pragma unroll
      for (int it = 0; it < 4; ++it) {
        const int w = it * 8 + warp;
        const int row = 8 * (w & 15) + (lane & 7), pc = (lane >> 3) + 4 * (w >> 4);
        const uint32_t base = ptx::smem_u32(sA) + (uint32_t)(row >> 3) * 1024u +
                              (uint32_t)pc * 128u + (uint32_t)(row & 7) * 16u;
        split_store8(v[it], base, kPrA / 3, 2 * (kPrA / 3));
      }
      ptx::fence_proxy_async_smem();
      ptx::tc_fence_before();
      __syncthreads();
      if (threadIdx.x == 0) {
        ptx::tc_fence_after();
        const int ksteps = (kreal - 64 * h) >= 64 ? 4 : ((kreal - 64 * h) + 15) / 16;
        for (int kk = 0; kk < ksteps; ++kk)
          mma3(tmem, ptx::smem_u32(sA) + (uint32_t)kk * 256u, kPrA / 3, 128u, 1024u,
               ptx::smem_u32(sB) + (uint32_t)(4 * h + kk) * 256u, bsbo, Nn, h == 0 && kk == 0);
      }
      if (u + 1 < nunit) load(u + 1);
      if (!commit_wait(&bar, phase, &s_abort)) {
        s_abort = 1;
        atomicOr(&g_bltc_error, kErrBlocking);
      }
      __syncthreads();
      if (s_abort) break;
      if (h < nkh - 1) continue;
      // epilogue of tile t: warps 0-3, lane r = tile row r; y = the sum of
      // the three column blocks
      if (warp < 4) {
        const int grow = 128 * t + 32 * warp + lane;
        const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16);
        for (int c0 = 0; c0 < jreal; c0 += 8) {
          float u0[8], u1[8], u2[8];
          ptx::tmem_ld8_sync(ta + (uint32_t)c0, u0);
          ptx::tmem_ld8_sync(ta + (uint32_t)(Nn + c0), u1);
          ptx::tmem_ld8_sync(ta + (uint32_t)(2 * Nn + c0), u2);
          if (grow < vb) {
            float* dst = reinterpret_cast<float*>(Fx + (int64_t)grow * R) + c0;
#pragma unroll
            for (int e = 0; e < 8; e += 4)
              if (c0 + e < jreal)
                *reinterpret_cast<float4*>(dst + e) =
                    make_float4(u0[e] + u1[e] + u2[e], u0[e + 1] + u1[e + 1] + u2[e + 1],
                                u0[e + 2] + u1[e + 2] + u2[e + 2], u0[e + 3] + u1[e + 3] + u2[e + 3]);
          }
        }
      }
      ptx::tc_fence_before();
      __syncthreads();
      ptx::tc_fence_after();
    }
    __syncthreads();     // sB is rebuilt for the next block
  }
  // every MMA of this CTA has completed before its tensor memory is freed
  if (threadIdx.x == 0) {
    ptx::mma_commit(&done);
    volatile int never = 0;
    ptx::mbar_wait(&done, 0, &never);
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, tcols);
  }
}

// ============================================================ project
// C(x) = B(x)^dagger F(x).  The block's fine rows are the contraction: chunks
// of four 16-row MMA steps, each step's operands B^T (M = 2 n_basis <= 128
// real columns) and F^T (N = 2 nrhs real columns) converted from global
// memory, lane = real column so that a warp's loads of a row are one line.
constexpr uint32_t kPjAStep = 3 * 128 * 16 * 2;       // A terms of one step (12 KB)
// smem: [A terms: 4 steps][F terms: 4 steps x 3 Nn x 16 bf16]
__global__ void __launch_bounds__(kBlThreads)
    k_project_tc(const float2* __restrict__ basis, const float2* __restrict__ F,
                 float2* __restrict__ Cc, int64_t nblk, int vb, int nbasis, int R) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t bar, done;
  __shared__ uint32_t tslot;
  __shared__ volatile int s_abort;
  const int kreal = 2 * nbasis, jreal = 2 * R;
  const int Nn = (jreal + 15) & ~15;
  const uint32_t fstep = (uint32_t)(3 * Nn) * 32u;     // F terms of one step
  uint8_t* sA = smem;
  uint8_t* sF = smem + 4 * kPjAStep;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t tcols = 3 * Nn <= 128 ? 128u : 256u;
  if (threadIdx.x == 0) {
    ptx::mbar_init(&bar, 1);
    ptx::mbar_init(&done, 1);
    ptx::fence_mbar_init();
    s_abort = 0;
  }
  if (warp == 0) {
    ptx::tmem_alloc(&tslot, tcols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = tslot;
  uint32_t phase = 0;
  const int nchunk = vb / 64;                          // vb is a multiple of 64
  const int nj = (Nn + 31) / 32;                       // 32-column blocks of F^T
  for (int64_t x = blockIdx.x; x < nblk && !s_abort; x += gridDim.x) {
    const float* Bx = reinterpret_cast<const float*>(basis + x * (int64_t)vb * nbasis);
    const float* Fx = reinterpret_cast<const float*>(F + x * (int64_t)vb * R);
    for (int c = 0; c < nchunk; ++c) {
      // B^T: task (step s, 8-row half kh, 32-column block mb) per warp, four
      // per warp, loads of all four first
      float v[4][8];
#pragma unroll
      for (int it = 0; it < 4; ++it) {
        const int task = it * 8 + warp;                  // 0..31
        const int s = task >> 3, kh = (task >> 2) & 1, mb = task & 3;
        const int m = 32 * mb + lane;
        const int64_t r0 = 64 * (int64_t)c + 16 * s + 8 * kh;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk)
          v[it][kk] = m < kreal ? __ldg(Bx + (r0 + kk) * kreal + m) : 0.f;
      }
#pragma unroll
      for (int it = 0; it < 4; ++it) {
        const int task = it * 8 + warp;
        const int s = task >> 3, kh = (task >> 2) & 1, mb = task & 3;
        const int m = 32 * mb + lane;
        const uint32_t base = ptx::smem_u32(sA) + (uint32_t)s * kPjAStep + (uint32_t)(m >> 3) * 256u +
                              (uint32_t)kh * 128u + (uint32_t)(m & 7) * 16u;
        split_store8(v[it], base, kPjAStep / 3, 2 * (kPjAStep / 3));
      }
      // F^T: task (step s, half kh, 32-column block jb)
      for (int task = warp; task < 8 * nj; task += 8) {
        const int s = task / (2 * nj), kh = (task / nj) & 1, jb = task % nj;
        const int j = 32 * jb + lane;
        if (j < Nn) {
          float f[8];
          const int64_t r0 = 64 * (int64_t)c + 16 * s + 8 * kh;
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) f[kk] = j < jreal ? __ldg(Fx + (r0 + kk) * jreal + j) : 0.f;
          const uint32_t base = ptx::smem_u32(sF) + (uint32_t)s * fstep + (uint32_t)(j >> 3) * 256u +
                                (uint32_t)kh * 128u + (uint32_t)(j & 7) * 16u;
          split_store8(f, base, (uint32_t)Nn * 32u, 2u * (uint32_t)Nn * 32u);
        }
      }
      ptx::fence_proxy_async_smem();
      ptx::tc_fence_before();
      __syncthreads();
      if (threadIdx.x == 0) {
        ptx::tc_fence_after();
        for (int s = 0; s < 4; ++s)
          mma3(tmem, ptx::smem_u32(sA) + (uint32_t)s * kPjAStep, kPjAStep / 3, 128u, 256u,
               ptx::smem_u32(sF) + (uint32_t)s * fstep, 256u, Nn, c == 0 && s == 0);
      }
      if (!commit_wait(&bar, phase, &s_abort)) {
        s_abort = 1;
        atomicOr(&g_bltc_error, kErrBlocking);
      }
      __syncthreads();
      if (s_abort) break;
    }
    if (s_abort) break;
    // epilogue: warps 0-3, lane m = B's real column; P[m][j] = the three
    // blocks' sum; the odd column's values come from the neighbouring lane
    if (warp < 4) {
      const int m = 32 * warp + lane;
      const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16);
      float2* Cx = Cc + x * (int64_t)nbasis * R;
      for (int c0 = 0; c0 < jreal; c0 += 8) {
        float u0[8], u1[8], u2[8], p[8], o[8];
        ptx::tmem_ld8_sync(ta + (uint32_t)c0, u0);
        ptx::tmem_ld8_sync(ta + (uint32_t)(Nn + c0), u1);
        ptx::tmem_ld8_sync(ta + (uint32_t)(2 * Nn + c0), u2);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          p[e] = u0[e] + u1[e] + u2[e];
          o[e] = __shfl_xor_sync(0xffffffffu, p[e], 1);
        }
        if ((m & 1) == 0 && m < kreal) {
          // row a = m / 2: C[a][r] = (P0[2r] + P1[2r+1]) + i (P0[2r+1] - P1[2r])
          float* dst = reinterpret_cast<float*>(Cx + (m >> 1) * R) + c0;
          *reinterpret_cast<float4*>(dst) =
              make_float4(p[0] + o[1], p[1] - o[0], p[2] + o[3], p[3] - o[2]);
          *reinterpret_cast<float4*>(dst + 4) =
              make_float4(p[4] + o[5], p[5] - o[4], p[6] + o[7], p[7] - o[6]);
        }
      }
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
  }
  if (threadIdx.x == 0) {
    ptx::mma_commit(&done);
    volatile int never = 0;
    ptx::mbar_wait(&done, 0, &never);
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, tcols);
  }
}

// dynamic shared memory that also caps the CTAs per SM so that their tensor
// memory fits the SM's 512 columns
size_t blocking_smem(size_t need, uint32_t tcols) {
  const int max_ctas = (int)(512 / tcols) > 3 ? 3 : (int)(512 / tcols);
  const size_t per_sm = 227 * 1024;
  const size_t floor_bytes = per_sm / (size_t)(max_ctas + 1) + 1024;
  return need > floor_bytes ? need : floor_bytes;
}

}  // namespace

bool blocking_tc_applies(const void* basis, const void* in, const void* out, int64_t nblk,
                         int vb, int nbasis, int R, int dtype) {
  auto a16 = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
  return g_block_tc_mode == 1 && dtype == MRHS_C64 && nblk >= 1 && vb >= 64 && vb % 64 == 0 &&
         nbasis >= 8 && nbasis <= 64 && nbasis % 8 == 0 && R >= 4 && R <= 32 && R % 4 == 0 &&
         a16(basis) && a16(in) && a16(out);
}

int blocking_tc(bool project, const void* basis, const void* in, void* out, int64_t nblk, int vb,
                int nbasis, int R, cudaStream_t s) {
  const int Nn = (2 * R + 15) & ~15, K16 = (2 * nbasis + 15) & ~15;
  const uint32_t tcols = 3 * Nn <= 128 ? 128u : 256u;
  const int max_ctas = (int)(512 / tcols) > 3 ? 3 : (int)(512 / tcols);
  const int64_t cap = (int64_t)num_sms() * max_ctas;
  const unsigned grid = (unsigned)(nblk < cap ? nblk : cap);
  if (project) {
    const size_t smem = blocking_smem(4 * (size_t)kPjAStep + 4 * (size_t)(3 * Nn) * 32, tcols);
    MRHS_CUDA_TRY(cudaFuncSetAttribute(k_project_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    { k_project_tc<<<grid, kBlThreads, smem, s>>>((const float2*)basis, (const float2*)in,
                                                  (float2*)out, nblk, vb, nbasis, R); count_launch(); }
  } else {
    const size_t bbytes = ((size_t)(3 * Nn) * K16 * 2 + 1023) & ~(size_t)1023;
    const size_t smem = blocking_smem(bbytes + kPrA, tcols);
    MRHS_CUDA_TRY(cudaFuncSetAttribute(k_promote_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    { k_promote_tc<<<grid, kBlThreads, smem, s>>>((const float2*)basis, (const float2*)in,
                                                  (float2*)out, nblk, vb, nbasis, R); count_launch(); }
  }
  MRHS_CUDA_TRY(cudaGetLastError());
  return MRHS_OK;
}

unsigned bltc_read_and_clear_error() {
  unsigned v = 0, z = 0;
  cudaMemcpyFromSymbol(&v, g_bltc_error, sizeof(v));
  cudaMemcpyToSymbol(g_bltc_error, &z, sizeof(z));
  return v;
}

}  // namespace mrhs
