// Block project / promote between fine and coarse degrees of freedom
// (Sec. 2.5.1, "Transfer between grids"): one small complex GEMM per coarse site x,
//   project:  C(x) = B(x)^dagger F(x)   (n_basis x nrhs)
//   promote:  F(x) = B(x) C(x)          (v_block x nrhs)
// with the basis B [n_blocks][v_block][n_basis], fine vectors
// [n_blocks][v_block][nrhs] and coarse vectors [n_blocks][n_basis][nrhs].
//
// The paper issues these as vendor batched GEMMs over pointer lists; here one
// CTA takes one block at a time (grid-stride over blocks), so the basis --
// the only large operand -- streams from HBM once per call, in a single
// launch, with no pointer lists.  Both kernels block in registers (a thread
// owns a small tile of outputs and reuses each loaded value across it), so
// complex64 runs near the memory roofline; FP64 runs on the FP64 pipe.
#include "internal.cuh"

namespace mrhs {
namespace {

constexpr int kThreads = 256;

// promote: thread tile of TS fine rows x TR right-hand sides; C(x) staged in
// shared memory; a thread walks its rows' basis entries four at a time (two
// 16-byte loads per row for complex64) against the staged C, so every
// multiply-add has its operands in registers.
template <typename C, int TS, int TR>
__global__ void __launch_bounds__(kThreads)
    k_promote(const C* __restrict__ basis, const C* __restrict__ Cc, C* __restrict__ F,
              int64_t nblk, int vb, int nbasis, int R) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sC = reinterpret_cast<C*>(smem_raw);      // [nbasis][R]
  const int ns = (vb + TS - 1) / TS, nr = (R + TR - 1) / TR, jobs = ns * nr;
  for (int64_t x = blockIdx.x; x < nblk; x += gridDim.x) {
    __syncthreads();
    for (int i = threadIdx.x; i < nbasis * R; i += kThreads) sC[i] = Cc[x * nbasis * R + i];
    __syncthreads();
    const C* Bx = basis + x * (int64_t)vb * nbasis;
    C* Fx = F + x * (int64_t)vb * R;
    for (int job = threadIdx.x; job < jobs; job += kThreads) {
      const int s0 = (job / nr) * TS, r0 = (job % nr) * TR;
      C acc[TS][TR];
#pragma unroll
      for (int i = 0; i < TS; ++i)
#pragma unroll
        for (int j = 0; j < TR; ++j) acc[i][j] = czero<C>();
      // four basis entries of each of the thread's rows per step (contiguous
      // in memory), then the tail one at a time
      int a = 0;
      for (; a + 4 <= nbasis; a += 4) {
        C b[TS][4];
#pragma unroll
        for (int i = 0; i < TS; ++i)
#pragma unroll
          for (int q = 0; q < 4; ++q)
            b[i][q] = (s0 + i < vb) ? __ldg(&Bx[(int64_t)(s0 + i) * nbasis + a + q]) : czero<C>();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          C c[TR];
#pragma unroll
          for (int j = 0; j < TR; ++j) c[j] = (r0 + j < R) ? sC[(a + q) * R + r0 + j] : czero<C>();
#pragma unroll
          for (int i = 0; i < TS; ++i)
#pragma unroll
            for (int j = 0; j < TR; ++j) acc[i][j] = cfma(b[i][q], c[j], acc[i][j]);
        }
      }
      for (; a < nbasis; ++a) {
        C b[TS], c[TR];
#pragma unroll
        for (int i = 0; i < TS; ++i)
          b[i] = (s0 + i < vb) ? __ldg(&Bx[(int64_t)(s0 + i) * nbasis + a]) : czero<C>();
#pragma unroll
        for (int j = 0; j < TR; ++j) c[j] = (r0 + j < R) ? sC[a * R + r0 + j] : czero<C>();
#pragma unroll
        for (int i = 0; i < TS; ++i)
#pragma unroll
          for (int j = 0; j < TR; ++j) acc[i][j] = cfma(b[i], c[j], acc[i][j]);
      }
#pragma unroll
      for (int i = 0; i < TS; ++i)
#pragma unroll
        for (int j = 0; j < TR; ++j)
          if (s0 + i < vb && r0 + j < R) Fx[(int64_t)(s0 + i) * R + r0 + j] = acc[i][j];
    }
  }
}

// project: thread tile of TA basis columns x TR right-hand sides over a
// share of the block's fine rows (the rows split into KS groups when the
// tiles leave threads idle), partial sums combined in shared memory in a
// fixed order.  Per fine row a thread reads TA consecutive basis entries
// (coalesced across the warp) and TR entries of F, then does TA x TR
// multiply-adds from registers.
template <typename C, int TA, int TR>
__global__ void __launch_bounds__(kThreads)
    k_project(const C* __restrict__ basis, const C* __restrict__ F, C* __restrict__ Cc,
              int64_t nblk, int vb, int nbasis, int R) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sP = reinterpret_cast<C*>(smem_raw);      // [KS][jobs][TA * TR] partial sums
  const int na = (nbasis + TA - 1) / TA, nr = (R + TR - 1) / TR, jobs = na * nr;
  int ks = kThreads / jobs;
  if (ks < 1) ks = 1;
  const int tpj = jobs < kThreads ? jobs : kThreads;     // threads per row group
  for (int64_t x = blockIdx.x; x < nblk; x += gridDim.x) {
    const C* Bx = basis + x * (int64_t)vb * nbasis;
    const C* Fx = F + x * (int64_t)vb * R;
    __syncthreads();
    const int g = threadIdx.x / tpj;
    if (g < ks) {
      for (int job = threadIdx.x % tpj; job < jobs; job += tpj) {
        const int a0 = (job % na) * TA, r0 = (job / na) * TR;
        C acc[TA][TR];
#pragma unroll
        for (int i = 0; i < TA; ++i)
#pragma unroll
          for (int j = 0; j < TR; ++j) acc[i][j] = czero<C>();
        for (int s = g; s < vb; s += ks) {
          C b[TA], f[TR];
#pragma unroll
          for (int i = 0; i < TA; ++i)
            b[i] = (a0 + i < nbasis) ? __ldg(&Bx[(int64_t)s * nbasis + a0 + i]) : czero<C>();
#pragma unroll
          for (int j = 0; j < TR; ++j)
            f[j] = (r0 + j < R) ? __ldg(&Fx[(int64_t)s * R + r0 + j]) : czero<C>();
#pragma unroll
          for (int i = 0; i < TA; ++i)
#pragma unroll
            for (int j = 0; j < TR; ++j) acc[i][j] = cfma_conj(b[i], f[j], acc[i][j]);
        }
        C* dst = sP + ((int64_t)g * jobs + job) * (TA * TR);
#pragma unroll
        for (int i = 0; i < TA; ++i)
#pragma unroll
          for (int j = 0; j < TR; ++j) dst[i * TR + j] = acc[i][j];
      }
    }
    __syncthreads();
    // combine the row groups in order and write C(x)
    C* Cx = Cc + x * (int64_t)nbasis * R;
    for (int e = threadIdx.x; e < jobs * TA * TR; e += kThreads) {
      const int job = e / (TA * TR), k = e % (TA * TR), i = k / TR, j = k % TR;
      const int a = (job % na) * TA + i, r = (job / na) * TR + j;
      if (a >= nbasis || r >= R) continue;
      C v = sP[(int64_t)job * (TA * TR) + k];
      for (int gg = 1; gg < ks; ++gg) {
        const C w = sP[((int64_t)gg * jobs + job) * (TA * TR) + k];
        v.x += w.x;
        v.y += w.y;
      }
      Cx[a * R + r] = v;
    }
  }
}

template <typename C>
int promote_t(const void* basis, const void* Cc, void* F, int64_t nblk, int vb, int nbasis, int R,
              cudaStream_t s) {
  const size_t smem = sizeof(C) * (size_t)nbasis * R;
  const int64_t cap = (int64_t)num_sms() * 4;
  const unsigned grid = (unsigned)(nblk < cap ? nblk : cap);
  auto go = [&](auto kern) -> int {
    MRHS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    { kern<<<grid, kThreads, smem, s>>>((const C*)basis, (const C*)Cc, (C*)F, nblk, vb, nbasis, R); count_launch(); }
    MRHS_CUDA_TRY(cudaGetLastError());
    return MRHS_OK;
  };
  if (R <= 2) return go(k_promote<C, 4, 2>);
  if (R <= 4) return go(k_promote<C, 4, 4>);
  if (R % 3 == 0 && R <= 12) return go(k_promote<C, 4, 3>);
  return go(k_promote<C, 4, 4>);
}

template <typename C>
int project_t(const void* basis, const void* F, void* Cc, int64_t nblk, int vb, int nbasis, int R,
              cudaStream_t s) {
  const int64_t cap = (int64_t)num_sms() * 4;
  const unsigned grid = (unsigned)(nblk < cap ? nblk : cap);
  auto go = [&](auto kern, int TA, int TR) -> int {
    const int jobs = ((nbasis + TA - 1) / TA) * ((R + TR - 1) / TR);
    const int ks = jobs < kThreads ? kThreads / jobs : 1;
    const size_t smem = sizeof(C) * (size_t)ks * jobs * TA * TR;
    MRHS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    { kern<<<grid, kThreads, smem, s>>>((const C*)basis, (const C*)F, (C*)Cc, nblk, vb, nbasis, R); count_launch(); }
    MRHS_CUDA_TRY(cudaGetLastError());
    return MRHS_OK;
  };
  if (R <= 2) return go(k_project<C, 4, 2>, 4, 2);
  if (R % 3 == 0 && R <= 12) return go(k_project<C, 4, 3>, 4, 3);
  return go(k_project<C, 4, 4>, 4, 4);
}

}  // namespace

int blocking(bool project, const void* basis, const void* in, void* out, int64_t nblk, int vb,
             int nbasis, int R, int dtype, cudaStream_t s) {
  if (blocking_tc_applies(basis, in, out, nblk, vb, nbasis, R, dtype))   // blocking_tc.cu
    return blocking_tc(project, basis, in, out, nblk, vb, nbasis, R, s);
  if (project)
    return dtype == MRHS_C128 ? project_t<double2>(basis, in, out, nblk, vb, nbasis, R, s)
                              : project_t<float2>(basis, in, out, nblk, vb, nbasis, R, s);
  return dtype == MRHS_C128 ? promote_t<double2>(basis, in, out, nblk, vb, nbasis, R, s)
                            : promote_t<float2>(basis, in, out, nblk, vb, nbasis, R, s);
}

}  // namespace mrhs
