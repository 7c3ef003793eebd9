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
// launch, with no pointer lists.
//   promote: C(x) is staged in shared memory; a thread owns one fine row s
//            and a chunk of RC right-hand sides and walks its basis row
//            (contiguous, cached in L1 across a) against the staged C.
//   project: F(x) is staged in shared memory in tiles of rows; a thread owns
//            one basis column a and up to K right-hand sides; for every row s
//            the CTA reads the basis row coalesced (consecutive a).
// FP64 runs on the FP64 pipe, complex64 on the FP32 pipes.
#include "internal.cuh"

namespace mrhs {
namespace {

constexpr int kThreads = 256;
constexpr int kTileRows = 32;    // fine rows of F(x) staged per step (project)

template <typename C, int RC>
__global__ void __launch_bounds__(kThreads)
    k_promote(const C* __restrict__ basis, const C* __restrict__ Cc, C* __restrict__ F,
              int64_t nblk, int vb, int nbasis, int R) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sC = reinterpret_cast<C*>(smem_raw);      // [nbasis][R]
  const int nchunk = (R + RC - 1) / RC;
  for (int64_t x = blockIdx.x; x < nblk; x += gridDim.x) {
    __syncthreads();
    for (int i = threadIdx.x; i < nbasis * R; i += kThreads) sC[i] = Cc[x * nbasis * R + i];
    __syncthreads();
    const C* Bx = basis + x * (int64_t)vb * nbasis;
    C* Fx = F + x * (int64_t)vb * R;
    for (int w = threadIdx.x; w < vb * nchunk; w += kThreads) {
      const int s = w / nchunk, r0 = (w % nchunk) * RC;
      C acc[RC];
#pragma unroll
      for (int j = 0; j < RC; ++j) acc[j] = czero<C>();
      const C* brow = Bx + (int64_t)s * nbasis;
      for (int a = 0; a < nbasis; ++a) {
        const C b = brow[a];
#pragma unroll
        for (int j = 0; j < RC; ++j)
          if (r0 + j < R) acc[j] = cfma(b, sC[a * R + r0 + j], acc[j]);
      }
#pragma unroll
      for (int j = 0; j < RC; ++j)
        if (r0 + j < R) Fx[(int64_t)s * R + r0 + j] = acc[j];
    }
  }
}

template <typename C, int K>
__global__ void __launch_bounds__(kThreads)
    k_project(const C* __restrict__ basis, const C* __restrict__ F, C* __restrict__ Cc,
              int64_t nblk, int vb, int nbasis, int R) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sF = reinterpret_cast<C*>(smem_raw);      // [kTileRows][R]
  const int groups = kThreads / nbasis;        // right-hand-side groups
  const int a = threadIdx.x % nbasis, g = threadIdx.x / nbasis;
  const bool active = g < groups;
  for (int64_t x = blockIdx.x; x < nblk; x += gridDim.x) {
    const C* Bx = basis + x * (int64_t)vb * nbasis;
    const C* Fx = F + x * (int64_t)vb * R;
    C acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = czero<C>();
    for (int s0 = 0; s0 < vb; s0 += kTileRows) {
      const int rows = (vb - s0) < kTileRows ? (vb - s0) : kTileRows;
      __syncthreads();
      for (int i = threadIdx.x; i < rows * R; i += kThreads) sF[i] = Fx[(int64_t)s0 * R + i];
      __syncthreads();
      if (active) {
        for (int s = 0; s < rows; ++s) {
          const C b = Bx[(int64_t)(s0 + s) * nbasis + a];
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const int r = g + k * groups;
            if (r < R) acc[k] = cfma_conj(b, sF[s * R + r], acc[k]);
          }
        }
      }
    }
    if (active) {
      C* Cx = Cc + x * (int64_t)nbasis * R;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int r = g + k * groups;
        if (r < R) Cx[a * R + r] = acc[k];
      }
    }
  }
}

template <typename C>
int promote_t(const void* basis, const void* Cc, void* F, int64_t nblk, int vb, int nbasis, int R,
              cudaStream_t s) {
  const size_t smem = sizeof(C) * (size_t)nbasis * R;
  const int64_t cap = (int64_t)num_sms() * 8;
  const unsigned grid = (unsigned)(nblk < cap ? nblk : cap);
  auto go = [&](auto kern) -> int {
    MRHS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    { kern<<<grid, kThreads, smem, s>>>((const C*)basis, (const C*)Cc, (C*)F, nblk, vb, nbasis, R); count_launch(); }
    MRHS_CUDA_TRY(cudaGetLastError());
    return MRHS_OK;
  };
  if (R <= 4) return go(k_promote<C, 4>);
  if (R <= 8) return go(k_promote<C, 8>);
  return go(k_promote<C, 16>);
}

template <typename C>
int project_t(const void* basis, const void* F, void* Cc, int64_t nblk, int vb, int nbasis, int R,
              cudaStream_t s) {
  const size_t smem = sizeof(C) * (size_t)kTileRows * R;
  const int64_t cap = (int64_t)num_sms() * 8;
  const unsigned grid = (unsigned)(nblk < cap ? nblk : cap);
  const int groups = kThreads / nbasis;
  const int K = (R + groups - 1) / groups;
  auto go = [&](auto kern) -> int {
    MRHS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    { kern<<<grid, kThreads, smem, s>>>((const C*)basis, (const C*)F, (C*)Cc, nblk, vb, nbasis, R); count_launch(); }
    MRHS_CUDA_TRY(cudaGetLastError());
    return MRHS_OK;
  };
  if (K <= 1) return go(k_project<C, 1>);
  if (K <= 2) return go(k_project<C, 2>);
  if (K <= 4) return go(k_project<C, 4>);
  if (K <= 8) return go(k_project<C, 8>);
  if (K <= 16) return go(k_project<C, 16>);
  return fail(MRHS_ERR_INVALID_ARG, "block_project: nrhs too large for n_basis");
}

}  // namespace

int blocking(bool project, const void* basis, const void* in, void* out, int64_t nblk, int vb,
             int nbasis, int R, int dtype, cudaStream_t s) {
  if (project)
    return dtype == MRHS_C128 ? project_t<double2>(basis, in, out, nblk, vb, nbasis, R, s)
                              : project_t<float2>(basis, in, out, nblk, vb, nbasis, R, s);
  return dtype == MRHS_C128 ? promote_t<double2>(basis, in, out, nblk, vb, nbasis, R, s)
                            : promote_t<float2>(basis, in, out, nblk, vb, nbasis, R, s);
}

}  // namespace mrhs
