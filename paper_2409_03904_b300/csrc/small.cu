// Small Hermitian factorisations of block CG (Fig. 2), one CTA, FP64.
//
// factor: G (r x r, Hermitian part taken) = S^dagger S with S upper triangular
// and a positive real diagonal when every pivot exceeds tau * max_i G_ii;
// otherwise a diagonally pivoted Cholesky stopped at numerical rank k, so
// that T = Q S with S k x r (rows k..r-1 zero) and W (r x r, columns k..r-1
// zero) with T W = Q.  A leading-block width k_in (from the previous
// iteration) restricts the factorisation to G[0:k_in, 0:k_in].
//
// r <= 64: right-looking elimination with the trailing block in shared
// memory, one sync per pivot; the triangular inverse by one back
// substitution per column and thread.
#include "internal.cuh"
#include "small.cuh"

namespace mrhs {

namespace {

__global__ void k_factor(const double2* G, double2* S, double2* W, int32_t* rank, int r,
                         double tau) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* sA = reinterpret_cast<double2*>(smem_raw);
  double2* sS = sA + r * r;
  double2* sW = sS + r * r;
  __shared__ int perm[MRHS_MAX_RHS];
  const int k = factor_block(G, r, r, r, tau, sA, sS, sW, perm, S, W);
  if (threadIdx.x == 0 && rank) *rank = k;
}

}  // namespace

size_t factor_smem_bytes(int r) { return 3 * sizeof(double2) * (size_t)r * r; }

int factor(const double2* G, double2* S, double2* W, int32_t* rank, int r, double tau,
           cudaStream_t s) {
  const size_t smem = factor_smem_bytes(r);
  MRHS_CUDA_TRY(cudaFuncSetAttribute(k_factor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
  { k_factor<<<1, 256, smem, s>>>(G, S, W, rank, r, tau); ::mrhs::count_launch(); }
  MRHS_CUDA_TRY(cudaGetLastError());
  return MRHS_OK;
}

}  // namespace mrhs
