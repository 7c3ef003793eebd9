// Stencil-projected outer product for the adjoints of the coarse operator
// and of the solve: GA_p(x) = alpha * sum_r G(x)[a][r] conj(X(x + delta_p)[b][r]).
//
// For Y = H X, grad A_p(x) = grad Y(x) X(x + delta_p)^dagger (alpha = 1); for
// X = H^-1 B, grad A_p(x) = -grad B(x) X(x + delta_p)^dagger (alpha = -1),
// both following from dY = dA X + A dX.  The result has the coefficients'
// shape, so this is a batched outer-product GEMM with K = nrhs that writes
// V * npts * nb^2 complex128 values (bound by that write at large nb).
// One CTA per (site, stencil point), G(x) and X(x + delta_p) staged in
// shared memory, one output entry per thread and step, FP64 accumulation.
#include "internal.cuh"

namespace mrhs {
namespace {

template <typename C>
__global__ void __launch_bounds__(256)
    k_outer(const C* __restrict__ G, const C* __restrict__ X, double2* __restrict__ GA,
            const int32_t* __restrict__ nbr, int64_t V, int nb, int npts, int R, double alpha) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* sG = reinterpret_cast<double2*>(smem_raw);
  double2* sX = sG + nb * R;
  const int64_t x = blockIdx.x;
  const int p = blockIdx.y;
  const int64_t y = nbr[(int64_t)p * V + x];
  for (int i = threadIdx.x; i < nb * R; i += blockDim.x) {
    const C g = G[x * nb * R + i], v = X[y * nb * R + i];
    sG[i] = make_double2((double)g.x, (double)g.y);
    sX[i] = make_double2((double)v.x, (double)v.y);
  }
  __syncthreads();
  double2* out = GA + ((x * npts + p) * (int64_t)nb) * nb;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int a = e / nb, b = e % nb;
    double2 acc = make_double2(0.0, 0.0);
    for (int r = 0; r < R; ++r) acc = cfma_conj(sX[b * R + r], sG[a * R + r], acc);
    out[e] = make_double2(alpha * acc.x, alpha * acc.y);
  }
}

}  // namespace

int outer(const mrhs_op_s* op, const void* G, const void* X, double2* GA, double alpha, int R,
          int dtype, cudaStream_t s) {
  const size_t smem = 2 * sizeof(double2) * (size_t)op->nb * R;
  dim3 grid((unsigned)op->V, (unsigned)op->npts);
  if (dtype == MRHS_C128) {
    MRHS_CUDA_TRY(cudaFuncSetAttribute(k_outer<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    { k_outer<double2><<<grid, 256, smem, s>>>((const double2*)G, (const double2*)X, GA,
                                               op->nbr_fwd, op->V, op->nb, op->npts, R, alpha); ::mrhs::count_launch(); }
  } else {
    MRHS_CUDA_TRY(cudaFuncSetAttribute(k_outer<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    { k_outer<float2><<<grid, 256, smem, s>>>((const float2*)G, (const float2*)X, GA,
                                              op->nbr_fwd, op->V, op->nb, op->npts, R, alpha); ::mrhs::count_launch(); }
  }
  MRHS_CUDA_TRY(cudaGetLastError());
  return MRHS_OK;
}

}  // namespace mrhs
