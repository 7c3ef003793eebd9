// FP64 / FP32 coarse operator on the CUDA cores (FMA pipes).
//
// Y(x) = sum_p A_p(x) X(x + delta_p)           (Sec. 2.6, "Applying the coarse
// operator": one GEMM per site and stencil point, batch = coarse volume),
// and the adjoint Y(x) = sum_p A_p(x - delta_p)^dagger X(x - delta_p).
//
// B300 design: one CTA per site (grid-stride), the stencil point's nb x nb
// block and the neighbour's nb x nrhs block staged in shared memory, so every
// coefficient is read from HBM once per application and reused for all nrhs
// right-hand sides (the "fictitious fifth dimension" of Sec. 2).  Thread t
// owns one RHS column r = t % nrhs and rows a = t / nrhs + k * (T / nrhs), so
// the neighbour value X[b][r] is loaded once per b and reused for all its
// rows while A[a][b] is a warp-wide broadcast.  On B300 the FP64 variant is
// bound by the FP64 pipe, the FP32 variant by FFMA issue.
#include "internal.cuh"

namespace mrhs {
namespace {

template <typename C, int OPT>
__global__ void __launch_bounds__(256) k_op_simt(const C* __restrict__ A, const C* __restrict__ X,
                                                 C* __restrict__ Y, const int32_t* __restrict__ nbr,
                                                 int64_t V, int nb, int npts, int R, int dag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sA = reinterpret_cast<C*>(smem_raw);
  C* sX = sA + nb * nb;
  const int T = blockDim.x;
  const int rows_per_pass = T / R;
  const int r = threadIdx.x % R;
  const int a0 = threadIdx.x / R;
  const bool lane_ok = threadIdx.x < rows_per_pass * R;
  for (int64_t x = blockIdx.x; x < V; x += gridDim.x) {
    C acc[OPT];
#pragma unroll
    for (int k = 0; k < OPT; ++k) acc[k] = czero<C>();
    for (int p = 0; p < npts; ++p) {
      const int64_t y = nbr[(int64_t)p * V + x];
      const C* Ap = A + ((dag ? y : x) * npts + p) * (int64_t)nb * nb;
      const C* Xp = X + y * (int64_t)nb * R;
      __syncthreads();
      for (int i = threadIdx.x; i < nb * nb; i += T) sA[i] = Ap[i];
      for (int i = threadIdx.x; i < nb * R; i += T) sX[i] = Xp[i];
      __syncthreads();
      if (lane_ok) {
        if (!dag) {
          for (int b = 0; b < nb; ++b) {
            const C xv = sX[b * R + r];
#pragma unroll
            for (int k = 0; k < OPT; ++k) {
              const int a = a0 + k * rows_per_pass;
              if (a < nb) acc[k] = cfma(sA[a * nb + b], xv, acc[k]);
            }
          }
        } else {
          for (int b = 0; b < nb; ++b) {
            const C xv = sX[b * R + r];
#pragma unroll
            for (int k = 0; k < OPT; ++k) {
              const int a = a0 + k * rows_per_pass;
              if (a < nb) acc[k] = cfma_conj(sA[b * nb + a], xv, acc[k]);
            }
          }
        }
      }
    }
    if (lane_ok) {
      C* Yx = Y + x * (int64_t)nb * R;
#pragma unroll
      for (int k = 0; k < OPT; ++k) {
        const int a = a0 + k * rows_per_pass;
        if (a < nb) Yx[a * R + r] = acc[k];
      }
    }
  }
}

template <typename C, int OPT>
int launch(const C* A, const C* X, C* Y, const int32_t* nbr, int64_t V, int nb, int npts, int R,
           int dag, int threads, cudaStream_t s) {
  const size_t smem = sizeof(C) * ((size_t)nb * nb + (size_t)nb * R);
  auto kern = k_op_simt<C, OPT>;
  MRHS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t grid = V < 1048576 ? V : 1048576;
  { kern<<<(unsigned)grid, threads, smem, s>>>(A, X, Y, nbr, V, nb, npts, R, dag); ::mrhs::count_launch(); }
  MRHS_CUDA_TRY(cudaGetLastError());
  return MRHS_OK;
}

template <typename C>
int dispatch(const C* A, const C* X, C* Y, const int32_t* nbr, int64_t V, int nb, int npts, int R,
             int dag, cudaStream_t s) {
  int rows = 256 / R;
  if (rows < 1) rows = 1;
  const int threads = rows * R;
  const int need = (nb + rows - 1) / rows;
  if (need <= 1) return launch<C, 1>(A, X, Y, nbr, V, nb, npts, R, dag, threads, s);
  if (need <= 2) return launch<C, 2>(A, X, Y, nbr, V, nb, npts, R, dag, threads, s);
  if (need <= 4) return launch<C, 4>(A, X, Y, nbr, V, nb, npts, R, dag, threads, s);
  if (need <= 6) return launch<C, 6>(A, X, Y, nbr, V, nb, npts, R, dag, threads, s);
  if (need <= 8) return launch<C, 8>(A, X, Y, nbr, V, nb, npts, R, dag, threads, s);
  if (need <= 16) return launch<C, 16>(A, X, Y, nbr, V, nb, npts, R, dag, threads, s);
  return fail(MRHS_ERR_INVALID_ARG, "simt apply: nb too large for nrhs");
}

}  // namespace

int simt_apply(mrhs_op_s* op, int prec, bool dag, const void* X, void* Y, int nrhs,
               cudaStream_t s) {
  const int32_t* nbr = dag ? op->nbr_bwd : op->nbr_fwd;
  int st = MRHS_ERR_UNSUPPORTED;
  timer_mark(op, prec, s);
  if (prec == MRHS_PREC_FP64)
    st = dispatch<double2>(op->a64, (const double2*)X, (double2*)Y, nbr, op->V, op->nb, op->npts,
                           nrhs, dag ? 1 : 0, s);
  else if (prec == MRHS_PREC_FP32)
    st = dispatch<float2>(op->a32, (const float2*)X, (float2*)Y, nbr, op->V, op->nb, op->npts,
                          nrhs, dag ? 1 : 0, s);
  timer_mark(op, prec, s);
  if (st == MRHS_ERR_UNSUPPORTED) return fail(st, "simt apply: precision");
  return st;
}

}  // namespace mrhs
