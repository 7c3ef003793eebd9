// FP64 / FP32 coarse operator on the CUDA cores (FMA pipes).
//
// Y(x) = sum_p A_p(x) X(x + delta_p)           (Sec. 2.6, "Applying the coarse
// operator": one GEMM per site and stencil point, batch = coarse volume),
// and the adjoint Y(x) = sum_p A_p(x - delta_p)^dagger X(x - delta_p).
//
// B300 design: one CTA per site (grid-stride), the stencil point's nb x nb
// block and the neighbour's nb x nrhs block staged in shared memory, so every
// coefficient is read from HBM once per application and reused for all nrhs
// right-hand sides (the extra dimension over right-hand sides of Sec. 2).  Thread t
// owns one RHS column r = t % nrhs and rows a = t / nrhs + k * (T / nrhs), so
// the neighbour value X[b][r] is loaded once per b and reused for all its
// rows while A[a][b] is a warp-wide broadcast.  On B300 the FP64 variant is
// bound by the FP64 pipe, the FP32 variant by shared-memory loads.
//
// The FP64 variant forms each complex product from three real products
// (Gauss / Karatsuba): with A = Ar + i Ai and x = Br + i Bi it accumulates
// T1 = sum Ar Br, T2 = sum Ai Bi and T3 = sum (Ar + Ai)(Br + Bi), and writes
// Re = T1 - T2, Im = T3 - T1 - T2 (for the adjoint, conj(A) x: T3 = sum
// (Ar - Ai)(Br + Bi), Re = T1 + T2, Im = T3 - T1 + T2).  Ar +- Ai is formed
// once per coefficient when it is staged, Br + Bi once per neighbour value,
// so the FP64 pipe does three fused multiply-adds per complex product
// instead of four.
//
// DF32 ("double-float"): the same FP64 coefficients and vectors, each value
// split on staging into an FP32 pair hi + lo (hi = fl32(v), lo = fl32(v - hi)),
// the three real products of the Gauss form computed on the FP32 pipes,
// whose issue rate on B300 is about sixty times the FP64 pipe's.  A product
// of pairs is formed exactly up to the lo x lo term with one FMA (Dekker /
// Knuth error-free product: p = ah bh, e = fma(ah, bh, -p) + ah bl + al bh);
// p joins the running hi sum through an error-free two-sum whose rounding
// error goes, with e, into the running lo sum; after each stencil point the
// pair is renormalised.  Sums are carried to about 2^-44 relative, enough for
// residuals far below tol / kappa (the outer defect correction's need).
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

template <int OPT>
__global__ void __launch_bounds__(256) k_op_fp64_k3(const double2* __restrict__ A,
                                                    const double2* __restrict__ X,
                                                    double2* __restrict__ Y,
                                                    const int32_t* __restrict__ nbr, int64_t V,
                                                    int nb, int npts, int R, int dag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* sA = reinterpret_cast<double2*>(smem_raw);
  double2* sX = sA + nb * nb;                 // (Br, Bi)
  double* sS = reinterpret_cast<double*>(sX + nb * R);   // Ar +- Ai
  double* sXs = sS + nb * nb;                 // Br + Bi
  const int T = blockDim.x;
  const int rows_per_pass = T / R;
  const int r = threadIdx.x % R;
  const int a0 = threadIdx.x / R;
  const bool lane_ok = threadIdx.x < rows_per_pass * R;
  const double sg = dag ? -1.0 : 1.0;
  for (int64_t x = blockIdx.x; x < V; x += gridDim.x) {
    double t1[OPT], t2[OPT], t3[OPT];
#pragma unroll
    for (int k = 0; k < OPT; ++k) t1[k] = t2[k] = t3[k] = 0.0;
    for (int p = 0; p < npts; ++p) {
      const int64_t y = nbr[(int64_t)p * V + x];
      const double2* Ap = A + ((dag ? y : x) * npts + p) * (int64_t)nb * nb;
      const double2* Xp = X + y * (int64_t)nb * R;
      __syncthreads();
      for (int i = threadIdx.x; i < nb * nb; i += T) {
        const double2 v = Ap[i];
        sA[i] = v;
        sS[i] = v.x + sg * v.y;
      }
      for (int i = threadIdx.x; i < nb * R; i += T) {
        const double2 v = Xp[i];
        sX[i] = v;
        sXs[i] = v.x + v.y;
      }
      __syncthreads();
      if (lane_ok) {
        // forward: coefficient (a, b) at a * nb + b; adjoint: conj of (b, a)
        const int sa = dag ? 1 : nb, sb = dag ? nb : 1;
        for (int b = 0; b < nb; ++b) {
          const double2 xv = sX[b * R + r];
          const double xs = sXs[b * R + r];
#pragma unroll
          for (int k = 0; k < OPT; ++k) {
            const int a = a0 + k * rows_per_pass;
            if (a < nb) {
              const int e = a * sa + b * sb;
              const double2 av = sA[e];
              t1[k] = fma(av.x, xv.x, t1[k]);
              t2[k] = fma(av.y, xv.y, t2[k]);
              t3[k] = fma(sS[e], xs, t3[k]);
            }
          }
        }
      }
    }
    if (lane_ok) {
      double2* Yx = Y + x * (int64_t)nb * R;
#pragma unroll
      for (int k = 0; k < OPT; ++k) {
        const int a = a0 + k * rows_per_pass;
        if (a < nb)
          Yx[a * R + r] = dag ? make_double2(t1[k] + t2[k], t3[k] - t1[k] + t2[k])
                              : make_double2(t1[k] - t2[k], t3[k] - t1[k] - t2[k]);
      }
    }
  }
}

template <int OPT>
int launch_k3(const double2* A, const double2* X, double2* Y, const int32_t* nbr, int64_t V,
              int nb, int npts, int R, int dag, int threads, cudaStream_t s) {
  const size_t smem = sizeof(double2) * ((size_t)nb * nb + (size_t)nb * R) +
                      sizeof(double) * ((size_t)nb * nb + (size_t)nb * R);
  auto kern = k_op_fp64_k3<OPT>;
  MRHS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t grid = V < 1048576 ? V : 1048576;
  { kern<<<(unsigned)grid, threads, smem, s>>>(A, X, Y, nbr, V, nb, npts, R, dag); ::mrhs::count_launch(); }
  MRHS_CUDA_TRY(cudaGetLastError());
  return MRHS_OK;
}

int dispatch_fp64(const double2* A, const double2* X, double2* Y, const int32_t* nbr, int64_t V,
                  int nb, int npts, int R, int dag, cudaStream_t s) {
  int rows = 256 / R;
  if (rows < 1) rows = 1;
  const int threads = rows * R;
  const int need = (nb + rows - 1) / rows;
  if (need <= 1) return launch_k3<1>(A, X, Y, nbr, V, nb, npts, R, dag, threads, s);
  if (need <= 2) return launch_k3<2>(A, X, Y, nbr, V, nb, npts, R, dag, threads, s);
  if (need <= 4) return launch_k3<4>(A, X, Y, nbr, V, nb, npts, R, dag, threads, s);
  if (need <= 6) return launch_k3<6>(A, X, Y, nbr, V, nb, npts, R, dag, threads, s);
  if (need <= 8) return launch_k3<8>(A, X, Y, nbr, V, nb, npts, R, dag, threads, s);
  if (need <= 16) return launch_k3<16>(A, X, Y, nbr, V, nb, npts, R, dag, threads, s);
  return fail(MRHS_ERR_INVALID_ARG, "simt apply: nb too large for nrhs");
}

// error-free sum s + e = a + b (Knuth two-sum), written with the _rn
// intrinsics so that no step is contracted into an FMA
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// (h, l) += (ah + al)(bh + bl), the al bl term dropped
__device__ __forceinline__ void df_mac(float& h, float& l, float ah, float al, float bh,
                                       float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  float s, t;
  two_sum(h, p, s, t);
  h = s;
  l = __fadd_rn(l, __fadd_rn(t, e));
}

__device__ __forceinline__ void df_norm(float& h, float& l) {
  float s, t;
  two_sum(h, l, s, t);
  h = s;
  l = t;
}

__device__ __forceinline__ float2 df_split(double v) {
  const float hi = __double2float_rn(v);
  return make_float2(hi, __double2float_rn(v - (double)hi));
}

template <int OPT>
__global__ void __launch_bounds__(256) k_op_df32(const double2* __restrict__ A,
                                                 const double2* __restrict__ X,
                                                 double2* __restrict__ Y,
                                                 const int32_t* __restrict__ nbr, int64_t V,
                                                 int nb, int npts, int R, int dag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* sA = reinterpret_cast<float4*>(smem_raw);   // (Ar hi, Ar lo, Ai hi, Ai lo)
  float4* sX = sA + nb * nb;                          // (Br hi, Br lo, Bi hi, Bi lo)
  float2* sS = reinterpret_cast<float2*>(sX + nb * R);   // Ar +- Ai
  float2* sXs = sS + nb * nb;                         // Br + Bi
  const int T = blockDim.x;
  const int rows_per_pass = T / R;
  const int r = threadIdx.x % R;
  const int a0 = threadIdx.x / R;
  const bool lane_ok = threadIdx.x < rows_per_pass * R;
  const double sg = dag ? -1.0 : 1.0;
  for (int64_t x = blockIdx.x; x < V; x += gridDim.x) {
    float t1h[OPT], t1l[OPT], t2h[OPT], t2l[OPT], t3h[OPT], t3l[OPT];
#pragma unroll
    for (int k = 0; k < OPT; ++k) t1h[k] = t1l[k] = t2h[k] = t2l[k] = t3h[k] = t3l[k] = 0.f;
    for (int p = 0; p < npts; ++p) {
      const int64_t y = nbr[(int64_t)p * V + x];
      const double2* Ap = A + ((dag ? y : x) * npts + p) * (int64_t)nb * nb;
      const double2* Xp = X + y * (int64_t)nb * R;
      __syncthreads();
      for (int i = threadIdx.x; i < nb * nb; i += T) {
        const double2 v = Ap[i];
        const float2 re = df_split(v.x), im = df_split(v.y);
        sA[i] = make_float4(re.x, re.y, im.x, im.y);
        sS[i] = df_split(v.x + sg * v.y);
      }
      for (int i = threadIdx.x; i < nb * R; i += T) {
        const double2 v = Xp[i];
        const float2 re = df_split(v.x), im = df_split(v.y);
        sX[i] = make_float4(re.x, re.y, im.x, im.y);
        sXs[i] = df_split(v.x + v.y);
      }
      __syncthreads();
      if (lane_ok) {
        const int sa = dag ? 1 : nb, sb = dag ? nb : 1;
        for (int b = 0; b < nb; ++b) {
          const float4 xv = sX[b * R + r];
          const float2 xs = sXs[b * R + r];
#pragma unroll
          for (int k = 0; k < OPT; ++k) {
            const int a = a0 + k * rows_per_pass;
            if (a < nb) {
              const int e = a * sa + b * sb;
              const float4 av = sA[e];
              const float2 as = sS[e];
              df_mac(t1h[k], t1l[k], av.x, av.y, xv.x, xv.y);
              df_mac(t2h[k], t2l[k], av.z, av.w, xv.z, xv.w);
              df_mac(t3h[k], t3l[k], as.x, as.y, xs.x, xs.y);
            }
          }
        }
#pragma unroll
        for (int k = 0; k < OPT; ++k) {
          df_norm(t1h[k], t1l[k]);
          df_norm(t2h[k], t2l[k]);
          df_norm(t3h[k], t3l[k]);
        }
      }
    }
    if (lane_ok) {
      double2* Yx = Y + x * (int64_t)nb * R;
#pragma unroll
      for (int k = 0; k < OPT; ++k) {
        const int a = a0 + k * rows_per_pass;
        if (a < nb) {
          const double t1 = (double)t1h[k] + (double)t1l[k];
          const double t2 = (double)t2h[k] + (double)t2l[k];
          const double t3 = (double)t3h[k] + (double)t3l[k];
          Yx[a * R + r] = dag ? make_double2(t1 + t2, t3 - t1 + t2)
                              : make_double2(t1 - t2, t3 - t1 - t2);
        }
      }
    }
  }
}

template <int OPT>
int launch_df32(const double2* A, const double2* X, double2* Y, const int32_t* nbr, int64_t V,
                int nb, int npts, int R, int dag, int threads, cudaStream_t s) {
  const size_t smem = (sizeof(float4) + sizeof(float2)) * ((size_t)nb * nb + (size_t)nb * R);
  auto kern = k_op_df32<OPT>;
  MRHS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t grid = V < 1048576 ? V : 1048576;
  { kern<<<(unsigned)grid, threads, smem, s>>>(A, X, Y, nbr, V, nb, npts, R, dag); ::mrhs::count_launch(); }
  MRHS_CUDA_TRY(cudaGetLastError());
  return MRHS_OK;
}

int dispatch_df32(const double2* A, const double2* X, double2* Y, const int32_t* nbr, int64_t V,
                  int nb, int npts, int R, int dag, cudaStream_t s) {
  int rows = 256 / R;
  if (rows < 1) rows = 1;
  const int threads = rows * R;
  const int need = (nb + rows - 1) / rows;
  if (need <= 1) return launch_df32<1>(A, X, Y, nbr, V, nb, npts, R, dag, threads, s);
  if (need <= 2) return launch_df32<2>(A, X, Y, nbr, V, nb, npts, R, dag, threads, s);
  if (need <= 4) return launch_df32<4>(A, X, Y, nbr, V, nb, npts, R, dag, threads, s);
  if (need <= 6) return launch_df32<6>(A, X, Y, nbr, V, nb, npts, R, dag, threads, s);
  if (need <= 8) return launch_df32<8>(A, X, Y, nbr, V, nb, npts, R, dag, threads, s);
  if (need <= 16) return launch_df32<16>(A, X, Y, nbr, V, nb, npts, R, dag, threads, s);
  return fail(MRHS_ERR_INVALID_ARG, "simt apply: nb too large for nrhs");
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
    st = dispatch_fp64(op->a64, (const double2*)X, (double2*)Y, nbr, op->V, op->nb, op->npts,
                       nrhs, dag ? 1 : 0, s);
  else if (prec == MRHS_PREC_DF32)
    st = dispatch_df32(op->a64, (const double2*)X, (double2*)Y, nbr, op->V, op->nb, op->npts,
                       nrhs, dag ? 1 : 0, s);
  else if (prec == MRHS_PREC_FP32)
    st = dispatch<float2>(op->a32, (const float2*)X, (float2*)Y, nbr, op->V, op->nb, op->npts,
                          nrhs, dag ? 1 : 0, s);
  timer_mark(op, prec, s);
  if (st == MRHS_ERR_UNSUPPORTED) return fail(st, "simt apply: precision");
  return st;
}

}  // namespace mrhs
