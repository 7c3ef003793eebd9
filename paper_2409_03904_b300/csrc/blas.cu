// Block inner products and block updates of block CG (Fig. 2), N x nrhs blocks.
//
// Gram G = X^dagger Y: the "ThinQR" reduction of Sec. 3.5 and Table 6 (12 x 12
// result, K ~ 1M).  The paper splits K into batched short GEMMs and sums the
// partial 12 x 12 matrices by hand; here one pass over the rows does the
// same thing in one launch: every CTA reduces a contiguous row range in
// registers (products in the vectors' precision, per-tile partial sums added
// into FP64 accumulators), writes its partial Gram, and a second one-CTA-per-
// entry pass sums the partials in a fixed order, so the FP64 result is
// bitwise reproducible run to run.
//
// Block update Y = beta Y + X M (X + D M C, Q - Z M, T S^-1, D S^dagger, ...):
// row tiles of X staged in shared memory (so Y may alias X), M in shared
// memory, one output element per thread and step.
#include <map>
#include <mutex>

#include "internal.cuh"

namespace mrhs {
namespace {

constexpr int kTile = 32;      // rows staged per step
constexpr int kThreads = 256;

template <typename C>
__global__ void __launch_bounds__(kThreads)
    k_gram_partial(const C* __restrict__ X, const C* __restrict__ Y, double2* __restrict__ part,
                   int64_t N, int rx, int ry, int64_t rows_per_block) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sX = reinterpret_cast<C*>(smem_raw);
  C* sY = sX + kTile * rx;
  constexpr int kMaxE = (MRHS_MAX_RHS * MRHS_MAX_RHS) / kThreads;
  const int ne = rx * ry;
  double2 acc[kMaxE];
#pragma unroll
  for (int k = 0; k < kMaxE; ++k) acc[k] = make_double2(0.0, 0.0);
  const int64_t n0 = (int64_t)blockIdx.x * rows_per_block;
  int64_t n1 = n0 + rows_per_block;
  if (n1 > N) n1 = N;
  for (int64_t t0 = n0; t0 < n1; t0 += kTile) {
    const int rows = (int)((n1 - t0) < kTile ? (n1 - t0) : kTile);
    __syncthreads();
    for (int i = threadIdx.x; i < rows * rx; i += kThreads) sX[i] = X[t0 * rx + i];
    for (int i = threadIdx.x; i < rows * ry; i += kThreads) sY[i] = Y[t0 * ry + i];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kMaxE; ++k) {
      const int e = threadIdx.x + k * kThreads;
      if (e < ne) {
        const int i = e / ry, j = e % ry;
        C s = czero<C>();
        for (int n = 0; n < rows; ++n) s = cfma_conj(sX[n * rx + i], sY[n * ry + j], s);
        acc[k].x += (double)s.x;
        acc[k].y += (double)s.y;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kMaxE; ++k) {
    const int e = threadIdx.x + k * kThreads;
    if (e < ne) part[(int64_t)blockIdx.x * ne + e] = acc[k];
  }
}

__global__ void k_gram_final(const double2* __restrict__ part, double2* __restrict__ G, int nblk,
                             int ne) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  double2 s = make_double2(0.0, 0.0);
  for (int b = 0; b < nblk; ++b) {
    const double2 v = part[(int64_t)b * ne + e];
    s.x += v.x;
    s.y += v.y;
  }
  G[e] = s;
}

template <typename C>
__device__ inline C from_c128(double2 v);
template <>
__device__ inline double2 from_c128<double2>(double2 v) { return v; }
template <>
__device__ inline float2 from_c128<float2>(double2 v) {
  return make_float2((float)v.x, (float)v.y);
}

template <typename C>
__global__ void __launch_bounds__(kThreads)
    k_axpy(C* Y, const C* X, const double2* __restrict__ M, double beta, int64_t N, int rin,
           int rout) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sM = reinterpret_cast<C*>(smem_raw);
  C* sX = sM + rin * rout;
  for (int i = threadIdx.x; i < rin * rout; i += kThreads) sM[i] = from_c128<C>(M[i]);
  using R = typename real_of<C>::type;
  const R b = (R)beta;
  for (int64_t t0 = (int64_t)blockIdx.x * kTile; t0 < N; t0 += (int64_t)gridDim.x * kTile) {
    const int rows = (int)((N - t0) < kTile ? (N - t0) : kTile);
    __syncthreads();
    for (int i = threadIdx.x; i < rows * rin; i += kThreads) sX[i] = X[t0 * rin + i];
    __syncthreads();
    for (int e = threadIdx.x; e < rows * rout; e += kThreads) {
      const int n = e / rout, j = e % rout;
      C s = czero<C>();
      if (beta != 0.0) {
        const C y = Y[t0 * rout + e];
        s.x = b * y.x;
        s.y = b * y.y;
      }
      for (int i = 0; i < rin; ++i) s = cfma(sX[n * rin + i], sM[i * rout + j], s);
      Y[t0 * rout + e] = s;
    }
  }
}

struct WsKey {
  int dev;
  cudaStream_t s;
  bool operator<(const WsKey& o) const { return dev != o.dev ? dev < o.dev : s < o.s; }
};
std::mutex g_ws_mu;
std::map<WsKey, Workspace>& ws_map() {
  static std::map<WsKey, Workspace> m;
  return m;
}

}  // namespace

int Workspace::ensure(size_t need) {
  if (need <= bytes) return MRHS_OK;
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  bytes = 0;
  size_t want = need + need / 4;
  if (cudaMalloc(&ptr, want) != cudaSuccess) {
    cudaGetLastError();
    ptr = nullptr;
    return fail(MRHS_ERR_NO_MEMORY, "workspace allocation of " + std::to_string(want) + " bytes");
  }
  bytes = want;
  return MRHS_OK;
}

void Workspace::release() {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  bytes = 0;
}

int gram_blocks(int64_t N) {
  const int64_t per = 4096;   // at least this many rows per CTA
  int64_t nblk = (N + per - 1) / per;
  const int64_t cap = (int64_t)num_sms() * 4;
  if (nblk > cap) nblk = cap;
  if (nblk < 1) nblk = 1;
  return (int)nblk;
}

size_t gram_workspace_bytes(int64_t N, int rx, int ry) {
  return (size_t)gram_blocks(N) * rx * ry * sizeof(double2);
}

int gram_ws(const void* X, const void* Y, double2* G, int64_t N, int rx, int ry, int dtype,
            double2* part, cudaStream_t s) {
  const int nblk = gram_blocks(N);
  int64_t per = (N + nblk - 1) / nblk;
  per = ((per + kTile - 1) / kTile) * kTile;
  const int ne = rx * ry;
  if (N == 0) {
    MRHS_CUDA_TRY(cudaMemsetAsync(G, 0, sizeof(double2) * ne, s));
    return MRHS_OK;
  }
  if (dtype == MRHS_C128) {
    const size_t smem = sizeof(double2) * kTile * (rx + ry);
    MRHS_CUDA_TRY(cudaFuncSetAttribute(k_gram_partial<double2>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    { k_gram_partial<double2><<<nblk, kThreads, smem, s>>>((const double2*)X, (const double2*)Y,
                                                          part, N, rx, ry, per); ::mrhs::count_launch(); }
  } else {
    const size_t smem = sizeof(float2) * kTile * (rx + ry);
    MRHS_CUDA_TRY(cudaFuncSetAttribute(k_gram_partial<float2>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    { k_gram_partial<float2><<<nblk, kThreads, smem, s>>>((const float2*)X, (const float2*)Y, part,
                                                         N, rx, ry, per); ::mrhs::count_launch(); }
  }
  MRHS_CUDA_TRY(cudaGetLastError());
  { k_gram_final<<<(ne + 127) / 128, 128, 0, s>>>(part, G, nblk, ne); ::mrhs::count_launch(); }
  MRHS_CUDA_TRY(cudaGetLastError());
  return MRHS_OK;
}

// Same two kernels as gram_ws, with the number of row blocks capped so that
// the partial Grams fit a caller-provided buffer of `max_entries` complex128
// values (used by the entry point that must not allocate).
int gram_ws_capped(const void* X, const void* Y, double2* G, int64_t N, int rx, int ry, int dtype,
                   double2* part, int64_t max_entries, cudaStream_t s) {
  const int ne = rx * ry;
  int nblk = gram_blocks(N);
  if ((int64_t)nblk * ne > max_entries) nblk = (int)(max_entries / ne);
  if (nblk < 1) return fail(MRHS_ERR_INVALID_ARG, "partial-Gram buffer too small");
  int64_t per = (N + nblk - 1) / nblk;
  per = ((per + kTile - 1) / kTile) * kTile;
  if (N == 0) {
    MRHS_CUDA_TRY(cudaMemsetAsync(G, 0, sizeof(double2) * ne, s));
    return MRHS_OK;
  }
  if (dtype == MRHS_C128) {
    const size_t smem = sizeof(double2) * kTile * (rx + ry);
    MRHS_CUDA_TRY(cudaFuncSetAttribute(k_gram_partial<double2>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    { k_gram_partial<double2><<<nblk, kThreads, smem, s>>>((const double2*)X, (const double2*)Y,
                                                          part, N, rx, ry, per); ::mrhs::count_launch(); }
  } else {
    const size_t smem = sizeof(float2) * kTile * (rx + ry);
    MRHS_CUDA_TRY(cudaFuncSetAttribute(k_gram_partial<float2>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    { k_gram_partial<float2><<<nblk, kThreads, smem, s>>>((const float2*)X, (const float2*)Y, part,
                                                         N, rx, ry, per); ::mrhs::count_launch(); }
  }
  MRHS_CUDA_TRY(cudaGetLastError());
  { k_gram_final<<<(ne + 127) / 128, 128, 0, s>>>(part, G, nblk, ne); ::mrhs::count_launch(); }
  MRHS_CUDA_TRY(cudaGetLastError());
  return MRHS_OK;
}

int gram(const void* X, const void* Y, double2* G, int64_t N, int rx, int ry, int dtype,
         cudaStream_t s) {
  int dev = 0;
  MRHS_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_ws_mu);
  Workspace& ws = ws_map()[WsKey{dev, s}];
  MRHS_TRY(ws.ensure(gram_workspace_bytes(N, rx, ry)));
  return gram_ws(X, Y, G, N, rx, ry, dtype, (double2*)ws.ptr, s);
}

int axpy(void* Y, const void* X, const double2* M, double beta, int64_t N, int rin, int rout,
         int dtype, cudaStream_t s) {
  if (N == 0) return MRHS_OK;
  int64_t grid = (N + kTile - 1) / kTile;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (grid > cap) grid = cap;
  if (dtype == MRHS_C128) {
    const size_t smem = sizeof(double2) * ((size_t)rin * rout + (size_t)kTile * rin);
    MRHS_CUDA_TRY(cudaFuncSetAttribute(k_axpy<double2>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    { k_axpy<double2><<<(unsigned)grid, kThreads, smem, s>>>((double2*)Y, (const double2*)X, M, beta,
                                                            N, rin, rout); ::mrhs::count_launch(); }
  } else {
    const size_t smem = sizeof(float2) * ((size_t)rin * rout + (size_t)kTile * rin);
    { k_axpy<float2><<<(unsigned)grid, kThreads, smem, s>>>((float2*)Y, (const float2*)X, M, beta, N,
                                                          rin, rout); ::mrhs::count_launch(); }
  }
  MRHS_CUDA_TRY(cudaGetLastError());
  return MRHS_OK;
}

}  // namespace mrhs
