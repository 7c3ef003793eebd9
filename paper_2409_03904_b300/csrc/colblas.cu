// Column-wise vector algebra for solvers that run one Krylov process per
// right-hand side in lockstep: the flexible ADEF2 CG of Fig. 1 and its
// fixed-iteration CG smoother (Sec. 2: "the separate right hand sides have
// the smoother implemented as distinct Krylov processes on each right hand
// side").  Every column j of an N x r block has its own scalars:
//   mrhs_col_dot:    out[j] = sum_n conj(X[n][j]) Y[n][j]   (FP64 sums, fixed order)
//   mrhs_col_ratio:  out[j] = scale * num[j] / den[j]       (0 if den[j] = 0 or
//                                                            the column is inactive)
//   mrhs_col_update: Y[n][j] = beta Y[n][j] + coef[j] X[n][j]
// The scalars stay on the device, so a step of all r processes is a few
// launches with no host round trip.
#include <map>
#include <mutex>

#include "internal.cuh"

namespace mrhs {
namespace {

constexpr int kThreads = 256;

template <typename C>
__device__ inline double2 widen(C v);
template <>
__device__ inline double2 widen<double2>(double2 v) { return v; }
template <>
__device__ inline double2 widen<float2>(float2 v) { return make_double2(v.x, v.y); }

// Per-CTA partial column dots: thread t owns column t % r and rows
// t / r, t / r + lanes, ... of the CTA's row range; the CTA sums each
// column's threads in a fixed order.
template <typename C>
__global__ void __launch_bounds__(kThreads) k_col_dot_part(const C* __restrict__ X,
                                                           const C* __restrict__ Y,
                                                           double2* __restrict__ part, int64_t N,
                                                           int r, int64_t per) {
  __shared__ double2 s[kThreads];
  const int lanes = kThreads / r;              // threads per column
  const int t = threadIdx.x;
  double2 acc = make_double2(0.0, 0.0);
  if (t < lanes * r) {
    const int j = t % r;
    const int64_t n0 = (int64_t)blockIdx.x * per, n1 = n0 + per < N ? n0 + per : N;
    for (int64_t n = n0 + t / r; n < n1; n += lanes) {
      const double2 a = widen(X[n * r + j]), b = widen(Y[n * r + j]);
      acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
      acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
    }
  }
  s[t] = acc;
  __syncthreads();
  if (t < r) {
    double2 v = make_double2(0.0, 0.0);
    for (int i = t; i < lanes * r; i += r) {
      v.x += s[i].x;
      v.y += s[i].y;
    }
    part[(int64_t)blockIdx.x * r + t] = v;
  }
}

__global__ void k_col_dot_final(const double2* __restrict__ part, double2* __restrict__ out,
                                int nblk, int r) {
  const int j = threadIdx.x;
  if (j >= r) return;
  double2 v = make_double2(0.0, 0.0);
  for (int b = 0; b < nblk; ++b) {
    v.x += part[(int64_t)b * r + j].x;
    v.y += part[(int64_t)b * r + j].y;
  }
  out[j] = v;
}

__global__ void k_col_ratio(const double2* __restrict__ num, const double2* __restrict__ den,
                            double2* __restrict__ out, const int32_t* __restrict__ active, int r,
                            double scale) {
  const int j = threadIdx.x;
  if (j >= r) return;
  const double2 a = num[j], b = den[j];
  const double d = b.x * b.x + b.y * b.y;
  if (d == 0.0 || (active && !active[j])) {
    out[j] = make_double2(0.0, 0.0);
    return;
  }
  // a / b = a conj(b) / |b|^2
  out[j] = make_double2(scale * (a.x * b.x + a.y * b.y) / d, scale * (a.y * b.x - a.x * b.y) / d);
}

template <typename C>
__global__ void __launch_bounds__(kThreads) k_col_update(C* Y, const C* __restrict__ X,
                                                         const double2* __restrict__ coef,
                                                         double beta, int64_t n, int r) {
  using R = typename real_of<C>::type;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(i % r);
    const double2 c = coef[j];
    const C x = X[i];
    C y;
    if (beta != 0.0) {
      const C y0 = Y[i];
      y.x = (R)(beta * (double)y0.x + c.x * (double)x.x - c.y * (double)x.y);
      y.y = (R)(beta * (double)y0.y + c.x * (double)x.y + c.y * (double)x.x);
    } else {
      y.x = (R)(c.x * (double)x.x - c.y * (double)x.y);
      y.y = (R)(c.x * (double)x.y + c.y * (double)x.x);
    }
    Y[i] = y;
  }
}

struct Key {
  int dev;
  cudaStream_t s;
  bool operator<(const Key& o) const { return dev != o.dev ? dev < o.dev : s < o.s; }
};
std::mutex g_mu;
std::map<Key, Workspace>& partials() {
  static std::map<Key, Workspace> m;
  return m;
}

}  // namespace
}  // namespace mrhs

using namespace mrhs;

extern "C" int mrhs_col_dot(const void* X, const void* Y, void* out, int64_t N, int32_t r,
                            int32_t dtype, void* stream) {
  if (N < 0 || r < 1 || r > MRHS_MAX_RHS) return fail(MRHS_ERR_INVALID_ARG, "mrhs_col_dot: sizes");
  if (dtype != MRHS_C128 && dtype != MRHS_C64) return fail(MRHS_ERR_INVALID_ARG, "dtype");
  if (!out || ((uintptr_t)out & 15u)) return fail(MRHS_ERR_INVALID_ARG, "out null or misaligned");
  if (N > 0 && (!X || !Y || (((uintptr_t)X | (uintptr_t)Y) & 15u)))
    return fail(MRHS_ERR_INVALID_ARG, "X or Y null or misaligned");
  cudaStream_t s = (cudaStream_t)stream;
  if (N == 0) {
    MRHS_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double2) * r, s));
    return MRHS_OK;
  }
  int nblk = num_sms() * 2;
  if ((int64_t)nblk > N) nblk = (int)N;
  const int64_t per = (N + nblk - 1) / nblk;
  int dev = 0;
  MRHS_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  Workspace& ws = partials()[Key{dev, s}];
  MRHS_TRY(ws.ensure(sizeof(double2) * (size_t)nblk * r));
  double2* part = (double2*)ws.ptr;
  if (dtype == MRHS_C128)
    k_col_dot_part<double2><<<nblk, kThreads, 0, s>>>((const double2*)X, (const double2*)Y, part,
                                                      N, r, per);
  else
    k_col_dot_part<float2><<<nblk, kThreads, 0, s>>>((const float2*)X, (const float2*)Y, part, N,
                                                     r, per);
  count_launch();
  k_col_dot_final<<<1, 64, 0, s>>>(part, (double2*)out, nblk, r);
  count_launch();
  MRHS_CUDA_TRY(cudaGetLastError());
  return MRHS_OK;
}

extern "C" int mrhs_col_ratio(const void* num, const void* den, void* out, const int32_t* active,
                              int32_t r, double scale, void* stream) {
  if (r < 1 || r > MRHS_MAX_RHS) return fail(MRHS_ERR_INVALID_ARG, "mrhs_col_ratio: r");
  if (!num || !den || !out) return fail(MRHS_ERR_INVALID_ARG, "mrhs_col_ratio: null pointer");
  k_col_ratio<<<1, 64, 0, (cudaStream_t)stream>>>((const double2*)num, (const double2*)den,
                                                  (double2*)out, active, r, scale);
  count_launch();
  MRHS_CUDA_TRY(cudaGetLastError());
  return MRHS_OK;
}

extern "C" int mrhs_col_update(void* Y, const void* X, const void* coef, double beta, int64_t N,
                               int32_t r, int32_t dtype, void* stream) {
  if (N < 0 || r < 1 || r > MRHS_MAX_RHS)
    return fail(MRHS_ERR_INVALID_ARG, "mrhs_col_update: sizes");
  if (dtype != MRHS_C128 && dtype != MRHS_C64) return fail(MRHS_ERR_INVALID_ARG, "dtype");
  if (!coef) return fail(MRHS_ERR_INVALID_ARG, "coef is null");
  if (N == 0) return MRHS_OK;
  if (!X || !Y || (((uintptr_t)X | (uintptr_t)Y) & 15u))
    return fail(MRHS_ERR_INVALID_ARG, "X or Y null or misaligned");
  const int64_t n = N * r;
  int64_t grid = (n + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (grid > cap) grid = cap;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == MRHS_C128)
    k_col_update<double2><<<(unsigned)grid, kThreads, 0, s>>>((double2*)Y, (const double2*)X,
                                                              (const double2*)coef, beta, n, r);
  else
    k_col_update<float2><<<(unsigned)grid, kThreads, 0, s>>>((float2*)Y, (const float2*)X,
                                                             (const double2*)coef, beta, n, r);
  count_launch();
  MRHS_CUDA_TRY(cudaGetLastError());
  return MRHS_OK;
}
