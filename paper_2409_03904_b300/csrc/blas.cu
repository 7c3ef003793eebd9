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

// Partial Gram of one row range per CTA.  A thread owns a T x T tile of
// entries (T = 1, 2 or 4 by the block width, so the tiles number at most 256)
// and the threads left over form row groups: group g takes rows g, g + G, ...
// of every staged tile, so all 256 threads work even for a 4 x 4 Gram.
// Products are summed in the vectors' precision over at most kFlushRows rows
// per thread and then added into FP64; the groups are summed in a fixed
// order, so the result is bitwise reproducible.
constexpr int kFlushRows = 64;

template <typename C, int T>
__global__ void __launch_bounds__(kThreads)
    k_gram_partial(const C* __restrict__ X, const C* __restrict__ Y, double2* __restrict__ part,
                   int64_t N, int rx, int ry, int64_t rows_per_block, int64_t ldx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sX = reinterpret_cast<C*>(smem_raw);
  C* sY = sX + kTile * rx;
  const int tx = (rx + T - 1) / T, ty = (ry + T - 1) / T;
  const int nt = tx * ty;
  const int G = kThreads / nt;
  const int tid = threadIdx.x;
  const int g = tid / nt, et = tid % nt;
  const bool worker = g < G;
  const int i0 = (et / ty) * T, j0 = (et % ty) * T;
  double2 acc[T][T];
  C sum[T][T];
#pragma unroll
  for (int a = 0; a < T; ++a)
#pragma unroll
    for (int b = 0; b < T; ++b) {
      acc[a][b] = make_double2(0.0, 0.0);
      sum[a][b] = czero<C>();
    }
  int pending = 0;
  const int64_t n0 = (int64_t)blockIdx.x * rows_per_block;
  int64_t n1 = n0 + rows_per_block;
  if (n1 > N) n1 = N;
  for (int64_t t0 = n0; t0 < n1; t0 += kTile) {
    const int rows = (int)((n1 - t0) < kTile ? (n1 - t0) : kTile);
    __syncthreads();
    if (ldx == rx) {
      for (int i = tid; i < rows * rx; i += kThreads) sX[i] = X[t0 * rx + i];
    } else {      // a column block of a wider matrix
      for (int i = tid; i < rows * rx; i += kThreads) sX[i] = X[(t0 + i / rx) * ldx + i % rx];
    }
    for (int i = tid; i < rows * ry; i += kThreads) sY[i] = Y[t0 * ry + i];
    __syncthreads();
    if (!worker) continue;
    for (int n = g; n < rows; n += G) {
      C xv[T], yv[T];
#pragma unroll
      for (int a = 0; a < T; ++a) xv[a] = (i0 + a < rx) ? sX[n * rx + i0 + a] : czero<C>();
#pragma unroll
      for (int b = 0; b < T; ++b) yv[b] = (j0 + b < ry) ? sY[n * ry + j0 + b] : czero<C>();
#pragma unroll
      for (int a = 0; a < T; ++a)
#pragma unroll
        for (int b = 0; b < T; ++b) sum[a][b] = cfma_conj(xv[a], yv[b], sum[a][b]);
      if (++pending == kFlushRows) {
#pragma unroll
        for (int a = 0; a < T; ++a)
#pragma unroll
          for (int b = 0; b < T; ++b) {
            acc[a][b].x += (double)sum[a][b].x;
            acc[a][b].y += (double)sum[a][b].y;
            sum[a][b] = czero<C>();
          }
        pending = 0;
      }
    }
  }
#pragma unroll
  for (int a = 0; a < T; ++a)
#pragma unroll
    for (int b = 0; b < T; ++b) {
      acc[a][b].x += (double)sum[a][b].x;
      acc[a][b].y += (double)sum[a][b].y;
    }
  const int ne = rx * ry;
  double2* out = part + (int64_t)blockIdx.x * ne;
  if (G == 1) {
    if (worker)
#pragma unroll
      for (int a = 0; a < T; ++a)
#pragma unroll
        for (int b = 0; b < T; ++b)
          if (i0 + a < rx && j0 + b < ry) out[(i0 + a) * ry + j0 + b] = acc[a][b];
    return;
  }
  // groups -> shared memory [G][nt][T][T], then a fixed-order sum per entry
  __syncthreads();
  double2* red = reinterpret_cast<double2*>(smem_raw);
  if (worker)
#pragma unroll
    for (int a = 0; a < T; ++a)
#pragma unroll
      for (int b = 0; b < T; ++b) red[((g * nt + et) * T + a) * T + b] = acc[a][b];
  __syncthreads();
  for (int e = tid; e < nt * T * T; e += kThreads) {
    const int t = e / (T * T), a = (e / T) % T, b = e % T;
    const int i = (t / ty) * T + a, j = (t % ty) * T + b;
    if (i >= rx || j >= ry) continue;
    double2 v = make_double2(0.0, 0.0);
    for (int gg = 0; gg < G; ++gg) {
      const double2 w = red[gg * nt * T * T + e];
      v.x += w.x;
      v.y += w.y;
    }
    out[i * ry + j] = v;
  }
}

// Sum of the partial Grams: one warp per entry, lanes striding over the
// blocks, then a fixed shuffle tree (bitwise reproducible).
__global__ void k_gram_final(const double2* __restrict__ part, double2* __restrict__ G, int nblk,
                             int ne) {
  const int e = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (e >= ne) return;
  double2 s = make_double2(0.0, 0.0);
  for (int b = lane; b < nblk; b += 32) {
    const double2 v = part[(int64_t)b * ne + e];
    s.x += v.x;
    s.y += v.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s.x += __shfl_down_sync(0xffffffffu, s.x, o);
    s.y += __shfl_down_sync(0xffffffffu, s.y, o);
  }
  if (lane == 0) G[e] = s;
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
           int rout, int64_t ldx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sM = reinterpret_cast<C*>(smem_raw);
  C* sX = sM + rin * rout;
  for (int i = threadIdx.x; i < rin * rout; i += kThreads) sM[i] = from_c128<C>(M[i]);
  using R = typename real_of<C>::type;
  const R b = (R)beta;
  for (int64_t t0 = (int64_t)blockIdx.x * kTile; t0 < N; t0 += (int64_t)gridDim.x * kTile) {
    const int rows = (int)((N - t0) < kTile ? (N - t0) : kTile);
    __syncthreads();
    if (ldx == rin) {
      for (int i = threadIdx.x; i < rows * rin; i += kThreads) sX[i] = X[t0 * rin + i];
    } else {      // a column block of a wider matrix
      for (int i = threadIdx.x; i < rows * rin; i += kThreads)
        sX[i] = X[(t0 + i / rin) * ldx + i % rin];
    }
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

// ---- complex64 blocks of at most 32 columns: one row per warp step
// The two kernels above stage row tiles for the whole CTA and spend two
// shared-memory loads per complex product.  For complex64 blocks of up to 32
// columns (the mixed solve's Krylov blocks) a lane owns one output column and
// keeps what it multiplies with in registers: the column M[:, j] for the block
// update, its Gram column's partial sums for the Gram.  Each warp stages its
// own kWarpRows rows of X (no block barrier) and reads them back as 16-byte
// broadcasts, so the FP32 pipes, not shared memory, set the pace.
constexpr int kWarpRows = 4;
constexpr int kWarpsW = 4;            // 128 threads (153 registers: three CTAs per SM)

// Y = beta Y + X M, rin, rout <= 32.  A warp reads its rows of X completely
// before it writes the same rows of Y, so Y may alias X.  The next step's rows
// are loaded into registers while the current ones are multiplied.
template <int MAXI>
__global__ void __launch_bounds__(kWarpsW * 32)
    k_axpy_w(float2* Y, const float2* X, const double2* __restrict__ M, float beta, int64_t N,
             int rin, int rout, int64_t ldx) {
  __shared__ __align__(16) float2 sx[kWarpsW][kWarpRows][MAXI];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2 m[MAXI];
#pragma unroll
  for (int i = 0; i < MAXI; ++i) {
    m[i] = make_float2(0.f, 0.f);
    if (i < rin && lane < rout) {
      const double2 v = M[i * rout + lane];
      m[i] = make_float2((float)v.x, (float)v.y);
    }
  }
  const int64_t step = (int64_t)gridDim.x * kWarpsW * kWarpRows;
  int64_t n0 = ((int64_t)blockIdx.x * kWarpsW + warp) * kWarpRows;
  float2 xn[kWarpRows], yn[kWarpRows];
  auto load = [&](int64_t base) {
#pragma unroll
    for (int r = 0; r < kWarpRows; ++r) {
      const int64_t n = base + r;
      xn[r] = yn[r] = make_float2(0.f, 0.f);
      if (n < N) {
        if (lane < rin) xn[r] = X[n * ldx + lane];
        if (beta != 0.f && lane < rout) yn[r] = Y[n * rout + lane];
      }
    }
  };
  load(n0);
  for (; n0 < N; n0 += step) {
    float2 acc[kWarpRows];
#pragma unroll
    for (int r = 0; r < kWarpRows; ++r) {
      if (lane < MAXI) sx[warp][r][lane] = xn[r];
      acc[r] = make_float2(beta * yn[r].x, beta * yn[r].y);
    }
    __syncwarp();
    load(n0 + step);
#pragma unroll
    for (int i = 0; i < MAXI; i += 2) {
#pragma unroll
      for (int r = 0; r < kWarpRows; ++r) {
        const float4 xx = *reinterpret_cast<const float4*>(&sx[warp][r][i]);
        acc[r] = cfma(make_float2(xx.x, xx.y), m[i], acc[r]);
        acc[r] = cfma(make_float2(xx.z, xx.w), m[i + 1], acc[r]);
      }
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < kWarpRows; ++r) {
      const int64_t n = n0 + r;
      if (lane < rout && n < N) Y[n * rout + lane] = acc[r];
    }
  }
}

// Partial Gram X^dagger Y of one row range per CTA, rx, ry <= 32: lane j keeps
// column j of the partial Gram (rx complex64 sums over at most kFlushRowsW rows
// of its warp, then added into the warp's FP64 row of shared memory; on B300
// an FP64 add costs about as much as sixty FP32 FMAs, so the flushes are kept
// rare); the warps' FP64 partials are summed in a fixed order at the end.  The
// next step's rows are loaded into registers while the current ones are used.
constexpr int kWarpsG = 4;            // 128 threads
constexpr int kGramRows = 8;          // rows per warp step
constexpr int kFlushRowsW = 256;
template <int MAXI>
__global__ void __launch_bounds__(kWarpsG * 32)
    k_gram_w(const float2* __restrict__ X, const float2* __restrict__ Y, double2* __restrict__ part,
             int64_t N, int rx, int ry, int64_t rows_per_block, int64_t ldx) {
  __shared__ __align__(16) float2 sx[kWarpsG][kGramRows][MAXI];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // the warps' FP64 partials [kWarpsG][MAXI][32] (dynamic: 64 KB at MAXI = 32)
  double2 (*sg)[MAXI][32] = reinterpret_cast<double2 (*)[MAXI][32]>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = 0; i < MAXI; ++i) sg[warp][i][lane] = make_double2(0.0, 0.0);
  float2 acc[MAXI];
#pragma unroll
  for (int i = 0; i < MAXI; ++i) acc[i] = make_float2(0.f, 0.f);
  const int64_t b0 = (int64_t)blockIdx.x * rows_per_block;
  int64_t b1 = b0 + rows_per_block;
  if (b1 > N) b1 = N;
  const int64_t step = kWarpsG * kGramRows;
  float2 xn[kGramRows], yn[kGramRows];
  auto load = [&](int64_t base) {
#pragma unroll
    for (int r = 0; r < kGramRows; ++r) {
      const int64_t n = base + r;
      xn[r] = yn[r] = make_float2(0.f, 0.f);
      if (n < b1) {
        if (lane < rx) xn[r] = X[n * ldx + lane];
        if (lane < ry) yn[r] = Y[n * ry + lane];
      }
    }
  };
  int pending = 0;
  int64_t n0 = b0 + warp * kGramRows;
  load(n0);
  for (; n0 < b1; n0 += step) {
    float2 yv[kGramRows];
#pragma unroll
    for (int r = 0; r < kGramRows; ++r) {
      if (lane < MAXI) sx[warp][r][lane] = xn[r];
      yv[r] = yn[r];
    }
    __syncwarp();
    load(n0 + step);
#pragma unroll
    for (int i = 0; i < MAXI; i += 2) {
#pragma unroll
      for (int r = 0; r < kGramRows; ++r) {
        const float4 xx = *reinterpret_cast<const float4*>(&sx[warp][r][i]);
        acc[i] = cfma_conj(make_float2(xx.x, xx.y), yv[r], acc[i]);
        acc[i + 1] = cfma_conj(make_float2(xx.z, xx.w), yv[r], acc[i + 1]);
      }
    }
    __syncwarp();
    pending += kGramRows;
    if (pending >= kFlushRowsW) {
#pragma unroll
      for (int i = 0; i < MAXI; ++i) {
        double2 g = sg[warp][i][lane];
        g.x += (double)acc[i].x;
        g.y += (double)acc[i].y;
        sg[warp][i][lane] = g;
        acc[i] = make_float2(0.f, 0.f);
      }
      pending = 0;
    }
  }
#pragma unroll
  for (int i = 0; i < MAXI; ++i) {
    double2 g = sg[warp][i][lane];
    g.x += (double)acc[i].x;
    g.y += (double)acc[i].y;
    sg[warp][i][lane] = g;
  }
  __syncthreads();
  double2* out = part + (int64_t)blockIdx.x * rx * ry;
  for (int e = threadIdx.x; e < rx * ry; e += blockDim.x) {
    const int i = e / ry, j = e % ry;
    double2 v = sg[0][i][j];
    for (int w = 1; w < kWarpsG; ++w) {
      v.x += sg[w][i][j].x;
      v.y += sg[w][i][j].y;
    }
    out[e] = v;
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
  const int64_t per = 512;    // at least this many rows per CTA
  int64_t nblk = (N + per - 1) / per;
  const int64_t cap = (int64_t)num_sms() * 2;
  if (nblk > cap) nblk = cap;
  if (nblk < 1) nblk = 1;
  return (int)nblk;
}

size_t gram_workspace_bytes(int64_t N, int rx, int ry) {
  return (size_t)gram_blocks(N) * rx * ry * sizeof(double2);
}

int gram_tile(int rx, int ry) {
  const int r = rx > ry ? rx : ry;
  return r <= 8 ? 1 : (r <= 16 ? 2 : 4);
}

template <typename C, int T>
int launch_gram(const void* X, const void* Y, double2* part, int64_t N, int rx, int ry,
                int nblk, int64_t per, int64_t ldx, cudaStream_t s) {
  const int nt = ((rx + T - 1) / T) * ((ry + T - 1) / T);
  const int G = kThreads / nt;
  const size_t stage = sizeof(C) * kTile * (rx + ry);
  const size_t red = G > 1 ? sizeof(double2) * (size_t)G * nt * T * T : 0;
  const size_t smem = stage > red ? stage : red;
  MRHS_CUDA_TRY(cudaFuncSetAttribute(k_gram_partial<C, T>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  { k_gram_partial<C, T><<<nblk, kThreads, smem, s>>>((const C*)X, (const C*)Y, part, N, rx, ry,
                                                      per, ldx); ::mrhs::count_launch(); }
  return MRHS_OK;
}

template <typename C>
int launch_gram(const void* X, const void* Y, double2* part, int64_t N, int rx, int ry,
                int nblk, int64_t per, int64_t ldx, cudaStream_t s) {
  switch (gram_tile(rx, ry)) {
    case 1: return launch_gram<C, 1>(X, Y, part, N, rx, ry, nblk, per, ldx, s);
    case 2: return launch_gram<C, 2>(X, Y, part, N, rx, ry, nblk, per, ldx, s);
    default: return launch_gram<C, 4>(X, Y, part, N, rx, ry, nblk, per, ldx, s);
  }
}

template <int MAXI>
int launch_gram_w_t(const void* X, const void* Y, double2* part, int64_t N, int rx, int ry,
                    int nblk, int64_t per, int64_t ldx, cudaStream_t s) {
  const size_t smem = sizeof(double2) * kWarpsG * MAXI * 32;
  MRHS_CUDA_TRY(cudaFuncSetAttribute(k_gram_w<MAXI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
  { k_gram_w<MAXI><<<nblk, kWarpsG * 32, smem, s>>>((const float2*)X, (const float2*)Y, part, N,
                                                    rx, ry, per, ldx); ::mrhs::count_launch(); }
  return MRHS_OK;
}

int launch_gram_w(const void* X, const void* Y, double2* part, int64_t N, int rx, int ry,
                  int nblk, int64_t per, int64_t ldx, cudaStream_t s) {
  if (rx <= 8) return launch_gram_w_t<8>(X, Y, part, N, rx, ry, nblk, per, ldx, s);
  if (rx <= 16) return launch_gram_w_t<16>(X, Y, part, N, rx, ry, nblk, per, ldx, s);
  return launch_gram_w_t<32>(X, Y, part, N, rx, ry, nblk, per, ldx, s);
}

int gram_ws(const void* X, const void* Y, double2* G, int64_t N, int rx, int ry, int dtype,
            double2* part, cudaStream_t s) {
  return gram_ws_capped(X, Y, G, N, rx, ry, dtype, part, (int64_t)gram_blocks(N) * rx * ry, s);
}

// The two Gram kernels with the number of row blocks capped so that the
// partial Grams fit a buffer of `max_entries` complex128 values (the entry
// point that must not allocate passes its own static buffer).
int gram_ws_capped(const void* X, const void* Y, double2* G, int64_t N, int rx, int ry, int dtype,
                   double2* part, int64_t max_entries, cudaStream_t s, int64_t ldx) {
  if (ldx <= 0) ldx = rx;
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
  if (gram_tc_applies(X, Y, N, rx, ry, dtype, ldx)) {     // tensor cores (blas_tc.cu)
    MRHS_TRY(gram_tc_partial(X, Y, part, N, rx, ry, max_entries / ne, &nblk, s));
    { k_gram_final<<<(unsigned)((ne * 32 + 255) / 256), 256, 0, s>>>(part, G, nblk, ne); ::mrhs::count_launch(); }
    MRHS_CUDA_TRY(cudaGetLastError());
    return MRHS_OK;
  }
  if (dtype == MRHS_C128) MRHS_TRY(launch_gram<double2>(X, Y, part, N, rx, ry, nblk, per, ldx, s));
  else if (rx <= 32 && ry <= 32) MRHS_TRY(launch_gram_w(X, Y, part, N, rx, ry, nblk, per, ldx, s));
  else MRHS_TRY(launch_gram<float2>(X, Y, part, N, rx, ry, nblk, per, ldx, s));
  MRHS_CUDA_TRY(cudaGetLastError());
  { k_gram_final<<<(unsigned)((ne * 32 + 255) / 256), 256, 0, s>>>(part, G, nblk, ne); ::mrhs::count_launch(); }
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
         int dtype, cudaStream_t s, int64_t ldx) {
  if (ldx <= 0) ldx = rin;
  if (N == 0) return MRHS_OK;
  if (update_tc_applies(Y, X, Y, N, rin, rout, dtype, ldx))   // tensor cores (blas_tc.cu)
    return update_tc(Y, X, Y, M, 0, beta, N, rin, rout, s);
  int64_t grid = (N + kTile - 1) / kTile;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (grid > cap) grid = cap;
  if (dtype == MRHS_C128) {
    const size_t smem = sizeof(double2) * ((size_t)rin * rout + (size_t)kTile * rin);
    MRHS_CUDA_TRY(cudaFuncSetAttribute(k_axpy<double2>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    { k_axpy<double2><<<(unsigned)grid, kThreads, smem, s>>>((double2*)Y, (const double2*)X, M, beta,
                                                            N, rin, rout, ldx); ::mrhs::count_launch(); }
  } else if (rin <= 32 && rout <= 32) {
    int64_t g = (N + kWarpsW * kWarpRows - 1) / (kWarpsW * kWarpRows);
    const int64_t capw = (int64_t)num_sms() * 3;   // the resident CTAs
    if (g > capw) g = capw;
    const float b = (float)beta;
    if (rin <= 8)
      { k_axpy_w<8><<<(unsigned)g, kWarpsW * 32, 0, s>>>((float2*)Y, (const float2*)X, M, b, N, rin,
                                                          rout, ldx); ::mrhs::count_launch(); }
    else if (rin <= 16)
      { k_axpy_w<16><<<(unsigned)g, kWarpsW * 32, 0, s>>>((float2*)Y, (const float2*)X, M, b, N, rin,
                                                           rout, ldx); ::mrhs::count_launch(); }
    else
      { k_axpy_w<32><<<(unsigned)g, kWarpsW * 32, 0, s>>>((float2*)Y, (const float2*)X, M, b, N, rin,
                                                           rout, ldx); ::mrhs::count_launch(); }
  } else {
    const size_t smem = sizeof(float2) * ((size_t)rin * rout + (size_t)kTile * rin);
    { k_axpy<float2><<<(unsigned)grid, kThreads, smem, s>>>((float2*)Y, (const float2*)X, M, beta, N,
                                                          rin, rout, ldx); ::mrhs::count_launch(); }
  }
  MRHS_CUDA_TRY(cudaGetLastError());
  return MRHS_OK;
}

}  // namespace mrhs
