// Block conjugate gradient solvers (Fig. 2) and the Chebyshev preconditioner
// (Sec. 2.3) on the device.
//
// BlockCGrQ (Fig. 2 left) and Preconditioned BlockCGrQ (Fig. 2 right) run
// as a host loop of stream-ordered launches: operator applications, Gram
// products, one-CTA FP64 kernels for the nrhs x nrhs algebra (Cholesky,
// inverse, C updates, stopping test) and fused row-wise block rotations.
// Nothing returns to the host inside the loop except a convergence word read
// every `check_every` iterations.  Readings of the figure taken here (the
// CPU reference takes the same ones): the solution update carries C_k (X += D M C), one Cholesky factor
// per iteration, Grams Hermitian-symmetrised, numerically null directions
// dropped by a pivoted factor (the block narrows; W and S carry zero
// columns/rows for the dropped directions, so every block keeps nrhs
// columns in memory).
//
// MRHS_SOLVE_MIXED is FP64-outer defect correction (the paper's observation
// that the preconditioner tolerates single precision while the outer solver
// keeps double, Sec. 4): r = B - H x with the FP64 operator, per-column
// scaling to complex64, an inner preconditioned block CG on complex64 vectors
// with the FP32 operator and a BF16/FP16 (or FP32) Chebyshev preconditioner,
// Grams accumulated in FP64 and factorised in FP64, and x += rho e in FP64.
#include <array>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "small.cuh"

namespace mrhs {
namespace {

constexpr int kTile = 32;
// inner target above which a refinement cycle is expected to end the solve
constexpr double kFinalCycleTarget = 0.1;
constexpr int kThreads = 256;

template <typename C>
__device__ inline C to_c(double2 v);
template <>
__device__ inline double2 to_c<double2>(double2 v) { return v; }
template <>
__device__ inline float2 to_c<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }

// ---------------------------------------------------------- elementwise
template <typename C>
__global__ void k_sub(C* out, const C* a, const C* b, int64_t n) {   // out = a - b
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const C x = a[i], y = b[i];
    C r;
    r.x = x.x - y.x;
    r.y = x.y - y.y;
    out[i] = r;
  }
}

// r32[n][j] = complex64(r[n][j] / rho[j]) (0 where rho[j] == 0)
__global__ void k_scale_to_c64(float2* out, const double2* r, const double* rho, int64_t N,
                               int R) {
  // the columns' reciprocals once per CTA (an FP64 division is many
  // instructions on B300's FP64 pipe); 0 for a column with rho <= 0
  __shared__ double s_inv[MRHS_MAX_RHS];
  for (int j = threadIdx.x; j < R; j += blockDim.x) s_inv[j] = rho[j] > 0.0 ? 1.0 / rho[j] : 0.0;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N * R;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double ip = s_inv[i % R];
    const double2 v = r[i];
    out[i] = make_float2((float)(v.x * ip), (float)(v.y * ip));
  }
}

// x[n][j] += rho[j] * e[n][j]  (FP64 solution update)
__global__ void k_update_x(double2* x, const float2* e, const double* rho, int64_t N, int R) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N * R;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double p = rho[i % R];
    const float2 v = e[i];
    double2 xv = x[i];
    xv.x = fma(p, (double)v.x, xv.x);
    xv.y = fma(p, (double)v.y, xv.y);
    x[i] = xv;
  }
}

template <typename C>
__global__ void k_zero_cols(C* x, const double* bnorm, int64_t N, int R) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N * R;
       i += (int64_t)gridDim.x * blockDim.x)
    if (!(bnorm[i % R] > 0.0)) x[i] = C{};
}

// Chebyshev recurrence, first step: T1 = a W + b X, P = c0 X + c1 T1
template <typename C>
__global__ void k_cheb_first(C* T1, C* P, const C* W, const C* X, double a, double b, double c0,
                             double c1, int64_t n) {
  using Rl = typename real_of<C>::type;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const C w = W[i], x = X[i];
    C t;
    t.x = (Rl)a * w.x + (Rl)b * x.x;
    t.y = (Rl)a * w.y + (Rl)b * x.y;
    T1[i] = t;
    C p;
    p.x = (Rl)c0 * x.x + (Rl)c1 * t.x;
    p.y = (Rl)c0 * x.y + (Rl)c1 * t.y;
    P[i] = p;
  }
}
// T_{j+1} = 2 (a W + b T_j) - T_{j-1} -> out (may alias Tp), P += c T_{j+1}
template <typename C>
__global__ void k_cheb_step(C* out, C* P, const C* W, const C* Tc, const C* Tp, double a,
                            double b, double c, int64_t n) {
  using Rl = typename real_of<C>::type;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const C w = W[i], tc = Tc[i], tp = Tp[i];
    C t;
    t.x = (Rl)2 * ((Rl)a * w.x + (Rl)b * tc.x) - tp.x;
    t.y = (Rl)2 * ((Rl)a * w.y + (Rl)b * tc.y) - tp.y;
    out[i] = t;
    C p = P[i];
    p.x += (Rl)c * t.x;
    p.y += (Rl)c * t.y;
    P[i] = p;
  }
}

// ---------------------------------------------------------- column norms
template <typename C>
__global__ void k_colnorm_partial(const C* X, double* part, int64_t N, int R,
                                  int64_t rows_per_block) {
  __shared__ double s[kThreads];
  const int64_t n0 = (int64_t)blockIdx.x * rows_per_block;
  int64_t n1 = n0 + rows_per_block;
  if (n1 > N) n1 = N;
  if (kThreads % R == 0) {
    // thread t owns column t % R and every (kThreads / R)-th row, so a warp
    // reads whole rows; the row groups are combined in a fixed order
    const int j = (int)threadIdx.x % R, g = (int)threadIdx.x / R, G = kThreads / R;
    double acc = 0.0;
    for (int64_t n = n0 + g; n < n1; n += G) {
      const C v = X[n * R + j];
      acc += (double)v.x * v.x + (double)v.y * v.y;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    if ((int)threadIdx.x < R) {
      double t = 0.0;
      for (int gg = 0; gg < G; ++gg) t += s[gg * R + threadIdx.x];
      part[(int64_t)blockIdx.x * R + threadIdx.x] = t;
    }
    return;
  }
  for (int j = 0; j < R; ++j) {
    double acc = 0.0;
    for (int64_t n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
      const C v = X[n * R + j];
      acc += (double)v.x * v.x + (double)v.y * v.y;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * R + j] = s[0];
    __syncthreads();
  }
}
__global__ void k_colnorm_final(const double* part, double* out, int nblk, int R) {
  const int j = threadIdx.x;
  if (j >= R) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * R + j];
  out[j] = sqrt(s);
}

// ---------------------------------------------------------- row rotations
// P1 <- P1 W; (P2 <- P2 W); D <- (P2 ? P2 : P1) + D S^dagger.  W, S: R x R.
template <typename C>
__global__ void __launch_bounds__(kThreads)
    k_rotate(C* P1, C* P2, C* D, const double2* __restrict__ Wm, const double2* __restrict__ Sm,
             int64_t N, int R) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sW = reinterpret_cast<C*>(smem_raw);
  C* sSh = sW + R * R;          // S^dagger
  C* sP1 = sSh + R * R;
  C* sP2 = sP1 + kTile * R;
  C* sD = sP2 + kTile * R;
  for (int i = threadIdx.x; i < R * R; i += kThreads) {
    sW[i] = to_c<C>(Wm[i]);
    const int a = i / R, b = i % R;   // S^dagger[a][b] = conj(S[b][a])
    const double2 v = Sm[b * R + a];
    sSh[i] = to_c<C>(make_double2(v.x, -v.y));
  }
  for (int64_t t0 = (int64_t)blockIdx.x * kTile; t0 < N; t0 += (int64_t)gridDim.x * kTile) {
    const int rows = (int)((N - t0) < kTile ? (N - t0) : kTile);
    __syncthreads();
    for (int i = threadIdx.x; i < rows * R; i += kThreads) {
      sP1[i] = P1[t0 * R + i];
      if (P2) sP2[i] = P2[t0 * R + i];
      sD[i] = D[t0 * R + i];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < rows * R; e += kThreads) {
      const int n = e / R, j = e % R;
      C a1 = czero<C>(), a2 = czero<C>(), dd = czero<C>();
      for (int i = 0; i < R; ++i) {
        a1 = cfma(sP1[n * R + i], sW[i * R + j], a1);
        if (P2) a2 = cfma(sP2[n * R + i], sW[i * R + j], a2);
        dd = cfma(sD[n * R + i], sSh[i * R + j], dd);
      }
      P1[t0 * R + e] = a1;
      if (P2) P2[t0 * R + e] = a2;
      const C base = P2 ? a2 : a1;
      dd.x += base.x;
      dd.y += base.y;
      D[t0 * R + e] = dd;
    }
  }
}

// The same for complex64 blocks of at most 32 columns: lane j keeps W[:, j]
// and S^dagger[:, j] in registers and each warp stages its own kRotRows rows
// of P1, P2 and D (no block barrier), read back as 16-byte broadcasts; the
// next rows are loaded into registers while the current ones are multiplied.
// A warp reads its rows completely before it writes them.
constexpr int kRotRows = 2;
constexpr int kRotWarps = 4;
template <int MAXI>
__global__ void __launch_bounds__(kRotWarps * 32)
    k_rotate_w(float2* P1, float2* P2, float2* D, const double2* __restrict__ Wm,
               const double2* __restrict__ Sm, int64_t N, int R) {
  __shared__ __align__(16) float2 sp[3][kRotWarps][kRotRows][MAXI];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2 w[MAXI], sh[MAXI];
#pragma unroll
  for (int i = 0; i < MAXI; ++i) {
    w[i] = sh[i] = make_float2(0.f, 0.f);
    if (i < R && lane < R) {
      const double2 a = Wm[i * R + lane];
      const double2 b = Sm[lane * R + i];      // S^dagger[i][j] = conj(S[j][i])
      w[i] = make_float2((float)a.x, (float)a.y);
      sh[i] = make_float2((float)b.x, -(float)b.y);
    }
  }
  const bool two = P2 != nullptr;
  const int64_t step = (int64_t)gridDim.x * kRotWarps * kRotRows;
  int64_t n0 = ((int64_t)blockIdx.x * kRotWarps + warp) * kRotRows;
  float2 pa[kRotRows], pb[kRotRows], pd[kRotRows];
  auto load = [&](int64_t base) {
#pragma unroll
    for (int r = 0; r < kRotRows; ++r) {
      const int64_t n = base + r;
      pa[r] = pb[r] = pd[r] = make_float2(0.f, 0.f);
      if (lane < R && n < N) {
        pa[r] = P1[n * R + lane];
        if (two) pb[r] = P2[n * R + lane];
        pd[r] = D[n * R + lane];
      }
    }
  };
  load(n0);
  for (; n0 < N; n0 += step) {
#pragma unroll
    for (int r = 0; r < kRotRows; ++r)
      if (lane < MAXI) {
        sp[0][warp][r][lane] = pa[r];
        sp[1][warp][r][lane] = pb[r];
        sp[2][warp][r][lane] = pd[r];
      }
    __syncwarp();
    load(n0 + step);
    float2 a1[kRotRows], a2[kRotRows], dd[kRotRows];
#pragma unroll
    for (int r = 0; r < kRotRows; ++r) a1[r] = a2[r] = dd[r] = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < MAXI; i += 2) {
#pragma unroll
      for (int r = 0; r < kRotRows; ++r) {
        const float4 x1 = *reinterpret_cast<const float4*>(&sp[0][warp][r][i]);
        const float4 xd = *reinterpret_cast<const float4*>(&sp[2][warp][r][i]);
        a1[r] = cfma(make_float2(x1.x, x1.y), w[i], a1[r]);
        a1[r] = cfma(make_float2(x1.z, x1.w), w[i + 1], a1[r]);
        dd[r] = cfma(make_float2(xd.x, xd.y), sh[i], dd[r]);
        dd[r] = cfma(make_float2(xd.z, xd.w), sh[i + 1], dd[r]);
        if (two) {
          const float4 x2 = *reinterpret_cast<const float4*>(&sp[1][warp][r][i]);
          a2[r] = cfma(make_float2(x2.x, x2.y), w[i], a2[r]);
          a2[r] = cfma(make_float2(x2.z, x2.w), w[i + 1], a2[r]);
        }
      }
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < kRotRows; ++r) {
      const int64_t n = n0 + r;
      if (lane < R && n < N) {
        P1[n * R + lane] = a1[r];
        if (two) P2[n * R + lane] = a2[r];
        const float2 base = two ? a2[r] : a1[r];
        D[n * R + lane] = make_float2(dd[r].x + base.x, dd[r].y + base.y);
      }
    }
  }
}

// ---------------------------------------------------------- small algebra
struct Small {           // device-resident solver state (R <= 64)
  double2 C[64 * 64];    // k x R (rows >= k zero)
  double2 S[64 * 64];
  double2 W[64 * 64];
  double2 M[64 * 64];    // inverse of D^dagger Z on the active block
  double2 MC[64 * 64];   // M C
  double2 negM[64 * 64];
  double2 G[64 * 64];    // Gram workspace (filled by gram kernels)
  double2 G2[64 * 64];   // second Gram (t^dagger t)
  double2 Y[64 * 64];    // projection coefficients N_i D_i^dagger F (kept blocks)
  double est[64];        // per-column residual estimate (relative)
  double target[64];     // per-column stopping level (absolute, same units)
  int32_t rank;
  int32_t flag;          // bit 0 converged, bit 1 breakdown, bit 2 non-finite
};

// Start: factor G = Gram of the initial residual block -> C = S, W (q <- q W).
__global__ void k_small_start(Small* st, int R, double tau) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* sA = reinterpret_cast<double2*>(smem_raw);
  double2* sS = sA + R * R;
  double2* sW = sS + R * R;
  __shared__ int perm[64];
  const int k = factor_block(st->G, R, R, R, tau, sA, sS, sW, perm, st->C, st->W);
  for (int i = threadIdx.x; i < R * R; i += blockDim.x) st->S[i] = st->C[i];
  if (threadIdx.x == 0) {
    st->rank = k;
    st->flag = 0;
    for (int i = 0; i < R * R; ++i)
      if (!isfinite(st->G[i].x) || !isfinite(st->G[i].y)) st->flag |= 4;
  }
}

// The nrhs x nrhs steps of an iteration, split so that only the
// factorisation (inherently sequential) runs on one CTA; the products run
// one CTA per row or column (on B300 one SM's FP64 rate made them the bulk
// of a single-CTA kernel).  Sums run in the same order as a plain loop, so
// the results do not depend on the split.
//
// M step: factor the Gram D^dagger Z (rank checked against the block's), then
// M = W W^dagger, negM = -M (k_small_WWh) and MC = M C (k_small_mul).
// A Gram whose diagonal is not finite: a NaN or Inf in either block makes
// some diagonal entry non-finite (|NaN|^2 and |Inf|^2 are), where the pivoted
// factorisation would only see rank loss and the loop would run to its cap.
__device__ bool diag_finite(const double2* G, int R) {
  for (int j = 0; j < R; ++j)
    if (!isfinite(G[j * R + j].x)) return false;
  return true;
}

__global__ void k_small_Mf(Small* st, int R, double tau) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* sA = reinterpret_cast<double2*>(smem_raw);
  double2* sS = sA + R * R;
  double2* sW = sS + R * R;
  __shared__ int perm[64];
  const int k_in = st->rank;
  const int k = factor_block(st->G, R, R, k_in, tau, sA, sS, sW, perm, nullptr, st->W);
  if (threadIdx.x == 0) {
    if (k < k_in) st->flag |= 2;                      // D^dagger H D lost rank
    if (!diag_finite(st->G, R)) st->flag |= 4;        // a NaN or Inf reached the Gram
  }
}

// M = W W^dagger and negM = -M: block i (row), thread j (column)
__global__ void k_small_WWh(Small* st, int R) {
  const int i = blockIdx.x, j = threadIdx.x;
  if (j >= R) return;
  double2 acc = make_double2(0.0, 0.0);
  for (int l = 0; l < R; ++l) {
    const double2 a = st->W[i * R + l], b = st->W[j * R + l];
    acc = cfma(a, make_double2(b.x, -b.y), acc);
  }
  st->M[i * R + j] = acc;
  st->negM[i * R + j] = make_double2(-acc.x, -acc.y);
}

// S step.  Preconditioned form first: est_j^2 = (C^dagger G2 C)_jj with
// G2 = t^dagger t and the old C; block j (column), thread a.
__global__ void k_small_est_pre(Small* st, int R) {
  __shared__ double part[64];
  const int j = blockIdx.x, a = threadIdx.x;
  if (a < R) {
    double2 v = make_double2(0.0, 0.0);
    for (int b = 0; b < R; ++b) v = cfma(st->G2[a * R + b], st->C[b * R + j], v);
    const double2 c = st->C[a * R + j];
    part[a] = c.x * v.x + c.y * v.y;                 // Re(conj(C_aj) v_aj)
  }
  __syncthreads();
  if (a == 0) {
    double s = 0.0;
    for (int i = 0; i < R; ++i) s += part[i];
    st->est[j] = sqrt(fmax(s, 0.0));
  }
}

// factor T^dagger t -> S, W and the new rank (one CTA)
__global__ void k_small_Sf(Small* st, int R, double tau) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* sA = reinterpret_cast<double2*>(smem_raw);
  double2* sS = sA + R * R;
  double2* sW = sS + R * R;
  __shared__ int perm[64];
  const int k_in = st->rank;
  const int k = factor_block(st->G, R, R, k_in, tau, sA, sS, sW, perm, st->S, st->W);
  if (threadIdx.x == 0) {
    st->rank = k;
    if (!diag_finite(st->G, R)) st->flag |= 4;        // a NaN or Inf reached the Gram
  }
}

// C <- S C in place, block j owning column j; unpreconditioned form: est_j =
// |(S C) e_j| (Q orthonormal)
__global__ void k_small_SC(Small* st, int R, int precond) {
  __shared__ double2 col[64];
  __shared__ double part[64];
  const int j = blockIdx.x, i = threadIdx.x;
  if (i < R) col[i] = st->C[i * R + j];
  __syncthreads();
  if (i < R) {
    double2 acc = make_double2(0.0, 0.0);
    for (int l = 0; l < R; ++l) acc = cfma(st->S[i * R + l], col[l], acc);
    st->C[i * R + j] = acc;
    part[i] = acc.x * acc.x + acc.y * acc.y;
  }
  __syncthreads();
  if (!precond && i == 0) {
    double s = 0.0;
    for (int a = 0; a < R; ++a) s += part[a];
    st->est[j] = sqrt(s);
  }
}

// convergence, breakdown and non-finite flags of the S step
__global__ void k_small_flags(Small* st, int R) {
  if (threadIdx.x != 0) return;
  int conv = 1;
  for (int j = 0; j < R; ++j) {
    if (!isfinite(st->est[j])) st->flag |= 4;
    if (!(st->est[j] <= st->target[j])) conv = 0;
  }
  if (st->rank == 0) conv = 1;
  if (conv) st->flag |= 1;
}

// deterministic start vector in [-1, 1] (an integer hash of the index)
template <typename C>
__global__ void k_init_vec(C* v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t h = (uint64_t)i * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    h ^= h >> 31;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 29;
    C c;
    c.x = (typename real_of<C>::type)((double)(h & 0xFFFFFF) / 8388608.0 - 1.0);
    c.y = (typename real_of<C>::type)((double)((h >> 24) & 0xFFFFFF) / 8388608.0 - 1.0);
    v[i] = c;
  }
}
template <typename C>
__global__ void k_scale_vec(C* out, const C* in, double f, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    C c = in[i];
    c.x = (typename real_of<C>::type)(c.x * f);
    c.y = (typename real_of<C>::type)(c.y * f);
    out[i] = c;
  }
}

// Keep this iteration's search block: D -> slot ctr[0] (if below the
// available count ctr[2] and the block has full rank R) and
// N = (D^dagger H D)^-1 beside it; the last block to finish advances
// ctr[0].  Every block reads ctr[0] before any block takes its ticket, so
// all of them see the same slot; the counters live on the device, so a
// captured CUDA graph replays this correctly.
__global__ void __launch_bounds__(256) k_store_block(void* const* table, double2* nmat,
                                                     int32_t* ctr, const float2* __restrict__ D,
                                                     const double2* __restrict__ M,
                                                     const int32_t* rank, int R, int64_t n) {
  __shared__ int s_slot, s_avail, s_full;
  if (threadIdx.x == 0) {
    s_slot = ((volatile int32_t*)ctr)[0];
    s_avail = ((volatile int32_t*)ctr)[2];
    s_full = *rank == R;   // a block that lost rank is not kept
  }
  __syncthreads();
  const int slot = s_slot;
  const int RR = R * R;
  const bool keep = slot < s_avail && s_full;
  if (keep) {
    float4* dst = (float4*)table[slot];
    const float4* src = (const float4*)D;
    const int64_t n4 = n >> 1;   // two complex64 per 16 bytes
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * blockDim.x)
      dst[i] = src[i];
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) ((float2*)dst)[n - 1] = D[n - 1];
    if (blockIdx.x == 0)
      for (int e = threadIdx.x; e < RR; e += blockDim.x) nmat[(int64_t)slot * RR + e] = M[e];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd((unsigned*)&ctr[1], 1u);
    if (t == gridDim.x - 1) {
      ctr[1] = 0;
      if (keep) ctr[0] = slot + 1;
      __threadfence();
    }
  }
}

// Galerkin start accepted per column only if it lowers the energy
// functional phi_j = e_j^dagger H e_j - 2 Re e_j^dagger f_j below its value
// at e_j = 0 (phi = |e - e*|_H^2 - |e*|_H^2): G = E^dagger (H E), G2 =
// E^dagger F; a rejected column of E and of H E is zeroed.
__global__ void k_start_guard(Small* st, int R) {
  const int j = threadIdx.x;
  if (j < R) {
    const double phi = st->G[j * R + j].x - 2.0 * st->G2[j * R + j].x;
    st->est[j] = phi < 0.0 ? 1.0 : 0.0;    // est[] is free before the first iteration
  }
}
__global__ void k_mask_cols(float2* E, float2* HE, const Small* st, int64_t N, int R) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N * R;
       i += (int64_t)gridDim.x * blockDim.x)
    if (st->est[i % R] == 0.0) {
      E[i] = make_float2(0.f, 0.f);
      HE[i] = make_float2(0.f, 0.f);
    }
}

// Y = A B for R x R complex matrices (row-major): block i, thread j
__global__ void k_small_mul(double2* Y, const double2* A, const double2* B, int R) {
  const int i = blockIdx.x, j = threadIdx.x;
  if (j >= R) return;
  double2 acc = make_double2(0.0, 0.0);
  for (int l = 0; l < R; ++l) acc = cfma(A[i * R + l], B[l * R + j], acc);
  Y[i * R + j] = acc;
}

int grid_for(int64_t n) {
  int64_t g = (n + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

// A NaN or Inf in a right-hand side or an initial guess shows as a
// non-finite column norm (so does an entry above about 1e154, whose square
// overflows the FP64 sum); the solves refuse such input before iterating
// instead of treating the column as a zero one.
// Inner tolerance of refinement cycle `cycle` (0: the first).  A later cycle
// starts from a residual whose low modes dominate, and for those the Krylov
// operator's own error bounds the reduction the cycle can reach.
double cycle_inner_tol(const mrhs_solve_params& p, int cycle) {
  return (cycle > 0 && p.inner_tol_later > 0.0) ? p.inner_tol_later : p.inner_tol;
}

int finite_columns(const std::vector<double>& norm, const std::string& what) {
  for (size_t j = 0; j < norm.size(); ++j)
    if (!std::isfinite(norm[j]))
      return fail(MRHS_ERR_NONFINITE,
                  what + " column " + std::to_string(j) + " is not finite");
  return MRHS_OK;
}

// ---------------------------------------------------------- host driver
struct Ctx {
  mrhs_op_s* op;
  cudaStream_t s;
  int R;
  int64_t N;
  double tau;
  Small* st = nullptr;        // device
  double2* gpart = nullptr;   // Gram partials
  double* npart = nullptr;    // column-norm partials
  int64_t applies[MRHS_NUM_PREC] = {};
  bool use_graph = true;
  // bump allocation from one grow-only operator-owned workspace: a first
  // pass with base == nullptr only sums the sizes
  char* base = nullptr;
  size_t used = 0;
  template <typename T>
  int alloc(T** p, size_t count) {
    const size_t off = (used + 255) / 256 * 256;
    used = off + sizeof(T) * count;
    *p = base ? (T*)(base + off) : nullptr;
    return MRHS_OK;
  }
  int apply(int prec, const void* X, void* Y) {
    applies[prec]++;
    return op_apply(op, prec, false, X, Y, R, s);
  }
  template <typename C>
  int gram(const C* X, const C* Y, double2* G) {
    return gram_ws(X, Y, G, N, R, R, sizeof(C) == 16 ? MRHS_C128 : MRHS_C64, gpart, s);
  }
  template <typename C>
  int colnorms(const C* X, double* out) {
    int nblk = num_sms() * 2;
    int64_t per = (N + nblk - 1) / nblk;
    if (per < 1) per = 1;
    nblk = (int)((N + per - 1) / per);
    if (nblk < 1) nblk = 1;
    { k_colnorm_partial<C><<<nblk, kThreads, 0, s>>>(X, npart, N, R, per); ::mrhs::count_launch(); }
    { k_colnorm_final<<<1, 64, 0, s>>>(npart, out, nblk, R); ::mrhs::count_launch(); }
    MRHS_CUDA_TRY(cudaGetLastError());
    return MRHS_OK;
  }
  int small_launch(int which, int precond = 0) {
    const size_t smem = factor_smem_bytes(R);
    if (which == 0) {
      MRHS_CUDA_TRY(cudaFuncSetAttribute(k_small_start, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      { k_small_start<<<1, 256, smem, s>>>(st, R, tau); ::mrhs::count_launch(); }
    } else if (which == 1) {
      MRHS_CUDA_TRY(cudaFuncSetAttribute(k_small_Mf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      { k_small_Mf<<<1, 256, smem, s>>>(st, R, tau); ::mrhs::count_launch(); }
      { k_small_WWh<<<R, 64, 0, s>>>(st, R); ::mrhs::count_launch(); }
      { k_small_mul<<<R, 64, 0, s>>>(st->MC, st->M, st->C, R); ::mrhs::count_launch(); }
    } else {
      if (precond) { k_small_est_pre<<<R, 64, 0, s>>>(st, R); ::mrhs::count_launch(); }
      MRHS_CUDA_TRY(cudaFuncSetAttribute(k_small_Sf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      { k_small_Sf<<<1, 256, smem, s>>>(st, R, tau); ::mrhs::count_launch(); }
      { k_small_SC<<<R, 64, 0, s>>>(st, R, precond); ::mrhs::count_launch(); }
      { k_small_flags<<<1, 32, 0, s>>>(st, R); ::mrhs::count_launch(); }
    }
    MRHS_CUDA_TRY(cudaGetLastError());
    return MRHS_OK;
  }
  template <typename C>
  int rotate(C* P1, C* P2, C* D) {
    if (sizeof(C) == sizeof(float2) &&
        update_tc_applies(P1, P1, D, N, R, R, MRHS_C64, R) &&
        (P2 == nullptr || update_tc_applies(P2, P2, D, N, R, R, MRHS_C64, R))) {
      // tensor cores (blas_tc.cu): P1 <- P1 W, P2 <- P2 W, D <- P + D S^dagger
      MRHS_TRY(update_tc(P1, P1, nullptr, st->W, 0, 0.0, N, R, R, s));
      if (P2) MRHS_TRY(update_tc(P2, P2, nullptr, st->W, 0, 0.0, N, R, R, s));
      return update_tc(D, D, P2 ? P2 : P1, st->S, 1, 1.0, N, R, R, s);
    }
    if (sizeof(C) == sizeof(float2) && R <= 32) {
      float2 *p1 = (float2*)P1, *p2 = (float2*)P2, *d = (float2*)D;
      int64_t g = (N + kRotWarps * kRotRows - 1) / (kRotWarps * kRotRows);
      const int64_t capw = (int64_t)num_sms() * 2;   // the resident CTAs (241 registers)
      if (g > capw) g = capw;
      if (R <= 8)
        { k_rotate_w<8><<<(unsigned)g, kRotWarps * 32, 0, s>>>(p1, p2, d, st->W, st->S, N, R); ::mrhs::count_launch(); }
      else if (R <= 16)
        { k_rotate_w<16><<<(unsigned)g, kRotWarps * 32, 0, s>>>(p1, p2, d, st->W, st->S, N, R); ::mrhs::count_launch(); }
      else
        { k_rotate_w<32><<<(unsigned)g, kRotWarps * 32, 0, s>>>(p1, p2, d, st->W, st->S, N, R); ::mrhs::count_launch(); }
      MRHS_CUDA_TRY(cudaGetLastError());
      return MRHS_OK;
    }
    const size_t smem = sizeof(C) * (2 * (size_t)R * R + 3 * (size_t)kTile * R);
    MRHS_CUDA_TRY(cudaFuncSetAttribute(k_rotate<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int64_t grid = (N + kTile - 1) / kTile;
    const int64_t cap = (int64_t)num_sms() * 16;
    if (grid > cap) grid = cap;
    { k_rotate<C><<<(unsigned)grid, kThreads, smem, s>>>(P1, P2, D, st->W, st->S, N, R); ::mrhs::count_launch(); }
    MRHS_CUDA_TRY(cudaGetLastError());
    return MRHS_OK;
  }
};

void cheb_coeffs(double lo, double hi, int order, std::vector<double>& c) {
  const int m1 = order + 1;
  c.assign(m1, 0.0);
  for (int j = 0; j < m1; ++j) {
    double s = 0.0;
    for (int k = 0; k < m1; ++k) {
      const double th = M_PI * (k + 0.5) / m1;
      const double x = 0.5 * ((hi - lo) * std::cos(th) + hi + lo);
      s += std::cos(j * th) / x;
    }
    c[j] = 2.0 * s / m1;
  }
  c[0] *= 0.5;
}

// P = p(H) X, recurrence buffers W, T1, T2 (each N x R of type C).
template <typename C>
int cheb_run(Ctx& cx, int prec, double lo, double hi, int order, const C* X, C* P, C* W, C* T1,
             C* T2) {
  std::vector<double> c;
  cheb_coeffs(lo, hi, order, c);
  const double a = 2.0 / (hi - lo), b = -(hi + lo) / (hi - lo);
  const int64_t n = cx.N * cx.R;
  const int g = grid_for(n);
  if (order == 0) {
    { k_cheb_first<C><<<g, kThreads, 0, cx.s>>>(T1, P, X, X, 0.0, 0.0, c[0], 0.0, n); ::mrhs::count_launch(); }
    MRHS_CUDA_TRY(cudaGetLastError());
    return MRHS_OK;
  }
  if (MRHS_PREC_IS_TC(prec) && sizeof(C) == sizeof(float2)) {
    // each step inside the operator's epilogue: W is never stored, and the
    // step's output column maxima are ready for the next application's packing
    ChebFuse f;
    f.mode = 1;
    f.a = (float)a;
    f.b = (float)b;
    f.c0 = (float)c[0];
    f.c = (float)c[1];
    f.Tout = T1;
    f.P = P;
    f.colmax_next = order >= 2;
    const void* in = X;
    void* none = nullptr;
    int32_t R = cx.R;
    mrhs_op_s* op = cx.op;
    cx.applies[prec]++;
    MRHS_TRY(tc_apply_batch(&op, 1, prec, &in, &none, &R, nullptr, cx.s, nullptr, &f));
    const C* Tprev = X;
    C* Tcur = T1;
    for (int j = 2; j <= order; ++j) {
      C* dst = (Tprev == X) ? T2 : const_cast<C*>(Tprev);
      f.mode = 2;
      f.c = (float)c[j];
      f.Tout = dst;
      f.Tp = Tprev;
      f.colmax_next = j < order;
      f.colmax_ready = true;
      in = Tcur;
      cx.applies[prec]++;
      MRHS_TRY(tc_apply_batch(&op, 1, prec, &in, &none, &R, nullptr, cx.s, nullptr, &f));
      Tprev = Tcur;
      Tcur = dst;
    }
    return MRHS_OK;
  }
  MRHS_TRY(cx.apply(prec, X, W));
  { k_cheb_first<C><<<g, kThreads, 0, cx.s>>>(T1, P, W, X, a, b, c[0], c[1], n); ::mrhs::count_launch(); }
  MRHS_CUDA_TRY(cudaGetLastError());
  const C* Tprev = X;   // T_{j-1}
  C* Tcur = T1;         // T_j
  for (int j = 2; j <= order; ++j) {
    MRHS_TRY(cx.apply(prec, Tcur, W));
    // T_{j+1} goes over T_{j-1}, except that the input X is never written
    C* dst = (Tprev == X) ? T2 : const_cast<C*>(Tprev);
    { k_cheb_step<C><<<g, kThreads, 0, cx.s>>>(dst, P, W, Tcur, Tprev, a, b, c[j], n); ::mrhs::count_launch(); }
    MRHS_CUDA_TRY(cudaGetLastError());
    Tprev = Tcur;
    Tcur = dst;
  }
  return MRHS_OK;
}

// ---------------------------------------------------------- kept search blocks
constexpr int kRecycleMax = 256;       // slots in the device table
constexpr int kRecycleDefault = 128;   // cap when recycle_max_blocks = 0
constexpr int kRecycleHeadroom = 64;   // slots made available ahead of a cycle

struct RecycleStore {
  mrhs_op_s* op = nullptr;
  double2* nmat = nullptr;   // [kRecycleMax][R][R]
  int64_t n = 0;             // complex64 elements per block (N R)
  int R = 0, cap = 0;
  int used = 0;              // slots holding blocks of finished cycles
  int avail = 0;             // slots with memory behind them
  std::vector<std::pair<int, int>> cycles;   // [first, end) per finished cycle
  const float2* block(int slot) const { return (const float2*)op->rc_slots[slot]; }
  const double2* N(int slot) const { return nmat + (int64_t)slot * R * R; }
  // launched inside the block-CG iteration (also under graph capture)
  int store(cudaStream_t s, const float2* D, const double2* M, const int32_t* rank) const {
    int g = num_sms() * 4;
    const int64_t need = (n / 2 + 255) / 256;
    if (need < g) g = need > 0 ? (int)need : 1;
    { k_store_block<<<g, 256, 0, s>>>(op->rc_table, nmat, op->rc_ctr, D, M, rank, R, n); ::mrhs::count_launch(); }
    MRHS_CUDA_TRY(cudaGetLastError());
    return MRHS_OK;
  }
};

int recycle_setup(mrhs_op_s* op, int64_t N, int R, int max_blocks, cudaStream_t s,
                  RecycleStore* rs) {
  const size_t bytes = sizeof(float2) * (size_t)N * R;
  if (op->rc_slot_bytes < bytes) {
    recycle_release(op);
    op->rc_slot_bytes = bytes;
  }
  if (!op->rc_table) MRHS_CUDA_TRY(cudaMalloc(&op->rc_table, sizeof(void*) * kRecycleMax));
  if (!op->rc_ctr) MRHS_CUDA_TRY(cudaMalloc(&op->rc_ctr, 4 * sizeof(int32_t)));
  MRHS_TRY(op->ws_rcn.ensure(sizeof(double2) * kRecycleMax * R * R));
  rs->op = op;
  rs->nmat = (double2*)op->ws_rcn.ptr;
  rs->n = N * R;
  rs->R = R;
  rs->cap = max_blocks > 0 ? std::min(max_blocks, kRecycleMax) : kRecycleDefault;
  rs->used = 0;
  rs->avail = 0;
  rs->cycles.clear();
  MRHS_CUDA_TRY(cudaMemsetAsync(op->rc_ctr, 0, 4 * sizeof(int32_t), s));
  return MRHS_OK;
}

// Before a cycle: slots up to used + headroom (within the cap), allocating
// while free memory stays above max(4 GiB, 1/16 of the device); the table
// and the counters {used, 0, avail} go to the device.
int recycle_grow(RecycleStore& rs, cudaStream_t s) {
  mrhs_op_s* op = rs.op;
  const int want = std::min(rs.cap, rs.used + kRecycleHeadroom);
  size_t fr = 0, tot = 0;
  MRHS_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
  const size_t reserve = std::max<size_t>((size_t)4 << 30, tot / 16);
  const size_t before = op->rc_slots.size();
  while ((int)op->rc_slots.size() < want && fr >= op->rc_slot_bytes + reserve) {
    void* ptr = nullptr;
    if (cudaMalloc(&ptr, op->rc_slot_bytes) != cudaSuccess) {
      cudaGetLastError();
      break;
    }
    op->rc_slots.push_back(ptr);
    fr -= op->rc_slot_bytes;
  }
  rs.avail = std::min(want, (int)op->rc_slots.size());
  if (op->rc_slots.size() != before || before == 0)
    MRHS_CUDA_TRY(cudaMemcpyAsync(op->rc_table, op->rc_slots.data(),
                                  sizeof(void*) * op->rc_slots.size(), cudaMemcpyHostToDevice, s));
  const int32_t ctr[4] = {rs.used, 0, rs.avail, 0};
  MRHS_CUDA_TRY(cudaMemcpyAsync(op->rc_ctr, ctr, sizeof(ctr), cudaMemcpyHostToDevice, s));
  MRHS_CUDA_TRY(cudaStreamSynchronize(s));   // ctr lives on this stack frame
  return MRHS_OK;
}

// After a cycle (stream synchronised): the slots it filled.
int recycle_close_cycle(RecycleStore& rs, cudaStream_t s) {
  int32_t next = 0;
  MRHS_CUDA_TRY(cudaMemcpyAsync(&next, rs.op->rc_ctr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  MRHS_CUDA_TRY(cudaStreamSynchronize(s));
  const int end = std::min((int)next, rs.avail);
  if (end > rs.used) rs.cycles.push_back({rs.used, end});
  rs.used = std::max(rs.used, end);
  return MRHS_OK;
}

// Galerkin start of a refinement cycle from the kept blocks.  The blocks of
// one earlier cycle are mutually H-conjugate (D_i^dagger H D_j = 0, i != j,
// and N_i = (D_i^dagger H D_i)^-1), so the correction over that cycle's span
// is sum_i D_i N_i D_i^dagger Fr.  Earlier cycles are taken one after
// another, Fr = F - H E recomputed before each, `sweeps` times over all.
int recycle_project(Ctx& cx, const RecycleStore& rs, int sweeps, int prec, const float2* F,
                    float2* E, float2* Fr, float2* HE, int* nproj) {
  const int64_t n = cx.N * cx.R;
  const int g = grid_for(n);
  bool zero = true;   // E is still zero: Fr = F
  for (int sw = 0; sw < sweeps; ++sw)
    for (const auto& c : rs.cycles) {
      const float2* fr = F;
      if (!zero) {
        MRHS_TRY(cx.apply(prec, E, HE));
        { k_sub<float2><<<g, kThreads, 0, cx.s>>>(Fr, F, HE, n); ::mrhs::count_launch(); }
        MRHS_CUDA_TRY(cudaGetLastError());
        fr = Fr;
      }
      for (int slot = c.first; slot < c.second; ++slot) {
        MRHS_TRY(cx.gram<float2>(rs.block(slot), fr, cx.st->G));            // D_i^dagger Fr
        { k_small_mul<<<cx.R, 64, 0, cx.s>>>(cx.st->Y, rs.N(slot), cx.st->G, cx.R); ::mrhs::count_launch(); }
        MRHS_CUDA_TRY(cudaGetLastError());
        MRHS_TRY(axpy(E, rs.block(slot), cx.st->Y, 1.0, cx.N, cx.R, cx.R, MRHS_C64, cx.s));
        ++*nproj;
      }
      zero = false;
    }
  return MRHS_OK;
}

template <typename C>
struct BcgBufs {
  C *q = nullptr, *Q = nullptr, *D = nullptr, *z = nullptr, *Zz = nullptr;
  C *cw = nullptr, *c1 = nullptr, *c2 = nullptr;
  void carve(Ctx& cx, int64_t n, bool precond) {
    cx.alloc(&q, n);
    cx.alloc(&D, n);
    cx.alloc(&z, n);
    if (precond) {
      cx.alloc(&Q, n);
      cx.alloc(&Zz, n);
      cx.alloc(&cw, n);
      cx.alloc(&c1, n);
      cx.alloc(&c2, n);
    } else {
      Q = q;
    }
  }
};

// One block-CG run on H E = F (type C), E in/out. target[j]: absolute
// stopping level of column j (estimates are in the units of F).
template <typename C>
int run_bcg(Ctx& cx, BcgBufs<C>& b, int prec, const C* F, C* E, const double* target_host,
            bool precond, int pprec, double lo, double hi, int order, int maxiter,
            int check_every, int* iters, int* flag_out, const RecycleStore* keep = nullptr,
            bool guard_start = false, bool e_zero = false) {
  const int64_t n = cx.N * cx.R;
  const int g = grid_for(n);
  const int dt = sizeof(C) == 16 ? MRHS_C128 : MRHS_C64;
  C *q = b.q, *Q = b.Q, *D = b.D, *z = b.z;
  MRHS_CUDA_TRY(cudaMemcpyAsync(cx.st->target, target_host, sizeof(double) * cx.R,
                                cudaMemcpyHostToDevice, cx.s));
  MRHS_CUDA_TRY(cudaMemsetAsync(&cx.st->flag, 0, sizeof(int), cx.s));
  // r0 = F - H E; with E known to be zero (H 0 = 0 exactly) r0 = F
  if (e_zero) {
    MRHS_CUDA_TRY(cudaMemcpyAsync(q, F, sizeof(C) * n, cudaMemcpyDeviceToDevice, cx.s));
  } else {
    MRHS_TRY(cx.apply(prec, E, z));
    if (guard_start && sizeof(C) == sizeof(float2)) {
      MRHS_TRY(cx.gram<C>(E, z, cx.st->G));                                    // E^dag H E
      MRHS_TRY(cx.gram<C>(E, F, cx.st->G2));                                   // E^dag F
      { k_start_guard<<<1, 64, 0, cx.s>>>(cx.st, cx.R); ::mrhs::count_launch(); }
      { k_mask_cols<<<g, kThreads, 0, cx.s>>>((float2*)E, (float2*)z, cx.st, cx.N, cx.R); ::mrhs::count_launch(); }
      MRHS_CUDA_TRY(cudaGetLastError());
    }
    { k_sub<C><<<g, kThreads, 0, cx.s>>>(q, F, z, n); ::mrhs::count_launch(); }
    MRHS_CUDA_TRY(cudaGetLastError());
  }
  if (precond) {
    MRHS_TRY(cheb_run<C>(cx, pprec, lo, hi, order, q, Q, b.cw, b.c1, b.c2));   // Z0 = M^-1 r0
    MRHS_TRY(cx.gram<C>(Q, q, cx.st->G));                                      // Z0^dag r0
  } else {
    MRHS_TRY(cx.gram<C>(q, q, cx.st->G));                                      // R0^dag R0
  }
  MRHS_TRY(cx.small_launch(0));
  // q <- q W (Q <- Q W), D <- Q: rotate with D = 0 and S = 0
  MRHS_CUDA_TRY(cudaMemsetAsync(D, 0, sizeof(C) * n, cx.s));
  MRHS_CUDA_TRY(cudaMemsetAsync(cx.st->S, 0, sizeof(double2) * 64 * 64, cx.s));
  MRHS_TRY(cx.rotate<C>(q, precond ? Q : nullptr, D));
  int it = 0, flag = 0, stalled = 0;
  double best = 1e300;
  std::vector<double> est(cx.R);
  const int stall_checks = check_every > 0 ? (32 + check_every - 1) / check_every : 0;
  // one block-CG iteration (Fig. 2): fixed launches on fixed buffers, so a
  // chunk of `check_every` of them can be captured once as a CUDA graph
  auto body = [&]() -> int {
    MRHS_TRY(cx.apply(prec, D, z));                                            // z = H D
    if (precond) MRHS_TRY(cheb_run<C>(cx, pprec, lo, hi, order, z, b.Zz, b.cw, b.c1, b.c2));
    MRHS_TRY(cx.gram<C>(D, z, cx.st->G));                                      // D^dag z
    MRHS_TRY(cx.small_launch(1));                                              // M, MC, -M
    if (keep && sizeof(C) == sizeof(float2))                                   // D, M kept
      MRHS_TRY(keep->store(cx.s, (const float2*)D, cx.st->M, &cx.st->rank));
    MRHS_TRY(axpy(E, D, cx.st->MC, 1.0, cx.N, cx.R, cx.R, dt, cx.s));          // E += D M C
    MRHS_TRY(axpy(q, z, cx.st->negM, 1.0, cx.N, cx.R, cx.R, dt, cx.s));        // t = q - z M
    if (precond) {
      MRHS_TRY(axpy(Q, b.Zz, cx.st->negM, 1.0, cx.N, cx.R, cx.R, dt, cx.s));   // T = Q - Z M
      MRHS_TRY(cx.gram<C>(Q, q, cx.st->G));                                    // T^dag t
      MRHS_TRY(cx.gram<C>(q, q, cx.st->G2));                                   // t^dag t
    } else {
      MRHS_TRY(cx.gram<C>(q, q, cx.st->G));                                    // T^dag T
    }
    MRHS_TRY(cx.small_launch(2, precond ? 1 : 0));                             // S, W, C = S C
    MRHS_TRY(cx.rotate<C>(q, precond ? Q : nullptr, D));                       // q, Q, D
    return MRHS_OK;
  };
  bool timing = false;
  for (const auto& t : cx.op->timer) timing = timing || t.on;
  bool graph_ok = cx.use_graph && !timing && check_every > 1;
  int64_t graph_launches = 0;
  cudaGraphExec_t exec = nullptr;
  int64_t graph_applies[MRHS_NUM_PREC] = {};
  auto cleanup = [&]() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
  };
  it = 0;
  while (it < maxiter) {
    const int chunk = (maxiter - it) < check_every ? (maxiter - it) : check_every;
    if (graph_ok && it >= 1 && chunk == check_every) {
      if (!exec) {
        // workspaces were sized by the iterations already run uncaptured;
        // if capture or instantiation fails the chunk runs uncaptured instead
        int64_t before[MRHS_NUM_PREC];
        for (int i = 0; i < MRHS_NUM_PREC; ++i) before[i] = cx.applies[i];
        const int64_t l0 = launch_count();
        cudaGraph_t gr = nullptr;
        int st = cudaStreamBeginCapture(cx.s, cudaStreamCaptureModeThreadLocal) == cudaSuccess
                     ? MRHS_OK : MRHS_ERR_CUDA;
        for (int j = 0; j < chunk && st == MRHS_OK; ++j) st = body();
        const cudaError_t ce = cudaStreamEndCapture(cx.s, &gr);
        const bool ok = st == MRHS_OK && ce == cudaSuccess && gr &&
                        cudaGraphInstantiate(&exec, gr, 0) == cudaSuccess;
        if (gr) cudaGraphDestroy(gr);
        for (int i = 0; i < MRHS_NUM_PREC; ++i) {
          graph_applies[i] = cx.applies[i] - before[i];
          cx.applies[i] = before[i];
        }
        graph_launches = launch_count() - l0;
        add_launches(-graph_launches);
        if (!ok) {
          cudaGetLastError();
          if (exec) cudaGraphExecDestroy(exec);
          exec = nullptr;
          graph_ok = false;
          continue;   // nothing of the chunk ran: redo it uncaptured
        }
      }
      const cudaError_t le = cudaGraphLaunch(exec, cx.s);
      if (le != cudaSuccess) {
        cleanup();
        return fail(MRHS_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(le));
      }
      for (int i = 0; i < MRHS_NUM_PREC; ++i) cx.applies[i] += graph_applies[i];
      add_launches(graph_launches);
    } else {
      for (int j = 0; j < chunk; ++j) {
        const int st = body();
        if (st != MRHS_OK) {
          cleanup();
          return st;
        }
      }
    }
    it += chunk;
    MRHS_CUDA_TRY(cudaMemcpyAsync(&flag, &cx.st->flag, sizeof(int), cudaMemcpyDeviceToHost, cx.s));
    MRHS_CUDA_TRY(cudaMemcpyAsync(est.data(), cx.st->est, sizeof(double) * cx.R,
                                  cudaMemcpyDeviceToHost, cx.s));
    MRHS_CUDA_TRY(cudaStreamSynchronize(cx.s));
    if (flag & (1 | 4)) break;
    // stagnation: the worst column's distance to its target has not shrunk
    // by 30% over `stall_checks` reads (a low-precision preconditioner is
    // not exactly linear, so the recurrences can plateau above the target;
    // the caller then restarts from the true residual)
    double worst = 0.0;
    for (int j = 0; j < cx.R; ++j)
      if (target_host[j] > 0.0) worst = std::fmax(worst, est[j] / target_host[j]);
    if (worst < 0.7 * best) {
      best = worst;
      stalled = 0;
    } else if (stall_checks > 0 && ++stalled >= stall_checks) {
      flag |= 8;
      break;
    }
  }
  cleanup();
  if (it > maxiter) it = maxiter;
  *iters = it;
  *flag_out = flag;
  return MRHS_OK;
}

struct SolveBufs {
  double *bnorm_d = nullptr, *rnorm_d = nullptr, *rho_d = nullptr;
  double2* r64 = nullptr;
  float2 *f32 = nullptr, *e32 = nullptr;
  BcgBufs<double2> b64;
  BcgBufs<float2> b32;
  void carve(Ctx& cx, int R, int64_t n, bool mixed, bool precond) {
    const int nblk = num_sms() * 4;
    cx.alloc(&cx.st, 1);
    cx.alloc(&cx.gpart, gram_workspace_bytes(cx.N, R, R) / sizeof(double2) + 1);
    cx.alloc(&cx.npart, (size_t)nblk * R + R);
    cx.alloc(&bnorm_d, R);
    cx.alloc(&rnorm_d, R);
    cx.alloc(&rho_d, R);
    cx.alloc(&r64, n);
    if (mixed) {
      cx.alloc(&f32, n);
      cx.alloc(&e32, n);
      b32.carve(cx, n, precond);
    } else {
      b64.carve(cx, n, precond);
    }
  }
};

template <typename C>
int power_run(mrhs_op_s* op, int prec, int iters, cudaStream_t s, double* lam) {
  const int64_t n = op->V * op->nb;
  const size_t vb = (sizeof(C) * n + 255) / 256 * 256;
  const size_t part = gram_workspace_bytes(n, 1, 1);
  MRHS_TRY(op->ws_small.ensure(2 * vb + part + 256));
  char* base = (char*)op->ws_small.ptr;
  C* v = (C*)base;
  C* w = (C*)(base + vb);
  double2* G = (double2*)(base + 2 * vb);           // two 1 x 1 Grams
  double2* gp = G + 2;
  const int g = grid_for(n);
  const int dt = sizeof(C) == 16 ? MRHS_C128 : MRHS_C64;
  { k_init_vec<C><<<g, kThreads, 0, s>>>(v, n); ::mrhs::count_launch(); }
  double2 h[2];
  MRHS_TRY(gram_ws(v, v, G, n, 1, 1, dt, gp, s));
  MRHS_CUDA_TRY(cudaMemcpyAsync(h, G, sizeof(double2), cudaMemcpyDeviceToHost, s));
  MRHS_CUDA_TRY(cudaStreamSynchronize(s));
  { k_scale_vec<C><<<g, kThreads, 0, s>>>(v, v, 1.0 / std::sqrt(h[0].x), n); ::mrhs::count_launch(); }
  double est = 0.0;
  for (int it = 0; it < iters; ++it) {
    MRHS_TRY(op_apply(op, prec, false, v, w, 1, s));
    MRHS_TRY(gram_ws(v, w, G, n, 1, 1, dt, gp, s));       // v^dag H v (|v| = 1)
    MRHS_TRY(gram_ws(w, w, G + 1, n, 1, 1, dt, gp, s));   // |H v|^2
    MRHS_CUDA_TRY(cudaMemcpyAsync(h, G, 2 * sizeof(double2), cudaMemcpyDeviceToHost, s));
    MRHS_CUDA_TRY(cudaStreamSynchronize(s));
    est = h[0].x;
    if (!(h[1].x > 0.0) || !std::isfinite(h[1].x)) break;
    { k_scale_vec<C><<<g, kThreads, 0, s>>>(v, w, 1.0 / std::sqrt(h[1].x), n); ::mrhs::count_launch(); }
  }
  MRHS_CUDA_TRY(cudaGetLastError());
  // a NaN or Inf in the coefficients reaches the estimate: report it as such
  // (the Chebyshev interval built from it would only fail as an argument)
  if (!std::isfinite(est))
    return fail(MRHS_ERR_NONFINITE, "power-method estimate of lambda_max is not finite "
                                    "(non-finite operator coefficients?)");
  *lam = est;
  return MRHS_OK;
}

}  // namespace

void recycle_release(mrhs_op_s* op) {
  for (void* ptr : op->rc_slots) cudaFree(ptr);
  op->rc_slots.clear();
  op->rc_slot_bytes = 0;
  if (op->rc_table) cudaFree(op->rc_table);
  op->rc_table = nullptr;
  if (op->rc_ctr) cudaFree(op->rc_ctr);
  op->rc_ctr = nullptr;
  op->ws_rcn.release();
}

// Largest-eigenvalue estimate by the power method (Sec. 2.3 obtains the
// Chebyshev upper bound from a few power-method steps):
// Rayleigh quotient of H^k v0, one right-hand side, operator in `prec`.
int lambda_max(mrhs_op_s* op, int prec, int iters, cudaStream_t s, double* lam) {
  if (MRHS_PREC_IS_WIDE(prec))
    return power_run<double2>(op, prec, iters, s, lam);
  return power_run<float2>(op, prec, iters, s, lam);
}

int solve(mrhs_op_s* op, const double2* B, double2* X, int R, const mrhs_solve_params& p,
          mrhs_solve_info* info, cudaStream_t s) {
  auto t0 = std::chrono::steady_clock::now();
  Ctx cx;
  cx.op = op;
  cx.s = s;
  cx.R = R;
  cx.N = op->V * op->nb;
  cx.tau = p.breakdown_tau > 0 ? p.breakdown_tau : 1e-12;
  cx.use_graph = p.use_graph != 0;
  const int64_t n = cx.N * R;
  const int g = grid_for(n);
  const bool mixed = p.mode == MRHS_SOLVE_MIXED;
  SolveBufs sb;
  sb.carve(cx, R, n, mixed, p.precond != 0);          // sizing pass
  MRHS_TRY(op->ws_solve.ensure(cx.used));
  cx.base = (char*)op->ws_solve.ptr;
  cx.used = 0;
  sb.carve(cx, R, n, mixed, p.precond != 0);          // assignment pass
  MRHS_CUDA_TRY(cudaMemsetAsync(cx.st, 0, sizeof(Small), s));

  double lo = p.cheb_lo, hi = p.cheb_hi;
  if (p.precond && hi <= 0.0) {
    // cached power-method estimate in the preconditioner's precision, with
    // a margin: p(x) must not see eigenvalues above hi
    double& cached = op->lam_max[p.precond_prec];
    if (!(cached > 0.0)) MRHS_TRY(lambda_max(op, p.precond_prec, 40, s, &cached));
    hi = 1.08 * cached;
  }
  if (p.precond && lo <= 0.0) lo = hi / 400.0;
  if (p.precond && !(lo < hi)) return fail(MRHS_ERR_INVALID_ARG, "cheb_lo must be < cheb_hi");

  MRHS_TRY(cx.colnorms<double2>(B, sb.bnorm_d));
  std::vector<double> bnorm(R), rnorm(R), target(R);
  MRHS_CUDA_TRY(cudaMemcpyAsync(bnorm.data(), sb.bnorm_d, sizeof(double) * R,
                                cudaMemcpyDeviceToHost, s));
  MRHS_CUDA_TRY(cudaStreamSynchronize(s));
  MRHS_TRY(finite_columns(bnorm, "B"));
  { k_zero_cols<double2><<<g, kThreads, 0, s>>>(X, sb.bnorm_d, cx.N, R); ::mrhs::count_launch(); }
  int total_iters = 0, cycles = 0, status = MRHS_OK, flag = 0;

  // r64 = B - H X with the operator of precision `rp` (FP64 or DF32), rnorm
  auto residual_in = [&](int rp) -> int {
    MRHS_TRY(cx.apply(rp, X, sb.r64));
    { k_sub<double2><<<g, kThreads, 0, s>>>(sb.r64, B, sb.r64, n); ::mrhs::count_launch(); }
    MRHS_CUDA_TRY(cudaGetLastError());
    MRHS_TRY(cx.colnorms<double2>(sb.r64, sb.rnorm_d));
    MRHS_CUDA_TRY(cudaMemcpyAsync(rnorm.data(), sb.rnorm_d, sizeof(double) * R,
                                  cudaMemcpyDeviceToHost, s));
    MRHS_CUDA_TRY(cudaStreamSynchronize(s));
    return MRHS_OK;
  };
  auto all_done = [&]() {
    for (int j = 0; j < R; ++j)
      if (bnorm[j] > 0 && !(rnorm[j] <= p.tol * bnorm[j])) return false;
    return true;
  };
  // the cycle residual in residual_prec; one that meets tol is confirmed with
  // the FP64 operator (fp64_prec: native FP64 or the digit-sliced OZ form), so
  // convergence is always decided on an FP64 residual
  const int f64 = p.fp64_prec;
  const int res_prec = (mixed && p.residual_prec >= 0) ? p.residual_prec : f64;
  auto true_residual = [&]() -> int {
    MRHS_TRY(residual_in(res_prec));
    if (res_prec != f64 && all_done()) MRHS_TRY(residual_in(f64));
    return MRHS_OK;
  };
  // a zero initial guess needs no operator application: r = B
  bool x0_zero = false;
  auto initial_residual = [&]() -> int {
    std::vector<double> xn(R);
    MRHS_TRY(cx.colnorms<double2>(X, sb.rnorm_d));
    MRHS_CUDA_TRY(cudaMemcpyAsync(xn.data(), sb.rnorm_d, sizeof(double) * R,
                                  cudaMemcpyDeviceToHost, s));
    MRHS_CUDA_TRY(cudaStreamSynchronize(s));
    MRHS_TRY(finite_columns(xn, "X0"));
    bool zero = true;
    for (double v : xn) zero = zero && v == 0.0;
    x0_zero = zero;
    if (!zero) return true_residual();
    MRHS_CUDA_TRY(cudaMemcpyAsync(sb.r64, B, sizeof(double2) * n, cudaMemcpyDeviceToDevice, s));
    rnorm = bnorm;
    return MRHS_OK;
  };
  auto max_rel = [&]() {
    double m = 0.0;
    for (int j = 0; j < R; ++j)
      if (bnorm[j] > 0) m = std::fmax(m, rnorm[j] / bnorm[j]);
    return m;
  };
  const int every = p.check_every > 0 ? p.check_every : 1;
  if (info) {
    for (int c = 0; c < MRHS_MAX_CYCLES; ++c) {
      info->cycle_iters[c] = 0;
      info->cycle_resid[c] = 0.0;
      info->cycle_flag[c] = 0;
    }
    info->recycle_blocks = 0;
    info->recycle_projections = 0;
  }

  if (!mixed) {
    for (int j = 0; j < R; ++j) target[j] = p.tol * bnorm[j];
    MRHS_TRY(initial_residual());
    cycles = 0;
    if (!all_done()) {
      int it = 0;
      MRHS_TRY(run_bcg<double2>(cx, sb.b64, f64, B, X, target.data(), p.precond != 0,
                                p.precond_prec, lo, hi, p.cheb_order, p.maxiter, every, &it,
                                &flag, nullptr, false, x0_zero));
      total_iters = it;
      cycles = 1;
      MRHS_TRY(true_residual());
    }
  } else {
    MRHS_TRY(initial_residual());
    // search blocks of finished cycles, for the Galerkin start of the next
    RecycleStore keep;
    bool recycle = p.recycle > 0;
    int nproj = 0;
    if (recycle) MRHS_TRY(recycle_setup(op, cx.N, R, p.recycle_max_blocks, s, &keep));
    for (cycles = 0; cycles < p.max_cycles && !all_done() && total_iters < p.maxiter; ++cycles) {
      // scale each residual column to unit norm; inner target relative to 1
      std::vector<double> rho(R);
      // a cycle that needs less than a tenfold reduction on every column is
      // expected to finish the solve (TC32 inner solves reach 1/20..1/50 per
      // cycle even at kappa 1e4): its residual goes straight to FP64
      bool final_cycle = true;
      const double tol_c = cycle_inner_tol(p, cycles);
      for (int j = 0; j < R; ++j) {
        rho[j] = (bnorm[j] > 0 && rnorm[j] > p.tol * bnorm[j]) ? rnorm[j] : 0.0;
        const double want = rho[j] > 0 ? 0.5 * p.tol * bnorm[j] / rho[j] : 1.0;
        target[j] = std::fmax(tol_c, want);
        if (rho[j] > 0 && want < std::fmax(tol_c, kFinalCycleTarget)) final_cycle = false;
      }
      MRHS_CUDA_TRY(cudaMemcpyAsync(sb.rho_d, rho.data(), sizeof(double) * R,
                                    cudaMemcpyHostToDevice, s));
      { k_scale_to_c64<<<g, kThreads, 0, s>>>(sb.f32, sb.r64, sb.rho_d, cx.N, R); ::mrhs::count_launch(); }
      MRHS_CUDA_TRY(cudaMemsetAsync(sb.e32, 0, sizeof(float2) * n, s));
      MRHS_CUDA_TRY(cudaGetLastError());
      const bool projected = recycle && !keep.cycles.empty();
      if (recycle) {
        // E_0 from the earlier cycles' blocks (the inner solve's q and z
        // buffers serve as scratch before it starts), then room for this
        // cycle's blocks
        if (projected)
          MRHS_TRY(recycle_project(cx, keep, p.recycle, p.krylov_prec, sb.f32, sb.e32,
                                   sb.b32.q, sb.b32.z, &nproj));
        MRHS_TRY(recycle_grow(keep, s));
      }
      const std::vector<double> rnorm_before = rnorm;
      int it = 0;
      // the cycle expected to end the solve needs few iterations and leaves
      // no blocks for a later start, so it reads its flags at least every
      // second iteration (the earlier cycles' extra iterations between
      // checks deepen their reduction, which the recycled start builds on)
      const int every_cycle = final_cycle && every > 2 ? 2 : every;
      MRHS_TRY(run_bcg<float2>(cx, sb.b32, p.krylov_prec, sb.f32, sb.e32, target.data(),
                               p.precond != 0, p.precond_prec, lo, hi, p.cheb_order,
                               p.maxiter - total_iters, every_cycle, &it, &flag,
                               recycle && keep.avail > keep.used ? &keep : nullptr, projected,
                               !projected));
      if (recycle) MRHS_TRY(recycle_close_cycle(keep, s));
      total_iters += it;
      { k_update_x<<<g, kThreads, 0, s>>>(X, sb.e32, sb.rho_d, cx.N, R); ::mrhs::count_launch(); }
      MRHS_CUDA_TRY(cudaGetLastError());
      if (final_cycle) MRHS_TRY(residual_in(f64));
      else MRHS_TRY(true_residual());
      // a cycle that started from kept blocks and made no progress on some
      // column ends the recycling for this solve (plain restarts follow)
      if (projected)
        for (int j = 0; j < R; ++j)
          if (rho[j] > 0 && !(rnorm[j] < rnorm_before[j])) recycle = false;
      if (info && cycles < MRHS_MAX_CYCLES) {
        info->cycle_iters[cycles] = it;
        info->cycle_resid[cycles] = max_rel();
        info->cycle_flag[cycles] = flag;
      }
      if (flag & 4) break;
    }
    if (info) {
      info->recycle_blocks = keep.used;
      info->recycle_projections = nproj;
    }
  }
  if (flag & 4) status = MRHS_ERR_NONFINITE;
  else if (!all_done()) status = MRHS_ERR_NOT_CONVERGED;
  if (info) {
    info->status = status;
    info->iters = total_iters;
    info->cycles = cycles;
    info->nrhs = R;
    for (int i = 0; i < MRHS_NUM_PREC; ++i) info->applies[i] = cx.applies[i];
    for (int j = 0; j < MRHS_MAX_RHS; ++j)
      info->resid[j] = j < R ? (bnorm[j] > 0 ? rnorm[j] / bnorm[j] : 0.0) : 0.0;
    info->cheb_lo = lo;
    info->cheb_hi = hi;
    info->krylov_prec = mixed ? p.krylov_prec : f64;
    info->precond_prec = p.precond ? p.precond_prec : -1;
  }
  MRHS_CUDA_TRY(cudaStreamSynchronize(s));
  if (info)
    info->ms_total =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (status != MRHS_OK)
    set_error(status == MRHS_ERR_NONFINITE ? "non-finite value in block CG" : "not converged");
  return status;
}

// standalone Chebyshev application (entry point cheby_apply); recurrence
// buffers come from the operator's grow-only workspace, so calls on one
// operator must not overlap on the GPU.
int cheby(mrhs_op_s* op, int prec, double lo, double hi, int order, const void* X, void* P,
          int R, cudaStream_t s) {
  Ctx cx;
  cx.op = op;
  cx.s = s;
  cx.R = R;
  cx.N = op->V * op->nb;
  const int64_t n = cx.N * R;
  const bool wide = MRHS_PREC_IS_WIDE(prec);
  const size_t es = wide ? sizeof(double2) : sizeof(float2);
  MRHS_TRY(op->ws_cheb.ensure(3 * (n * es + 256)));
  char* base = (char*)op->ws_cheb.ptr;
  const size_t stride = (n * es + 255) / 256 * 256;
  if (wide)
    return cheb_run<double2>(cx, prec, lo, hi, order, (const double2*)X, (double2*)P,
                             (double2*)base, (double2*)(base + stride),
                             (double2*)(base + 2 * stride));
  return cheb_run<float2>(cx, prec, lo, hi, order, (const float2*)X, (float2*)P, (float2*)base,
                          (float2*)(base + stride), (float2*)(base + 2 * stride));
}


// ---------------------------------------------------------------- batches
// Many independent problems solved side by side (mixed mode, Chebyshev-
// preconditioned).  The problems advance in lockstep: every operator
// application of an iteration -- the Krylov step and each Chebyshev step --
// is one persistent tensor-core launch over the sites of all active problems
// (tc_apply_batch); the per-problem nrhs x nrhs algebra and block updates are
// ordinary launches in the same stream.  Chunks of check_every iterations are
// captured once as a CUDA graph and replayed.  A problem whose inner solve
// reached its target (or stalled) is masked out of the batched launches
// through a device flag; its search block and rank are zeroed, so the
// remaining iterations of the chunk leave it unchanged.
namespace {

struct BatchProb {
  Ctx cx;
  SolveBufs sb;
  std::vector<double> bnorm, rnorm, target, est;
  double lo = 0, hi = 0, best = 1e300;
  int iters = 0, cycles = 0, flag = 0, stalled = 0;
  bool done = false, in_cycle = false, inner_live = false, final_cycle = false;
  double cycle_resid[MRHS_MAX_CYCLES] = {0};
  int cycle_iters[MRHS_MAX_CYCLES] = {0}, cycle_flag[MRHS_MAX_CYCLES] = {0};
};

}  // namespace

int solve_batch(mrhs_op_s* const* ops, int n, const double2* const* B, double2* const* X,
                const int32_t* nrhs, const mrhs_solve_params& p, mrhs_solve_info* infos,
                cudaStream_t s) {
  auto t0 = std::chrono::steady_clock::now();
  std::vector<BatchProb> P(n);
  int32_t* d_active = nullptr;
  for (int i = 0; i < n; ++i) {
    BatchProb& b = P[i];
    Ctx& cx = b.cx;
    cx.op = ops[i];
    cx.s = s;
    cx.R = nrhs[i];
    cx.N = ops[i]->V * ops[i]->nb;
    cx.tau = p.breakdown_tau > 0 ? p.breakdown_tau : 1e-12;
    const int64_t nn = cx.N * cx.R;
    b.sb.carve(cx, cx.R, nn, true, true);
    int32_t* act = nullptr;
    cx.alloc(&act, MRHS_MAX_BATCH);
    MRHS_TRY(ops[i]->ws_solve.ensure(cx.used));
    cx.base = (char*)ops[i]->ws_solve.ptr;
    cx.used = 0;
    b.sb.carve(cx, cx.R, nn, true, true);
    cx.alloc(&act, MRHS_MAX_BATCH);
    if (i == 0) d_active = act;
    MRHS_CUDA_TRY(cudaMemsetAsync(cx.st, 0, sizeof(Small), s));
    b.bnorm.resize(cx.R);
    b.rnorm.resize(cx.R);
    b.target.resize(cx.R);
    b.est.resize(cx.R);
    // Chebyshev interval of this problem
    b.hi = p.cheb_hi;
    if (b.hi <= 0.0) {
      double& cached = ops[i]->lam_max[p.precond_prec];
      if (!(cached > 0.0)) MRHS_TRY(lambda_max(ops[i], p.precond_prec, 40, s, &cached));
      b.hi = 1.08 * cached;
    }
    b.lo = p.cheb_lo > 0.0 ? p.cheb_lo : b.hi / 400.0;
    MRHS_TRY(cx.colnorms<double2>(B[i], b.sb.bnorm_d));
    MRHS_CUDA_TRY(cudaMemcpyAsync(b.bnorm.data(), b.sb.bnorm_d, sizeof(double) * cx.R,
                                  cudaMemcpyDeviceToHost, s));
  }
  MRHS_CUDA_TRY(cudaStreamSynchronize(s));
  for (int i = 0; i < n; ++i)
    MRHS_TRY(finite_columns(P[i].bnorm, "problem " + std::to_string(i) + ": B"));
  for (int i = 0; i < n; ++i) {
    BatchProb& b = P[i];
    { k_zero_cols<double2><<<grid_for(b.cx.N * b.cx.R), kThreads, 0, s>>>(X[i], b.sb.bnorm_d, b.cx.N, b.cx.R); ::mrhs::count_launch(); }
  }

  // one side stream per problem: the per-problem block algebra of an
  // iteration forks onto them (event fork / join), so inside a captured graph
  // the problems' small kernels are parallel branches instead of a chain
  struct Side {
    std::vector<cudaStream_t> st;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    ~Side() {
      for (cudaStream_t x : st) if (x) cudaStreamDestroy(x);
      for (cudaEvent_t e : join) if (e) cudaEventDestroy(e);
      if (fork) cudaEventDestroy(fork);
    }
  } side;
  side.st.assign(n, nullptr);
  side.join.assign(n, nullptr);
  MRHS_CUDA_TRY(cudaEventCreateWithFlags(&side.fork, cudaEventDisableTiming));
  for (int i = 0; i < n; ++i) {
    MRHS_CUDA_TRY(cudaStreamCreateWithFlags(&side.st[i], cudaStreamNonBlocking));
    MRHS_CUDA_TRY(cudaEventCreateWithFlags(&side.join[i], cudaEventDisableTiming));
  }
  // run fn(k, stream) for every problem idx[k] on its side stream, joined back
  auto fork_each = [&](const std::vector<int>& ids, auto&& fn) -> int {
    MRHS_CUDA_TRY(cudaEventRecord(side.fork, s));
    for (int k = 0; k < (int)ids.size(); ++k) {
      const int i = ids[k];
      MRHS_CUDA_TRY(cudaStreamWaitEvent(side.st[i], side.fork, 0));
      P[i].cx.s = side.st[i];
      const int st = fn(k, side.st[i]);
      P[i].cx.s = s;
      if (st != MRHS_OK) return st;
      MRHS_CUDA_TRY(cudaEventRecord(side.join[i], side.st[i]));
    }
    for (int k = 0; k < (int)ids.size(); ++k)
      MRHS_CUDA_TRY(cudaStreamWaitEvent(s, side.join[ids[k]], 0));
    return MRHS_OK;
  };

  auto residual_in = [&](BatchProb& b, int i, int rp) -> int {
    Ctx& cx = b.cx;
    const int64_t nn = cx.N * cx.R;
    MRHS_TRY(cx.apply(rp, X[i], b.sb.r64));
    { k_sub<double2><<<grid_for(nn), kThreads, 0, s>>>(b.sb.r64, B[i], b.sb.r64, nn); ::mrhs::count_launch(); }
    MRHS_TRY(cx.colnorms<double2>(b.sb.r64, b.sb.rnorm_d));
    MRHS_CUDA_TRY(cudaMemcpyAsync(b.rnorm.data(), b.sb.rnorm_d, sizeof(double) * cx.R,
                                  cudaMemcpyDeviceToHost, s));
    return MRHS_OK;
  };
  auto problem_done = [&](BatchProb& b) {
    for (int j = 0; j < b.cx.R; ++j)
      if (b.bnorm[j] > 0 && !(b.rnorm[j] <= p.tol * b.bnorm[j])) return false;
    return true;
  };
  // the cycle residual in residual_prec, confirmed with the FP64 operator
  // (fp64_prec) once it meets tol
  const int f64 = p.fp64_prec;
  const int res_prec = p.residual_prec >= 0 ? p.residual_prec : f64;
  auto true_residual = [&](BatchProb& b, int i) -> int {
    MRHS_TRY(residual_in(b, i, res_prec));
    if (res_prec != f64) {
      MRHS_CUDA_TRY(cudaStreamSynchronize(s));
      if (problem_done(b)) MRHS_TRY(residual_in(b, i, f64));
    }
    return MRHS_OK;
  };
  // initial residuals: a zero guess needs no operator application
  for (int i = 0; i < n; ++i) {
    BatchProb& b = P[i];
    std::vector<double> xn(b.cx.R);
    MRHS_TRY(b.cx.colnorms<double2>(X[i], b.sb.rnorm_d));
    MRHS_CUDA_TRY(cudaMemcpyAsync(xn.data(), b.sb.rnorm_d, sizeof(double) * b.cx.R,
                                  cudaMemcpyDeviceToHost, s));
    MRHS_CUDA_TRY(cudaStreamSynchronize(s));
    MRHS_TRY(finite_columns(xn, "problem " + std::to_string(i) + ": X0"));
    bool zero = true;
    for (double v : xn) zero = zero && v == 0.0;
    if (zero) {
      MRHS_CUDA_TRY(cudaMemcpyAsync(b.sb.r64, B[i], sizeof(double2) * b.cx.N * b.cx.R,
                                    cudaMemcpyDeviceToDevice, s));
      b.rnorm = b.bnorm;
    } else {
      MRHS_TRY(true_residual(b, i));
    }
  }
  MRHS_CUDA_TRY(cudaStreamSynchronize(s));
  for (auto& b : P) b.done = problem_done(b);

  const int kp = p.krylov_prec, pp = p.precond_prec, order = p.cheb_order;
  const int every = p.check_every > 1 ? p.check_every : 2;
  std::vector<int32_t> h_active(MRHS_MAX_BATCH, 0);
  std::vector<std::vector<double>> coef(n);
  for (int i = 0; i < n; ++i) cheb_coeffs(P[i].lo, P[i].hi, order, coef[i]);
  int total_iters = 0;

  for (int cycle = 0; cycle < p.max_cycles; ++cycle) {
    // problems taking part in this refinement cycle
    std::vector<int> idx;
    for (int i = 0; i < n; ++i) {
      P[i].in_cycle = !P[i].done;
      if (P[i].in_cycle) idx.push_back(i);
    }
    if (idx.empty() || total_iters >= p.maxiter) break;
    const int m = (int)idx.size();
    std::vector<mrhs_op_s*> bops(m);
    std::vector<int32_t> bR(m);
    for (int k = 0; k < m; ++k) {
      const int i = idx[k];
      BatchProb& b = P[i];
      Ctx& cx = b.cx;
      bops[k] = ops[i];
      bR[k] = cx.R;
      std::vector<double> rho(cx.R);
      b.final_cycle = true;      // less than a tenfold reduction left: FP64 residual directly
      const double tol_c = cycle_inner_tol(p, cycle);
      for (int j = 0; j < cx.R; ++j) {
        rho[j] = (b.bnorm[j] > 0 && b.rnorm[j] > p.tol * b.bnorm[j]) ? b.rnorm[j] : 0.0;
        const double want = rho[j] > 0 ? 0.5 * p.tol * b.bnorm[j] / rho[j] : 1.0;
        b.target[j] = std::fmax(tol_c, want);
        if (rho[j] > 0 && want < std::fmax(tol_c, kFinalCycleTarget)) b.final_cycle = false;
      }
      const int64_t nn = cx.N * cx.R;
      MRHS_CUDA_TRY(cudaMemcpyAsync(b.sb.rho_d, rho.data(), sizeof(double) * cx.R,
                                    cudaMemcpyHostToDevice, s));
      MRHS_CUDA_TRY(cudaMemcpyAsync(cx.st->target, b.target.data(), sizeof(double) * cx.R,
                                    cudaMemcpyHostToDevice, s));
      MRHS_CUDA_TRY(cudaMemsetAsync(&cx.st->flag, 0, sizeof(int), s));
      { k_scale_to_c64<<<grid_for(nn), kThreads, 0, s>>>(b.sb.f32, b.sb.r64, b.sb.rho_d, cx.N, cx.R); ::mrhs::count_launch(); }
      MRHS_CUDA_TRY(cudaMemsetAsync(b.sb.e32, 0, sizeof(float2) * nn, s));
      // zero inner guess: r0 = F
      MRHS_CUDA_TRY(cudaMemcpyAsync(b.sb.b32.q, b.sb.f32, sizeof(float2) * nn,
                                    cudaMemcpyDeviceToDevice, s));
      b.inner_live = true;
      b.flag = 0;
      b.stalled = 0;
      b.best = 1e300;
      h_active[k] = 1;
    }
    for (int k = m; k < MRHS_MAX_BATCH; ++k) h_active[k] = 0;
    MRHS_CUDA_TRY(cudaMemcpyAsync(d_active, h_active.data(), sizeof(int32_t) * MRHS_MAX_BATCH,
                                  cudaMemcpyHostToDevice, s));

    // batched operator application: inputs in[k], outputs out[k]
    std::vector<const void*> in(m);
    std::vector<void*> out(m);
    auto bapply = [&](int prec) -> int {
      for (int k = 0; k < m; ++k) P[idx[k]].cx.applies[prec]++;
      return tc_apply_batch(bops.data(), m, prec, in.data(), out.data(), bR.data(), d_active, s);
    };
    // batched Chebyshev: P_k = p(H_k) X_k for all problems of the cycle
    auto bcheb = [&](float2* const* Xs, float2* const* Ps) -> int {
      std::vector<const float2*> Tprev(m);
      std::vector<float2*> Tcur(m);
      if (order > 0) {
        // every step inside the batched operator's epilogue (W never stored)
        std::vector<ChebFuse> f(m);
        std::vector<void*> none(m, nullptr);
        for (int k = 0; k < m; ++k) {
          BatchProb& b = P[idx[k]];
          const std::vector<double>& c = coef[idx[k]];
          const double a = 2.0 / (b.hi - b.lo), bb = -(b.hi + b.lo) / (b.hi - b.lo);
          f[k].mode = 1;
          f[k].a = (float)a;
          f[k].b = (float)bb;
          f[k].c0 = (float)c[0];
          f[k].c = (float)c[1];
          f[k].Tout = b.sb.b32.c1;
          f[k].P = Ps[k];
          f[k].colmax_next = order >= 2;
          in[k] = Xs[k];
          Tprev[k] = Xs[k];
          Tcur[k] = b.sb.b32.c1;
          b.cx.applies[pp]++;
        }
        MRHS_TRY(tc_apply_batch(bops.data(), m, pp, in.data(), none.data(), bR.data(), d_active,
                                s, nullptr, f.data()));
        for (int j = 2; j <= order; ++j) {
          for (int k = 0; k < m; ++k) {
            BatchProb& b = P[idx[k]];
            float2* dst = (Tprev[k] == Xs[k]) ? b.sb.b32.c2 : const_cast<float2*>(Tprev[k]);
            f[k].mode = 2;
            f[k].c = (float)coef[idx[k]][j];
            f[k].Tout = dst;
            f[k].Tp = Tprev[k];
            f[k].colmax_next = j < order;
            f[k].colmax_ready = true;
            in[k] = Tcur[k];
            Tprev[k] = Tcur[k];
            Tcur[k] = dst;
            b.cx.applies[pp]++;
          }
          MRHS_TRY(tc_apply_batch(bops.data(), m, pp, in.data(), none.data(), bR.data(), d_active,
                                  s, nullptr, f.data()));
        }
        return MRHS_OK;
      }
      for (int k = 0; k < m; ++k) {
        in[k] = Xs[k];
        out[k] = P[idx[k]].sb.b32.cw;
      }
      MRHS_TRY(bapply(pp));
      MRHS_TRY(fork_each(idx, [&](int k, cudaStream_t ss) -> int {
        BatchProb& b = P[idx[k]];
        const std::vector<double>& c = coef[idx[k]];
        const double a = 2.0 / (b.hi - b.lo), bb = -(b.hi + b.lo) / (b.hi - b.lo);
        const int64_t nn = b.cx.N * b.cx.R;
        { k_cheb_first<float2><<<grid_for(nn), kThreads, 0, ss>>>(b.sb.b32.c1, Ps[k], b.sb.b32.cw, Xs[k], a, bb, c[0], order > 0 ? c[1] : 0.0, nn); ::mrhs::count_launch(); }
        Tprev[k] = Xs[k];
        Tcur[k] = b.sb.b32.c1;
        return MRHS_OK;
      }));
      for (int j = 2; j <= order; ++j) {
        for (int k = 0; k < m; ++k) {
          in[k] = Tcur[k];
          out[k] = P[idx[k]].sb.b32.cw;
        }
        MRHS_TRY(bapply(pp));
        MRHS_TRY(fork_each(idx, [&](int k, cudaStream_t ss) -> int {
          BatchProb& b = P[idx[k]];
          const std::vector<double>& c = coef[idx[k]];
          const double a = 2.0 / (b.hi - b.lo), bb = -(b.hi + b.lo) / (b.hi - b.lo);
          const int64_t nn = b.cx.N * b.cx.R;
          float2* dst = (Tprev[k] == Xs[k]) ? b.sb.b32.c2 : const_cast<float2*>(Tprev[k]);
          { k_cheb_step<float2><<<grid_for(nn), kThreads, 0, ss>>>(dst, Ps[k], b.sb.b32.cw, Tcur[k], Tprev[k], a, bb, c[j], nn); ::mrhs::count_launch(); }
          Tprev[k] = Tcur[k];
          Tcur[k] = dst;
          return MRHS_OK;
        }));
      }
      MRHS_CUDA_TRY(cudaGetLastError());
      return MRHS_OK;
    };

    // start: Z0 = M^-1 r0, C0 from Z0^dag r0, q <- q W, Q <- Q W, D <- Q
    {
      std::vector<float2*> Xs(m), Ps(m);
      for (int k = 0; k < m; ++k) {
        Xs[k] = P[idx[k]].sb.b32.q;
        Ps[k] = P[idx[k]].sb.b32.Q;
      }
      MRHS_TRY(bcheb(Xs.data(), Ps.data()));
      MRHS_TRY(fork_each(idx, [&](int k, cudaStream_t ss) -> int {
        BatchProb& b = P[idx[k]];
        Ctx& cx = b.cx;
        MRHS_TRY(cx.gram<float2>(b.sb.b32.Q, b.sb.b32.q, cx.st->G));
        MRHS_TRY(cx.small_launch(0));
        MRHS_CUDA_TRY(cudaMemsetAsync(b.sb.b32.D, 0, sizeof(float2) * cx.N * cx.R, ss));
        MRHS_CUDA_TRY(cudaMemsetAsync(cx.st->S, 0, sizeof(double2) * 64 * 64, ss));
        MRHS_TRY(cx.rotate<float2>(b.sb.b32.q, b.sb.b32.Q, b.sb.b32.D));
        return MRHS_OK;
      }));
    }
    auto body = [&]() -> int {
      for (int k = 0; k < m; ++k) {
        in[k] = P[idx[k]].sb.b32.D;
        out[k] = P[idx[k]].sb.b32.z;
      }
      MRHS_TRY(bapply(kp));                                          // z = H D
      std::vector<float2*> Xs(m), Ps(m);
      for (int k = 0; k < m; ++k) {
        Xs[k] = P[idx[k]].sb.b32.z;
        Ps[k] = P[idx[k]].sb.b32.Zz;
      }
      MRHS_TRY(bcheb(Xs.data(), Ps.data()));                         // Z = M^-1 z
      return fork_each(idx, [&](int k, cudaStream_t ss) -> int {
        BatchProb& b = P[idx[k]];
        Ctx& cx = b.cx;
        BcgBufs<float2>& q = b.sb.b32;
        MRHS_TRY(cx.gram<float2>(q.D, q.z, cx.st->G));
        MRHS_TRY(cx.small_launch(1));
        MRHS_TRY(axpy(b.sb.e32, q.D, cx.st->MC, 1.0, cx.N, cx.R, cx.R, MRHS_C64, ss));
        MRHS_TRY(axpy(q.q, q.z, cx.st->negM, 1.0, cx.N, cx.R, cx.R, MRHS_C64, ss));
        MRHS_TRY(axpy(q.Q, q.Zz, cx.st->negM, 1.0, cx.N, cx.R, cx.R, MRHS_C64, ss));
        MRHS_TRY(cx.gram<float2>(q.Q, q.q, cx.st->G));
        MRHS_TRY(cx.gram<float2>(q.q, q.q, cx.st->G2));
        MRHS_TRY(cx.small_launch(2, 1));
        MRHS_TRY(cx.rotate<float2>(q.q, q.Q, q.D));
        return MRHS_OK;
      });
    };

    cudaGraphExec_t exec = nullptr;
    bool graph_ok = p.use_graph != 0;
    int64_t graph_launches = 0;
    std::vector<std::array<int64_t, MRHS_NUM_PREC>> graph_applies(m);
    int it = 0;
    const int maxit = p.maxiter - total_iters;
    const int stall_checks = (32 + every - 1) / every;
    while (it < maxit) {
      const int chunk = (maxit - it) < every ? (maxit - it) : every;
      if (graph_ok && it >= 1 && chunk == every) {
        if (!exec) {
          std::vector<std::array<int64_t, MRHS_NUM_PREC>> before(m);
          for (int k = 0; k < m; ++k)
            for (int q = 0; q < MRHS_NUM_PREC; ++q) before[k][q] = P[idx[k]].cx.applies[q];
          const int64_t l0 = launch_count();
          cudaGraph_t gr = nullptr;
          int st = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess
                       ? MRHS_OK : MRHS_ERR_CUDA;
          for (int j = 0; j < chunk && st == MRHS_OK; ++j) st = body();
          const cudaError_t ce = cudaStreamEndCapture(s, &gr);
          const bool ok = st == MRHS_OK && ce == cudaSuccess && gr &&
                          cudaGraphInstantiate(&exec, gr, 0) == cudaSuccess;
          if (gr) cudaGraphDestroy(gr);
          for (int k = 0; k < m; ++k)
            for (int q = 0; q < MRHS_NUM_PREC; ++q) {
              graph_applies[k][q] = P[idx[k]].cx.applies[q] - before[k][q];
              P[idx[k]].cx.applies[q] = before[k][q];
            }
          graph_launches = launch_count() - l0;
          add_launches(-graph_launches);
          if (!ok) {
            cudaGetLastError();
            if (exec) cudaGraphExecDestroy(exec);
            exec = nullptr;
            graph_ok = false;
            continue;
          }
        }
        if (cudaGraphLaunch(exec, s) != cudaSuccess) {
          cudaGraphExecDestroy(exec);
          return fail(MRHS_ERR_CUDA, "batched graph launch failed");
        }
        add_launches(graph_launches);
        for (int k = 0; k < m; ++k)
          for (int q = 0; q < MRHS_NUM_PREC; ++q) P[idx[k]].cx.applies[q] += graph_applies[k][q];
      } else {
        for (int j = 0; j < chunk; ++j) {
          const int st = body();
          if (st != MRHS_OK) {
            if (exec) cudaGraphExecDestroy(exec);
            return st;
          }
        }
      }
      it += chunk;
      for (int k = 0; k < m; ++k) {
        BatchProb& b = P[idx[k]];
        if (!b.inner_live) continue;
        MRHS_CUDA_TRY(cudaMemcpyAsync(&b.flag, &b.cx.st->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        MRHS_CUDA_TRY(cudaMemcpyAsync(b.est.data(), b.cx.st->est, sizeof(double) * b.cx.R,
                                      cudaMemcpyDeviceToHost, s));
      }
      MRHS_CUDA_TRY(cudaStreamSynchronize(s));
      bool any = false, changed = false;
      for (int k = 0; k < m; ++k) {
        BatchProb& b = P[idx[k]];
        if (!b.inner_live) continue;
        b.iters += chunk;
        bool stop = (b.flag & (1 | 4)) != 0;
        if (!stop) {
          double worst = 0.0;
          for (int j = 0; j < b.cx.R; ++j)
            if (b.target[j] > 0.0) worst = std::fmax(worst, b.est[j] / b.target[j]);
          if (worst < 0.7 * b.best) {
            b.best = worst;
            b.stalled = 0;
          } else if (++b.stalled >= stall_checks) {
            b.flag |= 8;
            stop = true;
          }
        }
        if (stop) {
          // freeze: out of the batched launches, zero search block and rank
          b.inner_live = false;
          h_active[k] = 0;
          changed = true;
          MRHS_CUDA_TRY(cudaMemsetAsync(b.sb.b32.D, 0, sizeof(float2) * b.cx.N * b.cx.R, s));
          MRHS_CUDA_TRY(cudaMemsetAsync(&b.cx.st->rank, 0, sizeof(int32_t), s));
        } else {
          any = true;
        }
      }
      if (changed)
        MRHS_CUDA_TRY(cudaMemcpyAsync(d_active, h_active.data(), sizeof(int32_t) * MRHS_MAX_BATCH,
                                      cudaMemcpyHostToDevice, s));
      if (!any) break;
    }
    if (exec) cudaGraphExecDestroy(exec);
    total_iters += it;
    // FP64 outer step for every problem of the cycle
    for (int k = 0; k < m; ++k) {
      const int i = idx[k];
      BatchProb& b = P[i];
      Ctx& cx = b.cx;
      { k_update_x<<<grid_for(cx.N * cx.R), kThreads, 0, s>>>(X[i], b.sb.e32, b.sb.rho_d, cx.N, cx.R); ::mrhs::count_launch(); }
      if (b.final_cycle) MRHS_TRY(residual_in(b, i, f64));
      else MRHS_TRY(true_residual(b, i));
    }
    MRHS_CUDA_TRY(cudaStreamSynchronize(s));
    for (int k = 0; k < m; ++k) {
      BatchProb& b = P[idx[k]];
      if (b.cycles < MRHS_MAX_CYCLES) {
        double mr = 0.0;
        for (int j = 0; j < b.cx.R; ++j)
          if (b.bnorm[j] > 0) mr = std::fmax(mr, b.rnorm[j] / b.bnorm[j]);
        b.cycle_resid[b.cycles] = mr;
        b.cycle_iters[b.cycles] = b.iters;
        b.cycle_flag[b.cycles] = b.flag;
      }
      b.cycles++;
      b.done = problem_done(b) || (b.flag & 4);
    }
  }
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  int worst = MRHS_OK;
  for (int i = 0; i < n; ++i) {
    BatchProb& b = P[i];
    const int status = (b.flag & 4) ? MRHS_ERR_NONFINITE : (problem_done(b) ? MRHS_OK : MRHS_ERR_NOT_CONVERGED);
    if (status != MRHS_OK && worst == MRHS_OK) worst = status;
    if (!infos) continue;
    mrhs_solve_info& inf = infos[i];
    inf.recycle_blocks = 0;      // lockstep batches restart each cycle afresh
    inf.recycle_projections = 0;
    inf.status = status;
    inf.iters = b.iters;
    inf.cycles = b.cycles;
    inf.nrhs = b.cx.R;
    for (int q = 0; q < MRHS_NUM_PREC; ++q) inf.applies[q] = b.cx.applies[q];
    for (int j = 0; j < MRHS_MAX_RHS; ++j)
      inf.resid[j] = j < b.cx.R ? (b.bnorm[j] > 0 ? b.rnorm[j] / b.bnorm[j] : 0.0) : 0.0;
    inf.cheb_lo = b.lo;
    inf.cheb_hi = b.hi;
    inf.ms_total = ms;
    inf.krylov_prec = kp;
    inf.precond_prec = pp;
    for (int c = 0; c < MRHS_MAX_CYCLES; ++c) {
      inf.cycle_iters[c] = c < b.cycles ? b.cycle_iters[c] - (c ? b.cycle_iters[c - 1] : 0) : 0;
      inf.cycle_resid[c] = b.cycle_resid[c];
      inf.cycle_flag[c] = b.cycle_flag[c];
    }
  }
  if (worst != MRHS_OK) set_error(worst == MRHS_ERR_NONFINITE ? "non-finite value in a batched solve" : "a batched problem did not converge");
  return worst;
}

}  // namespace mrhs

// ---------------------------------------------------------------- 5D CG
// The coarse solve as one enlarged five-dimensional system (Sec. 2.1): plain
// CG on the whole [V][nb][R] block, alpha and beta from inner products summed
// over every right-hand side, so the block algebra is two scalar reductions
// and three vector updates per iteration instead of Grams and a Hermitian
// factorisation.  The scalars stay on the device; the host reads per-column
// residual norms every check_every iterations to stop.
namespace mrhs {
namespace {

// per-block partial sums of Re <x, y> over a row range, fixed order
__global__ void k_dot5d_partial(const double2* __restrict__ x, const double2* __restrict__ y,
                                double* part, int64_t n, int64_t per) {
  __shared__ double sm[kThreads];
  const int64_t i0 = (int64_t)blockIdx.x * per;
  const int64_t i1 = (i0 + per) < n ? (i0 + per) : n;
  double acc = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kThreads) {
    const double2 a = x[i], b = y[i];
    acc = fma(a.x, b.x, fma(a.y, b.y, acc));
  }
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

__global__ void k_dot5d_final(const double* __restrict__ part, int nblk, double* out) {
  __shared__ double sm[kThreads];
  double acc = 0.0;
  for (int b = threadIdx.x; b < nblk; b += kThreads) acc += part[b];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sm[0];
}

// sc = {rr, pw, rr_new}: X += a p, r -= a w with a = rr / pw, and the
// partial sums of |r|^2 of the updated residual
__global__ void k_cg5d_update(double2* X, double2* r, const double2* __restrict__ p,
                              const double2* __restrict__ w, const double* __restrict__ sc,
                              double* part, int64_t n, int64_t per) {
  __shared__ double sm[kThreads];
  const double a = sc[0] / sc[1];
  const int64_t i0 = (int64_t)blockIdx.x * per;
  const int64_t i1 = (i0 + per) < n ? (i0 + per) : n;
  double acc = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kThreads) {
    const double2 pv = p[i], wv = w[i];
    double2 xv = X[i], rv = r[i];
    xv.x = fma(a, pv.x, xv.x);
    xv.y = fma(a, pv.y, xv.y);
    rv.x = fma(-a, wv.x, rv.x);
    rv.y = fma(-a, wv.y, rv.y);
    X[i] = xv;
    r[i] = rv;
    acc = fma(rv.x, rv.x, fma(rv.y, rv.y, acc));
  }
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int wd = kThreads / 2; wd > 0; wd >>= 1) {
    if (threadIdx.x < wd) sm[threadIdx.x] += sm[threadIdx.x + wd];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

// p = r + b p with b = rr_new / rr
__global__ void k_cg5d_dir(double2* p, const double2* __restrict__ r,
                           const double* __restrict__ sc, int64_t n) {
  const double b = sc[2] / sc[0];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double2 rv = r[i];
    double2 pv = p[i];
    pv.x = fma(b, pv.x, rv.x);
    pv.y = fma(b, pv.y, rv.y);
    p[i] = pv;
  }
}

__global__ void k_cg5d_roll(double* sc) { sc[0] = sc[2]; }

}  // namespace

int cg5d(mrhs_op_s* op, const double2* B, double2* X, int R, const mrhs_solve_params& p,
         mrhs_solve_info* info, cudaStream_t s) {
  auto t0 = std::chrono::steady_clock::now();
  const int prec = p.krylov_prec >= 0 ? p.krylov_prec : MRHS_PREC_FP64;
  Ctx cx;
  cx.op = op;
  cx.s = s;
  cx.R = R;
  cx.N = op->V * op->nb;
  const int64_t n = cx.N * R;
  const int nblk = num_sms() * 4;
  const int64_t per = (n + nblk - 1) / nblk;
  double2 *r = nullptr, *pv = nullptr, *w = nullptr;
  double *part = nullptr, *sc = nullptr, *bnorm_d = nullptr, *rnorm_d = nullptr;
  for (int pass = 0; pass < 2; ++pass) {      // sizing, then assignment
    cx.used = 0;
    cx.alloc(&r, n);
    cx.alloc(&pv, n);
    cx.alloc(&w, n);
    cx.alloc(&part, nblk);
    cx.alloc(&sc, 4);
    cx.alloc(&bnorm_d, R);
    cx.alloc(&rnorm_d, R);
    cx.alloc(&cx.npart, (size_t)num_sms() * 2 * R + R);
    if (pass == 0) {
      MRHS_TRY(op->ws_solve.ensure(cx.used));
      cx.base = (char*)op->ws_solve.ptr;
    }
  }
  const int g = grid_for(n);
  std::vector<double> bnorm(R), rnorm(R);
  MRHS_TRY(cx.colnorms<double2>(B, bnorm_d));
  MRHS_CUDA_TRY(cudaMemcpyAsync(bnorm.data(), bnorm_d, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
  MRHS_CUDA_TRY(cudaStreamSynchronize(s));
  MRHS_TRY(finite_columns(bnorm, "B"));
  { k_zero_cols<double2><<<g, kThreads, 0, s>>>(X, bnorm_d, cx.N, R); ::mrhs::count_launch(); }
  {
    std::vector<double> xn(R);
    MRHS_TRY(cx.colnorms<double2>(X, rnorm_d));
    MRHS_CUDA_TRY(cudaMemcpyAsync(xn.data(), rnorm_d, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
    MRHS_CUDA_TRY(cudaStreamSynchronize(s));
    MRHS_TRY(finite_columns(xn, "X0"));
  }
  // r = B - H X (X = 0: r = B)
  MRHS_TRY(cx.apply(prec, X, r));
  { k_sub<double2><<<g, kThreads, 0, s>>>(r, B, r, n); ::mrhs::count_launch(); }
  MRHS_CUDA_TRY(cudaMemcpyAsync(pv, r, sizeof(double2) * n, cudaMemcpyDeviceToDevice, s));
  { k_dot5d_partial<<<nblk, kThreads, 0, s>>>(r, r, part, n, per); ::mrhs::count_launch(); }
  { k_dot5d_final<<<1, kThreads, 0, s>>>(part, nblk, sc); ::mrhs::count_launch(); }
  MRHS_CUDA_TRY(cudaGetLastError());
  auto all_done = [&]() {
    for (int j = 0; j < R; ++j)
      if (bnorm[j] > 0 && !(rnorm[j] <= p.tol * bnorm[j])) return false;
    return true;
  };
  const int every = p.check_every > 0 ? p.check_every : 1;
  int it = 0;
  bool done = false;
  while (it < p.maxiter && !done) {
    const int chunk = (p.maxiter - it) < every ? (p.maxiter - it) : every;
    for (int j = 0; j < chunk; ++j) {
      MRHS_TRY(cx.apply(prec, pv, w));                                            // w = H p
      { k_dot5d_partial<<<nblk, kThreads, 0, s>>>(pv, w, part, n, per); ::mrhs::count_launch(); }
      { k_dot5d_final<<<1, kThreads, 0, s>>>(part, nblk, sc + 1); ::mrhs::count_launch(); }
      { k_cg5d_update<<<nblk, kThreads, 0, s>>>(X, r, pv, w, sc, part, n, per); ::mrhs::count_launch(); }
      { k_dot5d_final<<<1, kThreads, 0, s>>>(part, nblk, sc + 2); ::mrhs::count_launch(); }
      { k_cg5d_dir<<<g, kThreads, 0, s>>>(pv, r, sc, n); ::mrhs::count_launch(); }
      { k_cg5d_roll<<<1, 1, 0, s>>>(sc); ::mrhs::count_launch(); }
    }
    MRHS_CUDA_TRY(cudaGetLastError());
    it += chunk;
    MRHS_TRY(cx.colnorms<double2>(r, rnorm_d));
    MRHS_CUDA_TRY(cudaMemcpyAsync(rnorm.data(), rnorm_d, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
    MRHS_CUDA_TRY(cudaStreamSynchronize(s));
    bool finite = true;
    for (double v : rnorm) finite = finite && std::isfinite(v);
    if (!finite) break;
    done = all_done();
  }
  // true residual with the FP64 operator (fp64_prec)
  MRHS_TRY(cx.apply(p.fp64_prec, X, w));
  { k_sub<double2><<<g, kThreads, 0, s>>>(w, B, w, n); ::mrhs::count_launch(); }
  MRHS_TRY(cx.colnorms<double2>(w, rnorm_d));
  MRHS_CUDA_TRY(cudaMemcpyAsync(rnorm.data(), rnorm_d, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
  MRHS_CUDA_TRY(cudaStreamSynchronize(s));
  bool finite = true;
  for (double v : rnorm) finite = finite && std::isfinite(v);
  const int status = !finite ? MRHS_ERR_NONFINITE : (all_done() ? MRHS_OK : MRHS_ERR_NOT_CONVERGED);
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->status = status;
    info->iters = it;
    info->cycles = 1;
    info->nrhs = R;
    for (int i = 0; i < MRHS_NUM_PREC; ++i) info->applies[i] = cx.applies[i];
    for (int j = 0; j < R; ++j) info->resid[j] = bnorm[j] > 0 ? rnorm[j] / bnorm[j] : 0.0;
    info->krylov_prec = prec;
    info->precond_prec = -1;
    info->ms_total =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  if (status != MRHS_OK)
    set_error(status == MRHS_ERR_NONFINITE ? "non-finite value in CG" : "not converged");
  return status;
}

}  // namespace mrhs
