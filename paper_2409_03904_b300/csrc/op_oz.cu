// Coarse operator Y(x) = sum_p A_p(x) X(x + delta_p) (Sec. 2.6) to FP64
// accuracy on the tcgen05 tensor cores, by digit slicing: the error-free
// splitting of Ozaki, Ogita, Oishi and Rump (2012) in the fixed-point form
// that Mukunoki, Ozaki, Ogita and Imamura ("DGEMM using Tensor Cores, and Its
// Accurate and Reproducible Versions", ISC 2020) run on FP16 tensor cores.
//
// Both operands become fixed-point numbers with few bits per digit (balanced
// base-64 digits of rint(2^47 v / scale), see digits_of):
//   coefficients, per site x:  A_p(x) - d_x I = s_x 2^-5 sum_s a_s 2^(-6(s-1))
//   input, per column r:       X[:, r]         = sigma_r 2^-5 sum_t e_t 2^(-6(t-1))
// with s, t = 1..8, s_x and sigma_r powers of two above the largest entry
// (d_x = mean real self diagonal, applied exactly in FP64), and integer digits
// |a_s|, |e_t| <= 32, each held exactly by an fp16 code; the representation
// error is 2^-48 of the scale.  A digit product is at most 2^10 and exact in
// FP32; level c = s + t gathers c - 1 products per term, so a level sum over
// npts * nb terms stays below 2^24 -- exact in the FP32 tensor-memory
// accumulator -- for c <= 5 at 81 x 48 terms in the worst case; deeper levels
// sit 2^-24 below the first and their rounding is far below the target.
// Levels c <= 9 are kept (the first dropped one, c = 10, is 2^-48 of the
// scales per term):
//   Y = s_x sigma_r 2^-46 (sum_{c<=8} D_c 2^(6 (8 - c)) + rint(D_9 2^-6)) + d_x X;
// with |D_c| < 2^25 the sum fits an int64 exactly; level 9 enters rounded to
// the unit of level 8 (half a unit per contribution), and one rounding to
// FP64 follows.
//
// Tensor-core mapping (M = input rows, N = coefficient rows, as in op_tc.cu):
// digit t of the input is a block of 2 rb rows [Re X_t ; Im X_t] (rb =
// round8(R)); in shared memory the blocks follow a zero block X_0, so every
// window [X_t ; X_(t+1)] is one contiguous 4 rb-row operand.  Accumulator j
// (j = 0..3, 128 TMEM columns apart) holds levels (2j + 2, 2j + 3) on its two
// row halves: for coefficient digit s it receives the MMA of window
// [X_(c-s) ; X_(c+1-s)], c = 2j + 2, against the [Re A_s ; Im A_s] tile.
// 2 + 4 + 6 + 8 = 20 MMAs (M = 128, N = 2 nb8, K = 16) per stencil point and
// 16-column K step.  The epilogue converts each level sum to an integer,
// weights it by its power of two in int64, combines the Xi rows' and the
// upper level's contributions with the Xr rows' through shared memory (as
// op_tc.cu does in FP32), and writes complex128 Y.
//
// Layout: the digit image holds, per site, stencil point and K step, one slab
// [digit s][N rows][16 columns] in the canonical no-swizzle K-major layout
// (8 x 16-byte core matrices, 128 bytes apart along K, 256 bytes apart per
// 8 rows); the packed input holds per site and K step [digit t][2 rb][16].  A
// pipeline stage is one (site, point, K step): the coefficient slab, the zero
// block (written once at start) and the input slab, two 1-D bulk copies.
//
// Kernel: persistent, one CTA per SM (the four accumulators take the 512 TMEM
// columns), warp-specialised as in op_tc.cu: warp 0 TMA producer, warp 1 MMA
// issuer, warps 2-5 epilogue.  Every wait is bounded (1 s); on expiry the
// kernel records an error, drains its copies, frees TMEM and returns.
#include <cuda_fp16.h>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace mrhs {

// error bits of this file's kernels (a device variable is private to its
// translation unit without relocatable device code): 8 producer, 16 MMA
// issuer, 32 epilogue wait expired
__device__ unsigned int g_oz_error = 0;
// limit of the epilogue's accumulator wait in ns (0: the default 1 s); set
// only by the debugging entry point mrhs_debug_wait_limit
__device__ unsigned long long g_oz_wait_ns = 0;

namespace {

constexpr int kDigits = 8;        // digits per operand
constexpr int kBeta = 6;          // bits per digit
constexpr int kTopShift = 5;      // first digit: |a_1| <= 2^5
constexpr int kLevels = 8;        // levels 2..8 combined exactly, level 9 rounded into them
constexpr int kNormShift = 2 * kTopShift + (kLevels - 2) * kBeta;   // 46
constexpr int kThreads = 192;
constexpr int kAccCols = 128;
constexpr int kNumAcc = 4;
constexpr uint32_t kTmemCols = kNumAcc * kAccCols;   // 512
constexpr int kChunk = 8;
constexpr int kM = 128;
constexpr size_t kSmemBudget = 220 * 1024;
constexpr int kMaxStages = 16;
constexpr size_t kSmemOneCta = 120 * 1024;

// One MMA of a stage: input window w (digit blocks w, w + 1), coefficient
// digit sd, accumulator acc (levels 2 acc + 2 and 2 acc + 3 = w + sd and
// w + sd + 1); first: the accumulator's first MMA of a site; coll: 0 alone,
// 1 fill, 2 use, 3 lastuse of the A collector.  Ordered by window, so the
// MMAs of one window share its A operand.
struct OzMma {
  int8_t w, sd, acc, first, coll;
};
constexpr int kOzMmas = 20;
__device__ __constant__ const OzMma kOzOrder[kOzMmas] = {
    {0, 2, 0, 1, 1}, {0, 4, 1, 1, 2}, {0, 6, 2, 1, 2}, {0, 8, 3, 1, 3},
    {1, 1, 0, 0, 1}, {1, 3, 1, 0, 2}, {1, 5, 2, 0, 2}, {1, 7, 3, 0, 3},
    {2, 2, 1, 0, 1}, {2, 4, 2, 0, 2}, {2, 6, 3, 0, 3},
    {3, 1, 1, 0, 1}, {3, 3, 2, 0, 2}, {3, 5, 3, 0, 3},
    {4, 2, 2, 0, 1}, {4, 4, 3, 0, 3},
    {5, 1, 2, 0, 1}, {5, 3, 3, 0, 3},
    {6, 2, 3, 0, 0},
    {7, 1, 3, 0, 0}};

struct OzGeom {
  int nb, nbp8, N, K, nk;   // N = 2 nb8 (MMA N), K = nb16, nk = K / 16
  int R, rb;
  uint32_t aslab;           // coefficient slab: kDigits x N rows x 32 bytes
  uint32_t zbytes;          // one input digit block: 2 rb rows x 32 bytes
  uint32_t xslab;           // input slab: kDigits blocks
  uint32_t stage;           // aslab + zbytes + xslab
};

OzGeom make_oz_geom(int nb, int R) {
  OzGeom g;
  g.nb = nb;
  g.nbp8 = (nb + 7) / 8 * 8;
  g.N = 2 * g.nbp8;
  g.K = (nb + 15) / 16 * 16;
  g.nk = g.K / 16;
  g.R = R;
  g.rb = (R + 7) / 8 * 8;
  g.aslab = (uint32_t)kDigits * g.N * 32u;
  g.zbytes = (uint32_t)(2 * g.rb) * 32u;
  g.xslab = (uint32_t)kDigits * g.zbytes;
  g.stage = g.aslab + g.zbytes + g.xslab;
  return g;
}

// byte offset of (row, k) in a 16-column canonical slab
__host__ __device__ inline uint32_t slab_off(int row, int k) {
  return (uint32_t)(row >> 3) * 256u + (uint32_t)(k >> 3) * 128u + (uint32_t)(row & 7) * 16u +
         (uint32_t)(k & 7) * 2u;
}

// smallest power of two >= m (1 for m = 0; NaN for a non-finite m, so that a
// non-finite operand gives a non-finite result)
__device__ inline double pow2_at_least(double m) {
  if (!isfinite(m)) return __longlong_as_double(0x7ff8000000000000ll);
  if (!(m > 0.0)) return 1.0;
  int e;
  const double f = frexp(m, &e);
  if (f == 0.5) e -= 1;
  return ldexp(1.0, e);
}

// The kDigits digits of w (|w| <= 2^5): the fixed-point integer
// n = rint(w 2^42) (one rounding, so |w - n 2^-42| <= 2^-43, i.e. 2^-48 of
// the scale), then its balanced base-64 digits from the bottom,
// d = ((n + 32) mod 64) - 32 in [-32, 31] and n <- (n - d) / 64 exactly; the
// remaining top digit lies in [-32, 32].  Every digit is exact in fp16.  One
// FP64 product and one conversion per value (the FP64 pipe is thin on this
// part); the rest is integer arithmetic.  A NaN gives NaN digits, so a
// non-finite operand yields a non-finite result.
__device__ inline void digits_of(double w, uint16_t* out) {
  if (w != w) {
#pragma unroll
    for (int s = 0; s < kDigits; ++s) out[s] = 0x7E00u;   // fp16 NaN
    return;
  }
  long long n = __double2ll_rn(w * 4398046511104.0);    // w 2^42, an exact scaling
#pragma unroll
  for (int s = kDigits - 1; s >= 1; --s) {
    const long long d = ((n + 32) & 63) - 32;
    out[s] = __half_as_ushort(__int2half_rn((int)d));
    n = (n - d) >> kBeta;
  }
  out[0] = __half_as_ushort(__int2half_rn((int)n));
}

__device__ inline uint4 pack8(const uint16_t* h) {
  uint4 v;
  v.x = (uint32_t)h[0] | ((uint32_t)h[1] << 16);
  v.y = (uint32_t)h[2] | ((uint32_t)h[3] << 16);
  v.z = (uint32_t)h[4] | ((uint32_t)h[5] << 16);
  v.w = (uint32_t)h[6] | ((uint32_t)h[7] << 16);
  return v;
}

// One CTA per site: d_x (FP64 mean real self diagonal), s_x and the digit
// slabs of every stencil point and K step.  dag: the block of point p at x is
// A_p(x - delta_p)^dagger.
__global__ void __launch_bounds__(256) k_oz_pack_coef(const double2* __restrict__ A,
                                                      uint8_t* digits, double* scale,
                                                      double* diag,
                                                      const int32_t* __restrict__ nbr_bwd,
                                                      int64_t V, int npts, OzGeom g, int dag) {
  const int64_t x = blockIdx.x;
  if (x >= V) return;
  const int nb = g.nb;
  __shared__ double s_red[256];
  __shared__ double s_d, s_scale;
  auto src = [&](int p, int a, int b) -> double2 {
    if (!dag) return A[((x * npts + p) * (int64_t)nb) * nb + a * nb + b];
    const int64_t y = nbr_bwd[(int64_t)p * V + x];
    const double2 v = A[((y * npts + p) * (int64_t)nb) * nb + b * nb + a];
    return make_double2(v.x, -v.y);
  };
  double acc = 0.0;
  for (int a = threadIdx.x; a < nb; a += blockDim.x) acc += src(0, a, a).x;
  s_red[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) t += s_red[i];
    s_d = t / nb;
  }
  __syncthreads();
  const double d = s_d;
  const int nn = nb * nb;
  double m = 0.0;
  for (int i = threadIdx.x; i < npts * nn; i += blockDim.x) {
    const int p = i / nn, a = (i % nn) / nb, b = i % nb;
    double2 v = src(p, a, b);
    if (p == 0 && a == b) v.x -= d;
    // fmax drops NaN: carry it explicitly
    const double mv = fmax(fabs(v.x), fabs(v.y));
    m = (mv != mv || m != m) ? __longlong_as_double(0x7ff8000000000000ll) : fmax(m, mv);
  }
  s_red[threadIdx.x] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i)
      t = (s_red[i] != s_red[i] || t != t) ? s_red[i] + t : fmax(t, s_red[i]);
    s_scale = pow2_at_least(t);
    scale[x] = s_scale;
    diag[x] = d;
  }
  __syncthreads();
  const double inv = (double)(1 << kTopShift) / s_scale;   // exact: powers of two
  // one unit: 8 consecutive k of one row of one (point, K step)
  const int units = npts * g.nk * g.N * 2;
  uint8_t* base = digits + (uint64_t)x * npts * g.nk * g.aslab;
  for (int u = threadIdx.x; u < units; u += blockDim.x) {
    const int row = u % g.N;
    const int kh = (u / g.N) & 1;
    const int pj = u / (2 * g.N);          // p * nk + j
    const int p = pj / g.nk, j = pj % g.nk;
    const bool re = row < g.nbp8;          // [Re A ; Im A]
    const int a = re ? row : row - g.nbp8;
    uint16_t dg[kDigits][8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int b = j * 16 + kh * 8 + e;
      double v = 0.0;
      if (a < nb && b < nb) {
        double2 c = src(p, a, b);
        if (p == 0 && a == b) c.x -= d;
        v = (re ? c.x : c.y) * inv;
      }
      uint16_t t[kDigits];
      digits_of(v, t);
#pragma unroll
      for (int s = 0; s < kDigits; ++s) dg[s][e] = t[s];
    }
    uint8_t* slab = base + (uint64_t)pj * g.aslab;
#pragma unroll
    for (int s = 0; s < kDigits; ++s)
      *reinterpret_cast<uint4*>(slab + (uint32_t)s * g.N * 32u + slab_off(row, kh * 8)) =
          pack8(dg[s]);
  }
}

// Per-column maxima of |Re|, |Im| of a complex128 [rows][R] block, as the bit
// patterns of non-negative doubles (ordered like the values; NaN above all).
__global__ void k_oz_colmax(const double2* __restrict__ X, unsigned long long* colmax,
                            int64_t rows, int R) {
  const int per = blockDim.x / R;
  const int t = threadIdx.x;
  __shared__ unsigned long long s_m[MRHS_MAX_RHS];
  for (int i = t; i < R; i += blockDim.x) s_m[i] = 0ull;
  __syncthreads();
  if (t < per * R) {
    const int c = t % R;
    unsigned long long m = 0ull;
    for (int64_t row = (int64_t)blockIdx.x * per + t / R; row < rows;
         row += (int64_t)gridDim.x * per) {
      const double2 v = X[row * R + c];
      const unsigned long long a = (unsigned long long)__double_as_longlong(fabs(v.x));
      const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(v.y));
      m = m > a ? m : a;
      m = m > b ? m : b;
    }
    atomicMax(&s_m[c], m);
  }
  __syncthreads();
  for (int i = t; i < R; i += blockDim.x)
    if (s_m[i]) atomicMax(&colmax[i], s_m[i]);
}

// sigma_r (NaN for a non-finite column); the maxima are cleared for the next
// application.
__global__ void k_oz_colscale(unsigned long long* colmax, double* sigma, int R) {
  const int r = threadIdx.x;
  if (r < R) {
    sigma[r] = pow2_at_least(__longlong_as_double((long long)colmax[r]));
    colmax[r] = 0ull;
  }
}

// Input digit slabs: one unit = 8 consecutive k of one row (Re or Im of a
// column) of one (site, K step), all kDigits digits.
__global__ void k_oz_pack_x(const double2* __restrict__ X, const double* __restrict__ sigma,
                            uint8_t* xb, int64_t V, OzGeom g) {
  const int rows = 2 * g.rb;
  const int64_t units = V * g.nk * 2 * rows;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < units;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int row = (int)(u % rows);
    const int kh = (int)((u / rows) & 1);
    const int64_t xj = u / (2 * rows);     // x * nk + j
    const int j = (int)(xj % g.nk);
    const int64_t x = xj / g.nk;
    const int grp = row / g.rb, r = row % g.rb;
    const bool live = r < g.R;
    const double inv = live ? (double)(1 << kTopShift) / sigma[r] : 0.0;
    uint16_t dg[kDigits][8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int b = j * 16 + kh * 8 + e;
      double v = 0.0;
      if (live && b < g.nb) {
        const double2 xv = X[(x * g.nb + b) * g.R + r];
        v = (grp ? xv.y : xv.x) * inv;
      }
      uint16_t t[kDigits];
      digits_of(v, t);
#pragma unroll
      for (int s = 0; s < kDigits; ++s) dg[s][e] = t[s];
    }
    uint8_t* slab = xb + (uint64_t)xj * g.xslab;
#pragma unroll
    for (int s = 0; s < kDigits; ++s)
      *reinterpret_cast<uint4*>(slab + (uint32_t)s * g.zbytes + slab_off(row, kh * 8)) =
          pack8(dg[s]);
  }
}

struct OzStencil {
  int32_t L[4];            // output lattice
  int32_t Lin[4];          // input lattice: L + 2 h (an input halo h in {0, 1} per dimension)
  int32_t h[4];
  int32_t sign;            // +1: x + delta_p (forward); -1: x - delta_p (adjoint)
  int8_t d[MRHS_MAX_PTS][4];
};

struct OzDesc {
  const uint8_t* coef;      // digit image
  const uint8_t* xb;        // packed input digits
  const double* scale;      // s_x
  const double* diag;       // d_x
  const double* sigma;      // sigma_r
  const double2* X;         // complex128 input, for d_x X(x)
  double2* Y;               // complex128 output
  int64_t V;
  int32_t npts;
  uint32_t idesc;
  OzGeom g;
  OzStencil st;
};

__global__ void __launch_bounds__(kThreads, 1)
    k_op_oz(const __grid_constant__ OzDesc od, int nstages) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + nstages;
  uint64_t* acc_full = empty + nstages;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* mma_done = acc_empty + 1;     // every MMA of this CTA has completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
  uint8_t* stages = smem + 1024;
  const OzGeom g = od.g;
  const uint32_t stage_bytes = g.stage;
  // exchange buffers (two, of 3 rb rows x 16 int64) after the ring
  long long* ex = reinterpret_cast<long long*>(stages + (size_t)nstages * stage_bytes);
  __shared__ volatile int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < nstages; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    ptx::mbar_init(acc_full, 1);
    ptx::mbar_init(acc_empty, 4);
    ptx::mbar_init(mma_done, 1);
    ptx::fence_mbar_init();
    s_abort = 0;
  }
  // the zero digit block X_0 of every stage (never written by the copies)
  for (int s = 0; s < nstages; ++s) {
    uint4* z = reinterpret_cast<uint4*>(stages + (size_t)s * stage_bytes + g.aslab);
    for (uint32_t i = threadIdx.x; i < g.zbytes / 16u; i += blockDim.x) z[i] = make_uint4(0, 0, 0, 0);
  }
  ptx::fence_proxy_async_smem();
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, kTmemCols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int64_t V = od.V;
  const int npts = od.npts, nk = g.nk;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- producer: one stage per (site, point, K step)
      const uint64_t pol_stream = ptx::policy_evict_first();
      const uint64_t pol_keep = ptx::policy_evict_last();
      const uint8_t* coef = od.coef;
      const uint8_t* xbp = od.xb;
      const uint32_t aslab = g.aslab, xslab = g.xslab, xoff = g.aslab + g.zbytes;
      const int sign = od.st.sign;
      const uint32_t* dwords = reinterpret_cast<const uint32_t*>(&od.st.d[0][0]);
      int Lm[4], Ln[4], hm[4];
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) {
        Lm[mu] = od.st.L[mu];
        Ln[mu] = od.st.Lin[mu];
        hm[mu] = od.st.h[mu];
      }
      int s = 0;
      uint32_t ph = 0;
      int64_t issued = 0;
      bool ok = true;
      for (int64_t x = blockIdx.x; x < V && ok; x += gridDim.x) {
        int c[4];
        {
          int64_t r = x;
#pragma unroll
          for (int mu = 0; mu < 4; ++mu) {
            c[mu] = (int)(r % Lm[mu]);
            r /= Lm[mu];
          }
        }
        for (int p = 0; p < npts && ok; ++p) {
          const uint32_t dw = dwords[p];      // delta_p, four signed bytes
          int64_t y = 0;
#pragma unroll
          for (int mu = 3; mu >= 0; --mu) {
            int v = c[mu] + sign * (int)(int8_t)(dw >> (8 * mu));
            v += hm[mu];                      // input coordinates: shifted by the halo
            v += (v < 0) ? Ln[mu] : 0;
            v -= (v >= Ln[mu]) ? Ln[mu] : 0;
            y = y * Ln[mu] + v;
          }
          for (int j = 0; j < nk; ++j) {
            if (!ptx::mbar_wait(&empty[s], ph ^ 1u, &s_abort)) { ok = false; break; }
            uint8_t* st_smem = stages + (size_t)s * stage_bytes;
            ptx::mbar_arrive_expect_tx(&full[s], aslab + xslab);
            ptx::bulk_g2s(st_smem, coef + ((uint64_t)(x * npts + p) * nk + j) * aslab, aslab,
                          &full[s], pol_stream);
            ptx::bulk_g2s(st_smem + xoff, xbp + ((uint64_t)y * nk + j) * xslab, xslab, &full[s],
                          pol_keep);
            ++issued;
            if (++s == nstages) { s = 0; ph ^= 1u; }
          }
        }
      }
      if (!ok) {
        s_abort = 1;
        atomicOr(&g_oz_error, 8u);
      }
      // drain: every copy this thread issued has landed before the CTA exits
      const int64_t last = issued < nstages ? issued : nstages;
      for (int64_t i = 0; i < last; ++i) {
        const int64_t n = issued - 1 - i;
        const int ss = (int)(n % nstages);
        const uint32_t par = (uint32_t)((n / nstages) & 1);
        volatile int never = 0;
        ptx::mbar_wait(&full[ss], par, &never);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer: 20 MMAs per stage
      const uint32_t idesc = od.idesc, zb = g.zbytes, aslice = (uint32_t)g.N * 32u;
      const uint32_t aslab = g.aslab;
      int s = 0;
      uint32_t ph = 0, aph = 0;
      bool ok = true;
      for (int64_t x = blockIdx.x; x < V && ok; x += gridDim.x) {
        if (!ptx::mbar_wait(acc_empty, aph ^ 1u, &s_abort)) { ok = false; break; }
        ptx::tc_fence_after();
        for (int p = 0; p < npts && ok; ++p) {
          for (int j = 0; j < nk; ++j) {
            if (!ptx::mbar_wait(&full[s], ph, &s_abort)) { ok = false; break; }
            ptx::tc_fence_after();
            const uint32_t sa = ptx::smem_u32(stages + (size_t)s * stage_bytes);
            const uint32_t sz = sa + aslab;           // X_0, then X_1..X_7
            const bool first = p == 0 && j == 0;
            // the 20 MMAs grouped by input window [X_w ; X_(w+1)]: those of one
            // window share the A operand through the tensor core's collector,
            // so shared memory serves 8 window reads instead of 20
#pragma unroll
            for (int m = 0; m < kOzMmas; ++m) {
              const OzMma& q = kOzOrder[m];
              const uint64_t adesc = ptx::smem_desc(sz + (uint32_t)q.w * zb, 128u, 256u);
              const uint64_t bdesc = ptx::smem_desc(sa + (uint32_t)(q.sd - 1) * aslice, 128u, 256u);
              const uint32_t td = tmem_base + (uint32_t)(q.acc * kAccCols);
              const uint32_t accum = (first && q.first) ? 0u : 1u;
              if (q.coll == 0) ptx::mma_f16(td, adesc, bdesc, idesc, accum);
              else if (q.coll == 1) ptx::mma_f16_coll<ptx::CollA::fill>(td, adesc, bdesc, idesc, accum);
              else if (q.coll == 2) ptx::mma_f16_coll<ptx::CollA::use>(td, adesc, bdesc, idesc, accum);
              else ptx::mma_f16_coll<ptx::CollA::lastuse>(td, adesc, bdesc, idesc, accum);
            }
            ptx::mma_commit(&empty[s]);
            if (++s == nstages) { s = 0; ph ^= 1u; }
          }
        }
        if (!ok) break;
        ptx::mma_commit(acc_full);
        aph ^= 1u;
      }
      if (!ok) {
        s_abort = 1;
        atomicOr(&g_oz_error, 16u);
      }
      // every MMA issued has completed before tensor memory is freed (also
      // after an abort left accumulators unread)
      ptx::mma_commit(mma_done);
      volatile int never = 0;
      ptx::mbar_wait(mma_done, 0, &never);
    }
  } else {
    // ---------------- epilogue, warps 2..5 -> TMEM lane quarters 2,3,0,1
    const int q = warp & 3;
    const int m = 32 * q + lane;                 // D row = TMEM lane
    const int rb = g.rb, R = g.R, nb = g.nb, nbp8 = g.nbp8;
    // row group: 0 Re X (level c), 1 Im X (level c), 2 Re X (c + 1), 3 Im X (c + 1)
    const int grp = m / rb, r = m % rb;
    const bool live = r < R && grp < 4;
    const bool writer = live && grp == 0;
    const bool imag = (grp & 1) != 0;
    const int up = (grp >> 1) & 1;
    const double2* Xp = od.X;
    double2* Yp = od.Y;
    const double sig = writer ? ldexp(__ldg(&od.sigma[r]), -kNormShift) : 0.0;
    const unsigned long long lim_dbg = g_oz_wait_ns;
    const uint64_t wait_ns = lim_dbg ? lim_dbg : 1000000000ull;
    int xbuf = 0;
    uint32_t aph = 0;
    for (int64_t x = blockIdx.x; x < V; x += gridDim.x) {
      double sc = 0.0, dx = 0.0;
      int64_t xin = x;             // x on the input lattice (differs with an input halo)
      if (writer) {
        sc = __ldg(&od.scale[x]) * sig;
        dx = __ldg(&od.diag[x]);
        int64_t rr = x, acc_in = 0, stride = 1;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
          const int c = (int)(rr % od.st.L[mu]);
          rr /= od.st.L[mu];
          acc_in += (int64_t)(c + od.st.h[mu]) * stride;
          stride *= od.st.Lin[mu];
        }
        xin = acc_in;
      }
      const bool got = ptx::mbar_wait(acc_full, aph, &s_abort, wait_ns);
      if (!ptx::epilogue_all(got)) {
        s_abort = 1;
        atomicOr(&g_oz_error, 32u);
        break;
      }
      ptx::tc_fence_after();
      const uint32_t taddr = tmem_base + ((uint32_t)(32 * q) << 16);
      for (int c0 = 0; c0 < nbp8; c0 += kChunk) {
        long long vre[kChunk], vim[kChunk];
#pragma unroll
        for (int e = 0; e < kChunk; ++e) vre[e] = vim[e] = 0;
#pragma unroll
        for (int a = 0; a < kNumAcc; ++a) {
          // every lane loads (tcgen05.ld is warp-collective): u = D[.][a'],
          // w = D[.][nb8 + a'] for the chunk's output rows a'
          float u[kChunk], w[kChunk];
          ptx::tmem_ld8_sync(taddr + (uint32_t)(a * kAccCols + c0), u);
          ptx::tmem_ld8_sync(taddr + (uint32_t)(a * kAccCols + nbp8 + c0), w);
          // level 2a + 2 + up, weight 2^(6 (8 - level)); level 9 (a = 3,
          // upper half) enters rounded to the unit of level 8 (the product
          // by 2^-6 is exact in FP32)
          const int sh = kBeta * (kLevels - 2 - 2 * a - up);
#pragma unroll
          for (int e = 0; e < kChunk; ++e) {
            long long iu, iw;
            if (sh >= 0) {
              iu = (long long)__float2int_rn(u[e]) << sh;
              iw = (long long)__float2int_rn(w[e]) << sh;
            } else {
              iu = __float2ll_rn(u[e] * 0.015625f);
              iw = __float2ll_rn(w[e] * 0.015625f);
            }
            if (!imag) {          // Re X row: (Re A x, Im A x)
              vre[e] += iu;
              vim[e] += iw;
            } else {              // Im X row: (-Im A x, Re A x)
              vre[e] -= iw;
              vim[e] += iu;
            }
          }
        }
        if (c0 + kChunk >= nbp8) {      // last chunk read: release the accumulators
          ptx::tc_fence_before();
          __syncwarp();
          if (lane == 0) ptx::mbar_arrive(acc_empty);
        }
        // exchange layout [group - 1][value][row r]: consecutive lanes touch
        // consecutive 8-byte words (no bank conflicts)
        long long* xe = ex + xbuf * (3 * rb * 2 * kChunk);
        if (live && !writer) {
          long long* slot = xe + (grp - 1) * 2 * kChunk * rb + r;
#pragma unroll
          for (int e = 0; e < kChunk; ++e) {
            slot[e * rb] = vre[e];
            slot[(kChunk + e) * rb] = vim[e];
          }
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (writer) {
#pragma unroll
          for (int gg = 0; gg < 3; ++gg) {
            const long long* slot = xe + gg * 2 * kChunk * rb + r;
#pragma unroll
            for (int e = 0; e < kChunk; ++e) {
              vre[e] += slot[e * rb];
              vim[e] += slot[(kChunk + e) * rb];
            }
          }
#pragma unroll
          for (int e = 0; e < kChunk; ++e) {
            const int ar = c0 + e;
            if (ar < nb) {
              const int64_t idx = ((int64_t)x * nb + ar) * R + r;
              const double2 xv = __ldg(&Xp[((int64_t)xin * nb + ar) * R + r]);
              Yp[idx] = make_double2(fma(sc, (double)vre[e], dx * xv.x),
                                     fma(sc, (double)vim[e], dx * xv.y));
            }
          }
        }
        xbuf ^= 1;
      }
      aph ^= 1u;
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem_base, kTmemCols);
  }
}

// Shared memory of a launch: barriers (1 KB), the ring, the two exchange
// buffers, and the rows an M = 128 operand read runs past the last stage's
// input area (a window starts at most 2 (kDigits - 1) rb rows in, the area
// holds 2 (kDigits + 1) rb; rows of D beyond 4 rb are never read).
struct OzRing {
  int nstages = 0;
  size_t smem = 0;
};

OzRing plan_oz_ring(const OzGeom& g) {
  OzRing out;
  const size_t ex = 2 * (size_t)3 * g.rb * 2 * kChunk * sizeof(long long);
  const int over = kM - 4 * g.rb;
  const size_t tail = (size_t)(over > 0 ? over : 0) * 32u;
  const size_t fixed = 1024 + ex + tail;
  if (kSmemBudget < fixed + 2 * (size_t)g.stage) return out;
  int ns = (int)((kSmemBudget - fixed) / g.stage);
  if (ns > kMaxStages) ns = kMaxStages;
  out.nstages = ns;
  out.smem = fixed + (size_t)ns * g.stage;
  // more than half the shared memory keeps the CTA alone on its SM (it holds
  // all 512 TMEM columns)
  if (out.smem < kSmemOneCta) out.smem = kSmemOneCta;
  return out;
}

}  // namespace

int oz_supported(const mrhs_op_s* op, int nrhs) {
  if (op->nb > 64 || nrhs < 1 || nrhs > 32) return 0;
  return plan_oz_ring(make_oz_geom(op->nb, nrhs)).nstages >= 2;
}

int oz_build(mrhs_op_s* op, bool dag, const double2* A, cudaStream_t s) {
  OzImage& img = dag ? op->oz_dag : op->oz;
  if (img.digits) return MRHS_OK;
  if (!A) return fail(MRHS_ERR_INVALID_ARG, "no source coefficients for the digit image");
  const OzGeom g = make_oz_geom(op->nb, 1);
  img.bytes = (size_t)op->V * op->npts * g.nk * g.aslab;
  if (cudaMalloc(&img.digits, img.bytes) != cudaSuccess ||
      cudaMalloc(&img.scale, sizeof(double) * op->V) != cudaSuccess ||
      cudaMalloc(&img.diag, sizeof(double) * op->V) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(img.digits);
    cudaFree(img.scale);
    cudaFree(img.diag);
    img = OzImage();
    return fail(MRHS_ERR_NO_MEMORY, "digit-sliced coefficient image");
  }
  { k_oz_pack_coef<<<(unsigned)op->V, 256, 0, s>>>(A, (uint8_t*)img.digits, img.scale, img.diag,
                                                   op->nbr_bwd, op->V, op->npts, g, dag ? 1 : 0);
    count_launch(); }
  MRHS_CUDA_TRY(cudaGetLastError());
  return MRHS_OK;
}

int oz_apply(mrhs_op_s* op, bool dag, const void* X, void* Y, int nrhs, cudaStream_t s) {
  if (!oz_supported(op, nrhs))
    return fail(MRHS_ERR_UNSUPPORTED, "digit-sliced operator: nb <= 64, nrhs <= 32");
  if (dag && !op->oz_dag.digits) {
    if (!op->a64) return fail(MRHS_ERR_UNSUPPORTED, "daggered digit image needs FP64 coefficients");
    MRHS_TRY(oz_build(op, true, op->a64, s));
  }
  const OzImage& img = dag ? op->oz_dag : op->oz;
  if (!img.digits) return fail(MRHS_ERR_UNSUPPORTED, "digit-sliced image not built");
  const OzGeom g = make_oz_geom(op->nb, nrhs);
  const OzRing ring = plan_oz_ring(g);
  // column maxima and scales at a fixed head (the maxima stay zero between
  // applications), the input digits after it
  constexpr size_t kHead = 1024;
  const size_t before = op->ws_ozpack.bytes;
  MRHS_TRY(op->ws_ozpack.ensure(kHead + (size_t)op->Vin * g.nk * g.xslab));
  unsigned long long* colmax = (unsigned long long*)op->ws_ozpack.ptr;
  double* sigma = (double*)(colmax + MRHS_MAX_RHS);
  uint8_t* xb = (uint8_t*)op->ws_ozpack.ptr + kHead;
  if (op->ws_ozpack.bytes != before)
    MRHS_CUDA_TRY(cudaMemsetAsync(colmax, 0, sizeof(unsigned long long) * MRHS_MAX_RHS, s));
  const int sms = num_sms();
  { k_oz_colmax<<<sms * 4, 256, 0, s>>>((const double2*)X, colmax, op->Vin * op->nb, nrhs);
    count_launch(); }
  { k_oz_colscale<<<1, 64, 0, s>>>(colmax, sigma, nrhs); count_launch(); }
  { k_oz_pack_x<<<sms * 8, 256, 0, s>>>((const double2*)X, sigma, xb, op->Vin, g); count_launch(); }
  MRHS_CUDA_TRY(cudaGetLastError());
  OzDesc od;
  od.coef = (const uint8_t*)img.digits;
  od.xb = xb;
  od.scale = img.scale;
  od.diag = img.diag;
  od.sigma = sigma;
  od.X = (const double2*)X;
  od.Y = (double2*)Y;
  od.V = op->V;
  od.npts = op->npts;
  od.idesc = ptx::idesc_f16(kM, g.N, false);
  od.g = g;
  for (int mu = 0; mu < 4; ++mu) {
    od.st.L[mu] = op->L[mu];
    od.st.Lin[mu] = op->Lin[mu];
    od.st.h[mu] = op->halo[mu];
  }
  od.st.sign = dag ? -1 : 1;
  for (int p = 0; p < op->npts; ++p)
    for (int mu = 0; mu < 4; ++mu) od.st.d[p][mu] = op->disp[p][mu];
  MRHS_CUDA_TRY(cudaFuncSetAttribute(k_op_oz, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)ring.smem));
  const int64_t grid = op->V < sms ? op->V : sms;
  timer_mark(op, MRHS_PREC_OZ, s);
  { k_op_oz<<<(unsigned)grid, kThreads, ring.smem, s>>>(od, ring.nstages); count_launch(); }
  timer_mark(op, MRHS_PREC_OZ, s);
  MRHS_CUDA_TRY(cudaGetLastError());
  return MRHS_OK;
}

int oz_set_wait_limit(unsigned long long ns) {
  MRHS_CUDA_TRY(cudaMemcpyToSymbol(g_oz_wait_ns, &ns, sizeof(ns)));
  return MRHS_OK;
}

unsigned oz_read_and_clear_error() {
  unsigned v = 0, z = 0;
  cudaMemcpyFromSymbol(&v, g_oz_error, sizeof(v));
  cudaMemcpyToSymbol(g_oz_error, &z, sizeof(z));
  return v;
}

}  // namespace mrhs
