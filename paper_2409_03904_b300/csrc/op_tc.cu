// Coarse operator on the 5th-generation tensor cores (tcgen05): BF16, FP16,
// and two split forms (FP16X, TC32) that reach FP32-class accuracy from
// 16-bit operands.
//
// Y(x) = sum_p A_p(x) X(x + delta_p)   (Sec. 2.6, "Applying the coarse
// operator"), in the quantised form: the mean real diagonal d_x of the self
// block is carried exactly in FP32, the remainder of the site's coefficient
// block is stored as 16-bit codes times a power-of-two site scale s_x, every
// RHS column of the input as codes times a power-of-two sigma_r, and
//   Y(x) = s_x sigma_r sum_p Ahat_p(x) Xhat(x + delta_p) + d_x X(x),
// with the sum accumulated in FP32 in tensor memory.
//
// Complex GEMM with the real and imaginary coefficient blocks stacked along
// N.  For one site and stencil point, with the coefficient tile
//     AT = [Re A ; Im A]   (2 nb8 rows: rows a < nb8 = Re A[a][:], rows
//                           nb8 + a = Im A[a][:]; K = nb16 columns over b)
// and input rows Xr_r = Re X[:,r], Xi_r = Im X[:,r] (K = nb16 columns),
//     D (rows x 2 nb8) = XT . AT^T
// gives on an Xr row the products Xr.Re A^T | Xr.Im A^T and on an Xi row
// Xi.Re A^T | Xi.Im A^T, so
//     Re Y[a][r] = D[Xr_r][a] - D[Xi_r][nb8 + a]
//     Im Y[a][r] = D[Xr_r][nb8 + a] + D[Xi_r][a].
// Neither operand is duplicated and one MMA of N = 2 nb8 covers both parts:
// M = 128, N = 2 nb8, K = 16, nb16/16 MMAs per stencil point, summed over all
// points into one accumulator.  The tensor core reads the whole 128-row A
// operand from shared memory for every MMA, so few wide MMAs (large N) keep
// that read traffic, which shares shared-memory bandwidth with the TMA
// writes, low.  The epilogue combines the Xi row's values with the Xr row's
// through shared memory.
//
// Split forms (up to 32 right-hand sides): a value u is held as hi = fp16(u),
// lo = fp16((u - hi) 2^11).  XSPLIT adds the input's lo rows (Xr_lo, Xi_lo)
// as two more row groups of the same operand, so one MMA also gives Ahi Xlo;
// ASPLIT stacks the coefficients' lo tile under the hi tile along N (the two
// tiles are contiguous with the same layout), so one MMA of N = 4 nb8 also
// gives Alo X in the accumulator columns 2 nb8 .. 4 nb8 (used on the hi rows).
// An MMA of twice the width costs the tensor core far less than two.  The epilogue adds 2^-11 times
// the lo contributions.  FP16X = FP16 coefficients with a two-term input
// (linear in X to ~2^-22, for a stationary preconditioner); TC32 = both
// operands in two terms (FP32-class operator, same bytes per coefficient as
// complex64).
//
// Both operands are pre-packed in global memory in the canonical K-major
// no-swizzle tcgen05 layout (8 x 16-byte core matrices, K groups 128 bytes
// apart, 8-row groups K/8*128 bytes apart), so a single 1-D bulk TMA copy
// per tile lands it ready for the MMA.  Element (row, k) of a tile with K
// columns sits at byte (row/8)*(K/8)*128 + (k/8)*128 + (row%8)*16 + (k%8)*2.
//
// Kernel: persistent, two CTAs per SM by default (two independent rings;
// TC32, whose two double-buffered accumulators fill the tensor memory, runs
// one),
// warp-specialised:
//   warp 0      TMA producer: per stage the coefficient tiles of `pps`
//               consecutive stencil points of one site (contiguous, one bulk
//               copy, L2 evict-first) and their neighbours' packed X tiles
//               (L2 evict-last), into an nstage ring of shared memory
//   warp 1      allocates TMEM, issues tcgen05.mma (one elected thread) into
//               two alternating sets of accumulators, commits stage releases
//   warps 2-5   epilogue: tcgen05.ld of their 32-lane quarter in 8-column
//               chunks, every row group's contribution posted to shared
//               memory; then all 128 threads split the chunk's outputs, sum
//               the groups, scale, add d_x X(x) (and the Chebyshev step) and
//               store complex64 Y, the chunk's global reads issued ahead
// Every mbarrier wait is bounded (1 s); on expiry the kernel records an
// error, drains its own copies, frees TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace mrhs {

__device__ unsigned int g_tc_error = 0;
// limit of the epilogue's accumulator wait in ns (0: the default 1 s); set
// only by the debugging entry point mrhs_debug_wait_limit
__device__ unsigned long long g_tc_wait_ns = 0;

namespace {

constexpr int kThreadsTc = 192;
constexpr int kAccCols = 128;    // TMEM columns per accumulator (n_mma <= 128)
constexpr int kChunk = 8;        // epilogue columns per tcgen05.ld
constexpr int kExFloats = 4 * 2 * kChunk * 32;   // one exchange buffer ([4][2][8][32] or [2][2][8][64])
constexpr int kM = 128;
constexpr size_t kSmemBudget = 220 * 1024;   // dynamic shared memory per SM
constexpr size_t kSmemOneCta = 120 * 1024;   // at least this much keeps a CTA alone on its SM
constexpr float kLoScale = 1.0f / 2048.0f;   // 2^-11

struct Geom {
  int nb, nbp8, nb16, K, n_mma;   // K = nb16, N = 2 nb8
  int R, rb, xrows;         // rb = round8(R): rows per input row group
  int xsplit, asplit;
  uint32_t coef1;           // one coefficient tile (hi or lo)
  uint32_t coef_bytes;      // coefficient bytes per stencil point (x2 if asplit)
  uint32_t xb_bytes, sbo;
};

Geom make_geom(int nb, int R, bool xsplit, bool asplit) {
  Geom g;
  g.nb = nb;
  g.nbp8 = (nb + 7) / 8 * 8;
  g.nb16 = (nb + 15) / 16 * 16;
  g.K = g.nb16;
  g.n_mma = 2 * g.nbp8;
  g.R = R;
  g.xsplit = xsplit;
  g.asplit = asplit;
  // input row groups Xr, Xi (then Xr_lo, Xi_lo), round8(R) rows each
  g.rb = (R + 7) / 8 * 8;
  g.xrows = (xsplit ? 4 : 2) * g.rb;
  g.coef1 = (uint32_t)(2 * g.nbp8) * g.K * 2;
  g.coef_bytes = g.coef1 * (asplit ? 2u : 1u);
  g.xb_bytes = (uint32_t)g.xrows * g.K * 2;
  g.sbo = (uint32_t)(g.K / 8) * 128;
  return g;
}

// Stencil geometry by value in the kernel parameters, so the TMA producer
// forms x +- delta_p with a few integer operations instead of a dependent
// global load per tile.
struct Stencil {
  int32_t L[4];
  int32_t sign;            // +1: x + delta_p (forward); -1: x - delta_p (adjoint)
  int8_t d[MRHS_MAX_PTS][4];
};

__host__ __device__ inline uint32_t canon_off(int row, int k, int K) {
  return (uint32_t)(row >> 3) * (uint32_t)(K >> 3) * 128u + (uint32_t)(k >> 3) * 128u +
         (uint32_t)(row & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

__device__ inline double pow2_ceil(double m) {
  if (!(m > 0.0)) return 1.0;
  int e;
  const double f = frexp(m, &e);
  if (f == 0.5) e -= 1;
  return ldexp(1.0, e);
}

template <bool BF16>
__device__ inline uint16_t code16(float v) {
  if (BF16) return __bfloat16_as_ushort(__float2bfloat16_rn(v));
  return __half_as_ushort(__float2half_rn(v));
}
// two-term split of an FP32 value: hi = fp16(u), lo = fp16((u - hi) 2^11)
__device__ inline void split16(float u, uint16_t& hi, uint16_t& lo) {
  const __half h = __float2half_rn(u);
  hi = __half_as_ushort(h);
  lo = __half_as_ushort(__float2half_rn((u - __half2float(h)) * 2048.0f));
}

int image_index(int prec) {
  switch (prec) {
    case MRHS_PREC_BF16: return 0;
    case MRHS_PREC_FP16:
    case MRHS_PREC_FP16X: return 1;
    case MRHS_PREC_TC32: return 2;
    default: return -1;
  }
}

// One CTA per site: d_x, s_x and the codes of the site's coefficient tiles.
// dag: the block of stencil point p at site x is A_p(x - delta_p)^dagger.
// ASPLIT: each point gets a hi tile followed by a lo tile.
// Largest |Re|, |Im| of the coefficients over all sites, the mean real
// diagonal of each site's self block removed as in k_pack_coef (double bits,
// ordered like the values): the one scale of an image whose tiles are shared
// between sites (Hermitian pairing).
__global__ void __launch_bounds__(256) k_coef_gmax(const double2* __restrict__ A, int64_t V,
                                                   int npts, int nb,
                                                   unsigned long long* gmax) {
  const int64_t x = blockIdx.x;
  if (x >= V) return;
  __shared__ double s_red[256];
  const double2* Ax = A + x * npts * (int64_t)nb * nb;
  double acc = 0.0;
  for (int a = threadIdx.x; a < nb; a += blockDim.x) acc += Ax[a * nb + a].x;
  s_red[threadIdx.x] = acc;
  __syncthreads();
  __shared__ float s_d;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) t += s_red[i];
    s_d = __double2float_rn(t / nb);
  }
  __syncthreads();
  const double d = (double)s_d;
  const int nn = nb * nb;
  double m = 0.0;
  for (int i = threadIdx.x; i < npts * nn; i += blockDim.x) {
    double2 v = Ax[i];
    if (i < nn && (i / nb) == (i % nb)) v.x -= d;
    m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
  }
  atomicMax(gmax, (unsigned long long)__double_as_longlong(m));
}

__global__ void k_coef_gscale(const unsigned long long* gmax, double* gscale) {
  *gscale = pow2_ceil(__longlong_as_double((long long)*gmax));
}

template <bool BF16, bool ASPLIT>
__global__ void __launch_bounds__(256) k_pack_coef(const double2* __restrict__ A, uint8_t* codes,
                                                   float* scale, float* diag,
                                                   const int32_t* __restrict__ nbr_bwd, int64_t V,
                                                   int npts, int nb, Geom g, int dag,
                                                   const double* __restrict__ gscale) {
  const int64_t x = blockIdx.x;
  if (x >= V) return;
  __shared__ double s_red[256];
  __shared__ float s_d;
  __shared__ double s_scale;
  const int nn = nb * nb;
  auto src = [&](int p, int a, int b) -> double2 {
    if (!dag) return A[((x * npts + p) * (int64_t)nb) * nb + a * nb + b];
    const int64_t y = nbr_bwd[(int64_t)p * V + x];
    const double2 v = A[((y * npts + p) * (int64_t)nb) * nb + b * nb + a];
    return make_double2(v.x, -v.y);
  };
  // d_x: mean real diagonal of the self block, rounded to FP32
  double acc = 0.0;
  for (int a = threadIdx.x; a < nb; a += blockDim.x) acc += src(0, a, a).x;
  s_red[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) t += s_red[i];
    s_d = __double2float_rn(t / nb);
  }
  __syncthreads();
  const double d = (double)s_d;
  double m = 0.0;
  for (int i = threadIdx.x; i < npts * nn; i += blockDim.x) {
    const int p = i / nn, a = (i % nn) / nb, b = i % nb;
    double2 v = src(p, a, b);
    if (p == 0 && a == b) v.x -= d;
    m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
  }
  s_red[threadIdx.x] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) t = fmax(t, s_red[i]);
    s_scale = gscale ? *gscale : pow2_ceil(t);   // one scale for all sites, or the site's own
    scale[x] = (float)s_scale;
    diag[x] = s_d;
  }
  __syncthreads();
  const double inv = 1.0 / s_scale;   // exact: power of two
  const int tile_elems = 2 * g.nbp8 * g.K;
  for (int p = 0; p < npts; ++p) {
    uint8_t* tile = codes + ((uint64_t)x * npts + p) * g.coef_bytes;
    for (int i = threadIdx.x; i < tile_elems; i += blockDim.x) {
      const int row = i / g.K, b = i % g.K;
      const bool re = row < g.nbp8;           // [Re A ; Im A], nb8 rows each
      const int a = re ? row : row - g.nbp8;
      float v = 0.f;
      if (a < nb && b < nb) {
        double2 c = src(p, a, b);
        if (p == 0 && a == b) c.x -= d;
        v = __double2float_rn((re ? c.x : c.y) * inv);
      }
      if (ASPLIT) {
        uint16_t hi, lo;
        split16(v, hi, lo);
        *reinterpret_cast<uint16_t*>(tile + canon_off(row, b, g.K)) = hi;
        *reinterpret_cast<uint16_t*>(tile + g.coef1 + canon_off(row, b, g.K)) = lo;
      } else {
        *reinterpret_cast<uint16_t*>(tile + canon_off(row, b, g.K)) = code16<BF16>(v);
      }
    }
  }
}

// Input packing of every problem of a launch, three launches in all: column
// maxima, column scales, real-split tiles.  Each kernel runs a 2-D grid whose
// blockIdx.y is the problem; a problem masked out by `active` returns at once.
struct PackProb {
  const float2* X;          // complex64 [V][nb][R]
  unsigned* colmax;         // [64] float bits, zero on entry (reset by k_colscale)
  float* sigma;             // [64]
  uint8_t* xb;              // packed tiles
  int64_t V;
  Geom g;
};
struct PackBatch {
  int32_t n;
  const int32_t* active;
  PackProb p[MRHS_MAX_BATCH];
};

__device__ __forceinline__ bool pack_live(const PackBatch& pb, int k) {
  return pb.active == nullptr || pb.active[k] != 0;
}

// Per-column max |Re|, |Im| of a problem's [N][R] block (as float bits): a
// thread keeps one column, so the maximum stays in a register until the end.
__global__ void k_colmax(const __grid_constant__ PackBatch pb) {
  const int k = blockIdx.y;
  if (!pack_live(pb, k)) return;
  const PackProb& pp = pb.p[k];
  const int R = pp.g.R;
  const int rows_per_block = blockDim.x / R;
  const int t = threadIdx.x;
  __shared__ unsigned s_m[MRHS_MAX_RHS];
  for (int i = t; i < R; i += blockDim.x) s_m[i] = 0u;
  __syncthreads();
  if (t < rows_per_block * R) {
    const int c = t % R;
    const int64_t N = pp.V * pp.g.nb;
    const float2* X = pp.X;
    float m = 0.f;
    for (int64_t row = (int64_t)blockIdx.x * rows_per_block + t / R; row < N;
         row += (int64_t)gridDim.x * rows_per_block) {
      const float2 v = X[row * R + c];
      m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    atomicMax(&s_m[c], __float_as_uint(m));
  }
  __syncthreads();
  for (int i = t; i < R; i += blockDim.x)
    if (s_m[i]) atomicMax(&pp.colmax[i], s_m[i]);
}

// sigma_r = 2^e >= column max (1 for a zero column); stored as float.  The
// maxima are cleared for the next application.
__global__ void k_colscale(const __grid_constant__ PackBatch pb) {
  const int k = blockIdx.x;
  if (!pack_live(pb, k)) return;
  const PackProb& pp = pb.p[k];
  const int r = threadIdx.x;
  if (r < pp.g.R) {
    pp.sigma[r] = (float)pow2_ceil((double)__uint_as_float(pp.colmax[r]));
    pp.colmax[r] = 0u;
  }
}

// Packed input tiles, one [xrows][K] canonical tile per site: row group 0
// holds Re X[:,r] / sigma_r in row r, group 1 Im X[:,r] / sigma_r (groups
// round8(R) rows apart, K = nb16 columns over b); XSPLIT: groups 0, 1 the hi
// terms, groups 2, 3 the lo terms.  A thread takes one (site, 8-column group,
// column r): it reads the eight complex values once and writes the 16-byte
// unit of every row group (consecutive threads: consecutive r, so both the
// reads and the 8-row core-matrix writes are coalesced).
template <bool BF16, bool XSPLIT>
__global__ void k_pack_xb(const __grid_constant__ PackBatch pb) {
  const int k = blockIdx.y;
  if (!pack_live(pb, k)) return;
  const PackProb& pp = pb.p[k];
  const Geom g = pp.g;
  const float2* __restrict__ X = pp.X;
  const float* __restrict__ sigma = pp.sigma;
  uint8_t* xb = pp.xb;
  const int nb = g.nb, R = g.R, rb = g.rb;
  const int nkc = g.K / 8;
  const int64_t total = pp.V * nkc * rb;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < total;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(u % rb);
    const int64_t t = u / rb;
    const int kc = (int)(t % nkc);
    const int64_t x = t / nkc;
    const bool live = r < R;
    const float inv = live ? 1.0f / sigma[r] : 0.f;
    uint16_t h[4][8];        // row groups: Re hi, Im hi, Re lo, Im lo
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int b = kc * 8 + e;
      float2 v = make_float2(0.f, 0.f);
      if (live && b < nb) {
        const float2 xv = X[(x * nb + b) * R + r];
        v = make_float2(xv.x * inv, xv.y * inv);
      }
      if (XSPLIT) {
        split16(v.x, h[0][e], h[2][e]);
        split16(v.y, h[1][e], h[3][e]);
      } else {
        h[0][e] = code16<BF16>(v.x);
        h[1][e] = code16<BF16>(v.y);
      }
    }
    uint8_t* tile = xb + (uint64_t)x * g.xb_bytes;
#pragma unroll
    for (int grp = 0; grp < (XSPLIT ? 4 : 2); ++grp) {
      uint4 pk;
      pk.x = (uint32_t)h[grp][0] | ((uint32_t)h[grp][1] << 16);
      pk.y = (uint32_t)h[grp][2] | ((uint32_t)h[grp][3] << 16);
      pk.z = (uint32_t)h[grp][4] | ((uint32_t)h[grp][5] << 16);
      pk.w = (uint32_t)h[grp][6] | ((uint32_t)h[grp][7] << 16);
      *reinterpret_cast<uint4*>(tile + canon_off(grp * rb + r, kc * 8, g.K)) = pk;
    }
  }
}

// One problem of a launch: its operands, geometry and stencil.
struct ProbDesc {
  const uint8_t* coef;      // packed coefficient image
  const uint8_t* xb;        // packed input tiles
  const float* scale;       // s_x
  const float* diag;        // d_x
  const float* sigma;       // sigma_r
  const float* X;           // complex64 input (as floats), for d_x X(x)
  float* Y;                 // complex64 output
  int64_t V, item0;         // sites; first item of this problem in the work list
  int32_t npts, nb, nbp8, K, n_mma, R, pps, rb;
  uint32_t coef1, coef_bytes, xb_bytes, sbo, idesc, xb_off;
  // Chebyshev step in the epilogue (cheb != 0): W = H X is not stored; with
  // the recurrence's a, b and coefficient c (c0 too for the first step)
  //   cheb 1:  T = a W + b X,             P = c0 X + c T
  //   cheb 2:  T = 2 (a W + b X) - Tp,    P = P + c T
  // T goes to Tout (may be Tp); colmax_next, when set, receives the column
  // maxima of T for the next application's packing.
  int32_t cheb;
  float ca, cb, cc, c0;
  float* Tout;
  const float* Tp;
  float* P;
  unsigned* colmax_next;
  // Hermitian pairing (herm != 0): one stage per pair (p, -p) of the nf
  // points fpts[] plus the self term; sites visited in blocks bl[4]; the
  // partner tile A_p(x - delta_p) is read transposed (idesc_t: Re half,
  // idesc_tn: Im half negated) to give A_{-p}(x) = A_p(x - delta_p)^dagger
  int32_t herm, nf;
  int32_t bl[4];
  uint32_t idesc_t, idesc_tn;
  int8_t fpts[MRHS_MAX_PTS / 2];
  Stencil st;
};

// Every problem of one launch, by value in the kernel parameters (large
// kernel parameters: no upload, nothing to capture separately in a graph).
struct Batch {
  int32_t n;
  int64_t total;            // items (sites) over all problems
  const int32_t* active;    // per problem 0/1, or null (all active)
  ProbDesc p[MRHS_MAX_BATCH];
};

__device__ __forceinline__ int find_prob(const Batch& bt, int64_t t) {
  int k = 0;
  for (int i = 1; i < bt.n; ++i)
    if (t >= bt.p[i].item0) k = i;
  return k;
}
// Site of a problem's i-th work item: linear order, or (paired mode) blocks
// of bl[0] x .. x bl[3] sites, so that the sites in flight together are
// neighbours and share their coefficient tiles through L2.
__device__ __forceinline__ int64_t site_of(const ProbDesc& pd, int64_t i) {
  if (!pd.herm) return i;
  const int b0 = pd.bl[0], b1 = pd.bl[1], b2 = pd.bl[2], b3 = pd.bl[3];
  const int64_t bvol = (int64_t)b0 * b1 * b2 * b3;
  int64_t blk = i / bvol;
  int in = (int)(i - blk * bvol);
  const int c0 = in % b0;
  in /= b0;
  const int c1 = in % b1;
  in /= b1;
  const int c2 = in % b2;
  const int c3 = in / b2;
  const int n0 = pd.st.L[0] / b0, n1 = pd.st.L[1] / b1, n2 = pd.st.L[2] / b2;
  const int q0 = (int)(blk % n0);
  blk /= n0;
  const int q1 = (int)(blk % n1);
  blk /= n1;
  const int q2 = (int)(blk % n2);
  const int q3 = (int)(blk / n2);
  (void)b3;
  const int64_t x0 = q0 * b0 + c0, x1 = q1 * b1 + c1, x2 = q2 * b2 + c2, x3 = q3 * b3 + c3;
  return x0 + pd.st.L[0] * (x1 + (int64_t)pd.st.L[1] * (x2 + (int64_t)pd.st.L[2] * x3));
}

__device__ __forceinline__ bool item_live(const Batch& bt, int k) {
  return bt.active == nullptr || bt.active[k] != 0;
}

template <bool BF16, bool XSPLIT, bool ASPLIT>
__global__ void __launch_bounds__(kThreadsTc, ASPLIT ? 1 : 2)
    k_op_tc(const __grid_constant__ Batch bt, int nstages, uint32_t stage_bytes) {
  extern __shared__ __align__(1024) uint8_t smem[];
  // accumulators per buffer: D, and for ASPLIT the lo-coefficient D2 in the
  // n_mma columns right after it (one MMA of N = 2 n_mma writes both)
  constexpr int kAccStride = (ASPLIT ? 2 : 1) * kAccCols;   // TMEM cols per buffer
  constexpr uint32_t kTmemCols = 2u * kAccStride;           // two buffers
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + nstages;
  uint64_t* acc_full = empty + nstages;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* mma_done = acc_empty + 2;     // every MMA of this CTA has completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
  uint8_t* stages = smem + 1024;
  // a stage holds up to `pps` consecutive stencil points of one site: their
  // coefficient tiles (contiguous in HBM, one bulk copy) at the start, their
  // neighbour input tiles from the problem's `xb_off` on (one stage size for
  // all problems; each packs as many points as fit)
  // two exchange buffers (Xi and lo rows -> Xr rows), after the ring
  float* ex = reinterpret_cast<float*>(stages + (size_t)nstages * stage_bytes);
  __shared__ volatile int s_abort;
  __shared__ unsigned s_cm[MRHS_MAX_RHS];   // epilogue: column maxima of the Chebyshev output

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < nstages; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      ptx::mbar_init(&acc_full[i], 1);
      ptx::mbar_init(&acc_empty[i], 4);
    }
    ptx::mbar_init(mma_done, 1);
    ptx::fence_mbar_init();
    s_abort = 0;
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, kTmemCols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- producer
      const uint64_t pol_stream = ptx::policy_evict_first();
      const uint64_t pol_shared = ptx::policy_evict_normal();
      const uint64_t pol_keep = ptx::policy_evict_last();
      int s = 0;
      uint32_t ph = 0;
      int64_t issued = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < bt.total && ok; t += gridDim.x) {
        const int k = find_prob(bt, t);
        if (!item_live(bt, k)) continue;
        // the problem's fields in registers: the waits and copies below
        // clobber memory, and would otherwise reload them from the parameters
        const ProbDesc& pd = bt.p[k];
        const int64_t x = site_of(pd, t - pd.item0);
        const uint8_t* coef = pd.coef;
        const uint8_t* xbp = pd.xb;
        const int npts = pd.npts, pps = pd.pps, sign = pd.st.sign;
        const uint32_t cbytes = pd.coef_bytes, xbytes = pd.xb_bytes, xb_off = pd.xb_off;
        const uint32_t* dwords = reinterpret_cast<const uint32_t*>(&pd.st.d[0][0]);
        int Lm[4], c[4];
        {
          int64_t r = x;
#pragma unroll
          for (int mu = 0; mu < 4; ++mu) {
            Lm[mu] = pd.st.L[mu];
            c[mu] = (int)(r % Lm[mu]);
            r /= Lm[mu];
          }
        }
        if (pd.herm) {
          // one stage per pair (p, -p): A_p(x) and X(x + delta_p), the
          // partner tile A_p(x - delta_p) and X(x - delta_p); the self term
          // first.  Tiles are left in L2 for the neighbour that shares them.
          const int nf = pd.nf;
          for (int j = 0; j <= nf && ok; ++j) {
            if (!ptx::mbar_wait(&empty[s], ph ^ 1u, &s_abort)) { ok = false; break; }
            uint8_t* st_smem = stages + (size_t)s * stage_bytes;
            if (j == 0) {
              ptx::mbar_arrive_expect_tx(&full[s], cbytes + xbytes);
              ptx::bulk_g2s(st_smem, coef + (uint64_t)x * npts * cbytes, cbytes, &full[s],
                            pol_shared);
              ptx::bulk_g2s(st_smem + xb_off, xbp + (uint64_t)x * xbytes, xbytes, &full[s],
                            pol_shared);
            } else {
              const int p = pd.fpts[j - 1];
              const uint32_t dw = dwords[p];
              int64_t yf = 0, yb = 0;
#pragma unroll
              for (int mu = 3; mu >= 0; --mu) {
                const int d = (int)(int8_t)(dw >> (8 * mu));
                int vf = c[mu] + d, vb = c[mu] - d;
                vf += (vf < 0) ? Lm[mu] : 0;
                vf -= (vf >= Lm[mu]) ? Lm[mu] : 0;
                vb += (vb < 0) ? Lm[mu] : 0;
                vb -= (vb >= Lm[mu]) ? Lm[mu] : 0;
                yf = yf * Lm[mu] + vf;
                yb = yb * Lm[mu] + vb;
              }
              ptx::mbar_arrive_expect_tx(&full[s], 2u * (cbytes + xbytes));
              ptx::bulk_g2s(st_smem, coef + ((uint64_t)x * npts + p) * cbytes, cbytes, &full[s],
                            pol_shared);
              ptx::bulk_g2s(st_smem + cbytes, coef + ((uint64_t)yb * npts + p) * cbytes, cbytes,
                            &full[s], pol_shared);
              ptx::bulk_g2s(st_smem + xb_off, xbp + (uint64_t)yf * xbytes, xbytes, &full[s],
                            pol_shared);
              ptx::bulk_g2s(st_smem + xb_off + xbytes, xbp + (uint64_t)yb * xbytes, xbytes,
                            &full[s], pol_shared);
            }
            ++issued;
            if (++s == nstages) { s = 0; ph ^= 1u; }
          }
          continue;
        }
        for (int p0 = 0; p0 < npts; p0 += pps) {
          const int np = (npts - p0) < pps ? (npts - p0) : pps;
          if (!ptx::mbar_wait(&empty[s], ph ^ 1u, &s_abort)) { ok = false; break; }
          uint8_t* st_smem = stages + (size_t)s * stage_bytes;
          ptx::mbar_arrive_expect_tx(&full[s], (uint32_t)np * (cbytes + xbytes));
          ptx::bulk_g2s(st_smem, coef + ((uint64_t)x * npts + p0) * cbytes,
                        (uint32_t)np * cbytes, &full[s], pol_stream);
          for (int i = 0; i < np; ++i) {
            const uint32_t dw = dwords[p0 + i];      // delta_p, four signed bytes
            int64_t y = 0;
#pragma unroll
            for (int mu = 3; mu >= 0; --mu) {
              int v = c[mu] + sign * (int)(int8_t)(dw >> (8 * mu));
              v += (v < 0) ? Lm[mu] : 0;
              v -= (v >= Lm[mu]) ? Lm[mu] : 0;
              y = y * Lm[mu] + v;
            }
            ptx::bulk_g2s(st_smem + xb_off + (uint32_t)i * xbytes, xbp + (uint64_t)y * xbytes,
                          xbytes, &full[s], pol_keep);
          }
          ++issued;
          if (++s == nstages) { s = 0; ph ^= 1u; }
        }
      }
      if (!ok) {
        s_abort = 1;
        atomicOr(&g_tc_error, 1u);
      }
      // drain: every copy this thread issued has landed before the CTA exits
      const int64_t last = issued < nstages ? issued : nstages;
      for (int64_t i = 0; i < last; ++i) {
        const int64_t n = issued - 1 - i;           // issue index
        const int ss = (int)(n % nstages);
        const uint32_t par = (uint32_t)((n / nstages) & 1);
        volatile int never = 0;
        ptx::mbar_wait(&full[ss], par, &never);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      int s = 0, acc = 0;
      uint32_t ph = 0, aph = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < bt.total && ok; t += gridDim.x) {
        const int k = find_prob(bt, t);
        if (!item_live(bt, k)) continue;
        const ProbDesc& pd = bt.p[k];
        const int nk = pd.K / 16, npts = pd.npts, pps = pd.pps;
        const uint32_t cbytes = pd.coef_bytes, xbytes = pd.xb_bytes, sbo = pd.sbo,
                       idesc = pd.idesc, coef1 = pd.coef1, xb_off = pd.xb_off;
        const uint32_t lo_off = (uint32_t)pd.n_mma;     // D2: columns n_mma .. 2 n_mma
        const uint32_t idesc2 = ptx::idesc_f16(kM, 2 * pd.n_mma, false);
        if (!ptx::mbar_wait(&acc_empty[acc], aph ^ 1u, &s_abort)) { ok = false; break; }
        ptx::tc_fence_after();
        const uint32_t tmem_d = tmem_base + (uint32_t)(acc * kAccStride);
        if (pd.herm) {
          // stage j: forward A_p(x) X(x + delta_p) as usual, then the partner
          // tile read transposed: its Re half into the Re-A columns, its Im
          // half negated into the Im-A columns, giving A_p(x - delta_p)^dagger
          // X(x - delta_p) in the same accumulator
          const int nf = pd.nf;
          const uint32_t idesc_t = pd.idesc_t, idesc_tn = pd.idesc_tn;
          const uint32_t im_row = (uint32_t)(pd.nbp8 / 8) * sbo;   // Im half: row nb8
          const uint32_t im_col = (uint32_t)pd.nbp8;                // TMEM columns of the Im half
          for (int j = 0; j <= nf && ok; ++j) {
            if (!ptx::mbar_wait(&full[s], ph, &s_abort)) { ok = false; break; }
            ptx::tc_fence_after();
            const uint32_t sb = ptx::smem_u32(stages + (size_t)s * stage_bytes);
            const uint32_t ab = sb + xb_off;
            for (int kk = 0; kk < nk; ++kk) {
              const uint32_t accum = (j > 0 || kk > 0) ? 1u : 0u;
              const uint64_t adesc = ptx::smem_desc(ab + (uint32_t)kk * 256u, 128u, sbo);
              const uint64_t bhi = ptx::smem_desc(sb + (uint32_t)kk * 256u, 128u, sbo);
              // hi and lo tiles stacked: one MMA of N = 2 n_mma (ASPLIT)
              ptx::mma_f16(tmem_d, adesc, bhi, ASPLIT ? idesc2 : idesc, accum);
            }
            if (j > 0) {
              const uint32_t cbk = sb + cbytes, abk = ab + xbytes;
              for (int kk = 0; kk < nk; ++kk) {
                const uint64_t adesc = ptx::smem_desc(abk + (uint32_t)kk * 256u, 128u, sbo);
                const uint32_t rows = (uint32_t)kk * 2u * sbo;      // tile rows 16 kk ..
                // (the collector buffer is not used here: reusing the input
                // operand across these transposed, negated MMAs gave wrong sums)
                ptx::mma_f16(tmem_d, adesc, ptx::smem_desc(cbk + rows, sbo, 128u), idesc_t, 1u);
                ptx::mma_f16(tmem_d + im_col, adesc, ptx::smem_desc(cbk + im_row + rows, sbo, 128u),
                             idesc_tn, 1u);
                if (ASPLIT) {
                  ptx::mma_f16(tmem_d + lo_off, adesc,
                               ptx::smem_desc(cbk + coef1 + rows, sbo, 128u), idesc_t, 1u);
                  ptx::mma_f16(tmem_d + lo_off + im_col, adesc,
                               ptx::smem_desc(cbk + coef1 + im_row + rows, sbo, 128u), idesc_tn,
                               1u);
                }
              }
            }
            ptx::mma_commit(&empty[s]);
            if (++s == nstages) { s = 0; ph ^= 1u; }
          }
          if (!ok) break;
          ptx::mma_commit(&acc_full[acc]);
          if (++acc == 2) { acc = 0; aph ^= 1u; }
          continue;
        }
        for (int p0 = 0; p0 < npts; p0 += pps) {
          const int np = (npts - p0) < pps ? (npts - p0) : pps;
          if (!ptx::mbar_wait(&full[s], ph, &s_abort)) { ok = false; break; }
          ptx::tc_fence_after();
          const uint32_t sb = ptx::smem_u32(stages + (size_t)s * stage_bytes);
          for (int i = 0; i < np; ++i) {
            const uint32_t cb = sb + (uint32_t)i * cbytes;
            const uint32_t ab = sb + xb_off + (uint32_t)i * xbytes;
            const uint32_t first = (p0 > 0 || i > 0) ? 1u : 0u;
            for (int j = 0; j < nk; ++j) {
              const uint32_t accum = (first || j > 0) ? 1u : 0u;
              const uint64_t adesc = ptx::smem_desc(ab + (uint32_t)j * 256u, 128u, sbo);
              const uint64_t bhi = ptx::smem_desc(cb + (uint32_t)j * 256u, 128u, sbo);
              // ASPLIT: the hi and lo coefficient tiles, contiguous, form one
              // operand of 2 n_mma rows; one MMA gives both accumulators
              ptx::mma_f16(tmem_d, adesc, bhi, ASPLIT ? idesc2 : idesc, accum);
            }
          }
          ptx::mma_commit(&empty[s]);
          if (++s == nstages) { s = 0; ph ^= 1u; }
        }
        if (!ok) break;
        ptx::mma_commit(&acc_full[acc]);
        if (++acc == 2) { acc = 0; aph ^= 1u; }
      }
      if (!ok) {
        s_abort = 1;
        atomicOr(&g_tc_error, 2u);
      }
      // wait until every MMA this thread issued has completed, so that tensor
      // memory is freed only after its last write, also when an abort left
      // accumulators that nobody reads
      ptx::mma_commit(mma_done);
      volatile int never = 0;
      ptx::mbar_wait(mma_done, 0, &never);
    }
  } else {
    // ---------------- epilogue, warps 2..5 -> TMEM lane quarters 2,3,0,1
    // Per 8-column chunk every live row posts its row group's contribution
    // to (Re Y, Im Y) through shared memory; then the 128 threads split the
    // chunk's 8 R outputs (item i = e R + r, consecutive in Y) and each sums
    // the groups, applies the scales and the Chebyshev step and does the
    // global reads and writes.  The reads of a chunk are issued before its
    // tensor-memory loads (the first chunk's before the accumulator wait), so
    // their latency overlaps the exchange.
    const int q = warp & 3;
    const int mrow = 32 * q + lane;              // D row = TMEM lane
    const int et = (int)threadIdx.x - 64;        // epilogue thread 0..127
    int acc = 0, xbuf = 0;
    uint32_t aph = 0;
    const unsigned long long lim_dbg = g_tc_wait_ns;
    const uint64_t wait_ns = lim_dbg ? lim_dbg : 1000000000ull;
    // column maxima of the Chebyshev output of the current problem
    for (int i = et; i < MRHS_MAX_RHS; i += 128) s_cm[i] = 0u;
    asm volatile("bar.sync 1, 128;" ::: "memory");
    int cm_prob = -1;
    unsigned* cm_dst = nullptr;
    auto post_maxima = [&]() {
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (cm_dst)
        for (int i = et; i < MRHS_MAX_RHS; i += 128)
          if (s_cm[i]) atomicMax(&cm_dst[i], s_cm[i]);
      asm volatile("bar.sync 1, 128;" ::: "memory");
      for (int i = et; i < MRHS_MAX_RHS; i += 128) s_cm[i] = 0u;
    };
    constexpr int kMaxItems = kChunk * MRHS_MAX_RHS / 128;   // outputs per thread and chunk
    for (int64_t t = blockIdx.x; t < bt.total; t += gridDim.x) {
      const int k = find_prob(bt, t);
      if (!item_live(bt, k)) continue;
      const ProbDesc& pd = bt.p[k];
      const int64_t x = site_of(pd, t - pd.item0);
      const int R = pd.R, nb = pd.nb, nbp8 = pd.nbp8, rb = pd.rb;
      const float2* Xp = reinterpret_cast<const float2*>(pd.X);
      float2* Yp = reinterpret_cast<float2*>(pd.Y);
      const int cheb = pd.cheb;
      if (k != cm_prob) {      // a new problem: post the previous one's column maxima
        post_maxima();
        cm_prob = k;
        cm_dst = pd.colmax_next;
      }
      // row group of this lane: 0 Xr, 1 Xi, 2 Xr_lo, 3 Xi_lo
      constexpr int kGroups = XSPLIT ? 4 : 2;
      const int grp = mrow / rb, r_row = mrow % rb;
      const bool live = r_row < R && grp < kGroups;
      const bool imag = (grp & 1) != 0;
      const float gs = grp >= 2 ? kLoScale : 1.0f;
      const float sx = __ldg(&pd.scale[x]), dx = __ldg(&pd.diag[x]);
      const int nitem = kChunk * R;
      const int64_t site0 = (int64_t)x * nb * R;
      // this thread's outputs of a chunk: items et + 128 j
      float2 xv[kMaxItems], tp[kMaxItems], pv[kMaxItems];
      auto load_items = [&](int c0) {
#pragma unroll
        for (int j = 0; j < kMaxItems; ++j) {
          const int i = et + 128 * j;
          const int e = i / R;
          const bool in = i < nitem && c0 + e < nb;
          const int64_t idx = site0 + (int64_t)c0 * R + i;
          xv[j] = in ? __ldg(&Xp[idx]) : make_float2(0.f, 0.f);
          tp[j] = pv[j] = make_float2(0.f, 0.f);
          if (cheb == 2 && in) {
            tp[j] = reinterpret_cast<const float2*>(pd.Tp)[idx];   // may be Tout: no .nc load
            pv[j] = reinterpret_cast<const float2*>(pd.P)[idx];
          }
        }
      };
      load_items(0);
      const bool got = ptx::mbar_wait(&acc_full[acc], aph, &s_abort, wait_ns);
      // give up together: tcgen05.ld below is .aligned per warp and the four
      // epilogue warps meet at named barriers
      if (!ptx::epilogue_all(got)) {
        s_abort = 1;
        atomicOr(&g_tc_error, 4u);
        break;
      }
      ptx::tc_fence_after();
      const uint32_t taddr =
          tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * kAccStride);
      for (int c0 = 0; c0 < nbp8; c0 += kChunk) {
        // every lane loads (tcgen05.ld is warp-collective), whatever its row:
        // u = D[.][a] (times Re A), w = D[.][nb8 + a] (times Im A)
        float u[kChunk], w[kChunk];
        ptx::tmem_ld8_sync(taddr + (uint32_t)c0, u);
        ptx::tmem_ld8_sync(taddr + (uint32_t)(nbp8 + c0), w);
        if (ASPLIT) {      // + 2^-11 Alo X, kept on the hi rows
          float u2[kChunk], w2[kChunk];
          ptx::tmem_ld8_sync(taddr + (uint32_t)(2 * nbp8 + c0), u2);
          ptx::tmem_ld8_sync(taddr + (uint32_t)(3 * nbp8 + c0), w2);
          if (grp < 2) {
#pragma unroll
            for (int e = 0; e < kChunk; ++e) {
              u[e] = fmaf(kLoScale, u2[e], u[e]);
              w[e] = fmaf(kLoScale, w2[e], w[e]);
            }
          }
        }
        if (c0 + kChunk >= nbp8) {      // last chunk read: release the buffer
          ptx::tc_fence_before();
          __syncwarp();
          if (lane == 0) ptx::mbar_arrive(&acc_empty[acc]);
        }
        // contribution of this row to (Re Y, Im Y)[a][r]: an Xr row gives
        // (u, w), an Xi row (-w, u); lo rows scaled by 2^-11.  Exchange
        // layout [group][value][column e][row r]: consecutive lanes touch
        // consecutive words, free of bank conflicts both ways
        float* xe = ex + xbuf * kExFloats;
        if (live) {
          float* slot = xe + grp * 2 * kChunk * rb + r_row;
#pragma unroll
          for (int e = 0; e < kChunk; ++e) {
            slot[e * rb] = gs * (imag ? -w[e] : u[e]);
            slot[(kChunk + e) * rb] = gs * (imag ? u[e] : w[e]);
          }
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
#pragma unroll
        for (int j = 0; j < kMaxItems; ++j) {
          const int i = et + 128 * j;
          const int e = i / R, r = i - e * R;
          if (i >= nitem || c0 + e >= nb) continue;
          // the groups summed in order 0, 1, 2, 3
          const float* col = xe + e * rb + r;
          float re = col[0], im = col[kChunk * rb];
#pragma unroll
          for (int gg = 1; gg < kGroups; ++gg) {
            re += col[gg * 2 * kChunk * rb];
            im += col[(gg * 2 + 1) * kChunk * rb];
          }
          const float sc = sx * __ldg(&pd.sigma[r]);
          const int64_t idx = site0 + (int64_t)c0 * R + i;
          const float2 y = make_float2(fmaf(sc, re, dx * xv[j].x), fmaf(sc, im, dx * xv[j].y));
          if (cheb == 0) {
            Yp[idx] = y;
            continue;
          }
          const float ca = pd.ca, cb = pd.cb, cc = pd.cc;
          float2 tv = make_float2(ca * y.x + cb * xv[j].x, ca * y.y + cb * xv[j].y);
          float2 p;
          if (cheb == 1) {
            p = make_float2(pd.c0 * xv[j].x + cc * tv.x, pd.c0 * xv[j].y + cc * tv.y);
          } else {
            tv = make_float2(2.f * tv.x - tp[j].x, 2.f * tv.y - tp[j].y);
            p = make_float2(pv[j].x + cc * tv.x, pv[j].y + cc * tv.y);
          }
          reinterpret_cast<float2*>(pd.Tout)[idx] = tv;
          reinterpret_cast<float2*>(pd.P)[idx] = p;
          if (cm_dst) atomicMax(&s_cm[r], __float_as_uint(fmaxf(fabsf(tv.x), fabsf(tv.y))));
        }
        xbuf ^= 1;      // the next chunk writes the other buffer
        if (c0 + kChunk < nbp8) load_items(c0 + kChunk);
      }
      if (++acc == 2) { acc = 0; aph ^= 1u; }
    }
    post_maxima();
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem_base, kTmemCols);
  }
}

// Ring layout for a launch: one stage size for every problem, set by the
// largest request; a stage of problem i holds pps[i] coefficient tiles and,
// from xb_off[i] on, pps[i] input tiles.  After the size is fixed each
// problem's pps grows to fill the stage (at most 8 and its stencil size).
struct Ring {
  int nstages = 0;
  uint32_t stage_bytes = 0;
  size_t smem = 0;
};

int plan_ring(const Geom* g, int* pps, const int* npts, int n, size_t budget, int max_stages,
              Ring* out, uint32_t* xb_off) {
  size_t stage = 0, tail = 0;
  bool xs = false;
  for (int i = 0; i < n; ++i) {
    stage = std::max(stage, (size_t)pps[i] * (g[i].coef_bytes + g[i].xb_bytes));
    // the M = 128 operand read runs past an input tile of fewer than 128
    // rows (the coefficient tile has exactly the N = 2 nb8 rows read)
    const size_t row_bytes = (size_t)g[i].K * 2;
    tail = std::max(tail, (size_t)(kM - g[i].xrows) * row_bytes);
    xs = xs || g[i].xsplit;
  }
  tail += 1024;
  tail += 2 * (size_t)kExFloats * sizeof(float);
  (void)xs;
  if (budget < 1024 + tail + 2 * stage) return 0;
  int ns = (int)((budget - 1024 - tail) / stage);
  if (ns > max_stages) ns = max_stages;
  if (ns > 32) ns = 32;                 // barrier area: 2 * 32 + 4 words < 1024 bytes
  if (ns < 2) return 0;
  for (int i = 0; i < n && xb_off; ++i) {
    const size_t u = g[i].coef_bytes + g[i].xb_bytes;
    int fit = (int)(stage / u);
    if (fit > 8) fit = 8;
    if (fit > npts[i]) fit = npts[i];
    if (fit > pps[i]) pps[i] = fit;
    xb_off[i] = (uint32_t)pps[i] * g[i].coef_bytes;
  }
  out->nstages = ns;
  out->stage_bytes = (uint32_t)stage;
  out->smem = 1024 + (size_t)ns * stage + tail;
  return ns;
}

int default_pps(const Geom& g) {
  // points per stage: aim for >= 16 KB of coefficients per copy
  int pps = (int)((16384 + g.coef_bytes - 1) / g.coef_bytes);
  return pps > 8 ? 8 : (pps < 1 ? 1 : pps);
}

template <bool BF16, bool XS, bool AS>
int launch_tc(const Batch& bt, const Ring& ring, int64_t grid, cudaStream_t s) {
  auto kern = k_op_tc<BF16, XS, AS>;
  MRHS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)ring.smem));
  { kern<<<(unsigned)grid, kThreadsTc, ring.smem, s>>>(bt, ring.nstages, ring.stage_bytes); ::mrhs::count_launch(); }
  return MRHS_OK;
}

bool xsplit_of(int prec) { return prec == MRHS_PREC_FP16X || prec == MRHS_PREC_TC32; }

// Reserve one problem's packing workspace (column maxima and scales at a
// fixed offset, so the maxima stay zero between applications; tiles after)
// and fill its kernel and packing descriptors.
constexpr size_t kXpackHead = 1024;

int prepare(mrhs_op_s* op, int prec, bool dag, const void* X, void* Y, int nrhs, int pps_req,
            cudaStream_t s, ProbDesc* pd, PackProb* pk, Geom* gout) {
  const int i = image_index(prec);
  if (dag && op->herm) dag = false;      // H^dagger = H exactly: the forward image serves
  if (dag && !op->tc_dag[i].codes) {
    if (!op->a64) return fail(MRHS_ERR_UNSUPPORTED, "daggered low-precision image needs FP64 coefficients");
    MRHS_TRY(tc_build(op, prec, true, op->a64, s));
  }
  const TcImage& img = dag ? op->tc_dag[i] : op->tc[i];
  const bool xs = xsplit_of(prec);
  const Geom g = make_geom(op->nb, nrhs, xs, prec == MRHS_PREC_TC32);
  const size_t xb_bytes = (size_t)op->V * g.xb_bytes;
  const size_t before = op->ws_xpack.bytes;      // grows on every reallocation
  MRHS_TRY(op->ws_xpack.ensure(kXpackHead + xb_bytes));
  unsigned* colmax = (unsigned*)op->ws_xpack.ptr;
  float* sigma = (float*)(colmax + MRHS_MAX_RHS);
  uint8_t* xb = (uint8_t*)op->ws_xpack.ptr + kXpackHead;
  if (op->ws_xpack.bytes != before)
    MRHS_CUDA_TRY(cudaMemsetAsync(colmax, 0, sizeof(unsigned) * MRHS_MAX_RHS, s));
  pk->X = (const float2*)X;
  pk->colmax = colmax;
  pk->sigma = sigma;
  pk->xb = xb;
  pk->V = op->V;
  pk->g = g;
  pd->coef = (const uint8_t*)img.codes;
  pd->xb = xb;
  pd->scale = img.scale;
  pd->diag = img.diag;
  pd->sigma = sigma;
  pd->X = (const float*)X;
  pd->Y = (float*)Y;
  pd->V = op->V;
  pd->npts = op->npts;
  pd->nb = op->nb;
  pd->K = g.K;
  pd->n_mma = g.n_mma;
  pd->R = nrhs;
  pd->nbp8 = g.nbp8;
  pd->rb = g.rb;
  pd->pps = pps_req > 0 ? pps_req : default_pps(g);
  if (pd->pps > op->npts) pd->pps = op->npts;
  pd->coef1 = g.coef1;
  pd->coef_bytes = g.coef_bytes;
  pd->xb_bytes = g.xb_bytes;
  pd->sbo = g.sbo;
  pd->idesc = ptx::idesc_f16(kM, g.n_mma, prec == MRHS_PREC_BF16);
  // Hermitian pairing: exact Hermiticity checked at creation, tiles whose
  // row and column extents agree (nb a multiple of 16), one pair per stage
  const bool pair_here =
      op->herm_mode == 1 || (op->herm_mode == 2 && prec == MRHS_PREC_TC32);
  pd->herm = (!dag && pair_here && op->nb % 16 == 0 && op->herm_nf > 0) ? 1 : 0;
  pd->nf = op->herm_nf;
  for (int j = 0; j < op->herm_nf; ++j) pd->fpts[j] = op->herm_f[j];
  for (int mu = 0; mu < 4; ++mu) {     // visiting blocks: largest divisor of L <= 4
    int b = 1;
    for (int c = 4; c >= 1; --c)
      if (op->L[mu] % c == 0) { b = c; break; }
    pd->bl[mu] = b;
  }
  pd->idesc_t = ptx::idesc_f16(kM, op->nb, prec == MRHS_PREC_BF16) | (1u << 16);
  pd->idesc_tn = pd->idesc_t | (1u << 14);
  if (pd->herm) pd->pps = 2;           // a stage holds two tiles and two inputs
  pd->cheb = 0;
  pd->ca = pd->cb = pd->cc = pd->c0 = 0.f;
  pd->Tout = nullptr;
  pd->Tp = nullptr;
  pd->P = nullptr;
  pd->colmax_next = nullptr;
  for (int mu = 0; mu < 4; ++mu) pd->st.L[mu] = op->L[mu];
  pd->st.sign = dag ? -1 : 1;
  for (int p = 0; p < op->npts; ++p)
    for (int mu = 0; mu < 4; ++mu) pd->st.d[p][mu] = op->disp[p][mu];
  *gout = g;
  return MRHS_OK;
}

// The three packing launches for every problem of `pb`.
// colmax_ready: the previous launch (a fused Chebyshev step) already
// accumulated the column maxima of this input.
int pack_batch(const PackBatch& pb, int prec, cudaStream_t s, bool colmax_ready = false) {
  const int sms = num_sms();
  const dim3 g4((unsigned)(sms * 4), (unsigned)pb.n), g8((unsigned)(sms * 8), (unsigned)pb.n);
  if (!colmax_ready) { k_colmax<<<g4, 256, 0, s>>>(pb); ::mrhs::count_launch(); }
  { k_colscale<<<pb.n, 64, 0, s>>>(pb); ::mrhs::count_launch(); }
  if (prec == MRHS_PREC_BF16)
    { k_pack_xb<true, false><<<g8, 256, 0, s>>>(pb); ::mrhs::count_launch(); }
  else if (!xsplit_of(prec))
    { k_pack_xb<false, false><<<g8, 256, 0, s>>>(pb); ::mrhs::count_launch(); }
  else
    { k_pack_xb<false, true><<<g8, 256, 0, s>>>(pb); ::mrhs::count_launch(); }
  MRHS_CUDA_TRY(cudaGetLastError());
  return MRHS_OK;
}

int run_batch(Batch& bt, Geom* geoms, int prec, const TcTune& tune, bool tune_set, int timer_prec,
              mrhs_op_s* timer_op, cudaStream_t s) {
  // TC32 holds 512 TMEM columns (two buffers of four accumulators): one CTA
  // per SM, kept alone there by its shared-memory request
  const bool tc32 = prec == MRHS_PREC_TC32;
  int ctas = tc32 ? 1 : (tune_set ? tune.ctas_per_sm : 2);
  const int max_stages = tune_set ? tune.max_stages : 32;
  Ring ring;
  int pps[MRHS_MAX_BATCH], npts[MRHS_MAX_BATCH];
  uint32_t xb_off[MRHS_MAX_BATCH];
  for (int i = 0; i < bt.n; ++i) {
    pps[i] = bt.p[i].pps;
    npts[i] = bt.p[i].npts;
  }
  for (;;) {   // fall back to fewer points per stage, then one CTA per SM
    if (plan_ring(geoms, pps, npts, bt.n, kSmemBudget / (size_t)ctas, max_stages, &ring, xb_off) >= 2)
      break;
    bool shrunk = false;
    for (int i = 0; i < bt.n; ++i)       // a paired problem keeps its two tiles per stage
      if (pps[i] > 1 && !bt.p[i].herm) { pps[i] = (pps[i] + 1) / 2; shrunk = true; }
    if (!shrunk) {
      if (ctas == 1) return fail(MRHS_ERR_UNSUPPORTED, "tensor-core ring does not fit");
      ctas = 1;
      for (int i = 0; i < bt.n; ++i) pps[i] = bt.p[i].pps;
    }
  }
  for (int i = 0; i < bt.n; ++i) {
    if (bt.p[i].herm) {                // plan_ring may have grown pps to fill the stage
      pps[i] = 2;
      xb_off[i] = 2u * geoms[i].coef_bytes;
    }
    bt.p[i].pps = pps[i];
    bt.p[i].xb_off = xb_off[i];
  }
  if (tc32 && ring.smem < kSmemOneCta) ring.smem = kSmemOneCta;
  bt.total = 0;
  for (int i = 0; i < bt.n; ++i) {
    bt.p[i].item0 = bt.total;
    bt.total += bt.p[i].V;
  }
  const int64_t cap = (int64_t)num_sms() * ctas;
  const int64_t grid = bt.total < cap ? bt.total : cap;
  if (timer_op) timer_mark(timer_op, timer_prec, s);
  int st;
  if (prec == MRHS_PREC_BF16) st = launch_tc<true, false, false>(bt, ring, grid, s);
  else if (prec == MRHS_PREC_FP16) st = launch_tc<false, false, false>(bt, ring, grid, s);
  else if (prec == MRHS_PREC_FP16X) st = launch_tc<false, true, false>(bt, ring, grid, s);
  else st = launch_tc<false, true, true>(bt, ring, grid, s);
  if (timer_op) timer_mark(timer_op, timer_prec, s);
  MRHS_TRY(st);
  MRHS_CUDA_TRY(cudaGetLastError());
  return MRHS_OK;
}

}  // namespace

int tc_supported(const mrhs_op_s* op, int prec, int nrhs) {
  if (op->nb > 64 || nrhs > 64 || nrhs < 1) return 0;
  const bool xs = xsplit_of(prec);
  if (xs && nrhs > 32) return 0;      // four row groups of round8(R) <= 128 rows
  const Geom g = make_geom(op->nb, nrhs, xs, prec == MRHS_PREC_TC32);
  int one = 1;
  Ring r;
  return plan_ring(&g, &one, &one, 1, kSmemBudget, 32, &r, nullptr) > 0;
}

int tc_build(mrhs_op_s* op, int prec, bool dag, const double2* A, cudaStream_t s) {
  const int i = image_index(prec);
  if (i < 0) return fail(MRHS_ERR_UNSUPPORTED, "tensor-core precision");
  TcImage& img = dag ? op->tc_dag[i] : op->tc[i];
  if (img.codes) return MRHS_OK;
  const Geom g = make_geom(op->nb, 1, false, i == 2);
  if (!A) return fail(MRHS_ERR_INVALID_ARG, "no source coefficients for the packed image");
  img.bytes = (size_t)op->V * op->npts * g.coef_bytes;
  if (cudaMalloc(&img.codes, img.bytes) != cudaSuccess ||
      cudaMalloc(&img.scale, sizeof(float) * op->V) != cudaSuccess ||
      cudaMalloc(&img.diag, sizeof(float) * op->V) != cudaSuccess) {
    cudaGetLastError();
    return fail(MRHS_ERR_NO_MEMORY, "tensor-core coefficient image");
  }
  const unsigned grid = (unsigned)op->V;
  // a Hermitian operator's tiles serve two sites (pairing): one scale for all
  double* gscale = nullptr;
  unsigned long long* gmax = nullptr;
  if (op->pairable && !dag) {
    if (cudaMalloc(&gmax, sizeof(unsigned long long) + sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return fail(MRHS_ERR_NO_MEMORY, "coefficient scale");
    }
    gscale = (double*)(gmax + 1);
    MRHS_CUDA_TRY(cudaMemsetAsync(gmax, 0, sizeof(unsigned long long), s));
    { k_coef_gmax<<<grid, 256, 0, s>>>(A, op->V, op->npts, op->nb, gmax); ::mrhs::count_launch(); }
    { k_coef_gscale<<<1, 1, 0, s>>>(gmax, gscale); ::mrhs::count_launch(); }
  }
  if (i == 0)
    { k_pack_coef<true, false><<<grid, 256, 0, s>>>(A, (uint8_t*)img.codes, img.scale, img.diag,
                                                     op->nbr_bwd, op->V, op->npts, op->nb, g,
                                                     dag ? 1 : 0, gscale); ::mrhs::count_launch(); }
  else if (i == 1)
    { k_pack_coef<false, false><<<grid, 256, 0, s>>>(A, (uint8_t*)img.codes, img.scale, img.diag,
                                                      op->nbr_bwd, op->V, op->npts, op->nb, g,
                                                      dag ? 1 : 0, gscale); ::mrhs::count_launch(); }
  else
    { k_pack_coef<false, true><<<grid, 256, 0, s>>>(A, (uint8_t*)img.codes, img.scale, img.diag,
                                                     op->nbr_bwd, op->V, op->npts, op->nb, g,
                                                     dag ? 1 : 0, gscale); ::mrhs::count_launch(); }
  if (gmax) {
    MRHS_CUDA_TRY(cudaStreamSynchronize(s));
    cudaFree(gmax);
  }
  MRHS_CUDA_TRY(cudaGetLastError());
  return MRHS_OK;
}

int tc_apply(mrhs_op_s* op, int prec, bool dag, const void* X, void* Y, int nrhs,
             cudaStream_t s) {
  const int i = image_index(prec);
  if (i < 0) return fail(MRHS_ERR_UNSUPPORTED, "tensor-core precision");
  if (!tc_supported(op, prec, nrhs))
    return fail(MRHS_ERR_UNSUPPORTED,
                "tensor-core shape (nb <= 64; nrhs <= 64, or <= 32 for FP16X/TC32)");
  // launch shape: set on the operator, else tuned for this shape, else default
  TcTune tune = op->tc_tune;
  bool set = op->tc_set;
  if (!set) {
    const int32_t r = nrhs;
    set = tune_lookup(&op, &r, 1, prec, &tune);
  }
  Batch bt;
  bt.n = 1;
  bt.active = nullptr;
  PackBatch pb;
  pb.n = 1;
  pb.active = nullptr;
  Geom g;
  MRHS_TRY(prepare(op, prec, dag, X, Y, nrhs, set ? tune.pps : 0, s, &bt.p[0], &pb.p[0], &g));
  MRHS_TRY(pack_batch(pb, prec, s));
  return run_batch(bt, &g, prec, tune, set, prec, op, s);
}

// Many operators in one persistent launch (each with its own inputs).
int tc_apply_batch(mrhs_op_s* const* ops, int n, int prec, const void* const* X,
                   void* const* Y, const int32_t* nrhs, const int32_t* active, cudaStream_t s,
                   const TcTune* force, const ChebFuse* fuse) {
  if (n < 1 || n > MRHS_MAX_BATCH) return fail(MRHS_ERR_INVALID_ARG, "batch size 1..16");
  if (image_index(prec) < 0) return fail(MRHS_ERR_UNSUPPORTED, "tensor-core precision");
  TcTune tune = ops[0]->tc_tune;
  bool set = ops[0]->tc_set;
  if (force) {
    tune = *force;
    set = true;
  } else if (!set) {
    set = tune_lookup(ops, nrhs, n, prec, &tune);
  }
  Batch bt;
  bt.n = n;
  bt.active = active;
  PackBatch pb;
  pb.n = n;
  pb.active = active;
  Geom g[MRHS_MAX_BATCH];
  for (int i = 0; i < n; ++i) {
    if (!tc_supported(ops[i], prec, nrhs[i]))
      return fail(MRHS_ERR_UNSUPPORTED, "tensor-core shape of a batch member");
    MRHS_TRY(prepare(ops[i], prec, false, X[i], Y[i], nrhs[i], set ? tune.pps : 0, s, &bt.p[i],
                     &pb.p[i], &g[i]));
  }
  bool colmax_ready = fuse != nullptr;
  for (int i = 0; i < n && fuse; ++i) {
    const ChebFuse& f = fuse[i];
    ProbDesc& pd = bt.p[i];
    pd.cheb = f.mode;
    pd.ca = f.a;
    pd.cb = f.b;
    pd.cc = f.c;
    pd.c0 = f.c0;
    pd.Tout = (float*)f.Tout;
    pd.Tp = (const float*)f.Tp;
    pd.P = (float*)f.P;
    pd.colmax_next = f.colmax_next ? pb.p[i].colmax : nullptr;
    colmax_ready = colmax_ready && f.colmax_ready;
  }
  MRHS_TRY(pack_batch(pb, prec, s, colmax_ready));
  // a single problem keeps its operator's kernel timer
  return run_batch(bt, g, prec, tune, set, prec, n == 1 ? ops[0] : nullptr, s);
}

int tc_set_wait_limit(unsigned long long ns) {
  MRHS_CUDA_TRY(cudaMemcpyToSymbol(g_tc_wait_ns, &ns, sizeof(ns)));
  return MRHS_OK;
}

unsigned tc_read_and_clear_error() {
  unsigned v = 0, z = 0;
  cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(v));
  cudaMemcpyToSymbol(g_tc_error, &z, sizeof(z));
  return v;
}

}  // namespace mrhs
