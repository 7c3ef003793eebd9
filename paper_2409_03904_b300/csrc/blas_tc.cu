// Block algebra of the mixed solve on the tensor cores (tcgen05), complex64
// blocks of at most 32 columns, N rows:
//   Gram          G = X^dagger Y                 (Fig. 2: D^dagger z, T^dagger t,
//                                                  t^dagger t; the ThinQR shape of
//                                                  Sec. 3.5 and Table 6)
//   block update  Out = beta Add + X M           (Fig. 2: X + D M C, q - z M,
//                                                  T S^-1, Q + D S^dagger)
//
// Precision.  Every FP32 value v is split exactly into three bf16 terms by
// truncation: h = v with its low 16 bits cleared, m the same of v - h, and
// l = v - h - m (8 + 8 + 8 significant bits, so l is exact in bf16).  Of the
// nine term products the six down to order 2^-16 (hh, hm, mh, mm, hl, lh) are
// accumulated, each product exact in FP32, into FP32 tensor memory; the
// dropped ones are below 2^-23 of |x||y|, the size of an FP32 rounding.  The
// Gram adds its FP32 accumulators every 512 rows into double-float sums
// (an FP32 pair updated by the error-free TwoSum, ~2^-48 relative; B300's
// FP64 adds would cost sixty times as much) and sums the CTAs' partials in
// FP64 in a fixed order, so it is bitwise reproducible.
//
// Real forms.  A complex64 row of r columns is 2r interleaved reals
// (k = 2c + part).  The Gram's real product P = Xre^T Yre gives
//   G[c][d] = (P[2c][2d] + P[2c+1][2d+1]) + i (P[2c][2d+1] - P[2c+1][2d]),
// and the update multiplies a real row by the 2rin x 2rout real form of M:
//   Mre[2c][2d] = Re M, Mre[2c+1][2d] = -Im M, Mre[2c][2d+1] = Im M,
//   Mre[2c+1][2d+1] = Re M.
//
// Operand layouts: canonical K-major, no swizzle (8-row x 16-byte core
// matrices, K groups 128 bytes apart, 8-row groups `sbo` apart), written by
// converter warps.
//
//   Gram: K = 16 rows of the vectors per MMA step.  The A operand (M = 128)
//   is a window of two 64-row term blocks of X stored in the order
//   [m, h, l, 0], B (N = 192 or 64) term blocks of Y in the order [m, h, l]:
//     [m; h] x [m; h; l]  (N = 192)  ->  mm, mh, ml | hm, hh, hl
//     [l; 0] x h          (N = 64)   ->  lh | 0
//   into one 128 x 192 accumulator D, so P[i][j] is the sum of D[i][j],
//   D[i][64+j], D[i][128+j] and the same three of row 64 + i (ml, below
//   2^-24, is kept as it comes).  Two MMAs per step: the issue of an MMA, not
//   its size, sets the pace at these widths.  When X and Y are the same
//   block, X's term blocks serve as B as well.
//
//   Update: M = 128 rows of X, K = 2 rin (in steps of 16), the small matrix's
//   terms stacked along N as [Mh; Mm; Ml] (Nn = round16(2 rout) rows each):
//     Xh x [Mh; Mm; Ml]  ->  D[:, 0:3Nn]  = hh | hm | hl
//     Xm x [Mh; Mm]      ->  D[:, 0:2Nn] += mh | mm
//     Xl x Mh            ->  D[:, 0:Nn]  += lh
//   and row n of the result is D[n][j] + D[n][Nn+j] + D[n][2Nn+j].
//
// Kernels are persistent, one CTA per SM, warp-specialised:
//   warp 0       bulk copies of raw row tiles into a ring
//   warp 1       allocates tensor memory, issues the MMAs (one thread)
//   warps 2-5    epilogue (tensor-memory lane quarters 2, 3, 0, 1); the
//                update has a second epilogue group in warps 6-9, the two
//                taking alternate tiles
//   the rest     converters: raw rows in shared memory -> bf16 term operands
//                (eight warps for the Gram, four for the update)
// Every mbarrier wait is bounded (1 s); on expiry the kernel records an error
// bit (mrhs_device_error), drains its own copies and MMAs, frees its tensor
// memory and returns.
#include "bf16x3.cuh"
#include "internal.cuh"
#include "tc_ptx.cuh"

namespace mrhs {

__device__ unsigned int g_btc_error = 0;
// limit of the epilogue's accumulator wait in ns (0: 1 s), debugging only
__device__ unsigned long long g_btc_wait_ns = 0;

namespace {

constexpr int kConvWarps = 8;
constexpr int kBtcThreads = (6 + kConvWarps) * 32;   // 448
constexpr uint32_t kErrProducer = 64u, kErrMma = 128u, kErrEpi = 256u, kErrConv = 512u;

// converters' shared-memory stores visible to the MMA (async proxy), then one
// arrival per warp
__device__ __forceinline__ void conv_publish(uint64_t* bar, int lane) {
  ptx::fence_proxy_async_smem();
  __syncwarp();
  if (lane == 0) ptx::mbar_arrive(bar);
}
__device__ __forceinline__ void bar_epi() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// The epilogue's bounded wait.  With the default limit (1 s) it is the
// suspending wait of the other roles; with a shorter debugging limit it polls
// the barrier without suspending (mbarrier.test_wait), because a suspended
// try_wait may sleep for longer than such a limit.
__device__ __forceinline__ bool wait_epi(uint64_t* bar, uint32_t parity, volatile int* abort,
                                         uint64_t limit_ns) {
  if (limit_ns >= 1000000000ull) return ptx::mbar_wait(bar, parity, abort, limit_ns);
  const uint64_t t0 = ptx::globaltimer();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(ptx::smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (*abort) return false;
    if (ptx::globaltimer() - t0 > limit_ns) return false;
  }
}

// ============================================================ Gram
constexpr int kGRaw = 2;                         // raw ring depth
constexpr int kGTerm = 8;                        // term ring depth (16-row MMA steps)
constexpr int kGFlush = 32;                      // MMA steps per FP64 flush (512 rows)
constexpr uint32_t kGRawBytes = 32 * 1024;       // 64 rows of X and Y, or 128 rows of X (herm)
constexpr uint32_t kGBlk = 64 * 16 * 2;          // one term block: 64 x 16 bf16 = 2 KB
constexpr uint32_t kGTermX = 4 * kGBlk;          // X: m, h, l, zero
constexpr uint32_t kGTermBytes = kGTermX + 3 * kGBlk;   // + Y: m, h, l
constexpr uint32_t kGOffRaw = 1024;
constexpr uint32_t kGOffTerm = kGOffRaw + kGRaw * kGRawBytes;
constexpr uint32_t kGOffEx = kGOffTerm + kGTerm * kGTermBytes;
constexpr uint32_t kGOffAcc = kGOffEx + 64 * 32 * 4;       // exchange: 32 columns x 64 rows
constexpr uint32_t kGSmem = kGOffAcc + 64 * 64 * 8;        // double-float sums [j][i]: hi, lo

// Partial Grams of contiguous row ranges: CTA b reduces rows
// [b per, min(N, (b + 1) per)) into part[b][rx][ry] (complex128).
// Requires rx, ry multiples of 4 in [4, 32], X and Y 16-byte aligned, per a
// multiple of 128; herm: Y is X.  A raw tile is 64 rows of X and Y (128 of X
// alone with herm), landed by one bulk copy per block.  Converter lanes are
// real columns, so the reads of a row are conflict-free.  Without herm warps
// 0-3 convert X and 4-7 Y, every step; with herm warps 0-3 convert the even
// steps of X and 4-7 the odd ones; either way a warp converts two of its
// steps per pass and publishes them after one proxy fence.
__global__ void __launch_bounds__(kBtcThreads, 1)
    k_gram_tc(const float2* __restrict__ X, const float2* __restrict__ Y,
              double2* __restrict__ part, int64_t N, int rx, int ry, int64_t per, int herm) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* raw_full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* raw_empty = raw_full + kGRaw;
  uint64_t* term_full = raw_empty + kGRaw;
  uint64_t* term_empty = term_full + kGTerm;
  uint64_t* acc_full = term_empty + kGTerm;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* mma_done = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
  uint8_t* raw = smem + kGOffRaw;
  uint8_t* term = smem + kGOffTerm;
  float* ex = reinterpret_cast<float*>(smem + kGOffEx);
  float* acc_hi = reinterpret_cast<float*>(smem + kGOffAcc);      // [j][i]
  float* acc_lo = acc_hi + 64 * 64;
  __shared__ volatile int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t b0 = (int64_t)blockIdx.x * per;
  int64_t b1 = b0 + per;
  if (b1 > N) b1 = N;
  const int trows = herm ? 128 : 64;             // rows per raw tile
  const int tsteps = trows / 16;
  const int ntile = b1 > b0 ? (int)((b1 - b0 + trows - 1) / trows) : 0;
  const int nstep = tsteps * ntile;
  const int nflush = (nstep + kGFlush - 1) / kGFlush;
  const int xr = 2 * rx, yr = 2 * ry;            // reals per row

  if (threadIdx.x == 0) {
    for (int s = 0; s < kGRaw; ++s) {
      ptx::mbar_init(&raw_full[s], 1);
      ptx::mbar_init(&raw_empty[s], kConvWarps);
    }
    for (int s = 0; s < kGTerm; ++s) {
      ptx::mbar_init(&term_full[s], herm ? kConvWarps / 2 : kConvWarps);
      ptx::mbar_init(&term_empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      ptx::mbar_init(&acc_full[i], 1);
      ptx::mbar_init(&acc_empty[i], 4);
    }
    ptx::mbar_init(mma_done, 1);
    ptx::fence_mbar_init();
    s_abort = 0;
  }
  // the zero block of every X term stage, and the double-float accumulators
  for (int i = threadIdx.x; i < kGTerm * (int)(kGBlk / 16); i += blockDim.x) {
    const int s = i / (kGBlk / 16), o = i % (kGBlk / 16);
    uint4* z = reinterpret_cast<uint4*>(term + s * kGTermBytes + 3 * kGBlk) + o;
    *z = make_uint4(0u, 0u, 0u, 0u);
  }
  for (int i = threadIdx.x; i < 2 * 64 * 64; i += blockDim.x) acc_hi[i] = 0.f;
  ptx::fence_proxy_async_smem();
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, 512);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- producer: raw rows of X (and Y) per tile
      const uint64_t pol = ptx::policy_evict_first();
      int issued = 0;
      bool ok = true;
      for (int i = 0; i < ntile && ok; ++i) {
        const int s = i % kGRaw;
        const uint32_t ph = (uint32_t)(i / kGRaw) & 1u;
        if (!ptx::mbar_wait(&raw_empty[s], ph ^ 1u, &s_abort)) { ok = false; break; }
        const int64_t n0 = b0 + (int64_t)i * trows;
        const int64_t rows = (b1 - n0) < trows ? (b1 - n0) : trows;
        const uint32_t xb = (uint32_t)(rows * rx * 8), yb = herm ? 0u : (uint32_t)(rows * ry * 8);
        uint8_t* dst = raw + (size_t)s * kGRawBytes;
        ptx::mbar_arrive_expect_tx(&raw_full[s], xb + yb);
        ptx::bulk_g2s(dst, X + n0 * rx, xb, &raw_full[s], pol);
        if (yb) ptx::bulk_g2s(dst + kGRawBytes / 2, Y + n0 * ry, yb, &raw_full[s], pol);
        ++issued;
      }
      if (!ok) {
        s_abort = 1;
        atomicOr(&g_btc_error, kErrProducer);
      }
      const int last = issued < kGRaw ? issued : kGRaw;
      for (int k = 0; k < last; ++k) {      // drain: every copy has landed
        const int n = issued - 1 - k;
        volatile int never = 0;
        ptx::mbar_wait(&raw_full[n % kGRaw], (uint32_t)(n / kGRaw) & 1u, &never);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      const uint32_t id192 = ptx::idesc_f16(128, 192, true), id64 = ptx::idesc_f16(128, 64, true);
      const uint32_t tb = ptx::smem_u32(term);
      int acc = 0, in_acc = 0;
      uint32_t aph = 0;
      bool ok = true;
      for (int g = 0; g < nstep && ok; ++g) {
        if (in_acc == 0) {
          if (!ptx::mbar_wait(&acc_empty[acc], aph ^ 1u, &s_abort)) { ok = false; break; }
          ptx::tc_fence_after();
        }
        const int ts = g % kGTerm;
        if (!ptx::mbar_wait(&term_full[ts], (uint32_t)(g / kGTerm) & 1u, &s_abort)) {
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        const uint32_t xa = tb + (uint32_t)ts * kGTermBytes;
        const uint32_t ya = herm ? xa : xa + kGTermX;
        const uint32_t d = tmem_base + (uint32_t)(acc * 256);
        ptx::mma_f16(d, ptx::smem_desc(xa, 128u, 256u), ptx::smem_desc(ya, 128u, 256u), id192,
                     in_acc > 0 ? 1u : 0u);                                  // [m;h] x [m;h;l]
        ptx::mma_f16(d, ptx::smem_desc(xa + 2 * kGBlk, 128u, 256u),
                     ptx::smem_desc(ya + kGBlk, 128u, 256u), id64, 1u);       // [l;0] x h
        ptx::mma_commit(&term_empty[ts]);
        if (++in_acc == kGFlush || g == nstep - 1) {
          ptx::mma_commit(&acc_full[acc]);
          in_acc = 0;
          if (++acc == 2) { acc = 0; aph ^= 1u; }
        }
      }
      if (!ok) {
        s_abort = 1;
        atomicOr(&g_btc_error, kErrMma);
      }
      ptx::mma_commit(mma_done);
      volatile int never = 0;
      ptx::mbar_wait(mma_done, 0, &never);
    }
  } else if (warp < 6) {
    // ---------------- epilogue: lane L of the accumulator = A row L
    const int q = warp & 3;
    const int L = 32 * q + lane;
    const unsigned long long lim = g_btc_wait_ns;
    const uint64_t wait_ns = lim ? lim : 1000000000ull;
    for (int f = 0; f < nflush; ++f) {
      const int buf = f & 1;
      const bool got = wait_epi(&acc_full[buf], (uint32_t)(f >> 1) & 1u, &s_abort, wait_ns);
      if (!ptx::epilogue_all(got)) {
        s_abort = 1;
        atomicOr(&g_btc_error, kErrEpi);
        break;
      }
      ptx::tc_fence_after();
      const uint32_t ta = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * 256);
      // rows 64 + i hand their sums to row i through shared memory, one
      // 32-column half at a time; row i adds them into its double-float
      // accumulators (hi + lo, the error of each FP32 add kept exactly by
      // TwoSum: ~2^-48 relative, at FP32 speed; layout [j][i])
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        float sv[32];
#pragma unroll
        for (int sub = 0; sub < 2; ++sub) {
          float a[16], b[16], c[16];
          ptx::tmem_ld16_sync(ta + (uint32_t)(32 * half + 16 * sub), a);
          ptx::tmem_ld16_sync(ta + (uint32_t)(64 + 32 * half + 16 * sub), b);
          ptx::tmem_ld16_sync(ta + (uint32_t)(128 + 32 * half + 16 * sub), c);
#pragma unroll
          for (int j = 0; j < 16; ++j) sv[16 * sub + j] = (a[j] + b[j]) + c[j];
        }
        if (half == 1) {        // the last tensor-memory read of this flush
          ptx::tc_fence_before();
          __syncwarp();
          if (lane == 0) ptx::mbar_arrive(&acc_empty[buf]);
        }
        if (L >= 64)
#pragma unroll
          for (int j = 0; j < 32; ++j) ex[j * 64 + (L - 64)] = sv[j];
        bar_epi();
        if (L < 64)
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int idx = (32 * half + j) * 64 + L;
            const float v = sv[j] + ex[j * 64 + L];
            const float a = acc_hi[idx];
            const float sum = a + v, bv = sum - a;
            acc_hi[idx] = sum;
            acc_lo[idx] += (a - (sum - bv)) + (v - bv);
          }
        bar_epi();
      }
    }
    bar_epi();
    const int et = (int)threadIdx.x - 64;
    const int ne = rx * ry;
    double2* out = part + (int64_t)blockIdx.x * ne;
    if (!s_abort)
      for (int e = et; e < ne; e += 128) {
        const int c = e / ry, dd = e - c * ry;
        auto P = [&](int ii, int jj) {
          return (double)acc_hi[jj * 64 + ii] + (double)acc_lo[jj * 64 + ii];
        };
        const double p00 = P(2 * c, 2 * dd), p11 = P(2 * c + 1, 2 * dd + 1);
        const double p01 = P(2 * c, 2 * dd + 1), p10 = P(2 * c + 1, 2 * dd);
        out[e] = make_double2(p00 + p11, p01 - p10);
      }
  } else {
    // ---------------- converters: lane = real column m (mod 32), one 8-row
    // half of a 16-row step per warp
    const int cw = warp - 6;
    const int S = herm ? 2 : 1, o = herm ? (cw >> 2) : 0;    // steps of a tile: o, o + S, ...
    const int op = herm ? 0 : (cw >> 2);
    const int sub = cw & 3;
    const int kh = sub >> 1, m = (sub & 1) * 32 + lane;
    const int width = op ? yr : xr;
    const uint32_t boff = (uint32_t)(m >> 3) * 256u + (uint32_t)kh * 128u + (uint32_t)(m & 7) * 16u;
    bool ok = true;
    for (int i = 0; i < ntile && ok; ++i) {
      const int rs = i % kGRaw;
      if (!ptx::mbar_wait(&raw_full[rs], (uint32_t)(i / kGRaw) & 1u, &s_abort)) { ok = false; break; }
      const int64_t n0 = b0 + (int64_t)i * trows;
      const int rows = (b1 - n0) < trows ? (int)(b1 - n0) : trows;
      const float* src = reinterpret_cast<const float*>(raw + (size_t)rs * kGRawBytes +
                                                        (op ? kGRawBytes / 2 : 0u));
      // this warp's four steps of the tile, two at a time: both steps'
      // loads and splits are independent, and one proxy fence serves both
#pragma unroll
      for (int pr = 0; pr < 2; ++pr) {
        const int ja = o + 2 * pr * S, jb = ja + S;
        const int ga = tsteps * i + ja, gb = tsteps * i + jb;
        const int tsa = ga % kGTerm, tsb = gb % kGTerm;
        if (!ptx::mbar_wait(&term_empty[tsa], ((uint32_t)(ga / kGTerm) & 1u) ^ 1u, &s_abort) ||
            !ptx::mbar_wait(&term_empty[tsb], ((uint32_t)(gb / kGTerm) & 1u) ^ 1u, &s_abort)) {
          ok = false;
          break;
        }
        float va[8], vb[8];
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const int ra = 16 * ja + 8 * kh + kk, rb = 16 * jb + 8 * kh + kk;
          va[kk] = (m < width && ra < rows) ? src[ra * width + m] : 0.f;
          vb[kk] = (m < width && rb < rows) ? src[rb * width + m] : 0.f;
        }
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const float* v = h2 ? vb : va;
          uint32_t hh[8], mm[8], ll[8];
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) split3(v[kk], hh[kk], mm[kk], ll[kk]);
          const uint32_t base = ptx::smem_u32(term + (size_t)(h2 ? tsb : tsa) * kGTermBytes +
                                              (op ? kGTermX : 0u)) + boff;
          // blocks m, h, l
          sts128(base, pack_bf16(mm[0], mm[1]), pack_bf16(mm[2], mm[3]),
                 pack_bf16(mm[4], mm[5]), pack_bf16(mm[6], mm[7]));
          sts128(base + kGBlk, pack_bf16(hh[0], hh[1]), pack_bf16(hh[2], hh[3]),
                 pack_bf16(hh[4], hh[5]), pack_bf16(hh[6], hh[7]));
          sts128(base + 2 * kGBlk, pack_bf16(ll[0], ll[1]), pack_bf16(ll[2], ll[3]),
                 pack_bf16(ll[4], ll[5]), pack_bf16(ll[6], ll[7]));
        }
        ptx::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          ptx::mbar_arrive(&term_full[tsa]);
          ptx::mbar_arrive(&term_full[tsb]);
        }
      }
      if (!ok) break;
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&raw_empty[rs]);
    }
    if (!ok) {
      s_abort = 1;
      atomicOr(&g_btc_error, kErrConv);
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem_base, 512);
  }
}

// ============================================================ block update
constexpr int kURows = 128;                      // rows per tile (M of the MMA)
constexpr int kURaw = 2;
constexpr int kUTerm = 2;
constexpr int kUConv = 4;                        // converter warps (10..13)
constexpr uint32_t kURawBytes = kURows * 32 * 8;           // 32 KB
constexpr uint32_t kUTermBlk = kURows * 64 * 2;            // one term, K <= 64: 16 KB
constexpr uint32_t kUTermBytes = 3 * kUTermBlk;            // 48 KB
constexpr uint32_t kUBBytes = 3 * 64 * 64 * 2;             // [Mh; Mm; Ml], 24 KB
constexpr int kUExStride = 36;                             // floats per exchange row (32 + 4)
constexpr uint32_t kUExBytes = kURows * kUExStride * 4;    // one group's exchange: 18 KB
constexpr uint32_t kUOffRaw = 1024;
constexpr uint32_t kUOffTerm = kUOffRaw + kURaw * kURawBytes;
constexpr uint32_t kUOffB = kUOffTerm + kUTerm * kUTermBytes;
constexpr uint32_t kUOffEx = kUOffB + kUBBytes;
constexpr uint32_t kUSmem = kUOffEx + 2 * kUExBytes;
static_assert(kUSmem + 1024 <= 227 * 1024, "block update: shared memory");
static_assert(kGSmem + 1024 <= 227 * 1024, "Gram: shared memory");

struct UpdArgs {
  const float2* X;     // [N][rin]
  const float2* Add;   // [N][rout] or null (beta = 0)
  float2* Out;         // [N][rout]; may be X (rin = rout) and/or Add
  const double2* M;    // mode 0: M [rin][rout]; mode 1: S [rout][rin], M[c][d] = conj(S[d][c])
  int64_t N;
  int rin, rout, mode;
  float beta;
};

// AND of pred over the 128 threads of epilogue group grp (named barrier 1 + grp)
__device__ __forceinline__ bool group_all(bool pred, int grp) {
  uint32_t r;
  if (grp == 0)
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred)
        : "memory");
  else
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 2, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred)
        : "memory");
  return r != 0;
}
__device__ __forceinline__ void bar_group(int grp) {
  if (grp == 0)
    asm volatile("bar.sync 1, 128;" ::: "memory");
  else
    asm volatile("bar.sync 2, 128;" ::: "memory");
}

// Out = beta Add + X M, 128-row tiles handed out round robin.  Requires rin,
// rout multiples of 4 in [4, 32] and 16-byte aligned vectors.  A tile's rows
// of X are in shared memory before any of its rows of Out are written, and
// its rows of Add are read by the thread that writes them, so Out may alias
// X and Add.  Two epilogue groups (warps 2-5 and 6-9) take alternate tiles,
// each with its own accumulator and exchange buffer, so the global reads of
// Add for one tile overlap the other group's work.
__global__ void __launch_bounds__(kBtcThreads, 1) k_update_tc(const __grid_constant__ UpdArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* raw_full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* raw_empty = raw_full + kURaw;
  uint64_t* term_full = raw_empty + kURaw;
  uint64_t* term_empty = term_full + kUTerm;
  uint64_t* acc_full = term_empty + kUTerm;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* mma_done = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
  uint8_t* raw = smem + kUOffRaw;
  uint8_t* term = smem + kUOffTerm;
  uint8_t* bmat = smem + kUOffB;
  __shared__ volatile int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rin = a.rin, rout = a.rout;
  const int kin = 2 * rin, kout = 2 * rout;            // reals per row
  const int K16 = (kin + 15) & ~15, Nn = (kout + 15) & ~15;
  const uint32_t sbo = (uint32_t)K16 * 16u;            // 8-row group stride (K16/8 x 128 B)
  const int64_t ntiles = (a.N + kURows - 1) / kURows;
  int mytiles = 0;
  if ((int64_t)blockIdx.x < ntiles) mytiles = (int)((ntiles - 1 - blockIdx.x) / gridDim.x) + 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kURaw; ++s) {
      ptx::mbar_init(&raw_full[s], 1);
      ptx::mbar_init(&raw_empty[s], kUConv);
    }
    for (int s = 0; s < kUTerm; ++s) {
      ptx::mbar_init(&term_full[s], kUConv);
      ptx::mbar_init(&term_empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      ptx::mbar_init(&acc_full[i], 1);
      ptx::mbar_init(&acc_empty[i], 4);
    }
    ptx::mbar_init(mma_done, 1);
    ptx::fence_mbar_init();
    s_abort = 0;
  }
  // the small matrix's terms, B[t Nn + j][k] = term t of Mre[k][j], zero
  // outside 2 rin x 2 rout
  for (int e = threadIdx.x; e < Nn * K16; e += blockDim.x) {
    const int j = e / K16, k = e - j * K16;
    float v = 0.f;
    if (j < kout && k < kin) {
      const int c = k >> 1, p = k & 1, d = j >> 1, qq = j & 1;
      const double2 z = a.mode ? a.M[d * rin + c] : a.M[c * rout + d];
      const double re = z.x, im = a.mode ? -z.y : z.y;
      // Mre[2c + p][2d + q]: (p, q) = (0,0) Re, (1,0) -Im, (0,1) Im, (1,1) Re
      v = (float)(p == qq ? re : (p ? -im : im));
    }
    uint32_t h, m, l;
    split3(v, h, m, l);
    const uint32_t terms[3] = {h, m, l};
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const int n = t * Nn + j;
      const uint32_t off = (uint32_t)(n >> 3) * sbo + (uint32_t)(k >> 3) * 128u +
                           (uint32_t)(n & 7) * 16u + (uint32_t)(k & 7) * 2u;
      *reinterpret_cast<uint16_t*>(bmat + off) = (uint16_t)(terms[t] >> 16);
    }
  }
  ptx::fence_proxy_async_smem();
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, 512);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- producer: raw rows of X per tile
      const uint64_t pol = ptx::policy_evict_first();
      int issued = 0;
      bool ok = true;
      for (int i = 0; i < mytiles && ok; ++i) {
        const int s = i % kURaw;
        if (!ptx::mbar_wait(&raw_empty[s], (((uint32_t)(i / kURaw)) & 1u) ^ 1u, &s_abort)) {
          ok = false;
          break;
        }
        const int64_t n0 = ((int64_t)blockIdx.x + (int64_t)i * gridDim.x) * kURows;
        const int64_t rows = (a.N - n0) < kURows ? (a.N - n0) : kURows;
        const uint32_t xb = (uint32_t)(rows * rin * 8);
        ptx::mbar_arrive_expect_tx(&raw_full[s], xb);
        ptx::bulk_g2s(raw + (size_t)s * kURawBytes, a.X + n0 * rin, xb, &raw_full[s], pol);
        ++issued;
      }
      if (!ok) {
        s_abort = 1;
        atomicOr(&g_btc_error, kErrProducer);
      }
      const int last = issued < kURaw ? issued : kURaw;
      for (int k = 0; k < last; ++k) {
        const int n = issued - 1 - k;
        volatile int never = 0;
        ptx::mbar_wait(&raw_full[n % kURaw], (uint32_t)(n / kURaw) & 1u, &never);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer: tile i into accumulator i & 1
      const uint32_t id3 = ptx::idesc_f16(128, 3 * Nn, true), id2 = ptx::idesc_f16(128, 2 * Nn, true),
                     id1 = ptx::idesc_f16(128, Nn, true);
      const uint32_t tb = ptx::smem_u32(term), bb = ptx::smem_u32(bmat);
      const int nk = K16 / 16;
      bool ok = true;
      for (int i = 0; i < mytiles && ok; ++i) {
        const int acc = i & 1;
        if (!ptx::mbar_wait(&acc_empty[acc], (((uint32_t)(i >> 1)) & 1u) ^ 1u, &s_abort)) {
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        const int ts = i % kUTerm;
        if (!ptx::mbar_wait(&term_full[ts], (uint32_t)(i / kUTerm) & 1u, &s_abort)) {
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        const uint32_t xa = tb + (uint32_t)ts * kUTermBytes;
        const uint32_t d = tmem_base + (uint32_t)(acc * 256);
        for (int kk = 0; kk < nk; ++kk) {
          const uint32_t ko = (uint32_t)kk * 256u;
          const uint64_t bdesc = ptx::smem_desc(bb + ko, 128u, sbo);
          ptx::mma_f16(d, ptx::smem_desc(xa + ko, 128u, sbo), bdesc, id3, kk > 0 ? 1u : 0u);
          ptx::mma_f16(d, ptx::smem_desc(xa + kUTermBlk + ko, 128u, sbo), bdesc, id2, 1u);
          ptx::mma_f16(d, ptx::smem_desc(xa + 2 * kUTermBlk + ko, 128u, sbo), bdesc, id1, 1u);
        }
        ptx::mma_commit(&term_empty[ts]);
        ptx::mma_commit(&acc_full[acc]);
      }
      if (!ok) {
        s_abort = 1;
        atomicOr(&g_btc_error, kErrMma);
      }
      ptx::mma_commit(mma_done);
      volatile int never = 0;
      ptx::mbar_wait(mma_done, 0, &never);
    }
  } else if (warp < 10) {
    // ---------------- epilogue group grp (warps 2-5: tiles 0, 2, ...; warps
    // 6-9: tiles 1, 3, ...): lane r of the accumulator = tile row r
    const int grp = (warp - 2) >> 2;
    const int q = warp & 3;
    const int r = 32 * q + lane;
    const int et = 32 * ((warp - 2) & 3) + lane;        // 0..127 within the group
    float* ex = reinterpret_cast<float*>(smem + kUOffEx + (size_t)grp * kUExBytes);
    const unsigned long long lim = g_btc_wait_ns;
    const uint64_t wait_ns = lim ? lim : 1000000000ull;
    const int v4row = kout / 4;                 // float4 per output row
    const int hw = kout < 32 ? kout : 32;       // reals per row in one exchange pass
    const int v4half = hw / 4;
    constexpr int kMaxV4 = kURows * 16 / 128;   // per thread and tile (rout <= 32)
    const float beta = a.beta;
    for (int i = grp; i < mytiles; i += 2) {
      const int acc = grp;
      const int64_t n0 = ((int64_t)blockIdx.x + (int64_t)i * gridDim.x) * kURows;
      const int rows = (a.N - n0) < kURows ? (int)(a.N - n0) : kURows;
      const int nv4 = rows * v4row;
      // this thread's outputs: pass h, item u -> row e / v4half, float4 e % v4half
      float4 add[kMaxV4];
      const float4* addp = reinterpret_cast<const float4*>(a.Add + n0 * rout);
#pragma unroll
      for (int u = 0; u < kMaxV4; ++u) {
        const int h = u / (kMaxV4 / 2), e = et + 128 * (u % (kMaxV4 / 2));
        const int rr = e / v4half, cc = e - rr * v4half + h * v4half;
        const bool in = rr < rows && cc < v4row;
        add[u] = (beta != 0.f && in) ? addp[rr * v4row + cc] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      const bool got = wait_epi(&acc_full[acc], (uint32_t)(i >> 1) & 1u, &s_abort, wait_ns);
      if (!group_all(got, grp)) {
        s_abort = 1;
        atomicOr(&g_btc_error, kErrEpi);
        break;
      }
      ptx::tc_fence_after();
      const uint32_t ta = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * 256);
      float4* outp = reinterpret_cast<float4*>(a.Out + n0 * rout);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h * 32 >= kout) break;
        // reals 32 h .. 32 h + 31 of every row into the exchange, then out
        for (int c0 = 32 * h; c0 < kout && c0 < 32 * h + 32; c0 += 8) {
          float u0[8], u1[8], u2[8];
          ptx::tmem_ld8_sync(ta + (uint32_t)c0, u0);
          ptx::tmem_ld8_sync(ta + (uint32_t)(Nn + c0), u1);
          ptx::tmem_ld8_sync(ta + (uint32_t)(2 * Nn + c0), u2);
          float* row = ex + r * kUExStride + (c0 - 32 * h);
#pragma unroll
          for (int e = 0; e < 8; e += 4)
            *reinterpret_cast<float4*>(row + e) =
                make_float4(u0[e] + u1[e] + u2[e], u0[e + 1] + u1[e + 1] + u2[e + 1],
                            u0[e + 2] + u1[e + 2] + u2[e + 2], u0[e + 3] + u1[e + 3] + u2[e + 3]);
        }
        if (32 * h + 32 >= kout) {      // the last tensor-memory read of this tile
          ptx::tc_fence_before();
          __syncwarp();
          if (lane == 0) ptx::mbar_arrive(&acc_empty[acc]);
        }
        bar_group(grp);
#pragma unroll
        for (int uu = 0; uu < kMaxV4 / 2; ++uu) {
          const int u = h * (kMaxV4 / 2) + uu;
          const int e = et + 128 * uu;
          const int rr = e / v4half, cl = e - rr * v4half, cc = cl + h * v4half;
          if (rr >= rows || cc >= v4row) continue;
          const float4 y = *reinterpret_cast<const float4*>(ex + rr * kUExStride + 4 * cl);
          outp[rr * v4row + cc] = make_float4(fmaf(beta, add[u].x, y.x), fmaf(beta, add[u].y, y.y),
                                              fmaf(beta, add[u].z, y.z), fmaf(beta, add[u].w, y.w));
        }
        bar_group(grp);
      }
    }
  } else {
    // ---------------- converters (warps 10-13): row r of a tile, its
    // 8-real (32-byte) pieces visited in the lane-rotated order
    // (q + lane) mod 8 and each read in two 16-byte halves, first the half
    // (lane >> 2) & 1, so that eight consecutive rows (256-byte stride) hit
    // distinct banks
    const int cw = warp - 10;
    const int r = 32 * cw + lane;
    const int npc = K16 / 8;                      // pieces per row (<= 8)
    const int h0 = (lane >> 2) & 1;
    bool ok = true;
    for (int i = 0; i < mytiles && ok; ++i) {
      const int rs = i % kURaw, ts = i % kUTerm;
      if (!ptx::mbar_wait(&raw_full[rs], (uint32_t)(i / kURaw) & 1u, &s_abort)) { ok = false; break; }
      if (!ptx::mbar_wait(&term_empty[ts], ((uint32_t)(i / kUTerm) & 1u) ^ 1u, &s_abort)) {
        ok = false;
        break;
      }
      const int64_t n0 = ((int64_t)blockIdx.x + (int64_t)i * gridDim.x) * kURows;
      const int rows = (a.N - n0) < kURows ? (int)(a.N - n0) : kURows;
      const uint8_t* src = raw + (size_t)rs * kURawBytes + (size_t)r * rin * 8;
      const uint32_t tbase = ptx::smem_u32(term + (size_t)ts * kUTermBytes) +
                             (uint32_t)(r >> 3) * sbo + (uint32_t)(r & 7) * 16u;
      // two pieces per pass (npc is even): both pieces' loads are issued
      // before either is split, so their latencies overlap
      for (int qq = 0; qq < npc; qq += 2) {
        float v[2][8];
        int pcs[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int pc = (qq + u + (lane & 7)) % npc;
          pcs[u] = pc;
          if (r < rows && 8 * pc < kin) {
            const float4 x0 = *reinterpret_cast<const float4*>(src + pc * 32 + h0 * 16);
            const float4 x1 = *reinterpret_cast<const float4*>(src + pc * 32 + (h0 ^ 1) * 16);
            const float4 lo = h0 ? x1 : x0, hi = h0 ? x0 : x1;
            v[u][0] = lo.x; v[u][1] = lo.y; v[u][2] = lo.z; v[u][3] = lo.w;
            v[u][4] = hi.x; v[u][5] = hi.y; v[u][6] = hi.z; v[u][7] = hi.w;
          } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) v[u][e] = 0.f;
          }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          uint32_t hh[8], mm[8], ll[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) split3(v[u][e], hh[e], mm[e], ll[e]);
          const uint32_t o = tbase + (uint32_t)pcs[u] * 128u;
          sts128(o, pack_bf16(hh[0], hh[1]), pack_bf16(hh[2], hh[3]), pack_bf16(hh[4], hh[5]),
                 pack_bf16(hh[6], hh[7]));
          sts128(o + kUTermBlk, pack_bf16(mm[0], mm[1]), pack_bf16(mm[2], mm[3]),
                 pack_bf16(mm[4], mm[5]), pack_bf16(mm[6], mm[7]));
          sts128(o + 2 * kUTermBlk, pack_bf16(ll[0], ll[1]), pack_bf16(ll[2], ll[3]),
                 pack_bf16(ll[4], ll[5]), pack_bf16(ll[6], ll[7]));
        }
      }
      conv_publish(&term_full[ts], lane);
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&raw_empty[rs]);
    }
    if (!ok) {
      s_abort = 1;
      atomicOr(&g_btc_error, kErrConv);
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem_base, 512);
  }
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
bool width_ok(int r) { return r >= 4 && r <= 32 && (r & 3) == 0; }

}  // namespace

// 0: SIMT kernels only; 1: the tensor-core kernels where they apply
int g_block_tc_mode = 1;

bool gram_tc_applies(const void* X, const void* Y, int64_t N, int rx, int ry, int dtype,
                     int64_t ldx) {
  return g_block_tc_mode == 1 && dtype == MRHS_C64 && N >= 1024 && width_ok(rx) &&
         width_ok(ry) && ldx == rx && aligned16(X) && aligned16(Y);
}

// Partial Grams into part (at most max_blocks blocks of rx x ry complex128);
// *nblk_out is the number written.
int gram_tc_partial(const void* X, const void* Y, double2* part, int64_t N, int rx, int ry,
                    int64_t max_blocks, int* nblk_out, cudaStream_t s) {
  int64_t nblk = num_sms();
  const int64_t by_rows = (N + 511) / 512;
  if (nblk > by_rows) nblk = by_rows;
  if (nblk > max_blocks) nblk = max_blocks;
  if (nblk < 1) return fail(MRHS_ERR_INVALID_ARG, "partial-Gram buffer too small");
  int64_t per = (N + nblk - 1) / nblk;
  per = (per + 127) / 128 * 128;
  nblk = (N + per - 1) / per;
  const int herm = (X == Y && rx == ry) ? 1 : 0;
  MRHS_CUDA_TRY(cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kGSmem));
  { k_gram_tc<<<(unsigned)nblk, kBtcThreads, kGSmem, s>>>((const float2*)X, (const float2*)Y, part,
                                                          N, rx, ry, per, herm); ::mrhs::count_launch(); }
  MRHS_CUDA_TRY(cudaGetLastError());
  *nblk_out = (int)nblk;
  return MRHS_OK;
}

bool update_tc_applies(const void* Out, const void* X, const void* Add, int64_t N, int rin,
                       int rout, int dtype, int64_t ldx) {
  return g_block_tc_mode == 1 && dtype == MRHS_C64 && N >= 1024 && width_ok(rin) &&
         width_ok(rout) && ldx == rin && aligned16(X) && aligned16(Out) &&
         (Add == nullptr || aligned16(Add));
}

// Out = beta Add + X M (mode 0: M [rin][rout]; mode 1: M = S^dagger, S
// [rout][rin]), complex64.
int update_tc(void* Out, const void* X, const void* Add, const double2* M, int mode, double beta,
              int64_t N, int rin, int rout, cudaStream_t s) {
  if (N == 0) return MRHS_OK;
  UpdArgs a;
  a.X = (const float2*)X;
  a.Add = beta != 0.0 ? (const float2*)Add : nullptr;
  a.Out = (float2*)Out;
  a.M = M;
  a.N = N;
  a.rin = rin;
  a.rout = rout;
  a.mode = mode;
  a.beta = (float)beta;
  if (a.beta != 0.f && !a.Add) return fail(MRHS_ERR_INVALID_ARG, "update: beta != 0 without Add");
  const int64_t ntiles = (N + kURows - 1) / kURows;
  int64_t grid = num_sms();
  if (grid > ntiles) grid = ntiles;
  MRHS_CUDA_TRY(cudaFuncSetAttribute(k_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kUSmem));
  { k_update_tc<<<(unsigned)grid, kBtcThreads, kUSmem, s>>>(a); ::mrhs::count_launch(); }
  MRHS_CUDA_TRY(cudaGetLastError());
  return MRHS_OK;
}

int btc_set_wait_limit(unsigned long long ns) {
  MRHS_CUDA_TRY(cudaMemcpyToSymbol(g_btc_wait_ns, &ns, sizeof(ns)));
  return MRHS_OK;
}

unsigned btc_read_and_clear_error() {
  unsigned v = 0, z = 0;
  cudaMemcpyFromSymbol(&v, g_btc_error, sizeof(v));
  cudaMemcpyToSymbol(g_btc_error, &z, sizeof(z));
  return v;
}

}  // namespace mrhs
