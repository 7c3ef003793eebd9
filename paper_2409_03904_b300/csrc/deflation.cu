// Deflated Chebyshev coarse solve Q^{Cheby+defl} (Sec. 2.3, "two step
// deflated/Chebyshev coarse solve").
//
// With the n_ev lowest eigenpairs (lambda_i, u_i) of the Hermitian coarse
// operator, every right-hand side b is split into its parts along and across
// the deflation space; the first is inverted exactly, the second goes through
// the Chebyshev approximation p of 1/x on [lo, hi]:
//     X = U Lambda^-1 (U^dagger B) + p(H) (B - U (U^dagger B)).
// The deflation is three passes of tall-skinny GEMMs over U ([N][n_ev], the
// layout of a block of n_ev right-hand sides), done with the Gram and block
// update kernels on column blocks of at most 64 eigenvectors (Sec. 3.5's
// multi-RHS deflation GEMM, n_ev x N x R): G = U^dagger B, then
// B_perp = B - U G and X = U (Lambda^-1 G).  The polynomial is the
// Chebyshev recurrence with the operator in the requested precision.
#include "internal.cuh"

namespace mrhs {
namespace {

constexpr int kThreads = 256;
constexpr int kColBlock = 64;    // eigenvectors per Gram / update pass

// Gs[i][r] = G[i][r] / lambda_i, Gn[i][r] = -G[i][r]
__global__ void k_defl_scale(const double2* __restrict__ G, const double* __restrict__ lam,
                             double2* Gs, double2* Gn, int n_ev, int R) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_ev * R) return;
  const double2 g = G[e];
  const double inv = 1.0 / lam[e / R];
  Gs[e] = make_double2(g.x * inv, g.y * inv);
  Gn[e] = make_double2(-g.x, -g.y);
}

template <typename C>
__global__ void k_add_into(C* X, const C* __restrict__ P, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const C a = X[i], b = P[i];
    C c;
    c.x = a.x + b.x;
    c.y = a.y + b.y;
    X[i] = c;
  }
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

int defl_cheby(mrhs_op_s* op, int prec, const void* U, const double* lam_host, int n_ev,
               double lo, double hi, int order, const void* B, void* X, int R, cudaStream_t s) {
  const bool wide = MRHS_PREC_IS_WIDE(prec);
  const int dtype = wide ? MRHS_C128 : MRHS_C64;
  const size_t es = wide ? sizeof(double2) : sizeof(float2);
  const int64_t N = op->V * op->nb;
  const int64_t n = N * R;
  const int g = num_sms() * 8;

  // workspace: lambda, G, Gs, Gn (n_ev x R complex128), Gram partials,
  // B_perp and p(H) B_perp (N x R)
  const size_t part_bytes = gram_workspace_bytes(N, kColBlock, R);
  const size_t small = align256(sizeof(double) * n_ev) + 3 * align256(sizeof(double2) * n_ev * R);
  const size_t need = small + align256(part_bytes) + 2 * align256(es * n);
  MRHS_TRY(op->ws_defl.ensure(need > 0 ? need : 256));
  char* base = (char*)op->ws_defl.ptr;
  double* lam = (double*)base;
  double2* G = (double2*)(base + align256(sizeof(double) * n_ev));
  double2* Gs = (double2*)((char*)G + align256(sizeof(double2) * n_ev * R));
  double2* Gn = (double2*)((char*)Gs + align256(sizeof(double2) * n_ev * R));
  double2* part = (double2*)((char*)Gn + align256(sizeof(double2) * n_ev * R));
  char* Bp = (char*)part + align256(part_bytes);
  char* Pp = Bp + align256(es * n);
  if (n_ev == 0) {      // nothing deflated: X = p(H) B (B copied, X may equal B)
    MRHS_CUDA_TRY(cudaMemcpyAsync(Bp, B, es * n, cudaMemcpyDeviceToDevice, s));
    return cheby(op, prec, lo, hi, order, Bp, X, R, s);
  }
  MRHS_CUDA_TRY(cudaMemcpyAsync(lam, lam_host, sizeof(double) * n_ev, cudaMemcpyHostToDevice, s));

  // G = U^dagger B, one Gram per column block of U
  const int64_t max_entries = (int64_t)(part_bytes / sizeof(double2));
  for (int i0 = 0; i0 < n_ev; i0 += kColBlock) {
    const int w = (n_ev - i0) < kColBlock ? (n_ev - i0) : kColBlock;
    MRHS_TRY(gram_ws_capped((const char*)U + es * i0, B, G + (int64_t)i0 * R, N, w, R, dtype,
                            part, max_entries, s, n_ev));
  }
  { k_defl_scale<<<(n_ev * R + kThreads - 1) / kThreads, kThreads, 0, s>>>(G, lam, Gs, Gn, n_ev, R); count_launch(); }
  // B_perp = B - U G and X = U Lambda^-1 G, block by block
  MRHS_CUDA_TRY(cudaMemcpyAsync(Bp, B, es * n, cudaMemcpyDeviceToDevice, s));
  for (int i0 = 0; i0 < n_ev; i0 += kColBlock) {
    const int w = (n_ev - i0) < kColBlock ? (n_ev - i0) : kColBlock;
    const void* Ub = (const char*)U + es * i0;
    MRHS_TRY(axpy(Bp, Ub, Gn + (int64_t)i0 * R, 1.0, N, w, R, dtype, s, n_ev));
    MRHS_TRY(axpy(X, Ub, Gs + (int64_t)i0 * R, i0 == 0 ? 0.0 : 1.0, N, w, R, dtype, s, n_ev));
  }
  // X += p(H) B_perp
  MRHS_TRY(cheby(op, prec, lo, hi, order, Bp, Pp, R, s));
  if (wide) { k_add_into<double2><<<g, kThreads, 0, s>>>((double2*)X, (const double2*)Pp, n); count_launch(); }
  else { k_add_into<float2><<<g, kThreads, 0, s>>>((float2*)X, (const float2*)Pp, n); count_launch(); }
  MRHS_CUDA_TRY(cudaGetLastError());
  return MRHS_OK;
}

}  // namespace mrhs
