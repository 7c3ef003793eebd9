// Coarsening a fine stencil operator onto a blocked basis (Sec. 2.6, "Coarse
// operator"), FP64.
//
// The fine operator is one of this library's operators (a stencil inside
// {-1,0,1}^4 on the fine lattice, nb_f components per site); coarse site b
// owns the fine sites y with floor(y / block) = b and the basis vectors
// basis[b][s][k], s = i * nb_f + a (i: position inside the block, first
// direction fastest).  The coarse matrix elements
//     A_p(b)[j][k] = <phi_j^b | M | phi_k^(b + delta_p)>
// come from the momentum-phase method: for every coarse stencil point p, M is
// applied once to the phased basis phi~^p_k = sum_b exp(i b.q^p) phi_k^b
// (q^p = 2 pi delta^p / L_c; all n_basis vectors as right-hand sides of one
// multi-RHS application), the result is block-projected onto the basis with
// the phase removed, T^p(b) = sum_p' alpha_{p,p'} A_p'(b) with
// alpha_{p,p'} = exp(i delta^p'.q^p), and A_p' = sum_p (alpha^-1)_{p',p} T^p.
// npts fine applications resolve all npts x n_basis^2 elements per block.
#include <complex>
#include <vector>

#include "internal.cuh"

namespace mrhs {
namespace {

constexpr int kThreads = 256;

struct Geo {
  int32_t Lf[4], Lc[4], blk[4];
  int32_t nbf, nbasis, bvol;
};

// fraction f with exp(i b.q) = exp(2 pi i f), f = sum_mu b_mu d_mu / Lc_mu
// (each term reduced mod Lc_mu first, so f stays small and exact)
__device__ __forceinline__ double phase_frac(const int* b, const int8_t* d, const Geo& g) {
  double f = 0.0;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    int t = (b[mu] * (int)d[mu]) % g.Lc[mu];
    if (t < 0) t += g.Lc[mu];
    f += (double)t / (double)g.Lc[mu];
  }
  return f;
}

// fine site y -> (coarse block coordinates, position inside the block)
__device__ __forceinline__ void split_site(int64_t y, const Geo& g, int* bc, int& inner,
                                           int64_t& bidx) {
  int ic[4];
  int64_t r = y;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const int c = (int)(r % g.Lf[mu]);
    r /= g.Lf[mu];
    bc[mu] = c / g.blk[mu];
    ic[mu] = c % g.blk[mu];
  }
  inner = ic[0] + g.blk[0] * (ic[1] + g.blk[1] * (ic[2] + g.blk[2] * ic[3]));
  bidx = bc[0] + (int64_t)g.Lc[0] * (bc[1] + (int64_t)g.Lc[1] * (bc[2] + (int64_t)g.Lc[2] * bc[3]));
}

// Phi[y][a][k] = exp(i b(y).q) basis[b(y)][i(y) nb_f + a][k]
__global__ void k_phase_scatter(double2* Phi, const double2* __restrict__ basis, Geo g,
                                int8_t d0, int8_t d1, int8_t d2, int8_t d3, int64_t n) {
  const int8_t d[4] = {d0, d1, d2, d3};
  const int vb = g.bvol * g.nbf;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e % g.nbasis);
    const int64_t t = e / g.nbasis;
    const int a = (int)(t % g.nbf);
    const int64_t y = t / g.nbf;
    int bc[4], inner;
    int64_t b;
    split_site(y, g, bc, inner, b);
    double sn, cs;
    sincospi(2.0 * phase_frac(bc, d, g), &sn, &cs);
    const double2 v = basis[(b * vb + (int64_t)inner * g.nbf + a) * g.nbasis + k];
    Phi[e] = make_double2(cs * v.x - sn * v.y, cs * v.y + sn * v.x);
  }
}

// Yb[b][i nb_f + a][k] = exp(-i b.q) Y[y(b, i)][a][k]
__global__ void k_gather_phase(double2* Yb, const double2* __restrict__ Y, Geo g, int8_t d0,
                               int8_t d1, int8_t d2, int8_t d3, int64_t n) {
  const int8_t d[4] = {d0, d1, d2, d3};
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e % g.nbasis);
    const int64_t t = e / g.nbasis;
    const int a = (int)(t % g.nbf);
    const int64_t y = t / g.nbf;
    int bc[4], inner;
    int64_t b;
    split_site(y, g, bc, inner, b);
    double sn, cs;
    sincospi(2.0 * phase_frac(bc, d, g), &sn, &cs);
    const double2 v = Y[e];
    const int vb = g.bvol * g.nbf;
    Yb[(b * vb + (int64_t)inner * g.nbf + a) * g.nbasis + k] =
        make_double2(cs * v.x + sn * v.y, cs * v.y - sn * v.x);
  }
}

// A[b][p'][j][k] = sum_p ainv[p'][p] T[p][b][j][k]
__global__ void k_unmix(double2* A, const double2* __restrict__ T, const double2* __restrict__ ainv,
                        int npts, int64_t Vc, int nb2) {
  const int64_t n = Vc * npts * nb2;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int jk = (int)(e % nb2);
    const int64_t t = e / nb2;
    const int q = (int)(t % npts);
    const int64_t b = t / npts;
    double2 acc = make_double2(0.0, 0.0);
    for (int p = 0; p < npts; ++p)
      acc = cfma(ainv[q * npts + p], T[((int64_t)p * Vc + b) * nb2 + jk], acc);
    A[e] = acc;
  }
}

// inverse of the phase matrix alpha[p][p'] = exp(i delta^p'.q^p) by
// Gauss-Jordan elimination with partial pivoting (host, npts <= 81)
int invert_alpha(const int8_t (*disp)[4], int npts, const int32_t* Lc,
                 std::vector<double2>& out) {
  using cd = std::complex<double>;
  const double pi = 3.14159265358979323846;
  std::vector<cd> a((size_t)npts * 2 * npts, cd(0.0, 0.0));
  for (int p = 0; p < npts; ++p) {
    for (int q = 0; q < npts; ++q) {
      double f = 0.0;
      for (int mu = 0; mu < 4; ++mu) f += (double)disp[p][mu] * disp[q][mu] / (double)Lc[mu];
      a[(size_t)p * 2 * npts + q] = std::polar(1.0, 2.0 * pi * f);
    }
    a[(size_t)p * 2 * npts + npts + p] = cd(1.0, 0.0);
  }
  const int w = 2 * npts;
  for (int c = 0; c < npts; ++c) {
    int piv = c;
    for (int r = c + 1; r < npts; ++r)
      if (std::abs(a[(size_t)r * w + c]) > std::abs(a[(size_t)piv * w + c])) piv = r;
    if (std::abs(a[(size_t)piv * w + c]) < 1e-10)
      return fail(MRHS_ERR_INVALID_ARG, "coarsening: phase matrix singular (coarse extents must be >= 3 "
                                        "and the stencil displacements distinct)");
    if (piv != c)
      for (int k = 0; k < w; ++k) std::swap(a[(size_t)piv * w + k], a[(size_t)c * w + k]);
    const cd inv = 1.0 / a[(size_t)c * w + c];
    for (int k = 0; k < w; ++k) a[(size_t)c * w + k] *= inv;
    for (int r = 0; r < npts; ++r) {
      if (r == c) continue;
      const cd f = a[(size_t)r * w + c];
      if (f == cd(0.0, 0.0)) continue;
      for (int k = 0; k < w; ++k) a[(size_t)r * w + k] -= f * a[(size_t)c * w + k];
    }
  }
  out.resize((size_t)npts * npts);
  for (int p = 0; p < npts; ++p)
    for (int q = 0; q < npts; ++q) {
      const cd v = a[(size_t)p * w + npts + q];
      out[(size_t)p * npts + q] = make_double2(v.real(), v.imag());
    }
  return MRHS_OK;
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

int coarsen(mrhs_op_s* op, const int32_t* block, const void* basis, int nbasis,
            const int8_t (*disp)[4], int npts, void* A_out, cudaStream_t s) {
  Geo g;
  int64_t Vc = 1;
  g.bvol = 1;
  for (int mu = 0; mu < 4; ++mu) {
    g.Lf[mu] = op->L[mu];
    g.blk[mu] = block[mu];
    g.Lc[mu] = op->L[mu] / block[mu];
    Vc *= g.Lc[mu];
    g.bvol *= block[mu];
  }
  g.nbf = op->nb;
  g.nbasis = nbasis;
  std::vector<double2> ainv;
  MRHS_TRY(invert_alpha(disp, npts, g.Lc, ainv));
  const int64_t nfine = op->V * op->nb * nbasis;
  const int nb2 = nbasis * nbasis;
  const size_t need = 3 * align256(sizeof(double2) * nfine) +
                      align256(sizeof(double2) * (size_t)npts * Vc * nb2) +
                      align256(sizeof(double2) * (size_t)npts * npts);
  MRHS_TRY(op->ws_coarsen.ensure(need));
  char* base = (char*)op->ws_coarsen.ptr;
  double2* Phi = (double2*)base;
  double2* Y = (double2*)(base + align256(sizeof(double2) * nfine));
  double2* Yb = (double2*)(base + 2 * align256(sizeof(double2) * nfine));
  double2* T = (double2*)(base + 3 * align256(sizeof(double2) * nfine));
  double2* dinv = (double2*)((char*)T + align256(sizeof(double2) * (size_t)npts * Vc * nb2));
  MRHS_CUDA_TRY(cudaMemcpyAsync(dinv, ainv.data(), sizeof(double2) * npts * npts,
                                cudaMemcpyHostToDevice, s));
  const int grid = num_sms() * 8;
  const int vb = g.bvol * g.nbf;
  for (int p = 0; p < npts; ++p) {
    const int8_t* d = disp[p];
    { k_phase_scatter<<<grid, kThreads, 0, s>>>(Phi, (const double2*)basis, g, d[0], d[1], d[2], d[3], nfine); count_launch(); }
    MRHS_TRY(op_apply(op, MRHS_PREC_FP64, false, Phi, Y, nbasis, s));
    { k_gather_phase<<<grid, kThreads, 0, s>>>(Yb, Y, g, d[0], d[1], d[2], d[3], nfine); count_launch(); }
    MRHS_TRY(blocking(true, basis, Yb, T + (size_t)p * Vc * nb2, Vc, vb, nbasis, nbasis, MRHS_C128, s));
  }
  { k_unmix<<<grid, kThreads, 0, s>>>((double2*)A_out, T, dinv, npts, Vc, nb2); count_launch(); }
  MRHS_CUDA_TRY(cudaGetLastError());
  return MRHS_OK;
}

}  // namespace mrhs
