/* Oracle coarse operator as plain C loops (FP64 complex), OpenMP over sites.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
 * baseline leg of the benchmark; never linked into the product library.
 *
 * Y(x) = sum_p A_p(x) X(x + delta_p)       (Sec. 2.6, "Applying the coarse
 * operator"), periodic lattice, site x = x0 + L0*(x1 + L1*(x2 + L2*x3)).
 * Layouts: A[x][p][a][b], X/Y[x][b][r], complex as (re, im) double pairs.
 *
 * oracle_op_apply_sites evaluates the rows of a list of sites only, with the
 * coefficients of those sites passed in (A_sites[s][p][a][b]) and the full
 * input vector X: this is how sampled outputs of very large lattices are
 * checked without holding every coefficient on the host.
 *
 * oracle_op_apply_herm_half applies a Hermitian stencil from its self block
 * and its positive-displacement blocks only:
 *   (H X)(x) = A_0(x) X(x) + sum_{delta_p > 0} [ A_p(x) X(x + delta_p)
 *              + A_p(x - delta_p)^dagger X(x - delta_p) ],
 * which follows from A_{-p}(x + delta_p) = A_p(x)^dagger.
 */
#include <complex.h>
#include <stdint.h>
#include <string.h>

static int64_t shift_site(const int32_t* L, int64_t x, const int8_t* d, int sign) {
  int64_t c[4];
  int64_t r = x;
  for (int mu = 0; mu < 4; ++mu) {
    c[mu] = r % L[mu];
    r /= L[mu];
  }
  int64_t y = 0;
  for (int mu = 3; mu >= 0; --mu) {
    int64_t v = (c[mu] + sign * (int64_t)d[mu]) % L[mu];
    if (v < 0) v += L[mu];
    y = y * L[mu] + v;
  }
  return y;
}

/* Y_rows[s] = sum_p A_sites[s][p] X(site_s + delta_p) */
void oracle_op_apply_sites(const double _Complex* A_sites, const double _Complex* X,
                           double _Complex* Y_rows, const int32_t* L, int32_t nb,
                           int32_t npts, const int8_t* disp, int32_t nrhs,
                           const int64_t* sites, int64_t nsites) {
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < nsites; ++s) {
    double _Complex* y = Y_rows + s * (int64_t)nb * nrhs;
    for (int64_t i = 0; i < (int64_t)nb * nrhs; ++i) y[i] = 0.0;
    for (int p = 0; p < npts; ++p) {
      int64_t n = shift_site(L, sites[s], disp + 4 * p, +1);
      const double _Complex* a = A_sites + ((s * npts + p) * (int64_t)nb) * nb;
      const double _Complex* xv = X + n * (int64_t)nb * nrhs;
      for (int i = 0; i < nb; ++i)
        for (int b = 0; b < nb; ++b) {
          double _Complex aib = a[i * nb + b];
          for (int r = 0; r < nrhs; ++r) y[i * nrhs + r] += aib * xv[b * nrhs + r];
        }
    }
  }
}

void oracle_op_apply(const double _Complex* A, const double _Complex* X, double _Complex* Y,
                     const int32_t* L, int32_t nb, int32_t npts, const int8_t* disp,
                     int32_t nrhs) {
  int64_t V = (int64_t)L[0] * L[1] * L[2] * L[3];
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < V; ++x) {
    double _Complex* y = Y + x * (int64_t)nb * nrhs;
    for (int64_t i = 0; i < (int64_t)nb * nrhs; ++i) y[i] = 0.0;
    for (int p = 0; p < npts; ++p) {
      int64_t n = shift_site(L, x, disp + 4 * p, +1);
      const double _Complex* a = A + ((x * npts + p) * (int64_t)nb) * nb;
      const double _Complex* xv = X + n * (int64_t)nb * nrhs;
      for (int i = 0; i < nb; ++i)
        for (int b = 0; b < nb; ++b) {
          double _Complex aib = a[i * nb + b];
          for (int r = 0; r < nrhs; ++r) y[i * nrhs + r] += aib * xv[b * nrhs + r];
        }
    }
  }
}

/* Ahalf[x][k][a][b]: k = 0 the self block, k = 1.. the blocks of the
 * positive displacements listed in pos_disp[k-1][4]. */
void oracle_op_apply_herm_half(const double _Complex* Ahalf, const double _Complex* X,
                               double _Complex* Y, const int32_t* L, int32_t nb,
                               int32_t npos, const int8_t* pos_disp, int32_t nrhs) {
  int64_t V = (int64_t)L[0] * L[1] * L[2] * L[3];
  int64_t blk = (int64_t)nb * nb;
  int32_t nk = npos + 1;
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < V; ++x) {
    double _Complex* y = Y + x * (int64_t)nb * nrhs;
    for (int64_t i = 0; i < (int64_t)nb * nrhs; ++i) y[i] = 0.0;
    /* self */
    {
      const double _Complex* a = Ahalf + (x * nk) * blk;
      const double _Complex* xv = X + x * (int64_t)nb * nrhs;
      for (int i = 0; i < nb; ++i)
        for (int b = 0; b < nb; ++b)
          for (int r = 0; r < nrhs; ++r) y[i * nrhs + r] += a[i * nb + b] * xv[b * nrhs + r];
    }
    for (int k = 1; k < nk; ++k) {
      const int8_t* d = pos_disp + 4 * (k - 1);
      int64_t fwd = shift_site(L, x, d, +1);
      int64_t bwd = shift_site(L, x, d, -1);
      const double _Complex* a = Ahalf + (x * nk + k) * blk;       /* A_p(x) */
      const double _Complex* ab = Ahalf + (bwd * nk + k) * blk;    /* A_p(x - delta) */
      const double _Complex* xf = X + fwd * (int64_t)nb * nrhs;
      const double _Complex* xb = X + bwd * (int64_t)nb * nrhs;
      for (int i = 0; i < nb; ++i)
        for (int b = 0; b < nb; ++b) {
          double _Complex af = a[i * nb + b];
          double _Complex ad = conj(ab[b * nb + i]);
          for (int r = 0; r < nrhs; ++r)
            y[i * nrhs + r] += af * xf[b * nrhs + r] + ad * xb[b * nrhs + r];
        }
    }
  }
}
