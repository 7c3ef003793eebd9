/* mrhs.h -- C ABI of libmrhs, the multi-right-hand-side coarse-grid operator
 * and block conjugate gradient kernels of P. Boyle, "Multiple right hand side
 * multigrid for domain wall fermions with a multigrid preconditioned block
 * conjugate gradient algorithm" (arXiv:2409.03904), for NVIDIA B300 (sm_103a).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Lattice: four periodic dimensions L[0..3], V = L0*L1*L2*L3 sites, site
 *   index x = x0 + L0*(x1 + L1*(x2 + L2*x3)).
 * Stencil: npts displacements delta_p in {-1,0,1}^4 (disp[p][4], host
 *   memory), p = 0 must be the self term (0,0,0,0); at most 81 points
 *   (Sec. 2.6, "Coarse operator": the full 3^4 neighbourhood).
 * Coefficients: complex128 A[x][p][a][b], a, b < nb (row-major nb x nb
 *   block for every site and stencil point), as (re, im) double pairs.
 * Vectors: a block of nrhs coarse vectors is stored [x][b][r] (RHS index r
 *   fastest), i.e. an N x nrhs row-major complex matrix with N = V*nb; the
 *   element type is complex128 (MRHS_C128) or complex64 (MRHS_C64).
 * Memory: every vector, matrix and coefficient pointer is caller-owned
 *   DEVICE memory unless stated otherwise, 16-byte aligned; the library never
 *   frees it.  Host pointers are marked "host".
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Apply-type calls are asynchronous on that stream.
 * Errors: every call returns MRHS_OK (0) or a negative MRHS_ERR_* code and
 *   never aborts or traps; mrhs_last_error() returns a thread-local message
 *   for the last failure.  A CUDA failure inside a call returns MRHS_ERR_CUDA.
 */
#ifndef MRHS_H
#define MRHS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  MRHS_OK = 0,
  MRHS_ERR_INVALID_ARG = -1,   /* bad size, pointer, alignment or enum */
  MRHS_ERR_CUDA = -2,          /* a CUDA runtime call or launch failed */
  MRHS_ERR_NOT_CONVERGED = -3, /* maxiter reached; X and info still written */
  MRHS_ERR_BREAKDOWN = -4,     /* block Gram not positive (solve only) */
  MRHS_ERR_NONFINITE = -5,     /* NaN/Inf met in the solve */
  MRHS_ERR_UNSUPPORTED = -6,   /* precision not built into this operator */
  MRHS_ERR_NO_MEMORY = -7,     /* device allocation failed */
  MRHS_ERR_DEVICE = -8         /* a kernel's bounded wait expired, or a device
                                  self-check failed (mrhs_device_error) */
};

/* Operator precisions (coefficients and arithmetic of one application). */
enum {
  MRHS_PREC_FP64 = 0, /* complex128 coefficients, FP64 FMA; vectors complex128 */
  MRHS_PREC_FP32 = 1, /* complex64 coefficients, FP32 FMA; vectors complex64 */
  MRHS_PREC_BF16 = 2, /* bf16 codes x per-site power-of-two scale, tcgen05
                         tensor cores, FP32 accumulation; vectors complex64 */
  MRHS_PREC_FP16 = 3, /* as BF16 with fp16 codes */
  MRHS_PREC_FP16X = 4, /* fp16 coefficient codes, input in two fp16 terms
                          (hi + 2^-11 lo): linear in X to ~2^-22; nrhs <= 32 */
  MRHS_PREC_TC32 = 5, /* coefficients and input in two fp16 terms, lo x lo
                          dropped: FP32-class accuracy on the tensor cores,
                          8 bytes per complex coefficient; nrhs <= 32 */
  MRHS_PREC_DF32 = 6, /* the FP64 coefficients and complex128 vectors in
                          double-float arithmetic (FP32 pairs, error-free
                          products and sums) on the FP32 pipes: about 2^-44
                          relative; built whenever FP64 is */
  MRHS_PREC_OZ = 7    /* FP64 operator on the tensor cores by digit
                          slicing (Ozaki scheme): coefficients (per site) and
                          input (per column) as eight signed 6-bit fixed-point
                          digits held exactly in fp16 (2^-48 of the scale),
                          digit products with s + t <= 9 summed in FP32
                          tensor memory, recombined in int64 and FP64;
                          vectors complex128; a few 2^-48 of the site and
                          column scales per term (relative error ~1e-13, held
                          to the FP64 tolerance 1e-12 in the tests);
                          nrhs <= 32; 32 bytes per complex coefficient.
                          Needs no FP64 copy: block_cg_solve runs its FP64
                          operator applications with it (see fp64_prec) */
};
#define MRHS_NUM_PREC 8
#define MRHS_PREC_IS_TC(p) ((p) >= MRHS_PREC_BF16 && (p) <= MRHS_PREC_TC32)
/* precisions whose vectors are complex128 (the others: complex64) */
#define MRHS_PREC_IS_WIDE(p) \
  ((p) == MRHS_PREC_FP64 || (p) == MRHS_PREC_DF32 || (p) == MRHS_PREC_OZ)
#define MRHS_PREC_BIT(p) (1u << (p))

/* The four tensor-core forms share one design (op_tc.cu): per site, the
 * mean real self diagonal d_x in FP32, the rest as codes times a power-of-two
 * site scale, each input column times a power-of-two scale, FP32 accumulation
 * in tensor memory.  Two-term values are hi = fp16(u), lo = fp16((u-hi)2^11). */

/* Vector element types. */
enum { MRHS_C128 = 0, MRHS_C64 = 1 };

#define MRHS_MAX_RHS 64
#define MRHS_MAX_PTS 81
#define MRHS_MAX_CYCLES 16
#define MRHS_MAX_BATCH 16

typedef struct mrhs_op_s* mrhs_op;

/* Create a coarse operator (Sec. 2.6: the object holds the coarse matrix
 * coefficients itself).
 *   L      host int32[4], each >= 1
 *   nb     basis size per site, 1..64
 *   npts   stencil points, 1..81; disp host int8[npts][4] in {-1,0,1}, disp[0]=0
 *   A      device complex128 [V][npts][nb][nb]; read during the call only
 *   prec_mask  OR of MRHS_PREC_BIT(p): the precisions to build.  The operator
 *          owns a packed copy of A for each (complex128, complex64, or
 *          16-bit codes with a float scale and diagonal per site; FP16 and
 *          FP16X share one image; OZ keeps eight fp16 digit tiles per
 *          coefficient tile, 32 bytes per complex coefficient, with double
 *          scales and diagonals); A may be freed after the call returns.
 *          DF32 runs on the FP64 copy, so FP64 and DF32 come together.  OZ
 *          does not need the FP64 copy; its adjoint image is built from the
 *          FP64 copy on first use, so coarse_op_apply_dag with OZ needs FP64
 *          built as well (MRHS_ERR_UNSUPPORTED otherwise).
 * On success *out holds the handle.  Synchronises `stream`. */
int mrhs_op_create(mrhs_op* out, const int32_t L[4], int32_t nb, int32_t npts,
                   const int8_t* disp, const void* A, uint32_t prec_mask, void* stream);

/* One rank's part of a coarse operator on a 4D-decomposed lattice (Sec. 2.6,
 * "Applying the coarse operator": the input vector lives on the padded local
 * volume that includes the ghost zones, the result on the owned local volume
 * only, the coefficients stay local).
 *   L      host int32[4]: the local (owned) extents; V = prod(L) output sites
 *   halo   host int32[4], each 0 or 1: a ghost layer of depth 1 on both sides
 *          of dimension mu.  Input vectors are [Vin][nb][nrhs] on the padded
 *          lattice Lin = L + 2 halo (site index over Lin, first dimension
 *          fastest); owned site x with coordinates c reads its neighbour
 *          c + halo + delta_p of the input without wrapping in a padded
 *          dimension and with periodic wrap (on L) in the others.  Every
 *          input site an application reads must be filled by the caller
 *          (mrhs_gather_rows / mrhs_scatter_rows and a message exchange).
 *   A      device complex128 [V][npts][nb][nb]: the owned sites' coefficients
 *   prec_mask  FP64, FP32, DF32 and OZ only (MRHS_ERR_UNSUPPORTED otherwise)
 * Only coarse_op_apply takes such an operator; the adjoint, the solvers and
 * the other operator calls return MRHS_ERR_UNSUPPORTED (they need the whole
 * periodic lattice; the decomposed solve is driven from the host, see
 * domain.py).  halo = {0,0,0,0} gives the same operator as mrhs_op_create.
 * Synchronises `stream`. */
int mrhs_op_create_halo(mrhs_op* out, const int32_t L[4], const int32_t halo[4], int32_t nb,
                        int32_t npts, const int8_t* disp, const void* A, uint32_t prec_mask,
                        void* stream);

/* Row copies between a site-indexed array and a contiguous buffer, for the
 * ghost-zone exchange of Sec. 2.6 (faces are gathered into message buffers,
 * received messages scattered into the ghost layers, one dimension after the
 * other so that corner sites travel through the earlier dimensions' layers):
 *   mrhs_gather_rows:  dst[i] = src[idx[i]],   i < n  (src has src_rows rows)
 *   mrhs_scatter_rows: dst[idx[i]] = src[i],   i < n  (dst has dst_rows rows)
 * A row is row_bytes bytes (a positive multiple of 16; for a vector block,
 * nb * nrhs * element size).  src, dst: device, 16-byte aligned; idx: device
 * int64[n].  An index outside [0, rows) is skipped.  Indices of a scatter
 * must be distinct.  Asynchronous on `stream`. */
int mrhs_gather_rows(const void* src, int64_t src_rows, const int64_t* idx, int64_t n, void* dst,
                     int64_t row_bytes, void* stream);
int mrhs_scatter_rows(const void* src, int64_t n, const int64_t* idx, void* dst,
                      int64_t dst_rows, int64_t row_bytes, void* stream);

/* Release the operator and its device copies (after its last use is done). */
int mrhs_op_destroy(mrhs_op op);

/* Y = H X,  Y(x) = sum_p A_p(x) X(x + delta_p)   (Sec. 2.6, "Applying the
 * coarse operator", the per-stencil-point batched GEMM summed over p).
 *   prec   MRHS_PREC_*; must be in the operator's prec_mask
 *   X, Y   device [V][nb][nrhs]: complex128 for FP64, DF32 and OZ (see
 *          MRHS_PREC_IS_WIDE), complex64 otherwise;
 *          X and Y must not overlap
 *   nrhs   1..MRHS_MAX_RHS */
int coarse_op_apply(mrhs_op op, int32_t prec, const void* X, void* Y, int32_t nrhs,
                    void* stream);

/* Y = H^dagger X,  Y(x) = sum_p A_p(x - delta_p)^dagger X(x - delta_p): the
 * adjoint of the operator above (the reversed, daggered stencil).  Same
 * arguments.  For the tensor-core precisions (BF16 ... TC32, OZ) the first
 * call builds a packed image of the daggered coefficients inside the
 * operator. */
int coarse_op_apply_dag(mrhs_op op, int32_t prec, const void* X, void* Y, int32_t nrhs,
                        void* stream);

/* GA_p(x) = alpha * sum_r G(x)[a][r] conj(X(x + delta_p)[b][r]): the
 * coefficient-shaped outer product that gives the adjoints of the operator
 * (grad A = grad Y X^dagger on the stencil, alpha = 1) and of the solve
 * (grad A = -grad B X^dagger, alpha = -1), from dY = dA X + A dX with
 * Y(x) = sum_p A_p(x) X(x + delta_p) (Sec. 2.6).
 *   G, X   device [V][nb][nrhs], both complex128 or both complex64 (dtype)
 *   GA     device complex128 [V][npts][nb][nb] (written), FP64 accumulation
 * Asynchronous. */
int coarse_op_outer(mrhs_op op, const void* G, const void* X, void* GA, double alpha,
                    int32_t nrhs, int32_t dtype, void* stream);

/* G = X^dagger Y, the nrhs_x x nrhs_y block inner product of block CG
 * (Fig. 2: D^dagger Z, T^dagger t, ...; Sec. 3.5 and Table 6, the "ThinQR" Gram).
 *   X [N][rx], Y [N][ry] of element type dtype (MRHS_C128 or MRHS_C64)
 *   G device complex128 [rx][ry] row-major (written, not accumulated)
 *   N >= 0 rows, 1 <= rx, ry <= MRHS_MAX_RHS
 * Products are formed in the vectors' precision and summed in FP64 over a
 * fixed reduction tree, so the result is bitwise reproducible.  Complex64
 * blocks of 4..32 columns (multiples of 4; X rows contiguous, 16-byte
 * aligned, N >= 1024) run on the tensor cores (mrhs_block_tc): each FP32
 * value split exactly into three bf16 terms, the six products down to order
 * 2^-16 summed in FP32 over at most 512 rows, then in FP64.  Uses a
 * library-owned device workspace. */
int block_inner(const void* X, const void* Y, void* G, int64_t N, int32_t rx, int32_t ry,
                int32_t dtype, void* stream);

/* Same product as block_inner, for callers that may not allocate device
 * memory (the paper has no counterpart: this is a deployment variant).
 * block_inner grows a library-owned cudaMalloc workspace; this call instead
 * keeps its partial Grams in a fixed 2 MiB array compiled into the library
 * (held by every GPU that loads it until exit) and allocates nothing.
 *   Arguments as block_inner; rx, ry <= 64 (larger is rejected with
 *   MRHS_ERR_INVALID_ARG); the number of row blocks is capped so the partials
 *   fit, so the summation order (not the result beyond rounding) may differ
 *   from block_inner's.
 * The first call on a device looks up the array's device address with that
 * device current (cudaGetSymbolAddress); under CUDA's lazy module loading
 * (the default) that lookup is also what loads the library's device code on
 * the device and creates the array, so the first call may take device memory
 * (and fails with MRHS_ERR_CUDA if none is left); later calls take none.
 * Make that first call at set-up (N = 0 is enough), before any stream
 * capture.  The address is cached per device for the life of the process:
 * do not use the library across a cudaDeviceReset.  All calls on a device
 * share the array: calls that overlap on the GPU race and give wrong
 * results.  Each call writes every partial it reads, so nothing carries over
 * between calls. */
int block_inner_noalloc(const void* X, const void* Y, void* G, int64_t N, int32_t rx, int32_t ry,
                        int32_t dtype, void* stream);

/* Column-wise algebra for one Krylov process per right-hand side, run in
 * lockstep over the columns of an N x r block (the flexible ADEF2 CG of
 * Fig. 1 and its fixed-iteration CG smoother, which Sec. 2 runs as distinct
 * processes per right-hand side).  Scalars live on the device as complex128
 * [r] arrays.
 *   mrhs_col_dot:    out[j] = sum_n conj(X[n][j]) Y[n][j], FP64 sums in a
 *                    fixed order (bitwise reproducible); X, Y of dtype;
 *                    uses a library-owned workspace per (device, stream)
 *   mrhs_col_ratio:  out[j] = scale * num[j] / den[j]; 0 where den[j] = 0 or
 *                    active[j] = 0 (active: device int32[r], or NULL = all)
 *   mrhs_col_update: Y[n][j] = beta Y[n][j] + coef[j] X[n][j] (Y may be X)
 * 1 <= r <= MRHS_MAX_RHS; N >= 0.  Asynchronous on `stream`. */
int mrhs_col_dot(const void* X, const void* Y, void* out, int64_t N, int32_t r, int32_t dtype,
                 void* stream);
int mrhs_col_ratio(const void* num, const void* den, void* out, const int32_t* active, int32_t r,
                   double scale, void* stream);
int mrhs_col_update(void* Y, const void* X, const void* coef, double beta, int64_t N, int32_t r,
                    int32_t dtype, void* stream);

/* Y = beta*Y + X M  (Fig. 2 block updates X + D M, Q - Z M, D S^dagger, ...)
 *   X [N][rin], Y [N][rout] of element type dtype; Y may alias X when
 *   rin == rout (the update is done row tile by row tile)
 *   M device complex128 [rin][rout] row-major; beta real
 * For MRHS_C64 the arithmetic is FP32 with M rounded to complex64: on the
 * tensor cores (mrhs_block_tc) for 4..32 columns (multiples of 4), 16-byte
 * aligned blocks and N >= 1024, from exact three-term bf16 splits of X and M
 * (six products, FP32 accumulation over the 2 rin reals of a row). */
int block_axpy(void* Y, const void* X, const void* M, double beta, int64_t N, int32_t rin,
               int32_t rout, int32_t dtype, void* stream);

/* Factor a Hermitian block Gram G = T^dagger T (r x r, device complex128) as
 * T = Q S (Fig. 2: "Q_{k+1} S_{k+1} = Q_k - Z_k M_k", C_0 from R_0):
 *   S  device complex128 [r][r]: upper triangular with a positive real
 *      diagonal (S^dagger S = G) when every pivot exceeds tau * max_i G_ii;
 *      otherwise the diagonally pivoted factor stopped at rank k, rows k..r-1
 *      zero (breakdown-free block CG, dropping numerically null directions)
 *   W  device complex128 [r][r]: T W = Q (W = S^-1 at full rank; columns
 *      k..r-1 zero otherwise)
 *   rank  device int32[1]: k
 * G is Hermitian-symmetrised first.  One CTA, FP64.  Asynchronous. */
int herm_factor(const void* G, void* S, void* W, int32_t* rank, int32_t r, double tau,
                void* stream);

/* P = p(H) X with p the degree-`order` Chebyshev interpolant of 1/x on
 * [lo, hi] (Sec. 2.3: "a Chebyshev approximation to 1/x ... coefficients
 * at the Chebyshev interpolation points"), applied by the three-term
 * recurrence on t(H) = (2H - (hi + lo))/(hi - lo) with the operator in
 * precision `prec`.  X, P complex64 (FP32/BF16/FP16) or complex128 (FP64),
 * [V][nb][nrhs]; uses operator-owned workspace; asynchronous.  0 < lo < hi. */
int cheby_apply(mrhs_op op, int32_t prec, double lo, double hi, int32_t order, const void* X,
                void* P, int32_t nrhs, void* stream);

/* Block project and promote between fine and coarse degrees of freedom
 * (Sec. 2.5.1, "Transfer between grids"): one GEMM per coarse site x,
 *   block_project:  C(x) = B(x)^dagger F(x)   (n_basis x nrhs)
 *   block_promote:  F(x) = B(x) C(x)          (v_block x nrhs)
 * basis: device [n_blocks][v_block][n_basis]; F: device
 * [n_blocks][v_block][nrhs]; C: device [n_blocks][n_basis][nrhs] (the coarse
 * vector layout [V][nb][nrhs] with V = n_blocks, nb = n_basis).  dtype
 * MRHS_C128 (FP64 arithmetic) or MRHS_C64 (FP32) for all three arrays.
 * Complex64 with v_block a multiple of 64, n_basis a multiple of 8 up to 64,
 * nrhs a multiple of 4 up to 32 and 16-byte aligned arrays runs on the
 * tensor cores (mrhs_block_tc): exact three-term bf16 splits, six products
 * summed in FP32.
 * 1 <= v_block, 1 <= n_basis <= 256, 1 <= nrhs <= 64 (project also needs
 * nrhs <= 16 * (256 / n_basis)); n_blocks = 0 does nothing.  The output
 * must not overlap the inputs.  Asynchronous on `stream`. */
int block_project(const void* basis, const void* F, void* C, int64_t n_blocks, int32_t v_block,
                  int32_t n_basis, int32_t nrhs, int32_t dtype, void* stream);
int block_promote(const void* basis, const void* C, void* F, int64_t n_blocks, int32_t v_block,
                  int32_t n_basis, int32_t nrhs, int32_t dtype, void* stream);

/* Coarse operator of a fine one on a blocked basis (Sec. 2.6, "Coarse
 * operator"): A_p(b)[j][k] = <phi_j^b | M | phi_k^(b + delta_p)> for the npts
 * coarse displacements disp (host int8 [npts][4] in {-1,0,1}, distinct; they
 * must cover every coarse coupling of M, which holds for the full 81-point
 * set when M's own stencil lies inside {-1,0,1}^4).  fine: an operator with
 * FP64 built (lattice L_f, nb_f components); block[4] divides L_f, and every
 * coarse extent L_f / block is >= 3.  basis: device complex128
 * [V_c][v_block][n_basis], v_block = prod(block) * nb_f, row s = i * nb_f + a
 * for fine component a of the site at position i inside the block (first
 * direction fastest); 1 <= n_basis <= min(64, v_block).  A: device complex128
 * [V_c][npts][n_basis][n_basis], the layout mrhs_op_create takes.  Method
 * (momentum phases): one multi-RHS FP64 application of M per displacement to
 * the phased basis, block projections, and the inverse of the npts x npts
 * phase matrix.  Uses workspace of `fine`; asynchronous on `stream`. */
int coarsen_op(mrhs_op fine, const int32_t block[4], const void* basis, int32_t nbasis,
               const int8_t* disp, int32_t npts, void* A, void* stream);

/* Deflated Chebyshev coarse solve Q^{Cheby+defl} (Sec. 2.3, the "two step
 * deflated/Chebyshev coarse solve"):
 *   X = U Lambda^-1 U^dagger B + p(H) (B - U U^dagger B),
 * the exact inverse on the span of n_ev eigenvectors u_i (eigenvalues
 * lambda_i) of the Hermitian operator plus the degree-`order` Chebyshev
 * approximation p of 1/x on [lo, hi] (as cheby_apply) on the rest.
 * U: device, [V][nb][n_ev] (column i = u_i, the layout of a block of n_ev
 * right-hand sides), orthonormal columns expected (not checked); lambda:
 * host, n_ev positive values; B, X: device [V][nb][nrhs].  Element type of
 * U, B and X: complex128 for FP64/DF32, complex64 for the other precisions
 * (the deflation GEMMs and the recurrence run in it; the n_ev x nrhs
 * coefficients are summed in FP64).  n_ev = 0 reduces to cheby_apply; U may
 * then be NULL.  X may equal B; U must not overlap either.  Uses
 * operator-owned workspace (calls on one operator must not overlap on the
 * GPU); asynchronous on `stream` apart from the copy of lambda. */
int coarse_solve_defl_cheby(mrhs_op op, int32_t prec, const void* U, const double* lambda,
                            int32_t n_ev, double lo, double hi, int32_t order, const void* B,
                            void* X, int32_t nrhs, void* stream);

/* Largest-eigenvalue estimate of a Hermitian positive operator by the power
 * method (Sec. 2.3 takes the upper end of the Chebyshev interval from a
 * few power-method steps): Rayleigh quotient after
 * `iters` applications in precision `prec` to one deterministic start vector.
 * The estimate lies below the true maximum; it is cached on the operator and
 * block_cg_solve uses 1.08 x the cached value when cheb_hi <= 0.  A
 * non-finite estimate (NaN or Inf coefficients) returns MRHS_ERR_NONFINITE
 * and caches nothing.  Uses operator-owned workspace; synchronises
 * `stream`. */
int mrhs_op_lambda_max(mrhs_op op, int32_t prec, int32_t iters, double* lam, void* stream);

/* Solver parameters (block_cg_solve). */
typedef struct {
  double tol;           /* per-RHS relative true residual |b_r - H x_r| / |b_r| */
  int32_t maxiter;      /* cap on Krylov iterations (all cycles together) */
  int32_t mode;         /* MRHS_SOLVE_FP64, MRHS_SOLVE_MIXED or MRHS_SOLVE_CG5D */
  int32_t precond;      /* 0: BlockCGrQ (Fig. 2 left); 1: Chebyshev-preconditioned
                           BlockCGrQ (Fig. 2 right) */
  int32_t precond_prec; /* MRHS_PREC_* of the Chebyshev operator applications;
                           -1 (default): FP16X, FP16, BF16, TC32 or FP32, the
                           first one built that fits nrhs (FP16X/TC32: <= 32) */
  int32_t cheb_order;   /* polynomial degree */
  double cheb_lo;       /* Chebyshev interval; cheb_hi <= 0: hi = 1.08 x power- */
  double cheb_hi;       /*   method estimate; cheb_lo <= 0: lo = hi / 400 */
  double inner_tol;     /* MIXED: residual reduction of the first refinement
                           cycle, and of the later ones unless inner_tol_later
                           is set; in (0, 1).  A cycle also ends when the
                           recurrence estimate has not improved by 30% over 32
                           iterations (a low-precision preconditioner is not
                           exactly linear) */
  int32_t max_cycles;   /* MIXED: refinement cycles */
  int32_t check_every;  /* read the convergence flag every k iterations (MIXED:
                           at most every 2 in a refinement cycle that needs
                           less than a tenfold reduction, which is expected
                           to end the solve) */
  double breakdown_tau; /* relative Cholesky pivot threshold */
  int32_t krylov_prec;  /* MIXED: operator precision inside the inner Krylov loop,
                           MRHS_PREC_FP32 or MRHS_PREC_TC32; -1 (default): TC32
                           if built and nrhs <= 32, else FP32 */
  int32_t use_graph;    /* 1 (default): after a first uncaptured iteration, each
                           chunk of check_every block-CG iterations is captured
                           once as a CUDA graph and replayed */
  int32_t residual_prec; /* MIXED: operator of each cycle's residual B - H X:
                           MRHS_PREC_FP64, MRHS_PREC_DF32 or MRHS_PREC_OZ;
                           -1 (default): OZ if built and nrhs <= 32, else
                           DF32.  A residual in another precision than
                           fp64_prec that meets tol is recomputed with
                           fp64_prec before the solve returns, and a cycle
                           that needs less than a tenfold reduction computes
                           its residual with fp64_prec directly, so the
                           residuals reported are FP64 ones */
  int32_t recycle;      /* MIXED (block_cg_solve only): every inner iteration
                           keeps a copy of its search block D and of
                           N = (D^dagger H D)^-1; a new refinement cycle
                           starts from the Galerkin correction over the
                           blocks of all earlier cycles, E_0 = sum_i D_i N_i
                           D_i^dagger F, taken one cycle's blocks at a time
                           (the blocks of one cycle are H-conjugate) with
                           F - H E_0 refreshed between cycles, `recycle`
                           sweeps over them (0, the default: plain restarts;
                           1 and 2 are tested, 1 is the benchmark's setting).
                           A column keeps its E_0
                           only if that lowers the energy functional
                           e^dagger H e - 2 Re e^dagger f below zero; blocks of
                           iterations that lost rank are not kept; a cycle
                           that started from kept blocks and reduced some
                           column's residual by nothing ends the recycling
                           for the solve.  The copies are held by the
                           operator until mrhs_op_destroy */
  int32_t recycle_max_blocks; /* cap on kept blocks (each N x nrhs complex64);
                           0 (default): 128.  Fewer are kept when device
                           memory runs short (a reserve of max(4 GiB, 1/16
                           of the device) stays free) */
  int32_t fp64_prec;    /* the FP64 operator of the solve: every operator
                           application of MRHS_SOLVE_FP64 (Krylov loop,
                           residuals, FP64 preconditioner), and in MIXED and
                           CG5D the residual that decides convergence.
                           MRHS_PREC_FP64 (FP64 FMA pipes) or MRHS_PREC_OZ
                           (digit-sliced tensor-core form, held to the FP64
                           tolerance); -1 (default): OZ if built and
                           nrhs <= 32, else FP64 (MRHS_ERR_UNSUPPORTED if
                           neither is available) */
  double inner_tol_later; /* MIXED: residual reduction of the refinement cycles
                           after the first, in [0, 1); 0: inner_tol; default
                           1e-2.
                           Such a cycle starts from a residual whose low modes
                           dominate.  For those modes the Krylov operator's own
                           error, about its relative error times the condition
                           number, bounds what the cycle reaches (TC32 at
                           kappa 1e4: 1.5-2% of the start), and iterating the
                           recurrence estimate far below that bound lowers the
                           true residual no further.  1e-2 against inner_tol:
                           42 instead of 50-54 inner iterations at 12^4
                           (inner_tol 3e-4, four right-hand-side sets), 34
                           instead of 42 at 8^4, 24 instead of 26 at 6^4 with
                           kappa 1e3.  On a well-conditioned problem, where a
                           cycle is not bound that way, a loose later target
                           can cost an extra cycle */
} mrhs_solve_params;

enum {
  MRHS_SOLVE_FP64 = 0,  /* everything FP64 (plain FP64 block CG, with the
                           operator fp64_prec) */
  MRHS_SOLVE_MIXED = 1, /* FP64 outer defect correction (true residual, Gram
                           accumulation, Cholesky, solution update); inner block
                           CG on complex64 vectors with the TC32 (or FP32)
                           operator and the low-precision Chebyshev
                           preconditioner */
  MRHS_SOLVE_CG5D = 2   /* Sec. 2.1's single five-dimensional system: plain
                           CG on the whole block, alpha and beta from inner
                           products summed over all right-hand sides, no
                           preconditioner; operator krylov_prec = FP64 (default,
                           -1) or DF32; stops when every column's recurrence
                           residual meets tol, info reports FP64 true residuals */
};

typedef struct {
  int32_t status;     /* same code as the return value */
  int32_t iters;      /* Krylov iterations, all cycles */
  int32_t cycles;     /* refinement cycles (MIXED) or 1 */
  int32_t nrhs;
  int64_t applies[MRHS_NUM_PREC]; /* operator applications per precision */
  double resid[MRHS_MAX_RHS]; /* final true relative residual per RHS (FP64) */
  double cheb_lo, cheb_hi;    /* interval used */
  double ms_total;            /* wall time of the call */
  int32_t krylov_prec;        /* operator precision used in the Krylov loop */
  int32_t precond_prec;       /* operator precision used in the preconditioner (-1: none) */
  /* MIXED, per refinement cycle (first MRHS_MAX_CYCLES): inner iterations,
   * largest true relative residual after the cycle, and how the inner solve
   * ended (bit 0 target reached, bit 3 estimate stalled) */
  int32_t cycle_iters[MRHS_MAX_CYCLES];
  double cycle_resid[MRHS_MAX_CYCLES];
  int32_t cycle_flag[MRHS_MAX_CYCLES];
  int32_t recycle_blocks;      /* MIXED: search blocks kept (see recycle) */
  int32_t recycle_projections; /* MIXED: block projections of cycle starts */
} mrhs_solve_info;

/* Solve H X = B for nrhs right-hand sides with block CG (Fig. 2).
 *   B device complex128 [V][nb][nrhs] (read only); X device complex128: in,
 *   the initial guess X_0; out, the solution.  A zero column of B gives a
 *   zero column of X.  H must be Hermitian positive definite.
 * Returns after termination (synchronises `stream`); on MRHS_ERR_NOT_CONVERGED
 * X and *info hold the last iterate.  A NaN or Inf in B, or in a column of
 * X_0 whose column of B is not zero, returns MRHS_ERR_NONFINITE before any
 * iteration: *info is not written and X holds X_0 with the columns of zero B
 * cleared.  (A column norm that overflows, from entries above about 1e154,
 * counts as non-finite.)  A NaN or Inf met during the iteration also returns
 * MRHS_ERR_NONFINITE.  Workspace is allocated by the call. */
int block_cg_solve(mrhs_op op, const void* B, void* X, int32_t nrhs,
                   const mrhs_solve_params* params, mrhs_solve_info* info, void* stream);

/* Many independent operators in ONE persistent tensor-core launch: the work
 * list covers every site of every problem (uneven lattices, nb and nrhs
 * allowed), each problem keeps its own inputs, scales and packed images.
 *   ops    host array of n (1..MRHS_MAX_BATCH) distinct operators on the
 *          current device, all built with precision `prec` (BF16, FP16,
 *          FP16X or TC32)
 *   X, Y   host arrays of n device pointers ([V_i][nb_i][nrhs_i] complex64)
 *   nrhs   host array of n counts
 * Asynchronous. */
int mrhs_batch_apply(const mrhs_op* ops, int32_t n, int32_t prec, const void* const* X,
                     void* const* Y, const int32_t* nrhs, void* stream);

/* Solve n independent systems H_i X_i = B_i side by side.  With
 * MRHS_SOLVE_MIXED, precond = 1, nrhs_i <= 32 and TC32 plus a tensor-core
 * preconditioner precision built into every operator, the problems advance in
 * lockstep: each operator step (Krylov and Chebyshev) of an iteration is one
 * persistent launch over all still-active problems, chunks of check_every
 * iterations are captured once as a CUDA graph, and a problem that reaches
 * its inner target leaves the launches through a device mask.  Otherwise the
 * problems are solved one after another with block_cg_solve.
 *   B, X   host arrays of n device pointers (complex128 [V_i][nb_i][nrhs_i])
 *   info   host array of n records (may be NULL)
 * Returns MRHS_OK if every problem converged.  MRHS_ERR_NOT_CONVERGED means
 * some problem did not; all X and info are still written.  Non-finite input
 * in a problem's B or X_0 returns MRHS_ERR_NONFINITE, as in block_cg_solve:
 * in the lockstep path before any problem iterates (the message names the
 * problem), one after another when that problem's turn comes.  Any other
 * failure code may leave the X and info of problems other than the failing
 * one unwritten.  Synchronises `stream`. */
int mrhs_batch_solve(const mrhs_op* ops, int32_t n, const void* const* B, void* const* X,
                     const int32_t* nrhs, const mrhs_solve_params* params, mrhs_solve_info* info,
                     void* stream);

/* Default parameters for `mode`. */
void mrhs_solve_params_default(mrhs_solve_params* p, int32_t mode);

/* Returns and clears the sticky error word of the tensor-core kernels: 0 if
 * none, else a bit set by a bounded wait that expired inside a kernel (1 the
 * TMA producer, 2 the MMA issuer, 4 the epilogue of the BF16 ... TC32 kernel;
 * 8, 16, 32 the same roles in the OZ kernel; 64, 128, 256 the same and 512
 * the operand converters of the tensor-core Gram and block update
 * (mrhs_block_tc); 1024 the tensor-core block project / promote); such a
 * kernel records the
 * bit, drains its own copies, frees its tensor memory and returns, leaving
 * its output undefined.  Synchronises the current device. */
int32_t mrhs_device_error(void);

/* Which kernels run the complex64 block algebra of blocks of 4..32 columns
 * (block_inner, block_axpy and the updates inside the block-CG solves) and
 * the complex64 block project / promote of the shapes stated there:
 * mode 1 (default) the tcgen05 tensor-core kernels (Fig. 2's Grams and
 * block updates as MMAs on three-term bf16 splits, FP32-class products),
 * mode 0 the FP32 FMA kernels.  Process-wide; returns the previous mode, or
 * MRHS_ERR_INVALID_ARG for another value.  Not thread-safe against calls in
 * flight on other host threads. */
int32_t mrhs_block_tc(int32_t mode);

/* Debugging: the limit, in ns, of the bounded wait with which the epilogue
 * of the tensor-core kernels (BF16 ... TC32 and OZ) waits for its
 * accumulator; 0 restores the default of 1 s.  A short limit (a microsecond)
 * makes that wait run out on purpose: the kernel records bit 4 (BF16 ...
 * TC32) or 32 (OZ) in mrhs_device_error (the producer and the MMA issuer,
 * told to stop, may add theirs), waits for its own copies and MMAs, frees
 * its tensor memory and returns; its output is then undefined.  Lets a test
 * exercise the failure path without faulting the GPU.  Applies to the
 * current device; synchronous. */
int mrhs_debug_wait_limit(uint64_t ns);

/* Measurement hooks.  mrhs_op_kernel_timing(op, 1) makes every following
 * application of `op` record a CUDA event pair on its stream around the
 * operator's main kernel (the tcgen05 kernel for BF16/FP16, the FMA kernel
 * for FP64/FP32; input packing excluded); mrhs_op_kernel_time returns the
 * number of such launches for precision `prec` and their summed device time
 * in ms, then clears the record (it synchronises on the last event).
 * mrhs_launch_count returns the number of kernels this library has launched
 * in the process so far. */
int mrhs_op_kernel_timing(mrhs_op op, int32_t enable);

/* Hermitian pairing in the tensor-core kernels.  When the hop coefficients
 * satisfy A_q(x + delta_p) = A_p(x)^dagger exactly (q the point with
 * delta_q = -delta_p, p != 0; checked at creation, Sec. 2.6's Hermitian
 * coarse operator) and nb is a multiple of 16, the BF16/FP16/FP16X/TC32
 * kernels read
 * one coefficient tile per pair of points: the tile of (x, p) serves site x
 * directly and site x + delta_p transposed and conjugated, the second read
 * coming from L2 when both sites are in flight.  Sites are visited in 4D
 * blocks for that.  mode -1 queries, 0 disables, 1 enables for every
 * tensor-core form, 2 for TC32 only (MRHS_ERR_UNSUPPORTED if the hop pairs are
 * not exactly Hermitian); *active (may be null) receives the mode after the
 * call.  Default 0.  At 12^4, nb 48, 32 RHS the shared reads cut DRAM
 * traffic by 10% (FP16X) and 4% (TC32); the second, transposed use costs two
 * MMAs (N = nb) per K step that re-read the input tile.  FP16X gets slower
 * (2.82 against 2.66 ms); TC32 is 8-15% faster when timed alone but slower
 * inside the mixed solve (6.85 against 5.7 ms per launch).  Results equal
 * the unpaired kernel's up to FP32 summation order. */
int mrhs_op_hermitian(mrhs_op op, int32_t mode, int32_t* active);

/* Launch shape of this operator's BF16/FP16 tensor-core kernel (the knobs an
 * autotuner searches): stencil points per pipeline stage (1..16; 0 = built-in
 * choice of >= 16 KB of coefficients per copy), CTAs per SM (1 or 2, each
 * with its own copy/MMA ring; default 2) and the ring depth cap (2..32).  Shapes that
 * do not fit shared memory fall back to fewer points per stage.  Results do
 * not depend on the shape. */
int mrhs_op_tc_tune(mrhs_op op, int32_t pts_per_stage, int32_t ctas_per_sm, int32_t max_stages);

/* Launch-shape autotuner for the tensor-core kernel (the three knobs of
 * mrhs_op_tc_tune).  mrhs_autotune times candidate shapes for the `n`
 * operators ops[0..n-1] (n = 1: one operator; n > 1: their batched launch, as
 * mrhs_batch_apply makes it) in precision `prec` (BF16..TC32) at nrhs[i]
 * right-hand sides, on scratch inputs it allocates and frees itself: first
 * points per stage {built-in, 1, 2, 3, 4, 6, 8, 12} x CTAs per SM {1, 2} at
 * the deepest ring, then ring depths {2, 3, 4, 6, 8, 12, 16} for the best of
 * those.  Each candidate is timed over `reps` launches (<= 0: 3) after one
 * warm-up, with CUDA events on `stream`; every candidate's output must equal
 * the first one's bit for bit, else MRHS_ERR_DEVICE.  The winner is stored in
 * a process-wide cache keyed, per problem, on (SM count, V, nb, stencil
 * points, nrhs, prec); every later launch of exactly that shape (or list of
 * shapes, for a batch) without an explicit mrhs_op_tc_tune uses it.  `out`
 * (host, may be NULL) receives the winner, the number of candidates timed and
 * the best and built-in default times in ms per launch.  Synchronises
 * `stream`; MRHS_ERR_INVALID_ARG if `stream` is being captured into a graph.
 * mrhs_autotune_save / _load write / merge the cache as text, one entry per
 * line ("n", n x "sms V nb npts nrhs prec", "pps ctas stages ms"); a malformed
 * file is rejected whole (MRHS_ERR_INVALID_ARG).  mrhs_autotune_entries
 * returns the number of cached shapes; mrhs_autotune_clear empties the cache.
 * The cache calls are host-only and thread-safe. */
typedef struct {
  int32_t pts_per_stage, ctas_per_sm, max_stages, candidates;
  double ms, ms_default;
} mrhs_tune_result;
int mrhs_autotune(const mrhs_op* ops, int32_t n, int32_t prec, const int32_t* nrhs, int32_t reps,
                  mrhs_tune_result* out, void* stream);
int mrhs_autotune_save(const char* path);
int mrhs_autotune_load(const char* path);
int64_t mrhs_autotune_entries(void);
void mrhs_autotune_clear(void);
int mrhs_op_kernel_time(mrhs_op op, int32_t prec, int64_t* launches, double* ms);
int64_t mrhs_launch_count(void);

/* Thread-local message describing the last error ("" if none). */
const char* mrhs_last_error(void);

/* Library version string. */
const char* mrhs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MRHS_H */
