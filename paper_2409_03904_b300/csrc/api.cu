// C ABI entry points of libmrhs: argument checks, operator construction and
// dispatch to the kernels (see include/mrhs.h for the contract).
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>

#include "internal.cuh"

namespace mrhs {

static thread_local std::string t_last_error;

void set_error(const std::string& msg) { t_last_error = msg; }

int fail(int code, const std::string& msg) {
  set_error(msg);
  return code;
}

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t launch_count() { return (int64_t)g_launches.load(); }
void add_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void timer_mark(mrhs_op_s* op, int prec, cudaStream_t s) {
  KernelTimer& t = op->timer[prec];
  if (!t.on) return;
  if (t.used >= t.ev.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    t.ev.push_back(e);
  }
  cudaEventRecord(t.ev[t.used++], s);
}

int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 148;
  if (!cached[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 148;
    cached[dev] = n;
  }
  return cached[dev];
}

namespace {

struct Geom4 {
  int32_t L[4], Lin[4], h[4];
};

// Input-site index of x + delta_p (fwd) and x - delta_p (bwd) for every
// output site x: coordinates c of x on L, then c + h +- delta on the input
// lattice Lin, wrapped periodically (a padded dimension never wraps, since
// |delta| <= 1 = h there).
__global__ void k_neighbours(int32_t* fwd, int32_t* bwd, int64_t V, int npts, Geom4 g,
                             const int8_t* __restrict__ disp) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (x >= V) return;
  int c[4];
  int64_t r = x;
  for (int mu = 0; mu < 4; ++mu) {
    c[mu] = (int)(r % g.L[mu]);
    r /= g.L[mu];
  }
  int64_t yf = 0, yb = 0;
  for (int mu = 3; mu >= 0; --mu) {
    const int d = disp[4 * p + mu], n = g.Lin[mu], ci = c[mu] + g.h[mu];
    yf = yf * n + (ci + d + n) % n;
    yb = yb * n + (ci - d + n) % n;
  }
  fwd[(int64_t)p * V + x] = (int32_t)yf;
  bwd[(int64_t)p * V + x] = (int32_t)yb;
}

// Exact Hermiticity of the stencil operator, A_q(x + delta_p) = A_p(x)^dagger
// for the partner q of every point p (delta_q = -delta_p): one block per
// (site, point); a mismatch sets bad[0] for a hop pair, bad[1] for the self
// term (p = q = 0).
__global__ void k_herm_check(const double2* __restrict__ A, const int32_t* __restrict__ nbr_fwd,
                             const int8_t* __restrict__ partner, int64_t V, int npts, int nb,
                             int* bad) {
  const int64_t x = blockIdx.x;
  const int p = blockIdx.y;
  const int q = partner[p];
  const int64_t y = nbr_fwd[(int64_t)p * V + x];
  const double2* Ap = A + (x * npts + p) * (int64_t)nb * nb;
  const double2* Aq = A + (y * npts + q) * (int64_t)nb * nb;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int a = e / nb, b = e % nb;
    const double2 u = Ap[a * nb + b], v = Aq[b * nb + a];
    if (u.x != v.x || u.y != -v.y) atomicExch(&bad[p == 0 ? 1 : 0], 1);
  }
}

__global__ void k_to_c64(const double2* __restrict__ a, float2* __restrict__ b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = make_float2(__double2float_rn(a[i].x), __double2float_rn(a[i].y));
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int check_op(const mrhs_op_s* op) {
  if (!op) return fail(MRHS_ERR_INVALID_ARG, "null operator");
  return MRHS_OK;
}

// Entry points that need the whole periodic lattice on one operator: an
// operator with an input halo (one rank's part of a decomposed lattice)
// supports coarse_op_apply only.
int check_plain(const mrhs_op_s* op) {
  if (op->Vin != op->V)
    return fail(MRHS_ERR_UNSUPPORTED, "this entry point needs an operator without an input halo");
  return MRHS_OK;
}

// The mixed solve's per-cycle reductions: a target of 1 or more would end
// every cycle at once, and the solve would restart without progress.
int check_inner_tols(const mrhs_solve_params& p) {
  if (p.mode != MRHS_SOLVE_MIXED) return MRHS_OK;
  if (!(p.inner_tol > 0.0 && p.inner_tol < 1.0) ||
      !(p.inner_tol_later >= 0.0 && p.inner_tol_later < 1.0))
    return fail(MRHS_ERR_INVALID_ARG, "inner_tol must be in (0, 1) and inner_tol_later in [0, 1)");
  return MRHS_OK;
}

int check_vec(const void* p, const char* name) {
  if (!p) return fail(MRHS_ERR_INVALID_ARG, std::string(name) + " is null");
  if (!aligned16(p)) return fail(MRHS_ERR_INVALID_ARG, std::string(name) + " not 16-byte aligned");
  return MRHS_OK;
}

int check_prec(const mrhs_op_s* op, int prec) {
  if (prec < 0 || prec >= MRHS_NUM_PREC) return fail(MRHS_ERR_INVALID_ARG, "unknown precision");
  if (!(op->prec_mask & MRHS_PREC_BIT(prec)))
    return fail(MRHS_ERR_UNSUPPORTED, "precision not built into this operator");
  return MRHS_OK;
}

// Operator of the refinement cycles' residuals: FP64, DF32 (both on the FP64
// copy) or, when built and the shape fits, the digit-sliced tensor-core form.
int check_residual_prec(int rp, bool fp64_ok, bool oz_ok) {
  if (rp == MRHS_PREC_FP64 || rp == MRHS_PREC_DF32)
    return fp64_ok ? MRHS_OK : fail(MRHS_ERR_UNSUPPORTED, "residual_prec: FP64 not built");
  if (rp == MRHS_PREC_OZ)
    return oz_ok ? MRHS_OK
                 : fail(MRHS_ERR_UNSUPPORTED, "residual_prec OZ: not built or nrhs > 32");
  return fail(MRHS_ERR_INVALID_ARG, "residual_prec must be FP64, DF32 or OZ");
}

// The FP64 operator of a solve (fp64_prec): native FP64 or the digit-sliced
// form; -1 picks OZ when it is built and fits, else FP64.
int resolve_fp64_prec(int* fp, bool fp64_ok, bool oz_ok) {
  if (*fp < 0) *fp = oz_ok ? MRHS_PREC_OZ : MRHS_PREC_FP64;
  if (*fp == MRHS_PREC_FP64)
    return fp64_ok ? MRHS_OK
                   : fail(MRHS_ERR_UNSUPPORTED, "the solve needs the FP64 or the OZ operator "
                                                "(OZ: nrhs <= 32)");
  if (*fp == MRHS_PREC_OZ)
    return oz_ok ? MRHS_OK : fail(MRHS_ERR_UNSUPPORTED, "fp64_prec OZ: not built or nrhs > 32");
  return fail(MRHS_ERR_INVALID_ARG, "fp64_prec must be FP64 or OZ");
}

}  // namespace

int op_apply(mrhs_op_s* op, int prec, bool dag, const void* X, void* Y, int nrhs,
             cudaStream_t s) {
  if (prec == MRHS_PREC_OZ) return oz_apply(op, dag, X, Y, nrhs, s);
  if (!MRHS_PREC_IS_TC(prec)) return simt_apply(op, prec, dag, X, Y, nrhs, s);
  return tc_apply(op, prec, dag, X, Y, nrhs, s);
}

}  // namespace mrhs

using namespace mrhs;

extern "C" {

const char* mrhs_last_error(void) { return t_last_error.c_str(); }

const char* mrhs_version(void) { return "mrhs 0.1 (sm_103a)"; }

int32_t mrhs_device_error(void) {
  cudaDeviceSynchronize();
  return (int32_t)(tc_read_and_clear_error() | oz_read_and_clear_error() |
                   btc_read_and_clear_error() | bltc_read_and_clear_error());
}

int32_t mrhs_block_tc(int32_t mode) {
  if (mode != 0 && mode != 1) return fail(MRHS_ERR_INVALID_ARG, "block algebra mode is 0 or 1");
  const int32_t prev = g_block_tc_mode;
  g_block_tc_mode = mode;
  return prev;
}

static int op_create(mrhs_op* out, const int32_t L[4], const int32_t halo[4], int32_t nb,
                     int32_t npts, const int8_t* disp, const void* A, uint32_t prec_mask,
                     void* stream) {
  if (!out || !L || !disp || !A) return fail(MRHS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  bool any_halo = false;
  for (int mu = 0; mu < 4; ++mu) {
    if (halo[mu] != 0 && halo[mu] != 1) return fail(MRHS_ERR_INVALID_ARG, "halo must be 0 or 1");
    any_halo = any_halo || halo[mu] != 0;
  }
  if (any_halo && (prec_mask & ~(MRHS_PREC_BIT(MRHS_PREC_FP64) | MRHS_PREC_BIT(MRHS_PREC_FP32) |
                                 MRHS_PREC_BIT(MRHS_PREC_DF32) | MRHS_PREC_BIT(MRHS_PREC_OZ))))
    return fail(MRHS_ERR_UNSUPPORTED,
                "an operator with an input halo builds FP64, DF32, FP32 and OZ only");
  if (nb < 1 || nb > 64) return fail(MRHS_ERR_INVALID_ARG, "nb must be in 1..64");
  if (npts < 1 || npts > MRHS_MAX_PTS) return fail(MRHS_ERR_INVALID_ARG, "npts must be in 1..81");
  if (prec_mask == 0 || (prec_mask >> MRHS_NUM_PREC))
    return fail(MRHS_ERR_INVALID_ARG, "prec_mask must select precisions 0..7");
  // DF32 runs on the FP64 coefficients; with them it comes for free.  The
  // digit-sliced form stands alone (only its adjoint image is built from the
  // FP64 copy, on first use)
  if (prec_mask & MRHS_PREC_BIT(MRHS_PREC_DF32)) prec_mask |= MRHS_PREC_BIT(MRHS_PREC_FP64);
  if (prec_mask & MRHS_PREC_BIT(MRHS_PREC_FP64)) prec_mask |= MRHS_PREC_BIT(MRHS_PREC_DF32);
  if (!aligned16(A)) return fail(MRHS_ERR_INVALID_ARG, "A not 16-byte aligned");
  int64_t V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (L[mu] < 1) return fail(MRHS_ERR_INVALID_ARG, "lattice extents must be >= 1");
    V *= L[mu];
  }
  if (V * npts > INT32_MAX) return fail(MRHS_ERR_INVALID_ARG, "lattice too large");
  for (int p = 0; p < npts; ++p)
    for (int mu = 0; mu < 4; ++mu)
      if (disp[4 * p + mu] < -1 || disp[4 * p + mu] > 1)
        return fail(MRHS_ERR_INVALID_ARG, "displacements must lie in {-1,0,1}");
  for (int mu = 0; mu < 4; ++mu)
    if (disp[mu] != 0) return fail(MRHS_ERR_INVALID_ARG, "disp[0] must be the self term");
  cudaStream_t s = (cudaStream_t)stream;
  mrhs_op_s* op = new mrhs_op_s();
  op->Vin = 1;
  for (int mu = 0; mu < 4; ++mu) {
    op->L[mu] = L[mu];
    op->halo[mu] = halo[mu];
    op->Lin[mu] = L[mu] + 2 * halo[mu];
    op->Vin *= op->Lin[mu];
  }
  if (op->Vin * npts > INT32_MAX) {
    delete op;
    return fail(MRHS_ERR_INVALID_ARG, "lattice too large");
  }
  op->nb = nb;
  op->npts = npts;
  op->V = V;
  std::memcpy(op->disp, disp, 4 * (size_t)npts);
  op->prec_mask = prec_mask;
  cudaGetDevice(&op->device);
  auto bail = [&](int code) {
    mrhs_op_destroy(op);
    return code;
  };
  const size_t nA = (size_t)V * npts * nb * nb;
  int8_t* d_disp = nullptr;
  if (cudaMalloc(&op->nbr_fwd, sizeof(int32_t) * V * npts) != cudaSuccess ||
      cudaMalloc(&op->nbr_bwd, sizeof(int32_t) * V * npts) != cudaSuccess ||
      cudaMalloc(&d_disp, 4 * (size_t)npts) != cudaSuccess) {
    cudaGetLastError();
    if (d_disp) cudaFree(d_disp);
    return bail(fail(MRHS_ERR_NO_MEMORY, "neighbour tables"));
  }
  if (cudaMemcpyAsync(d_disp, disp, 4 * (size_t)npts, cudaMemcpyHostToDevice, s) != cudaSuccess) {
    cudaFree(d_disp);
    return bail(fail(MRHS_ERR_CUDA, "disp upload"));
  }
  {
    dim3 grid((unsigned)((V + 255) / 256), (unsigned)npts);
    Geom4 g4;
    for (int mu = 0; mu < 4; ++mu) {
      g4.L[mu] = op->L[mu];
      g4.Lin[mu] = op->Lin[mu];
      g4.h[mu] = op->halo[mu];
    }
    { k_neighbours<<<grid, 256, 0, s>>>(op->nbr_fwd, op->nbr_bwd, V, npts, g4, d_disp);
      ::mrhs::count_launch(); }
  }
  if (prec_mask & MRHS_PREC_BIT(MRHS_PREC_FP64)) {
    if (cudaMalloc(&op->a64, sizeof(double2) * nA) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(d_disp);
      return bail(fail(MRHS_ERR_NO_MEMORY, "FP64 coefficients"));
    }
    cudaMemcpyAsync(op->a64, A, sizeof(double2) * nA, cudaMemcpyDeviceToDevice, s);
  }
  if (prec_mask & MRHS_PREC_BIT(MRHS_PREC_FP32)) {
    if (cudaMalloc(&op->a32, sizeof(float2) * nA) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(d_disp);
      return bail(fail(MRHS_ERR_NO_MEMORY, "FP32 coefficients"));
    }
    { k_to_c64<<<num_sms() * 8, 256, 0, s>>>((const double2*)A, op->a32, (int64_t)nA); ::mrhs::count_launch(); }
  }
  // Hermitian stencil operators let the tensor-core kernel read one tile per
  // pair of points (p, -p): detect exact Hermiticity once (an operator with
  // an input halo holds no partner tiles across its boundary: not checked)
  if (!any_halo) {
    int8_t partner[MRHS_MAX_PTS];
    bool paired = true;
    for (int p = 0; p < npts && paired; ++p) {
      partner[p] = -1;
      for (int q = 0; q < npts; ++q)
        if (disp[4 * q] == -disp[4 * p] && disp[4 * q + 1] == -disp[4 * p + 1] &&
            disp[4 * q + 2] == -disp[4 * p + 2] && disp[4 * q + 3] == -disp[4 * p + 3])
          partner[p] = (int8_t)q;
      paired = partner[p] >= 0;
    }
    if (paired) {
      int8_t* d_partner = nullptr;
      int* d_bad = nullptr;
      int bad[2] = {1, 1};
      if (cudaMalloc(&d_partner, (size_t)npts) == cudaSuccess &&
          cudaMalloc(&d_bad, 2 * sizeof(int)) == cudaSuccess &&
          cudaMemcpyAsync(d_partner, partner, (size_t)npts, cudaMemcpyHostToDevice, s) == cudaSuccess &&
          cudaMemsetAsync(d_bad, 0, 2 * sizeof(int), s) == cudaSuccess) {
        dim3 grid((unsigned)V, (unsigned)npts);
        { k_herm_check<<<grid, 128, 0, s>>>((const double2*)A, op->nbr_fwd, d_partner, V, npts,
                                            nb, d_bad); ::mrhs::count_launch(); }
        if (cudaMemcpyAsync(bad, d_bad, 2 * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
          bad[0] = bad[1] = 1;
      }
      cudaGetLastError();
      cudaFree(d_partner);
      cudaFree(d_bad);
      // pairing needs the hop pairs only; H^dagger = H also the self term
      op->pairable = bad[0] == 0;
      op->herm = bad[0] == 0 && bad[1] == 0;
      // the points with a positive first nonzero displacement, one of each pair
      op->herm_nf = 0;
      for (int p = 1; p < npts; ++p) {
        int first = 0;
        for (int mu = 0; mu < 4 && first == 0; ++mu) first = disp[4 * p + mu];
        if (first > 0) op->herm_f[op->herm_nf++] = (int8_t)p;
      }
      op->herm_mode = 0;       // opt-in: see mrhs_op_hermitian
    }
  }
  for (int prec = MRHS_PREC_BF16; prec <= MRHS_PREC_TC32; ++prec)
    if (prec_mask & MRHS_PREC_BIT(prec)) {
      int st = tc_build(op, prec, false, (const double2*)A, s);
      if (st != MRHS_OK) {
        cudaFree(d_disp);
        return bail(st);
      }
    }
  if (prec_mask & MRHS_PREC_BIT(MRHS_PREC_OZ)) {
    int st = oz_build(op, false, (const double2*)A, s);
    if (st != MRHS_OK) {
      cudaFree(d_disp);
      return bail(st);
    }
  }
  cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(d_disp);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return bail(fail(MRHS_ERR_CUDA, std::string("op create: ") + cudaGetErrorString(e)));
  *out = op;
  return MRHS_OK;
}

int mrhs_debug_wait_limit(uint64_t ns) {
  if (ns > 10000000000ull) return fail(MRHS_ERR_INVALID_ARG, "wait limit above 10 s");
  MRHS_TRY(tc_set_wait_limit(ns));
  MRHS_TRY(oz_set_wait_limit(ns));
  MRHS_TRY(btc_set_wait_limit(ns));
  return MRHS_OK;
}

int mrhs_op_create(mrhs_op* out, const int32_t L[4], int32_t nb, int32_t npts, const int8_t* disp,
                   const void* A, uint32_t prec_mask, void* stream) {
  const int32_t none[4] = {0, 0, 0, 0};
  return op_create(out, L, none, nb, npts, disp, A, prec_mask, stream);
}

int mrhs_op_create_halo(mrhs_op* out, const int32_t L[4], const int32_t halo[4], int32_t nb,
                        int32_t npts, const int8_t* disp, const void* A, uint32_t prec_mask,
                        void* stream) {
  if (!halo) return fail(MRHS_ERR_INVALID_ARG, "null argument");
  return op_create(out, L, halo, nb, npts, disp, A, prec_mask, stream);
}

int mrhs_op_lambda_max(mrhs_op op, int32_t prec, int32_t iters, double* lam, void* stream) {
  MRHS_TRY(check_op(op));
  MRHS_TRY(check_plain(op));
  MRHS_TRY(check_prec(op, prec));
  if (!lam || iters < 1) return fail(MRHS_ERR_INVALID_ARG, "mrhs_op_lambda_max: arguments");
  MRHS_TRY(lambda_max(op, prec, iters, (cudaStream_t)stream, lam));
  op->lam_max[prec] = *lam;
  return MRHS_OK;
}

int mrhs_op_hermitian(mrhs_op op, int32_t mode, int32_t* active) {
  MRHS_TRY(check_op(op));
  if (mode < -1 || mode > 2)
    return fail(MRHS_ERR_INVALID_ARG, "mrhs_op_hermitian: mode -1, 0, 1 or 2");
  if (mode >= 1 && !op->pairable)
    return fail(MRHS_ERR_UNSUPPORTED,
                "hop pairs of the operator are not exactly Hermitian on a symmetric stencil");
  if (mode >= 0) op->herm_mode = (int8_t)mode;
  if (active) *active = op->herm_mode;
  return MRHS_OK;
}

int mrhs_op_tc_tune(mrhs_op op, int32_t pts_per_stage, int32_t ctas_per_sm, int32_t max_stages) {
  MRHS_TRY(check_op(op));
  if (pts_per_stage < 0 || pts_per_stage > 16 || ctas_per_sm < 1 || ctas_per_sm > 2 ||
      max_stages < 2 || max_stages > 32)
    return fail(MRHS_ERR_INVALID_ARG, "mrhs_op_tc_tune: pts 0..16, ctas 1..2, stages 2..32");
  op->tc_tune.pps = pts_per_stage;
  op->tc_tune.ctas_per_sm = ctas_per_sm;
  op->tc_tune.max_stages = max_stages;
  op->tc_set = true;
  return MRHS_OK;
}

int64_t mrhs_launch_count(void) { return (int64_t)g_launches.load(); }

int mrhs_op_kernel_timing(mrhs_op op, int32_t enable) {
  if (!op) return fail(MRHS_ERR_INVALID_ARG, "null operator");
  for (auto& t : op->timer) {
    t.on = enable != 0;
    t.used = 0;
  }
  return MRHS_OK;
}

int mrhs_op_kernel_time(mrhs_op op, int32_t prec, int64_t* launches, double* ms) {
  if (!op || !launches || !ms || prec < 0 || prec >= MRHS_NUM_PREC)
    return fail(MRHS_ERR_INVALID_ARG, "mrhs_op_kernel_time: arguments");
  KernelTimer& t = op->timer[prec];
  double total = 0.0;
  const size_t pairs = t.used / 2;
  if (pairs) MRHS_CUDA_TRY(cudaEventSynchronize(t.ev[2 * pairs - 1]));
  for (size_t i = 0; i < pairs; ++i) {
    float v = 0.f;
    MRHS_CUDA_TRY(cudaEventElapsedTime(&v, t.ev[2 * i], t.ev[2 * i + 1]));
    total += v;
  }
  *launches = (int64_t)pairs;
  *ms = total;
  t.used = 0;
  return MRHS_OK;
}

int mrhs_op_destroy(mrhs_op op) {
  if (!op) return MRHS_OK;
  for (auto& t : op->timer)
    for (cudaEvent_t e : t.ev) cudaEventDestroy(e);
  cudaFree(op->nbr_fwd);
  cudaFree(op->nbr_bwd);
  cudaFree(op->a64);
  cudaFree(op->a32);
  for (int i = 0; i < 3; ++i) {
    cudaFree(op->tc[i].codes);
    cudaFree(op->tc[i].scale);
    cudaFree(op->tc[i].diag);
    cudaFree(op->tc_dag[i].codes);
    cudaFree(op->tc_dag[i].scale);
    cudaFree(op->tc_dag[i].diag);
  }
  for (mrhs::OzImage* im : {&op->oz, &op->oz_dag}) {
    cudaFree(im->digits);
    cudaFree(im->scale);
    cudaFree(im->diag);
  }
  op->ws_xpack.release();
  op->ws_ozpack.release();
  op->ws_defl.release();
  op->ws_coarsen.release();
  op->ws_cheb.release();
  op->ws_small.release();
  op->ws_solve.release();
  recycle_release(op);
  delete op;
  return MRHS_OK;
}

static int apply_common(mrhs_op op, int32_t prec, const void* X, void* Y, int32_t nrhs,
                        void* stream, bool dag) {
  MRHS_TRY(check_op(op));
  MRHS_TRY(check_prec(op, prec));
  MRHS_TRY(check_vec(X, "X"));
  MRHS_TRY(check_vec(Y, "Y"));
  if (nrhs < 1 || nrhs > MRHS_MAX_RHS) return fail(MRHS_ERR_INVALID_ARG, "nrhs must be in 1..64");
  if (dag && op->Vin != op->V)
    return fail(MRHS_ERR_UNSUPPORTED, "the adjoint of an operator with an input halo needs "
                                      "coefficients of neighbouring sites it does not hold");
  const size_t es = MRHS_PREC_IS_WIDE(prec) ? 16 : 8;
  const size_t xbytes = es * (size_t)op->Vin * op->nb * nrhs;
  const size_t ybytes = es * (size_t)op->V * op->nb * nrhs;
  const char* x = (const char*)X;
  const char* y = (const char*)Y;
  if (x < y + ybytes && y < x + xbytes) return fail(MRHS_ERR_INVALID_ARG, "X and Y overlap");
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != op->device) return fail(MRHS_ERR_INVALID_ARG, "operator lives on another device");
  return op_apply(op, prec, dag, X, Y, nrhs, (cudaStream_t)stream);
}

int coarse_op_apply(mrhs_op op, int32_t prec, const void* X, void* Y, int32_t nrhs,
                    void* stream) {
  return apply_common(op, prec, X, Y, nrhs, stream, false);
}

int coarse_op_apply_dag(mrhs_op op, int32_t prec, const void* X, void* Y, int32_t nrhs,
                        void* stream) {
  return apply_common(op, prec, X, Y, nrhs, stream, true);
}

int coarse_op_outer(mrhs_op op, const void* G, const void* X, void* GA, double alpha,
                    int32_t nrhs, int32_t dtype, void* stream) {
  MRHS_TRY(check_op(op));
  MRHS_TRY(check_plain(op));
  MRHS_TRY(check_vec(G, "G"));
  MRHS_TRY(check_vec(X, "X"));
  MRHS_TRY(check_vec(GA, "GA"));
  if (nrhs < 1 || nrhs > MRHS_MAX_RHS) return fail(MRHS_ERR_INVALID_ARG, "nrhs must be in 1..64");
  if (dtype != MRHS_C128 && dtype != MRHS_C64) return fail(MRHS_ERR_INVALID_ARG, "dtype");
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != op->device) return fail(MRHS_ERR_INVALID_ARG, "operator lives on another device");
  return outer(op, G, X, (double2*)GA, alpha, nrhs, dtype, (cudaStream_t)stream);
}

int block_inner(const void* X, const void* Y, void* G, int64_t N, int32_t rx, int32_t ry,
                int32_t dtype, void* stream) {
  if (N < 0 || rx < 1 || ry < 1 || rx > MRHS_MAX_RHS || ry > MRHS_MAX_RHS)
    return fail(MRHS_ERR_INVALID_ARG, "block_inner: sizes");
  if (dtype != MRHS_C128 && dtype != MRHS_C64) return fail(MRHS_ERR_INVALID_ARG, "dtype");
  MRHS_TRY(check_vec(G, "G"));
  if (N > 0) {
    MRHS_TRY(check_vec(X, "X"));
    MRHS_TRY(check_vec(Y, "Y"));
  }
  return gram(X, Y, (double2*)G, N, rx, ry, dtype, (cudaStream_t)stream);
}

int block_axpy(void* Y, const void* X, const void* M, double beta, int64_t N, int32_t rin,
               int32_t rout, int32_t dtype, void* stream) {
  if (N < 0 || rin < 1 || rout < 1 || rin > MRHS_MAX_RHS || rout > MRHS_MAX_RHS)
    return fail(MRHS_ERR_INVALID_ARG, "block_axpy: sizes");
  if (dtype != MRHS_C128 && dtype != MRHS_C64) return fail(MRHS_ERR_INVALID_ARG, "dtype");
  MRHS_TRY(check_vec(M, "M"));
  if (N > 0) {
    MRHS_TRY(check_vec(X, "X"));
    MRHS_TRY(check_vec(Y, "Y"));
    if (X == Y && rin != rout)
      return fail(MRHS_ERR_INVALID_ARG, "block_axpy: in-place needs rin == rout");
    const size_t es = dtype == MRHS_C128 ? 16 : 8;
    const char* x = (const char*)X;
    const char* y = (const char*)Y;
    if (X != Y && x < y + es * N * rout && y < x + es * N * rin)
      return fail(MRHS_ERR_INVALID_ARG, "block_axpy: X and Y partially overlap");
  }
  return axpy(Y, X, (const double2*)M, beta, N, rin, rout, dtype, (cudaStream_t)stream);
}

int herm_factor(const void* G, void* S, void* W, int32_t* rank, int32_t r, double tau,
                void* stream) {
  if (r < 1 || r > MRHS_MAX_RHS) return fail(MRHS_ERR_INVALID_ARG, "herm_factor: r");
  if (!(tau >= 0.0)) return fail(MRHS_ERR_INVALID_ARG, "herm_factor: tau");
  MRHS_TRY(check_vec(G, "G"));
  MRHS_TRY(check_vec(S, "S"));
  MRHS_TRY(check_vec(W, "W"));
  if (!rank) return fail(MRHS_ERR_INVALID_ARG, "rank is null");
  return factor((const double2*)G, (double2*)S, (double2*)W, rank, r, tau, (cudaStream_t)stream);
}

int cheby_apply(mrhs_op op, int32_t prec, double lo, double hi, int32_t order, const void* X,
                void* P, int32_t nrhs, void* stream) {
  MRHS_TRY(check_op(op));
  MRHS_TRY(check_plain(op));
  MRHS_TRY(check_prec(op, prec));
  MRHS_TRY(check_vec(X, "X"));
  MRHS_TRY(check_vec(P, "P"));
  if (nrhs < 1 || nrhs > MRHS_MAX_RHS) return fail(MRHS_ERR_INVALID_ARG, "nrhs must be in 1..64");
  if (!(lo > 0.0 && lo < hi)) return fail(MRHS_ERR_INVALID_ARG, "need 0 < lo < hi");
  if (order < 0 || order > 10000) return fail(MRHS_ERR_INVALID_ARG, "order");
  if (X == P) return fail(MRHS_ERR_INVALID_ARG, "X and P must differ");
  return cheby(op, prec, lo, hi, order, X, P, nrhs, (cudaStream_t)stream);
}

static int blocking_common(bool project, const void* basis, const void* in, void* out,
                           int64_t nblk, int32_t vb, int32_t nbasis, int32_t nrhs, int32_t dtype,
                           void* stream) {
  const char* name = project ? "block_project" : "block_promote";
  if (nblk < 0 || vb < 1 || nbasis < 1 || nbasis > 256 || nrhs < 1 || nrhs > MRHS_MAX_RHS)
    return fail(MRHS_ERR_INVALID_ARG, std::string(name) + ": sizes");
  if (dtype != MRHS_C128 && dtype != MRHS_C64) return fail(MRHS_ERR_INVALID_ARG, "dtype");
  if (project && nrhs > 16 * (256 / nbasis))
    return fail(MRHS_ERR_INVALID_ARG, "block_project: nrhs > 16 x (256 / n_basis)");
  if (nblk == 0) return MRHS_OK;
  MRHS_TRY(check_vec(basis, "basis"));
  MRHS_TRY(check_vec(in, project ? "F" : "C"));
  MRHS_TRY(check_vec(out, project ? "C" : "F"));
  const size_t es = dtype == MRHS_C128 ? 16 : 8;
  const size_t nF = es * (size_t)nblk * vb * nrhs, nC = es * (size_t)nblk * nbasis * nrhs;
  const size_t nB = es * (size_t)nblk * vb * nbasis;
  const size_t in_b = project ? nF : nC, out_b = project ? nC : nF;
  const char* o = (const char*)out;
  for (auto pr : {std::make_pair((const char*)in, in_b), std::make_pair((const char*)basis, nB)})
    if (o < pr.first + pr.second && pr.first < o + out_b)
      return fail(MRHS_ERR_INVALID_ARG, std::string(name) + ": output overlaps an input");
  return blocking(project, basis, in, out, nblk, vb, nbasis, nrhs, dtype, (cudaStream_t)stream);
}

int block_project(const void* basis, const void* F, void* C, int64_t n_blocks, int32_t v_block,
                  int32_t n_basis, int32_t nrhs, int32_t dtype, void* stream) {
  return blocking_common(true, basis, F, C, n_blocks, v_block, n_basis, nrhs, dtype, stream);
}

int block_promote(const void* basis, const void* C, void* F, int64_t n_blocks, int32_t v_block,
                  int32_t n_basis, int32_t nrhs, int32_t dtype, void* stream) {
  return blocking_common(false, basis, C, F, n_blocks, v_block, n_basis, nrhs, dtype, stream);
}

int coarsen_op(mrhs_op fine, const int32_t block[4], const void* basis, int32_t nbasis,
               const int8_t* disp, int32_t npts, void* A, void* stream) {
  MRHS_TRY(check_op(fine));
  MRHS_TRY(check_plain(fine));
  MRHS_TRY(check_prec(fine, MRHS_PREC_FP64));
  if (!block || !disp) return fail(MRHS_ERR_INVALID_ARG, "coarsen_op: null argument");
  MRHS_TRY(check_vec(basis, "basis"));
  MRHS_TRY(check_vec(A, "A"));
  int64_t Vc = 1, bvol = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (block[mu] < 1 || fine->L[mu] % block[mu] != 0)
      return fail(MRHS_ERR_INVALID_ARG, "coarsen_op: block must divide the fine lattice");
    if (fine->L[mu] / block[mu] < 3)
      return fail(MRHS_ERR_INVALID_ARG, "coarsen_op: every coarse extent must be >= 3");
    Vc *= fine->L[mu] / block[mu];
    bvol *= block[mu];
  }
  if (nbasis < 1 || nbasis > MRHS_MAX_RHS || nbasis > bvol * fine->nb)
    return fail(MRHS_ERR_INVALID_ARG, "coarsen_op: 1 <= n_basis <= min(64, v_block)");
  if (npts < 1 || npts > MRHS_MAX_PTS) return fail(MRHS_ERR_INVALID_ARG, "coarsen_op: npts 1..81");
  for (int p = 0; p < npts; ++p)
    for (int mu = 0; mu < 4; ++mu)
      if (disp[4 * p + mu] < -1 || disp[4 * p + mu] > 1)
        return fail(MRHS_ERR_INVALID_ARG, "coarsen_op: displacements must be in {-1,0,1}");
  const size_t ab = 16 * (size_t)Vc * npts * nbasis * nbasis;
  const size_t bb = 16 * (size_t)Vc * bvol * fine->nb * nbasis;
  const char* a = (const char*)A;
  const char* b = (const char*)basis;
  if (a < b + bb && b < a + ab) return fail(MRHS_ERR_INVALID_ARG, "coarsen_op: A overlaps basis");
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != fine->device) return fail(MRHS_ERR_INVALID_ARG, "operator lives on another device");
  return coarsen(fine, block, basis, nbasis, reinterpret_cast<const int8_t(*)[4]>(disp), npts, A,
                 (cudaStream_t)stream);
}

int coarse_solve_defl_cheby(mrhs_op op, int32_t prec, const void* U, const double* lambda,
                            int32_t n_ev, double lo, double hi, int32_t order, const void* B,
                            void* X, int32_t nrhs, void* stream) {
  MRHS_TRY(check_op(op));
  MRHS_TRY(check_plain(op));
  MRHS_TRY(check_prec(op, prec));
  MRHS_TRY(check_vec(B, "B"));
  MRHS_TRY(check_vec(X, "X"));
  if (nrhs < 1 || nrhs > MRHS_MAX_RHS) return fail(MRHS_ERR_INVALID_ARG, "nrhs must be in 1..64");
  if (!(lo > 0.0 && lo < hi)) return fail(MRHS_ERR_INVALID_ARG, "need 0 < lo < hi");
  if (order < 0 || order > 10000) return fail(MRHS_ERR_INVALID_ARG, "order");
  if (n_ev < 0 || n_ev > 65536) return fail(MRHS_ERR_INVALID_ARG, "n_ev must be in 0..65536");
  if (n_ev > 0) {
    MRHS_TRY(check_vec(U, "U"));
    if (!lambda) return fail(MRHS_ERR_INVALID_ARG, "lambda is null");
    for (int i = 0; i < n_ev; ++i)
      if (!(lambda[i] > 0.0) || !std::isfinite(lambda[i]))
        return fail(MRHS_ERR_INVALID_ARG, "lambda must be positive and finite");
    const size_t es = MRHS_PREC_IS_WIDE(prec) ? 16 : 8;
    const size_t ub = es * (size_t)op->V * op->nb * n_ev, vb = es * (size_t)op->V * op->nb * nrhs;
    const char* u = (const char*)U;
    for (const void* v : {B, (const void*)X}) {
      const char* c = (const char*)v;
      if (u < c + vb && c < u + ub) return fail(MRHS_ERR_INVALID_ARG, "U overlaps B or X");
    }
  }
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != op->device) return fail(MRHS_ERR_INVALID_ARG, "operator lives on another device");
  return defl_cheby(op, prec, U, lambda, n_ev, lo, hi, order, B, X, nrhs, (cudaStream_t)stream);
}

int block_cg_solve(mrhs_op op, const void* B, void* X, int32_t nrhs,
                   const mrhs_solve_params* params, mrhs_solve_info* info, void* stream) {
  MRHS_TRY(check_op(op));
  MRHS_TRY(check_plain(op));
  if (!params) return fail(MRHS_ERR_INVALID_ARG, "params is null");
  MRHS_TRY(check_vec(B, "B"));
  MRHS_TRY(check_vec(X, "X"));
  if (nrhs < 1 || nrhs > MRHS_MAX_RHS) return fail(MRHS_ERR_INVALID_ARG, "nrhs must be in 1..64");
  const mrhs_solve_params& p = *params;
  if (!(p.tol > 0.0) || p.maxiter < 1) return fail(MRHS_ERR_INVALID_ARG, "tol / maxiter");
  if (p.mode != MRHS_SOLVE_FP64 && p.mode != MRHS_SOLVE_MIXED && p.mode != MRHS_SOLVE_CG5D)
    return fail(MRHS_ERR_INVALID_ARG, "mode");
  if (p.recycle < 0 || p.recycle_max_blocks < 0)
    return fail(MRHS_ERR_INVALID_ARG, "recycle / recycle_max_blocks must be >= 0");
  MRHS_TRY(check_inner_tols(p));
  auto built = [&](int pr) { return (op->prec_mask & MRHS_PREC_BIT(pr)) != 0; };
  const bool fp64_ok = built(MRHS_PREC_FP64);
  const bool oz_ok = built(MRHS_PREC_OZ) && oz_supported(op, nrhs);
  if (p.mode == MRHS_SOLVE_CG5D) {
    mrhs_solve_params q = p;
    MRHS_TRY(resolve_fp64_prec(&q.fp64_prec, fp64_ok, oz_ok));
    if (q.krylov_prec < 0) q.krylov_prec = q.fp64_prec;
    if (q.krylov_prec != MRHS_PREC_FP64 && q.krylov_prec != MRHS_PREC_DF32 &&
        q.krylov_prec != MRHS_PREC_OZ)
      return fail(MRHS_ERR_INVALID_ARG, "CG5D runs the FP64, DF32 or OZ operator");
    if ((q.krylov_prec == MRHS_PREC_OZ && !oz_ok) || (q.krylov_prec != MRHS_PREC_OZ && !fp64_ok))
      return fail(MRHS_ERR_UNSUPPORTED, "CG5D: operator precision not built");
    if (q.precond) return fail(MRHS_ERR_INVALID_ARG, "CG5D takes no preconditioner");
    if (X == B) return fail(MRHS_ERR_INVALID_ARG, "X and B must differ");
    return cg5d(op, (const double2*)B, (double2*)X, nrhs, q, info, (cudaStream_t)stream);
  }
  mrhs_solve_params q = p;   // resolve the automatic precision choices
  auto fits = [&](int pr) {
    if (pr == MRHS_PREC_OZ) return oz_ok;
    return !MRHS_PREC_IS_TC(pr) || tc_supported(op, pr, nrhs) != 0;
  };
  MRHS_TRY(resolve_fp64_prec(&q.fp64_prec, fp64_ok, oz_ok));
  if (q.mode == MRHS_SOLVE_MIXED) {
    if (q.residual_prec < 0) q.residual_prec = oz_ok ? MRHS_PREC_OZ : MRHS_PREC_DF32;
    MRHS_TRY(check_residual_prec(q.residual_prec, fp64_ok, oz_ok));
    if (q.krylov_prec < 0)
      q.krylov_prec = (built(MRHS_PREC_TC32) && fits(MRHS_PREC_TC32)) ? MRHS_PREC_TC32 : MRHS_PREC_FP32;
    if (q.krylov_prec != MRHS_PREC_FP32 && q.krylov_prec != MRHS_PREC_TC32)
      return fail(MRHS_ERR_INVALID_ARG, "krylov_prec must be FP32 or TC32");
    if (!built(q.krylov_prec) || !fits(q.krylov_prec))
      return fail(MRHS_ERR_UNSUPPORTED, "mixed mode needs the FP32 or TC32 operator");
  }
  if (q.precond && q.precond_prec < 0) {
    const int order[] = {MRHS_PREC_FP16X, MRHS_PREC_FP16, MRHS_PREC_BF16, MRHS_PREC_TC32,
                         MRHS_PREC_FP32};
    q.precond_prec = q.mode == MRHS_SOLVE_FP64 ? q.fp64_prec : -1;
    if (q.mode == MRHS_SOLVE_MIXED)
      for (int pr : order)
        if (built(pr) && fits(pr)) { q.precond_prec = pr; break; }
  }
  const mrhs_solve_params& pp = q;
  if (pp.precond) {
    if (pp.precond_prec < 0 || pp.precond_prec >= MRHS_NUM_PREC)
      return fail(MRHS_ERR_INVALID_ARG, "precond_prec");
    if (!fits(pp.precond_prec))
      return fail(MRHS_ERR_UNSUPPORTED, "preconditioner precision does not fit this shape");
    if (!built(pp.precond_prec))
      return fail(MRHS_ERR_UNSUPPORTED, "preconditioner precision not built");
    if (pp.mode == MRHS_SOLVE_FP64 && pp.precond_prec != MRHS_PREC_FP64 &&
        pp.precond_prec != MRHS_PREC_OZ)
      return fail(MRHS_ERR_INVALID_ARG, "FP64 mode takes an FP64 (or OZ) preconditioner");
    if (pp.mode == MRHS_SOLVE_MIXED && MRHS_PREC_IS_WIDE(pp.precond_prec))
      return fail(MRHS_ERR_INVALID_ARG, "mixed mode takes a low-precision preconditioner");
    if (pp.cheb_order < 0) return fail(MRHS_ERR_INVALID_ARG, "cheb_order");
  }
  if (X == B) return fail(MRHS_ERR_INVALID_ARG, "X and B must differ");
  return solve(op, (const double2*)B, (double2*)X, nrhs, pp, info, (cudaStream_t)stream);
}

int mrhs_autotune(const mrhs_op* ops, int32_t n, int32_t prec, const int32_t* nrhs, int32_t reps,
                  mrhs_tune_result* out, void* stream) {
  if (!ops || !nrhs || n < 1 || n > MRHS_MAX_BATCH)
    return fail(MRHS_ERR_INVALID_ARG, "mrhs_autotune: arguments (1 <= n <= 16)");
  if (!MRHS_PREC_IS_TC(prec))
    return fail(MRHS_ERR_UNSUPPORTED, "only the tensor-core kernel has a tuned launch shape");
  int dev = 0;
  cudaGetDevice(&dev);
  for (int i = 0; i < n; ++i) {
    MRHS_TRY(check_op(ops[i]));
    MRHS_TRY(check_plain(ops[i]));
    MRHS_TRY(check_prec(ops[i], prec));
    if (ops[i]->device != dev) return fail(MRHS_ERR_INVALID_ARG, "operator on another device");
    if (nrhs[i] < 1 || nrhs[i] > MRHS_MAX_RHS) return fail(MRHS_ERR_INVALID_ARG, "nrhs[i]");
    for (int j = 0; j < i; ++j)
      if (ops[j] == ops[i]) return fail(MRHS_ERR_INVALID_ARG, "an operator appears twice");
  }
  return autotune(const_cast<mrhs_op_s* const*>(ops), n, prec, nrhs, reps, out,
                  (cudaStream_t)stream);
}

int mrhs_autotune_save(const char* path) {
  if (!path) return fail(MRHS_ERR_INVALID_ARG, "path");
  return tune_save(path);
}

int mrhs_autotune_load(const char* path) {
  if (!path) return fail(MRHS_ERR_INVALID_ARG, "path");
  return tune_load(path);
}

int64_t mrhs_autotune_entries(void) { return tune_entries(); }

void mrhs_autotune_clear(void) { tune_clear(); }

int mrhs_batch_apply(const mrhs_op* ops, int32_t n, int32_t prec, const void* const* X,
                     void* const* Y, const int32_t* nrhs, void* stream) {
  if (!ops || !X || !Y || !nrhs || n < 1 || n > MRHS_MAX_BATCH)
    return fail(MRHS_ERR_INVALID_ARG, "mrhs_batch_apply: arguments (1 <= n <= 16)");
  if (!MRHS_PREC_IS_TC(prec))
    return fail(MRHS_ERR_UNSUPPORTED, "batched applications run on the tensor cores only");
  int dev = 0;
  cudaGetDevice(&dev);
  for (int i = 0; i < n; ++i) {
    MRHS_TRY(check_op(ops[i]));
    MRHS_TRY(check_plain(ops[i]));
    MRHS_TRY(check_prec(ops[i], prec));
    MRHS_TRY(check_vec(X[i], "X[i]"));
    MRHS_TRY(check_vec(Y[i], "Y[i]"));
    if (ops[i]->device != dev) return fail(MRHS_ERR_INVALID_ARG, "operator on another device");
    if (nrhs[i] < 1 || nrhs[i] > MRHS_MAX_RHS) return fail(MRHS_ERR_INVALID_ARG, "nrhs[i]");
    for (int j = 0; j < i; ++j)
      if (ops[j] == ops[i]) return fail(MRHS_ERR_INVALID_ARG, "an operator appears twice (its input workspace is shared)");
  }
  return tc_apply_batch(const_cast<mrhs_op_s* const*>(ops), n, prec, X, Y, nrhs, nullptr,
                        (cudaStream_t)stream);
}

int mrhs_batch_solve(const mrhs_op* ops, int32_t n, const void* const* B, void* const* X,
                     const int32_t* nrhs, const mrhs_solve_params* params, mrhs_solve_info* info,
                     void* stream) {
  if (!ops || !B || !X || !nrhs || !params || n < 1 || n > MRHS_MAX_BATCH)
    return fail(MRHS_ERR_INVALID_ARG, "mrhs_batch_solve: arguments (1 <= n <= 16)");
  mrhs_solve_params q = *params;
  bool batched = q.mode == MRHS_SOLVE_MIXED && q.precond;
  int dev = 0;
  cudaGetDevice(&dev);
  for (int i = 0; i < n; ++i) {
    MRHS_TRY(check_op(ops[i]));
    MRHS_TRY(check_plain(ops[i]));
    MRHS_TRY(check_vec(B[i], "B[i]"));
    MRHS_TRY(check_vec(X[i], "X[i]"));
    if (ops[i]->device != dev) return fail(MRHS_ERR_INVALID_ARG, "operator on another device");
    if (nrhs[i] < 1 || nrhs[i] > MRHS_MAX_RHS) return fail(MRHS_ERR_INVALID_ARG, "nrhs[i]");
    for (int j = 0; j < i; ++j)
      if (ops[j] == ops[i]) return fail(MRHS_ERR_INVALID_ARG, "an operator appears twice");
    const uint32_t m = ops[i]->prec_mask;
    const bool oz_i = (m & MRHS_PREC_BIT(MRHS_PREC_OZ)) && oz_supported(ops[i], nrhs[i]);
    if (!(m & MRHS_PREC_BIT(MRHS_PREC_FP64)) && !oz_i)
      return fail(MRHS_ERR_UNSUPPORTED, "the FP64 or the OZ operator is needed");
    if (nrhs[i] > 32 || !(m & MRHS_PREC_BIT(MRHS_PREC_TC32))) batched = false;
  }
  // the batched path: TC32 in the Krylov loop and a tensor-core preconditioner
  // shared by all problems; otherwise each problem is solved in turn
  if (batched) {
    bool oz = true, f64 = true;
    for (int i = 0; i < n; ++i) {
      oz = oz && (ops[i]->prec_mask & MRHS_PREC_BIT(MRHS_PREC_OZ)) && oz_supported(ops[i], nrhs[i]);
      f64 = f64 && (ops[i]->prec_mask & MRHS_PREC_BIT(MRHS_PREC_FP64));
    }
    MRHS_TRY(resolve_fp64_prec(&q.fp64_prec, f64, oz));
    if (q.residual_prec < 0) q.residual_prec = oz ? MRHS_PREC_OZ : MRHS_PREC_DF32;
    MRHS_TRY(check_residual_prec(q.residual_prec, f64, oz));
    if (q.krylov_prec < 0) q.krylov_prec = MRHS_PREC_TC32;
    if (q.precond_prec < 0) {
      const int order[] = {MRHS_PREC_FP16X, MRHS_PREC_FP16, MRHS_PREC_BF16, MRHS_PREC_TC32};
      for (int pr : order) {
        bool all = true;
        for (int i = 0; i < n; ++i) all = all && (ops[i]->prec_mask & MRHS_PREC_BIT(pr));
        if (all) { q.precond_prec = pr; break; }
      }
    }
    batched = q.krylov_prec == MRHS_PREC_TC32 && q.precond_prec >= MRHS_PREC_BF16;
    for (int i = 0; i < n && batched; ++i)
      batched = (ops[i]->prec_mask & MRHS_PREC_BIT(q.precond_prec)) != 0;
  }
  if (batched) {
    if (!(q.tol > 0.0) || q.maxiter < 1 || q.cheb_order < 0)
      return fail(MRHS_ERR_INVALID_ARG, "tol / maxiter / cheb_order");
    MRHS_TRY(check_inner_tols(q));
    for (int i = 0; i < n; ++i)
      if (B[i] == X[i]) return fail(MRHS_ERR_INVALID_ARG, "X and B must differ");
    return solve_batch(const_cast<mrhs_op_s* const*>(ops), n, (const double2* const*)B,
                       (double2* const*)X, nrhs, q, info, (cudaStream_t)stream);
  }
  int worst = MRHS_OK;
  for (int i = 0; i < n; ++i) {
    const int st = block_cg_solve(ops[i], B[i], X[i], nrhs[i], params, info ? info + i : nullptr,
                                  stream);
    if (st != MRHS_OK && st != MRHS_ERR_NOT_CONVERGED) return st;
    if (st != MRHS_OK && worst == MRHS_OK) worst = st;
  }
  return worst;
}

void mrhs_solve_params_default(mrhs_solve_params* p, int32_t mode) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->tol = 1e-8;
  p->maxiter = 5000;
  p->mode = mode;
  p->precond = mode == MRHS_SOLVE_MIXED ? 1 : 0;
  p->precond_prec = -1;
  p->krylov_prec = -1;
  p->use_graph = 1;
  p->residual_prec = -1;
  p->cheb_order = 8;
  p->cheb_lo = 0.0;
  p->cheb_hi = 0.0;
  p->inner_tol = 1e-3;
  p->max_cycles = 12;
  p->check_every = 4;
  p->breakdown_tau = 1e-12;
  p->recycle = 0;
  p->recycle_max_blocks = 0;
  p->fp64_prec = -1;
  p->inner_tol_later = mode == MRHS_SOLVE_MIXED ? 1e-2 : 0.0;
}

}  // extern "C"
