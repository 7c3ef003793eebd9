// Internal declarations of libmrhs (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "mrhs.h"

namespace mrhs {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

#define MRHS_CUDA_TRY(expr)                                                        \
  do {                                                                             \
    cudaError_t _e = (expr);                                                       \
    if (_e != cudaSuccess)                                                         \
      return ::mrhs::fail(MRHS_ERR_CUDA, std::string(#expr) + ": " +              \
                                             cudaGetErrorString(_e));             \
  } while (0)

#define MRHS_TRY(expr)          \
  do {                          \
    int _s = (expr);            \
    if (_s != MRHS_OK) return _s; \
  } while (0)

// ---------------------------------------------------------------- complex
__host__ __device__ inline double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 cfma(double2 a, double2 b, double2 c) {  // a*b + c
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__host__ __device__ inline double2 cfma_conj(double2 a, double2 b, double2 c) {  // conj(a)*b + c
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));
}
__host__ __device__ inline float2 cfma(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__host__ __device__ inline float2 cfma_conj(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(-a.y, b.x, c.y)));
}
template <typename C> struct real_of;
template <> struct real_of<double2> { using type = double; };
template <> struct real_of<float2> { using type = float; };
template <typename C> __host__ __device__ inline C czero();
template <> __host__ __device__ inline double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <> __host__ __device__ inline float2 czero<float2>() { return make_float2(0.f, 0.f); }

// ---------------------------------------------------------------- operator
struct TcImage {             // tensor-core packed coefficients (BF16/FP16)
  void* codes = nullptr;     // see op_tc.cu for the layout
  float* scale = nullptr;    // [V] power-of-two site scales
  float* diag = nullptr;     // [V] mean real self diagonal d_x (FP32)
  size_t bytes = 0;
};

struct OzImage {             // digit-sliced coefficients (op_oz.cu)
  void* digits = nullptr;    // [V][npts][nb16/16] slabs of 8 fp16 digit tiles
  double* scale = nullptr;   // [V] power-of-two site scales s_x
  double* diag = nullptr;    // [V] mean real self diagonal d_x (FP64)
  size_t bytes = 0;
};

// CUDA-event timing of an operator's main kernel, one (start, stop) pair per
// launch while enabled; read and cleared by mrhs_op_kernel_time.
struct KernelTimer {
  bool on = false;
  std::vector<cudaEvent_t> ev;
  size_t used = 0;
};

// Launch shape of the tensor-core operator (pps <= 0: built-in default).
struct TcTune {
  int pps = 0;           // stencil points per pipeline stage
  int ctas_per_sm = 1;   // CTAs per SM (each with its own ring)
  int max_stages = 32;   // ring depth cap
};

// A Chebyshev recurrence step carried out in the epilogue of the tensor-core
// operator (op_tc.cu, ProbDesc): with W = H X (not stored),
//   mode 1:  Tout = a W + b X,           P = c0 X + c Tout
//   mode 2:  Tout = 2 (a W + b X) - Tp,  P = P + c Tout
// complex64 vectors; Tout may be Tp, never X.
struct ChebFuse {
  int mode = 0;
  float a = 0.f, b = 0.f, c = 0.f, c0 = 0.f;
  void* Tout = nullptr;
  const void* Tp = nullptr;
  void* P = nullptr;
  bool colmax_next = false;   // accumulate Tout's column maxima for the next application
  bool colmax_ready = false;  // this application's input maxima are accumulated already
};

struct Workspace {           // grow-only device scratch
  void* ptr = nullptr;
  size_t bytes = 0;
  int ensure(size_t need);
  void release();
};

}  // namespace mrhs

struct mrhs_op_s {
  int32_t L[4];
  int32_t nb, npts;
  int64_t V;
  // input halo (mrhs_op_create_halo): the input vectors live on the padded
  // lattice Lin = L + 2 halo (halo[mu] in {0, 1}; no wrap in a padded
  // dimension, periodic wrap in the others), Vin sites; the output on L.
  // Without a halo Lin = L and Vin = V.
  int32_t halo[4] = {0, 0, 0, 0};
  int32_t Lin[4] = {0, 0, 0, 0};
  int64_t Vin = 0;
  int8_t disp[MRHS_MAX_PTS][4];
  int device;
  uint32_t prec_mask;
  int32_t* nbr_fwd = nullptr;   // [npts][V]  x + delta_p
  int32_t* nbr_bwd = nullptr;   // [npts][V]  x - delta_p
  double2* a64 = nullptr;       // [V][npts][nb][nb]
  float2* a32 = nullptr;        // [V][npts][nb][nb]
  mrhs::TcImage tc[3];          // BF16, FP16 (also FP16X), TC32: forward stencil
  mrhs::TcImage tc_dag[3];      // the same for the daggered stencil (on demand)
  mrhs::OzImage oz;             // digit-sliced image, forward stencil
  mrhs::OzImage oz_dag;         // the same for the daggered stencil (on demand)
  mrhs::Workspace ws_xpack;     // packed input vectors for the tensor path
  mrhs::Workspace ws_ozpack;    // input digits of the digit-sliced operator
  mrhs::Workspace ws_defl;      // deflated Chebyshev solve: Grams, B_perp, p(H) B_perp
  mrhs::Workspace ws_coarsen;   // coarsening: phased basis, M phi, blocked copy, T
  mrhs::Workspace ws_cheb;      // Chebyshev recurrence vectors
  mrhs::Workspace ws_small;     // column scales etc.
  mrhs::Workspace ws_solve;     // block CG vectors and state
  // search blocks kept across the mixed solve's refinement cycles (solver.cu):
  // one device allocation of rc_slot_bytes per slot, their addresses in the
  // device table rc_table, the matching (D^dagger H D)^-1 in ws_rcn, and the
  // device counters rc_ctr = {next slot, block ticket, slots available}
  std::vector<void*> rc_slots;
  size_t rc_slot_bytes = 0;
  void** rc_table = nullptr;
  int32_t* rc_ctr = nullptr;
  mrhs::Workspace ws_rcn;
  mrhs::KernelTimer timer[MRHS_NUM_PREC];   // per precision
  double lam_max[MRHS_NUM_PREC] = {};   // cached power-method estimates
  bool herm = false;                 // A_q(x + delta_p) = A_p(x)^dagger exactly (q: -p), all p
  bool pairable = false;             // the same for every hop pair (p != 0)
  int8_t herm_mode = 0;              // point-pair tile reading: 0 off (default), 1 all
                                     // tensor-core forms, 2 TC32 only
  int32_t herm_nf = 0;               // points with a positive first displacement
  int8_t herm_f[MRHS_MAX_PTS / 2];   // ... their indices
  mrhs::TcTune tc_tune;              // tensor-core launch shape
  bool tc_set = false;               // tc_tune set explicitly
};

namespace mrhs {

void count_launch();
int64_t launch_count();
void add_launches(int64_t n);   // kernels launched by a graph replay
void timer_mark(mrhs_op_s* op, int prec, cudaStream_t s);   // call before and after

// op_simt.cu
int simt_apply(mrhs_op_s* op, int prec, bool dag, const void* X, void* Y, int nrhs,
               cudaStream_t s);
// op_tc.cu
int tc_build(mrhs_op_s* op, int prec, bool dag, const double2* A, cudaStream_t s);
unsigned tc_read_and_clear_error();
int tc_set_wait_limit(unsigned long long ns);
int tc_apply_batch(mrhs_op_s* const* ops, int n, int prec, const void* const* X,
                   void* const* Y, const int32_t* nrhs, const int32_t* active, cudaStream_t s,
                   const TcTune* force = nullptr, const ChebFuse* fuse = nullptr);
// launch-shape cache (tune.cu)
bool tune_lookup(mrhs_op_s* const* ops, const int32_t* nrhs, int n, int prec, TcTune* out);
int autotune(mrhs_op_s* const* ops, int n, int prec, const int32_t* nrhs, int reps,
             mrhs_tune_result* res, cudaStream_t s);
int64_t tune_entries();
void tune_clear();
int tune_save(const char* path);
int tune_load(const char* path);
int tc_apply(mrhs_op_s* op, int prec, bool dag, const void* X, void* Y, int nrhs,
             cudaStream_t s);
int tc_supported(const mrhs_op_s* op, int prec, int nrhs);
// op_oz.cu
int oz_build(mrhs_op_s* op, bool dag, const double2* A, cudaStream_t s);
int oz_apply(mrhs_op_s* op, bool dag, const void* X, void* Y, int nrhs, cudaStream_t s);
int oz_supported(const mrhs_op_s* op, int nrhs);
unsigned oz_read_and_clear_error();
int oz_set_wait_limit(unsigned long long ns);
// blas.cu
int gram(const void* X, const void* Y, double2* G, int64_t N, int rx, int ry, int dtype,
         cudaStream_t s);
int axpy(void* Y, const void* X, const double2* M, double beta, int64_t N, int rin, int rout,
         int dtype, cudaStream_t s, int64_t ldx = 0);   // ldx: X's row stride (0: rin)
// blas_tc.cu: complex64 Gram and block update on the tensor cores
extern int g_block_tc_mode;   // 0: SIMT kernels only, 1: tensor cores where they apply
bool gram_tc_applies(const void* X, const void* Y, int64_t N, int rx, int ry, int dtype,
                     int64_t ldx);
int gram_tc_partial(const void* X, const void* Y, double2* part, int64_t N, int rx, int ry,
                    int64_t max_blocks, int* nblk_out, cudaStream_t s);
bool update_tc_applies(const void* Out, const void* X, const void* Add, int64_t N, int rin,
                       int rout, int dtype, int64_t ldx);
int update_tc(void* Out, const void* X, const void* Add, const double2* M, int mode, double beta,
              int64_t N, int rin, int rout, cudaStream_t s);
int btc_set_wait_limit(unsigned long long ns);
unsigned btc_read_and_clear_error();
// blocking_tc.cu: complex64 block project / promote on the tensor cores
bool blocking_tc_applies(const void* basis, const void* in, const void* out, int64_t nblk,
                         int vb, int nbasis, int R, int dtype);
int blocking_tc(bool project, const void* basis, const void* in, void* out, int64_t nblk, int vb,
                int nbasis, int R, cudaStream_t s);
unsigned bltc_read_and_clear_error();
// small.cu
int factor(const double2* G, double2* S, double2* W, int32_t* rank, int r, double tau,
           cudaStream_t s);
int gram_ws(const void* X, const void* Y, double2* G, int64_t N, int rx, int ry, int dtype,
            double2* part, cudaStream_t s);
size_t gram_workspace_bytes(int64_t N, int rx, int ry);
int gram_ws_capped(const void* X, const void* Y, double2* G, int64_t N, int rx, int ry, int dtype,
                   double2* part, int64_t max_entries, cudaStream_t s,
                   int64_t ldx = 0);   // ldx: X's row stride (0: rx)

// solver.cu
int solve(mrhs_op_s* op, const double2* B, double2* X, int R, const mrhs_solve_params& p,
          mrhs_solve_info* info, cudaStream_t s);
int cg5d(mrhs_op_s* op, const double2* B, double2* X, int R, const mrhs_solve_params& p,
         mrhs_solve_info* info, cudaStream_t s);
int cheby(mrhs_op_s* op, int prec, double lo, double hi, int order, const void* X, void* P,
          int R, cudaStream_t s);
int defl_cheby(mrhs_op_s* op, int prec, const void* U, const double* lam_host, int n_ev,
               double lo, double hi, int order, const void* B, void* X, int R, cudaStream_t s);
int blocking(bool project, const void* basis, const void* in, void* out, int64_t nblk, int vb,
             int nbasis, int R, int dtype, cudaStream_t s);
int coarsen(mrhs_op_s* op, const int32_t* block, const void* basis, int nbasis,
            const int8_t (*disp)[4], int npts, void* A_out, cudaStream_t s);
int lambda_max(mrhs_op_s* op, int prec, int iters, cudaStream_t s, double* lam);
void recycle_release(mrhs_op_s* op);   // frees the kept search blocks
int solve_batch(mrhs_op_s* const* ops, int n, const double2* const* B, double2* const* X,
                const int32_t* nrhs, const mrhs_solve_params& p, mrhs_solve_info* infos,
                cudaStream_t s);

// grad.cu
int outer(const mrhs_op_s* op, const void* G, const void* X, double2* GA, double alpha, int R,
          int dtype, cudaStream_t s);

// generic apply dispatch (api.cu)
int op_apply(mrhs_op_s* op, int prec, bool dag, const void* X, void* Y, int nrhs,
             cudaStream_t s);

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
int num_sms();

}  // namespace mrhs
