// Row gather and scatter for the ghost-zone exchange of a decomposed lattice
// (Sec. 2.6, "Applying the coarse operator": the input vector of the coarse
// operator lives on the padded local volume; its boundary layers are
// exchanged one dimension after the other, each exchange carrying the ghost
// zones already filled, so the corners of the 81-point stencil arrive through
// nearest-neighbour messages only).
//
// A "row" is everything one site holds: nb x nrhs complex values of a vector
// (or npts x nb x nb coefficients), row_bytes bytes, a multiple of 16.  The
// host side (domain.py) lists, per dimension, the padded-site indices of the
// faces to send and of the ghost layers to fill; these two kernels copy
// between such index lists and contiguous message buffers.  Rows move in
// 16-byte units, consecutive threads on consecutive units of a row.
#include "internal.cuh"

namespace mrhs {
namespace {

// gather: dst[i] = src[idx[i]];  scatter: dst[idx[i]] = src[i].  An index
// outside [0, rows) of the indexed array is skipped (no access).
template <bool kGather>
__global__ void k_rows(const uint4* __restrict__ src, uint4* __restrict__ dst,
                       const int64_t* __restrict__ idx, int64_t n, int64_t rows, int64_t per) {
  const int64_t units = n * per;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < units;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = u / per, k = u - i * per;
    const int64_t j = __ldg(&idx[i]);
    if (j < 0 || j >= rows) continue;
    if (kGather) dst[i * per + k] = src[j * per + k];
    else dst[j * per + k] = src[i * per + k];
  }
}

int rows_common(bool gather, const void* src, void* dst, const int64_t* idx, int64_t n,
                int64_t rows, int64_t row_bytes, cudaStream_t s) {
  if (n < 0 || rows < 0 || row_bytes < 16 || row_bytes % 16)
    return fail(MRHS_ERR_INVALID_ARG, "rows: n, rows >= 0 and row_bytes a positive multiple of 16");
  if (n == 0) return MRHS_OK;
  if (!src || !dst || !idx) return fail(MRHS_ERR_INVALID_ARG, "rows: null pointer");
  if (((uintptr_t)src | (uintptr_t)dst) & 15u)
    return fail(MRHS_ERR_INVALID_ARG, "rows: src and dst must be 16-byte aligned");
  if ((uintptr_t)idx & 7u) return fail(MRHS_ERR_INVALID_ARG, "rows: idx must be 8-byte aligned");
  const int64_t per = row_bytes / 16;
  const int64_t units = n * per;
  int64_t grid = (units + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (grid > cap) grid = cap;
  if (gather) {
    k_rows<true><<<(unsigned)grid, 256, 0, s>>>((const uint4*)src, (uint4*)dst, idx, n, rows, per);
  } else {
    k_rows<false><<<(unsigned)grid, 256, 0, s>>>((const uint4*)src, (uint4*)dst, idx, n, rows, per);
  }
  count_launch();
  MRHS_CUDA_TRY(cudaGetLastError());
  return MRHS_OK;
}

}  // namespace
}  // namespace mrhs

using namespace mrhs;

extern "C" int mrhs_gather_rows(const void* src, int64_t src_rows, const int64_t* idx, int64_t n,
                                void* dst, int64_t row_bytes, void* stream) {
  return rows_common(true, src, dst, idx, n, src_rows, row_bytes, (cudaStream_t)stream);
}

extern "C" int mrhs_scatter_rows(const void* src, int64_t n, const int64_t* idx, void* dst,
                                 int64_t dst_rows, int64_t row_bytes, void* stream) {
  return rows_common(false, src, dst, idx, n, dst_rows, row_bytes, (cudaStream_t)stream);
}
