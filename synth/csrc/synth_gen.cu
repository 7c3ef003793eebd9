// Device twin of synth/philox.py and synth/coarse.py: Philox-4x32-10
// (Salmon et al., SC'11) and the same seeded recipe for coarse operators and
// vectors, for lattices too large to generate on the host.  Random draws and
// index bookkeeping only.  Counter layout (element, site, point/row, stream);
// key (seed mod 2^32, seed >> 32).
#include <stdint.h>

namespace {

__device__ __forceinline__ void philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// standard complex normal, Box-Muller on the first two words
__device__ __forceinline__ double2 cnormal(uint32_t e, uint32_t site, uint32_t p, uint32_t stream,
                                           uint64_t seed) {
  uint32_t c[4] = {e, site, p, stream};
  philox(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const double u1 = ((double)c[0] + 0.5) * 2.3283064365386963e-10;   // 2^-32
  const double u2 = ((double)c[1] + 0.5) * 2.3283064365386963e-10;
  const double rho = sqrt(-log(u1));
  const double th = (2.0 * 3.141592653589793) * u2;
  return make_double2(rho * cos(th), rho * sin(th));
}

__global__ void k_gen_op(double2* A, int64_t V, int nb, int npts, int L0, int L1, int L2, int L3,
                         const int8_t* __restrict__ disp, const int32_t* __restrict__ pair,
                         uint64_t seed, double shift) {
  const int64_t per_site = (int64_t)npts * nb * nb;
  const int64_t total = V * per_site;
  const double inv = 1.0 / sqrt((double)nb);
  const int L[4] = {L0, L1, L2, L3};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = i / per_site;
    const int rem = (int)(i % per_site);
    const int p = rem / (nb * nb), a = (rem / nb) % nb, b = rem % nb;
    const int8_t* d = disp + 4 * p;
    int first = 0;
    for (int mu = 0; mu < 4; ++mu)
      if (d[mu] != 0) { first = d[mu]; break; }
    double2 v;
    if (first == 0) {
      double2 g1 = cnormal((uint32_t)(a * nb + b), (uint32_t)x, 0u, 2u, seed);
      double2 g2 = cnormal((uint32_t)(b * nb + a), (uint32_t)x, 0u, 2u, seed);
      // explicit roundings: a contracted multiply-add would round the [a][b]
      // and [b][a] entries differently and break exact Hermiticity
      g1.x = __dmul_rn(g1.x, inv); g1.y = __dmul_rn(g1.y, inv);
      g2.x = __dmul_rn(g2.x, inv); g2.y = __dmul_rn(g2.y, inv);
      v = make_double2(0.5 * __dadd_rn(g1.x, g2.x), 0.5 * __dsub_rn(g1.y, g2.y));
      if (a == b) v.x += shift;
    } else if (first > 0) {
      v = cnormal((uint32_t)(a * nb + b), (uint32_t)x, (uint32_t)p, 1u, seed);
      v.x *= inv; v.y *= inv;
    } else {
      int64_t r = x, y = 0, c[4];
      for (int mu = 0; mu < 4; ++mu) { c[mu] = r % L[mu]; r /= L[mu]; }
      for (int mu = 3; mu >= 0; --mu) y = y * L[mu] + (c[mu] + d[mu] + L[mu]) % L[mu];
      v = cnormal((uint32_t)(b * nb + a), (uint32_t)y, (uint32_t)pair[p], 1u, seed);
      v.x *= inv; v.y = -(v.y * inv);
    }
    A[i] = v;
  }
}

__global__ void k_gen_vec(double2* X, int64_t V, int nb, int R, uint64_t seed, uint32_t stream) {
  const int64_t total = V * nb * R;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i % R);
    const int a = (int)((i / R) % nb);
    const int64_t x = i / ((int64_t)R * nb);
    X[i] = cnormal((uint32_t)r, (uint32_t)x, (uint32_t)a, stream, seed);
  }
}

__global__ void k_philox_words(uint32_t* out, int64_t n, uint32_t c1, uint32_t c2, uint32_t c3,
                               uint64_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c[4] = {(uint32_t)i, c1, c2, c3};
    philox(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    for (int k = 0; k < 4; ++k) out[4 * i + k] = c[k];
  }
}

}  // namespace

extern "C" {

int synth_gen_op(void* A, int64_t V, int nb, int npts, const int32_t* L, const int8_t* disp_dev,
                 const int32_t* pair_dev, uint64_t seed, double shift, void* stream) {
  k_gen_op<<<148 * 16, 256, 0, (cudaStream_t)stream>>>((double2*)A, V, nb, npts, L[0], L[1], L[2],
                                                         L[3], disp_dev, pair_dev, seed, shift);
  return (int)cudaGetLastError();
}

int synth_gen_vec(void* X, int64_t V, int nb, int R, uint64_t seed, uint32_t stream_id,
                  void* stream) {
  k_gen_vec<<<148 * 16, 256, 0, (cudaStream_t)stream>>>((double2*)X, V, nb, R, seed, stream_id);
  return (int)cudaGetLastError();
}

int synth_philox_words(void* out, int64_t n, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t seed,
                       void* stream) {
  k_philox_words<<<148 * 4, 256, 0, (cudaStream_t)stream>>>((uint32_t*)out, n, c1, c2, c3, seed);
  return (int)cudaGetLastError();
}

}  // extern "C"
