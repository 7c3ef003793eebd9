// Device-side small Hermitian factorisation shared by the factor entry point
// and the block CG phase kernels (one CTA, FP64, r <= 64).
#pragma once
#include "internal.cuh"

namespace mrhs {

// Factor the leading k_in x k_in block of the Hermitian part of G (row
// stride ldg) as described in small.cu.  sA, sS, sW: r*r shared scratch each;
// perm: r shared ints.  S_out / W_out (r x r, caller order) may be null.
// Returns the rank k on every thread.  Must be called by the whole CTA.
__device__ inline int factor_block(const double2* __restrict__ G, int ldg, int r, int k_in, double tau,
                            double2* sA, double2* sS, double2* sW, int* perm, double2* S_out,
                            double2* W_out) {
  const int tid = threadIdx.x, T = blockDim.x;
  __shared__ double s_dmax, s_piv_d, s_sjj, s_isjj;
  __shared__ int s_fail, s_piv, s_rank;
  for (int pass = 0; pass < 2; ++pass) {
    const bool pivoting = pass == 1;
    for (int e = tid; e < r * r; e += T) {
      const int i = e / r, j = e % r;
      double2 v = make_double2(0.0, 0.0);
      if (i < k_in && j < k_in) {
        const double2 a = G[i * ldg + j], b = G[j * ldg + i];
        v = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
      }
      sA[e] = v;
      sS[e] = make_double2(0.0, 0.0);
    }
    for (int i = tid; i < r; i += T) perm[i] = i;
    __syncthreads();
    if (tid == 0) {
      double m = 0.0;
      for (int i = 0; i < k_in; ++i) m = fmax(m, sA[i * r + i].x);
      s_dmax = m;
      s_fail = 0;
      s_rank = k_in;
    }
    __syncthreads();
    for (int j = 0; j < k_in; ++j) {
      if (tid == 0) {
        int p = j;
        double d = sA[j * r + j].x;
        if (pivoting)
          for (int i = j + 1; i < k_in; ++i)
            if (sA[i * r + i].x > d) { d = sA[i * r + i].x; p = i; }
        s_piv = p;
        s_piv_d = d;
        if (!(d > tau * s_dmax) || !isfinite(d)) {
          s_fail = 1;
          s_rank = j;
        } else {
          // the pivot's square root and reciprocal, once per column: both
          // take many instructions on B300's FP64 pipe
          s_sjj = sqrt(d);
          s_isjj = 1.0 / s_sjj;
        }
      }
      __syncthreads();
      if (s_fail) break;
      const int p = s_piv;
      if (p != j) {   // symmetric swap of rows/cols j, p of A; columns of S (rows < j)
        for (int i = tid; i < r; i += T) {
          double2 t = sA[j * r + i]; sA[j * r + i] = sA[p * r + i]; sA[p * r + i] = t;
        }
        __syncthreads();
        for (int i = tid; i < r; i += T) {
          double2 t = sA[i * r + j]; sA[i * r + j] = sA[i * r + p]; sA[i * r + p] = t;
        }
        for (int i = tid; i < j; i += T) {
          double2 t = sS[i * r + j]; sS[i * r + j] = sS[i * r + p]; sS[i * r + p] = t;
        }
        if (tid == 0) { int t = perm[j]; perm[j] = perm[p]; perm[p] = t; }
        __syncthreads();
      }
      const double sjj = s_sjj, isjj = s_isjj;
      for (int i = j + tid; i < k_in; i += T) {
        const double2 a = sA[j * r + i];
        sS[j * r + i] = (i == j) ? make_double2(sjj, 0.0) : make_double2(a.x * isjj, a.y * isjj);
      }
      __syncthreads();
      const int m = k_in - j - 1;
      for (int e = tid; e < m * m; e += T) {
        const int i = j + 1 + e / m, c = j + 1 + e % m;
        const double2 si = sS[j * r + i], sc = sS[j * r + c];
        // A_ic -= conj(S_ji) S_jc
        double2 a = sA[i * r + c];
        a.x -= si.x * sc.x + si.y * sc.y;
        a.y -= si.x * sc.y - si.y * sc.x;
        sA[i * r + c] = a;
      }
      __syncthreads();
    }
    __syncthreads();
    if (!s_fail || pivoting) break;
    __syncthreads();
  }
  const int k = s_rank;
  // W = (leading k x k of S)^-1, column c by back substitution, with the
  // reciprocals of S's real diagonal formed once (in sA's first row, free now)
  double* inv_d = reinterpret_cast<double*>(sA);
  for (int i = tid; i < k; i += T) inv_d[i] = 1.0 / sS[i * r + i].x;
  __syncthreads();
  for (int e = tid; e < r * r; e += T) sW[e] = make_double2(0.0, 0.0);
  __syncthreads();
  if (T >= 8 * r && (T & 31) == 0) {
    // eight lanes per column c (c = tid / 8): row i of the column is
    // -(sum_{l = i+1..c} S[i][l] W[l][c]) / S[i][i]; the lanes split the sum
    // over l and combine it by shuffles in a fixed order, row by row from
    // the diagonal up (every lane of a warp runs the same r - 1 row steps)
    const int c = tid >> 3, part = tid & 7;
    const bool live = c < k;          // c < k <= r: lanes past the last column add zeros
    if (live && part == 0) sW[c * r + c] = make_double2(inv_d[c], 0.0);
    __syncwarp();
    if ((tid >> 5) * 32 < 8 * r) {     // whole warps: the shuffles take every lane
      for (int i = r - 2; i >= 0; --i) {
        double2 acc = make_double2(0.0, 0.0);
        if (live && i < c)
          for (int l = i + 1 + part; l <= c; l += 8) acc = cfma(sS[i * r + l], sW[l * r + c], acc);
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
          acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
          acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        if (live && i < c && part == 0) {
          const double inv = inv_d[i];
          sW[i * r + c] = make_double2(-acc.x * inv, -acc.y * inv);
        }
        __syncwarp();
      }
    }
  } else {
    for (int c = tid; c < r; c += T) {
      if (c < k) {
        sW[c * r + c] = make_double2(inv_d[c], 0.0);
        for (int i = c - 1; i >= 0; --i) {
          double2 acc = make_double2(0.0, 0.0);
          for (int l = i + 1; l <= c; ++l) acc = cfma(sS[i * r + l], sW[l * r + c], acc);
          const double inv = inv_d[i];
          sW[i * r + c] = make_double2(-acc.x * inv, -acc.y * inv);
        }
      }
    }
  }
  __syncthreads();
  // scatter back to the caller's column order: S_out[j][perm[c]] = S[j][c],
  // W_out[perm[i]][c] = W[i][c]
  if (S_out)
    for (int e = tid; e < r * r; e += T) {
      const int j = e / r, c = e % r;
      S_out[j * r + perm[c]] = (j < k) ? sS[j * r + c] : make_double2(0.0, 0.0);
    }
  if (W_out)
    for (int e = tid; e < r * r; e += T) {
      const int i = e / r, c = e % r;
      W_out[perm[i] * r + c] = (i < k && c < k) ? sW[i * r + c] : make_double2(0.0, 0.0);
    }
  __syncthreads();
  return k;
}

size_t factor_smem_bytes(int r);

}  // namespace mrhs
