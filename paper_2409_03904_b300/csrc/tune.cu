// Launch-shape autotuner for the tensor-core operator.
//
// The tcgen05 kernel has three free parameters that change its speed but not
// its result: stencil points per pipeline stage (the size of each bulk copy),
// CTAs per SM (one or two rings per SM) and the ring depth.  The best choice
// depends on the problem shape (V, nb, stencil, nrhs) and the precision form,
// so it is measured once per shape and kept in a process-wide cache that every
// later launch of that shape consults.  A batch of several problems is tuned
// as a whole under the list of its members' keys.
//
// Candidates are timed with CUDA events on the caller's stream over a few
// launches each; every candidate's output is compared bit for bit with the
// first one's (the per-site MMA order does not depend on the launch shape), so
// a tuning run is also a self-check of the kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace mrhs {
namespace {

using KeyItem = std::array<int64_t, 6>;   // SMs, V, nb, npts, nrhs, prec
using Key = std::vector<KeyItem>;

struct Entry {
  TcTune t;
  double ms = 0;
};

std::mutex g_mu;
std::map<Key, Entry>& cache() {
  static std::map<Key, Entry> c;
  return c;
}

Key make_key(mrhs_op_s* const* ops, const int32_t* nrhs, int n, int prec) {
  Key k(n);
  const int sms = num_sms();
  for (int i = 0; i < n; ++i)
    k[i] = {sms, ops[i]->V, ops[i]->nb, ops[i]->npts, nrhs[i], prec};
  return k;
}

// deterministic fill in [-1, 1) (integer hash of the index)
__global__ void k_fill(float2* v, int64_t n, uint32_t salt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t h = ((uint64_t)i + ((uint64_t)salt << 40)) * 0x9E3779B97F4A7C15ull;
    h ^= h >> 29;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 32;
    v[i] = make_float2((float)((double)(h & 0xFFFFFF) / 8388608.0 - 1.0),
                       (float)((double)((h >> 24) & 0xFFFFFF) / 8388608.0 - 1.0));
  }
}

__global__ void k_differs(const uint32_t* a, const uint32_t* b, int64_t n, unsigned* flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (a[i] != b[i]) *flag = 1u;
}

}  // namespace

bool tune_lookup(mrhs_op_s* const* ops, const int32_t* nrhs, int n, int prec, TcTune* out) {
  const Key k = make_key(ops, nrhs, n, prec);
  std::lock_guard<std::mutex> g(g_mu);
  auto it = cache().find(k);
  if (it == cache().end()) return false;
  *out = it->second.t;
  return true;
}

int autotune(mrhs_op_s* const* ops, int n, int prec, const int32_t* nrhs, int reps,
             mrhs_tune_result* res, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  MRHS_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone) return fail(MRHS_ERR_INVALID_ARG, "autotune while the stream is captured");
  for (int i = 0; i < n; ++i)
    if (!tc_supported(ops[i], prec, nrhs[i])) return fail(MRHS_ERR_UNSUPPORTED, "tensor-core shape of a tuned problem");
  if (reps < 1) reps = 3;

  // scratch inputs, outputs and the reference output of the first candidate
  std::vector<void*> X(n, nullptr), Y(n, nullptr), Y0(n, nullptr);
  unsigned* flag = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto release = [&]() {
    for (int i = 0; i < n; ++i) {
      cudaFree(X[i]);
      cudaFree(Y[i]);
      cudaFree(Y0[i]);
    }
    cudaFree(flag);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  std::vector<int64_t> elems(n);
  for (int i = 0; i < n; ++i) {
    elems[i] = ops[i]->V * ops[i]->nb * nrhs[i];
    const size_t bytes = sizeof(float2) * (size_t)elems[i];
    if (cudaMalloc(&X[i], bytes) != cudaSuccess || cudaMalloc(&Y[i], bytes) != cudaSuccess ||
        cudaMalloc(&Y0[i], bytes) != cudaSuccess) {
      cudaGetLastError();
      release();
      return fail(MRHS_ERR_NO_MEMORY, "autotune scratch vectors");
    }
    k_fill<<<num_sms() * 4, 256, 0, s>>>((float2*)X[i], elems[i], 17u + (uint32_t)i);
    count_launch();
  }
  if (cudaMalloc(&flag, sizeof(unsigned)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    release();
    return fail(MRHS_ERR_CUDA, "autotune events");
  }
  MRHS_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(unsigned), s));

  auto run = [&](const TcTune& t, float* ms) -> int {
    int st = tc_apply_batch(ops, n, prec, X.data(), Y.data(), nrhs, nullptr, s, &t);   // warm-up
    if (st != MRHS_OK) return st;
    if (cudaEventRecord(e0, s) != cudaSuccess) return fail(MRHS_ERR_CUDA, "event");
    for (int r = 0; r < reps && st == MRHS_OK; ++r)
      st = tc_apply_batch(ops, n, prec, X.data(), Y.data(), nrhs, nullptr, s, &t);
    if (st != MRHS_OK) return st;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
      return fail(MRHS_ERR_CUDA, "event");
    if (tc_read_and_clear_error() != 0u) return fail(MRHS_ERR_DEVICE, "tensor-core kernel gave up waiting");
    cudaEventElapsedTime(ms, e0, e1);
    *ms /= (float)reps;
    return MRHS_OK;
  };

  // candidates: points per stage x CTAs per SM at the deepest ring, then the
  // ring depth for the best of those
  int max_pts = 1;
  for (int i = 0; i < n; ++i) max_pts = std::max(max_pts, ops[i]->npts);
  std::vector<TcTune> first;
  for (int pps : {0, 1, 2, 3, 4, 6, 8, 12}) {
    if (pps > max_pts) continue;
    for (int ctas : {1, 2}) {
      TcTune t;
      t.pps = pps;
      t.ctas_per_sm = ctas;
      t.max_stages = 32;
      first.push_back(t);
    }
  }
  TcTune best;
  double best_ms = 1e300, default_ms = 0;
  int tried = 0;
  bool have_ref = false;
  auto consider = [&](const TcTune& t) -> int {
    float ms = 0;
    MRHS_TRY(run(t, &ms));
    ++tried;
    if (!have_ref) {
      for (int i = 0; i < n; ++i)
        MRHS_CUDA_TRY(cudaMemcpyAsync(Y0[i], Y[i], sizeof(float2) * (size_t)elems[i],
                                      cudaMemcpyDeviceToDevice, s));
      have_ref = true;
    } else {
      for (int i = 0; i < n; ++i) {
        k_differs<<<num_sms() * 4, 256, 0, s>>>((const uint32_t*)Y[i], (const uint32_t*)Y0[i],
                                                 2 * elems[i], flag);
        count_launch();
      }
    }
    if (t.pps == 0 && t.ctas_per_sm == 2 && t.max_stages == 32) default_ms = ms;
    if (ms < best_ms) {
      best_ms = ms;
      best = t;
    }
    return MRHS_OK;
  };
  int st = MRHS_OK;
  for (const TcTune& t : first)
    if ((st = consider(t)) != MRHS_OK) break;
  if (st == MRHS_OK) {
    const TcTune base = best;
    for (int ns : {2, 3, 4, 6, 8, 12, 16}) {
      TcTune t = base;
      t.max_stages = ns;
      if ((st = consider(t)) != MRHS_OK) break;
    }
  }
  unsigned bad = 0;
  if (st == MRHS_OK) {
    if (cudaMemcpyAsync(&bad, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      st = fail(MRHS_ERR_CUDA, "autotune check");
  }
  release();
  if (st != MRHS_OK) return st;
  if (bad) return fail(MRHS_ERR_DEVICE, "launch shapes gave different results");
  {
    std::lock_guard<std::mutex> g(g_mu);
    cache()[make_key(ops, nrhs, n, prec)] = Entry{best, best_ms};
  }
  if (res) {
    res->pts_per_stage = best.pps;
    res->ctas_per_sm = best.ctas_per_sm;
    res->max_stages = best.max_stages;
    res->candidates = tried;
    res->ms = best_ms;
    res->ms_default = default_ms;
  }
  return MRHS_OK;
}

int64_t tune_entries() {
  std::lock_guard<std::mutex> g(g_mu);
  return (int64_t)cache().size();
}

void tune_clear() {
  std::lock_guard<std::mutex> g(g_mu);
  cache().clear();
}

// Text format, one entry per line:
//   n  {sms V nb npts nrhs prec} x n  pps ctas stages ms
int tune_save(const char* path) {
  FILE* f = std::fopen(path, "w");
  if (!f) return fail(MRHS_ERR_INVALID_ARG, std::string("cannot write ") + path);
  std::lock_guard<std::mutex> g(g_mu);
  std::fprintf(f, "# mrhs tensor-core launch shapes v1\n");
  for (const auto& kv : cache()) {
    std::fprintf(f, "%zu", kv.first.size());
    for (const KeyItem& it : kv.first)
      for (int64_t v : it) std::fprintf(f, " %lld", (long long)v);
    std::fprintf(f, " %d %d %d %.6g\n", kv.second.t.pps, kv.second.t.ctas_per_sm,
                 kv.second.t.max_stages, kv.second.ms);
  }
  const bool ok = std::fclose(f) == 0;
  return ok ? MRHS_OK : fail(MRHS_ERR_INVALID_ARG, std::string("cannot write ") + path);
}

int tune_load(const char* path) {
  FILE* f = std::fopen(path, "r");
  if (!f) return fail(MRHS_ERR_INVALID_ARG, std::string("cannot read ") + path);
  std::map<Key, Entry> got;
  char line[4096];
  int st = MRHS_OK;
  while (std::fgets(line, sizeof line, f)) {
    if (line[0] == '#' || line[0] == '\n') continue;
    char* p = line;
    char* end = nullptr;
    const long n = std::strtol(p, &end, 10);
    if (end == p || n < 1 || n > MRHS_MAX_BATCH) { st = MRHS_ERR_INVALID_ARG; break; }
    p = end;
    Key k(n);
    bool ok = true;
    for (long i = 0; i < n && ok; ++i)
      for (int j = 0; j < 6 && ok; ++j) {
        k[i][j] = std::strtoll(p, &end, 10);
        ok = end != p;
        p = end;
      }
    Entry e;
    long vals[3];
    for (int j = 0; j < 3 && ok; ++j) {
      vals[j] = std::strtol(p, &end, 10);
      ok = end != p;
      p = end;
    }
    if (ok) {
      e.ms = std::strtod(p, &end);
      ok = end != p;
    }
    if (!ok || vals[0] < 0 || vals[0] > 16 || vals[1] < 1 || vals[1] > 2 || vals[2] < 2 ||
        vals[2] > 32) {
      st = MRHS_ERR_INVALID_ARG;
      break;
    }
    e.t.pps = (int)vals[0];
    e.t.ctas_per_sm = (int)vals[1];
    e.t.max_stages = (int)vals[2];
    got[k] = e;
  }
  std::fclose(f);
  if (st != MRHS_OK) return fail(st, std::string("malformed launch-shape cache ") + path);
  std::lock_guard<std::mutex> g(g_mu);
  for (auto& kv : got) cache()[kv.first] = kv.second;
  return MRHS_OK;
}

}  // namespace mrhs
