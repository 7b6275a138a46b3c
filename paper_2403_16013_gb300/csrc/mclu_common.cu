// Precision-independent C entry points: elementwise dispatch, status strings.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "../../include/mclu.h"

namespace mclu {
static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace mclu

extern "C" uint64_t mclu_launch_count(void) { return mclu::g_launches.load(std::memory_order_relaxed); }

namespace mclu {
struct ProfRec {
  int kind;
  cudaEvent_t e0, e1;
};
static std::mutex g_prof_mu;
static std::atomic<uint32_t> g_prof_mask{0};
static std::vector<ProfRec> g_prof;
bool prof_on(int kind) { return (g_prof_mask.load(std::memory_order_relaxed) >> kind) & 1u; }
void prof_push(int kind, cudaEvent_t e0, cudaEvent_t e1) {
  std::lock_guard<std::mutex> g(g_prof_mu);
  g_prof.push_back({kind, e0, e1});
}
}  // namespace mclu

extern "C" int mclu_profile_begin(uint32_t kind_mask) {
  std::lock_guard<std::mutex> g(mclu::g_prof_mu);
  for (auto &r : mclu::g_prof) {
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  mclu::g_prof.clear();
  mclu::g_prof_mask.store(kind_mask);
  return 0;
}

extern "C" int mclu_profile_end(double *ms, int64_t *launches, int nkinds) {
  mclu::g_prof_mask.store(0);
  std::lock_guard<std::mutex> g(mclu::g_prof_mu);
  for (int k = 0; k < nkinds; k++) {
    if (ms) ms[k] = 0.0;
    if (launches) launches[k] = 0;
  }
  int rc = 0;
  for (auto &r : mclu::g_prof) {
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(r.e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.e0, r.e1);
    if (e != cudaSuccess && rc == 0) rc = (int)e;
    if (r.kind < nkinds) {
      if (ms) ms[r.kind] += t;
      if (launches) launches[r.kind] += 1;
    }
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  mclu::g_prof.clear();
  return rc;
}

int mclu_vec_op_dd(int op, int64_t count, const double *x, const double *y, double *z, void *stream);
int mclu_vec_op_td(int op, int64_t count, const double *x, const double *y, double *z, void *stream);
int mclu_vec_op_qd(int op, int64_t count, const double *x, const double *y, double *z, void *stream);

extern "C" int mclu_vec_op(int op, int L, int64_t count, const double *x, const double *y, double *z,
                           void *stream) {
  switch (L) {
    case 2: return mclu_vec_op_dd(op, count, x, y, z, stream);
    case 3: return mclu_vec_op_td(op, count, x, y, z, stream);
    case 4: return mclu_vec_op_qd(op, count, x, y, z, stream);
    default: return -2;
  }
}

extern "C" const char *mclu_status_string(int status) {
  if (status == 0) return "ok";
  if (status == MCLU_ERR_UNSUPPORTED) return "request not supported by this build";
  if (status == MCLU_ERR_SCRATCH_CAPACITY) return "problem too large for the fixed scratch capacity of this entry point";
  if (status < 0) return "invalid argument (status = -index of the argument)";
  return cudaGetErrorString((cudaError_t)status);
}

extern "C" const char *mclu_version(void) { return "0.2.0"; }

namespace {
// FP64 throughput probe: every thread runs 8 independent DFMA chains, so the
// FP64 units see no dependency stalls; 4 CTAs of 256 threads per SM.
__global__ void k_fp64_probe(double *out, int iters, double mul, double add) {
  double a[8];
#pragma unroll
  for (int c = 0; c < 8; c++) a[c] = 1.0 + 1e-3 * c + 1e-9 * threadIdx.x;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int c = 0; c < 8; c++) a[c] = __fma_rn(a[c], mul, add);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 8; c++) s = __dadd_rn(s, a[c]);
  if (s == -1.0) out[0] = s;  // never true: keeps the chains live
}
}  // namespace

extern "C" int mclu_probe_fp64_rate(double *ops_per_second) {
  if (ops_per_second == nullptr) return -1;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return (int)e;
  double *d = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(&d, sizeof(double));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int grid = 4 * sms, block = 256, iters = 40000;
  if (e == cudaSuccess) {
    k_fp64_probe<<<grid, block, 0, st>>>(d, iters / 8, 0.9999999, 1e-7);  // warm-up
    e = cudaEventRecord(e0, st);
  }
  if (e == cudaSuccess) {
    k_fp64_probe<<<grid, block, 0, st>>>(d, iters, 0.9999999, 1e-7);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) *ops_per_second = (double)grid * block * iters * 8.0 / (ms * 1e-3);
  if (e1) cudaEventDestroy(e1);
  if (e0) cudaEventDestroy(e0);
  if (st) cudaStreamDestroy(st);
  if (d) cudaFree(d);
  return (int)e;
}
