// Double-double (L = 2) instantiation of the C entry points.
#include "lu_host.cuh"
MCLU_DEFINE_PRECISION(dd, 2)

// The inter-CTA wait of the cooperative panels on a flag that nothing sets:
// it must run out within its budget and leave the status word set.
__global__ void k_selftest_wait(const int *flag, int *status) {
  if (threadIdx.x == 0 && !mclu::coop_wait_flag(flag, 1)) atomicOr(status, 1);
}

extern "C" int mclu_selftest_wait_timeout(int32_t *status) {
  if (status == nullptr) return -1;
  int *d = nullptr;
  cudaError_t e = cudaMalloc(&d, 2 * sizeof(int));
  if (e != cudaSuccess) return (int)e;
  e = cudaMemset(d, 0, 2 * sizeof(int));
  if (e == cudaSuccess) {
    k_selftest_wait<<<1, 32>>>(d, d + 1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(status, d + 1, sizeof(int32_t), cudaMemcpyDeviceToHost);
  cudaFree(d);
  return (int)e;
}
