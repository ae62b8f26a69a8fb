// Self-test of the bounded waits that guard every TMA copy of the library (k_tma.cuh): one
// thread initialises an mbarrier for a 16-byte copy and waits for it with a time limit. With
// the copy issued the wait completes; without it nothing ever arrives, the wait gives up after
// the limit and the kernel reports SEM_ERR_TIMEOUT, the status a local-operator kernel sets
// when its factor or input copy does not arrive. Before leaving after a timeout the kernel
// waits, again with a time limit, for a copy it had issued; it does not guarantee that such a
// copy has landed if that second wait also gives up. The context stays usable.
#include "k_common.cuh"
#include "k_tma.cuh"

namespace sem {
namespace {

__global__ void k_probe_wait(const int4* __restrict__ src, int4* __restrict__ dst, int issue, uint64_t limit_ns,
                             int* __restrict__ status) {
  __shared__ alignas(16) int4 buf;
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_proxy_async();
  mbar_expect_tx(&bar, 16u);
  if (issue) tma_load_1d(&buf, src, 16u, &bar);
  const bool ok = mbar_wait_bounded(&bar, 0u, limit_ns);
  if (ok) {
    *dst = buf;
    *status = SEM_OK;
  } else {
    if (issue) mbar_wait_bounded(&bar, 0u, limit_ns);  // let the issued copy land before leaving
    *status = SEM_ERR_TIMEOUT;
  }
}

}  // namespace
}  // namespace sem

extern "C" sem_status sem_probe_bounded_wait(int64_t limit_ns, int issue_copy, double* elapsed_ms, void* stream) {
  using namespace sem;
  return guarded([&]() -> sem_status {
    if (!elapsed_ms) return fail(SEM_ERR_ARG, "elapsed_ms is null");
    if (limit_ns < 1000000 || limit_ns > 2000000000) return fail(SEM_ERR_ARG, "limit_ns must be in [1 ms, 2 s]");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int4* buf = nullptr;  // [0] source, [1] destination
    int* status = nullptr;
    SEM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&buf), 2 * sizeof(int4), s));
    sem_status st = SEM_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int h = -1;
    auto step = [&](cudaError_t e, const char* what) {
      if (st == SEM_OK && e != cudaSuccess) st = cuda_fail(e, what);
    };
    step(cudaMallocAsync(reinterpret_cast<void**>(&status), sizeof(int), s), "cudaMallocAsync");
    step(cudaMemsetAsync(buf, 0x5a, 2 * sizeof(int4), s), "cudaMemsetAsync");
    step(cudaMemsetAsync(status, 0xff, sizeof(int), s), "cudaMemsetAsync");
    step(cudaEventCreate(&e0), "cudaEventCreate");
    step(cudaEventCreate(&e1), "cudaEventCreate");
    if (st == SEM_OK) {
      cudaEventRecord(e0, s);
      k_probe_wait<<<1, 32, 0, s>>>(buf, buf + 1, issue_copy ? 1 : 0, static_cast<uint64_t>(limit_ns), status);
      count_launch();
      step(cudaGetLastError(), "k_probe_wait launch");
      cudaEventRecord(e1, s);
      step(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync");
      step(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    }
    if (st == SEM_OK) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      *elapsed_ms = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (status) cudaFreeAsync(status, s);
    cudaFreeAsync(buf, s);
    if (st != SEM_OK) return st;
    if (h == SEM_OK) return SEM_OK;
    if (h == SEM_ERR_TIMEOUT) return fail(SEM_ERR_TIMEOUT, "bounded wait gave up (no copy arrived)");
    return fail(SEM_ERR_CUDA, "the probe kernel did not report");
  });
}

// Self-test of the grid barrier of the persistent CG kernel (k_cg_small.cu): a cooperative launch
// of a few blocks meets at one bounded barrier. skip_one = 0: every block arrives, SEM_OK.
// skip_one = 1: the last block never arrives, the others give up after the barrier's limit (1 s)
// and report SEM_ERR_TIMEOUT; nothing faults and the context stays usable.
extern "C" sem_status sem_probe_grid_barrier(int skip_one, double* elapsed_ms, void* stream) {
  using namespace sem;
  return guarded([&]() -> sem_status {
    if (!elapsed_ms) return fail(SEM_ERR_ARG, "elapsed_ms is null");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    SEM_CUDA_TRY(cudaGetDevice(&dev));
    SEM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms < 8 ? sms : 8;
    if (blocks < 2) return fail(SEM_ERR_UNSUPPORTED, "needs two SMs");
    unsigned* bar = nullptr;
    int* status = nullptr;
    SEM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&bar), 2 * sizeof(unsigned), s));
    sem_status st = SEM_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int h = -2;
    auto step = [&](cudaError_t e, const char* what) {
      if (st == SEM_OK && e != cudaSuccess) st = cuda_fail(e, what);
    };
    step(cudaMallocAsync(reinterpret_cast<void**>(&status), sizeof(int), s), "cudaMallocAsync");
    step(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s), "cudaMemsetAsync");
    step(cudaMemsetAsync(status, 0xff, sizeof(int), s), "cudaMemsetAsync");
    step(cudaEventCreate(&e0), "cudaEventCreate");
    step(cudaEventCreate(&e1), "cudaEventCreate");
    if (st == SEM_OK) {
      cudaEventRecord(e0, s);
      st = launch_probe_barrier(bar, blocks, skip_one ? blocks - 1 : -1, status, s);
      cudaEventRecord(e1, s);
      step(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync");
      step(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    }
    if (st == SEM_OK) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      *elapsed_ms = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (status) cudaFreeAsync(status, s);
    cudaFreeAsync(bar, s);
    if (st != SEM_OK) return st;
    if (h == SEM_OK) return SEM_OK;
    if (h == SEM_ERR_TIMEOUT) return fail(SEM_ERR_TIMEOUT, "grid barrier gave up (a block never arrived)");
    return fail(SEM_ERR_CUDA, "the barrier probe did not report");
  });
}
