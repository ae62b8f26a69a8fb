// sem_glsc3_noalloc: the weighted inner product <a, b, c> of sem_glsc3, for callers that
// must not allocate device memory through the library - an application that hands all
// device memory out from its own pool, or a loop where the implicit device-wide
// synchronisation of cudaMalloc/cudaFree cannot be afforded. The per-block partial sums and
// the completion counter, which sem_glsc3 keeps in memory allocated with the mesh, live here
// in a file-scope static device array instead; the call itself allocates nothing.
//
// Limits and sharing rules:
//  - The array holds kNoAllocBlocks partials; each block reduces a fixed chunk of
//    kNoAllocChunk points, so n_local <= kNoAllocBlocks * kNoAllocChunk = 33,554,432.
//    Larger meshes are rejected with SEM_ERR_ARG.
//  - Every GPU that loads the library holds the array (32 KB + 256 B) until the process ends.
//  - All calls share the one array and it keeps the last call's contents: the counter is
//    cleared on the call's stream before each launch, and calls that overlap on the GPU
//    (different streams, or different host threads) race on the array and give wrong sums.
//  - The first call on each device looks up the array's device address with that device
//    current; make that first call before any stream capture is started. The address is kept
//    for the life of the process, so the call must not be used after cudaDeviceReset (or
//    after the device's primary context has been destroyed and created again).
#include <mutex>

#include "k_common.cuh"

namespace sem {
namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocBlocks = 4096;
constexpr int64_t kNoAllocChunk = 8192;
constexpr int kCounterBytes = 256;  // the completion counter, padded so the partials stay 256-byte aligned
constexpr int kMaxDevices = 64;

// [0, 256): completion counter; [256, 256 + 8 * kNoAllocBlocks): one double per block.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kCounterBytes + sizeof(double) * kNoAllocBlocks];

template <typename T>
__global__ void __launch_bounds__(kNoAllocThreads)
    k_glsc3_chunked(int64_t n, const T* __restrict__ a, const T* __restrict__ b, const uint8_t* __restrict__ mult,
                    const double* __restrict__ ctab, unsigned char* scratch, double* __restrict__ result) {
  __shared__ double sRed[kNoAllocThreads / 32];
  unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch);
  double* partials = reinterpret_cast<double*>(scratch + kCounterBytes);
  const int64_t lo = blockIdx.x * kNoAllocChunk;
  const int64_t hi = lo + kNoAllocChunk < n ? lo + kNoAllocChunk : n;
  double acc = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += kNoAllocThreads) {
    const unsigned m = mult[i];
    const double c = m == 1u ? 1.0 : __ldg(ctab + m);
    acc += static_cast<double>(a[i]) * static_cast<double>(b[i]) * c;
  }
  const double v[1] = {block_sum(acc, sRed)};
  if (publish_partials<1>(v, partials, ticket)) {
    const double s = sum_partials(partials, gridDim.x, 1, 0, sRed);
    if (threadIdx.x == 0) *result = s;
  }
}

// Device address of the static array, looked up once per device with that device current.
sem_status scratch_address(unsigned char** out) {
  static std::mutex mu;
  static void* addr[kMaxDevices] = {};
  int dev = 0;
  SEM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(SEM_ERR_UNSUPPORTED, "device ordinal beyond the supported range");
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(addr[dev]);
  return SEM_OK;
}

}  // namespace
}  // namespace sem

using namespace sem;

extern "C" sem_status sem_glsc3_noalloc(sem_mesh m, sem_prec prec, const void* a, const void* b, double* result,
                                        void* stream) {
  return guarded([&]() -> sem_status {
    sem_status st = check_mesh(m);
    if (st != SEM_OK) return st;
    if (prec != SEM_F64 && prec != SEM_F32) return fail(SEM_ERR_ARG, "precision must be SEM_F64 or SEM_F32");
    if ((st = check_ptr(a, "a_dev")) != SEM_OK || (st = check_ptr(b, "b_dev")) != SEM_OK) return st;
    if (!result) return fail(SEM_ERR_ARG, "result_dev is null");
    if (m->n > static_cast<int64_t>(kNoAllocBlocks) * kNoAllocChunk)
      return fail(SEM_ERR_ARG, "sem_glsc3_noalloc handles at most " +
                                   std::to_string(static_cast<int64_t>(kNoAllocBlocks) * kNoAllocChunk) +
                                   " local points (its static scratch holds " + std::to_string(kNoAllocBlocks) +
                                   " block partials); this mesh has " + std::to_string(m->n));
    unsigned char* scratch = nullptr;
    if ((st = scratch_address(&scratch)) != SEM_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    note_stream(m, s);  // sem_mesh_destroy waits for this stream before releasing mult and ctab
    SEM_CUDA_TRY(cudaMemsetAsync(scratch, 0, kCounterBytes, s));
    const int grid = static_cast<int>((m->n + kNoAllocChunk - 1) / kNoAllocChunk);
    if (prec == SEM_F64)
      k_glsc3_chunked<double><<<grid, kNoAllocThreads, 0, s>>>(m->n, static_cast<const double*>(a),
                                                                static_cast<const double*>(b), m->mult, m->ctab,
                                                                scratch, result);
    else
      k_glsc3_chunked<float><<<grid, kNoAllocThreads, 0, s>>>(m->n, static_cast<const float*>(a),
                                                               static_cast<const float*>(b), m->mult, m->ctab,
                                                               scratch, result);
    count_launch();
    SEM_CUDA_TRY(cudaGetLastError());
    return SEM_OK;
  });
}
