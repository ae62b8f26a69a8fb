// FP32 local operator kernels for 8..12 points per direction (stored and on-the-fly,
// plain and CG mode, both block shapes); the orders are split across translation units so
// that they compile in parallel.
#include "k_ax.cuh"

namespace sem {
sem_status launch_ax_f32_hi(int N, sem_ax_variant v, bool cg, const AxLaunch& a, cudaStream_t s) {
  return launch_ax_range<float, 8, 12>(N, v, cg, a, s);
}
}  // namespace sem
