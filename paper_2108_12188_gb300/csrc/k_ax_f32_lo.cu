// FP32 local operator kernels for 2..7 points per direction (stored and on-the-fly,
// plain and CG mode, both block shapes); the orders are split across translation units so
// that they compile in parallel.
#include "k_ax.cuh"

namespace sem {
sem_status launch_ax_f32_lo(int N, sem_ax_variant v, bool cg, const AxLaunch& a, cudaStream_t s) {
  return launch_ax_range<float, 2, 7>(N, v, cg, a, s);
}
}  // namespace sem
