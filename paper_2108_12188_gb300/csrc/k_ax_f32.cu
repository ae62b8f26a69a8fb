// FP32 instantiations of the local operator kernels (orders 1..SEM_MAX_N, stored and on-the-fly).
#include "k_ax.cuh"

namespace sem {
sem_status launch_ax_f32(int N, sem_ax_variant v, bool cg, const AxLaunch& a, cudaStream_t s) {
  return launch_ax_prec<float>(N, v, cg, a, s);
}
}  // namespace sem
