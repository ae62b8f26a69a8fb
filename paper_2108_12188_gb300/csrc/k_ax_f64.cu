// FP64 instantiations of the local operator kernels (orders 1..SEM_MAX_N, stored and on-the-fly).
#include "k_ax.cuh"

namespace sem {
sem_status launch_ax_f64(int N, sem_ax_variant v, bool cg, const AxLaunch& a, cudaStream_t s) {
  return launch_ax_prec<double>(N, v, cg, a, s);
}
}  // namespace sem
