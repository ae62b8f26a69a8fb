// FP64 local operator kernels for 2..7 points per direction (stored and on-the-fly,
// plain and CG mode, both block shapes); the orders are split across translation units so
// that they compile in parallel.
#include "k_ax.cuh"

namespace sem {
sem_status launch_ax_f64_lo(int N, sem_ax_variant v, bool cg, const AxLaunch& a, cudaStream_t s) {
  return launch_ax_range<double, 2, 7>(N, v, cg, a, s);
}
}  // namespace sem

namespace sem {
namespace {
template <int NP>
int epb_np(int shape) {
  return shape == 0 ? ax_epb<NP>() : ax_epb_alt<NP>();
}
}  // namespace

int ax_elements_per_block(int N, int shape) {
  switch (N + 1) {
    case 2: return epb_np<2>(shape);
    case 3: return epb_np<3>(shape);
    case 4: return epb_np<4>(shape);
    case 5: return epb_np<5>(shape);
    case 6: return epb_np<6>(shape);
    case 7: return epb_np<7>(shape);
    case 8: return epb_np<8>(shape);
    case 9: return epb_np<9>(shape);
    case 10: return epb_np<10>(shape);
    case 11: return epb_np<11>(shape);
    case 12: return epb_np<12>(shape);
    default: return 0;
  }
}
}  // namespace sem
