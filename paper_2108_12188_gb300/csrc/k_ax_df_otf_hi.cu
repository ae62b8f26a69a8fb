// Double-float local operator with the geometric factors rebuilt on the fly from the element's
// trilinear coefficients, 8 to 12 points per direction (kernel in k_ax_df.cuh).
#include "k_ax_df.cuh"

namespace sem {
namespace {

template <int NP>
struct DfOtf {
  static sem_status run(int N, bool cg, const AxLaunch& a, cudaStream_t s) {
    return cg ? launch_df_t<NP, true, kGkOtf>(N, a, s) : launch_df_t<NP, false, kGkOtf>(N, a, s);
  }
};

}  // namespace

sem_status launch_ax_f64x_otf_hi(int N, bool cg, const AxLaunch& a, cudaStream_t s) {
  return df_dispatch<DfOtf, 8, 12>(N, cg, a, s);
}

}  // namespace sem
