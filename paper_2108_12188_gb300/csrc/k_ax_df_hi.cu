// Double-float local operator with stored factors, 8 to 12 points per direction (kernel in
// k_ax_df.cuh).
#include "k_ax_df.cuh"

namespace sem {
namespace {

template <int NP>
struct DfStored {
  static sem_status run(int N, bool cg, const AxLaunch& a, cudaStream_t s) {
    if (a.g_pairs) return cg ? launch_df_t<NP, true, kGkPairs>(N, a, s) : launch_df_t<NP, false, kGkPairs>(N, a, s);
    return cg ? launch_df_t<NP, true, kGkF64>(N, a, s) : launch_df_t<NP, false, kGkF64>(N, a, s);
  }
};

}  // namespace

sem_status launch_ax_f64x_hi(int N, bool cg, const AxLaunch& a, cudaStream_t s) {
  return df_dispatch<DfStored, 8, 12>(N, cg, a, s);
}

}  // namespace sem
