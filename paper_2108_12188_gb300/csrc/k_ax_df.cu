// Double-float local operator with stored factors (FP64 values or float pairs), 2 to 7 points
// per direction; the kernel is in k_ax_df.cuh, the other orders and the on-the-fly variant in
// k_ax_df_hi.cu, k_ax_df_otf.cu and k_ax_df_otf_hi.cu (compiled in parallel).
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

sem_status launch_ax_f64x(int N, sem_ax_variant v, bool cg, const AxLaunch& a, cudaStream_t s) {
  if (v == SEM_AX_OTF) {
    if (!a.coef) return fail(SEM_ERR_ARG, "the mesh has no trilinear coefficients");
    return N + 1 <= 7 ? launch_ax_f64x_otf_lo(N, cg, a, s) : launch_ax_f64x_otf_hi(N, cg, a, s);
  }
  if (v != SEM_AX_STORED) return fail(SEM_ERR_UNSUPPORTED, "SEM_F64X runs the stored and on-the-fly variants");
  return N + 1 <= 7 ? df_dispatch<DfStored, 2, 7>(N, cg, a, s) : launch_ax_f64x_hi(N, cg, a, s);
}

}  // namespace sem
