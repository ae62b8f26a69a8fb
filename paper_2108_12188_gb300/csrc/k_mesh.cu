// Element geometry kernels: trilinear-map coefficients, geometric factors G and mass B
// (Eq. 4's G^e; Section 4.2's six factors per point), physical coordinates, the local
// diagonal of A_L (Jacobi), the right-hand side B f, and small vector utilities.
//
// A trilinear hexahedron with vertices X_v, v = a + 2b + 4c, is
//   x(xi, eta, gam) = sum_v X_v phi_a(xi) phi_b(eta) phi_c(gam),  phi_0 = (1-t)/2, phi_1 = (1+t)/2
//                   = a0 + a1 xi + a2 eta + a3 gam + a4 xi eta + a5 xi gam + a6 eta gam + a7 xi eta gam
// with a_m = (1/8) sum_v s_m(v) X_v and s_m the products of the corner signs (2a-1, 2b-1, 2c-1)
// selected by the monomial. a1..a7 are differences of vertices, so rounding them to FP32
// keeps their relative accuracy (absolute coordinates would lose bits to cancellation).
#include "k_common.cuh"

namespace sem {
namespace {

constexpr int kThreads = 256;

struct GllAll {  // xi and w of one order, FP64
  double xi[kMaxNp], w[kMaxNp];
};
GllAll gll_all(int N) {
  const GllTable& t = gll_table(N);
  GllAll g{};
  for (int a = 0; a <= N; ++a) {
    g.xi[a] = t.xi[a];
    g.w[a] = t.w[a];
  }
  return g;
}

__global__ void k_coefficients(int64_t E, const double* __restrict__ X, double* __restrict__ c64,
                               float* __restrict__ c32) {
  const int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (e >= E) return;
  const double* x = X + e * 24;
  for (int comp = 0; comp < 3; ++comp) {
    double a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int v = 0; v < 8; ++v) {
      const double sa = (v & 1) ? 1.0 : -1.0, sb = (v & 2) ? 1.0 : -1.0, sc = (v & 4) ? 1.0 : -1.0;
      const double xv = x[v * 3 + comp];
      a[0] += xv;
      a[1] += sa * xv;
      a[2] += sb * xv;
      a[3] += sc * xv;
      a[4] += sa * sb * xv;
      a[5] += sa * sc * xv;
      a[6] += sb * sc * xv;
      a[7] += sa * sb * sc * xv;
    }
    for (int m = 0; m < 8; ++m) {
      const double am = 0.125 * a[m];
      c64[e * 24 + m * 3 + comp] = am;
      c32[e * 24 + m * 3 + comp] = static_cast<float>(am);
    }
  }
}

struct PointGeom {
  double g[3][3];  // g[b] = dx/dxi_b
};

__device__ __forceinline__ void jacobian_columns(const double* a, double xi, double eta, double gam, double g0[3],
                                                 double g1[3], double g2[3]) {
  for (int c = 0; c < 3; ++c) {
    const double a1 = a[3 + c], a2 = a[6 + c], a3 = a[9 + c], a4 = a[12 + c], a5 = a[15 + c], a6 = a[18 + c],
                 a7 = a[21 + c];
    g0[c] = a1 + a4 * eta + a5 * gam + a7 * eta * gam;
    g1[c] = a2 + a4 * xi + a6 * gam + a7 * xi * gam;
    g2[c] = a3 + a5 * xi + a6 * eta + a7 * xi * eta;
  }
}

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double out[3]) {
  out[0] = a[1] * b[2] - a[2] * b[1];
  out[1] = a[2] * b[0] - a[0] * b[2];
  out[2] = a[0] * b[1] - a[1] * b[0];
}

// G = w |det J| J^-1 J^-T = (w / det) C C^T with C's rows c_b = g_{b+1} x g_{b+2}; B = w det.
__device__ void point_geometry(const double* a, double xi, double eta, double gam, double wq, double G[6],
                               double* B, double* det_out) {
  double g0[3], g1[3], g2[3], c0[3], c1[3], c2[3];
  jacobian_columns(a, xi, eta, gam, g0, g1, g2);
  cross3(g1, g2, c0);
  cross3(g2, g0, c1);
  cross3(g0, g1, c2);
  const double det = g0[0] * c0[0] + g0[1] * c0[1] + g0[2] * c0[2];
  const double s = wq / det;
  auto d = [](const double* p, const double* q) { return p[0] * q[0] + p[1] * q[1] + p[2] * q[2]; };
  G[0] = s * d(c0, c0);
  G[1] = s * d(c0, c1);
  G[2] = s * d(c0, c2);
  G[3] = s * d(c1, c1);
  G[4] = s * d(c1, c2);
  G[5] = s * d(c2, c2);
  *B = wq * det;
  *det_out = det;
}

__global__ void k_geometry(const __grid_constant__ GllAll tab, int Np, int64_t E, const double* __restrict__ coef,
                           double* __restrict__ G64, float* __restrict__ G32, double* __restrict__ B64,
                           float* __restrict__ B32, int* __restrict__ bad, int64_t gs64, int64_t gs32,
                           double* __restrict__ S64, float* __restrict__ S32, float* __restrict__ GX) {
  const int64_t P = static_cast<int64_t>(Np) * Np * Np;
  const int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (idx >= E * P) return;
  const int64_t e = idx / P;
  const int r = static_cast<int>(idx - e * P);
  const int i = r % Np, j = (r / Np) % Np, k = r / (Np * Np);
  double G[6], B, det;
  point_geometry(coef + e * 24, tab.xi[i], tab.xi[j], tab.xi[k], tab.w[i] * tab.w[j] * tab.w[k], G, &B, &det);
  if (!(det > 0.0) || !isfinite(det)) atomicOr(bad, 1);
  for (int m = 0; m < 6; ++m) {
    if (G64) G64[e * gs64 + m * P + r] = G[m];
    if (G32) G32[e * gs32 + m * P + r] = static_cast<float>(G[m]);
    if (GX) {  // float pair (high, low): high = G rounded to FP32, low = the rest rounded to FP32
      const float h = static_cast<float>(G[m]);
      GX[2 * (e * gs64 + m * P + r)] = h;
      GX[2 * (e * gs64 + m * P + r) + 1] = static_cast<float>(G[m] - static_cast<double>(h));
    }
  }
  if (B64) B64[idx] = B;
  if (B32) B32[idx] = static_cast<float>(B);
  const double sc = tab.w[i] * tab.w[j] * tab.w[k] / det;  // scale of the on-the-fly factors
  if (S64) S64[idx] = sc;
  if (S32) S32[idx] = static_cast<float>(sc);
}

__global__ void k_coords(const __grid_constant__ GllAll tab, int Np, int64_t E, const double* __restrict__ coef,
                         double* __restrict__ xyz, int64_t n) {
  const int64_t P = static_cast<int64_t>(Np) * Np * Np;
  const int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (idx >= E * P) return;
  const int64_t e = idx / P;
  const int r = static_cast<int>(idx - e * P);
  const double xi = tab.xi[r % Np], eta = tab.xi[(r / Np) % Np], gam = tab.xi[r / (Np * Np)];
  const double* a = coef + e * 24;
  for (int c = 0; c < 3; ++c)
    xyz[c * n + idx] = a[c] + a[3 + c] * xi + a[6 + c] * eta + a[9 + c] * gam + a[12 + c] * xi * eta +
                       a[15 + c] * xi * gam + a[18 + c] * eta * gam + a[21 + c] * xi * eta * gam;
}

// Diagonal of D^T G D at (i, j, k):
//   sum_l D_li^2 G11(l,j,k) + sum_l D_lj^2 G22(i,l,k) + sum_l D_lk^2 G33(i,j,l)
//   + 2 D_ii D_jj G12 + 2 D_ii D_kk G13 + 2 D_jj D_kk G23.
// One block per element; G of the element is built in shared memory first.
__global__ void k_local_diag(const __grid_constant__ GllTable tab, int Np, int64_t E, const double* __restrict__ coef,
                             double* __restrict__ d) {
  extern __shared__ double sG[];  // [6][P]
  const int P = Np * Np * Np;
  const int64_t e = blockIdx.x;
  for (int r = threadIdx.x; r < P; r += blockDim.x) {
    const int i = r % Np, j = (r / Np) % Np, k = r / (Np * Np);
    double G[6], B, det;
    point_geometry(coef + e * 24, tab.xi[i], tab.xi[j], tab.xi[k], tab.w[i] * tab.w[j] * tab.w[k], G, &B, &det);
    for (int m = 0; m < 6; ++m) sG[m * P + r] = G[m];
  }
  __syncthreads();
  for (int r = threadIdx.x; r < P; r += blockDim.x) {
    const int i = r % Np, j = (r / Np) % Np, k = r / (Np * Np);
    double s = 0.0;
    for (int l = 0; l < Np; ++l) {
      const double dli = tab.D[l * Np + i], dlj = tab.D[l * Np + j], dlk = tab.D[l * Np + k];
      s += dli * dli * sG[0 * P + (k * Np + j) * Np + l];
      s += dlj * dlj * sG[3 * P + (k * Np + l) * Np + i];
      s += dlk * dlk * sG[5 * P + (l * Np + j) * Np + i];
    }
    const double dii = tab.D[i * Np + i], djj = tab.D[j * Np + j], dkk = tab.D[k * Np + k];
    s += 2.0 * dii * djj * sG[1 * P + r] + 2.0 * dii * dkk * sG[2 * P + r] + 2.0 * djj * dkk * sG[4 * P + r];
    d[e * P + r] = s;
  }
}

// (B f)(x) with f = (a^2+b^2+c^2) pi^2 sin(a pi x) sin(b pi y) sin(c pi z).
__global__ void k_rhs_local(const __grid_constant__ GllAll tab, int Np, int64_t E, const double* __restrict__ coef,
                            int fa, int fb, int fc, double* __restrict__ out) {
  const int64_t P = static_cast<int64_t>(Np) * Np * Np;
  const int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (idx >= E * P) return;
  const int64_t e = idx / P;
  const int r = static_cast<int>(idx - e * P);
  const int i = r % Np, j = (r / Np) % Np, k = r / (Np * Np);
  const double xi = tab.xi[i], eta = tab.xi[j], gam = tab.xi[k];
  const double* a = coef + e * 24;
  double x[3];
  for (int c = 0; c < 3; ++c)
    x[c] = a[c] + a[3 + c] * xi + a[6 + c] * eta + a[9 + c] * gam + a[12 + c] * xi * eta + a[15 + c] * xi * gam +
           a[18 + c] * eta * gam + a[21 + c] * xi * eta * gam;
  double G[6], B, det;
  point_geometry(a, xi, eta, gam, tab.w[i] * tab.w[j] * tab.w[k], G, &B, &det);
  const double pi2 = 9.869604401089358;  // pi^2
  const double f = (fa * fa + fb * fb + fc * fc) * pi2 * sinpi(fa * x[0]) * sinpi(fb * x[1]) * sinpi(fc * x[2]);
  out[idx] = B * f;
}

template <typename T>
__global__ void k_scatter(int64_t n, const int32_t* __restrict__ glo, const T* __restrict__ ug, T* __restrict__ ul) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    ul[i] = ug[glo[i]];
}

__global__ void k_invert(int64_t n, const double* __restrict__ d, double* __restrict__ m64, float* __restrict__ m32) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double v = 1.0 / d[i];
    if (m64) m64[i] = v;
    if (m32) m32[i] = static_cast<float>(v);
  }
}

__global__ void k_cast(int64_t n, const double* __restrict__ in, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    out[i] = static_cast<float>(in[i]);
}

// One thread per item, at most 32 blocks per SM (grid-stride beyond).
int grid_for(int64_t n) {
  static const int cap = [] {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return 32 * (sms > 0 ? sms : 1);
  }();
  const int64_t b = (n + kThreads - 1) / kThreads;
  return static_cast<int>(b < cap ? (b > 0 ? b : 1) : cap);
}

}  // namespace

sem_status launch_coefficients(int64_t E, const double* X, double* coef64, float* coef32, cudaStream_t s) {
  k_coefficients<<<ceil_div(E, 128), 128, 0, s>>>(E, X, coef64, coef32);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

sem_status launch_geometry(int N, int64_t E, const double* coef64, double* G64, float* G32, double* B64, float* B32,
                           int* bad, int64_t gs64, int64_t gs32, cudaStream_t s, double* S64, float* S32,
                           float* GX) {
  const int Np = N + 1;
  const int64_t n = E * Np * Np * Np;
  k_geometry<<<ceil_div(n, kThreads), kThreads, 0, s>>>(gll_all(N), Np, E, coef64, G64, G32, B64, B32, bad, gs64,
                                                        gs32, S64, S32, GX);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

sem_status launch_coords(int N, int64_t E, const double* coef64, double* xyz, int64_t n, cudaStream_t s) {
  k_coords<<<ceil_div(n, kThreads), kThreads, 0, s>>>(gll_all(N), N + 1, E, coef64, xyz, n);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

sem_status launch_local_diag(int N, int64_t E, const double* coef64, double* d, cudaStream_t s) {
  const int Np = N + 1, P = Np * Np * Np;
  const size_t smem = 6 * static_cast<size_t>(P) * sizeof(double);
  static const cudaError_t attr = cudaFuncSetAttribute(k_local_diag, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       6 * kMaxNp * kMaxNp * kMaxNp * static_cast<int>(sizeof(double)));
  SEM_CUDA_TRY(attr);
  // E blocks: at most 2^31 / 8 elements (the local-size limit), within the grid x limit
  k_local_diag<<<static_cast<unsigned>(E), P < 512 ? P : 512, smem, s>>>(gll_table(N), Np, E, coef64, d);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

sem_status launch_rhs_local(int N, int64_t E, const double* coef64, int a, int b, int c, double* out, cudaStream_t s) {
  const int Np = N + 1;
  const int64_t n = E * Np * Np * Np;
  k_rhs_local<<<ceil_div(n, kThreads), kThreads, 0, s>>>(gll_all(N), Np, E, coef64, a, b, c, out);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

sem_status launch_scatter(sem_prec prec, int64_t n, const int32_t* glo, const void* ug, void* ul, cudaStream_t s) {
  if (prec == SEM_F64)
    k_scatter<double><<<grid_for(n), kThreads, 0, s>>>(n, glo, static_cast<const double*>(ug), static_cast<double*>(ul));
  else
    k_scatter<float><<<grid_for(n), kThreads, 0, s>>>(n, glo, static_cast<const float*>(ug), static_cast<float*>(ul));
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

sem_status launch_invert(int64_t n, const double* d, double* m64, float* m32, cudaStream_t s) {
  k_invert<<<grid_for(n), kThreads, 0, s>>>(n, d, m64, m32);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

sem_status launch_cast(int64_t n, const double* in, float* out, cudaStream_t s) {
  k_cast<<<grid_for(n), kThreads, 0, s>>>(n, in, out);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

}  // namespace sem
