// lmep_spectral.cu -- the Fourier symbol of a harvested row (Sec. 4.1's
// spectral footprints): G(theta) = sum_j w_j e^{i theta (j - r)}, the factor by
// which one step of a constant-coefficient periodic update multiplies the mode
// e^{i theta x / h}.  One thread per angle, FP64.
#include "lmep_internal.h"

namespace lmep {

namespace {
__global__ void k_symbol(const double* __restrict__ w, int n, int r, const double* __restrict__ theta, int64_t M,
                         double* __restrict__ G) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= M) return;
  const double t = theta[q];
  double re = 0.0, im = 0.0;
  for (int j = 0; j < n; ++j) {
    double sn, cs;
    sincos(t * double(j - r), &sn, &cs);
    re = fma(w[j], cs, re);
    im = fma(w[j], sn, im);
  }
  G[2 * q] = re;
  G[2 * q + 1] = im;
}
}  // namespace

cudaError_t launch_symbol(const double* w, int n, int r, const double* theta, int64_t M, double* G, cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  const int block = 256;
  k_symbol<<<unsigned((M + block - 1) / block), block, 0, s>>>(w, n, r, theta, M, G);
  return cudaGetLastError();
}

}  // namespace lmep
