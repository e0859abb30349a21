// k-sum of Eq. 2 (with Eq. 4's batching): S(E_F) = (1/N_k) sum_k sum_n occ(E_n(k)) Omega_n(k)
// for every (eta, E_F) pair.  Deterministic: every block sums a fixed k-range in order with
// Neumaier compensation, blocks are folded in index order, batches in call order.
#include "kubo_internal.cuh"

namespace kubo {

namespace {

__device__ __forceinline__ void neumaier_add(double& s, double& c, double x) {
  double t = s + x;
  if (fabs(s) >= fabs(x)) c += (s - t) + x;
  else c += (x - t) + s;
  s = t;
}

// occupation of a level at energy E for Fermi level EF: step (strict) or Fermi-Dirac
__device__ __forceinline__ double occupation(double E, double EF, double kT) {
  if (kT == 0.0) return E < EF ? 1.0 : 0.0;
  double x = (E - EF) / kT;
  double ex = exp(-fabs(x));
  return x > 0.0 ? ex / (1.0 + ex) : 1.0 / (1.0 + ex);
}

__global__ void ksum_partial_kernel(const double* __restrict__ E, const double* __restrict__ Om,
                                    int W, int n, int n_eta, int64_t eta_stride,
                                    const double* __restrict__ E_F, int n_EF, double kT,
                                    double2* __restrict__ part, int kpb) {
  const int b = blockIdx.x;
  const int kb = b * kpb, ke = min(n, kb + kpb);
  const int n_out = n_eta * n_EF;
  for (int o = threadIdx.x; o < n_out; o += blockDim.x) {
    const int e = o / n_EF, j = o % n_EF;
    const double ef = E_F[j];
    double s = 0.0, c = 0.0;
    for (int k = kb; k < ke; ++k) {
      const double* Ek = E + (size_t)k * W;
      const double* Ok = Om + e * eta_stride + (size_t)k * W;
      double v = 0.0;
      for (int q = 0; q < W; ++q) v = fma(occupation(Ek[q], ef, kT), Ok[q], v);
      neumaier_add(s, c, v);
    }
    part[(size_t)b * n_out + o] = make_double2(s, c);
  }
}

__global__ void ksum_fold_kernel(const double2* __restrict__ part, int n_blocks, int n_out,
                                 double2* __restrict__ acc) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < n_out; o += gridDim.x * blockDim.x) {
    double s = acc[o].x, c = acc[o].y;
    for (int b = 0; b < n_blocks; ++b) {
      double2 p = part[(size_t)b * n_out + o];
      neumaier_add(s, c, p.x);
      neumaier_add(s, c, p.y);
    }
    acc[o] = make_double2(s, c);
  }
}

__global__ void ksum_final_kernel(const double2* __restrict__ acc, int n_out, double inv_Nk,
                                  const DevStatus* st, double* __restrict__ out) {
  if (st->bits != 0) return;   // outputs are written only on success
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < n_out; o += gridDim.x * blockDim.x)
    out[o] = (acc[o].x + acc[o].y) * inv_Nk;
}

}  // namespace

cudaError_t launch_ksum_partial(const double* E, const double* Om, int W, int n, int n_eta,
                                int64_t eta_stride, const double* E_F, int n_EF, double kT,
                                double2* part, int kpb, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int nb = (n + kpb - 1) / kpb;
  ksum_partial_kernel<<<nb, 128, 0, s>>>(E, Om, W, n, n_eta, eta_stride, E_F, n_EF, kT, part, kpb);
  return cudaGetLastError();
}

cudaError_t launch_ksum_fold(const double2* part, int n_blocks, int n_out, double2* acc,
                             cudaStream_t s) {
  if (n_blocks <= 0) return cudaSuccess;
  ksum_fold_kernel<<<(n_out + 127) / 128, 128, 0, s>>>(part, n_blocks, n_out, acc);
  return cudaGetLastError();
}

cudaError_t launch_ksum_final(const double2* acc, int n_out, double inv_Nk, const DevStatus* st,
                              double* out, cudaStream_t s) {
  ksum_final_kernel<<<(n_out + 127) / 128, 128, 0, s>>>(acc, n_out, inv_Nk, st, out);
  return cudaGetLastError();
}

}  // namespace kubo
