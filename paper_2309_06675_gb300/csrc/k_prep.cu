// Model preparation: Hermitian-pairing check, packed real basis of the Fourier sum and
// the per-axis twiddle tables.  These run once per call, before the per-k batches.
#include "kubo_internal.cuh"

namespace kubo {

namespace {

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* p, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

// One thread per entry (r, i, j): deviation |H(-R)_ji - conj H(R)_ij| and |H(R)_ij|.
__global__ void check_hermitian_kernel(const double2* __restrict__ H, const int* __restrict__ neg,
                                       int N_R, int W, DevStatus* st) {
  const int64_t total = (int64_t)N_R * W * W;
  double dev = 0.0, mx = 0.0;
  bool bad = false;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(t / ((int64_t)W * W));
    int ij = (int)(t % ((int64_t)W * W));
    int i = ij / W, j = ij % W;
    double2 a = H[t];
    double2 b = H[((int64_t)neg[r] * W + j) * W + i];
    if (!isfinite(a.x) || !isfinite(a.y)) bad = true;
    double dr = b.x - a.x, di = b.y + a.y;
    dev = fmax(dev, fabs(dr) + fabs(di));
    mx = fmax(mx, fabs(a.x) + fabs(a.y));
  }
  // warp reduce
  for (int o = 16; o > 0; o >>= 1) {
    dev = fmax(dev, __shfl_xor_sync(0xffffffffu, dev, o));
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  unsigned anybad = __any_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(&st->herm_dev_bits, dev);
    atomic_max_nonneg(&st->herm_max_bits, mx);
    if (anybad) atomicOr(&st->bits, ST_NONFINITE);
  }
}

// every listed mesh index in [0, Nk)
__global__ void check_kidx_kernel(const int64_t* __restrict__ kidx, int64_t n, int64_t Nk,
                                  DevStatus* st) {
  bool bad = false;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = kidx[t];
    bad |= k < 0 || k >= Nk;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&st->bits, ST_BAD_INDEX);
}

__global__ void hermitian_verdict_kernel(DevStatus* st) {
  double dev = __longlong_as_double((long long)st->herm_dev_bits);
  double mx = __longlong_as_double((long long)st->herm_max_bits);
  if (!(dev <= 1e-12 * mx)) atomicOr(&st->bits, ST_NOT_HERMITIAN);
}

// Packed basis rows.  Thread per packed entry (i, j) of one row.
//   row 0      : P0 = packed (H0 + H0^dagger)/2
//   row 1 + 2h : A_h = H(R_h) + H(-R_h)
//   row 2 + 2h : B_h = i (H(R_h) - H(-R_h))
// Packed Hermitian: P[i][j] = Re M_ij (i <= j), P[i][j] = Im M_ji (i > j).
__global__ void pack_basis_kernel(const double2* __restrict__ H, const int* __restrict__ pairs,
                                  int idx0, int N_h, int W, double scale, double* __restrict__ Bp) {
  const int WW = W * W;
  const int K = 1 + 2 * N_h;
  const int64_t total = (int64_t)K * WW;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int row = (int)(t / WW);
    int ij = (int)(t % WW);
    int i = ij / W, j = ij % W;
    // element (p, q) of the Hermitian matrix M that this packed slot holds
    int p = i <= j ? i : j;
    int q = i <= j ? j : i;
    bool want_im = i > j;
    double2 m;
    if (row == 0) {
      double2 a = H[((int64_t)idx0 * W + p) * W + q];
      double2 b = H[((int64_t)idx0 * W + q) * W + p];
      m = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    } else {
      int h = (row - 1) >> 1;
      int rp = pairs[2 * h], rm = pairs[2 * h + 1];
      double2 a = H[((int64_t)rp * W + p) * W + q];
      double2 b = H[((int64_t)rm * W + p) * W + q];
      if (((row - 1) & 1) == 0) {
        m = make_double2(a.x + b.x, a.y + b.y);          // A = H(R) + H(-R)
      } else {
        m = make_double2(-(a.y - b.y), a.x - b.x);       // B = i (H(R) - H(-R))
      }
    }
    Bp[t] = (want_im ? m.y : m.x) * scale;
  }
}

__global__ void scale_pow2_kernel(double* __restrict__ x, int64_t n, double f) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    x[t] *= f;
}

__global__ void twiddle_kernel(double2* tab, int N1, int N2, int N3) {
  int n = N1 + N2 + N3;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    int N, j;
    if (t < N1) { N = N1; j = t; }
    else if (t < N1 + N2) { N = N2; j = t - N1; }
    else { N = N3; j = t - N1 - N2; }
    double s, c;
    sincospi(2.0 * (double)j / (double)N, &s, &c);
    tab[t] = make_double2(c, s);
    // the FP32-pair copy: h = fl32(x), l = fl32(x - h)
    const float ch = __double2float_rn(c), sh = __double2float_rn(s);
    reinterpret_cast<float4*>(tab + n)[t] =
        make_float4(ch, __double2float_rn(c - (double)ch), sh, __double2float_rn(s - (double)sh));
  }
}

int grid_for(int64_t total, int threads) {
  int64_t b = (total + threads - 1) / threads;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

cudaError_t launch_check_hermitian(const double2* H_R, const int* neg, int N_R, int W,
                                   DevStatus* st, cudaStream_t s) {
  int64_t total = (int64_t)N_R * W * W;
  check_hermitian_kernel<<<grid_for(total, 256), 256, 0, s>>>(H_R, neg, N_R, W, st);
  return cudaGetLastError();
}

cudaError_t launch_hermitian_verdict(DevStatus* st, cudaStream_t s) {
  hermitian_verdict_kernel<<<1, 1, 0, s>>>(st);
  return cudaGetLastError();
}

cudaError_t launch_pack_basis(const double2* H_R, const int* pairs, int idx0, int N_h, int W,
                              double* Bp, cudaStream_t s, int escale) {
  int64_t total = (int64_t)(1 + 2 * N_h) * W * W;
  pack_basis_kernel<<<grid_for(total, 256), 256, 0, s>>>(H_R, pairs, idx0, N_h, W,
                                                          ldexp(1.0, escale), Bp);
  return cudaGetLastError();
}

cudaError_t launch_scale_pow2(double* x, int64_t n, int e, cudaStream_t s) {
  if (n <= 0 || e == 0) return cudaSuccess;
  scale_pow2_kernel<<<grid_for(n, 256), 256, 0, s>>>(x, n, ldexp(1.0, e));
  return cudaGetLastError();
}

cudaError_t launch_check_kidx(const int64_t* kidx, int64_t n, int64_t Nk, DevStatus* st,
                              cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  check_kidx_kernel<<<grid_for(n, 256), 256, 0, s>>>(kidx, n, Nk, st);
  return cudaGetLastError();
}

cudaError_t launch_twiddles(double2* tab, int N1, int N2, int N3, cudaStream_t s) {
  twiddle_kernel<<<grid_for(N1 + N2 + N3, 256), 256, 0, s>>>(tab, N1, N2, N3);
  return cudaGetLastError();
}

}  // namespace kubo
