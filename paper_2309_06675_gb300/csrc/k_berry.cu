// Steps (3)-(4) of List 1/2 ("convert" + "evaluate"), FP64, one CTA per k-point:
//   v^a = U^dagger (d_a H) U            (a = x, y)
//   Omega_n = -2 sum_{m != n} Im(v^x_nm conj(v^y_nm)) / ((E_n - E_m)^2 + eta^2)   (Eq. 3)
// (v^y_mn = conj(v^y_nm) because v^y is Hermitian.)  Both rotations are register-tiled
// complex products over shared-memory operands; the curvature is reduced per band in a
// fixed order (deterministic), for every requested broadening eta at once.
#include "kubo_internal.cuh"

namespace kubo {

namespace {

constexpr int NT = 256;
constexpr int MAXE = 8;
constexpr int TM = 4;   // 16 x 16 threads, 4 x 4 tile each: W <= 64

// acc[i][j] = sum_q op(A)[r_i][q] * B[q][c_j],  r_i = ty + 16 i, c_j = tx + 16 j
template <bool ADJ>
__device__ __forceinline__ void cgemm_tile(const double2* __restrict__ A,
                                           const double2* __restrict__ B, int W, int LD,
                                           int ty, int tx, double2 (&acc)[TM][TM]) {
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TM; ++j) acc[i][j] = make_double2(0.0, 0.0);
  for (int q = 0; q < W; ++q) {
    double2 a[TM], bb[TM];
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      int r = ty + 16 * i;
      double2 v = make_double2(0.0, 0.0);
      if (r < W) {
        if (ADJ) { v = A[q * LD + r]; v.y = -v.y; }
        else v = A[r * LD + q];
      }
      a[i] = v;
    }
#pragma unroll
    for (int j = 0; j < TM; ++j) {
      int c = tx + 16 * j;
      bb[j] = c < W ? B[q * LD + c] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TM; ++j) {
        acc[i][j].x = fma(a[i].x, bb[j].x, acc[i][j].x);
        acc[i][j].x = fma(-a[i].y, bb[j].y, acc[i][j].x);
        acc[i][j].y = fma(a[i].x, bb[j].y, acc[i][j].y);
        acc[i][j].y = fma(a[i].y, bb[j].x, acc[i][j].y);
      }
  }
}

__device__ __forceinline__ void store_tile(double2* C, int W, int LD, int ty, int tx,
                                           const double2 (&acc)[TM][TM]) {
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TM; ++j) {
      int r = ty + 16 * i, c = tx + 16 * j;
      if (r < W && c < W) C[r * LD + c] = acc[i][j];
    }
}

__device__ __forceinline__ void unpack_hermitian(const double* __restrict__ P, double2* A, int W,
                                                 int LD, int t) {
  for (int idx = t; idx < W * W; idx += NT) {
    int i = idx / W, j = idx % W;
    double2 a;
    if (i < j) a = make_double2(P[i * W + j], P[j * W + i]);
    else if (i > j) a = make_double2(P[j * W + i], -P[i * W + j]);
    else a = make_double2(P[i * W + i], 0.0);
    A[i * LD + j] = a;
  }
}

__global__ void __launch_bounds__(NT) berry_fp64_kernel(const double* __restrict__ E,
                                                        const double2* __restrict__ U,
                                                        const double* __restrict__ Xp,
                                                        const double* __restrict__ Yp, int W,
                                                        const double* __restrict__ etas,
                                                        int n_eta, double* __restrict__ Om,
                                                        int64_t eta_stride) {
  extern __shared__ double2 sm[];
  const int LD = W + 1;
  double2* sU = sm;
  double2* sA = sU + W * LD;
  double2* sB = sA + W * LD;
  double* red = (double*)sB;   // reused after the last product
  __shared__ double sE[64];
  __shared__ double sEta[MAXE];
  __shared__ double s_emax;

  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int64_t k = blockIdx.x;
  const size_t WW = (size_t)W * W;

  for (int idx = t; idx < W * W; idx += NT) sU[(idx / W) * LD + idx % W] = U[k * WW + idx];
  unpack_hermitian(Xp + k * WW, sA, W, LD, t);
  for (int j = t; j < W; j += NT) sE[j] = E[k * W + j];
  if (t < n_eta) sEta[t] = etas[t];
  __syncthreads();
  if (t == 0) {
    double mx = 0.0;
    for (int j = 0; j < W; ++j) mx = fmax(mx, fabs(sE[j]));
    s_emax = mx;
  }

  double2 acc[TM][TM];
  cgemm_tile<false>(sA, sU, W, LD, ty, tx, acc);        // T = X U
  __syncthreads();
  store_tile(sA, W, LD, ty, tx, acc);
  __syncthreads();
  cgemm_tile<true>(sU, sA, W, LD, ty, tx, acc);         // v^x = U^H T
  __syncthreads();
  store_tile(sA, W, LD, ty, tx, acc);
  unpack_hermitian(Yp + k * WW, sB, W, LD, t);
  __syncthreads();
  cgemm_tile<false>(sB, sU, W, LD, ty, tx, acc);        // T = Y U
  __syncthreads();
  store_tile(sB, W, LD, ty, tx, acc);
  __syncthreads();
  cgemm_tile<true>(sU, sB, W, LD, ty, tx, acc);         // v^y = U^H T
  __syncthreads();                                      // sB is free from here on

  const double emax = s_emax;
  double rp[MAXE][TM];
#pragma unroll
  for (int e = 0; e < MAXE; ++e)
#pragma unroll
    for (int i = 0; i < TM; ++i) rp[e][i] = 0.0;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int n = ty + 16 * i;
    if (n >= W) continue;
    double En = sE[n];
#pragma unroll
    for (int j = 0; j < TM; ++j) {
      int m = tx + 16 * j;
      if (m >= W || m == n) continue;
      double2 vx = sA[n * LD + m];
      double2 vy = acc[i][j];
      double num = -2.0 * fma(vx.y, vy.x, -vx.x * vy.y);   // -2 Im(vx conj(vy))
      double dE = En - sE[m];
      double d2 = dE * dE;
#pragma unroll
      for (int e = 0; e < MAXE; ++e) {
        if (e >= n_eta) break;
        double eta = sEta[e];
        if (eta == 0.0 && fabs(dE) <= 1e-12 * emax) continue;
        rp[e][i] += num / fma(eta, eta, d2);
      }
    }
  }
#pragma unroll
  for (int e = 0; e < MAXE; ++e) {
    if (e >= n_eta) break;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      int n = ty + 16 * i;
      if (n < W) red[(e * W + n) * 16 + tx] = rp[e][i];
    }
  }
  __syncthreads();
  for (int idx = t; idx < n_eta * W; idx += NT) {
    int e = idx / W, n = idx % W;
    const double* p = red + (size_t)idx * 16;
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 16; ++q) s += p[q];
    Om[e * eta_stride + k * W + n] = s;
  }
}

}  // namespace

size_t berry_fp64_smem(int W, int n_eta) {
  size_t mat = (size_t)W * (W + 1) * sizeof(double2);
  size_t red = (size_t)n_eta * W * 16 * sizeof(double);
  return 2 * mat + (mat > red ? mat : red);
}

cudaError_t launch_berry_fp64(const double* E, const double2* U, const double* Xp,
                              const double* Yp, int W, int n, const double* etas, int n_eta,
                              double* Om, int64_t eta_stride, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  size_t sm = berry_fp64_smem(W, n_eta);
  cudaError_t e = cudaFuncSetAttribute(berry_fp64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  berry_fp64_kernel<<<n, NT, sm, s>>>(E, U, Xp, Yp, W, etas, n_eta, Om, eta_stride);
  return cudaGetLastError();
}

}  // namespace kubo
