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
// 16 x 16 threads, each a TM x TM tile of the W x W products: TM = 1, 2, 4 for W up to 16,
// 32, 64 (the smallest tile that covers W, so no thread multiplies padding)

// acc[i][j] = sum_q op(A)[r_i][q] * B[q][c_j],  r_i = ty + 16 i, c_j = tx + 16 j
template <int TM, bool ADJ>
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

template <int TM>
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

template <typename TIn>
__device__ __forceinline__ void unpack_hermitian(const TIn* __restrict__ P, double2* A, int W,
                                                 int LD, int t) {
  for (int idx = t; idx < W * W; idx += NT) {
    int i = idx / W, j = idx % W;
    double2 a;
    if (i < j) a = make_double2((double)P[i * W + j], (double)P[j * W + i]);
    else if (i > j) a = make_double2((double)P[j * W + i], -(double)P[i * W + j]);
    else a = make_double2((double)P[i * W + i], 0.0);
    A[i * LD + j] = a;
  }
}

// Curvature epilogue shared by both precisions.  Every pair is evaluated once (n < m) and
// enters Omega_n with +T_nm and Omega_m with -T_nm, so the antisymmetry T_mn = -T_nm that
// makes occupied-occupied pairs cancel holds exactly even when v is only Hermitian to FP32
// rounding.  Per-thread row / column partials go to `red` (2 * n_eta * W * 16 doubles, may
// alias sVx: a barrier separates the last read of sVx from the first write of red) and are
// summed in a fixed order (deterministic).
template <int TM, typename V>
__device__ __forceinline__ void curvature_epilogue(const V* sVx, const V (&vy)[TM][TM],
                                                   const double* sE, const double* sEta,
                                                   int n_eta, double emax, int W, int LD, int ty,
                                                   int tx, int t, double* red,
                                                   double* __restrict__ Om, int64_t eta_stride,
                                                   int64_t k) {
  double num[TM][TM], d2[TM][TM];
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int n = ty + 16 * i;
#pragma unroll
    for (int j = 0; j < TM; ++j) {
      const int m = tx + 16 * j;
      num[i][j] = 0.0;
      d2[i][j] = -1.0;   // marks "no pair"
      if (n < W && m < W && n < m) {
        const V vx = sVx[n * LD + m];
        num[i][j] = -2.0 * ((double)vx.y * (double)vy[i][j].x - (double)vx.x * (double)vy[i][j].y);
        const double dE = sE[n] - sE[m];
        d2[i][j] = dE * dE;
      }
    }
  }
  __syncthreads();
  const double thr2 = (1e-12 * emax) * (1e-12 * emax);
  for (int e = 0; e < n_eta; ++e) {
    const double eta = sEta[e];
    double rp[TM], cp[TM];
#pragma unroll
    for (int i = 0; i < TM; ++i) { rp[i] = 0.0; cp[i] = 0.0; }
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TM; ++j) {
        if (d2[i][j] < 0.0) continue;
        if (eta == 0.0 && d2[i][j] <= thr2) continue;
        const double T = num[i][j] / fma(eta, eta, d2[i][j]);
        rp[i] += T;
        cp[j] -= T;
      }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int n = ty + 16 * i;
      if (n < W) red[((size_t)(e * W + n) * 2) * 16 + tx] = rp[i];
      const int m = tx + 16 * i;
      if (m < W) red[((size_t)(e * W + m) * 2 + 1) * 16 + ty] = cp[i];
    }
  }
  __syncthreads();
  for (int idx = t; idx < n_eta * W; idx += NT) {
    const int e = idx / W, n = idx % W;
    const double* p = red + (size_t)idx * 2 * 16;
    double sr = 0.0, sc = 0.0;
#pragma unroll
    for (int q = 0; q < 16; ++q) { sr += p[q]; sc += p[16 + q]; }
    Om[e * eta_stride + k * W + n] = sr + sc;
  }
}

// X and Y: packed Hermitian rows of leading dimension ld (FP64 rows of the FP64 Fourier
// kernel, or FP32 rows of the tensor-core one).
template <typename TIn, int TM>
__global__ void __launch_bounds__(NT) berry_fp64_kernel(const double* __restrict__ E,
                                                        const double2* __restrict__ U,
                                                        const TIn* __restrict__ Xp,
                                                        const TIn* __restrict__ Yp, int64_t ld,
                                                        int W,
                                                        const double* __restrict__ etas,
                                                        int n_eta, double* __restrict__ Om,
                                                        int64_t eta_stride, int pad) {
  extern __shared__ double2 sm[];
  const int LD = W + pad;   // pad = 1: conflict-free column walks; 0: the padding ablation
  double2* sU = sm;
  double2* sA = sU + W * LD;
  double2* sB = sA + W * LD;
  double* red = (double*)sA;   // reused (sA and beyond) after the pair terms are formed
  __shared__ double sE[64];
  __shared__ double sEta[MAXE];
  __shared__ double s_emax;

  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int64_t k = blockIdx.x;
  const size_t WW = (size_t)W * W;

  for (int idx = t; idx < W * W; idx += NT) sU[(idx / W) * LD + idx % W] = U[k * WW + idx];
  unpack_hermitian(Xp + k * ld, sA, W, LD, t);
  for (int j = t; j < W; j += NT) sE[j] = E[k * W + j];
  if (t < n_eta) sEta[t] = etas[t];
  __syncthreads();
  if (t == 0) {
    double mx = 0.0;
    for (int j = 0; j < W; ++j) mx = fmax(mx, fabs(sE[j]));
    s_emax = mx;
  }

  double2 acc[TM][TM];
  cgemm_tile<TM, false>(sA, sU, W, LD, ty, tx, acc);        // T = X U
  __syncthreads();
  store_tile<TM>(sA, W, LD, ty, tx, acc);
  __syncthreads();
  cgemm_tile<TM, true>(sU, sA, W, LD, ty, tx, acc);         // v^x = U^H T
  __syncthreads();
  store_tile<TM>(sA, W, LD, ty, tx, acc);
  unpack_hermitian(Yp + k * ld, sB, W, LD, t);
  __syncthreads();
  cgemm_tile<TM, false>(sB, sU, W, LD, ty, tx, acc);        // T = Y U
  __syncthreads();
  store_tile<TM>(sB, W, LD, ty, tx, acc);
  __syncthreads();
  cgemm_tile<TM, true>(sU, sB, W, LD, ty, tx, acc);         // v^y = U^H T
  curvature_epilogue<TM, double2>(sA, acc, sE, sEta, n_eta, s_emax, W, LD, ty, tx, t, red, Om,
                              eta_stride, k);
}

// ------------------------------------------------------------------ mixed precision
// The two rotations in FP32 on the FP32 pipe (64x the FP64 rate on GB300): operands U
// (rounded from FP64) and the FP32 tensor-core Fourier output; the energy denominators,
// the pair terms and the band sums stay FP64.
template <int TM, bool ADJ>
__device__ __forceinline__ void cgemm_tile_f32(const float2* __restrict__ A,
                                               const float2* __restrict__ B, int W, int LD,
                                               int ty, int tx, float2 (&acc)[TM][TM]) {
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TM; ++j) acc[i][j] = make_float2(0.f, 0.f);
  for (int q = 0; q < W; ++q) {
    float2 a[TM], bb[TM];
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      int r = ty + 16 * i;
      float2 v = make_float2(0.f, 0.f);
      if (r < W) {
        if (ADJ) { v = A[q * LD + r]; v.y = -v.y; }
        else v = A[r * LD + q];
      }
      a[i] = v;
    }
#pragma unroll
    for (int j = 0; j < TM; ++j) {
      int c = tx + 16 * j;
      bb[j] = c < W ? B[q * LD + c] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TM; ++j) {
        acc[i][j].x = fmaf(a[i].x, bb[j].x, acc[i][j].x);
        acc[i][j].x = fmaf(-a[i].y, bb[j].y, acc[i][j].x);
        acc[i][j].y = fmaf(a[i].x, bb[j].y, acc[i][j].y);
        acc[i][j].y = fmaf(a[i].y, bb[j].x, acc[i][j].y);
      }
  }
}

template <int TM>
__device__ __forceinline__ void store_tile_f32(float2* C, int W, int LD, int ty, int tx,
                                               const float2 (&acc)[TM][TM]) {
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TM; ++j) {
      int r = ty + 16 * i, c = tx + 16 * j;
      if (r < W && c < W) C[r * LD + c] = acc[i][j];
    }
}

template <typename TIn>
__device__ __forceinline__ void unpack_hermitian_f32(const TIn* __restrict__ P, float2* A, int W,
                                                     int LD, int t) {
  for (int idx = t; idx < W * W; idx += NT) {
    int i = idx / W, j = idx % W;
    float2 a;
    if (i < j) a = make_float2((float)P[i * W + j], (float)P[j * W + i]);
    else if (i > j) a = make_float2((float)P[j * W + i], -(float)P[i * W + j]);
    else a = make_float2((float)P[i * W + i], 0.f);
    A[i * LD + j] = a;
  }
}

// U = Q D Z in FP32, in shared memory, from the FP64 factors of the eigensolver: Z (eigenvectors
// of the real tridiagonal, [W][W]), the phases D and the Householder reflectors (staged in
// `stage`, W (W - 1) / 2 complex).  Each column is transformed by its own 4 threads, so the
// reflectors are applied without block barriers.  The only consumer of this U is the FP32
// rotation, so it is formed at that precision.
__device__ __forceinline__ void assemble_u_f32(const double* __restrict__ Zk,
                                               const double2* __restrict__ ph,
                                               const double2* __restrict__ R,
                                               const double* __restrict__ tau, int W, int LD,
                                               int t, float2* sU, float2* stage) {
  for (int idx = t; idx < W * W; idx += NT) {
    const int r = idx / W, c = idx % W;
    const double z = Zk[idx];
    const double2 p = ph[r];
    sU[r * LD + c] = make_float2((float)(p.x * z), (float)(p.y * z));
  }
  auto roff = [&](int j) { return j * (W - 1) - (j * (j - 1)) / 2; };   // sum_{j'<j} (W-1-j')
  for (int idx = t; idx < W * W; idx += NT) {
    const int r = idx / W, c = idx % W;
    if (r > c && c < W - 2) {
      const double2 v = R[idx];
      stage[roff(c) + (r - c - 1)] = make_float2((float)v.x, (float)v.y);
    }
  }
  __syncthreads();
  const int q = t & 3, c = t >> 2;   // NT / 4 = 64 >= W columns
  const bool act = c < W;
  for (int j = W - 3; j >= 0; --j) {
    const float tj = (float)tau[j];
    if (tj == 0.f) continue;
    const int o = j + 1, m = W - 1 - j;
    const float2* v = stage + roff(j);
    float sx = 0.f, sy = 0.f;
    if (act) {
      for (int r = q; r < m; r += 4) {
        const float2 vv = v[r];
        const float2 u = sU[(o + r) * LD + c];
        sx = fmaf(vv.x, u.x, fmaf(vv.y, u.y, sx));   // conj(v) u
        sy = fmaf(vv.x, u.y, fmaf(-vv.y, u.x, sy));
      }
    }
    sx += __shfl_xor_sync(0xffffffffu, sx, 1);
    sy += __shfl_xor_sync(0xffffffffu, sy, 1);
    sx += __shfl_xor_sync(0xffffffffu, sx, 2);
    sy += __shfl_xor_sync(0xffffffffu, sy, 2);
    sx *= tj; sy *= tj;
    if (act) {
      for (int r = q; r < m; r += 4) {
        const float2 vv = v[r];
        float2 u = sU[(o + r) * LD + c];
        u.x = fmaf(-sx, vv.x, fmaf(sy, vv.y, u.x));   // u -= s v
        u.y = fmaf(-sx, vv.y, fmaf(-sy, vv.x, u.y));
        sU[(o + r) * LD + c] = u;
      }
    }
    __syncwarp();
  }
  __syncthreads();
}

// Leading dimension (in float2) of the FP32 shared-memory matrices.  Padded: W + P with
// W + P = 4 (mod 16), so that a row step moves 8 banks: the 4 rows x 2 columns of float2 that
// a quarter of a warp touches in the reflector application, and the 16 consecutive columns of
// a half warp elsewhere, fall on distinct banks.  Unpadded (the ablation): W.
__host__ __device__ __forceinline__ int mixed_ld(int W, int pad) {
  return pad ? W + ((4 - W) & 15) : W;
}

// X and Y: packed Hermitian rows of leading dimension ld.  FROMZ: U is assembled in FP32 from
// the eigensolver's factors (Z, eb.phase, eb.refl, eb.tau) instead of being read.
template <typename TIn, bool FROMZ, int TM>
__global__ void __launch_bounds__(NT) berry_mixed_kernel(const double* __restrict__ E,
                                                         const double2* __restrict__ U,
                                                         const double* __restrict__ Z,
                                                         EighBufs eb,
                                                         const TIn* __restrict__ Xp,
                                                         const TIn* __restrict__ Yp, int64_t ld,
                                                         int W, const double* __restrict__ etas,
                                                         int n_eta, double* __restrict__ Om,
                                                         int64_t eta_stride, int pad) {
  extern __shared__ float2 smf[];
  const int LD = mixed_ld(W, pad);
  float2* sU = smf;
  float2* sA = sU + W * LD;
  float2* sB = sA + W * LD;
  double* red = (double*)sA;   // reused (sA and beyond) after the pair terms are formed
  __shared__ double sE[64];
  __shared__ double sEta[MAXE];
  __shared__ double s_emax;

  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int64_t k = blockIdx.x;
  const size_t WW = (size_t)W * W;

  if (FROMZ) {
    assemble_u_f32(Z + k * WW, eb.phase + k * W, eb.refl + k * WW, eb.tau + k * W, W, LD, t, sU, sA);
  } else {
    for (int idx = t; idx < W * W; idx += NT) {
      double2 u = U[k * WW + idx];
      sU[(idx / W) * LD + idx % W] = make_float2((float)u.x, (float)u.y);
    }
  }
  unpack_hermitian_f32(Xp + k * ld, sA, W, LD, t);
  for (int j = t; j < W; j += NT) sE[j] = E[k * W + j];
  if (t < n_eta) sEta[t] = etas[t];
  __syncthreads();
  if (t == 0) {
    double mx = 0.0;
    for (int j = 0; j < W; ++j) mx = fmax(mx, fabs(sE[j]));
    s_emax = mx;
  }

  float2 acc[TM][TM];
  cgemm_tile_f32<TM, false>(sA, sU, W, LD, ty, tx, acc);   // T = X U
  __syncthreads();
  store_tile_f32<TM>(sA, W, LD, ty, tx, acc);
  __syncthreads();
  cgemm_tile_f32<TM, true>(sU, sA, W, LD, ty, tx, acc);    // v^x = U^H T
  __syncthreads();
  store_tile_f32<TM>(sA, W, LD, ty, tx, acc);
  unpack_hermitian_f32(Yp + k * ld, sB, W, LD, t);
  __syncthreads();
  cgemm_tile_f32<TM, false>(sB, sU, W, LD, ty, tx, acc);   // T = Y U
  __syncthreads();
  store_tile_f32<TM>(sB, W, LD, ty, tx, acc);
  __syncthreads();
  cgemm_tile_f32<TM, true>(sU, sB, W, LD, ty, tx, acc);    // v^y = U^H T
  curvature_epilogue<TM, float2>(sA, acc, sE, sEta, n_eta, s_emax, W, LD, ty, tx, t, red, Om,
                             eta_stride, k);
}

__global__ void unpack_rows_kernel(const double* __restrict__ C, int64_t ld, int W, int n,
                                   double* __restrict__ H, double* __restrict__ X,
                                   double* __restrict__ Y) {
  const int64_t WW = (int64_t)W * W;
  const int64_t total = (int64_t)n * WW;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = t / WW, q = t % WW;
    const double* r = C + k * ld;
    H[t] = r[q];
    X[t] = r[WW + q];
    Y[t] = r[2 * WW + q];
  }
}

}  // namespace

size_t berry_fp64_smem(int W, int n_eta) {
  size_t mat = (size_t)W * (W + 1) * sizeof(double2);
  size_t red = (size_t)n_eta * W * 2 * 16 * sizeof(double);
  return mat + (2 * mat > red ? 2 * mat : red);
}

template <typename TIn>
cudaError_t launch_berry_fp64_t(const double* E, const double2* U, const TIn* Xp, const TIn* Yp,
                                int64_t ld, int W, int n, const double* etas, int n_eta, double* Om,
                                int64_t eta_stride, cudaStream_t s, int pad) {
  if (n <= 0) return cudaSuccess;
  size_t sm = berry_fp64_smem(W, n_eta);
  auto go = [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    kern<<<n, NT, sm, s>>>(E, U, Xp, Yp, ld, W, etas, n_eta, Om, eta_stride, pad ? 1 : 0);
    return cudaGetLastError();
  };
  if (W <= 16) return go(berry_fp64_kernel<TIn, 1>);
  if (W <= 32) return go(berry_fp64_kernel<TIn, 2>);
  return go(berry_fp64_kernel<TIn, 4>);
}

cudaError_t launch_berry_fp64(const double* E, const double2* U, const double* Xp,
                              const double* Yp, int W, int n, const double* etas, int n_eta,
                              double* Om, int64_t eta_stride, cudaStream_t s, int pad) {
  return launch_berry_fp64_t<double>(E, U, Xp, Yp, (int64_t)W * W, W, n, etas, n_eta, Om,
                                     eta_stride, s, pad);
}

cudaError_t launch_berry_fp64_rows(const double* E, const double2* U, const double* C,
                                   int64_t ld, int W, int n, const double* etas, int n_eta,
                                   double* Om, int64_t eta_stride, cudaStream_t s, int pad) {
  const int64_t WW = (int64_t)W * W;
  return launch_berry_fp64_t<double>(E, U, C + WW, C + 2 * WW, ld, W, n, etas, n_eta, Om,
                                     eta_stride, s, pad);
}

size_t berry_mixed_smem(int W, int n_eta) {
  const size_t mat = (size_t)W * mixed_ld(W, 1) * sizeof(float2);
  const size_t red = (size_t)n_eta * W * 2 * 16 * sizeof(double);
  return mat + (2 * mat > red ? 2 * mat : red);
}

template <typename TIn, bool FROMZ>
cudaError_t launch_berry_mixed_t(const double* E, const double2* U, const double* Z,
                                 const EighBufs& eb, const TIn* Xp, const TIn* Yp,
                                 int64_t ld, int W, int n, const double* etas, int n_eta,
                                 double* Om, int64_t eta_stride, cudaStream_t s, int pad) {
  if (n <= 0) return cudaSuccess;
  size_t sm = berry_mixed_smem(W, n_eta);
  auto go = [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    kern<<<n, NT, sm, s>>>(E, U, Z, eb, Xp, Yp, ld, W, etas, n_eta, Om, eta_stride, pad ? 1 : 0);
    return cudaGetLastError();
  };
  if (W <= 16) return go(berry_mixed_kernel<TIn, FROMZ, 1>);
  if (W <= 32) return go(berry_mixed_kernel<TIn, FROMZ, 2>);
  return go(berry_mixed_kernel<TIn, FROMZ, 4>);
}

cudaError_t launch_berry_mixed_rows(const double* E, const double2* U, const double* C,
                                    int64_t ld, int W, int n, const double* etas, int n_eta,
                                    double* Om, int64_t eta_stride, cudaStream_t s, int pad) {
  const int64_t WW = (int64_t)W * W;
  return launch_berry_mixed_t<double, false>(E, U, nullptr, EighBufs{}, C + WW, C + 2 * WW, ld, W,
                                             n, etas, n_eta, Om, eta_stride, s, pad);
}

cudaError_t launch_berry_mixed_rows_z(const double* E, const double* Z, const EighBufs& eb,
                                      const double* C, int64_t ld, int W, int n,
                                      const double* etas, int n_eta, double* Om,
                                      int64_t eta_stride, cudaStream_t s, int pad) {
  const int64_t WW = (int64_t)W * W;
  return launch_berry_mixed_t<double, true>(E, nullptr, Z, eb, C + WW, C + 2 * WW, ld, W, n, etas,
                                            n_eta, Om, eta_stride, s, pad);
}

cudaError_t launch_berry_mixed_from_f64_z(const double* E, const double* Z, const EighBufs& eb,
                                          const double* Xp, const double* Yp, int W, int n,
                                          const double* etas, int n_eta, double* Om,
                                          int64_t eta_stride, cudaStream_t s, int pad) {
  return launch_berry_mixed_t<double, true>(E, nullptr, Z, eb, Xp, Yp, (int64_t)W * W, W, n, etas,
                                            n_eta, Om, eta_stride, s, pad);
}

cudaError_t launch_berry_mixed_from_f64(const double* E, const double2* U, const double* Xp,
                                        const double* Yp, int W, int n, const double* etas,
                                        int n_eta, double* Om, int64_t eta_stride,
                                        cudaStream_t s, int pad) {
  return launch_berry_mixed_t<double, false>(E, U, nullptr, EighBufs{}, Xp, Yp, (int64_t)W * W, W,
                                             n, etas, n_eta, Om, eta_stride, s, pad);
}

cudaError_t launch_unpack_rows(const double* C, int64_t ld, int W, int n, double* H, double* X,
                               double* Y, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int64_t total = (int64_t)n * W * W;
  int64_t b = (total + 255) / 256;
  if (b > 152 * 64) b = 152 * 64;
  unpack_rows_kernel<<<(int)b, 256, 0, s>>>(C, ld, W, n, H, X, Y);
  return cudaGetLastError();
}

}  // namespace kubo
