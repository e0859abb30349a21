// Steps (3)-(4) of List 1/2 ("convert" + "evaluate"), FP64, one CTA per k-point:
//   v^a = U^dagger (d_a H) U            (a = x, y)
//   Omega_n = -2 sum_{m != n} Im(v^x_nm conj(v^y_nm)) / ((E_n - E_m)^2 + eta^2)   (Eq. 3)
// (v^y_mn = conj(v^y_nm) because v^y is Hermitian.)  Both rotations are register-tiled
// complex products over shared-memory operands; the curvature is reduced per band in a
// fixed order (deterministic), for every requested broadening eta at once.
#include <algorithm>
#include <type_traits>

#include <cuda_bf16.h>

#include "kubo_internal.cuh"
#include "tc_ptx.cuh"

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
  const FastDiv dW(W);
  for (int idx = t; idx < W * W; idx += NT) {
    const int i = (int)dW.div(idx), j = idx - i * W;
    double2 a;
    if (i < j) a = make_double2((double)P[i * W + j], (double)P[j * W + i]);
    else if (i > j) a = make_double2((double)P[j * W + i], -(double)P[i * W + j]);
    else a = make_double2((double)P[i * W + i], 0.0);
    A[i * LD + j] = a;
  }
}

// max_j |E_j| of a shared array, by warp 0 on the bit patterns (for non-negative doubles the
// integer order is the numeric order; NaN patterns count as 0): no FP64 instruction, where a
// serial loop of FP64 maxima by one thread queued behind the FP64 pipe.  Every thread calls
// it; the value is read after a later barrier.
__device__ __forceinline__ void emax_warp0(const double* sE, int W, int t, double* out) {
  if (t < 32) {
    unsigned long long m = 0ull;
    for (int j = t; j < W; j += 32) {
      unsigned long long u = (unsigned long long)__double_as_longlong(sE[j]) & 0x7FFFFFFFFFFFFFFFull;
      if (u > 0x7FF0000000000000ull) u = 0ull;
      m = u > m ? u : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
      m = v > m ? v : m;
    }
    if (t == 0) *out = __longlong_as_double((long long)m);
  }
}

// a b - c d within 2 ulp (Kahan: the rounding error of c d is recovered exactly by an FMA)
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d) {
  const float w = __fmul_rn(c, d);
  const float e = fmaf(-c, d, w);     // w - c d, exact
  const float f = fmaf(a, b, -w);
  return __fadd_rn(f, e);
}

// (hi, lo) += x with the rounding error of hi + x carried exactly into lo (Knuth's TwoSum)
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bp = __fsub_rn(s, hi);
  const float ap = __fsub_rn(s, bp);
  const float err = __fadd_rn(__fsub_rn(hi, ap), __fsub_rn(x, bp));
  hi = s;
  lo = __fadd_rn(lo, err);
}

// Curvature epilogue shared by both precisions.  Every pair is evaluated once (n < m) and
// enters Omega_n with +T_nm and Omega_m with -T_nm, so the antisymmetry T_mn = -T_nm that
// makes occupied-occupied pairs cancel holds exactly even when v is only Hermitian to FP32
// rounding.  Per-thread row / column partials go to `red` (2 * n_eta * W * 16 doubles, may
// alias sVx: a barrier separates the last read of sVx from the first write of red) and are
// summed in a fixed order (deterministic).
//
// FP32 velocities (V = float2): the numerator carries FP32 rounding already, so the quotient
// T = num / (dE^2 + eta^2) is formed in FP32 too; only dE = E_n - E_m (a difference of close
// FP64 eigenvalues), its square and the eta = 0 cut-off stay in FP64.  The numerator is
// Kahan's difference of products (within 2 ulp of the exact Im part), and the partial sums are
// exact FP32 pairs (Knuth's TwoSum): a large term of a near-degenerate pair enters Omega_n and
// Omega_m with the same rounded value and no accumulation error, so it still cancels when
// both bands are occupied.  Every term is bounded (|num| <= 2 |v^x| |v^y|) while the FP32
// denominator is at least 2^-86; a thread whose tile holds a smaller one (eta and a gap below
// ~1e-13) takes the FP64 quotient for that eta.
template <int TM, typename V>
__device__ __forceinline__ void curvature_epilogue(const V* sVx, const V (&vy)[TM][TM],
                                                   const double* sE, const double* sEta,
                                                   int n_eta, double emax, int W, int LD, int ty,
                                                   int tx, int t, double* red,
                                                   double* __restrict__ Om, int64_t eta_stride,
                                                   int64_t k) {
  constexpr bool F32 = std::is_same<V, float2>::value;
  using R = typename std::conditional<F32, float, double>::type;
  const double thr2 = (1e-12 * emax) * (1e-12 * emax);
  R num[TM][TM];
  // (dE)^2 per pair: FP64 for FP64 velocities; for FP32 ones only its FP32 rounding is kept
  // (the FP64 fallback recomputes it), and the pair / cut-off tests are bit masks, so that the
  // per-eta loop issues no FP64 compare
  double d2[F32 ? 1 : TM][F32 ? 1 : TM];
  float d2f[TM][TM];
  unsigned pairs = 0;    // bit (i TM + j): n < m < W
  unsigned small0 = 0;   // bit (i TM + j): (dE)^2 <= thr2 (dropped when eta = 0)
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int n = ty + 16 * i;
#pragma unroll
    for (int j = 0; j < TM; ++j) {
      const int m = tx + 16 * j;
      num[i][j] = 0;
      d2f[i][j] = 0.f;
      if (n < W && m < W && n < m) {
        pairs |= 1u << (i * TM + j);
        const V vx = sVx[n * LD + m];
        if constexpr (F32)
          num[i][j] = -2.0f * diff_of_products(vx.y, vy[i][j].x, vx.x, vy[i][j].y);
        else
          num[i][j] = -2.0 * (vx.y * vy[i][j].x - vx.x * vy[i][j].y);
        const double dE = sE[n] - sE[m];
        const double q = dE * dE;
        if constexpr (F32) d2f[i][j] = (float)q;
        else d2[i][j] = q;
        if (q <= thr2) small0 |= 1u << (i * TM + j);
      }
    }
  }
  __syncthreads();
  for (int e = 0; e < n_eta; ++e) {
    const double eta = sEta[e];
    const bool eta0 = eta == 0.0;
    R rp[TM], cp[TM], rl[TM], cl[TM];   // (rl, cl: the FP32 pairs' low parts)
#pragma unroll
    for (int i = 0; i < TM; ++i) { rp[i] = 0; cp[i] = 0; rl[i] = 0; cl[i] = 0; }
    bool fp64 = !F32;
    if constexpr (F32) {
      const float eta2 = (float)(eta * eta);
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM; ++j) {
          if (!((pairs >> (i * TM + j)) & 1u)) continue;
          if (eta0 && ((small0 >> (i * TM + j)) & 1u)) continue;
          const float den = d2f[i][j] + eta2;
          if (den < 0x1p-86f) fp64 = true;
          const float T = num[i][j] / den;
          two_sum_acc(rp[i], rl[i], T);
          two_sum_acc(cp[j], cl[j], -T);
        }
    }
    if (fp64) {
      double rq[TM], cq[TM];
#pragma unroll
      for (int i = 0; i < TM; ++i) { rq[i] = 0.0; cq[i] = 0.0; }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM; ++j) {
          if (!((pairs >> (i * TM + j)) & 1u)) continue;
          if (eta0 && ((small0 >> (i * TM + j)) & 1u)) continue;
          double q;
          if constexpr (F32) {
            const double dE = sE[ty + 16 * i] - sE[tx + 16 * j];
            q = dE * dE;
          } else {
            q = d2[i][j];
          }
          const double T = (double)num[i][j] / fma(eta, eta, q);
          rq[i] += T;
          cq[j] -= T;
        }
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        const int n = ty + 16 * i;
        if (n < W) red[((size_t)(e * W + n) * 2) * 16 + tx] = rq[i];
        const int m = tx + 16 * i;
        if (m < W) red[((size_t)(e * W + m) * 2 + 1) * 16 + ty] = cq[i];
      }
    } else {
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        const int n = ty + 16 * i;
        if (n < W) red[((size_t)(e * W + n) * 2) * 16 + tx] = (double)rp[i] + (double)rl[i];
        const int m = tx + 16 * i;
        if (m < W) red[((size_t)(e * W + m) * 2 + 1) * 16 + ty] = (double)cp[i] + (double)cl[i];
      }
    }
  }
  __syncthreads();
  const FastDiv dW(W);
  for (int idx = t; idx < n_eta * W; idx += NT) {
    const int e = (int)dW.div(idx), n = idx - e * W;
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

  const FastDiv dW(W);
  for (int idx = t; idx < W * W; idx += NT) {
    const int r = (int)dW.div(idx);
    sU[r * LD + idx - r * W] = U[k * WW + idx];
  }
  unpack_hermitian(Xp + k * ld, sA, W, LD, t);
  for (int j = t; j < W; j += NT) sE[j] = E[k * W + j];
  if (t < n_eta) sEta[t] = etas[t];
  __syncthreads();
  emax_warp0(sE, W, t, &s_emax);

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
  const FastDiv dW(W);
  for (int idx = t; idx < W * W; idx += NT) {
    const int i = (int)dW.div(idx), j = idx - i * W;
    float2 a;
    if (i < j) a = make_float2((float)P[i * W + j], (float)P[j * W + i]);
    else if (i > j) a = make_float2((float)P[j * W + i], -(float)P[i * W + j]);
    else a = make_float2((float)P[i * W + i], 0.f);
    A[i * LD + j] = a;
  }
}

// U = Q D Z in FP32, in shared memory, from the FP64 factors of the eigensolver: Z (eigenvectors
// of the real tridiagonal, [W][W]), the phases D and the Householder reflectors (staged in
// `stage`, W (W - 1) / 2 complex, then 2 ceil((W - 2) / 4) x 16 complex of block factors).
// The only consumer of this U is the FP32 rotation, so it is formed at that precision.
//
// Q = H_0 H_1 ... H_{W-3} is applied in blocks of ASM_NB consecutive reflectors in the compact
// WY form H_j0 ... H_j0+3 = I - V T V^H (T upper triangular: T_ii = tau_i,
// T[0:i, i] = -tau_i T[0:i, 0:i] V[:, 0:i]^H v_i), last block first: U <- U - V (T (V^H U)).
// The block factors are formed once from the reflectors' inner products; each group of 4
// threads then applies a block to one column with ASM_NB independent dot chains, so the
// application is ceil((W - 2) / 4) dependent steps instead of W - 2.  (Blocks of 16 applied
// as register-tiled products were measured slower: their per-block serial phases are not
// hidden at two CTAs per SM.)
constexpr int ASM_NB = 4;

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ void assemble_u_f32(const double* __restrict__ Zk,
                                               const double2* __restrict__ ph,
                                               const double2* __restrict__ R,
                                               const double* __restrict__ tau, int W, int LD,
                                               int t, float2* sU, float2* stage) {
  auto roff = [&](int j) { return j * (W - 1) - (j * (j - 1)) / 2; };   // sum_{j'<j} (W-1-j')
  // the phases in FP32 once per row (the FP64 -> FP32 conversions issue on the FP64 pipe)
  __shared__ float2 sPh[64];   // W <= 64
  for (int j = t; j < W; j += NT) {
    const double2 p = ph[j];
    sPh[j] = make_float2((float)p.x, (float)p.y);
  }
  __syncthreads();
  const FastDiv dW(W);
  for (int idx = t; idx < W * W; idx += NT) {
    const int r = (int)dW.div(idx), c = idx - r * W;
    const float z = (float)Zk[idx];
    const float2 p = sPh[r];
    sU[r * LD + c] = make_float2(p.x * z, p.y * z);
    if (r > c && c < W - 2) {
      const double2 v = R[idx];
      stage[roff(c) + (r - c - 1)] = make_float2((float)v.x, (float)v.y);
    }
  }
  const int nref = W > 2 ? W - 2 : 0;
  const int nblk = (nref + ASM_NB - 1) / ASM_NB;
  float2* G = stage + W * (W - 1) / 2;        // [nblk][NB][NB]: v_a^H v_b (a < b)
  float2* Tm = G + nblk * ASM_NB * ASM_NB;    // [nblk][NB][NB]: T (upper triangular)
  __syncthreads();
  for (int d = t; d < nblk * ASM_NB * ASM_NB; d += NT) {
    const int bk = d / (ASM_NB * ASM_NB), a = (d / ASM_NB) % ASM_NB, a2 = d % ASM_NB;
    const int j0 = bk * ASM_NB, nj = min(ASM_NB, nref - j0), m0 = W - 1 - j0;
    float2 g = make_float2(0.f, 0.f);
    if (a < a2 && a2 < nj) {
      // rows j0 + 1 + rr, rr >= a2 (v_b vanishes above its first row)
      const float2* va = stage + roff(j0 + a) - a;
      const float2* vb = stage + roff(j0 + a2) - a2;
      for (int rr = a2; rr < m0; ++rr) {
        const float2 x = va[rr], y = vb[rr];
        g.x = fmaf(x.x, y.x, fmaf(x.y, y.y, g.x));   // conj(x) y
        g.y = fmaf(x.x, y.y, fmaf(-x.y, y.x, g.y));
      }
    }
    G[d] = g;
  }
  __syncthreads();
  for (int bk = t; bk < nblk; bk += NT) {
    const int j0 = bk * ASM_NB, nj = min(ASM_NB, nref - j0);
    float2* Tb = Tm + bk * ASM_NB * ASM_NB;
    const float2* Gb = G + bk * ASM_NB * ASM_NB;
    for (int e = 0; e < ASM_NB * ASM_NB; ++e) Tb[e] = make_float2(0.f, 0.f);
    for (int i = 0; i < nj; ++i) {
      const float ti = (float)tau[j0 + i];
      Tb[i * ASM_NB + i] = make_float2(ti, 0.f);
      for (int a = 0; a < i; ++a) {
        float2 acc = make_float2(0.f, 0.f);
        for (int k2 = a; k2 < i; ++k2) {
          const float2 pr = cmulf(Tb[a * ASM_NB + k2], Gb[k2 * ASM_NB + i]);
          acc.x += pr.x;
          acc.y += pr.y;
        }
        Tb[a * ASM_NB + i] = make_float2(-ti * acc.x, -ti * acc.y);
      }
    }
  }
  __syncthreads();
  // NT / 4 = 64 groups of four row lanes, one column each (W <= 64): the dot products of a
  // block are reduced over four lanes (two shuffle rounds of 2 ASM_NB values; with two columns
  // per group of eight lanes the three rounds of 4 ASM_NB values cost as much as the dot
  // products themselves).  A warp touches 4 rows x 8 columns of U: conflict-free with the
  // padded row (8 banks per row step).
  const int q = t & 3, c0 = t >> 2;
  const bool act0 = c0 < W;
  for (int bk = nblk - 1; bk >= 0; --bk) {
    const int j0 = bk * ASM_NB, nj = min(ASM_NB, nref - j0), m0 = W - 1 - j0, o = j0 + 1;
    const float2* Tb = Tm + bk * ASM_NB * ASM_NB;
    float2 s0[ASM_NB];
#pragma unroll
    for (int a = 0; a < ASM_NB; ++a) s0[a] = make_float2(0.f, 0.f);
    for (int rr = q; rr < m0; rr += 4) {
      const float2 u0 = act0 ? sU[(o + rr) * LD + c0] : make_float2(0.f, 0.f);
#pragma unroll
      for (int a = 0; a < ASM_NB; ++a) {
        if (a < nj && rr >= a) {
          const float2 v = stage[roff(j0 + a) + rr - a];
          s0[a].x = fmaf(v.x, u0.x, fmaf(v.y, u0.y, s0[a].x));   // conj(v) u
          s0[a].y = fmaf(v.x, u0.y, fmaf(-v.y, u0.x, s0[a].y));
        }
      }
    }
#pragma unroll
    for (int a = 0; a < ASM_NB; ++a)
#pragma unroll
      for (int o2 = 1; o2 < 4; o2 <<= 1) {
        s0[a].x += __shfl_xor_sync(0xffffffffu, s0[a].x, o2);
        s0[a].y += __shfl_xor_sync(0xffffffffu, s0[a].y, o2);
      }
    // t = T s (upper triangular)
    float2 t0[ASM_NB];
#pragma unroll
    for (int a = 0; a < ASM_NB; ++a) {
      t0[a] = make_float2(0.f, 0.f);
#pragma unroll
      for (int a2 = a; a2 < ASM_NB; ++a2) {
        const float2 p0 = cmulf(Tb[a * ASM_NB + a2], s0[a2]);
        t0[a].x += p0.x; t0[a].y += p0.y;
      }
    }
    for (int rr = q; rr < m0; rr += 4) {
      float2 u0 = act0 ? sU[(o + rr) * LD + c0] : make_float2(0.f, 0.f);
#pragma unroll
      for (int a = 0; a < ASM_NB; ++a) {
        if (a < nj && rr >= a) {
          const float2 v = stage[roff(j0 + a) + rr - a];
          u0.x = fmaf(-v.x, t0[a].x, fmaf(v.y, t0[a].y, u0.x));   // u -= v t
          u0.y = fmaf(-v.x, t0[a].y, fmaf(-v.y, t0[a].x, u0.y));
        }
      }
      if (act0) sU[(o + rr) * LD + c0] = u0;
    }
    __syncwarp();   // the group's rows shift between blocks: updates before the next reads
  }
  __syncthreads();
}

// U = Q D Z in FP32 as a kernel of its own (one CTA per k-point, several per SM), for the
// tensor-core rotation: U32 [n][W][W] float2, row-major.
__global__ void __launch_bounds__(NT) assemble_u_kernel(const double* __restrict__ Z, EighBufs eb,
                                                        float2* __restrict__ U32, int W, int LD) {
  extern __shared__ float2 au_smem[];
  float2* sU = au_smem;
  float2* stage = au_smem + (size_t)W * LD;
  const int64_t k = blockIdx.x;
  const int t = threadIdx.x;
  const size_t WW = (size_t)W * W;
  assemble_u_f32(Z + k * WW, eb.phase + k * W, eb.refl + k * WW, eb.tau + k * W, W, LD, t, sU,
                 stage);
  float2* dst = U32 + k * WW;
  const FastDiv dW(W);
  for (int idx = t; idx < W * W; idx += NT) {
    const int r = (int)dW.div(idx);
    dst[idx] = sU[r * LD + (idx - r * W)];
  }
}

// Leading dimension (in float2) of the FP32 shared-memory matrices.  Padded: W + P with
// W + P = 4 (mod 16), so that a row step moves 8 banks: the 4 rows x 4 columns of float2 that
// a half warp touches in the reflector application (four row lanes per column), and the 16
// consecutive columns of a half warp elsewhere, fall on distinct banks.  Unpadded (the
// ablation): W.
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
    const FastDiv dW(W);
    for (int idx = t; idx < W * W; idx += NT) {
      const double2 u = U[k * WW + idx];
      const int r = (int)dW.div(idx);
      sU[r * LD + idx - r * W] = make_float2((float)u.x, (float)u.y);
    }
  }
  unpack_hermitian_f32(Xp + k * ld, sA, W, LD, t);
  for (int j = t; j < W; j += NT) sE[j] = E[k * W + j];
  if (t < n_eta) sEta[t] = etas[t];
  __syncthreads();
  emax_warp0(sE, W, t, &s_emax);

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


// ------------------------------------------------------------------ rotations on the tensor cores
// Step (3) as exact fixed-point products on tcgen05 (the scheme of the tensor-core Fourier sum):
// every operand is scaled by a power of two to |x| <= 1 and cut into four 8-bit integer slices
// held exactly in BF16 (x = sum_i s_i 2^(-7-8i) + O(2^-32)); the ten slice pairs with i + j <= 3
// are multiplied into one FP32 TMEM accumulator per level l = i + j, where every partial sum
// is an integer below 2^24 (exact), and the levels are folded in int64.  The complex products
// are block-real GEMMs with M = 128, N = 64, K = 128 (W padded to 64):
//   T = X U:    [T_r; T_i] = [[X_r, -X_i], [X_i, X_r]] [U_r; U_i]
//   V = U^H T:  [V_r; V_i] = [[U_r^T, U_i^T], [-U_i^T, U_r^T]] [T_r; T_i]
// U = Q D Z is assembled in FP32 in shared memory first (its FP32 rounding is the dominant
// error, ~1e-7); T is re-sliced with its own exponent for the second product.  V^x waits in
// TMEM while V^y is formed; the curvature uses FP64 denominators as in the SIMT kernels.
// One persistent CTA per SM (226 KB of shared memory), k-points in turn.
constexpr int RT_NT = 256;
constexpr int RT_WP = 64;                                 // padded order
constexpr int RT_NS = 4;                                  // slices per operand
constexpr int RT_A_BLOCK = 128 * 128;                     // bytes: 128 rows x 64 K (BF16)
constexpr int RT_B_BLOCK = 64 * 128;                      // bytes: 64 rows x 64 K
constexpr int RT_A_BYTES = RT_NS * 2 * RT_A_BLOCK;        // 128 KB (4 slices x 2 K halves)
constexpr int RT_B_BYTES = RT_NS * 2 * RT_B_BLOCK;        // 64 KB
constexpr int RT_U_BYTES = RT_WP * RT_WP * 8;             // float2 [64][64]
constexpr int RT_TMEM_COLS = 512;                         // 4 levels x 64 + V^x (64)
constexpr int RT_VX_COL = 256;
constexpr uint32_t RT_WAIT_LIMIT = 1u << 20;              // a product takes microseconds
// instruction descriptor: kind::f16, BF16 operands, F32 accumulator, K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t rt_idesc_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// byte offset of element (row, k in 0..63) in a K-major 128-byte-swizzled block of 2-byte elements
__device__ __forceinline__ uint32_t sw128_off(int row, int k) {
  const uint32_t b = (uint32_t)k * 2u;
  return (uint32_t)row * 128u + ((((b >> 4) ^ (uint32_t)(row & 7)) & 7u) << 4) + (b & 15u);
}

// The operands are 31-bit fixed-point integers q (value q 2^-31, |q| <= 2^31 - 1) cut into
// four signed 8-bit slices with round-to-nearest carries in 32-bit integer arithmetic (no FP64
// and no 64-bit conversions, which share the slow FP64 pipe):
// q = s0 2^24 + s1 2^16 + s2 2^8 + s3, |s_i| <= 128, each exact in BF16.  round(q / 2^24) is
// formed as (floor(q / 2^23) + 1) >> 1, which cannot overflow; the remainder q - s0 2^24 lies
// in [-2^23, 2^23] and is formed modulo 2^32.
__device__ __forceinline__ void slice4(int q, uint16_t (&o)[RT_NS]) {
  const int s0 = ((q >> 23) + 1) >> 1;
  int r = (int)((uint32_t)q - ((uint32_t)s0 << 24));
  const int s1 = ((r >> 15) + 1) >> 1;
  r -= s1 * 65536;
  const int s2 = ((r >> 7) + 1) >> 1;
  const int s3 = r - s2 * 256;
  o[0] = __bfloat16_as_ushort(__int2bfloat16_rn(s0));
  o[1] = __bfloat16_as_ushort(__int2bfloat16_rn(s1));
  o[2] = __bfloat16_as_ushort(__int2bfloat16_rn(s2));
  o[3] = __bfloat16_as_ushort(__int2bfloat16_rn(s3));
}

constexpr int RT_QMAX = 2147483647;

// round(x 2^(31 - e)) for |x| <= 2^e (clamped to 2^31 - 1), from the bit pattern
__device__ __forceinline__ int fixed31(double x, int e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  const int sh = 1044 + e - ex;   // x 2^(31-e) = m 2^(ex - 1075 + 31 - e) = m 2^-sh
  if (ex == 0 || sh >= 63) return 0;   // zero, subnormal, or below half a unit
  const unsigned long long m = (b & ((1ull << 52) - 1)) | (1ull << 52);
  const unsigned long long q = sh <= 21 ? (1ull << 31) : (m + (1ull << (sh - 1))) >> sh;
  const int qi = q > (unsigned long long)RT_QMAX ? RT_QMAX : (int)q;
  return (b >> 63) ? -qi : qi;
}
// round(u 2^31) for an FP32 value |u| <= 1 (the conversion saturates at 2^31 - 1)
__device__ __forceinline__ int fixed31f(float u) { return __float2int_rn(u * 2147483648.0f); }

// |x| as an ordered unsigned integer (FP64 bit pattern), and the smallest e with |x| <= 2^e
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ int pow2_exponent_bits(unsigned long long ab) {
  if (ab == 0) return 0;
  const int ex = (int)(ab >> 52) - 1023;
  return (ab & ((1ull << 52) - 1)) ? ex + 1 : ex;
}

// store a pair of adjacent-K elements (k even) of all slices into the operand region
__device__ __forceinline__ void put2(unsigned char* region, int block_bytes, int row, int k,
                                     int v0, int v1) {
  uint16_t a[RT_NS], b[RT_NS];
  slice4(v0, a);
  slice4(v1, b);
  const int kc = k >> 6, kin = k & 63;
#pragma unroll
  for (int i = 0; i < RT_NS; ++i) {
    unsigned char* blk = region + (size_t)(kc * RT_NS + i) * block_bytes;
    *reinterpret_cast<uint32_t*>(blk + sw128_off(row, kin)) = (uint32_t)a[i] | ((uint32_t)b[i] << 16);
  }
}

// issue the 32 MMAs of one block-real product (4 A slices x 2 K halves x 4 K16 steps): the
// slice blocks of a K half are consecutive ([K half][slice]), so slices 0 .. 3-i of B form one
// K-major operand of N = 64 (4 - i) rows whose accumulator columns are those of levels i + j
// (levels contiguous in TMEM); A_0 comes first and initialises every level.
__device__ __forceinline__ void rot_issue(uint32_t tmem, uint32_t a_base, uint32_t b_base) {
  for (int kc = 0; kc < 2; ++kc)
    for (int kk = 0; kk < 4; ++kk) {
      const uint64_t db = tc::umma_desc_sw128(b_base + (uint32_t)(kc * RT_NS * RT_B_BLOCK + kk * 32));
#pragma unroll
      for (int i = 0; i < RT_NS; ++i) {
        const uint32_t acc = (i > 0 || kc > 0 || kk > 0) ? 1u : 0u;
        const uint64_t da = tc::umma_desc_sw128(a_base + (uint32_t)((kc * RT_NS + i) * RT_A_BLOCK + kk * 32));
        tc::umma_bf16(tmem + (uint32_t)(i * 64), da, db, rt_idesc_n(64 * (RT_NS - i)), acc);
      }
    }
}

// the 32 columns c0 .. c0 + 31 of this thread's TMEM lane, folded over the four levels:
// value = isum 2^(-46) in units of the operands' scales (exact integers)
__device__ __forceinline__ void rot_fold(uint32_t lane_addr, int c0, long long (&isum)[32]) {
#pragma unroll
  for (int j = 0; j < 32; ++j) isum[j] = 0;
#pragma unroll
  for (int l = 0; l < 4; ++l) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint32_t r[16];
      tc::tmem_ld16(lane_addr + (uint32_t)(l * 64 + c0 + 16 * h), r);
#pragma unroll
      for (int j = 0; j < 16; ++j)
        isum[16 * h + j] += (long long)__float2int_rn(__uint_as_float(r[j])) << (32 - 8 * l);
    }
  }
}

// block-wide maximum of 64-bit unsigned integers (256 threads)
__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v,
                                                            unsigned long long* red8) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red8[w] = v;
  __syncthreads();
  unsigned long long m = 0;
  for (int i = 0; i < RT_NT / 32; ++i) m = max(m, red8[i]);
  return m;
}

// an exact integer |v| < 2^62 to FP32 with 32-bit conversions only (two parts; the sum is
// rounded twice, an error below 2^-23 relative)
__device__ __forceinline__ float ll_to_float(long long v) {
  const int hi = (int)(v >> 31);
  const int lo = (int)(v & 0x7FFFFFFF);
  return fmaf((float)hi, 2147483648.0f, (float)lo);
}

template <typename TIn>
__global__ void __launch_bounds__(RT_NT, 1) berry_tc_kernel(
    const double* __restrict__ E, const double* __restrict__ Z, EighBufs eb,
    const TIn* __restrict__ Xp, const TIn* __restrict__ Yp, int64_t ld, int W, int n,
    const double* __restrict__ etas, int n_eta, double* __restrict__ Om, int64_t eta_stride,
    DevStatus* st) {
  extern __shared__ unsigned char rt_smem[];
  __shared__ double sE[64];
  __shared__ double sEta[MAXE];
  __shared__ double s_emax;
  __shared__ unsigned long long redl[RT_NT / 32];
  __shared__ __align__(8) uint64_t mma_bar;
  __shared__ uint32_t tmem_sh;
  __shared__ int s_ok;
  // [U float2 64 x 64][pad to 1024][A operand 128 KB][B operand 64 KB]
  float2* sU = reinterpret_cast<float2*>(rt_smem);
  unsigned char* opA = reinterpret_cast<unsigned char*>(
      ((uintptr_t)(rt_smem + RT_U_BYTES) + 1023) & ~(uintptr_t)1023);
  unsigned char* opB = opA + RT_A_BYTES;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int LDV = mixed_ld(RT_WP, 1);   // 68: the curvature matrices live in opB / opA
  const size_t WW = (size_t)W * W;

  if (t == 0) {
    tc::mbar_init(&mma_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc::smem_u32(&tmem_sh)), "r"(RT_TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_sh;
  const uint32_t a_base = tc::smem_u32(opA), b_base = tc::smem_u32(opB);
  // TMEM lane quarter and column half of this warp in the epilogues
  const int quarter = warp & 3, chalf = warp >> 2;
  const int mrow = quarter * 32 + lane;                   // row of [.._r; .._i]
  const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
  uint32_t phase = 0;
  bool ok = true;

  // run the MMAs of one product and wait (bounded) for them; false on timeout
  auto product = [&]() -> bool {
    tc::fence_proxy_async_smem();
    __syncthreads();
    if (t == 0) {
      tc::tc_fence_after();
      rot_issue(tmem, a_base, b_base);
      tc::umma_commit(&mma_bar);
      s_ok = tc::mbar_wait(&mma_bar, phase, RT_WAIT_LIMIT) ? 1 : 0;
    }
    __syncthreads();
    phase ^= 1u;
    tc::tc_fence_after();
    return s_ok != 0;
  };

  for (int64_t k = blockIdx.x; k < n && ok; k += gridDim.x) {
    __syncthreads();
    if (t < W) sE[t] = E[k * W + t];
    if (t < n_eta) sEta[t] = etas[t];
    // ---- U = Q D Z in FP32 (reflectors staged in the A operand region)
    for (int idx = t; idx < RT_WP * RT_WP; idx += RT_NT) sU[idx] = make_float2(0.f, 0.f);
    __syncthreads();
    assemble_u_f32(Z + k * WW, eb.phase + k * W, eb.refl + k * WW, eb.tau + k * W, W, RT_WP, t, sU,
                   reinterpret_cast<float2*>(opA));
    emax_warp0(sE, W, t, &s_emax);
    for (int a = 0; a < 2 && ok; ++a) {
      const TIn* P = (a == 0 ? Xp : Yp) + k * ld;
      // ---- A1 = [[X_r, -X_i], [X_i, X_r]] 2^-eX (W padded to 64)
      unsigned long long mx = 0;
      for (int idx = t; idx < W * W; idx += RT_NT) mx = max(mx, abs_bits(P[idx]));
      const int eX = pow2_exponent_bits(block_max_u64(mx, redl));
      for (int idx = t; idx < RT_WP * RT_WP / 2; idx += RT_NT) {
        const int r = idx / (RT_WP / 2), c = 2 * (idx % (RT_WP / 2));
        int qr[2] = {0, 0}, qi[2] = {0, 0};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int cc = c + q;
          if (r < W && cc < W) {
            if (r < cc) { qr[q] = fixed31(P[r * W + cc], eX); qi[q] = fixed31(P[cc * W + r], eX); }
            else if (r > cc) { qr[q] = fixed31(P[cc * W + r], eX); qi[q] = -fixed31(P[r * W + cc], eX); }
            else qr[q] = fixed31(P[r * W + r], eX);
          }
        }
        const int qr0 = qr[0], qr1 = qr[1], qi0 = qi[0], qi1 = qi[1];
        put2(opA, RT_A_BLOCK, r, c, qr0, qr1);
        put2(opA, RT_A_BLOCK, r, 64 + c, -qi0, -qi1);
        put2(opA, RT_A_BLOCK, 64 + r, c, qi0, qi1);
        put2(opA, RT_A_BLOCK, 64 + r, 64 + c, qr0, qr1);
      }
      // ---- B1[n][k] = U_r[k][n] (k < 64), U_i[k-64][n] (|U| <= 1: no scale)
      for (int idx = t; idx < RT_WP * RT_WP / 2; idx += RT_NT) {
        const int nn = idx / (RT_WP / 2), kk = 2 * (idx % (RT_WP / 2));
        const float2 u0 = sU[kk * RT_WP + nn], u1 = sU[(kk + 1) * RT_WP + nn];
        put2(opB, RT_B_BLOCK, nn, kk, fixed31f(u0.x), fixed31f(u1.x));
        put2(opB, RT_B_BLOCK, nn, 64 + kk, fixed31f(u0.y), fixed31f(u1.y));
      }
      if (!product()) { ok = false; break; }
      // ---- T' = [T_r; T_i] 2^-eX = isum 2^-46 from TMEM; re-cut as 31-bit fixed point
      // q = round(isum 2^-sh) with the smallest sh >= 0 that keeps |q| <= 2^31
      long long tv[32];
      rot_fold(lane_addr, chalf * 32, tv);
      unsigned long long tm = 0;
#pragma unroll
      for (int j = 0; j < 32; ++j) tm = max(tm, (unsigned long long)(tv[j] < 0 ? -tv[j] : tv[j]));
      tc::tc_fence_before();
      const unsigned long long tmax = block_max_u64(tm, redl);
      const int bits = tmax > 0 ? 64 - __clzll((long long)tmax) : 0;
      const int sh = bits > 31 ? bits - 31 : 0;
#pragma unroll
      for (int j = 0; j < 32; j += 2) {
        // B2 row = output column n of T, K index = mrow; a pair of adjacent K needs the
        // neighbouring lane's value (rounding can reach 2^31: clamp)
        const int v0 = (int)min((sh ? (tv[j] + (1ll << (sh - 1))) >> sh : tv[j]), (long long)RT_QMAX);
        const int v1 = (int)min((sh ? (tv[j + 1] + (1ll << (sh - 1))) >> sh : tv[j + 1]), (long long)RT_QMAX);
        const int w0 = __shfl_down_sync(0xffffffffu, v0, 1);
        const int w1 = __shfl_down_sync(0xffffffffu, v1, 1);
        if ((lane & 1) == 0) {
          put2(opB, RT_B_BLOCK, chalf * 32 + j, mrow, v0, w0);
          put2(opB, RT_B_BLOCK, chalf * 32 + j + 1, mrow, v1, w1);
        }
      }
      // ---- A2 = [[U_r^T, U_i^T], [-U_i^T, U_r^T]]
      for (int idx = t; idx < RT_WP * RT_WP / 2; idx += RT_NT) {
        const int r = idx / (RT_WP / 2), c = 2 * (idx % (RT_WP / 2));
        const float2 u0 = sU[c * RT_WP + r], u1 = sU[(c + 1) * RT_WP + r];   // U[c][r], U[c+1][r]
        const int ar0 = fixed31f(u0.x), ar1 = fixed31f(u1.x);
        const int ai0 = fixed31f(u0.y), ai1 = fixed31f(u1.y);
        put2(opA, RT_A_BLOCK, r, c, ar0, ar1);
        put2(opA, RT_A_BLOCK, r, 64 + c, ai0, ai1);
        put2(opA, RT_A_BLOCK, 64 + r, c, -ai0, -ai1);
        put2(opA, RT_A_BLOCK, 64 + r, 64 + c, ar0, ar1);
      }
      if (!product()) { ok = false; break; }
      // ---- V = [V_r; V_i]: the B2 slices stood for T' 2^(sh - 15) (q 2^-31 = isum 2^(sh-46)),
      // so V = isum2 2^-46 2^(sh - 15) 2^eX
      long long vi[32];
      rot_fold(lane_addr, chalf * 32, vi);
      const float sV = ldexpf(1.0f, eX + sh - 61);
      float vv[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) vv[j] = ll_to_float(vi[j]) * sV;
      if (a == 0) {
        // park V^x in TMEM columns RT_VX_COL.. (FP32) while V^y is formed
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t r[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) r[j] = __float_as_uint(vv[16 * h + j]);
          tc::tmem_st16(lane_addr + (uint32_t)(RT_VX_COL + chalf * 32 + 16 * h), r);
        }
        tc::tc_fence_before();
      } else {
        // V^y -> opA (float2 [64][LDV]), V^x (TMEM) -> opB
        float2* sVy = reinterpret_cast<float2*>(opA);
        float2* sVx = reinterpret_cast<float2*>(opB);
        __syncthreads();   // the product's operands are no longer read (it completed)
        const int rr = mrow & 63;
        const bool im = mrow >= 64;
        uint32_t px[32];
        tc::tmem_ld16(lane_addr + (uint32_t)(RT_VX_COL + chalf * 32), *reinterpret_cast<uint32_t(*)[16]>(px));
        tc::tmem_ld16(lane_addr + (uint32_t)(RT_VX_COL + chalf * 32 + 16), *reinterpret_cast<uint32_t(*)[16]>(px + 16));
        tc::tc_fence_before();
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int cn = chalf * 32 + j;
          float* vy = reinterpret_cast<float*>(&sVy[rr * LDV + cn]);
          float* vx = reinterpret_cast<float*>(&sVx[rr * LDV + cn]);
          vy[im ? 1 : 0] = vv[j];
          vx[im ? 1 : 0] = __uint_as_float(px[j]);
        }
      }
    }
    if (!ok) break;
    __syncthreads();
    // ---- curvature (FP64 denominators), as the SIMT kernels
    {
      const int tx = t & 15, ty = t >> 4;
      const float2* sVx = reinterpret_cast<const float2*>(opB);
      const float2* sVy = reinterpret_cast<const float2*>(opA);
      float2 vy[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) vy[i][j] = sVy[(ty + 16 * i) * LDV + tx + 16 * j];
      curvature_epilogue<4, float2>(sVx, vy, sE, sEta, n_eta, s_emax, W, LDV, ty, tx, t,
                                    reinterpret_cast<double*>(opA), Om, eta_stride, k);
    }
  }
  if (!ok && t == 0) atomicOr(&st->bits, ST_TIMEOUT);
  // no MMA may still write TMEM when it is released
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    if (lane == 0 && !ok) tc::mbar_wait(&mma_bar, phase, RT_WAIT_LIMIT);
    __syncwarp();
    tc::tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(RT_TMEM_COLS) : "memory");
  }
}

// ------------------------------------------------------------------ rotations in 3xTF32
// Step (3) on tcgen05 with kind::tf32 operands and FP32 accumulation in TMEM (the split-TF32
// scheme): every FP32 operand x is cut into hi = tf32(x) and lo = tf32(x - hi) (11 + 11
// significant bits, the cut exact), and a product is formed as hi lo + lo hi + hi hi; the
// dropped lo lo and the cut's residual are ~2^-24 relative: FP32-grade.  The tensor core's
// additions into its FP32 accumulator truncate, so each K phase of 32 (12 MMAs, the small
// cross terms first) starts a fresh accumulator and the phases are summed in registers with
// round-to-nearest: on the W = 64 workload this rotation is then slightly more accurate than
// the SIMT FP32 one (all 48 MMAs in one accumulator were ten times less accurate).
// The complex products are block-real GEMMs with M = 128, N = 64, K = 128 (W padded to 64):
//   T = X U:    [T_r; T_i] = [[X_r, -X_i], [X_i, X_r]] [U_r; U_i]
//   V = U^H T:  [V_r; V_i] = [[U_r^T, U_i^T], [-U_i^T, U_r^T]] [T_r; T_i]
// T is held in registers (each thread 32 entries of one row of [T_r; T_i], which is one K
// column of the second product's B operand); V^x waits in TMEM while V^y is formed.  The
// operands are staged one K phase (32 TF32 = one 128-byte swizzle row) at a time, 48 KB for
// A and B with their hi / lo parts -- a phase pairs 16 K of the real-part half with the same 16
// of the imaginary-part half, so that every block-real row pair is formed from one load and
// one split per value -- so that with U (FP32, assembled from the FP64 factors in
// shared memory) and the packed FP32 velocity rows (copied asynchronously into shared memory,
// rows of W + 1 floats: X while U is assembled, Y while the second product of X runs) a CTA
// needs ~100 KB and two CTAs share an SM: one stages operands while the other's MMAs run.
// Persistent over the k-points; every wait on the tensor core is bounded (ST_TIMEOUT).
constexpr int TF_NT = 256;
constexpr int TF_WP = 64;
constexpr int TF_A_TILE = 128 * 128;   // bytes: 128 rows x 32 TF32
constexpr int TF_B_TILE = 64 * 128;    // bytes: 64 rows x 32 TF32
constexpr int TF_OPS_BYTES = 2 * TF_A_TILE + 2 * TF_B_TILE;   // A hi, A lo, B hi, B lo: 48 KB
constexpr int TF_LDU = 68;                                    // = mixed_ld(64, 1)
constexpr int TF_U_BYTES = TF_WP * TF_LDU * 8;                // 34,816
constexpr int TF_X_BYTES = TF_WP * (TF_WP + 1) * 4;         // FP32 velocity, rows of W + 1
constexpr int TF_TMEM_COLS = 256;   // partial T at 0, partial V at 64, parked V^x at 128
constexpr uint32_t TF_WAIT_LIMIT = 1u << 20;
// instruction descriptor: D F32, A and B TF32 (K-major), N = 64, M = 128
constexpr uint32_t TF_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(64 >> 3) << 17) |
                              ((uint32_t)(128 >> 4) << 24);

// byte offset of element (row, k in 0..31) in a K-major 128-byte-swizzled tile of 4-byte elements
__device__ __forceinline__ uint32_t sw128_off32(int row, int k) {
  const uint32_t b = (uint32_t)k * 4u;
  return (uint32_t)row * 128u + ((((b >> 4) ^ (uint32_t)(row & 7)) & 7u) << 4) + (b & 15u);
}

// 4-byte asynchronous global -> shared copy (completion: cp_async_wait_all, then a barrier)
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(tc::smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(tc::smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
// x = hi + lo + O(2^-22 |x|), both TF32 (low 13 mantissa bits zero); x - hi is exact in FP32
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}

// The block-real rows of a complex operand in K columns 4 c4 .. + 3 (left) and 16 + 4 c4 .. + 3
// (right): NEG_TOP: row r0 = [x | -y], row r1 = [y | x]; else row r0 = [x | y], row r1 =
// [-y | x].  Each value is split once; a negation flips the sign bits of both parts (exact).
template <bool NEG_TOP>
__device__ __forceinline__ void put4_tf32_twin(unsigned char* hi_tile, unsigned char* lo_tile,
                                               int r0, int r1, int c4, const float (&x)[4],
                                               const float (&y)[4]) {
  uint4 xh, xl, yh, yl;
  tf32_split(x[0], xh.x, xl.x); tf32_split(x[1], xh.y, xl.y);
  tf32_split(x[2], xh.z, xl.z); tf32_split(x[3], xh.w, xl.w);
  tf32_split(y[0], yh.x, yl.x); tf32_split(y[1], yh.y, yl.y);
  tf32_split(y[2], yh.z, yl.z); tf32_split(y[3], yh.w, yl.w);
  const uint32_t S = 0x80000000u;
  const uint4 nyh = make_uint4(yh.x ^ S, yh.y ^ S, yh.z ^ S, yh.w ^ S);
  const uint4 nyl = make_uint4(yl.x ^ S, yl.y ^ S, yl.z ^ S, yl.w ^ S);
  const uint32_t a0 = sw128_off32(r0, 4 * c4), a1 = sw128_off32(r0, 16 + 4 * c4);
  const uint32_t b0 = sw128_off32(r1, 4 * c4), b1 = sw128_off32(r1, 16 + 4 * c4);
  *reinterpret_cast<uint4*>(hi_tile + a0) = xh;
  *reinterpret_cast<uint4*>(lo_tile + a0) = xl;
  *reinterpret_cast<uint4*>(hi_tile + a1) = NEG_TOP ? nyh : yh;
  *reinterpret_cast<uint4*>(lo_tile + a1) = NEG_TOP ? nyl : yl;
  *reinterpret_cast<uint4*>(hi_tile + b0) = NEG_TOP ? yh : nyh;
  *reinterpret_cast<uint4*>(lo_tile + b0) = NEG_TOP ? yl : nyl;
  *reinterpret_cast<uint4*>(hi_tile + b1) = xh;
  *reinterpret_cast<uint4*>(lo_tile + b1) = xl;
}
// row r of a tile: [x | y] in K columns 4 c4 .. + 3 and 16 + 4 c4 .. + 3
__device__ __forceinline__ void put4_tf32_pair(unsigned char* hi_tile, unsigned char* lo_tile, int r,
                                               int c4, const float (&x)[4], const float (&y)[4]) {
  uint4 xh, xl, yh, yl;
  tf32_split(x[0], xh.x, xl.x); tf32_split(x[1], xh.y, xl.y);
  tf32_split(x[2], xh.z, xl.z); tf32_split(x[3], xh.w, xl.w);
  tf32_split(y[0], yh.x, yl.x); tf32_split(y[1], yh.y, yl.y);
  tf32_split(y[2], yh.z, yl.z); tf32_split(y[3], yh.w, yl.w);
  const uint32_t a0 = sw128_off32(r, 4 * c4), a1 = sw128_off32(r, 16 + 4 * c4);
  *reinterpret_cast<uint4*>(hi_tile + a0) = xh; *reinterpret_cast<uint4*>(lo_tile + a0) = xl;
  *reinterpret_cast<uint4*>(hi_tile + a1) = yh; *reinterpret_cast<uint4*>(lo_tile + a1) = yl;
}

__device__ __forceinline__ void umma_tf32(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                          uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}

// the 12 MMAs of one K phase: (hi, lo), (lo, hi), then (hi, hi), x 4 K8 steps.  The small
// cross terms go first: each MMA's addition into the FP32 accumulator truncates at the
// accumulator's magnitude, so they are added while it is still ~2^-11 of its final size and
// only the four (hi, hi) steps truncate at full size.
__device__ __forceinline__ void tf_issue(uint32_t tmem_d, uint32_t ops, bool first) {
  const uint32_t a_hi = ops, a_lo = ops + TF_A_TILE;
  const uint32_t b_hi = ops + 2 * TF_A_TILE, b_lo = b_hi + TF_B_TILE;
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const uint32_t a = p == 1 ? a_lo : a_hi, b = p == 0 ? b_lo : b_hi;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
      umma_tf32(tmem_d, tc::umma_desc_sw128(a + kk * 32), tc::umma_desc_sw128(b + kk * 32),
                TF_IDESC, (first && p == 0 && kk == 0) ? 0u : 1u);
  }
}

// U32 (nullable): U = Q D Z already formed in FP32 ([n][W][W], assemble_u_kernel), copied
// into shared memory instead of being assembled here
template <typename TIn>
__global__ void __launch_bounds__(TF_NT, 2) berry_tf32_kernel(
    const double* __restrict__ E, const double* __restrict__ Z, EighBufs eb,
    const TIn* __restrict__ Xp, const TIn* __restrict__ Yp, int64_t ld, int W, int n,
    const double* __restrict__ etas, int n_eta, double* __restrict__ Om, int64_t eta_stride,
    DevStatus* st, const float2* __restrict__ U32) {
  extern __shared__ unsigned char tf_smem[];
  __shared__ double sE[64];
  __shared__ double sEta[MAXE];
  __shared__ double s_emax;
  __shared__ __align__(8) uint64_t mma_bar;
  __shared__ uint32_t tmem_sh;
  __shared__ int s_ok;
  float2* sU = reinterpret_cast<float2*>(tf_smem);
  // the operand tiles start on a 1024-byte boundary (the 128-byte swizzle pattern repeats every
  // 8 rows of 128 bytes and is taken from the address bits)
  unsigned char* ops = reinterpret_cast<unsigned char*>(
      ((uintptr_t)(tf_smem + TF_U_BYTES) + 1023) & ~(uintptr_t)1023);
  unsigned char* a_hi = ops;
  unsigned char* a_lo = ops + TF_A_TILE;
  unsigned char* b_hi = ops + 2 * TF_A_TILE;
  unsigned char* b_lo = b_hi + TF_B_TILE;
  // FP32 velocity input: the packed row of the current direction, rows of LDX floats
  constexpr bool XS = std::is_same<TIn, float>::value;
  float* sX = reinterpret_cast<float*>(ops + TF_OPS_BYTES);
  const int LDX = W + 1;   // odd: row and column walks of a warp fall on distinct banks
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const size_t WW = (size_t)W * W;
  const FastDiv dWx(W > 0 ? W : 1);
  auto fetch_x = [&](const TIn* P) {
    if constexpr (XS) {
      for (int idx = t; idx < W * W; idx += TF_NT) {
        const int r = (int)dWx.div(idx);
        cp_async4(sX + r * LDX + (idx - r * W), P + idx);
      }
    }
  };

  if (t == 0) {
    tc::mbar_init(&mma_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc::smem_u32(&tmem_sh)), "r"(TF_TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_sh;
  const uint32_t ops_u32 = tc::smem_u32(ops);
  // TMEM lane quarter and column half of this warp when reading an accumulator
  const int quarter = warp & 3, chalf = warp >> 2;
  const int mrow = quarter * 32 + lane;   // row of [.._r; .._i]
  const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
  uint32_t phase = 0;
  bool ok = true;

  // the MMAs of the staged K phase into TMEM column d_col; bounded wait (false on timeout)
  auto mma_quarter = [&](uint32_t d_col, bool first) -> bool {
    tc::fence_proxy_async_smem();
    __syncthreads();
    if (t == 0) {
      tc::tc_fence_after();
      tf_issue(tmem + d_col, ops_u32, first);
      tc::umma_commit(&mma_bar);
      s_ok = tc::mbar_wait(&mma_bar, phase, TF_WAIT_LIMIT) ? 1 : 0;
    }
    __syncthreads();
    phase ^= 1u;
    tc::tc_fence_after();
    return s_ok != 0;
  };

  for (int64_t k = blockIdx.x; k < n && ok; k += gridDim.x) {
    __syncthreads();   // the previous k-point's shared data is no longer read
    if (t < W) sE[t] = E[k * W + t];
    if (t < n_eta) sEta[t] = etas[t];
    for (int idx = t; idx < TF_WP * TF_LDU; idx += TF_NT) sU[idx] = make_float2(0.f, 0.f);
    __syncthreads();
    fetch_x(Xp + k * ld);   // lands while U is assembled (or copied)
    if (U32) {
      // ---- U = Q D Z, formed in FP32 by the assembly kernel: asynchronous copy (the zero
      // padding of rows / columns >= W is written above, behind the barrier)
      const float2* src = U32 + k * WW;
      for (int idx = t; idx < W * W; idx += TF_NT) {
        const int r = (int)dWx.div(idx);
        cp_async8(sU + r * TF_LDU + (idx - r * W), src + idx);
      }
      cp_async_wait_all();
      __syncthreads();
    } else {
      // ---- U = Q D Z in FP32 (the reflectors staged in the operand region)
      assemble_u_f32(Z + k * WW, eb.phase + k * W, eb.refl + k * WW, eb.tau + k * W, W, TF_LDU,
                     t, sU, reinterpret_cast<float2*>(ops));
    }
    emax_warp0(sE, W, t, &s_emax);
    float vacc[32];   // this thread's 32 entries of row mrow of [V_r; V_i]
    for (int a = 0; a < 2 && ok; ++a) {
      const TIn* P = (a == 0 ? Xp : Yp) + k * ld;
      // ---- product 1: [T_r; T_i] = A1 B1^T.  Each K phase accumulates into TMEM columns
      // 0..63 from zero and is added here in FP32 with round-to-nearest: the tensor core's
      // FP32 accumulation truncates, and one accumulator per phase keeps that to 12 steps
      // (all 48 in one accumulator left the result ten times less accurate than the SIMT
      // rotation's).  tv: this thread's 32 entries of row mrow of [T_r; T_i].
      float tv[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) tv[j] = 0.f;
      if constexpr (XS) cp_async_wait_all();   // this direction's rows (the barrier follows)
      for (int h = 0; h < 4 && ok; ++h) {
        __syncthreads();   // the stage area / previous phase's operands are free
        // Phase h pairs the X columns c = 16 h .. 16 h + 15 of both K halves: tile K columns
        // 0..15 are K = c (real parts), 16..31 are K = 64 + c (imaginary parts), in A and B
        // alike (the product sums over K in any order).  A1 rows i: [X_r | -X_i], rows
        // 64 + i: [X_i | X_r], each X value loaded and split once (-X_i by the sign bits).
        {
          const int i = t & 63, c4 = t >> 6;   // 64 rows x 4 groups of 4 columns: one per thread
          float xr[4], xi[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int c = 16 * h + 4 * c4 + q;
            float re = 0.f, im = 0.f;
            if (i < W && c < W) {
              if constexpr (XS) {
                if (i < c) { re = sX[i * LDX + c]; im = sX[c * LDX + i]; }
                else if (i > c) { re = sX[c * LDX + i]; im = -sX[i * LDX + c]; }
                else re = sX[i * LDX + i];
              } else {
                if (i < c) { re = (float)P[i * W + c]; im = (float)P[c * W + i]; }
                else if (i > c) { re = (float)P[c * W + i]; im = -(float)P[i * W + c]; }
                else re = (float)P[i * W + i];
              }
            }
            xr[q] = re;
            xi[q] = im;
          }
          put4_tf32_twin<true>(a_hi, a_lo, i, 64 + i, c4, xr, xi);
        }
        // B1 rows n: [U_r[c][n] | U_i[c][n]]
        {
          const int nn = t & 63, c4 = t >> 6;
          float ur[4], ui[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float2 v = sU[(16 * h + 4 * c4 + q) * TF_LDU + nn];
            ur[q] = v.x;
            ui[q] = v.y;
          }
          put4_tf32_pair(b_hi, b_lo, nn, c4, ur, ui);
        }
        if (!mma_quarter(0, true)) { ok = false; break; }
        // the last read of this direction's rows is behind the barrier: fetch Y (lands while
        // the second product of X runs)
        if (h == 3 && a == 0) fetch_x(Yp + k * ld);
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          uint32_t r[16];
          tc::tmem_ld16(lane_addr + (uint32_t)(chalf * 32 + 16 * hh), r);
#pragma unroll
          for (int j = 0; j < 16; ++j)
            tv[16 * hh + j] += __uint_as_float(r[j]);
        }
        tc::tc_fence_before();
      }
      if (!ok) break;
      // ---- product 2: [V_r; V_i] = A2 B2^T, per K phase in TMEM columns 64..127, summed here
#pragma unroll
      for (int j = 0; j < 32; ++j) vacc[j] = 0.f;
      for (int h = 0; h < 4 && ok; ++h) {
        __syncthreads();
        // Phase h pairs the rows r = 16 h .. 16 h + 15 of T_r (tile K 0..15) and of T_i (16..31).
        // A2 rows m: [U_r[r][m] | U_i[r][m]], rows 64 + m: [-U_i[r][m] | U_r[r][m]]
        {
          const int m = t & 63, c4 = t >> 6;
          float ur[4], ui[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float2 v = sU[(16 * h + 4 * c4 + q) * TF_LDU + m];   // U[r][m]
            ur[q] = v.x;
            ui[q] = v.y;
          }
          put4_tf32_twin<false>(a_hi, a_lo, m, 64 + m, c4, ur, ui);
        }
        // B2[n][K]: T_r[r][n] (K = r - 16 h) and T_i[r][n] (K = 16 + r - 16 h); row r of T_r is
        // TMEM lane r, of T_i lane 64 + r: held in tv by the threads of lanes 16 h .. 16 h + 15
        // (quarter h / 2) and 64 + those (quarter 2 + h / 2), each for its 32 columns n
        {
          const int r0 = 16 * (h & 1);   // lane offset within the quarter
          const bool mine = (quarter == (h >> 1) || quarter == 2 + (h >> 1)) && lane >= r0 &&
                            lane < r0 + 16;
          if (mine) {
            const int kc = (quarter >= 2 ? 16 : 0) + (lane - r0);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              uint32_t hi, lo;
              tf32_split(tv[j], hi, lo);
              const uint32_t off = sw128_off32(chalf * 32 + j, kc);
              *reinterpret_cast<uint32_t*>(b_hi + off) = hi;
              *reinterpret_cast<uint32_t*>(b_lo + off) = lo;
            }
          }
        }
        if (!mma_quarter(64, true)) { ok = false; break; }
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          uint32_t r[16];
          tc::tmem_ld16(lane_addr + (uint32_t)(64 + chalf * 32 + 16 * hh), r);
#pragma unroll
          for (int j = 0; j < 16; ++j)
            vacc[16 * hh + j] += __uint_as_float(r[j]);
        }
        tc::tc_fence_before();
      }
      if (!ok) break;
      if (a == 0) {
        // park V^x in TMEM columns 128..191 while V^y is formed
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          uint32_t r[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) r[j] = __float_as_uint(vacc[16 * hh + j]);
          tc::tmem_st16(lane_addr + (uint32_t)(128 + chalf * 32 + 16 * hh), r);
        }
        tc::tc_fence_before();
      }
    }
    if (!ok) break;
    // ---- V^x (TMEM) and V^y (registers) into shared memory (float2 [64][TF_LDU]; U and the
    // operands are no longer needed)
    __syncthreads();
    float2* sVx = reinterpret_cast<float2*>(tf_smem);
    float2* sVy = sVx + TF_WP * TF_LDU;
    {
      const int rr = mrow & 63;
      const int comp = mrow >= 64 ? 1 : 0;
      float* dx = reinterpret_cast<float*>(sVx);
      float* dy = reinterpret_cast<float*>(sVy);
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        uint32_t r[16];
        tc::tmem_ld16(lane_addr + (uint32_t)(128 + chalf * 32 + 16 * hh), r);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int o = 2 * (rr * TF_LDU + chalf * 32 + 16 * hh + j) + comp;
          dx[o] = __uint_as_float(r[j]);
          dy[o] = vacc[16 * hh + j];
        }
      }
    }
    tc::tc_fence_before();
    __syncthreads();
    // ---- curvature (FP64 energy differences), as the SIMT kernels
    {
      const int tx = t & 15, ty = t >> 4;
      float2 vy[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) vy[i][j] = sVy[(ty + 16 * i) * TF_LDU + tx + 16 * j];
      curvature_epilogue<4, float2>(sVx, vy, sE, sEta, n_eta, s_emax, W, TF_LDU, ty, tx, t,
                                    reinterpret_cast<double*>(tf_smem), Om, eta_stride, k);
    }
  }
  if (!ok && t == 0) atomicOr(&st->bits, ST_TIMEOUT);
  // no MMA may still write TMEM when it is released
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    if (lane == 0 && !ok) tc::mbar_wait(&mma_bar, phase, TF_WAIT_LIMIT);
    __syncwarp();
    tc::tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TF_TMEM_COLS) : "memory");
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

// bytes of the U assembly's staging area (reflectors, then the block factors G and T)
static size_t asm_stage_bytes(int W) {
  const size_t nref = W > 2 ? (size_t)W - 2 : 0;
  const size_t nblk = (nref + ASM_NB - 1) / ASM_NB;
  return ((size_t)W * (W - 1) / 2 + 2 * nblk * ASM_NB * ASM_NB) * sizeof(float2);
}

size_t berry_mixed_smem(int W, int n_eta) {
  const size_t mat = (size_t)W * mixed_ld(W, 1) * sizeof(float2);
  const size_t red = (size_t)n_eta * W * 2 * 16 * sizeof(double);
  return mat + std::max(std::max(2 * mat, red), asm_stage_bytes(W));
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
                                      int64_t eta_stride, cudaStream_t s, int pad, bool vel32) {
  const int64_t WW = (int64_t)W * W;
  if (vel32) {
    const float* X = reinterpret_cast<const float*>(C) + vel32_x0(W);
    return launch_berry_mixed_t<float, true>(E, nullptr, Z, eb, X, X + vel32_yoff(W), 2 * ld, W,
                                             n, etas, n_eta, Om, eta_stride, s, pad);
  }
  return launch_berry_mixed_t<double, true>(E, nullptr, Z, eb, C + WW, C + 2 * WW, ld, W, n, etas,
                                            n_eta, Om, eta_stride, s, pad);
}

size_t berry_tc_smem() { return (size_t)RT_U_BYTES + 1024 + RT_A_BYTES + RT_B_BYTES; }

template <typename TIn>
static cudaError_t launch_berry_tc_t(const double* E, const double* Z, const EighBufs& eb,
                                     const TIn* Xp, const TIn* Yp, int64_t ld, int W, int n,
                                     const double* etas, int n_eta, double* Om, int64_t eta_stride,
                                     DevStatus* st, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (W > RT_WP || n_eta > MAXE) return cudaErrorInvalidValue;
  const size_t sm = berry_tc_smem();
  cudaError_t e = cudaFuncSetAttribute(berry_tc_kernel<TIn>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  const int grid = std::min(n, std::max(1, sms));
  berry_tc_kernel<TIn><<<grid, RT_NT, sm, s>>>(E, Z, eb, Xp, Yp, ld, W, n, etas, n_eta, Om,
                                               eta_stride, st);
  return cudaGetLastError();
}

cudaError_t launch_berry_tc_rows(const double* E, const double* Z, const EighBufs& eb,
                                 const double* C, int64_t ld, int W, int n, const double* etas,
                                 int n_eta, double* Om, int64_t eta_stride, DevStatus* st,
                                 cudaStream_t s, bool vel32) {
  const int64_t WW = (int64_t)W * W;
  if (vel32) {
    const float* X = reinterpret_cast<const float*>(C) + vel32_x0(W);
    return launch_berry_tc_t<float>(E, Z, eb, X, X + vel32_yoff(W), 2 * ld, W, n, etas, n_eta,
                                    Om, eta_stride, st, s);
  }
  return launch_berry_tc_t<double>(E, Z, eb, C + WW, C + 2 * WW, ld, W, n, etas, n_eta, Om,
                                   eta_stride, st, s);
}

cudaError_t launch_berry_tc_from_f64(const double* E, const double* Z, const EighBufs& eb,
                                     const double* Xp, const double* Yp, int W, int n,
                                     const double* etas, int n_eta, double* Om,
                                     int64_t eta_stride, DevStatus* st, cudaStream_t s) {
  return launch_berry_tc_t<double>(E, Z, eb, Xp, Yp, (int64_t)W * W, W, n, etas, n_eta, Om,
                                   eta_stride, st, s);
}

size_t assemble_u_smem(int W) {
  return (size_t)W * mixed_ld(W, 1) * sizeof(float2) + asm_stage_bytes(W);
}

cudaError_t launch_assemble_u32(const double* Z, const EighBufs& eb, float2* U32, int W, int n,
                                cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (W > 64 || W < 1) return cudaErrorInvalidValue;
  const size_t sm = assemble_u_smem(W);
  cudaError_t e = cudaFuncSetAttribute(assemble_u_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  assemble_u_kernel<<<n, NT, sm, s>>>(Z, eb, U32, W, mixed_ld(W, 1));
  return cudaGetLastError();
}

// dynamic shared memory of the 3xTF32 rotation kernel: U and the operand stage, or the
// curvature's per-eta partial sums if larger (n_eta x 16 KB)
size_t berry_tf32_smem(int n_eta, bool xs) {
  const size_t base = (size_t)TF_U_BYTES + 1024 + TF_OPS_BYTES + (xs ? TF_X_BYTES : 0);
  const size_t red = (size_t)n_eta * TF_WP * 2 * 16 * sizeof(double);
  return std::max(base, red);
}

template <typename TIn>
static cudaError_t launch_berry_tf32_t(const double* E, const double* Z, const EighBufs& eb,
                                       const TIn* Xp, const TIn* Yp, int64_t ld, int W, int n,
                                       const double* etas, int n_eta, double* Om,
                                       int64_t eta_stride, DevStatus* st, cudaStream_t s,
                                       const float2* U32 = nullptr) {
  if (n <= 0) return cudaSuccess;
  if (W > TF_WP || n_eta > MAXE) return cudaErrorInvalidValue;
  const size_t sm = berry_tf32_smem(n_eta, std::is_same<TIn, float>::value);
  cudaError_t e = cudaFuncSetAttribute(berry_tf32_kernel<TIn>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  // the whole unified L1 / shared-memory array as shared memory, so that two CTAs fit
  cudaFuncSetAttribute(berry_tf32_kernel<TIn>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  // two CTAs per SM (128 registers x 256 threads each, 2 x 256 of the 512 TMEM columns) while
  // the shared memory allows (up to six broadenings); the CTAs are independent, so a grid
  // larger than what is resident only queues
  const int per_sm = sm <= (size_t)110 * 1024 ? 2 : 1;
  const int grid = (int)std::min<int64_t>(n, (int64_t)std::max(1, sms) * per_sm);
  berry_tf32_kernel<TIn><<<grid, TF_NT, sm, s>>>(E, Z, eb, Xp, Yp, ld, W, n, etas, n_eta, Om,
                                                 eta_stride, st, U32);
  return cudaGetLastError();
}

cudaError_t launch_berry_tf32_rows(const double* E, const double* Z, const EighBufs& eb,
                                   const double* C, int64_t ld, int W, int n, const double* etas,
                                   int n_eta, double* Om, int64_t eta_stride, DevStatus* st,
                                   cudaStream_t s, bool vel32, const float2* U32) {
  const int64_t WW = (int64_t)W * W;
  if (vel32) {
    const float* X = reinterpret_cast<const float*>(C) + vel32_x0(W);
    return launch_berry_tf32_t<float>(E, Z, eb, X, X + vel32_yoff(W), 2 * ld, W, n, etas, n_eta,
                                      Om, eta_stride, st, s, U32);
  }
  return launch_berry_tf32_t<double>(E, Z, eb, C + WW, C + 2 * WW, ld, W, n, etas, n_eta, Om,
                                     eta_stride, st, s);
}

cudaError_t launch_berry_tf32_from_f64(const double* E, const double* Z, const EighBufs& eb,
                                       const double* Xp, const double* Yp, int W, int n,
                                       const double* etas, int n_eta, double* Om,
                                       int64_t eta_stride, DevStatus* st, cudaStream_t s) {
  return launch_berry_tf32_t<double>(E, Z, eb, Xp, Yp, (int64_t)W * W, W, n, etas, n_eta, Om,
                                     eta_stride, st, s);
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
