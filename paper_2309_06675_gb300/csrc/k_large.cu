// Steps (2)-(4) for orders 64 < W <= 128, where a whole k-point no longer fits one CTA's
// shared memory.  Same arithmetic as the fused kernels, split into batched passes:
//   iit_kernel            eigenvalue sort + eigenvectors of the tridiagonal T by inverse
//                         iteration, one thread per cluster, persistent CTAs; LU factors in
//                         per-CTA global scratch laid out [i][thread] (coalesced), iterates in
//                         their column of Z (also used for W <= 64 when U is formed in FP32)
//   reflect_large_kernel  U = Q D Z for one 32-column block of one k-point per CTA
//   cgemm_herm_u_kernel   T = dH U   (dH from packed Hermitian rows)          } FP64 or FP32
//   cgemm_uh_t_kernel     V = U^H T                                            } arithmetic
//   curvature_large_kernel Omega_n = sum_{m != n} T_nm, every pair evaluated from the upper
//                         triangle (exact antisymmetry), FP64 energy differences for every
//                         eta (FP32 quotients for FP32 velocities)
#include <algorithm>
#include <type_traits>

#include "kubo_internal.cuh"

namespace kubo {

namespace {

constexpr int LW_MAX = LARGE_W_MAX;
// Solves per eigenvector: QL leaves every shift within ~eps ||T|| of its eigenvalue, so after
// two solves the other eigenvectors' share is ~(eps ||T|| / gap)^2 (clusters closer than
// 1e-3 ||T|| are orthogonalised explicitly); a third changes nothing at FP64 precision.
constexpr int IIT_SOLVES = 2;
constexpr int MAXE = 8;
constexpr int IIT_SMS = 152;   // GB300 SM count: persistent inverse-iteration grid

__device__ __forceinline__ unsigned long long order_key(double x) {
  unsigned long long u = (unsigned long long)__double_as_longlong(x);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// ------------------------------------------------------------------ inverse iteration
// Persistent: CTA b handles k = b, b + gridDim.x, ...; block = ldt = W rounded up to a warp;
// thread j handles the cluster starting at sorted index j.  Z: [n][W][W] real, column m =
// eigenvector of sorted eigenvalue m.  scratch: per CTA [4][W][ldt] (reciprocal pivots, U1,
// U2, multipliers), lane-interleaved so every access of a warp is one coalesced row segment.
// rq: the eigenvalues written are the FP64 Rayleigh quotients z^T T z of the finished unit
// eigenvectors (kept non-decreasing within a cluster) instead of the shifts b.lam -- for
// shifts from a reduced-precision QL, whose only role is then to make the iteration converge.
// (launch bounds: LW_MAX threads and 8 CTAs of them per SM = 64 registers a thread, the budget
// of the 16 (W <= 64) or 8 (W = 128) resident CTAs of iit_max_slots; without the CTA count,
// ptxas settled on 56 registers and spilled)
__global__ void __launch_bounds__(LW_MAX, 8) iit_kernel(int W, int n, EighBufs b,
                                                     double* __restrict__ Eout,
                                                     double* __restrict__ Z,
                                                     double* __restrict__ scratch, int rq) {
  __shared__ double ws[LW_MAX], dd[LW_MAX], ee[LW_MAX];
  __shared__ int newc[LW_MAX];
  __shared__ double s_onenrm;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int ldt = blockDim.x;
  const size_t plane = (size_t)W * ldt;
  double* rU0 = scratch + (size_t)blockIdx.x * 4 * plane;
  double* U1 = rU0 + plane;
  double* U2 = U1 + plane;
  double* ML = U2 + plane;
  const double eps = 2.220446049250313e-16;
  for (int64_t k = blockIdx.x; k < n; k += gridDim.x) {
    __syncthreads();   // the previous k-point's shared arrays are no longer read
    const double* lk = b.lam + k * W;
    if (t < W) {
      const double lj = lk[t];
      const unsigned long long kj = order_key(lj);
      int rnk = 0;
      for (int i = 0; i < W; ++i) {
        const unsigned long long ki = order_key(lk[i]);
        rnk += (ki < kj) || (ki == kj && i < t);
      }
      ws[rnk] = lj;
      Eout[k * W + rnk] = lj;
      dd[t] = b.d[k * W + t];
      ee[t] = b.e[k * W + t];
    }
    __syncthreads();
    if (warp == 0) {
      double mx = 0.0;
      for (int i = lane; i < W; i += 32)
        mx = fmax(mx, fabs(dd[i]) + (i > 0 ? ee[i - 1] : 0.0) + (i < W - 1 ? ee[i] : 0.0));
      for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0) s_onenrm = mx > 0.0 ? mx : 1.0;
    }
    __syncthreads();
    const double onenrm = s_onenrm;
    const double ortol = 1e-3 * onenrm, pertol = 10.0 * eps * onenrm, tiny = eps * onenrm;
    if (t < W) newc[t] = (t == 0) || (ws[t] - ws[t - 1] > ortol);
    __syncthreads();
    if (Z == nullptr) continue;

    double* Zk = Z + (size_t)k * W * W;
    const int j = t;
    if (j < W && newc[j]) {
      double lprev = 0.0, rprev = 0.0;
      for (int m = j; m < W && (m == j || !newc[m]); ++m) {
        double lam = ws[m];
        if (m > j && lam - lprev <= pertol) lam = lprev + pertol;
        lprev = lam;
        unsigned long long piv0 = 0ull, piv1 = 0ull;   // row interchanges, bits 0..127
        double q0 = dd[0] - lam, q1 = W > 1 ? ee[0] : 0.0, q2 = 0.0;
        // Gaussian elimination with partial pivoting of T - lam I (q2 is zero at every step).
        // The row interchange only selects operands (integer selects), so the lanes of a warp,
        // whose interchanges differ, issue one common sequence of FP64 instructions.
        for (int i = 0; i + 1 < W; ++i) {
          const double ei = ee[i];
          const double a = dd[i + 1] - lam;
          const double bb = i + 2 < W ? ee[i + 1] : 0.0;
          const size_t o = (size_t)i * ldt + t;
          const bool sw = mag_bits(q0) < mag_bits(ei);   // interchange rows i and i + 1
          const double den = sw ? ei : (mag_bits(q0) == 0ull ? tiny : q0);
          const double r = recip_nr(den);
          const double mlt = (sw ? q0 : ei) * r;
          rU0[o] = r; U1[o] = sw ? a : q1; U2[o] = sw ? bb : q2; ML[o] = mlt;
          if (sw) { if (i < 64) piv0 |= 1ull << i; else piv1 |= 1ull << (i - 64); }
          const double n0 = fma(-mlt, sw ? a : q1, sw ? q1 : a);
          q1 = fma(-mlt, sw ? bb : q2, sw ? q2 : bb);
          q0 = n0;
          q2 = 0.0;
        }
        if (mag_bits(q0) == 0ull) q0 = tiny;
        {
          const size_t o = (size_t)(W - 1) * ldt + t;
          rU0[o] = 1.0 / q0; U1[o] = 0.0; U2[o] = 0.0;
        }
        for (int i = 0; i < W; ++i) Zk[(size_t)i * W + m] = iit_start_vec(i, m);
        for (int it = 0; it < IIT_SOLVES; ++it) {
          for (int i = 0; i + 1 < W; ++i) {
            const double mlt = ML[(size_t)i * ldt + t];
            const double yi = Zk[(size_t)i * W + m], yn = Zk[(size_t)(i + 1) * W + m];
            const bool sw = i < 64 ? ((piv0 >> i) & 1ull) : ((piv1 >> (i - 64)) & 1ull);
            if (sw) Zk[(size_t)i * W + m] = yn;
            Zk[(size_t)(i + 1) * W + m] = fma(-mlt, sw ? yn : yi, sw ? yi : yn);
          }
          double x1 = 0.0, x2 = 0.0;
          for (int i = W - 1; i >= 0; --i) {
            const size_t o = (size_t)i * ldt + t;
            const double xi = (Zk[(size_t)i * W + m] - U1[o] * x1 - U2[o] * x2) * rU0[o];
            Zk[(size_t)i * W + m] = xi;
            x2 = x1;
            x1 = xi;
          }
          for (int q = j; q < m; ++q) {
            double c = 0.0;
            for (int i = 0; i < W; ++i) c = fma(Zk[(size_t)i * W + q], Zk[(size_t)i * W + m], c);
            for (int i = 0; i < W; ++i)
              Zk[(size_t)i * W + m] = fma(-c, Zk[(size_t)i * W + q], Zk[(size_t)i * W + m]);
          }
          if (it + 1 < IIT_SOLVES) {   // between solves: a power-of-two rescale (exact)
            pow2_rescale(Zk + m, W, (size_t)W);
            continue;
          }
          double s0 = 0.0, s1 = 0.0;
          int i = 0;
          for (; i + 1 < W; i += 2) {
            const double u = Zk[(size_t)i * W + m], v = Zk[(size_t)(i + 1) * W + m];
            s0 = fma(u, u, s0);
            s1 = fma(v, v, s1);
          }
          if (i < W) { const double u = Zk[(size_t)i * W + m]; s0 = fma(u, u, s0); }
          const double inv = 1.0 / sqrt(s0 + s1);
          for (int i2 = 0; i2 < W; ++i2) Zk[(size_t)i2 * W + m] *= inv;
        }
        if (rq) {
          // z^T T z = sum_i d_i z_i^2 + 2 sum_i e_i z_i z_{i+1} (z of unit norm)
          double q = 0.0, qe = 0.0, zi = Zk[m];
          for (int i = 0; i < W; ++i) {
            const double zn = i + 1 < W ? Zk[(size_t)(i + 1) * W + m] : 0.0;
            q = fma(dd[i] * zi, zi, q);
            if (i + 1 < W) qe = fma(ee[i] * zi, zn, qe);
            zi = zn;
          }
          q = fma(2.0, qe, q);
          if (m > j && q < rprev) q = rprev;   // ascending order within the cluster
          rprev = q;
          Eout[k * W + m] = q;
        }
      }
    }
  }
}

// ------------------------------------------------------------------ U = Q D Z, column blocks
// One CTA per (32-column block, k-point): the block of D Z in shared memory, the reflectors
// applied from the last to the first (U <- H_j U), eight reflectors at a time staged in shared
// memory from coalesced row segments of the reflector matrix.
template <typename T> struct cx;
template <> struct cx<double> { typedef double2 type; __device__ static double2 make(double a, double b) { return make_double2(a, b); } };
template <> struct cx<float> { typedef float2 type; __device__ static float2 make(double a, double b) { return make_float2((float)a, (float)b); } };

constexpr int RB_COLS = 32;
constexpr int RB_NT = 256;   // 8 threads per column
constexpr int RB_J = 8;      // reflectors per staged block

// T = float: U is formed in FP32 from the FP64 factors, for the FP32 rotations (its only
// consumer in that mode); T = double: the FP64 eigenvectors.
template <typename T>
__global__ void __launch_bounds__(RB_NT) reflect_large_kernel(int W, EighBufs b,
                                                              const double* __restrict__ Z,
                                                              typename cx<T>::type* __restrict__ Uout) {
  typedef typename cx<T>::type C2;
  extern __shared__ __align__(16) unsigned char rb_smem[];
  C2* ub = reinterpret_cast<C2*>(rb_smem);   // [W][RB_COLS + 1]
  __shared__ C2 vs[RB_J][LW_MAX + 1];
  const int LDB = RB_COLS + 1;
  const int t = threadIdx.x;
  const int c0 = blockIdx.y * RB_COLS;
  const int64_t k = blockIdx.x;
  const int ncol = min(RB_COLS, W - c0);
  const double* Zk = Z + (size_t)k * W * W;
  const double2* ph = b.phase + k * W;
  for (int idx = t; idx < W * RB_COLS; idx += RB_NT) {
    const int r = idx / RB_COLS, c = idx % RB_COLS;
    C2 u = cx<T>::make(0.0, 0.0);
    if (c < ncol) {
      const double z = Zk[(size_t)r * W + c0 + c];
      const double2 p = ph[r];
      u = cx<T>::make(p.x * z, p.y * z);
    }
    ub[r * LDB + c] = u;
  }
  const double2* R = b.refl + (size_t)k * W * W;
  const double* tau = b.tau + k * W;
  const int c = t >> 3, q = t & 7;
  const bool act = c < ncol;
  for (int jhi = W - 3; jhi >= 0; jhi -= RB_J) {
    const int jlo = max(0, jhi - RB_J + 1);
    __syncthreads();   // the previous block of reflectors is no longer read
    for (int idx = t; idx < W * RB_J; idx += RB_NT) {
      const int r = idx / RB_J, jj = idx % RB_J, j = jlo + jj;
      if (j <= jhi) {
        const double2 v = r > j ? R[(size_t)r * W + j] : make_double2(0.0, 0.0);
        vs[jj][r] = cx<T>::make(v.x, v.y);
      }
    }
    __syncthreads();
    for (int j = jhi; j >= jlo; --j) {
      const T tj = (T)tau[j];
      if (tj == (T)0) continue;
      const int o = j + 1, m = W - 1 - j;
      const C2* v = vs[j - jlo] + o;
      T sx = 0, sy = 0;
      if (act) {
        for (int r = q; r < m; r += 8) {
          const C2 vv = v[r];
          const C2 u = ub[(o + r) * LDB + c];
          sx = fma(vv.x, u.x, fma(vv.y, u.y, sx));   // conj(v) u
          sy = fma(vv.x, u.y, fma(-vv.y, u.x, sy));
        }
      }
#pragma unroll
      for (int s = 1; s < 8; s <<= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, s);
        sy += __shfl_xor_sync(0xffffffffu, sy, s);
      }
      sx *= tj; sy *= tj;
      if (act) {
        for (int r = q; r < m; r += 8) {
          const C2 vv = v[r];
          C2 u = ub[(o + r) * LDB + c];
          u.x = fma(-sx, vv.x, fma(sy, vv.y, u.x));   // u -= s v
          u.y = fma(-sx, vv.y, fma(-sy, vv.x, u.y));
          ub[(o + r) * LDB + c] = u;
        }
      }
      __syncwarp();
    }
  }
  __syncthreads();
  C2* Uk = Uout + (size_t)k * W * W;
  for (int idx = t; idx < W * RB_COLS; idx += RB_NT) {
    const int r = idx / RB_COLS, cc = idx % RB_COLS;
    if (cc < ncol) Uk[(size_t)r * W + c0 + cc] = ub[r * LDB + cc];
  }
}

// ------------------------------------------------------------------ U = Q D Z in FP32, blocked
// For the FP32 rotations: Q = H_0 ... H_{W-3} applied in blocks of WY_NB = 8 reflectors in the
// compact WY form I - V T V^H (T upper triangular: T_ii = tau_i,
// T[0:i, i] = -tau_i T[0:i, 0:i] G[0:i, i], G = V^H V), last block first.
//   wy_factors_kernel: one CTA per k-point; V of every block in FP32, row-major [W][WY_LDV]
//     (8 reflectors per row, zeros above each reflector's first row, rows padded to 80 bytes),
//     and T, into a per-k scratch.
//   reflect_wy_kernel: one CTA per (k-point, 32-column block); D Z of the block in shared
//     memory; thread (column c, row lane q) owns rows q, q + 8, ...; per block s = V^H u
//     (partial sums over the lane's rows from the block's first row down, three shuffles),
//     y_q = (T s)_q, an exchange, u -= V y.  Blocks are double-buffered by cp.async.
constexpr int WY_NB = 8;
constexpr int WY_LDV = 10;   // float2 per staged row (8 + 2 pad: 80 bytes)

__host__ __device__ __forceinline__ int wy_nblk(int W) { return W > 2 ? (W - 2 + WY_NB - 1) / WY_NB : 0; }
__host__ __device__ __forceinline__ size_t wy_v_elems(int W) { return (size_t)wy_nblk(W) * W * WY_LDV; }
__host__ __device__ __forceinline__ size_t wy_bytes_per_k(int W) {
  return (wy_v_elems(W) + (size_t)wy_nblk(W) * WY_NB * WY_NB) * sizeof(float2);
}

__device__ __forceinline__ float2 wy_cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__global__ void __launch_bounds__(256) wy_factors_kernel(int W, EighBufs b,
                                                         float2* __restrict__ wy) {
  __shared__ float2 sV[LW_MAX * WY_LDV];
  __shared__ float2 sG[WY_NB * WY_NB];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t k = blockIdx.x;
  const int nref = W - 2, nblk = wy_nblk(W);
  const double2* R = b.refl + (size_t)k * W * W;
  const double* tau = b.tau + k * W;
  float2* Vk = wy + (size_t)k * (wy_bytes_per_k(W) / sizeof(float2));
  float2* Tk = Vk + wy_v_elems(W);
  for (int bk = 0; bk < nblk; ++bk) {
    const int j0 = bk * WY_NB;
    __syncthreads();   // the previous block's stage is no longer read
    for (int idx = t; idx < W * WY_NB; idx += 256) {
      const int r = idx >> 3, a = idx & 7, c = j0 + a;
      float2 v = make_float2(0.f, 0.f);
      if (c < nref && r > c) {
        const double2 d = R[(size_t)r * W + c];
        v = make_float2((float)d.x, (float)d.y);
      }
      sV[r * WY_LDV + a] = v;
      Vk[((size_t)bk * W + r) * WY_LDV + a] = v;
    }
    __syncthreads();
    // G[a][a2] (a < a2): 32 lane groups of 8, group g sums pair g over rows q, q + 8, ...
    {
      const int g = warp * 4 + (lane >> 3), q = lane & 7;
      int a = 0, rem = g < WY_NB * (WY_NB - 1) / 2 ? g : 0;
      while (rem >= WY_NB - 1 - a) {
        rem -= WY_NB - 1 - a;
        ++a;
      }
      const int a2 = a + 1 + rem;
      float2 acc = make_float2(0.f, 0.f);
      for (int r = j0 + a2 + 1 + q; r < W; r += 8) {
        const float2 x = sV[r * WY_LDV + a], y = sV[r * WY_LDV + a2];
        acc.x = fmaf(x.x, y.x, fmaf(x.y, y.y, acc.x));   // conj(x) y
        acc.y = fmaf(x.x, y.y, fmaf(-x.y, y.x, acc.y));
      }
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o, 8);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o, 8);
      }
      if (q == 0 && g < WY_NB * (WY_NB - 1) / 2) sG[a * WY_NB + a2] = acc;
    }
    __syncthreads();
    // T: lane a of warp 0 keeps row a
    if (warp == 0) {
      float2 trow[WY_NB];
#pragma unroll
      for (int i = 0; i < WY_NB; ++i) {
        const float ti = j0 + i < nref ? (float)tau[j0 + i] : 0.f;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int k2 = 0; k2 < i; ++k2) {
          if (k2 >= lane) {
            const float2 pr = wy_cmul(trow[k2], sG[k2 * WY_NB + i]);
            acc.x += pr.x;
            acc.y += pr.y;
          }
        }
        trow[i] = lane < i ? make_float2(-ti * acc.x, -ti * acc.y)
                           : (lane == i ? make_float2(ti, 0.f) : make_float2(0.f, 0.f));
      }
      if (lane < WY_NB)
#pragma unroll
        for (int i = 0; i < WY_NB; ++i) Tk[((size_t)bk * WY_NB + lane) * WY_NB + i] = trow[i];
    }
  }
}

__device__ __forceinline__ void wy_cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}

__global__ void __launch_bounds__(RB_NT) reflect_wy_kernel(int W, EighBufs b,
                                                           const double* __restrict__ Z,
                                                           const float2* __restrict__ wy,
                                                           float2* __restrict__ Uout) {
  extern __shared__ __align__(16) unsigned char wy_smem[];
  const int LDB = RB_COLS + 1;
  float2* ub = reinterpret_cast<float2*>(wy_smem);                        // [W][LDB]
  float2* vbuf = ub + (((size_t)W * LDB + 1) & ~(size_t)1);             // 2 x [W][WY_LDV]
  float2* tbuf = vbuf + 2 * (size_t)W * WY_LDV;                           // 2 x [NB][NB]
  const int t = threadIdx.x;
  const int c0 = blockIdx.y * RB_COLS;
  const int64_t k = blockIdx.x;
  const int ncol = min(RB_COLS, W - c0);
  const int nblk = wy_nblk(W);
  const float2* Vk = wy + (size_t)k * (wy_bytes_per_k(W) / sizeof(float2));
  const float2* Tk = Vk + wy_v_elems(W);
  const size_t vblk = (size_t)W * WY_LDV;   // float2 per staged V block (a multiple of 2)
  auto fetch = [&](int bk, int buf) {
    const float4* src = reinterpret_cast<const float4*>(Vk + (size_t)bk * vblk);
    float4* dst = reinterpret_cast<float4*>(vbuf + (size_t)buf * vblk);
    for (int i = t; i < (int)(vblk / 2); i += RB_NT) wy_cp16(dst + i, src + i);
    const float4* ts = reinterpret_cast<const float4*>(Tk + (size_t)bk * WY_NB * WY_NB);
    float4* td = reinterpret_cast<float4*>(tbuf + (size_t)buf * WY_NB * WY_NB);
    if (t < WY_NB * WY_NB / 2) wy_cp16(td + t, ts + t);
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if (nblk > 0) fetch(nblk - 1, (nblk - 1) & 1);
  const double* Zk = Z + (size_t)k * W * W;
  const double2* ph = b.phase + k * W;
  for (int idx = t; idx < W * RB_COLS; idx += RB_NT) {
    const int r = idx / RB_COLS, c = idx % RB_COLS;
    float2 u = make_float2(0.f, 0.f);
    if (c < ncol) {
      const float z = (float)Zk[(size_t)r * W + c0 + c];
      const double2 p = ph[r];
      u = make_float2((float)p.x * z, (float)p.y * z);
    }
    ub[r * LDB + c] = u;
  }
  const int c = t >> 3, q = t & 7;
  for (int bk = nblk - 1; bk >= 0; --bk) {
    const int buf = bk & 1;
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();   // block bk landed; the other buffer (block bk + 1) is no longer read
    if (bk > 0) fetch(bk - 1, buf ^ 1);
    const float4* V4 = reinterpret_cast<const float4*>(vbuf + (size_t)buf * vblk);
    const float2* T = tbuf + (size_t)buf * WY_NB * WY_NB;
    const int r0 = bk * WY_NB + 1;   // first row a reflector of the block touches
    const int rs = q >= r0 ? q : q + ((r0 - q + 7) >> 3) * 8;   // first own row >= r0
    float2 sv[WY_NB];
#pragma unroll
    for (int a = 0; a < WY_NB; ++a) sv[a] = make_float2(0.f, 0.f);
    for (int r = rs; r < W; r += 8) {
      const float2 u = ub[r * LDB + c];
#pragma unroll
      for (int a2 = 0; a2 < WY_NB / 2; ++a2) {
        const float4 v = V4[r * (WY_LDV / 2) + a2];
        sv[2 * a2].x = fmaf(v.x, u.x, fmaf(v.y, u.y, sv[2 * a2].x));   // conj(v) u
        sv[2 * a2].y = fmaf(v.x, u.y, fmaf(-v.y, u.x, sv[2 * a2].y));
        sv[2 * a2 + 1].x = fmaf(v.z, u.x, fmaf(v.w, u.y, sv[2 * a2 + 1].x));
        sv[2 * a2 + 1].y = fmaf(v.z, u.y, fmaf(-v.w, u.x, sv[2 * a2 + 1].y));
      }
    }
#pragma unroll
    for (int a = 0; a < WY_NB; ++a)
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        sv[a].x += __shfl_xor_sync(0xffffffffu, sv[a].x, o);
        sv[a].y += __shfl_xor_sync(0xffffffffu, sv[a].y, o);
      }
    // lane q forms y_q = sum_{a2 >= q} T[q][a2] s[a2]; then every lane gathers all eight
    float2 yq = make_float2(0.f, 0.f);
#pragma unroll
    for (int a2 = 0; a2 < WY_NB; ++a2) {
      if (a2 >= q) {
        const float2 pr = wy_cmul(T[q * WY_NB + a2], sv[a2]);
        yq.x += pr.x;
        yq.y += pr.y;
      }
    }
    float2 y[WY_NB];
#pragma unroll
    for (int a = 0; a < WY_NB; ++a) {
      y[a].x = __shfl_sync(0xffffffffu, yq.x, a, 8);
      y[a].y = __shfl_sync(0xffffffffu, yq.y, a, 8);
    }
    for (int r = rs; r < W; r += 8) {
      float2 u = ub[r * LDB + c];
#pragma unroll
      for (int a2 = 0; a2 < WY_NB / 2; ++a2) {
        const float4 v = V4[r * (WY_LDV / 2) + a2];
        u.x = fmaf(-v.x, y[2 * a2].x, fmaf(v.y, y[2 * a2].y, u.x));   // u -= v y
        u.y = fmaf(-v.x, y[2 * a2].y, fmaf(-v.y, y[2 * a2].x, u.y));
        u.x = fmaf(-v.z, y[2 * a2 + 1].x, fmaf(v.w, y[2 * a2 + 1].y, u.x));
        u.y = fmaf(-v.z, y[2 * a2 + 1].y, fmaf(-v.w, y[2 * a2 + 1].x, u.y));
      }
      ub[r * LDB + c] = u;
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  float2* Uk = Uout + (size_t)k * W * W;
  for (int idx = t; idx < W * RB_COLS; idx += RB_NT) {
    const int r = idx / RB_COLS, cc = idx % RB_COLS;
    if (cc < ncol) Uk[(size_t)r * W + c0 + cc] = ub[r * LDB + cc];
  }
}

// ------------------------------------------------------------------ batched complex GEMMs
// 64 x 64 output tile per CTA, 16 x 16 threads with 4 x 4 strided micro-tiles, K tiles of 16.

constexpr int GT = 64, GK = 16;

// C[k] = H[k] U[k]; H from packed Hermitian rows P (leading dimension ldp), U complex in the
// compute type.
template <typename T>
__global__ void __launch_bounds__(256) cgemm_herm_u_kernel(const double* __restrict__ P, int64_t ldp,
                                                           const typename cx<T>::type* __restrict__ U,
                                                           int W,
                                                           typename cx<T>::type* __restrict__ C) {
  typedef typename cx<T>::type C2;
  __shared__ C2 As[GT][GK + 1];
  __shared__ C2 Bs[GK][GT + 1];
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int nt = (W + GT - 1) / GT;
  const int r0 = (blockIdx.y / nt) * GT, c0 = (blockIdx.y % nt) * GT;
  const int64_t k = blockIdx.x;
  const double* Pk = P + k * ldp;
  const C2* Uk = U + (size_t)k * W * W;
  T ax[4][4], ay[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { ax[i][j] = 0; ay[i][j] = 0; }
  for (int q0 = 0; q0 < W; q0 += GK) {
    for (int idx = t; idx < GT * GK; idx += 256) {
      const int r = idx / GK, q = idx % GK;
      const int gr = r0 + r, gq = q0 + q;
      C2 a = cx<T>::make(0.0, 0.0);
      if (gr < W && gq < W) {
        if (gr < gq) a = cx<T>::make(Pk[gr * W + gq], Pk[gq * W + gr]);
        else if (gr > gq) a = cx<T>::make(Pk[gq * W + gr], -Pk[gr * W + gq]);
        else a = cx<T>::make(Pk[gr * W + gr], 0.0);
      }
      As[r][q] = a;
    }
    for (int idx = t; idx < GK * GT; idx += 256) {
      const int q = idx / GT, c = idx % GT;
      const int gq = q0 + q, gc = c0 + c;
      C2 v = cx<T>::make(0.0, 0.0);
      if (gq < W && gc < W) v = Uk[(size_t)gq * W + gc];
      Bs[q][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < GK; ++q) {
      C2 a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[ty + 16 * i][q];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[q][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          ax[i][j] = fma(a[i].x, bb[j].x, ax[i][j]);
          ax[i][j] = fma(-a[i].y, bb[j].y, ax[i][j]);
          ay[i][j] = fma(a[i].x, bb[j].y, ay[i][j]);
          ay[i][j] = fma(a[i].y, bb[j].x, ay[i][j]);
        }
    }
    __syncthreads();
  }
  typename cx<T>::type* Ck = C + (size_t)k * W * W;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = r0 + ty + 16 * i, c = c0 + tx + 16 * j;
      if (r < W && c < W) { C2 v; v.x = ax[i][j]; v.y = ay[i][j]; Ck[(size_t)r * W + c] = v; }
    }
}

// V[k] = U[k]^H Tm[k]
template <typename T>
__global__ void __launch_bounds__(256) cgemm_uh_t_kernel(const typename cx<T>::type* __restrict__ U,
                                                         const typename cx<T>::type* __restrict__ Tm,
                                                         int W, typename cx<T>::type* __restrict__ V) {
  typedef typename cx<T>::type C2;
  __shared__ C2 As[GT][GK + 1];
  __shared__ C2 Bs[GK][GT + 1];
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int nt = (W + GT - 1) / GT;
  const int r0 = (blockIdx.y / nt) * GT, c0 = (blockIdx.y % nt) * GT;
  const int64_t k = blockIdx.x;
  const C2* Uk = U + (size_t)k * W * W;
  const C2* Tk = Tm + (size_t)k * W * W;
  if (r0 >= c0 + GT) return;   // strictly below the diagonal: V is Hermitian, never read
  T ax[4][4], ay[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { ax[i][j] = 0; ay[i][j] = 0; }
  for (int q0 = 0; q0 < W; q0 += GK) {
    for (int idx = t; idx < GT * GK; idx += 256) {
      const int q = idx / GT, r = idx % GT;   // coalesced along r (a row of U)
      const int gr = r0 + r, gq = q0 + q;
      C2 a = cx<T>::make(0.0, 0.0);
      if (gr < W && gq < W) { a = Uk[(size_t)gq * W + gr]; a.y = -a.y; }
      As[r][q] = a;
    }
    for (int idx = t; idx < GK * GT; idx += 256) {
      const int q = idx / GT, c = idx % GT;
      const int gq = q0 + q, gc = c0 + c;
      Bs[q][c] = (gq < W && gc < W) ? Tk[(size_t)gq * W + gc] : cx<T>::make(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < GK; ++q) {
      C2 a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[ty + 16 * i][q];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[q][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          ax[i][j] = fma(a[i].x, bb[j].x, ax[i][j]);
          ax[i][j] = fma(-a[i].y, bb[j].y, ax[i][j]);
          ay[i][j] = fma(a[i].x, bb[j].y, ay[i][j]);
          ay[i][j] = fma(a[i].y, bb[j].x, ay[i][j]);
        }
    }
    __syncthreads();
  }
  C2* Vk = V + (size_t)k * W * W;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = r0 + ty + 16 * i, c = c0 + tx + 16 * j;
      if (r < W && c < W) { C2 v; v.x = ax[i][j]; v.y = ay[i][j]; Vk[(size_t)r * W + c] = v; }
    }
}

// a b - c d within 2 ulp (Kahan: the rounding error of c d is recovered exactly by an FMA)
__device__ __forceinline__ float large_diff_of_products(float a, float b, float c, float d) {
  const float w = __fmul_rn(c, d);
  const float e = fmaf(-c, d, w);
  const float f = fmaf(a, b, -w);
  return __fadd_rn(f, e);
}
// (hi, lo) += x with the rounding error of hi + x carried exactly into lo (Knuth's TwoSum)
__device__ __forceinline__ void large_two_sum_acc(float& hi, float& lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bp = __fsub_rn(s, hi);
  const float ap = __fsub_rn(s, bp);
  const float err = __fadd_rn(__fsub_rn(hi, ap), __fsub_rn(x, bp));
  hi = s;
  lo = __fadd_rn(lo, err);
}

// ------------------------------------------------------------------ curvature, thread per band
template <typename T>
__global__ void __launch_bounds__(LW_MAX) curvature_large_kernel(const double* __restrict__ E,
                                                                 const typename cx<T>::type* __restrict__ Vx,
                                                                 const typename cx<T>::type* __restrict__ Vy,
                                                                 int W, const double* __restrict__ etas,
                                                                 int n_eta, double* __restrict__ Om,
                                                                 int64_t eta_stride) {
  __shared__ double sE[LW_MAX];
  __shared__ double s_emax;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t k = blockIdx.x;
  if (t < W) sE[t] = E[k * W + t];
  __syncthreads();
  if (warp == 0) {
    double mx = 0.0;
    for (int i = lane; i < W; i += 32) mx = fmax(mx, fabs(sE[i]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) s_emax = mx;
  }
  __syncthreads();
  const int n = t;
  if (n >= W) return;
  const double thr2 = (1e-12 * s_emax) * (1e-12 * s_emax);
  const size_t base = (size_t)k * W * W;
  if constexpr (std::is_same<T, float>::value) {
    // FP32 velocities: the numerator is FP32-grade already, so the quotient is formed in FP32
    // as in the W <= 64 kernels -- dE = E_p - E_q, its square and the eta = 0 cut-off in FP64,
    // Kahan's difference of products for Im(v^x v^y), the sums as exact FP32 pairs (Knuth's
    // TwoSum), and the FP64 quotient for a denominator below 2^-86 (eta and a gap below
    // ~1e-13).  Both orders of a pair read the same (p < q) entry with the same arithmetic, so
    // T_mn = -T_nm holds exactly.
    float hi[MAXE], lo[MAXE];
    float eta2[MAXE];
#pragma unroll
    for (int e = 0; e < MAXE; ++e) {
      hi[e] = 0.f;
      lo[e] = 0.f;
      eta2[e] = e < n_eta ? (float)(etas[e] * etas[e]) : 0.f;
    }
    double fb[MAXE];   // FP64 fallback terms
#pragma unroll
    for (int e = 0; e < MAXE; ++e) fb[e] = 0.0;
    for (int m = 0; m < W; ++m) {
      if (m == n) continue;
      const int p = n < m ? n : m, q = n < m ? m : n;
      const float2 vx = Vx[base + (size_t)p * W + q];
      const float2 vy = Vy[base + (size_t)p * W + q];
      const float num = -2.0f * large_diff_of_products(vx.y, vy.x, vx.x, vy.y);
      const double dE = sE[p] - sE[q];
      const double d2 = dE * dE;
      const float d2f = (float)d2;
      const bool small0 = d2 <= thr2;
      const float sgn = n < m ? 1.f : -1.f;
#pragma unroll
      for (int e = 0; e < MAXE; ++e) {
        if (e >= n_eta) break;
        if (eta2[e] == 0.f && small0) continue;
        const float den = d2f + eta2[e];
        if (den < 0x1p-86f) {
          fb[e] += (double)sgn * ((double)num / fma(etas[e], etas[e], d2));
        } else {
          large_two_sum_acc(hi[e], lo[e], sgn * (num / den));
        }
      }
    }
#pragma unroll
    for (int e = 0; e < MAXE; ++e) {
      if (e >= n_eta) break;
      Om[e * eta_stride + k * W + n] = ((double)hi[e] + (double)lo[e]) + fb[e];
    }
  } else {
    double rp[MAXE];
#pragma unroll
    for (int e = 0; e < MAXE; ++e) rp[e] = 0.0;
    for (int m = 0; m < W; ++m) {
      if (m == n) continue;
      const int p = n < m ? n : m, q = n < m ? m : n;
      const typename cx<T>::type vx = Vx[base + (size_t)p * W + q];
      const typename cx<T>::type vy = Vy[base + (size_t)p * W + q];
      const double num = -2.0 * ((double)vx.y * (double)vy.x - (double)vx.x * (double)vy.y);
      const double dE = sE[p] - sE[q];
      const double d2 = dE * dE;
      const double sgn = n < m ? 1.0 : -1.0;   // T_nm = -T_mn: evaluated from the (p < q) entry
#pragma unroll
      for (int e = 0; e < MAXE; ++e) {
        if (e >= n_eta) break;
        const double eta = etas[e];
        if (eta == 0.0 && d2 <= thr2) continue;
        rp[e] += sgn * (num / fma(eta, eta, d2));
      }
    }
#pragma unroll
    for (int e = 0; e < MAXE; ++e) {
      if (e >= n_eta) break;
      Om[e * eta_stride + k * W + n] = rp[e];
    }
  }
}

}  // namespace

// threads per inverse-iteration CTA and number of persistent CTAs (scratch slots): one warp
// per 32 orders; CTAs per SM so that about 1024 threads of each SM run inverse iteration
static int iit_threads(int W) { return (W + 31) / 32 * 32; }

int iit_max_slots(int W) { return IIT_SMS * std::min(32, 1024 / iit_threads(W)); }

size_t iit_scratch_doubles(int W, int slots) { return (size_t)slots * 4 * W * iit_threads(W); }

cudaError_t launch_iit(int W, int n, EighBufs b, double* E, double* Z, double* scratch, int slots,
                       cudaStream_t s, bool rq) {
  if (n <= 0) return cudaSuccess;
  if (W > LW_MAX || slots < 1) return cudaErrorInvalidValue;
  const int grid = std::min(n, slots);
  iit_kernel<<<grid, iit_threads(W), 0, s>>>(W, n, b, E, Z, scratch, (rq && Z) ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_reflect_large(int W, int n, EighBufs b, const double* Z, void* U, bool f32,
                                 cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  dim3 grid(n, (W + RB_COLS - 1) / RB_COLS);
  if (f32) {
    const size_t sm = (size_t)W * (RB_COLS + 1) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(reflect_large_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    reflect_large_kernel<float><<<grid, RB_NT, sm, s>>>(W, b, Z, (float2*)U);
  } else {
    const size_t sm = (size_t)W * (RB_COLS + 1) * sizeof(double2);
    cudaError_t e = cudaFuncSetAttribute(reflect_large_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    reflect_large_kernel<double><<<grid, RB_NT, sm, s>>>(W, b, Z, (double2*)U);
  }
  return cudaGetLastError();
}

size_t reflect_wy_scratch_bytes(int W) { return wy_bytes_per_k(W); }

cudaError_t launch_reflect_wy(int W, int n, EighBufs b, const double* Z, float2* U, float2* wy,
                              cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (W > LW_MAX || W < 3 || ((uintptr_t)wy & 15)) return cudaErrorInvalidValue;
  wy_factors_kernel<<<n, 256, 0, s>>>(W, b, wy);
  const size_t sm = ((((size_t)W * (RB_COLS + 1) + 1) & ~(size_t)1) + 2 * (size_t)W * WY_LDV +
                     2 * WY_NB * WY_NB) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(reflect_wy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  dim3 grid(n, (W + RB_COLS - 1) / RB_COLS);
  reflect_wy_kernel<<<grid, RB_NT, sm, s>>>(W, b, Z, wy, U);
  return cudaGetLastError();
}

// T[k] = X[k] U[k], X packed Hermitian rows of leading dimension ld, FP64 (any W <= 128)
cudaError_t launch_herm_u(const double* X, int64_t ld, const double2* U, double2* T, int W, int n,
                          cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (W > LW_MAX) return cudaErrorInvalidValue;
  const int tiles = (W + GT - 1) / GT;
  dim3 grid(n, tiles * tiles);
  cgemm_herm_u_kernel<double><<<grid, 256, 0, s>>>(X, ld, U, W, T);
  return cudaGetLastError();
}

// steps (3)-(4) for large W: X, Y packed Hermitian rows (leading dimension ld); U is float2
// when f32 (formed in FP32 by launch_reflect_large), double2 otherwise.
// f32 selects FP32 arithmetic for the products (mixed precision).  Tbuf, Vx, Vy: scratch of
// n * W * W complex elements of the arithmetic type each.
cudaError_t launch_berry_large(const double* E, const void* Uv, const double* X, const double* Y,
                               int64_t ld, int W, int n, const double* etas, int n_eta, double* Om,
                               int64_t eta_stride, bool f32, void* Tbuf, void* Vx, void* Vy,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (W > LW_MAX || n_eta > MAXE) return cudaErrorInvalidValue;
  const int tiles = (W + GT - 1) / GT;
  dim3 grid(n, tiles * tiles);
  if (f32) {
    const float2* U = (const float2*)Uv;
    cgemm_herm_u_kernel<float><<<grid, 256, 0, s>>>(X, ld, U, W, (float2*)Tbuf);
    cgemm_uh_t_kernel<float><<<grid, 256, 0, s>>>(U, (const float2*)Tbuf, W, (float2*)Vx);
    cgemm_herm_u_kernel<float><<<grid, 256, 0, s>>>(Y, ld, U, W, (float2*)Tbuf);
    cgemm_uh_t_kernel<float><<<grid, 256, 0, s>>>(U, (const float2*)Tbuf, W, (float2*)Vy);
    curvature_large_kernel<float><<<n, LW_MAX, 0, s>>>(E, (const float2*)Vx, (const float2*)Vy, W,
                                                        etas, n_eta, Om, eta_stride);
  } else {
    const double2* U = (const double2*)Uv;
    cgemm_herm_u_kernel<double><<<grid, 256, 0, s>>>(X, ld, U, W, (double2*)Tbuf);
    cgemm_uh_t_kernel<double><<<grid, 256, 0, s>>>(U, (const double2*)Tbuf, W, (double2*)Vx);
    cgemm_herm_u_kernel<double><<<grid, 256, 0, s>>>(Y, ld, U, W, (double2*)Tbuf);
    cgemm_uh_t_kernel<double><<<grid, 256, 0, s>>>(U, (const double2*)Tbuf, W, (double2*)Vy);
    curvature_large_kernel<double><<<n, LW_MAX, 0, s>>>(E, (const double2*)Vx, (const double2*)Vy,
                                                         W, etas, n_eta, Om, eta_stride);
  }
  return cudaGetLastError();
}

}  // namespace kubo
