// Reverse mode of steps (1)-(4) (Eq. 2-3): the gradient of L = sum_{e,j} g[e][j] S_e(E_F_j)
// with respect to every entry of H(R), FP64 throughout.
//
// Per k-point, from the forward quantities E, U, v^x = U^dagger dxH U, v^y = U^dagger dyH U:
//   a[e][n]  = sum_j g[e][j] occ_j(E_n) / N_k,   a'[e][n] = sum_j g[e][j] occ_j'(E_n) / N_k
//   num_nm   = -2 Im(v^x_nm v^y_mn),  D^e_nm = (E_n - E_m)^2 + eta_e^2
//   B_nm     = sum_e (a[e][n] - a[e][m]) / D^e_nm                       (antisymmetric)
//   vbar^x   = -i B o v^y,  vbar^y = i B o v^x                          (Hermitian)
//   Ebar_n   = sum_e a'[e][n] Omega^e_n - 2 sum_m (E_n - E_m) num_nm sum_e (a[e][n] - a[e][m]) / (D^e_nm)^2
//   N        = vbar^x v^x + vbar^y v^y
//   Gp       = diag(Ebar) + F o (N^dagger - N),  F_ij = (E_j - E_i) / ((E_j - E_i)^2 + eps^2)
//   Hbar     = U Gp U^dagger,  dxHbar = U vbar^x U^dagger,  dyHbar = U vbar^y U^dagger
// (first-order perturbation theory of the Hermitian eigenproblem for the Gp step), and then
// the transposed Fourier sum
//   G(R) = sum_k e^{-ik.R} [Hbar - i R_x dxHbar - i R_y dyHbar],
// evaluated as one real GEMM over the canonical half set of R: rows (1, cos k.R_h, sin k.R_h)
// against the packed Hermitian columns [Hbar | dxHbar | dyHbar], accumulated over batches in
// a fixed order (deterministic), and unfolded into G(R_h), G(-R_h) = G(R_h)^dagger, G(0).
#include <algorithm>

#include "kubo_internal.cuh"

namespace kubo {

namespace {

constexpr int GT = 64, GK = 16;   // GEMM tiles: up to 64 x 64 outputs, K steps of 16
constexpr int MAXE = 8;
constexpr int PW = 128;            // threads of the per-k kernels (W <= 128)

// ------------------------------------------------------------------ batched complex GEMM
// C[k] = op(A[k]) op(B[k]) (+ C[k]), W x W complex FP64, op = identity or conjugate transpose.
// Output tile T = 16 TM (TM x TM per thread); TM = 2 for W <= 32 so no thread multiplies padding.
template <bool HA, bool HB, bool ACC, int TM>
__global__ void __launch_bounds__(256) zgemm_kernel(const double2* __restrict__ A,
                                                    const double2* __restrict__ B,
                                                    double2* __restrict__ C, int W) {
  constexpr int T = 16 * TM;
  __shared__ double2 As[T][GK + 1];
  __shared__ double2 Bs[GK][T + 1];
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int nt = (W + T - 1) / T;
  const int r0 = (blockIdx.y / nt) * T, c0 = (blockIdx.y % nt) * T;
  const size_t base = (size_t)blockIdx.x * W * W;
  const double2* Ak = A + base;
  const double2* Bk = B + base;
  double ax[TM][TM], ay[TM][TM];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TM; ++j) { ax[i][j] = 0.0; ay[i][j] = 0.0; }
  for (int q0 = 0; q0 < W; q0 += GK) {
    for (int idx = t; idx < T * GK; idx += 256) {
      int r, q;
      if (HA) { q = idx / T; r = idx % T; } else { r = idx / GK; q = idx % GK; }
      const int gr = r0 + r, gq = q0 + q;
      double2 a = make_double2(0.0, 0.0);
      if (gr < W && gq < W) {
        if (HA) { a = Ak[(size_t)gq * W + gr]; a.y = -a.y; }
        else a = Ak[(size_t)gr * W + gq];
      }
      As[r][q] = a;
    }
    for (int idx = t; idx < GK * T; idx += 256) {
      int q, c;
      if (HB) { c = idx / GK; q = idx % GK; } else { q = idx / T; c = idx % T; }
      const int gq = q0 + q, gc = c0 + c;
      double2 b = make_double2(0.0, 0.0);
      if (gq < W && gc < W) {
        if (HB) { b = Bk[(size_t)gc * W + gq]; b.y = -b.y; }
        else b = Bk[(size_t)gq * W + gc];
      }
      Bs[q][c] = b;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < GK; ++q) {
      double2 a[TM], b[TM];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[ty + 16 * i][q];
#pragma unroll
      for (int j = 0; j < TM; ++j) b[j] = Bs[q][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM; ++j) {
          ax[i][j] = fma(a[i].x, b[j].x, ax[i][j]);
          ax[i][j] = fma(-a[i].y, b[j].y, ax[i][j]);
          ay[i][j] = fma(a[i].x, b[j].y, ay[i][j]);
          ay[i][j] = fma(a[i].y, b[j].x, ay[i][j]);
        }
    }
    __syncthreads();
  }
  double2* Ck = C + base;
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TM; ++j) {
      const int r = r0 + ty + 16 * i, c = c0 + tx + 16 * j;
      if (r < W && c < W) {
        double2 v = make_double2(ax[i][j], ay[i][j]);
        if (ACC) { const double2 o = Ck[(size_t)r * W + c]; v.x += o.x; v.y += o.y; }
        Ck[(size_t)r * W + c] = v;
      }
    }
}

// ------------------------------------------------------------------ occupations
__device__ __forceinline__ void occ_and_derivative(double E, double EF, double kT, double& f,
                                                   double& fp) {
  if (kT == 0.0) {
    f = E < EF ? 1.0 : 0.0;
    fp = 0.0;
    return;
  }
  const double x = (E - EF) / kT;
  const double ex = exp(-fabs(x));
  f = x > 0.0 ? ex / (1.0 + ex) : 1.0 / (1.0 + ex);
  fp = -f * (1.0 - f) / kT;
}

// ------------------------------------------------------------------ per-k pair terms
// One CTA per k-point, thread per row p: vbar^x, vbar^y (full W x W) and Ebar.
__global__ void __launch_bounds__(PW) grad_pairs_kernel(
    const double* __restrict__ E, const double2* __restrict__ vx, const double2* __restrict__ vy,
    int W, const double* __restrict__ g, const double* __restrict__ E_F, int n_EF,
    const double* __restrict__ etas, int n_eta, double kT, double inv_Nk,
    double2* __restrict__ vbx, double2* __restrict__ vby, double* __restrict__ Ebar) {
  __shared__ double sE[PW];
  __shared__ double sa[MAXE][PW], sap[MAXE][PW];
  __shared__ double s_emax;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t k = blockIdx.x;
  if (t < W) {
    const double En = E[k * W + t];
    sE[t] = En;
    for (int e = 0; e < n_eta; ++e) {
      double a = 0.0, ap = 0.0;
      for (int j = 0; j < n_EF; ++j) {
        double f, fp;
        occ_and_derivative(En, E_F[j], kT, f, fp);
        const double w = g[e * n_EF + j];
        a = fma(w, f, a);
        ap = fma(w, fp, ap);
      }
      sa[e][t] = a * inv_Nk;
      sap[e][t] = ap * inv_Nk;
    }
  }
  __syncthreads();
  if (warp == 0) {
    double mx = 0.0;
    for (int i = lane; i < W; i += 32) mx = fmax(mx, fabs(sE[i]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) s_emax = mx;
  }
  __syncthreads();
  const int p = t;
  if (p >= W) return;
  const double thr2 = (1e-12 * s_emax) * (1e-12 * s_emax);
  const size_t row = (size_t)k * W * W + (size_t)p * W;
  const double Ep = sE[p];
  double om[MAXE];
#pragma unroll
  for (int e = 0; e < MAXE; ++e) om[e] = 0.0;
  double eb = 0.0;
  for (int m = 0; m < W; ++m) {
    const double2 x = vx[row + m], y = vy[row + m];
    double B = 0.0;
    if (m != p) {
      const double num = -2.0 * (x.y * y.x - x.x * y.y);   // -2 Im(v^x_pm conj(v^y_pm))
      const double dE = Ep - sE[m];
      const double d2 = dE * dE;
      double s2 = 0.0;
#pragma unroll
      for (int e = 0; e < MAXE; ++e) {
        if (e >= n_eta) break;
        const double eta = etas[e];
        if (eta == 0.0 && d2 <= thr2) continue;
        const double D = fma(eta, eta, d2);
        const double iD = 1.0 / D;
        const double da = sa[e][p] - sa[e][m];
        B = fma(da, iD, B);
        s2 = fma(da, iD * iD, s2);
        om[e] = fma(num, iD, om[e]);
      }
      eb = fma(-2.0 * dE * num, s2, eb);
    }
    vbx[row + m] = make_double2(B * y.y, -B * y.x);    // -i B v^y
    vby[row + m] = make_double2(-B * x.y, B * x.x);    //  i B v^x
  }
#pragma unroll
  for (int e = 0; e < MAXE; ++e) {
    if (e >= n_eta) break;
    eb = fma(sap[e][p], om[e], eb);
  }
  Ebar[k * W + p] = eb;
}

// Gp = diag(Ebar) + F o (N^dagger - N), one CTA per k-point
__global__ void __launch_bounds__(256) grad_gp_kernel(const double* __restrict__ E,
                                                      const double* __restrict__ Ebar,
                                                      const double2* __restrict__ N, int W,
                                                      double grad_eps, double2* __restrict__ Gp) {
  __shared__ double sE[PW];
  __shared__ double s_eps2;
  const int t = threadIdx.x;
  const int64_t k = blockIdx.x;
  if (t < W) sE[t] = E[k * W + t];
  __syncthreads();
  if (t == 0) {
    double eps = grad_eps;
    if (!(eps > 0.0)) {
      double mx = 0.0;
      for (int i = 0; i < W; ++i) mx = fmax(mx, fabs(sE[i]));
      eps = 1e-12 * mx;
    }
    s_eps2 = eps * eps;
  }
  __syncthreads();
  const double eps2 = s_eps2;
  const size_t base = (size_t)k * W * W;
  for (int idx = t; idx < W * W; idx += 256) {
    const int i = idx / W, j = idx % W;
    double2 v;
    if (i == j) {
      v = make_double2(Ebar[k * W + i], 0.0);
    } else {
      const double dji = sE[j] - sE[i];
      const double den = fma(dji, dji, eps2);
      const double F = den > 0.0 ? dji / den : 0.0;
      const double2 a = N[base + (size_t)j * W + i], b = N[base + idx];
      v = make_double2(F * (a.x - b.x), F * (-a.y - b.y));   // F (conj(N_ji) - N_ij)
    }
    Gp[base + idx] = v;
  }
}

// Hermitian parts of three full complex matrices -> packed rows [k][3 W^2]
__global__ void pack3_kernel(const double2* __restrict__ A0, const double2* __restrict__ A1,
                             const double2* __restrict__ A2, int W, int n,
                             double* __restrict__ out) {
  const int64_t WW = (int64_t)W * W;
  const int64_t total = (int64_t)n * WW;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = t / WW;
    const int q = (int)(t % WW), i = q / W, j = q % W;
    const int lo = min(i, j), hi = max(i, j);
    const size_t u = (size_t)k * WW + (size_t)lo * W + hi;   // upper element (lo, hi)
    const size_t l = (size_t)k * WW + (size_t)hi * W + lo;   // its mirror
    const double2* src[3] = {A0, A1, A2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double2 x = src[a][u], y = src[a][l];
      // Hermitian part h_lo,hi = (x + conj(y)) / 2: Re above (and on) the diagonal, Im below
      const double v = i <= j ? 0.5 * (x.x + y.x) : 0.5 * (x.y - y.y);
      out[k * 3 * WW + a * WW + q] = v;
    }
  }
}

// Coef[row][kk] for row 0 (R = 0: 1), 1 + h (cos k.R_h), 1 + N_h + h (sin k.R_h)
__global__ void grad_coef_kernel(Model md, Mesh mesh, KList kl, int ldc, double* __restrict__ Coef) {
  const int64_t total = (int64_t)(md.N_h + 1) * kl.n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int h = (int)(t / kl.n) - 1;
    const int kk = (int)(t % kl.n);
    if (h < 0) {
      Coef[kk] = 1.0;
      continue;
    }
    int j1, j2, j3;
    mesh_coords(mesh, klist_get(kl, kk), j1, j2, j3);
    const int* r = md.Rh + 3 * h;
    const double2 e = mesh_phase(md.tab, md.tab_off, mesh, j1, j2, j3, r[0], r[1], r[2]);
    Coef[(size_t)(1 + h) * ldc + kk] = e.x;
    Coef[(size_t)(1 + md.N_h + h) * ldc + kk] = e.y;
  }
}

// Gacc[M][N] += Coef[M][K] Mbar[K][N], real FP64, 64 x 64 tiles; K in order (deterministic)
__global__ void __launch_bounds__(256) grad_fourier_t_kernel(const double* __restrict__ Coef,
                                                             int ldc, const double* __restrict__ Mb,
                                                             int M, int N, int K,
                                                             double* __restrict__ Gacc) {
  __shared__ double As[GT][GK + 1];
  __shared__ double Bs[GK][GT + 1];
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int r0 = blockIdx.y * GT, c0 = blockIdx.x * GT;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int q0 = 0; q0 < K; q0 += GK) {
    for (int idx = t; idx < GT * GK; idx += 256) {
      const int r = idx / GK, q = idx % GK;
      const int gr = r0 + r, gq = q0 + q;
      As[r][q] = (gr < M && gq < K) ? Coef[(size_t)gr * ldc + gq] : 0.0;
    }
    for (int idx = t; idx < GK * GT; idx += 256) {
      const int q = idx / GT, c = idx % GT;
      const int gq = q0 + q, gc = c0 + c;
      Bs[q][c] = (gq < K && gc < N) ? Mb[(size_t)gq * N + gc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < GK; ++q) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[ty + 16 * i][q];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[q][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = r0 + ty + 16 * i, c = c0 + tx + 16 * j;
      if (r < M && c < N) Gacc[(size_t)r * N + c] += acc[i][j];
    }
}

// unpack element (i, j) of the Hermitian matrix whose packed form is P (W x W reals)
__device__ __forceinline__ double2 herm_at(const double* P, int W, int i, int j) {
  if (i < j) return make_double2(P[i * W + j], P[j * W + i]);
  if (i > j) return make_double2(P[j * W + i], -P[i * W + j]);
  return make_double2(P[i * W + i], 0.0);
}

// G(R) from the accumulated rows: thread per (h or R = 0, i, j)
__global__ void grad_finalize_kernel(const double* __restrict__ Gacc, const int* __restrict__ pairs,
                                     const int* __restrict__ Rh, int idx0, int N_h, int W,
                                     double2* __restrict__ G) {
  const int64_t WW = (int64_t)W * W;
  const int64_t N = 3 * WW;
  const int64_t total = (int64_t)(N_h + 1) * WW;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int h = (int)(t / WW) - 1;
    const int q = (int)(t % WW), i = q / W, j = q % W;
    if (h < 0) {
      G[(size_t)idx0 * WW + q] = herm_at(Gacc, W, i, j);
      continue;
    }
    const double* C = Gacc + (size_t)(1 + h) * N;          // cos row: [CH | CX | CY]
    const double* S = Gacc + (size_t)(1 + N_h + h) * N;    // sin row: [SH | SX | SY]
    const double rx = (double)Rh[3 * h], ry = (double)Rh[3 * h + 1];
    const double2 ch = herm_at(C, W, i, j), cx = herm_at(C + WW, W, i, j), cy = herm_at(C + 2 * WW, W, i, j);
    const double2 sh = herm_at(S, W, i, j), sx = herm_at(S + WW, W, i, j), sy = herm_at(S + 2 * WW, W, i, j);
    // P1 = CH - R_x SX - R_y SY, P2 = SH + R_x CX + R_y CY, G(R_h) = P1 - i P2
    const double2 p1 = make_double2(ch.x - rx * sx.x - ry * sy.x, ch.y - rx * sx.y - ry * sy.y);
    const double2 p2 = make_double2(sh.x + rx * cx.x + ry * cy.x, sh.y + rx * cx.y + ry * cy.y);
    const double2 gv = make_double2(p1.x + p2.y, p1.y - p2.x);
    G[(size_t)pairs[2 * h] * WW + q] = gv;
    G[(size_t)pairs[2 * h + 1] * WW + (size_t)j * W + i] = make_double2(gv.x, -gv.y);   // G(-R) = G(R)^dagger
  }
}

}  // namespace

cudaError_t launch_zgemm_batched(bool hA, bool hB, bool acc, const double2* A, const double2* B,
                                 double2* C, int W, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int T = W <= 32 ? 32 : GT;
  const int tiles = (W + T - 1) / T;
  dim3 grid(n, tiles * tiles);
#define ZG(a, b, c)                                                          \
  do {                                                                       \
    if (T == 32) zgemm_kernel<a, b, c, 2><<<grid, 256, 0, s>>>(A, B, C, W);  \
    else zgemm_kernel<a, b, c, 4><<<grid, 256, 0, s>>>(A, B, C, W);          \
  } while (0)
  if (!hA && !hB && !acc) ZG(false, false, false);
  else if (!hA && !hB && acc) ZG(false, false, true);
  else if (hA && !hB && !acc) ZG(true, false, false);
  else if (!hA && hB && !acc) ZG(false, true, false);
  else return cudaErrorInvalidValue;
#undef ZG
  return cudaGetLastError();
}

cudaError_t launch_grad_pairs(const double* E, const double2* vx, const double2* vy, int W, int n,
                              const double* g, const double* E_F, int n_EF, const double* etas,
                              int n_eta, double kT, double inv_Nk, double2* vbx, double2* vby,
                              double* Ebar, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (W > PW || n_eta > MAXE) return cudaErrorInvalidValue;
  grad_pairs_kernel<<<n, PW, 0, s>>>(E, vx, vy, W, g, E_F, n_EF, etas, n_eta, kT, inv_Nk, vbx,
                                     vby, Ebar);
  return cudaGetLastError();
}

cudaError_t launch_grad_gp(const double* E, const double* Ebar, const double2* N, int W, int n,
                           double grad_eps, double2* Gp, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (W > PW) return cudaErrorInvalidValue;
  grad_gp_kernel<<<n, 256, 0, s>>>(E, Ebar, N, W, grad_eps, Gp);
  return cudaGetLastError();
}

cudaError_t launch_pack3(const double2* A0, const double2* A1, const double2* A2, int W, int n,
                         double* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t total = (int64_t)n * W * W;
  const int b = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  pack3_kernel<<<b, 256, 0, s>>>(A0, A1, A2, W, n, out);
  return cudaGetLastError();
}

cudaError_t launch_grad_coef(const Model& md, const Mesh& mesh, const KList& kl, int ldc,
                             double* Coef, cudaStream_t s) {
  if (kl.n <= 0) return cudaSuccess;
  const int64_t total = (int64_t)(md.N_h + 1) * kl.n;
  const int b = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  grad_coef_kernel<<<b, 256, 0, s>>>(md, mesh, kl, ldc, Coef);
  return cudaGetLastError();
}

cudaError_t launch_grad_fourier_t(const double* Coef, int ldc, const double* Mbar, int M, int N,
                                  int K, double* Gacc, cudaStream_t s) {
  if (K <= 0) return cudaSuccess;
  dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT);
  grad_fourier_t_kernel<<<grid, 256, 0, s>>>(Coef, ldc, Mbar, M, N, K, Gacc);
  return cudaGetLastError();
}

cudaError_t launch_grad_finalize(const double* Gacc, const int* pairs, const int* Rh, int idx0,
                                 int N_h, int W, double2* G, cudaStream_t s) {
  const int64_t total = (int64_t)(N_h + 1) * W * W;
  const int b = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  grad_finalize_kernel<<<b, 256, 0, s>>>(Gacc, pairs, Rh, idx0, N_h, W, G);
  return cudaGetLastError();
}

}  // namespace kubo
