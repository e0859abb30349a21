// Step (1) of the paper's List 1/2 ("define_matrices"): H(k), d_x H(k), d_y H(k) for a
// batch of mesh points, FP64.
//
// The Fourier sum is written as a real contraction over the canonical half set of R
// (Hermitian pairing H(-R) = H(R)^dagger):
//   H(k)     = P0 + sum_h [ c_h A_h + s_h B_h ]
//   d_a H(k) = sum_h R_h,a [ c_h B_h - s_h A_h ]          (c_h, s_h) = (cos, sin)(k.R_h)
// where A_h, B_h are packed Hermitian rows of the basis (see kubo_internal.cuh).  Phases are
// generated on the fly from per-axis twiddle tables with exact integer argument reduction,
// so no phase matrix ever touches HBM.
//
// FP64 on GB300 issues one warp instruction per 16 SM cycles; this kernel is a register-
// tiled SIMT contraction (6 DFMA per (k, column, h)), bound by that pipe.
#include "kubo_internal.cuh"

namespace kubo {

namespace {

constexpr int TK = 16;    // k-points per CTA
constexpr int TN = 128;   // packed columns per CTA
constexpr int HB = 16;    // half-set vectors per phase block (TK * HB == threads)
constexpr int NT = 256;

__global__ void __launch_bounds__(NT) fourier_fp64_kernel(Model md, Mesh mesh, KList kl,
                                                          double* __restrict__ Hp,
                                                          double* __restrict__ Xp,
                                                          double* __restrict__ Yp) {
  __shared__ double2 ph[HB][TK];
  __shared__ double rxs[HB], rys[HB];
  __shared__ int jk[TK][3];

  const int WW = md.W * md.W;
  const int t = threadIdx.x;
  const int k0 = blockIdx.y * TK;
  const int n0 = blockIdx.x * TN;
  const int cg = t & 31, kg = t >> 5;   // 4 columns, 2 k-points per thread

  if (t < TK) {
    int kk = min(k0 + t, kl.n - 1);
    int j1, j2, j3;
    mesh_coords(mesh, klist_get(kl, kk), j1, j2, j3);
    jk[t][0] = j1; jk[t][1] = j2; jk[t][2] = j3;
  }

  double aH[2][4], aX[2][4], aY[2][4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    int col = n0 + cg + 32 * c;
    double p0 = col < WW ? md.Bp[col] : 0.0;
#pragma unroll
    for (int q = 0; q < 2; ++q) { aH[q][c] = p0; aX[q][c] = 0.0; aY[q][c] = 0.0; }
  }
  __syncthreads();

  for (int hb = 0; hb < md.N_h; hb += HB) {
    {
      int kk = t % TK, hh = t / TK;
      int h = hb + hh;
      double2 e = make_double2(0.0, 0.0);
      if (h < md.N_h) {
        const int* r = md.Rh + 3 * h;
        e = mesh_phase(md.tab, md.tab_off, mesh, jk[kk][0], jk[kk][1], jk[kk][2], r[0], r[1], r[2]);
      }
      ph[hh][kk] = e;
      if (kk == 0) {
        rxs[hh] = h < md.N_h ? (double)md.Rh[3 * h] : 0.0;
        rys[hh] = h < md.N_h ? (double)md.Rh[3 * h + 1] : 0.0;
      }
    }
    __syncthreads();
    const int hmax = min(HB, md.N_h - hb);
    for (int hh = 0; hh < hmax; ++hh) {
      const double* rowA = md.Bp + (size_t)(1 + 2 * (hb + hh)) * WW;
      const double* rowB = rowA + WW;
      double A[4], B[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        int col = n0 + cg + 32 * c;
        A[c] = col < WW ? __ldg(rowA + col) : 0.0;
        B[c] = col < WW ? __ldg(rowB + col) : 0.0;
      }
      const double rx = rxs[hh], ry = rys[hh];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const double2 e = ph[hh][kg * 2 + q];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          double t1 = fma(e.x, B[c], -e.y * A[c]);     // c B - s A
          aH[q][c] = fma(e.x, A[c], aH[q][c]);
          aH[q][c] = fma(e.y, B[c], aH[q][c]);
          aX[q][c] = fma(rx, t1, aX[q][c]);
          aY[q][c] = fma(ry, t1, aY[q][c]);
        }
      }
    }
    __syncthreads();
  }

#pragma unroll
  for (int q = 0; q < 2; ++q) {
    int kk = k0 + kg * 2 + q;
    if (kk >= kl.n) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int col = n0 + cg + 32 * c;
      if (col >= WW) continue;
      size_t o = (size_t)kk * WW + col;
      Hp[o] = aH[q][c];
      Xp[o] = aX[q][c];
      Yp[o] = aY[q][c];
    }
  }
}

}  // namespace

cudaError_t launch_fourier_fp64(const Model& md, const Mesh& mesh, const KList& kl, double* Hp,
                                double* Xp, double* Yp, cudaStream_t s) {
  if (kl.n <= 0) return cudaSuccess;
  const int WW = md.W * md.W;
  dim3 grid((WW + TN - 1) / TN, (kl.n + TK - 1) / TK);
  fourier_fp64_kernel<<<grid, NT, 0, s>>>(md, mesh, kl, Hp, Xp, Yp);
  return cudaGetLastError();
}

}  // namespace kubo
