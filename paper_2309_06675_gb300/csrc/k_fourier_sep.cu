// Step (1) as three one-axis sums (the separable variant of the Fourier sum; FP64):
//
//   H(k) = sum_{R1} e^{i k1 R1} sum_{R2} e^{i k2 R2} sum_{R3} e^{i k3 R3} H(R1, R2, R3)
//
// over the bounding box of the R set (absent vectors contribute nothing).  Hermitian pairing
// H(-R) = H(R)^dagger gives B_{-R1}(k2, k3) = B_{R1}(k2, k3)^dagger for the partial sums
// B_{R1}(k2, k3) = sum_{R2, R3} e^{i (k2 R2 + k3 R3)} H(R1, R2, R3), so only R1 >= 0 is formed:
//
//   stage A (once per call):   A[j3][R1][R2] = sum_{R3} e^{i k3 R3} H(R1, R2, R3)
//   stage B (per pair block):  B[p][R1]  = sum_{R2} e^{i k2 R2} A[j3][R1][R2]
//                              By[p][R1] = sum_{R2} i R2 e^{i k2 R2} A[j3][R1][R2]
//   stage C (per k-point):     H   = B_0 + sum_{R1>0} (e^{i k1 R1} B_R1 + e^{-i k1 R1} B_R1^dagger)
//                              dxH = sum_{R1>0} i R1 (e^{i k1 R1} B_R1 - e^{-i k1 R1} B_R1^dagger)
//                              dyH = By_0 + sum_{R1>0} (e^{i k1 R1} By_R1 + e^{-i k1 R1} By_R1^dagger)
//
// with the mesh phases of the twiddle tables (exact argument reduction).  A batch is a block
// of (k2, k3) pairs times every k1-plane of the requested range, so each B is reused by all of
// the range's planes.  Per k-point this is O((n2 / planes + 3) (h1 + 1) W^2) work instead of
// the dense contraction's 6 N_R W^2 real flops.
#include <algorithm>

#include "kubo_internal.cuh"

namespace kubo {

namespace {

__device__ __forceinline__ double2 axis_phase(const double2* __restrict__ tab, int off, int N,
                                              int j, int r) {
  int a = (int)(((long long)j * r) % N);
  if (a < 0) a += N;
  return tab[off + a];
}

__device__ __forceinline__ void cmac(double2& acc, double2 p, double2 h) {
  acc.x = fma(p.x, h.x, fma(-p.y, h.y, acc.x));
  acc.y = fma(p.x, h.y, fma(p.y, h.x, acc.y));
}

// A[(j3 * (h1 + 1) + R1) * n2 + (R2 + h2)][q], R1 in 0..h1
__global__ void sep_stage_a_kernel(const double2* __restrict__ H_R, const int* __restrict__ box,
                                   SepBox sb, int WW, Mesh mesh, const double2* __restrict__ tab,
                                   int off3, double2* __restrict__ A) {
  const int n2 = 2 * sb.h2 + 1, n3 = 2 * sb.h3 + 1;
  const int64_t combos = (int64_t)mesh.N3 * (sb.h1 + 1) * n2;
  for (int64_t cb = blockIdx.y; cb < combos; cb += gridDim.y) {
    const int r2i = (int)(cb % n2);
    const int R1 = (int)((cb / n2) % (sb.h1 + 1));
    const int j3 = (int)(cb / ((int64_t)n2 * (sb.h1 + 1)));
    const int* brow = box + ((size_t)(R1 + sb.h1) * n2 + r2i) * n3;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < WW; q += gridDim.x * blockDim.x) {
      double2 acc = make_double2(0.0, 0.0);
      for (int r3 = 0; r3 < n3; ++r3) {
        const int idx = brow[r3];
        if (idx < 0) continue;
        cmac(acc, axis_phase(tab, off3, mesh.N3, j3, r3 - sb.h3), H_R[(size_t)idx * WW + q]);
      }
      A[(size_t)cb * WW + q] = acc;
    }
  }
}

// B[p][R1][q], By[p][R1][q] for the pairs p0 .. p0 + np - 1 (pair = j2 * N3 + j3)
__global__ void sep_stage_b_kernel(const double2* __restrict__ A, SepBox sb, int WW, Mesh mesh,
                                   const double2* __restrict__ tab, int off2, int64_t p0, int np,
                                   double2* __restrict__ B, double2* __restrict__ By) {
  const int n2 = 2 * sb.h2 + 1;
  const int64_t combos = (int64_t)np * (sb.h1 + 1);
  for (int64_t cb = blockIdx.y; cb < combos; cb += gridDim.y) {
    const int R1 = (int)(cb % (sb.h1 + 1));
    const int64_t p = cb / (sb.h1 + 1);
    const int64_t pair = p0 + p;
    const int j2 = (int)(pair / mesh.N3), j3 = (int)(pair % mesh.N3);
    const double2* Arow = A + ((size_t)j3 * (sb.h1 + 1) + R1) * n2 * WW;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < WW; q += gridDim.x * blockDim.x) {
      double2 b = make_double2(0.0, 0.0), by = make_double2(0.0, 0.0);
      for (int r2i = 0; r2i < n2; ++r2i) {
        const int R2 = r2i - sb.h2;
        const double2 ph = axis_phase(tab, off2, mesh.N2, j2, R2);
        const double2 a = Arow[(size_t)r2i * WW + q];
        double2 t = make_double2(0.0, 0.0);
        cmac(t, ph, a);
        b.x += t.x;
        b.y += t.y;
        by.x = fma(-(double)R2, t.y, by.x);   // i R2 t
        by.y = fma((double)R2, t.x, by.y);
      }
      B[(size_t)cb * WW + q] = b;
      By[(size_t)cb * WW + q] = by;
    }
  }
}

// packed H, dxH, dyH of every k-point of the batch (local t -> pair p = t / np1, plane
// j1 = j1a + t % np1); thread per (k, upper element)
__global__ void sep_stage_c_kernel(const double2* __restrict__ B, const double2* __restrict__ By,
                                   SepBox sb, int W, Mesh mesh, const double2* __restrict__ tab,
                                   int off1, int j1a, int np1, int n, double* __restrict__ Hp,
                                   double* __restrict__ Xp, double* __restrict__ Yp) {
  const int WW = W * W;
  const int nup = W * (W + 1) / 2;
  const int64_t total = (int64_t)n * nup;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(g / nup);
    const int e = (int)(g % nup);
    // upper element e -> (i, j), i <= j, row-major over the upper triangle: row i starts at
    // off(i) = i W - i (i - 1) / 2 (a float estimate, then exact integer corrections)
    const float bq = 2.0f * (float)W + 1.0f;
    int i = (int)((bq - sqrtf(fmaxf(bq * bq - 8.0f * (float)e, 0.0f))) * 0.5f);
    i = min(max(i, 0), W - 1);
    while (i > 0 && i * W - i * (i - 1) / 2 > e) --i;
    while (i + 1 < W && (i + 1) * W - (i + 1) * i / 2 <= e) ++i;
    const int j = i + (e - (i * W - i * (i - 1) / 2));
    const int p = t / np1, j1 = j1a + t % np1;
    const double2* Bp = B + (size_t)p * (sb.h1 + 1) * WW;
    const double2* Byp = By + (size_t)p * (sb.h1 + 1) * WW;
    const int ij = i * W + j, ji = j * W + i;
    double2 h = Bp[ij], y = Byp[ij], x = make_double2(0.0, 0.0);
    for (int R1 = 1; R1 <= sb.h1; ++R1) {
      const double2 ph = axis_phase(tab, off1, mesh.N1, j1, R1);   // e^{i k1 R1}
      const double2 b = Bp[(size_t)R1 * WW + ij], bt = Bp[(size_t)R1 * WW + ji];
      const double2 c = Byp[(size_t)R1 * WW + ij], ct = Byp[(size_t)R1 * WW + ji];
      // u = e^{i th} b, w = e^{-i th} conj(bt) = conj(e^{i th} bt)
      const double2 u = make_double2(ph.x * b.x - ph.y * b.y, ph.x * b.y + ph.y * b.x);
      const double2 w = make_double2(ph.x * bt.x - ph.y * bt.y, -(ph.x * bt.y + ph.y * bt.x));
      h.x += u.x + w.x;
      h.y += u.y + w.y;
      // i R1 (u - w)
      x.x = fma(-(double)R1, u.y - w.y, x.x);
      x.y = fma((double)R1, u.x - w.x, x.y);
      const double2 uy = make_double2(ph.x * c.x - ph.y * c.y, ph.x * c.y + ph.y * c.x);
      const double2 wy = make_double2(ph.x * ct.x - ph.y * ct.y, -(ph.x * ct.y + ph.y * ct.x));
      y.x += uy.x + wy.x;
      y.y += uy.y + wy.y;
    }
    const size_t o = (size_t)t * WW;
    Hp[o + ij] = h.x;
    Xp[o + ij] = x.x;
    Yp[o + ij] = y.x;
    if (i < j) {
      Hp[o + ji] = h.y;
      Xp[o + ji] = x.y;
      Yp[o + ji] = y.y;
    }
  }
}

int grid_1d(int64_t total, int threads) {
  int64_t b = (total + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

}  // namespace

size_t sep_a_elems(const SepBox& sb, int W, int N3) {
  return (size_t)N3 * (sb.h1 + 1) * (2 * sb.h2 + 1) * W * W;
}
size_t sep_b_elems_per_pair(const SepBox& sb, int W) { return (size_t)(sb.h1 + 1) * W * W; }

cudaError_t launch_sep_stage_a(const double2* H_R, const int* box, const SepBox& sb, int W,
                               const Mesh& mesh, const double2* tab, int off3, double2* A,
                               cudaStream_t s) {
  const int WW = W * W;
  const int64_t combos = (int64_t)mesh.N3 * (sb.h1 + 1) * (2 * sb.h2 + 1);
  dim3 grid((WW + 255) / 256, (unsigned)std::min<int64_t>(combos, 65535));
  sep_stage_a_kernel<<<grid, 256, 0, s>>>(H_R, box, sb, WW, mesh, tab, off3, A);
  return cudaGetLastError();
}

cudaError_t launch_sep_batch(const double2* A, const SepBox& sb, int W, const Mesh& mesh,
                             const double2* tab, const int tab_off[3], int64_t p0, int np,
                             int j1a, int np1, double2* B, double2* By, double* Hp, double* Xp,
                             double* Yp, cudaStream_t s) {
  if (np <= 0 || np1 <= 0) return cudaSuccess;
  const int WW = W * W;
  const int64_t combos = (int64_t)np * (sb.h1 + 1);
  dim3 gb((WW + 255) / 256, (unsigned)std::min<int64_t>(combos, 65535));
  sep_stage_b_kernel<<<gb, 256, 0, s>>>(A, sb, WW, mesh, tab, tab_off[1], p0, np, B, By);
  const int n = np * np1;
  sep_stage_c_kernel<<<grid_1d((int64_t)n * (W * (W + 1) / 2), 256), 256, 0, s>>>(
      B, By, sb, W, mesh, tab, tab_off[0], j1a, np1, n, Hp, Xp, Yp);
  return cudaGetLastError();
}

}  // namespace kubo
