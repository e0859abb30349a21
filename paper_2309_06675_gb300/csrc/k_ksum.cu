// k-sum of Eq. 2 (with Eq. 4's batching): S(E_F) = (1/N_k) sum_k sum_n occ(E_n(k)) Omega_n(k)
// for every (eta, E_F) pair.  Deterministic: every block sums a fixed k-range in order with
// Neumaier compensation, blocks are folded in index order, batches in call order.
//
// Step occupation (kT = 0): the levels of a k-point are ascending, so the occupied ones are a
// prefix of the bands and the per-k term is an inclusive prefix sum of Omega over the bands,
// looked up at the count of levels below E_F (binary search): O(log W) per (k, E_F) instead of
// O(W).  The prefix is accumulated in band order, so the per-k term is bit-identical to the
// direct sum over occupied bands.
#include <algorithm>

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

// Omega_n(k) <- sum_{m <= n} Omega_m(k), in place, for every eta (thread per (eta, k))
__global__ void band_prefix_kernel(double* __restrict__ Om, int W, int n, int n_eta,
                                   int64_t eta_stride) {
  const int64_t total = (int64_t)n_eta * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(t / n);
    const int64_t k = t % n;
    double* o = Om + e * eta_stride + k * W;
    double s = 0.0;
    for (int q = 0; q < W; ++q) {
      s += o[q];
      o[q] = s;
    }
  }
}

constexpr int KS_MAXE = 8;

// kT = 0: thread per E_F (all etas), k-range of the block in order
__global__ void ksum_step_kernel(const double* __restrict__ E, const double* __restrict__ P,
                                 int W, int n, int n_eta, int64_t eta_stride,
                                 const double* __restrict__ E_F, int n_EF,
                                 double2* __restrict__ part, int kpb) {
  const int b = blockIdx.x;
  const int kb = b * kpb, ke = min(n, kb + kpb);
  const int n_out = n_eta * n_EF;
  for (int j = threadIdx.x; j < n_EF; j += blockDim.x) {
    const double ef = E_F[j];
    double s[KS_MAXE], c[KS_MAXE];
#pragma unroll
    for (int e = 0; e < KS_MAXE; ++e) { s[e] = 0.0; c[e] = 0.0; }
    for (int k = kb; k < ke; ++k) {
      const double* Ek = E + (size_t)k * W;
      int lo = 0, hi = W;   // number of levels strictly below E_F
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (Ek[mid] < ef) lo = mid + 1;
        else hi = mid;
      }
      if (lo == 0) continue;
      const double* Pk = P + (size_t)k * W + (lo - 1);
#pragma unroll
      for (int e = 0; e < KS_MAXE; ++e)
        if (e < n_eta) neumaier_add(s[e], c[e], Pk[e * eta_stride]);
    }
#pragma unroll
    for (int e = 0; e < KS_MAXE; ++e)
      if (e < n_eta) part[(size_t)b * n_out + e * n_EF + j] = make_double2(s[e], c[e]);
  }
}

// one CTA per output: thread i folds the partials i, i + FOLD_NT, ... in order (Neumaier),
// then the per-thread (sum, compensation) pairs are combined in a fixed tree and added to the
// running accumulator (deterministic: the assignment and the order are fixed)
constexpr int FOLD_NT = 256;
__global__ void __launch_bounds__(FOLD_NT) ksum_fold_kernel(const double2* __restrict__ part,
                                                           int n_blocks, int n_out,
                                                           double2* __restrict__ acc) {
  __shared__ double ss[FOLD_NT], cc[FOLD_NT];
  const int t = threadIdx.x;
  for (int o = blockIdx.x; o < n_out; o += gridDim.x) {
    double s = 0.0, c = 0.0;
    for (int b = t; b < n_blocks; b += FOLD_NT) {
      const double2 p = part[(size_t)b * n_out + o];
      neumaier_add(s, c, p.x);
      neumaier_add(s, c, p.y);
    }
    ss[t] = s;
    cc[t] = c;
    __syncthreads();
    for (int h = FOLD_NT / 2; h > 0; h >>= 1) {
      if (t < h) {
        double s2 = ss[t], c2 = cc[t];
        neumaier_add(s2, c2, ss[t + h]);
        ss[t] = s2;
        cc[t] = c2 + cc[t + h];
      }
      __syncthreads();
    }
    if (t == 0) {
      double s2 = acc[o].x, c2 = acc[o].y;
      neumaier_add(s2, c2, ss[0]);
      acc[o] = make_double2(s2, c2 + cc[0]);
    }
    __syncthreads();
  }
}

__global__ void ksum_final_kernel(const double2* __restrict__ acc, int n_out, double inv_Nk,
                                  const DevStatus* st, double* __restrict__ out) {
  if (st->bits != 0) return;   // outputs are written only on success
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < n_out; o += gridDim.x * blockDim.x)
    out[o] = (acc[o].x + acc[o].y) * inv_Nk;
}

// ------------------------------------------------------------------ mixed-precision fix-up
// Two kinds of k-point carry most of the mixed path's error and are redone in FP64:
//  * a level within tau_k = rel * max_n |E_n(k)| of some Fermi level (its occupation could
//    flip under the FP32-level energy error);
//  * the spiky tail: ||Omega(k)||_inf among the largest `frac` of the batch (near-degenerate
//    pairs, whose curvature error ~ |Omega| dE / gap dominates the k-sum).
// Pass 1 (this kernel): per k the near-E_F flag and the bin of log2 ||Omega(k)||_inf.
constexpr int NBIN = 512;            // quarter-octave bins of log2 |Omega|
constexpr int BIN_OFFSET = 256;      // bin of |Omega| = 1

__global__ void fixup_flag_kernel(const double* __restrict__ E, const double* __restrict__ Om,
                                  int W, int n, int n_eta, int64_t eta_stride,
                                  const double* __restrict__ E_F, int n_EF, double rel,
                                  int* __restrict__ flag, int* __restrict__ bin) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const double* Ek = E + (size_t)k * W;
    double mx = 0.0;
    for (int q = 0; q < W; ++q) mx = fmax(mx, fabs(Ek[q]));
    const double tau = rel * mx;
    int f = 0;
    for (int j = 0; j < n_EF && !f; ++j) {
      const double ef = E_F[j];
      for (int q = 0; q < W; ++q)
        if (fabs(Ek[q] - ef) < tau) { f = 1; break; }
    }
    double om = 0.0;
    for (int e = 0; e < n_eta; ++e)
      for (int q = 0; q < W; ++q) om = fmax(om, fabs(Om[e * eta_stride + (size_t)k * W + q]));
    int b = 0;
    if (om > 0.0) {
      b = (int)floorf(4.0f * log2f((float)om)) + BIN_OFFSET;
      b = b < 0 ? 0 : (b >= NBIN ? NBIN - 1 : b);
    }
    flag[k] = f;
    bin[k] = b;
  }
}

// Pass 2 (one block): integer histogram of the bins -> threshold bin of the top `frac`
// (deterministic), then order-preserving compaction: pos[c] = local index, kid[c] = mesh index
// of the c-th flagged k-point, *count = number flagged.
__global__ void fixup_compact_kernel(const int* __restrict__ flag, const int* __restrict__ bin,
                                     int n, double frac, KList kl, int* __restrict__ pos,
                                     int64_t* __restrict__ kid, int* __restrict__ count) {
  __shared__ int hist[NBIN];
  __shared__ int warp_tot[32];
  __shared__ int base_sh, thr_sh;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int b = threadIdx.x; b < NBIN; b += blockDim.x) hist[b] = 0;
  if (threadIdx.x == 0) base_sh = 0;
  __syncthreads();
  for (int t = threadIdx.x; t < n; t += blockDim.x) atomicAdd(&hist[bin[t]], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    const int budget = (int)(frac * (double)n);
    int acc = 0, thr = NBIN;          // no k-point flagged by curvature when budget == 0
    for (int b = NBIN - 1; b > 0; --b) {
      if (acc + hist[b] > budget) break;
      acc += hist[b];
      thr = b;
    }
    thr_sh = thr;
  }
  __syncthreads();
  const int thr = thr_sh;
  for (int c0 = 0; c0 < n; c0 += blockDim.x) {
    const int t = c0 + threadIdx.x;
    const int f = t < n ? (flag[t] | (bin[t] >= thr ? 1 : 0)) : 0;
    const unsigned b = __ballot_sync(0xffffffffu, f);
    const int within = __popc(b & ((1u << lane) - 1u));
    if (lane == 0) warp_tot[warp] = __popc(b);
    __syncthreads();
    int off = base_sh;
    for (int w = 0; w < warp; ++w) off += warp_tot[w];
    if (f) {
      pos[off + within] = t;
      kid[off + within] = klist_get(kl, t);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int w = 0; w < nw; ++w) tot += warp_tot[w];
      base_sh += tot;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = base_sh;
}

// E[pos[c]] = Efix[c], Om[e][pos[c]] = Omfix[e][c]
__global__ void fixup_scatter_kernel(const int* __restrict__ pos, int cnt, int W, int n_eta,
                                     const double* __restrict__ Efix,
                                     const double* __restrict__ Omfix, int64_t fix_eta_stride,
                                     double* __restrict__ E, double* __restrict__ Om,
                                     int64_t eta_stride) {
  const int64_t total = (int64_t)cnt * W;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t / W), q = (int)(t % W);
    const int64_t k = pos[c];
    E[k * W + q] = Efix[t];
    for (int e = 0; e < n_eta; ++e) Om[e * eta_stride + k * W + q] = Omfix[e * fix_eta_stride + t];
  }
}

}  // namespace

cudaError_t launch_ksum_partial(const double* E, double* Om, int W, int n, int n_eta,
                                int64_t eta_stride, const double* E_F, int n_EF, double kT,
                                double2* part, int kpb, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int nb = (n + kpb - 1) / kpb;
  if (kT == 0.0 && n_eta <= KS_MAXE) {
    const int64_t rows = (int64_t)n_eta * n;
    const int pb = (int)std::min<int64_t>((rows + 127) / 128, 152 * 16);
    band_prefix_kernel<<<pb, 128, 0, s>>>(Om, W, n, n_eta, eta_stride);
    const int nt = std::min(256, (n_EF + 31) / 32 * 32);
    ksum_step_kernel<<<nb, nt, 0, s>>>(E, Om, W, n, n_eta, eta_stride, E_F, n_EF, part, kpb);
  } else {
    ksum_partial_kernel<<<nb, 128, 0, s>>>(E, Om, W, n, n_eta, eta_stride, E_F, n_EF, kT, part, kpb);
  }
  return cudaGetLastError();
}

cudaError_t launch_ksum_fold(const double2* part, int n_blocks, int n_out, double2* acc,
                             cudaStream_t s) {
  if (n_blocks <= 0) return cudaSuccess;
  ksum_fold_kernel<<<std::min(n_out, 152 * 8), FOLD_NT, 0, s>>>(part, n_blocks, n_out, acc);
  return cudaGetLastError();
}

cudaError_t launch_ksum_final(const double2* acc, int n_out, double inv_Nk, const DevStatus* st,
                              double* out, cudaStream_t s) {
  ksum_final_kernel<<<(n_out + 127) / 128, 128, 0, s>>>(acc, n_out, inv_Nk, st, out);
  return cudaGetLastError();
}

cudaError_t launch_fixup_flag(const double* E, const double* Om, int W, int n, int n_eta,
                              int64_t eta_stride, const double* E_F, int n_EF, double rel,
                              int* flag, int* bin, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  fixup_flag_kernel<<<(n + 255) / 256, 256, 0, s>>>(E, Om, W, n, n_eta, eta_stride, E_F, n_EF, rel,
                                                    flag, bin);
  return cudaGetLastError();
}

cudaError_t launch_fixup_compact(const int* flag, const int* bin, int n, double frac,
                                 const KList& kl, int* pos, int64_t* kid, int* count,
                                 cudaStream_t s) {
  fixup_compact_kernel<<<1, 1024, 0, s>>>(flag, bin, n, frac, kl, pos, kid, count);
  return cudaGetLastError();
}

cudaError_t launch_fixup_scatter(const int* pos, int cnt, int W, int n_eta, const double* Efix,
                                 const double* Omfix, int64_t fix_eta_stride, double* E, double* Om,
                                 int64_t eta_stride, cudaStream_t s) {
  if (cnt <= 0) return cudaSuccess;
  int64_t total = (int64_t)cnt * W;
  int b = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  fixup_scatter_kernel<<<b, 256, 0, s>>>(pos, cnt, W, n_eta, Efix, Omfix, fix_eta_stride, E, Om,
                                         eta_stride);
  return cudaGetLastError();
}

}  // namespace kubo
