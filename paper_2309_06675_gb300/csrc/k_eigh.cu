// Step (2) of List 1/2 ("diagonalize"): batched FP64 Hermitian eigendecomposition.
//
// The paper batches an EISPACK-derived solver along the vector dimension of a vector
// engine (Sec. 2.3): l_B matrices advance in lock-step, one per vector lane.  On GB300 an
// FP64 warp instruction occupies the SM's FP64 pipe for 16 cycles whatever its active
// mask, and a dependent DFMA has 64 cycles of latency, so the solver is split by the kind
// of parallelism each stage has:
//
//   tridiag_kernel   one CTA per k-point.  Householder reduction H = Q T_c Q^dagger with
//                    Hermitian reflectors I - tau v v^dagger (tau real); the reduction is
//                    vectorised over matrix rows/elements.  T_c is made real by the diagonal
//                    unitary D (T_c = D T D^dagger, T[j+1][j] = |beta_j|).
//   ql_kernel        one LANE per k-point (the paper's batching along the vector length):
//                    implicit QL with Wilkinson shifts on the real tridiagonal T, eigenvalues
//                    only.  The rotation recurrence is inherently scalar, so 32 k-points share
//                    each warp instruction; each lane advances through its own eigenvalues.
//   backtransform_kernel  one CTA per k-point: sorts the eigenvalues, computes the
//                    eigenvectors Z of T by inverse iteration and forms U = Q D Z by applying
//                    the reflectors to the columns of D Z.
//
// Padded leading dimensions (W+1) keep column walks conflict-free in shared memory (the
// GPU counterpart of the paper's padding against memory-bank conflicts).
#include <climits>

#include "kubo_internal.cuh"

namespace kubo {

namespace {

constexpr int NT = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------ K2a: tridiagonalise
// The Hermitian matrix is held as its lower triangle, packed by rows: element (r, c <= r) at
// r (r + 1) / 2 + c (33 KB at W = 64), so that several CTAs share an SM and hide each
// other's scalar Householder steps.
__device__ __forceinline__ int tri(int r, int c) { return (r * (r + 1) >> 1) + c; }

// Packed rows of leading dimension ld (W*W for the FP64 Fourier kernel, the padded row of
// H | dxH | dyH for the tensor-core one).  The reduction is FP64.
// threads of the one-k reduction's CTA (orders W > 64; W <= 64 runs two k-points per CTA in
// tridiag2_kernel below)
constexpr int TRI_NT = 512;

// Column partitions of the symv for trailing order m on nt threads: the count P up to
// min(nt / m, cap) with the fewest FP64 warp instructions -- thread t takes row t mod m and part
// t / m, so warp w's lanes start at part 32 w / m and run ceil((m - part) / P) columns of 4 FMAs,
// and the partial-sum pass runs ceil(m / 32) warps of 2 P + 2 operations.  For the two-k
// reduction, whose three CTAs per SM keep the FP64 pipe fed while one of them runs a phase on
// few warps.
__device__ __forceinline__ int symv_partitions(int m, int nt, int cap) {
  const int pmax = max(1, min(nt / m, cap));
  int best = 1, bcost = INT_MAX;
  for (int P = 1; P <= pmax; ++P) {
    int c = ((m + 31) >> 5) * (2 * P + 2);
    for (int w = 0; 32 * w < m * P; ++w) c += 4 * ((m - (32 * w) / m + P - 1) / P);
    if (c < bcost) { bcost = c; best = P; }
  }
  return best;
}

// NTT = 512 threads: one CTA (136 KB of shared memory at W = 128) holds an SM, and more warps
// than 256 cover its barriers (W = 128: 235 -> 229 ms per 18,432 k-points; 1,024 threads
// with twice the symv parts: 240 ms)
template <typename T, int NTT>
__global__ void __launch_bounds__(NTT, 1) tridiag_kernel(const T* __restrict__ Hp, int64_t ld, int W,
                                                     EighBufs b) {
  // the reflector is read from its column of A (not copied), the symv partials share their
  // array with p, and beta_i, tau_i go to the outputs as they are formed (beta_i into the phase
  // row, which is rewritten at the end): the triangle plus NTT partials of shared memory
  extern __shared__ double2 smem2[];
  double2* A = smem2;                              // lower triangle, packed by rows
  double2* sp = A + (size_t)W * (W + 1) / 2;       // [NTT] partial sums of the symv
  double2* pb = sp;                                // [W] p, then w (the symv's part-0 slots)
  __shared__ double s_tau, s_K;
  double2* beg = b.phase + blockIdx.x * (int64_t)W;   // beta_i until the phases replace them
  double* tout = b.tau + blockIdx.x * (int64_t)W;

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t k = blockIdx.x;
  const T* P = Hp + (size_t)k * ld;

  for (int idx = t; idx < W * (W + 1) / 2; idx += NTT) {
    int r = (int)((sqrtf(8.0f * (float)idx + 1.0f) - 1.0f) * 0.5f);
    while (tri(r, 0) > idx) --r;
    while (tri(r + 1, 0) <= idx) ++r;
    const int c = idx - tri(r, 0);
    A[idx] = r == c ? make_double2((double)P[r * W + r], 0.0)
                    : make_double2((double)P[c * W + r], -(double)P[r * W + c]);   // conj(A_cr)
  }
  __syncthreads();

  for (int i = 0; i < W - 2; ++i) {
    const int o = i + 1;       // first row of the trailing block
    const int m = W - 1 - i;   // its size
    if (warp == 0) {
      double s2 = 0.0;
      for (int r = o + 1 + lane; r < W; r += 32) {
        double2 x = A[tri(r, i)];
        s2 = fma(x.x, x.x, fma(x.y, x.y, s2));
      }
      s2 = warp_sum(s2);
      // H = I - tau v v^H with v = x - beta e1, beta = -e^{i arg alpha} |x|:
      // v0 = alpha + e^{i arg alpha} |x|, tau = 2 / v^H v = 1 / (|x| (|x| + |alpha|)).
      // Few lanes run this, and every FP64 instruction takes a whole warp slot of the pipe
      // whatever its active mask, so the two independent halves run side by side in lanes 0
      // and 1: |x| = n2 rsqrt(n2) and |alpha| = aa2 rsqrt(aa2) in one rsqrt, then the real and
      // imaginary parts of the unit phase alpha / |alpha|, of beta and of v0 in one instruction
      // each.
      if (lane < 2) {
        const double2 al = A[tri(o, i)];
        const double aa2 = fma(al.x, al.x, al.y * al.y);
        const double x2 = lane == 0 ? aa2 + s2 : aa2;     // |x|^2 (lane 0), |alpha|^2 (lane 1)
        const double rx = mag_bits(x2) != 0ull ? rsqrt(x2) : 0.0;   // (sums of squares: integer tests)
        const double xn = x2 * rx;                         // |x| (lane 0), |alpha| (lane 1)
        const double nrm = __shfl_sync(0x3u, xn, 0);
        const double aa = __shfl_sync(0x3u, xn, 1);
        const double ra = __shfl_sync(0x3u, rx, 1);
        const double comp = lane == 0 ? al.x : al.y;
        // the unit phase of alpha (1 for alpha = 0)
        const double ph = mag_bits(aa2) != 0ull ? comp * ra : (lane == 0 ? 1.0 : 0.0);
        if (mag_bits(s2) != 0ull) {
          const double bet = -ph * nrm;
          const double v0 = fma(ph, nrm, comp);
          double* Ao = reinterpret_cast<double*>(&A[tri(o, i)]);
          double* bo = reinterpret_cast<double*>(&beg[i]);
          Ao[lane] = v0;
          bo[lane] = bet;
          if (lane == 0) {
            const double tau = recip_nr(nrm * (nrm + aa));
            s_tau = tau;
            tout[i] = tau;
          }
        } else {
          reinterpret_cast<double*>(&beg[i])[lane] = comp;   // beta = alpha, no reflection
          if (lane == 0) {
            s_tau = 0.0;
            tout[i] = 0.0;
          }
        }
      }
    }
    __syncthreads();
    const double tau = s_tau;
    if (tau != 0.0) {
      // v: column i of A from row o (its first entry v0 written by the scalar step); the symv
      // reads it there (one address per warp), the later phases from a copy at sp + W
      double2* vb = sp + W;
      // p = tau * A22 v  (lower storage: A22[r][c] = conj(A22[c][r]) for c > r).  The m x m
      // product is spread over the block: thread t takes row r = t mod m and the columns
      // c = part, part + P, ... (part = t / m, P = min(NTT / m, cap) parts per row, cap = 4 by
      // default), so that the warps issue full; the P partial sums of a row are added in part
      // order by the m row threads.  P is capped: for a small trailing block more parts would
      // shorten the product but lengthen that sum, whose warps run with m of their 32 lanes.
      // (The two-k kernel picks P per m by instruction count instead; here, with one CTA per
      // SM at W = 128, fewer parts leave the FP64 pipe without other warps to issue: 6 %
      // slower.)  The conjugate of the mirrored element flips a sign bit on the integer side
      // (no FP64 instruction).
      {
        const int P = max(1, min(NTT / m, b.symv_parts));
        const int r = t % m, part = t / m;
        if (part < P) {
          double ax = 0.0, ay = 0.0;
          const int rowb = tri(o + r, o);
          for (int c = part; c < m; c += P) {
            const int idx = c <= r ? rowb + c : tri(o + c, o + r);
            double2 a = A[idx];
            const unsigned long long flip = c > r ? 0x8000000000000000ull : 0ull;
            a.y = __longlong_as_double(__double_as_longlong(a.y) ^ flip);
            const double2 v = A[tri(o + c, i)];
            ax = fma(a.x, v.x, ax); ax = fma(-a.y, v.y, ax);
            ay = fma(a.x, v.y, ay); ay = fma(a.y, v.x, ay);
          }
          sp[part * m + r] = make_double2(ax, ay);
        }
        __syncthreads();
        for (int rr = t; rr < m; rr += NTT) {
          double sx = 0.0, sy = 0.0;
          for (int q = 0; q < P; ++q) {
            const double2 v = sp[q * m + rr];
            sx += v.x;
            sy += v.y;
          }
          pb[rr] = make_double2(tau * sx, tau * sy);
        }
      }
      __syncthreads();
      if (warp == 0) {
        double sum = 0.0;   // Re(v^H p)
        for (int r = lane; r < m; r += 32) {
          const double2 v = A[tri(o + r, i)], p = pb[r];
          sum = fma(v.x, p.x, fma(v.y, p.y, sum));
        }
        sum = warp_sum(sum);
        if (lane == 0) s_K = 0.5 * tau * sum;
      } else {
        for (int r = t - 32; r < m; r += NTT - 32) vb[r] = A[tri(o + r, i)];
      }
      __syncthreads();
      const double K = s_K;
      for (int r = t; r < m; r += NTT) {
        const double2 p = pb[r], v = vb[r];
        pb[r] = make_double2(fma(-K, v.x, p.x), fma(-K, v.y, p.y));
      }
      __syncthreads();
      // A22 <- A22 - v w^H - w v^H on the lower triangle: the strictly lower elements (c < r),
      // eight FMAs each with every lane busy, then the diagonal (real part only)
      const int nlow = m * (m - 1) / 2;
      for (int idx = t; idx < nlow; idx += NTT) {
        int r = (int)((sqrtf(8.0f * (float)idx + 1.0f) + 1.0f) * 0.5f);
        while (r * (r - 1) / 2 > idx) --r;
        while ((r + 1) * r / 2 <= idx) ++r;
        const int c = idx - r * (r - 1) / 2;
        const double2 vr = vb[r], wr = pb[r], vc = vb[c], wc = pb[c];
        double2 a = A[tri(o + r, o + c)];
        // v_r conj(w_c) + w_r conj(v_c)
        a.x = fma(-vr.x, wc.x, a.x); a.x = fma(-vr.y, wc.y, a.x);
        a.x = fma(-wr.x, vc.x, a.x); a.x = fma(-wr.y, vc.y, a.x);
        a.y = fma(-vr.y, wc.x, a.y); a.y = fma(vr.x, wc.y, a.y);
        a.y = fma(-wr.y, vc.x, a.y); a.y = fma(wr.x, vc.y, a.y);
        A[tri(o + r, o + c)] = a;
      }
      for (int r = t; r < m; r += NTT) {
        const double2 vr = vb[r], wr = pb[r];
        double2 a = A[tri(o + r, o + r)];
        a.x = fma(-vr.x, wr.x, a.x); a.x = fma(-vr.y, wr.y, a.x);
        a.x = fma(-wr.x, vr.x, a.x); a.x = fma(-wr.y, vr.y, a.x);
        a.y = 0.0;
        A[tri(o + r, o + r)] = a;
      }
    }
    __syncthreads();
  }

  // outputs: d, |e|, phases D, tau, reflectors
  double* dout = b.d + k * W;
  double* eout = b.e + k * W;
  double2* phout = b.phase + k * W;   // = beg: beta_j until the running product replaces them
  // |beta_j| and the unit phases beta_j / |beta_j| in parallel, then their running product
  // D_{j+1} = D_j beta_j / |beta_j| by one thread (4 FP64 operations per step)
  if (t == 0 && W >= 2) beg[W - 2] = A[tri(W - 1, W - 2)];
  __syncthreads();
  for (int j = t; j + 1 < W; j += NTT) {
    const double2 bj = beg[j];
    const double a2 = fma(bj.x, bj.x, bj.y * bj.y);
    double a = 0.0;
    double2 u = make_double2(1.0, 0.0);
    if (a2 > 0.0) {
      const double ra = rsqrt(a2);
      a = a2 * ra;
      u = make_double2(bj.x * ra, bj.y * ra);
    }
    eout[j] = a;
    sp[j] = u;
  }
  __syncthreads();
  if (t < 32) {
    // D_0 = 1, D_{j+1} = D_j u_j as a warp scan: lane l takes u_4l .. u_4l+3 (W <= 128)
    double2 u[4];
    double2 pr = make_double2(1.0, 0.0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = 4 * t + q;
      u[q] = j + 1 < W ? sp[j] : make_double2(1.0, 0.0);
      pr = cmul(pr, u[q]);
    }
    double2 sc = pr;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      double2 o2;
      o2.x = __shfl_up_sync(0xffffffffu, sc.x, off);
      o2.y = __shfl_up_sync(0xffffffffu, sc.y, off);
      if (t >= off) sc = cmul(o2, sc);
    }
    double2 D;
    D.x = __shfl_up_sync(0xffffffffu, sc.x, 1);
    D.y = __shfl_up_sync(0xffffffffu, sc.y, 1);
    if (t == 0) D = make_double2(1.0, 0.0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = 4 * t + q;
      if (j < W) phout[j] = D;
      D = cmul(D, u[q]);
    }
    if (t == 0) eout[W - 1] = 0.0;
  }
  for (int j = t; j < W; j += NTT) {
    dout[j] = A[tri(j, j)].x;
    if (j >= W - 2) tout[j] = 0.0;   // tau_j of the reflections: written as formed
  }
  double2* rout = b.refl + (size_t)k * W * W;
  for (int idx = t; idx < W * W; idx += NTT) {
    int r = idx / W, c = idx % W;
    rout[idx] = r > c ? A[tri(r, c)] : make_double2(0.0, 0.0);
  }
}

// Two k-points per 512-thread CTA (W <= 64; three CTAs per SM, the same six k-points per SM
// as the one-k kernel).  Half h = t / 256 works on k-point 2 blockIdx + h with the one-k
// kernel's thread layout; the per-column steps that one warp runs -- the norm of the column,
// the Householder scalar step and Re(v^H p) -- run for both k-points in warp 0 (lanes 0-15 /
// 16-31 for the reductions, lanes 0-1 / 2-3 for the scalar step), so each of those FP64
// instructions serves two k-points, and every block barrier serves two.  A half whose
// k-point is absent (odd count) or whose column needs no reflection idles through the phases.
__global__ void __launch_bounds__(512, 3) tridiag2_kernel(const double* __restrict__ Hp,
                                                          int64_t ld, int W, int n, EighBufs b) {
  extern __shared__ double2 smem2[];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int h = t >> 8, th = t & 255;
  const size_t per_k = (size_t)W * (W + 1) / 2 + 256;   // triangle + partials
  double2* A = smem2 + h * per_k;
  double2* sp = A + (size_t)W * (W + 1) / 2;
  double2* pb = sp;
  __shared__ double s_tau[2], s_K[2];
  __shared__ unsigned char s_parts[64];   // symv column partitions for trailing order m
  const int64_t k = 2 * (int64_t)blockIdx.x + h;
  const bool live = k < n;
  double2* beg = b.phase + k * W;
  if (t >= 1 && t < W) s_parts[t] = (unsigned char)symv_partitions(t, 256, b.symv_parts);
  double* tout = b.tau + k * W;
  const double* P = Hp + (size_t)k * ld;

  if (live)
    for (int idx = th; idx < W * (W + 1) / 2; idx += 256) {
      int r = (int)((sqrtf(8.0f * (float)idx + 1.0f) - 1.0f) * 0.5f);
      while (tri(r, 0) > idx) --r;
      while (tri(r + 1, 0) <= idx) ++r;
      const int c = idx - tri(r, 0);
      A[idx] = r == c ? make_double2(P[r * W + r], 0.0)
                      : make_double2(P[c * W + r], -P[r * W + c]);   // conj(A_cr)
    }
  __syncthreads();

  for (int i = 0; i < W - 2; ++i) {
    const int o = i + 1;       // first row of the trailing block
    const int m = W - 1 - i;   // its size
    if (warp == 0) {
      // lanes 0-15: k-point of half 0, 16-31: half 1
      const int hh = lane >> 4, l16 = lane & 15;
      const double2* Ah = smem2 + hh * per_k;
      const bool lv = 2 * (int64_t)blockIdx.x + hh < n;
      double s2 = 0.0;
      if (lv)
        for (int r = o + 1 + l16; r < W; r += 16) {
          const double2 x = Ah[tri(r, i)];
          s2 = fma(x.x, x.x, fma(x.y, x.y, s2));
        }
#pragma unroll
      for (int off = 8; off > 0; off >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, off);
      // the scalar step (see the one-k kernel): lanes 2 kk, 2 kk + 1 for the k-point of half kk
      const double s2k = __shfl_sync(0xffffffffu, s2, (lane >> 1) << 4);
      if (lane < 4) {
        const int kk = lane >> 1, sub = lane & 1;
        const bool lk = 2 * (int64_t)blockIdx.x + kk < n;
        double2* Ak = smem2 + kk * per_k;
        const double2 al = lk ? Ak[tri(o, i)] : make_double2(0.0, 0.0);
        const double aa2 = fma(al.x, al.x, al.y * al.y);
        const double x2 = sub == 0 ? aa2 + s2k : aa2;    // |x|^2, |alpha|^2
        // (x2, aa2 and s2k are sums of squares: "> 0" is a non-zero bit pattern, tested on the
        // integer side -- these FP64 instructions would issue with four lanes active)
        const double rx = mag_bits(x2) != 0ull ? rsqrt(x2) : 0.0;
        const double xn = x2 * rx;                         // |x|, |alpha|
        const double nrm = __shfl_sync(0xFu, xn, 2 * kk);
        const double aa = __shfl_sync(0xFu, xn, 2 * kk + 1);
        const double ra = __shfl_sync(0xFu, rx, 2 * kk + 1);
        const double comp = sub == 0 ? al.x : al.y;
        const double ph = mag_bits(aa2) != 0ull ? comp * ra : (sub == 0 ? 1.0 : 0.0);
        double2* begk = b.phase + (2 * (int64_t)blockIdx.x + kk) * W;
        double* toutk = b.tau + (2 * (int64_t)blockIdx.x + kk) * W;
        if (lk) {
          if (mag_bits(s2k) != 0ull) {
            const double bet = -ph * nrm;
            const double v0 = fma(ph, nrm, comp);
            reinterpret_cast<double*>(&Ak[tri(o, i)])[sub] = v0;
            reinterpret_cast<double*>(&begk[i])[sub] = bet;
            if (sub == 0) {
              const double tau = recip_nr(nrm * (nrm + aa));
              s_tau[kk] = tau;
              toutk[i] = tau;
            }
          } else {
            reinterpret_cast<double*>(&begk[i])[sub] = comp;   // beta = alpha, no reflection
            if (sub == 0) {
              s_tau[kk] = 0.0;
              toutk[i] = 0.0;
            }
          }
        } else if (sub == 0) {
          s_tau[kk] = 0.0;
        }
      }
    }
    __syncthreads();
    const double tau = s_tau[h];
    const bool act = live && tau != 0.0;
    double2* vb = sp + W;
    // p = tau * A22 v (the one-k kernel's partition over the half's 256 threads, with the
    // partition count of the table)
    const int P2 = s_parts[m];
    {
      const int r = th % m, part = th / m;
      if (act && part < P2) {
        double ax = 0.0, ay = 0.0;
        const int rowb = tri(o + r, o);
        for (int c = part; c < m; c += P2) {
          const int idx = c <= r ? rowb + c : tri(o + c, o + r);
          double2 a = A[idx];
          const unsigned long long flip = c > r ? 0x8000000000000000ull : 0ull;
          a.y = __longlong_as_double(__double_as_longlong(a.y) ^ flip);
          const double2 v = A[tri(o + c, i)];
          ax = fma(a.x, v.x, ax); ax = fma(-a.y, v.y, ax);
          ay = fma(a.x, v.y, ay); ay = fma(a.y, v.x, ay);
        }
        sp[part * m + r] = make_double2(ax, ay);
      }
    }
    __syncthreads();
    if (act)
      for (int rr = th; rr < m; rr += 256) {
        double sx = 0.0, sy = 0.0;
        for (int q = 0; q < P2; ++q) {
          const double2 v = sp[q * m + rr];
          sx += v.x;
          sy += v.y;
        }
        pb[rr] = make_double2(tau * sx, tau * sy);
      }
    __syncthreads();
    if (warp == 0) {
      const int hh = lane >> 4, l16 = lane & 15;
      const double2* Ah = smem2 + hh * per_k;
      const double2* ph2 = Ah + (size_t)W * (W + 1) / 2;
      const double tk = s_tau[hh];
      double sum = 0.0;   // Re(v^H p)
      if (tk != 0.0)
        for (int r = l16; r < m; r += 16) {
          const double2 v = Ah[tri(o + r, i)], p = ph2[r];
          sum = fma(v.x, p.x, fma(v.y, p.y, sum));
        }
#pragma unroll
      for (int off = 8; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
      if (l16 == 0) s_K[hh] = 0.5 * tk * sum;
    } else if (act) {
      // the copy of v: half 0 without its warp 0 (busy above), half 1 whole
      const int base = h == 0 ? 32 : 0;
      for (int r = th - base; r < m; r += 256 - base) vb[r] = A[tri(o + r, i)];
    }
    __syncthreads();
    const double K = s_K[h];
    if (act)
      for (int r = th; r < m; r += 256) {
        const double2 p = pb[r], v = vb[r];
        pb[r] = make_double2(fma(-K, v.x, p.x), fma(-K, v.y, p.y));
      }
    __syncthreads();
    if (act) {
      // A22 <- A22 - v w^H - w v^H on the lower triangle: the strictly lower elements (c < r),
      // eight FMAs each with every lane busy, then the diagonal (real part only)
      const int nlow = m * (m - 1) / 2;
      for (int idx = th; idx < nlow; idx += 256) {
        int r = (int)((sqrtf(8.0f * (float)idx + 1.0f) + 1.0f) * 0.5f);
        while (r * (r - 1) / 2 > idx) --r;
        while ((r + 1) * r / 2 <= idx) ++r;
        const int c = idx - r * (r - 1) / 2;
        const double2 vr = vb[r], wr = pb[r], vc = vb[c], wc = pb[c];
        double2 a = A[tri(o + r, o + c)];
        a.x = fma(-vr.x, wc.x, a.x); a.x = fma(-vr.y, wc.y, a.x);
        a.x = fma(-wr.x, vc.x, a.x); a.x = fma(-wr.y, vc.y, a.x);
        a.y = fma(-vr.y, wc.x, a.y); a.y = fma(vr.x, wc.y, a.y);
        a.y = fma(-wr.y, vc.x, a.y); a.y = fma(wr.x, vc.y, a.y);
        A[tri(o + r, o + c)] = a;
      }
      for (int r = th; r < m; r += 256) {
        const double2 vr = vb[r], wr = pb[r];
        double2 a = A[tri(o + r, o + r)];
        a.x = fma(-vr.x, wr.x, a.x); a.x = fma(-vr.y, wr.y, a.x);
        a.x = fma(-wr.x, vr.x, a.x); a.x = fma(-wr.y, vr.y, a.x);
        a.y = 0.0;
        A[tri(o + r, o + r)] = a;
      }
    }
    __syncthreads();
  }
  if (!live) return;   // no block barrier follows

  // outputs (as the one-k kernel)
  double* dout = b.d + k * W;
  double* eout = b.e + k * W;
  double2* phout = beg;
  if (th == 0 && W >= 2) beg[W - 2] = A[tri(W - 1, W - 2)];
  // the half's own threads only from here: named barrier 1 + h over its 256 threads
  asm volatile("bar.sync %0, 256;" ::"r"(1 + h) : "memory");
  for (int j = th; j + 1 < W; j += 256) {
    const double2 bj = beg[j];
    const double a2 = fma(bj.x, bj.x, bj.y * bj.y);
    double a = 0.0;
    double2 u = make_double2(1.0, 0.0);
    if (a2 > 0.0) {
      const double ra = rsqrt(a2);
      a = a2 * ra;
      u = make_double2(bj.x * ra, bj.y * ra);
    }
    eout[j] = a;
    sp[j] = u;
  }
  asm volatile("bar.sync %0, 256;" ::"r"(1 + h) : "memory");
  if (th < 32) {
    // D_0 = 1, D_{j+1} = D_j u_j as a warp scan (a serial chain of 63 complex products in one
    // thread would hold the CTA's shared memory while it queues behind the FP64 pipe): lane l
    // takes u_2l, u_2l+1, then the lanes' products are scanned in five steps
    const int j0 = 2 * th, j1 = j0 + 1;
    const double2 u0 = j0 + 1 < W ? sp[j0] : make_double2(1.0, 0.0);
    const double2 u1 = j1 + 1 < W ? sp[j1] : make_double2(1.0, 0.0);
    const double2 pr = cmul(u0, u1);
    double2 sc = pr;   // inclusive scan of the lanes' pair products
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      double2 o2;
      o2.x = __shfl_up_sync(0xffffffffu, sc.x, off);
      o2.y = __shfl_up_sync(0xffffffffu, sc.y, off);
      if (th >= off) sc = cmul(o2, sc);
    }
    double2 ex;        // product of u_0 .. u_{2l-1}
    ex.x = __shfl_up_sync(0xffffffffu, sc.x, 1);
    ex.y = __shfl_up_sync(0xffffffffu, sc.y, 1);
    if (th == 0) ex = make_double2(1.0, 0.0);
    if (j0 < W) phout[j0] = ex;
    if (j1 < W) phout[j1] = cmul(ex, u0);
    if (th == 0) eout[W - 1] = 0.0;
  }
  for (int j = th; j < W; j += 256) {
    dout[j] = A[tri(j, j)].x;
    if (j >= W - 2) tout[j] = 0.0;
  }
  double2* rout = b.refl + (size_t)k * W * W;
  for (int idx = th; idx < W * W; idx += 256) {
    int r = idx / W, c = idx % W;
    rout[idx] = r > c ? A[tri(r, c)] : make_double2(0.0, 0.0);
  }
}

// ------------------------------------------------------------------ K2b: QL, lane per k
// Eigenvalues of the real symmetric tridiagonal T by implicit QL with Wilkinson shifts, one
// k-point per lane.  Smem per warp: d and e as [W][32] (lane-interleaved: conflict-free for
// any mix of indices across lanes).  Iterations per eigenvalue are capped (-> ST_NO_CONVERGENCE).
__global__ void __launch_bounds__(32) ql_kernel(int W, int n, EighBufs b, DevStatus* st) {
  extern __shared__ double qsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  double* D = qsm + (size_t)warp * 2 * W * 32 + lane;
  double* E = D + (size_t)W * 32;
  if (k >= n) return;
  for (int i = 0; i < W; ++i) {
    D[i * 32] = b.d[(size_t)k * W + i];
    E[i * 32] = b.e[(size_t)k * W + i];
  }
  bool fail = false;
  // Each lane advances through its own eigenvalues: one pass of the loop either deflates the
  // current eigenvalue l (|e| small at m = l) or runs one QL sweep on its block l..m.  A lane is
  // never held at an eigenvalue by the other lanes of the warp, whose matrices need a
  // different number of sweeps for it (with the eigenvalue loop outermost, every lane would
  // wait at each l for the slowest lane's sweeps, about half of the warp's issued work).
  // The deflation test |e_m| <= eps (|d_m| + |d_m+1|) is taken in its slightly stricter form
  // |e_m| <= 2^-52 max(|d_m|, |d_m+1|) on the bit patterns (non-negative doubles order like
  // their bits, and adding 52 to the exponent field multiplies by 2^52), so that the scan,
  // about a sixth of the kernel's floating-point work, issues no FP64 instruction.
  int l = 0, iter = 0;
  while (l < W) {
    int m = l;
    for (; m < W - 1; ++m) {
      const long long e = __double_as_longlong(E[m * 32]) & 0x7FFFFFFFFFFFFFFFll;
      const long long a = __double_as_longlong(D[m * 32]) & 0x7FFFFFFFFFFFFFFFll;
      const long long c = __double_as_longlong(D[(m + 1) * 32]) & 0x7FFFFFFFFFFFFFFFll;
      if (e == 0 || e + (52ll << 52) <= (a > c ? a : c)) break;
    }
    if (m == l) {
      ++l;
      iter = 0;
      continue;
    }
    if (++iter > b.ql_cap) { fail = true; break; }
    // Wilkinson shift from the leading 2x2 of the block, then chase up from the bottom.
    double dl = D[l * 32], el = E[l * 32];
    double g = (D[(l + 1) * 32] - dl) / (2.0 * el);
    double r = hypot(g, 1.0);
    g = D[m * 32] - dl + el / (g + copysign(r, g));
    double s = 1.0, c = 1.0, p = 0.0;
    bool early = false;
    for (int i = m - 1; i >= l; --i) {
      double ei = E[i * 32];
      double f = s * ei, bb = c * ei;
      // r = |(f, g)| and (s, c) = (f, g) / r from one reciprocal square root (the entries of
      // T are far from the FP64 overflow/underflow range, so no scaling is needed)
      const double r2 = fma(f, f, g * g);
      if ((__double_as_longlong(r2) << 1) == 0) {   // r2 = +-0: the chase stops here (split)
        E[(i + 1) * 32] = 0.0;
        D[(i + 1) * 32] -= p;
        E[m * 32] = 0.0;
        early = true;
        break;
      }
      const double ir = rsqrt(r2);
      r = r2 * ir;
      E[(i + 1) * 32] = r;
      s = f * ir;
      c = g * ir;
      double gi = D[(i + 1) * 32] - p;
      double rr = fma(D[i * 32] - gi, s, 2.0 * c * bb);
      p = s * rr;
      D[(i + 1) * 32] = gi + p;
      g = fma(c, rr, -bb);
    }
    if (early) continue;
    D[l * 32] -= p;
    E[l * 32] = g;
    E[m * 32] = 0.0;
  }
  for (int i = 0; i < W; ++i) b.lam[(size_t)k * W + i] = D[i * 32];
  if (fail) atomicOr(&st->bits, ST_NO_CONVERGENCE);
}

// ------------------------------------------------------------------ K2c: eigenvectors + back-transform
// Eigenvectors of T by inverse iteration, then U = Q D Z.
//   * eigenvalues are sorted (rank by integer keys); clusters are runs of sorted eigenvalues
//     closer than 1e-3 ||T||_1; one thread handles one cluster (almost always one vector).
//   * for each eigenvalue: LU of T - lambda I with partial pivoting (row interchanges), 3
//     solves from a fixed pseudo-random start, modified Gram-Schmidt against the cluster's
//     previous vectors, normalisation.  Coincident eigenvalues are separated by 10 eps ||T||_1.
//   * a warp at a time: the factors of 32 vectors live lane-interleaved in the U region;
//     the iterate lives in its column of Z.
__device__ __forceinline__ unsigned long long order_key(double x) {
  unsigned long long u = (unsigned long long)__double_as_longlong(x);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// double2 slots of the U region: the W x (W+1) matrix, or the inverse-iteration factors of
// 32 vectors (4 arrays of W x 32 doubles)
__host__ __device__ __forceinline__ size_t bt_u_slots(int W) {
  const size_t mat = (size_t)W * (W + 1);
  const size_t lu = (size_t)64 * W;
  return mat > lu ? mat : lu;
}

constexpr int IIT_SOLVES = 3;

__global__ void __launch_bounds__(NT) backtransform_kernel(int W, EighBufs b, double* __restrict__ Eout,
                                                           double2* __restrict__ Uout, int pad) {
  extern __shared__ double2 smem2[];
  const int LDU = W + pad;   // pad = 1: conflict-free column walks; 0: the padding ablation
  double2* U = smem2;                               // [W][LDU] complex (LU scratch before)
  double* Z = (double*)(U + bt_u_slots(W));         // [W][LDU] eigenvectors of T (by sorted index)
  double* ws = Z + (size_t)W * LDU;                 // [W] sorted eigenvalues
  double* dd = ws + W;                              // [W] diagonal of T
  double* ee = dd + W;                              // [W] off-diagonal of T
  int* rank = (int*)(ee + W);                       // [W]
  int* newc = rank + W;                             // [W] 1 = starts a cluster
  __shared__ double s_onenrm;

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t k = blockIdx.x;
  const double* lk = b.lam + k * W;

  // ascending order of the eigenvalues (ties broken by index)
  for (int j = t; j < W; j += NT) {
    const double lj = lk[j];
    const unsigned long long kj = order_key(lj);
    int rnk = 0;
    for (int i = 0; i < W; ++i) {
      const unsigned long long ki = order_key(lk[i]);
      rnk += (ki < kj) || (ki == kj && i < j);
    }
    rank[j] = rnk;
    ws[rnk] = lj;
    Eout[k * W + rnk] = lj;
    dd[j] = b.d[k * W + j];
    ee[j] = b.e[k * W + j];
  }
  if (Uout == nullptr) return;
  __syncthreads();
  if (warp == 0) {   // ||T||_1
    double mx = 0.0;
    for (int i = lane; i < W; i += 32)
      mx = fmax(mx, fabs(dd[i]) + (i > 0 ? ee[i - 1] : 0.0) + (i < W - 1 ? ee[i] : 0.0));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) s_onenrm = mx > 0.0 ? mx : 1.0;
  }
  __syncthreads();
  const double onenrm = s_onenrm;
  const double ortol = 1e-3 * onenrm;
  const double eps = 2.220446049250313e-16;
  const double pertol = 10.0 * eps * onenrm;
  const double tiny = eps * onenrm;
  for (int j = t; j < W; j += NT) newc[j] = (j == 0) || (ws[j] - ws[j - 1] > ortol);
  __syncthreads();

  double* rU0 = (double*)U;                 // [W][32] reciprocal pivots
  double* U1 = rU0 + (size_t)W * 32;        // [W][32] first super-diagonal of U
  double* U2 = U1 + (size_t)W * 32;         // [W][32] second super-diagonal of U
  double* ML = U2 + (size_t)W * 32;         // [W][32] multipliers
  for (int p0 = 0; p0 < W; p0 += 32) {
    const int j = p0 + lane;
    if (warp == 0 && j < W && newc[j]) {
      double lprev = 0.0;
      for (int m = j; m < W && (m == j || !newc[m]); ++m) {
        double lam = ws[m];
        if (m > j && lam - lprev <= pertol) lam = lprev + pertol;
        lprev = lam;
        // ---- LU of T - lam I with row interchanges
        unsigned long long piv = 0ull;
        double q0 = dd[0] - lam, q1 = W > 1 ? ee[0] : 0.0, q2 = 0.0;
        for (int i = 0; i + 1 < W; ++i) {
          const double ei = ee[i];
          const double a = dd[i + 1] - lam;
          const double bb = i + 2 < W ? ee[i + 1] : 0.0;
          // the interchange only selects operands: one FP64 sequence for the whole warp
          const bool sw = mag_bits(q0) < mag_bits(ei);
          const double den = sw ? ei : (mag_bits(q0) == 0ull ? tiny : q0);
          const double r = 1.0 / den;
          const double mlt = (sw ? q0 : ei) * r;
          rU0[i * 32 + lane] = r; U1[i * 32 + lane] = sw ? a : q1; U2[i * 32 + lane] = sw ? bb : q2;
          ML[i * 32 + lane] = mlt;
          if (sw) piv |= 1ull << i;
          const double n0 = fma(-mlt, sw ? a : q1, sw ? q1 : a);
          q1 = fma(-mlt, sw ? bb : q2, sw ? q2 : bb);
          q0 = n0;
          q2 = 0.0;
        }
        if (mag_bits(q0) == 0ull) q0 = tiny;
        rU0[(W - 1) * 32 + lane] = 1.0 / q0;
        U1[(W - 1) * 32 + lane] = 0.0;   // the last row of U has no super-diagonals; the
        U2[(W - 1) * 32 + lane] = 0.0;   // back-substitution reads them (times zero)
        if (W >= 2) U2[(W - 2) * 32 + lane] = 0.0;
        // ---- inverse iteration in column m of Z
        for (int i = 0; i < W; ++i) Z[i * LDU + m] = iit_start_vec(i, m);
        for (int it = 0; it < IIT_SOLVES; ++it) {
          for (int i = 0; i + 1 < W; ++i) {
            const double mlt = ML[i * 32 + lane];
            const double yi = Z[i * LDU + m], yn = Z[(i + 1) * LDU + m];
            const bool sw = (piv >> i) & 1ull;
            if (sw) Z[i * LDU + m] = yn;
            Z[(i + 1) * LDU + m] = fma(-mlt, sw ? yn : yi, sw ? yi : yn);
          }
          double x1 = 0.0, x2 = 0.0;   // x_{i+1}, x_{i+2}
          for (int i = W - 1; i >= 0; --i) {
            const double xi = (Z[i * LDU + m] - U1[i * 32 + lane] * x1 - U2[i * 32 + lane] * x2) *
                              rU0[i * 32 + lane];
            Z[i * LDU + m] = xi;
            x2 = x1;
            x1 = xi;
          }
          // orthogonalise against the cluster's previous vectors (modified Gram-Schmidt)
          for (int q = j; q < m; ++q) {
            double c = 0.0;
            for (int i = 0; i < W; ++i) c = fma(Z[i * LDU + q], Z[i * LDU + m], c);
            for (int i = 0; i < W; ++i) Z[i * LDU + m] = fma(-c, Z[i * LDU + q], Z[i * LDU + m]);
          }
          if (it + 1 < IIT_SOLVES) {   // between solves: a power-of-two rescale (exact)
            pow2_rescale(Z + m, W, (size_t)LDU);
            continue;
          }
          double s0 = 0.0, s1 = 0.0;
          int i = 0;
          for (; i + 1 < W; i += 2) {
            const double u = Z[i * LDU + m], v = Z[(i + 1) * LDU + m];
            s0 = fma(u, u, s0);
            s1 = fma(v, v, s1);
          }
          if (i < W) { const double u = Z[i * LDU + m]; s0 = fma(u, u, s0); }
          const double inv = 1.0 / sqrt(s0 + s1);
          for (int i2 = 0; i2 < W; ++i2) Z[i2 * LDU + m] *= inv;
        }
      }
    }
    __syncthreads();
  }

  // U = D Z, columns in the original (unsorted) eigenvalue order of rank[]: column c of U holds
  // the vector of sorted index c (the output below writes U[:, c] to column c).
  const double2* ph = b.phase + k * W;
  for (int idx = t; idx < W * W; idx += NT) {
    int r = idx / W, c = idx % W;
    double z = Z[r * LDU + c];
    double2 p = ph[r];
    U[r * LDU + c] = make_double2(p.x * z, p.y * z);
  }
  __syncthreads();

  // stage the reflectors in Z's space: reflector j (length m = W-1-j) at offset roff(j)
  double2* Rs = (double2*)Z;
  const double2* R = b.refl + (size_t)k * W * W;
  auto roff = [&](int j) { return j * (W - 1) - (j * (j - 1)) / 2; };   // sum_{j'<j} (W-1-j')
  for (int idx = t; idx < W * W; idx += NT) {
    const int r = idx / W, c = idx % W;
    if (r > c && c < W - 2) Rs[roff(c) + (r - c - 1)] = R[idx];
  }
  __syncthreads();

  // U <- H_j U for j = W-3 .. 0; 4 threads per column, rows strided by 4
  const double* tau = b.tau + k * W;
  const int q = t & 3;
  for (int c0 = 0; c0 < W; c0 += NT / 4) {
    const int c = c0 + (t >> 2);
    const bool act = c < W;
    for (int j = W - 3; j >= 0; --j) {
      const double tj = tau[j];
      if (tj == 0.0) continue;
      const int o = j + 1, m = W - 1 - j;
      const double2* v_j = Rs + roff(j);
      double sx = 0.0, sy = 0.0;
      if (act) {
        for (int r = q; r < m; r += 4) {
          double2 v = v_j[r];
          double2 u = U[(o + r) * LDU + c];
          sx = fma(v.x, u.x, fma(v.y, u.y, sx));     // conj(v) u
          sy = fma(v.x, u.y, fma(-v.y, u.x, sy));
        }
      }
      sx += __shfl_xor_sync(0xffffffffu, sx, 1);
      sy += __shfl_xor_sync(0xffffffffu, sy, 1);
      sx += __shfl_xor_sync(0xffffffffu, sx, 2);
      sy += __shfl_xor_sync(0xffffffffu, sy, 2);
      sx *= tj; sy *= tj;
      if (act) {
        for (int r = q; r < m; r += 4) {
          double2 v = v_j[r];
          double2 u = U[(o + r) * LDU + c];
          u.x = fma(-sx, v.x, fma(sy, v.y, u.x));    // u -= s v
          u.y = fma(-sx, v.y, fma(-sy, v.x, u.y));
          U[(o + r) * LDU + c] = u;
        }
      }
      __syncwarp();
    }
  }
  __syncthreads();
  double2* Uk = Uout + (size_t)k * W * W;
  for (int idx = t; idx < W * W; idx += NT) Uk[idx] = U[(idx / W) * LDU + idx % W];
}

}  // namespace

size_t tridiag_smem(int W) {
  // packed triangle + the symv partials (at least 2 W: p and the copy of v)
  return ((size_t)W * (W + 1) / 2 + std::max(TRI_NT, 2 * W)) * sizeof(double2);
}
size_t backtransform_smem(int W) {
  return bt_u_slots(W) * sizeof(double2) + (size_t)W * (W + 1) * sizeof(double) +
         (size_t)3 * W * sizeof(double) + (size_t)2 * W * sizeof(int);
}
// threads per QL block: one warp (d and e of a warp take 2 W 32 doubles of shared memory, so
// single-warp blocks pack the most warps onto an SM: 7 at W = 64)
static int ql_threads(int W) { (void)W; return 32; }
size_t ql_smem(int W) { return (size_t)(ql_threads(W) / 32) * 2 * W * 32 * sizeof(double); }

static cudaError_t launch_tridiag_ld(const double* Hp, int64_t ld, int W, int n, EighBufs b,
                                     cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const size_t sm = tridiag_smem(W);
  auto go = [&](auto kern, int nt) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    kern<<<n, nt, sm, s>>>(Hp, ld, W, b);
    return cudaGetLastError();
  };
  if (W <= 64) {
    // two k-points per 512-thread CTA
    const size_t sm2 = 2 * ((size_t)W * (W + 1) / 2 + 256) * sizeof(double2);
    cudaError_t e = cudaFuncSetAttribute(tridiag2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm2);
    if (e != cudaSuccess) return e;
    tridiag2_kernel<<<(n + 1) / 2, 512, sm2, s>>>(Hp, ld, W, n, b);
    return cudaGetLastError();
  }
  return go(tridiag_kernel<double, TRI_NT>, TRI_NT);
}

cudaError_t launch_tridiag(const double* Hp, int W, int n, EighBufs b, cudaStream_t s) {
  return launch_tridiag_ld(Hp, (int64_t)W * W, W, n, b, s);
}

cudaError_t launch_tridiag_rows(const double* Hp, int64_t ld, int W, int n, EighBufs b,
                                cudaStream_t s) {
  return launch_tridiag_ld(Hp, ld, W, n, b, s);
}

cudaError_t launch_ql(int W, int n, EighBufs b, DevStatus* st, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  size_t sm = ql_smem(W);
  cudaError_t e = cudaFuncSetAttribute(ql_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int nt = ql_threads(W);
  ql_kernel<<<(n + nt - 1) / nt, nt, sm, s>>>(W, n, b, st);
  return cudaGetLastError();
}

cudaError_t launch_backtransform(int W, int n, EighBufs b, double* E, double2* U, cudaStream_t s,
                                 int pad) {
  if (n <= 0) return cudaSuccess;
  size_t sm = backtransform_smem(W);
  cudaError_t e = cudaFuncSetAttribute(backtransform_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  backtransform_kernel<<<n, NT, sm, s>>>(W, b, E, U, pad ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace kubo
