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
//                    implicit QL with Wilkinson shifts on the real tridiagonal T.  The
//                    rotation recurrence is inherently scalar, so 32 k-points share each
//                    warp instruction.  Every Givens rotation (c, s, i) is logged.
//   backtransform_kernel  one CTA per k-point: replays the logged rotations on Z (T = Z L
//                    Z^T; rows in parallel), sorts the eigenvalues, and forms
//                    U = Q D Z by applying the reflectors to the columns of D Z.
//
// Padded leading dimensions (W+1) keep column walks conflict-free in shared memory (the
// GPU counterpart of the paper's padding against memory-bank conflicts).
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
template <typename T>
__global__ void __launch_bounds__(NT, 5) tridiag_kernel(const T* __restrict__ Hp, int64_t ld, int W,
                                                     EighBufs b) {
  extern __shared__ double2 smem2[];
  double2* A = smem2;                              // lower triangle, packed by rows
  double2* vb = A + (size_t)W * (W + 1) / 2;       // [W] reflector (contiguous copy)
  double2* pb = vb + W;                            // [W] p, then w
  double2* be = pb + W;                            // [W] complex sub-diagonal beta_i
  double* tb = (double*)(be + W);                  // [W] tau_i
  __shared__ double s_tau, s_K;

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t k = blockIdx.x;
  const T* P = Hp + (size_t)k * ld;

  for (int idx = t; idx < W * (W + 1) / 2; idx += NT) {
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
      if (lane == 0) {
        double2 al = A[tri(o, i)];
        double tau = 0.0;
        double2 beta = al;
        if (s2 != 0.0) {
          // H = I - tau v v^H with v = x - beta e1, beta = -e^{i arg alpha} |x|:
          // v0 = alpha + e^{i arg alpha} |x|, tau = 2 / v^H v = 1 / (|x| (|x| + |alpha|))
          const double aa2 = fma(al.x, al.x, al.y * al.y);
          const double aa = sqrt(aa2);
          const double nrm = sqrt(aa2 + s2);
          double pr = 1.0, pi = 0.0;
          if (aa > 0.0) { const double ia = 1.0 / aa; pr = al.x * ia; pi = al.y * ia; }
          beta = make_double2(-pr * nrm, -pi * nrm);
          A[tri(o, i)] = make_double2(fma(pr, nrm, al.x), fma(pi, nrm, al.y));
          tau = 1.0 / (nrm * (nrm + aa));
        }
        s_tau = tau;
        be[i] = beta;
        tb[i] = tau;
      }
    }
    __syncthreads();
    const double tau = s_tau;
    if (tau != 0.0) {
      for (int r = t; r < m; r += NT) vb[r] = A[tri(o + r, i)];
      __syncthreads();
      // p = tau * A22 v  (lower storage: A22[r][c] = conj(A22[c][r]) for c > r)
      for (int r = t; r < m; r += NT) {
        double ax = 0.0, ay = 0.0, bx = 0.0, by = 0.0;
        const int rowb = tri(o + r, o);
        int c = 0;
        for (; c + 1 < m; c += 2) {
          const int i0 = c <= r ? rowb + c : tri(o + c, o + r);
          const int i1 = c + 1 <= r ? rowb + c + 1 : tri(o + c + 1, o + r);
          double2 a0 = A[i0], a1 = A[i1];
          if (c > r) a0.y = -a0.y;
          if (c + 1 > r) a1.y = -a1.y;
          const double2 v0 = vb[c], v1 = vb[c + 1];
          ax = fma(a0.x, v0.x, ax); ax = fma(-a0.y, v0.y, ax);
          ay = fma(a0.x, v0.y, ay); ay = fma(a0.y, v0.x, ay);
          bx = fma(a1.x, v1.x, bx); bx = fma(-a1.y, v1.y, bx);
          by = fma(a1.x, v1.y, by); by = fma(a1.y, v1.x, by);
        }
        if (c < m) {
          const int i0 = c <= r ? rowb + c : tri(o + c, o + r);
          double2 a0 = A[i0];
          if (c > r) a0.y = -a0.y;
          const double2 v0 = vb[c];
          ax = fma(a0.x, v0.x, ax); ax = fma(-a0.y, v0.y, ax);
          ay = fma(a0.x, v0.y, ay); ay = fma(a0.y, v0.x, ay);
        }
        pb[r] = make_double2(tau * (ax + bx), tau * (ay + by));
      }
      __syncthreads();
      if (warp == 0) {
        double sum = 0.0;   // Re(v^H p)
        for (int r = lane; r < m; r += 32) {
          const double2 v = vb[r], p = pb[r];
          sum = fma(v.x, p.x, fma(v.y, p.y, sum));
        }
        sum = warp_sum(sum);
        if (lane == 0) s_K = 0.5 * tau * sum;
      }
      __syncthreads();
      const double K = s_K;
      for (int r = t; r < m; r += NT) {
        const double2 p = pb[r], v = vb[r];
        pb[r] = make_double2(fma(-K, v.x, p.x), fma(-K, v.y, p.y));
      }
      __syncthreads();
      // A22 <- A22 - v w^H - w v^H on the lower triangle (c <= r)
      const int ntri = m * (m + 1) / 2;
      for (int idx = t; idx < ntri; idx += NT) {
        int r = (int)((sqrtf(8.0f * (float)idx + 1.0f) - 1.0f) * 0.5f);
        while (r * (r + 1) / 2 > idx) --r;
        while ((r + 1) * (r + 2) / 2 <= idx) ++r;
        const int c = idx - r * (r + 1) / 2;
        const double2 vr = vb[r], wr = pb[r], vc = vb[c], wc = pb[c];
        double2 a = A[tri(o + r, o + c)];
        // v_r conj(w_c) + w_r conj(v_c)
        a.x = fma(-vr.x, wc.x, a.x); a.x = fma(-vr.y, wc.y, a.x);
        a.x = fma(-wr.x, vc.x, a.x); a.x = fma(-wr.y, vc.y, a.x);
        if (c == r) {
          a.y = 0.0;
        } else {
          a.y = fma(-vr.y, wc.x, a.y); a.y = fma(vr.x, wc.y, a.y);
          a.y = fma(-wr.y, vc.x, a.y); a.y = fma(wr.x, vc.y, a.y);
        }
        A[tri(o + r, o + c)] = a;
      }
    }
    __syncthreads();
  }

  // outputs: d, |e|, phases D, tau, reflectors
  double* dout = b.d + k * W;
  double* eout = b.e + k * W;
  double2* phout = b.phase + k * W;
  double* tout = b.tau + k * W;
  if (t == 0) {
    if (W >= 2) be[W - 2] = A[tri(W - 1, W - 2)];
    double2 D = make_double2(1.0, 0.0);
    phout[0] = D;
    for (int j = 0; j + 1 < W; ++j) {
      double2 bj = be[j];
      double a = hypot(bj.x, bj.y);
      eout[j] = a;
      if (a > 0.0) D = cmul(D, make_double2(bj.x / a, bj.y / a));
      phout[j + 1] = D;
    }
    eout[W - 1] = 0.0;
  }
  for (int j = t; j < W; j += NT) {
    dout[j] = A[tri(j, j)].x;
    tout[j] = j < W - 2 ? tb[j] : 0.0;
  }
  double2* rout = b.refl + (size_t)k * W * W;
  for (int idx = t; idx < W * W; idx += NT) {
    int r = idx / W, c = idx % W;
    rout[idx] = r > c ? A[tri(r, c)] : make_double2(0.0, 0.0);
  }
}

// ------------------------------------------------------------------ K2b: QL, lane per k
// Smem per warp: d and e as [W][32] (lane-interleaved: conflict-free for any index mix).
__global__ void __launch_bounds__(64) ql_kernel(int W, int n, EighBufs b, DevStatus* st) {
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
  const int cap = b.cap;
  double2* rot = b.rot + (size_t)k * cap;
  short* rc = b.rcol + (size_t)k * cap;
  int nrot = 0;
  bool fail = false;
  const double eps = 2.220446049250313e-16;
  for (int l = 0; l < W && !fail; ++l) {
    int iter = 0;
    while (true) {
      int m = l;
      for (; m < W - 1; ++m) {
        double dd = fabs(D[m * 32]) + fabs(D[(m + 1) * 32]);
        if (fabs(E[m * 32]) <= eps * dd) break;
      }
      if (m == l) break;
      if (++iter > 60) { fail = true; break; }
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
        r = hypot(f, g);
        E[(i + 1) * 32] = r;
        if (r == 0.0) {   // split: the chase stops here
          D[(i + 1) * 32] -= p;
          E[m * 32] = 0.0;
          early = true;
          break;
        }
        s = f / r;
        c = g / r;
        double gi = D[(i + 1) * 32] - p;
        double rr = fma(D[i * 32] - gi, s, 2.0 * c * bb);
        p = s * rr;
        D[(i + 1) * 32] = gi + p;
        g = fma(c, rr, -bb);
        if (nrot < cap) { rot[nrot] = make_double2(c, s); rc[nrot] = (short)i; }
        ++nrot;
      }
      if (early) continue;
      D[l * 32] -= p;
      E[l * 32] = g;
      E[m * 32] = 0.0;
    }
  }
  for (int i = 0; i < W; ++i) b.d[(size_t)k * W + i] = D[i * 32];
  b.nrot[k] = nrot;
  if (fail) atomicOr(&st->bits, ST_NO_CONVERGENCE);
  if (nrot > cap) atomicOr(&st->bits, ST_LOG_OVERFLOW);
}

// ------------------------------------------------------------------ K2c: replay + back-transform
__device__ __forceinline__ unsigned long long order_key(double x) {
  unsigned long long u = (unsigned long long)__double_as_longlong(x);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// Log chunk staged in shared memory while the rows replay the previous one
constexpr int LOG_CHUNK = 1024;

// double2 slots of the U region: the W x (W+1) matrix, or two log chunks ((c, s) + indices)
__host__ __device__ __forceinline__ size_t bt_u_slots(int W) {
  const size_t mat = (size_t)W * (W + 1);
  const size_t logs = 2 * LOG_CHUNK + (2 * LOG_CHUNK * sizeof(short) + 15) / 16;
  return mat > logs ? mat : logs;
}

__global__ void __launch_bounds__(NT) backtransform_kernel(int W, EighBufs b, double* __restrict__ Eout,
                                                           double2* __restrict__ Uout) {
  extern __shared__ double2 smem2[];
  const int LDU = W + 1;
  double2* U = smem2;                               // [W][LDU] complex
  double* Z = (double*)(U + bt_u_slots(W));         // [W][LDU] real
  int* rank = (int*)(Z + (size_t)W * LDU);          // [W]
  // during the replay U's space holds two log chunks: (c, s) pairs, then column indices
  double2* logcs = U;                               // [2][LOG_CHUNK]
  short* logi = (short*)(U + 2 * LOG_CHUNK);        // [2][LOG_CHUNK]
  // after U = D Z, Z's space holds the reflectors: column j (rows j+1..W-1) at tri(W-2-j) offsets
  double2* Rs = (double2*)Z;

  const int t = threadIdx.x;
  const int64_t k = blockIdx.x;
  const double* dk = b.d + k * W;

  // ascending order of the eigenvalues (ties broken by index)
  for (int j = t; j < W; j += NT) {
    unsigned long long kj = order_key(dk[j]);
    int rnk = 0;
    for (int i = 0; i < W; ++i) {
      unsigned long long ki = order_key(dk[i]);
      rnk += (ki < kj) || (ki == kj && i < j);
    }
    rank[j] = rnk;
    Eout[k * W + rnk] = dk[j];
  }
  if (Uout == nullptr) return;

  for (int idx = t; idx < W * W; idx += NT) {
    int r = idx / W, c = idx % W;
    Z[r * LDU + c] = r == c ? 1.0 : 0.0;
  }

  // Replay the QL rotations: row r of Z is owned by thread r (< W); the other threads stage the
  // next chunk of the log.  Rotation i acts on columns (i, i+1); within a sweep the indices
  // descend, so column i of one rotation is column i+1 of the next and is carried in a
  // register (`cur`, column `ci`): two dependent FP64 operations per rotation.
  const int nr = min(b.nrot[k], b.cap);
  const double2* rot = b.rot + k * b.cap;
  const short* rc = b.rcol + k * b.cap;
  const int nchunk = (nr + LOG_CHUNK - 1) / LOG_CHUNK;
  for (int q = t; q < min(nr, LOG_CHUNK); q += NT) {
    logcs[q] = rot[q];
    logi[q] = rc[q];
  }
  __syncthreads();
  double cur = 0.0;
  int ci = -2;   // no carried column
  double* zr = Z + (t < W ? t : 0) * LDU;
  for (int ch = 0; ch < nchunk; ++ch) {
    const int buf = ch & 1;
    const int q0 = ch * LOG_CHUNK;
    const int qn = min(LOG_CHUNK, nr - q0);
    if (t < W) {
      const double2* cs_b = logcs + buf * LOG_CHUNK;
      const short* i_b = logi + buf * LOG_CHUNK;
      for (int q = 0; q < qn; ++q) {
        const double2 cs = cs_b[q];
        const int i = i_b[q];
        double f;                  // column i+1
        if (ci == i + 1) {
          f = cur;
        } else {
          if (ci >= 0) zr[ci] = cur;
          f = zr[i + 1];
        }
        const double zi = zr[i];
        zr[i + 1] = fma(cs.y, zi, cs.x * f);
        cur = fma(cs.x, zi, -cs.y * f);
        ci = i;
      }
    } else if (ch + 1 < nchunk) {
      const int nb = buf ^ 1;
      const int q1 = q0 + LOG_CHUNK;
      const int qn1 = min(LOG_CHUNK, nr - q1);
      for (int q = t - W; q < qn1; q += NT - W) {
        logcs[nb * LOG_CHUNK + q] = rot[q1 + q];
        logi[nb * LOG_CHUNK + q] = rc[q1 + q];
      }
    }
    __syncthreads();
  }
  if (t < W && ci >= 0) zr[ci] = cur;
  __syncthreads();

  // U = D Z (overwrites the log buffers)
  const double2* ph = b.phase + k * W;
  for (int idx = t; idx < W * W; idx += NT) {
    int r = idx / W, c = idx % W;
    double z = Z[r * LDU + c];
    double2 p = ph[r];
    U[r * LDU + c] = make_double2(p.x * z, p.y * z);
  }
  __syncthreads();

  // stage the reflectors in Z's space: reflector j (length m = W-1-j) at offset roff(j)
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
  for (int idx = t; idx < W * W; idx += NT) {
    int r = idx / W, c = idx % W;
    Uk[r * W + rank[c]] = U[r * LDU + c];
  }
}

}  // namespace

size_t tridiag_smem(int W) {
  return ((size_t)W * (W + 1) / 2 + 3 * (size_t)W) * sizeof(double2) + (size_t)W * sizeof(double);
}
size_t backtransform_smem(int W) {
  return bt_u_slots(W) * sizeof(double2) + (size_t)W * (W + 1) * sizeof(double) +
         (size_t)W * sizeof(int);
}
size_t ql_smem(int W) { return (size_t)2 * 2 * W * 32 * sizeof(double); }

cudaError_t launch_tridiag(const double* Hp, int W, int n, EighBufs b, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  size_t sm = tridiag_smem(W);
  cudaError_t e = cudaFuncSetAttribute(tridiag_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  tridiag_kernel<double><<<n, NT, sm, s>>>(Hp, (int64_t)W * W, W, b);
  return cudaGetLastError();
}

cudaError_t launch_tridiag_rows(const double* Hp, int64_t ld, int W, int n, EighBufs b,
                                cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  size_t sm = tridiag_smem(W);
  cudaError_t e = cudaFuncSetAttribute(tridiag_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  tridiag_kernel<double><<<n, NT, sm, s>>>(Hp, ld, W, b);
  return cudaGetLastError();
}

cudaError_t launch_ql(int W, int n, EighBufs b, DevStatus* st, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  size_t sm = ql_smem(W);
  cudaError_t e = cudaFuncSetAttribute(ql_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  ql_kernel<<<(n + 63) / 64, 64, sm, s>>>(W, n, b, st);
  return cudaGetLastError();
}

cudaError_t launch_backtransform(int W, int n, EighBufs b, double* E, double2* U, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  size_t sm = backtransform_smem(W);
  cudaError_t e = cudaFuncSetAttribute(backtransform_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  backtransform_kernel<<<n, NT, sm, s>>>(W, b, E, U);
  return cudaGetLastError();
}

}  // namespace kubo
