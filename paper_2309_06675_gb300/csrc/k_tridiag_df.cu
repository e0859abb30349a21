// Step (2), first half, for the MIXED mode: the Householder tridiagonalisation H = Q T_c Q^dagger
// of the FP64 eigensolver with its O(W^3) part in double-float arithmetic.
//
// On GB300 a warp FP64 instruction holds the SM's FP64 pipe for 16 cycles, 64 times the cost
// of an FP32 one, and the FP64 reduction is bound by that pipe.  Here every element of the
// packed lower triangle, the reflector v, p = tau A v and w are unevaluated pairs (hi, lo) of
// FP32 numbers with hi + lo the value and |lo| <= ulp(hi) / 2: products by FMA-exact
// TwoProd, sums by Knuth's TwoSum, so each operation keeps about 46 bits (relative error
// ~2^-46, against 2^-53 for FP64).  The symv and the rank-2 update (16/3 W^3 of the
// reduction's flops) run on the FP32 pipe; the scalar Householder step of each column
// (norm, square roots, tau) and the outputs stay FP64.  The reduction's backward error is
// then ~W 2^-46 ||H|| (1e-12 ||H|| at W = 64): the eigenvalues move by that much, four orders
// below what the FP32 rotations and eta ~ 1e-3 of the MIXED mode resolve.  Same algorithm,
// same outputs (FP64 d, |e|, phases, tau, reflectors) as the FP64 kernel in k_eigh.cu.
#include "kubo_internal.cuh"

namespace kubo {

namespace {

constexpr int NT = 256;

__device__ __forceinline__ int tri(int r, int c) { return (r * (r + 1) >> 1) + c; }

// exact s + e = a + b (Knuth's TwoSum; no ordering of |a|, |b| needed)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float ap = __fsub_rn(s, bp);
  e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

// (h, l) normalised from s + e with |s| >= |e| (Dekker's Fast2Sum)
__device__ __forceinline__ void fast_two_sum(float s, float e, float& h, float& l) {
  h = __fadd_rn(s, e);
  l = __fsub_rn(e, __fsub_rn(h, s));
}

// accumulator (sh, sl) += (xh + xl)(yh + yl); sl stays unnormalised until the end.  The
// dropped xl yl is below 2^-48 of the product.
__device__ __forceinline__ void df_mac(float& sh, float& sl, float xh, float xl, float yh,
                                       float yl) {
  const float p = __fmul_rn(xh, yh);
  float q = fmaf(xh, yh, -p);   // the rounding error of p, exactly
  q = fmaf(xh, yl, q);
  q = fmaf(xl, yh, q);
  float s, e;
  two_sum(sh, p, s, e);
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(e, q));
}

__device__ __forceinline__ void df_norm(float& h, float& l) { fast_two_sum(h, l, h, l); }

__device__ __forceinline__ float2 df_split(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}

// The conversions between FP64 and FP32 pairs run on the FP64 pipe; for the bulk input and
// output they are done on the bit patterns instead (integer pipe), with the FP64 conversion
// only for exponents outside a safe range (zero included on the input side).
// x = hi + lo with hi = x truncated to 24 significant bits and lo the remaining 29 bits
// rounded to FP32 (|x - hi - lo| <= 2^-48 |x|).
__device__ __forceinline__ float2 df_split_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex < 1023 - 70 || ex > 1023 + 70) return df_split(x);
  const uint32_t sgn = (uint32_t)(b >> 63) << 31;
  const uint32_t hb = sgn | ((uint32_t)(ex - 1023 + 127) << 23) | (uint32_t)((b >> 29) & 0x7FFFFFu);
  // the low 29 bits are worth low29 2^(ex - 1075); 2^(ex - 1075) = 2^(ex - 1023 - 52) is a
  // normal FP32 for the exponents admitted above
  const float scale = __uint_as_float((uint32_t)(ex - 1023 - 52 + 127) << 23);
  const float lo = __uint2float_rn((uint32_t)(b & 0x1FFFFFFFu)) * scale;
  return make_float2(__uint_as_float(hb), sgn ? -lo : lo);
}

// exact FP32 -> FP64 widening on the bit pattern (zero exactly; subnormals, inf and NaN by
// the FP64 conversion)
__device__ __forceinline__ double widen_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t ex = (u >> 23) & 0xFFu;
  if ((u & 0x7FFFFFFFu) == 0) return __longlong_as_double((long long)((unsigned long long)u << 32));
  if (ex == 0 || ex == 0xFFu) return (double)f;
  return __longlong_as_double((long long)(((unsigned long long)(u >> 31) << 63) |
                                          ((unsigned long long)(ex + 896) << 52) |
                                          ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}
__device__ __forceinline__ double df_val(float h, float l) { return widen_bits(h) + widen_bits(l); }

// complex element as float4 (re_h, re_l, im_h, im_l)
__device__ __forceinline__ float4 cdf_split(double re, double im) {
  const float2 a = df_split_bits(re), b = df_split_bits(im);
  return make_float4(a.x, a.y, b.x, b.y);
}

// a += x * y (complex double-float; conjugate x when CX)
template <bool CX>
__device__ __forceinline__ void cdf_mac(float4& a, const float4& x, const float4& y) {
  // re += x.re y.re -/+ x.im y.im ; im += x.re y.im +/- x.im y.re
  df_mac(a.x, a.y, x.x, x.y, y.x, y.y);
  if (CX) df_mac(a.x, a.y, x.z, x.w, y.z, y.w);
  else df_mac(a.x, a.y, -x.z, -x.w, y.z, y.w);
  df_mac(a.z, a.w, x.x, x.y, y.z, y.w);
  if (CX) df_mac(a.z, a.w, -x.z, -x.w, y.x, y.y);
  else df_mac(a.z, a.w, x.z, x.w, y.x, y.y);
}

__device__ __forceinline__ float4 cdf_norm(float4 a) {
  df_norm(a.x, a.y);
  df_norm(a.z, a.w);
  return a;
}

// double-float warp sum: exact TwoSum of the high parts, low parts added
__device__ __forceinline__ void warp_sum_df(float& h, float& l) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o);
    const float ol = __shfl_xor_sync(0xffffffffu, l, o);
    float s, e;
    two_sum(h, oh, s, e);
    h = s;
    l = __fadd_rn(l, __fadd_rn(ol, e));
  }
}

// Packed rows of leading dimension ld (the [H | dxH | dyH] rows of the tensor-core Fourier
// sum).  Shared memory: the lower triangle packed by rows (element (r, c <= r) at
// r (r + 1) / 2 + c) as complex double-float, then v, p / w, the symv partials.
__global__ void __launch_bounds__(NT, 5) tridiag_df_kernel(const double* __restrict__ Hp,
                                                           int64_t ld, int W, EighBufs b) {
  extern __shared__ float4 sm4[];
  float4* A = sm4;                                  // W (W + 1) / 2
  float4* vb = A + (size_t)W * (W + 1) / 2;         // [W] reflector
  float4* pb = vb + W;                              // [W] p, then w
  float4* sp = pb + W;                              // [NT] symv partial sums
  double2* be = reinterpret_cast<double2*>(sp + NT);   // [W] complex sub-diagonal beta_i
  double* tb = reinterpret_cast<double*>(be + W);      // [W] tau_i
  __shared__ float2 s_tdf, s_Kdf;   // tau and K as FP32 pairs
  __shared__ int s_act;             // tau != 0

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t k = blockIdx.x;
  const double* P = Hp + (size_t)k * ld;

  for (int idx = t; idx < W * (W + 1) / 2; idx += NT) {
    int r = (int)((sqrtf(8.0f * (float)idx + 1.0f) - 1.0f) * 0.5f);
    while (tri(r, 0) > idx) --r;
    while (tri(r + 1, 0) <= idx) ++r;
    const int c = idx - tri(r, 0);
    A[idx] = r == c ? cdf_split(P[r * W + r], 0.0)
                    : cdf_split(P[c * W + r], -P[r * W + c]);   // conj(A_cr)
  }
  __syncthreads();

  for (int i = 0; i < W - 2; ++i) {
    const int o = i + 1;       // first row of the trailing block
    const int m = W - 1 - i;   // its size
    if (warp == 0) {
      float sh = 0.f, sl = 0.f;   // |x|^2 below the sub-diagonal
      for (int r = o + 1 + lane; r < W; r += 32) {
        const float4 x = A[tri(r, i)];
        df_mac(sh, sl, x.x, x.y, x.x, x.y);
        df_mac(sh, sl, x.z, x.w, x.z, x.w);
      }
      warp_sum_df(sh, sl);
      if (lane == 0) {
        const double s2 = df_val(sh, sl);
        const float4 a4 = A[tri(o, i)];
        const double alx = df_val(a4.x, a4.y), aly = df_val(a4.z, a4.w);
        double tau = 0.0;
        double2 beta = make_double2(alx, aly);
        if (s2 > 0.0) {
          // H = I - tau v v^H, v = x - beta e1, beta = -e^{i arg alpha} |x|,
          // v0 = alpha + e^{i arg alpha} |x|, tau = 1 / (|x| (|x| + |alpha|))
          const double aa2 = fma(alx, alx, aly * aly);
          const double n2 = aa2 + s2;
          const double nrm = n2 * rsqrt(n2);
          double pr = 1.0, pi = 0.0, aa = 0.0;
          if (aa2 > 0.0) {
            const double ra = rsqrt(aa2);
            aa = aa2 * ra;
            pr = alx * ra;
            pi = aly * ra;
          }
          beta = make_double2(-pr * nrm, -pi * nrm);
          A[tri(o, i)] = cdf_split(fma(pr, nrm, alx), fma(pi, nrm, aly));
          tau = 1.0 / (nrm * (nrm + aa));
        }
        s_tdf = df_split(tau);
        s_act = tau != 0.0;
        be[i] = beta;
        tb[i] = tau;
      }
    }
    __syncthreads();
    if (s_act) {
      for (int r = t; r < m; r += NT) vb[r] = A[tri(o + r, i)];
      __syncthreads();
      // p = tau A22 v, spread densely: thread t takes row r = t mod m and the columns
      // c = part, part + P, ... (part = t / m, P = NT / m); the P partials of a row are added
      // in part order.  Mirrored elements (c > r) are conjugated by flipping the sign bits of
      // both imaginary halves.
      {
        const int Pp = NT / m;
        const int r = t % m, part = t / m;
        if (part < Pp) {
          float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
          const int rowb = tri(o + r, o);
          for (int c = part; c < m; c += Pp) {
            const bool up = c > r;
            float4 a = A[up ? tri(o + c, o + r) : rowb + c];
            if (up) {
              a.z = -a.z;
              a.w = -a.w;
            }
            cdf_mac<false>(acc, a, vb[c]);
          }
          sp[part * m + r] = acc;
        }
        __syncthreads();
        const float2 tdf = s_tdf;
        for (int rr = t; rr < m; rr += NT) {
          float4 s = sp[rr];
          for (int q = 1; q < Pp; ++q) {
            const float4 v = sp[q * m + rr];
            float e;
            two_sum(s.x, v.x, s.x, e);
            s.y = __fadd_rn(s.y, __fadd_rn(v.y, e));
            two_sum(s.z, v.z, s.z, e);
            s.w = __fadd_rn(s.w, __fadd_rn(v.w, e));
          }
          s = cdf_norm(s);
          float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
          df_mac(p.x, p.y, tdf.x, tdf.y, s.x, s.y);
          df_mac(p.z, p.w, tdf.x, tdf.y, s.z, s.w);
          pb[rr] = cdf_norm(p);
        }
      }
      __syncthreads();
      if (warp == 0) {
        float sh = 0.f, sl = 0.f;   // Re(v^H p)
        for (int r = lane; r < m; r += 32) {
          const float4 v = vb[r], p = pb[r];
          df_mac(sh, sl, v.x, v.y, p.x, p.y);
          df_mac(sh, sl, v.z, v.w, p.z, p.w);
        }
        warp_sum_df(sh, sl);
        if (lane == 0) s_Kdf = df_split(0.5 * df_val(s_tdf.x, s_tdf.y) * df_val(sh, sl));
      }
      __syncthreads();
      {
        const float2 K = s_Kdf;
        for (int r = t; r < m; r += NT) {
          float4 p = pb[r];
          const float4 v = vb[r];
          df_mac(p.x, p.y, -K.x, -K.y, v.x, v.y);
          df_mac(p.z, p.w, -K.x, -K.y, v.z, v.w);
          pb[r] = cdf_norm(p);
        }
      }
      __syncthreads();
      // A22 <- A22 - v w^H - w v^H on the lower triangle (c <= r)
      const int ntri = m * (m + 1) / 2;
      for (int idx = t; idx < ntri; idx += NT) {
        int r = (int)((sqrtf(8.0f * (float)idx + 1.0f) - 1.0f) * 0.5f);
        while (r * (r + 1) / 2 > idx) --r;
        while ((r + 1) * (r + 2) / 2 <= idx) ++r;
        const int c = idx - r * (r + 1) / 2;
        const float4 vr = vb[r], wr = pb[r], vc = vb[c], wc = pb[c];
        float4 a = A[tri(o + r, o + c)];
        // re -= vr.re wc.re + vr.im wc.im + wr.re vc.re + wr.im vc.im
        df_mac(a.x, a.y, -vr.x, -vr.y, wc.x, wc.y);
        df_mac(a.x, a.y, -vr.z, -vr.w, wc.z, wc.w);
        df_mac(a.x, a.y, -wr.x, -wr.y, vc.x, vc.y);
        df_mac(a.x, a.y, -wr.z, -wr.w, vc.z, vc.w);
        df_norm(a.x, a.y);
        if (c == r) {
          a.z = 0.f;
          a.w = 0.f;
        } else {
          // im -= vr.im wc.re - vr.re wc.im + wr.im vc.re - wr.re vc.im
          df_mac(a.z, a.w, -vr.z, -vr.w, wc.x, wc.y);
          df_mac(a.z, a.w, vr.x, vr.y, wc.z, wc.w);
          df_mac(a.z, a.w, -wr.z, -wr.w, vc.x, vc.y);
          df_mac(a.z, a.w, wr.x, wr.y, vc.z, vc.w);
          df_norm(a.z, a.w);
        }
        A[tri(o + r, o + c)] = a;
      }
    }
    __syncthreads();
  }

  // outputs (FP64): d, |e|, phases D, tau, reflectors
  double* dout = b.d + k * W;
  double* eout = b.e + k * W;
  double2* phout = b.phase + k * W;
  double* tout = b.tau + k * W;
  if (t == 0 && W >= 2) {
    const float4 a = A[tri(W - 1, W - 2)];
    be[W - 2] = make_double2(df_val(a.x, a.y), df_val(a.z, a.w));
  }
  __syncthreads();
  double2* ub = reinterpret_cast<double2*>(vb);   // unit phases (vb / pb no longer needed)
  for (int j = t; j + 1 < W; j += NT) {
    const double2 bj = be[j];
    const double a2 = fma(bj.x, bj.x, bj.y * bj.y);
    double a = 0.0;
    double2 u = make_double2(1.0, 0.0);
    if (a2 > 0.0) {
      const double ra = rsqrt(a2);
      a = a2 * ra;
      u = make_double2(bj.x * ra, bj.y * ra);
    }
    eout[j] = a;
    ub[j] = u;
  }
  __syncthreads();
  if (t == 0) {
    double2 D = make_double2(1.0, 0.0);
    phout[0] = D;
    for (int j = 0; j + 1 < W; ++j) {
      D = cmul(D, ub[j]);
      phout[j + 1] = D;
    }
    eout[W - 1] = 0.0;
  }
  for (int j = t; j < W; j += NT) {
    const float4 a = A[tri(j, j)];
    dout[j] = df_val(a.x, a.y);
    tout[j] = j < W - 2 ? tb[j] : 0.0;
  }
  double2* rout = b.refl + (size_t)k * W * W;
  for (int idx = t; idx < W * W; idx += NT) {
    const int r = idx / W, c = idx % W;
    double2 v = make_double2(0.0, 0.0);
    if (r > c) {
      const float4 a = A[tri(r, c)];
      v = make_double2(df_val(a.x, a.y), df_val(a.z, a.w));
    }
    rout[idx] = v;
  }
}

}  // namespace

size_t tridiag_df_smem(int W) {
  return ((size_t)W * (W + 1) / 2 + 2 * (size_t)W + NT) * sizeof(float4) +
         (size_t)W * (sizeof(double2) + sizeof(double));
}

cudaError_t launch_tridiag_df_rows(const double* Hp, int64_t ld, int W, int n, EighBufs b,
                                   cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const size_t sm = tridiag_df_smem(W);
  cudaError_t e = cudaFuncSetAttribute(tridiag_df_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  tridiag_df_kernel<<<n, NT, sm, s>>>(Hp, ld, W, b);
  return cudaGetLastError();
}

}  // namespace kubo
