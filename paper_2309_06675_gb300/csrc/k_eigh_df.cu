// Step (2) for the MIXED mode: the Householder tridiagonalisation H = Q T_c Q^dagger and the
// implicit QL eigenvalue iteration of the FP64 eigensolver in double-float arithmetic.
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
#include <algorithm>

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
// only for exponents outside a safe range.  That rare path is a call, which the compiler
// branches around: inlined, it would be issued predicated off for every element, and a
// predicated-off FP64 instruction still takes its slots on the FP64 pipe.
__device__ __noinline__ float2 df_split_slow(double x);
__device__ __noinline__ double widen_slow(float f) { return (double)f; }
// x = hi + lo with hi = x truncated to 24 significant bits and lo the remaining 29 bits
// rounded to FP32 (|x - hi - lo| <= 2^-48 |x|).
__device__ __forceinline__ float2 df_split_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex < 1023 - 70 || ex > 1023 + 70) {
    // +-0 as df_split gives it: (+-0, +0)
    if ((b << 1) == 0ull) return make_float2(__uint_as_float((uint32_t)(b >> 32)), 0.f);
    return df_split_slow(x);
  }
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
  if (ex == 0 || ex == 0xFFu) return widen_slow(f);
  return __longlong_as_double((long long)(((unsigned long long)(u >> 31) << 63) |
                                          ((unsigned long long)(ex + 896) << 52) |
                                          ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}
__device__ __forceinline__ double df_val(float h, float l) { return widen_bits(h) + widen_bits(l); }

__device__ __noinline__ float2 df_split_slow(double x) { return df_split(x); }

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

// Scalar double-float operations (value h + l): results normalised, ~2^-46 relative.
struct Df {
  float h, l;
};
__device__ __forceinline__ Df dfv(float h, float l = 0.f) { return Df{h, l}; }
__device__ __forceinline__ Df df_add(Df a, Df b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  Df r;
  fast_two_sum(s, e, r.h, r.l);
  return r;
}
__device__ __forceinline__ Df df_neg(Df a) { return Df{-a.h, -a.l}; }
__device__ __forceinline__ Df df_sub(Df a, Df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ Df df_mul(Df a, Df b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  Df r;
  fast_two_sum(p, e, r.h, r.l);
  return r;
}
// a * b + c
__device__ __forceinline__ Df df_fma(Df a, Df b, Df c) { return df_add(df_mul(a, b), c); }
// 1 / sqrt(a), a > 0: the FP32 estimate and one Newton step, y + y (1 - a y^2) / 2, whose
// correction is ~2^-22 of y and needs FP32 precision only
__device__ __forceinline__ Df df_rsqrt(Df a) {
  const float y = rsqrtf(a.h);
  const float y2 = __fmul_rn(y, y);
  const Df t = df_mul(a, Df{y2, fmaf(y, y, -y2)});
  const float r = __fadd_rn(__fsub_rn(1.0f, t.h), -t.l);
  Df out;
  fast_two_sum(y, 0.5f * y * r, out.h, out.l);
  return out;
}
// sqrt(a), a >= 0: y + (a - y^2) / (2 y) from an approximate FP32 root (the correction
// absorbs its few-ulp error)
__device__ __forceinline__ Df df_sqrt(Df a) {
  if (!(a.h > 0.f)) return Df{0.f, 0.f};
  const float ry = rsqrtf(a.h);
  const float y = a.h * ry;
  const float y2 = __fmul_rn(y, y);
  const Df d = df_sub(a, Df{y2, fmaf(y, y, -y2)});
  Df out;
  fast_two_sum(y, d.h * (0.5f * ry), out.h, out.l);
  return out;
}
// FP32 reciprocal estimate (one MUFU instruction, ~1 ulp)
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// a / b: an approximate FP32 quotient q1 = a rcp(b), then the quotient of the remainder
// a - q1 b (exact to 2^-46): ~2^-45 relative in all
__device__ __forceinline__ Df df_div(Df a, Df b) {
  const float rb = rcp_approx(b.h);
  const float q1 = a.h * rb;
  const Df r = df_sub(a, df_mul(b, Df{q1, 0.f}));
  Df out;
  fast_two_sum(q1, r.h * rb, out.h, out.l);
  return out;
}

// Householder step j's scalar part on warp 0: the norm of column j below the sub-diagonal,
// the reflector H = I - tau v v^H with v = x - beta e1, beta = -e^{i arg alpha} |x|,
// v0 = alpha + e^{i arg alpha} |x|, tau = 1 / (|x| (|x| + |alpha|)) (FP64 on lane 0), and the
// copy of v into vdst.  Column j must be final (its last update done by this warp).
__device__ __forceinline__ void householder_warp0(float4* A, int W, int j, float4* vdst,
                                                  double2* be, double* tb, float2* s_tdf,
                                                  int* s_act, int lane) {
  const int o = j + 1, m = W - 1 - j;
  float sh = 0.f, sl = 0.f;
  for (int r = o + 1 + lane; r < W; r += 32) {
    const float4 x = A[tri(r, j)];
    df_mac(sh, sl, x.x, x.y, x.x, x.y);
    df_mac(sh, sl, x.z, x.w, x.z, x.w);
  }
  warp_sum_df(sh, sl);
  if (lane == 0) {
    // in FP32 pairs: the FP64 pipe would serialise this lane behind 16-cycle slots
    Df s2;
    fast_two_sum(sh, sl, s2.h, s2.l);
    const float4 a4 = A[tri(o, j)];
    const Df alx = Df{a4.x, a4.y}, aly = Df{a4.z, a4.w};
    Df tau = Df{0.f, 0.f};
    Df bx = alx, by = aly;   // beta
    if (s2.h > 0.f) {
      const Df aa2 = df_fma(alx, alx, df_mul(aly, aly));
      const Df nrm = df_sqrt(df_add(aa2, s2));
      Df pr = Df{1.f, 0.f}, pi = Df{0.f, 0.f}, aa = Df{0.f, 0.f};
      if (aa2.h > 0.f) {
        const Df ra = df_rsqrt(aa2);
        aa = df_mul(aa2, ra);
        pr = df_mul(alx, ra);
        pi = df_mul(aly, ra);
      }
      bx = df_neg(df_mul(pr, nrm));
      by = df_neg(df_mul(pi, nrm));
      const Df v0x = df_fma(pr, nrm, alx), v0y = df_fma(pi, nrm, aly);
      A[tri(o, j)] = make_float4(v0x.h, v0x.l, v0y.h, v0y.l);
      tau = df_div(Df{1.f, 0.f}, df_mul(nrm, df_add(nrm, aa)));
    }
    *s_tdf = make_float2(tau.h, tau.l);
    *s_act = tau.h != 0.f;
    be[j] = make_double2(df_val(bx.h, bx.l), df_val(by.h, by.l));
    tb[j] = df_val(tau.h, tau.l);
  }
  __syncwarp();
  for (int r = lane; r < m; r += 32) vdst[r] = A[tri(o + r, j)];
}

// a -= vr conj(wc) + wr conj(vc) (the rank-2 update of one lower element; diag: real)
__device__ __forceinline__ void rank2_elem(float4& a, const float4& vr, const float4& wr,
                                           const float4& vc, const float4& wc, bool diag) {
  df_mac(a.x, a.y, -vr.x, -vr.y, wc.x, wc.y);
  df_mac(a.x, a.y, -vr.z, -vr.w, wc.z, wc.w);
  df_mac(a.x, a.y, -wr.x, -wr.y, vc.x, vc.y);
  df_mac(a.x, a.y, -wr.z, -wr.w, vc.z, vc.w);
  df_norm(a.x, a.y);
  if (diag) {
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
}

// FastDiv magics ceil(2^32 / d) of the trailing-block orders 2 <= d <= 256: the symv's row /
// part split of each column step reads one (the same for the whole block) instead of running
// two integer-divide sequences.
struct DivMagic {
  uint32_t v[257];
};
constexpr DivMagic make_div_magic() {
  DivMagic t{};
  for (uint32_t d = 2; d <= 256; ++d) t.v[d] = 0xFFFFFFFFu / d + 1u;
  return t;
}
__constant__ DivMagic c_divmag = make_div_magic();

// Packed rows of leading dimension ld (the [H | dxH | dyH] rows of the tensor-core Fourier
// sum).  Shared memory: the lower triangle packed by rows (element (r, c <= r) at
// r (r + 1) / 2 + c) as complex double-float, two reflector buffers, p / w, the symv
// partials.  Per column step three block barriers: after the symv partials, after w, and
// after the rank-2 update, during which warp 0 first finishes the next column and prepares
// the next reflector (so the serial Householder step overlaps the other warps' update).
__global__ void __launch_bounds__(NT, 5) tridiag_df_kernel(const double* __restrict__ Hp,
                                                           int64_t ld, int W, EighBufs b) {
  extern __shared__ float4 sm4[];
  float4* A = sm4;                                  // W (W + 1) / 2
  float4* vbuf = A + (size_t)W * (W + 1) / 2;       // [2][W] reflectors of even / odd steps
  float4* pb = vbuf + 2 * W;                        // [W] p, then w
  float4* sp = pb + W;                              // [NT] symv partial sums
  double2* be = reinterpret_cast<double2*>(sp + NT);   // [W] complex sub-diagonal beta_i
  double* tb = reinterpret_cast<double*>(be + W);      // [W] tau_i
  // row of each packed lower-triangle index (the same for every triangle in row-packed order)
  unsigned char* rowof = reinterpret_cast<unsigned char*>(tb + W);   // [W (W + 1) / 2]
  // tau as an FP32 pair and tau != 0, by step parity (warp 0 writes step i + 1's while the
  // other warps may still read step i's)
  __shared__ float2 s_tdf[2];
  __shared__ int s_act[2];
  __shared__ float2 s_vp[4];  // per-warp parts of Re(v^H p) (warps 0..3)

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t k = blockIdx.x;
  const double* P = Hp + (size_t)k * ld;

  for (int r = t; r < W; r += NT)
    for (int c = 0; c <= r; ++c) rowof[tri(r, c)] = (unsigned char)r;
  __syncthreads();
  for (int idx = t; idx < W * (W + 1) / 2; idx += NT) {
    const int r = rowof[idx];
    const int c = idx - tri(r, 0);
    A[idx] = r == c ? cdf_split(P[r * W + r], 0.0)
                    : cdf_split(P[c * W + r], -P[r * W + c]);   // conj(A_cr)
  }
  __syncthreads();
  if (W > 2 && warp == 0) householder_warp0(A, W, 0, vbuf, be, tb, &s_tdf[0], &s_act[0], lane);
  __syncthreads();

  for (int i = 0; i < W - 2; ++i) {
    const int o = i + 1;       // first row of the trailing block
    const int m = W - 1 - i;   // its size
    const float4* vb = vbuf + (i & 1) * W;
    float4* vnext = vbuf + ((i + 1) & 1) * W;
    const bool next = i + 1 < W - 2;
    const int ph = i & 1, nph = ph ^ 1;
    if (!s_act[ph]) {
      // no reflection: the trailing block is unchanged; prepare the next step
      if (next && warp == 0) householder_warp0(A, W, o, vnext, be, tb, &s_tdf[nph], &s_act[nph], lane);
      __syncthreads();
      continue;
    }
    // p = tau A22 v, spread densely: thread t takes row r = t mod m and the columns
    // c = part, part + P, ... (part = t / m, P = NT / m); the P partials of a row are added
    // in part order.  Mirrored elements (c > r) are conjugated by flipping the sign bits of
    // both imaginary halves (one loop for all columns keeps the warp convergent: its threads
    // have different rows r).
    {
      const uint32_t mag = c_divmag.v[m];   // floor(a / m) = umulhi(a, mag) for a <= NT
      const int Pp = (int)__umulhi(NT, mag);
      const int part = (int)__umulhi(t, mag), r = t - part * m;
      if (part < Pp) {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        // running packed indices of (r, c) (row-contiguous, + Pp per step of c) and of the
        // mirror (c, r) = tri(o + c, o + r), whose step (o + c) Pp + Pp (Pp + 1) / 2 itself
        // grows by Pp^2
        int ilo = tri(o + r, o) + part;
        int iup = tri(o + part, o + r);
        int dup = (o + part) * Pp + ((Pp * (Pp + 1)) >> 1);
        const int pp2 = Pp * Pp;
        for (int c = part; c < m; c += Pp) {
          const bool up = c > r;
          float4 a = A[up ? iup : ilo];
          if (up) {
            a.z = -a.z;
            a.w = -a.w;
          }
          cdf_mac<false>(acc, a, vb[c]);
          ilo += Pp;
          iup += dup;
          dup += pp2;
        }
        sp[part * m + r] = acc;
      }
    }
    __syncthreads();
    // warps 0..3 (m <= 127 rows): p_t = tau sum of the partials, K = tau Re(v^H p) / 2,
    // w_t = p_t - K v_t
    if (t < 128) {
      const int Pp = (int)__umulhi(NT, c_divmag.v[m]);
      float4 p = make_float4(0.f, 0.f, 0.f, 0.f), v = make_float4(0.f, 0.f, 0.f, 0.f);
      float dh = 0.f, dl = 0.f;
      if (t < m) {
        float4 s = sp[t];
        for (int q = 1; q < Pp; ++q) {
          const float4 u = sp[q * m + t];
          float e;
          two_sum(s.x, u.x, s.x, e);
          s.y = __fadd_rn(s.y, __fadd_rn(u.y, e));
          two_sum(s.z, u.z, s.z, e);
          s.w = __fadd_rn(s.w, __fadd_rn(u.w, e));
        }
        s = cdf_norm(s);
        const float2 tdf = s_tdf[ph];
        df_mac(p.x, p.y, tdf.x, tdf.y, s.x, s.y);
        df_mac(p.z, p.w, tdf.x, tdf.y, s.z, s.w);
        p = cdf_norm(p);
        v = vb[t];
        df_mac(dh, dl, v.x, v.y, p.x, p.y);
        df_mac(dh, dl, v.z, v.w, p.z, p.w);
      }
      warp_sum_df(dh, dl);
      if (lane == 0) s_vp[warp] = make_float2(dh, dl);
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (t < m) {
        float vh = s_vp[0].x, vl = s_vp[0].y;
        for (int q = 1; q < 4; ++q) {
          float e;
          two_sum(vh, s_vp[q].x, vh, e);
          vl = __fadd_rn(vl, __fadd_rn(s_vp[q].y, e));
        }
        // K = tau (vh + vl) / 2 as an FP32 pair (the factor 1/2 is exact)
        const float2 tdf = s_tdf[ph];
        float Kh = 0.f, Kl = 0.f;
        df_mac(Kh, Kl, 0.5f * tdf.x, 0.5f * tdf.y, vh, vl);
        df_norm(Kh, Kl);
        const float2 Kd = make_float2(Kh, Kl);
        df_mac(p.x, p.y, -Kd.x, -Kd.y, v.x, v.y);
        df_mac(p.z, p.w, -Kd.x, -Kd.y, v.z, v.w);
        pb[t] = cdf_norm(p);
      }
    }
    __syncthreads();
    // A22 <- A22 - v w^H - w v^H on the lower triangle (c <= r).  Warp 0: column 0 of the
    // block (it becomes column o of A, the next step's), then the next Householder step;
    // warps 1..: the columns 1 .. m-1 (a triangle of order m - 1).
    if (warp == 0) {
      const float4 v0 = vb[0], w0 = pb[0];
      for (int r = lane; r < m; r += 32) {
        float4 a = A[tri(o + r, o)];
        rank2_elem(a, vb[r], pb[r], v0, w0, r == 0);
        A[tri(o + r, o)] = a;
      }
      __syncwarp();
      if (next) householder_warp0(A, W, o, vnext, be, tb, &s_tdf[nph], &s_act[nph], lane);
    } else {
      const int n1 = m - 1;
      const int ntri = n1 * (n1 + 1) / 2;
      // element (r + 1, c + 1) of the trailing block sits at tri(o + r + 1, o + c + 1)
      // = idx + r (o + 1) + tri(o + 1, o + 1) for idx = tri(r, c)
      const int o1 = o + 1, base = tri(o + 1, o + 1);
      for (int idx = t - 32; idx < ntri; idx += NT - 32) {
        const int r = rowof[idx];
        const int c = idx - tri(r, 0);
        const int ia = idx + r * o1 + base;
        float4 a = A[ia];
        rank2_elem(a, vb[r + 1], pb[r + 1], vb[c + 1], pb[c + 1], r == c);
        A[ia] = a;
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
  double2* ub = reinterpret_cast<double2*>(vbuf);   // unit phases (the reflector buffers are free)
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
  if (t < 32) {
    // D_0 = 1, D_{j+1} = D_j u_j as a warp scan (lane l takes u_4l .. u_4l+3, W <= 128)
    // rather than one thread's serial chain of complex products on the FP64 pipe
    double2 u[4];
    double2 pr = make_double2(1.0, 0.0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = 4 * t + q;
      u[q] = j + 1 < W ? ub[j] : make_double2(1.0, 0.0);
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
  for (int j = t; j < W; j += NT) {
    const float4 a = A[tri(j, j)];
    dout[j] = df_val(a.x, a.y);
    tout[j] = j < W - 2 ? tb[j] : 0.0;
  }
  double2* rout = b.refl + (size_t)k * W * W;
  for (int r = warp; r < W; r += NT / 32)
    for (int c = lane; c < W; c += 32) {
      double2 v = make_double2(0.0, 0.0);
      if (r > c) {
        const float4 a = A[tri(r, c)];
        v = make_double2(df_val(a.x, a.y), df_val(a.z, a.w));
      }
      rout[r * W + c] = v;
    }
}

// ------------------------------------------------------------------ QL in double-float
// Eigenvalues of the real symmetric tridiagonal T (FP64 d, |e|) by implicit QL with Wilkinson
// shifts, one k-point per lane, in double-float: the same chase as the FP64 kernel, with the
// deflation test |e_m| <= 2^-44 (|d_m| + |d_m+1|) matched to the pair precision.  d and e live
// lane-interleaved in shared memory as [W][32] pairs.
__global__ void __launch_bounds__(32) ql_df_kernel(int W, int n, EighBufs b, DevStatus* st) {
  extern __shared__ float2 qsm2[];
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  float2* D = qsm2 + lane;
  float2* E = D + (size_t)W * 32;
  if (k >= n) return;
  for (int i = 0; i < W; ++i) {
    D[i * 32] = df_split_bits(b.d[(size_t)k * W + i]);
    E[i * 32] = df_split_bits(b.e[(size_t)k * W + i]);
  }
  auto ld = [&](const float2* a, int i) { const float2 v = a[i * 32]; return Df{v.x, v.y}; };
  auto st2 = [&](float2* a, int i, Df v) { a[i * 32] = make_float2(v.h, v.l); };
  bool fail = false;
  const float eps = 0x1p-44f;
  // each lane advances through its own eigenvalues (as the FP64 kernel): one pass deflates the
  // current eigenvalue or runs one sweep on its block
  int l = 0, iter = 0;
  while (l < W) {
    {
      int m = l;
      for (; m < W - 1; ++m) {
        const float dd = fabsf(D[m * 32].x) + fabsf(D[(m + 1) * 32].x);
        if (fabsf(E[m * 32].x) <= eps * dd) break;
      }
      if (m == l) {
        ++l;
        iter = 0;
        continue;
      }
      if (++iter > b.ql_cap) { fail = true; break; }
      // Wilkinson shift from the leading 2x2 of the block, then chase up from the bottom
      const Df dl = ld(D, l), el = ld(E, l);
      Df g = df_div(df_sub(ld(D, l + 1), dl), Df{2.0f * el.h, 2.0f * el.l});
      const Df r0 = df_sqrt(df_fma(g, g, dfv(1.0f)));
      g = df_add(df_sub(ld(D, m), dl), df_div(el, df_add(g, g.h >= 0.f ? r0 : df_neg(r0))));
      Df s = dfv(1.0f), c = dfv(1.0f), p = dfv(0.0f);
      bool early = false;
      for (int i = m - 1; i >= l; --i) {
        const Df ei = ld(E, i);
        const Df f = df_mul(s, ei), bb = df_mul(c, ei);
        const Df r2 = df_fma(f, f, df_mul(g, g));
        if (r2.h == 0.f) {   // split: the chase stops here
          st2(E, i + 1, dfv(0.f));
          st2(D, i + 1, df_sub(ld(D, i + 1), p));
          st2(E, m, dfv(0.f));
          early = true;
          break;
        }
        const Df ir = df_rsqrt(r2);
        st2(E, i + 1, df_mul(r2, ir));
        s = df_mul(f, ir);
        c = df_mul(g, ir);
        const Df gi = df_sub(ld(D, i + 1), p);
        const Df cb = df_mul(c, bb);
        const Df rr = df_fma(df_sub(ld(D, i), gi), s, df_add(cb, cb));
        p = df_mul(s, rr);
        st2(D, i + 1, df_add(gi, p));
        g = df_sub(df_mul(c, rr), bb);
      }
      if (early) continue;
      st2(D, l, df_sub(ld(D, l), p));
      st2(E, l, g);
      st2(E, m, dfv(0.f));
    }
  }
  for (int i = 0; i < W; ++i) {
    const float2 v = D[i * 32];
    b.lam[(size_t)k * W + i] = df_val(v.x, v.y);
  }
  if (fail) atomicOr(&st->bits, ST_NO_CONVERGENCE);
}

// ------------------------------------------------------------------ inverse iteration in double-float
__device__ __forceinline__ unsigned long long order_key(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// deterministic start vector in [0.5, 1.5) from an integer hash of (row, vector): 23 hash bits
// as the mantissa of a number in [1, 2), minus 1/2
__device__ __forceinline__ float iit_start_f(int i, int j) {
  unsigned h = (unsigned)i * 0x9E3779B1u ^ ((unsigned)j * 0x85EBCA77u + 0x165667B1u);
  h ^= h >> 15; h *= 0x2C1B3C6Du; h ^= h >> 12; h *= 0x297A2D39u; h ^= h >> 15;
  return __fsub_rn(__uint_as_float(0x3F800000u | (h >> 9)), 0.5f);
}

// Two solves: the shifts are the QL eigenvalues to ~2^-45 ||T|| (delta), so one solve from a
// start with O(1) components leaves a contamination ~delta / gap along the other eigenvectors
// and two leave (delta / gap)^2 (1e-12 at gap = 1e-7 ||T||), far below the FP32 rounding of U
// that consumes them; closer eigenvalues form a cluster and are orthogonalised.
constexpr int IIT_DF_SOLVES = 2;

// Eigenvectors of the tridiagonal T by inverse iteration, as the FP64 kernel (sort, clusters
// closer than 1e-3 ||T||_1 on one thread, LU of T - lambda I with row interchanges, solves
// (two here, three there) from a fixed pseudo-random start, modified Gram-Schmidt inside a cluster,
// normalisation), in FP32 pairs: the solves' backward error ~2^-46 ||T|| sets the residual,
// and the eigenvectors are accurate to ~2^-46 ||T|| / gap.  Coincident eigenvalues are
// separated by 10 2^-46 ||T||_1.
// Memory: each thread's iterate lives in shared memory ([W][ldt], lane-interleaved); the LU
// factors go to the per-CTA global scratch (L2-resident) as three planes: reciprocal pivots,
// multipliers and the first super-diagonal of U (the second, nonzero only on swapped rows, is
// the next e of T).  Finished vectors are written to Z in FP64; Gram-Schmidt reads a
// cluster's earlier vectors from there.
__global__ void __launch_bounds__(128) iit_df_kernel(int W, int n, EighBufs b,
                                                     double* __restrict__ Eout,
                                                     double* __restrict__ Z,
                                                     double* __restrict__ scratch) {
  extern __shared__ float2 zsm[];               // [W][ldt] iterates
  __shared__ float2 ws[128], dd[128], ee[128];
  __shared__ int newc[128];
  __shared__ float s_onenrm;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int ldt = blockDim.x;
  const size_t plane = (size_t)W * ldt;
  float2* __restrict__ RP = reinterpret_cast<float2*>(scratch) + (size_t)blockIdx.x * 3 * plane;
  float2* __restrict__ ML = RP + plane;   // multipliers
  float2* __restrict__ U1 = ML + plane;   // first super-diagonal of U
  float2* Zs = zsm + t;
  auto ldf = [](const float2* a, size_t i) { const float2 v = a[i]; return Df{v.x, v.y}; };
  auto sdf = [](float2* a, size_t i, Df v) { a[i] = make_float2(v.h, v.l); };
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
      ws[rnk] = df_split_bits(lj);
      Eout[k * W + rnk] = lj;
      dd[t] = df_split_bits(b.d[k * W + t]);
      ee[t] = df_split_bits(b.e[k * W + t]);
    }
    __syncthreads();
    if (warp == 0) {
      float mx = 0.f;
      for (int i = lane; i < W; i += 32)
        mx = fmaxf(mx, fabsf(dd[i].x) + (i > 0 ? ee[i - 1].x : 0.f) + (i < W - 1 ? ee[i].x : 0.f));
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0) s_onenrm = mx > 0.f ? mx : 1.f;
    }
    __syncthreads();
    const float onenrm = s_onenrm;
    const float ortol = 1e-3f * onenrm, pertol = 10.0f * 0x1p-46f * onenrm;
    const float tiny = 0x1p-46f * onenrm;
    if (t < W) {
      const Df gap = t > 0 ? df_sub(ldf(ws, t), ldf(ws, t - 1)) : Df{0.f, 0.f};
      newc[t] = (t == 0) || (gap.h > ortol);
    }
    __syncthreads();

    double* __restrict__ Zd = Z + (size_t)k * W * W;
    const int j = t;
    if (j < W && newc[j]) {
      Df lprev = Df{0.f, 0.f};
      for (int m = j; m < W && (m == j || !newc[m]); ++m) {
        Df lam = ldf(ws, m);
        if (m > j && df_sub(lam, lprev).h <= pertol) lam = df_add(lprev, Df{pertol, 0.f});
        lprev = lam;
        // ---- LU of T - lam I with row interchanges (the carried third entry of a row is
        // always 0 after a step, so a row of U is (q0, q1, 0) or swapped (e_i, a, e_i+1))
        unsigned long long piv0 = 0ull, piv1 = 0ull;   // row interchanges, bits 0..127
        Df q0 = df_sub(ldf(dd, 0), lam), q1 = W > 1 ? ldf(ee, 0) : Df{0.f, 0.f};
        for (int i = 0; i + 1 < W; ++i) {
          const Df ei = ldf(ee, i);
          const Df a = df_sub(ldf(dd, i + 1), lam);
          const Df bb = i + 2 < W ? ldf(ee, i + 1) : Df{0.f, 0.f};
          const size_t o = (size_t)i * ldt + t;
          // the interchange only selects operands: one instruction sequence for the warp
          const bool sw = !(fabsf(q0.h) >= fabsf(ei.h));
          const Df den = sw ? ei : (q0.h == 0.f ? Df{tiny, 0.f} : q0);
          const Df r = df_div(Df{1.f, 0.f}, den);
          const Df mlt = df_mul(sw ? q0 : ei, r);
          sdf(RP, o, r); sdf(ML, o, mlt); sdf(U1, o, sw ? a : q1);
          if (sw) { if (i < 64) piv0 |= 1ull << i; else piv1 |= 1ull << (i - 64); }
          const Df n0 = df_sub(sw ? q1 : a, df_mul(mlt, sw ? a : q1));
          const Df mb = df_mul(mlt, bb);
          q1 = sw ? df_neg(mb) : bb;
          q0 = n0;
        }
        if (q0.h == 0.f) q0 = Df{tiny, 0.f};
        sdf(RP, (size_t)(W - 1) * ldt + t, df_div(Df{1.f, 0.f}, q0));
        sdf(U1, (size_t)(W - 1) * ldt + t, Df{0.f, 0.f});
        for (int i = 0; i < W; ++i) Zs[(size_t)i * ldt] = make_float2(iit_start_f(i, m), 0.f);
        for (int it = 0; it < IIT_DF_SOLVES; ++it) {
          // forward elimination L y = P b; the running row value is carried in registers
          Df cur = ldf(Zs, 0);
#pragma unroll 8
          for (int i = 0; i + 1 < W; ++i) {
            const bool sw = i < 64 ? ((piv0 >> i) & 1ull) : ((piv1 >> (i - 64)) & 1ull);
            const Df mlt = ldf(ML, (size_t)i * ldt + t);
            const Df yn = ldf(Zs, (size_t)(i + 1) * ldt);
            const Df f = sw ? yn : cur, g = sw ? cur : yn;
            sdf(Zs, (size_t)i * ldt, f);
            cur = df_sub(g, df_mul(mlt, f));
          }
          sdf(Zs, (size_t)(W - 1) * ldt, cur);
          // back substitution U x = y (U2 of row i: e_i+1 on swapped rows, else 0)
          Df x1 = Df{0.f, 0.f}, x2 = Df{0.f, 0.f};
#pragma unroll 8
          for (int i = W - 1; i >= 0; --i) {
            const bool sw = i + 1 < W && (i < 64 ? ((piv0 >> i) & 1ull) : ((piv1 >> (i - 64)) & 1ull));
            const size_t o = (size_t)i * ldt + t;
            const Df y = ldf(Zs, (size_t)i * ldt);
            Df num = df_sub(y, df_mul(ldf(U1, o), x1));
            if (sw && i + 2 < W) num = df_sub(num, df_mul(ldf(ee, i + 1), x2));
            const Df xi = df_mul(num, ldf(RP, o));
            sdf(Zs, (size_t)i * ldt, xi);
            x2 = x1;
            x1 = xi;
          }
          for (int q = j; q < m; ++q) {   // earlier vectors of the cluster (FP64 in Z)
            float ch = 0.f, cl = 0.f;
            for (int i = 0; i < W; ++i) {
              const float2 zq = df_split_bits(Zd[(size_t)i * W + q]);
              const Df zm = ldf(Zs, (size_t)i * ldt);
              df_mac(ch, cl, zq.x, zq.y, zm.h, zm.l);
            }
            Df c;
            fast_two_sum(ch, cl, c.h, c.l);
            for (int i = 0; i < W; ++i) {
              const float2 zq = df_split_bits(Zd[(size_t)i * W + q]);
              sdf(Zs, (size_t)i * ldt, df_sub(ldf(Zs, (size_t)i * ldt), df_mul(c, Df{zq.x, zq.y})));
            }
          }
          float sh = 0.f, sl = 0.f;
          for (int i = 0; i < W; ++i) {
            const Df u = ldf(Zs, (size_t)i * ldt);
            df_mac(sh, sl, u.h, u.l, u.h, u.l);
          }
          Df s2;
          fast_two_sum(sh, sl, s2.h, s2.l);
          const Df inv = df_rsqrt(s2);
          for (int i = 0; i < W; ++i)
            sdf(Zs, (size_t)i * ldt, df_mul(ldf(Zs, (size_t)i * ldt), inv));
        }
        for (int i = 0; i < W; ++i) {
          const float2 v = Zs[(size_t)i * ldt];
          Zd[(size_t)i * W + m] = df_val(v.x, v.y);
        }
      }
    }
  }
}

}  // namespace

size_t tridiag_df_smem(int W) {
  return ((size_t)W * (W + 1) / 2 + 3 * (size_t)W + NT) * sizeof(float4) +
         (size_t)W * (sizeof(double2) + sizeof(double)) + (size_t)W * (W + 1) / 2;
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

size_t ql_df_smem(int W) { return (size_t)2 * W * 32 * sizeof(float2); }

cudaError_t launch_ql_df(int W, int n, EighBufs b, DevStatus* st, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const size_t sm = ql_df_smem(W);
  cudaError_t e = cudaFuncSetAttribute(ql_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  ql_df_kernel<<<(n + 31) / 32, 32, sm, s>>>(W, n, b, st);
  return cudaGetLastError();
}

// persistent CTAs of the double-float inverse iteration: as many per SM as the iterate
// arrays (W x ldt pairs of shared memory per CTA) allow within 220 KB (6 at W = 64: 12 warps
// per SM, measured faster than 5); each uses 3 W ldt pairs of the scratch
int iit_df_ctas(int W) {
  const int ldt = (W + 31) / 32 * 32;
  const size_t sm = (size_t)W * ldt * sizeof(float2) + 4 * 1024;
  return 152 * (int)std::max<size_t>(1, std::min<size_t>(16, (220 * 1024) / sm));
}

cudaError_t launch_iit_df(int W, int n, EighBufs b, double* E, double* Z, double* scratch,
                          int slots, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (W > 128 || slots < 1 || Z == nullptr) return cudaErrorInvalidValue;
  const int ldt = (W + 31) / 32 * 32;
  const size_t sm = (size_t)W * ldt * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(iit_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  // the FP64 scratch of `slots` CTAs (4 planes each) holds at least as many of these (3)
  const int grid = std::min(std::min(n, slots), iit_df_ctas(W));
  iit_df_kernel<<<grid, ldt, sm, s>>>(W, n, b, E, Z, scratch);
  return cudaGetLastError();
}

}  // namespace kubo
