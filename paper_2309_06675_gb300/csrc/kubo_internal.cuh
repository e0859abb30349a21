// Internal declarations shared by the CUDA translation units of libkubo.
// Nothing here is part of the public ABI (see include/kubo.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kubo.h"

namespace kubo {

// ---------------------------------------------------------------- device status word
// Bits OR-ed into the status word by kernels; read back by the host at the end of a call.
enum : unsigned {
  ST_NOT_HERMITIAN = 1u,   // H(-R) != H(R)^dagger beyond tolerance
  ST_NONFINITE = 2u,       // NaN/Inf in H(R)
  ST_NO_CONVERGENCE = 4u,  // QL iteration cap reached at some k
  ST_TIMEOUT = 16u,        // a bounded device-side wait gave up
  ST_BAD_INDEX = 32u,      // a listed mesh index outside [0, N_k)
};

struct DevStatus {
  unsigned int bits;
  unsigned int pad;
  unsigned long long herm_dev_bits;  // max |H(-R)_ji - conj H(R)_ij| as double bits
  unsigned long long herm_max_bits;  // max |H(R)_ij| as double bits
  unsigned long long pad2;
};

// ---------------------------------------------------------------- batch of k-points
// Local index t of a batch maps to the linear mesh index idx[t] (list) or base + t (range).
struct KList {
  const int64_t* idx;
  int64_t base;
  int n;
};

__device__ __forceinline__ int64_t klist_get(const KList& l, int t) {
  return l.idx ? l.idx[t] : l.base + t;
}

struct Mesh {
  int N1, N2, N3;
  int64_t Nk;
};

// ---------------------------------------------------------------- prepared model (device)
// H(k) = P0 + sum_h [cos(th_h) A_h + sin(th_h) B_h]
// d_a H(k) = sum_h R_h,a [cos(th_h) B_h - sin(th_h) A_h]
// with A_h = H(R_h) + H(-R_h), B_h = i (H(R_h) - H(-R_h)) over the canonical half set
// (first non-zero component of R_h positive).  Rows of Bp: 0 -> P0, 1+2h -> A_h, 2+2h -> B_h,
// each packed Hermitian (W*W doubles).
struct Model {
  int W, N_R, N_h, K;
  const double* Bp;       // [K][W*W]
  const int* Rh;          // [N_h][3]
  const double2* tab;     // twiddles: tab[tab_off[a] + j] = e^{2 pi i j / N_a}
  const float4* tab_df;   // the same twiddles as FP32 pairs (re_h, re_l, im_h, im_l)
  int tab_off[3];
};

// ---------------------------------------------------------------- separable Fourier sum
// Bounding box |R_a| <= h_a of the R set (k_fourier_sep.cu).
struct SepBox {
  int h1, h2, h3;
};

// ---------------------------------------------------------------- small helpers
// |x| as an ordered integer (non-NaN x): |x| < |y| iff mag_bits(x) < mag_bits(y), and x == 0
// iff mag_bits(x) == 0 -- integer compares in place of FP64 compares (GB300 issues those on the
// FP64 pipe, at 1/64 of the FP32 rate)
__device__ __forceinline__ unsigned long long mag_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// x_i <- x_i 2^-e (i < n, stride apart), e the exponent of max |x_i|, on the bit patterns: the
// exponent fields are shifted by integer subtraction (exact); zeros, subnormals and entries
// that would leave the normal range become signed zeros (all below 2^-1022 of the largest or
// of the normal range), and a zero or non-finite vector is left alone.  The inverse
// iterations rescale their iterate this way between solves (no FP64 square root, reciprocal
// or multiplies; only the last solve's vector is normalised in FP64).
__device__ __forceinline__ void pow2_rescale(double* x, int n, size_t stride) {
  unsigned long long mx = 0ull;
  for (int i = 0; i < n; ++i) {
    const unsigned long long u = mag_bits(x[i * stride]);
    mx = u > mx ? u : mx;
  }
  const int ex = (int)(mx >> 52);
  if (ex == 0 || ex >= 0x7FF || ex == 1023) return;
  const int e = ex - 1023;
  for (int i = 0; i < n; ++i) {
    const long long b = __double_as_longlong(x[i * stride]);
    const int bex = (int)((b >> 52) & 0x7FF);
    const long long r = (bex >= 1 && bex - e >= 1) ? b - ((long long)e << 52)
                                                   : (b & (long long)0x8000000000000000ull);
    x[i * stride] = __longlong_as_double(r);
  }
}

// 1 / d by Newton-Raphson (r <- r + r (1 - d r), the relative error squaring each step) from
// the hardware's approximate FP64 reciprocal (~2^-22): 2^-44, then below an ulp before the
// final rounding.  Four FMAs after the estimate, where an IEEE division issues more FP64
// instructions (the LU of every inverse-iteration vector takes W of these, the Householder
// reduction one per column).  For |d| and 1 / |d| in the normal range (the callers' pivots
// are at least eps ||T||, the reduction's |x| (|x| + |alpha|) a positive sum of squares).
__device__ __forceinline__ double recip_nr(double d) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  double e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  e = fma(-d, r, 1.0);
  return fma(r, e, r);
}

// start vector of the inverse iterations: 0.5 + (h >> 8) 2^-24 in [0.5, 1.5) from an integer hash
// of (row, vector); 1 + (h >> 8) 2^-24 is assembled from its bits (exponent of 1, the 24-bit
// integer as the leading mantissa bits) and 0.5 subtracted exactly, instead of an integer ->
// FP64 conversion and a multiply-add, both on the FP64 pipe
__device__ __forceinline__ double iit_start_vec(int i, int j) {
  unsigned h = (unsigned)i * 0x9E3779B1u ^ ((unsigned)j * 0x85EBCA77u + 0x165667B1u);
  h ^= h >> 15; h *= 0x2C1B3C6Du; h ^= h >> 12; h *= 0x297A2D39u; h ^= h >> 15;
  return __longlong_as_double((long long)((0x3FFull << 52) | ((unsigned long long)(h >> 8) << 28))) - 0.5;
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}

// floor(a / d) by one multiply-high with mag = ceil(2^32 / d), exact for a d < 2^32 (the
// rounding excess of mag, below 1, times a stays under 2^32 / d).  The integer-divide sequence
// it replaces is about a dozen instructions (a float reciprocal estimate, two conversions and
// the integer corrections).  mag = 0 marks d = 1.
struct FastDiv {
  uint32_t d, mag;
  __host__ __device__ static uint32_t magic(uint32_t dd) { return dd > 1 ? 0xFFFFFFFFu / dd + 1u : 0u; }
  __device__ explicit FastDiv(uint32_t dd) : d(dd), mag(magic(dd)) {}
  __device__ __forceinline__ uint32_t div(uint32_t a) const { return mag ? __umulhi(a, mag) : a; }
};

// e^{i k.R} from per-axis twiddle tables with exact integer argument reduction.
__device__ __forceinline__ double2 mesh_phase(const double2* __restrict__ tab, const int* off,
                                              const Mesh& m, int j1, int j2, int j3, int r1,
                                              int r2, int r3) {
  int a1 = (int)(((long long)j1 * r1) % m.N1); if (a1 < 0) a1 += m.N1;
  int a2 = (int)(((long long)j2 * r2) % m.N2); if (a2 < 0) a2 += m.N2;
  int a3 = (int)(((long long)j3 * r3) % m.N3); if (a3 < 0) a3 += m.N3;
  double2 p = cmul(tab[off[0] + a1], tab[off[1] + a2]);
  return cmul(p, tab[off[2] + a3]);
}

__device__ __forceinline__ void mesh_coords(const Mesh& m, int64_t k, int& j1, int& j2, int& j3) {
  j3 = (int)(k % m.N3);
  int64_t q = k / m.N3;
  j2 = (int)(q % m.N2);
  j1 = (int)(q / m.N2);
}

// ---------------------------------------------------------------- eigensolver buffers
// Per-k intermediate layout of the three eigensolver kernels (all device memory).
struct EighBufs {
  double* d;        // [n][W]  diagonal of the real tridiagonal T
  double* e;        // [n][W]  off-diagonal |beta_i| (e[W-1] unused)
  double2* phase;   // [n][W]  D of T_complex = D T D^dagger
  double2* refl;    // [n][W*W] Householder vectors v_i stored in column i, rows i+1..W-1
  double* tau;      // [n][W]
  double* lam;      // [n][W]  eigenvalues of T (unordered)
  int ql_cap = 60;  // implicit-QL sweeps allowed per eigenvalue before ST_NO_CONVERGENCE
  int symv_parts = 4;  // Householder reduction: column partitions per row of its symv (1..8)
};

// ---------------------------------------------------------------- launchers
// All launchers are asynchronous on `s` and return the launch error (cudaSuccess on success).
cudaError_t launch_check_hermitian(const double2* H_R, const int* neg, int N_R, int W,
                                   DevStatus* st, cudaStream_t s);
cudaError_t launch_hermitian_verdict(DevStatus* st, cudaStream_t s);
cudaError_t launch_check_kidx(const int64_t* kidx, int64_t n, int64_t Nk, DevStatus* st,
                              cudaStream_t s);
// escale: the basis is multiplied by 2^escale (exact; 0 = unscaled)
cudaError_t launch_pack_basis(const double2* H_R, const int* pairs, int idx0, int N_h, int W,
                              double* Bp, cudaStream_t s, int escale = 0);
// x[i] *= 2^e for i < n (exact unless the result leaves the FP64 range)
cudaError_t launch_scale_pow2(double* x, int64_t n, int e, cudaStream_t s);
// tab: [N1 + N2 + N3] double2, followed by the same twiddles as FP32 pairs ([N1 + N2 + N3]
// float4: re_h, re_l, im_h, im_l; twiddle_bytes(...) in all)
cudaError_t launch_twiddles(double2* tab, int N1, int N2, int N3, cudaStream_t s);
inline size_t twiddle_bytes(int N1, int N2, int N3) {
  return (sizeof(double2) + sizeof(float4)) * (size_t)(N1 + N2 + N3);
}

cudaError_t launch_fourier_fp64(const Model& md, const Mesh& mesh, const KList& kl, double* Hp,
                                double* Xp, double* Yp, cudaStream_t s);

// pad (fused back-transform and rotation kernels): leading dimension W + pad of the shared-
// memory matrices; 1 (default) keeps column walks conflict-free, 0 is the padding ablation
cudaError_t launch_tridiag(const double* Hp, int W, int n, EighBufs b, cudaStream_t s);
// same reduction reading packed H from rows of leading dimension ld (tensor-core output)
cudaError_t launch_tridiag_rows(const double* Hp, int64_t ld, int W, int n, EighBufs b,
                                cudaStream_t s);
// the same reduction with its symv and rank-2 updates in double-float (FP32 pairs, ~2^-46
// per operation) on the FP32 pipe; FP64 outputs (MIXED mode)
cudaError_t launch_tridiag_df_rows(const double* Hp, int64_t ld, int W, int n, EighBufs b,
                                   cudaStream_t s);
cudaError_t launch_ql(int W, int n, EighBufs b, DevStatus* st, cudaStream_t s);
// the same QL iteration in double-float (MIXED mode; FP64 eigenvalues out)
cudaError_t launch_ql_df(int W, int n, EighBufs b, DevStatus* st, cudaStream_t s);
// eigenvectors of T by inverse iteration in double-float (MIXED mode; same layout, scratch and
// outputs as launch_iit, Z required)
cudaError_t launch_iit_df(int W, int n, EighBufs b, double* E, double* Z, double* scratch,
                          int slots, cudaStream_t s);
cudaError_t launch_backtransform(int W, int n, EighBufs b, double* E, double2* U,
                                 cudaStream_t s, int pad = 1);

cudaError_t launch_berry_fp64(const double* E, const double2* U, const double* Xp,
                              const double* Yp, int W, int n, const double* etas, int n_eta,
                              double* Om, int64_t eta_stride, cudaStream_t s, int pad = 1);

// rotations from packed dH rows of leading dimension ld (d_x H at column offset W*W, d_y H at
// 2*W*W, as written by the tensor-core Fourier kernel): in FP32 (mixed) or in FP64
cudaError_t launch_berry_mixed_rows(const double* E, const double2* U, const double* C,
                                    int64_t ld, int W, int n, const double* etas, int n_eta,
                                    double* Om, int64_t eta_stride, cudaStream_t s, int pad = 1);
cudaError_t launch_berry_fp64_rows(const double* E, const double2* U, const double* C,
                                   int64_t ld, int W, int n, const double* etas, int n_eta,
                                   double* Om, int64_t eta_stride, cudaStream_t s, int pad = 1);

// FP32 rotations with U = Q D Z assembled in FP32 inside the kernel from Z and the eigensolver
// factors in eb (phase, refl, tau), W <= 64.  vel32 (these and the two tensor-core forms
// below): the velocity rows of C are FP32 (vel32_x0 layout), else FP64 after the H columns.
cudaError_t launch_berry_mixed_rows_z(const double* E, const double* Z, const EighBufs& eb,
                                      const double* C, int64_t ld, int W, int n,
                                      const double* etas, int n_eta, double* Om,
                                      int64_t eta_stride, cudaStream_t s, int pad = 1,
                                      bool vel32 = false);
cudaError_t launch_berry_mixed_from_f64_z(const double* E, const double* Z, const EighBufs& eb,
                                          const double* Xp, const double* Yp, int W, int n,
                                          const double* etas, int n_eta, double* Om,
                                          int64_t eta_stride, cudaStream_t s, int pad = 1);

// the same rotations as exact fixed-point BF16-slice products on the tensor cores (U assembled
// in FP32 from Z and eb), W <= 64; a stalled MMA completion sets ST_TIMEOUT in st
cudaError_t launch_berry_tc_rows(const double* E, const double* Z, const EighBufs& eb,
                                 const double* C, int64_t ld, int W, int n, const double* etas,
                                 int n_eta, double* Om, int64_t eta_stride, DevStatus* st,
                                 cudaStream_t s, bool vel32 = false);
// the same two rotations in 3xTF32 on tcgen05 (kind::tf32, FP32 accumulation), W <= 64; U is
// assembled in FP32 from Z and eb; a stalled MMA completion sets ST_TIMEOUT in st
cudaError_t launch_berry_tf32_rows(const double* E, const double* Z, const EighBufs& eb,
                                   const double* C, int64_t ld, int W, int n, const double* etas,
                                   int n_eta, double* Om, int64_t eta_stride, DevStatus* st,
                                   cudaStream_t s, bool vel32 = false,
                                   const float2* U32 = nullptr);
// U = Q D Z in FP32 from Z and the eigensolver factors in eb, W <= 64: U32 [n][W][W] float2
// (the tensor-core rotation's input when it is formed by a kernel of its own)
cudaError_t launch_assemble_u32(const double* Z, const EighBufs& eb, float2* U32, int W, int n,
                                cudaStream_t s);
cudaError_t launch_berry_tf32_from_f64(const double* E, const double* Z, const EighBufs& eb,
                                       const double* Xp, const double* Yp, int W, int n,
                                       const double* etas, int n_eta, double* Om,
                                       int64_t eta_stride, DevStatus* st, cudaStream_t s);
cudaError_t launch_berry_tc_from_f64(const double* E, const double* Z, const EighBufs& eb,
                                     const double* Xp, const double* Yp, int W, int n,
                                     const double* etas, int n_eta, double* Om,
                                     int64_t eta_stride, DevStatus* st, cudaStream_t s);

// FP32 rotation from FP64 packed arrays (error-budget mode)
cudaError_t launch_berry_mixed_from_f64(const double* E, const double2* U, const double* Xp,
                                        const double* Yp, int W, int n, const double* etas,
                                        int n_eta, double* Om, int64_t eta_stride,
                                        cudaStream_t s, int pad = 1);

// tensor-core Fourier sum (k_fourier_tc.cu)
int tc_pad_m(int n);
int tc_pad_n(int W);
int tc_pad_k(int N_R);
int tc_slices();
cudaError_t launch_basis_split(const double* Bp, const int* Rh, int N_h, int W, int Npad, int Kp,
                               int* col_exp, void* Bt, cudaStream_t s);
cudaError_t launch_coef_split(const Model& md, const Mesh& mesh, const KList& kl, int Mpad, int Kp,
                              void* A, cudaStream_t s);
// FP32 velocity rows: the packed dH_x and dH_y of an output row r (ldc doubles, the packed H
// in its first W^2) as FP32, at float indices vel32_x0(W) and vel32_x0(W) + vel32_yoff(W) of
// the row (float row stride 2 ldc; both 16-byte aligned, after the H columns)
inline int vel32_x0(int W) { return (2 * W * W + 3) / 4 * 4; }
inline int vel32_yoff(int W) { return (W * W + 3) / 4 * 4; }
// red_n0: first output column whose tile may keep three slices (FP32-grade; Npad = none).
// vel_w > 0: the 2 W^2 velocity columns after the first W^2 = vel_w^2 are stored as FP32 in the
// layout above (their only consumer is an FP32 rotation); 0: every column as FP64.
cudaError_t launch_fourier_tc(const void* A, const void* Bt, const int* col_exp, int Mpad, int Npad,
                              int Kp, int n_rows, double* out, int ldc, DevStatus* st,
                              cudaStream_t s, int red_n0,
                              int group_m = 8, int vel_w = 0);
// the tensor-core kernel's bounded mbarrier wait on a barrier that never completes
cudaError_t launch_bounded_wait_check(uint32_t limit, DevStatus* st, cudaStream_t s);
// rows [n][ld] (H | dxH | dyH packed) -> three packed arrays [n][W*W]
cudaError_t launch_unpack_rows(const double* C, int64_t ld, int W, int n, double* H, double* X,
                               double* Y, cudaStream_t s);

// per-block partial sums; with kT = 0 Om is overwritten by its prefix sums over the bands
// (E must be ascending per k-point)
cudaError_t launch_ksum_partial(const double* E, double* Om, int W, int n, int n_eta,
                                int64_t eta_stride, const double* E_F, int n_EF, double kT,
                                double2* part, int k_per_block, cudaStream_t s);
cudaError_t launch_ksum_fold(const double2* part, int n_blocks, int n_out, double2* acc,
                             cudaStream_t s);
cudaError_t launch_ksum_final(const double2* acc, int n_out, double inv_Nk,
                              const DevStatus* st, double* out, cudaStream_t s);

// mixed-precision fix-up (k_ksum.cu)
cudaError_t launch_fixup_flag(const double* E, const double* Om, int W, int n, int n_eta,
                              int64_t eta_stride, const double* E_F, int n_EF, double rel,
                              int* flag, int* bin, cudaStream_t s);
cudaError_t launch_fixup_compact(const int* flag, const int* bin, int n, double frac,
                                 const KList& kl, int* pos, int64_t* kid, int* count,
                                 cudaStream_t s);
cudaError_t launch_fixup_scatter(const int* pos, int cnt, int W, int n_eta, const double* Efix,
                                 const double* Omfix, int64_t fix_eta_stride, double* E, double* Om,
                                 int64_t eta_stride, cudaStream_t s);

// k_large.cu: sorted eigenvalues E and eigenvectors Z of T by inverse iteration ([n][W][W]
// real, column m for sorted eigenvalue m; Z may be null: eigenvalues only), any W <= 128,
// at most `slots` persistent CTAs (iit_max_slots(W) fill the GPU) with
// iit_scratch_doubles(W, slots) doubles of scratch in total; then, for 64 < W <= 128,
// U = Q D Z by column blocks
constexpr int LARGE_W_MAX = 128;
int iit_max_slots(int W);
size_t iit_scratch_doubles(int W, int slots);
cudaError_t launch_iit(int W, int n, EighBufs b, double* E, double* Z, double* scratch, int slots,
                       cudaStream_t s,
                       bool rq = false);
// U: float2 [n][W][W] when f32 (formed in FP32 for the FP32 rotations), else double2
cudaError_t launch_reflect_large(int W, int n, EighBufs b, const double* Z, void* U, bool f32,
                                 cudaStream_t s);
// U = Q D Z in FP32 by blocked compact-WY products (W > 64, the FP32-rotation modes): per-k
// FP32 factors in wy (reflect_wy_scratch_bytes(W) per k-point, 16-byte aligned)
size_t reflect_wy_scratch_bytes(int W);
cudaError_t launch_reflect_wy(int W, int n, EighBufs b, const double* Z, float2* U, float2* wy,
                              cudaStream_t s);
// steps (3)-(4) as batched complex GEMMs: X, Y packed Hermitian rows of leading dimension ld;
// f32 = FP32 products.  Tbuf, Vx, Vy: n * W * W complex elements (of the product type) each.
cudaError_t launch_berry_large(const double* E, const void* U, const double* X, const double* Y,
                               int64_t ld, int W, int n, const double* etas, int n_eta, double* Om,
                               int64_t eta_stride, bool f32, void* Tbuf, void* Vx, void* Vy,
                               cudaStream_t s);

// separable Fourier sum (k_fourier_sep.cu).  box: [2h1+1][2h2+1][2h3+1] index of (R1, R2, R3)
// in the R list or -1.  Stage A once per call into A (sep_a_elems complex); per batch the
// pairs p0 .. p0+np-1 (pair = j2 N3 + j3) times the planes j1a .. j1a+np1-1: B and By hold
// np * sep_b_elems_per_pair complex each, Hp / Xp / Yp receive the packed FP64 matrices of the
// batch's k-points in pair-major order (local t -> pair p0 + t / np1, plane j1a + t % np1).
size_t sep_a_elems(const SepBox& sb, int W, int N3);
size_t sep_b_elems_per_pair(const SepBox& sb, int W);
cudaError_t launch_sep_stage_a(const double2* H_R, const int* box, const SepBox& sb, int W,
                               const Mesh& mesh, const double2* tab, int off3, double2* A,
                               cudaStream_t s);
cudaError_t launch_sep_batch(const double2* A, const SepBox& sb, int W, const Mesh& mesh,
                             const double2* tab, const int tab_off[3], int64_t p0, int np,
                             int j1a, int np1, double2* B, double2* By, double* Hp, double* Xp,
                             double* Yp, cudaStream_t s);

// T = X U with X packed Hermitian rows (leading dimension ld), FP64
cudaError_t launch_herm_u(const double* X, int64_t ld, const double2* U, double2* T, int W, int n,
                          cudaStream_t s);

// reverse mode (k_grad.cu)
cudaError_t launch_zgemm_batched(bool hA, bool hB, bool acc, const double2* A, const double2* B,
                                 double2* C, int W, int n, cudaStream_t s);
cudaError_t launch_grad_pairs(const double* E, const double2* vx, const double2* vy, int W, int n,
                              const double* g, const double* E_F, int n_EF, const double* etas,
                              int n_eta, double kT, double inv_Nk, double2* vbx, double2* vby,
                              double* Ebar, cudaStream_t s);
cudaError_t launch_grad_gp(const double* E, const double* Ebar, const double2* N, int W, int n,
                           double grad_eps, double2* Gp, cudaStream_t s);
cudaError_t launch_pack3(const double2* A0, const double2* A1, const double2* A2, int W, int n,
                         double* out, cudaStream_t s);
cudaError_t launch_grad_coef(const Model& md, const Mesh& mesh, const KList& kl, int ldc,
                             double* Coef, cudaStream_t s);
cudaError_t launch_grad_fourier_t(const double* Coef, int ldc, const double* Mbar, int M, int N,
                                  int K, double* Gacc, cudaStream_t s);
cudaError_t launch_grad_finalize(const double* Gacc, const int* pairs, const int* Rh, int idx0,
                                 int N_h, int W, double2* G, cudaStream_t s);

size_t tridiag_smem(int W);
size_t tridiag_df_smem(int W);
size_t backtransform_smem(int W);
size_t ql_smem(int W);
size_t berry_fp64_smem(int W, int n_eta);

}  // namespace kubo
