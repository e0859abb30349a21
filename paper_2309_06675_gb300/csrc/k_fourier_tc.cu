// Step (1) of List 1/2 on the 5th-generation tensor cores.
//
// The three outputs of the Fourier sum share one real coefficient row per k-point,
//   coef(k) = [cos th_0, sin th_0, cos th_1, sin th_1, ..., cos th_{N_h-1}, sin th_{N_h-1}, 1],
// once the derivative weights are moved into the basis:
//   H   = sum_h c_h A_h + s_h B_h + P0
//   d_a H = sum_h c_h (R_h,a B_h) + s_h (-R_h,a A_h)
// so the whole step is ONE dense contraction C[n_k x 3W^2] = Coef[n_k x N_R] . Basis[N_R x 3W^2]
// with the stacked basis [B^H | B^X | B^Y].
//
// Arithmetic: fixed-point slicing (the Ozaki scheme) on BF16 MMAs.  Every coefficient
// (|c| <= 1) and every basis entry (scaled by 2^-e_n, e_n the exponent of its column's
// largest magnitude) is written as x = sum_{i<4} s_i 2^(-7-8i) with integer slices
// |s_i| <= 128, exact in BF16.  A product of slices is an integer below 2^14, so the sum of one
// 64-wide K block of all slice pairs of one level l = i + j (at most 4 pairs) stays an integer
// below 2^22 and is EXACT in the FP32 tensor-memory accumulator, whatever rounding the tensor
// core applies.  The epilogue converts each level to an integer (exact), accumulates the K
// blocks and levels exactly in one int64 per column, and scales once in FP64:
//   C = 2^e_n sum_l 2^(-14-8l) I_l   (levels l <= 3: 10 slice pairs).
// The result carries ~31 fractional bits relative to the operand scales (phases to ~2^-46,
// FP64 basis), versus ~24 for a split-BF16 product with FP32 accumulation.
//
// Kernels:
//   basis_scale_kernel  once per call: column exponents e_n of the stacked basis
//   basis_slice_kernel  once per call: stacked basis -> Bt[4 slices][Npad][Kp] (K-major, bf16)
//   coef_slice_kernel   per batch: phases with exact integer argument reduction, the three
//                       twiddles multiplied in FP32 pairs (~2^-46) -> A[4][Mpad][Kp]
//   fourier_tc_kernel   per batch: tcgen05.mma (kind::f16, M=128, K=16; one MMA per A slice
//                       against the stacked B slices, N = 64 x (slices - i)), operands staged
//                       by TMA (128-byte swizzle, 2-stage mbarrier pipeline), 4 level
//                       accumulators x 2 buffers filling the 512 TMEM columns, integer
//                       epilogue, FP64 rows in HBM; persistent (one CTA per SM over the
//                       tiles, the epilogue of a tile overlapping the next tile's MMAs).
//
// Every mbarrier wait is bounded; on timeout the CTA records ST_TIMEOUT, drains its own
// copies (bounded), frees its TMEM and returns.
#include <algorithm>
#include <climits>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "kubo_internal.cuh"
#include "tc_ptx.cuh"

namespace kubo {

namespace {

using namespace tc;

constexpr int BM = 128;           // k-points per tile (UMMA M)
constexpr int BN = 64;            // output columns per tile (UMMA N)
constexpr int BK = 64;            // K per stage (one 128-byte swizzle row of bf16) = one exact chunk
constexpr int NSTAGE = 2;
constexpr int NSLICE = 4;         // slices per operand: 7 + 3 x 8 = 31 fractional bits
constexpr int NLEVEL = 4;         // levels l = i + j <= 3 kept: 10 slice pairs
constexpr int NACC = 2;           // level-accumulator sets in flight (double buffer)
constexpr int DRAIN = 4;          // K blocks summed in TMEM before the epilogue drains a set:
                                  // 4 blocks x 4 pairs x 64 x 2^14 = 2^24, still exact in FP32
constexpr int TILE_A_BYTES = BM * BK * 2;            // 16 KB per slice
constexpr int TILE_B_BYTES = BN * BK * 2;            // 8 KB per slice
constexpr int STAGE_BYTES = NSLICE * (TILE_A_BYTES + TILE_B_BYTES);   // 96 KB
constexpr int TC_THREADS = 320;                      // 10 warps: TMA, MMA, 8 epilogue
constexpr int EPI_THREADS = TC_THREADS - 64;         // 2 per TMEM lane quarter, 32 columns each
constexpr int EPI_COLS = BN / 2;
constexpr int TMEM_COLS = 512;                       // = NACC * NLEVEL * BN

// PTX wrappers: tc_ptx.cuh

// Failure-detection check: the same bounded wait on a barrier that nothing ever completes.
// Thread 0 gives up after `limit` tries and records ST_TIMEOUT; the kernel then returns, so
// the context stays usable.
__global__ void bounded_wait_check_kernel(uint32_t limit, DevStatus* st) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0, limit)) atomicOr(&st->bits, ST_TIMEOUT);
}

// Instruction descriptor: kind::f16, A = B = BF16, D = F32, both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

// Fixed-point slices of x 2^-e (|x| <= 2^e): x 2^-e = sum_i s_i 2^(-7-8i) + O(2^-32),
// |s_i| <= 128, from the FP64 bit pattern with integer operations (fixed31_ll, slice4_bf16 in
// tc_ptx.cuh): no FP64 instruction, which GB300 issues at 1/64 of the FP32 rate.
__device__ __forceinline__ void slice_scaled(double x, int e, __nv_bfloat16 (&sl)[NSLICE]) {
  slice4_bf16(fixed31_ll(x, e), sl);
}

// ------------------------------------------------------------------ operand preparation
// value of the stacked basis at (output column n < 3 W^2, K index k)
__device__ __forceinline__ double stacked_basis(const double* __restrict__ Bp,
                                                const int* __restrict__ Rh, int N_h, int WW, int n,
                                                int k) {
  const int alpha = n / WW, q = n % WW;
  if (k < 2 * N_h) {
    const int h = k >> 1;
    const bool is_sin = k & 1;
    const double Ah = Bp[(size_t)(1 + 2 * h) * WW + q];
    const double Bh = Bp[(size_t)(2 + 2 * h) * WW + q];
    if (alpha == 0) return is_sin ? Bh : Ah;
    const double r = (double)Rh[3 * h + (alpha - 1)];
    return is_sin ? -r * Ah : r * Bh;
  }
  if (k == 2 * N_h && alpha == 0) return Bp[q];
  return 0.0;
}

// e[n]: exponent with max_k |basis(n, k)| < 2^e[n] (0 for an all-zero column).  Block: 128
// columns (x, coalesced) x SCALE_KY slices of K (y), maxima combined in shared memory.
constexpr int SCALE_KY = 8;
__global__ void basis_scale_kernel(const double* __restrict__ Bp, const int* __restrict__ Rh,
                                   int N_h, int W, int Npad, int* __restrict__ e) {
  __shared__ double red[SCALE_KY][128];
  const int WW = W * W;
  const int n = blockIdx.x * 128 + threadIdx.x;
  double mx = 0.0;
  if (n < 3 * WW)
    for (int k = threadIdx.y; k <= 2 * N_h; k += SCALE_KY)
      mx = fmax(mx, fabs(stacked_basis(Bp, Rh, N_h, WW, n, k)));
  red[threadIdx.y][threadIdx.x] = mx;
  __syncthreads();
  if (threadIdx.y == 0 && n < Npad) {
    for (int y = 1; y < SCALE_KY; ++y) mx = fmax(mx, red[y][threadIdx.x]);
    int ex = 0;
    if (mx > 0.0) frexp(mx, &ex);   // mx = f 2^ex, f in [0.5, 1)
    e[n] = ex;
  }
}

// Bt[s][n][k] (n < Npad rows, k < Kp contiguous): slices of basis(n, k) * 2^-e[n]
__global__ void basis_slice_kernel(const double* __restrict__ Bp, const int* __restrict__ Rh,
                                   const int* __restrict__ e, int N_h, int W, int Npad, int Kp,
                                   __nv_bfloat16* __restrict__ Bt) {
  const int WW = W * W;
  const int64_t plane = (int64_t)Npad * Kp;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < plane;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(t / Kp), k = (int)(t % Kp);
    double v = 0.0;
    if (n < 3 * WW && k <= 2 * N_h) v = stacked_basis(Bp, Rh, N_h, WW, n, k);
    __nv_bfloat16 sl[NSLICE];
    slice_scaled(v, n < 3 * WW ? e[n] : 0, sl);   // |v| < 2^e[n] by construction
#pragma unroll
    for (int i = 0; i < NSLICE; ++i) Bt[i * plane + t] = sl[i];
  }
}

// ---- FP32-pair (double-float) arithmetic for the phases: ~2^-46 relative, on the FP32 pipe
struct Pf {
  float h, l;
};
// exact h + l = a + b (Knuth's TwoSum)
__device__ __forceinline__ Pf pf_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  return Pf{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp))};
}
__device__ __forceinline__ Pf pf_norm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return Pf{h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ Pf pf_mul(Pf a, Pf b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);   // the rounding error of p, exactly
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return pf_norm(p, e);
}
__device__ __forceinline__ Pf pf_add(Pf a, Pf b) {
  const Pf s = pf_two_sum(a.h, b.h);
  return pf_norm(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ Pf pf_neg(Pf a) { return Pf{-a.h, -a.l}; }
// (a.re + i a.im)(b.re + i b.im), operands as float4 (re_h, re_l, im_h, im_l)
__device__ __forceinline__ float4 pf_cmul(const float4& a, const float4& b) {
  const Pf ar{a.x, a.y}, ai{a.z, a.w}, br{b.x, b.y}, bi{b.z, b.w};
  const Pf re = pf_add(pf_mul(ar, br), pf_neg(pf_mul(ai, bi)));
  const Pf im = pf_add(pf_mul(ar, bi), pf_mul(ai, br));
  return make_float4(re.h, re.l, im.h, im.l);
}
// v 2^62 as an integer for an FP32 v with |v| <= 2 (bits below 2^-62 dropped), from the bits
__device__ __forceinline__ long long f32_fix62(float v) {
  const uint32_t b = __float_as_uint(v);
  const int ex = (int)((b >> 23) & 0xFFu);
  if (ex == 0) return 0;   // zero or subnormal (below 2^-126)
  const long long m = (long long)((b & 0x7FFFFFu) | 0x800000u);
  const int sh = ex - 150 + 62;   // v 2^62 = m 2^(ex - 150 + 62)
  const long long mag = sh >= 0 ? (m << sh) : (sh > -40 ? (m >> -sh) : 0);
  return (b >> 31) ? -mag : mag;
}
// round((h + l) 2^31) for |h + l| <= 1 + 2^-40: the pair's parts as 62-bit fixed-point
// integers, summed exactly, rounded to 31 fractional bits (ties away from zero)
__device__ __forceinline__ long long pf_fixed31(float h, float l) {
  const long long q = f32_fix62(h) + f32_fix62(l);
  const long long aq = q < 0 ? -q : q;
  const long long r = (aq + (1ll << 30)) >> 31;
  return q < 0 ? -r : r;
}
// x mod d in [0, d) for |x| < 2^32, by the multiply-high division
__device__ __forceinline__ int posmod(long long x, const FastDiv& f) {
  const unsigned long long ax = x < 0 ? (unsigned long long)(-x) : (unsigned long long)x;
  uint32_t r;
  if (ax < 0x100000000ull) {
    const uint32_t a = (uint32_t)ax;
    r = a - f.div(a) * f.d;
  } else {
    r = (uint32_t)(ax % f.d);
  }
  return (x < 0 && r) ? (int)(f.d - r) : (int)r;
}

// A[s][m][k] for m < Mpad (rows >= n are zero), k < Kp.  Persistent CTAs over the rows
// (k-points); a row's mesh coordinates once per row, then per (m, h) the three per-axis
// twiddles by exact integer argument reduction (multiply-high modulo) and their product as two
// complex multiplies in FP32 pairs (~2^-46: the FP64 products would run on the FP64 pipe, at
// 1/64 of the FP32 rate), rounded to 31 fractional bits from the pair with integer operations.
constexpr int CS_NT = 256;
__global__ void __launch_bounds__(CS_NT) coef_slice_kernel(Model md, Mesh mesh, KList kl, int Mpad,
                                                           int Kp, __nv_bfloat16* __restrict__ A) {
  const int npair = Kp / 2;
  const int64_t plane = (int64_t)Mpad * Kp;
  const FastDiv f1((uint32_t)mesh.N1), f2((uint32_t)mesh.N2), f3((uint32_t)mesh.N3);
  const float4* t1 = md.tab_df + md.tab_off[0];
  const float4* t2 = md.tab_df + md.tab_off[1];
  const float4* t3 = md.tab_df + md.tab_off[2];
  __shared__ int s_j[3];
  for (int m = blockIdx.x; m < Mpad; m += gridDim.x) {
    const bool live = m < kl.n;
    if (threadIdx.x == 0 && live) mesh_coords(mesh, klist_get(kl, m), s_j[0], s_j[1], s_j[2]);
    __syncthreads();
    const int j1 = s_j[0], j2 = s_j[1], j3 = s_j[2];
    for (int h = threadIdx.x; h < npair; h += CS_NT) {
      long long qc = 0, qs = 0;
      if (live) {
        if (h < md.N_h) {
          const int* r = md.Rh + 3 * h;
          const float4 e = pf_cmul(pf_cmul(t1[posmod((long long)j1 * r[0], f1)],
                                           t2[posmod((long long)j2 * r[1], f2)]),
                                   t3[posmod((long long)j3 * r[2], f3)]);
          qc = pf_fixed31(e.x, e.y);
          qs = pf_fixed31(e.z, e.w);
        } else if (h == md.N_h) {
          qc = 1ll << 31;   // the R = 0 term (column 2 N_h); its partner column stays 0
        }
      }
      __nv_bfloat16 cs[NSLICE], ss[NSLICE];
      slice4_bf16(qc, cs);
      slice4_bf16(qs, ss);
      const int64_t o = (int64_t)m * Kp + 2 * h;
#pragma unroll
      for (int i = 0; i < NSLICE; ++i)
        *reinterpret_cast<__nv_bfloat162*>(A + i * plane + o) = __halves2bfloat162(cs[i], ss[i]);
    }
    __syncthreads();   // s_j is rewritten for the next row
  }
}

// ------------------------------------------------------------------ the tcgen05 GEMM
// Persistent: one CTA per SM walks the tiles tau = blockIdx.x, + gridDim.x, ... of the column
// tiles nt0 .. nt0 + ntc - 1 (grouped rasterisation, below).  The K-block counter of the
// TMA / MMA pipeline and the drain-group counter of the two TMEM accumulator sets run across
// tiles, so the epilogue of one tile (its last drain, the FP64 conversion and the stores)
// overlaps the loads and MMAs of the next, and TMEM, barriers and pipeline fill are paid once
// per SM.  out: FP64 [n rows][ldc], rows >= n_rows not written.
// NS = slices per operand kept: 4 (levels i + j <= 3, 10 slice pairs, ~31 fractional bits) or
// 3 (levels <= 2, 6 pairs, ~23 bits: for the velocity columns when their only consumer is the
// FP32 rotation, whose own input rounding is 2^-24).
template <int NS>
__global__ void __launch_bounds__(TC_THREADS, 1)
    fourier_tc_kernel(const __grid_constant__ CUtensorMap mapA,
                      const __grid_constant__ CUtensorMap mapB, const int* __restrict__ col_exp,
                      int Mpad, int Npad, int nkb, int n_rows, double* __restrict__ out, int ldc,
                      DevStatus* st, int nt0, int ntc, int group_m, int vel0, int vw2,
                      int vx0, int vyoff) {
  constexpr int NLEV = NS;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[NSTAGE], empty_bar[NSTAGE];
  __shared__ __align__(8) uint64_t acc_full[NACC], acc_empty[NACC], done_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_mt = Mpad / BM, n_tiles = n_mt * ntc;
  const int groups_per_tile = (nkb + DRAIN - 1) / DRAIN;
  // grouped rasterisation: group_m consecutive M tiles per column tile, so one B tile serves
  // several tiles in a row and the group's A tiles stay resident in L2 across column tiles
  auto tile_origin = [&](int id, int& m0, int& n0) {
    const int per_group = group_m * ntc;
    const int grp = id / per_group;
    const int gm0 = grp * group_m;
    const int gsz = min(group_m, n_mt - gm0);
    const int in = id - grp * per_group;
    n0 = (nt0 + in / gsz) * BN;
    m0 = (gm0 + in % gsz) * BM;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int a = 0; a < NACC; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], EPI_THREADS);   // every epilogue thread arrives
    }
    mbar_init(&done_bar, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;

  auto stageA = [&](int s, int sl) { return base + (size_t)s * STAGE_BYTES + (size_t)sl * TILE_A_BYTES; };
  auto stageB = [&](int s, int sl) {
    return base + (size_t)s * STAGE_BYTES + NSLICE * TILE_A_BYTES + (size_t)sl * TILE_B_BYTES;
  };

  if (warp == 0) {
    // ---------------- TMA producer (g: K blocks issued by this CTA over all its tiles)
    if (lane == 0) {
      int g = 0;
      for (int id = blockIdx.x; id < n_tiles && !abort_sh; id += gridDim.x) {
        int m0, n0;
        tile_origin(id, m0, n0);
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int s = g % NSTAGE;
          if (abort_sh) break;
          if (g >= NSTAGE && !mbar_wait(&empty_bar[s], ((uint32_t)(g / NSTAGE) & 1u) ^ 1u)) {
            atomicOr(&st->bits, ST_TIMEOUT);
            abort_sh = 1;
            break;
          }
          mbar_expect_tx(&full_bar[s], (uint32_t)NS * (TILE_A_BYTES + TILE_B_BYTES));
          for (int sl = 0; sl < NS; ++sl)
            tma_load_2d(stageA(s, sl), &mapA, &full_bar[s], kb * BK, sl * Mpad + m0);
          for (int sl = 0; sl < NS; ++sl)
            tma_load_2d(stageB(s, sl), &mapB, &full_bar[s], kb * BK, sl * Npad + n0);
        }
      }
      // drain: every issued stage's copies must have landed before the CTA may exit
      for (int q = (g > NSTAGE ? g - NSTAGE : 0); q < g; ++q)
        mbar_wait(&full_bar[q % NSTAGE], (uint32_t)(q / NSTAGE) & 1u);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: drain group G (global) accumulates into set G % NACC
    if (lane == 0) {
      int g = 0, G = 0;
      for (int id = blockIdx.x; id < n_tiles && !abort_sh; id += gridDim.x) {
        for (int kb = 0; kb < nkb && !abort_sh; ++kb, ++g) {
          const int s = g % NSTAGE;
          const bool first = kb % DRAIN == 0;
          const bool last = kb % DRAIN == DRAIN - 1 || kb == nkb - 1;
          const int a = G % NACC;
          if (first && G >= NACC && !mbar_wait(&acc_empty[a], (uint32_t)(G / NACC - 1) & 1u)) {
            atomicOr(&st->bits, ST_TIMEOUT);
            abort_sh = 1;
            break;
          }
          if (!mbar_wait(&full_bar[s], (uint32_t)(g / NSTAGE) & 1u)) {
            atomicOr(&st->bits, ST_TIMEOUT);
            abort_sh = 1;
            break;
          }
          tc_fence_after();
          // One MMA per A slice i against the stacked B slices 0 .. NS-1-i: the B tiles of a
          // stage are consecutive 8-row-group runs of one 128-byte-swizzled K-major operand,
          // so rows j*BN .. j*BN+BN-1 of the N = (NS-i) BN operand are slice j, and the
          // accumulator columns they write are those of level i + j (levels are contiguous
          // within a set).  A_i is read from shared memory once per K step instead of once per
          // pair; A_0 comes first and initialises every level of a drain group.
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t db = umma_desc_sw128(smem_u32(stageB(s, 0)) + kk * 32);
#pragma unroll
            for (int i = 0; i < NS; ++i) {
              const uint32_t acc = (i > 0 || !first || kk > 0) ? 1u : 0u;
              const uint64_t da = umma_desc_sw128(smem_u32(stageA(s, i)) + kk * 32);
              umma_bf16(tmem + (uint32_t)((a * NLEVEL + i) * BN), da, db, idesc_n((NS - i) * BN), acc);
            }
          }
          umma_commit(&empty_bar[s]);   // stage free once these MMAs have read it
          if (last) {
            umma_commit(&acc_full[a]);  // level sums of this drain group complete
            ++G;
          }
        }
      }
      umma_commit(&done_bar);         // all issued MMAs complete
    }
  } else {
    // ---------------- epilogue: warps 2..9; warp w owns TMEM lanes 32 (w % 4) .. + 31 (the
    // lanes a warp may access) and the column half (w - 2) / 4 of the tile
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const int c_lo = ((warp - 2) >> 2) * EPI_COLS;
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
    bool ok = true;
    int G = 0;
    for (int id = blockIdx.x; id < n_tiles && ok; id += gridDim.x) {
      int m0, n0;
      tile_origin(id, m0, n0);
      // One exact integer per column: sum over drain groups and levels of I_l 2^(32 - 8 l).  A
      // group's level sum is at most 2^24 in magnitude, so the total stays below 2^57.
      long long isum[EPI_COLS];
#pragma unroll
      for (int j = 0; j < EPI_COLS; ++j) isum[j] = 0;
      for (int gi = 0; gi < groups_per_tile; ++gi, ++G) {
        const int a = G % NACC;
        ok = mbar_wait(&acc_full[a], (uint32_t)(G / NACC) & 1u);
        ok = __all_sync(0xffffffffu, ok && !abort_sh);   // tcgen05.ld is warp-collective
        if (!ok) break;
        tc_fence_after();
        // NLEV x 2 loads of 16 columns, double-buffered: the conversion of one buffer overlaps
        // the TMEM load of the next
        constexpr int NQ = EPI_COLS / 16, NSTEP = NLEV * NQ;
        uint32_t rb[2][16];
        const uint32_t set_addr = lane_addr + (uint32_t)(a * NLEVEL * BN + c_lo);
        tmem_ld16_async(set_addr, rb[0]);
        tmem_wait_ld16(rb[0]);
#pragma unroll
        for (int q = 0; q < NSTEP; ++q) {
          const int l = q / NQ, c0 = (q % NQ) * 16;
          if (q + 1 < NSTEP)
            tmem_ld16_async(set_addr + (uint32_t)(((q + 1) / NQ) * BN + ((q + 1) % NQ) * 16), rb[(q + 1) & 1]);
#pragma unroll
          for (int j = 0; j < 16; ++j)
            isum[c0 + j] += (long long)__float2int_rn(__uint_as_float(rb[q & 1][j])) << (32 - 8 * l);
          if (q + 1 < NSTEP) tmem_wait_ld16(rb[(q + 1) & 1]);
        }
        tc_fence_before();
        mbar_arrive(&acc_empty[a]);
      }
      if (!ok) break;
      const int grow = m0 + row;
      if (grow < n_rows) {
        // C = 2^e_n * isum * 2^(-14 - 32): a power-of-two scale, exact apart from the final
        // rounding of the 57-bit integer to FP64
        double* dst = out + (size_t)grow * ldc + n0 + c_lo;
        const int* ce = col_exp + n0 + c_lo;
        if (n0 + c_lo + EPI_COLS <= vel0) {
#pragma unroll
          for (int j = 0; j < EPI_COLS; j += 2) {
            const double s0 = __longlong_as_double((long long)(1023 - 46 + ce[j]) << 52);
            const double s1 = __longlong_as_double((long long)(1023 - 46 + ce[j + 1]) << 52);
            *reinterpret_cast<double2*>(dst + j) =
                make_double2((double)isum[j] * s0, (double)isum[j + 1] * s1);
          }
        } else {
          // velocity columns as FP32 (vel32_x0 layout of the row), padding columns dropped
          // (pairs: even W^2 keeps both entries of a pair in one row, 8-byte aligned)
          float* o32 = reinterpret_cast<float*>(out) + (size_t)grow * 2 * ldc;
#pragma unroll
          for (int j = 0; j < EPI_COLS; j += 2) {
            const int cc = n0 + c_lo + j;
            const double v0 =
                (double)isum[j] * __longlong_as_double((long long)(1023 - 46 + ce[j]) << 52);
            const double v1 =
                (double)isum[j + 1] * __longlong_as_double((long long)(1023 - 46 + ce[j + 1]) << 52);
            if (!(vw2 & 1) && cc >= vel0 && cc + 1 < vel0 + 2 * vw2) {
              const int u = cc - vel0;
              *reinterpret_cast<float2*>(o32 + (u < vw2 ? vx0 + u : vx0 + vyoff + (u - vw2))) =
                  make_float2((float)v0, (float)v1);
            } else {
#pragma unroll
              for (int q = 0; q < 2; ++q) {
                const int c2 = cc + q;
                const double v = q ? v1 : v0;
                if (c2 < vel0) {
                  dst[j + q] = v;
                } else if (c2 < vel0 + 2 * vw2) {
                  const int u = c2 - vel0;
                  o32[u < vw2 ? vx0 + u : vx0 + vyoff + (u - vw2)] = (float)v;
                }
              }
            }
          }
        }
      }
    }
    if (!ok) {
      atomicOr(&st->bits, ST_TIMEOUT);
      abort_sh = 1;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    if (lane == 0) mbar_wait(&done_bar, 0);   // no MMA may still be writing TMEM
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// ------------------------------------------------------------------ host helpers
PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

bool encode_2d(CUtensorMap* map, const void* gptr, uint64_t inner, uint64_t outer, uint32_t box_inner,
               uint32_t box_outer) {
  auto enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {inner * 2};   // bytes between rows
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(gptr), dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int grid_for(int64_t total, int threads) {
  int64_t b = (total + threads - 1) / threads;
  if (b > 152 * 64) b = 152 * 64;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

int tc_pad_m(int n) { return (n + BM - 1) / BM * BM; }
int tc_pad_n(int W) { return (3 * W * W + BN - 1) / BN * BN; }
int tc_pad_k(int N_R) { return (N_R + BK - 1) / BK * BK; }
int tc_slices() { return NSLICE; }

cudaError_t launch_bounded_wait_check(uint32_t limit, DevStatus* st, cudaStream_t s) {
  bounded_wait_check_kernel<<<1, 32, 0, s>>>(limit, st);
  return cudaGetLastError();
}
size_t fourier_tc_smem() { return (size_t)NSTAGE * STAGE_BYTES + 1024; }

cudaError_t launch_basis_split(const double* Bp, const int* Rh, int N_h, int W, int Npad, int Kp,
                               int* col_exp, void* Bt, cudaStream_t s) {
  basis_scale_kernel<<<(Npad + 127) / 128, dim3(128, SCALE_KY), 0, s>>>(Bp, Rh, N_h, W, Npad, col_exp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  basis_slice_kernel<<<grid_for((int64_t)Npad * Kp, 256), 256, 0, s>>>(Bp, Rh, col_exp, N_h, W, Npad,
                                                                        Kp, (__nv_bfloat16*)Bt);
  return cudaGetLastError();
}

cudaError_t launch_coef_split(const Model& md, const Mesh& mesh, const KList& kl, int Mpad, int Kp,
                              void* A, cudaStream_t s) {
  int dev = 0, nsm = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::max(1, std::min(Mpad, 8 * std::max(nsm, 1)));   // persistent over the rows
  coef_slice_kernel<<<grid, CS_NT, 0, s>>>(md, mesh, kl, Mpad, Kp, (__nv_bfloat16*)A);
  return cudaGetLastError();
}

cudaError_t launch_fourier_tc(const void* A, const void* Bt, const int* col_exp, int Mpad, int Npad,
                              int Kp, int n_rows, double* out, int ldc, DevStatus* st,
                              cudaStream_t s, int red_n0, int group_m, int vel_w) {
  if (n_rows <= 0) return cudaSuccess;
  if (Mpad % BM || Npad % BN || Kp % BK || ldc % 2) return cudaErrorInvalidValue;
  if (group_m < 1 || group_m > 64) return cudaErrorInvalidValue;
  const int vw2 = vel_w * vel_w;
  if (vel_w < 0 || (vel_w > 0 && (3 * vw2 > Npad ||
                                  vel32_x0(vel_w) + vel32_yoff(vel_w) + vw2 > 2 * ldc)))
    return cudaErrorInvalidValue;
  const int vel0 = vel_w > 0 ? vw2 : INT_MAX;
  CUtensorMap mA, mB;
  if (!encode_2d(&mA, A, (uint64_t)Kp, (uint64_t)NSLICE * Mpad, BK, BM)) return cudaErrorInvalidValue;
  if (!encode_2d(&mB, Bt, (uint64_t)Kp, (uint64_t)NSLICE * Npad, BK, BN)) return cudaErrorInvalidValue;
  const size_t sm = fourier_tc_smem();
  const int nt = Npad / BN;
  // first column tile that lies entirely at or after red_n0
  const int rt = std::min(nt, (std::max(red_n0, 0) + BN - 1) / BN);
  auto go = [&](auto kern, int t0, int tc, int gm) -> cudaError_t {
    if (tc <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::min(tc * (Mpad / BM), std::max(nsm, 1));   // persistent: one per SM
    kern<<<grid, TC_THREADS, sm, s>>>(mA, mB, col_exp, Mpad, Npad, Kp / BK, n_rows, out, ldc, st,
                                      t0, tc, gm, vel0, vw2, vel32_x0(vel_w),
                                      vel32_yoff(vel_w));
    return cudaGetLastError();
  };
  // M tiles rasterised together: group_m for the H columns, four times that (at most 64) for the
  // velocity columns, whose A tiles are three-quarters the size (3 slices) and whose basis is
  // half again as large (8,192 vs 4,096 columns at W = 64).  Measured DRAM reads per 65,536-k
  // launch at W = 64, N_R = 1331 (H / velocity kernel): groups of 8: 2.50 / 3.93 GB; of 32:
  // 3.54 / 1.85 GB; of 1: 2.85 / 5.58 GB -- the same time in every case (the kernels are bound
  // by their operand intake, not by DRAM).
  cudaError_t e = go(fourier_tc_kernel<NSLICE>, 0, rt, group_m);
  if (e != cudaSuccess) return e;
  return go(fourier_tc_kernel<NSLICE - 1>, rt, nt - rt, std::min(64, 4 * group_m));
}

}  // namespace kubo
