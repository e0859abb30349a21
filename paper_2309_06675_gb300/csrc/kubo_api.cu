// C ABI of libkubo (include/kubo.h): argument validation, analysis of the R set, workspace
// planning and the batched k-point pipeline (the paper's List 2 loop over batches).
#include <algorithm>
#include <atomic>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "kubo_internal.cuh"

using namespace kubo;

namespace {

constexpr int MAX_W = LARGE_W_MAX;
constexpr int SMALL_W_MAX = 64;      // beyond: the multi-pass eigenvector / rotation kernels
constexpr int MAX_ETA = 8;
constexpr int KSUM_KPB = 32;         // k-points per deterministic k-sum block (at least)
constexpr size_t KSUM_PART_BYTES = (size_t)256 << 20;   // cap on the per-block partials
// mixed precision: share of each batch (largest ||Omega(k)||_inf) redone in FP64
constexpr double kFixupSpikyFraction = 0.005;
constexpr size_t ALIGN = 256;

// ------------------------------------------------------------------ options
kubo_options defaults() {
  kubo_options o;
  std::memset(&o, 0, sizeof(o));
  o.precision = KUBO_FP64;
  return o;
}

// FP32-grade rotation kernels for W <= 64 (kubo_options.rotation_tc: 0 = automatic, 1 = exact
// slices, 2 = SIMT, 3 = 3xTF32)
enum { ROT_TF32 = 0, ROT_EXACT_SLICES = 1, ROT_SIMT = 2 };

// The automatic choice: the 3xTF32 tensor-core kernel pads every k-point to W = 64, so it is
// taken only above W = 40, where it (with its separate U assembly) is at least as fast as the
// FP32 FMA kernel with the assembly inside (eigenvector + rotation stages on 65,536 k-points:
// W = 40 25.0 vs 25.2 ms, W = 48 28.6 vs 30.6, W = 64 36.9 vs 43.5; W = 32 17.6 vs 9.6).
int rotation_kernel(int option, int W, bool unpadded) {
  if (unpadded) return ROT_SIMT;   // the padding ablation concerns the SIMT kernel's layout
  switch (option) {
    case 1: return ROT_EXACT_SLICES;
    case 2: return ROT_SIMT;
    case 3: return ROT_TF32;
    default: return W > 40 ? ROT_TF32 : ROT_SIMT;
  }
}

// ------------------------------------------------------------------ R set
struct RInfo {
  std::vector<int> neg;     // [N_R] index of -R
  std::vector<int> pairs;   // [N_h][2] (index of R_h, index of -R_h), canonical R_h
  std::vector<int> Rh;      // [N_h][3]
  int idx0 = -1;
  int N_h = 0;
  std::vector<int> box;     // separable Fourier sum: bounding-box index table (or empty)
};

kubo_status analyze_R(const int32_t* R, int N_R, RInfo& info) {
  std::map<std::array<int, 3>, int> idx;
  for (int i = 0; i < N_R; ++i) {
    std::array<int, 3> key{R[3 * i], R[3 * i + 1], R[3 * i + 2]};
    if (!idx.emplace(key, i).second) return KUBO_ERR_R_NOT_CLOSED;   // duplicate
  }
  auto z = idx.find({0, 0, 0});
  if (z == idx.end()) return KUBO_ERR_R_NOT_CLOSED;
  info.idx0 = z->second;
  info.neg.assign(N_R, -1);
  for (int i = 0; i < N_R; ++i) {
    auto it = idx.find({-R[3 * i], -R[3 * i + 1], -R[3 * i + 2]});
    if (it == idx.end()) return KUBO_ERR_R_NOT_CLOSED;
    info.neg[i] = it->second;
    const int r0 = R[3 * i], r1 = R[3 * i + 1], r2 = R[3 * i + 2];
    const bool canon = r0 > 0 || (r0 == 0 && (r1 > 0 || (r1 == 0 && r2 > 0)));
    if (canon) {
      info.pairs.push_back(i);
      info.pairs.push_back(it->second);
      info.Rh.push_back(r0);
      info.Rh.push_back(r1);
      info.Rh.push_back(r2);
    }
  }
  info.N_h = (int)info.pairs.size() / 2;
  if (1 + 2 * info.N_h != N_R) return KUBO_ERR_R_NOT_CLOSED;
  return KUBO_OK;
}

// ------------------------------------------------------------------ workspace plan
struct Bump {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t o = off;
    off += (bytes + ALIGN - 1) / ALIGN * ALIGN;
    return o;
  }
};

// precision modes whose step (1) runs on the tensor cores / whose step (3) runs in FP32 /
// whose eigensolver runs in double-float
bool tc_fourier(int prec) {
  return prec == KUBO_MIXED || prec == KUBO_MIXED_FOURIER || prec == KUBO_MIXED_DF;
}
bool f32_rotation(int prec) {
  return prec == KUBO_MIXED || prec == KUBO_MIXED_ROTATION || prec == KUBO_MIXED_DF;
}
bool df_eigh(int prec) { return prec == KUBO_MIXED_DF; }
// MIXED: the QL iteration runs in double-float as well, but only to supply the shifts of the
// FP64 inverse iteration; the eigenvalues reported are the FP64 Rayleigh quotients of its
// eigenvectors
// (kubo_options.ql_fp64 keeps the MIXED mode's QL in FP64 and its eigenvalues)
bool df_ql(int prec, bool ql_fp64) {
  return (prec == KUBO_MIXED && !ql_fp64) || prec == KUBO_MIXED_DF;
}
bool rq_eigenvalues(int prec, bool ql_fp64) { return prec == KUBO_MIXED && !ql_fp64; }

// Power-of-two exponent s that brings max |H(R)| into [1, 2) when it lies outside
// [2^-20, 2^20] (0 otherwise, and for zero or non-finite maxima).  S(E_F) is homogeneous of
// degree zero in (H, eta, E, kT), and scaling by 2^s is exact, so the FP32 steps see O(1)
// magnitudes whatever the input's units.
int range_exponent(double mx) {
  if (!(mx > 0.0) || !std::isfinite(mx)) return 0;
  int e = 0;
  std::frexp(mx, &e);   // mx = f 2^e, f in [0.5, 1)
  const int lg = e - 1; // mx in [2^lg, 2^(lg+1))
  if (lg >= -20 && lg <= 20) return 0;
  return -lg;
}

struct Plan {
  int W = 0, N_R = 0, N_h = 0, K = 0, n_EF = 0, n_eta = 1, chunk = 0;
  int precision = KUBO_FP64;
  int Npad = 0, Kp = 0, Mpad = 0;   // tensor-core operand padding (mixed precision)
  int kpb = KSUM_KPB;               // k-points per k-sum block
  int pad = 1;                      // leading dimension W + pad in the fused kernels' smem
  int rot = 0;                      // FP32-grade rotation kernel (W <= 64): ROT_* below
  bool scale_ok = false;            // the call may rescale H(R) by a power of two (range_exponent)
  int escale = 0;                   // that power: the basis holds 2^escale H(R)
  int ql_cap = 0;                   // QL sweeps per eigenvalue (0 = the kernels' default)
  bool ql_fp64 = false;             // MIXED: FP64 QL and its eigenvalues (kubo_options.ql_fp64)
  int group_m = 8;                  // tensor-core Fourier sum: M tiles rasterised together
  int symv_parts = 4;               // Householder reduction: column partitions of its symv
  bool model = false;   // needs the prepared Fourier basis
  bool eigh = false;    // needs eigensolver buffers
  bool berry = false;   // needs velocity / curvature buffers
  bool ksum = false;    // needs k-sum buffers
  bool lbuf = false;    // W > SMALL_W_MAX: scratch of the multi-pass kernels
  bool grad = false;    // reverse-mode buffers (kubo_ahc_grad)
  bool iit = false;     // inverse-iteration scratch (separate eigenvector kernel)
  int iit_slots = 0;
  // separable Fourier sum: bounding box, pairs per batch, planes of the range
  bool sep = false;
  SepBox sb{0, 0, 0};
  int sep_np = 0, sep_np1 = 0, sep_j1a = 0;
  Mesh mesh{1, 1, 1, 1};
  size_t o_status = 0, o_neg = 0, o_pairs = 0, o_Rh = 0, o_tab = 0, o_Bp = 0, o_etas = 0,
         o_acc = 0, o_Hp = 0, o_Xp = 0, o_Yp = 0, o_E = 0, o_U = 0, o_Om = 0, o_d = 0, o_e = 0,
         o_ph = 0, o_refl = 0, o_tau = 0, o_lam = 0, o_part = 0,
         o_HR = 0, o_EF = 0, o_out = 0, o_Bt = 0, o_A = 0, o_C64 = 0, o_cexp = 0, o_L = 0,
         o_iit = 0, o_box = 0, o_sepA = 0, o_sepB = 0, o_sepBy = 0;
  // reverse mode: six complex W x W work matrices per k, Ebar, packed [Hbar|dxHbar|dyHbar],
  // the Fourier coefficient rows of the batch and the accumulated G rows
  size_t o_gw = 0, o_Ebar = 0, o_Mbar = 0, o_Coef = 0, o_Gacc = 0;
  // mixed-precision fix-up buffers
  bool fixup = false;
  int fix_cap = 0;
  size_t o_flag = 0, o_bin = 0, o_pos = 0, o_kid = 0, o_cnt = 0, o_fHp = 0, o_fXp = 0, o_fYp = 0,
         o_fE = 0, o_fOm = 0;
  size_t total = 0;
};

// Per k-point scratch of the W > SMALL_W_MAX kernels, reused by stage: the eigenvectors Z of
// the tridiagonal, then the FP64 rotation products T, V^x, V^y (the larger of the two).
size_t large_region_bytes(int W) {
  const size_t WW = (size_t)W * W;
  // (Z and the FP32 compact-WY factors of the U assembly, 256 bytes of alignment per batch
  // included, fit in the rotation products' share at every W > 64)
  return std::max(WW * sizeof(double) + reflect_wy_scratch_bytes(W) + 256,
                  3 * WW * sizeof(double2));
}

// persistent inverse-iteration CTAs of a plan (their LU scratch is per CTA)
int iit_slots_for(int W, int chunk) { return std::max(1, std::min(chunk, iit_max_slots(W))); }

size_t bytes_per_k(int W, int n_eta) {
  size_t WW = (size_t)W * W;
  return 3 * WW * 8 + WW * 16 /*U*/ + WW * 16 /*refl*/ + (size_t)W * (8 * 5 + 16) +
         (size_t)n_eta * W * 8 + 64 + (W > SMALL_W_MAX ? large_region_bytes(W) : 0);
}

// k-points per batch: a fixed 24 GiB of batch buffers (of GB300's 288 GB), at most 65,536.
// Larger batches give the lane-per-k QL more resident warps (65,536 at W = 64: 13 per SM);
// the budget is a constant so that a size query and the call agree.
int auto_chunk(int W, int n_eta, int64_t n_total, size_t extra_per_k = 0) {
  const size_t budget = (size_t)24 << 30;
  int64_t c = (int64_t)(budget / (bytes_per_k(W, n_eta) + extra_per_k));
  c = std::max<int64_t>(1024, std::min<int64_t>(c, 65536));
  c = c / 1024 * 1024;
  return (int)std::max<int64_t>(1, std::min<int64_t>(c, n_total));
}

void plan_layout(Plan& p, bool host_io, int64_t n_list_outputs_unused) {
  (void)n_list_outputs_unused;
  Bump b;
  const size_t WW = (size_t)p.W * p.W;
  p.o_status = b.take(sizeof(DevStatus));
  p.o_etas = b.take(sizeof(double) * MAX_ETA);
  if (p.model) {
    p.o_neg = b.take(sizeof(int) * p.N_R);
    p.o_pairs = b.take(sizeof(int) * 2 * std::max(1, p.N_h));
    p.o_Rh = b.take(sizeof(int) * 3 * std::max(1, p.N_h));
    p.o_tab = b.take(twiddle_bytes(p.mesh.N1, p.mesh.N2, p.mesh.N3));
    p.o_Bp = b.take(sizeof(double) * (size_t)p.K * WW);
    if (p.sep) {
      p.o_box = b.take(sizeof(int) * (size_t)(2 * p.sb.h1 + 1) * (2 * p.sb.h2 + 1) * (2 * p.sb.h3 + 1));
      p.o_sepA = b.take(sizeof(double2) * sep_a_elems(p.sb, p.W, p.mesh.N3));
      p.o_sepB = b.take(sizeof(double2) * sep_b_elems_per_pair(p.sb, p.W) * (size_t)std::max(1, p.sep_np));
      p.o_sepBy = b.take(sizeof(double2) * sep_b_elems_per_pair(p.sb, p.W) * (size_t)std::max(1, p.sep_np));
    }
    if (tc_fourier(p.precision)) {
      p.Npad = tc_pad_n(p.W);
      p.Kp = tc_pad_k(p.N_R);
      p.Mpad = tc_pad_m(std::max(1, p.chunk));
      p.o_Bt = b.take((size_t)2 * tc_slices() * p.Npad * p.Kp);
      p.o_cexp = b.take(sizeof(int) * (size_t)p.Npad);
      p.o_A = b.take((size_t)2 * tc_slices() * p.Mpad * p.Kp);
      p.o_C64 = b.take(sizeof(double) * (size_t)p.chunk * p.Npad);
    } else {
      p.o_Hp = b.take(sizeof(double) * (size_t)p.chunk * WW);
      p.o_Xp = b.take(sizeof(double) * (size_t)p.chunk * WW);
      p.o_Yp = b.take(sizeof(double) * (size_t)p.chunk * WW);
    }
  }
  if (p.eigh) {
    p.o_d = b.take(sizeof(double) * (size_t)p.chunk * p.W);
    p.o_e = b.take(sizeof(double) * (size_t)p.chunk * p.W);
    p.o_ph = b.take(sizeof(double2) * (size_t)p.chunk * p.W);
    p.o_tau = b.take(sizeof(double) * (size_t)p.chunk * p.W);
    p.o_refl = b.take(sizeof(double2) * (size_t)p.chunk * WW);
    p.o_lam = b.take(sizeof(double) * (size_t)p.chunk * p.W);
  }
  if (p.berry) {
    p.o_E = b.take(sizeof(double) * (size_t)p.chunk * p.W);
    p.o_U = b.take(sizeof(double2) * (size_t)p.chunk * WW);
    p.o_Om = b.take(sizeof(double) * (size_t)p.chunk * p.W * p.n_eta);
  }
  if (p.fixup) {
    p.fix_cap = std::min(std::max(1, p.chunk), std::max(256, p.chunk / 8));
    p.o_flag = b.take(sizeof(int) * (size_t)p.chunk);
    p.o_bin = b.take(sizeof(int) * (size_t)p.chunk);
    p.o_pos = b.take(sizeof(int) * (size_t)p.chunk);
    p.o_kid = b.take(sizeof(int64_t) * (size_t)p.chunk);
    p.o_cnt = b.take(sizeof(int));
    p.o_fHp = b.take(sizeof(double) * (size_t)p.fix_cap * WW);
    p.o_fXp = b.take(sizeof(double) * (size_t)p.fix_cap * WW);
    p.o_fYp = b.take(sizeof(double) * (size_t)p.fix_cap * WW);
    p.o_fE = b.take(sizeof(double) * (size_t)p.fix_cap * p.W);
    p.o_fOm = b.take(sizeof(double) * (size_t)p.fix_cap * p.W * p.n_eta);
  }
  if (p.lbuf) p.o_L = b.take(large_region_bytes(p.W) * (size_t)std::max(1, p.chunk));
  p.iit = p.eigh && (p.W > SMALL_W_MAX || f32_rotation(p.precision));
  if (p.iit) {
    p.iit_slots = iit_slots_for(p.W, std::max(1, p.chunk));
    p.o_iit = b.take(sizeof(double) * iit_scratch_doubles(p.W, p.iit_slots));
  }
  if (p.grad) {
    const size_t ch = (size_t)std::max(1, p.chunk);
    p.o_gw = b.take(6 * sizeof(double2) * ch * WW);
    p.o_Ebar = b.take(sizeof(double) * ch * p.W);
    p.o_Mbar = b.take(3 * sizeof(double) * ch * WW);
    p.o_Coef = b.take(sizeof(double) * (size_t)(2 * p.N_h + 1) * ch);
    p.o_Gacc = b.take(3 * sizeof(double) * (size_t)(2 * p.N_h + 1) * WW);
  }
  if (p.ksum) {
    const int n_out = p.n_eta * p.n_EF;
    p.o_acc = b.take(sizeof(double2) * n_out);
    const int64_t max_blocks = std::max<int64_t>(1, (int64_t)(KSUM_PART_BYTES / (sizeof(double2) * n_out)));
    const int64_t ch = std::max(1, p.chunk);
    p.kpb = (int)std::max<int64_t>(KSUM_KPB, (ch + max_blocks - 1) / max_blocks);
    p.o_part = b.take(sizeof(double2) * (size_t)n_out * ((ch + p.kpb - 1) / p.kpb));
  }
  if (host_io) {
    p.o_HR = b.take(sizeof(double2) * (size_t)p.N_R * WW);
    p.o_EF = b.take(sizeof(double) * p.n_EF);
    p.o_out = b.take(sizeof(double) * (size_t)p.n_eta * p.n_EF);
  }
  p.total = b.off;
}

// ------------------------------------------------------------------ device allocations
// Every device allocation the library makes goes through lib_malloc_async, which honours the
// test hook kubo_debug_fail_allocations (pending simulated failures).
std::atomic<int> g_fail_allocs{0};

cudaError_t lib_malloc_async(void** p, size_t bytes, cudaStream_t s) {
  int n = g_fail_allocs.load();
  while (n > 0) {
    if (g_fail_allocs.compare_exchange_weak(n, n - 1)) {
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
  }
  return cudaMallocAsync(p, bytes, s);
}

// ------------------------------------------------------------------ call context
// The library-managed workspace comes from the device's default stream-ordered pool.  With
// the pool's default release threshold (0) the freed workspace is unmapped at the next
// synchronisation and every call pays for mapping it again (GBs at the default batch); the
// threshold is raised to the largest workspace seen, so one workspace stays mapped between
// calls.  (A caller-supplied workspace bypasses the pool.)
inline void retain_pool_memory(size_t bytes) {
  int dev = 0;
  cudaMemPool_t pool;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  uint64_t cur = 0;
  if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &cur) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  if (cur < (uint64_t)bytes) {
    uint64_t thr = (uint64_t)bytes;
    if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr) != cudaSuccess)
      cudaGetLastError();
  }
}

struct Call {
  cudaStream_t s = nullptr;
  char* ws = nullptr;
  bool owned = false;
  Plan p;
  kubo_status st = KUBO_OK;
  // optional per-stage timing: event pairs recorded around launches, read after the sync
  struct Ev { int stage, launches; cudaEvent_t a, b; };
  kubo_profile* prof = nullptr;
  std::vector<Ev> evs;

  ~Call() { collect(); }
  void collect() {
    if (evs.empty()) return;
    cudaStreamSynchronize(s);
    for (auto& e : evs) {
      float ms = 0.f;
      if (prof && cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) {
        prof->ms[e.stage] += ms;
        prof->launches[e.stage] += e.launches;
      }
      cudaEventDestroy(e.a);
      cudaEventDestroy(e.b);
    }
    evs.clear();
    cudaGetLastError();
  }

  template <class T>
  T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }

  kubo_status acquire(const kubo_options& o) {
    if (o.workspace) {
      if (o.workspace_bytes < p.total) return KUBO_ERR_WORKSPACE;
      ws = (char*)o.workspace;
      return KUBO_OK;
    }
    retain_pool_memory(p.total);
    if (lib_malloc_async((void**)&ws, p.total, s) != cudaSuccess) {
      cudaGetLastError();
      ws = nullptr;
      return KUBO_ERR_OOM;
    }
    owned = true;
    return KUBO_OK;
  }
  void release() {
    if (owned && ws) cudaFreeAsync(ws, s);
    ws = nullptr;
    owned = false;
  }
};

// Records a CUDA event pair on the call's stream around the launches of one stage.
struct StageTimer {
  Call& c;
  Call::Ev ev{0, 0, nullptr, nullptr};
  StageTimer(Call& call, int stage, int launches) : c(call) {
    if (!c.prof) return;
    ev.stage = stage;
    ev.launches = launches;
    if (cudaEventCreate(&ev.a) != cudaSuccess || cudaEventCreate(&ev.b) != cudaSuccess) {
      cudaGetLastError();
      ev.a = ev.b = nullptr;
      return;
    }
    cudaEventRecord(ev.a, c.s);
  }
  ~StageTimer() {
    if (!c.prof || !ev.a) return;
    cudaEventRecord(ev.b, c.s);
    c.evs.push_back(ev);
  }
};

#define KCHECK(expr)                                  \
  do {                                                \
    cudaError_t _e = (expr);                          \
    if (_e != cudaSuccess) {                          \
      cudaGetLastError();                             \
      return KUBO_ERR_CUDA;                           \
    }                                                 \
  } while (0)

kubo_status bits_to_status(unsigned bits) {
  if (bits & ST_BAD_INDEX) return KUBO_ERR_INVALID_ARG;
  if (bits & (ST_NOT_HERMITIAN | ST_NONFINITE)) return KUBO_ERR_NOT_HERMITIAN;
  if (bits & ST_TIMEOUT) return KUBO_ERR_TIMEOUT;
  if (bits & ST_NO_CONVERGENCE) return KUBO_ERR_NO_CONVERGENCE;
  return KUBO_OK;
}

kubo_status read_status(Call& c, DevStatus* full = nullptr) {
  DevStatus h;
  KCHECK(cudaMemcpyAsync(&h, c.at<DevStatus>(c.p.o_status), sizeof(h), cudaMemcpyDeviceToHost, c.s));
  KCHECK(cudaStreamSynchronize(c.s));
  if (full) *full = h;
  return bits_to_status(h.bits);
}

double herm_max(const DevStatus& h) {
  double mx;
  std::memcpy(&mx, &h.herm_max_bits, sizeof(mx));
  return mx;
}

bool finite_nonneg(double x) { return std::isfinite(x) && x >= 0.0; }

kubo_status validate_common(int W, int N_R, const int32_t* kmesh, const kubo_options& o,
                            int& n_eta) {
  if (W < 1 || N_R < 1 || !kmesh) return KUBO_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a)
    if (kmesh[a] < 1) return KUBO_ERR_INVALID_ARG;
  if (o.precision < KUBO_FP64 || o.precision > KUBO_MIXED_DF) return KUBO_ERR_UNSUPPORTED;
  if (W > MAX_W) return KUBO_ERR_UNSUPPORTED;
  if (!finite_nonneg(o.kT)) return KUBO_ERR_INVALID_ARG;
  if (o.n_eta < 0) return KUBO_ERR_INVALID_ARG;
  if (o.n_eta > 0) {
    if (!o.etas) return KUBO_ERR_INVALID_ARG;
    if (o.n_eta > MAX_ETA) return KUBO_ERR_UNSUPPORTED;
    for (int e = 0; e < o.n_eta; ++e)
      if (!finite_nonneg(o.etas[e])) return KUBO_ERR_INVALID_ARG;
  }
  if (o.chunk_k < 0 || o.ql_max_sweeps < 0) return KUBO_ERR_INVALID_ARG;
  if (o.ql_fp64 < 0 || o.ql_fp64 > 1) return KUBO_ERR_INVALID_ARG;
  if (o.rotation_tc < 0 || o.rotation_tc > 3) return KUBO_ERR_INVALID_ARG;
  if (!std::isfinite(o.mixed_fixup_rel)) return KUBO_ERR_INVALID_ARG;
  n_eta = o.n_eta > 0 ? o.n_eta : 1;
  return KUBO_OK;
}

// Device k-list check before any output is written: every index in [0, N_k) (one host sync).
kubo_status check_klist(Call& c, const int64_t* kidx, int64_t n) {
  KCHECK(cudaMemsetAsync(c.at<char>(c.p.o_status), 0, sizeof(DevStatus), c.s));
  KCHECK(launch_check_kidx(kidx, n, c.p.mesh.Nk, c.at<DevStatus>(c.p.o_status), c.s));
  return read_status(c);
}

// Prepare the model: status reset, Hermitian check (one host sync, which also gives max |H(R)|
// and so the range exponent of the call), twiddles, packed basis (scaled by 2^escale).
kubo_status prepare_model(Call& c, const double* H_R, const RInfo& ri) {
  Plan& p = c.p;
  KCHECK(cudaMemsetAsync(c.at<char>(p.o_status), 0, sizeof(DevStatus), c.s));
  KCHECK(cudaMemcpyAsync(c.at<int>(p.o_neg), ri.neg.data(), sizeof(int) * p.N_R, cudaMemcpyHostToDevice, c.s));
  if (p.N_h > 0) {
    KCHECK(cudaMemcpyAsync(c.at<int>(p.o_pairs), ri.pairs.data(), sizeof(int) * 2 * p.N_h, cudaMemcpyHostToDevice, c.s));
    KCHECK(cudaMemcpyAsync(c.at<int>(p.o_Rh), ri.Rh.data(), sizeof(int) * 3 * p.N_h, cudaMemcpyHostToDevice, c.s));
  }
  DevStatus* st = c.at<DevStatus>(p.o_status);
  {
    StageTimer tm(c, KUBO_STAGE_PREP, 2);
    KCHECK(launch_check_hermitian((const double2*)H_R, c.at<int>(p.o_neg), p.N_R, p.W, st, c.s));
    KCHECK(launch_hermitian_verdict(st, c.s));
  }
  DevStatus h;
  kubo_status hv = read_status(c, &h);
  if (hv != KUBO_OK) return hv;
  p.escale = p.scale_ok ? range_exponent(herm_max(h)) : 0;
  {
    StageTimer tm(c, KUBO_STAGE_PREP, 2);
    KCHECK(launch_twiddles(c.at<double2>(p.o_tab), p.mesh.N1, p.mesh.N2, p.mesh.N3, c.s));
    KCHECK(launch_pack_basis((const double2*)H_R, c.at<int>(p.o_pairs), ri.idx0, p.N_h, p.W, c.at<double>(p.o_Bp), c.s, p.escale));
  }
  if (p.sep) {
    StageTimer tm(c, KUBO_STAGE_PREP, 1);
    KCHECK(cudaMemcpyAsync(c.at<int>(p.o_box), ri.box.data(), sizeof(int) * ri.box.size(), cudaMemcpyHostToDevice, c.s));
    KCHECK(launch_sep_stage_a((const double2*)H_R, c.at<int>(p.o_box), p.sb, p.W, p.mesh, c.at<double2>(p.o_tab), p.mesh.N1 + p.mesh.N2, c.at<double2>(p.o_sepA), c.s));
  }
  if (tc_fourier(p.precision)) {
    StageTimer tm(c, KUBO_STAGE_PREP, 1);
    KCHECK(launch_basis_split(c.at<double>(p.o_Bp), c.at<int>(p.o_Rh), p.N_h, p.W, p.Npad, p.Kp, c.at<int>(p.o_cexp), c.at<char>(p.o_Bt), c.s));
  }
  return read_status(c);
}

Model make_model(const Call& c) {
  Model md;
  md.W = c.p.W;
  md.N_R = c.p.N_R;
  md.N_h = c.p.N_h;
  md.K = c.p.K;
  md.Bp = c.at<double>(c.p.o_Bp);
  md.Rh = c.at<int>(c.p.o_Rh);
  md.tab = c.at<double2>(c.p.o_tab);
  md.tab_df = reinterpret_cast<const float4*>(md.tab + (c.p.mesh.N1 + c.p.mesh.N2 + c.p.mesh.N3));
  md.tab_off[0] = 0;
  md.tab_off[1] = c.p.mesh.N1;
  md.tab_off[2] = c.p.mesh.N1 + c.p.mesh.N2;
  return md;
}

EighBufs make_eigh_bufs(const Call& c) {
  EighBufs b;
  b.d = c.at<double>(c.p.o_d);
  b.e = c.at<double>(c.p.o_e);
  b.phase = c.at<double2>(c.p.o_ph);
  b.refl = c.at<double2>(c.p.o_refl);
  b.tau = c.at<double>(c.p.o_tau);
  b.lam = c.at<double>(c.p.o_lam);
  if (c.p.ql_cap > 0) b.ql_cap = c.p.ql_cap;
  b.symv_parts = c.p.symv_parts;
  return b;
}

// Eigenvalues (sorted) and eigenvectors U = Q D Z of n tridiagonalised matrices whose
// eigenvalues QL left in eb.lam (U may be null: eigenvalues only).  f32u (W > 64 only): U is
// formed in FP32 (float2) for the FP32 rotations, its only consumer in that mode.  rq (W > 64
// only): eigenvalues from the Rayleigh quotients of the eigenvectors instead of eb.lam.
cudaError_t eigh_vectors(const Call& c, int n, const EighBufs& eb, double* E, double2* U,
                         bool f32u = false, bool rq = false) {
  const Plan& p = c.p;
  if (p.W <= SMALL_W_MAX) return launch_backtransform(p.W, n, eb, E, U, c.s, p.pad);
  double* Z = U ? c.at<double>(p.o_L) : nullptr;
  cudaError_t e = Z && df_eigh(p.precision)
                      ? launch_iit_df(p.W, n, eb, E, Z, c.at<double>(p.o_iit), p.iit_slots, c.s)
                      : launch_iit(p.W, n, eb, E, Z, c.at<double>(p.o_iit), p.iit_slots, c.s, rq);
  if (e != cudaSuccess || !U) return e;
  if (f32u) {
    // the blocked WY factors in the large region after Z (16-byte aligned, within its size)
    const uintptr_t after_z = (uintptr_t)(Z + (size_t)std::max(1, p.chunk) * p.W * p.W);
    float2* wy = reinterpret_cast<float2*>((after_z + 255) & ~(uintptr_t)255);
    return launch_reflect_wy(p.W, n, eb, Z, reinterpret_cast<float2*>(U), wy, c.s);
  }
  return launch_reflect_large(p.W, n, eb, Z, U, f32u, c.s);
}

// Steps (3)-(4) from packed Hermitian dH rows X, Y of leading dimension ld; f32 = FP32
// products.  rows = X and Y are the W*W and 2*W*W column offsets of tensor-core output rows.
cudaError_t berry_any(const Call& c, const double* E, const double2* U, const double* X,
                      const double* Y, int64_t ld, bool rows, int n, bool f32, double* Om,
                      int64_t om_stride) {
  const Plan& p = c.p;
  const double* etas = c.at<double>(p.o_etas);
  if (p.W > SMALL_W_MAX) {
    const size_t WW = (size_t)p.W * p.W;
    const size_t es = f32 ? sizeof(float2) : sizeof(double2);
    char* L = c.at<char>(p.o_L);
    const size_t cap = (size_t)std::max(1, p.chunk) * WW * es;
    return launch_berry_large(E, U, X, Y, ld, p.W, n, etas, p.n_eta, Om, om_stride, f32, L, L + cap,
                              L + 2 * cap, c.s);
  }
  if (rows) {
    const double* C = X - (size_t)p.W * p.W;   // the row start (H | dxH | dyH)
    return f32 ? launch_berry_mixed_rows(E, U, C, ld, p.W, n, etas, p.n_eta, Om, om_stride, c.s, p.pad)
               : launch_berry_fp64_rows(E, U, C, ld, p.W, n, etas, p.n_eta, Om, om_stride, c.s, p.pad);
  }
  return f32 ? launch_berry_mixed_from_f64(E, U, X, Y, p.W, n, etas, p.n_eta, Om, om_stride, c.s, p.pad)
             : launch_berry_fp64(E, U, X, Y, p.W, n, etas, p.n_eta, Om, om_stride, c.s, p.pad);
}

// Steps (1)-(4) for one batch [t0, t0+n) of a k-list; E and U go to the chunk buffers, Omega
// to Om (eta stride om_stride).  Eout may redirect the sorted eigenvalues.
// Mixed precision: step (1) on the tensor cores into rows [H | dxH | dyH], the eigensolver
// in FP64 from those rows, the rotations in FP32 (or FP64) with FP64 denominators.
kubo_status run_batch_mixed(Call& c, const Model& md, const KList& kl, double* Eout, double* Om,
                            int64_t om_stride) {
  Plan& p = c.p;
  EighBufs eb = make_eigh_bufs(c);
  DevStatus* st = c.at<DevStatus>(p.o_status);
  double2* U = c.at<double2>(p.o_U);
  double* C64 = c.at<double>(p.o_C64);
  const int Mb = tc_pad_m(kl.n);
  // W <= 64 with an FP32-grade rotation: the velocity rows are stored in FP32 (their only
  // consumer reads them in FP32: half the bytes, no conversions on the FP64 pipe)
  const bool vel32 = f32_rotation(p.precision) && p.W <= SMALL_W_MAX;
  {
    // the velocity columns feed only the FP32 rotation in the MIXED mode: FP32-grade slices
    // (a second tensor-core launch over those column tiles)
    const int red_n0 = f32_rotation(p.precision) ? p.W * p.W : p.Npad;
    StageTimer tm(c, KUBO_STAGE_FOURIER, red_n0 < p.Npad ? 3 : 2);
    KCHECK(launch_coef_split(md, p.mesh, kl, Mb, p.Kp, c.at<char>(p.o_A), c.s));
    KCHECK(launch_fourier_tc(c.at<char>(p.o_A), c.at<char>(p.o_Bt), c.at<int>(p.o_cexp), Mb, p.Npad, p.Kp, kl.n, C64, p.Npad, st, c.s, red_n0, p.group_m, vel32 ? p.W : 0));
  }
  {
    // MIXED_DF: the reduction and the QL iteration in double-float on the FP32 pipe (both are
    // FP64-pipe-bound otherwise); every other mode: FP64
    StageTimer tm(c, KUBO_STAGE_TRIDIAG, 1);
    if (df_eigh(p.precision))
      KCHECK(launch_tridiag_df_rows(C64, p.Npad, p.W, kl.n, eb, c.s));
    else
      KCHECK(launch_tridiag_rows(C64, p.Npad, p.W, kl.n, eb, c.s));
  }
  {
    StageTimer tm(c, KUBO_STAGE_QL, 1);
    if (df_ql(p.precision, p.ql_fp64))
      KCHECK(launch_ql_df(p.W, kl.n, eb, st, c.s));
    else
      KCHECK(launch_ql(p.W, kl.n, eb, st, c.s));
  }
  const size_t WW = (size_t)p.W * p.W;
  if (f32_rotation(p.precision) && p.W <= SMALL_W_MAX) {
    // FP32 rotations: U = Q D Z is formed in FP32 (inside the SIMT and exact-slice rotation
    // kernels, by assemble_u_kernel for the 3xTF32 one) from the FP64 eigenvectors Z of the
    // tridiagonal (kept in the U buffer) and the reflectors
    double* Z = reinterpret_cast<double*>(U);
    // the tensor-core rotation takes U = Q D Z formed by a kernel of its own (FP32, in the
    // second half of the U buffer: Z holds the first n W^2 doubles)
    float2* U32 = p.rot == ROT_TF32 ? reinterpret_cast<float2*>(Z + (size_t)kl.n * WW) : nullptr;
    {
      StageTimer tm(c, KUBO_STAGE_BACKTRANSFORM, U32 ? 2 : 1);
      if (df_eigh(p.precision))
        KCHECK(launch_iit_df(p.W, kl.n, eb, Eout, Z, c.at<double>(p.o_iit), p.iit_slots, c.s));
      else
        KCHECK(launch_iit(p.W, kl.n, eb, Eout, Z, c.at<double>(p.o_iit), p.iit_slots, c.s,
                           rq_eigenvalues(p.precision, p.ql_fp64)));
      if (U32) KCHECK(launch_assemble_u32(Z, eb, U32, p.W, kl.n, c.s));
    }
    StageTimer tm(c, KUBO_STAGE_BERRY, 1);
    if (p.rot == ROT_TF32)
      KCHECK(launch_berry_tf32_rows(Eout, Z, eb, C64, p.Npad, p.W, kl.n, c.at<double>(p.o_etas), p.n_eta, Om, om_stride, st, c.s, vel32, U32));
    else if (p.rot == ROT_EXACT_SLICES)
      KCHECK(launch_berry_tc_rows(Eout, Z, eb, C64, p.Npad, p.W, kl.n, c.at<double>(p.o_etas), p.n_eta, Om, om_stride, st, c.s, vel32));
    else
      KCHECK(launch_berry_mixed_rows_z(Eout, Z, eb, C64, p.Npad, p.W, kl.n, c.at<double>(p.o_etas), p.n_eta, Om, om_stride, c.s, p.pad, vel32));
    return KUBO_OK;
  }
  {
    StageTimer tm(c, KUBO_STAGE_BACKTRANSFORM, p.W > SMALL_W_MAX ? 2 : 1);
    KCHECK(eigh_vectors(c, kl.n, eb, Eout, U, f32_rotation(p.precision),
                        rq_eigenvalues(p.precision, p.ql_fp64)));
  }
  {
    StageTimer tm(c, KUBO_STAGE_BERRY, p.W > SMALL_W_MAX ? 5 : 1);
    KCHECK(berry_any(c, Eout, U, C64 + WW, C64 + 2 * WW, p.Npad, true, kl.n, f32_rotation(p.precision), Om, om_stride));
  }
  return KUBO_OK;
}

// fourier_done: step (1) already wrote Hp / Xp / Yp (separable Fourier sum)
kubo_status run_batch_steps(Call& c, const Model& md, const KList& kl, double* Eout, double* Om,
                            int64_t om_stride, bool fourier_done) {
  Plan& p = c.p;
  if (tc_fourier(p.precision)) return run_batch_mixed(c, md, kl, Eout, Om, om_stride);
  double* Hp = c.at<double>(p.o_Hp);
  double* Xp = c.at<double>(p.o_Xp);
  double* Yp = c.at<double>(p.o_Yp);
  EighBufs eb = make_eigh_bufs(c);
  DevStatus* st = c.at<DevStatus>(p.o_status);
  double2* U = c.at<double2>(p.o_U);
  if (!fourier_done) {
    StageTimer tm(c, KUBO_STAGE_FOURIER, 1);
    KCHECK(launch_fourier_fp64(md, p.mesh, kl, Hp, Xp, Yp, c.s));
  }
  {
    StageTimer tm(c, KUBO_STAGE_TRIDIAG, 1);
    KCHECK(launch_tridiag(Hp, p.W, kl.n, eb, c.s));
  }
  {
    StageTimer tm(c, KUBO_STAGE_QL, 1);
    KCHECK(launch_ql(p.W, kl.n, eb, st, c.s));
  }
  if (f32_rotation(p.precision) && p.W <= SMALL_W_MAX) {
    double* Z = reinterpret_cast<double*>(U);
    {
      StageTimer tm(c, KUBO_STAGE_BACKTRANSFORM, 1);
      if (df_eigh(p.precision))
        KCHECK(launch_iit_df(p.W, kl.n, eb, Eout, Z, c.at<double>(p.o_iit), p.iit_slots, c.s));
      else
        KCHECK(launch_iit(p.W, kl.n, eb, Eout, Z, c.at<double>(p.o_iit), p.iit_slots, c.s));
    }
    StageTimer tm(c, KUBO_STAGE_BERRY, 1);
    if (p.rot == ROT_TF32)
      KCHECK(launch_berry_tf32_from_f64(Eout, Z, eb, Xp, Yp, p.W, kl.n, c.at<double>(p.o_etas), p.n_eta, Om, om_stride, st, c.s));
    else if (p.rot == ROT_EXACT_SLICES)
      KCHECK(launch_berry_tc_from_f64(Eout, Z, eb, Xp, Yp, p.W, kl.n, c.at<double>(p.o_etas), p.n_eta, Om, om_stride, st, c.s));
    else
      KCHECK(launch_berry_mixed_from_f64_z(Eout, Z, eb, Xp, Yp, p.W, kl.n, c.at<double>(p.o_etas), p.n_eta, Om, om_stride, c.s, p.pad));
    return KUBO_OK;
  }
  {
    StageTimer tm(c, KUBO_STAGE_BACKTRANSFORM, p.W > SMALL_W_MAX ? 2 : 1);
    KCHECK(eigh_vectors(c, kl.n, eb, Eout, U, f32_rotation(p.precision)));
  }
  {
    StageTimer tm(c, KUBO_STAGE_BERRY, p.W > SMALL_W_MAX ? 5 : 1);
    KCHECK(berry_any(c, Eout, U, Xp, Yp, (int64_t)p.W * p.W, false, kl.n, f32_rotation(p.precision), Om, om_stride));
  }
  return KUBO_OK;
}

// Steps (1)-(4) of one batch; with a rescaled model (escale != 0) the eigenvalues are brought
// back to the caller's units (the curvatures are scale-free).
kubo_status run_batch(Call& c, const Model& md, const KList& kl, double* Eout, double* Om,
                      int64_t om_stride, bool fourier_done = false) {
  kubo_status r = run_batch_steps(c, md, kl, Eout, Om, om_stride, fourier_done);
  if (r != KUBO_OK) return r;
  KCHECK(launch_scale_pow2(Eout, (int64_t)kl.n * c.p.W, -c.p.escale, c.s));
  return KUBO_OK;
}

// The broadenings on the device, scaled like H(R) (2^escale: call after prepare_model).
kubo_status upload_etas(Call& c, const kubo_options& o, double eta) {
  double h[MAX_ETA] = {0};
  if (o.n_eta > 0) for (int e = 0; e < o.n_eta; ++e) h[e] = o.etas[e];
  else h[0] = eta;
  for (double& x : h) x = std::ldexp(x, c.p.escale);
  KCHECK(cudaMemcpyAsync(c.at<double>(c.p.o_etas), h, sizeof(h), cudaMemcpyHostToDevice, c.s));
  return KUBO_OK;
}

// Mixed precision: re-evaluate in FP64 the k-points of this batch that have a level within
// tau_k = rel * max|E(k)| of a Fermi level, and overwrite their E and Omega in place (the
// k-sum order is unchanged, so the result stays deterministic).
kubo_status fixup_batch(Call& c, const Model& md, const KList& kl, const double* E_F, double rel,
                        double frac, double* E, double* Om) {
  Plan& p = c.p;
  int* flag = c.at<int>(p.o_flag);
  int* pos = c.at<int>(p.o_pos);
  int64_t* kid = c.at<int64_t>(p.o_kid);
  int cnt = 0;
  {
    StageTimer tm(c, KUBO_STAGE_FIXUP, 2);
    KCHECK(launch_fixup_flag(E, Om, p.W, kl.n, p.n_eta, (int64_t)kl.n * p.W, E_F, p.n_EF, rel, flag, c.at<int>(p.o_bin), c.s));
    KCHECK(launch_fixup_compact(flag, c.at<int>(p.o_bin), kl.n, frac, kl, pos, kid, c.at<int>(p.o_cnt), c.s));
  }
  KCHECK(cudaMemcpyAsync(&cnt, c.at<int>(p.o_cnt), sizeof(int), cudaMemcpyDeviceToHost, c.s));
  KCHECK(cudaStreamSynchronize(c.s));
  if (c.prof) c.prof->fixup_k += cnt;
  if (cnt <= 0) return KUBO_OK;
  EighBufs eb = make_eigh_bufs(c);
  DevStatus* st = c.at<DevStatus>(p.o_status);
  double2* U = c.at<double2>(p.o_U);
  double* fE = c.at<double>(p.o_fE);
  double* fOm = c.at<double>(p.o_fOm);
  const int64_t fstride = (int64_t)p.fix_cap * p.W;
  for (int c0 = 0; c0 < cnt; c0 += p.fix_cap) {
    const int nf = std::min(p.fix_cap, cnt - c0);
    KList fl{kid + c0, 0, nf};
    StageTimer tm(c, KUBO_STAGE_FIXUP, p.W > SMALL_W_MAX ? 11 : 6);
    KCHECK(launch_fourier_fp64(md, p.mesh, fl, c.at<double>(p.o_fHp), c.at<double>(p.o_fXp), c.at<double>(p.o_fYp), c.s));
    KCHECK(launch_tridiag(c.at<double>(p.o_fHp), p.W, nf, eb, c.s));
    KCHECK(launch_ql(p.W, nf, eb, st, c.s));
    KCHECK(eigh_vectors(c, nf, eb, fE, U));
    KCHECK(berry_any(c, fE, U, c.at<double>(p.o_fXp), c.at<double>(p.o_fYp), (int64_t)p.W * p.W, false, nf, false, fOm, fstride));
    KCHECK(launch_scale_pow2(fE, (int64_t)nf * p.W, -p.escale, c.s));
    KCHECK(launch_fixup_scatter(pos + c0, nf, p.W, p.n_eta, fE, fOm, fstride, E, Om, (int64_t)kl.n * p.W, c.s));
  }
  return KUBO_OK;
}

// Shared body of kubo_ahc and kubo_ahc_host (device pointers by now).
kubo_status ahc_device(Call& c, const kubo_options& o, const double* H_R, const RInfo& ri,
                       const double* E_F, double eta, double* out, int64_t kb, int64_t ke) {
  Plan& p = c.p;
  kubo_status r = prepare_model(c, H_R, ri);
  if (r != KUBO_OK) return r;
  r = upload_etas(c, o, eta);
  if (r != KUBO_OK) return r;
  const int n_out = p.n_eta * p.n_EF;
  KCHECK(cudaMemsetAsync(c.at<char>(p.o_acc), 0, sizeof(double2) * n_out, c.s));
  const Model md = make_model(c);
  double* E = c.at<double>(p.o_E);
  double* Om = c.at<double>(p.o_Om);
  double2* part = c.at<double2>(p.o_part);
  double2* acc = c.at<double2>(p.o_acc);
  const int64_t plane = (int64_t)p.mesh.N2 * p.mesh.N3;
  for (int64_t base = kb; base < ke; base += p.chunk) {
    KList kl{nullptr, base, (int)std::min<int64_t>(p.chunk, ke - base)};
    bool done = false;
    if (p.sep) {
      // batch = pairs [p0, p0 + np) x every plane of the range (pair-major); the loop index
      // base counts k-points of the range, so p0 = (base - kb) / np1
      const int64_t p0 = (base - kb) / p.sep_np1;
      const int np = (int)std::min<int64_t>(p.sep_np, plane - p0);
      kl = KList{nullptr, 0, np * p.sep_np1};
      StageTimer tm(c, KUBO_STAGE_FOURIER, 2);
      KCHECK(launch_sep_batch(c.at<double2>(p.o_sepA), p.sb, p.W, p.mesh, md.tab, md.tab_off, p0, np,
                              p.sep_j1a, p.sep_np1, c.at<double2>(p.o_sepB), c.at<double2>(p.o_sepBy),
                              c.at<double>(p.o_Hp), c.at<double>(p.o_Xp), c.at<double>(p.o_Yp), c.s));
      done = true;
    }
    r = run_batch(c, md, kl, E, Om, (int64_t)kl.n * p.W, done);
    if (r != KUBO_OK) return r;
    if (p.fixup) {
      r = fixup_batch(c, md, kl, E_F, o.mixed_fixup_rel, kFixupSpikyFraction, E, Om);
      if (r != KUBO_OK) return r;
    }
    StageTimer tm(c, KUBO_STAGE_KSUM, o.kT == 0.0 ? 3 : 2);
    KCHECK(launch_ksum_partial(E, Om, p.W, kl.n, p.n_eta, (int64_t)kl.n * p.W, E_F, p.n_EF, o.kT, part, p.kpb, c.s));
    KCHECK(launch_ksum_fold(part, (kl.n + p.kpb - 1) / p.kpb, n_out, acc, c.s));
  }
  {
    StageTimer tm(c, KUBO_STAGE_KSUM, 1);
    KCHECK(launch_ksum_final(acc, n_out, 1.0 / (double)p.mesh.Nk, c.at<DevStatus>(p.o_status), out, c.s));
  }
  return read_status(c);
}

// Separable Fourier sum: the bounding box of the R set, its index table, and the batch shape
// (pairs of (k2, k3) per batch x the k1-planes of the range; the batch k-count becomes the
// chunk).  Requires whole k1-planes and a box of at most 8 N_R vectors.
kubo_status setup_separable(Plan& p, const int32_t* R, int N_R, int64_t kb, int64_t ke, RInfo& ri) {
  if (p.precision != KUBO_FP64 && p.precision != KUBO_MIXED_ROTATION) return KUBO_ERR_UNSUPPORTED;
  const int64_t plane = (int64_t)p.mesh.N2 * p.mesh.N3;
  if (kb % plane != 0 || ke % plane != 0 || ke <= kb) return KUBO_ERR_UNSUPPORTED;
  int h[3] = {0, 0, 0};
  for (int i = 0; i < N_R; ++i)
    for (int a = 0; a < 3; ++a) h[a] = std::max(h[a], std::abs(R[3 * i + a]));
  const int64_t n1 = 2 * h[0] + 1, n2 = 2 * h[1] + 1, n3 = 2 * h[2] + 1;
  if (n1 * n2 * n3 > 8 * (int64_t)N_R) return KUBO_ERR_UNSUPPORTED;
  ri.box.assign((size_t)(n1 * n2 * n3), -1);
  for (int i = 0; i < N_R; ++i)
    ri.box[((size_t)(R[3 * i] + h[0]) * n2 + (R[3 * i + 1] + h[1])) * n3 + (R[3 * i + 2] + h[2])] = i;
  p.sep = true;
  p.sb = SepBox{h[0], h[1], h[2]};
  const int64_t np1 = (ke - kb) / plane;
  if (np1 > 65536) return KUBO_ERR_UNSUPPORTED;
  p.sep_np1 = (int)np1;
  p.sep_j1a = (int)(kb / plane);
  // pairs per batch: about the automatic batch size, B and By within 4 GiB
  const size_t per_pair = 2 * sizeof(double2) * sep_b_elems_per_pair(p.sb, p.W);
  int64_t np = std::max<int64_t>(1, (int64_t)p.chunk / np1);
  np = std::min<int64_t>(np, std::max<int64_t>(1, (int64_t)(((size_t)4 << 30) / per_pair)));
  np = std::min<int64_t>(np, plane);
  p.sep_np = (int)np;
  p.chunk = (int)(np * np1);
  return KUBO_OK;
}

kubo_status setup_ahc(Call& c, const kubo_options& o, const int32_t* R_vecs, int W, int N_R,
                      const int32_t* kmesh, int n_EF, RInfo& ri, int64_t& kb, int64_t& ke,
                      bool host_io) {
  int n_eta = 1;
  kubo_status r = validate_common(W, N_R, kmesh, o, n_eta);
  if (r != KUBO_OK) return r;
  if (!R_vecs || n_EF < 1) return KUBO_ERR_INVALID_ARG;
  r = analyze_R(R_vecs, N_R, ri);
  if (r != KUBO_OK) return r;
  Plan& p = c.p;
  p.W = W; p.N_R = N_R; p.N_h = ri.N_h; p.K = N_R; p.n_EF = n_EF; p.n_eta = n_eta;
  p.precision = o.precision;
  p.mesh = Mesh{kmesh[0], kmesh[1], kmesh[2], (int64_t)kmesh[0] * kmesh[1] * kmesh[2]};
  kb = o.k_begin; ke = o.k_end;
  if (kb == 0 && ke == 0) ke = p.mesh.Nk;
  if (kb < 0 || ke > p.mesh.Nk || kb > ke) return KUBO_ERR_INVALID_ARG;
  p.chunk = o.chunk_k > 0 ? o.chunk_k : auto_chunk(W, n_eta, std::max<int64_t>(1, ke - kb));
  p.model = p.eigh = p.berry = p.ksum = true;
  p.lbuf = W > SMALL_W_MAX;
  p.fixup = tc_fourier(p.precision) && o.mixed_fixup_rel > 0.0;
  p.pad = o.layout_unpadded ? 0 : 1;
  p.ql_cap = o.ql_max_sweeps;
  p.ql_fp64 = o.ql_fp64 != 0;
  p.rot = rotation_kernel(o.rotation_tc, W, o.layout_unpadded != 0);
  if (o.fourier_separable) {
    if (o.workspace) return KUBO_ERR_UNSUPPORTED;   // its size depends on the R set
    r = setup_separable(p, R_vecs, N_R, kb, ke, ri);
    if (r != KUBO_OK) return r;
  }
  // the separable stage A reads H(R) itself, not the (scalable) packed basis
  p.scale_ok = f32_rotation(p.precision) && !p.sep;
  plan_layout(p, host_io, 0);
  c.s = (cudaStream_t)o.stream;
  c.prof = o.profile;
  return KUBO_OK;
}

// per-k bytes of the reverse-mode buffers (for the automatic batch size)
size_t grad_bytes_per_k(int W, int N_R) {
  const size_t WW = (size_t)W * W;
  return 6 * 16 * WW + 8 * (size_t)W + 3 * 8 * WW + 8 * (size_t)N_R;
}

// Body of kubo_ahc_grad (device pointers): per batch the forward steps (1)-(3) in FP64, the
// optional forward k-sum, then the reverse pass and the transposed Fourier accumulation.
kubo_status ahc_grad_device(Call& c, const kubo_options& o, const double* H_R, const RInfo& ri,
                            const double* E_F, double eta, const double* g, double2* G,
                            double* out, int64_t kb, int64_t ke) {
  Plan& p = c.p;
  kubo_status r = prepare_model(c, H_R, ri);
  if (r != KUBO_OK) return r;
  r = upload_etas(c, o, eta);
  if (r != KUBO_OK) return r;
  const int n_out = p.n_eta * p.n_EF;
  const size_t WW = (size_t)p.W * p.W;
  const int M = 2 * p.N_h + 1;
  KCHECK(cudaMemsetAsync(c.at<char>(p.o_acc), 0, sizeof(double2) * n_out, c.s));
  KCHECK(cudaMemsetAsync(c.at<char>(p.o_Gacc), 0, 3 * sizeof(double) * (size_t)M * WW, c.s));
  const Model md = make_model(c);
  EighBufs eb = make_eigh_bufs(c);
  DevStatus* st = c.at<DevStatus>(p.o_status);
  double* Hp = c.at<double>(p.o_Hp);
  double* Xp = c.at<double>(p.o_Xp);
  double* Yp = c.at<double>(p.o_Yp);
  double* E = c.at<double>(p.o_E);
  double* Om = c.at<double>(p.o_Om);
  double2* U = c.at<double2>(p.o_U);
  double2* part = c.at<double2>(p.o_part);
  double2* acc = c.at<double2>(p.o_acc);
  const size_t cap = (size_t)std::max(1, p.chunk) * WW;
  double2* bw[6];
  for (int q = 0; q < 6; ++q) bw[q] = c.at<double2>(p.o_gw) + q * cap;
  double* Ebar = c.at<double>(p.o_Ebar);
  double* Mbar = c.at<double>(p.o_Mbar);
  double* Coef = c.at<double>(p.o_Coef);
  double* Gacc = c.at<double>(p.o_Gacc);
  const double* etas = c.at<double>(p.o_etas);
  const double inv_Nk = 1.0 / (double)p.mesh.Nk;
  for (int64_t base = kb; base < ke; base += p.chunk) {
    KList kl{nullptr, base, (int)std::min<int64_t>(p.chunk, ke - base)};
    const int n = kl.n;
    {
      StageTimer tm(c, KUBO_STAGE_FOURIER, 1);
      KCHECK(launch_fourier_fp64(md, p.mesh, kl, Hp, Xp, Yp, c.s));
    }
    {
      StageTimer tm(c, KUBO_STAGE_TRIDIAG, 1);
      KCHECK(launch_tridiag(Hp, p.W, n, eb, c.s));
    }
    {
      StageTimer tm(c, KUBO_STAGE_QL, 1);
      KCHECK(launch_ql(p.W, n, eb, st, c.s));
    }
    {
      StageTimer tm(c, KUBO_STAGE_BACKTRANSFORM, p.W > SMALL_W_MAX ? 2 : 1);
      KCHECK(eigh_vectors(c, n, eb, E, U));
    }
    if (out) {
      {
        StageTimer tm(c, KUBO_STAGE_BERRY, p.W > SMALL_W_MAX ? 5 : 1);
        KCHECK(berry_any(c, E, U, Xp, Yp, (int64_t)WW, false, n, false, Om, (int64_t)n * p.W));
      }
      StageTimer tm(c, KUBO_STAGE_KSUM, o.kT == 0.0 ? 3 : 2);
      KCHECK(launch_ksum_partial(E, Om, p.W, n, p.n_eta, (int64_t)n * p.W, E_F, p.n_EF, o.kT, part, p.kpb, c.s));
      KCHECK(launch_ksum_fold(part, (n + p.kpb - 1) / p.kpb, n_out, acc, c.s));
    }
    StageTimer tm(c, KUBO_STAGE_ADJOINT, 17);
    // v^x, v^y (full): b0 = U^H (X U), b1 = U^H (Y U)
    KCHECK(launch_herm_u(Xp, (int64_t)WW, U, bw[5], p.W, n, c.s));
    KCHECK(launch_zgemm_batched(true, false, false, U, bw[5], bw[0], p.W, n, c.s));
    KCHECK(launch_herm_u(Yp, (int64_t)WW, U, bw[5], p.W, n, c.s));
    KCHECK(launch_zgemm_batched(true, false, false, U, bw[5], bw[1], p.W, n, c.s));
    // vbar^x -> b2, vbar^y -> b3, Ebar
    KCHECK(launch_grad_pairs(E, bw[0], bw[1], p.W, n, g, E_F, p.n_EF, etas, p.n_eta, o.kT, inv_Nk, bw[2], bw[3], Ebar, c.s));
    // N = vbar^x v^x + vbar^y v^y -> b4; Gp -> b0
    KCHECK(launch_zgemm_batched(false, false, false, bw[2], bw[0], bw[4], p.W, n, c.s));
    KCHECK(launch_zgemm_batched(false, false, true, bw[3], bw[1], bw[4], p.W, n, c.s));
    KCHECK(launch_grad_gp(E, Ebar, bw[4], p.W, n, o.grad_eps, bw[0], c.s));
    // Hbar = U Gp U^H -> b1, dxHbar = U vbar^x U^H -> b0, dyHbar = U vbar^y U^H -> b4
    KCHECK(launch_zgemm_batched(false, false, false, U, bw[0], bw[5], p.W, n, c.s));
    KCHECK(launch_zgemm_batched(false, true, false, bw[5], U, bw[1], p.W, n, c.s));
    KCHECK(launch_zgemm_batched(false, false, false, U, bw[2], bw[5], p.W, n, c.s));
    KCHECK(launch_zgemm_batched(false, true, false, bw[5], U, bw[0], p.W, n, c.s));
    KCHECK(launch_zgemm_batched(false, false, false, U, bw[3], bw[5], p.W, n, c.s));
    KCHECK(launch_zgemm_batched(false, true, false, bw[5], U, bw[4], p.W, n, c.s));
    KCHECK(launch_pack3(bw[1], bw[0], bw[4], p.W, n, Mbar, c.s));
    // transposed Fourier sum of the batch into the G rows
    KCHECK(launch_grad_coef(md, p.mesh, kl, n, Coef, c.s));
    KCHECK(launch_grad_fourier_t(Coef, n, Mbar, M, (int)(3 * WW), n, Gacc, c.s));
  }
  r = read_status(c);
  if (r != KUBO_OK) return r;
  {
    StageTimer tm(c, KUBO_STAGE_ADJOINT, 1);
    KCHECK(launch_grad_finalize(Gacc, c.at<int>(p.o_pairs), c.at<int>(p.o_Rh), ri.idx0, p.N_h, p.W, G, c.s));
  }
  if (out) {
    StageTimer tm(c, KUBO_STAGE_KSUM, 1);
    KCHECK(launch_ksum_final(acc, n_out, inv_Nk, st, out, c.s));
  }
  return read_status(c);
}

// ------------------------------------------------------------------ batched models
// One model of a kubo_ahc_batched call: its validated plan (laid out inside the buffer of the
// stream it runs on), its R analysis and its device tables.
struct Job {
  int idx = 0;          // index in the caller's problem array
  RInfo ri;
  Plan p;
  double cost = 0.0;    // estimated device work (LPT order)
  int stream = 0;
  size_t o_tables = 0;  // offset of neg / pairs / Rh / status in the tables region
};

// Estimated device time of a model in units of FP64 flops: the FP64 pipe runs the eigensolver
// (and, in FP64 mode, everything else); tensor-core and FP32 work is discounted by its rate.
double job_cost(const Plan& p) {
  const double W = p.W, NR = p.N_R, Nk = (double)p.mesh.Nk;
  const double fourier = 6.0 * NR * W * W * (tc_fourier(p.precision) ? 10.0 / 1500.0 : 1.0);
  // the double-float eigensolver runs about 2.5x faster than the FP64 one at W = 64
  const double eig = (16.0 / 3.0 * W * W * W + 72.0 * W * W) * (df_eigh(p.precision) ? 0.4 : 1.0);
  const double rot = 24.0 * W * W * W * (f32_rotation(p.precision) ? 1.0 / 48.0 : 1.0);
  return Nk * (fourier + eig + rot + 1e4);   // + per-k fixed cost (launch/latency share)
}

// Kernel parameters of a batch, chosen by the autotuner (applied to every model): the tensor-
// core Fourier sum's rasterisation group, the reduction's symv partition cap and the option
// value of the FP32-grade rotation kernel (kubo_options.rotation_tc).
struct KernelParams {
  int group_m = 8, symv_parts = 4, rotation = 0;
};

struct BatchRun {
  std::vector<Job> jobs;
  KernelParams kp;
  int streams = 1;
  std::vector<size_t> stream_off, stream_bytes;   // stream buffers inside the workspace
  size_t tables_bytes = 0, total = 0;
};

size_t align_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

// Tables region at the start of the workspace: neg, pairs, Rh and a status word per model
// (laid out once per call; independent of the schedule).
void layout_tables(BatchRun& br) {
  Bump t;
  for (auto& j : br.jobs)
    j.o_tables = t.take(sizeof(DevStatus) + sizeof(double) * MAX_ETA +
                        sizeof(int) * (j.p.N_R + 2 * std::max(1, j.p.N_h) + 3 * std::max(1, j.p.N_h)));
  br.tables_bytes = align_up(t.off);
}

// Lay out a batch for S streams with batches of at most chunk_cap k-points: LPT assignment of
// the models (longest first, to the least loaded stream), one buffer per stream sized for its
// largest model.
void layout_batch(BatchRun& br, int S, int chunk_cap, int n_eta) {
  br.streams = S;
  std::vector<Job*> order;
  for (auto& j : br.jobs) order.push_back(&j);
  std::stable_sort(order.begin(), order.end(), [](const Job* a, const Job* b) { return a->cost > b->cost; });
  std::vector<double> load(S, 0.0);
  for (Job* j : order) {
    int best = 0;
    for (int q = 1; q < S; ++q) if (load[q] < load[best]) best = q;
    j->stream = best;
    load[best] += j->cost;
  }
  const size_t stream_budget = ((size_t)12 << 30) / (size_t)S;
  br.stream_bytes.assign(S, 0);
  for (auto& j : br.jobs) {
    Plan& p = j.p;
    p.group_m = br.kp.group_m;
    p.symv_parts = br.kp.symv_parts;
    p.rot = rotation_kernel(br.kp.rotation, p.W, false);
    const int64_t nk = p.mesh.Nk;
    int64_t c = (int64_t)(stream_budget / bytes_per_k(p.W, n_eta));
    c = std::max<int64_t>(1, std::min<int64_t>(c, chunk_cap));
    p.chunk = (int)std::min<int64_t>(c, nk);
    plan_layout(p, false, 0);
    br.stream_bytes[j.stream] = std::max(br.stream_bytes[j.stream], align_up(p.total));
  }
  br.stream_off.assign(S, 0);
  size_t off = br.tables_bytes;
  for (int q = 0; q < S; ++q) { br.stream_off[q] = off; off += br.stream_bytes[q]; }
  br.total = off;
}

struct JobTables {
  DevStatus* st;
  double* etas;   // [MAX_ETA] this model's broadenings
  int *neg, *pairs, *Rh;
};

JobTables job_tables(char* base, const Job& j) {
  char* t = base + j.o_tables;
  JobTables jt;
  jt.st = (DevStatus*)t;
  jt.etas = (double*)(t + sizeof(DevStatus));
  jt.neg = (int*)(t + sizeof(DevStatus) + sizeof(double) * MAX_ETA);
  jt.pairs = jt.neg + j.p.N_R;
  jt.Rh = jt.pairs + 2 * std::max(1, j.p.N_h);
  return jt;
}

// Everything of one model after its Hermitian check, stream-ordered on c.s without host
// synchronisation (capturable): twiddles, packed basis (and its tensor-core split), every
// k-batch, the k-sum, and a copy of the model's status word into its table slot.
kubo_status run_job(Call& c, const Job& j, const kubo_problem& pr, const kubo_options& o,
                    const JobTables& jt, double* out, int64_t nk) {
  const Plan& p = c.p;
  DevStatus* st = c.at<DevStatus>(p.o_status);
  KCHECK(cudaMemsetAsync(st, 0, sizeof(DevStatus), c.s));
  KCHECK(cudaMemcpyAsync(c.at<double>(p.o_etas), jt.etas, sizeof(double) * MAX_ETA, cudaMemcpyDeviceToDevice, c.s));
  KCHECK(launch_twiddles(c.at<double2>(p.o_tab), p.mesh.N1, p.mesh.N2, p.mesh.N3, c.s));
  KCHECK(launch_pack_basis((const double2*)pr.H_R, jt.pairs, j.ri.idx0, p.N_h, p.W, c.at<double>(p.o_Bp), c.s, p.escale));
  if (tc_fourier(p.precision))
    KCHECK(launch_basis_split(c.at<double>(p.o_Bp), jt.Rh, p.N_h, p.W, p.Npad, p.Kp, c.at<int>(p.o_cexp), c.at<char>(p.o_Bt), c.s));
  const int n_out = p.n_eta * p.n_EF;
  KCHECK(cudaMemsetAsync(c.at<char>(p.o_acc), 0, sizeof(double2) * n_out, c.s));
  Model md = make_model(c);
  md.Rh = jt.Rh;
  double* E = c.at<double>(p.o_E);
  double* Om = c.at<double>(p.o_Om);
  double2* part = c.at<double2>(p.o_part);
  double2* acc = c.at<double2>(p.o_acc);
  for (int64_t base = 0; base < nk; base += p.chunk) {
    KList kl{nullptr, base, (int)std::min<int64_t>(p.chunk, nk - base)};
    kubo_status r = run_batch(c, md, kl, E, Om, (int64_t)kl.n * p.W);
    if (r != KUBO_OK) return r;
    KCHECK(launch_ksum_partial(E, Om, p.W, kl.n, p.n_eta, (int64_t)kl.n * p.W, pr.E_F, p.n_EF, o.kT, part, p.kpb, c.s));
    KCHECK(launch_ksum_fold(part, (kl.n + p.kpb - 1) / p.kpb, n_out, acc, c.s));
  }
  KCHECK(launch_ksum_final(acc, n_out, 1.0 / (double)p.mesh.Nk, st, out, c.s));
  KCHECK(cudaMemcpyAsync(jt.st, st, sizeof(DevStatus), cudaMemcpyDeviceToDevice, c.s));
  return KUBO_OK;
}

// Issue the whole batch: fork the origin stream into S streams, run every model on its
// stream, join.  With graph != nullptr the work is captured and instantiated into *graph
// (one CUDA graph, launched by the caller); otherwise it is issued directly.  probe_out:
// per-model scratch outputs and k-limits for autotuner probes (empty = real run).
kubo_status issue_batch(const BatchRun& br, const std::vector<kubo_problem>& probs,
                        const kubo_options& o, char* ws, cudaStream_t origin,
                        const std::vector<cudaStream_t>& streams, cudaGraphExec_t* graph,
                        double* probe_out, const std::vector<int64_t>& probe_nk) {
  std::vector<cudaEvent_t> evs(br.streams + 1, nullptr);
  for (auto& e : evs)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      for (auto& x : evs) if (x) cudaEventDestroy(x);
      return KUBO_ERR_CUDA;
    }
  if (graph && cudaStreamBeginCapture(origin, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    for (auto& x : evs) cudaEventDestroy(x);
    return KUBO_ERR_CUDA;
  }
  kubo_status r = KUBO_OK;
  if (cudaEventRecord(evs[0], origin) != cudaSuccess) r = KUBO_ERR_CUDA;
  for (int q = 0; q < br.streams && r == KUBO_OK; ++q)
    if (cudaStreamWaitEvent(streams[q], evs[0], 0) != cudaSuccess) r = KUBO_ERR_CUDA;
  for (size_t i = 0; i < br.jobs.size() && r == KUBO_OK; ++i) {
    const Job& j = br.jobs[i];
    Call c;
    c.p = j.p;
    c.s = streams[j.stream];
    c.ws = ws + br.stream_off[j.stream];
    const kubo_problem& pr = probs[j.idx];
    double* out = probe_out ? probe_out + i * (size_t)(j.p.n_eta * j.p.n_EF) : pr.out;
    const int64_t nk = probe_out ? probe_nk[i] : j.p.mesh.Nk;
    r = run_job(c, j, pr, o, job_tables(ws, j), out, nk);
    c.ws = nullptr;
  }
  for (int q = 0; q < br.streams && r == KUBO_OK; ++q) {
    if (cudaEventRecord(evs[q + 1], streams[q]) != cudaSuccess ||
        cudaStreamWaitEvent(origin, evs[q + 1], 0) != cudaSuccess)
      r = KUBO_ERR_CUDA;
  }
  if (graph) {
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture(origin, &g) != cudaSuccess) r = KUBO_ERR_CUDA;
    if (r == KUBO_OK && cudaGraphInstantiate(graph, g, 0) != cudaSuccess) {
      *graph = nullptr;
      r = KUBO_ERR_CUDA;
    }
    if (g) cudaGraphDestroy(g);
  }
  if (r != KUBO_OK) cudaGetLastError();
  for (auto& x : evs) cudaEventDestroy(x);
  return r;
}

// Run a laid-out batch once (graph or direct) and return the device time of the launch.
kubo_status run_batch_once(const BatchRun& br, const std::vector<kubo_problem>& probs,
                           const kubo_options& o, char* ws, cudaStream_t origin,
                           const std::vector<cudaStream_t>& streams, bool graph,
                           double* probe_out, const std::vector<int64_t>& probe_nk, float* ms) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    cudaGetLastError();
    if (a) cudaEventDestroy(a);
    return KUBO_ERR_CUDA;
  }
  kubo_status r = KUBO_OK;
  cudaGraphExec_t ge = nullptr;
  if (graph) r = issue_batch(br, probs, o, ws, origin, streams, &ge, probe_out, probe_nk);
  if (r == KUBO_OK && cudaEventRecord(a, origin) != cudaSuccess) r = KUBO_ERR_CUDA;
  if (r == KUBO_OK) {
    if (graph) {
      if (cudaGraphLaunch(ge, origin) != cudaSuccess) r = KUBO_ERR_CUDA;
    } else {
      r = issue_batch(br, probs, o, ws, origin, streams, nullptr, probe_out, probe_nk);
    }
  }
  if (r == KUBO_OK && cudaEventRecord(b, origin) != cudaSuccess) r = KUBO_ERR_CUDA;
  if (cudaStreamSynchronize(origin) != cudaSuccess) r = KUBO_ERR_CUDA;
  if (r == KUBO_OK && ms && cudaEventElapsedTime(ms, a, b) != cudaSuccess) r = KUBO_ERR_CUDA;
  if (ge) cudaGraphExecDestroy(ge);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (r != KUBO_OK) cudaGetLastError();
  return r;
}

// process-wide cache of tuned schedules, keyed by the batch signature
std::mutex g_tune_mutex;
struct TunedSchedule {
  int streams, chunk;
  KernelParams kp;
};
std::map<std::vector<int64_t>, TunedSchedule> g_tune_cache;

std::vector<int64_t> batch_signature(const std::vector<Job>& jobs, const kubo_options& o) {
  std::vector<int64_t> sig{o.precision, o.kT > 0.0 ? 1 : 0, o.n_eta, o.rotation_tc, o.layout_unpadded};
  std::vector<std::array<int64_t, 3>> m;
  for (const auto& j : jobs) m.push_back({j.p.W, j.p.N_R, j.p.mesh.Nk});
  std::sort(m.begin(), m.end());
  for (auto& x : m) sig.insert(sig.end(), x.begin(), x.end());
  return sig;
}

}  // namespace

// ====================================================================== public ABI
extern "C" {

void kubo_options_init(kubo_options* opt) {
  if (opt) *opt = defaults();
}

const char* kubo_status_string(kubo_status s) {
  switch (s) {
    case KUBO_OK: return "KUBO_OK";
    case KUBO_ERR_INVALID_ARG: return "KUBO_ERR_INVALID_ARG: invalid argument";
    case KUBO_ERR_NOT_HERMITIAN: return "KUBO_ERR_NOT_HERMITIAN: H(-R) != H(R)^dagger or non-finite H(R)";
    case KUBO_ERR_R_NOT_CLOSED: return "KUBO_ERR_R_NOT_CLOSED: R set not closed under -R, missing R=0, or duplicate R";
    case KUBO_ERR_UNSUPPORTED: return "KUBO_ERR_UNSUPPORTED: size or precision not supported by this build";
    case KUBO_ERR_OOM: return "KUBO_ERR_OOM: device allocation failed";
    case KUBO_ERR_CUDA: return "KUBO_ERR_CUDA: CUDA runtime error";
    case KUBO_ERR_NO_CONVERGENCE: return "KUBO_ERR_NO_CONVERGENCE: eigensolver iteration cap reached";
    case KUBO_ERR_WORKSPACE: return "KUBO_ERR_WORKSPACE: workspace smaller than kubo_workspace_size()";
    case KUBO_ERR_TIMEOUT: return "KUBO_ERR_TIMEOUT: a bounded device-side wait gave up";
  }
  return "KUBO_ERR_UNKNOWN";
}

void kubo_debug_fail_allocations(int n) { g_fail_allocs.store(n > 0 ? n : 0); }

int kubo_max_orbitals(int precision) {
  return (precision >= KUBO_FP64 && precision <= KUBO_MIXED_DF) ? MAX_W : 0;
}

size_t kubo_workspace_size(int W, int N_R, const int32_t* kmesh, int n_EF,
                           const kubo_options* opt) {
  kubo_options o = opt ? *opt : defaults();
  if (o.fourier_separable) return 0;   // depends on the R set: library allocation only
  int n_eta = 1;
  if (validate_common(W, N_R, kmesh, o, n_eta) != KUBO_OK || n_EF < 1) return 0;
  Plan p;
  p.W = W; p.N_R = N_R; p.N_h = (N_R - 1) / 2; p.K = N_R; p.n_EF = n_EF; p.n_eta = n_eta;
  p.precision = o.precision;
  p.mesh = Mesh{kmesh[0], kmesh[1], kmesh[2], (int64_t)kmesh[0] * kmesh[1] * kmesh[2]};
  int64_t kb = o.k_begin, ke = o.k_end;
  if (kb == 0 && ke == 0) ke = p.mesh.Nk;
  p.chunk = o.chunk_k > 0 ? o.chunk_k : auto_chunk(W, n_eta, std::max<int64_t>(1, ke - kb));
  p.model = p.eigh = p.berry = p.ksum = true;
  p.lbuf = W > SMALL_W_MAX;
  p.fixup = tc_fourier(p.precision) && o.mixed_fixup_rel > 0.0;
  plan_layout(p, false, 0);
  return p.total;
}

size_t kubo_grad_workspace_size(int W, int N_R, const int32_t* kmesh, int n_EF,
                                const kubo_options* opt) {
  kubo_options o = opt ? *opt : defaults();
  int n_eta = 1;
  if (validate_common(W, N_R, kmesh, o, n_eta) != KUBO_OK || n_EF < 1) return 0;
  if (o.precision != KUBO_FP64) return 0;
  Plan p;
  p.W = W; p.N_R = N_R; p.N_h = (N_R - 1) / 2; p.K = N_R; p.n_EF = n_EF; p.n_eta = n_eta;
  p.precision = o.precision;
  p.mesh = Mesh{kmesh[0], kmesh[1], kmesh[2], (int64_t)kmesh[0] * kmesh[1] * kmesh[2]};
  int64_t kb = o.k_begin, ke = o.k_end;
  if (kb == 0 && ke == 0) ke = p.mesh.Nk;
  p.chunk = o.chunk_k > 0 ? o.chunk_k
                          : auto_chunk(W, n_eta, std::max<int64_t>(1, ke - kb), grad_bytes_per_k(W, N_R));
  p.model = p.eigh = p.berry = p.ksum = p.grad = true;
  p.lbuf = W > SMALL_W_MAX;
  plan_layout(p, false, 0);
  return p.total;
}

kubo_status kubo_ahc(const double* H_R, const int32_t* R_vecs, int W, int N_R,
                     const int32_t* kmesh, const double* E_F, int n_EF, double eta, double* out,
                     const kubo_options* opt) {
  try {
    kubo_options o = opt ? *opt : defaults();
    if (!H_R || !E_F || !out) return KUBO_ERR_INVALID_ARG;
    if (o.n_eta == 0 && !finite_nonneg(eta)) return KUBO_ERR_INVALID_ARG;
    Call c;
    RInfo ri;
    int64_t kb, ke;
    kubo_status r = setup_ahc(c, o, R_vecs, W, N_R, kmesh, n_EF, ri, kb, ke, false);
    if (r != KUBO_OK) return r;
    r = c.acquire(o);
    if (r != KUBO_OK) return r;
    r = ahc_device(c, o, H_R, ri, E_F, eta, out, kb, ke);
    c.release();
    if (r == KUBO_OK && cudaStreamSynchronize(c.s) != cudaSuccess) r = KUBO_ERR_CUDA;
    return r;
  } catch (const std::bad_alloc&) {
    return KUBO_ERR_OOM;
  } catch (...) {
    return KUBO_ERR_CUDA;
  }
}

kubo_status kubo_ahc_host(const double* H_R, const int32_t* R_vecs, int W, int N_R,
                          const int32_t* kmesh, const double* E_F, int n_EF, double eta,
                          double* out, const kubo_options* opt) {
  try {
    kubo_options o = opt ? *opt : defaults();
    if (!H_R || !E_F || !out) return KUBO_ERR_INVALID_ARG;
    if (o.n_eta == 0 && !finite_nonneg(eta)) return KUBO_ERR_INVALID_ARG;
    Call c;
    RInfo ri;
    int64_t kb, ke;
    kubo_status r = setup_ahc(c, o, R_vecs, W, N_R, kmesh, n_EF, ri, kb, ke, true);
    if (r != KUBO_OK) return r;
    r = c.acquire(o);
    if (r != KUBO_OK) return r;
    const Plan& p = c.p;
    const size_t hr_bytes = sizeof(double2) * (size_t)N_R * W * W;
    if (cudaMemcpyAsync(c.at<char>(p.o_HR), H_R, hr_bytes, cudaMemcpyHostToDevice, c.s) != cudaSuccess ||
        cudaMemcpyAsync(c.at<char>(p.o_EF), E_F, sizeof(double) * n_EF, cudaMemcpyHostToDevice, c.s) != cudaSuccess) {
      cudaGetLastError();
      c.release();
      return KUBO_ERR_CUDA;
    }
    r = ahc_device(c, o, c.at<double>(p.o_HR), ri, c.at<double>(p.o_EF), eta, c.at<double>(p.o_out), kb, ke);
    if (r == KUBO_OK) {
      if (cudaMemcpyAsync(out, c.at<double>(p.o_out), sizeof(double) * p.n_eta * n_EF, cudaMemcpyDeviceToHost, c.s) != cudaSuccess ||
          cudaStreamSynchronize(c.s) != cudaSuccess) {
        cudaGetLastError();
        r = KUBO_ERR_CUDA;
      }
    }
    c.release();
    if (cudaStreamSynchronize(c.s) != cudaSuccess && r == KUBO_OK) r = KUBO_ERR_CUDA;
    return r;
  } catch (const std::bad_alloc&) {
    return KUBO_ERR_OOM;
  } catch (...) {
    return KUBO_ERR_CUDA;
  }
}

kubo_status kubo_ahc_grad(const double* H_R, const int32_t* R_vecs, int W, int N_R,
                          const int32_t* kmesh, const double* E_F, int n_EF, double eta,
                          const double* dL_dout, double* grad_H_R, double* out,
                          const kubo_options* opt) {
  try {
    kubo_options o = opt ? *opt : defaults();
    if (!H_R || !E_F || !dL_dout || !grad_H_R) return KUBO_ERR_INVALID_ARG;
    if (o.fourier_separable) return KUBO_ERR_UNSUPPORTED;
    if (o.n_eta == 0 && !finite_nonneg(eta)) return KUBO_ERR_INVALID_ARG;
    if (!std::isfinite(o.grad_eps)) return KUBO_ERR_INVALID_ARG;
    Call c;
    RInfo ri;
    int64_t kb, ke;
    kubo_status r = setup_ahc(c, o, R_vecs, W, N_R, kmesh, n_EF, ri, kb, ke, false);
    if (r != KUBO_OK) return r;
    if (o.precision != KUBO_FP64) return KUBO_ERR_UNSUPPORTED;
    Plan& p = c.p;
    p.grad = true;
    p.fixup = false;
    p.chunk = o.chunk_k > 0 ? o.chunk_k
                            : auto_chunk(W, p.n_eta, std::max<int64_t>(1, ke - kb), grad_bytes_per_k(W, N_R));
    plan_layout(p, false, 0);
    r = c.acquire(o);
    if (r != KUBO_OK) return r;
    r = ahc_grad_device(c, o, H_R, ri, E_F, eta, dL_dout, (double2*)grad_H_R, out, kb, ke);
    c.release();
    if (cudaStreamSynchronize(c.s) != cudaSuccess && r == KUBO_OK) r = KUBO_ERR_CUDA;
    return r;
  } catch (const std::bad_alloc&) {
    return KUBO_ERR_OOM;
  } catch (...) {
    return KUBO_ERR_CUDA;
  }
}

kubo_status kubo_ahc_batched(kubo_problem* probs, int n_probs, const kubo_options* opt,
                             kubo_batch_schedule* sched) {
  std::vector<cudaStream_t> streams;
  char* ws = nullptr;
  cudaStream_t user = nullptr, origin = nullptr;   // origin: the library's own capture stream
  auto finish = [&](kubo_status r) {
    for (auto& q : streams)
      if (q && cudaStreamSynchronize(q) != cudaSuccess && r == KUBO_OK) r = KUBO_ERR_CUDA;
    if (origin) {
      if (ws) cudaFreeAsync(ws, origin);
      if (cudaStreamSynchronize(origin) != cudaSuccess && r == KUBO_OK) r = KUBO_ERR_CUDA;
      cudaStreamDestroy(origin);
    }
    for (auto& q : streams) if (q) cudaStreamDestroy(q);
    cudaGetLastError();
    return r;
  };
  try {
    kubo_options o = opt ? *opt : defaults();
    if (!probs || n_probs < 1) return KUBO_ERR_INVALID_ARG;
    if (o.k_begin != 0 || o.k_end != 0 || o.workspace) return KUBO_ERR_INVALID_ARG;
    if (o.fourier_separable) return KUBO_ERR_UNSUPPORTED;
    kubo_batch_schedule sc{};
    if (sched) sc = *sched;
    if (sc.streams < 0 || sc.chunk_k < 0) return KUBO_ERR_INVALID_ARG;
    user = (cudaStream_t)o.stream;
    // ---- validate every model; invalid ones are skipped (their status says why)
    std::vector<kubo_problem> P(probs, probs + n_probs);
    BatchRun br;
    kubo_status first = KUBO_OK;
    int n_eta = 1;
    for (int i = 0; i < n_probs; ++i) {
      kubo_problem& q = probs[i];
      kubo_status r = KUBO_OK;
      if (!q.H_R || !q.E_F || !q.out || !q.R_vecs || q.n_EF < 1) r = KUBO_ERR_INVALID_ARG;
      else if (o.n_eta == 0 && !finite_nonneg(q.eta)) r = KUBO_ERR_INVALID_ARG;
      if (r == KUBO_OK) r = validate_common(q.W, q.N_R, q.kmesh, o, n_eta);
      Job j;
      if (r == KUBO_OK) r = analyze_R(q.R_vecs, q.N_R, j.ri);
      q.status = r;
      if (r != KUBO_OK) {
        if (first == KUBO_OK) first = r;
        continue;
      }
      j.idx = i;
      Plan& p = j.p;
      p.W = q.W; p.N_R = q.N_R; p.N_h = j.ri.N_h; p.K = q.N_R; p.n_EF = q.n_EF; p.n_eta = n_eta;
      p.precision = o.precision;
      p.mesh = Mesh{q.kmesh[0], q.kmesh[1], q.kmesh[2], (int64_t)q.kmesh[0] * q.kmesh[1] * q.kmesh[2]};
      p.model = p.eigh = p.berry = p.ksum = true;
      p.lbuf = q.W > SMALL_W_MAX;
      p.fixup = false;
      p.scale_ok = f32_rotation(p.precision);
      p.ql_cap = o.ql_max_sweeps;
      p.ql_fp64 = o.ql_fp64 != 0;
      p.rot = rotation_kernel(o.rotation_tc, q.W, o.layout_unpadded != 0);
      j.cost = job_cost(p);
      br.jobs.push_back(std::move(j));
    }
    if (br.jobs.empty()) return first;
    const int n_jobs = (int)br.jobs.size();
    // ---- schedule: given, cached, tuned or default
    const int kStreamsMax = 16;
    int S = sc.streams > 0 ? std::min({sc.streams, n_jobs, kStreamsMax}) : 0;
    int chunk = sc.chunk_k > 0 ? sc.chunk_k : 0;
    const bool graph = sc.graph >= 0;
    sc.probe_ms = 0.0;
    sc.tuned_candidates = 0;
    if (sc.fourier_group_m < 0 || sc.fourier_group_m > 64 || sc.symv_parts < 0 || sc.symv_parts > 8 ||
        sc.rotation < 0 || sc.rotation > 3)
      return KUBO_ERR_INVALID_ARG;
    // kernel parameters: given, else the defaults (tuned below when tune = 1)
    br.kp.group_m = sc.fourier_group_m > 0 ? sc.fourier_group_m : 8;
    br.kp.symv_parts = sc.symv_parts > 0 ? sc.symv_parts : 4;
    br.kp.rotation = o.layout_unpadded ? 2 : (sc.rotation > 0 ? sc.rotation : o.rotation_tc);
    const bool tune_gm = sc.tune && sc.fourier_group_m == 0 && tc_fourier(o.precision);
    const bool tune_sp = sc.tune && sc.symv_parts == 0;
    const bool tune_rot = sc.tune && sc.rotation == 0 && !o.layout_unpadded && o.rotation_tc == 0 &&
                          f32_rotation(o.precision);
    std::vector<int64_t> sig;
    bool need_tune = sc.tune && (S == 0 || chunk == 0 || tune_gm || tune_sp || tune_rot);
    if (need_tune) {
      sig = batch_signature(br.jobs, o);
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      auto it = g_tune_cache.find(sig);
      if (it != g_tune_cache.end()) {
        if (S == 0) S = std::min(it->second.streams, n_jobs);
        if (chunk == 0) chunk = it->second.chunk;
        if (tune_gm) br.kp.group_m = it->second.kp.group_m;
        if (tune_sp) br.kp.symv_parts = it->second.kp.symv_parts;
        if (tune_rot) br.kp.rotation = it->second.kp.rotation;
        need_tune = false;
      }
    }
    // ---- one allocation for the largest layout any candidate can need, plus probe outputs
    std::vector<int> cand_S, cand_C;
    if (need_tune) {
      for (int v : {1, 2, 4, 8}) if ((S == 0 || v == S) && v <= n_jobs) cand_S.push_back(v);
      if (S != 0 && cand_S.empty()) cand_S.push_back(S);
      for (int v : {8192, 65536}) if (chunk == 0 || v == chunk) cand_C.push_back(v);
      if (chunk != 0 && cand_C.empty()) cand_C.push_back(chunk);
    } else {
      cand_S.push_back(S > 0 ? S : std::min(4, n_jobs));
      cand_C.push_back(chunk > 0 ? chunk : 65536);
    }
    layout_tables(br);
    size_t need = 0;
    for (int cs : cand_S)
      for (int cc : cand_C) {
        layout_batch(br, cs, cc, n_eta);
        need = std::max(need, br.total);
      }
    size_t probe_doubles = 0;
    for (const auto& j : br.jobs) probe_doubles += (size_t)j.p.n_eta * j.p.n_EF;
    const size_t probe_off = align_up(need);
    // the batch runs behind the caller's stream on a stream of its own (the legacy default
    // stream cannot be captured), and the call returns when it is done
    {
      cudaEvent_t ev = nullptr;
      if (cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        origin = nullptr;
        return finish(KUBO_ERR_CUDA);
      }
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventRecord(ev, user) != cudaSuccess || cudaStreamWaitEvent(origin, ev, 0) != cudaSuccess) {
        if (ev) cudaEventDestroy(ev);
        return finish(KUBO_ERR_CUDA);
      }
      cudaEventDestroy(ev);
    }
    if (lib_malloc_async((void**)&ws, probe_off + sizeof(double) * probe_doubles, origin) != cudaSuccess) {
      cudaGetLastError();
      ws = nullptr;
      return finish(KUBO_ERR_OOM);
    }
    const int max_S = *std::max_element(cand_S.begin(), cand_S.end());
    streams.assign(max_S, nullptr);
    for (auto& q : streams)
      if (cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        q = nullptr;
        return finish(KUBO_ERR_CUDA);
      }
    // ---- tables and the Hermitian check of every model (one host synchronisation)
#define BCHECK(expr)                                  \
  do {                                                \
    if ((expr) != cudaSuccess) return finish(KUBO_ERR_CUDA); \
  } while (0)
    std::vector<std::array<double, MAX_ETA>> eta_h(br.jobs.size());
    for (size_t i = 0; i < br.jobs.size(); ++i) {
      eta_h[i].fill(0.0);
      if (o.n_eta > 0) for (int e = 0; e < o.n_eta; ++e) eta_h[i][e] = o.etas[e];
      else eta_h[i][0] = probs[br.jobs[i].idx].eta;
    }
    for (size_t i = 0; i < br.jobs.size(); ++i) {
      const Job& j = br.jobs[i];
      const JobTables jt = job_tables(ws, j);
      BCHECK(cudaMemsetAsync(jt.st, 0, sizeof(DevStatus), origin));
      BCHECK(cudaMemcpyAsync(jt.etas, eta_h[i].data(), sizeof(double) * MAX_ETA, cudaMemcpyHostToDevice, origin));
      BCHECK(cudaMemcpyAsync(jt.neg, j.ri.neg.data(), sizeof(int) * j.p.N_R, cudaMemcpyHostToDevice, origin));
      if (j.p.N_h > 0) {
        BCHECK(cudaMemcpyAsync(jt.pairs, j.ri.pairs.data(), sizeof(int) * 2 * j.p.N_h, cudaMemcpyHostToDevice, origin));
        BCHECK(cudaMemcpyAsync(jt.Rh, j.ri.Rh.data(), sizeof(int) * 3 * j.p.N_h, cudaMemcpyHostToDevice, origin));
      }
      BCHECK(launch_check_hermitian((const double2*)probs[j.idx].H_R, jt.neg, j.p.N_R, j.p.W, jt.st, origin));
      BCHECK(launch_hermitian_verdict(jt.st, origin));
    }
    std::vector<DevStatus> hs(br.jobs.size());
    for (size_t i = 0; i < br.jobs.size(); ++i)
      BCHECK(cudaMemcpyAsync(&hs[i], job_tables(ws, br.jobs[i]).st, sizeof(DevStatus), cudaMemcpyDeviceToHost, origin));
    BCHECK(cudaStreamSynchronize(origin));
    {
      std::vector<Job> ok;
      for (size_t i = 0; i < br.jobs.size(); ++i) {
        const kubo_status r = bits_to_status(hs[i].bits);
        if (r != KUBO_OK) {
          probs[br.jobs[i].idx].status = r;
          if (first == KUBO_OK) first = r;
        } else {
          // a model outside the FP32 steps' comfortable range is scaled by a power of two
          // (basis and broadenings; its eigenvalues are scaled back per batch)
          Job& j = br.jobs[i];
          j.p.escale = j.p.scale_ok ? range_exponent(herm_max(hs[i])) : 0;
          if (j.p.escale != 0) {
            for (double& x : eta_h[i]) x = std::ldexp(x, j.p.escale);
            BCHECK(cudaMemcpyAsync(job_tables(ws, j).etas, eta_h[i].data(), sizeof(double) * MAX_ETA,
                                   cudaMemcpyHostToDevice, origin));
          }
          ok.push_back(std::move(j));
        }
      }
      br.jobs.swap(ok);
    }
    if (br.jobs.empty()) return finish(first);
    std::vector<kubo_problem> PP(probs, probs + n_probs);
    double* probe_out = (double*)(ws + probe_off);
    // ---- autotune: time every candidate schedule on a probe of each model's first k-points
    if (need_tune) {
      std::vector<int64_t> probe_nk;
      for (const auto& j : br.jobs)
        probe_nk.push_back(std::min<int64_t>(j.p.mesh.Nk, std::max<int64_t>(4096, j.p.mesh.Nk / 16)));
      float best = -1.f;
      int bS = cand_S[0], bC = cand_C[0];
      for (int cs : cand_S)
        for (int cc : cand_C) {
          layout_batch(br, std::min(cs, (int)br.jobs.size()), cc, n_eta);
          float ms = 0.f;
          kubo_status r = run_batch_once(br, PP, o, ws, origin, streams, graph, probe_out, probe_nk, &ms);
          if (r != KUBO_OK) return finish(r);
          ++sc.tuned_candidates;
          if (best < 0.f || ms < best) { best = ms; bS = cs; bC = cc; }
        }
      S = bS;
      chunk = bC;
      // then the kernel parameters, one at a time from the defaults (coordinate search), on
      // the chosen schedule
      layout_batch(br, std::min(S, (int)br.jobs.size()), chunk, n_eta);
      auto try_params = [&](KernelParams kp) -> kubo_status {
        const KernelParams keep = br.kp;
        br.kp = kp;
        layout_batch(br, std::min(S, (int)br.jobs.size()), chunk, n_eta);
        float ms = 0.f;
        kubo_status r = run_batch_once(br, PP, o, ws, origin, streams, graph, probe_out, probe_nk, &ms);
        if (r != KUBO_OK) return r;
        ++sc.tuned_candidates;
        if (ms < best) best = ms;
        else br.kp = keep;
        return KUBO_OK;
      };
      if (tune_gm)
        for (int v : {4, 16}) {
          KernelParams kp = br.kp;
          kp.group_m = v;
          kubo_status r = try_params(kp);
          if (r != KUBO_OK) return finish(r);
        }
      if (tune_sp)
        for (int v : {2, 8}) {
          KernelParams kp = br.kp;
          kp.symv_parts = v;
          kubo_status r = try_params(kp);
          if (r != KUBO_OK) return finish(r);
        }
      if (tune_rot)
        for (int v : {2, 3}) {   // FP32 SIMT everywhere, 3xTF32 everywhere (vs the automatic rule)
          KernelParams kp = br.kp;
          kp.rotation = v;
          kubo_status r = try_params(kp);
          if (r != KUBO_OK) return finish(r);
        }
      sc.probe_ms = best;
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      g_tune_cache[sig] = TunedSchedule{S, chunk, br.kp};
    } else {
      S = cand_S[0];
      chunk = cand_C[0];
    }
    // ---- the real run
    layout_batch(br, std::min(S, (int)br.jobs.size()), chunk, n_eta);
    kubo_status r = run_batch_once(br, PP, o, ws, origin, streams, graph, nullptr, {}, nullptr);
    if (r != KUBO_OK) return finish(r);
    for (size_t i = 0; i < br.jobs.size(); ++i)
      BCHECK(cudaMemcpyAsync(&hs[i], job_tables(ws, br.jobs[i]).st, sizeof(DevStatus), cudaMemcpyDeviceToHost, origin));
    BCHECK(cudaStreamSynchronize(origin));
    for (size_t i = 0; i < br.jobs.size(); ++i) {
      const kubo_status rj = bits_to_status(hs[i].bits);
      probs[br.jobs[i].idx].status = rj;
      if (rj != KUBO_OK && first == KUBO_OK) first = rj;
    }
    sc.streams = br.streams;
    sc.chunk_k = chunk;
    sc.graph = graph ? 1 : -1;
    sc.fourier_group_m = br.kp.group_m;
    sc.symv_parts = br.kp.symv_parts;
    sc.rotation = br.kp.rotation;
    if (sched) *sched = sc;
    return finish(first);
#undef BCHECK
  } catch (const std::bad_alloc&) {
    return finish(KUBO_ERR_OOM);
  } catch (...) {
    return finish(KUBO_ERR_CUDA);
  }
}

kubo_status kubo_check_bounded_wait(uint32_t spins, void* stream) {
  try {
    if (spins < 1) return KUBO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    DevStatus* st = nullptr;
    if (cudaMallocAsync((void**)&st, sizeof(DevStatus), s) != cudaSuccess) {
      cudaGetLastError();
      return KUBO_ERR_OOM;
    }
    kubo_status r = KUBO_OK;
    DevStatus h;
    if (cudaMemsetAsync(st, 0, sizeof(DevStatus), s) != cudaSuccess ||
        launch_bounded_wait_check(spins, st, s) != cudaSuccess ||
        cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      r = KUBO_ERR_CUDA;
    else
      r = bits_to_status(h.bits);
    cudaFreeAsync(st, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && r == KUBO_OK) r = KUBO_ERR_CUDA;
    cudaGetLastError();
    return r;
  } catch (...) {
    return KUBO_ERR_CUDA;
  }
}

kubo_status kubo_ahc_k(const double* H_R, const int32_t* R_vecs, int W, int N_R,
                       const int32_t* kmesh, const int64_t* kidx, int64_t n_k, double eta,
                       double* E, double* Omega, const kubo_options* opt) {
  try {
    kubo_options o = opt ? *opt : defaults();
    if (!H_R || !kidx || !E || !Omega || n_k < 1) return KUBO_ERR_INVALID_ARG;
    if (o.fourier_separable) return KUBO_ERR_UNSUPPORTED;
    if (o.n_eta == 0 && !finite_nonneg(eta)) return KUBO_ERR_INVALID_ARG;
    o.k_begin = o.k_end = 0;
    Call c;
    RInfo ri;
    int64_t kb, ke;
    kubo_status r = setup_ahc(c, o, R_vecs, W, N_R, kmesh, 1, ri, kb, ke, false);
    if (r != KUBO_OK) return r;
    // per-k mode: no k-sum, batches over the list
    Plan& p = c.p;
    p.ksum = false;
    p.fixup = false;   // per-k results carry no Fermi level to protect
    p.chunk = o.chunk_k > 0 ? o.chunk_k : auto_chunk(W, p.n_eta, n_k);
    plan_layout(p, false, 0);
    r = c.acquire(o);
    if (r != KUBO_OK) return r;
    r = check_klist(c, kidx, n_k);
    if (r == KUBO_OK) r = prepare_model(c, H_R, ri);
    if (r == KUBO_OK) r = upload_etas(c, o, eta);
    if (r == KUBO_OK) {
      const Model md = make_model(c);
      for (int64_t t0 = 0; t0 < n_k && r == KUBO_OK; t0 += p.chunk) {
        KList kl{kidx + t0, 0, (int)std::min<int64_t>(p.chunk, n_k - t0)};
        r = run_batch(c, md, kl, E + t0 * W, Omega + t0 * W, n_k * W);
      }
      if (r == KUBO_OK) r = read_status(c);
    }
    c.release();
    if (cudaStreamSynchronize(c.s) != cudaSuccess && r == KUBO_OK) r = KUBO_ERR_CUDA;
    return r;
  } catch (const std::bad_alloc&) {
    return KUBO_ERR_OOM;
  } catch (...) {
    return KUBO_ERR_CUDA;
  }
}

kubo_status kubo_bloch(const double* H_R, const int32_t* R_vecs, int W, int N_R,
                       const int32_t* kmesh, const int64_t* kidx, int64_t n_k, double* Hk,
                       double* dHx, double* dHy, const kubo_options* opt) {
  try {
    kubo_options o = opt ? *opt : defaults();
    if (!H_R || !kidx || !Hk || !dHx || !dHy || n_k < 1) return KUBO_ERR_INVALID_ARG;
    int n_eta = 1;
    kubo_status r = validate_common(W, N_R, kmesh, o, n_eta);
    if (r != KUBO_OK) return r;
    if (!R_vecs) return KUBO_ERR_INVALID_ARG;
    RInfo ri;
    r = analyze_R(R_vecs, N_R, ri);
    if (r != KUBO_OK) return r;
    Call c;
    Plan& p = c.p;
    p.W = W; p.N_R = N_R; p.N_h = ri.N_h; p.K = N_R; p.n_EF = 1; p.n_eta = 1;
    p.precision = o.precision;
    p.mesh = Mesh{kmesh[0], kmesh[1], kmesh[2], (int64_t)kmesh[0] * kmesh[1] * kmesh[2]};
    p.chunk = tc_fourier(o.precision) ? (int)std::min<int64_t>(n_k, o.chunk_k > 0 ? o.chunk_k : 8192) : 0;
    p.model = true;
    plan_layout(p, false, 0);
    c.s = (cudaStream_t)o.stream;
    c.prof = o.profile;
    r = c.acquire(o);
    if (r != KUBO_OK) return r;
    r = check_klist(c, kidx, n_k);
    if (r == KUBO_OK) r = prepare_model(c, H_R, ri);
    if (r == KUBO_OK) {
      const Model md = make_model(c);
      const size_t WW = (size_t)W * W;
      if (tc_fourier(p.precision)) {
        DevStatus* st = c.at<DevStatus>(p.o_status);
        double* C64 = c.at<double>(p.o_C64);
        for (int64_t t0 = 0; t0 < n_k && r == KUBO_OK; t0 += p.chunk) {
          KList kl{kidx + t0, 0, (int)std::min<int64_t>(p.chunk, n_k - t0)};
          const int Mb = tc_pad_m(kl.n);
          if (launch_coef_split(md, p.mesh, kl, Mb, p.Kp, c.at<char>(p.o_A), c.s) != cudaSuccess ||
              launch_fourier_tc(c.at<char>(p.o_A), c.at<char>(p.o_Bt), c.at<int>(p.o_cexp), Mb, p.Npad, p.Kp, kl.n, C64, p.Npad, st, c.s, p.Npad) != cudaSuccess ||
              launch_unpack_rows(C64, p.Npad, W, kl.n, Hk + t0 * WW, dHx + t0 * WW, dHy + t0 * WW, c.s) != cudaSuccess) {
            cudaGetLastError();
            r = KUBO_ERR_CUDA;
          }
        }
        if (r == KUBO_OK) r = read_status(c);
      }
      const int64_t step = 1 << 19;   // grid.y = step / 16 <= 65535
      for (int64_t t0 = 0; t0 < n_k && r == KUBO_OK && !tc_fourier(p.precision); t0 += step) {
        KList kl{kidx + t0, 0, (int)std::min<int64_t>(step, n_k - t0)};
        if (launch_fourier_fp64(md, p.mesh, kl, Hk + t0 * WW, dHx + t0 * WW, dHy + t0 * WW, c.s) != cudaSuccess) {
          cudaGetLastError();
          r = KUBO_ERR_CUDA;
        }
      }
      if (r == KUBO_OK) r = read_status(c);
    }
    c.release();
    if (cudaStreamSynchronize(c.s) != cudaSuccess && r == KUBO_OK) r = KUBO_ERR_CUDA;
    return r;
  } catch (...) {
    return KUBO_ERR_CUDA;
  }
}

kubo_status kubo_eigh_batched(const double* A, int W, int64_t n, double* E, double* U,
                              const kubo_options* opt) {
  try {
    kubo_options o = opt ? *opt : defaults();
    if (!A || !E || n < 1 || W < 1 || o.chunk_k < 0 || o.ql_max_sweeps < 0) return KUBO_ERR_INVALID_ARG;
    if (W > MAX_W) return KUBO_ERR_UNSUPPORTED;
    Call c;
    Plan& p = c.p;
    p.W = W; p.n_eta = 1; p.n_EF = 1;
    p.chunk = o.chunk_k > 0 ? o.chunk_k : auto_chunk(W, 1, n);
    p.ql_cap = o.ql_max_sweeps;
    p.eigh = true;
    p.lbuf = W > SMALL_W_MAX;
    plan_layout(p, false, 0);
    c.s = (cudaStream_t)o.stream;
    kubo_status r = c.acquire(o);
    if (r != KUBO_OK) return r;
    if (cudaMemsetAsync(c.at<char>(p.o_status), 0, sizeof(DevStatus), c.s) != cudaSuccess) r = KUBO_ERR_CUDA;
    EighBufs eb = make_eigh_bufs(c);
    DevStatus* st = c.at<DevStatus>(p.o_status);
    const size_t WW = (size_t)W * W;
    for (int64_t t0 = 0; t0 < n && r == KUBO_OK; t0 += p.chunk) {
      int nn = (int)std::min<int64_t>(p.chunk, n - t0);
      if (launch_tridiag(A + t0 * WW, W, nn, eb, c.s) != cudaSuccess ||
          launch_ql(W, nn, eb, st, c.s) != cudaSuccess ||
          eigh_vectors(c, nn, eb, E + t0 * W, U ? (double2*)U + t0 * WW : nullptr) != cudaSuccess) {
        cudaGetLastError();
        r = KUBO_ERR_CUDA;
      }
    }
    if (r == KUBO_OK) r = read_status(c);
    c.release();
    if (cudaStreamSynchronize(c.s) != cudaSuccess && r == KUBO_OK) r = KUBO_ERR_CUDA;
    return r;
  } catch (...) {
    return KUBO_ERR_CUDA;
  }
}

kubo_status kubo_berry_batched(const double* E, const double* U, const double* dHx,
                               const double* dHy, int W, int64_t n, double eta, double* Omega,
                               const kubo_options* opt) {
  try {
    kubo_options o = opt ? *opt : defaults();
    if (!E || !U || !dHx || !dHy || !Omega || n < 1 || W < 1) return KUBO_ERR_INVALID_ARG;
    if (W > MAX_W) return KUBO_ERR_UNSUPPORTED;
    if (o.n_eta > MAX_ETA) return KUBO_ERR_UNSUPPORTED;
    if (o.n_eta == 0 && !finite_nonneg(eta)) return KUBO_ERR_INVALID_ARG;
    for (int e = 0; e < o.n_eta; ++e)
      if (!o.etas || !finite_nonneg(o.etas[e])) return KUBO_ERR_INVALID_ARG;
    Call c;
    Plan& p = c.p;
    p.W = W; p.n_eta = o.n_eta > 0 ? o.n_eta : 1; p.n_EF = 1;
    p.lbuf = W > SMALL_W_MAX;   // the GEMM products of large orders go through the workspace
    p.chunk = p.lbuf ? (o.chunk_k > 0 ? o.chunk_k : auto_chunk(W, p.n_eta, n)) : 0;
    plan_layout(p, false, 0);
    c.s = (cudaStream_t)o.stream;
    kubo_status r = c.acquire(o);
    if (r != KUBO_OK) return r;
    r = upload_etas(c, o, eta);
    const size_t WW = (size_t)W * W;
    const int64_t step = p.lbuf ? p.chunk : 1 << 30;
    for (int64_t t0 = 0; t0 < n && r == KUBO_OK; t0 += step) {
      int nn = (int)std::min<int64_t>(step, n - t0);
      if (berry_any(c, E + t0 * W, (const double2*)U + t0 * WW, dHx + t0 * WW, dHy + t0 * WW, (int64_t)WW,
                    false, nn, false, Omega + t0 * W, n * W) != cudaSuccess) {
        cudaGetLastError();
        r = KUBO_ERR_CUDA;
      }
    }
    c.release();
    if (cudaStreamSynchronize(c.s) != cudaSuccess && r == KUBO_OK) r = KUBO_ERR_CUDA;
    return r;
  } catch (...) {
    return KUBO_ERR_CUDA;
  }
}

}  // extern "C"
