// Allocation-free variant of the batched Hermitian eigensolver entry point.
//
// Some callers cannot let a library allocate device memory during a call: applications
// whose own allocator reserves (nearly) all of the GPU's memory up front, so a cudaMalloc
// from inside the library fails or fragments their pool; and latency-critical loops in
// which a cudaMalloc/cudaFree would synchronise the device and stall every other stream.
// kubo_eigh_batched_noalloc serves them: its intermediates live in one fixed block of
// device memory that is part of the library image itself (a file-scope __device__ array),
// so the call performs no allocation of any kind.  It runs the same three kernels as
// kubo_eigh_batched, over passes of as many matrices as fit in that block.
#include "kubo_internal.cuh"

namespace kubo {
namespace {

constexpr size_t kScratchBytes = (size_t)32 << 20;   // 32 MiB, held by every GPU that loads the library
constexpr int kMaxW = 64;
constexpr size_t kAlign = 256;

static __device__ __align__(256) unsigned char noalloc_scratch[kScratchBytes];

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// bytes of the block used by a pass of B matrices of order W (status word first)
size_t pass_bytes(int W, int64_t B) {
  return align_up(sizeof(DevStatus)) + 4 * align_up(sizeof(double) * B * W) +
         align_up(sizeof(double2) * B * W) + align_up(sizeof(double2) * B * W * W);
}

int64_t pass_capacity(int W) {
  const size_t per = sizeof(double) * 4 * W + sizeof(double2) * W + sizeof(double2) * W * W;
  int64_t B = (int64_t)(kScratchBytes / per);
  while (B > 0 && pass_bytes(W, B) > kScratchBytes) --B;
  return B;
}

// Device address of the block on the current device.  The host-side symbol is only a stand-in
// and must never reach a kernel.  The address is looked up on every call, with the caller's
// device current: the lookup allocates nothing, and a cached address could outlive a reset of
// the device's primary context, after which the block may be loaded elsewhere.
kubo_status scratch_address(char** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, noalloc_scratch);
  if (e != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return KUBO_ERR_CUDA;
  }
  *out = (char*)p;
  return KUBO_OK;
}

}  // namespace
}  // namespace kubo

using namespace kubo;

extern "C" kubo_status kubo_eigh_batched_noalloc(const double* A, int W, int64_t n, double* E,
                                                 double* U, void* stream) {
  try {
    if (!A || !E || n < 1 || W < 1) return KUBO_ERR_INVALID_ARG;
    if (W > kMaxW) return KUBO_ERR_UNSUPPORTED;   // beyond the block's and the kernels' limit
    const int64_t B = pass_capacity(W);
    if (B < 1) return KUBO_ERR_UNSUPPORTED;
    char* base = nullptr;
    kubo_status r = scratch_address(&base);
    if (r != KUBO_OK) return r;
    cudaStream_t s = (cudaStream_t)stream;

    // carve the block for a pass of B matrices
    size_t off = 0;
    auto take = [&](size_t bytes) { char* p = base + off; off += align_up(bytes); return p; };
    DevStatus* st = (DevStatus*)take(sizeof(DevStatus));
    EighBufs b;
    b.d = (double*)take(sizeof(double) * B * W);
    b.e = (double*)take(sizeof(double) * B * W);
    b.tau = (double*)take(sizeof(double) * B * W);
    b.lam = (double*)take(sizeof(double) * B * W);
    b.phase = (double2*)take(sizeof(double2) * B * W);
    b.refl = (double2*)take(sizeof(double2) * B * W * W);

    // the block keeps the previous call's contents: the status word must start at zero;
    // every other buffer is fully written before it is read
    if (cudaMemsetAsync(st, 0, sizeof(DevStatus), s) != cudaSuccess) {
      cudaGetLastError();
      return KUBO_ERR_CUDA;
    }
    const size_t WW = (size_t)W * W;
    for (int64_t t0 = 0; t0 < n; t0 += B) {
      const int nn = (int)(n - t0 < B ? n - t0 : B);
      if (launch_tridiag(A + t0 * WW, W, nn, b, s) != cudaSuccess ||
          launch_ql(W, nn, b, st, s) != cudaSuccess ||
          launch_backtransform(W, nn, b, E + t0 * W, U ? (double2*)U + t0 * WW : nullptr, s) !=
              cudaSuccess) {
        cudaGetLastError();
        return KUBO_ERR_CUDA;
      }
    }
    DevStatus h;
    if (cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      return KUBO_ERR_CUDA;
    }
    if (h.bits & ST_NO_CONVERGENCE) return KUBO_ERR_NO_CONVERGENCE;
    return KUBO_OK;
  } catch (...) {
    return KUBO_ERR_CUDA;
  }
}
