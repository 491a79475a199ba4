// lmfao_cart_variances_noalloc: the CART split variances of lmfao_cart_variances without
// any device allocation.
//
// lmfao_cart_variances stages one small descriptor per query (where its COUNT, SUM(y) and
// SUM(y^2) cells live) in device memory that it allocates on every call. Some callers
// cannot allocate device memory at that point: a framework that hands the engine a fixed
// device-memory budget through its own caching allocator and forbids other allocations,
// or a host loop that evaluates the splits of every tree level and must not pay the
// implicit device-wide synchronisation that cudaMalloc / cudaFree may trigger. For them
// this entry point keeps the descriptors in a file-scope device array of fixed size
// instead, so a call only copies and launches.
//
// The array holds at most LMFAO_NOALLOC_MAX_QUERIES descriptors (6 x int64 each, 192 KiB);
// every GPU that loads this library keeps one copy of it until the process exits. All
// calls on a device share that copy: two calls whose work overlaps on the GPU (different
// streams, or contexts used from several threads) race on it. Each call overwrites the
// descriptors it uses before its kernel reads them, and the kernel reads nothing else
// from the array, so no clearing is needed between calls.
//
// On the host side the descriptors are built in one process-wide staging array and copied
// with cudaMemcpyAsync from it; a mutex is held from the first descriptor written until that
// copy has returned (a copy from pageable memory has left the source buffer when it returns),
// so calls from several host threads, on the same device or on different ones, do not mix
// their descriptors.
#include <mutex>
#include <unordered_map>

#include "ctx.h"

namespace {

constexpr int kDescWords = lmfao::kCartDescWords;

// Descriptor scratch: [query][icnt base, fsum base, buckets, aggregates, SUM(y) index, SUM(y^2) index].
static __device__ __align__(256) long long g_cart_desc[LMFAO_NOALLOC_MAX_QUERIES * kDescWords];

// Host staging copy of the descriptors (the source of the host-to-device copy); guarded by g_mu.
int64_t g_host_desc[LMFAO_NOALLOC_MAX_QUERIES * kDescWords];

std::mutex g_mu;                          // guards g_host_desc and g_addr
std::unordered_map<int, void *> g_addr;  // device -> device address of g_cart_desc

// Device address of the scratch array on `device`, which must be the current device; the
// caller holds g_mu. The name g_cart_desc in host code is only a host-side stand-in for the
// symbol; kernels must receive the address obtained here.
void *scratch_address_locked(int device) {
  auto it = g_addr.find(device);
  if (it != g_addr.end()) return it->second;
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_cart_desc);
  if (e != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    throw lmfao::Error(LMFAO_ERR_CUDA, std::string("cudaGetSymbolAddress of the descriptor array failed: ") +
                                           cudaGetErrorString(e));
  }
  g_addr[device] = p;
  return p;
}

}  // namespace

extern "C" int lmfao_cart_variances_noalloc(lmfao_ctx *ctx, const int *qids, int n, double *out, void *stream) {
  if (!ctx) return LMFAO_ERR_ARG;
  try {
    ctx->last_error.clear();
    if (ctx->device < 0) throw lmfao::Error(LMFAO_ERR_NOT_PLANNED, "host-only context");
    if (n < 0 || (n && (!qids || !out))) throw lmfao::Error(LMFAO_ERR_ARG, "bad arguments");
    if (n > LMFAO_NOALLOC_MAX_QUERIES)
      throw lmfao::Error(LMFAO_ERR_ARG, "lmfao_cart_variances_noalloc takes at most " +
                                            std::to_string(LMFAO_NOALLOC_MAX_QUERIES) + " queries per call (got " +
                                            std::to_string(n) + ")");
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
      cudaGetLastError();
      throw lmfao::Error(LMFAO_ERR_CUDA, "cudaSetDevice failed");
    }
    // the same checks as lmfao_cart_variances, without writing descriptors yet
    lmfao::PhysPlan *PP = nullptr;
    const int nb = lmfao::cart_descriptors(ctx, qids, n, nullptr, &PP);
    if (!n || nb < 2) return LMFAO_OK;
    lmfao::PhysPlan &P = *PP;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(g_mu);
    // First call on this device: look up the array's device address (the device is current).
    void *desc = scratch_address_locked(ctx->device);
    lmfao::cart_descriptors(ctx, qids, n, g_host_desc, nullptr);
    cudaError_t e = cudaMemcpyAsync(desc, g_host_desc, (size_t)n * kDescWords * sizeof(int64_t),
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw lmfao::Error(LMFAO_ERR_CUDA, std::string("descriptor copy failed: ") + cudaGetErrorString(e));
    }
    lmfao::launch_cart_variances(P.icnt, P.fsum, (const int64_t *)desc, n, nb, out, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) throw lmfao::Error(LMFAO_ERR_CUDA, std::string("launch failed: ") + cudaGetErrorString(e));
    return LMFAO_OK;
  } catch (const lmfao::Error &err) {
    ctx->last_error = err.what();
    return err.code;
  } catch (const std::exception &err) {
    ctx->last_error = err.what();
    return LMFAO_ERR_ARG;
  }
}
