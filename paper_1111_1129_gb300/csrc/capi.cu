// Error reporting, device memory, handle release and version of the C ABI.
#include <cstdint>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <string>

#include "lbm_internal.cuh"

namespace lbm {

namespace {
thread_local std::string g_last_error;
// The caller's allocator (both null: the library's own) and the number of
// blocks handed out and not yet released.
lbm_alloc_fn g_alloc = nullptr;
lbm_free_fn g_release = nullptr;
void* g_alloc_ctx = nullptr;
std::atomic<int64_t> g_live{0};
}

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t stream, bool ordered) {
  *p = nullptr;
  if (g_alloc) {
    void* q = g_alloc(bytes, (void*)stream, g_alloc_ctx);
    if (!q) return cudaErrorMemoryAllocation;
    if (reinterpret_cast<uintptr_t>(q) % 16 != 0) {   // the kernels use vector accesses
      if (g_release) g_release(q, (void*)stream, g_alloc_ctx);
      return cudaErrorMemoryAllocation;
    }
    *p = q;
  } else {
    const cudaError_t e = ordered ? cudaMallocAsync(p, bytes, stream) : cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
      *p = nullptr;
      return e;
    }
  }
  ++g_live;
  return cudaSuccess;
}

void dev_free(void* p, cudaStream_t stream, bool ordered) {
  if (!p) return;
  --g_live;
  if (g_release) g_release(p, (void*)stream, g_alloc_ctx);
  else if (ordered) cudaFreeAsync(p, stream);
  else cudaFree(p);
}

int fail(int status, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return status;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s (%s)", what,
              cudaGetErrorString(e), cudaGetErrorName(e));
}

void clear_error() { g_last_error.clear(); }

void free_sparse(lbm_sparse* sp) {
  if (!sp) return;
  const cudaStream_t s = sp->stream;
  for (void* p : {(void*)sp->cells, (void*)sp->inv, (void*)sp->adj, (void*)sp->adj_ld})
    dev_free(p, s, true);
  cudaStreamSynchronize(s);
  sp->magic = 0;
  delete sp;
}

}  // namespace lbm

extern "C" void lbm_free(void* handle) {
  if (!handle) return;
  const uint32_t magic = *static_cast<const uint32_t*>(handle);
  if (magic == lbm::kMagicSparse) lbm::free_sparse(static_cast<lbm_sparse*>(handle));
  else if (magic == lbm::kMagicState) lbm::free_state(static_cast<lbm_state*>(handle));
  else if (magic == lbm::kMagicAdjoint) lbm::free_adjoint(static_cast<lbm_adjoint*>(handle));
}

extern "C" const char* lbm_last_error(void) { return lbm::g_last_error.c_str(); }

extern "C" int lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn release, void* ctx) {
  lbm::clear_error();
  if ((alloc == nullptr) != (release == nullptr))
    return lbm::fail(LBM_EINVAL, "give both allocator functions or neither");
  const int64_t live = lbm::g_live.load();
  if (live != 0)
    return lbm::fail(LBM_EINVAL, "%lld device blocks of existing handles are still live",
                     (long long)live);
  lbm::g_alloc = alloc;
  lbm::g_release = release;
  lbm::g_alloc_ctx = ctx;
  return LBM_OK;
}

extern "C" int32_t lbm_abi_version(void) { return 2; }
