// Error reporting, handle release and version of the C ABI.
#include <cstdarg>
#include <cstdio>
#include <string>

#include "lbm_internal.cuh"

namespace lbm {

namespace {
thread_local std::string g_last_error;
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
  for (void* p : {(void*)sp->cells, (void*)sp->inv, (void*)sp->adj})
    if (p) cudaFreeAsync(p, s);
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

extern "C" int32_t lbm_abi_version(void) { return 1; }
