// The D3Q19 TRT stream-collide sweep over the sparse representation
// (Sec. 1: TRT on D3Q19; Sec. 2: sparse representation with implicit bounce
// back; Sec. 7: pull scheme, structure of arrays, nontemporal stores).
//
// One thread updates one fluid cell per step (two adjacent cells in the
// plain steps of the 16-bit forms, sweep_pair_kernel):
//   gather   g_0 = f[n], g_i = f[adj[i-1][n]]     (pull through the list)
//   collide  TRT with body force and Brinkman damping, written on the nine
//            (c, -c) pairs: with s = g_a + g_b, d = g_a - g_b,
//              f*_a = P + Q,  f*_b = P - Q,
//              P = (1 - w+)/2 s + w+ e+,   Q = (1 - w-)/2 d + c.V,
//              w+ e+ = w+ w (rho - 1.5 u.u) + 4.5 w+ w (c.u)^2,
//              V = 3 w (w- u + (1 - w-/2) F_n),
//            which is the same update as f* = g - w+(g+ - e+) - w-(g- - e-)
//            + (1 - w-/2) 3 w c.F_n, with fewer operations;
//   store    f'[q][n] with streaming (evict-first) stores, the GPU analogue
//            of the paper's nontemporal stores.
// The last step of a call also reduces rho and u to per-warp FP64 sums.
// The steps of a call after its first are chained (programmatic dependent
// launch, except in FP64 arithmetic), and long calls replay CUDA graphs.
//
// Storage forms: FP64 / FP32 PDFs, or the deviation d_q = f_q - w_q from
// the rest state in FP32, FP16 or BF16 (16-bit forms scaled by 2^k).  The
// collision on deviations is the same formula with rho replaced by
// rho - 1, because w_q is the equilibrium of rho = 1, u = 0.
//
// A state's PDF rows, and the link rows its steps read, have the stride
// sp->ld (N rounded up to 64), so that every row starts on a 128-byte
// boundary; the links name slots r ld + m.  Host-facing copies (set/get
// PDFs, moments) use the plain [19][N] layout.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <mutex>
#include <thread>

#include "lbm_kernels.cuh"

namespace lbm {

namespace {

// Stored value of every slot of row q at rest, in the storage form: w_q, or
// the deviation 0 for the shifted forms.
template <int PREC>
struct RestRow {
  typename Form<PREC>::S v[19];
};

// One row q = blockIdx.y per grid row, so no slot index is divided by N.
// From rest the stored value comes from `rest`; from f the value is
// converted as the form stores it (the deviation f - w in FP64, then
// rounded).  f is [19][n]; dst has rows of stride ld.
template <int PREC>
__global__ void set_pdfs_kernel(typename Form<PREC>::S* __restrict__ dst,
                                const double* __restrict__ f, int32_t n, int32_t ld, double scale,
                                RestRow<PREC> rest) {
  const int q = (int)blockIdx.y;
  using C = typename Form<PREC>::C;
  const double w = weight(q);
  const typename Form<PREC>::S r = rest.v[q];
  // a grid-stride loop: one-element threads made this kernel bound by
  // block scheduling (2.9 ms for 1.25 GB)
  for (int32_t i = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x); i < n;
       i += (int32_t)(gridDim.x * blockDim.x)) {
    const int64_t t = (int64_t)q * ld + i;
    if (!f) {
      dst[t] = r;
    } else {
      const double fv = f[(int64_t)q * n + i];
      C c;
      if constexpr (Form<PREC>::kShifted) c = (C)(fv - w);
      else c = (C)fv;
      dst[t] = encode<PREC>(c, (C)scale);
    }
  }
}

// The inverse of set_pdfs_kernel from f: src rows of stride ld, f [19][n].
template <int PREC>
__global__ void get_pdfs_kernel(const typename Form<PREC>::S* __restrict__ src, double* f,
                                int32_t n, int32_t ld, double inv_scale) {
  const int q = (int)blockIdx.y;
  using C = typename Form<PREC>::C;
  const double w = weight(q);
  for (int32_t i = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x); i < n;
       i += (int32_t)(gridDim.x * blockDim.x)) {
    const double v = (double)decode<PREC>(src[(int64_t)q * ld + i], (C)inv_scale);
    f[(int64_t)q * n + i] = Form<PREC>::kShifted ? w + v : v;
  }
}

// Grid of the row kernels above: x blocks of 256 threads per row, 19 rows.
dim3 row_grid(int64_t n) { return dim3((unsigned)std::min<int64_t>((n + 255) / 256, 2048), 19); }

template <class C>
__global__ void set_alpha_kernel(C* dst, const double* a, int32_t n) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (C)a[i];
}

}  // namespace

size_t storage_bytes(int prec) {
  switch (prec) {
    case LBM_F64: case LBM_F64X: return 8;
    case LBM_F32: case LBM_F32S: return 4;
    default: return 2;
  }
}
size_t compute_bytes(int prec) { return (prec == LBM_F64 || prec == LBM_F64X) ? 8 : 4; }
bool is_shifted(int prec) { return prec == LBM_F32S || prec == LBM_F16S || prec == LBM_BF16S; }

static double g_timeout_s = 600.0;

int wait_event(cudaEvent_t ev, cudaStream_t stream, double timeout_s) {
  LBM_CUDA_TRY(cudaEventRecord(ev, stream));
  const double limit = timeout_s > 0 ? timeout_s : g_timeout_s;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return LBM_OK;
    if (e != cudaErrorNotReady) return cuda_fail(e, "cudaEventQuery");
    const double el =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el > limit)
      return fail(LBM_ETIMEOUT, "queued work still running after %.1f s", limit);
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

bool valid_state(const lbm_state* st) { return st && st->magic == kMagicState; }

namespace {

template <int PREC>
int launch_steps(lbm_state* st, int32_t n_steps, double wp, double wm, const double F[3],
                 cudaStream_t stream, bool reduce_last) {
  using S = typename Form<PREC>::S;
  using C = typename Form<PREC>::C;
  const int32_t n = (int32_t)st->sp->n;
  const int32_t ld = (int32_t)st->sp->ld;
  if constexpr (PREC == LBM_F64X) return launch_steps_fx(st, n_steps, wp, wm, F, stream, reduce_last);
  const Coef<C> k = make_coef<C>(wp, wm, F, st->scale_exp);
  const unsigned grid = (unsigned)st->nblocks;
  const C* alpha = (const C*)st->alpha;
  // the 16-bit forms take two adjacent cells per thread in their plain steps
  // on grids of more than one wave
  constexpr bool kPairForm = LBM_PAIR_SWEEP && (PREC == LBM_F16S || PREC == LBM_BF16S);
  constexpr int64_t kPairCells = 2 * (int64_t)kPairThreads;
  const unsigned grid_pair = (unsigned)((n + kPairCells - 1) / kPairCells);
  for (int32_t t = 0; t < n_steps; ++t) {
    const S* src = (const S*)st->buf[st->cur];
    S* dst = (S*)st->buf[st->cur ^ 1];
    const bool last = reduce_last && t == n_steps - 1;
    if (n > 0) {
      const int32_t* adj = state_links(st->sp);
      // Steps in FP64 arithmetic are not chained: a chained grid's blocks are
      // placed while the previous grid still holds its SMs, which packs
      // them onto fewer SMs, and these steps are bound by each SM's FP64
      // rate (32x32x64 bed: 2,333 against 2,580 MFLUP/s unchained).
      constexpr bool kMemoryBound = PREC != LBM_F64 && PREC != LBM_F64X;
      const bool chained = kMemoryBound && t > 0;
      // a grid of one wave loads its links before the wait (sweep_kernel)
      const bool links_first = kMemoryBound && st->one_wave && !last;
      if constexpr (kPairForm) {
        if (!last && !st->one_wave) {
          if (alpha) LBM_CUDA_TRY(launch_chained(sweep_pair_kernel<PREC, true>, grid_pair, (unsigned)kPairThreads, stream, chained, src, dst, adj, n, ld, k, alpha));
          else LBM_CUDA_TRY(launch_chained(sweep_pair_kernel<PREC, false>, grid_pair, (unsigned)kPairThreads, stream, chained, src, dst, adj, n, ld, k, alpha));
          st->cur ^= 1;
          continue;
        }
      }
      if (alpha) {
        if (last) LBM_CUDA_TRY(launch_sweep(sweep_kernel<PREC, true, kWarpSums>, grid, stream, chained, src, dst, adj, n, ld, k, alpha, st->partials));
        else if (links_first) LBM_CUDA_TRY(launch_sweep(sweep_kernel<PREC, true, kNoReduce, kMemoryBound>, grid, stream, chained, src, dst, adj, n, ld, k, alpha, st->partials));
        else LBM_CUDA_TRY(launch_sweep(sweep_kernel<PREC, true, kNoReduce>, grid, stream, chained, src, dst, adj, n, ld, k, alpha, st->partials));
      } else {
        if (last) LBM_CUDA_TRY(launch_sweep(sweep_kernel<PREC, false, kWarpSums>, grid, stream, chained, src, dst, adj, n, ld, k, alpha, st->partials));
        else if (links_first) LBM_CUDA_TRY(launch_sweep(sweep_kernel<PREC, false, kNoReduce, kMemoryBound>, grid, stream, chained, src, dst, adj, n, ld, k, alpha, st->partials));
        else LBM_CUDA_TRY(launch_sweep(sweep_kernel<PREC, false, kNoReduce>, grid, stream, chained, src, dst, adj, n, ld, k, alpha, st->partials));
      }
    }
    st->cur ^= 1;
  }
  return LBM_OK;
}

template <int PREC>
int launch_moments(const lbm_state* st, double* rho, double* u) {
  using S = typename Form<PREC>::S;
  using C = typename Form<PREC>::C;
  const int32_t n = (int32_t)st->sp->n;
  if (n == 0) return LBM_OK;
  const Coef<C> k = make_coef<C>(st->last_wp, st->last_wm, st->last_force, st->scale_exp);
  const S* prev = (const S*)st->buf[st->cur ^ 1];
  const C* alpha = (const C*)st->alpha;
  if (alpha)
    moments_kernel<PREC, true><<<(unsigned)st->nblocks, kSweepThreads, 0, st->sp->stream>>>(prev, state_links(st->sp), n, (int32_t)st->sp->ld, k, alpha, rho, u);
  else
    moments_kernel<PREC, false><<<(unsigned)st->nblocks, kSweepThreads, 0, st->sp->stream>>>(prev, state_links(st->sp), n, (int32_t)st->sp->ld, k, alpha, rho, u);
  LBM_CUDA_TRY(cudaGetLastError());
  return LBM_OK;
}

// A batched state in several L2 groups keeps its arrays in the group layout:
// set and get go through the plain layout in the other PDF grid, which
// holds nothing between the steps of a batched state.
template <int PREC>
int launch_set(lbm_state* st, const double* f, int from_rest) {
  const int64_t total = 19 * st->sp->n;
  if (total == 0) return LBM_OK;
  const bool grouped = batch_grouped(st);
  using S = typename Form<PREC>::S;
  using C = typename Form<PREC>::C;
  RestRow<PREC> rest;
  for (int q = 0; q < 19; ++q) {
    const double w = weight(q);
    if constexpr (Form<PREC>::kShifted) {
      rest.v[q] = S{};   // a zero deviation: all-zero bits in every shifted form
    } else {
      rest.v[q] = (S)(C)w;
    }
  }
  const int32_t n = (int32_t)st->sp->n;
  set_pdfs_kernel<PREC><<<row_grid(n), 256, 0, st->sp->stream>>>(
      (S*)st->buf[grouped ? st->cur ^ 1 : st->cur], from_rest ? nullptr : f, n,
      (int32_t)st->sp->ld, std::ldexp(1.0, st->scale_exp), rest);
  LBM_CUDA_TRY(cudaGetLastError());
  if (grouped) return batch_relayout_pdfs(st, st->cur ^ 1, st->cur, false);
  return LBM_OK;
}

template <int PREC>
int launch_get(const lbm_state* st, double* f) {
  const int64_t total = 19 * st->sp->n;
  if (total == 0) return LBM_OK;
  const bool grouped = batch_grouped(st);
  if (grouped) {
    const int rc = batch_relayout_pdfs(st, st->cur, st->cur ^ 1, true);
    if (rc != LBM_OK) return rc;
  }
  get_pdfs_kernel<PREC><<<row_grid(st->sp->n), 256, 0, st->sp->stream>>>(
      (const typename Form<PREC>::S*)st->buf[grouped ? st->cur ^ 1 : st->cur], f,
      (int32_t)st->sp->n, (int32_t)st->sp->ld, std::ldexp(1.0, -st->scale_exp));
  LBM_CUDA_TRY(cudaGetLastError());
  return LBM_OK;
}

#define LBM_DISPATCH(prec, fn, ...)                          \
  switch (prec) {                                            \
    case LBM_F64: return fn<LBM_F64>(__VA_ARGS__);           \
    case LBM_F64X: return fn<LBM_F64X>(__VA_ARGS__);         \
    case LBM_F32: return fn<LBM_F32>(__VA_ARGS__);           \
    case LBM_F32S: return fn<LBM_F32S>(__VA_ARGS__);         \
    case LBM_F16S: return fn<LBM_F16S>(__VA_ARGS__);         \
    default: return fn<LBM_BF16S>(__VA_ARGS__);              \
  }

int dispatch_set(lbm_state* st, const double* f, int from_rest) {
  LBM_DISPATCH(st->precision, launch_set, st, f, from_rest)
}
int dispatch_get(const lbm_state* st, double* f) { LBM_DISPATCH(st->precision, launch_get, st, f) }
int dispatch_steps(lbm_state* st, int32_t n_steps, double wp, double wm, const double F[3],
                   cudaStream_t stream, bool reduce_last) {
  LBM_DISPATCH(st->precision, launch_steps, st, n_steps, wp, wm, F, stream, reduce_last)
}

void free_graph(lbm_state* st) {
  StepGraph* g = st->graph;
  if (!g) return;
  for (int p = 0; p < 2; ++p)
    if (g->exec[p]) cudaGraphExecDestroy(g->exec[p]);
  if (g->capture) cudaStreamDestroy(g->capture);
  delete g;
  st->graph = nullptr;
}

// The graph of kGraphSteps non-reducing steps from the current parity with
// these arguments, captured on first use (or when the arguments changed).
int step_graph(lbm_state* st, double wp, double wm, const double F[3], cudaGraphExec_t* out) {
  if (!st->graph) {
    st->graph = new StepGraph{};
    const cudaError_t e = cudaStreamCreateWithFlags(&st->graph->capture, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      free_graph(st);
      return cuda_fail(e, "cudaStreamCreateWithFlags");
    }
  }
  StepGraph* g = st->graph;
  const int p = st->cur;
  if (g->exec[p] && g->wp[p] == wp && g->wm[p] == wm && g->F[p][0] == F[0] &&
      g->F[p][1] == F[1] && g->F[p][2] == F[2] && g->alpha[p] == st->alpha) {
    *out = g->exec[p];
    return LBM_OK;
  }
  if (g->exec[p]) {
    cudaGraphExecDestroy(g->exec[p]);
    g->exec[p] = nullptr;
  }
  LBM_CUDA_TRY(cudaStreamBeginCapture(g->capture, cudaStreamCaptureModeThreadLocal));
  const int rc = dispatch_steps(st, kGraphSteps, wp, wm, F, g->capture, false);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(g->capture, &graph);
  st->cur = p;   // the capture only recorded the launches
  if (rc != LBM_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  const cudaError_t e2 = cudaGraphInstantiate(&g->exec[p], graph, 0);
  cudaGraphDestroy(graph);
  if (e2 != cudaSuccess) {
    g->exec[p] = nullptr;
    return cuda_fail(e2, "cudaGraphInstantiate");
  }
  g->wp[p] = wp;
  g->wm[p] = wm;
  for (int d = 0; d < 3; ++d) g->F[p][d] = F[d];
  g->alpha[p] = st->alpha;
  *out = g->exec[p];
  return LBM_OK;
}

// n_steps steps on the state's stream.  Launching a kernel costs the host a
// few microseconds, as much as a whole step of a bed of ~10^5 cells, so a
// call long enough to replay the cached graph of kGraphSteps steps at least
// twice runs its bulk that way; the remaining steps, the reducing last one
// included, are launched one by one.  The kernels and their order are the
// same either way, so the results are bit-identical.
int run_steps(lbm_state* st, int32_t n_steps, double wp, double wm, const double F[3]) {
  const cudaStream_t stream = st->sp->stream;
  int32_t replays = st->sp->n > 0 ? (n_steps - 1) / kGraphSteps : 0;
  if (replays >= 2) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    LBM_CUDA_TRY(cudaStreamIsCapturing(stream, &cs));
    if (cs != cudaStreamCaptureStatusNone) replays = 0;   // the caller is capturing
  } else {
    replays = 0;
  }
  if (replays > 0) {
    cudaGraphExec_t exec = nullptr;
    const int rc = step_graph(st, wp, wm, F, &exec);
    if (rc != LBM_OK) return rc;
    for (int32_t r = 0; r < replays; ++r) LBM_CUDA_TRY(cudaGraphLaunch(exec, stream));
  }
  return dispatch_steps(st, n_steps - replays * kGraphSteps, wp, wm, F, stream, true);
}
int dispatch_moments(const lbm_state* st, double* rho, double* u) {
  LBM_DISPATCH(st->precision, launch_moments, st, rho, u)
}

}  // namespace

void free_state(lbm_state* st) {
  if (!st) return;
  // the sparse handle may already be released (a garbage collector may free
  // the two in either order): only the stream kept here is used
  const cudaStream_t s = st->stream;
  cudaStreamSynchronize(s);
  for (void* p : {st->buf[0], st->buf[1], st->alpha, (void*)st->alpha_fx, (void*)st->partials,
                  (void*)st->red_dev})
    dev_free(p, s, false);
  if (st->red_host) cudaFreeHost(st->red_host);
  if (st->done) cudaEventDestroy(st->done);
  if (st->t0) cudaEventDestroy(st->t0);
  if (st->t1) cudaEventDestroy(st->t1);
  free_graph(st);
  if (st->batch) free_batch(st);
  st->magic = 0;
  delete st;
}

}  // namespace lbm

using namespace lbm;

extern "C" int lbm_state_create(const lbm_sparse* sp, int32_t precision, int32_t scale_exp,
                                lbm_state** out) {
  clear_error();
  if (!out) return fail(LBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!sp || sp->magic != kMagicSparse) return fail(LBM_EINVAL, "not a sparse handle");
  if (sp->ld < sp->n || (sp->ld != sp->n && !sp->adj_ld))
    return fail(LBM_EINVAL, "sparse handle without a valid row layout");
  if (precision < LBM_F64 || precision > LBM_F64X)
    return fail(LBM_EINVAL, "unknown precision %d", precision);
  if ((precision == LBM_F16S || precision == LBM_BF16S) && (scale_exp < 0 || scale_exp > 40))
    return fail(LBM_EINVAL, "scale_exp %d outside [0, 40]", scale_exp);
  lbm_state* st = new lbm_state{};
  st->magic = kMagicState;
  st->sp = sp;
  st->stream = sp->stream;
  st->precision = precision;
  st->scale_exp = (precision == LBM_F16S || precision == LBM_BF16S) ? scale_exp : 0;
  const int64_t n = sp->n;
  st->nblocks = (n + kSweepThreads - 1) / kSweepThreads;
  if (st->nblocks < 1) st->nblocks = 1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    sms = 0;
  }
  // one wave at the 4 resident blocks per SM of the FP32 and 16-bit sweeps
  st->one_wave = st->nblocks <= 4 * (int64_t)sms;
  // rows of sp->ld elements; the padding slots past n are never read
  const size_t bytes = storage_bytes(precision) * 19 * (size_t)(sp->ld > 0 ? sp->ld : 1);
  const cudaStream_t stream = sp->stream;
  bool ok = dev_alloc(&st->buf[0], bytes, stream, false) == cudaSuccess &&
            dev_alloc(&st->buf[1], bytes, stream, false) == cudaSuccess &&
            dev_alloc(&st->partials, sizeof(double) * 4 * (kWarpsPerBlock + 1) * st->nblocks,
                      stream, false) == cudaSuccess &&
            dev_alloc(&st->red_dev, sizeof(double) * 4, stream, false) == cudaSuccess &&
            cudaMallocHost(&st->red_host, sizeof(double) * 4) == cudaSuccess &&
            cudaEventCreateWithFlags(&st->done, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_state(st);
    return fail(LBM_ENOMEM, "state allocation of 2 x %zu bytes failed", bytes);
  }
  int rc = dispatch_set(st, nullptr, 1);
  // The first step writes every slot of the second grid before anything
  // reads it.  A concatenated batch (ord.kind -1) also has padding cells
  // that no step writes: zero its second grid so that they read back as 0.
  if (rc == LBM_OK && sp->ord.kind == -1) {
    const cudaError_t e = cudaMemsetAsync(st->buf[1], 0, bytes, sp->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemsetAsync");
  }
  if (rc != LBM_OK) {
    free_state(st);
    return rc;
  }
  *out = st;
  return LBM_OK;
}

extern "C" int lbm_state_set_pdfs(lbm_state* st, const double* f_dev) {
  clear_error();
  if (!valid_state(st)) return fail(LBM_EINVAL, "not a state handle");
  if (!f_dev && st->sp->n > 0) return fail(LBM_EINVAL, "f_dev is NULL");
  st->steps = 0;
  return dispatch_set(st, f_dev, 0);
}

// Raw copies between the state's padded rows (stride sp->ld) and [19][N].
static int copy_raw(const lbm_state* st, void* dst, size_t dpitch, const void* src,
                    size_t spitch) {
  const size_t row = (size_t)st->sp->n * storage_bytes(st->precision);
  LBM_CUDA_TRY(cudaMemcpy2DAsync(dst, dpitch, src, spitch, row, 19, cudaMemcpyDefault,
                                 st->sp->stream));
  return LBM_OK;
}

extern "C" int lbm_state_get_raw(const lbm_state* st, void* raw) {
  clear_error();
  if (!valid_state(st)) return fail(LBM_EINVAL, "not a state handle");
  if (st->batch) return fail(LBM_EINVAL, "raw copies are not available on a batched state");
  if (st->sp->n == 0) return LBM_OK;
  if (!raw) return fail(LBM_EINVAL, "raw is NULL");
  const size_t e = storage_bytes(st->precision);
  return copy_raw(st, raw, (size_t)st->sp->n * e, st->buf[st->cur], (size_t)st->sp->ld * e);
}

extern "C" int lbm_state_set_raw(lbm_state* st, const void* raw) {
  clear_error();
  if (!valid_state(st)) return fail(LBM_EINVAL, "not a state handle");
  if (st->batch) return fail(LBM_EINVAL, "raw copies are not available on a batched state");
  st->steps = 0;
  if (st->sp->n == 0) return LBM_OK;
  if (!raw) return fail(LBM_EINVAL, "raw is NULL");
  const size_t e = storage_bytes(st->precision);
  return copy_raw(st, st->buf[st->cur], (size_t)st->sp->ld * e, raw, (size_t)st->sp->n * e);
}

extern "C" int lbm_state_reset(lbm_state* st) {
  clear_error();
  if (!valid_state(st)) return fail(LBM_EINVAL, "not a state handle");
  st->steps = 0;
  return dispatch_set(st, nullptr, 1);
}

extern "C" int lbm_state_get_pdfs(const lbm_state* st, double* f_dev) {
  clear_error();
  if (!valid_state(st)) return fail(LBM_EINVAL, "not a state handle");
  if (!f_dev && st->sp->n > 0) return fail(LBM_EINVAL, "f_dev is NULL");
  return dispatch_get(st, f_dev);
}

extern "C" int lbm_set_damping(lbm_state* st, const double* alpha_dev) {
  clear_error();
  if (!valid_state(st)) return fail(LBM_EINVAL, "not a state handle");
  if (st->batch) return fail(LBM_EINVAL, "damping is not supported on a batched state");
  if (!alpha_dev) {
    if (st->alpha) {
      cudaStreamSynchronize(st->sp->stream);
      dev_free(st->alpha, st->sp->stream, false);
      dev_free(st->alpha_fx, st->sp->stream, false);
    }
    st->alpha = nullptr;
    st->alpha_fx = nullptr;
    return LBM_OK;
  }
  const int64_t n = st->sp->n;
  if (!st->alpha) {
    const size_t nn = (size_t)(n > 0 ? n : 1);
    void* afx = nullptr;
    if (dev_alloc(&st->alpha, compute_bytes(st->precision) * nn, st->sp->stream, false) !=
            cudaSuccess ||
        (st->precision == LBM_F64X &&
         dev_alloc(&afx, 2 * sizeof(int64_t) * nn, st->sp->stream, false) != cudaSuccess)) {
      cudaGetLastError();
      dev_free(st->alpha, st->sp->stream, false);
      st->alpha = nullptr;
      return fail(LBM_ENOMEM, "damping field allocation failed");
    }
    st->alpha_fx = (int64_t*)afx;
  }
  if (n > 0) {
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (compute_bytes(st->precision) == 8)   // the FP64 forms, FP64 storage in fixed point included
      set_alpha_kernel<double><<<grid, 256, 0, st->sp->stream>>>((double*)st->alpha, alpha_dev, (int32_t)n);
    else
      set_alpha_kernel<float><<<grid, 256, 0, st->sp->stream>>>((float*)st->alpha, alpha_dev, (int32_t)n);
    LBM_CUDA_TRY(cudaGetLastError());
    if (st->alpha_fx) {
      const int rc = set_alpha_fx(st, alpha_dev);
      if (rc != LBM_OK) return rc;
    }
  }
  return LBM_OK;
}

extern "C" int lbm_step(lbm_state* st, int32_t n_steps, double omega_plus, double omega_minus,
                        const double force[3]) {
  clear_error();
  if (!valid_state(st)) return fail(LBM_EINVAL, "not a state handle");
  if (n_steps < 0) return fail(LBM_EINVAL, "n_steps = %d < 0", n_steps);
  if (!(omega_plus > 0.0 && omega_plus < 2.0) || !(omega_minus > 0.0 && omega_minus < 2.0))
    return fail(LBM_EINVAL, "relaxation rates must lie in (0, 2): %g, %g", omega_plus, omega_minus);
  if (!force) return fail(LBM_EINVAL, "force is NULL");
  const int n_force = st->batch ? 3 * st->batch->n_beds : 3;
  for (int d = 0; d < n_force; ++d)
    if (!std::isfinite(force[d])) return fail(LBM_EINVAL, "force[%d] is not finite", d);
  if (n_steps == 0) return LBM_OK;
  const int rc = st->batch ? batch_steps(st, n_steps, omega_plus, omega_minus, force)
                           : run_steps(st, n_steps, omega_plus, omega_minus, force);
  if (rc != LBM_OK) return rc;
  st->steps += n_steps;
  st->last_wp = omega_plus;
  st->last_wm = omega_minus;
  for (int d = 0; d < 3; ++d) st->last_force[d] = force[d];
  return LBM_OK;
}

extern "C" int lbm_step_timed(lbm_state* st, int32_t n_steps, double omega_plus,
                              double omega_minus, const double force[3], double* ms_out) {
  clear_error();
  if (!valid_state(st)) return fail(LBM_EINVAL, "not a state handle");
  if (!ms_out) return fail(LBM_EINVAL, "ms_out is NULL");
  if (!st->t0) {
    if (cudaEventCreate(&st->t0) != cudaSuccess || cudaEventCreate(&st->t1) != cudaSuccess) {
      cudaGetLastError();
      if (st->t0) cudaEventDestroy(st->t0);
      st->t0 = st->t1 = nullptr;
      return fail(LBM_ECUDA, "cudaEventCreate failed");
    }
  }
  const cudaStream_t stream = st->sp->stream;
  LBM_CUDA_TRY(cudaEventRecord(st->t0, stream));
  int rc = lbm_step(st, n_steps, omega_plus, omega_minus, force);
  if (rc != LBM_OK) return rc;
  LBM_CUDA_TRY(cudaEventRecord(st->t1, stream));
  rc = wait_event(st->done, stream, 0.0);
  if (rc != LBM_OK) return rc;
  float ms = 0.f;
  LBM_CUDA_TRY(cudaEventElapsedTime(&ms, st->t0, st->t1));
  *ms_out = (double)ms;
  return LBM_OK;
}

extern "C" int lbm_reduce_flux(lbm_state* st, int32_t axis, double* mass_out, double* flux_out) {
  clear_error();
  if (!valid_state(st)) return fail(LBM_EINVAL, "not a state handle");
  if (axis < 0 || axis > 2) return fail(LBM_EINVAL, "axis %d outside {0,1,2}", axis);
  if (st->steps < 1) return fail(LBM_EINVAL, "no step taken yet");
  if (st->batch) return batch_reduce(st, axis, mass_out, flux_out);
  const cudaStream_t stream = st->sp->stream;
  const int64_t n = st->sp->n;
  if (n > 0) {
    // group sums after the warp slots (room for nblocks values of 4)
    double* groups = st->partials + 4 * kWarpsPerBlock * st->nblocks;
    const int64_t ngroups = (st->nblocks + kCollapseThreads - 1) / kCollapseThreads;
    collapse_warp_sums_kernel<<<(unsigned)ngroups, kCollapseThreads, 0, stream>>>(
        st->partials, st->nblocks, groups);
    final_sum_kernel<<<1, 1024, 0, stream>>>(groups, ngroups, st->red_dev);
    LBM_CUDA_TRY(cudaGetLastError());
    LBM_CUDA_TRY(cudaMemcpyAsync(st->red_host, st->red_dev, sizeof(double) * 4,
                                 cudaMemcpyDeviceToHost, stream));
    const int rc = wait_event(st->done, stream, 0.0);
    if (rc != LBM_OK) return rc;
  } else {
    for (int j = 0; j < 4; ++j) st->red_host[j] = 0.0;
  }
  const bool shifted = is_shifted(st->precision);
  const double mass = shifted ? (double)n + st->red_host[0] : st->red_host[0];
  const double flux = n > 0 ? st->red_host[1 + axis] / (double)n : 0.0;
  if (!std::isfinite(mass) || !std::isfinite(flux))
    return fail(LBM_ENONFINITE, "non-finite mass (%g) or flux (%g)", mass, flux);
  if (mass_out) *mass_out = mass;
  if (flux_out) *flux_out = flux;
  return LBM_OK;
}

extern "C" int lbm_moments(const lbm_state* st, double* rho_dev, double* u_dev) {
  clear_error();
  if (!valid_state(st)) return fail(LBM_EINVAL, "not a state handle");
  if ((!rho_dev || !u_dev) && st->sp->n > 0) return fail(LBM_EINVAL, "rho_dev / u_dev is NULL");
  if (st->steps < 1) return fail(LBM_EINVAL, "no step taken yet");
  if (st->batch) return fail(LBM_EINVAL, "lbm_moments is not available on a batched state");
  return dispatch_moments(st, rho_dev, u_dev);
}

extern "C" int lbm_state_steps(const lbm_state* st, int64_t* steps) {
  clear_error();
  if (!valid_state(st)) return fail(LBM_EINVAL, "not a state handle");
  if (steps) *steps = st->steps;
  return LBM_OK;
}

extern "C" int lbm_synchronize(const lbm_state* st, double timeout_s) {
  clear_error();
  if (!valid_state(st)) return fail(LBM_EINVAL, "not a state handle");
  return wait_event(st->done, st->sp->stream, timeout_s);
}

extern "C" void lbm_set_timeout(double timeout_s) {
  if (timeout_s > 0) g_timeout_s = timeout_s;
}

// ---------------------------------------------------------------------------
// Allocation-free FP64 step.  The paper has no counterpart.  Some callers
// cannot allocate device memory: a host application that owns all of the
// GPU's memory and hands this library only the arrays it works on, or a
// time-stepping loop with a fixed memory budget that cannot absorb the
// device-wide synchronisation and latency of a cudaMalloc.  This entry point
// takes every input and output from the caller and keeps its one piece of
// scratch -- the FP64 block partial sums of the reduction -- in a fixed
// static device array.  Under lazy module loading the driver reserves the
// array on a device when this file's device code is first used there (at
// the latest by the first call of this entry point on that device); the
// device then holds it until the process exits.
namespace lbm {
namespace {

constexpr int64_t kStaticMaxBlocks = 65536;
constexpr int64_t kStaticMaxCells = kStaticMaxBlocks * kSweepThreads;  // 16,777,216
static __device__ __align__(256) double g_static_partials[kStaticMaxBlocks * 4];  // 2 MiB

// Device address of g_static_partials on the current device, looked up once
// per device (in host code the symbol is only a host-side stand-in).
int static_partials(double** out) {
  constexpr int kMaxDevices = 64;
  static std::mutex mu;
  static double* addr[kMaxDevices] = {};
  int dev = 0;
  LBM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(LBM_EINVAL, "device ordinal %d unsupported", dev);
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    double* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_static_partials);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_static_partials)");
    addr[dev] = p;
  }
  *out = addr[dev];
  return LBM_OK;
}

}  // namespace
}  // namespace lbm

extern "C" int lbm_step_f64_noalloc(const double* f_src_dev, double* f_dst_dev,
                                    const int32_t* adj_dev, int64_t n_fluid, double omega_plus,
                                    double omega_minus, const double force[3],
                                    const double* alpha_dev, double* sums_dev, void* stream_v) {
  clear_error();
  if (n_fluid < 0 || n_fluid > kStaticMaxCells)
    return fail(LBM_EINVAL,
                "lbm_step_f64_noalloc handles at most %lld fluid cells (its static scratch "
                "holds %lld block sums); got %lld",
                (long long)kStaticMaxCells, (long long)kStaticMaxBlocks, (long long)n_fluid);
  if (!sums_dev) return fail(LBM_EINVAL, "sums_dev is NULL");
  if (n_fluid > 0 && (!f_src_dev || !f_dst_dev || !adj_dev))
    return fail(LBM_EINVAL, "f_src_dev, f_dst_dev and adj_dev must be non-NULL");
  if (n_fluid > 0 && f_src_dev == f_dst_dev)
    return fail(LBM_EINVAL, "f_src_dev and f_dst_dev must be different arrays");
  if (!(omega_plus > 0.0 && omega_plus < 2.0) || !(omega_minus > 0.0 && omega_minus < 2.0))
    return fail(LBM_EINVAL, "relaxation rates must lie in (0, 2): %g, %g", omega_plus, omega_minus);
  if (!force) return fail(LBM_EINVAL, "force is NULL");
  for (int d = 0; d < 3; ++d)
    if (!std::isfinite(force[d])) return fail(LBM_EINVAL, "force[%d] is not finite", d);
  double* partials = nullptr;
  int rc = static_partials(&partials);
  if (rc != LBM_OK) return rc;
  const cudaStream_t stream = (cudaStream_t)stream_v;
  if (n_fluid == 0) {
    LBM_CUDA_TRY(cudaMemsetAsync(sums_dev, 0, 4 * sizeof(double), stream));
    return LBM_OK;
  }
  const int32_t n = (int32_t)n_fluid;
  const int64_t nblocks = (n_fluid + kSweepThreads - 1) / kSweepThreads;
  const Coef<double> k = make_coef<double>(omega_plus, omega_minus, force, 0);
  if (alpha_dev)
    sweep_kernel<LBM_F64, true, kBlockSums><<<(unsigned)nblocks, kSweepThreads, 0, stream>>>(
        f_src_dev, f_dst_dev, adj_dev, n, n, k, alpha_dev, partials);
  else
    sweep_kernel<LBM_F64, false, kBlockSums><<<(unsigned)nblocks, kSweepThreads, 0, stream>>>(
        f_src_dev, f_dst_dev, adj_dev, n, n, k, nullptr, partials);
  final_sum_kernel<<<1, 1024, 0, stream>>>(partials, nblocks, sums_dev);
  LBM_CUDA_TRY(cudaGetLastError());
  return LBM_OK;
}
