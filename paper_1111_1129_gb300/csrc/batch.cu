// Batched sweep: many independent packed beds of uneven size in one launch
// per time step.
//
// The beds' sparse representations are concatenated into one list; each bed
// starts at a multiple of kBatchChunk (2048) cells, so any tile of
// block x cells-per-thread <= 2048 cells lies inside one bed and finds its
// bed from a per-chunk table -- no per-cell bed id is stored or read.  The
// adjacency is remapped to the concatenated slots (q*N + m of a bed becomes
// q*N_pad + begin + m); padding cells bounce every link onto themselves and
// are never read or written by the sweep.  Each bed has its own body force,
// taken from a small table.  The step that reduces runs with the 256-thread,
// one-cell-per-thread layout of the single-bed sweep and reduces each bed
// over its own 256-cell blocks in the same order, so a bed's PDFs and flux
// are bit-identical to running it alone.
//
// Launch shape: the non-reducing steps use (block, cells per thread) from
// {128, 256, 512} x {1, 2, 4}, picked by lbm_batch_tune; all shapes give the
// same per-cell arithmetic.  A sequence of K steps is captured once into a
// CUDA graph (on a private stream) and replayed on the caller's stream.
#include <cmath>
#include <vector>

#include "lbm_kernels.cuh"

namespace lbm {
namespace {

template <class C>
struct BedForce {
  C F[3], hF[3], bF1[3];
};

__global__ void self_bounce_kernel(int32_t* __restrict__ adj, int32_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 18 * (int64_t)n) return;
  const int q = (int)(t / n) + 1;
  const int32_t i = (int32_t)(t % n);
  adj[t] = opp(q) * n + i;
}

__global__ void concat_adj_kernel(const int32_t* __restrict__ adj_b, int32_t nb, int32_t off,
                                  int32_t ntot, int32_t* __restrict__ adj) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 18 * (int64_t)nb) return;
  const int32_t row = (int32_t)(t / nb), i = (int32_t)(t % nb);
  const int32_t s = adj_b[t];
  const int32_t q = s / nb, m = s - q * nb;
  adj[(int64_t)row * ntot + off + i] = q * ntot + off + m;
}

template <int PREC, bool REDUCE, int CPT>
__global__ void __launch_bounds__(512)
    batch_sweep_kernel(const typename Form<PREC>::S* __restrict__ src,
                       typename Form<PREC>::S* __restrict__ dst, const int32_t* __restrict__ adj,
                       int32_t n, Coef<typename Form<PREC>::C> k,
                       const BedForce<typename Form<PREC>::C>* __restrict__ forces,
                       const int32_t* __restrict__ chunk_bed, const int64_t* __restrict__ begin,
                       const int32_t* __restrict__ count, double* __restrict__ partials) {
  using C = typename Form<PREC>::C;
  const int64_t base = (int64_t)blockIdx.x * blockDim.x * CPT;
  const int bed = chunk_bed[base / kBatchChunk];
  const int64_t end = begin[bed] + count[bed];
  Coef<C> kb = k;
  const BedForce<C> bf = forces[bed];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    kb.F[d] = bf.F[d];
    kb.hF[d] = bf.hF[d];
    kb.bF1[d] = bf.bF1[d];
  }
  C rho = C(0), u[3] = {C(0), C(0), C(0)};
  bool live = false;
#pragma unroll
  for (int j = 0; j < CPT; ++j) {
    const int64_t i = base + (int64_t)j * blockDim.x + threadIdx.x;
    if (i < end) {
      C g[19];
      gather<PREC>(src, adj, n, (int32_t)i, kb.inv_scale, g);
      collide<C, false>(g, kb, C(0), rho, u);
      live = true;
#pragma unroll
      for (int q = 0; q < 19; ++q)
        store_stream<PREC>(dst + q * n + i, encode<PREC>(g[q], kb.scale));
    }
  }
  if constexpr (REDUCE) {   // runs with 256 threads and CPT = 1
    double w[4];
    warp_flux_sums<C, Form<PREC>::kShifted>(live, rho, u, w);
    store_warp_sums(w, partials);
  }
}

// Per-bed final sums over the warp sums of the bed's 256-cell blocks, in the
// same order as the single-bed final sum.
__global__ void __launch_bounds__(1024)
    batch_final_kernel(const double* __restrict__ part, const int64_t* __restrict__ begin,
                       const int32_t* __restrict__ count, double* __restrict__ out) {
  __shared__ double sm[1024][4];
  const int bed = blockIdx.x;
  const double* p = part + 4 * kWarpsPerBlock * (begin[bed] / kSweepThreads);
  const int64_t nblocks = ((int64_t)count[bed] + kSweepThreads - 1) / kSweepThreads;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t b = threadIdx.x; b < nblocks; b += 1024)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      double v = 0.0;
      for (int k = 0; k < kWarpsPerBlock; ++k) v += p[4 * (b * kWarpsPerBlock + k) + j];
      acc[j] += v;
    }
#pragma unroll
  for (int j = 0; j < 4; ++j) sm[threadIdx.x][j] = acc[j];
  __syncthreads();
  for (int s = 512; s > 0; s >>= 1) {
    if (threadIdx.x < s)
#pragma unroll
      for (int j = 0; j < 4; ++j) sm[threadIdx.x][j] += sm[threadIdx.x + s][j];
    __syncthreads();
  }
  if (threadIdx.x < 4) out[4 * bed + threadIdx.x] = sm[0][threadIdx.x];
}

template <int PREC, bool REDUCE>
void launch_one(lbm_state* st, int block, int cpt, cudaStream_t stream,
                const Coef<typename Form<PREC>::C>& k) {
  using S = typename Form<PREC>::S;
  using C = typename Form<PREC>::C;
  Batch* b = st->batch;
  const int32_t n = (int32_t)st->sp->n;
  const S* src = (const S*)st->buf[st->cur];
  S* dst = (S*)st->buf[st->cur ^ 1];
  const unsigned grid = (unsigned)(n / (block * cpt));
  const BedForce<C>* forces = (const BedForce<C>*)b->d_force;
#define LBM_BATCH_LAUNCH(CPT)                                                          \
  batch_sweep_kernel<PREC, REDUCE, CPT><<<grid, block, 0, stream>>>(                   \
      src, dst, st->sp->adj, n, k, forces, b->d_chunk_bed, b->d_begin, b->d_count,     \
      st->partials)
  if (cpt == 1) LBM_BATCH_LAUNCH(1);
  else if (cpt == 2) LBM_BATCH_LAUNCH(2);
  else LBM_BATCH_LAUNCH(4);
#undef LBM_BATCH_LAUNCH
  st->cur ^= 1;
}

// Enqueues n_steps steps on `stream` (the last one reduces).
template <int PREC>
void enqueue_steps(lbm_state* st, int32_t n_steps, double wp, double wm, int block, int cpt,
                   cudaStream_t stream) {
  using C = typename Form<PREC>::C;
  const double zero[3] = {0.0, 0.0, 0.0};
  const Coef<C> k = make_coef<C>(wp, wm, zero, st->scale_exp);
  for (int32_t t = 0; t < n_steps; ++t) {
    if (t == n_steps - 1) launch_one<PREC, true>(st, kSweepThreads, 1, stream, k);
    else launch_one<PREC, false>(st, block, cpt, stream, k);
  }
}

template <int PREC>
int fill_forces(lbm_state* st, double wm, const double* forces, cudaStream_t stream) {
  using C = typename Form<PREC>::C;
  Batch* b = st->batch;
  // the previous call's upload must have left the staging buffer
  LBM_CUDA_TRY(cudaStreamSynchronize(stream));
  BedForce<C>* h = (BedForce<C>*)b->h_force;
  const double b1 = 3.0 * (1.0 - 0.5 * wm) / 18.0;
  for (int i = 0; i < b->n_beds; ++i)
    for (int d = 0; d < 3; ++d) {
      const double F = forces[3 * i + d];
      h[i].F[d] = (C)F;
      h[i].hF[d] = (C)(0.5 * F);
      h[i].bF1[d] = (C)(b1 * F);
    }
  LBM_CUDA_TRY(cudaMemcpyAsync(b->d_force, b->h_force, sizeof(BedForce<C>) * b->n_beds,
                               cudaMemcpyHostToDevice, stream));
  return LBM_OK;
}

template <int PREC>
int run_batch(lbm_state* st, int32_t n_steps, double wp, double wm, const double* forces) {
  Batch* b = st->batch;
  const cudaStream_t stream = st->sp->stream;
  int rc = fill_forces<PREC>(st, wm, forces, stream);
  if (rc != LBM_OK) return rc;
  if (st->sp->n == 0) {
    st->cur ^= (n_steps & 1);
    return LBM_OK;
  }
  if (!b->use_graph) {
    enqueue_steps<PREC>(st, n_steps, wp, wm, b->block, b->cpt, stream);
    LBM_CUDA_TRY(cudaGetLastError());
    return LBM_OK;
  }
  const bool hit = b->graph && b->g_steps == n_steps && b->g_parity == st->cur &&
                   b->g_block == b->block && b->g_cpt == b->cpt && b->g_wp == wp &&
                   b->g_wm == wm;
  if (!hit) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    const int parity = st->cur;
    LBM_CUDA_TRY(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
    enqueue_steps<PREC>(st, n_steps, wp, wm, b->block, b->cpt, b->capture);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->capture, &g);
    st->cur = parity;  // capture only recorded the launches
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    const cudaError_t e2 = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) {
      b->graph = nullptr;
      return cuda_fail(e2, "cudaGraphInstantiate");
    }
    b->g_steps = n_steps;
    b->g_parity = parity;
    b->g_block = b->block;
    b->g_cpt = b->cpt;
    b->g_wp = wp;
    b->g_wm = wm;
  }
  LBM_CUDA_TRY(cudaGraphLaunch(b->graph, stream));
  st->cur ^= (n_steps & 1);
  return LBM_OK;
}

template <int PREC>
size_t force_bytes() {
  return sizeof(BedForce<typename Form<PREC>::C>);
}

#define LBM_BATCH_DISPATCH(prec, fn, ...)                    \
  switch (prec) {                                            \
    case LBM_F64: return fn<LBM_F64>(__VA_ARGS__);           \
    case LBM_F64X: return fn<LBM_F64X>(__VA_ARGS__);         \
    case LBM_F32: return fn<LBM_F32>(__VA_ARGS__);           \
    case LBM_F32S: return fn<LBM_F32S>(__VA_ARGS__);         \
    case LBM_F16S: return fn<LBM_F16S>(__VA_ARGS__);         \
    default: return fn<LBM_BF16S>(__VA_ARGS__);              \
  }

size_t dispatch_force_bytes(int prec) { LBM_BATCH_DISPATCH(prec, force_bytes) }

bool valid_batch(const lbm_state* st) { return valid_state(st) && st->batch; }

}  // namespace

int batch_steps(lbm_state* st, int32_t n_steps, double wp, double wm, const double* forces) {
  LBM_BATCH_DISPATCH(st->precision, run_batch, st, n_steps, wp, wm, forces)
}

int batch_reduce(lbm_state* st, int32_t axis, double* mass_out, double* flux_out) {
  Batch* b = st->batch;
  const cudaStream_t stream = st->sp->stream;
  if (st->sp->n > 0) {
    batch_final_kernel<<<b->n_beds, 1024, 0, stream>>>(st->partials, b->d_begin, b->d_count,
                                                       b->d_red);
    LBM_CUDA_TRY(cudaGetLastError());
    LBM_CUDA_TRY(cudaMemcpyAsync(b->h_red, b->d_red, sizeof(double) * 4 * b->n_beds,
                                 cudaMemcpyDeviceToHost, stream));
    const int rc = wait_event(st->done, stream, 0.0);
    if (rc != LBM_OK) return rc;
  } else {
    for (int i = 0; i < 4 * b->n_beds; ++i) b->h_red[i] = 0.0;
  }
  const bool shifted = is_shifted(st->precision);
  for (int i = 0; i < b->n_beds; ++i) {
    const double cnt = (double)b->h_count[i];
    const double mass = shifted ? cnt + b->h_red[4 * i] : b->h_red[4 * i];
    const double flux = b->h_count[i] > 0 ? b->h_red[4 * i + 1 + axis] / cnt : 0.0;
    if (!std::isfinite(mass) || !std::isfinite(flux))
      return fail(LBM_ENONFINITE, "bed %d: non-finite mass (%g) or flux (%g)", i, mass, flux);
    if (mass_out) mass_out[i] = mass;
    if (flux_out) flux_out[i] = flux;
  }
  return LBM_OK;
}

void free_batch(lbm_state* st) {
  Batch* b = st->batch;
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->capture) cudaStreamDestroy(b->capture);
  for (void* p : {(void*)b->d_begin, (void*)b->d_count, (void*)b->d_chunk_bed, b->d_force,
                  (void*)b->d_red})
    if (p) cudaFree(p);
  for (void* p : {b->h_force, (void*)b->h_red})
    if (p) cudaFreeHost(p);
  delete[] b->h_begin;
  delete[] b->h_count;
  delete b;
  st->batch = nullptr;
  free_sparse(const_cast<lbm_sparse*>(st->sp));
  st->sp = nullptr;
}

}  // namespace lbm

using namespace lbm;

extern "C" int lbm_state_create_batched(const lbm_sparse* const* beds, int32_t n_beds,
                                        int32_t precision, int32_t scale_exp, lbm_state** out) {
  clear_error();
  if (!out) return fail(LBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!beds || n_beds < 1) return fail(LBM_EINVAL, "need at least one bed");
  for (int i = 0; i < n_beds; ++i)
    if (!beds[i] || beds[i]->magic != kMagicSparse)
      return fail(LBM_EINVAL, "beds[%d] is not a sparse handle", i);
  const cudaStream_t stream = beds[0]->stream;
  std::vector<int64_t> begin(n_beds), count(n_beds);
  int64_t total = 0;
  for (int i = 0; i < n_beds; ++i) {
    begin[i] = total;
    count[i] = beds[i]->n;
    total += (count[i] + kBatchChunk - 1) / kBatchChunk * kBatchChunk;
  }
  if (19 * total >= ((int64_t)1 << 31))
    return fail(LBM_EOVERFLOW, "%lld padded cells: 19*N exceeds the int32 adjacency range",
                (long long)total);
  // concatenated sparse representation (owned by the state)
  lbm_sparse* cat = new lbm_sparse{};
  cat->magic = kMagicSparse;
  cat->n = total;
  cat->stream = stream;
  cat->ord.kind = -1;
  if (cudaMalloc(&cat->adj, sizeof(int32_t) * 18 * (size_t)(total > 0 ? total : 1)) !=
      cudaSuccess) {
    cudaGetLastError();
    delete cat;
    return fail(LBM_ENOMEM, "batched adjacency allocation failed");
  }
  if (total > 0) {
    const int64_t t = 18 * total;
    self_bounce_kernel<<<(unsigned)((t + 255) / 256), 256, 0, stream>>>(cat->adj, (int32_t)total);
    for (int i = 0; i < n_beds; ++i)
      if (count[i] > 0)
        concat_adj_kernel<<<(unsigned)((18 * count[i] + 255) / 256), 256, 0, stream>>>(
            beds[i]->adj, (int32_t)count[i], (int32_t)begin[i], (int32_t)total, cat->adj);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    free_sparse(cat);
    return cuda_fail(e, "batched adjacency");
  }
  lbm_state* st = nullptr;
  int rc = lbm_state_create(cat, precision, scale_exp, &st);
  if (rc != LBM_OK) {
    free_sparse(cat);
    return rc;
  }
  Batch* b = new Batch{};
  st->batch = b;
  b->n_beds = n_beds;
  b->h_begin = new int64_t[n_beds];
  b->h_count = new int64_t[n_beds];
  std::vector<int32_t> count32(n_beds);
  for (int i = 0; i < n_beds; ++i) {
    b->h_begin[i] = begin[i];
    b->h_count[i] = count[i];
    count32[i] = (int32_t)count[i];
  }
  const int64_t n_chunks = total / kBatchChunk;
  std::vector<int32_t> chunk_bed((size_t)(n_chunks > 0 ? n_chunks : 1), 0);
  for (int i = 0; i < n_beds; ++i)
    for (int64_t c = begin[i] / kBatchChunk; c < (begin[i] + count[i] + kBatchChunk - 1) / kBatchChunk; ++c)
      chunk_bed[c] = i;
  b->block = kSweepThreads;
  b->cpt = 1;
  b->use_graph = 1;
  const size_t fbytes = dispatch_force_bytes(precision);
  bool ok = cudaMalloc(&b->d_begin, sizeof(int64_t) * n_beds) == cudaSuccess &&
            cudaMalloc(&b->d_count, sizeof(int32_t) * n_beds) == cudaSuccess &&
            cudaMalloc(&b->d_chunk_bed, sizeof(int32_t) * chunk_bed.size()) == cudaSuccess &&
            cudaMalloc(&b->d_force, fbytes * n_beds) == cudaSuccess &&
            cudaMallocHost(&b->h_force, fbytes * n_beds) == cudaSuccess &&
            cudaMalloc(&b->d_red, sizeof(double) * 4 * n_beds) == cudaSuccess &&
            cudaMallocHost(&b->h_red, sizeof(double) * 4 * n_beds) == cudaSuccess &&
            cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_state(st);
    return fail(LBM_ENOMEM, "batch tables allocation failed");
  }
  e = cudaMemcpyAsync(b->d_begin, begin.data(), sizeof(int64_t) * n_beds, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_count, count32.data(), sizeof(int32_t) * n_beds, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_chunk_bed, chunk_bed.data(), sizeof(int32_t) * chunk_bed.size(),
                        cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    free_state(st);
    return cuda_fail(e, "batch tables upload");
  }
  *out = st;
  return LBM_OK;
}

extern "C" int lbm_batch_layout(const lbm_state* st, int32_t* n_beds, int64_t* begin_out,
                                int64_t* count_out, int64_t* n_padded) {
  clear_error();
  if (!valid_batch(st)) return fail(LBM_EINVAL, "not a batched state");
  const Batch* b = st->batch;
  if (n_beds) *n_beds = b->n_beds;
  if (n_padded) *n_padded = st->sp->n;
  for (int i = 0; i < b->n_beds; ++i) {
    if (begin_out) begin_out[i] = b->h_begin[i];
    if (count_out) count_out[i] = b->h_count[i];
  }
  return LBM_OK;
}

extern "C" int lbm_batch_config(lbm_state* st, int32_t block, int32_t cells_per_thread,
                                int32_t use_graph) {
  clear_error();
  if (!valid_batch(st)) return fail(LBM_EINVAL, "not a batched state");
  if (block != 128 && block != 256 && block != 512)
    return fail(LBM_EINVAL, "block %d not in {128, 256, 512}", block);
  if (cells_per_thread != 1 && cells_per_thread != 2 && cells_per_thread != 4)
    return fail(LBM_EINVAL, "cells per thread %d not in {1, 2, 4}", cells_per_thread);
  st->batch->block = block;
  st->batch->cpt = cells_per_thread;
  st->batch->use_graph = use_graph != 0;
  return LBM_OK;
}

extern "C" int lbm_batch_tune(lbm_state* st, int32_t steps_per_candidate, double omega_plus,
                              double omega_minus, const double* forces, int32_t* block_out,
                              int32_t* cpt_out, float* ms_out /* [9] or NULL */) {
  clear_error();
  if (!valid_batch(st)) return fail(LBM_EINVAL, "not a batched state");
  if (steps_per_candidate < 1) return fail(LBM_EINVAL, "steps_per_candidate must be >= 1");
  Batch* b = st->batch;
  const int blocks[3] = {128, 256, 512}, cpts[3] = {1, 2, 4};
  const int saved_graph = b->use_graph;
  b->use_graph = 0;
  cudaEvent_t e0, e1;
  LBM_CUDA_TRY(cudaEventCreate(&e0));
  LBM_CUDA_TRY(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_b = b->block, best_c = b->cpt, idx = 0;
  int rc = LBM_OK;
  for (int bi = 0; bi < 3 && rc == LBM_OK; ++bi)
    for (int ci = 0; ci < 3 && rc == LBM_OK; ++ci, ++idx) {
      b->block = blocks[bi];
      b->cpt = cpts[ci];
      rc = lbm_step(st, 1, omega_plus, omega_minus, forces);  // warm the shape
      if (rc != LBM_OK) break;
      cudaEventRecord(e0, st->sp->stream);
      rc = lbm_step(st, steps_per_candidate, omega_plus, omega_minus, forces);
      cudaEventRecord(e1, st->sp->stream);
      if (rc != LBM_OK) break;
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = cuda_fail(cudaGetLastError(), "timing a candidate shape");
        break;
      }
      if (ms_out) ms_out[idx] = ms;
      if (ms < best) {
        best = ms;
        best_b = blocks[bi];
        best_c = cpts[ci];
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->block = best_b;
  b->cpt = best_c;
  b->use_graph = saved_graph;
  if (rc != LBM_OK) return rc;
  if (block_out) *block_out = best_b;
  if (cpt_out) *cpt_out = best_c;
  return LBM_OK;
}
