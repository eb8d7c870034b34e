// Batched sweep: many independent packed beds of uneven size in one launch
// per time step.
//
// The beds' sparse representations are concatenated into one list; each bed
// starts at a multiple of kBatchChunk (2048) cells, so any tile of
// block x cells-per-thread <= 2048 cells lies inside one bed and finds its
// bed from a per-chunk table -- no per-cell bed id is stored or read.  The
// adjacency is remapped to the concatenated slots (q*N + m of a bed becomes
// q*N_pad + begin + m, before the L2 groups below relayout it); padding
// cells bounce every link onto themselves and
// are never read or written by the sweep.  Each bed has its own body force,
// taken from a small table.  The step that reduces runs with the 256-thread,
// one-cell-per-thread layout of the single-bed sweep and reduces each bed
// over its own 256-cell blocks in the same order, so a bed's PDFs and flux
// are bit-identical to running it alone.
//
// Launch shape: the non-reducing steps use (block, cells per thread) from
// {128, 256, 512} x {1, 2, 4}, picked by lbm_batch_tune; all shapes give the
// same per-cell arithmetic.  The launches of a call are captured once into a
// CUDA graph (on a private stream) and replayed on the caller's stream.
//
// L2 groups: the beds, in list order, form groups whose working set fits a
// budget (by default 0.6 of the L2), and a call takes all its steps on one
// group before the next, so that a group's steps stream from L2.  Each
// group keeps its arrays contiguous -- 19 PDF rows and 18 link rows of its
// own padded length, links holding group-local slots -- and lbm_state_get/
// set_pdfs convert to and from the plain [19][N_pad] layout.  Beds are
// independent and every bed takes the same steps in the same order, so the
// grouping changes no result.
//
// Resident steps (lbm_batch_resident): a group that fits one 1024-thread
// block per SM, each keeping the links of its run of cells in shared
// memory, takes all but its reducing step in one cooperative launch with a
// bounded grid barrier between steps.
#include <algorithm>
#include <cmath>
#include <cstdint>
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

// LINKS_FIRST (one cell per thread, not reducing): the bed tables, the
// force and the cell's links, which no step writes, are read before the
// wait for the previous step, so a chained launch overlaps them with that
// step's end.  A group's launch lasts ~10 us, so that overlap is a large
// part of it.  256 beds in L2 groups, 1000 steps, MFLUP/s: FP32S 41,417 ->
// 45,679, FP16S 51,422 -> 53,846; as one group FP32S 31,354 -> 30,751,
// FP16S 36,384 -> 39,202.
#ifndef LBM_BATCH_LINKS_FIRST
#define LBM_BATCH_LINKS_FIRST 1
#endif
template <int PREC, bool REDUCE, int CPT, bool LINKS_FIRST = false>
__global__ void __launch_bounds__(512)
    batch_sweep_kernel(const typename Form<PREC>::S* __restrict__ src,
                       typename Form<PREC>::S* __restrict__ dst, const int32_t* __restrict__ adj,
                       int32_t n, Coef<typename Form<PREC>::C> k,
                       const BedForce<typename Form<PREC>::C>* __restrict__ forces,
                       const int32_t* __restrict__ chunk_bed, const int64_t* __restrict__ begin,
                       const int32_t* __restrict__ count, int64_t cell0,
                       double* __restrict__ partials) {
  using C = typename Form<PREC>::C;
  static_assert(!LINKS_FIRST || (CPT == 1 && !REDUCE), "links first: one cell, not reducing");
  // A chained launch waits here for the previous step.  The zero it returns
  // offsets every index and the sums pointer, so no access is scheduled
  // ahead of the wait.
  int32_t z = 0;
  if constexpr (!LINKS_FIRST) z = prior_step_done();
  // src, dst and adj are the group's arrays, n its padded length; `base` is
  // local to the group, cell0 + base the padded index in the whole list
  const int64_t base = (int64_t)blockIdx.x * blockDim.x * CPT + z;
  const int bed = chunk_bed[(cell0 + base) / kBatchChunk];
  const int64_t end = begin[bed] + count[bed] - cell0;
  Coef<C> kb = k;
  const BedForce<C> bf = forces[bed];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    kb.F[d] = bf.F[d];
    kb.hF[d] = bf.hF[d];
    kb.bF1[d] = bf.bF1[d];
  }
  C rho = C(0), u[3] = {C(0), C(0), C(0)};
  if constexpr (LINKS_FIRST) {
    const int64_t i = base + threadIdx.x;
    int32_t idx[18];
    if (i < end) load_links(adj, n, (int32_t)i, idx);
    z = prior_step_done();   // PDF accesses are volatile asm: kept behind the wait
    if (i < end) {
      C g[19];
      pull<PREC>(src, idx, (int32_t)i + z, kb.inv_scale, g);
      collide<C, false>(g, kb, C(0), rho, u);
#pragma unroll
      for (int q = 0; q < 19; ++q)
        store_stream<PREC>(dst + q * n + i + z, encode<PREC>(g[q], kb.scale));
    }
    return;
  }
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
    store_warp_sums(w, partials + z);
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

// ---- resident steps ------------------------------------------------------------
// One cooperative launch takes all non-reducing steps of an L2 group: one
// block of kResidentThreads per SM, each owning a run of up to res_tile
// consecutive cells whose links it reads once into shared memory.  Between
// steps every block waits at a grid barrier, so a step reads only the PDFs
// (from L2) and not the links, which are half of a 16-bit step's bytes.
// Loads that may meet data written earlier in the same launch go through
// L2 (ld.global.cg): the non-coherent path may hold stale lines.  On a
// periodic 80x80x72 box, 1000 FP16S steps: 64,400 MFLUP/s against 56,700
// for chained per-step launches; the barrier costs 1.4 us per step.  On 256
// packed beds, 1000 steps: FP16S 55,729 and FP32S 49,157 MFLUP/s against
// 54,012 and 45,852 for per-step launches in L2 groups.  Its warps wait
// mostly at the barriers, but two or four independent groups per launch
// (one block of each per SM, to fill those waits) ran no faster.
constexpr int kResidentThreads = 1024;
// Chunks of kBatchChunk cells that one block's run of cells can touch.
constexpr int kResidentMaxChunks = 4;
// A barrier wait gives up after this long (all blocks are co-resident, so
// only a fault elsewhere can hold one back); the check mode's waits never
// end by themselves and give up after the short limit.
constexpr uint64_t kBarrierLimitNs = 2000000000ull;
constexpr uint64_t kBarrierCheckLimitNs = 20000000ull;

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned short ld_cg(const unsigned short* p) {
  unsigned short v;
  asm volatile("ld.global.cg.u16 %0, [%1];" : "=h"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float ld_cg(const float* p) {
  float v;
  asm volatile("ld.global.cg.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ void st_wb(unsigned short* p, unsigned short v) {
  asm volatile("st.global.u16 [%0], %1;" ::"l"(p), "h"(v) : "memory");
}
__device__ __forceinline__ void st_wb(float* p, float v) {
  asm volatile("st.global.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

template <int PREC>
__device__ __forceinline__ typename Form<PREC>::C load_coherent(const typename Form<PREC>::S* p,
                                                               typename Form<PREC>::C inv_scale) {
  if constexpr (PREC == LBM_F16S)
    return decode<PREC>(__ushort_as_half(ld_cg(reinterpret_cast<const unsigned short*>(p))),
                        inv_scale);
  else if constexpr (PREC == LBM_BF16S)
    return decode<PREC>(__ushort_as_bfloat16(ld_cg(reinterpret_cast<const unsigned short*>(p))),
                        inv_scale);
  else
    return ld_cg(p);
}

template <int PREC>
__device__ __forceinline__ void store_wb(typename Form<PREC>::S* p, typename Form<PREC>::C v,
                                         typename Form<PREC>::C scale) {
  if constexpr (PREC == LBM_F16S)
    st_wb(reinterpret_cast<unsigned short*>(p), __half_as_ushort(encode<PREC>(v, scale)));
  else if constexpr (PREC == LBM_BF16S)
    st_wb(reinterpret_cast<unsigned short*>(p), __bfloat16_as_ushort(encode<PREC>(v, scale)));
  else
    st_wb(p, v);
}

// Forms with resident steps: FP32 and 16-bit arithmetic (the FP64 steps
// need more than the 64 registers a 1024-thread block leaves a thread).
constexpr bool resident_form(int prec) { return prec != LBM_F64 && prec != LBM_F64X; }

// Every block adds one to *counter and waits until it reaches target.  The
// release add and the acquire poll of thread 0, between two block barriers,
// order every thread's stores of this step before every thread's loads of
// the next.  A wait that runs past limit_ns sets *err; once *err is set
// every wait returns at once, so the launch always ends.
__device__ __forceinline__ void grid_barrier(uint32_t* counter, uint32_t target, int32_t* err,
                                             uint64_t limit_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(counter) : "memory");
    const uint64_t t0 = global_ns();
    for (;;) {
      uint32_t v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(counter) : "memory");
      if (v >= target) break;
      if (*(volatile int32_t*)err) break;
      if (global_ns() - t0 > limit_ns) {
        atomicExch(err, 1);
        break;
      }
    }
  }
  __syncthreads();
}

template <class C>
struct ChunkBed {
  BedForce<C> f;
  int64_t end;   // group-local end of the live cells of the chunk's bed
};

// `steps` non-reducing steps of the group's padded cells [0, n) (global
// cells cell0 + i), from buf0 (steps even: ending in buf0, odd: in buf1).
// Block b owns cells [b tile, b tile + tile).  check: each barrier waits for
// one arrival more than the grid makes (tests the time limit).
template <int PREC>
__global__ void __launch_bounds__(kResidentThreads, 1)
    batch_resident_kernel(typename Form<PREC>::S* buf0, typename Form<PREC>::S* buf1,
                          const int32_t* __restrict__ adj, int32_t n, int32_t tile,
                          Coef<typename Form<PREC>::C> k,
                          const BedForce<typename Form<PREC>::C>* __restrict__ forces,
                          const int32_t* __restrict__ chunk_bed, const int64_t* __restrict__ begin,
                          const int32_t* __restrict__ count, int64_t cell0, int32_t steps,
                          uint32_t* counter, int32_t* err, int32_t check) {
  using C = typename Form<PREC>::C;
  using S = typename Form<PREC>::S;
  extern __shared__ int32_t links[];   // [18][tile]
  __shared__ ChunkBed<C> tab[kResidentMaxChunks];
  const int64_t c0 = (int64_t)blockIdx.x * tile;
  const int cnt = (int)min((int64_t)tile, (int64_t)n - c0);
  const int64_t ch0 = (cell0 + c0) / kBatchChunk;
  if (threadIdx.x < kResidentMaxChunks && cnt > 0 &&
      ch0 + threadIdx.x <= (cell0 + c0 + cnt - 1) / kBatchChunk) {
    const int bed = chunk_bed[ch0 + threadIdx.x];
    tab[threadIdx.x].f = forces[bed];
    tab[threadIdx.x].end = begin[bed] + count[bed] - cell0;
  }
  for (int e = threadIdx.x; e < 18 * tile; e += kResidentThreads) {
    const int q = e / tile, j = e - q * tile;
    links[e] = j < cnt ? adj[(int64_t)q * n + c0 + j] : 0;
  }
  __syncthreads();
  const uint64_t limit = check ? kBarrierCheckLimitNs : kBarrierLimitNs;
  for (int s = 0; s < steps; ++s) {
    const S* src = (s & 1) ? buf1 : buf0;
    S* dst = (s & 1) ? buf0 : buf1;
    for (int j = threadIdx.x; j < cnt; j += kResidentThreads) {
      const int64_t i = c0 + j;
      const ChunkBed<C>& cb = tab[(cell0 + i) / kBatchChunk - ch0];
      if (i >= cb.end) continue;   // padding after the bed's last cell
      Coef<C> kb = k;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        kb.F[d] = cb.f.F[d];
        kb.hF[d] = cb.f.hF[d];
        kb.bF1[d] = cb.f.bF1[d];
      }
      C g[19], rho, u[3];
      g[0] = load_coherent<PREC>(src + i, kb.inv_scale);
#pragma unroll
      for (int q = 1; q < 19; ++q)
        g[q] = load_coherent<PREC>(src + links[(q - 1) * tile + j], kb.inv_scale);
      collide<C, false>(g, kb, C(0), rho, u);
#pragma unroll
      for (int q = 0; q < 19; ++q) store_wb<PREC>(dst + (int64_t)q * n + i, g[q], kb.scale);
    }
    if (s + 1 < steps)
      grid_barrier(counter, (uint32_t)(s + 1) * gridDim.x + (check ? 1u : 0u), err, limit);
  }
}

// ---- group layout ------------------------------------------------------------
// A layout on the device: the group of each 2048-cell chunk and each group's
// first padded cell and length; chunk_group null: one group of all cells.
struct GroupLayout {
  const int32_t* chunk_group;
  const int64_t* cell0;
  const int64_t* span;
};

__device__ __forceinline__ void group_of(const GroupLayout& L, int64_t i, int64_t n, int64_t& c0,
                                         int64_t& span) {
  if (!L.chunk_group) {
    c0 = 0;
    span = n;
    return;
  }
  const int g = L.chunk_group[i / kBatchChunk];
  c0 = L.cell0[g];
  span = L.span[g];
}

// dst in layout `to` = src in layout `from`, element (q, i) for q < 19.
template <class T>
__global__ void relayout_pdfs_kernel(const T* __restrict__ src, T* __restrict__ dst, int64_t n,
                                     GroupLayout from, GroupLayout to) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 19 * n) return;
  const int64_t q = e / n, i = e - q * n;
  int64_t ca, sa, cb, sb;
  group_of(from, i, n, ca, sa);
  group_of(to, i, n, cb, sb);
  dst[19 * cb + q * sb + (i - cb)] = src[19 * ca + q * sa + (i - ca)];
}

// The links in layout `to` from those in layout `from`: a link is a slot
// q' * span + j local to the cell's group, and the pulled cell c0 + j lies in
// the same bed, hence in the same group of either layout.
__global__ void relayout_adj_kernel(const int32_t* __restrict__ src, int32_t* __restrict__ dst,
                                    int64_t n, GroupLayout from, GroupLayout to) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 18 * n) return;
  const int64_t r = e / n, i = e - r * n;
  int64_t ca, sa, cb, sb;
  group_of(from, i, n, ca, sa);
  group_of(to, i, n, cb, sb);
  const int64_t v = src[18 * ca + r * sa + (i - ca)];
  const int64_t q = v / sa, j = v - q * sa;
  dst[18 * cb + r * sb + (i - cb)] = (int32_t)(q * sb + (ca + j - cb));
}

GroupLayout layout_of(const Batch* b) {
  if (b->group_cell0.size() <= 1) return GroupLayout{nullptr, nullptr, nullptr};
  return GroupLayout{b->d_chunk_group, b->d_group_cell0, b->d_group_span};
}

int relayout_pdfs(const lbm_state* st, int from_buf, int to_buf, GroupLayout from,
                  GroupLayout to) {
  const int64_t n = st->sp->n;
  if (n == 0) return LBM_OK;
  const unsigned grid = (unsigned)((19 * n + 255) / 256);
  const cudaStream_t stream = st->sp->stream;
  switch (storage_bytes(st->precision)) {
    case 2:
      relayout_pdfs_kernel<uint16_t><<<grid, 256, 0, stream>>>(
          (const uint16_t*)st->buf[from_buf], (uint16_t*)st->buf[to_buf], n, from, to);
      break;
    case 4:
      relayout_pdfs_kernel<uint32_t><<<grid, 256, 0, stream>>>(
          (const uint32_t*)st->buf[from_buf], (uint32_t*)st->buf[to_buf], n, from, to);
      break;
    default:
      relayout_pdfs_kernel<uint64_t><<<grid, 256, 0, stream>>>(
          (const uint64_t*)st->buf[from_buf], (uint64_t*)st->buf[to_buf], n, from, to);
  }
  LBM_CUDA_TRY(cudaGetLastError());
  return LBM_OK;
}

// One step of the padded cells [cell0, cell0 + span) (whole beds, span a
// multiple of kBatchChunk).  `chained`: the previous launch on the stream is
// a step of the same call (not in FP64 arithmetic, which chaining slows
// down; see lbm_step).
template <int PREC, bool REDUCE>
cudaError_t launch_one(lbm_state* st, int block, int cpt, cudaStream_t stream,
                       const Coef<typename Form<PREC>::C>& k, bool chained, int64_t cell0,
                       int64_t span) {
  using S = typename Form<PREC>::S;
  using C = typename Form<PREC>::C;
  Batch* b = st->batch;
  const int32_t n = (int32_t)span;
  const S* src = (const S*)st->buf[st->cur] + 19 * cell0;
  S* dst = (S*)st->buf[st->cur ^ 1] + 19 * cell0;
  const int32_t* adj = st->sp->adj + 18 * cell0;
  const unsigned grid = (unsigned)(span / (block * cpt));
  const BedForce<C>* forces = (const BedForce<C>*)b->d_force;
  const bool pdl = chained && PREC != LBM_F64 && PREC != LBM_F64X;
  // the reducing step's warp slots are indexed by global 256-cell block
  double* partials = st->partials + 4 * kWarpsPerBlock * (cell0 / kSweepThreads);
#define LBM_BATCH_LAUNCH(CPT)                                                          \
  launch_chained(batch_sweep_kernel<PREC, REDUCE, CPT>, grid, (unsigned)block, stream, pdl, \
                 src, dst, adj, n, k, forces,                                          \
                 (const int32_t*)b->d_chunk_bed, (const int64_t*)b->d_begin,           \
                 (const int32_t*)b->d_count, cell0, partials)
  cudaError_t e;
  if (LBM_BATCH_LINKS_FIRST && !REDUCE && cpt == 1)
    e = launch_chained(batch_sweep_kernel<PREC, false, 1, true>, grid, (unsigned)block, stream,
                       pdl, src, dst, adj, n, k, forces, (const int32_t*)b->d_chunk_bed,
                       (const int64_t*)b->d_begin, (const int32_t*)b->d_count, cell0, partials);
  else if (cpt == 1) e = LBM_BATCH_LAUNCH(1);
  else if (cpt == 2) e = LBM_BATCH_LAUNCH(2);
  else e = LBM_BATCH_LAUNCH(4);
#undef LBM_BATCH_LAUNCH
  st->cur ^= 1;
  return e;
}

// The first n_steps steps of the cells [cell0, cell0 + span) in one
// cooperative launch (resident steps); counter: the group's barrier count,
// zeroed before the call.
template <int PREC>
cudaError_t launch_resident(lbm_state* st, cudaStream_t stream,
                            const Coef<typename Form<PREC>::C>& k, int64_t cell0, int64_t span,
                            int32_t n_steps, uint32_t* counter) {
  using S = typename Form<PREC>::S;
  using C = typename Form<PREC>::C;
  Batch* b = st->batch;
  const int64_t blocks = b->res_cells / b->res_tile;
  // the group's cells spread evenly over the SMs, 64 cells at a time
  const int64_t tile = ((span + blocks - 1) / blocks + 63) / 64 * 64;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeCooperative;
  attr.val.cooperative = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((span + tile - 1) / tile));
  cfg.blockDim = dim3(kResidentThreads);
  cfg.dynamicSmemBytes = (size_t)(18 * sizeof(int32_t) * tile);
  cfg.stream = stream;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  S* src = (S*)st->buf[st->cur] + 19 * cell0;
  S* dst = (S*)st->buf[st->cur ^ 1] + 19 * cell0;
  const cudaError_t e = cudaLaunchKernelEx(
      &cfg, batch_resident_kernel<PREC>, src, dst, (const int32_t*)(st->sp->adj + 18 * cell0),
      (int32_t)span, (int32_t)tile, k, (const BedForce<C>*)b->d_force,
      (const int32_t*)b->d_chunk_bed, (const int64_t*)b->d_begin, (const int32_t*)b->d_count,
      cell0, n_steps, counter, b->d_sync_err, (int32_t)(b->resident < 0));
  st->cur ^= (n_steps & 1);
  return e;
}

// Enqueues n_steps steps of the cells [cell0, cell0 + span) (group `group`)
// on `stream` (the last one reduces); the first launch is chained when
// `chain_first`.  With resident steps on and a group that fits, all but the
// last step are one cooperative launch.
template <int PREC>
cudaError_t enqueue_steps(lbm_state* st, int32_t n_steps, double wp, double wm, int block,
                          int cpt, cudaStream_t stream, int64_t cell0, int64_t span,
                          bool chain_first, size_t group) {
  using C = typename Form<PREC>::C;
  const double zero[3] = {0.0, 0.0, 0.0};
  const Coef<C> k = make_coef<C>(wp, wm, zero, st->scale_exp);
  cudaError_t err = cudaSuccess;
  if constexpr (resident_form(PREC)) {
    const Batch* b = st->batch;
    if (b->resident != 0 && n_steps >= 2 && span <= b->res_cells) {
      err = launch_resident<PREC>(st, stream, k, cell0, span, n_steps - 1, b->d_sync + group);
      const cudaError_t e =
          launch_one<PREC, true>(st, kSweepThreads, 1, stream, k, false, cell0, span);
      return err != cudaSuccess ? err : e;
    }
  }
  for (int32_t t = 0; t < n_steps; ++t) {
    const bool chained = t > 0 || chain_first;
    const cudaError_t e =
        t == n_steps - 1
            ? launch_one<PREC, true>(st, kSweepThreads, 1, stream, k, chained, cell0, span)
            : launch_one<PREC, false>(st, block, cpt, stream, k, chained, cell0, span);
    if (err == cudaSuccess) err = e;
  }
  return err;
}

// All steps of one group, then of the next: every group starts from the
// call's parity and ends at parity ^ (n_steps & 1).
template <int PREC>
cudaError_t enqueue_grouped(lbm_state* st, int32_t n_steps, double wp, double wm,
                            cudaStream_t stream) {
  Batch* b = st->batch;
  const int parity = st->cur;
  cudaError_t err = cudaSuccess;
  for (size_t g = 0; g < b->group_cell0.size(); ++g) {
    st->cur = parity;
    const cudaError_t e = enqueue_steps<PREC>(st, n_steps, wp, wm, b->block, b->cpt, stream,
                                              b->group_cell0[g], b->group_span[g], g > 0, g);
    if (err == cudaSuccess) err = e;
  }
  st->cur = parity ^ (n_steps & 1);
  return err;
}

// The launches of one call: grouped, or every step over all beds.
template <int PREC>
cudaError_t enqueue_call(lbm_state* st, int32_t n_steps, double wp, double wm,
                         cudaStream_t stream) {
  Batch* b = st->batch;
  if (b->group_cell0.size() > 1) return enqueue_grouped<PREC>(st, n_steps, wp, wm, stream);
  return enqueue_steps<PREC>(st, n_steps, wp, wm, b->block, b->cpt, stream, 0, st->sp->n, false,
                             0);
}

// Largest graph (kernel nodes) a call is captured into; longer calls launch
// their kernels one by one.
constexpr int64_t kMaxBatchGraphNodes = 1 << 18;

// After the stream has drained: LBM_ETIMEOUT (and the flag cleared) when a
// grid barrier wait of the last resident call ran out of time.
int take_barrier_error(lbm_state* st, cudaStream_t stream) {
  Batch* b = st->batch;
  if (*b->h_sync_err == 0) return LBM_OK;
  *b->h_sync_err = 0;
  LBM_CUDA_TRY(cudaMemsetAsync(b->d_sync_err, 0, sizeof(int32_t), stream));
  return fail(LBM_ETIMEOUT,
              "a grid barrier wait of the last resident call ran out of time: its results are "
              "not valid");
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
  int rc = fill_forces<PREC>(st, wm, forces, stream);   // drains the stream first
  if (rc != LBM_OK) return rc;
  rc = take_barrier_error(st, stream);
  if (rc != LBM_OK) return rc;
  if (st->sp->n == 0) {
    st->cur ^= (n_steps & 1);
    return LBM_OK;
  }
  if (resident_form(PREC) && b->resident != 0) {
    // a few launches per group: launched directly, no graph
    LBM_CUDA_TRY(cudaMemsetAsync(b->d_sync, 0, sizeof(uint32_t) * b->group_cell0.size(), stream));
    LBM_CUDA_TRY(enqueue_call<PREC>(st, n_steps, wp, wm, stream));
    LBM_CUDA_TRY(cudaMemcpyAsync(b->h_sync_err, b->d_sync_err, sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, stream));
    return LBM_OK;
  }
  const int64_t nodes = (int64_t)b->group_cell0.size() * n_steps;
  if (!b->use_graph || nodes > kMaxBatchGraphNodes) {
    LBM_CUDA_TRY(enqueue_call<PREC>(st, n_steps, wp, wm, stream));
    return LBM_OK;
  }
  const bool hit = b->graph && b->g_steps == n_steps && b->g_parity == st->cur &&
                   b->g_block == b->block && b->g_cpt == b->cpt && b->g_wp == wp &&
                   b->g_wm == wm && b->g_group_bytes == b->group_bytes;
  if (!hit) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    const int parity = st->cur;
    LBM_CUDA_TRY(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
    const cudaError_t el = enqueue_call<PREC>(st, n_steps, wp, wm, b->capture);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->capture, &g);
    st->cur = parity;  // capture only recorded the launches
    if (el != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(el, "batch step launch under capture");
    }
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
    b->g_group_bytes = b->group_bytes;
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

// The resident capacity of the state's form on the current device: the
// largest run of cells (a multiple of 64) whose links fit one block's
// shared memory, times one block per SM.  Raises the kernel's dynamic
// shared-memory limit to that run.
template <int PREC>
int setup_resident(lbm_state* st) {
  if constexpr (!resident_form(PREC)) {
    return fail(LBM_EINVAL, "resident steps need FP32 or 16-bit arithmetic");
  } else {
    int dev = 0, sms = 0, optin = 0;
    LBM_CUDA_TRY(cudaGetDevice(&dev));
    LBM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    LBM_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    LBM_CUDA_TRY(cudaFuncGetAttributes(&fa, batch_resident_kernel<PREC>));
    const int64_t per_cell = 18 * (int64_t)sizeof(int32_t);
    // The longest run that fits (3,200 cells on GB300).  Runs of whole
    // 1024-cell rounds (3,072) made more groups and ran 1% slower on the 256
    // beds in both FP16S and FP32S.
    int64_t tile = ((int64_t)optin - (int64_t)fa.sharedSizeBytes) / per_cell / 64 * 64;
    // a run must touch at most kResidentMaxChunks chunks
    tile = std::min<int64_t>(tile, (kResidentMaxChunks - 1) * kBatchChunk);
    if (tile < 64) return fail(LBM_EINVAL, "too little shared memory for resident steps");
    LBM_CUDA_TRY(cudaFuncSetAttribute(batch_resident_kernel<PREC>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(per_cell * tile)));
    int per_sm = 0;
    LBM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, batch_resident_kernel<PREC>, kResidentThreads, (size_t)(per_cell * tile)));
    if (per_sm < 1) return fail(LBM_EINVAL, "a resident block does not fit an SM");
    st->batch->res_tile = tile;
    st->batch->res_cells = tile * sms;
    return LBM_OK;
  }
}

int dispatch_setup_resident(int prec, lbm_state* st) { LBM_BATCH_DISPATCH(prec, setup_resident, st) }

bool valid_batch(const lbm_state* st) { return valid_state(st) && st->batch; }

// Splits the beds, in layout order, into groups whose working set (two PDF
// grids and the adjacency, per padded cell) fits `bytes`; a bed larger than
// that is a group of its own.  bytes <= 0: one group of all beds.  With
// resident steps the working set is the PDF grids, and a group also holds
// at most res_cells cells.
void split_groups(const lbm_state* st, int64_t bytes, std::vector<int64_t>& cell0_out,
                  std::vector<int64_t>& span_out) {
  const Batch* b = st->batch;
  cell0_out.clear();
  span_out.clear();
  const int64_t n_pad = st->sp->n;
  if (bytes <= 0 || n_pad == 0) {
    cell0_out.push_back(0);
    span_out.push_back(n_pad);
    return;
  }
  // resident steps keep the links in shared memory: the PDFs are the working
  // set, and a group holds at most res_cells cells
  const bool res = b->resident != 0;
  const int64_t per_cell = 2 * 19 * (int64_t)storage_bytes(st->precision) + (res ? 0 : 18 * 4);
  const int64_t max_cells = res ? b->res_cells : INT64_MAX;
  int64_t cell0 = 0, span = 0;
  for (int i = 0; i < b->n_beds; ++i) {
    const int64_t s = (b->h_count[i] + kBatchChunk - 1) / kBatchChunk * kBatchChunk;
    if (s == 0) continue;
    if (span > 0 && ((span + s) * per_cell > bytes || span + s > max_cells)) {
      cell0_out.push_back(cell0);
      span_out.push_back(span);
      cell0 = b->h_begin[i];
      span = 0;
    }
    span += s;
  }
  cell0_out.push_back(cell0);
  span_out.push_back(span);
}

void free_group_tables(Batch* b, cudaStream_t stream) {
  for (void* p : {(void*)b->d_chunk_group, (void*)b->d_group_cell0, (void*)b->d_group_span})
    dev_free(p, stream, false);
  b->d_chunk_group = nullptr;
  b->d_group_cell0 = nullptr;
  b->d_group_span = nullptr;
}

// Sets the L2 groups for a budget of `bytes` and moves the current PDFs and
// the links into their layout (the other PDF grid is scratch).  Allocates
// the new group tables and a second link array while it runs.
int regroup(lbm_state* st, int64_t bytes) {
  Batch* b = st->batch;
  std::vector<int64_t> c0, span;
  split_groups(st, bytes, c0, span);
  b->group_bytes = bytes > 0 ? bytes : 0;
  if (c0 == b->group_cell0 && span == b->group_span) return LBM_OK;
  const cudaStream_t stream = st->sp->stream;
  const int64_t n = st->sp->n;
  const GroupLayout from = layout_of(b);
  // new tables
  int32_t* d_chunk_group = nullptr;
  int64_t *d_c0 = nullptr, *d_span = nullptr;
  int32_t* adj_new = nullptr;
  const size_t G = c0.size();
  std::vector<int32_t> chunk_group((size_t)(n / kBatchChunk > 0 ? n / kBatchChunk : 1), 0);
  for (size_t g = 0; g < G; ++g)
    for (int64_t c = c0[g] / kBatchChunk; c < (c0[g] + span[g]) / kBatchChunk; ++c)
      chunk_group[(size_t)c] = (int32_t)g;
  bool ok = dev_alloc(&adj_new, sizeof(int32_t) * 18 * (size_t)(n > 0 ? n : 1), stream, true) ==
            cudaSuccess;
  if (ok && G > 1)
    ok = dev_alloc(&d_chunk_group, sizeof(int32_t) * chunk_group.size(), stream, false) ==
             cudaSuccess &&
         dev_alloc(&d_c0, sizeof(int64_t) * G, stream, false) == cudaSuccess &&
         dev_alloc(&d_span, sizeof(int64_t) * G, stream, false) == cudaSuccess;
  auto release_new = [&]() {
    dev_free(d_chunk_group, stream, false);
    dev_free(d_c0, stream, false);
    dev_free(d_span, stream, false);
    dev_free(adj_new, stream, true);
  };
  if (!ok) {
    cudaGetLastError();
    release_new();
    return fail(LBM_ENOMEM, "allocation for the L2 group layout failed");
  }
  cudaError_t e = cudaSuccess;
  if (G > 1) {
    e = cudaMemcpyAsync(d_chunk_group, chunk_group.data(), sizeof(int32_t) * chunk_group.size(),
                        cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_c0, c0.data(), sizeof(int64_t) * G, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_span, span.data(), sizeof(int64_t) * G, cudaMemcpyHostToDevice,
                          stream);
  }
  const GroupLayout to = G > 1 ? GroupLayout{d_chunk_group, d_c0, d_span}
                               : GroupLayout{nullptr, nullptr, nullptr};
  int rc = LBM_OK;
  if (e == cudaSuccess && n > 0) {
    rc = relayout_pdfs(st, st->cur, st->cur ^ 1, from, to);
    if (rc == LBM_OK) {
      relayout_adj_kernel<<<(unsigned)((18 * n + 255) / 256), 256, 0, stream>>>(
          st->sp->adj, adj_new, n, from, to);
      e = cudaGetLastError();
    }
  }
  // whatever was queued finishes before anything is freed
  const cudaError_t es = cudaStreamSynchronize(stream);
  if (e == cudaSuccess) e = es;
  if (e != cudaSuccess || rc != LBM_OK) {
    release_new();
    cudaStreamSynchronize(stream);
    return rc != LBM_OK ? rc : cuda_fail(e, "L2 group relayout");
  }
  // the cached graph holds the old link array
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  lbm_sparse* sp = const_cast<lbm_sparse*>(st->sp);
  dev_free(sp->adj, stream, true);
  sp->adj = adj_new;
  st->cur ^= 1;
  free_group_tables(b, stream);
  b->d_chunk_group = d_chunk_group;
  b->d_group_cell0 = d_c0;
  b->d_group_span = d_span;
  b->group_cell0 = c0;
  b->group_span = span;
  return LBM_OK;
}

// Default group budget: 0.6 of the L2 (77 MB of GB300's 129 MB).  On 256
// beds of 34.6 M cells in all (FP32 shifted), budgets of 64 and 96 MiB ran
// at 39,500 and 40,000 MFLUP/s, 128 MiB at 32,500, and one group at 31,400.
int64_t default_group_bytes() {
  int dev = 0, l2 = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (int64_t)(0.6 * (double)l2);
}

}  // namespace

bool batch_grouped(const lbm_state* st) {
  return st->batch && st->batch->group_cell0.size() > 1;
}

int batch_relayout_pdfs(const lbm_state* st, int from, int to, bool to_plain) {
  const GroupLayout plain{nullptr, nullptr, nullptr}, grouped = layout_of(st->batch);
  return to_plain ? relayout_pdfs(st, from, to, grouped, plain)
                  : relayout_pdfs(st, from, to, plain, grouped);
}

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
    int rc = wait_event(st->done, stream, 0.0);
    if (rc == LBM_OK) rc = take_barrier_error(st, stream);
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
  const cudaStream_t stream = st->stream;
  cudaStreamSynchronize(stream);
  for (void* p : {(void*)b->d_begin, (void*)b->d_count, (void*)b->d_chunk_bed, b->d_force,
                  (void*)b->d_red, (void*)b->d_sync, (void*)b->d_sync_err})
    dev_free(p, stream, false);
  free_group_tables(b, stream);
  for (void* p : {b->h_force, (void*)b->h_red, (void*)b->h_sync_err})
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
  for (int i = 0; i < n_beds; ++i) {
    if (!beds[i] || beds[i]->magic != kMagicSparse)
      return fail(LBM_EINVAL, "beds[%d] is not a sparse handle", i);
    // the concatenation copies each bed's public links
    const int rc = public_links(beds[i], nullptr);
    if (rc != LBM_OK) return rc;
  }
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
  cat->ld = total;   // a multiple of kBatchChunk: rows already aligned
  cat->stream = stream;
  cat->ord.kind = -1;
  if (dev_alloc(&cat->adj, sizeof(int32_t) * 18 * (size_t)(total > 0 ? total : 1), stream,
                true) != cudaSuccess) {
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
  b->group_cell0.assign(1, 0);
  b->group_span.assign(1, total);
  const size_t fbytes = dispatch_force_bytes(precision);
  bool ok = dev_alloc(&b->d_begin, sizeof(int64_t) * n_beds, stream, false) == cudaSuccess &&
            dev_alloc(&b->d_count, sizeof(int32_t) * n_beds, stream, false) == cudaSuccess &&
            dev_alloc(&b->d_chunk_bed, sizeof(int32_t) * chunk_bed.size(), stream, false) ==
                cudaSuccess &&
            dev_alloc(&b->d_force, fbytes * n_beds, stream, false) == cudaSuccess &&
            cudaMallocHost(&b->h_force, fbytes * n_beds) == cudaSuccess &&
            dev_alloc(&b->d_red, sizeof(double) * 4 * n_beds, stream, false) == cudaSuccess &&
            cudaMallocHost(&b->h_red, sizeof(double) * 4 * n_beds) == cudaSuccess &&
            dev_alloc(&b->d_sync, sizeof(uint32_t) * (size_t)(n_chunks + 1), stream, false) ==
                cudaSuccess &&
            dev_alloc(&b->d_sync_err, sizeof(int32_t), stream, false) == cudaSuccess &&
            cudaMallocHost(&b->h_sync_err, sizeof(int32_t)) == cudaSuccess &&
            cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_state(st);
    return fail(LBM_ENOMEM, "batch tables allocation failed");
  }
  *b->h_sync_err = 0;
  e = cudaMemsetAsync(b->d_sync_err, 0, sizeof(int32_t), stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_begin, begin.data(), sizeof(int64_t) * n_beds, cudaMemcpyHostToDevice,
                        stream);
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
  rc = regroup(st, default_group_bytes());
  if (rc != LBM_OK) {
    free_state(st);
    return rc;
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

extern "C" int lbm_batch_groups(lbm_state* st, int64_t bytes, int32_t* n_groups_out) {
  clear_error();
  if (!valid_batch(st)) return fail(LBM_EINVAL, "not a batched state");
  const int rc = regroup(st, bytes < 0 ? default_group_bytes() : bytes);
  if (rc != LBM_OK) return rc;
  if (n_groups_out) *n_groups_out = (int32_t)st->batch->group_cell0.size();
  return LBM_OK;
}

extern "C" int lbm_batch_resident(lbm_state* st, int32_t mode, int32_t* n_groups_out,
                                  int64_t* cells_out) {
  clear_error();
  if (!valid_batch(st)) return fail(LBM_EINVAL, "not a batched state");
  if (mode != 0 && mode != 1 && mode != -1) return fail(LBM_EINVAL, "mode %d not in {0, 1, -1}", mode);
  Batch* b = st->batch;
  if (mode != 0) {
    const int rc = dispatch_setup_resident(st->precision, st);
    if (rc != LBM_OK) return rc;
  }
  const int saved = b->resident;
  b->resident = mode;
  const int rc = regroup(st, b->group_bytes);
  if (rc != LBM_OK) {
    b->resident = saved;
    return rc;
  }
  if (n_groups_out) *n_groups_out = (int32_t)b->group_cell0.size();
  if (cells_out) *cells_out = mode != 0 ? b->res_cells : 0;
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
