// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

#include "lbm.h"

namespace lbm {

constexpr uint32_t kMagicSparse = 0x4C53504Bu;
constexpr uint32_t kMagicState = 0x4C535354u;
constexpr uint32_t kMagicAdjoint = 0x4C53414Du;
constexpr int kSweepThreads = 256;
constexpr int kWarpsPerBlock = kSweepThreads / 32;

// Records a message for lbm_last_error() and returns `status`.
int fail(int status, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
void clear_error();
// Device memory of every handle: the caller's allocator when one is set
// (lbm_set_allocator), else cudaMallocAsync / cudaFreeAsync on `stream`
// (ordered) or cudaMalloc / cudaFree.  An unordered free expects the work
// on the block to have finished.
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t stream, bool ordered);
void dev_free(void* p, cudaStream_t stream, bool ordered);
template <class T>
cudaError_t dev_alloc(T** p, size_t bytes, cudaStream_t stream, bool ordered) {
  return dev_alloc(reinterpret_cast<void**>(p), bytes, stream, ordered);
}

#define LBM_CUDA_TRY(expr)                                         \
  do {                                                             \
    cudaError_t lbm_err_ = (expr);                                 \
    if (lbm_err_ != cudaSuccess) return ::lbm::cuda_fail(lbm_err_, #expr); \
  } while (0)

// D3Q19 velocity set: 0 rest; 1..6 axis; 7..18 face diagonals; the odd
// member of each (odd, odd+1) pair is +c, the even one -c.
__host__ __device__ __forceinline__ int cx(int q) {
  switch (q) {
    case 1: case 7: case 9: case 11: case 13: return 1;
    case 2: case 8: case 10: case 12: case 14: return -1;
    default: return 0;
  }
}
__host__ __device__ __forceinline__ int cy(int q) {
  switch (q) {
    case 3: case 7: case 10: case 15: case 17: return 1;
    case 4: case 8: case 9: case 16: case 18: return -1;
    default: return 0;
  }
}
__host__ __device__ __forceinline__ int cz(int q) {
  switch (q) {
    case 5: case 11: case 14: case 15: case 18: return 1;
    case 6: case 12: case 13: case 16: case 17: return -1;
    default: return 0;
  }
}
__host__ __device__ __forceinline__ int opp(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }
__host__ __device__ __forceinline__ double weight(int q) {
  return q == 0 ? 1.0 / 3.0 : (q <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// Numbering-scheme key of box cell (x, y, z) (Sec. 3 "Numbering scheme").
struct KeySpace {
  int32_t kind;
  int64_t nx, ny, nz;
  int64_t bx, by, bz, nbx, nby, nbz;
  int32_t hbits;  // Hilbert: bits per axis of the enclosing cube
  uint64_t size;  // every key is < size
};

// Hilbert curve on a 2^bits cube (Skilling, "Programming the Hilbert
// curve", AIP Conf. Proc. 707, 2004): the coordinates become a "transposed"
// index by undoing, from the top level down, the rotations and reflections
// of the recursive construction and then Gray-encoding; the key reads the
// transposed index level by level in the order x, y, z.
__host__ __device__ inline uint64_t hilbert_encode(int bits, uint64_t x, uint64_t y, uint64_t z) {
  uint64_t X[3] = {x, y, z};
  const uint64_t top = 1ull << (bits - 1);
  for (uint64_t q = top; q > 1; q >>= 1) {
    const uint64_t p = q - 1;
    for (int i = 0; i < 3; ++i) {
      if (X[i] & q) {
        X[0] ^= p;
      } else {
        const uint64_t t = (X[0] ^ X[i]) & p;
        X[0] ^= t;
        X[i] ^= t;
      }
    }
  }
  X[1] ^= X[0];
  X[2] ^= X[1];
  uint64_t t = 0;
  for (uint64_t q = top; q > 1; q >>= 1)
    if (X[2] & q) t ^= q - 1;
  X[0] ^= t;
  X[1] ^= t;
  X[2] ^= t;
  uint64_t key = 0;
  for (int lvl = bits - 1; lvl >= 0; --lvl)
    key = (key << 3) | (((X[0] >> lvl) & 1ull) << 2) | (((X[1] >> lvl) & 1ull) << 1) |
          ((X[2] >> lvl) & 1ull);
  return key;
}

// Inverse of hilbert_encode: Gray-decode the transposed index, then redo
// the level transformations from the bottom up.
__host__ __device__ inline void hilbert_decode(int bits, uint64_t key, uint64_t& x, uint64_t& y,
                                               uint64_t& z) {
  uint64_t X[3] = {0, 0, 0};
  for (int lvl = 0; lvl < bits; ++lvl) {
    X[0] |= ((key >> (3 * lvl + 2)) & 1ull) << lvl;
    X[1] |= ((key >> (3 * lvl + 1)) & 1ull) << lvl;
    X[2] |= ((key >> (3 * lvl)) & 1ull) << lvl;
  }
  const uint64_t t0 = X[2] >> 1;
  X[2] ^= X[1];
  X[1] ^= X[0];
  X[0] ^= t0;
  for (uint64_t q = 2; q != (1ull << bits); q <<= 1) {
    const uint64_t p = q - 1;
    for (int i = 2; i >= 0; --i) {
      if (X[i] & q) {
        X[0] ^= p;
      } else {
        const uint64_t t = (X[0] ^ X[i]) & p;
        X[0] ^= t;
        X[i] ^= t;
      }
    }
  }
  x = X[0];
  y = X[1];
  z = X[2];
}

__host__ __device__ inline uint64_t key_of(const KeySpace& ks, int64_t x, int64_t y, int64_t z) {
  switch (ks.kind) {
    case LBM_ORDER_HILBERT:
      return hilbert_encode(ks.hbits, (uint64_t)x, (uint64_t)y, (uint64_t)z);
    case LBM_ORDER_LEX:
      return (uint64_t)(x + ks.nx * (y + ks.ny * z));
    case LBM_ORDER_BLOCKED: {
      const int64_t blk = x / ks.bx + ks.nbx * (y / ks.by + ks.nby * (z / ks.bz));
      const int64_t loc = x % ks.bx + ks.bx * (y % ks.by + ks.by * (z % ks.bz));
      return (uint64_t)(blk * (ks.bx * ks.by * ks.bz) + loc);
    }
    case LBM_ORDER_MORTON1: {
      uint64_t k = 0;
      for (int b = 0; b < 21; ++b) {
        k |= (((uint64_t)x >> b) & 1u) << (3 * b);
        k |= (((uint64_t)y >> b) & 1u) << (3 * b + 1);
        k |= (((uint64_t)z >> b) & 1u) << (3 * b + 2);
      }
      return k;
    }
    default: {  // LBM_ORDER_MORTON2
      uint64_t k = 0;
      for (int g = 0; g < 10; ++g) {
        k |= (((uint64_t)x >> (2 * g)) & 3u) << (6 * g);
        k |= (((uint64_t)y >> (2 * g)) & 3u) << (6 * g + 2);
        k |= (((uint64_t)z >> (2 * g)) & 3u) << (6 * g + 4);
      }
      return k;
    }
  }
}

// Inverse of key_of: the box cell of key k, or false if k names no cell of
// the box (the key space of blocked and Morton orders has gaps).
__host__ __device__ inline bool cell_of(const KeySpace& ks, uint64_t k, int64_t& x, int64_t& y,
                                        int64_t& z) {
  // Keys, block sizes and block counts below 2^32 (every lexicographic key
  // of a box below 2^31 cells) take 32-bit division, several times cheaper
  // on the GPU than 64-bit division; the results are the same.
  constexpr uint64_t k32 = 1ull << 32;
  switch (ks.kind) {
    case LBM_ORDER_LEX: {
      if (k < k32) {
        const uint32_t kk = (uint32_t)k, nx = (uint32_t)ks.nx, ny = (uint32_t)ks.ny;
        const uint32_t t = kk / nx;
        x = (int64_t)(kk - t * nx);
        y = (int64_t)(t % ny);
        z = (int64_t)(t / ny);
        break;
      }
      x = (int64_t)(k % (uint64_t)ks.nx);
      const uint64_t t = k / (uint64_t)ks.nx;
      y = (int64_t)(t % (uint64_t)ks.ny);
      z = (int64_t)(t / (uint64_t)ks.ny);
      break;
    }
    case LBM_ORDER_BLOCKED: {
      const uint64_t bsz = (uint64_t)(ks.bx * ks.by * ks.bz);
      if (k < k32 && bsz < k32 && (uint64_t)(ks.bx * ks.by) < k32 &&
          (uint64_t)(ks.nbx * ks.nby) < k32) {
        const uint32_t kk = (uint32_t)k, b = (uint32_t)bsz, bx = (uint32_t)ks.bx,
                       by = (uint32_t)ks.by, nbx = (uint32_t)ks.nbx, nby = (uint32_t)ks.nby;
        const uint32_t blk = kk / b, loc = kk - blk * b;
        const uint32_t lyz = loc / bx, biyz = blk / nbx;
        x = (int64_t)(blk - biyz * nbx) * ks.bx + (int64_t)(loc - lyz * bx);
        y = (int64_t)(biyz % nby) * ks.by + (int64_t)(lyz % by);
        z = (int64_t)(biyz / nby) * ks.bz + (int64_t)(loc / (bx * by));
        break;
      }
      const uint64_t blk = k / bsz, loc = k % bsz;
      const int64_t lx = (int64_t)(loc % (uint64_t)ks.bx);
      const int64_t ly = (int64_t)((loc / (uint64_t)ks.bx) % (uint64_t)ks.by);
      const int64_t lz = (int64_t)(loc / (uint64_t)(ks.bx * ks.by));
      const int64_t ix = (int64_t)(blk % (uint64_t)ks.nbx);
      const int64_t iy = (int64_t)((blk / (uint64_t)ks.nbx) % (uint64_t)ks.nby);
      const int64_t iz = (int64_t)(blk / (uint64_t)(ks.nbx * ks.nby));
      x = ix * ks.bx + lx;
      y = iy * ks.by + ly;
      z = iz * ks.bz + lz;
      break;
    }
    case LBM_ORDER_HILBERT: {
      uint64_t ux, uy, uz;
      hilbert_decode(ks.hbits, k, ux, uy, uz);
      x = (int64_t)ux;
      y = (int64_t)uy;
      z = (int64_t)uz;
      break;
    }
    case LBM_ORDER_MORTON1: {
      x = y = z = 0;
      for (int b = 0; b < 21; ++b) {
        x |= (int64_t)((k >> (3 * b)) & 1u) << b;
        y |= (int64_t)((k >> (3 * b + 1)) & 1u) << b;
        z |= (int64_t)((k >> (3 * b + 2)) & 1u) << b;
      }
      break;
    }
    default: {
      x = y = z = 0;
      for (int g = 0; g < 10; ++g) {
        x |= (int64_t)((k >> (6 * g)) & 3u) << (2 * g);
        y |= (int64_t)((k >> (6 * g + 2)) & 3u) << (2 * g);
        z |= (int64_t)((k >> (6 * g + 4)) & 3u) << (2 * g);
      }
      break;
    }
  }
  return k < ks.size && x < ks.nx && y < ks.ny && z < ks.nz;
}

// Validates dims/ordering and fills the key space; returns LBM_OK or an error.
// clamp_blocks shrinks blocking factors larger than the box (same order,
// smaller key space) for the assembly walk.
int make_key_space(const int32_t dims[3], const lbm_ordering& ord, bool clamp_blocks,
                   KeySpace* ks);

}  // namespace lbm

struct lbm_sparse {
  uint32_t magic;
  int32_t dims[3];
  lbm_ordering ord;
  int64_t n;
  int32_t* cells;  // [n]
  int32_t* inv;    // [box]
  // [18 * n], source slot q n + m (the layout lbm_sparse_info presents).
  // When ld != n the assembly writes adj_ld only, and adj is derived from
  // it on first request (public_links); null until then.
  int32_t* adj;
  // Row stride of the state arrays: n rounded up to kRowAlign (a batch: its
  // padded total).  adj_ld holds the links in that layout, rows of ld
  // entries naming slot r ld + m; null when ld == n (adj serves).
  int64_t ld;
  int32_t* adj_ld;
  cudaStream_t stream;
};

namespace lbm {
// Every row of a state's PDF grids, and of the links its sweeps read, starts
// on a 128-byte boundary: rows of kRowAlign elements.  On the 1024x256x256
// bed, a list of a multiple of 64 cells (fluid cells made solid) against the
// odd list of the same bed, MFLUP/s: FP16 45,537 / 43,390, FP32 31,502 /
// 30,742, FP64 storage 18,314 / 18,076 (an even list: 45,124 / 31,404 /
// 18,276).  Misaligned rows cost the 2-byte forms their paired 4-byte stores
// on every other row, and every form's warp accesses straddle one more line.
constexpr int64_t kRowAlign = 64;
inline int64_t row_stride(int64_t n) { return (n + kRowAlign - 1) / kRowAlign * kRowAlign; }
// The links the sweeps of a state on sp read: rows of sp->ld entries.
inline const int32_t* state_links(const lbm_sparse* sp) { return sp->adj_ld ? sp->adj_ld : sp->adj; }
// The public links of sp (*out may be null), built from adj_ld on the first
// request and kept (one kernel on sp's stream, which is then synchronised).
int public_links(const lbm_sparse* sp, const int32_t** out);
}  // namespace lbm

namespace lbm {
// Batched state: beds concatenated, each padded to kBatchChunk cells so that
// every tile of every launch configuration lies inside one bed.
constexpr int64_t kBatchChunk = 2048;
static_assert(kBatchChunk % kRowAlign == 0, "a batch's padded rows stay aligned");
struct Batch {
  int32_t n_beds;
  int64_t* h_begin;      // [n_beds] first padded-list index of each bed (host)
  int64_t* h_count;      // [n_beds] fluid cells of each bed (host)
  int64_t* d_begin;      // device copies
  int32_t* d_count;
  int32_t* d_chunk_bed;  // [n_pad / kBatchChunk] bed of each chunk
  void* d_force;         // [n_beds] per-bed force constants (arithmetic type)
  void* h_force;         // pinned staging for d_force
  double* d_red;         // [n_beds][4] per-bed final sums
  double* h_red;         // pinned
  int block, cpt;        // launch configuration of the non-reducing steps
  cudaStream_t capture;  // private stream used to capture graphs
  cudaGraphExec_t graph; // cached K-step graph (or null)
  int32_t g_steps, g_parity, g_block, g_cpt;
  double g_wp, g_wm;
  int use_graph;
  // L2 groups: consecutive beds whose working set (both PDF grids and the
  // adjacency) fits group_bytes.  With more than one group, a call runs all
  // its steps on one group, then on the next, so each group's steps stream
  // from L2 rather than HBM.  group_bytes 0: one group of all beds.
  // Each group's arrays are contiguous: the PDFs of its padded cells
  // [c0, c0 + span) are 19 rows of span at offset 19 c0, its links 18 rows
  // at 18 c0, holding slots local to the group.  One group is the plain
  // [19][N_pad] layout that lbm_state_get/set_pdfs present.
  int64_t group_bytes, g_group_bytes;  // current; the cached graph's
  std::vector<int64_t> group_cell0, group_span;  // padded first cell and length
  int32_t* d_chunk_group;  // [N_pad / kBatchChunk] group of each chunk (null: one group)
  int64_t* d_group_cell0;  // [groups]
  int64_t* d_group_span;   // [groups]
  // Resident steps (lbm_batch_resident): a group of at most res_cells cells
  // takes all but its reducing step in one cooperative launch of one
  // 1024-thread block per SM, each block holding its cells' links (at most
  // res_tile cells) in shared memory; blocks meet at a grid barrier.
  int resident;            // 0 off, 1 on, -1 barrier check (every wait runs out)
  int64_t res_cells, res_tile;
  uint32_t* d_sync;        // [N_pad / kBatchChunk + 1] barrier counter of each group
  int32_t* d_sync_err;     // set by a barrier wait that ran out of time
  int32_t* h_sync_err;     // pinned copy, read after the stream has drained
};

// Single-state step graphs: kGraphSteps non-reducing steps captured once per
// grid parity and replayed by long lbm_step calls.  kGraphSteps is even, so
// a replay leaves the parity where it found it.  A graph is keyed by the
// launch arguments it baked in.
constexpr int32_t kGraphSteps = 128;
struct StepGraph {
  cudaStream_t capture;     // private stream the launches are captured on
  cudaGraphExec_t exec[2];  // per parity of st->cur, or null
  double wp[2], wm[2], F[2][3];
  const void* alpha[2];
};

// Launches a sweep on `stream` in blocks of kSweepThreads.  `chained` means
// the previous launch on the stream is a sweep of the same lbm_step call: the
// launch then allows programmatic stream serialisation, so its blocks can
// start (and load their adjacency entries) while that sweep finishes.  The
// sweep kernels order every other access behind prior_step_done().  Build
// with -DLBM_CHAIN_STEPS=0 to launch every sweep normally.
#ifndef LBM_CHAIN_STEPS
#define LBM_CHAIN_STEPS 1
#endif
template <class... P, class... A>
cudaError_t launch_chained(void (*kernel)(P...), unsigned grid, unsigned block,
                           cudaStream_t stream, bool chained, A... args) {
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr.val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  const bool pdl = LBM_CHAIN_STEPS && chained;
  cfg.attrs = pdl ? &attr : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}
template <class... P, class... A>
cudaError_t launch_sweep(void (*kernel)(P...), unsigned grid, cudaStream_t stream, bool chained,
                         A... args) {
  return launch_chained(kernel, grid, (unsigned)kSweepThreads, stream, chained, args...);
}
}  // namespace lbm

struct lbm_state {
  uint32_t magic;
  const lbm_sparse* sp;
  cudaStream_t stream;   // sp's stream, kept so that releasing the state needs no sp
  int32_t precision;
  int32_t scale_exp;
  void* buf[2];        // PDF grids, 19 rows of sp->ld elements of the storage type (n used)
  int cur;             // index of the grid holding the current PDFs
  void* alpha;         // [n] damping in the arithmetic precision, or nullptr
  int64_t* alpha_fx;   // LBM_F64X with damping: [2][n] alpha 2^63 (-1: the cell takes the
                       // IEEE path) and e 2^63, e = (alpha/2) / (1 + alpha/2)
  double* partials;    // [nblocks * kWarpsPerBlock * 4] FP64 warp sums of the last step,
                       // then [nblocks * 4] room for the group values of lbm_reduce_flux
  int64_t nblocks;
  bool one_wave;       // nblocks <= 4 x SMs: plain FP32/16-bit steps load links first
  double* red_dev;     // [4] final sums
  double* red_host;    // [4] pinned
  int64_t steps;
  double last_force[3];
  double last_wp, last_wm;
  cudaEvent_t done;    // recorded to wait for the stream with a time limit
  cudaEvent_t t0, t1;  // timing events of lbm_step_timed (created on first use)
  lbm::StepGraph* graph;  // cached CUDA graphs of non-reducing steps, or null
  lbm::Batch* batch;   // non-null for a batched state (sp is then owned)
};

namespace lbm {
void free_state(lbm_state* st);
void free_sparse(lbm_sparse* sp);
void free_adjoint(lbm_adjoint* ad);
size_t storage_bytes(int prec);   // bytes per stored PDF of a precision form
size_t compute_bytes(int prec);   // bytes of the arithmetic type of a form
bool is_shifted(int prec);        // stores f - w_q rather than f
// Fixed-point FP64-storage sweep (sweep_fx.cu), undamped: n_steps launches
// on `stream`; the last one writes the warp sums when reduce_last is set.
// One fixed-point step of FP64-storage state st (its damping) from src to
// dst, arrays of rows of stride ld read through links adj (not reducing),
// queued on `stream`.
int launch_fx_step(const lbm_state* st, const double* src, double* dst, const int32_t* adj,
                   int32_t ld, double wp, double wm, const double F[3], cudaStream_t stream,
                   bool chained);
// Fills the fixed-point damping rows (alpha_fx) of an FP64-storage state
// from FP64 alpha on the device.
int set_alpha_fx(lbm_state* st, const double* alpha_dev);
int launch_steps_fx(lbm_state* st, int32_t n_steps, double wp, double wm, const double F[3],
                    cudaStream_t stream, bool reduce_last);
bool valid_state(const lbm_state* st);
// Records `ev` on `stream` and polls it with a wall-clock limit (<= 0: the
// library default); LBM_ETIMEOUT if the work is still running then.
int wait_event(cudaEvent_t ev, cudaStream_t stream, double timeout_s);
// Batched-state hooks (batch.cu).
int batch_steps(lbm_state* st, int32_t n_steps, double wp, double wm, const double* forces);
int batch_reduce(lbm_state* st, int32_t axis, double* mass_out, double* flux_out);
void free_batch(lbm_state* st);
// True if a batched state's arrays are in a layout of several L2 groups.
bool batch_grouped(const lbm_state* st);
// Copies the PDFs of buf[from] into buf[to], from the group layout into the
// plain [19][N_pad] one (to_plain) or back.
int batch_relayout_pdfs(const lbm_state* st, int from, int to, bool to_plain);
}  // namespace lbm
