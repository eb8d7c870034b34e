// Assembly of the sparse representation on the GPU (Sec. 2-3):
//   numbering scheme I(x,y,z) -> contiguous index I_c (rank of the fluid
//   cells in key order, solids dropped) -> pull adjacency with implicit
//   bounce back.
//
// The paper removes the gaps of the index with distributed run descriptors
// merged up an octree of MPI ranks (Sec. 3, "In- and outcells",
// "Contiguous index generation").  On one GPU the same result is a stream
// compaction in key order.  Instead of sorting keys, the kernels walk the
// key space itself: key k is inverted to its cell (every scheme here is a
// bijection onto a superset of the box), so a tile of consecutive keys is a
// contiguous run of the final order, and ranks come from a tile count, a
// scan of the counts and an in-tile ballot scan.  No key array is stored.
#include <cstdio>

#include "lbm_internal.cuh"

namespace lbm {

namespace {

constexpr int kTileThreads = 256;
constexpr int kTileRounds = 16;
constexpr uint64_t kTileKeys = (uint64_t)kTileThreads * kTileRounds;

__global__ void keys_kernel(KeySpace ks, uint64_t* keys, int64_t box) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= box) return;
  const int64_t x = c % ks.nx, y = (c / ks.nx) % ks.ny, z = c / (ks.nx * ks.ny);
  keys[c] = key_of(ks, x, y, z);
}

// Pass 1: number of fluid cells in each tile of kTileKeys consecutive keys;
// flags other than 0/1 raise *bad.
__global__ void __launch_bounds__(kTileThreads)
    tile_count_kernel(KeySpace ks, const uint8_t* __restrict__ flags, uint32_t* counts,
                      int* bad) {
  const uint64_t base = (uint64_t)blockIdx.x * kTileKeys;
  uint32_t mine = 0;
  for (int r = 0; r < kTileRounds; ++r) {
    const uint64_t k = base + (uint64_t)r * kTileThreads + threadIdx.x;
    int64_t x, y, z;
    if (cell_of(ks, k, x, y, z)) {
      const uint8_t f = flags[x + ks.nx * (y + ks.ny * z)];
      if (f > 1) atomicOr(bad, 1);
      mine += f == 0;
    }
  }
  // block sum in a fixed order
  __shared__ uint32_t warp_sum[kTileThreads / 32];
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    for (int w = 0; w < kTileThreads / 32; ++w) s += warp_sum[w];
    counts[blockIdx.x] = s;
  }
}

// Pass 2: exclusive scan of the tile counts by one block; total -> *total.
__global__ void __launch_bounds__(1024)
    tile_scan_kernel(const uint32_t* __restrict__ counts, int64_t ntiles, int64_t* offsets,
                     int64_t* total) {
  __shared__ int64_t s[1024];
  const int t = threadIdx.x;
  const int64_t chunk = (ntiles + 1023) / 1024;
  const int64_t b = (int64_t)t * chunk;
  const int64_t e = b + chunk < ntiles ? b + chunk : ntiles;
  int64_t mine = 0;
  for (int64_t i = b; i < e; ++i) mine += counts[i];
  s[t] = mine;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int64_t v = t >= off ? s[t - off] : 0;
    __syncthreads();
    s[t] += v;
    __syncthreads();
  }
  int64_t run = s[t] - mine;
  for (int64_t i = b; i < e; ++i) {
    offsets[i] = run;
    run += counts[i];
  }
  if (t == 1023) *total = s[1023];
}

// Pass 3: walk each tile again in key order and scatter: cells[rank] = box
// index, inv[box index] = rank (or -1 for a solid cell).
__global__ void __launch_bounds__(kTileThreads)
    tile_scatter_kernel(KeySpace ks, const uint8_t* __restrict__ flags,
                        const int64_t* __restrict__ offsets, int32_t* cells, int32_t* inv) {
  __shared__ uint32_t warp_cnt[kTileThreads / 32];
  const uint64_t base = (uint64_t)blockIdx.x * kTileKeys;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t run = offsets[blockIdx.x];
  for (int r = 0; r < kTileRounds; ++r) {
    const uint64_t k = base + (uint64_t)r * kTileThreads + threadIdx.x;
    int64_t x, y, z, c = -1;
    bool fluid = false;
    if (cell_of(ks, k, x, y, z)) {
      c = x + ks.nx * (y + ks.ny * z);
      fluid = flags[c] == 0;
    }
    const uint32_t ballot = __ballot_sync(0xffffffffu, fluid);
    if (lane == 0) warp_cnt[warp] = __popc(ballot);
    __syncthreads();
    int64_t before = 0, total = 0;
    for (int w = 0; w < kTileThreads / 32; ++w) {
      before += w < warp ? warp_cnt[w] : 0;
      total += warp_cnt[w];
    }
    if (c >= 0) {
      if (fluid) {
        const int64_t rank = run + before + __popc(ballot & ((1u << lane) - 1u));
        cells[rank] = (int32_t)c;
        inv[c] = (int32_t)rank;
      } else {
        inv[c] = -1;
      }
    }
    run += total;
    __syncthreads();
  }
}

// ---- lexicographic order: the key is the box index --------------------------
// A tile is then kTileKeys consecutive flag bytes, and thread t takes the
// 16 at tile + 16 t with one 16-byte load (flags 16-byte aligned; the last,
// partial chunk of the box byte by byte).  The generic passes above walk
// their 16 keys one by one and were bound by those dependent rounds.
static_assert(kTileKeys == 16 * kTileThreads, "16 keys per thread");

// The 16 flags of thread t's chunk (1 past the box) and how many are inside.
__device__ __forceinline__ int lex_chunk(const uint8_t* __restrict__ flags, int64_t box,
                                         int64_t k0, uint32_t w[4]) {
  if (k0 + 16 <= box) {
    const uint4 v = *reinterpret_cast<const uint4*>(flags + k0);
    w[0] = v.x;
    w[1] = v.y;
    w[2] = v.z;
    w[3] = v.w;
    return 16;
  }
  const int valid = k0 < box ? (int)(box - k0) : 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) w[j] = 0x01010101u;
  for (int b = 0; b < valid; ++b)
    w[b >> 2] = (w[b >> 2] & ~(0xffu << (8 * (b & 3)))) | ((uint32_t)flags[k0 + b] << (8 * (b & 3)));
  return valid;
}

// Pass 1 in lexicographic order (as tile_count_kernel).
__global__ void __launch_bounds__(kTileThreads)
    tile_count_lex_kernel(const uint8_t* __restrict__ flags, int64_t box, uint32_t* counts,
                          int* bad) {
  uint32_t w[4];
  lex_chunk(flags, box, (int64_t)blockIdx.x * kTileKeys + 16 * (int64_t)threadIdx.x, w);
  uint32_t mine = 0;
  bool any_bad = false;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    any_bad |= (w[j] & 0xfefefefeu) != 0;   // a byte other than 0 or 1
    mine += 4u - (uint32_t)__popc(w[j]);     // bytes 0/1: popc counts the solid ones
  }
  if (any_bad) atomicOr(bad, 1);
  __shared__ uint32_t warp_sum[kTileThreads / 32];
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    for (int wv = 0; wv < kTileThreads / 32; ++wv) s += warp_sum[wv];
    counts[blockIdx.x] = s;
  }
}

// Pass 3 in lexicographic order (as tile_scatter_kernel): each thread's
// fluid cells take consecutive ranks after those of the threads before it
// (a block scan of the per-thread counts); inv is written 16 ints at a time.
__global__ void __launch_bounds__(kTileThreads)
    tile_scatter_lex_kernel(const uint8_t* __restrict__ flags, int64_t box,
                            const int64_t* __restrict__ offsets, int32_t* cells, int32_t* inv) {
  __shared__ uint32_t warp_tot[kTileThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t k0 = (int64_t)blockIdx.x * kTileKeys + 16 * (int64_t)threadIdx.x;
  uint32_t w[4];
  const int valid = lex_chunk(flags, box, k0, w);
  uint32_t mine = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) mine += 4u - (uint32_t)__popc(w[j]);
  // inclusive scan within the warp, then over the warps in order
  uint32_t incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  uint32_t before = incl - mine;
  for (int wv = 0; wv < warp; ++wv) before += warp_tot[wv];
  int64_t rank = offsets[blockIdx.x] + before;
  int32_t out[16];
#pragma unroll
  for (int b = 0; b < 16; ++b) {
    const bool fluid = ((w[b >> 2] >> (8 * (b & 3))) & 0xffu) == 0;
    out[b] = fluid ? (int32_t)rank : -1;
    if (fluid) {
      cells[rank] = (int32_t)(k0 + b);
      ++rank;
    }
  }
  if (valid == 16) {
    int4* o = reinterpret_cast<int4*>(inv + k0);
#pragma unroll
    for (int j = 0; j < 4; ++j) o[j] = make_int4(out[4 * j], out[4 * j + 1], out[4 * j + 2], out[4 * j + 3]);
  } else {
    for (int b = 0; b < valid; ++b) inv[k0 + b] = out[b];
  }
}

// Pull adjacency (Sec. 2): source slot of direction i for fluid cell n, in
// rows of ld >= n entries naming slot r ld + m (ld = n: the public layout).
__global__ void adjacency_kernel(int32_t nx, int32_t ny, int32_t nz, uint32_t periodic,
                                 const int32_t* __restrict__ cells,
                                 const int32_t* __restrict__ inv, int32_t* __restrict__ adj,
                                 int32_t n, int32_t ld) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t c = cells[i];
  const int32_t x = c % nx, y = (c / nx) % ny, z = c / (nx * ny);
#pragma unroll
  for (int q = 1; q < 19; ++q) {
    int32_t sx = x - cx(q), sy = y - cy(q), sz = z - cz(q);
    bool inside = true;
    if (sx < 0 || sx >= nx) {
      if (periodic & 1u) sx = sx < 0 ? sx + nx : sx - nx; else inside = false;
    }
    if (sy < 0 || sy >= ny) {
      if (periodic & 2u) sy = sy < 0 ? sy + ny : sy - ny; else inside = false;
    }
    if (sz < 0 || sz >= nz) {
      if (periodic & 4u) sz = sz < 0 ? sz + nz : sz - nz; else inside = false;
    }
    int32_t m = -1;
    if (inside) m = inv[sx + nx * (sy + ny * sz)];
    adj[(q - 1) * ld + i] = m >= 0 ? q * ld + m : opp(q) * ld + i;
  }
}

// The public links (rows of n, slot q n + m) from links in rows of ld > n
// (slot r ld + m); grid (cells, 18 rows).
__global__ void public_links_kernel(const int32_t* __restrict__ adj_ld, int32_t ld, int32_t n,
                                    int32_t* __restrict__ adj) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const int32_t q = (int32_t)blockIdx.y;
  if (i >= n) return;
  const uint32_t s = (uint32_t)adj_ld[q * ld + i];
  const uint32_t r = s / (uint32_t)ld;
  adj[q * n + i] = (int32_t)(r * (uint32_t)n + (s - r * (uint32_t)ld));
}

}  // namespace

int make_key_space(const int32_t dims[3], const lbm_ordering& ord, bool clamp_blocks,
                   KeySpace* ks) {
  if (!dims) return fail(LBM_EINVAL, "dims is NULL");
  for (int k = 0; k < 3; ++k)
    if (dims[k] < 1) return fail(LBM_EINVAL, "dims[%d] = %d must be >= 1", k, dims[k]);
  const int64_t box = (int64_t)dims[0] * dims[1] * dims[2];
  if (box >= (int64_t)1 << 31)
    return fail(LBM_EOVERFLOW, "box of %lld cells: the bounding box must stay below 2^31 cells",
                (long long)box);
  if (ord.kind < LBM_ORDER_LEX || ord.kind > LBM_ORDER_HILBERT)
    return fail(LBM_EINVAL, "unknown ordering kind %d", ord.kind);
  if (ord.periodic > 7u) return fail(LBM_EINVAL, "periodic mask %u has bits beyond 0..2", ord.periodic);
  KeySpace s{};
  s.kind = ord.kind;
  s.nx = dims[0];
  s.ny = dims[1];
  s.nz = dims[2];
  s.bx = s.by = s.bz = 1;
  if (ord.kind == LBM_ORDER_BLOCKED) {
    for (int k = 0; k < 3; ++k)
      if (ord.block[k] < 1) return fail(LBM_EINVAL, "block[%d] = %d must be >= 1", k, ord.block[k]);
    s.bx = ord.block[0];
    s.by = ord.block[1];
    s.bz = ord.block[2];
    // A block wider than the box along an axis visits that axis
    // lexicographically either way; clamping leaves the order unchanged but
    // keeps the walked key space small.  Keys handed out keep the literal
    // blocking factors.
    if (clamp_blocks) {
      if (s.bx > s.nx) s.bx = s.nx;
      if (s.by > s.ny) s.by = s.ny;
      if (s.bz > s.nz) s.bz = s.nz;
    }
    if ((double)s.bx * (double)s.by * (double)s.bz >= 9.0e18)
      return fail(LBM_EOVERFLOW, "blocking factors too large");
  }
  s.nbx = (s.nx + s.bx - 1) / s.bx;
  s.nby = (s.ny + s.by - 1) / s.by;
  s.nbz = (s.nz + s.bz - 1) / s.bz;
  s.hbits = 1;
  while ((1LL << s.hbits) < s.nx || (1LL << s.hbits) < s.ny || (1LL << s.hbits) < s.nz) ++s.hbits;
  if (ord.kind == LBM_ORDER_BLOCKED) {
    s.size = (uint64_t)(s.nbx * s.nby * s.nbz) * (uint64_t)(s.bx * s.by * s.bz);
  } else if (ord.kind == LBM_ORDER_HILBERT) {
    // the Hilbert curve wanders through the whole enclosing cube
    s.size = 1ull << (3 * s.hbits);
  } else {
    s.size = ~0ull;
    // lexicographic and Z-curve keys are monotone in each coordinate: the
    // far corner holds the largest key
    s.size = key_of(s, s.nx - 1, s.ny - 1, s.nz - 1) + 1;
  }
  *ks = s;
  return LBM_OK;
}

int public_links(const lbm_sparse* sp_c, const int32_t** out) {
  // logically const: the public links are a cached view of adj_ld
  lbm_sparse* sp = const_cast<lbm_sparse*>(sp_c);
  if (!sp->adj) {
    const cudaStream_t stream = sp->stream;
    int32_t* adj = nullptr;
    if (dev_alloc(&adj, sizeof(int32_t) * 18 * (size_t)(sp->n > 0 ? sp->n : 1), stream, true) !=
        cudaSuccess) {
      cudaGetLastError();
      return fail(LBM_ENOMEM, "public adjacency allocation failed (%lld fluid cells)",
                  (long long)sp->n);
    }
    if (sp->n > 0)
      public_links_kernel<<<dim3((unsigned)((sp->n + 255) / 256), 18), 256, 0, stream>>>(
          sp->adj_ld, (int32_t)sp->ld, (int32_t)sp->n, adj);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
      dev_free(adj, stream, true);
      cudaStreamSynchronize(stream);
      return cuda_fail(e, "public adjacency");
    }
    sp->adj = adj;
  }
  if (out) *out = sp->adj;
  return LBM_OK;
}

}  // namespace lbm

using namespace lbm;

extern "C" int lbm_ordering_keys(const int32_t dims[3], lbm_ordering ord, uint64_t* keys_dev,
                                 void* stream) {
  clear_error();
  KeySpace ks;
  int rc = make_key_space(dims, ord, false, &ks);
  if (rc) return rc;
  if (!keys_dev) return fail(LBM_EINVAL, "keys_dev is NULL");
  const int64_t box = ks.nx * ks.ny * ks.nz;
  const int threads = 256;
  keys_kernel<<<(unsigned)((box + threads - 1) / threads), threads, 0, (cudaStream_t)stream>>>(
      ks, keys_dev, box);
  LBM_CUDA_TRY(cudaGetLastError());
  return LBM_OK;
}

extern "C" int lbm_build_sparse(const uint8_t* flags, const int32_t dims[3], lbm_ordering ord,
                                void* stream_v, lbm_sparse** out) {
  clear_error();
  if (!out) return fail(LBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!flags) return fail(LBM_EINVAL, "flags is NULL");
  KeySpace ks;
  int rc = make_key_space(dims, ord, true, &ks);
  if (rc) return rc;
  cudaStream_t stream = (cudaStream_t)stream_v;
  const int64_t box = ks.nx * ks.ny * ks.nz;
  const int64_t ntiles = (int64_t)((ks.size + kTileKeys - 1) / kTileKeys);
  if (ntiles >= (int64_t)1 << 31) return fail(LBM_EOVERFLOW, "key space too large");
  // host flags (pinned or pageable) are copied to the device first
  cudaPointerAttributes attr{};
  const cudaError_t pe = cudaPointerGetAttributes(&attr, flags);
  if (pe != cudaSuccess) return cuda_fail(pe, "cudaPointerGetAttributes(flags)");
  const bool on_host = attr.type == cudaMemoryTypeHost || attr.type == cudaMemoryTypeUnregistered;

  // scratch: tile counts, tile offsets, total, error flag
  uint32_t* counts = nullptr;
  int64_t* offsets = nullptr;
  int64_t* scal = nullptr;  // [0] total, [1] bad-flag word
  uint8_t* flags_copy = nullptr;
  lbm_sparse* sp = new lbm_sparse{};
  sp->magic = kMagicSparse;
  for (int k = 0; k < 3; ++k) sp->dims[k] = dims[k];
  sp->ord = ord;
  sp->stream = stream;
  auto release = [&](void* p) { dev_free(p, stream, true); };
  auto cleanup = [&](int status) {
    release(counts);
    release(offsets);
    release(scal);
    release(flags_copy);
    if (status != LBM_OK) {
      release(sp->cells);
      release(sp->inv);
      release(sp->adj);
      release(sp->adj_ld);
      delete sp;
    }
    cudaStreamSynchronize(stream);
    return status;
  };
  if (dev_alloc(&counts, sizeof(uint32_t) * ntiles, stream, true) != cudaSuccess ||
      dev_alloc(&offsets, sizeof(int64_t) * ntiles, stream, true) != cudaSuccess ||
      dev_alloc(&scal, sizeof(int64_t) * 2, stream, true) != cudaSuccess ||
      dev_alloc(&sp->inv, sizeof(int32_t) * box, stream, true) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(fail(LBM_ENOMEM, "device allocation failed (box %lld cells)", (long long)box));
  }
  if (cudaMemsetAsync(scal, 0, sizeof(int64_t) * 2, stream) != cudaSuccess)
    return cleanup(cuda_fail(cudaGetLastError(), "cudaMemsetAsync"));
  const uint8_t* flags_dev = flags;
  if (on_host) {
    if (dev_alloc(&flags_copy, (size_t)box, stream, true) != cudaSuccess) {
      cudaGetLastError();
      return cleanup(fail(LBM_ENOMEM, "device copy of the host flags (%lld bytes) failed",
                          (long long)box));
    }
    const cudaError_t ce =
        cudaMemcpyAsync(flags_copy, flags, (size_t)box, cudaMemcpyHostToDevice, stream);
    if (ce != cudaSuccess) return cleanup(cuda_fail(ce, "cudaMemcpyAsync(flags)"));
    flags_dev = flags_copy;
  }
  // lexicographic order with 16-byte aligned flags takes the vector passes
  const bool lex_vec = ks.kind == LBM_ORDER_LEX && reinterpret_cast<uintptr_t>(flags_dev) % 16 == 0;
  if (lex_vec)
    tile_count_lex_kernel<<<(unsigned)ntiles, kTileThreads, 0, stream>>>(flags_dev, box, counts,
                                                                        (int*)(scal + 1));
  else
    tile_count_kernel<<<(unsigned)ntiles, kTileThreads, 0, stream>>>(ks, flags_dev, counts,
                                                                    (int*)(scal + 1));
  tile_scan_kernel<<<1, 1024, 0, stream>>>(counts, ntiles, offsets, scal);
  int64_t host_scal[2] = {0, 0};
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_scal, scal, sizeof(host_scal), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "sparse assembly: tile count/scan"));
  if (host_scal[1] != 0) return cleanup(fail(LBM_EFLAGS, "flags must be 0 (fluid) or 1 (solid)"));
  const int64_t n = host_scal[0];
  const int64_t ld = row_stride(n);
  if (19 * ld >= ((int64_t)1 << 31))
    return cleanup(fail(LBM_EOVERFLOW,
                        "%lld fluid cells: 19*L PDF slots (rows of L = %lld, N rounded up to 64) "
                        "exceed the int32 adjacency range",
                        (long long)n, (long long)ld));
  sp->n = n;
  sp->ld = ld;
  const size_t nn = (size_t)(n > 0 ? n : 1);
  // the links in the state layout; they are the public ones when ld == n
  int32_t** links = ld == n ? &sp->adj : &sp->adj_ld;
  if (dev_alloc(&sp->cells, sizeof(int32_t) * nn, stream, true) != cudaSuccess ||
      dev_alloc(links, sizeof(int32_t) * 18 * (size_t)(ld > 0 ? ld : 1), stream, true) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(fail(LBM_ENOMEM, "device allocation failed (%lld fluid cells)", (long long)n));
  }
  if (lex_vec)
    tile_scatter_lex_kernel<<<(unsigned)ntiles, kTileThreads, 0, stream>>>(
        flags_dev, box, offsets, sp->cells, sp->inv);
  else
    tile_scatter_kernel<<<(unsigned)ntiles, kTileThreads, 0, stream>>>(ks, flags_dev, offsets,
                                                                      sp->cells, sp->inv);
  if (n > 0) {
    const int threads = 256;
    adjacency_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, stream>>>(
        dims[0], dims[1], dims[2], ord.periodic, sp->cells, sp->inv, *links, (int32_t)n,
        (int32_t)ld);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "sparse assembly: scatter/adjacency"));
  *out = sp;
  return cleanup(LBM_OK);
}

extern "C" int lbm_sparse_info(const lbm_sparse* sp, int64_t* n_fluid, const int32_t** cells_dev,
                               const int32_t** adj_dev, const int32_t** inv_dev) {
  clear_error();
  if (!sp || sp->magic != kMagicSparse) return fail(LBM_EINVAL, "not a sparse handle");
  if (n_fluid) *n_fluid = sp->n;
  if (cells_dev) *cells_dev = sp->cells;
  if (adj_dev) {
    const int rc = public_links(sp, adj_dev);
    if (rc != LBM_OK) return rc;
  }
  if (inv_dev) *inv_dev = sp->inv;
  return LBM_OK;
}
