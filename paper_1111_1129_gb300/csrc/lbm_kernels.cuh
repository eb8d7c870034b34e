// Device code shared by the sweep and the adjoint: storage forms, per-launch
// coefficients, the pull gather, the TRT collision, the sweep kernel and the
// fixed-order reductions.  Included by sweep.cu and adjoint.cu; everything
// here has internal linkage.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>

#include "lbm_internal.cuh"

namespace lbm {
namespace {

template <int PREC>
struct Form;
template <>
struct Form<LBM_F64> {
  using S = double;
  using C = double;
  static constexpr bool kShifted = false;
};
template <>
struct Form<LBM_F64X> {  // FP64 storage; the sweep itself runs in fixed point
  using S = double;
  using C = double;
  static constexpr bool kShifted = false;
};
template <>
struct Form<LBM_F32> {
  using S = float;
  using C = float;
  static constexpr bool kShifted = false;
};
template <>
struct Form<LBM_F32S> {
  using S = float;
  using C = float;
  static constexpr bool kShifted = true;
};
template <>
struct Form<LBM_F16S> {
  using S = __half;
  using C = float;
  static constexpr bool kShifted = true;
};
template <>
struct Form<LBM_BF16S> {
  using S = __nv_bfloat16;
  using C = float;
  static constexpr bool kShifted = true;
};

// Per-launch coefficients in the arithmetic precision C.
template <class C>
struct Coef {
  C hp, hm;        // (1 - w+)/2, (1 - w-)/2
  C one_m_wp;      // 1 - w+
  C w0p, w1p;      // w+ / 3, w+ / 18
  C k1, k2;        // 4.5 w+ / 18, 4.5 w+ / 36
  C a1, b1;        // 3 w- / 18, 3 (1 - w-/2) / 18
  C F[3], hF[3];   // F, F / 2
  C bF1[3];        // b1 F (used without damping)
  C scale, inv_scale;
};

template <class C>
Coef<C> make_coef(double wp, double wm, const double F[3], int scale_exp) {
  Coef<C> k;
  k.hp = (C)(0.5 * (1.0 - wp));
  k.hm = (C)(0.5 * (1.0 - wm));
  k.one_m_wp = (C)(1.0 - wp);
  k.w0p = (C)(wp / 3.0);
  k.w1p = (C)(wp / 18.0);
  k.k1 = (C)(4.5 * wp / 18.0);
  k.k2 = (C)(4.5 * wp / 36.0);
  k.a1 = (C)(3.0 * wm / 18.0);
  const double b1 = 3.0 * (1.0 - 0.5 * wm) / 18.0;
  k.b1 = (C)b1;
  for (int d = 0; d < 3; ++d) {
    k.F[d] = (C)F[d];
    k.hF[d] = (C)(0.5 * F[d]);
    k.bF1[d] = (C)(b1 * F[d]);
  }
  k.scale = (C)std::ldexp(1.0, scale_exp);
  k.inv_scale = (C)std::ldexp(1.0, -scale_exp);
  return k;
}

// ---- storage conversion -------------------------------------------------
template <int PREC>
__device__ __forceinline__ typename Form<PREC>::C decode(typename Form<PREC>::S v,
                                                         typename Form<PREC>::C inv_scale) {
  if constexpr (PREC == LBM_F16S) return __half2float(v) * inv_scale;
  else if constexpr (PREC == LBM_BF16S) return __bfloat162float(v) * inv_scale;
  else return v;
}

template <int PREC>
__device__ __forceinline__ typename Form<PREC>::S encode(typename Form<PREC>::C v,
                                                         typename Form<PREC>::C scale) {
  if constexpr (PREC == LBM_F16S) return __float2half_rn(v * scale);
  else if constexpr (PREC == LBM_BF16S) return __float2bfloat16_rn(v * scale);
  else return v;
}

// Global loads through the non-coherent path and streaming (evict-first)
// stores, as volatile inline PTX.  The compiler keeps volatile asm in program
// order, so in a chained step (prior_step_done() below) no PDF is read or
// written before the wait.  Loads ask L2 to fetch 256-byte blocks
// (LBM_LD_HINT): consecutive cells pull along the same rows, and the next
// warp's values then arrive with this one's.  On the 1024x256x256 bed,
// two alternating runs each: f64x 18,051 -> 18,099, FP32 shifted 30,605 ->
// 30,688, FP16 shifted 40,443 -> 40,644 MFLUP/s; a 128-byte hint changed
// nothing.
#ifndef LBM_LD_HINT
#define LBM_LD_HINT ".L2::256B"
#endif
__device__ __forceinline__ double ld_nc(const double* p) {
  double v;
  asm volatile("ld.global.nc" LBM_LD_HINT ".f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float ld_nc(const float* p) {
  float v;
  asm volatile("ld.global.nc" LBM_LD_HINT ".f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ int32_t ld_nc(const int32_t* p) {
  int32_t v;
  asm volatile("ld.global.nc" LBM_LD_HINT ".s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ unsigned short ld_nc(const unsigned short* p) {
  unsigned short v;
  asm volatile("ld.global.nc" LBM_LD_HINT ".u16 %0, [%1];" : "=h"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ void st_cs(double* p, double v) {
  asm volatile("st.global.cs.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ void st_cs(float* p, float v) {
  asm volatile("st.global.cs.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void st_cs(unsigned short* p, unsigned short v) {
  asm volatile("st.global.cs.u16 [%0], %1;" ::"l"(p), "h"(v) : "memory");
}

template <int PREC>
__device__ __forceinline__ typename Form<PREC>::S load_ro(const typename Form<PREC>::S* p) {
  if constexpr (PREC == LBM_F16S) {
    return __ushort_as_half(ld_nc(reinterpret_cast<const unsigned short*>(p)));
  } else if constexpr (PREC == LBM_BF16S) {
    return __ushort_as_bfloat16(ld_nc(reinterpret_cast<const unsigned short*>(p)));
  } else {
    return ld_nc(p);
  }
}

template <int PREC>
__device__ __forceinline__ void store_stream(typename Form<PREC>::S* p, typename Form<PREC>::S v) {
  if constexpr (PREC == LBM_F16S) {
    st_cs(reinterpret_cast<unsigned short*>(p), __half_as_ushort(v));
  } else if constexpr (PREC == LBM_BF16S) {
    st_cs(reinterpret_cast<unsigned short*>(p), __bfloat16_as_ushort(v));
  } else {
    st_cs(p, v);
  }
}

// ---- the collision ----------------------------------------------------------
// g[19] in: pulled PDFs (or deviations); out: post-collision values.
template <class C, bool DAMPED>
__device__ __forceinline__ void collide(C g[19], const Coef<C>& k, C alpha, C& rho_out,
                                        C u_out[3]) {
  C s[9], d[9];
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    s[p] = g[2 * p + 1] + g[2 * p + 2];
    d[p] = g[2 * p + 1] - g[2 * p + 2];
  }
  // pairs: 0:(1,2)=+x 1:(3,4)=+y 2:(5,6)=+z 3:(7,8)=(1,1,0) 4:(9,10)=(1,-1,0)
  // 5:(11,12)=(1,0,1) 6:(13,14)=(1,0,-1) 7:(15,16)=(0,1,1) 8:(17,18)=(0,1,-1)
  const C rho = g[0] + (((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7])) + s[8]);
  const C jx = ((d[0] + d[3]) + (d[4] + d[5])) + d[6];
  const C jy = ((d[1] + d[3]) - (d[4] - d[7])) + d[8];
  const C jz = ((d[2] + d[5]) - (d[6] - d[7])) - d[8];
  C ux, uy, uz, Vx, Vy, Vz;
  if constexpr (DAMPED) {
    const C ia = C(1) / (C(1) + C(0.5) * alpha);
    ux = (jx + k.hF[0]) * ia;
    uy = (jy + k.hF[1]) * ia;
    uz = (jz + k.hF[2]) * ia;
    Vx = k.a1 * ux + k.b1 * (k.F[0] - alpha * ux);
    Vy = k.a1 * uy + k.b1 * (k.F[1] - alpha * uy);
    Vz = k.a1 * uz + k.b1 * (k.F[2] - alpha * uz);
  } else {
    ux = jx + k.hF[0];
    uy = jy + k.hF[1];
    uz = jz + k.hF[2];
    Vx = k.a1 * ux + k.bF1[0];
    Vy = k.a1 * uy + k.bF1[1];
    Vz = k.a1 * uz + k.bF1[2];
  }
  const C usq = ux * ux + uy * uy + uz * uz;
  const C rp = rho - C(1.5) * usq;
  const C R1 = k.w1p * rp, R2 = C(0.5) * R1;
  g[0] = k.one_m_wp * g[0] + k.w0p * rp;
#define LBM_PAIR(P, CU, CV, R, K, HALF)                    \
  {                                                        \
    const C cu_ = (CU);                                    \
    const C cv_ = HALF ? C(0.5) * (CV) : (CV);             \
    const C P_ = k.hp * s[P] + (K * (cu_ * cu_) + R);      \
    const C Q_ = k.hm * d[P] + cv_;                        \
    g[2 * P + 1] = P_ + Q_;                                \
    g[2 * P + 2] = P_ - Q_;                                \
  }
  LBM_PAIR(0, ux, Vx, R1, k.k1, false)
  LBM_PAIR(1, uy, Vy, R1, k.k1, false)
  LBM_PAIR(2, uz, Vz, R1, k.k1, false)
  LBM_PAIR(3, ux + uy, Vx + Vy, R2, k.k2, true)
  LBM_PAIR(4, ux - uy, Vx - Vy, R2, k.k2, true)
  LBM_PAIR(5, ux + uz, Vx + Vz, R2, k.k2, true)
  LBM_PAIR(6, ux - uz, Vx - Vz, R2, k.k2, true)
  LBM_PAIR(7, uy + uz, Vy + Vz, R2, k.k2, true)
  LBM_PAIR(8, uy - uz, Vy - Vz, R2, k.k2, true)
#undef LBM_PAIR
  rho_out = rho;
  u_out[0] = ux;
  u_out[1] = uy;
  u_out[2] = uz;
}

// ---- the flux reduction --------------------------------------------------------
// The reducing step sums rho and u over its cells.  FP64 adds issue at 1/64
// of the FP32 rate on GB300, and a shuffle tree costs every lane 20 of them
// per cell: in FP64 the reduction made a reducing step of the 16-bit forms
// 2.4x as long as a plain one.  Instead each cell's rho - 1 and u are turned
// into int64 fixed point in units of 2^-60 (exact for |x| >= 2^-37 in FP32
// and |x| >= 2^-8 in FP64; smaller values round to the unit, error below
// 2^-61 per cell) and summed exactly per warp; each warp sum becomes FP64
// once.  A warp holding a value of magnitude >= 1/4, a NaN or an infinity
// sums in FP64 instead, so such values (NaN included) still reach the
// result.  Warp sums are combined in warp order, then over blocks in a
// fixed order: run-to-run identical.
__device__ __forceinline__ int64_t fixed60(float x) {   // |x| < 1/4
  const uint32_t b = __float_as_uint(x);
  const int e = (int)((b >> 23) & 0xffu);
  if (e == 0) return 0;
  const int64_t m = (int64_t)((b & 0x7fffffu) | 0x800000u);
  const int s = e - 90;   // x = m 2^(e - 150) = m 2^s units
  const int64_t v = s >= 0 ? (m << s) : (s > -25 ? ((m >> (-s - 1)) + 1) >> 1 : 0);
  return (b >> 31) ? -v : v;
}

__device__ __forceinline__ int64_t fixed60(double x) {   // |x| < 1/4
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ffu);
  if (e == 0) return 0;
  const int64_t m = (int64_t)((b & 0xfffffffffffffull) | (1ull << 52));
  const int s = e - 1015;   // x = m 2^(e - 1075) = m 2^s units
  const int64_t v = s >= 0 ? (m << s) : (s > -54 ? ((m >> (-s - 1)) + 1) >> 1 : 0);
  return (b >> 63) ? -v : v;
}

// Exact sum over the warp of int64 values with |v| < 2^58, on every lane:
// v + 2^58 (in [0, 2^59)) is cut into three pieces of at most 20 bits, each
// summed by one redux.sync over 32-bit values (each sum below 2^25), and
// recombined modulo 2^64.  Three instructions instead of a five-level tree of
// 64-bit shuffles and adds: the fixed-point FP64-storage reducing step went
// from 2.033 to 1.983 ms on the 1024x256x256 bed.
__device__ __forceinline__ int64_t warp_sum_i64(int64_t v) {
  const uint64_t u = (uint64_t)v + (1ull << 58);
  const uint64_t s0 = __reduce_add_sync(0xffffffffu, (unsigned)(u & 0xfffffu));
  const uint64_t s1 = __reduce_add_sync(0xffffffffu, (unsigned)((u >> 20) & 0xfffffu));
  const uint64_t s2 = __reduce_add_sync(0xffffffffu, (unsigned)(u >> 40));
  return (int64_t)(s0 + (s1 << 20) + (s2 << 40) - (32ull << 58));
}

// Warp sums of the cell's moments; lane 0 receives w[0] = sum rho (or
// sum (rho - 1) for the shifted forms, whose rho is already rho - 1) and
// w[1..3] = sum u (the other lanes' w is not the sum).  Every lane of the
// warp must call it.  Only lane 0 converts the fixed-point sums to FP64:
// 64-bit integer-to-float conversions and FP64 arithmetic issue at the
// FP64 rate, 1/64 of FP32 on GB300.  On the 1024x256x256 bed that took the
// reducing step of FP32S from 1.157 to 1.125 ms and of FP16S from 0.964 to
// 0.933 ms (the same change in the fixed-point FP64-storage step left it
// at 2.03 ms).
template <class C, bool SHIFTED>
__device__ __forceinline__ void warp_flux_sums(bool live, C rho, const C u[3], double w[4]) {
  const C v[4] = {live ? (SHIFTED ? rho : rho - C(1)) : C(0), live ? u[0] : C(0),
                  live ? u[1] : C(0), live ? u[2] : C(0)};
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 4; ++j) ok &= fabs(v[j]) < C(0.25);
  int cnt = live && !SHIFTED ? 1 : 0;
  if (__all_sync(0xffffffffu, ok)) {
    // a shuffle tree: warp_sum_i64 (redux) measured 0.8% slower here on the
    // FP16S reducing step, 0.946 against 0.938 ms
    int64_t s[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) s[j] = fixed60(v[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int j = 0; j < 4; ++j) s[j] += __shfl_down_sync(0xffffffffu, s[j], o);
      cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
      for (int j = 0; j < 4; ++j) w[j] = (double)s[j] * 0x1p-60;
      w[0] += (double)cnt;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) w[j] = 0.0;
    }
  } else {
    w[0] = live ? (SHIFTED ? (double)rho : (double)rho - 1.0) : 0.0;
#pragma unroll
    for (int j = 1; j < 4; ++j) w[j] = (double)v[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int j = 0; j < 4; ++j) w[j] += __shfl_down_sync(0xffffffffu, w[j], o);
      cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    }
    w[0] += (double)cnt;
  }
}

// Writes a warp's sums to its own slot: out[4 * (block * kWarpsPerBlock + warp) + j].
__device__ __forceinline__ void store_warp_sums(const double w[4], double* partials) {
  if ((threadIdx.x & 31) == 0) {
    double* o = partials + 4 * ((int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5));
#pragma unroll
    for (int j = 0; j < 4; ++j) o[j] = w[j];
  }
}

// Combines the block's warp sums in warp order into out[0..3] (the value
// collapse_warp_sums_kernel forms from store_warp_sums slots); has a block
// barrier.
__device__ __forceinline__ void store_block_sums(const double w[4], double* out) {
  __shared__ double sm[kWarpsPerBlock][4];
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int j = 0; j < 4; ++j) sm[threadIdx.x >> 5][j] = w[j];
  __syncthreads();
  if (threadIdx.x < 4) {
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < kWarpsPerBlock; ++k) acc += sm[k][threadIdx.x];
    out[threadIdx.x] = acc;
  }
}

// The 18 adjacency entries of cell i (the source slot of each pulled q > 0)
// from link rows of stride ld.
__device__ __forceinline__ void load_links(const int32_t* __restrict__ adj, int32_t ld, int32_t i,
                                           int32_t idx[18]) {
#pragma unroll
  for (int q = 0; q < 18; ++q) idx[q] = ld_nc(adj + q * ld + i);
}

// The 19 pulled values of cell i, given its adjacency entries.
template <int PREC>
__device__ __forceinline__ void pull(const typename Form<PREC>::S* __restrict__ src,
                                     const int32_t idx[18], int32_t i,
                                     typename Form<PREC>::C inv_scale,
                                     typename Form<PREC>::C g[19]) {
  g[0] = decode<PREC>(load_ro<PREC>(src + i), inv_scale);
#pragma unroll
  for (int q = 1; q < 19; ++q) g[q] = decode<PREC>(load_ro<PREC>(src + idx[q - 1]), inv_scale);
}

// Gathers the 19 pulled values of cell i (link rows of stride ld).
template <int PREC>
__device__ __forceinline__ void gather(const typename Form<PREC>::S* __restrict__ src,
                                       const int32_t* __restrict__ adj, int32_t ld, int32_t i,
                                       typename Form<PREC>::C inv_scale,
                                       typename Form<PREC>::C g[19]) {
  int32_t idx[18];
  load_links(adj, ld, i, idx);
  pull<PREC>(src, idx, i, inv_scale, g);
}

// ---- chained steps (programmatic dependent launch) --------------------------
// The second and later sweeps of an lbm_step call are launched with
// programmatic stream serialisation, so their blocks may start while the
// previous sweep still runs.  A sweep first loads its adjacency entries,
// which no step writes.  prior_step_done() then waits until the previous grid
// has completed and its writes are visible, and lets the next sweep's blocks
// launch.  PDF and damping accesses are volatile asm (ld_nc, st_cs), which the
// compiler keeps behind the wait.  The warp sums are plain C++ accesses: the
// wait returns zero, which the compiler cannot know, and the sums pointer is
// offset by it.  In a normal launch the wait returns at once.
__device__ __forceinline__ int32_t prior_step_done() {
  int32_t zero;
  asm volatile(
      "griddepcontrol.wait;\n\t"
      "griddepcontrol.launch_dependents;\n\t"
      "mov.b32 %0, 0;"
      : "=r"(zero)::"memory");
  return zero;
}

#ifndef LBM_SWEEP_MIN_BLOCKS
#define LBM_SWEEP_MIN_BLOCKS 4
#endif
// Resident 256-thread blocks per SM that the register budget of the FP32 and
// 16-bit sweeps is sized for (the FP64-arithmetic sweeps are bound by their
// arithmetic).  4 holds them at 64 registers, with all 18 indices and 19
// pulled values of a cell in flight and no spills; left free, the compiler
// takes 66-78 registers (3 blocks per SM).  On the 1024x256x256 bed forcing
// 5, 6, 7 or 8 blocks per SM cut the FP16 sweep by 3%, 4%, 8% and 8%.
template <int PREC>
constexpr int sweep_min_blocks() {
  return PREC == LBM_F64 || PREC == LBM_F64X ? 1 : LBM_SWEEP_MIN_BLOCKS;
}

// RED: 0 no reduction; 1 warp sums into per-warp slots (no block barrier);
// 2 block sums into per-block slots.  Both give the same final sums.
enum { kNoReduce = 0, kWarpSums = 1, kBlockSums = 2 };

// Resident blocks per SM the reducing variants of the FP32 and 16-bit
// forms are fitted to: 4 keeps them at the plain variant's 64 registers
// (1024x256x256 bed: FP16 reducing step 1.00 ms against 1.19 ms at the 72
// registers the compiler picks unconstrained; a plain step takes 0.86 ms).
#ifndef LBM_RED_MIN_BLOCKS
#define LBM_RED_MIN_BLOCKS 4
#endif

template <int PREC, int RED>
constexpr int sweep_launch_min_blocks() {
  return RED != kNoReduce && PREC != LBM_F64 && PREC != LBM_F64X ? LBM_RED_MIN_BLOCKS
                                                                 : sweep_min_blocks<PREC>();
}

// n cells; the PDF rows of src and dst and the link rows of adj have stride
// ld >= n, and the links name slots r ld + m.
// LINKS_FIRST: load the adjacency entries before waiting for the previous
// step (a chained launch then overlaps them with that step's end), instead of
// after.  On a grid of one wave (the 32x32x64 bed) that made the FP32 and
// 16-bit steps 15-17% faster; on the 1024x256x256 bed it cost the FP16 step
// 0.9%, and the fixed-point kernel spilled with it.
template <int PREC, bool DAMPED, int RED, bool LINKS_FIRST = false>
__global__ void __launch_bounds__(kSweepThreads, sweep_launch_min_blocks<PREC, RED>())
    sweep_kernel(const typename Form<PREC>::S* __restrict__ src,
                 typename Form<PREC>::S* __restrict__ dst, const int32_t* __restrict__ adj,
                 int32_t n, int32_t ld, Coef<typename Form<PREC>::C> k,
                 const typename Form<PREC>::C* __restrict__ alpha, double* __restrict__ partials) {
  using C = typename Form<PREC>::C;
  const int32_t i = blockIdx.x * kSweepThreads + threadIdx.x;
  C rho = C(0), u[3] = {C(0), C(0), C(0)};
  int32_t idx[18];
  int32_t z = 0;
  if constexpr (!LINKS_FIRST) z = prior_step_done();
  if (i < n) load_links(adj, ld, i, idx);
  if constexpr (LINKS_FIRST) z = prior_step_done();
  if (i < n) {
    C g[19];
    pull<PREC>(src, idx, i, k.inv_scale, g);
    collide<C, DAMPED>(g, k, DAMPED ? ld_nc(alpha + i) : C(0), rho, u);
#pragma unroll
    for (int q = 0; q < 19; ++q) store_stream<PREC>(dst + q * ld + i, encode<PREC>(g[q], k.scale));
  }
  if constexpr (RED != kNoReduce) {
    double w[4];
    warp_flux_sums<C, Form<PREC>::kShifted>(i < n, rho, u, w);
    if constexpr (RED == kWarpSums) store_warp_sums(w, partials + z);
    else store_block_sums(w, partials + z + 4 * (int64_t)blockIdx.x);
  }
}

template <int PREC>
__device__ __forceinline__ float bits_to_c(uint32_t h, float inv_scale) {
  if constexpr (PREC == LBM_F16S) return __half2float(__ushort_as_half((unsigned short)h)) * inv_scale;
  else return __bfloat162float(__ushort_as_bfloat16((unsigned short)h)) * inv_scale;
}
template <int PREC>
__device__ __forceinline__ uint32_t c_to_bits(float v, float scale) {
  if constexpr (PREC == LBM_F16S) return __half_as_ushort(__float2half_rn(v * scale));
  else return __bfloat16_as_ushort(__float2bfloat16_rn(v * scale));
}

// ---- two adjacent cells per thread (16-bit forms) ----------------------------
// A thread updates cells i and i + 1 (i even), so a warp covers 64
// consecutive cells and has twice the cells in flight at the same 64
// registers (4 blocks per SM).  The two accesses of a row are issued back to
// back -- both cells' links, both pulls, and, after both collisions, both
// stores -- so each pair lands on the same sectors at once and L1 and L2
// merge them.  Loads stay scalar; a row whose element q ld + i is even
// (every row: the row stride ld is a multiple of kRowAlign) takes the pair's
// two stores as one 4-byte store, which cuts the store instructions the LSU
// queue holds.  FP16 on the 1024x256x256 bed (N odd), MFLUP/s: with rows of
// stride N, alternating runs: one cell per thread 40,579-40,653; pair, all
// scalar 42,434-42,453; pair with the 4-byte stores on the even rows
// 43,307-43,376.  With every row aligned (this kernel) 45,779-45,784.
// Measured slower, on rows of stride N: 4-byte stores on the odd rows too,
// built with a lane shuffle, 41,923; one 4-byte load for both pulls where they share a word 29,135;
// 8-byte link loads on the aligned rows 29,844-30,936 (with and without the
// L2 hint, non-coherent or coherent; with registers to spare, 78 at 3 blocks
// per SM, 25,215 against 41,622 for scalar loads at that occupancy, so not
// register pressure); link rows through bulk copies into
// shared memory, completed on an mbarrier 36,780; three or four cells per
// thread 33,154 / 28,450; cells i and i + 32 of a warp's 64 40,189; links
// loaded before the wait for the previous step 37,263; write-back stores
// 42,277 (against 42,447); 2-byte rest-row loads 42,249; 128-thread blocks
// 41,209.  The per-cell arithmetic is that of sweep_kernel, so results are
// bit-identical to it.
#ifndef LBM_PAIR_SWEEP
#define LBM_PAIR_SWEEP 1
#endif
#ifndef LBM_PAIR_REST_U32
#define LBM_PAIR_REST_U32 1
#endif
#ifndef LBM_PAIR_THREADS
#define LBM_PAIR_THREADS 256
#endif
constexpr int kPairThreads = LBM_PAIR_THREADS;

__device__ __forceinline__ uint32_t ld_nc_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.global.nc" LBM_LD_HINT ".u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

// Pulls, both collisions and the stores of the pair (i, i + 1), given their
// links a (cell i) and b (cell i + 1); dst rows of stride ld.
template <int PREC, bool DAMPED>
__device__ __forceinline__ void pair_body(const typename Form<PREC>::S* __restrict__ src,
                                          typename Form<PREC>::S* __restrict__ dst, int32_t ld,
                                          const Coef<float>& k, const float* __restrict__ alpha,
                                          int32_t i, bool two, bool odd_ld, const int32_t a[18],
                                          const int32_t b[18]) {
  const unsigned short* src16 = reinterpret_cast<const unsigned short*>(src);
  // pulled values, packed: low half cell i, high half cell i + 1
  uint32_t g[19];
  if (LBM_PAIR_REST_U32 && two) {   // the rest row is aligned at even i
    g[0] = ld_nc_u32(reinterpret_cast<const uint32_t*>(src) + (i >> 1));
  } else {
    g[0] = ld_nc(src16 + i);
    if (two) g[0] |= (uint32_t)ld_nc(src16 + i + 1) << 16;
  }
#pragma unroll
  for (int q = 0; q < 18; ++q) {
    const uint32_t lo = ld_nc(src16 + a[q]);
    const uint32_t hi = two ? (uint32_t)ld_nc(src16 + b[q]) : 0u;
    g[q + 1] = lo | (hi << 16);
  }
  uint32_t out[19];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    if (c == 0 || two) {
      float v[19], rho, u[3];
#pragma unroll
      for (int q = 0; q < 19; ++q) v[q] = bits_to_c<PREC>(c ? g[q] >> 16 : g[q] & 0xffffu, k.inv_scale);
      collide<float, DAMPED>(v, k, DAMPED ? ld_nc(alpha + i + c) : 0.f, rho, u);
#pragma unroll
      for (int q = 0; q < 19; ++q) {
        const uint32_t h = c_to_bits<PREC>(v[q], k.scale);
        out[q] = c ? out[q] | (h << 16) : h;
      }
    }
  }
  unsigned short* dst16 = reinterpret_cast<unsigned short*>(dst);
#pragma unroll
  for (int q = 0; q < 19; ++q) {
    const int32_t e = q * ld + i;
    if (two && !(odd_ld && (q & 1))) {   // element e is even: one 4-byte store of the pair
      asm volatile("st.global.cs.u32 [%0], %1;" ::"l"(dst16 + e), "r"(out[q]) : "memory");
    } else {
      st_cs(dst16 + e, (unsigned short)(out[q] & 0xffffu));
      if (two) st_cs(dst16 + e + 1, (unsigned short)(out[q] >> 16));
    }
  }
}

template <int PREC, bool DAMPED>
__global__ void __launch_bounds__(kPairThreads, 4 * 256 / kPairThreads)
    sweep_pair_kernel(const typename Form<PREC>::S* __restrict__ src,
                      typename Form<PREC>::S* __restrict__ dst, const int32_t* __restrict__ adj,
                      int32_t n, int32_t ld, Coef<float> k, const float* __restrict__ alpha) {
  static_assert(PREC == LBM_F16S || PREC == LBM_BF16S, "16-bit forms only");
  const int32_t z = prior_step_done();
  const int32_t i = 2 * (int32_t)(blockIdx.x * kPairThreads + threadIdx.x) + z;
  if (i >= n) return;
  const bool two = i + 1 < n;   // false only for the last cell of an odd-length list
  const bool odd_ld = (ld & 1) != 0;
  int32_t a[18], b[18];
#pragma unroll
  for (int q = 0; q < 18; ++q) {
    const int32_t* p = adj + q * ld + i;
    a[q] = ld_nc(p);
    b[q] = two ? ld_nc(p + 1) : 0;
  }
  pair_body<PREC, DAMPED>(src, dst, ld, k, alpha, i, two, odd_ld, a, b);
}

// Per-cell moments of the collision that a step from `src` performs (rows
// of stride ld; rho_out [n], u_out [3][n]).
template <int PREC, bool DAMPED>
__global__ void __launch_bounds__(kSweepThreads)
    moments_kernel(const typename Form<PREC>::S* __restrict__ src, const int32_t* __restrict__ adj,
                   int32_t n, int32_t ld, Coef<typename Form<PREC>::C> k,
                   const typename Form<PREC>::C* __restrict__ alpha, double* __restrict__ rho_out,
                   double* __restrict__ u_out) {
  using C = typename Form<PREC>::C;
  const int32_t i = blockIdx.x * kSweepThreads + threadIdx.x;
  if (i >= n) return;
  C g[19];
  gather<PREC>(src, adj, ld, i, k.inv_scale, g);
  C rho, u[3];
  collide<C, DAMPED>(g, k, DAMPED ? alpha[i] : C(0), rho, u);
  rho_out[i] = Form<PREC>::kShifted ? 1.0 + (double)rho : (double)rho;
  u_out[i] = (double)u[0];
  u_out[n + i] = (double)u[1];
  u_out[2 * (int64_t)n + i] = (double)u[2];
}

// Group values from per-warp slots: thread b forms block b's value (its
// kWarpsPerBlock slots in slot order, the value store_block_sums forms
// inside a block), and each 256-thread CTA adds its
// 256 block values by a fixed tree into groups[4 g + j].  final_sum_kernel
// then adds the ceil(nblocks / 256) groups.  One 1024-thread block reading
// all block values had cost 0.15 ms per call on the 1024x256x256 bed.
constexpr int kCollapseThreads = 256;
__global__ void __launch_bounds__(kCollapseThreads)
    collapse_warp_sums_kernel(const double* __restrict__ part, int64_t nblocks,
                              double* __restrict__ groups) {
  __shared__ double sm[kCollapseThreads][4];
  const int64_t b = (int64_t)blockIdx.x * kCollapseThreads + threadIdx.x;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  if (b < nblocks) {
    const double* p = part + 4 * kWarpsPerBlock * b;
#pragma unroll
    for (int k = 0; k < kWarpsPerBlock; ++k)
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] += p[4 * k + j];
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) sm[threadIdx.x][j] = v[j];
  __syncthreads();
  for (int s = kCollapseThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
#pragma unroll
      for (int j = 0; j < 4; ++j) sm[threadIdx.x][j] += sm[threadIdx.x + s][j];
    __syncthreads();
  }
  if (threadIdx.x < 4) groups[4 * blockIdx.x + threadIdx.x] = sm[0][threadIdx.x];
}

// Final fixed-order sum of the block values: out[j] = sum_b part[4 b + j].
__global__ void __launch_bounds__(1024)
    final_sum_kernel(const double* __restrict__ part, int64_t nblocks, double* out) {
  __shared__ double sm[1024][4];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t b = threadIdx.x; b < nblocks; b += 1024)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] += part[4 * b + j];
#pragma unroll
  for (int j = 0; j < 4; ++j) sm[threadIdx.x][j] = acc[j];
  __syncthreads();
  for (int s = 512; s > 0; s >>= 1) {
    if (threadIdx.x < s)
#pragma unroll
      for (int j = 0; j < 4; ++j) sm[threadIdx.x][j] += sm[threadIdx.x + s][j];
    __syncthreads();
  }
  if (threadIdx.x < 4) out[threadIdx.x] = sm[0][threadIdx.x];
}

}  // namespace
}  // namespace lbm
