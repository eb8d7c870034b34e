// FP64-storage sweep in exact 64-bit fixed point (precision form LBM_F64X).
//
// GB300 issues FP64 at about 1/64 of its FP32 rate, so a TRT update in
// IEEE FP64 arithmetic (~140 FP64 instructions) is bound by the FP64 pipe
// at ~4.3 GLUP/s, a quarter of what HBM could feed.  This kernel keeps the
// PDFs in FP64 but computes without FP64 instructions:
//
//  * Every f_q lies near its weight w_q (1/3, 1/18, 1/36), inside the same
//    binary range [2^E_q, 2^(E_q+1)).  There the difference of the raw
//    64-bit patterns, bits(f_q) - bits(w_q), is the exact deviation
//    f_q - w_q in units of the range's ulp 2^(E_q-52).  Shifting it to the
//    common unit U = 2^-58 gives an exact int64 X_q; the store converts
//    back the same way.  No FP64 conversion is needed on this path.
//  * Pair sums/differences, rho - 1 and j are then exact integer sums.
//  * Products with the relaxation constants use 64x64 -> high-64 integer
//    multiplies with the constants scaled by 2^63 (relative precision
//    2^-62).  The quadratic velocity terms come from the six products
//    u_a u_b, each built from three 32x32 -> 64 integer products and exact
//    to 2 units (7e-18); this needs |u| < 2^-6.
//  * After rounding to the storage units, the rest population takes the
//    remainder rho - 1 - sum_{q>0} X*_q (and a diagonal population the last
//    sub-unit part), so every collision conserves the stored mass exactly.
//
// Brinkman damping alpha_n stays in fixed point too.  lbm_set_damping stores
// per cell A = alpha 2^63 and E = e 2^63 with e = (alpha/2) / (1 + alpha/2),
// so that u = (j + F/2)/(1 + alpha/2) = (j + F/2) - e (j + F/2), and the
// odd-part coefficient w-/6 - b1 alpha (b1 = (1 - w-/2)/6) is an integer
// product of two 63-bit constants: the damped step issues no FP64
// instruction either, and reads 16 bytes more per update.
//
// A cell with any PDF outside its range, with |u| >= 2^-6 (fast flow,
// random test states, NaN) or with alpha outside [0, 1/2) takes the IEEE
// FP64 collision instead, and an output that leaves its range is written
// through FP64; both are exact to FP64 round-off.  The
// update is the TRT update of the FP64 form (same pair formulation), with
// errors below FP64 round-off of f.
#include "lbm_kernels.cuh"

namespace lbm {
namespace {

struct FxCoef {
  int64_t hp, hm, w1p, a1;  // (1-w+)/2, (1-w-)/2, w+/18, w-/6, each * 2^63
  int32_t hp_shift;         // when (1-w+)/2 = hp_sign * 2^-hp_shift exactly
  int32_t hp_sign;
  int64_t q1;               // w+/36 (quadratic terms) * 2^63
  int64_t hF[3];            // F/2 in units U
  int64_t bF1[3];           // (1 - w-/2) F / 6 in units U
  int64_t b1x2;             // 2 (1 - w-/2)/6 * 2^63: mul.hi with alpha 2^63 gives b1 alpha 2^63
};

// (a * b) / 2^58 for |a|, |b| < 2^52, from three 32x32 -> 64 products:
// with a = ah 2^29 + al (0 <= al < 2^29), a b / 2^58 = ah bh +
// (ah bl + al bh) / 2^29 + al bl / 2^58; the last term (< 1) and the floor
// of the middle one make it exact to within 2 units.
__device__ __forceinline__ int64_t uprod(int64_t a, int64_t b) {
  const int32_t ah = (int32_t)(a >> 29), bh = (int32_t)(b >> 29);
  const int32_t al = (int32_t)(a & 0x1FFFFFFF), bl = (int32_t)(b & 0x1FFFFFFF);
  return (int64_t)ah * bh + (((int64_t)ah * bl + (int64_t)al * bh) >> 29);
}

constexpr int64_t kW0Bits = 0x3FD5555555555555LL;  // 1/3
constexpr int64_t kW1Bits = 0x3FAC71C71C71C71CLL;  // 1/18
constexpr int64_t kW2Bits = 0x3F9C71C71C71C71CLL;  // 1/36

__device__ __forceinline__ int64_t wbits(int q) { return q == 0 ? kW0Bits : (q <= 6 ? kW1Bits : kW2Bits); }
__device__ __forceinline__ int64_t wexp(int q) { return q == 0 ? 0x3FD : (q <= 6 ? 0x3FA : 0x3F9); }
__device__ __forceinline__ int wshift(int q) { return q == 0 ? 4 : (q <= 6 ? 1 : 0); }

// x * c for a constant c = c63 / 2^63 (|c| < 1/2), |x| < 2^59: floor.
__device__ __forceinline__ int64_t fxmul(int64_t x, int64_t c63) { return __mul64hi(2 * x, c63); }

// Resident blocks of 256 threads per SM the register budget is fitted to:
// on the 1024x256x256 bed 3 (80 registers) beat 2 (120 registers) by 15%
// and 4 (64 registers, heavy spills) by 5%.  The reducing kernel, which
// runs once per lbm_step call, is fitted to 3 as well: 1.98 ms per launch
// there (2.19 ms at 2 blocks, 128 registers, and at 4, 64 registers with
// 168 bytes spilled), against 1.80 ms for a plain step.
#ifndef LBM_FX_MIN_BLOCKS
#define LBM_FX_MIN_BLOCKS 3
#endif
#ifndef LBM_FX_RED_MIN_BLOCKS
#define LBM_FX_RED_MIN_BLOCKS 3
#endif

// Warp sums of rho and u for the flux reduction, in two parts.  Cells on the
// fixed-point path give exact int64 moments in units U (rho - 1 below
// 2^57.4 and u below 2^56 in magnitude, so a warp's sum stays below 2^63);
// they are summed exactly as soon as the moments are known, so nothing of
// the reduction stays live through the collision, and lane 0 writes the
// warp's slot.  Cells that took the IEEE path add their FP64 rho and u to
// the slot afterwards, in warps that have one.  The final sum combines the
// slots in warp order, then over blocks in a fixed order.
__device__ __forceinline__ void fx_fixed_warp_sums(int64_t drho, int64_t ux, int64_t uy,
                                                   int64_t uz, int nfix, double* partials) {
  // below 2^58 units, as warp_sum_i64 needs
  int64_t iv[4] = {warp_sum_i64(drho), warp_sum_i64(ux), warp_sum_i64(uy), warp_sum_i64(uz)};
  nfix = (int)__reduce_add_sync(0xffffffffu, (unsigned)nfix);
  double w[4];
  w[0] = (double)nfix + (double)iv[0] * 0x1p-58;
#pragma unroll
  for (int j = 1; j < 4; ++j) w[j] = (double)iv[j] * 0x1p-58;
  store_warp_sums(w, partials);
}

__device__ __forceinline__ void fx_ieee_warp_add(double dv[4], bool ieee, double* partials) {
  if (!__any_sync(0xffffffffu, ieee)) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int j = 0; j < 4; ++j) dv[j] += __shfl_down_sync(0xffffffffu, dv[j], o);
  if ((threadIdx.x & 31) == 0) {
    double* o = partials + 4 * ((int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5));
#pragma unroll
    for (int j = 0; j < 4; ++j) o[j] += dv[j];
  }
}

// Pulls the raw bits of cell i's 19 PDFs, given its adjacency entries.
__device__ __forceinline__ void fx_pull(const double* __restrict__ src, const int32_t idx[18],
                                        int32_t i, int64_t b[19]) {
  b[0] = __double_as_longlong(ld_nc(src + i));
#pragma unroll
  for (int q = 1; q < 19; ++q) b[q] = __double_as_longlong(ld_nc(src + idx[q - 1]));
}

// The exact moments of the pulled values: pair sums S, pair differences D,
// rho - 1 and u, in units U.  False if the cell must take the IEEE path (a
// PDF outside its binary range, or |u| >= 2^-6).
__device__ __forceinline__ bool fx_moments(const int64_t b[19], const FxCoef& k, int64_t S[9],
                                           int64_t D[9], int64_t& drho, int64_t& ux,
                                           int64_t& uy, int64_t& uz) {
  bool fast = true;
#pragma unroll
  for (int q = 0; q < 19; ++q) fast &= (b[q] >> 52) == wexp(q);
  if (!fast) return false;
  int64_t X[19];
#pragma unroll
  for (int q = 0; q < 19; ++q) X[q] = (b[q] - wbits(q)) << wshift(q);
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    S[p] = X[2 * p + 1] + X[2 * p + 2];
    D[p] = X[2 * p + 1] - X[2 * p + 2];
  }
  drho = X[0] + (((S[0] + S[1]) + (S[2] + S[3])) + ((S[4] + S[5]) + (S[6] + S[7])) + S[8]);
  ux = (((D[0] + D[3]) + (D[4] + D[5])) + D[6]) + k.hF[0];
  uy = (((D[1] + D[3]) - (D[4] - D[7])) + D[8]) + k.hF[1];
  uz = (((D[2] + D[5]) - (D[6] - D[7])) - D[8]) + k.hF[2];
  // exact quadratic terms need |u| < 2^-6 (2^52 units)
  const int64_t lim = 1LL << 52;
  return ux > -lim && ux < lim && uy > -lim && uy < lim && uz > -lim && uz < lim;
}

// The fixed-point TRT collision of one cell from its exact moments, and the
// store of its 19 results.  HP_POW2: (1 - w+)/2 is +-2^-k (w+ = 1.25, 1.5,
// 0.75, ...), so the nine even-part products are shifts.
template <bool HP_POW2>
__device__ __forceinline__ void fx_collide_store(const int64_t S[9], const int64_t D[9],
                                                 int64_t drho, int64_t ux, int64_t uy,
                                                 int64_t uz, const FxCoef& k, int64_t a1,
                                                 double* __restrict__ dst, int32_t ld, int32_t i) {
  // a1: the odd-part coefficient w-/6 (undamped) or w-/6 - b1 alpha, * 2^63
  const int64_t V1x = fxmul(ux, a1) + k.bF1[0];
  const int64_t V1y = fxmul(uy, a1) + k.bF1[1];
  const int64_t V1z = fxmul(uz, a1) + k.bF1[2];
  const int64_t V2x = V1x >> 1, V2y = V1y >> 1, V2z = V1z >> 1;
  // Quadratic terms w+ w_p (4.5 (c.u)^2 - 1.5 u.u) = (w+ w_p / 2)
  // (9 (c.u)^2 - 3 u.u): with v = (w+/36) u, the products
  // T_ab = v_a u_b carry the class-1 factor (w+ w1 / 2 = w+/36), so
  // quad_1 = 9 T_aa - 3 T_tr and quad_2 = that expression / 2 for the
  // diagonal (c.u)^2 = T_aa + T_bb +- 2 T_ab.
  const int64_t vx = fxmul(ux, k.q1), vy = fxmul(uy, k.q1), vz = fxmul(uz, k.q1);
  const int64_t Txx = uprod(vx, ux), Tyy = uprod(vy, uy), Tzz = uprod(vz, uz);
  const int64_t Txy2 = 2 * uprod(vx, uy), Txz2 = 2 * uprod(vx, uz), Tyz2 = 2 * uprod(vy, uz);
  const int64_t Ttr3 = 3 * (Txx + Tyy + Tzz);
  const int64_t R1 = fxmul(drho, k.w1p);
  const int64_t R2 = R1 >> 1;
  int64_t out[19];
#define LBM_FX_PAIR(P, QUAD, R, VX)                                         \
  {                                                                         \
    const int64_t hS_ = HP_POW2 ? (k.hp_sign > 0 ? S[P] >> k.hp_shift       \
                                             : -(S[P] >> k.hp_shift))   \
                            : fxmul(S[P], k.hp);                        \
    const int64_t P_ = hS_ + R + (QUAD);                                    \
    const int64_t Q_ = fxmul(D[P], k.hm) + (VX);                            \
    out[2 * P + 1] = P_ + Q_;                                               \
    out[2 * P + 2] = P_ - Q_;                                               \
  }
  LBM_FX_PAIR(0, 9 * Txx - Ttr3, R1, V1x)
  LBM_FX_PAIR(1, 9 * Tyy - Ttr3, R1, V1y)
  LBM_FX_PAIR(2, 9 * Tzz - Ttr3, R1, V1z)
  LBM_FX_PAIR(3, (9 * (Txx + Tyy + Txy2) - Ttr3) >> 1, R2, V2x + V2y)
  LBM_FX_PAIR(4, (9 * (Txx + Tyy - Txy2) - Ttr3) >> 1, R2, V2x - V2y)
  LBM_FX_PAIR(5, (9 * (Txx + Tzz + Txz2) - Ttr3) >> 1, R2, V2x + V2z)
  LBM_FX_PAIR(6, (9 * (Txx + Tzz - Txz2) - Ttr3) >> 1, R2, V2x - V2z)
  LBM_FX_PAIR(7, (9 * (Tyy + Tzz + Tyz2) - Ttr3) >> 1, R2, V2y + V2z)
  LBM_FX_PAIR(8, (9 * (Tyy + Tzz - Tyz2) - Ttr3) >> 1, R2, V2y - V2z)
#undef LBM_FX_PAIR
  // Round the moving populations to their storage units (2^-57 axis,
  // 2^-58 diagonal); the rest population takes the remainder rounded to
  // its unit 2^-54, and the last -8..7 units go to a diagonal
  // population, so the stored deviations sum exactly to drho: every
  // step conserves the stored mass bit for bit.
  int64_t d[19];
  int64_t stored = 0;
#pragma unroll
  for (int q = 1; q < 19; ++q) {
    const int s = wshift(q);
    d[q] = s ? (out[q] + (1LL << (s - 1))) >> s : out[q];
    stored += d[q] << s;
  }
  const int64_t rem = drho - stored;
  d[0] = (rem + 8) >> 4;
  d[7] += rem - (d[0] << 4);
  // Store the fixed-point result; an output that left its binary range
  // (rare) is rewritten through FP64 in a separate branch, so the
  // common path issues no FP64 instruction at all.
  uint32_t out_of_range = 0;
#pragma unroll
  for (int q = 0; q < 19; ++q) {
    const int64_t bits = wbits(q) + d[q];
    out_of_range |= (uint32_t)((bits >> 52) != wexp(q)) << q;
    st_cs(dst + q * ld + i, __longlong_as_double(bits));
  }
  if (out_of_range) {
    for (int q = 0; q < 19; ++q)
      if ((out_of_range >> q) & 1u)
        dst[q * ld + i] = weight(q) + (double)(d[q] << wshift(q)) * 0x1p-58;
  }
}

// The IEEE FP64 collision of one cell (out-of-range cells) and its store.
template <bool DAMPED>
__device__ __forceinline__ void fx_ieee_collide_store(double g[19], const Coef<double>& kd,
                                                      double alpha, double* __restrict__ dst,
                                                      int32_t ld, int32_t i, double red[4]) {
  double rho, u[3];
  collide<double, DAMPED>(g, kd, alpha, rho, u);
#pragma unroll
  for (int q = 0; q < 19; ++q) st_cs(dst + q * ld + i, g[q]);
  red[0] = rho;
  red[1] = u[0];
  red[2] = u[1];
  red[3] = u[2];
}

// Damping of cell i in fixed point: u <- u - e u (u = j + F/2 in units U)
// and the odd-part coefficient w-/6 - b1 alpha (* 2^63).  False if the cell
// must take the IEEE path (alpha outside [0, 1/2)).
template <bool DAMPED>
__device__ __forceinline__ bool fx_damp(const int64_t* __restrict__ alpha_fx, int32_t n,
                                        int32_t i, const FxCoef& k, int64_t& ux, int64_t& uy,
                                        int64_t& uz, int64_t& a1) {
  a1 = k.a1;
  if constexpr (DAMPED) {
    const int64_t A = __ldg(alpha_fx + i);
    if (A < 0) return false;
    const int64_t E = __ldg(alpha_fx + n + i);
    ux -= fxmul(ux, E);
    uy -= fxmul(uy, E);
    uz -= fxmul(uz, E);
    a1 -= __mul64hi(k.b1x2, A);
  }
  return true;
}

// A step that does not reduce: n cells, PDF and link rows of stride ld.
template <bool HP_POW2, bool DAMPED>
__global__ void __launch_bounds__(kSweepThreads, LBM_FX_MIN_BLOCKS)
    sweep_fx_kernel(const double* __restrict__ src, double* __restrict__ dst,
                    const int32_t* __restrict__ adj, int32_t n, int32_t ld, FxCoef k,
                    Coef<double> kd, const double* __restrict__ alpha,
                    const int64_t* __restrict__ alpha_fx) {
  const int32_t i = blockIdx.x * kSweepThreads + threadIdx.x;
  prior_step_done();  // a chained launch waits here for the previous step
  if (i < n) {
    int32_t idx[18];
    int64_t b[19];
    load_links(adj, ld, i, idx);
    fx_pull(src, idx, i, b);
    int64_t S[9], D[9], drho = 0, ux = 0, uy = 0, uz = 0, a1 = 0;
    if (fx_moments(b, k, S, D, drho, ux, uy, uz) &&
        fx_damp<DAMPED>(alpha_fx, n, i, k, ux, uy, uz, a1)) {
      fx_collide_store<HP_POW2>(S, D, drho, ux, uy, uz, k, a1, dst, ld, i);
    } else {
      double g[19], red[4];
#pragma unroll
      for (int q = 0; q < 19; ++q) g[q] = __longlong_as_double(b[q]);
      fx_ieee_collide_store<DAMPED>(g, kd, DAMPED ? ld_nc(alpha + i) : 0.0, dst, ld, i, red);
    }
  }
}

// The reducing step.  The fixed-point moments are summed per warp before the
// collision, and a cell that takes the IEEE path pulls its values again
// rather than keep the raw bits live: the reduction then adds little to the
// registers the collision needs.  (Sharing this structure with the plain
// step made that one spill.)
template <bool HP_POW2, bool DAMPED>
__global__ void __launch_bounds__(kSweepThreads, LBM_FX_RED_MIN_BLOCKS)
    sweep_fx_reduce_kernel(const double* __restrict__ src, double* __restrict__ dst,
                           const int32_t* __restrict__ adj, int32_t n, int32_t ld, FxCoef k,
                           Coef<double> kd, const double* __restrict__ alpha,
                           const int64_t* __restrict__ alpha_fx, double* __restrict__ partials) {
  const int32_t i = blockIdx.x * kSweepThreads + threadIdx.x;
  const bool live = i < n;
  bool fast = false;
  int64_t S[9], D[9], drho = 0, ux = 0, uy = 0, uz = 0, a1 = 0;
  const int32_t z = prior_step_done();  // zero, after the previous step has finished
  if (live) {
    int32_t idx[18];
    int64_t b[19];
    load_links(adj, ld, i, idx);
    fx_pull(src, idx, i, b);
    fast = fx_moments(b, k, S, D, drho, ux, uy, uz) &&
           fx_damp<DAMPED>(alpha_fx, n, i, k, ux, uy, uz, a1);
  }
  fast ? fx_fixed_warp_sums(drho, ux, uy, uz, 1, partials + z)
       : fx_fixed_warp_sums(0, 0, 0, 0, 0, partials + z);
  double red[4] = {0.0, 0.0, 0.0, 0.0};   // IEEE-path cells: rho, u
  if (live) {
    if (fast) {
      fx_collide_store<HP_POW2>(S, D, drho, ux, uy, uz, k, a1, dst, ld, i);
    } else {
      double g[19];
      g[0] = ld_nc(src + i);
#pragma unroll
      for (int q = 1; q < 19; ++q) g[q] = ld_nc(src + __ldg(adj + (q - 1) * ld + i));
      fx_ieee_collide_store<DAMPED>(g, kd, DAMPED ? ld_nc(alpha + i) : 0.0, dst, ld, i, red);
    }
  }
  fx_ieee_warp_add(red, live && !fast, partials + z);
}

int64_t c63(double c) { return (int64_t)std::llround(c * 0x1p63); }
int64_t units(double v) { return (int64_t)std::llround(v * 0x1p58); }

}  // namespace

namespace {

// Fixed-point coefficients of a step with these rates and force; *pow2:
// (1 - w+)/2 is an exact power of two, so the even-part products are shifts.
FxCoef make_fx_coef(double wp, double wm, const double F[3], bool* pow2) {
  FxCoef k{};
  k.hp = c63(0.5 * (1.0 - wp));
  // exact power of two (the mantissa of |hp| is 1/2) between 2^-1 and 2^-40
  const double hp = 0.5 * (1.0 - wp);
  int e = 0;
  const double m = hp != 0.0 ? std::frexp(std::fabs(hp), &e) : 0.0;
  *pow2 = m == 0.5 && -e + 1 >= 1 && -e + 1 <= 40;
  k.hp_shift = *pow2 ? 1 - e : 0;
  k.hp_sign = hp < 0 ? -1 : 1;
  k.hm = c63(0.5 * (1.0 - wm));
  k.w1p = c63(wp / 18.0);
  k.a1 = c63(wm / 6.0);
  for (int d = 0; d < 3; ++d) {
    k.hF[d] = units(0.5 * F[d]);
    k.bF1[d] = units((1.0 - 0.5 * wm) * F[d] / 6.0);
  }
  k.q1 = c63(wp / 36.0);
  k.b1x2 = 2 * c63((1.0 - 0.5 * wm) / 6.0);
  return k;
}

// One fixed-point step of state st (its damping included) from src to dst,
// arrays of rows of stride ld read through links adj; partials non-null: the
// reducing variant.
cudaError_t launch_fx(const lbm_state* st, const double* src, double* dst, const int32_t* adj,
                      int32_t ld, const FxCoef& k, bool pow2, const Coef<double>& kd,
                      cudaStream_t stream, bool chained, double* partials) {
  const int32_t n = (int32_t)st->sp->n;
  const unsigned grid = (unsigned)st->nblocks;
  const double* alpha = (const double*)st->alpha;
  const int64_t* afx = st->alpha_fx;
#define LBM_FX_LAUNCH(P2, DA)                                                                       \
  return partials ? launch_sweep(sweep_fx_reduce_kernel<P2, DA>, grid, stream, chained, src, dst, adj, n, ld, k, kd, alpha, afx, partials) \
                  : launch_sweep(sweep_fx_kernel<P2, DA>, grid, stream, chained, src, dst, adj, n, ld, k, kd, alpha, afx)
  if (alpha) {
    if (pow2) LBM_FX_LAUNCH(true, true);
    LBM_FX_LAUNCH(false, true);
  }
  if (pow2) LBM_FX_LAUNCH(true, false);
  LBM_FX_LAUNCH(false, false);
#undef LBM_FX_LAUNCH
}

}  // namespace

int launch_steps_fx(lbm_state* st, int32_t n_steps, double wp, double wm, const double F[3],
                    cudaStream_t stream, bool reduce_last) {
  bool pow2 = false;
  const FxCoef k = make_fx_coef(wp, wm, F, &pow2);
  const Coef<double> kd = make_coef<double>(wp, wm, F, 0);
  for (int32_t t = 0; t < n_steps; ++t) {
    const double* src = (const double*)st->buf[st->cur];
    double* dst = (double*)st->buf[st->cur ^ 1];
    if (st->sp->n > 0) {
      const bool last = reduce_last && t == n_steps - 1;
      LBM_CUDA_TRY(launch_fx(st, src, dst, state_links(st->sp), (int32_t)st->sp->ld, k, pow2, kd,
                             stream, t > 0, last ? st->partials : nullptr));
    }
    st->cur ^= 1;
  }
  return LBM_OK;
}

int launch_fx_step(const lbm_state* st, const double* src, double* dst, const int32_t* adj,
                   int32_t ld, double wp, double wm, const double F[3], cudaStream_t stream,
                   bool chained) {
  if (st->sp->n == 0) return LBM_OK;
  bool pow2 = false;
  const FxCoef k = make_fx_coef(wp, wm, F, &pow2);
  const Coef<double> kd = make_coef<double>(wp, wm, F, 0);
  LBM_CUDA_TRY(launch_fx(st, src, dst, adj, ld, k, pow2, kd, stream, chained, nullptr));
  return LBM_OK;
}

namespace {
// alpha_fx of a damped FP64-storage state: A = alpha 2^63 (or -1 where alpha
// is outside [0, 1/2): that cell takes the IEEE path) and
// E = e 2^63, e = (alpha/2) / (1 + alpha/2).
__global__ void set_alpha_fx_kernel(const double* __restrict__ a, int32_t n,
                                    int64_t* __restrict__ out) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double al = a[i];
  const bool ok = al >= 0.0 && al < 0.5;
  const double e = ok ? (0.5 * al) / (1.0 + 0.5 * al) : 0.0;
  out[i] = ok ? (int64_t)llrint(al * 0x1p63) : -1;
  out[n + i] = ok ? (int64_t)llrint(e * 0x1p63) : 0;
}
}  // namespace

int set_alpha_fx(lbm_state* st, const double* alpha_dev) {
  const int64_t n = st->sp->n;
  if (n == 0) return LBM_OK;
  set_alpha_fx_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st->sp->stream>>>(
      alpha_dev, (int32_t)n, st->alpha_fx);
  LBM_CUDA_TRY(cudaGetLastError());
  return LBM_OK;
}

}  // namespace lbm
