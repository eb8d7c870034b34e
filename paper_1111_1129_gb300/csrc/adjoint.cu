// Reverse mode (adjoint) of the sweep, for gradients of the mean axial
// velocity J = (1/N) sum_n u_axis,n of the collision of step K with respect
// to the body force F and a per-cell Brinkman damping alpha_n.
//
// Forward: f_0 given; for t = 1..K: g_t = S f_{t-1} (pull through the
// adjacency list), f_t = C(g_t; F, alpha) (TRT collision).  Reverse:
//   lam_g_K = dJ/dg_K,  lam_f_{t-1} = S^T lam_g_t,
//   lam_g_t = C'(g_t)^T lam_f_t  (t = K-1 .. 1),
// with dJ/dF and dJ/dalpha accumulated from every step.
//
// S^T needs no second index array: slot (q, m) is read in the forward pull
// either by the downstream cell k = m + c_q in direction q, whose
// adj[q-1][k] = q N + m, or -- when m + c_q is solid or beyond a closed
// face -- by m itself in direction opp(q) (bounce back).  Both cases are
// visible in adj[opp(q)-1][m], the pull of direction opp(q) at m, whose
// source is exactly m + c_q.
//
// C'^T is applied in closed form.  Writing the collision as
//   f*_q = L(g)_q + E_q(rho, u) + S_q(u),
//   L(g)_q = (1 - (w+ + w-)/2) g_q + ((w- - w+)/2) g_opp(q),
//   E_q = w+ w_q (rho + 4.5 (c_q.u)^2 - 1.5 u.u) + 3 w- w_q c_q.u,
//   S_q = (1 - w-/2) 3 w_q c_q.(F - alpha u),
// with drho/dg_r = 1 and du/dg_r = s c_r (s = 1/(1 + alpha/2)), one gets
//   lam_g_r = L^T(lam)_r + w+ M0 + s c_r.G,
//   G = 9 w+ M2 u - 3 w+ M0 u + 3 (w- - alpha (1 - w-/2)) M1,
//   dJ/dF     += (s/2) G + 3 (1 - w-/2) M1,
//   dJ/dalpha += -(s/2) G.u - 3 (1 - w-/2) M1.u,
// where M0 = sum w_q lam_q, M1 = sum w_q lam_q c_q, M2 = sum w_q lam_q c_q c_q^T.
//
// Memory: checkpoints of f every `stride` steps (stride ~ sqrt(K)) in the
// state's storage form, one segment of `stride` recomputed states, two
// adjoint buffers in the arithmetic precision.
#include <cmath>

#include "lbm_kernels.cuh"

struct lbm_adjoint {
  uint32_t magic;
  const lbm_state* st;
  cudaStream_t stream;   // the state's stream, kept so that freeing needs no state
  int32_t K, stride, n_ckpt;
  void* ckpt;       // n_ckpt states of 19 N storage elements
  void* seg;        // max(stride, 2) states
  void* lam[2];     // 19 N arithmetic-precision adjoints
  double* part;     // [nblocks][4]: dJ/dF_x, dJ/dF_y, dJ/dF_z, sum u_axis
  double* dalpha;   // [N]
  double* red_dev;  // [4]
  double* red_host; // [4], pinned
  cudaEvent_t done;
  int have_forward;
  double wp, wm, F[3];
  int32_t axis;
};

namespace lbm {
namespace {

// Coefficients of the reverse step, for its two forms (adjoint_step_kernel):
// the weighted form, and the pair form, which carries the weighted moments
// M of the adjoint as M' = 36 M (w0 = 12/36, w1 = 2/36, w2 = 1/36) with the
// 1/36 in the coefficients that multiply them.
template <class C>
struct AdjCoef {
  C wp, one_m_wp;  // w+, 1 - w+
  C k1, k2;        // 1 - (w+ + w-)/2, (w- - w+)/2
  C wm, src;       // w-, 1 - w-/2
  C hp, hm;        // (1 - w+)/2, (1 - w-)/2: the pair form of L^T
  C wp36, wp12, wp4;   // w+/36 (base), 3 w+/36, 9 w+/36 (G)
  C wm12, src12;   // beta/36 = w-/12 - alpha src/12
  C inv_n;         // 1 / N
};

template <class C>
AdjCoef<C> make_adj_coef(double wp, double wm, int64_t n) {
  AdjCoef<C> a;
  a.wp = (C)wp;
  a.one_m_wp = (C)(1.0 - wp);
  a.k1 = (C)(1.0 - 0.5 * (wp + wm));
  a.k2 = (C)(0.5 * (wm - wp));
  a.wm = (C)wm;
  a.src = (C)(1.0 - 0.5 * wm);
  a.hp = (C)(0.5 * (1.0 - wp));
  a.hm = (C)(0.5 * (1.0 - wm));
  a.wp36 = (C)(wp / 36.0);
  a.wp12 = (C)(wp / 12.0);
  a.wp4 = (C)(0.25 * wp);
  a.wm12 = (C)(wm / 12.0);
  a.src12 = (C)((1.0 - 0.5 * wm) / 12.0);
  a.inv_n = (C)(n > 0 ? 1.0 / (double)n : 0.0);
  return a;
}

// Flat slot, in the adjoint of the pulled values, that holds the adjoint of
// stored slot (q, i): s = adj[opp(q)-1][i].
__device__ __forceinline__ int32_t reverse_slot(int q, int32_t s, int32_t n, int32_t i) {
  const int o = opp(q);
  return s == q * n + i ? o * n + i : s + (q - o) * n;
}

// Velocity of the collision of the pulled values g (same arithmetic as the
// collision) and s = 1 / (1 + alpha/2).
template <class C, bool DAMPED>
__device__ __forceinline__ void velocity(const C g[19], const Coef<C>& k, C alpha, C u[3], C& s) {
  C d[9];
#pragma unroll
  for (int p = 0; p < 9; ++p) d[p] = g[2 * p + 1] - g[2 * p + 2];
  const C jx = ((d[0] + d[3]) + (d[4] + d[5])) + d[6];
  const C jy = ((d[1] + d[3]) - (d[4] - d[7])) + d[8];
  const C jz = ((d[2] + d[5]) - (d[6] - d[7])) - d[8];
  s = DAMPED ? C(1) / (C(1) + C(0.5) * alpha) : C(1);
  u[0] = (jx + k.hF[0]) * s;
  u[1] = (jy + k.hF[1]) * s;
  u[2] = (jz + k.hF[2]) * s;
}

__device__ __forceinline__ int axis_component(int q, int axis) {
  return axis == 0 ? cx(q) : (axis == 1 ? cy(q) : cz(q));
}

// Block-sum 4 values and add them to acc[4] (each block owns its slot;
// launches on one stream are ordered, so the accumulation is race free).
// The warp level sums in the arithmetic precision T of the values: FP64
// adds issue at 1/64 of the FP32 rate on GB300, and a shuffle tree costs
// every lane 20 of them per cell, most of an FP32 adjoint step.  Warp sums
// then accumulate in FP64.
template <class T>
__device__ __forceinline__ void block_accumulate4(T v[4], double* acc, bool assign) {
  __shared__ double sm[kSweepThreads / 32][4];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int j = 0; j < 4; ++j) sm[warp][j] = (double)v[j];
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kSweepThreads / 32; ++w) s += sm[w][threadIdx.x];
    acc[threadIdx.x] = assign ? s : acc[threadIdx.x] + s;
  }
}

// Seed: lam_g_K = dJ/dg_K from f_{K-1}; initialises dJ/dF, dJ/dalpha and
// the sum of u_axis (J = sum / N).
template <int PREC, bool DAMPED>
__global__ void __launch_bounds__(kSweepThreads)
    adjoint_seed_kernel(const typename Form<PREC>::S* __restrict__ f_prev,
                        const int32_t* __restrict__ adj, int32_t n,
                        Coef<typename Form<PREC>::C> k, AdjCoef<typename Form<PREC>::C> a,
                        const typename Form<PREC>::C* __restrict__ alpha, int axis,
                        typename Form<PREC>::C* __restrict__ lam_out, double* __restrict__ part,
                        double* __restrict__ dalpha) {
  using C = typename Form<PREC>::C;
  // A chained launch waits for the previous kernel here.  The zero it returns
  // offsets every index and pointer, so no access can be scheduled earlier.
  const int32_t z = prior_step_done();
  const int32_t i = blockIdx.x * kSweepThreads + threadIdx.x + z;
  double red[4] = {0.0, 0.0, 0.0, 0.0};
  if (i < n) {
    C g[19];
    gather<PREC>(f_prev, adj, n, i, k.inv_scale, g);
    C u[3], s;
    const C al = DAMPED ? alpha[i] : C(0);
    velocity<C, DAMPED>(g, k, al, u, s);
    const C seed = s * a.inv_n;
#pragma unroll
    for (int q = 0; q < 19; ++q) lam_out[q * n + i] = C(axis_component(q, axis)) * seed;
    red[axis] = 0.5 * (double)seed;
    red[3] = (double)u[axis];
    dalpha[i] = -0.5 * (double)seed * (double)u[axis];
  }
  block_accumulate4(red, part + z + 4 * (int64_t)blockIdx.x, true);
}

// One reverse step t: lam_f_t = S^T lam_g_{t+1} (gathered), then
// lam_g_t = C'(g_t)^T lam_f_t with g_t pulled from f_{t-1}.
template <int PREC, bool DAMPED>
__global__ void __launch_bounds__(kSweepThreads)
    adjoint_step_kernel(const typename Form<PREC>::S* __restrict__ f_prev,
                        const int32_t* __restrict__ adj, int32_t n,
                        Coef<typename Form<PREC>::C> k, AdjCoef<typename Form<PREC>::C> a,
                        const typename Form<PREC>::C* __restrict__ alpha,
                        const typename Form<PREC>::C* __restrict__ lam_in,
                        typename Form<PREC>::C* __restrict__ lam_out, double* __restrict__ part,
                        double* __restrict__ dalpha) {
  using C = typename Form<PREC>::C;
  const int32_t z = prior_step_done();  // as in adjoint_seed_kernel
  const int32_t i = blockIdx.x * kSweepThreads + threadIdx.x + z;
  C red[4] = {C(0), C(0), C(0), C(0)};
  if (i < n) {
    int32_t idx[18];
#pragma unroll
    for (int q = 0; q < 18; ++q) idx[q] = __ldg(adj + q * n + i);
    // all 36 pulls of the cell are independent: issue them back to back
    C lf[19], g[19];
    lf[0] = lam_in[i];
    g[0] = decode<PREC>(load_ro<PREC>(f_prev + i), k.inv_scale);
#pragma unroll
    for (int q = 1; q < 19; ++q) g[q] = decode<PREC>(load_ro<PREC>(f_prev + idx[q - 1]), k.inv_scale);
#pragma unroll
    for (int q = 1; q < 19; ++q) lf[q] = __ldg(lam_in + reverse_slot(q, idx[opp(q) - 1], n, i));
    C u[3], s;
    const C al = DAMPED ? alpha[i] : C(0);
    velocity<C, DAMPED>(g, k, al, u, s);
    C S[9], D[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
      S[p] = lf[2 * p + 1] + lf[2 * p + 2];
      D[p] = lf[2 * p + 1] - lf[2 * p + 2];
    }
    // Two forms of the same update.  FP64 arithmetic takes the pair form:
    // the outputs of pair (a, b) are e +- o, e = (1 - w+)/2 S + base and
    // o = (1 - w-)/2 D + s G (L^T's k1 la + k2 lb and k1 lb + k2 la have sum
    // (1 - w+) S and difference (1 - w-) D), with the moments carried as
    // 36 M.  It issues about a quarter fewer FP64 instructions: on the damped
    // 128^3 bed the IEEE reverse step took 371 us against 448 and the
    // reverse pass 1,297 ms against 1,450.  FP32 arithmetic keeps the
    // weighted form: there the pair form took 40 registers instead of 48,
    // ran 6 blocks per SM instead of 5, and was slower, 57.6 us against 53.2
    // (DRAM 65% against 71%; reverse pass 187 ms against 178).
    if constexpr (sizeof(C) == 8) {
      const C s34 = S[3] + S[4], s56 = S[5] + S[6], s78 = S[7] + S[8];
      const C M0 = C(12) * lf[0] + C(2) * ((S[0] + S[1]) + S[2]) + ((s34 + s56) + s78);
      const C M1x = C(2) * D[0] + ((D[3] + D[4]) + (D[5] + D[6]));
      const C M1y = C(2) * D[1] + ((D[3] - D[4]) + (D[7] + D[8]));
      const C M1z = C(2) * D[2] + ((D[5] - D[6]) + (D[7] - D[8]));
      const C Mxx = C(2) * S[0] + (s34 + s56);
      const C Myy = C(2) * S[1] + (s34 + s78);
      const C Mzz = C(2) * S[2] + (s56 + s78);
      const C Mxy = S[3] - S[4], Mxz = S[5] - S[6], Myz = S[7] - S[8];
      // G = 9 w+ M2 u - 3 w+ M0 u + beta M1, beta = 3 (w- - alpha (1 - w-/2))
      const C m0 = a.wp12 * M0;
      const C beta = a.wm12 - al * a.src12;
      const C Gx = a.wp4 * (Mxx * u[0] + Mxy * u[1] + Mxz * u[2]) - m0 * u[0] + beta * M1x;
      const C Gy = a.wp4 * (Mxy * u[0] + Myy * u[1] + Myz * u[2]) - m0 * u[1] + beta * M1y;
      const C Gz = a.wp4 * (Mxz * u[0] + Myz * u[1] + Mzz * u[2]) - m0 * u[2] + beta * M1z;
      const C base = a.wp36 * M0;
      lam_out[i] = a.one_m_wp * lf[0] + base;
#define LBM_ADJ_PAIR(P, CG)                                                    \
  {                                                                            \
    const C e_ = a.hp * S[P] + base;                                           \
    const C o_ = a.hm * D[P] + s * (CG);                                       \
    lam_out[(2 * P + 1) * n + i] = e_ + o_;                                    \
    lam_out[(2 * P + 2) * n + i] = e_ - o_;                                    \
  }
      LBM_ADJ_PAIR(0, Gx)
      LBM_ADJ_PAIR(1, Gy)
      LBM_ADJ_PAIR(2, Gz)
      LBM_ADJ_PAIR(3, Gx + Gy)
      LBM_ADJ_PAIR(4, Gx - Gy)
      LBM_ADJ_PAIR(5, Gx + Gz)
      LBM_ADJ_PAIR(6, Gx - Gz)
      LBM_ADJ_PAIR(7, Gy + Gz)
      LBM_ADJ_PAIR(8, Gy - Gz)
#undef LBM_ADJ_PAIR
      // dJ/dF += (s/2) G + 3 (1 - w-/2) M1; dJ/dalpha += -(s/2) G.u - 3 (1 - w-/2) M1.u
      const C hs = C(0.5) * s;
      red[0] = hs * Gx + a.src12 * M1x;
      red[1] = hs * Gy + a.src12 * M1y;
      red[2] = hs * Gz + a.src12 * M1z;
      const C Gu = Gx * u[0] + Gy * u[1] + Gz * u[2];
      const C M1u = M1x * u[0] + M1y * u[1] + M1z * u[2];
      dalpha[i] += (double)(-hs * Gu - a.src12 * M1u);
    } else {
      // weighted moments of the adjoint
      const C w0 = C(1.0 / 3.0), w1 = C(1.0 / 18.0), w2 = C(1.0 / 36.0);
      const C M0 = w0 * lf[0] + w1 * (S[0] + S[1] + S[2]) +
                   w2 * (((S[3] + S[4]) + (S[5] + S[6])) + (S[7] + S[8]));
      const C M1x = w1 * D[0] + w2 * ((D[3] + D[4]) + (D[5] + D[6]));
      const C M1y = w1 * D[1] + w2 * ((D[3] - D[4]) + (D[7] + D[8]));
      const C M1z = w1 * D[2] + w2 * ((D[5] - D[6]) + (D[7] - D[8]));
      const C Mxx = w1 * S[0] + w2 * ((S[3] + S[4]) + (S[5] + S[6]));
      const C Myy = w1 * S[1] + w2 * ((S[3] + S[4]) + (S[7] + S[8]));
      const C Mzz = w1 * S[2] + w2 * ((S[5] + S[6]) + (S[7] + S[8]));
      const C Mxy = w2 * (S[3] - S[4]);
      const C Mxz = w2 * (S[5] - S[6]);
      const C Myz = w2 * (S[7] - S[8]);
      const C nine_wp = C(9) * a.wp, three_wp_m0 = C(3) * a.wp * M0;
      const C beta = C(3) * (a.wm - al * a.src);
      const C Gx = nine_wp * (Mxx * u[0] + Mxy * u[1] + Mxz * u[2]) - three_wp_m0 * u[0] + beta * M1x;
      const C Gy = nine_wp * (Mxy * u[0] + Myy * u[1] + Myz * u[2]) - three_wp_m0 * u[1] + beta * M1y;
      const C Gz = nine_wp * (Mxz * u[0] + Myz * u[1] + Mzz * u[2]) - three_wp_m0 * u[2] + beta * M1z;
      const C base = a.wp * M0;
      lam_out[i] = a.one_m_wp * lf[0] + base;
#define LBM_ADJ_PAIR(P, CG)                                                    \
  {                                                                            \
    const C sg_ = s * (CG);                                                    \
    lam_out[(2 * P + 1) * n + i] = a.k1 * lf[2 * P + 1] + a.k2 * lf[2 * P + 2] + base + sg_; \
    lam_out[(2 * P + 2) * n + i] = a.k1 * lf[2 * P + 2] + a.k2 * lf[2 * P + 1] + base - sg_; \
  }
      LBM_ADJ_PAIR(0, Gx)
      LBM_ADJ_PAIR(1, Gy)
      LBM_ADJ_PAIR(2, Gz)
      LBM_ADJ_PAIR(3, Gx + Gy)
      LBM_ADJ_PAIR(4, Gx - Gy)
      LBM_ADJ_PAIR(5, Gx + Gz)
      LBM_ADJ_PAIR(6, Gx - Gz)
      LBM_ADJ_PAIR(7, Gy + Gz)
      LBM_ADJ_PAIR(8, Gy - Gz)
#undef LBM_ADJ_PAIR
      const C hs = C(0.5) * s, three_src = C(3) * a.src;
      red[0] = hs * Gx + three_src * M1x;
      red[1] = hs * Gy + three_src * M1y;
      red[2] = hs * Gz + three_src * M1z;
      const C Gu = Gx * u[0] + Gy * u[1] + Gz * u[2];
      const C M1u = M1x * u[0] + M1y * u[1] + M1z * u[2];
      dalpha[i] += (double)(-hs * Gu - three_src * M1u);
    }
  }
  block_accumulate4(red, part + z + 4 * (int64_t)blockIdx.x, false);
}

// ---- FP64-storage adjoint in double-single arithmetic --------------------------
// For LBM_F64X the reverse step keeps FP64-level accuracy without FP64
// instructions on its common path.  lambda is stored as a pair of FP32
// values (hi, lo) whose unevaluated sum carries ~48 significant bits, and
// is computed with error-free transformations: Knuth's TwoSum, Dekker's
// Fast2Sum (|a| >= |b|), and the product of two FP32 values with its exact
// error from one FMA (Ogita, Rump and Oishi, 2005).  The forward velocity
// comes exact from the FP64 bit patterns in 64-bit fixed point, as in the
// fixed-point sweep (units 2^-58), damping included (u - e u); a cell whose
// PDFs leave their binary ranges computes it in FP64 instead.
struct ds {
  float hi, lo;
};

__device__ __forceinline__ ds ds_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ds ds_fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ ds ds_add(ds x, ds y) {
  const ds s = ds_two_sum(x.hi, y.hi);
  return ds_fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}
__device__ __forceinline__ ds ds_neg(ds x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ ds ds_sub(ds x, ds y) { return ds_add(x, ds_neg(y)); }
__device__ __forceinline__ ds ds_mul(ds x, ds y) {
  const float p = x.hi * y.hi;
  const float e = fmaf(x.hi, y.hi, -p);
  return ds_fast_two_sum(p, fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e)));
}
// x times a power of two c (exact, barring overflow and underflow)
__device__ __forceinline__ ds ds_scale_pow2(ds x, float c) { return {x.hi * c, x.lo * c}; }
__device__ __forceinline__ double ds_to_double(ds x) { return (double)x.hi + (double)x.lo; }
// Host and device: the pair nearest to v (|lo| <= ulp(hi)/2).
__host__ __device__ __forceinline__ ds ds_from_double(double v) {
  const float hi = (float)v;
  return {hi, (float)(v - (double)hi)};
}
// An int64 value in units 2^-sc (sc = 58 or 63, |v| < 2^62), to ~48 bits.
// 64-bit integer conversions issue at the FP64 rate on GB300, so v is cut
// into three 21-bit pieces, each converted exactly as a 32-bit integer, and
// the pieces are summed as pairs.
__device__ __forceinline__ ds ds_from_fixed(int64_t v, int sc) {
  const float a = (float)(int32_t)(v >> 42) * 0x1p42f;                 // exact
  const float b = (float)(int32_t)((v >> 21) & 0x1FFFFF) * 0x1p21f;    // exact
  const float c = (float)(int32_t)(v & 0x1FFFFF);                      // exact
  const ds ab = ds_two_sum(a, b);
  const ds r = ds_add(ab, ds{c, 0.f});
  const float scale = sc == 58 ? 0x1p-58f : 0x1p-63f;   // exact: powers of two
  return {r.hi * scale, r.lo * scale};
}

// Coefficients of the reverse step as pairs (those of AdjCoef).
struct AdjCoefDS {
  ds one_m_wp, hp, hm, wp36, wp12, wp4, wm12, src12;
  int64_t fhF[3];   // F/2 in units 2^-58, for the fixed-point velocity
};

AdjCoefDS make_adj_coef_ds(double wp, double wm, const double F[3]) {
  AdjCoefDS a;
  a.one_m_wp = ds_from_double(1.0 - wp);
  a.hp = ds_from_double(0.5 * (1.0 - wp));
  a.hm = ds_from_double(0.5 * (1.0 - wm));
  a.wp36 = ds_from_double(wp / 36.0);
  a.wp12 = ds_from_double(wp / 12.0);
  a.wp4 = ds_from_double(0.25 * wp);
  a.wm12 = ds_from_double(wm / 12.0);
  a.src12 = ds_from_double((1.0 - 0.5 * wm) / 12.0);
  for (int d = 0; d < 3; ++d) a.fhF[d] = (int64_t)std::llround(0.5 * F[d] * 0x1p58);
  return a;
}

constexpr int64_t kAdjW0Bits = 0x3FD5555555555555LL;  // bits of 1/3, 1/18, 1/36
constexpr int64_t kAdjW1Bits = 0x3FAC71C71C71C71CLL;
constexpr int64_t kAdjW2Bits = 0x3F9C71C71C71C71CLL;

// Velocity and damping factor s = 1/(1 + alpha/2) of the collision of the
// pulled FP64 values g, as pairs: from the bit patterns in fixed point where
// every value lies in its weight's binary range (and alpha in [0, 1/2)),
// else in FP64.
template <bool DAMPED>
__device__ __forceinline__ void ds_velocity(const double g[19], const AdjCoefDS& a,
                                            const Coef<double>& kd,
                                            const double* __restrict__ alpha,
                                            const int64_t* __restrict__ alpha_fx, int32_t n,
                                            int32_t i, ds u[3], ds& s) {
  bool fast = true;
  int64_t X[19];
#pragma unroll
  for (int q = 0; q < 19; ++q) {
    const int64_t b = __double_as_longlong(g[q]);
    const int64_t wb = q == 0 ? kAdjW0Bits : (q <= 6 ? kAdjW1Bits : kAdjW2Bits);
    const int sh = q == 0 ? 4 : (q <= 6 ? 1 : 0);
    fast &= (b >> 52) == (wb >> 52);
    X[q] = (b - wb) << sh;   // exact deviation in units 2^-58 when in range
  }
  int64_t E = 0;
  if constexpr (DAMPED) {
    const int64_t A = __ldg(alpha_fx + i);
    fast &= A >= 0;
    E = __ldg(alpha_fx + n + i);
  }
  if (fast) {
    int64_t D[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) D[p] = X[2 * p + 1] - X[2 * p + 2];
    int64_t j[3] = {(((D[0] + D[3]) + (D[4] + D[5])) + D[6]) + a.fhF[0],
                    (((D[1] + D[3]) - (D[4] - D[7])) + D[8]) + a.fhF[1],
                    (((D[2] + D[5]) - (D[6] - D[7])) - D[8]) + a.fhF[2]};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if constexpr (DAMPED) j[d] -= __mul64hi(2 * j[d], E);   // u = j - e j
      u[d] = ds_from_fixed(j[d], 58);
    }
    s = DAMPED ? ds_sub(ds{1.f, 0.f}, ds_from_fixed(E, 63)) : ds{1.f, 0.f};
  } else {
    double ud[3], sd;
    velocity<double, DAMPED>(g, kd, DAMPED ? alpha[i] : 0.0, ud, sd);
#pragma unroll
    for (int d = 0; d < 3; ++d) u[d] = ds_from_double(ud[d]);
    s = ds_from_double(sd);
  }
}

// Block sums of four pairs, added to acc[4] in FP64 (as block_accumulate4).
__device__ __forceinline__ void block_accumulate4_ds(ds v[4], double* acc, bool assign) {
  __shared__ double sm[kSweepThreads / 32][4];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const ds w = {__shfl_down_sync(0xffffffffu, v[j].hi, o),
                    __shfl_down_sync(0xffffffffu, v[j].lo, o)};
      v[j] = ds_add(v[j], w);
    }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int j = 0; j < 4; ++j) sm[warp][j] = ds_to_double(v[j]);
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kSweepThreads / 32; ++w) t += sm[w][threadIdx.x];
    acc[threadIdx.x] = assign ? t : acc[threadIdx.x] + t;
  }
}

// Seed of the FP64-storage adjoint: as adjoint_seed_kernel, lambda written
// as pairs (float2 [19][N]).
template <bool DAMPED>
__global__ void __launch_bounds__(kSweepThreads)
    adjoint_seed_ds_kernel(const double* __restrict__ f_prev, const int32_t* __restrict__ adj,
                           int32_t n, Coef<double> k, AdjCoef<double> a,
                           const double* __restrict__ alpha, int axis, float2* __restrict__ lam_out,
                           double* __restrict__ part, double* __restrict__ dalpha) {
  const int32_t i = blockIdx.x * kSweepThreads + threadIdx.x;
  double red[4] = {0.0, 0.0, 0.0, 0.0};
  if (i < n) {
    double g[19];
    gather<LBM_F64>(f_prev, adj, n, i, 1.0, g);
    double u[3], s;
    const double al = DAMPED ? alpha[i] : 0.0;
    velocity<double, DAMPED>(g, k, al, u, s);
    const double seed = s * a.inv_n;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
      const ds v = ds_from_double((double)axis_component(q, axis) * seed);
      lam_out[q * n + i] = make_float2(v.hi, v.lo);
    }
    red[axis] = 0.5 * seed;
    red[3] = u[axis];
    dalpha[i] = -0.5 * seed * u[axis];
  }
  block_accumulate4(red, part + 4 * (int64_t)blockIdx.x, true);
}

// One reverse step of the FP64-storage adjoint (adjoint_step_kernel's
// formulas) in double-single arithmetic.
// 3 resident blocks per SM (80 registers, 36 bytes spilled): the damped
// 128^3 reverse pass took 0.392 s against 0.426 s at the 102 registers (2
// blocks) the compiler picks unbounded, two alternating runs each.
#ifndef LBM_ADJ_DS_MIN_BLOCKS
#define LBM_ADJ_DS_MIN_BLOCKS 3
#endif
template <bool DAMPED>
__global__ void __launch_bounds__(kSweepThreads, LBM_ADJ_DS_MIN_BLOCKS)
    adjoint_step_ds_kernel(const double* __restrict__ f_prev, const int32_t* __restrict__ adj,
                           int32_t n, Coef<double> kd, AdjCoefDS a,
                           const double* __restrict__ alpha, const int64_t* __restrict__ alpha_fx,
                           const float2* __restrict__ lam_in, float2* __restrict__ lam_out,
                           double* __restrict__ part, double* __restrict__ dalpha) {
  const int32_t i = blockIdx.x * kSweepThreads + threadIdx.x;
  ds red[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  if (i < n) {
    int32_t idx[18];
#pragma unroll
    for (int q = 0; q < 18; ++q) idx[q] = __ldg(adj + q * n + i);
    double g[19];
    float2 l2[19];
    g[0] = ld_nc(f_prev + i);
#pragma unroll
    for (int q = 1; q < 19; ++q) g[q] = ld_nc(f_prev + idx[q - 1]);
    l2[0] = __ldg(lam_in + i);
#pragma unroll
    for (int q = 1; q < 19; ++q) l2[q] = __ldg(lam_in + reverse_slot(q, idx[opp(q) - 1], n, i));
    ds u[3], s;
    ds_velocity<DAMPED>(g, a, kd, alpha, alpha_fx, n, i, u, s);
    ds lf[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) lf[q] = {l2[q].x, l2[q].y};
    // moments carried as 36 M, as in adjoint_step_kernel; the scalings by
    // 2, 4 and 8 are exact
    ds S[9], D[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
      S[p] = ds_add(lf[2 * p + 1], lf[2 * p + 2]);
      D[p] = ds_sub(lf[2 * p + 1], lf[2 * p + 2]);
    }
    const ds s34 = ds_add(S[3], S[4]), s56 = ds_add(S[5], S[6]), s78 = ds_add(S[7], S[8]);
    const ds M0 = ds_add(ds_add(ds_add(ds_scale_pow2(lf[0], 8.f), ds_scale_pow2(lf[0], 4.f)),
                                ds_scale_pow2(ds_add(ds_add(S[0], S[1]), S[2]), 2.f)),
                         ds_add(ds_add(s34, s56), s78));
    const ds M1x = ds_add(ds_scale_pow2(D[0], 2.f), ds_add(ds_add(D[3], D[4]), ds_add(D[5], D[6])));
    const ds M1y = ds_add(ds_scale_pow2(D[1], 2.f), ds_add(ds_sub(D[3], D[4]), ds_add(D[7], D[8])));
    const ds M1z = ds_add(ds_scale_pow2(D[2], 2.f), ds_add(ds_sub(D[5], D[6]), ds_sub(D[7], D[8])));
    const ds Mxx = ds_add(ds_scale_pow2(S[0], 2.f), ds_add(s34, s56));
    const ds Myy = ds_add(ds_scale_pow2(S[1], 2.f), ds_add(s34, s78));
    const ds Mzz = ds_add(ds_scale_pow2(S[2], 2.f), ds_add(s56, s78));
    const ds Mxy = ds_sub(S[3], S[4]);
    const ds Mxz = ds_sub(S[5], S[6]);
    const ds Myz = ds_sub(S[7], S[8]);
    const ds m0 = ds_mul(a.wp12, M0);
    // beta/36 = w-/12 - alpha src/12; alpha from its fixed-point value
    ds beta = a.wm12;
    if constexpr (DAMPED) {
      const int64_t A = __ldg(alpha_fx + i);
      const ds al = A >= 0 ? ds_from_fixed(A, 63) : ds_from_double(alpha[i]);
      beta = ds_sub(beta, ds_mul(a.src12, al));
    }
    const ds Gx = ds_add(ds_sub(ds_mul(a.wp4, ds_add(ds_add(ds_mul(Mxx, u[0]), ds_mul(Mxy, u[1])), ds_mul(Mxz, u[2]))),
                                ds_mul(m0, u[0])), ds_mul(beta, M1x));
    const ds Gy = ds_add(ds_sub(ds_mul(a.wp4, ds_add(ds_add(ds_mul(Mxy, u[0]), ds_mul(Myy, u[1])), ds_mul(Myz, u[2]))),
                                ds_mul(m0, u[1])), ds_mul(beta, M1y));
    const ds Gz = ds_add(ds_sub(ds_mul(a.wp4, ds_add(ds_add(ds_mul(Mxz, u[0]), ds_mul(Myz, u[1])), ds_mul(Mzz, u[2]))),
                                ds_mul(m0, u[2])), ds_mul(beta, M1z));
    const ds base = ds_mul(a.wp36, M0);
    {
      const ds v = ds_add(ds_mul(a.one_m_wp, lf[0]), base);
      lam_out[i] = make_float2(v.hi, v.lo);
    }
#define LBM_ADJ_DS_PAIR(P, CG)                                                                  \
  {                                                                                             \
    const ds e_ = ds_add(ds_mul(a.hp, S[P]), base);                                             \
    const ds o_ = ds_add(ds_mul(a.hm, D[P]), ds_mul(s, (CG)));                                  \
    const ds va_ = ds_add(e_, o_);                                                              \
    const ds vb_ = ds_sub(e_, o_);                                                              \
    lam_out[(2 * P + 1) * n + i] = make_float2(va_.hi, va_.lo);                                \
    lam_out[(2 * P + 2) * n + i] = make_float2(vb_.hi, vb_.lo);                                \
  }
    LBM_ADJ_DS_PAIR(0, Gx)
    LBM_ADJ_DS_PAIR(1, Gy)
    LBM_ADJ_DS_PAIR(2, Gz)
    LBM_ADJ_DS_PAIR(3, ds_add(Gx, Gy))
    LBM_ADJ_DS_PAIR(4, ds_sub(Gx, Gy))
    LBM_ADJ_DS_PAIR(5, ds_add(Gx, Gz))
    LBM_ADJ_DS_PAIR(6, ds_sub(Gx, Gz))
    LBM_ADJ_DS_PAIR(7, ds_add(Gy, Gz))
    LBM_ADJ_DS_PAIR(8, ds_sub(Gy, Gz))
#undef LBM_ADJ_DS_PAIR
    const ds hs = ds_scale_pow2(s, 0.5f);
    red[0] = ds_add(ds_mul(hs, Gx), ds_mul(a.src12, M1x));
    red[1] = ds_add(ds_mul(hs, Gy), ds_mul(a.src12, M1y));
    red[2] = ds_add(ds_mul(hs, Gz), ds_mul(a.src12, M1z));
    const ds Gu = ds_add(ds_add(ds_mul(Gx, u[0]), ds_mul(Gy, u[1])), ds_mul(Gz, u[2]));
    const ds M1u = ds_add(ds_add(ds_mul(M1x, u[0]), ds_mul(M1y, u[1])), ds_mul(M1z, u[2]));
    dalpha[i] += ds_to_double(ds_neg(ds_add(ds_mul(hs, Gu), ds_mul(a.src12, M1u))));
  }
  block_accumulate4_ds(red, part + 4 * (int64_t)blockIdx.x, false);
}

// lam_f_0 of the FP64-storage adjoint (lambda as pairs).
__global__ void __launch_bounds__(kSweepThreads)
    adjoint_initial_ds_kernel(const int32_t* __restrict__ adj, int32_t n,
                              const float2* __restrict__ lam_in, double* __restrict__ out) {
  const int32_t i = blockIdx.x * kSweepThreads + threadIdx.x;
  if (i >= n) return;
  const float2 v0 = lam_in[i];
  out[i] = (double)v0.x + (double)v0.y;
#pragma unroll
  for (int q = 1; q < 19; ++q) {
    const float2 v = lam_in[reverse_slot(q, adj[(opp(q) - 1) * n + i], n, i)];
    out[q * n + i] = (double)v.x + (double)v.y;
  }
}

// lam_f_0 = S^T lam_g_1 (gradient with respect to the initial PDFs).
template <class C>
__global__ void __launch_bounds__(kSweepThreads)
    adjoint_initial_kernel(const int32_t* __restrict__ adj, int32_t n,
                           const C* __restrict__ lam_in, double* __restrict__ out) {
  const int32_t i = blockIdx.x * kSweepThreads + threadIdx.x;
  if (i >= n) return;
  out[i] = (double)lam_in[i];
#pragma unroll
  for (int q = 1; q < 19; ++q)
    out[q * n + i] = (double)lam_in[reverse_slot(q, adj[(opp(q) - 1) * n + i], n, i)];
}

// ---- host orchestration -------------------------------------------------------

template <int PREC>
struct Runner {
  using S = typename Form<PREC>::S;
  using C = typename Form<PREC>::C;
  lbm_adjoint* ad;
  const lbm_state* st;
  int32_t n;
  cudaStream_t stream;
  unsigned grid;
  Coef<C> k;
  AdjCoef<C> a;
  const C* alpha;
  size_t state_elems;
  // Kernels after the first of a forward or backward pass are chained
  // (programmatic dependent launch; the kernels wait for their predecessor),
  // except in FP64 arithmetic, which chaining slows down.
  static constexpr bool kChain = PREC != LBM_F64 && PREC != LBM_F64X;
  mutable bool chained = false;
  mutable cudaError_t err = cudaSuccess;

  AdjCoefDS ads;   // LBM_F64X: the reverse step in double-single arithmetic
  Runner(lbm_adjoint* ad_) : ad(ad_), st(ad_->st) {
    n = (int32_t)st->sp->n;
    stream = st->sp->stream;
    grid = (unsigned)st->nblocks;
    k = make_coef<C>(ad->wp, ad->wm, ad->F, st->scale_exp);
    a = make_adj_coef<C>(ad->wp, ad->wm, n);
    alpha = (const C*)st->alpha;
    state_elems = 19 * (size_t)n;
    if constexpr (PREC == LBM_F64X) ads = make_adj_coef_ds(ad->wp, ad->wm, ad->F);
  }
  float2* lam2(int i) const { return (float2*)ad->lam[i]; }
  S* ckpt(int j) const { return (S*)ad->ckpt + (size_t)j * state_elems; }
  S* seg(int i) const { return (S*)ad->seg + (size_t)i * state_elems; }
  C* lam(int i) const { return (C*)ad->lam[i]; }

  template <class... P, class... A>
  void launch(void (*kernel)(P...), A... args) const {
    const cudaError_t e = launch_sweep(kernel, grid, stream, kChain && chained, args...);
    if (err == cudaSuccess) err = e;
    chained = true;
  }
  void step(const S* src, S* dst) const {
    if constexpr (PREC == LBM_F64X) {
      // FP64 storage: the fixed-point sweep, as lbm_step takes it
      const int rc = launch_fx_step(st, (const double*)src, (double*)dst, st->sp->adj, n, ad->wp,
                                    ad->wm, ad->F, stream, false);
      if (rc != LBM_OK && err == cudaSuccess) err = cudaErrorLaunchFailure;
      chained = true;
      return;
    }
    if (alpha) launch(sweep_kernel<PREC, true, kNoReduce>, src, dst, st->sp->adj, n, n, k, alpha, (double*)nullptr);
    else launch(sweep_kernel<PREC, false, kNoReduce>, src, dst, st->sp->adj, n, n, k, alpha, (double*)nullptr);
  }
  void seed(const S* f_prev) const {
    if constexpr (PREC == LBM_F64X) {
      const double* al = (const double*)alpha;
      if (alpha) launch(adjoint_seed_ds_kernel<true>, (const double*)f_prev, st->sp->adj, n, k, a, al, ad->axis, lam2(0), ad->part, ad->dalpha);
      else launch(adjoint_seed_ds_kernel<false>, (const double*)f_prev, st->sp->adj, n, k, a, al, ad->axis, lam2(0), ad->part, ad->dalpha);
      return;
    }
    if (alpha) launch(adjoint_seed_kernel<PREC, true>, f_prev, st->sp->adj, n, k, a, alpha, ad->axis, lam(0), ad->part, ad->dalpha);
    else launch(adjoint_seed_kernel<PREC, false>, f_prev, st->sp->adj, n, k, a, alpha, ad->axis, lam(0), ad->part, ad->dalpha);
  }
  void reverse(const S* f_prev, int in) const {
    if constexpr (PREC == LBM_F64X) {
      const double* al = (const double*)alpha;
      if (alpha) launch(adjoint_step_ds_kernel<true>, (const double*)f_prev, st->sp->adj, n, k, ads, al, (const int64_t*)st->alpha_fx, (const float2*)lam2(in), lam2(in ^ 1), ad->part, ad->dalpha);
      else launch(adjoint_step_ds_kernel<false>, (const double*)f_prev, st->sp->adj, n, k, ads, al, (const int64_t*)st->alpha_fx, (const float2*)lam2(in), lam2(in ^ 1), ad->part, ad->dalpha);
      return;
    }
    if (alpha) launch(adjoint_step_kernel<PREC, true>, f_prev, st->sp->adj, n, k, a, alpha, lam(in), lam(in ^ 1), ad->part, ad->dalpha);
    else launch(adjoint_step_kernel<PREC, false>, f_prev, st->sp->adj, n, k, a, alpha, lam(in), lam(in ^ 1), ad->part, ad->dalpha);
  }

  // Forward pass from the state's current PDFs: checkpoints f_{j*stride};
  // *last receives where f_{K-1} is.  The adjoint's arrays are [19][N] and
  // read through the plain links; the state's rows have stride sp->ld.
  int forward(const S** last) const {
    LBM_CUDA_TRY(cudaMemcpy2DAsync(ckpt(0), (size_t)n * sizeof(S), st->buf[st->cur],
                                   (size_t)st->sp->ld * sizeof(S), (size_t)n * sizeof(S), 19,
                                   cudaMemcpyDeviceToDevice, stream));
    chained = false;
    const S* cur = ckpt(0);
    for (int32_t t = 1; t <= ad->K - 1; ++t) {
      S* dst = (t % ad->stride == 0) ? ckpt(t / ad->stride) : seg(t & 1);
      step(cur, dst);
      cur = dst;
    }
    *last = cur;
    return LBM_OK;
  }

  // Recompute segment j: f_{j*stride + i} for i = 0..last into seg slots
  // (slot 0 is the checkpoint itself).
  void recompute(int j, int last) const {
    const S* cur = ckpt(j);
    for (int i = 1; i <= last; ++i) {
      step(cur, seg(i));
      cur = seg(i);
    }
  }
  const S* state_at(int j, int i) const { return i == 0 ? ckpt(j) : seg(i); }

  int backward(double* dJdf0) const {
    const int K = ad->K, s = ad->stride;
    int j = (K - 1) / s;
    chained = false;
    recompute(j, (K - 1) - j * s);
    seed(state_at(j, (K - 1) - j * s));
    int in = 0;
    for (int t = K - 1; t >= 1; --t) {
      const int jj = (t - 1) / s;
      if (jj != j) {
        j = jj;
        recompute(j, s - 1);
      }
      reverse(state_at(j, (t - 1) - j * s), in);
      in ^= 1;
    }
    if (dJdf0) {
      if constexpr (PREC == LBM_F64X)
        adjoint_initial_ds_kernel<<<grid, kSweepThreads, 0, stream>>>(st->sp->adj, n, lam2(in), dJdf0);
      else
        adjoint_initial_kernel<C><<<grid, kSweepThreads, 0, stream>>>(st->sp->adj, n, lam(in), dJdf0);
    }
    LBM_CUDA_TRY(err);
    LBM_CUDA_TRY(cudaGetLastError());
    return LBM_OK;
  }
};

template <int PREC>
int run_forward(lbm_adjoint* ad) {
  Runner<PREC> r(ad);
  if (r.n == 0) return LBM_OK;
  const typename Runner<PREC>::S* last = nullptr;
  const int rc = r.forward(&last);
  if (rc != LBM_OK) return rc;
  r.seed(last);
  LBM_CUDA_TRY(r.err);
  LBM_CUDA_TRY(cudaGetLastError());
  return LBM_OK;
}

template <int PREC>
int run_backward(lbm_adjoint* ad, double* dJdf0) {
  Runner<PREC> r(ad);
  if (r.n == 0) return LBM_OK;
  return r.backward(dJdf0);
}

#define LBM_ADJ_DISPATCH(prec, fn, ...)                      \
  switch (prec) {                                            \
    case LBM_F64: return fn<LBM_F64>(__VA_ARGS__);           \
    case LBM_F64X: return fn<LBM_F64X>(__VA_ARGS__);         \
    case LBM_F32: return fn<LBM_F32>(__VA_ARGS__);           \
    case LBM_F32S: return fn<LBM_F32S>(__VA_ARGS__);         \
    case LBM_F16S: return fn<LBM_F16S>(__VA_ARGS__);         \
    default: return fn<LBM_BF16S>(__VA_ARGS__);              \
  }

int dispatch_forward(lbm_adjoint* ad) { LBM_ADJ_DISPATCH(ad->st->precision, run_forward, ad) }
int dispatch_backward(lbm_adjoint* ad, double* dJdf0) {
  LBM_ADJ_DISPATCH(ad->st->precision, run_backward, ad, dJdf0)
}

bool valid_adjoint(const lbm_adjoint* ad) { return ad && ad->magic == kMagicAdjoint; }

// Final sums of the per-block accumulators into red_host.
int finish_sums(lbm_adjoint* ad) {
  const cudaStream_t stream = ad->st->sp->stream;
  if (ad->st->sp->n == 0) {
    for (int j = 0; j < 4; ++j) ad->red_host[j] = 0.0;
    return LBM_OK;
  }
  final_sum_kernel<<<1, 1024, 0, stream>>>(ad->part, ad->st->nblocks, ad->red_dev);
  LBM_CUDA_TRY(cudaGetLastError());
  LBM_CUDA_TRY(cudaMemcpyAsync(ad->red_host, ad->red_dev, 4 * sizeof(double),
                               cudaMemcpyDeviceToHost, stream));
  return wait_event(ad->done, stream, 0.0);
}

}  // namespace

void free_adjoint(lbm_adjoint* ad) {
  if (!ad) return;
  // the state may already be released (a garbage collector may free the two
  // in either order): only the stream kept here is used
  const cudaStream_t s = ad->stream;
  cudaStreamSynchronize(s);
  for (void* p : {ad->ckpt, ad->seg, ad->lam[0], ad->lam[1], (void*)ad->part,
                  (void*)ad->dalpha, (void*)ad->red_dev})
    dev_free(p, s, false);
  if (ad->red_host) cudaFreeHost(ad->red_host);
  if (ad->done) cudaEventDestroy(ad->done);
  ad->magic = 0;
  delete ad;
}

}  // namespace lbm

using namespace lbm;

extern "C" int lbm_adjoint_create(const lbm_state* st, int32_t n_steps, int32_t stride,
                                  lbm_adjoint** out) {
  clear_error();
  if (!out) return fail(LBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!valid_state(st)) return fail(LBM_EINVAL, "not a state handle");
  if (st->batch) return fail(LBM_EINVAL, "the adjoint is not available on a batched state");
  if (n_steps < 1) return fail(LBM_EINVAL, "n_steps = %d must be >= 1", n_steps);
  if (stride < 0) return fail(LBM_EINVAL, "checkpoint stride %d < 0", stride);
  if (stride == 0) stride = (int32_t)std::ceil(std::sqrt((double)n_steps));
  if (stride > n_steps) stride = n_steps;
  // the adjoint's arrays are [19][N], read through the public links
  const int rc = public_links(st->sp, nullptr);
  if (rc != LBM_OK) return rc;
  lbm_adjoint* ad = new lbm_adjoint{};
  ad->magic = kMagicAdjoint;
  ad->st = st;
  ad->stream = st->sp->stream;
  ad->K = n_steps;
  ad->stride = stride;
  ad->n_ckpt = (n_steps - 1) / stride + 1;
  const size_t n = (size_t)(st->sp->n > 0 ? st->sp->n : 1);
  const size_t sbytes = storage_bytes(st->precision) * 19 * n;
  const size_t cbytes = compute_bytes(st->precision) * 19 * n;
  const int nseg = stride > 2 ? stride : 2;
  const cudaStream_t s = st->sp->stream;
  bool ok = dev_alloc(&ad->ckpt, sbytes * ad->n_ckpt, s, false) == cudaSuccess &&
            dev_alloc(&ad->seg, sbytes * nseg, s, false) == cudaSuccess &&
            dev_alloc(&ad->lam[0], cbytes, s, false) == cudaSuccess &&
            dev_alloc(&ad->lam[1], cbytes, s, false) == cudaSuccess &&
            dev_alloc(&ad->part, sizeof(double) * 4 * st->nblocks, s, false) == cudaSuccess &&
            dev_alloc(&ad->dalpha, sizeof(double) * n, s, false) == cudaSuccess &&
            dev_alloc(&ad->red_dev, sizeof(double) * 4, s, false) == cudaSuccess &&
            cudaMallocHost(&ad->red_host, sizeof(double) * 4) == cudaSuccess &&
            cudaEventCreateWithFlags(&ad->done, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_adjoint(ad);
    return fail(LBM_ENOMEM, "adjoint allocation failed (%d checkpoints + %d segment states of %zu bytes)",
                (int)((n_steps - 1) / stride + 1), nseg, sbytes);
  }
  *out = ad;
  return LBM_OK;
}

extern "C" int lbm_adjoint_forward(lbm_adjoint* ad, double omega_plus, double omega_minus,
                                   const double force[3], int32_t axis, double* J_out) {
  clear_error();
  if (!valid_adjoint(ad)) return fail(LBM_EINVAL, "not an adjoint handle");
  if (!valid_state(ad->st)) return fail(LBM_EINVAL, "the adjoint's state was released");
  if (axis < 0 || axis > 2) return fail(LBM_EINVAL, "axis %d outside {0,1,2}", axis);
  if (!(omega_plus > 0.0 && omega_plus < 2.0) || !(omega_minus > 0.0 && omega_minus < 2.0))
    return fail(LBM_EINVAL, "relaxation rates must lie in (0, 2): %g, %g", omega_plus, omega_minus);
  if (!force) return fail(LBM_EINVAL, "force is NULL");
  for (int d = 0; d < 3; ++d)
    if (!std::isfinite(force[d])) return fail(LBM_EINVAL, "force[%d] is not finite", d);
  ad->wp = omega_plus;
  ad->wm = omega_minus;
  for (int d = 0; d < 3; ++d) ad->F[d] = force[d];
  ad->axis = axis;
  int rc = dispatch_forward(ad);
  if (rc != LBM_OK) return rc;
  rc = finish_sums(ad);
  if (rc != LBM_OK) return rc;
  const int64_t n = ad->st->sp->n;
  const double J = n > 0 ? ad->red_host[3] / (double)n : 0.0;
  if (!std::isfinite(J)) return fail(LBM_ENONFINITE, "objective is not finite");
  ad->have_forward = 1;
  if (J_out) *J_out = J;
  return LBM_OK;
}

extern "C" int lbm_adjoint_backward(lbm_adjoint* ad, double dJdF_out[3], double* dJdalpha_dev,
                                    double* dJdf0_dev) {
  clear_error();
  if (!valid_adjoint(ad)) return fail(LBM_EINVAL, "not an adjoint handle");
  if (!valid_state(ad->st)) return fail(LBM_EINVAL, "the adjoint's state was released");
  if (!ad->have_forward) return fail(LBM_EINVAL, "lbm_adjoint_forward has not run");
  int rc = dispatch_backward(ad, dJdf0_dev);
  if (rc != LBM_OK) return rc;
  const cudaStream_t stream = ad->st->sp->stream;
  const int64_t n = ad->st->sp->n;
  if (dJdalpha_dev && n > 0)
    LBM_CUDA_TRY(cudaMemcpyAsync(dJdalpha_dev, ad->dalpha, sizeof(double) * n,
                                 cudaMemcpyDeviceToDevice, stream));
  rc = finish_sums(ad);
  if (rc != LBM_OK) return rc;
  for (int d = 0; d < 3; ++d)
    if (!std::isfinite(ad->red_host[d])) return fail(LBM_ENONFINITE, "dJ/dF is not finite");
  if (dJdF_out)
    for (int d = 0; d < 3; ++d) dJdF_out[d] = ad->red_host[d];
  return LBM_OK;
}

extern "C" int lbm_adjoint_step(lbm_state* st, lbm_adjoint* ad, int32_t n_steps,
                                double omega_plus, double omega_minus, const double force[3],
                                int32_t axis, double* J_out, double dJdF_out[3],
                                double* dJdalpha_dev) {
  clear_error();
  if (!valid_adjoint(ad)) return fail(LBM_EINVAL, "not an adjoint handle");
  if (ad->st != st) return fail(LBM_EINVAL, "the adjoint was created for another state");
  if (n_steps != ad->K)
    return fail(LBM_EINVAL, "the adjoint was created for %d steps, not %d", ad->K, n_steps);
  int rc = lbm_adjoint_forward(ad, omega_plus, omega_minus, force, axis, J_out);
  if (rc != LBM_OK) return rc;
  return lbm_adjoint_backward(ad, dJdF_out, dJdalpha_dev, nullptr);
}
