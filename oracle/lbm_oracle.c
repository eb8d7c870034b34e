/*
 * CPU oracle for the sparse D3Q19 TRT lattice Boltzmann path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU baseline of
 * the benchmark do.  It shares no code, header or table with the CUDA path.
 *
 * Plain, slow, obviously correct FP64 code, written in the order of the
 * method's definition:
 *
 *   - the numbering scheme I(x,y,z) (lexicographic, lexicographic with
 *     blocking, Z curve with 1-bit and 2-bit interleave, and the Hilbert
 *     curve by Skilling's transform) applied to all cells, and the contiguous index I_c = rank of a fluid cell in that
 *     order, solids excluded (Sec. 3, "Numbering scheme" and the definition
 *     of I_c in [1, N_f]);
 *   - the adjacency list of the sparse representation with implicit bounce
 *     back (Sec. 2, sparse representation), built by inspecting the
 *     neighbourhood of each fluid cell in the full representation (Sec. 3,
 *     end of "Contiguous index generation");
 *   - the flow solver as a full-array (marker-and-cell) D3Q19 TRT solver
 *     (Sec. 2 full arrays; Sec. 1 TRT on D3Q19; Sec. 7 pull scheme): every
 *     fluid cell pulls its 19 PDFs by coordinates from the dense grid, with
 *     half-way bounce back at solid cells and closed faces, then collides.
 *     It never touches an adjacency list, so an adjacency bug cannot cancel.
 *   - the adjoint (reverse mode) of the time loop through the exact Jacobian
 *     of the collision, for gradients of the mean axial velocity;
 *   - one step on a given sparse list (pull through an explicit adjacency,
 *     then the same collision), used to check chunked runs whose lists
 *     carry ghost slots.
 *
 * The paper names TRT [Ginzburg] but does not print its equations.  The
 * readings used here, which the GPU path shares:
 *   rho = sum_q g_q,  j = sum_q c_q g_q,  rho0 = 1 (incompressible form),
 *   u   = (j + F/2) / (1 + alpha/2)          (implicit Brinkman, half force),
 *   F_n = F - alpha u                        (Brinkman-damped body force),
 *   e_q = w_q (rho + 3 c_q.u + 9/2 (c_q.u)^2 - 3/2 u.u),
 *   f*_q = g_q - w+ (g+_q - e+_q) - w- (g-_q - e-_q) + (1 - w-/2) 3 w_q c_q.F_n,
 *   with x+_q = (x_q + x_opp(q))/2, x-_q = (x_q - x_opp(q))/2.
 *
 * Velocity set: 0 rest; 1..6 axis (+x,-x,+y,-y,+z,-z); 7..18 face
 * diagonals; opp(q) = q+1 for odd q, q-1 for even q > 0.
 * Layouts: flags[z][y][x] (x fastest), 0 fluid / 1 solid; dense PDFs
 * f[q][z][y][x]; sparse PDFs f[q*N + n]; adjacency adj[(i-1)*N + n].
 *
 * Parity pins (tests): exact mass and momentum balance of one collision,
 * equilibrium moments, plane Poiseuille exact at Lambda = 3/16, square duct
 * second-order convergence, uniform acceleration, mirror symmetry, Morton
 * order by octant recursion, blocking-factor invariants, adjoint against
 * central finite differences of the forward solver.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

static const int CQ[19][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static double weight(int q) {
  if (q == 0) return 1.0 / 3.0;
  if (q <= 6) return 1.0 / 18.0;
  return 1.0 / 36.0;
}

static int opposite(int q) {
  if (q == 0) return 0;
  return (q % 2 == 1) ? q + 1 : q - 1;
}

void oracle_velocity_set(int32_t* c /* [19][3] */, double* w /* [19] */, int32_t* opp /* [19] */) {
  for (int q = 0; q < 19; ++q) {
    for (int k = 0; k < 3; ++k) c[3 * q + k] = CQ[q][k];
    w[q] = weight(q);
    opp[q] = opposite(q);
  }
}

/* ------------------------------------------------------------------------
 * Numbering schemes I(x, y, z) (Sec. 3, "Numbering scheme").
 * kind 0: lexicographic, x fastest.
 * kind 1: lexicographic with blocking: blocks of bx*by*bz cells visited
 *         lexicographically, cells inside a block lexicographically; edge
 *         blocks are clipped (the key leaves gaps, which only matter for
 *         order).  Blocking factor 1 equals plain lexicographic order.
 * kind 2: Z curve, 1-bit interleave: key bit 3k = x_k, 3k+1 = y_k,
 *         3k+2 = z_k.
 * kind 3: Z curve, 2-bit interleave: key bits 6k..6k+1 = x bits 2k..2k+1,
 *         6k+2..6k+3 = y bits 2k..2k+1, 6k+4..6k+5 = z bits 2k..2k+1.
 * kind 4: Hilbert curve over the enclosing 2^b cube (b bits per axis, the
 *         smallest b with 2^b >= every dimension), computed with Skilling's
 *         transform ("Programming the Hilbert curve", AIP Conf. Proc. 707,
 *         2004): coordinates -> "transposed" index by undoing the excess
 *         rotations/reflections level by level and Gray-encoding, then the
 *         index bits read level by level in the order x, y, z.
 */
static int hilbert_bits(const int32_t dims[3]) {
  int b = 1;
  for (int k = 0; k < 3; ++k)
    while ((1ll << b) < dims[k]) ++b;
  return b;
}

static uint64_t hilbert_key(int bits, int64_t x, int64_t y, int64_t z) {
  uint64_t X[3] = {(uint64_t)x, (uint64_t)y, (uint64_t)z};
  const uint64_t top = 1ull << (bits - 1);
  /* undo the excess work of the recursive construction, top level down */
  for (uint64_t q = top; q > 1; q >>= 1) {
    const uint64_t p = q - 1;
    for (int i = 0; i < 3; ++i) {
      if (X[i] & q) {
        X[0] ^= p; /* invert the low bits of x */
      } else {
        const uint64_t t = (X[0] ^ X[i]) & p; /* exchange low bits of x and X[i] */
        X[0] ^= t;
        X[i] ^= t;
      }
    }
  }
  /* Gray encode */
  for (int i = 1; i < 3; ++i) X[i] ^= X[i - 1];
  uint64_t t = 0;
  for (uint64_t q = top; q > 1; q >>= 1)
    if (X[2] & q) t ^= q - 1;
  for (int i = 0; i < 3; ++i) X[i] ^= t;
  /* read the transposed index: level by level, x then y then z */
  uint64_t key = 0;
  for (int lvl = bits - 1; lvl >= 0; --lvl)
    for (int i = 0; i < 3; ++i) key = (key << 1) | ((X[i] >> lvl) & 1ull);
  return key;
}

uint64_t oracle_key(int32_t kind, const int32_t dims[3], const int32_t block[3], int64_t x,
                    int64_t y, int64_t z) {
  const int64_t nx = dims[0], ny = dims[1];
  if (kind == 0) return (uint64_t)(x + nx * (y + ny * z));
  if (kind == 4) return hilbert_key(hilbert_bits(dims), x, y, z);
  if (kind == 1) {
    const int64_t bx = block[0], by = block[1], bz = block[2];
    const int64_t nbx = (dims[0] + bx - 1) / bx, nby = (dims[1] + by - 1) / by;
    const int64_t blk = (x / bx) + nbx * ((y / by) + nby * (z / bz));
    const int64_t loc = (x % bx) + bx * ((y % by) + by * (z % bz));
    return (uint64_t)(blk * (bx * by * bz) + loc);
  }
  uint64_t key = 0;
  const uint64_t p[3] = {(uint64_t)x, (uint64_t)y, (uint64_t)z};
  if (kind == 2) {
    for (int bit = 0; bit < 21; ++bit)
      for (int k = 0; k < 3; ++k) key |= ((p[k] >> bit) & 1ull) << (3 * bit + k);
    return key;
  }
  /* kind == 3 */
  for (int grp = 0; grp < 10; ++grp)
    for (int k = 0; k < 3; ++k) key |= ((p[k] >> (2 * grp)) & 3ull) << (6 * grp + 2 * k);
  return key;
}

typedef struct {
  uint64_t key;
  int64_t cell;
} keyed_t;

static int cmp_keyed(const void* a, const void* b) {
  const keyed_t* x = (const keyed_t*)a;
  const keyed_t* y = (const keyed_t*)b;
  if (x->key < y->key) return -1;
  if (x->key > y->key) return 1;
  return (x->cell < y->cell) ? -1 : (x->cell > y->cell);
}

int64_t oracle_count_fluid(const uint8_t* flags, const int32_t dims[3]) {
  const int64_t box = (int64_t)dims[0] * dims[1] * dims[2];
  int64_t n = 0;
  for (int64_t c = 0; c < box; ++c) n += flags[c] == 0;
  return n;
}

/* Source cell of the pull along direction q at (x,y,z): x - c_q, wrapped on
 * periodic axes.  Returns -1 outside a closed face. */
static int64_t pull_source(const int32_t dims[3], uint32_t periodic, int64_t x, int64_t y,
                           int64_t z, int q) {
  int64_t s[3] = {x - CQ[q][0], y - CQ[q][1], z - CQ[q][2]};
  for (int k = 0; k < 3; ++k) {
    if (s[k] < 0 || s[k] >= dims[k]) {
      if (!((periodic >> k) & 1u)) return -1;
      s[k] = (s[k] % dims[k] + dims[k]) % dims[k];
    }
  }
  return s[0] + (int64_t)dims[0] * (s[1] + (int64_t)dims[1] * s[2]);
}

/*
 * The sparse representation (Sec. 2-3): cells[n] = linear box index of the
 * fluid cell with contiguous index I_c = n + 1 (fluid cells sorted by the
 * numbering scheme), inv[box] = n or -1 for solids, and the pull adjacency
 * adj[(i-1)*N + n] (i = 1..18) = q*N + m with q = i when the source cell m is
 * fluid, or opp(i)*N + n (implicit bounce back) when it is solid or lies
 * beyond a closed face.  Returns N, or -1 on bad input.
 */
int64_t oracle_build_sparse(const uint8_t* flags, const int32_t dims[3], int32_t kind,
                            const int32_t block[3], uint32_t periodic, int32_t* cells,
                            int32_t* inv, int32_t* adj) {
  const int64_t box = (int64_t)dims[0] * dims[1] * dims[2];
  const int64_t n = oracle_count_fluid(flags, dims);
  keyed_t* list = (keyed_t*)malloc(sizeof(keyed_t) * (size_t)(n > 0 ? n : 1));
  if (!list) return -1;
  int64_t k = 0;
  for (int64_t z = 0; z < dims[2]; ++z)
    for (int64_t y = 0; y < dims[1]; ++y)
      for (int64_t x = 0; x < dims[0]; ++x) {
        const int64_t c = x + dims[0] * (y + dims[1] * z);
        if (flags[c] != 0) continue;
        list[k].key = oracle_key(kind, dims, block, x, y, z);
        list[k].cell = c;
        ++k;
      }
  qsort(list, (size_t)n, sizeof(keyed_t), cmp_keyed);
  for (int64_t c = 0; c < box; ++c) inv[c] = -1;
  for (int64_t i = 0; i < n; ++i) {
    cells[i] = (int32_t)list[i].cell;
    inv[list[i].cell] = (int32_t)i;
  }
  free(list);
  if (adj) {
    for (int64_t i = 0; i < n; ++i) {
      const int64_t c = cells[i];
      const int64_t x = c % dims[0], y = (c / dims[0]) % dims[1], z = c / ((int64_t)dims[0] * dims[1]);
      for (int q = 1; q < 19; ++q) {
        const int64_t s = pull_source(dims, periodic, x, y, z, q);
        int64_t slot;
        if (s >= 0 && flags[s] == 0)
          slot = (int64_t)q * n + inv[s];
        else
          slot = (int64_t)opposite(q) * n + i;
        adj[(int64_t)(q - 1) * n + i] = (int32_t)slot;
      }
    }
  }
  return n;
}

/* ------------------------------------------------------------------------
 * One TRT collision of a cell (Sec. 1: TRT on D3Q19; formulas in the header
 * comment).  g = pulled (post-stream) PDFs, F = body force, alpha = Brinkman
 * damping of the cell.  Writes f* and the cell's rho and u. */
void oracle_collide(const double g[19], const double F[3], double alpha, double omega_p,
                    double omega_m, double fout[19], double* rho_out, double u_out[3]) {
  double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
  for (int q = 0; q < 19; ++q) {
    rho += g[q];
    for (int k = 0; k < 3; ++k) j[k] += CQ[q][k] * g[q];
  }
  double u[3], Fn[3];
  for (int k = 0; k < 3; ++k) u[k] = (j[k] + 0.5 * F[k]) / (1.0 + 0.5 * alpha);
  for (int k = 0; k < 3; ++k) Fn[k] = F[k] - alpha * u[k];
  const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  double e[19];
  for (int q = 0; q < 19; ++q) {
    const double cu = CQ[q][0] * u[0] + CQ[q][1] * u[1] + CQ[q][2] * u[2];
    e[q] = weight(q) * (rho + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
  }
  for (int q = 0; q < 19; ++q) {
    const int o = opposite(q);
    const double gp = 0.5 * (g[q] + g[o]), gm = 0.5 * (g[q] - g[o]);
    const double ep = 0.5 * (e[q] + e[o]), em = 0.5 * (e[q] - e[o]);
    const double cF = CQ[q][0] * Fn[0] + CQ[q][1] * Fn[1] + CQ[q][2] * Fn[2];
    fout[q] = g[q] - omega_p * (gp - ep) - omega_m * (gm - em) +
              (1.0 - 0.5 * omega_m) * 3.0 * weight(q) * cF;
  }
  if (rho_out) *rho_out = rho;
  if (u_out)
    for (int k = 0; k < 3; ++k) u_out[k] = u[k];
}

/* Pull of the 19 PDFs of fluid cell (x,y,z) from the dense grid f[q][box]:
 * from the source cell when it is fluid, else the cell's own opposite PDF
 * (half-way bounce back; Sec. 2). */
static void pull_dense(const uint8_t* flags, const int32_t dims[3], uint32_t periodic,
                       const double* f, int64_t box, int64_t x, int64_t y, int64_t z,
                       double g[19]) {
  const int64_t c = x + (int64_t)dims[0] * (y + (int64_t)dims[1] * z);
  g[0] = f[c];
  for (int q = 1; q < 19; ++q) {
    const int64_t s = pull_source(dims, periodic, x, y, z, q);
    if (s >= 0 && flags[s] == 0)
      g[q] = f[(int64_t)q * box + s];
    else
      g[q] = f[(int64_t)opposite(q) * box + c];
  }
}

/* Rest state f_q = w_q * rho0 (rho0 = 1) on fluid cells, 0 on solids. */
void oracle_rest_state(const uint8_t* flags, const int32_t dims[3], double* f) {
  const int64_t box = (int64_t)dims[0] * dims[1] * dims[2];
  for (int q = 0; q < 19; ++q)
    for (int64_t c = 0; c < box; ++c) f[(int64_t)q * box + c] = flags[c] == 0 ? weight(q) : 0.0;
}

/*
 * n_steps full time steps on the dense grid (pull then collide, two grids
 * swapped; Sec. 7).  f (dense [19][box]) is the state in and out.  alpha is
 * a dense [box] field or NULL (no damping).  If obs != NULL, obs[4*t + 0..3]
 * receive sum rho, sum u_x, sum u_y, sum u_z over fluid cells of the
 * collision of step t+1.  If rho_last / u_last (dense [box], [3][box]) are
 * given they receive the per-cell moments of the last step's collision.
 */
int oracle_run(const uint8_t* flags, const int32_t dims[3], uint32_t periodic, double omega_p,
               double omega_m, const double F[3], const double* alpha, int32_t n_steps,
               double* f, double* obs, double* rho_last, double* u_last) {
  const int64_t box = (int64_t)dims[0] * dims[1] * dims[2];
  double* tmp = (double*)malloc(sizeof(double) * 19 * (size_t)box);
  if (!tmp) return -1;
  double* src = f;
  double* dst = tmp;
  for (int64_t i = 0; i < 19 * box; ++i) dst[i] = src[i];
  for (int32_t t = 0; t < n_steps; ++t) {
    const int last = t == n_steps - 1;
    double s_rho = 0.0, s_ux = 0.0, s_uy = 0.0, s_uz = 0.0;
#pragma omp parallel for collapse(2) schedule(static) reduction(+ : s_rho, s_ux, s_uy, s_uz)
    for (int64_t z = 0; z < dims[2]; ++z)
      for (int64_t y = 0; y < dims[1]; ++y)
        for (int64_t x = 0; x < dims[0]; ++x) {
          const int64_t c = x + (int64_t)dims[0] * (y + (int64_t)dims[1] * z);
          if (flags[c] != 0) continue;
          double g[19], fo[19], rho, u[3];
          pull_dense(flags, dims, periodic, src, box, x, y, z, g);
          oracle_collide(g, F, alpha ? alpha[c] : 0.0, omega_p, omega_m, fo, &rho, u);
          for (int q = 0; q < 19; ++q) dst[(int64_t)q * box + c] = fo[q];
          s_rho += rho;
          s_ux += u[0];
          s_uy += u[1];
          s_uz += u[2];
          if (last && rho_last) rho_last[c] = rho;
          if (last && u_last)
            for (int k = 0; k < 3; ++k) u_last[(int64_t)k * box + c] = u[k];
        }
    if (obs) {
      obs[4 * t + 0] = s_rho;
      obs[4 * t + 1] = s_ux;
      obs[4 * t + 2] = s_uy;
      obs[4 * t + 3] = s_uz;
    }
    double* sw = src;
    src = dst;
    dst = sw;
  }
  if (src != f)
    for (int64_t i = 0; i < 19 * box; ++i) f[i] = src[i];
  free(tmp);
  return 0;
}

/* ------------------------------------------------------------------------
 * Adjoint.  Forward: f_0 given; for t = 1..K: g_t = S f_{t-1} (pull),
 * f_t = C(g_t; F, alpha).  Objective: J = (1/N) sum_n u_axis(g_K)_n, the
 * mean axial velocity of the collision of step K.  Reverse mode:
 *   lam_g_K = dJ/dg_K;  lam_f_{t-1} = S^T lam_g_t;
 *   lam_g_t = (dC/dg(g_t))^T lam_f_t  for t = K-1 .. 1,
 * with dJ/dF and dJ/dalpha accumulated from every step's dC/dF, dC/dalpha
 * and from the direct dependence of J on F and alpha.
 */

/* Jacobian of one collision: Jg[q][r] = d f*_q / d g_r, JF[q][k] =
 * d f*_q / d F_k, Ja[q] = d f*_q / d alpha. */
static void collide_jacobian(const double g[19], const double F[3], double alpha,
                             double omega_p, double omega_m, double Jg[19][19],
                             double JF[19][3], double Ja[19]) {
  double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
  for (int q = 0; q < 19; ++q) {
    rho += g[q];
    for (int k = 0; k < 3; ++k) j[k] += CQ[q][k] * g[q];
  }
  const double s = 1.0 / (1.0 + 0.5 * alpha);
  double u[3];
  for (int k = 0; k < 3; ++k) u[k] = (j[k] + 0.5 * F[k]) * s;
  /* derivatives of u: du_k/dg_r = c_rk s; du_k/dF_m = delta_km s/2;
   * du_k/dalpha = -u_k s / 2 */
  double du_dg[19][3], du_dF[3][3], du_da[3];
  for (int r = 0; r < 19; ++r)
    for (int k = 0; k < 3; ++k) du_dg[r][k] = CQ[r][k] * s;
  for (int m = 0; m < 3; ++m)
    for (int k = 0; k < 3; ++k) du_dF[m][k] = (k == m) ? 0.5 * s : 0.0;
  for (int k = 0; k < 3; ++k) du_da[k] = -0.5 * u[k] * s;
  /* de_q/du_k = w_q (3 c_qk + 9 (c_q.u) c_qk - 3 u_k); de_q/drho = w_q */
  double de_du[19][3];
  for (int q = 0; q < 19; ++q) {
    const double cu = CQ[q][0] * u[0] + CQ[q][1] * u[1] + CQ[q][2] * u[2];
    for (int k = 0; k < 3; ++k)
      de_du[q][k] = weight(q) * (3.0 * CQ[q][k] + 9.0 * cu * CQ[q][k] - 3.0 * u[k]);
  }
  for (int q = 0; q < 19; ++q) {
    const int o = opposite(q);
    const double src = (1.0 - 0.5 * omega_m) * 3.0 * weight(q);
    /* with respect to g_r */
    for (int r = 0; r < 19; ++r) {
      double de_q = weight(q), de_o = weight(o); /* drho/dg_r = 1 */
      for (int k = 0; k < 3; ++k) {
        de_q += de_du[q][k] * du_dg[r][k];
        de_o += de_du[o][k] * du_dg[r][k];
      }
      const double dgp = 0.5 * ((q == r) + (o == r)), dgm = 0.5 * ((q == r) - (o == r));
      const double dep = 0.5 * (de_q + de_o), dem = 0.5 * (de_q - de_o);
      double dcF = 0.0; /* dF_n/dg_r = -alpha du/dg_r */
      for (int k = 0; k < 3; ++k) dcF += CQ[q][k] * (-alpha * du_dg[r][k]);
      Jg[q][r] = (q == r) - omega_p * (dgp - dep) - omega_m * (dgm - dem) + src * dcF;
    }
    /* with respect to F_m */
    for (int m = 0; m < 3; ++m) {
      double de_q = 0.0, de_o = 0.0;
      for (int k = 0; k < 3; ++k) {
        de_q += de_du[q][k] * du_dF[m][k];
        de_o += de_du[o][k] * du_dF[m][k];
      }
      const double dep = 0.5 * (de_q + de_o), dem = 0.5 * (de_q - de_o);
      double dcF = 0.0; /* dF_n/dF_m = e_m - alpha du/dF_m */
      for (int k = 0; k < 3; ++k) dcF += CQ[q][k] * (((k == m) ? 1.0 : 0.0) - alpha * du_dF[m][k]);
      JF[q][m] = omega_p * dep + omega_m * dem + src * dcF;
    }
    /* with respect to alpha */
    {
      double de_q = 0.0, de_o = 0.0;
      for (int k = 0; k < 3; ++k) {
        de_q += de_du[q][k] * du_da[k];
        de_o += de_du[o][k] * du_da[k];
      }
      const double dep = 0.5 * (de_q + de_o), dem = 0.5 * (de_q - de_o);
      double dcF = 0.0; /* dF_n/dalpha = -u - alpha du/dalpha */
      for (int k = 0; k < 3; ++k) dcF += CQ[q][k] * (-u[k] - alpha * du_da[k]);
      Ja[q] = omega_p * dep + omega_m * dem + src * dcF;
    }
  }
}

/*
 * Gradient of J = (1/N) sum_n u_axis(g_K)_n with respect to the force F
 * (dJdF[3]), the damping field (dJdalpha, dense [box], zero on solids) and
 * the initial state (lam0, dense [19][box], zero on solids; may be NULL).
 * f0 is the dense initial state.  Stores all K states (small cases only).
 * Also returns J.
 */
int oracle_adjoint(const uint8_t* flags, const int32_t dims[3], uint32_t periodic,
                   double omega_p, double omega_m, const double F[3], const double* alpha,
                   int32_t n_steps, int32_t axis, const double* f0, double* J_out,
                   double* dJdF, double* dJdalpha, double* lam0) {
  const int64_t box = (int64_t)dims[0] * dims[1] * dims[2];
  const int64_t nf = oracle_count_fluid(flags, dims);
  if (n_steps < 1 || nf <= 0 || axis < 0 || axis > 2) return -1;
  const int K = n_steps;
  /* states f_0 .. f_{K-1} */
  double* states = (double*)malloc(sizeof(double) * 19 * (size_t)box * (size_t)K);
  double* lam_f = (double*)calloc(19 * (size_t)box, sizeof(double));
  double* lam_g = (double*)calloc(19 * (size_t)box, sizeof(double));
  if (!states || !lam_f || !lam_g) {
    free(states); free(lam_f); free(lam_g);
    return -1;
  }
  memcpy(states, f0, sizeof(double) * 19 * (size_t)box);
  for (int t = 1; t < K; ++t) {
    double* cur = states + (size_t)t * 19 * (size_t)box;
    memcpy(cur, cur - 19 * box, sizeof(double) * 19 * (size_t)box);
    if (oracle_run(flags, dims, periodic, omega_p, omega_m, F, alpha, 1, cur, NULL, NULL, NULL))
      return -1;
  }
  for (int k = 0; k < 3; ++k) dJdF[k] = 0.0;
  for (int64_t c = 0; c < box; ++c) dJdalpha[c] = 0.0;

  /* seed: dJ/dg_K and the direct terms, from f_{K-1} */
  double J = 0.0;
  {
    const double* fprev = states + (size_t)(K - 1) * 19 * (size_t)box;
    for (int64_t z = 0; z < dims[2]; ++z)
      for (int64_t y = 0; y < dims[1]; ++y)
        for (int64_t x = 0; x < dims[0]; ++x) {
          const int64_t c = x + (int64_t)dims[0] * (y + (int64_t)dims[1] * z);
          if (flags[c] != 0) continue;
          double g[19], fo[19], rho, u[3];
          pull_dense(flags, dims, periodic, fprev, box, x, y, z, g);
          const double a = alpha ? alpha[c] : 0.0;
          oracle_collide(g, F, a, omega_p, omega_m, fo, &rho, u);
          const double s = 1.0 / (1.0 + 0.5 * a);
          J += u[axis] / (double)nf;
          for (int q = 0; q < 19; ++q) lam_g[(int64_t)q * box + c] = CQ[q][axis] * s / (double)nf;
          dJdF[axis] += 0.5 * s / (double)nf;
          dJdalpha[c] += -0.5 * u[axis] * s / (double)nf;
        }
  }
  for (int t = K - 1; t >= 0; --t) {
    /* lam_f_t = S^T lam_g_{t+1}: every pulled value sends its adjoint back
     * to the slot it was read from */
    memset(lam_f, 0, sizeof(double) * 19 * (size_t)box);
    for (int64_t z = 0; z < dims[2]; ++z)
      for (int64_t y = 0; y < dims[1]; ++y)
        for (int64_t x = 0; x < dims[0]; ++x) {
          const int64_t c = x + (int64_t)dims[0] * (y + (int64_t)dims[1] * z);
          if (flags[c] != 0) continue;
          lam_f[c] += lam_g[c];
          for (int q = 1; q < 19; ++q) {
            const int64_t s = pull_source(dims, periodic, x, y, z, q);
            if (s >= 0 && flags[s] == 0)
              lam_f[(int64_t)q * box + s] += lam_g[(int64_t)q * box + c];
            else
              lam_f[(int64_t)opposite(q) * box + c] += lam_g[(int64_t)q * box + c];
          }
        }
    if (t == 0) break;
    /* lam_g_t = (dC/dg(g_t))^T lam_f_t, g_t = S f_{t-1} */
    const double* fprev = states + (size_t)(t - 1) * 19 * (size_t)box;
    for (int64_t z = 0; z < dims[2]; ++z)
      for (int64_t y = 0; y < dims[1]; ++y)
        for (int64_t x = 0; x < dims[0]; ++x) {
          const int64_t c = x + (int64_t)dims[0] * (y + (int64_t)dims[1] * z);
          if (flags[c] != 0) continue;
          double g[19], Jg[19][19], JF[19][3], Ja[19], lf[19];
          pull_dense(flags, dims, periodic, fprev, box, x, y, z, g);
          const double a = alpha ? alpha[c] : 0.0;
          collide_jacobian(g, F, a, omega_p, omega_m, Jg, JF, Ja);
          for (int q = 0; q < 19; ++q) lf[q] = lam_f[(int64_t)q * box + c];
          for (int r = 0; r < 19; ++r) {
            double acc = 0.0;
            for (int q = 0; q < 19; ++q) acc += Jg[q][r] * lf[q];
            lam_g[(int64_t)r * box + c] = acc;
          }
          for (int k = 0; k < 3; ++k)
            for (int q = 0; q < 19; ++q) dJdF[k] += JF[q][k] * lf[q];
          for (int q = 0; q < 19; ++q) dJdalpha[c] += Ja[q] * lf[q];
        }
  }
  if (lam0) memcpy(lam0, lam_f, sizeof(double) * 19 * (size_t)box);
  if (J_out) *J_out = J;
  free(states);
  free(lam_f);
  free(lam_g);
  return 0;
}

/* Numbering-scheme key of every box cell, keys[x + nx*(y + ny*z)]. */
void oracle_keys(int32_t kind, const int32_t dims[3], const int32_t block[3], uint64_t* keys) {
  for (int64_t z = 0; z < dims[2]; ++z)
    for (int64_t y = 0; y < dims[1]; ++y)
      for (int64_t x = 0; x < dims[0]; ++x)
        keys[x + (int64_t)dims[0] * (y + (int64_t)dims[1] * z)] =
            oracle_key(kind, dims, block, x, y, z);
}

/* One time step on the sparse representation (Sec. 2 and Sec. 7): each of
 * the n cells pulls g_0 = f_src[i] and g_q = f_src[adj[(q-1)*n + i]], then
 * collides; f_dst[q*n + i] = f*_q.  f_src may be longer than 19 n (for
 * example a rank's ghost cells after its own PDFs); adj entries index it.
 * alpha: per-cell damping [n] or NULL.  Used to emulate the ranks of a
 * chunked run; pinned against the dense pull solver by the tests. */
void oracle_sparse_step(const double* f_src, double* f_dst, const int32_t* adj, int64_t n,
                        const double F[3], const double* alpha, double omega_p,
                        double omega_m) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double g[19], fo[19];
    g[0] = f_src[i];
    for (int q = 1; q < 19; ++q) g[q] = f_src[adj[(int64_t)(q - 1) * n + i]];
    oracle_collide(g, F, alpha ? alpha[i] : 0.0, omega_p, omega_m, fo, NULL, NULL);
    for (int q = 0; q < 19; ++q) f_dst[(int64_t)q * n + i] = fo[q];
  }
}
