/*
 * Seeded synthetic inputs: voxelised packed beds (a tube filled with spheres
 * by random sequential addition) and per-cell random fields.
 *
 * These stand in for the paper's benchmark geometries, the "channel" (an
 * empty tube) and the "packing" (a tube filled with spheres) of size
 * (5d) x d x d (Sec. 6, Fig. 2), whose files are not available.  The module
 * holds no lattice Boltzmann arithmetic: it only decides which voxels are
 * solid and draws uniform random numbers, and both the CPU oracle and the
 * CUDA path consume what it writes.
 *
 * Random numbers come from a counter-based generator: SplitMix64 (Steele,
 * Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA
 * 2014), applied to a hash of (seed, stream, counter).  It uses only 64-bit
 * integer arithmetic, so x86-64 and AArch64 hosts draw the same numbers.
 * Build with -ffp-contract=off so that no host fuses a*b+c differently.
 *
 * Flags layout: uint8 flags[z][y][x] (x fastest), 0 = fluid, 1 = solid.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

static uint64_t sm64_mix(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Uniform double in [0, 1) with 53 random bits for draw `counter` of
 * `stream` under `seed`. */
double pb_uniform(uint64_t seed, uint64_t stream, uint64_t counter) {
  uint64_t key = sm64_mix(seed ^ sm64_mix(stream + 0x5851F42D4C957F2Dull));
  uint64_t r = sm64_mix(key + counter * 0x9E3779B97F4A7C15ull);
  return (double)(r >> 11) * (1.0 / 9007199254740992.0);
}

/* out[i] = lo + (hi - lo) * U(seed, stream, i) for i in [0, n). */
void pb_uniform_field(int64_t n, uint64_t seed, uint64_t stream, double lo, double hi,
                      double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = lo + (hi - lo) * pb_uniform(seed, stream, (uint64_t)i);
}

typedef struct {
  double c[3];
} sphere_t;

static int64_t imax64(int64_t a, int64_t b) { return a > b ? a : b; }

/*
 * Tube of diameter tube_d along `axis` (0 = x, 1 = y, 2 = z), centred in the
 * cross-section, periodic along that axis, filled by random sequential
 * addition of non-overlapping spheres of radius `radius`:
 *   - a candidate centre is uniform along the axis and uniform in the tube's
 *     cross-section disc (spheres may cut the tube wall);
 *   - it is rejected if it lies closer than 2*radius to an accepted centre
 *     (minimum image along the periodic axis);
 *   - addition stops once the box porosity (fluid cells / box cells) is at or
 *     below target_porosity, or after max_rejects consecutive rejections.
 * A cell is fluid iff its centre (i + 1/2) lies inside the tube and outside
 * every sphere.  tube_d <= 0 means "no tube" (the whole box is the fluid
 * region, spheres uniform in the box); radius <= 0 means no spheres.
 * Returns 0 on success, -1 on bad arguments, -2 on allocation failure.
 */
int pb_packed_bed(int32_t nx, int32_t ny, int32_t nz, int32_t axis, double tube_d,
                  double radius, double target_porosity, int64_t max_rejects, uint64_t seed,
                  uint8_t* flags, int64_t* n_spheres_out, int64_t* n_fluid_out) {
  if (nx <= 0 || ny <= 0 || nz <= 0 || axis < 0 || axis > 2 || !flags) return -1;
  const int64_t dims[3] = {nx, ny, nz};
  const int64_t box = dims[0] * dims[1] * dims[2];
  const int a0 = axis, a1 = (axis + 1) % 3, a2 = (axis + 2) % 3;
  const double cu = 0.5 * (double)dims[a1], cv = 0.5 * (double)dims[a2];
  const double tr = 0.5 * tube_d;
  const int have_tube = tube_d > 0.0;

  int64_t n_fluid = 0;
  for (int64_t z = 0; z < nz; ++z)
    for (int64_t y = 0; y < ny; ++y)
      for (int64_t x = 0; x < nx; ++x) {
        const int64_t p[3] = {x, y, z};
        int fluid = 1;
        if (have_tube) {
          const double du = (double)p[a1] + 0.5 - cu, dv = (double)p[a2] + 0.5 - cv;
          fluid = du * du + dv * dv < tr * tr;
        }
        flags[x + nx * (y + ny * z)] = fluid ? 0 : 1;
        n_fluid += fluid;
      }

  int64_t n_spheres = 0;
  if (radius > 0.0 && box > 0) {
    /* Hash grid of bin edge >= 2r: an overlapping centre lies in a
     * neighbouring bin. */
    const double r = radius, d2min = 4.0 * r * r;
    int64_t nb[3];
    for (int k = 0; k < 3; ++k) {
      nb[k] = (int64_t)floor((double)dims[k] / (2.0 * r));
      if (nb[k] < 1) nb[k] = 1;
    }
    const int64_t nbins = nb[0] * nb[1] * nb[2];
    int64_t* head = (int64_t*)malloc(sizeof(int64_t) * (size_t)nbins);
    int64_t cap = 1024, *next = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
    sphere_t* sp = (sphere_t*)malloc(sizeof(sphere_t) * (size_t)cap);
    if (!head || !next || !sp) {
      free(head); free(next); free(sp);
      return -2;
    }
    for (int64_t b = 0; b < nbins; ++b) head[b] = -1;

    uint64_t counter = 0;
    int64_t rejects = 0;
    const int64_t attempt_cap = imax64(1000000000LL, 100 * max_rejects);
    for (int64_t attempt = 0; attempt < attempt_cap; ++attempt) {
      if ((double)n_fluid <= target_porosity * (double)box) break;
      if (rejects >= max_rejects) break;
      double c[3];
      c[a0] = pb_uniform(seed, 1, counter++) * (double)dims[a0];
      if (have_tube) {
        double du, dv;
        do {
          du = (2.0 * pb_uniform(seed, 1, counter++) - 1.0) * tr;
          dv = (2.0 * pb_uniform(seed, 1, counter++) - 1.0) * tr;
        } while (du * du + dv * dv >= tr * tr);
        c[a1] = cu + du;
        c[a2] = cv + dv;
      } else {
        c[a1] = pb_uniform(seed, 1, counter++) * (double)dims[a1];
        c[a2] = pb_uniform(seed, 1, counter++) * (double)dims[a2];
      }
      /* overlap test against the neighbouring bins */
      int64_t bc[3];
      for (int k = 0; k < 3; ++k) {
        bc[k] = (int64_t)floor(c[k] / (double)dims[k] * (double)nb[k]);
        if (bc[k] < 0) bc[k] = 0;
        if (bc[k] >= nb[k]) bc[k] = nb[k] - 1;
      }
      int overlap = 0;
      for (int64_t o2 = -1; o2 <= 1 && !overlap; ++o2)
        for (int64_t o1 = -1; o1 <= 1 && !overlap; ++o1)
          for (int64_t o0 = -1; o0 <= 1 && !overlap; ++o0) {
            const int64_t off[3] = {o0, o1, o2};
            int64_t bb[3];
            int skip = 0;
            for (int k = 0; k < 3; ++k) {
              bb[k] = bc[k] + off[k];
              if (k == a0) {
                bb[k] = ((bb[k] % nb[k]) + nb[k]) % nb[k];
              } else if (bb[k] < 0 || bb[k] >= nb[k]) {
                skip = 1;
              }
            }
            if (skip) continue;
            /* with fewer than three bins along the axis, wrapped offsets
             * revisit a bin; visiting it twice is harmless */
            for (int64_t s = head[bb[0] + nb[0] * (bb[1] + nb[1] * bb[2])]; s >= 0; s = next[s]) {
              double d2 = 0.0;
              for (int k = 0; k < 3; ++k) {
                double d = c[k] - sp[s].c[k];
                if (k == a0) {
                  const double L = (double)dims[k];
                  d = d - L * floor(d / L + 0.5);
                }
                d2 += d * d;
              }
              if (d2 < d2min) { overlap = 1; break; }
            }
          }
      if (overlap) { ++rejects; continue; }
      rejects = 0;
      if (n_spheres == cap) {
        cap *= 2;
        int64_t* nn = (int64_t*)realloc(next, sizeof(int64_t) * (size_t)cap);
        if (!nn) { free(head); free(next); free(sp); return -2; }
        next = nn;
        sphere_t* ns = (sphere_t*)realloc(sp, sizeof(sphere_t) * (size_t)cap);
        if (!ns) { free(head); free(next); free(sp); return -2; }
        sp = ns;
      }
      for (int k = 0; k < 3; ++k) sp[n_spheres].c[k] = c[k];
      const int64_t bin = bc[0] + nb[0] * (bc[1] + nb[1] * bc[2]);
      next[n_spheres] = head[bin];
      head[bin] = n_spheres;
      ++n_spheres;
      /* stamp the sphere: cells whose centre lies strictly inside */
      int64_t lo[3], hi[3];
      for (int k = 0; k < 3; ++k) {
        lo[k] = (int64_t)floor(c[k] - r - 1.0);
        hi[k] = (int64_t)ceil(c[k] + r + 1.0);
        if (k != a0) {
          if (lo[k] < 0) lo[k] = 0;
          if (hi[k] > dims[k] - 1) hi[k] = dims[k] - 1;
        } else if (hi[k] - lo[k] + 1 > dims[k]) {
          hi[k] = lo[k] + dims[k] - 1;
        }
      }
      for (int64_t q2 = lo[2]; q2 <= hi[2]; ++q2)
        for (int64_t q1 = lo[1]; q1 <= hi[1]; ++q1)
          for (int64_t q0 = lo[0]; q0 <= hi[0]; ++q0) {
            const int64_t q[3] = {q0, q1, q2};
            double d2 = 0.0;
            int64_t w[3];
            for (int k = 0; k < 3; ++k) {
              double d = (double)q[k] + 0.5 - c[k];
              w[k] = q[k];
              if (k == a0) {
                const double L = (double)dims[k];
                d = d - L * floor(d / L + 0.5);
                w[k] = ((q[k] % dims[k]) + dims[k]) % dims[k];
              }
              d2 += d * d;
            }
            if (d2 < r * r) {
              uint8_t* f = &flags[w[0] + dims[0] * (w[1] + dims[1] * w[2])];
              if (*f == 0) { *f = 1; --n_fluid; }
            }
          }
    }
    free(head);
    free(next);
    free(sp);
  }
  if (n_spheres_out) *n_spheres_out = n_spheres;
  if (n_fluid_out) *n_fluid_out = n_fluid;
  return 0;
}
