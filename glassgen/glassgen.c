/*
 * glassgen.c -- seeded synthetic binary-glass spring networks (input generator).
 *
 * This module produces INPUTS only: atom positions, types, masses and the bond list
 * (i, j, k_ij, unit vector r_hat_ij).  It holds none of the eigensolver's arithmetic:
 * neither the Hessian assembly (Delta blocks, mass weighting) nor anything of the filter.
 * Both the CPU oracle and the GPU library consume its output, each assembling H on its own.
 *
 * Workload shape (stands in for the Lennard-Jones binary glasses of the paper's Sec. 4.2,
 * whose MD structures are not available): periodic cube of side L = (N/rho)^(1/3),
 * positions by random sequential addition (RSA) with a minimum-image distance >= d_min,
 * a fraction f_A of type A (mass m_A) and the rest type B (mass m_B) assigned by a seeded
 * shuffle, bonds between every pair closer than r_c, spring constants k_ij lognormal with
 * median k_med and log-standard-deviation sigma.
 *
 * Random numbers: SplitMix64 (Steele, Lea & Flood 2014) seeds xoshiro256** (Blackman &
 * Vigna 2018); uniforms take the top 53 bits; normals come from the Box-Muller transform.
 * The order of draws is fixed: all RSA proposals, then the type shuffle, then one normal per
 * bond in (i, j) lexicographic order.
 *
 * After RSA the atoms are renumbered in Morton (Z-curve) order of r_c-sized cells so that
 * atoms close in space are close in index (what a spatially sorted MD dump looks like).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  uint64_t s[4];
} gg_rng;

static uint64_t gg_splitmix64(uint64_t *x) {
  uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

static uint64_t gg_rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static void gg_seed(gg_rng *r, uint64_t seed) {
  uint64_t x = seed;
  for (int i = 0; i < 4; ++i) r->s[i] = gg_splitmix64(&x);
}

static uint64_t gg_next(gg_rng *r) {
  uint64_t *s = r->s;
  const uint64_t result = gg_rotl(s[1] * 5, 7) * 9;
  const uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = gg_rotl(s[3], 45);
  return result;
}

/* uniform in [0, 1) with 53 random bits */
static double gg_uniform(gg_rng *r) { return (double)(gg_next(r) >> 11) * 0x1.0p-53; }

/* standard normal, Box-Muller (one of the pair; deterministic, no caching) */
static double gg_normal(gg_rng *r) {
  double u1 = 1.0 - gg_uniform(r); /* (0, 1] */
  double u2 = gg_uniform(r);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925 * u2);
}

/* per-sample sub-seed: SplitMix64 of (seed XOR index) */
uint64_t gg_subseed(uint64_t seed, uint64_t index) {
  uint64_t x = seed ^ index;
  return gg_splitmix64(&x);
}

static double gg_wrap(double d, double L) {
  /* minimum-image displacement component */
  return d - L * nearbyint(d / L);
}

static int gg_cell_of(double p, double L, int nc) {
  int c = (int)floor(p / L * nc);
  if (c < 0) c = 0;
  if (c >= nc) c = nc - 1;
  return c;
}

static uint64_t gg_spread3(uint64_t v) {
  /* spread the low 21 bits of v to every third bit */
  v &= 0x1fffffULL;
  v = (v | (v << 32)) & 0x1f00000000ffffULL;
  v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
  v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
  v = (v | (v << 2)) & 0x1249249249249249ULL;
  return v;
}

typedef struct {
  uint64_t key;
  int32_t idx;
} gg_keyed;

static int gg_cmp_keyed(const void *a, const void *b) {
  const gg_keyed *x = (const gg_keyed *)a, *y = (const gg_keyed *)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

static int gg_cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return x < y ? -1 : (x > y);
}

/*
 * Generate one glass.
 *   pos[3N], mass[N], type[N] (0 = A, 1 = B) are written by the call.
 *   bonds: up to bond_cap entries of bi[] < bj[], kk[], rhat[3*]; *nbonds receives the
 *   number found (also when it exceeds bond_cap, in which case nothing past the cap is
 *   written and the call returns -2 so that the caller can retry with a larger buffer).
 * Returns 0 on success, -1 on bad arguments, -2 bond buffer too small, -3 RSA gave up
 * (attempt cap reached: the requested packing is too close to jamming), -4 out of memory.
 */
int gg_generate(int32_t N, uint64_t seed, double rho, double d_min, double r_c, double frac_a,
                double m_a, double m_b, double k_med, double k_sigma, int spatial_sort,
                double *pos, double *mass, int32_t *type, double *box_L, int64_t bond_cap,
                int64_t *nbonds, int32_t *bi, int32_t *bj, double *kk, double *rhat) {
  if (N <= 0 || rho <= 0 || d_min < 0 || r_c <= 0 || !pos || !mass || !type || !box_L || !nbonds)
    return -1;
  const double L = cbrt((double)N / rho);
  *box_L = L;
  gg_rng rng;
  gg_seed(&rng, seed);

  /* ---- RSA with a cell list of cell size >= d_min ---- */
  int nc = (d_min > 0) ? (int)floor(L / d_min) : 1;
  if (nc < 1) nc = 1;
  if (nc > 1024) nc = 1024;
  const int64_t ncell = (int64_t)nc * nc * nc;
  int32_t *head = (int32_t *)malloc(sizeof(int32_t) * ncell);
  int32_t *next = (int32_t *)malloc(sizeof(int32_t) * N);
  double *p = (double *)malloc(sizeof(double) * 3 * (size_t)N);
  if (!head || !next || !p) {
    free(head); free(next); free(p);
    return -4;
  }
  for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
  const double dmin2 = d_min * d_min;
  const int64_t max_attempts = (int64_t)N * 100000 + 1000000;
  int64_t attempts = 0;
  int placed = 0;
  const int reach = (nc >= 3) ? 1 : 0; /* with < 3 cells per side a brute-force scan is used */
  while (placed < N) {
    if (++attempts > max_attempts) {
      free(head); free(next); free(p);
      return -3;
    }
    double x = gg_uniform(&rng) * L, y = gg_uniform(&rng) * L, z = gg_uniform(&rng) * L;
    int ok = 1;
    if (reach) {
      int cx = gg_cell_of(x, L, nc), cy = gg_cell_of(y, L, nc), cz = gg_cell_of(z, L, nc);
      for (int dz = -1; dz <= 1 && ok; ++dz)
        for (int dy = -1; dy <= 1 && ok; ++dy)
          for (int dx = -1; dx <= 1 && ok; ++dx) {
            int ux = (cx + dx + nc) % nc, uy = (cy + dy + nc) % nc, uz = (cz + dz + nc) % nc;
            for (int32_t a = head[((int64_t)uz * nc + uy) * nc + ux]; a >= 0; a = next[a]) {
              double ddx = gg_wrap(p[3 * a] - x, L), ddy = gg_wrap(p[3 * a + 1] - y, L),
                     ddz = gg_wrap(p[3 * a + 2] - z, L);
              if (ddx * ddx + ddy * ddy + ddz * ddz < dmin2) {
                ok = 0;
                break;
              }
            }
          }
    } else {
      for (int a = 0; a < placed; ++a) {
        double ddx = gg_wrap(p[3 * a] - x, L), ddy = gg_wrap(p[3 * a + 1] - y, L),
               ddz = gg_wrap(p[3 * a + 2] - z, L);
        if (ddx * ddx + ddy * ddy + ddz * ddz < dmin2) {
          ok = 0;
          break;
        }
      }
    }
    if (!ok) continue;
    p[3 * placed] = x;
    p[3 * placed + 1] = y;
    p[3 * placed + 2] = z;
    int64_t c = ((int64_t)gg_cell_of(z, L, nc) * nc + gg_cell_of(y, L, nc)) * nc + gg_cell_of(x, L, nc);
    next[placed] = head[c];
    head[c] = placed;
    ++placed;
  }
  free(head);
  free(next);

  /* ---- spatial renumbering: Morton order of r_c cells ---- */
  int ncb = (int)floor(L / r_c);
  if (ncb < 1) ncb = 1;
  if (ncb > 1024) ncb = 1024;
  gg_keyed *keys = (gg_keyed *)malloc(sizeof(gg_keyed) * N);
  if (!keys) {
    free(p);
    return -4;
  }
  for (int a = 0; a < N; ++a) {
    keys[a].idx = a;
    if (spatial_sort) {
      uint64_t cx = gg_cell_of(p[3 * a], L, ncb), cy = gg_cell_of(p[3 * a + 1], L, ncb),
               cz = gg_cell_of(p[3 * a + 2], L, ncb);
      keys[a].key = gg_spread3(cx) | (gg_spread3(cy) << 1) | (gg_spread3(cz) << 2);
    } else {
      keys[a].key = 0;
    }
  }
  qsort(keys, N, sizeof(gg_keyed), gg_cmp_keyed);
  for (int a = 0; a < N; ++a) {
    int s = keys[a].idx;
    pos[3 * a] = p[3 * s];
    pos[3 * a + 1] = p[3 * s + 1];
    pos[3 * a + 2] = p[3 * s + 2];
  }
  free(keys);
  free(p);

  /* ---- types: f_A of the atoms are A, assigned by a Fisher-Yates shuffle ---- */
  int32_t n_a = (int32_t)llround(frac_a * N);
  for (int a = 0; a < N; ++a) type[a] = (a < n_a) ? 0 : 1;
  for (int a = N - 1; a > 0; --a) {
    int b = (int)(gg_uniform(&rng) * (a + 1));
    if (b > a) b = a;
    int32_t t = type[a];
    type[a] = type[b];
    type[b] = t;
  }
  for (int a = 0; a < N; ++a) mass[a] = type[a] == 0 ? m_a : m_b;

  /* ---- bonds: every pair within r_c (minimum image), i < j, lexicographic ---- */
  int ncr = (int)floor(L / r_c);
  if (ncr > 1024) ncr = 1024;
  const int use_cells = ncr >= 3;
  int64_t ncell_r = use_cells ? (int64_t)ncr * ncr * ncr : 1;
  int32_t *chead = (int32_t *)malloc(sizeof(int32_t) * ncell_r);
  int32_t *cnext = (int32_t *)malloc(sizeof(int32_t) * N);
  int32_t *nb = (int32_t *)malloc(sizeof(int32_t) * (size_t)N); /* scratch neighbour list */
  int nb_cap = N;
  if (!chead || !cnext || !nb) {
    free(chead); free(cnext); free(nb);
    return -4;
  }
  for (int64_t c = 0; c < ncell_r; ++c) chead[c] = -1;
  if (use_cells) {
    for (int a = N - 1; a >= 0; --a) {
      int64_t c = ((int64_t)gg_cell_of(pos[3 * a + 2], L, ncr) * ncr + gg_cell_of(pos[3 * a + 1], L, ncr)) * ncr +
                  gg_cell_of(pos[3 * a], L, ncr);
      cnext[a] = chead[c];
      chead[c] = a;
    }
  }
  const double rc2 = r_c * r_c;
  int64_t nbond = 0;
  for (int i = 0; i < N; ++i) {
    int cnt = 0;
    if (use_cells) {
      int cx = gg_cell_of(pos[3 * i], L, ncr), cy = gg_cell_of(pos[3 * i + 1], L, ncr),
          cz = gg_cell_of(pos[3 * i + 2], L, ncr);
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            int ux = (cx + dx + ncr) % ncr, uy = (cy + dy + ncr) % ncr, uz = (cz + dz + ncr) % ncr;
            for (int32_t j = chead[((int64_t)uz * ncr + uy) * ncr + ux]; j >= 0; j = cnext[j]) {
              if (j <= i) continue;
              double ddx = gg_wrap(pos[3 * j] - pos[3 * i], L), ddy = gg_wrap(pos[3 * j + 1] - pos[3 * i + 1], L),
                     ddz = gg_wrap(pos[3 * j + 2] - pos[3 * i + 2], L);
              if (ddx * ddx + ddy * ddy + ddz * ddz < rc2 && cnt < nb_cap) nb[cnt++] = j;
            }
          }
    } else {
      for (int j = i + 1; j < N; ++j) {
        double ddx = gg_wrap(pos[3 * j] - pos[3 * i], L), ddy = gg_wrap(pos[3 * j + 1] - pos[3 * i + 1], L),
               ddz = gg_wrap(pos[3 * j + 2] - pos[3 * i + 2], L);
        if (ddx * ddx + ddy * ddy + ddz * ddz < rc2) nb[cnt++] = j;
      }
    }
    qsort(nb, cnt, sizeof(int32_t), gg_cmp_i32);
    for (int t = 0; t < cnt; ++t) {
      int j = nb[t];
      double z = gg_normal(&rng);
      if (nbond < bond_cap && bi && bj && kk && rhat) {
        double ddx = gg_wrap(pos[3 * j] - pos[3 * i], L), ddy = gg_wrap(pos[3 * j + 1] - pos[3 * i + 1], L),
               ddz = gg_wrap(pos[3 * j + 2] - pos[3 * i + 2], L);
        double r = sqrt(ddx * ddx + ddy * ddy + ddz * ddz);
        bi[nbond] = i;
        bj[nbond] = j;
        kk[nbond] = k_med * exp(k_sigma * z);
        rhat[3 * nbond] = ddx / r;
        rhat[3 * nbond + 1] = ddy / r;
        rhat[3 * nbond + 2] = ddz / r;
      }
      ++nbond;
    }
  }
  free(chead);
  free(cnext);
  free(nb);
  *nbonds = nbond;
  return nbond > bond_cap ? -2 : 0;
}
