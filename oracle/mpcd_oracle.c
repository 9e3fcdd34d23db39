/*
 * mpcd_oracle.c -- FP64 CPU oracle for one SRD time step.
 *
 * TEST INFRASTRUCTURE ONLY: it is the slow, plain statement that the CUDA path is checked
 * against, and nothing in the library calls it.  Compile with -ffp-contract=off: the only
 * fused multiply-adds are the explicit fma() calls below.
 *
 * The method (arXiv 2212.11878, Sec. 2): particles stream, the collision grid is shifted at
 * random every step, particles are sorted into the shifted cells (Sec. 3.1, Listing 1), each
 * cell's mass and momentum are summed (Sec. 3.3, Listing 4), and each particle's velocity
 * relative to the cell's centre of mass is split along a random axis and its perpendicular
 * part rotated by a fixed angle (Sec. 2, parts (i)-(iii)).  The readings R1..R14 that fill in
 * what the paper leaves open are listed in mpcd_oracle.h.
 */
#include "mpcd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static const double ORC_PI = 3.14159265358979323846;

/* ---------------------------------------------------------------- Philox4x64-10 ---- */
/* Salmon et al., "Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 4:
 * each round multiplies counter words 0 and 2 by two odd constants, keeps the 64-bit high
 * and low halves, and mixes the high halves with words 1 and 3 and the round key; the key
 * advances by two Weyl constants between rounds.  Ten rounds. */
static const uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ULL;
static const uint64_t PHILOX_M1 = 0xCA5A826395121157ULL;
static const uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ULL; /* golden ratio */
static const uint64_t PHILOX_W1 = 0xBB67AE8584CAA73BULL; /* sqrt(3) - 1 */

static void mul_hi_lo(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
  unsigned __int128 prod = (unsigned __int128)a * (unsigned __int128)b;
  *lo = (uint64_t)prod;
  *hi = (uint64_t)(prod >> 64);
}

void orc_philox(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t hi0, lo0, hi1, lo1;
    mul_hi_lo(PHILOX_M0, x0, &hi0, &lo0);
    mul_hi_lo(PHILOX_M1, x2, &hi1, &lo1);
    uint64_t y0 = hi1 ^ x1 ^ k0;
    uint64_t y1 = lo1;
    uint64_t y2 = hi0 ^ x3 ^ k1;
    uint64_t y3 = lo0;
    x0 = y0;
    x1 = y1;
    x2 = y2;
    x3 = y3;
  }
  out[0] = x0;
  out[1] = x1;
  out[2] = x2;
  out[3] = x3;
}

double orc_u53(uint64_t w) { return (double)(w >> 11) * 0x1.0p-53; }

static void draw(const orc_params* p, uint64_t c0, uint64_t c1, uint64_t tag, uint64_t w[4]) {
  uint64_t ctr[4] = {c0, c1, tag, 0};
  uint64_t key[2] = {p->seed, 0};
  orc_philox(ctr, key, w);
}

/* Box-Muller: two uniforms -> two independent standard normals. */
static void box_muller(uint64_t w0, uint64_t w1, double* g0, double* g1) {
  double u1 = 1.0 - orc_u53(w0); /* (0, 1] */
  double u2 = orc_u53(w1);
  double rad = sqrt(-2.0 * log(u1));
  double ang = 2.0 * ORC_PI * u2;
  *g0 = rad * cos(ang);
  *g1 = rad * sin(ang);
}

/* ------------------------------------------------------------------- geometry ---- */
int64_t orc_num_cells(const orc_params* p) {
  int64_t lz = p->L[2] + (p->walls_z ? 1 : 0);
  return (int64_t)p->L[0] * p->L[1] * lz;
}

static double box_len(const orc_params* p, int d) { return (double)p->L[d] * p->a; }

void orc_shift(const orc_params* p, int64_t t, double s[3]) {
  uint64_t w[4];
  draw(p, (uint64_t)t, 0, ORC_TAG_SHIFT, w);
  for (int d = 0; d < 3; ++d) s[d] = (orc_u53(w[d]) - 0.5) * p->a;
  if (p->walls_z && s[2] < 0.0) s[2] += p->a; /* R4: fold into [0, a) */
}

int64_t orc_cell_key(const orc_params* p, const double r[3], const double s[3]) {
  int64_t c[3];
  for (int d = 0; d < 3; ++d) {
    double q = (r[d] - s[d]) / p->a;
    int64_t k = (int64_t)floor(q);
    if (d == 2 && p->walls_z) {
      /* layers 0 .. Lz; for z just below H, (z - s)/a can round up to Lz when a is not a
       * power of two, so the layer is clamped into range */
      c[d] = k + 1;
      if (c[d] < 0) c[d] = 0;
      if (c[d] > p->L[2]) c[d] = p->L[2];
    } else {
      int64_t L = p->L[d];
      c[d] = ((k % L) + L) % L;
    }
  }
  return c[0] + (int64_t)p->L[0] * (c[1] + (int64_t)p->L[1] * c[2]);
}

void orc_axis(const orc_params* p, int64_t t, int64_t cell, double n[3]) {
  /* z uniform on [-1, 1) and azimuth uniform on [0, 2 pi): uniform on the sphere
   * (Archimedes' hat-box theorem). */
  uint64_t w[4];
  draw(p, (uint64_t)t, (uint64_t)cell, ORC_TAG_AXIS, w);
  double z = 2.0 * orc_u53(w[0]) - 1.0;
  double phi = 2.0 * ORC_PI * orc_u53(w[1]);
  double rho = sqrt((1.0 - z) * (1.0 + z));
  n[0] = rho * cos(phi);
  n[1] = rho * sin(phi);
  n[2] = z;
}

/* Marsaglia and Tsang, "A simple method for generating gamma variables", ACM TOMS 26(3),
 * 2000: for shape a >= 1 put d = a - 1/3 and c = 1/sqrt(9 d); draw x standard normal and
 * u uniform on (0, 1]; with t = 1 + c x > 0 and v = t^3, d v is accepted when
 * u < 1 - 0.0331 x^4 (the squeeze) or log u < x^2/2 + d (1 - v + log v); else draw again.
 * Attempt k takes its three uniforms from Philox counter (t, cell, THERMO, k): the normal
 * from words 0 and 1 by Box-Muller (the cosine branch), u from word 2. */
double orc_mbs_gamma(const orc_params* p, int64_t t, int64_t cell, double shape) {
  double d = shape - 1.0 / 3.0;
  double c = 1.0 / sqrt(9.0 * d);
  for (uint64_t k = 0; k < 64; ++k) {
    uint64_t ctr[4] = {(uint64_t)t, (uint64_t)cell, ORC_TAG_THERMO, k};
    uint64_t key[2] = {p->seed, 0};
    uint64_t w[4];
    orc_philox(ctr, key, w);
    double x = sqrt(-2.0 * log(1.0 - orc_u53(w[0]))) * cos(2.0 * ORC_PI * orc_u53(w[1]));
    double tt = 1.0 + c * x;
    if (tt <= 0.0) continue;
    double v = tt * tt * tt;
    double u = 1.0 - orc_u53(w[2]);
    double x2 = x * x;
    if (u < 1.0 - 0.0331 * (x2 * x2)) return d * v;
    if (log(u) < 0.5 * x2 + d * (1.0 - v + log(v))) return d * v;
  }
  return d;
}

void orc_cell_local(const orc_params* p, const double r[3], const double s[3], double l[3]) {
  for (int d = 0; d < 3; ++d) {
    double q = (r[d] - s[d]) / p->a;
    l[d] = q - floor(q);
  }
}

static void cross(const double a[3], const double b[3], double out[3]) {
  out[0] = a[1] * b[2] - a[2] * b[1];
  out[1] = a[2] * b[0] - a[0] * b[2];
  out[2] = a[0] * b[1] - a[1] * b[0];
}

/* Mass of the particle in storage slot i: its own (R24) or the box's. */
static double mass_of(const orc_params* p, const double* mass, int64_t i) { return mass ? mass[i] : p->mass; }

/* Angular momentum about the cell's centre of mass, sum m_i rho_i x v_i (R23). */
static void cell_angular_momentum(const orc_params* p, const double* mass, const double* rho, const double* v,
                                  const int32_t* perm, int32_t j0, int32_t j1, double L[3]) {
  L[0] = L[1] = L[2] = 0.0;
  for (int32_t j = j0; j < j1; ++j) {
    double c[3];
    cross(&rho[3 * (int64_t)(j - j0)], &v[3 * (int64_t)perm[j]], c);
    for (int d = 0; d < 3; ++d) L[d] += mass_of(p, mass, perm[j]) * c[d];
  }
}

void orc_rotate(const double n[3], double alpha, const double u[3], double v[3]) {
  double d[3], cr[3], out[3];
  for (int k = 0; k < 3; ++k) d[k] = v[k] - u[k];               /* relative velocity */
  double par = n[0] * d[0] + n[1] * d[1] + n[2] * d[2];           /* component along n */
  cr[0] = n[1] * d[2] - n[2] * d[1];                              /* n x d */
  cr[1] = n[2] * d[0] - n[0] * d[2];
  cr[2] = n[0] * d[1] - n[1] * d[0];
  double c = cos(alpha), s = sin(alpha);
  for (int k = 0; k < 3; ++k) {
    double perp = d[k] - par * n[k];                              /* perpendicular part */
    out[k] = par * n[k] + c * perp + s * cr[k];                   /* rotated by alpha */
  }
  for (int k = 0; k < 3; ++k) v[k] = u[k] + out[k];
}

/* -------------------------------------------------------------------- streaming ---- */
/* Periodic wrap into [0, B) (R3). */
static double wrap(double x, double B) {
  if (x >= B)
    x -= B;
  else if (x < 0.0)
    x += B;
  if (x >= B || x < 0.0) {
    x = fmod(x, B);
    if (x < 0.0) x += B;
    if (x >= B) x = 0.0;
  }
  return x;
}

/* Ballistic move over dt under the constant acceleration g: r += v dt + g dt^2 / 2 and
 * v += g dt, written as r = fma(v, dt, r + h) and v = fma(g, dt, v) with h = g dt^2 / 2.
 * With walls (R13), a particle that reaches z = 0 or z = H has its whole velocity reversed
 * at the crossing time and moves on for the rest of the step. */
static void stream_one(const orc_params* p, double* r, double* v) {
  double H = box_len(p, 2);
  if (!p->walls_z) {
    for (int d = 0; d < 3; ++d) {
      double h = 0.5 * p->g[d] * p->dt * p->dt;
      r[d] = fma(v[d], p->dt, r[d] + h);
      v[d] = fma(p->g[d], p->dt, v[d]);
      r[d] = wrap(r[d], box_len(p, d));
    }
    return;
  }
  double left = p->dt;
  for (int bounce = 0; bounce < 64 && left > 0.0; ++bounce) {
    double z1 = r[2] + v[2] * left; /* g has no z component with walls */
    double tau = left;
    double wall = -1.0;
    if (z1 < 0.0) {
      tau = (0.0 - r[2]) / v[2];
      wall = 0.0;
    } else if (z1 >= H) {
      tau = (H - r[2]) / v[2];
      wall = H;
    }
    if (tau < 0.0) tau = 0.0;
    if (tau > left) tau = left;
    for (int d = 0; d < 2; ++d) {
      double h = 0.5 * p->g[d] * tau * tau;
      r[d] = fma(v[d], tau, r[d] + h);
      v[d] = fma(p->g[d], tau, v[d]);
    }
    if (wall < 0.0) {
      r[2] = fma(v[2], tau, r[2]);
      left = 0.0;
    } else {
      r[2] = wall;
      for (int d = 0; d < 3; ++d) v[d] = -v[d];
      left -= tau;
    }
  }
  for (int d = 0; d < 2; ++d) r[d] = wrap(r[d], box_len(p, d));
  if (r[2] >= H) r[2] = nextafter(H, 0.0);
  if (r[2] < 0.0) r[2] = 0.0;
}

/* ---------------------------------------------------------------------- init ---- */
void orc_init(const orc_params* p, int64_t n, double* r, double* v) {
  double sigma = sqrt(p->kT / p->mass);
  double mean[3] = {0.0, 0.0, 0.0};
  for (int64_t i = 0; i < n; ++i) {
    uint64_t w[4];
    draw(p, (uint64_t)i, 0, ORC_TAG_INIT, w);
    for (int d = 0; d < 3; ++d) r[3 * i + d] = orc_u53(w[d]) * box_len(p, d);
    draw(p, (uint64_t)i, 1, ORC_TAG_INIT, w);
    double g[4];
    box_muller(w[0], w[1], &g[0], &g[1]);
    box_muller(w[2], w[3], &g[2], &g[3]);
    for (int d = 0; d < 3; ++d) {
      v[3 * i + d] = sigma * g[d];
      mean[d] += v[3 * i + d];
    }
  }
  if (n > 0)
    for (int d = 0; d < 3; ++d) mean[d] /= (double)n;
  for (int64_t i = 0; i < n; ++i)
    for (int d = 0; d < 3; ++d) v[3 * i + d] -= mean[d];
}

/* ---------------------------------------------------------------------- step ---- */
int orc_step(const orc_params* p, int64_t n, int64_t t, double* r, double* v, int32_t* id,
             int32_t* keys_out, int32_t* counts_out, int32_t* offsets_out, int32_t* perm_out,
             double* moments_out, double* shift_out) {
  return orc_step_m(p, n, t, r, v, id, NULL, keys_out, counts_out, offsets_out, perm_out, moments_out, shift_out);
}

int orc_step_m(const orc_params* p, int64_t n, int64_t t, double* r, double* v, int32_t* id, double* mass,
               int32_t* keys_out, int32_t* counts_out, int32_t* offsets_out, int32_t* perm_out,
               double* moments_out, double* shift_out) {
  if (!p || n < 0 || t < 1 || p->a <= 0.0 || p->mass <= 0.0) return -1;
  if (mass)
    for (int64_t i = 0; i < n; ++i)
      if (!(mass[i] > 0.0)) return -1;
  for (int d = 0; d < 3; ++d)
    if (p->L[d] < 1) return -1;
  if (p->walls_z && p->g[2] != 0.0) return -1;
  if (p->angular && p->walls_z) return -1; /* R23 */
  int64_t C = orc_num_cells(p);
  if (C > INT32_MAX || n > INT32_MAX) return -1;

  int32_t* key = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int32_t* cnt = (int32_t*)calloc((size_t)C, sizeof(int32_t));
  int32_t* off = (int32_t*)malloc(sizeof(int32_t) * (size_t)(C + 1));
  int32_t* cur = (int32_t*)malloc(sizeof(int32_t) * (size_t)C);
  int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  double* rho = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1)); /* R23, per cell */
  if (!key || !cnt || !off || !cur || !perm || !rho) {
    free(key); free(cnt); free(off); free(cur); free(perm); free(rho);
    return -2;
  }

  /* 1. streaming (R1) */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) stream_one(p, &r[3 * i], &v[3 * i]);

  /* 2. grid shift of this step (R2) */
  double s[3];
  orc_shift(p, t, s);

  /* 3. cell of every particle on the shifted grid (Sec. 3.1) */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) key[i] = (int32_t)orc_cell_key(p, &r[3 * i], s);

  /* 4. linked-cell list as a stable counting sort (R6) */
  for (int64_t i = 0; i < n; ++i) cnt[key[i]] += 1;
  off[0] = 0;
  for (int64_t c = 0; c < C; ++c) off[c + 1] = off[c] + cnt[c];
  for (int64_t c = 0; c < C; ++c) cur[c] = off[c];
  for (int64_t i = 0; i < n; ++i) perm[cur[key[i]]++] = (int32_t)i;

  /* 5.-7. per cell: centre of mass (Listing 4), relative velocity, rotation (Sec. 2) */
  const double m = p->mass;
  /* cells are independent: each reads and writes only its own members and its own slice
   * rho[3 off[c] ..] of the R23 scratch (the OpenMP build runs them in parallel) */
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t c = 0; c < C; ++c) {
    int32_t nc = cnt[c];
    double* rc = rho + 3 * (int64_t)off[c];
    double M = 0.0, P[3] = {0.0, 0.0, 0.0}, E = 0.0;
    for (int32_t j = off[c]; j < off[c + 1]; ++j) {
      const double* vi = &v[3 * (int64_t)perm[j]];
      const double mi = mass_of(p, mass, perm[j]); /* Listing 4 weights by mass */
      for (int d = 0; d < 3; ++d) P[d] += mi * vi[d];
      M += mi;
      E += 0.5 * mi * (vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2]);
    }
    if (moments_out) {
      moments_out[5 * c + 0] = M;
      moments_out[5 * c + 1] = P[0];
      moments_out[5 * c + 2] = P[1];
      moments_out[5 * c + 3] = P[2];
      moments_out[5 * c + 4] = E;
    }
    if (nc == 0) continue;

    /* R13: a cell cut by a wall is filled up to ppc with virtual particles at rest on
     * average, whose summed momentum is Gaussian with variance M_virtual kT. */
    int virt = 0;
    if (p->walls_z && s[2] > 0.0) {
      int64_t layer = c / ((int64_t)p->L[0] * p->L[1]);
      if ((layer == 0 || layer == p->L[2]) && (double)nc < p->ppc) {
        double Mv = (p->ppc - (double)nc) * m;
        uint64_t w[4];
        draw(p, (uint64_t)t, (uint64_t)c, ORC_TAG_WALL, w);
        double g[4];
        box_muller(w[0], w[1], &g[0], &g[1]);
        box_muller(w[2], w[3], &g[2], &g[3]);
        double sd = sqrt(Mv * p->kT);
        for (int d = 0; d < 3; ++d) P[d] += sd * g[d];
        M += Mv;
        virt = 1;
      }
    }
    if (nc < 2 && !virt) continue; /* R12 */

    double u[3];
    for (int d = 0; d < 3; ++d) u[d] = P[d] / M; /* R7 */
    double ax[3];
    orc_axis(p, t, c, ax);

    /* R23: positions relative to the cell's centre of mass and the angular momentum about it
     * before the collision */
    double Lb[3] = {0.0, 0.0, 0.0};
    if (p->angular) {
      double mean[3] = {0.0, 0.0, 0.0};
      for (int32_t j = off[c]; j < off[c + 1]; ++j) {
        double* l = &rc[3 * (int64_t)(j - off[c])];
        orc_cell_local(p, &r[3 * (int64_t)perm[j]], s, l);
        /* the centre of mass: with particle masses (R24) weighted, else the plain mean */
        for (int d = 0; d < 3; ++d) mean[d] += mass ? mass[perm[j]] * l[d] : l[d];
      }
      for (int d = 0; d < 3; ++d) mean[d] /= mass ? M : (double)nc;
      for (int32_t j = off[c]; j < off[c + 1]; ++j)
        for (int d = 0; d < 3; ++d) rc[3 * (int64_t)(j - off[c]) + d] = p->a * (rc[3 * (int64_t)(j - off[c]) + d] - mean[d]);
      cell_angular_momentum(p, mass, rc, v, perm, off[c], off[c + 1], Lb);
    }

    for (int32_t j = off[c]; j < off[c + 1]; ++j) orc_rotate(ax, p->alpha, u, &v[3 * (int64_t)perm[j]]);

    if (p->thermostat && nc >= 2) {
      /* R14: rescale the relative velocities so the cell's relative kinetic energy is
       * (3/2)(n_c - 1) kT; R22 (MBS): kT times a Gamma(3/2 (n_c - 1)) draw instead. */
      double target = p->thermostat == 2 ? p->kT * orc_mbs_gamma(p, t, c, 1.5 * (double)(nc - 1))
                                         : 1.5 * (double)(nc - 1) * p->kT;
      double K = 0.0;
      for (int32_t j = off[c]; j < off[c + 1]; ++j) {
        const double* vi = &v[3 * (int64_t)perm[j]];
        const double mi = mass_of(p, mass, perm[j]);
        for (int d = 0; d < 3; ++d) K += 0.5 * mi * (vi[d] - u[d]) * (vi[d] - u[d]);
      }
      if (K > 0.0) {
        double f = sqrt(target / K);
        for (int32_t j = off[c]; j < off[c + 1]; ++j) {
          double* vi = &v[3 * (int64_t)perm[j]];
          for (int d = 0; d < 3; ++d) vi[d] = u[d] + f * (vi[d] - u[d]);
        }
      }
    }

    if (p->angular) {
      /* R23: omega = I^-1 (L_before - L_after) with I = m sum (|rho|^2 1 - rho rho^T); then
       * v_i += omega x rho_i, which keeps the cell's momentum (sum rho_i = 0) and restores
       * its angular momentum (sum m rho_i x (omega x rho_i) = I omega). */
      double La[3], dL[3], I[3][3] = {{0.0}}, rr = 0.0, rrm = 0.0;
      cell_angular_momentum(p, mass, rc, v, perm, off[c], off[c + 1], La);
      for (int d = 0; d < 3; ++d) dL[d] = Lb[d] - La[d];
      for (int32_t j = off[c]; j < off[c + 1]; ++j) {
        const double* q = &rc[3 * (int64_t)(j - off[c])];
        double q2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
        const double mi = mass_of(p, mass, perm[j]);
        rr += q2;
        rrm += mi * q2;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) I[a][b] += mi * ((a == b ? q2 : 0.0) - q[a] * q[b]);
      }
      double w[3] = {0.0, 0.0, 0.0};
      int apply = 0;
      if (nc == 2) {
        /* two particles: rho_2 = -rho_1, I = m rr (1 - e e^T) with e = rho_1/|rho_1|; the
         * change of L is normal to e, where I acts as m rr */
        double e2 = rr > 0.0 ? 2.0 / rr : 0.0; /* 1/|rho_1|^2 */
        const double* q = &rc[0];
        double along = (q[0] * dL[0] + q[1] * dL[1] + q[2] * dL[2]) * e2;
        if (rr > 0.0 && !mass) {
          for (int d = 0; d < 3; ++d) w[d] = (dL[d] - along * q[d]) / (p->mass * rr);
          apply = 1;
        } else if (rr > 0.0) {
          /* unequal masses (R24): m_1 rho_1 + m_2 rho_2 = 0 keeps the pair on one line, and I
           * acts as sum m_i |rho_i|^2 normal to it */
          double qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
          double al = (q[0] * dL[0] + q[1] * dL[1] + q[2] * dL[2]) / qq;
          for (int d = 0; d < 3; ++d) w[d] = (dL[d] - al * q[d]) / rrm;
          apply = 1;
        }
      } else {
        /* the inverse by cofactors */
        double cof[3][3];
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            int a1 = (a + 1) % 3, a2 = (a + 2) % 3, b1 = (b + 1) % 3, b2 = (b + 2) % 3;
            cof[a][b] = I[a1][b1] * I[a2][b2] - I[a1][b2] * I[a2][b1];
          }
        double det = I[0][0] * cof[0][0] + I[0][1] * cof[0][1] + I[0][2] * cof[0][2];
        double tr = (I[0][0] + I[1][1] + I[2][2]) / 3.0;
        if (det > 1e-12 * tr * tr * tr) {
          for (int a = 0; a < 3; ++a) /* I symmetric: inverse = cof^T / det = cof / det */
            w[a] = (cof[a][0] * dL[0] + cof[a][1] * dL[1] + cof[a][2] * dL[2]) / det;
          apply = 1;
        }
      }
      if (apply)
        for (int32_t j = off[c]; j < off[c + 1]; ++j) {
          double corr[3];
          cross(w, &rc[3 * (int64_t)(j - off[c])], corr);
          double* vi = &v[3 * (int64_t)perm[j]];
          for (int d = 0; d < 3; ++d) vi[d] += corr[d];
        }
    }
  }

  if (keys_out) memcpy(keys_out, key, sizeof(int32_t) * (size_t)n);
  if (counts_out) memcpy(counts_out, cnt, sizeof(int32_t) * (size_t)C);
  if (offsets_out) memcpy(offsets_out, off, sizeof(int32_t) * (size_t)(C + 1));
  if (perm_out) memcpy(perm_out, perm, sizeof(int32_t) * (size_t)n);
  if (shift_out)
    for (int d = 0; d < 3; ++d) shift_out[d] = s[d];
  free(rho);

  /* 8. every k steps the storage itself is put into cell order (Listing 1, permute) */
  if (p->resort_k > 0 && t % p->resort_k == 0 && n > 0) {
    double* r2 = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    double* v2 = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    int32_t* id2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    double* m2 = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!r2 || !v2 || !id2 || !m2) {
      free(r2); free(v2); free(id2); free(m2);
      free(key); free(cnt); free(off); free(cur); free(perm);
      return -2;
    }
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
      int64_t i = perm[j];
      for (int d = 0; d < 3; ++d) {
        r2[3 * j + d] = r[3 * i + d];
        v2[3 * j + d] = v[3 * i + d];
      }
      id2[j] = id ? id[i] : (int32_t)i;
      m2[j] = mass ? mass[i] : 0.0;
    }
    memcpy(r, r2, sizeof(double) * 3 * (size_t)n);
    memcpy(v, v2, sizeof(double) * 3 * (size_t)n);
    if (id) memcpy(id, id2, sizeof(int32_t) * (size_t)n);
    if (mass) memcpy(mass, m2, sizeof(double) * (size_t)n);
    free(r2); free(v2); free(id2); free(m2);
  }

  free(key); free(cnt); free(off); free(cur); free(perm);
  return 0;
}

/* ------------------------------------------------------------------- presort ---- */
/* R25: a stable counting sort of the storage by the cell of each position on the unshifted
 * grid, then the permutation applied to every per-particle array. */
int orc_presort(const orc_params* p, int64_t n, double* r, double* v, int32_t* id, double* mass) {
  if (!p || n < 0) return -1;
  if (n == 0) return 0;
  int64_t C = orc_num_cells(p);
  const double s0[3] = {0.0, 0.0, 0.0};
  int32_t* key = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int64_t* start = (int64_t*)calloc((size_t)C + 1, sizeof(int64_t));
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  double* tmp = (double*)malloc(sizeof(double) * 3 * (size_t)n);
  int32_t* itmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!key || !start || !order || !tmp || !itmp) {
    free(key); free(start); free(order); free(tmp); free(itmp);
    return -2;
  }
  for (int64_t i = 0; i < n; ++i) {
    key[i] = (int32_t)orc_cell_key(p, &r[3 * i], s0);
    start[key[i] + 1] += 1;
  }
  for (int64_t c = 0; c < C; ++c) start[c + 1] += start[c];
  for (int64_t i = 0; i < n; ++i) order[start[key[i]]++] = i; /* slot j holds old slot order[j] */
  for (int64_t j = 0; j < n; ++j)
    for (int d = 0; d < 3; ++d) tmp[3 * j + d] = r[3 * order[j] + d];
  memcpy(r, tmp, sizeof(double) * 3 * (size_t)n);
  for (int64_t j = 0; j < n; ++j)
    for (int d = 0; d < 3; ++d) tmp[3 * j + d] = v[3 * order[j] + d];
  memcpy(v, tmp, sizeof(double) * 3 * (size_t)n);
  if (id) {
    for (int64_t j = 0; j < n; ++j) itmp[j] = id[order[j]];
    memcpy(id, itmp, sizeof(int32_t) * (size_t)n);
  }
  if (mass) {
    for (int64_t j = 0; j < n; ++j) tmp[j] = mass[order[j]];
    memcpy(mass, tmp, sizeof(double) * (size_t)n);
  }
  free(key); free(start); free(order); free(tmp); free(itmp);
  return 0;
}
