/*
 * h4d_oracle.c -- FP64 CPU oracle of the H4D grand-canonical method (arXiv:2307.11447).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU-baseline leg
 * of the benchmark, never by the CUDA library.  Everything is double precision, written
 * for a reader checking it against the paper:
 *   Sec. II.A   constant-velocity altitude protocol (Eq. 2), NVE time evolution,
 *               symmetric two-end momentum reversal, pair-exchange Metropolis rule
 *               (Eqs. 3-8).
 *   Sec. II.B.1 flying ions keep their 3D positions during NEMD.
 *   Sec. II.B.2 short-range 4D Coulomb with altitude screening (Eqs. 9-11).
 *   Sec. II.D   truncated-shifted LJ (Eq. 19), Coulomb (Eq. 20), Lorentz-Berthelot,
 *               rigid water.
 *   SI Sec. S5  altitude schedules w_v and w_x (Eqs. S6-S7).
 * Readings of points the paper leaves open (which energies Delta H compares, flyer momenta,
 * step ordering, reversal details, move choice, Coulomb shift, thermostat) are stated
 * at the code that takes them.
 *
 * Parity status: pinned by the not-gpu tests (closed forms, brute force, finite
 * differences, 3D recovery, NVE drift, exact reversibility, ideal-gas laws).
 */
#include "h4d_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of a multiply-xor      */
/* bijection keyed by a Weyl sequence.                                                   */
/* ------------------------------------------------------------------------------------ */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
  __uint128_t prod = (__uint128_t)a * (__uint128_t)b;
  *hi = (uint64_t)(prod >> 64);
  *lo = (uint64_t)prod;
}

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo64(0xD2E7470EE14C6C93ULL, c0, &hi0, &lo0);
    mulhilo64(0xCA5A826395121157ULL, c2, &hi1, &lo1);
    uint64_t n0 = hi1 ^ c1 ^ k0;
    uint64_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B97F4A7C15ULL;
    k1 += 0xBB67AE8584CAA73BULL;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw(const orc_params* p, uint64_t c0, uint64_t c1, uint64_t purpose, uint64_t out[4]) {
  uint64_t ctr[4] = {c0, c1, purpose, 0};
  uint64_t key[2] = {p->seed, p->replica};
  orc_philox4x64_10(ctr, key, out);
}

/* uniform in [0,1) and in (0,1] from the top 53 bits */
static double u01(uint64_t r) { return (double)(r >> 11) * 0x1.0p-53; }
static double u01_open(uint64_t r) { return (double)((r >> 11) + 1) * 0x1.0p-53; }
/* uniform integer in [0, n) from the top 32 bits (multiply-shift) */
static int32_t pick(uint64_t r, int32_t n) {
  return (int32_t)(((r >> 32) * (uint64_t)n) >> 32);
}
/* standard normal, Box-Muller cosine branch */
static double gauss_cos(uint64_t ra, uint64_t rb) {
  return sqrt(-2.0 * log(u01_open(ra))) * cos(2.0 * M_PI * u01(rb));
}
static double gauss_sin(uint64_t ra, uint64_t rb) {
  return sqrt(-2.0 * log(u01_open(ra))) * sin(2.0 * M_PI * u01(rb));
}

/* ------------------------------------------------------------------------------------ */
/* System layout                                                                         */
/* ------------------------------------------------------------------------------------ */
int orc_atom_type(const orc_params* p, int a) {
  int nsolv = 3 * p->n_water;
  if (a < nsolv) return (a % 3 == 0) ? 2 : 3;
  if (p->single) return 0; /* single-particle exchange: one species */
  return (a - nsolv) & 1;
}

static int excluded(const orc_params* p, int i, int j) {
  int nsolv = 3 * p->n_water;
  return i < nsolv && j < nsolv && (i / 3) == (j / 3);
}

static double mass_of(const orc_params* p, int a) { return p->mass[orc_atom_type(p, a)]; }

static double minimg(double d, double L) { return d - L * nearbyint(d / L); }

static double wrap(double x, double L) {
  double y = x - L * floor(x / L);
  if (y >= L) y -= L; /* guards x/L rounding up to the next integer */
  return y;
}

/* ------------------------------------------------------------------------------------ */
/* Pair potential                                                                        */
/* ------------------------------------------------------------------------------------ */
/* LJ truncated and shifted at rc_lj (Eq. 19) with Lorentz-Berthelot mixing (Sec. II.D.2);
 * Coulomb short-range part K q_i q_j erfc(alpha r)/r (Eqs. 9, 20), shifted to zero at
 * rc_coul (reading: energy shifted like the LJ, force unshifted), multiplied by the
 * altitude screening g (Eq. 11).  r is the 4D distance of Sec. II.A. */
void orc_pair(const orc_params* p, int ti, int tj, double r, double g, double* u, double* dudr) {
  double uu = 0.0, du = 0.0;
  double sig = 0.5 * (p->sig[ti] + p->sig[tj]);
  double eps = sqrt(p->eps[ti] * p->eps[tj]);
  if (eps > 0.0 && r < p->rc_lj) {
    double sr6 = pow(sig / r, 6.0);
    double sc6 = pow(sig / p->rc_lj, 6.0);
    uu += 4.0 * eps * (sr6 * sr6 - sr6) - 4.0 * eps * (sc6 * sc6 - sc6);
    du += 4.0 * eps * (-12.0 * sr6 * sr6 + 6.0 * sr6) / r;
  }
  double qq = p->q[ti] * p->q[tj];
  if (qq != 0.0 && r < p->rc_coul) {
    double a = p->alpha;
    double kq = p->kcoul * qq * g;
    uu += kq * (erfc(a * r) / r - erfc(a * p->rc_coul) / p->rc_coul);
    du += kq * (-erfc(a * r) / (r * r) - 2.0 * a / sqrt(M_PI) * exp(-a * a * r * r) / r);
  }
  *u = uu;
  *dudr = du;
}

/* mean altitude of the flyers (Sec. II.B.2: the screening uses the average altitude) */
static double mean_flyer_w(int n, const double* w, const uint8_t* fly) {
  if (!w || !fly) return 0.0;
  double s = 0.0;
  int m = 0;
  for (int i = 0; i < n; ++i)
    if (fly[i] == 1) { s += w[i]; ++m; }
  return m ? s / m : 0.0;
}

/* screening of Eq. 11: f_ij = 1 only when exactly one of i, j flies; other pairs keep
 * their unscreened interaction (reading of the f_ij definition) */
static double screen(const orc_params* p, const uint8_t* fly, int i, int j, double wbar) {
  if (!fly) return 1.0;
  int fi = fly[i] == 1, fj = fly[j] == 1;
  return (fi != fj) ? exp(-p->kappa_sr * wbar) : 1.0;
}

/* one pair: accumulate energy and forces; absent atoms (fly == 2) are skipped */
static double pair_term(const orc_params* p, const double* x, const double* w, const uint8_t* fly,
                        double wbar, int i, int j, double* F) {
  if (fly && (fly[i] == 2 || fly[j] == 2)) return 0.0;
  if (excluded(p, i, j)) return 0.0;
  double d[3];
  double r2 = 0.0;
  for (int c = 0; c < 3; ++c) {
    d[c] = minimg(x[3 * j + c] - x[3 * i + c], p->L);
    r2 += d[c] * d[c];
  }
  double dw = w ? (w[i] - w[j]) : 0.0;
  double r4 = sqrt(r2 + dw * dw);
  double rmax = p->rc_lj > p->rc_coul ? p->rc_lj : p->rc_coul;
#ifdef ORC_FP32_FORCES
  /* Tolerance-derivation build only (liboracle_fp32.so): the same pair force evaluated in
   * binary32 (distance, cut-off test, LJ and Coulomb derivative), everything else FP64.
   * Comparing it with the FP64 build measures how far FP32 pair forces alone move a
   * trajectory's work. */
  if (F) {
    int ti = orc_atom_type(p, i), tj = orc_atom_type(p, j);
    float df[3] = {(float)d[0], (float)d[1], (float)d[2]};
    float dwf = (float)dw;
    float r2f = df[0] * df[0] + df[1] * df[1] + df[2] * df[2] + dwf * dwf;
    float rmf = (float)rmax;
    if (r2f >= rmf * rmf) return 0.0;
    float rf = sqrtf(r2f);
    float sig = (float)(0.5 * (p->sig[ti] + p->sig[tj])), eps = (float)sqrt(p->eps[ti] * p->eps[tj]);
    float du = 0.f;
    if (eps > 0.f && r2f < (float)(p->rc_lj * p->rc_lj)) {
      float s2 = sig * sig / r2f, s6 = s2 * s2 * s2;
      du += 4.f * eps * (-12.f * s6 * s6 + 6.f * s6) / rf;
    }
    if (p->q[ti] * p->q[tj] != 0.0 && r2f < (float)(p->rc_coul * p->rc_coul)) {
      float a = (float)p->alpha;
      float kq = (float)(p->kcoul * p->q[ti] * p->q[tj] * screen(p, fly, i, j, wbar));
      du += kq * (-erfcf(a * rf) / r2f - 2.f * a / sqrtf((float)M_PI) * expf(-a * a * r2f) / rf);
    }
    for (int c = 0; c < 3; ++c) {
      float f = du * df[c] / rf;
      F[3 * i + c] += f;
      F[3 * j + c] -= f;
    }
    if (r4 >= rmax) return 0.0;
    double u, dudr;
    orc_pair(p, ti, tj, r4, screen(p, fly, i, j, wbar), &u, &dudr);
    return u;
  }
#endif
  if (r4 >= rmax) return 0.0;
  double u, dudr;
  orc_pair(p, orc_atom_type(p, i), orc_atom_type(p, j), r4, screen(p, fly, i, j, wbar), &u, &dudr);
  if (F) {
    /* F_i = -du/dx_i = u'(r4) (x_j - x_i)/r4 ; F_j = -F_i (3D components only) */
    for (int c = 0; c < 3; ++c) {
      double f = dudr * d[c] / r4;
      F[3 * i + c] += f;
      F[3 * j + c] -= f;
    }
  }
  return u;
}

static double energy_brute(const orc_params* p, int n, const double* x, const double* w,
                           const uint8_t* fly, double* F) {
  double wbar = mean_flyer_w(n, w, fly);
  double U = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) U += pair_term(p, x, w, fly, wbar, i, j, F);
  return U;
}

/* plain cell list with cells no smaller than the largest cut-off; a 3D criterion is a
 * valid superset in 4D because r4 >= r */
static double energy_cells(const orc_params* p, int n, const double* x, const double* w,
                           const uint8_t* fly, double* F) {
  double rmax = p->rc_lj > p->rc_coul ? p->rc_lj : p->rc_coul;
  int nc = (int)floor(p->L / rmax);
  if (nc < 3) return energy_brute(p, n, x, w, fly, F);
  double wbar = mean_flyer_w(n, w, fly);
  int ncell = nc * nc * nc;
  int* head = (int*)malloc(sizeof(int) * ncell);
  int* next = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
  for (int c = 0; c < ncell; ++c) head[c] = -1;
  for (int i = n - 1; i >= 0; --i) {
    int cx = (int)(x[3 * i + 0] / p->L * nc) % nc;
    int cy = (int)(x[3 * i + 1] / p->L * nc) % nc;
    int cz = (int)(x[3 * i + 2] / p->L * nc) % nc;
    int c = (cx * nc + cy) * nc + cz;
    next[i] = head[c];
    head[c] = i;
  }
  double U = 0.0;
  for (int cx = 0; cx < nc; ++cx)
    for (int cy = 0; cy < nc; ++cy)
      for (int cz = 0; cz < nc; ++cz) {
        int c = (cx * nc + cy) * nc + cz;
        for (int dx = -1; dx <= 1; ++dx)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
              int ex = (cx + dx + nc) % nc, ey = (cy + dy + nc) % nc, ez = (cz + dz + nc) % nc;
              int e = (ex * nc + ey) * nc + ez;
              for (int i = head[c]; i >= 0; i = next[i])
                for (int j = head[e]; j >= 0; j = next[j])
                  if (i < j) U += pair_term(p, x, w, fly, wbar, i, j, F);
            }
      }
  free(head);
  free(next);
  return U;
}

double orc_energy_forces(const orc_params* p, int n, const double* x, const double* w,
                         const uint8_t* fly, double* F) {
  if (F) memset(F, 0, sizeof(double) * 3 * (size_t)n);
  return p->use_cells ? energy_cells(p, n, x, w, fly, F) : energy_brute(p, n, x, w, fly, F);
}

/* energy of the pairs that involve at least one flyer, the flyers at altitude wf */
/* altitude of flyer i when the cation's altitude is w: the anion's is scaled by
 * r_w = w_max,a / w_max,c (1 with one w_max for both species) */
static double species_w(const orc_params* p, int i, double w) {
  if (p->fw <= 0.0 || orc_atom_type(p, i) != 1) return w;
  return w * (1.0 + 0.5 * (p->sig[0] + p->sig[1]) * p->fw / p->w_max);
}

static double flyer_energy(const orc_params* p, int n, const double* x, const uint8_t* fly, double wf,
                           double* wbuf) {
  for (int i = 0; i < n; ++i) wbuf[i] = (fly[i] == 1) ? species_w(p, i, wf) : 0.0;
  double wbar = mean_flyer_w(n, wbuf, fly);
  double U = 0.0;
  for (int i = 0; i < n; ++i) {
    if (fly[i] != 1) continue;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      if (fly[j] == 1 && j < i) continue; /* flyer-flyer pair counted once */
      U += pair_term(p, x, wbuf, fly, wbar, i, j, NULL);
    }
  }
  return U;
}

/* ------------------------------------------------------------------------------------ */
/* Fixed-point neighbour criterion (definition shared by name with the GPU path):        */
/* X = round(x/L * 2^32) mod 2^32 per coordinate; (i,j) is a list pair iff              */
/* sum_c ((int32)(X_i - X_j))^2 <= floor((r_list/L * 2^32)^2).                           */
/* ------------------------------------------------------------------------------------ */
static uint32_t fixpt(double x, double L) {
  double s = nearbyint(wrap(x, L) / L * 4294967296.0);
  return (uint32_t)((uint64_t)s & 0xffffffffULL);
}

/* early rejection: the anion (fixed point Xa) lies in the cube of volume v_ex centred on
 * the cation (Xc), per axis on the minimum-image fixed-point offset */
static int in_excluded_volume(const orc_params* p, const uint32_t Xc[3], const uint32_t Xa[3]) {
  if (!(p->v_ex > 0.0)) return 0;
  double half = nearbyint(0.5 * cbrt(p->v_ex) / p->L * 4294967296.0);
  for (int d = 0; d < 3; ++d) {
    double off = fabs((double)(int32_t)(Xa[d] - Xc[d]));
    if (!(off <= half)) return 0;
  }
  return 1;
}

int orc_in_excluded_volume(const orc_params* p, const double* xc, const double* xa) {
  uint32_t Xc[3], Xa[3];
  for (int d = 0; d < 3; ++d) {
    Xc[d] = fixpt(xc[d], p->L);
    Xa[d] = fixpt(xa[d], p->L);
  }
  return in_excluded_volume(p, Xc, Xa);
}

int64_t orc_neighbor_pairs(int n, const double* x, double L, double r_list, int32_t* out_i,
                           int32_t* out_j, int64_t cap) {
  double s = r_list / L * 4294967296.0;
  uint64_t T = (uint64_t)(s * s);
  int64_t m = 0;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      uint64_t d2 = 0;
      for (int c = 0; c < 3; ++c) {
        int64_t d = (int32_t)(fixpt(x[3 * i + c], L) - fixpt(x[3 * j + c], L));
        d2 += (uint64_t)(d * d);
      }
      if (d2 <= T) {
        if (m < cap) { out_i[m] = i; out_j[m] = j; }
        ++m;
      }
    }
  return m;
}

/* ------------------------------------------------------------------------------------ */
/* Protocol: altitude of a flyer at step k (Eq. 2 and SI Eqs. S6-S7).                    */
/* Insertion runs w_max -> 0, deletion 0 -> w_max; the deletion schedule is the time     */
/* reverse of the insertion schedule.                                                    */
/* ------------------------------------------------------------------------------------ */
double orc_altitude(const orc_params* p, int insertion, int k) {
  /* Deletion runs the insertion schedule backwards in time: w_del(t) = w_ins(t_f + t_i - t).
   * Reading: the deletion forms printed in Eqs. S6-S7 are swapped between w_v and w_x (as
   * printed, neither is the time reverse of its insertion form, and the text describes
   * a removal that is fast early for w_v); the time-reverse definition restores the
   * symmetric schedules that Sec. II.A requires for detailed balance. */
  int kk = insertion ? k : p->n_f - k;
  double xi = (double)kk / (double)p->n_f; /* x_i = (t - t_i)/(t_f - t_i) of the insertion */
  double n = p->sched_n;
  double s; /* w / w_max */
  if (p->schedule == ORC_SCHED_WV) s = 1.0 - pow(xi, n);      /* Eq. S6, insertion */
  else if (p->schedule == ORC_SCHED_WX) s = pow(1.0 - xi, n); /* Eq. S7, insertion */
  else s = 1.0 - xi;                                          /* Eq. 2: constant v_f */
  return p->w_max * s;
}

/* ------------------------------------------------------------------------------------ */
/* Velocity Verlet with RATTLE for rigid waters                                          */
/* ------------------------------------------------------------------------------------ */
double orc_kinetic(const orc_params* p, int n, const double* v, const uint8_t* fly) {
  double K = 0.0;
  for (int i = 0; i < n; ++i) {
    if (fly && fly[i]) continue;
    double m = mass_of(p, i);
    K += 0.5 * m * p->mvv2e * (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2]);
  }
  return K;
}

static void kick(const orc_params* p, int n, double* v, const double* F, const uint8_t* fly, double h) {
  for (int i = 0; i < n; ++i) {
    if (fly && fly[i]) continue; /* flyers keep their 3D state (Sec. II.B.1) */
    double a = h / (mass_of(p, i) * p->mvv2e);
    for (int c = 0; c < 3; ++c) v[3 * i + c] += a * F[3 * i + c];
  }
}

static void drift(const orc_params* p, int n, double* x, const double* v, const uint8_t* fly, double h) {
  for (int i = 0; i < n; ++i) {
    if (fly && fly[i]) continue;
    for (int c = 0; c < 3; ++c) x[3 * i + c] = wrap(x[3 * i + c] + h * v[3 * i + c], p->L);
  }
}

/* the three distance constraints of a rigid water: (O,H1), (O,H2), (H1,H2) */
static void water_constraint(const orc_params* p, int k, int* a, int* b, double* d) {
  static const int A[3] = {0, 0, 1}, B[3] = {1, 2, 2};
  *a = A[k];
  *b = B[k];
  *d = (k < 2) ? p->d_oh : p->d_hh;
}

/* SHAKE position stage of RATTLE (Andersen 1983): after an unconstrained drift, iterate
 * pairwise corrections along the old bond vectors until every bond length holds; the
 * same impulse corrects the half-step velocities. xold holds positions before the drift. */
static void shake(const orc_params* p, double* x, double* v, const double* xold, double h, const uint8_t* fly) {
  for (int m = 0; m < p->n_water; ++m) {
    if (fly && fly[3 * m] == 1) continue; /* a flying water is frozen in 3D */
    for (int it = 0; it < 1000; ++it) {
      double worst = 0.0;
      for (int k = 0; k < 3; ++k) {
        int a, b;
        double d;
        water_constraint(p, k, &a, &b, &d);
        int ia = 3 * m + a, ib = 3 * m + b;
        double rn[3], ro[3], rn2 = 0.0, dot = 0.0;
        for (int c = 0; c < 3; ++c) {
          rn[c] = minimg(x[3 * ia + c] - x[3 * ib + c], p->L);
          ro[c] = minimg(xold[3 * ia + c] - xold[3 * ib + c], p->L);
          rn2 += rn[c] * rn[c];
          dot += rn[c] * ro[c];
        }
        double diff = rn2 - d * d;
        double rel = fabs(diff) / (d * d);
        if (rel > worst) worst = rel;
        double ima = 1.0 / mass_of(p, ia), imb = 1.0 / mass_of(p, ib);
        double gk = diff / (2.0 * dot * (ima + imb));
        for (int c = 0; c < 3; ++c) {
          x[3 * ia + c] = wrap(x[3 * ia + c] - gk * ima * ro[c], p->L);
          x[3 * ib + c] = wrap(x[3 * ib + c] + gk * imb * ro[c], p->L);
          v[3 * ia + c] -= gk * ima * ro[c] / h;
          v[3 * ib + c] += gk * imb * ro[c] / h;
        }
      }
      if (worst < 1e-14) break;
    }
  }
}

/* RATTLE velocity stage: remove the bond-parallel relative velocity of every constraint */
static void rattle_v(const orc_params* p, const double* x, double* v, const uint8_t* fly) {
  for (int m = 0; m < p->n_water; ++m) {
    if (fly && fly[3 * m] == 1) continue;
    for (int it = 0; it < 1000; ++it) {
      double worst = 0.0;
      for (int k = 0; k < 3; ++k) {
        int a, b;
        double d;
        water_constraint(p, k, &a, &b, &d);
        int ia = 3 * m + a, ib = 3 * m + b;
        double r[3], dv = 0.0;
        for (int c = 0; c < 3; ++c) {
          r[c] = minimg(x[3 * ia + c] - x[3 * ib + c], p->L);
          dv += r[c] * (v[3 * ia + c] - v[3 * ib + c]);
        }
        if (fabs(dv) / (d * d) > worst) worst = fabs(dv) / (d * d);
        double ima = 1.0 / mass_of(p, ia), imb = 1.0 / mass_of(p, ib);
        double kk = dv / (d * d * (ima + imb));
        for (int c = 0; c < 3; ++c) {
          v[3 * ia + c] -= kk * ima * r[c];
          v[3 * ib + c] += kk * imb * r[c];
        }
      }
      if (worst < 1e-15) break;
    }
  }
}

/* one velocity-Verlet step. Reading of the step order (not stated in the paper): kick with
 * F(x, w_k), drift, move the altitude to w_{k+1}, force F(x, w_{k+1}), kick.  This map is
 * exactly time-reversible under v -> -v with the reversed schedule. */
static void vv_step(const orc_params* p, int n, double* x, double* v, double* F, const uint8_t* fly,
                    double* w, double w_next, double* xold) {
  double h = p->dt;
  kick(p, n, v, F, fly, 0.5 * h);
  if (p->n_water) memcpy(xold, x, sizeof(double) * 3 * (size_t)(3 * p->n_water));
  drift(p, n, x, v, fly, h);
  if (p->n_water) shake(p, x, v, xold, h, fly);
  if (w && fly)
    for (int i = 0; i < n; ++i) w[i] = (fly[i] == 1) ? w_next : 0.0;
  orc_energy_forces(p, n, x, w, fly, F);
  kick(p, n, v, F, fly, 0.5 * h);
  if (p->n_water) rattle_v(p, x, v, fly);
}

/* atoms of a state with n_pairs exchange units: ion pairs, or particles in single mode */
static int n_atoms(const orc_params* p, int n_pairs) { return 3 * p->n_water + (p->single ? 1 : 2) * n_pairs; }

/* the parameters with the state's number of waters (water exchange: the count varies) */
static const orc_params* with_waters(const orc_params* p, const orc_state* s, orc_params* tmp) {
  if (!p->water_ex) return p;
  *tmp = *p;
  tmp->n_water = s->n_water;
  return tmp;
}

double orc_nve(const orc_params* p, orc_state* s, int64_t n_steps, double* e_trace) {
  orc_params pw;
  p = with_waters(p, s, &pw);
  int n = n_atoms(p, s->n_pairs);
  double* F = (double*)calloc(3 * (size_t)(n + 1), sizeof(double));
  double* xold = (double*)calloc(3 * (size_t)(n + 1), sizeof(double));
  double U = orc_energy_forces(p, n, s->x, NULL, NULL, F);
  for (int64_t k = 0; k < n_steps; ++k) {
    vv_step(p, n, s->x, s->v, F, NULL, NULL, 0.0, xold);
    if (e_trace) {
      U = orc_energy_forces(p, n, s->x, NULL, NULL, NULL);
      e_trace[k] = U + orc_kinetic(p, n, s->v, NULL);
    }
  }
  U = orc_energy_forces(p, n, s->x, NULL, NULL, NULL);
  free(F);
  free(xold);
  return U;
}

/* ------------------------------------------------------------------------------------ */
/* Thermostat for equilibrium MD: CSVR (Bussi, Donadio, Parrinello, JCP 126, 014101      */
/* (2007), Eq. A7).  The chi-square variate with (dof-1) degrees uses the gamma sampler */
/* of Marsaglia and Tsang (ACM TOMS 26, 363 (2000)).                                    */
/* ------------------------------------------------------------------------------------ */
static double chi2_draw(const orc_params* p, uint64_t step, double dof) {
  double k = 0.5 * dof; /* gamma shape; chi2(dof) = 2 Gamma(dof/2, 1) */
  if (k <= 0.0) return 0.0;
  double boost = 1.0;
  if (k < 1.0) k += 1.0; /* shape < 1 handled by the standard boost U^(1/k) */
  double d = k - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * d);
  double g = d;
  for (uint64_t attempt = 0; attempt < 4096; ++attempt) {
    uint64_t r[4];
    draw(p, step, attempt, ORC_PUR_GAMMA, r);
    double z = gauss_cos(r[0], r[1]);
    double t = 1.0 + c * z;
    if (t <= 0.0) continue;
    t = t * t * t;
    double u = u01_open(r[2]);
    if (log(u) < 0.5 * z * z + d - d * t + d * log(t)) {
      g = d * t;
      if (0.5 * dof < 1.0) boost = pow(u01_open(r[3]), 1.0 / (0.5 * dof));
      break;
    }
  }
  return 2.0 * g * boost;
}

static void csvr(const orc_params* p, int n, double* v, uint64_t step) {
  double dof = 3.0 * n - 3.0 * p->n_water;
  if (dof < 1.0 || p->tau_t <= 0.0) return;
  double K = orc_kinetic(p, n, v, NULL);
  if (K <= 0.0) return;
  double Kbar = 0.5 * dof / p->beta;
  double c = exp(-p->dt / p->tau_t);
  uint64_t r[4];
  draw(p, step, 0, ORC_PUR_THERMO, r);
  double R1 = gauss_cos(r[0], r[1]);
  double S = chi2_draw(p, step, dof - 1.0);
  double Knew = K + (1.0 - c) * (Kbar * (S + R1 * R1) / dof - K) +
                2.0 * R1 * sqrt(Kbar * K * (1.0 - c) * c / dof);
  double alpha = sqrt(Knew / K);
  if (R1 + sqrt(dof * K * c / (Kbar * (1.0 - c))) < 0.0) alpha = -alpha;
  for (int i = 0; i < 3 * n; ++i) v[i] *= alpha;
}

void orc_md(const orc_params* p, orc_state* s, int64_t n_steps) {
  orc_params pw;
  p = with_waters(p, s, &pw);
  int n = n_atoms(p, s->n_pairs);
  double* F = (double*)calloc(3 * (size_t)(n + 1), sizeof(double));
  double* xold = (double*)calloc(3 * (size_t)(n + 1), sizeof(double));
  orc_energy_forces(p, n, s->x, NULL, NULL, F);
  for (int64_t k = 0; k < n_steps; ++k) {
    vv_step(p, n, s->x, s->v, F, NULL, NULL, 0.0, xold);
    csvr(p, n, s->v, s->step_ctr);
    s->step_ctr++;
  }
  free(F);
  free(xold);
}

/* Maxwell-Boltzmann velocities (Sec. II.A): three normals per atom from the atom's own
 * counter; waters then lose their bond-parallel components (RATTLE projection). */
static void mb_velocity(const orc_params* p, int type, const uint64_t r[4], double v[3]) {
  double sd = sqrt(1.0 / (p->beta * p->mass[type] * p->mvv2e));
  v[0] = sd * gauss_cos(r[0], r[1]);
  v[1] = sd * gauss_sin(r[0], r[1]);
  v[2] = sd * gauss_cos(r[2], r[3]);
}

void orc_init_velocities(const orc_params* p, orc_state* s) {
  orc_params pw;
  p = with_waters(p, s, &pw);
  int n = n_atoms(p, s->n_pairs);
  for (int i = 0; i < n; ++i) {
    uint64_t r[4];
    draw(p, (uint64_t)i, 0, ORC_PUR_VINIT, r);
    mb_velocity(p, orc_atom_type(p, i), r, &s->v[3 * i]);
  }
  if (p->n_water) rattle_v(p, s->x, s->v, NULL);
}

/* ------------------------------------------------------------------------------------ */
/* NEMD along the altitude schedule (Sec. II.A, II.B.1)                                  */
/* ------------------------------------------------------------------------------------ */
static double nemd(const orc_params* p, int n, double* x, double* v, const uint8_t* fly, int insertion) {
  double* F = (double*)calloc(3 * (size_t)n, sizeof(double));
  double* w = (double*)calloc((size_t)n, sizeof(double));
  double* wbuf = (double*)calloc((size_t)n, sizeof(double));
  double* xold = (double*)calloc(3 * (size_t)n, sizeof(double));
  double w0 = orc_altitude(p, insertion, 0);
  for (int i = 0; i < n; ++i) w[i] = (fly[i] == 1) ? species_w(p, i, w0) : 0.0;
  orc_energy_forces(p, n, x, w, fly, F);
  double wprot = 0.0;
  for (int k = 0; k < p->n_f; ++k) {
    double wk = orc_altitude(p, insertion, k), wk1 = orc_altitude(p, insertion, k + 1);
    /* the protocol work of step k is taken at the drifted positions, where the altitude
     * switches from w_k to w_{k+1} */
    double h = p->dt;
    kick(p, n, v, F, fly, 0.5 * h);
    if (p->n_water) memcpy(xold, x, sizeof(double) * 9 * (size_t)p->n_water);
    drift(p, n, x, v, fly, h);
    if (p->n_water) shake(p, x, v, xold, h, fly);
    wprot += flyer_energy(p, n, x, fly, wk1, wbuf) - flyer_energy(p, n, x, fly, wk, wbuf);
    for (int i = 0; i < n; ++i) w[i] = (fly[i] == 1) ? species_w(p, i, wk1) : 0.0;
    orc_energy_forces(p, n, x, w, fly, F);
    kick(p, n, v, F, fly, 0.5 * h);
    if (p->n_water) rattle_v(p, x, v, fly);
  }
  free(F);
  free(w);
  free(wbuf);
  free(xold);
  return wprot;
}

double orc_nemd_path(const orc_params* p, orc_state* s, const int32_t* flyers, int n_flyers,
                     int insertion, double* U_end) {
  orc_params pw;
  p = with_waters(p, s, &pw);
  int n = n_atoms(p, s->n_pairs);
  uint8_t* fly = (uint8_t*)calloc((size_t)n, 1);
  for (int k = 0; k < n_flyers; ++k) fly[flyers[k]] = 1;
  double wprot = nemd(p, n, s->x, s->v, fly, insertion);
  if (U_end) {
    double* w = (double*)calloc((size_t)n, sizeof(double));
    double wf = orc_altitude(p, insertion, p->n_f);
    for (int i = 0; i < n; ++i) w[i] = fly[i] ? species_w(p, i, wf) : 0.0;
    *U_end = orc_energy_forces(p, n, s->x, w, fly, NULL);
    free(w);
  }
  free(fly);
  return wprot;
}

/* ------------------------------------------------------------------------------------ */
/* Bimodal flyer-distance bias (Sec. II.B.3)                                             */
/* ------------------------------------------------------------------------------------ */
double orc_bias_density(double alpha, double xb, double L, double x) {
  double sa = sqrt(alpha);
  double num = exp(-alpha * (x - xb) * (x - xb)) + exp(-alpha * (x + xb) * (x + xb));
  double den = erf(sa * (xb + 0.5 * L)) - erf(sa * (xb - 0.5 * L));
  return sqrt(alpha / M_PI) * num / den;
}

/* inverse error function: Winitzki's closed-form approximation (a = 0.147) as the start,
 * then Newton steps x <- x - (erf(x) - y) / (2/sqrt(pi) exp(-x^2)) */
double orc_erfinv(double y) {
  const double a = 0.147;
  double w = log((1.0 - y) * (1.0 + y));
  double t = 2.0 / (M_PI * a) + 0.5 * w;
  double x = copysign(sqrt(sqrt(t * t - w / a) - t), y);
  for (int k = 0; k < 6; ++k) {
    double d = 2.0 / sqrt(M_PI) * exp(-x * x);
    if (!(d > 0.0)) break;
    x -= (erf(x) - y) / d;
  }
  return x;
}

double orc_bias_offset(double alpha, double xb, double L, uint64_t r_mode, uint64_t r_u) {
  double c = (r_mode >> 63) ? xb : -xb;
  double sa = sqrt(alpha);
  double lo = erf(sa * (-0.5 * L - c)), hi = erf(sa * (0.5 * L - c));
  double u = ((double)(r_u >> 11) + 0.5) * 0x1.0p-53; /* in (0, 1) */
  return c + orc_erfinv(lo + u * (hi - lo)) / sa;
}

/* B^ins of the anion at xa relative to the cation at xc: V prod_i b(x_ac,i) (Eq. 14) */
static double bias_B(const orc_params* p, const double* xa, const double* xc) {
  double B = p->L * p->L * p->L;
  for (int k = 0; k < 3; ++k) B *= orc_bias_density(p->bias_alpha, p->bias_xb, p->L, minimg(xa[k] - xc[k], p->L));
  return B;
}

/* ------------------------------------------------------------------------------------ */
/* Learned insertion-site proposal (definitions in h4d_oracle.h)                         */
/* ------------------------------------------------------------------------------------ */
static int species_of(int type) { return type <= 2 ? type : -1; } /* water H is not counted */

/* cell coordinate of a fixed-point coordinate X: floor(X G / 2^32) */
static int cell_coord(uint32_t X, int G) { return (int)(((uint64_t)X * (uint64_t)G) >> 32); }

static int cell_of_atom(const double* x, double L, int G) {
  int gx = cell_coord(fixpt(x[0], L), G), gy = cell_coord(fixpt(x[1], L), G), gz = cell_coord(fixpt(x[2], L), G);
  return (gx * G + gy) * G + gz;
}

int orc_proposal_features(const orc_params* p, int G, int n, const double* x, int ex0, int ex1,
                          double* feat) {
  int nc = G * G * G;
  double h = p->L / G;
  memset(feat, 0, sizeof(double) * (size_t)nc * ORC_NFEAT);
  for (int a = 0; a < n; ++a) {
    if (a == ex0 || a == ex1) continue;
    int t = orc_atom_type(p, a);
    int sp = species_of(t);
    double qa = p->q[t];
    int g[3];
    for (int k = 0; k < 3; ++k) g[k] = cell_coord(fixpt(x[3 * a + k], p->L), G);
    for (int dx = -1; dx <= 1; ++dx)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dz = -1; dz <= 1; ++dz) {
          /* cell c = g + d sees this atom at neighbour offset -d */
          int c[3] = {(g[0] + dx + G) % G, (g[1] + dy + G) % G, (g[2] + dz + G) % G};
          double* f = feat + (size_t)((c[0] * G + c[1]) * G + c[2]) * ORC_NFEAT;
          int slot = (1 - dx) * 9 + (1 - dy) * 3 + (1 - dz);
          if (sp >= 0) f[sp * 27 + slot] += 0.25;
          if (qa != 0.0) {
            double d[3], r2 = 0.0;
            for (int k = 0; k < 3; ++k) {
              d[k] = minimg((c[k] + 0.5) * h - x[3 * a + k], p->L);
              r2 += d[k] * d[k];
            }
            double r = fmax(sqrt(r2), 0.5);
            for (int k = 0; k < 3; ++k) f[81 + k] += 0.1 * qa * d[k] / (r * r * r);
          }
        }
  }
  return 0;
}

/* round to bfloat16 (nearest, ties to even) through binary32 */
static double bf16r(double v) {
  float f = (float)v;
  uint32_t u;
  memcpy(&u, &f, 4);
  u += 0x7fffu + ((u >> 16) & 1u);
  u &= 0xffff0000u;
  memcpy(&f, &u, 4);
  return (double)f;
}

/* one dense layer y = act(x W + b) of nin -> nout (W row-major [nin][nout]) */
static void dense(const double* xin, int nin, const double* W, const double* b, int nout, int relu,
                  int bf16, double* y) {
  for (int j = 0; j < nout; ++j) {
    double s = 0.0;
    for (int i = 0; i < nin; ++i) {
      double wij = W[(size_t)i * nout + j];
      s += (bf16 ? bf16r(xin[i]) * bf16r(wij) : xin[i] * wij);
    }
    if (bf16) s = (double)((float)s + (float)b[j]);
    else s += b[j];
    y[j] = (relu && s < 0.0) ? 0.0 : s;
  }
}

int orc_proposal_logits(const orc_params* p, const orc_proposal* q, int n, const double* x,
                        int ex0, int ex1, double* logits) {
  int nc = q->G * q->G * q->G;
  double* feat = (double*)malloc(sizeof(double) * (size_t)nc * ORC_NFEAT);
  orc_proposal_features(p, q->G, n, x, ex0, ex1, feat);
  const double* W1 = q->w;
  const double* b1 = W1 + ORC_NFEAT * ORC_HID;
  const double* W2 = b1 + ORC_HID;
  const double* b2 = W2 + ORC_HID * ORC_HID;
  const double* W3 = b2 + ORC_HID;
  const double* b3 = W3 + ORC_HID * 2;
  double h1[ORC_HID], h2[ORC_HID];
  for (int c = 0; c < nc; ++c) {
    dense(feat + (size_t)c * ORC_NFEAT, ORC_NFEAT, W1, b1, ORC_HID, 1, q->bf16, h1);
    dense(h1, ORC_HID, W2, b2, ORC_HID, 1, q->bf16, h2);
    dense(h2, ORC_HID, W3, b3, 2, 0, q->bf16, logits + 2 * (size_t)c);
  }
  free(feat);
  return 0;
}

/* softmax weights e_k = exp(l_k - max l) of species s and their sum */
static double soft_weights(const double* logits, int s, int nc, double* e) {
  double m = -INFINITY, Z = 0.0;
  for (int k = 0; k < nc; ++k) m = fmax(m, logits[2 * k + s]);
  for (int k = 0; k < nc; ++k) {
    e[k] = exp(logits[2 * k + s] - m);
    Z += e[k];
  }
  return Z;
}

/* draw a cell of species s: with probability eps a uniform cell, else inverse CDF of the
 * softmax (first cell whose running sum exceeds u Z) */
static int draw_cell(const double* e, double Z, int nc, double eps, uint64_t r_mix, uint64_t r_cell) {
  if (u01(r_mix) < eps) return pick(r_cell, nc);
  double target = u01(r_cell) * Z, cum = 0.0;
  int last = 0;
  for (int k = 0; k < nc; ++k) {
    if (e[k] > 0.0) last = k;
    cum += e[k];
    if (cum > target) return k;
  }
  return last;
}

static double ln_qn(const double* e, double Z, int nc, double eps, int k) {
  return log(((1.0 - eps) * e[k] / Z + eps / nc) * nc);
}

/* a fixed-point coordinate uniform over the cell's coordinates: X in [ceil(g 2^32/G),
 * ceil((g+1) 2^32/G)) */
static uint32_t place_in_cell(int g, int G, uint32_t r32) {
  uint64_t lo = (((uint64_t)g << 32) + (uint64_t)G - 1) / (uint64_t)G;
  uint64_t hi = (((uint64_t)(g + 1) << 32) + (uint64_t)G - 1) / (uint64_t)G;
  return (uint32_t)(lo + (((uint64_t)r32 * (hi - lo)) >> 32));
}

/* ------------------------------------------------------------------------------------ */
/* One pair-exchange trial                                                               */
/* ------------------------------------------------------------------------------------ */
static void flip_all(double* v, int n) {
  for (int i = 0; i < 3 * n; ++i) v[i] = -v[i];
}

/* Trial t of this chain.  Draw table (counter {t, block, TRIAL, 0}):
 *   block 0: [0] top bit = insertion, [1] top bit = reverse momenta before NEMD,
 *            [2] top bit = reverse after the decision, [3] acceptance uniform in (0,1]
 *   block 1: deletion: [0] cation index, [1] anion index (uniform in [0,N));
 *            insertion: [0..2] cation x,y,z and [3] anion x as 32-bit box fractions
 *   block 2: insertion: [0..1] anion y,z
 *   blocks 3-4: Maxwell-Boltzmann velocities of the inserted cation and anion
 *   block 5: learned proposal only: [0], [1] choose the uniform component (u < eps) for
 *            the cation and the anion cell, [2], [3] draw the cation and the anion cell;
 *            the 32-bit draws of blocks 1-2 then place each ion inside its cell
 *   block 6: bimodal bias only: [0..2] top bit picks the mode (+x_b or -x_b) of the
 *            anion offset on x, y, z; the anion's position words of blocks 1-2 then
 *            drive the inverse CDF of that truncated Gaussian.  Deletion with the bias
 *            picks the anion by inverse CDF of B^ins with u01 of block 1 word 1.
 * Readings: insertion and deletion are proposed with probability 1/2 each; the cation
 * and the anion are chosen independently (Eq. 3 squares 1/(N+1)); the momentum
 * reversal flips every velocity with probability 1/2 before NEMD and again after the
 * decision, and a rejection restores the state saved after the first flip.
 * Delta H compares the equilibrium Hamiltonians of the two end states: for insertion
 * H_{N+1}(end, all 3D) - H_N(start, flyers absent); for deletion the reverse.  The
 * flyers' kinetic energy is left out: insertion draws it from Maxwell-Boltzmann and a
 * deletion discards it, so it cancels against the e^{-beta K}/N_k factors of Eqs. 3-4.
 */
static int trial_single(const orc_params* p, orc_state* s, orc_record* rec);
static int trial_water(const orc_params* p, orc_state* s, orc_record* rec);

int orc_trial_prop(const orc_params* p, const orc_proposal* q, orc_state* s, orc_record* rec,
                   double* site_feat, double* site_y) {
  if (p->water_ex) return trial_water(p, s, rec); /* likewise */
  if (p->single) return trial_single(p, s, rec); /* no proposal, bias or early rejection */
  uint64_t t = s->trial_ctr++;
  uint64_t b0[4], b1[4], b2[4], b3[4], b4[4], b5[4], b6[4];
  draw(p, t, 0, ORC_PUR_TRIAL, b0);
  draw(p, t, 1, ORC_PUR_TRIAL, b1);
  draw(p, t, 2, ORC_PUR_TRIAL, b2);
  draw(p, t, 3, ORC_PUR_TRIAL, b3);
  draw(p, t, 4, ORC_PUR_TRIAL, b4);
  draw(p, t, 5, ORC_PUR_TRIAL, b5);
  draw(p, t, 6, ORC_PUR_TRIAL, b6);
  int insertion = (int)(b0[0] >> 63);
  int flip_start = (int)(b0[1] >> 63), flip_end = (int)(b0[2] >> 63);
  double ln_u = log(u01_open(b0[3]));
  int N = s->n_pairs;
  int base = 3 * p->n_water;
  int n = n_atoms(p, N);
  double V = p->L * p->L * p->L;

  memset(rec, 0, sizeof(*rec));
  rec->move = insertion;
  rec->n_before = N;
  rec->n_after = N;
  rec->cation = rec->anion = -1;
  rec->cell_c = rec->cell_a = -1;
  rec->ln_u = ln_u;
  int learned = q && q->mode == 1;
  int biased = p->bias_alpha > 0.0 && !learned;
  int G = q ? q->G : 0, nc = G * G * G;
  double ln_q = 0.0;

  if (flip_start) flip_all(s->v, n);
  if ((!insertion && N == 0) || (insertion && N >= s->cap_pairs)) {
    rec->status = insertion ? 2 : 1;
    if (flip_end) flip_all(s->v, n);
    return 0;
  }

  int ntot = insertion ? n + 2 : n;
  double* xs = (double*)malloc(sizeof(double) * 3 * (size_t)ntot);
  double* vs = (double*)malloc(sizeof(double) * 3 * (size_t)ntot);
  memcpy(xs, s->x, sizeof(double) * 3 * (size_t)n);
  memcpy(vs, s->v, sizeof(double) * 3 * (size_t)n);
  uint8_t* fly = (uint8_t*)calloc((size_t)ntot, 1);
  double* w0 = (double*)calloc((size_t)ntot, sizeof(double));
  double Ustart, Uend, Kstart, Kend;
  int ci, ai;

  if (insertion) {
    ci = base + 2 * N;
    ai = ci + 1;
    double h = p->L / 4294967296.0;
    uint32_t X[6] = {(uint32_t)(b1[0] >> 32), (uint32_t)(b1[1] >> 32), (uint32_t)(b1[2] >> 32),
                     (uint32_t)(b1[3] >> 32), (uint32_t)(b2[0] >> 32), (uint32_t)(b2[1] >> 32)};
    if (learned) {
      /* draw the two cells from the proposal of the start state (flyers absent), then
       * place each ion uniformly inside its cell with the same 32-bit draws */
      double* lg = (double*)malloc(sizeof(double) * 2 * (size_t)nc);
      double* e = (double*)malloc(sizeof(double) * (size_t)nc);
      orc_proposal_logits(p, q, n, s->x, -1, -1, lg);
      for (int sp = 0; sp < 2; ++sp) {
        double Z = soft_weights(lg, sp, nc, e);
        int k = draw_cell(e, Z, nc, q->eps, b5[sp], b5[2 + sp]);
        ln_q += ln_qn(e, Z, nc, q->eps, k);
        int g[3] = {k / (G * G), (k / G) % G, k % G};
        for (int d = 0; d < 3; ++d) X[3 * sp + d] = place_in_cell(g[d], G, X[3 * sp + d]);
      }
      free(lg);
      free(e);
    }
    if (biased) {
      /* the anion at a biased offset from the cation, per axis, in 32-bit box units */
      for (int d = 0; d < 3; ++d) {
        double off = orc_bias_offset(p->bias_alpha, p->bias_xb, p->L, b6[d], d == 0 ? b1[3] : b2[d - 1]);
        int64_t k = (int64_t)nearbyint(off / p->L * 4294967296.0);
        X[3 + d] = (uint32_t)((uint64_t)((int64_t)X[d] + k) & 0xffffffffULL);
      }
    }
    for (int d = 0; d < 3; ++d) {
      s->x[3 * ci + d] = (double)X[d] * h;
      s->x[3 * ai + d] = (double)X[3 + d] * h;
    }
    if (q) {
      rec->cell_c = cell_of_atom(&s->x[3 * ci], p->L, G);
      rec->cell_a = cell_of_atom(&s->x[3 * ai], p->L, G);
      if (site_feat) {
        double* f = (double*)malloc(sizeof(double) * (size_t)nc * ORC_NFEAT);
        orc_proposal_features(p, G, n, s->x, -1, -1, f);
        memcpy(site_feat, f + (size_t)rec->cell_c * ORC_NFEAT, sizeof(double) * ORC_NFEAT);
        memcpy(site_feat + ORC_NFEAT, f + (size_t)rec->cell_a * ORC_NFEAT, sizeof(double) * ORC_NFEAT);
        free(f);
      }
    }
    double sdc = sqrt(1.0 / (p->beta * p->mass[0] * p->mvv2e));
    double sda = sqrt(1.0 / (p->beta * p->mass[1] * p->mvv2e));
    s->v[3 * ci + 0] = sdc * gauss_cos(b3[0], b3[1]);
    s->v[3 * ci + 1] = sdc * gauss_sin(b3[0], b3[1]);
    s->v[3 * ci + 2] = sdc * gauss_cos(b3[2], b3[3]);
    s->v[3 * ai + 0] = sda * gauss_sin(b3[2], b3[3]);
    s->v[3 * ai + 1] = sda * gauss_cos(b4[0], b4[1]);
    s->v[3 * ai + 2] = sda * gauss_sin(b4[0], b4[1]);
    fly[ci] = fly[ai] = 1;
    /* H_start: the N-pair system, flyers absent */
    Ustart = orc_energy_forces(p, n, s->x, NULL, NULL, NULL);
    Kstart = orc_kinetic(p, ntot, s->v, fly);
    /* early rejection: an anion inside the excluded cube is inserted instantaneously */
    rec->instant = in_excluded_volume(p, X, X + 3);
    rec->w_prot = rec->instant ? 0.0 : nemd(p, ntot, s->x, s->v, fly, 1);
    /* H_end: the N+1-pair system, everyone in 3D */
    Uend = orc_energy_forces(p, ntot, s->x, NULL, NULL, NULL);
    Kend = orc_kinetic(p, ntot, s->v, fly);
    if (biased) {
      /* B^ins / B^del of the reverse deletion, in the end state: the mean of B^ins over
       * the N+1 anions relative to the inserted cation (Eq. 15) */
      double sum = 0.0;
      for (int k = 0; k <= N; ++k) sum += bias_B(p, &s->x[3 * (base + 2 * k + 1)], &s->x[3 * ci]);
      ln_q = log(sum / (double)(N + 1));
    }
  } else {
    int c = pick(b1[0], N), a = pick(b1[1], N);
    if (biased) {
      /* the anion with probability B^ins(r_a,n | r_c) / sum_n B^ins (Eq. 15); the factor
       * B^ins / B^del is the mean of B^ins over the N anions of the start state */
      double* Bn = (double*)malloc(sizeof(double) * (size_t)N);
      double sum = 0.0;
      for (int k = 0; k < N; ++k) {
        Bn[k] = bias_B(p, &s->x[3 * (base + 2 * k + 1)], &s->x[3 * (base + 2 * c)]);
        sum += Bn[k];
      }
      double target = u01(b1[1]) * sum, cum = 0.0;
      a = N - 1;
      for (int k = 0; k < N; ++k) {
        cum += Bn[k];
        if (cum > target) { a = k; break; }
      }
      ln_q = log(sum / (double)N);
      free(Bn);
    }
    rec->cation = c;
    rec->anion = a;
    ci = base + 2 * c;
    ai = base + 2 * a + 1;
    fly[ci] = fly[ai] = 1;
    Ustart = orc_energy_forces(p, n, s->x, NULL, NULL, NULL);
    Kstart = orc_kinetic(p, n, s->v, fly);
    /* early rejection: the same cube classifies the pair to delete */
    uint32_t Xc[3], Xa[3];
    for (int d = 0; d < 3; ++d) {
      Xc[d] = fixpt(s->x[3 * ci + d], p->L);
      Xa[d] = fixpt(s->x[3 * ai + d], p->L);
    }
    rec->instant = in_excluded_volume(p, Xc, Xa);
    rec->w_prot = rec->instant ? 0.0 : nemd(p, n, s->x, s->v, fly, 0);
    /* H_end: the N-1-pair system, flyers absent */
    uint8_t* gone = (uint8_t*)calloc((size_t)n, 1);
    gone[ci] = gone[ai] = 2;
    Uend = orc_energy_forces(p, n, s->x, NULL, gone, NULL);
    Kend = orc_kinetic(p, n, s->v, fly);
    free(gone);
    if (q) {
      /* the reverse insertion would draw these cells from the end state, flyers removed */
      rec->cell_c = cell_of_atom(&s->x[3 * ci], p->L, G);
      rec->cell_a = cell_of_atom(&s->x[3 * ai], p->L, G);
      if (learned) {
        double* lg = (double*)malloc(sizeof(double) * 2 * (size_t)nc);
        double* e = (double*)malloc(sizeof(double) * (size_t)nc);
        orc_proposal_logits(p, q, n, s->x, ci, ai, lg);
        for (int sp = 0; sp < 2; ++sp) {
          double Z = soft_weights(lg, sp, nc, e);
          ln_q += ln_qn(e, Z, nc, q->eps, sp == 0 ? rec->cell_c : rec->cell_a);
        }
        free(lg);
        free(e);
      }
      if (site_feat) {
        double* f = (double*)malloc(sizeof(double) * (size_t)nc * ORC_NFEAT);
        orc_proposal_features(p, G, n, s->x, ci, ai, f);
        memcpy(site_feat, f + (size_t)rec->cell_c * ORC_NFEAT, sizeof(double) * ORC_NFEAT);
        memcpy(site_feat + ORC_NFEAT, f + (size_t)rec->cell_a * ORC_NFEAT, sizeof(double) * ORC_NFEAT);
        free(f);
      }
    }
  }
  double dH = (Uend + Kend) - (Ustart + Kstart);
  rec->dH = dH;
  /* Eqs. 6 and 8 with Lambda_s = 1; Delta M is defined in the insertion direction */
  double x_acc;
  if (insertion) {
    rec->beta_dM = p->beta * dH - 2.0 * log(V / (double)(N + 1));
    x_acc = -rec->beta_dM + p->beta_mu;
  } else {
    rec->beta_dM = -p->beta * dH - 2.0 * log(V / (double)N);
    x_acc = rec->beta_dM - p->beta_mu;
  }
  if (site_y) *site_y = insertion ? x_acc : -x_acc;
  /* the proposal density relative to uniform: q(site) G^3 per ion */
  x_acc += insertion ? -ln_q : ln_q;
  rec->ln_q = ln_q;
  rec->x_acc = x_acc;
  int accept = isfinite(dH) && (ln_u < x_acc) && !p->no_accept;
  if (!isfinite(dH)) rec->status = 3;
  if (accept) {
    if (insertion) {
      s->n_pairs = N + 1;
    } else {
      /* swap-with-last removal keeps the interleaved cation/anion layout */
      int lc = base + 2 * (N - 1), la = lc + 1;
      for (int k = 0; k < 3; ++k) {
        s->x[3 * ci + k] = s->x[3 * lc + k];
        s->v[3 * ci + k] = s->v[3 * lc + k];
        s->x[3 * ai + k] = s->x[3 * la + k];
        s->v[3 * ai + k] = s->v[3 * la + k];
      }
      s->n_pairs = N - 1;
    }
  } else {
    memcpy(s->x, xs, sizeof(double) * 3 * (size_t)n);
    memcpy(s->v, vs, sizeof(double) * 3 * (size_t)n);
  }
  rec->accepted = accept;
  rec->n_after = s->n_pairs;
  if (flip_end) flip_all(s->v, n_atoms(p, s->n_pairs));
  free(xs);
  free(vs);
  free(fly);
  free(w0);
  return 0;
}

/* Single-particle exchange (Sec. II.A: the Metropolis rule of Eqs. 3-8 translated to one
 * flying particle; the flyer keeps its 3D position, Sec. II.B.1).  Draw table (counter
 * {t, block, TRIAL, 0}):
 *   block 0: as for pairs ([0] insertion, [1] and [2] the two reversals, [3] the uniform)
 *   block 1: insertion: [0..2] x, y, z as 32-bit box fractions; deletion: [0] the particle
 *   block 3: Maxwell-Boltzmann velocity of the inserted particle ([0],[1] cos and sin, [2],[3] cos)
 * With one flyer the phase-space factor of Eqs. 3-4 appears once: insertion
 * beta dM = beta dH - ln(V/(N+1)), accepted iff ln u < -beta dM + beta mu; deletion
 * beta dM = -beta dH - ln(V/N), accepted iff ln u < beta dM - beta mu (Lambda = 1).
 * Delta H and the momentum reversals follow the readings of the pair trial. */
static int trial_single(const orc_params* p, orc_state* s, orc_record* rec) {
  uint64_t t = s->trial_ctr++;
  uint64_t b0[4], b1[4], b3[4];
  draw(p, t, 0, ORC_PUR_TRIAL, b0);
  draw(p, t, 1, ORC_PUR_TRIAL, b1);
  draw(p, t, 3, ORC_PUR_TRIAL, b3);
  int insertion = (int)(b0[0] >> 63);
  int flip_start = (int)(b0[1] >> 63), flip_end = (int)(b0[2] >> 63);
  double ln_u = log(u01_open(b0[3]));
  int N = s->n_pairs;
  int base = 3 * p->n_water;
  int n = n_atoms(p, N);
  double V = p->L * p->L * p->L;

  memset(rec, 0, sizeof(*rec));
  rec->move = insertion;
  rec->n_before = N;
  rec->n_after = N;
  rec->cation = rec->anion = -1;
  rec->cell_c = rec->cell_a = -1;
  rec->ln_u = ln_u;
  if (flip_start) flip_all(s->v, n);
  if ((!insertion && N == 0) || (insertion && N >= s->cap_pairs)) {
    rec->status = insertion ? 2 : 1;
    if (flip_end) flip_all(s->v, n);
    return 0;
  }
  int ntot = insertion ? n + 1 : n;
  double* xs = (double*)malloc(sizeof(double) * 3 * (size_t)ntot);
  double* vs = (double*)malloc(sizeof(double) * 3 * (size_t)ntot);
  memcpy(xs, s->x, sizeof(double) * 3 * (size_t)n);
  memcpy(vs, s->v, sizeof(double) * 3 * (size_t)n);
  uint8_t* fly = (uint8_t*)calloc((size_t)ntot, 1);
  double Ustart, Uend, Kstart, Kend;
  int fi;
  if (insertion) {
    fi = n;
    double h = p->L / 4294967296.0;
    for (int d = 0; d < 3; ++d) s->x[3 * fi + d] = (double)(uint32_t)(b1[d] >> 32) * h;
    double sd = sqrt(1.0 / (p->beta * p->mass[0] * p->mvv2e));
    s->v[3 * fi + 0] = sd * gauss_cos(b3[0], b3[1]);
    s->v[3 * fi + 1] = sd * gauss_sin(b3[0], b3[1]);
    s->v[3 * fi + 2] = sd * gauss_cos(b3[2], b3[3]);
    fly[fi] = 1;
    /* H_start: the N-particle system, flyer absent; H_end: N + 1 particles in 3D */
    Ustart = orc_energy_forces(p, n, s->x, NULL, NULL, NULL);
    Kstart = orc_kinetic(p, ntot, s->v, fly);
    rec->w_prot = nemd(p, ntot, s->x, s->v, fly, 1);
    Uend = orc_energy_forces(p, ntot, s->x, NULL, NULL, NULL);
    Kend = orc_kinetic(p, ntot, s->v, fly);
  } else {
    int k = pick(b1[0], N);
    fi = base + k;
    rec->cation = k;
    fly[fi] = 1;
    Ustart = orc_energy_forces(p, n, s->x, NULL, NULL, NULL);
    Kstart = orc_kinetic(p, n, s->v, fly);
    rec->w_prot = nemd(p, n, s->x, s->v, fly, 0);
    /* H_end: the N - 1-particle system, flyer absent */
    uint8_t* gone = (uint8_t*)calloc((size_t)n, 1);
    gone[fi] = 2;
    Uend = orc_energy_forces(p, n, s->x, NULL, gone, NULL);
    Kend = orc_kinetic(p, n, s->v, fly);
    free(gone);
  }
  double dH = (Uend + Kend) - (Ustart + Kstart);
  rec->dH = dH;
  double x_acc;
  if (insertion) {
    rec->beta_dM = p->beta * dH - log(V / (double)(N + 1));
    x_acc = -rec->beta_dM + p->beta_mu;
  } else {
    rec->beta_dM = -p->beta * dH - log(V / (double)N);
    x_acc = rec->beta_dM - p->beta_mu;
  }
  rec->x_acc = x_acc;
  int accept = isfinite(dH) && (ln_u < x_acc) && !p->no_accept;
  if (!isfinite(dH)) rec->status = 3;
  if (accept) {
    if (insertion) {
      s->n_pairs = N + 1;
    } else {
      int last = base + N - 1; /* swap-with-last removal */
      for (int d = 0; d < 3; ++d) {
        s->x[3 * fi + d] = s->x[3 * last + d];
        s->v[3 * fi + d] = s->v[3 * last + d];
      }
      s->n_pairs = N - 1;
    }
  } else {
    memcpy(s->x, xs, sizeof(double) * 3 * (size_t)n);
    memcpy(s->v, vs, sizeof(double) * 3 * (size_t)n);
  }
  rec->accepted = accept;
  rec->n_after = s->n_pairs;
  if (flip_end) flip_all(s->v, n_atoms(p, s->n_pairs));
  free(xs);
  free(vs);
  free(fly);
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Rigid-water exchange (Sec. II.A: the exchange rule with one flyer; Sec. II.C: a       */
/* flying rigid water gets Maxwell-Boltzmann velocities drawn in its molecular frame)    */
/* ------------------------------------------------------------------------------------ */

/* The water in its body frame: O at the origin, the H atoms in the xy plane at
 * (+-d_oh sin(theta/2), d_oh cos(theta/2), 0), so the y axis is the symmetry axis and the
 * body axes are principal axes.  com: centre of mass; I: principal moments about it. */
typedef struct {
  double h[2][3], com[3], M, I[3];
} water_body;

static void water_frame(const orc_params* p, water_body* b) {
  double sh = 0.5 * p->d_hh / p->d_oh, ch = sqrt(1.0 - sh * sh);
  double mO = p->mass[2], mH = p->mass[3];
  b->h[0][0] = p->d_oh * sh;
  b->h[1][0] = -p->d_oh * sh;
  b->h[0][1] = b->h[1][1] = p->d_oh * ch;
  b->h[0][2] = b->h[1][2] = 0.0;
  b->M = mO + 2.0 * mH;
  b->com[0] = b->com[2] = 0.0;
  b->com[1] = 2.0 * mH * p->d_oh * ch / b->M;
  double yo = -b->com[1], yh = p->d_oh * ch - b->com[1], xh = p->d_oh * sh;
  b->I[0] = mO * yo * yo + 2.0 * mH * yh * yh; /* sum m (y^2 + z^2) */
  b->I[1] = 2.0 * mH * xh * xh;                /* sum m (x^2 + z^2) */
  b->I[2] = b->I[0] + b->I[1];                 /* sum m (x^2 + y^2), planar body */
}

/* A uniformly distributed rotation from three uniforms: the unit quaternion
 * (sqrt(1-u1) sin 2 pi u2, sqrt(1-u1) cos 2 pi u2, sqrt(u1) sin 2 pi u3, sqrt(u1) cos 2 pi u3)
 * (Shoemake, Graphics Gems III, 1992) and its rotation matrix. */
static void random_rotation(double u1, double u2, double u3, double R[3][3]) {
  double a = sqrt(1.0 - u1), b = sqrt(u1);
  double qx = a * sin(2.0 * M_PI * u2), qy = a * cos(2.0 * M_PI * u2);
  double qz = b * sin(2.0 * M_PI * u3), qw = b * cos(2.0 * M_PI * u3);
  R[0][0] = 1.0 - 2.0 * (qy * qy + qz * qz);
  R[0][1] = 2.0 * (qx * qy - qw * qz);
  R[0][2] = 2.0 * (qx * qz + qw * qy);
  R[1][0] = 2.0 * (qx * qy + qw * qz);
  R[1][1] = 1.0 - 2.0 * (qx * qx + qz * qz);
  R[1][2] = 2.0 * (qy * qz - qw * qx);
  R[2][0] = 2.0 * (qx * qz - qw * qy);
  R[2][1] = 2.0 * (qy * qz + qw * qx);
  R[2][2] = 1.0 - 2.0 * (qx * qx + qy * qy);
}

/* Place an inserted water (atoms O, H, H at x[0..8], v[0..8]).  Position: the O at the
 * 32-bit box fractions of block 1 words 0-2; each H at the O's fixed-point coordinate plus
 * its rotated body offset rounded to the 32-bit grid.  Orientation: uniform, from the
 * three uniforms of block 2.  Velocities, drawn in the molecular frame and handed to the
 * lab frame: centre-of-mass velocity V with N(0, kT/M) per axis and angular velocity
 * omega with N(0, kT/I_k) on body axis k (six normals from blocks 3-4: V_x, V_y, V_z,
 * omega_x, omega_y, omega_z in the order of the pair draws); atom a moves with
 * V + R (omega x (a_body - com)). */
static void place_water(const orc_params* p, const uint64_t b1[4], const uint64_t b2[4], const uint64_t b3[4],
                        const uint64_t b4[4], double* x, double* v) {
  water_body wb;
  water_frame(p, &wb);
  double R[3][3];
  random_rotation(u01(b2[0]), u01(b2[1]), u01(b2[2]), R);
  double q = p->L / 4294967296.0;
  uint32_t XO[3];
  for (int d = 0; d < 3; ++d) {
    XO[d] = (uint32_t)(b1[d] >> 32);
    x[d] = (double)XO[d] * q;
  }
  for (int k = 0; k < 2; ++k)
    for (int d = 0; d < 3; ++d) {
      double off = R[d][0] * wb.h[k][0] + R[d][1] * wb.h[k][1] + R[d][2] * wb.h[k][2];
      int64_t dk = (int64_t)nearbyint(off / p->L * 4294967296.0);
      x[3 * (k + 1) + d] = (double)(uint32_t)(XO[d] + (uint32_t)dk) * q;
    }
  double kT = 1.0 / (p->beta * p->mvv2e);
  double sv = sqrt(kT / wb.M);
  double V[3] = {sv * gauss_cos(b3[0], b3[1]), sv * gauss_sin(b3[0], b3[1]), sv * gauss_cos(b3[2], b3[3])};
  double om[3] = {sqrt(kT / wb.I[0]) * gauss_sin(b3[2], b3[3]), sqrt(kT / wb.I[1]) * gauss_cos(b4[0], b4[1]),
                  sqrt(kT / wb.I[2]) * gauss_sin(b4[0], b4[1])};
  for (int a = 0; a < 3; ++a) {
    double r[3];
    for (int d = 0; d < 3; ++d) r[d] = (a == 0 ? 0.0 : wb.h[a - 1][d]) - wb.com[d];
    double u[3] = {om[1] * r[2] - om[2] * r[1], om[2] * r[0] - om[0] * r[2], om[0] * r[1] - om[1] * r[0]};
    for (int d = 0; d < 3; ++d) v[3 * a + d] = V[d] + R[d][0] * u[0] + R[d][1] * u[1] + R[d][2] * u[2];
  }
}

/* Trial t of a water-exchange chain.  Draws as for pairs: block 0 (move, reversals,
 * acceptance uniform); block 1: deletion [0] the water (uniform in [0, N_w)), insertion
 * [0..2] the O position; block 2: insertion [0..2] the orientation; blocks 3-4: the
 * velocities.  The flying water stays frozen in 3D (Sec. II.B.1 for ions, read the same
 * way for a molecule: no drift, no kick, no constraint step) while its altitude follows
 * the schedule; Delta H, the momentum reversals and the exponents are those of a single
 * particle (reading of Sec. II.A: V/(N_w+1) once), N counting waters.  Layout: the
 * inserted water is the last water, so the ions move up by three atoms; a deletion moves
 * the last water into the deleted slot and the ions down by three. */
static int trial_water(const orc_params* p, orc_state* s, orc_record* rec) {
  uint64_t t = s->trial_ctr++;
  uint64_t b0[4], b1[4], b2[4], b3[4], b4[4];
  draw(p, t, 0, ORC_PUR_TRIAL, b0);
  draw(p, t, 1, ORC_PUR_TRIAL, b1);
  draw(p, t, 2, ORC_PUR_TRIAL, b2);
  draw(p, t, 3, ORC_PUR_TRIAL, b3);
  draw(p, t, 4, ORC_PUR_TRIAL, b4);
  int insertion = (int)(b0[0] >> 63);
  int flip_start = (int)(b0[1] >> 63), flip_end = (int)(b0[2] >> 63);
  double ln_u = log(u01_open(b0[3]));
  int N = s->n_water;
  int n_ion = 2 * s->n_pairs;
  int n = 3 * N + n_ion;
  double V = p->L * p->L * p->L;

  memset(rec, 0, sizeof(*rec));
  rec->move = insertion;
  rec->n_before = N;
  rec->n_after = N;
  rec->cation = rec->anion = -1;
  rec->cell_c = rec->cell_a = -1;
  rec->ln_u = ln_u;
  if (flip_start) flip_all(s->v, n);
  if ((!insertion && N == 0) || (insertion && N >= s->cap_water)) {
    rec->status = insertion ? 2 : 1;
    if (flip_end) flip_all(s->v, n);
    return 0;
  }
  int ntot = insertion ? n + 3 : n;
  double* xs = (double*)malloc(sizeof(double) * 3 * (size_t)n);
  double* vs = (double*)malloc(sizeof(double) * 3 * (size_t)n);
  memcpy(xs, s->x, sizeof(double) * 3 * (size_t)n);
  memcpy(vs, s->v, sizeof(double) * 3 * (size_t)n);
  uint8_t* fly = (uint8_t*)calloc((size_t)ntot, 1);
  uint8_t* gone = (uint8_t*)calloc((size_t)ntot, 1);
  orc_params pt = *p; /* the layout of the trial: an inserted water counts among the waters */
  pt.n_water = insertion ? N + 1 : N;
  int m = insertion ? N : pick(b1[0], N);
  for (int a = 3 * m; a < 3 * m + 3; ++a) fly[a] = 1, gone[a] = 2;
  double Ustart, Uend, Kstart, Kend;
  if (insertion) {
    memmove(s->x + 9 * (N + 1), s->x + 9 * N, sizeof(double) * 3 * (size_t)n_ion);
    memmove(s->v + 9 * (N + 1), s->v + 9 * N, sizeof(double) * 3 * (size_t)n_ion);
    place_water(p, b1, b2, b3, b4, s->x + 9 * N, s->v + 9 * N);
    /* H_start: the N-water system, the flyer absent; H_end: N + 1 waters in 3D */
    Ustart = orc_energy_forces(&pt, ntot, s->x, NULL, gone, NULL);
    Kstart = orc_kinetic(&pt, ntot, s->v, fly);
    rec->w_prot = nemd(&pt, ntot, s->x, s->v, fly, 1);
    Uend = orc_energy_forces(&pt, ntot, s->x, NULL, NULL, NULL);
    Kend = orc_kinetic(&pt, ntot, s->v, fly);
  } else {
    rec->cation = m; /* the deleted water */
    Ustart = orc_energy_forces(&pt, n, s->x, NULL, NULL, NULL);
    Kstart = orc_kinetic(&pt, n, s->v, fly);
    rec->w_prot = nemd(&pt, n, s->x, s->v, fly, 0);
    Uend = orc_energy_forces(&pt, n, s->x, NULL, gone, NULL);
    Kend = orc_kinetic(&pt, n, s->v, fly);
  }
  double dH = (Uend + Kend) - (Ustart + Kstart);
  rec->dH = dH;
  double x_acc;
  if (insertion) {
    rec->beta_dM = p->beta * dH - log(V / (double)(N + 1));
    x_acc = -rec->beta_dM + p->beta_mu;
  } else {
    rec->beta_dM = -p->beta * dH - log(V / (double)N);
    x_acc = rec->beta_dM - p->beta_mu;
  }
  rec->x_acc = x_acc;
  int accept = isfinite(dH) && (ln_u < x_acc) && !p->no_accept;
  if (!isfinite(dH)) rec->status = 3;
  if (accept) {
    if (insertion) {
      s->n_water = N + 1;
    } else {
      memcpy(s->x + 9 * m, s->x + 9 * (N - 1), sizeof(double) * 9); /* swap-with-last */
      memcpy(s->v + 9 * m, s->v + 9 * (N - 1), sizeof(double) * 9);
      memmove(s->x + 9 * (N - 1), s->x + 9 * N, sizeof(double) * 3 * (size_t)n_ion);
      memmove(s->v + 9 * (N - 1), s->v + 9 * N, sizeof(double) * 3 * (size_t)n_ion);
      s->n_water = N - 1;
    }
  } else {
    memcpy(s->x, xs, sizeof(double) * 3 * (size_t)n);
    memcpy(s->v, vs, sizeof(double) * 3 * (size_t)n);
  }
  rec->accepted = accept;
  rec->n_after = s->n_water;
  if (flip_end) flip_all(s->v, 3 * s->n_water + n_ion);
  free(xs);
  free(vs);
  free(fly);
  free(gone);
  return 0;
}

int orc_trial(const orc_params* p, orc_state* s, orc_record* rec) {
  return orc_trial_prop(p, NULL, s, rec, NULL, NULL);
}

int orc_run_cycles_prop(const orc_params* p, const orc_proposal* q, orc_state* s, int64_t n_cycles,
                        int64_t n_eq, orc_record* recs) {
  for (int64_t c = 0; c < n_cycles; ++c) {
    if (n_eq > 0) orc_md(p, s, n_eq);
    orc_trial_prop(p, q, s, &recs[c], NULL, NULL);
  }
  return 0;
}

int orc_run_cycles(const orc_params* p, orc_state* s, int64_t n_cycles, int64_t n_eq, orc_record* recs) {
  return orc_run_cycles_prop(p, NULL, s, n_cycles, n_eq, recs);
}

/* ------------------------------------------------------------------------------------ */
/* Ewald sum (Sec. II.B.2, Eqs. 9-10)                                                    */
/* ------------------------------------------------------------------------------------ */
double orc_ewald(const orc_params* p, int n, const double* x, double alpha, int kmax, double rcut,
                 double* U_real, double* U_recip, double* U_self, double* U_excl, double* F_recip) {
  const double L = p->L, V = L * L * L, K = p->kcoul;
  double ur = 0.0, uk = 0.0, us = 0.0, ue = 0.0;
  double* q = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int i = 0; i < n; ++i) {
    q[i] = p->q[orc_atom_type(p, i)];
    us -= K * alpha / sqrt(M_PI) * q[i] * q[i];
  }
  /* real space and the intramolecular corrections */
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      double r2 = 0.0;
      for (int c = 0; c < 3; ++c) {
        double d = minimg(x[3 * j + c] - x[3 * i + c], L);
        r2 += d * d;
      }
      double r = sqrt(r2);
      if (excluded(p, i, j)) ue -= K * q[i] * q[j] * erf(alpha * r) / r;
      else if (r < rcut) ur += K * q[i] * q[j] * erfc(alpha * r) / r;
    }
  /* reciprocal space: every k = 2 pi n / L with 0 < max |n_d| <= kmax */
  if (F_recip) memset(F_recip, 0, sizeof(double) * 3 * (size_t)n);
  double* cs = (double*)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
  for (int nx = -kmax; nx <= kmax; ++nx)
    for (int ny = -kmax; ny <= kmax; ++ny)
      for (int nz = -kmax; nz <= kmax; ++nz) {
        if (nx == 0 && ny == 0 && nz == 0) continue;
        double k[3] = {2.0 * M_PI * nx / L, 2.0 * M_PI * ny / L, 2.0 * M_PI * nz / L};
        double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        double a = exp(-k2 / (4.0 * alpha * alpha)) / k2;
        double re = 0.0, im = 0.0;
        for (int j = 0; j < n; ++j) {
          double th = k[0] * x[3 * j] + k[1] * x[3 * j + 1] + k[2] * x[3 * j + 2];
          cs[2 * j] = cos(th);
          cs[2 * j + 1] = sin(th);
          re += q[j] * cs[2 * j];
          im += q[j] * cs[2 * j + 1];
        }
        uk += 2.0 * M_PI * K / V * a * (re * re + im * im);
        if (F_recip)
          for (int j = 0; j < n; ++j) {
            /* -d/dr_j of (2 pi K / V) a |S|^2 = (4 pi K q_j / V) a k (re sin - im cos) */
            double f = 4.0 * M_PI * K * q[j] / V * a * (re * cs[2 * j + 1] - im * cs[2 * j]);
            for (int c = 0; c < 3; ++c) F_recip[3 * j + c] += f * k[c];
          }
      }
  free(cs);
  free(q);
  if (U_real) *U_real = ur;
  if (U_recip) *U_recip = uk;
  if (U_self) *U_self = us;
  if (U_excl) *U_excl = ue;
  return ur + uk + us + ue;
}
