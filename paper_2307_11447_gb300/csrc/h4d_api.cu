// h4d_api.cu -- host side of the libh4d C ABI (declared in include/h4d.h): parameter
// checking, device buffers, launch plan, state transfer and checkpoints.  All simulation
// steps run in the kernels of h4d_engine.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/h4d.h"
#include "h4d_engine.cuh"

using namespace h4d;

// device buffers of the proposal network and its training (one set per context, or a
// temporary set for the stateless gradient entry point)
struct PropDev {
  float* w = nullptr;      // [kPropNW] FP32 masters
  float* m = nullptr;      // Adam first moments
  float* v = nullptr;      // Adam second moments
  float* grad = nullptr;   // [kPropNW]
  uint2* w1 = nullptr;
  uint2* w2 = nullptr;
  uint2* w3 = nullptr;
  uint2* w2t = nullptr;
  float* w3r = nullptr;
  float* b = nullptr;
  long long adam_t = 0;
  // grid
  int cells = 0;
  int4* cnt = nullptr;
  long long* fld = nullptr;
  float2* logit = nullptr;
  double2* chunk = nullptr;
  // records
  int n_rec = 0;
  float* rfeat = nullptr;
  double* ry = nullptr;
  int2* rmeta = nullptr;
  // training scratch for up to cap_rows rows
  int cap_rows = 0;
  int* valid = nullptr;
  int* n_valid = nullptr;
  float* bfeat = nullptr;
  float* btgt = nullptr;
  uint16_t *xT = nullptr, *h1T = nullptr, *dz1T = nullptr, *h2T = nullptr, *dz2T = nullptr, *dlT = nullptr;
  float* loss_rows = nullptr;
  double* loss = nullptr;
  float* fout = nullptr;  // [cells][96] feature dump of h4d_proposal_logits
};

static void prop_free_train(PropDev* P) {
  void* ptrs[] = {P->bfeat, P->btgt, P->xT, P->h1T, P->dz1T, P->h2T, P->dz2T, P->dlT, P->loss_rows};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  P->bfeat = P->btgt = nullptr;
  P->xT = P->h1T = P->dz1T = P->h2T = P->dz2T = P->dlT = nullptr;
  P->loss_rows = nullptr;
  P->cap_rows = 0;
}

static void prop_free(PropDev* P) {
  if (!P) return;
  prop_free_train(P);
  void* ptrs[] = {P->w, P->m, P->v, P->grad, P->w1, P->w2, P->w3, P->w2t, P->w3r, P->b, P->cnt, P->fld,
                  P->logit, P->chunk, P->rfeat, P->ry, P->rmeta, P->valid, P->n_valid, P->loss, P->fout};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete P;
}

#define CKP(x)                                 \
  do {                                         \
    if ((x) != cudaSuccess) return H4D_ECUDA; \
  } while (0)

static int prop_alloc_net(PropDev* P) {
  CKP(cudaMalloc(&P->w, kPropNW * sizeof(float)));
  CKP(cudaMalloc(&P->m, kPropNW * sizeof(float)));
  CKP(cudaMalloc(&P->v, kPropNW * sizeof(float)));
  CKP(cudaMalloc(&P->grad, kPropNW * sizeof(float)));
  CKP(cudaMalloc(&P->w1, 1536 * sizeof(uint2)));
  CKP(cudaMalloc(&P->w2, 1024 * sizeof(uint2)));
  CKP(cudaMalloc(&P->w3, 128 * sizeof(uint2)));
  CKP(cudaMalloc(&P->w2t, 1024 * sizeof(uint2)));
  CKP(cudaMalloc(&P->w3r, 128 * sizeof(float)));
  CKP(cudaMalloc(&P->b, 130 * sizeof(float)));
  CKP(cudaMalloc(&P->loss, sizeof(double)));
  CKP(cudaMemset(P->w, 0, kPropNW * sizeof(float)));
  CKP(cudaMemset(P->m, 0, kPropNW * sizeof(float)));
  CKP(cudaMemset(P->v, 0, kPropNW * sizeof(float)));
  return H4D_OK;
}

// training scratch for `rows` rows (a multiple of 16)
static int prop_ensure_rows(PropDev* P, int rows) {
  if (rows <= P->cap_rows) return H4D_OK;
  prop_free_train(P);
  const size_t r = (size_t)rows;
  CKP(cudaMalloc(&P->bfeat, r * 96 * sizeof(float)));
  CKP(cudaMalloc(&P->btgt, r * sizeof(float)));
  CKP(cudaMalloc(&P->xT, 96 * r * sizeof(uint16_t)));
  CKP(cudaMalloc(&P->h1T, 64 * r * sizeof(uint16_t)));
  CKP(cudaMalloc(&P->dz1T, 64 * r * sizeof(uint16_t)));
  CKP(cudaMalloc(&P->h2T, 64 * r * sizeof(uint16_t)));
  CKP(cudaMalloc(&P->dz2T, 64 * r * sizeof(uint16_t)));
  CKP(cudaMalloc(&P->dlT, 8 * r * sizeof(uint16_t)));
  CKP(cudaMalloc(&P->loss_rows, r * sizeof(float)));
  CKP(cudaMemset(P->dlT, 0, 8 * r * sizeof(uint16_t)));  // rows 2..7 of dl stay zero
  P->cap_rows = rows;
  return H4D_OK;
}

static PropNet prop_net(const PropDev* P) {
  PropNet n;
  n.w1 = P->w1; n.w2 = P->w2; n.w3 = P->w3; n.w2t = P->w2t; n.w3r = P->w3r; n.b = P->b;
  return n;
}

// loss and gradient of n records already in P->bfeat / P->btgt (rows_pad rows)
static int prop_loss_grad(PropDev* P, int n, int rows_pad, cudaStream_t s) {
  int rc = launch_prop_fwd_bwd(prop_net(P), P->bfeat, P->btgt, n, 1.0f / (float)n, P->xT, P->h1T, P->dz1T, P->h2T,
                               P->dz2T, P->dlT, P->loss_rows, rows_pad, s);
  if (rc) return rc;
  return launch_prop_wgrad(P->xT, P->h1T, P->dz1T, P->h2T, P->dz2T, P->dlT, P->loss_rows, rows_pad, P->grad,
                           P->loss, s);
}

struct h4d_ctx {
  h4d_params prm;
  uint64_t seed;
  cudaStream_t stream;
  bool own_stream = false;
  int sm_count = 152;
  // captured launches of h4d_run_trials / h4d_run_md, keyed by (cycles, n_eq, do_trial)
  std::map<std::tuple<long long, int, int>, cudaGraphExec_t> graphs;
  int R;
  int total_atoms;
  int max_nbr;
  int max_out;
  int cta_threads;
  int n_ctas;
  size_t smem;
  std::vector<Rep> rep_h;
  std::vector<Group> groups_h;
  std::vector<int> cta_groups_h;
  Eng eng;
  // device allocations
  Rep* d_rep = nullptr;
  Group* d_groups = nullptr;
  int* d_cta_groups = nullptr;
  uint4* d_pos = nullptr;
  float4* d_vhi = nullptr;
  float4* d_vlo = nullptr;
  float4* d_force = nullptr;
  uint4* d_pos_save = nullptr;
  float4* d_vhi_save = nullptr;
  float4* d_vlo_save = nullptr;
  uint4* d_ref = nullptr;
  uint16_t* d_nbr = nullptr;
  int* d_ncnt = nullptr;
  uint16_t* d_nbr_out = nullptr;
  int* d_ncnt_out = nullptr;
  uint4* d_ref_out = nullptr;
  uint16_t* d_lrank = nullptr;  // Verlet-row layout: rank of each atom, atom at each position
  uint16_t* d_lord = nullptr;
  double* d_red = nullptr;
  h4d_record* d_rec = nullptr;
  double* d_scratch = nullptr;
  unsigned long long* d_count = nullptr;
  // learned proposal: network (FP32 masters, Adam moments, packed bf16 fragments), grid,
  // training records and training scratch
  PropDev* prop = nullptr;
};

#define CK(x)                                  \
  do {                                         \
    if ((x) != cudaSuccess) return H4D_ECUDA; \
  } while (0)

static const double kTwo32 = 4294967296.0;

static uint32_t __float_as_uint_host(float f) {
  uint32_t u;
  std::memcpy(&u, &f, sizeof(u));
  return u;
}

// fixed-point box fraction of a coordinate (matches the criterion stated in h4d.h)
static uint32_t to_fixed(double x, double L) {
  double y = x - L * std::floor(x / L);
  if (y >= L) y -= L;
  double s = std::nearbyint(y / L * kTwo32);
  return (uint32_t)((uint64_t)s & 0xffffffffULL);
}

static double rmax_of(const h4d_params& p) { return std::max(p.rc_lj, p.rc_coul); }

static int check_params(const h4d_params* p) {
  if (!p) return H4D_EINVAL;
  if (p->system != H4D_SYS_LJ && p->system != H4D_SYS_AQ) return H4D_EINVAL;
  if (p->ntypes < 2 || p->ntypes > 4) return H4D_EINVAL;
  if (!(p->beta > 0) || !(p->dt > 0) || !(p->rc_lj > 0) || !(p->rc_coul > 0)) return H4D_EINVAL;
  if (p->n_f < 1 || p->w_max < 0 || p->skin < 0 || p->skin_outer < 0) return H4D_EINVAL;
  if (p->schedule < 0 || p->schedule > 2) return H4D_EINVAL;
  if (p->threads_per_atom != 0 && (p->threads_per_atom & (p->threads_per_atom - 1))) return H4D_EINVAL;
  if (p->threads_per_atom > 32) return H4D_EINVAL;
  for (int t = 0; t < p->ntypes; ++t)
    if (!(p->mass[t] > 0) || p->sig[t] < 0 || p->eps[t] < 0) return H4D_EINVAL;
  if (p->system == H4D_SYS_LJ) {
    // the LJ specialisation assumes equal sizes/energies and charges +q/-q
    if (p->sig[0] != p->sig[1] || p->eps[0] != p->eps[1] || p->q[0] != -p->q[1]) return H4D_EINVAL;
  }
  if (p->exchange != H4D_EXCHANGE_PAIR && p->exchange != H4D_EXCHANGE_SINGLE && p->exchange != H4D_EXCHANGE_WATER)
    return H4D_EINVAL;
  // rigid-water exchange needs the water model: the aqueous system with its bond lengths
  if (p->exchange == H4D_EXCHANGE_WATER &&
      (p->system != H4D_SYS_AQ || p->ntypes < 4 || !(p->d_oh > 0) || !(p->d_hh > 0) || !(p->d_hh < 2 * p->d_oh)))
    return H4D_EINVAL;
  // single particles: one neutral species (a lone charge would leave the box charged)
  if (p->exchange == H4D_EXCHANGE_SINGLE && (p->system != H4D_SYS_LJ || p->q[0] != 0.0 || p->q[1] != 0.0))
    return H4D_EINVAL;
  return H4D_OK;
}

// atoms per exchange unit
static int unit_of(const h4d_params& p) { return p.exchange == H4D_EXCHANGE_SINGLE ? 1 : 2; }

// ratio of the anion's w_max to the cation's: (w_max + 0.5 (sig_c + sig_a) f_w) / w_max
static double species_rw(const h4d_params& p, double f_w) {
  if (!(f_w > 0) || !(p.w_max > 0)) return 1.0;
  return 1.0 + 0.5 * (p.sig[0] + p.sig[1]) * f_w / p.w_max;
}

// Screened-Coulomb force term of the LJ electrolyte as a polynomial.  With x = alpha r,
//   -du/dr / r = kq g (erfc(x) + 2x/sqrt(pi) e^{-x^2}) / r^3 = kq g (r^-3 + alpha^3 H(x^2)),
//   H(v) = (erfc(x) + 2x/sqrt(pi) e^{-v} - 1) / x^3 = -(4/sqrt(pi)) sum_n (-v)^n / ((2n + 3) n!),
// an entire function of v = x^2 (the bracket is 1 - (4/sqrt(pi)) int_0^x t^2 e^{-t^2} dt, odd
// in x from x^3 on).  C(s) = alpha^3 H(alpha^2 s) is interpolated in s = r^2 at the 8
// Chebyshev nodes of [0, rc^2]; the kernel then needs one rsqrt per pair and no exp, rcp or
// erfc.  The float evaluation of r^-3 + C loses 1/G(alpha rc) to cancellation at the
// cut-off, so the form is used for alpha rc <= 1.3 (relative error of the polynomial below
// 2e-7 there); otherwise the kernel keeps the erfc form.
static double coul_H(double v) {
  double s = 0.0, term = 1.0;  // term = v^n / n!
  for (int n = 0; n < 400; ++n) {
    s += ((n & 1) ? -term : term) / (2 * n + 3);
    term *= v / (n + 1);
    if (n > 4 && term < 1e-20) break;
  }
  return -4.0 / std::sqrt(M_PI) * s;
}

// fills cp[0..7] and returns 1 when the polynomial form applies to (alpha, rc), else 0
static int fit_coul_poly(double a, double rc, float* cp) {
  for (int j = 0; j < 8; ++j) cp[j] = 0.0f;
  if (!(rc > 0) || !(a >= 0) || a * rc > 1.3) return 0;
  const int D = 8;
  const double S = rc * rc;
  double A[D][D + 1];
  for (int k = 0; k < D; ++k) {  // interpolation conditions in u = s / S, u in [0, 1]
    const double u = 0.5 * (1.0 - std::cos(M_PI * (k + 0.5) / D));
    double pw = 1.0;
    for (int j = 0; j < D; ++j) { A[k][j] = pw; pw *= u; }
    A[k][D] = a * a * a * coul_H(a * a * u * S);
  }
  for (int col = 0; col < D; ++col) {  // Gaussian elimination, partial pivoting
    int piv = col;
    for (int r = col + 1; r < D; ++r)
      if (std::fabs(A[r][col]) > std::fabs(A[piv][col])) piv = r;
    for (int j = 0; j <= D; ++j) std::swap(A[col][j], A[piv][j]);
    for (int r = 0; r < D; ++r) {
      if (r == col) continue;
      const double f = A[r][col] / A[col][col];
      for (int j = col; j <= D; ++j) A[r][j] -= f * A[col][j];
    }
  }
  double c[D];
  double sc = 1.0;
  for (int j = 0; j < D; ++j) { c[j] = A[j][D] / A[j][j] / sc; sc *= S; }
  // check the interpolant against the series on a fine grid of r in (0, rc]
  double worst = 0.0;
  for (int k = 1; k <= 2000; ++k) {
    const double r = rc * k / 2000.0, s = r * r;
    double poly = 0.0;
    for (int j = D - 1; j >= 0; --j) poly = poly * s + c[j];
    const double exact = 1.0 / (r * r * r) + a * a * a * coul_H(a * a * s);
    worst = std::max(worst, std::fabs(poly - a * a * a * coul_H(a * a * s)) / std::fabs(exact));
  }
  if (!(worst < 2e-7)) return 0;
  for (int j = 0; j < D; ++j) cp[j] = (float)c[j];
  return 1;
}

static void fill_pot(const h4d_params& p, Pot& P, Proto& pr) {
  std::memset(&P, 0, sizeof(P));
  P.sys = p.system;
  P.ntypes = p.ntypes;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      int k = i * 4 + j;
      bool ok = i < p.ntypes && j < p.ntypes;
      double sig = ok ? 0.5 * (p.sig[i] + p.sig[j]) : 0.0;
      double eps = ok ? std::sqrt(p.eps[i] * p.eps[j]) : 0.0;
      double sc6 = (sig > 0) ? std::pow(sig / p.rc_lj, 6.0) : 0.0;
      double shift = 4.0 * eps * (sc6 * sc6 - sc6);
      double kq = ok ? p.kcoul * p.q[i] * p.q[j] : 0.0;
      P.dsig2[k] = sig * sig;
      P.deps4[k] = 4.0 * eps;
      P.dljshift[k] = shift;
      P.dkq[k] = kq;
      P.sig2[k] = (float)(sig * sig);
      P.eps4[k] = (float)(4.0 * eps);
      P.ljshift[k] = (float)shift;
      P.kq[k] = (float)kq;
    }
  if (p.system == H4D_SYS_LJ) {
    // LJ specialisation reads kq[0] for like and kq[1] for unlike charges
    P.kq[0] = (float)(p.kcoul * p.q[0] * p.q[0]);
    P.kq[1] = (float)(p.kcoul * p.q[0] * p.q[1]);
  }
  P.rc2_lj = (float)(p.rc_lj * p.rc_lj);
  P.rc2_c = (float)(p.rc_coul * p.rc_coul);
  P.rc2_max = std::max(P.rc2_lj, P.rc2_c);
  P.alpha = (float)p.alpha;
  P.shift_c = (float)(std::erfc(p.alpha * p.rc_coul) / p.rc_coul);
  P.two_alpha_sqrtpi = (float)(2.0 * p.alpha / std::sqrt(M_PI));
  P.kappa_sr = (float)p.kappa_sr;
  P.drc2_lj = p.rc_lj * p.rc_lj;
  P.drc2_c = p.rc_coul * p.rc_coul;
  P.dalpha = p.alpha;
  P.dshift_c = std::erfc(p.alpha * p.rc_coul) / p.rc_coul;
  P.dkappa_sr = p.kappa_sr;
  for (int t = 0; t < 4; ++t) {
    // single-particle exchange: both parities of the ion block are the one species
    const int tt = (p.exchange == H4D_EXCHANGE_SINGLE && t == 1) ? 0 : t;
    double m = (t < p.ntypes) ? p.mass[tt] * p.mvv2e : 1.0;
    P.dm[t] = m;
    P.inv_m[t] = (float)(1.0 / m);
    P.m_f[t] = (float)m;
    P.inv_m_d[t] = 1.0 / m;
  }
  P.d_oh2 = p.d_oh * p.d_oh;
  P.d_hh2 = p.d_hh * p.d_hh;
  for (int t = 0; t < 4; ++t) P.q[t] = (t < p.ntypes) ? (float)p.q[t] : 0.f;
  P.erfcx_fit = p.alpha * p.rc_coul <= 3.2 ? 1 : 0;  // the fit's range (fit_erfcx.py)
  P.coul_poly = (p.system == H4D_SYS_LJ) ? fit_coul_poly(p.alpha, p.rc_coul, P.cpoly) : 0;
  P.lj12 = 12.0f * P.eps4[0];
  P.lj6 = 6.0f * P.eps4[0];
  std::memset(&pr, 0, sizeof(pr));
  pr.n_f = p.n_f;
  pr.schedule = p.schedule;
  pr.w_max = p.w_max;
  pr.sched_n = p.sched_n;
  pr.dt = p.dt;
  pr.tau_t = p.tau_t;
  pr.beta = p.beta;
  pr.beta_mu = p.beta_mu;
  pr.rw = 1.0;
  pr.single = p.exchange == H4D_EXCHANGE_SINGLE;
  pr.unit = unit_of(p);
  pr.water = p.exchange == H4D_EXCHANGE_WATER;
  if (pr.water) {
    // body frame of the rigid water: O at the origin, H at (+-d_oh sin(t/2), d_oh cos(t/2), 0)
    const double sh = 0.5 * p.d_hh / p.d_oh, ch = std::sqrt(1.0 - sh * sh);
    const double mO = p.mass[2], mH = p.mass[3];
    pr.wh[0][0] = p.d_oh * sh;
    pr.wh[1][0] = -p.d_oh * sh;
    pr.wh[0][1] = pr.wh[1][1] = p.d_oh * ch;
    pr.wh[0][2] = pr.wh[1][2] = 0.0;
    const double M = mO + 2.0 * mH;
    pr.wcom_y = 2.0 * mH * p.d_oh * ch / M;
    const double yo = -pr.wcom_y, yh = p.d_oh * ch - pr.wcom_y, xh = p.d_oh * sh;
    const double Ix = mO * yo * yo + 2.0 * mH * yh * yh;  // about x: sum m (y^2 + z^2)
    const double Iy = 2.0 * mH * xh * xh;                 // about y: sum m (x^2 + z^2)
    // mass and moments times mvv2e: the velocity draw of an insertion has
    // var V = 1 / (beta M mvv2e) and var omega_k = 1 / (beta I_k mvv2e)
    pr.wM = M * p.mvv2e;
    pr.wI[0] = Ix * p.mvv2e;
    pr.wI[1] = Iy * p.mvv2e;
    pr.wI[2] = (Ix + Iy) * p.mvv2e;  // about z (a planar body)
  }
}

// neighbour-row capacity from the densest plausible packing (about one particle per sigma^3
// for the LJ electrolyte, liquid water for the aqueous system)
static double outer_skin(const h4d_params& p) {
  return std::max(p.skin_outer > 0 ? p.skin_outer : 4.0 * p.skin, p.skin);
}

static int derive_max_rows(const h4d_params& p, double rl) {
  double rho = (p.system == H4D_SYS_LJ) ? 1.05 / std::pow(p.sig[0], 3) : 0.105;
  int m = (int)std::ceil(4.0 / 3.0 * M_PI * rl * rl * rl * rho * 1.1) + 16;
  return ((m + 127) / 128) * 128;
}

static int derive_max_nbr(const h4d_params& p) {
  double rl = rmax_of(p) + p.skin;
  double rho = (p.system == H4D_SYS_LJ) ? 1.05 / std::pow(p.sig[0], 3) : 0.105;
  int m = (int)std::ceil(4.0 / 3.0 * M_PI * rl * rl * rl * rho * 1.1) + 16;
  return ((m + 31) / 32) * 32;
}

static int choose_tpa(const h4d_params& p, int n_atoms) {
  if (p.threads_per_atom > 0) return p.threads_per_atom;
  if (n_atoms >= 2048) return 4;
  if (n_atoms >= 512) return 8;
  return 16;
}

static int choose_threads(int n_atoms) {
  if (n_atoms >= 2048) return 512;
  if (n_atoms >= 256) return 256;
  return 128;
}

static void set_rep_geometry(const h4d_params& p, Rep& r, double L) {
  r.L = L;
  r.scale = (float)(L / kTwo32);
  r.c_drift = (float)(p.dt * kTwo32 / L);
  double rl = rmax_of(p) + p.skin;
  double ro = rmax_of(p) + outer_skin(p);
  // cells (for the outer list) of at least r_outer with a 3^3 stencil, else all pairs;
  // capped so the cell table stays small in shared memory (bigger cells remain valid)
  int nc1 = std::min((int)std::floor(L / ro), 8);
  if (nc1 >= 3) { r.nc = nc1; r.reach = 1; }
  else { r.nc = 0; r.reach = 0; }
  double s = rl / L * kTwo32;
  r.T_list = (unsigned long long)(s * s);
  double h = 0.5 * p.skin / L * kTwo32;
  r.T_move = (unsigned long long)(h * h);
  r.skin_fx = (float)(p.skin / L * kTwo32);
  double so = ro / L * kTwo32;
  r.T_out = (unsigned long long)(so * so);
  // 16-bit coordinates floor each difference, so |d16| <= |d|/q + 1 per axis and the
  // 16-bit length is at most |d|/q + sqrt(3); a radius of ceil(r/q) + 2 covers it
  double r16 = std::ceil(ro / L * 65536.0) + 2.0;
  r.T16_out = (unsigned)std::min(r16 * r16, 4.0e9);
  double r8 = std::ceil(ro / L * 256.0) + 2.0;  // same bound on 8-bit coordinates
  r.T8_out = (unsigned)std::min(r8 * r8, 4.0e9);
  r.skin_out_fx = (float)(outer_skin(p) / L * kTwo32);
}

static int alloc_all(h4d_ctx* c) {
  size_t na = (size_t)c->total_atoms;
  CK(cudaMalloc(&c->d_pos, na * sizeof(uint4)));
  CK(cudaMalloc(&c->d_vhi, na * sizeof(float4)));
  CK(cudaMalloc(&c->d_vlo, na * sizeof(float4)));
  CK(cudaMalloc(&c->d_force, na * sizeof(float4)));
  CK(cudaMalloc(&c->d_pos_save, na * sizeof(uint4)));
  CK(cudaMalloc(&c->d_vhi_save, na * sizeof(float4)));
  CK(cudaMalloc(&c->d_vlo_save, na * sizeof(float4)));
  CK(cudaMalloc(&c->d_ref, na * sizeof(uint4)));
  CK(cudaMalloc(&c->d_nbr, na * (size_t)c->max_nbr * sizeof(uint16_t)));
  CK(cudaMalloc(&c->d_ncnt, na * sizeof(int)));
  CK(cudaMalloc(&c->d_nbr_out, na * (size_t)c->max_out * sizeof(uint16_t)));
  CK(cudaMalloc(&c->d_ncnt_out, na * sizeof(int)));
  CK(cudaMalloc(&c->d_ref_out, na * sizeof(uint4)));
  CK(cudaMalloc(&c->d_lrank, na * sizeof(uint16_t)));
  CK(cudaMalloc(&c->d_lord, na * sizeof(uint16_t)));
  CK(cudaMalloc(&c->d_red, na * sizeof(double)));
  CK(cudaMemset(c->d_ncnt_out, 0, na * sizeof(int)));
  CK(cudaMemset(c->d_pos, 0, na * sizeof(uint4)));
  CK(cudaMemset(c->d_vhi, 0, na * sizeof(float4)));
  CK(cudaMemset(c->d_vlo, 0, na * sizeof(float4)));
  CK(cudaMemset(c->d_force, 0, na * sizeof(float4)));
  CK(cudaMemset(c->d_ncnt, 0, na * sizeof(int)));
  size_t nrec = 0;
  for (auto& r : c->rep_h) nrec += (size_t)r.rec_cap;
  CK(cudaMalloc(&c->d_rec, nrec * sizeof(h4d_record)));
  CK(cudaMemset(c->d_rec, 0, nrec * sizeof(h4d_record)));
  CK(cudaMalloc(&c->d_rep, c->rep_h.size() * sizeof(Rep)));
  CK(cudaMalloc(&c->d_groups, c->groups_h.size() * sizeof(Group)));
  CK(cudaMalloc(&c->d_cta_groups, (c->rep_h.size() + 1) * sizeof(int)));  // at most one CTA per replica
  CK(cudaMalloc(&c->d_scratch, 2 * c->rep_h.size() * sizeof(double)));
  CK(cudaMalloc(&c->d_count, sizeof(unsigned long long)));
  return H4D_OK;
}

static void fill_eng(h4d_ctx* c) {
  Eng& e = c->eng;
  fill_pot(c->prm, e.pot, e.proto);
  e.rows_by_index = 0;
  e.rep = c->d_rep;
  e.groups = c->d_groups;
  e.cta_groups = c->d_cta_groups;
  e.pos = c->d_pos;
  e.vhi = c->d_vhi;
  e.vlo = c->d_vlo;
  e.force = c->d_force;
  e.pos_save = c->d_pos_save;
  e.vhi_save = c->d_vhi_save;
  e.vlo_save = c->d_vlo_save;
  e.ref = c->d_ref;
  e.nbr = c->d_nbr;
  e.ncnt = c->d_ncnt;
  e.nbr_out = c->d_nbr_out;
  e.ncnt_out = c->d_ncnt_out;
  e.ref_out = c->d_ref_out;
  e.lrank = c->d_lrank;
  e.lord = c->d_lord;
  e.rec = c->d_rec;
  e.red = c->d_red;
  e.max_nbr = c->max_nbr;
  e.max_out = c->max_out;
  e.seed = c->seed;
}

static int push_plan(h4d_ctx* c) {
  CK(cudaMemcpyAsync(c->d_rep, c->rep_h.data(), c->rep_h.size() * sizeof(Rep), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->d_groups, c->groups_h.data(), c->groups_h.size() * sizeof(Group), cudaMemcpyHostToDevice,
                     c->stream));
  CK(cudaMemcpyAsync(c->d_cta_groups, c->cta_groups_h.data(), c->cta_groups_h.size() * sizeof(int),
                     cudaMemcpyHostToDevice, c->stream));
  return H4D_OK;
}

static int pull_reps(h4d_ctx* c) {
  CK(cudaMemcpyAsync(c->rep_h.data(), c->d_rep, c->rep_h.size() * sizeof(Rep), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return H4D_OK;
}

// Maxwell-Boltzmann draw on the host (3 normals per atom from Philox counter {atom, 0, 4, 0})
static void mulhilo(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
  __uint128_t p = (__uint128_t)a * b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}
static void philox_host(uint64_t c[4], uint64_t k0, uint64_t k1) {
  for (int r = 0; r < 10; ++r) {
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo(0xD2E7470EE14C6C93ULL, c[0], &hi0, &lo0);
    mulhilo(0xCA5A826395121157ULL, c[2], &hi1, &lo1);
    uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += 0x9E3779B97F4A7C15ULL;
    k1 += 0xBB67AE8584CAA73BULL;
  }
}
static double h_u01(uint64_t r) { return (double)(r >> 11) * 0x1.0p-53; }
static double h_u01o(uint64_t r) { return (double)((r >> 11) + 1) * 0x1.0p-53; }

static int atom_type_host(int a, int nw3, int unit) {
  return a < nw3 ? ((a % 3 == 0) ? 2 : 3) : (unit == 1 ? 0 : ((a - nw3) & 1));
}

static void split_ff(double v, float& hi, float& lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}

// Remove the bond-parallel relative velocities of every rigid water (the velocity stage
// of RATTLE), so that drawn Maxwell-Boltzmann velocities respect the constraints.
static double min_image(double d, double L) { return d - L * std::nearbyint(d / L); }
static void project_water_velocities(const h4d_params& p, int n_water, double L, const double* x, double* v) {
  const int A[3] = {0, 0, 1}, B[3] = {1, 2, 2};
  const double d2[3] = {p.d_oh * p.d_oh, p.d_oh * p.d_oh, p.d_hh * p.d_hh};
  const double im[3] = {1.0 / p.mass[2], 1.0 / p.mass[3], 1.0 / p.mass[3]};
  for (int m = 0; m < n_water; ++m) {
    for (int it = 0; it < 500; ++it) {
      double worst = 0.0;
      for (int q = 0; q < 3; ++q) {
        const int a = 3 * m + A[q], b = 3 * m + B[q];
        double rab[3], dv = 0.0;
        for (int k = 0; k < 3; ++k) {
          rab[k] = min_image(x[3 * a + k] - x[3 * b + k], L);
          dv += rab[k] * (v[3 * a + k] - v[3 * b + k]);
        }
        worst = std::max(worst, std::fabs(dv) / d2[q]);
        const double kk = dv / (d2[q] * (im[A[q]] + im[B[q]]));
        for (int k = 0; k < 3; ++k) {
          v[3 * a + k] -= kk * im[A[q]] * rab[k];
          v[3 * b + k] += kk * im[B[q]] * rab[k];
        }
      }
      if (worst < 1e-15) break;
    }
  }
}

static int upload_replica(h4d_ctx* c, int r, int n_pairs, const double* x, const double* v) {
  Rep& R = c->rep_h[r];
  if (n_pairs < 0 || n_pairs > R.cap_pairs) return H4D_ECAPACITY;
  R.n_pairs = n_pairs;
  R.err = 0;  // the error flags describe the state they were raised on
  int n = R.nw3 + unit_of(c->prm) * n_pairs;
  std::vector<uint4> pos(n);
  std::vector<float4> vh(n), vl(n);
  std::vector<double> vdraw(v ? 0 : 3 * (size_t)n);
  for (int a = 0; a < n; ++a) {
    pos[a] = make_uint4(to_fixed(x[3 * a], R.L), to_fixed(x[3 * a + 1], R.L), to_fixed(x[3 * a + 2], R.L), 0u);
    double vv[3];
    if (v) {
      vv[0] = v[3 * a]; vv[1] = v[3 * a + 1]; vv[2] = v[3 * a + 2];
    } else {
      uint64_t q[4] = {(uint64_t)a, 0, 4, 0};
      philox_host(q, c->seed, R.key);
      int t = atom_type_host(a, R.nw3, unit_of(c->prm));
      double sd = std::sqrt(1.0 / (c->prm.beta * c->prm.mass[t] * c->prm.mvv2e));
      double rad0 = std::sqrt(-2.0 * std::log(h_u01o(q[0])));
      double rad1 = std::sqrt(-2.0 * std::log(h_u01o(q[2])));
      vv[0] = sd * rad0 * std::cos(2.0 * M_PI * h_u01(q[1]));
      vv[1] = sd * rad0 * std::sin(2.0 * M_PI * h_u01(q[1]));
      vv[2] = sd * rad1 * std::cos(2.0 * M_PI * h_u01(q[3]));
      vdraw[3 * a] = vv[0]; vdraw[3 * a + 1] = vv[1]; vdraw[3 * a + 2] = vv[2];
    }
    if (!v && R.n_water > 0) continue;  // waters are projected below, then split
    float h, l;
    split_ff(vv[0], h, l); vh[a].x = h; vl[a].x = l;
    split_ff(vv[1], h, l); vh[a].y = h; vl[a].y = l;
    split_ff(vv[2], h, l); vh[a].z = h; vl[a].z = l;
    vh[a].w = vl[a].w = 0.f;
  }
  if (!v && R.n_water > 0) {
    project_water_velocities(c->prm, R.n_water, R.L, x, vdraw.data());
    for (int a = 0; a < n; ++a) {
      float h, l;
      split_ff(vdraw[3 * a], h, l); vh[a].x = h; vl[a].x = l;
      split_ff(vdraw[3 * a + 1], h, l); vh[a].y = h; vl[a].y = l;
      split_ff(vdraw[3 * a + 2], h, l); vh[a].z = h; vl[a].z = l;
      vh[a].w = vl[a].w = 0.f;
    }
  }
  if (n > 0) {
    CK(cudaMemcpyAsync(c->d_pos + R.atom_off, pos.data(), n * sizeof(uint4), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_vhi + R.atom_off, vh.data(), n * sizeof(float4), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_vlo + R.atom_off, vl.data(), n * sizeof(float4), cudaMemcpyHostToDevice, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  return H4D_OK;
}

static int check_device() {
  int dev = 0, ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return H4D_ENODEV;
  if (cudaGetDevice(&dev) != cudaSuccess) return H4D_ENODEV;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return H4D_ENODEV;
  if (!(prop.major == 10 && prop.minor == 3)) return H4D_ENODEV;
  return H4D_OK;
}

// Launch plan.  Every replica is simulated by a group of whole warps; groups are packed
// into CTAs (first-fit decreasing) with at most 15 groups (named barriers 1..15): two
// 16-warp CTAs of at most 113 KB shared memory per SM, or one 32-warp CTA per SM when a
// replica needs more shared memory than that (a large aqueous box) or the replicas are
// uneven (a batch of sizes more than 2x apart: its largest members can then have twice
// the warps).  (Measured on one GPU: equal 4000-ion chains run 31% slower as pairs of
// groups in 32-warp CTAs than in 16-warp CTAs of their own; the uneven batch of 256
// runs 36% faster in 32-warp CTAs.)
// A group's warp count follows the replica's weight (expected work, or the work the
// autotuner measured), out of the warps one resident wave of CTAs holds, so that uneven
// replicas finish together; rounding that would spill into a second wave shrinks the
// budget.  A group spanning a whole CTA uses __syncthreads.
static const size_t kCtaSmem = (size_t)113 * 1024;  // two CTAs per SM
static const int kCtaWarps = 16, kMaxCtaWarps = 32;

static double default_weight(const Rep& r) {
  // pair count ~ atoms x density
  const double n = (double)r.cap_atoms;
  return n * n / (r.L * r.L * r.L) + 1.0;
}

static void invalidate_graphs(h4d_ctx* c) {
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
}

static int make_plan(h4d_ctx* c, const std::vector<double>* weight = nullptr) {
  invalidate_graphs(c);
  const int R = c->R;
  std::vector<double> w(R);
  double W = 0.0;
  for (int r = 0; r < R; ++r) {
    w[r] = (weight && (*weight)[r] > 0) ? (*weight)[r] : default_weight(c->rep_h[r]);
    W += w[r];
  }
  size_t max_smem = 0;
  int min_atoms = 1 << 30, max_atoms = 0;
  for (int r = 0; r < R; ++r) {
    max_smem = std::max(max_smem, group_smem_bytes(c->rep_h[r].cap_atoms, c->rep_h[r].nc, 0));
    min_atoms = std::min(min_atoms, c->rep_h[r].cap_atoms);
    max_atoms = std::max(max_atoms, c->rep_h[r].cap_atoms);
  }
  // One 32-warp CTA per SM when a replica needs more shared memory than half an SM, and
  // for batches of uneven replicas: their large members then get up to twice the warps,
  // so the launch no longer waits on them alone.  Equal replicas keep two 16-warp CTAs.
  const bool uneven = max_atoms > 2 * min_atoms;
  const bool one_per_sm = max_smem > kCtaSmem || uneven;
  const int cta_warps = one_per_sm ? kMaxCtaWarps : kCtaWarps;
  const size_t cta_smem = one_per_sm ? (size_t)227 * 1024 : kCtaSmem;
  const int max_ctas = c->sm_count * (one_per_sm ? 1 : 2);  // one resident wave
  struct Item { int rep, nw; size_t smem; };
  struct Cta { int warps = 0; size_t smem = 0; std::vector<int> members; };
  std::vector<Item> items(R);
  std::vector<Cta> ctas;
  // resident warps of the GPU under this plan, shared out by weight; if rounding makes
  // the packing spill into a second wave of CTAs, shrink the budget and pack again
  double budget = (double)max_ctas * cta_warps;
  for (int attempt = 0; attempt < 64; ++attempt) {
    for (int r = 0; r < R; ++r) {
      int nw = (int)std::ceil(budget * w[r] / W);
      nw = std::max(1, std::min(cta_warps, nw));
      items[r] = {r, nw, group_smem_bytes(c->rep_h[r].cap_atoms, c->rep_h[r].nc, 32 * nw)};
      if (items[r].smem > 227 * 1024) return H4D_ECAPACITY;
    }
    std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& b) { return a.nw > b.nw; });
    ctas.clear();
    for (int k = 0; k < R; ++k) {
      const Item& it = items[k];
      int placed = -1;
      for (size_t q = 0; q < ctas.size() && placed < 0; ++q) {
        Cta& t = ctas[q];
        if (t.warps + it.nw <= cta_warps && (int)t.members.size() < kMaxGroupsPerCta &&
            t.smem + it.smem <= cta_smem)
          placed = (int)q;
      }
      if (placed < 0) { ctas.emplace_back(); placed = (int)ctas.size() - 1; }
      Cta& t = ctas[placed];
      t.members.push_back(k);
      t.warps += it.nw;
      t.smem += it.smem;
    }
    if ((int)ctas.size() <= max_ctas) break;
    budget *= 0.95;
  }
  c->groups_h.clear();
  c->cta_groups_h.clear();
  size_t smem = 0;
  for (auto& t : ctas) {
    c->cta_groups_h.push_back((int)c->groups_h.size());
    int warp0 = 0, bar = 1;
    size_t off = 0;
    const bool whole = t.members.size() == 1 && items[t.members[0]].nw == cta_warps;
    for (int k : t.members) {
      Group g;
      g.rep = items[k].rep;
      g.warp0 = warp0;
      g.nwarps = items[k].nw;
      g.bar = whole ? 0 : bar++;
      g.smem_off = (int)off;
      g.pad = 0;
      c->groups_h.push_back(g);
      warp0 += g.nwarps;
      off += items[k].smem;
    }
    smem = std::max(smem, off);
  }
  c->cta_groups_h.push_back((int)c->groups_h.size());
  c->n_ctas = (int)ctas.size();
  c->cta_threads = 32 * cta_warps;
  c->smem = smem;
  return H4D_OK;
}

extern "C" {

const char* h4d_strerror(int code) {
  switch (code) {
    case H4D_OK: return "ok";
    case H4D_EINVAL: return "invalid argument";
    case H4D_ECAPACITY: return "capacity exceeded (neighbour rows, shared memory or ion pairs)";
    case H4D_ETIMEOUT: return "bounded device loop gave up";
    case H4D_ENAN: return "non-finite state in equilibrium MD";
    case H4D_ECUDA: return "CUDA runtime error";
    case H4D_ENODEV: return "no sm_103 CUDA device";
    default: return "unknown error";
  }
}

int h4d_create(const h4d_params* params, const h4d_system* sys, uint64_t seed, void* cuda_stream, h4d_ctx** out) {
  if (!out) return H4D_EINVAL;
  *out = nullptr;
  int rc = check_params(params);
  if (rc) return rc;
  if (!sys || sys->n_replicas < 1 || !sys->L || !sys->n_pairs || !sys->cap_pairs || !sys->host_x) return H4D_EINVAL;
  rc = check_device();
  if (rc) return rc;
  h4d_ctx* c = new (std::nothrow) h4d_ctx();
  if (!c) return H4D_ECUDA;
  c->prm = *params;
  c->seed = seed;
  c->stream = (cudaStream_t)cuda_stream;
  if (!c->stream) {  // graph capture needs a stream other than the legacy default stream
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return H4D_ECUDA; }
    c->own_stream = true;
  }
  {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess)
      c->sm_count = prop.multiProcessorCount;
  }
  c->R = sys->n_replicas;
  c->max_nbr = params->max_nbr > 0 ? params->max_nbr : derive_max_nbr(*params);
  c->rep_h.resize(c->R);
  int off = 0;
  for (int r = 0; r < c->R; ++r) {
    Rep& R = c->rep_h[r];
    std::memset(&R, 0, sizeof(Rep));
    int nw = sys->n_water ? sys->n_water[r] : 0;
    int cw = sys->cap_water ? sys->cap_water[r] : nw;
    if (nw < 0 || cw < nw || sys->n_pairs[r] < 0 || sys->cap_pairs[r] < sys->n_pairs[r] || !(sys->L[r] > 0)) {
      h4d_destroy(c);
      return H4D_EINVAL;
    }
    if (cw > 0 && params->system != H4D_SYS_AQ) { h4d_destroy(c); return H4D_EINVAL; }
    if (cw != nw && params->exchange != H4D_EXCHANGE_WATER) { h4d_destroy(c); return H4D_EINVAL; }
    R.n_water = nw;
    R.nw3 = 3 * nw;
    R.cap_water = cw;
    R.n_pairs = sys->n_pairs[r];
    R.cap_pairs = sys->cap_pairs[r];
    R.cap_atoms = 3 * cw + unit_of(*params) * R.cap_pairs;
    if (R.cap_atoms > 65535 || R.cap_atoms < 1) { h4d_destroy(c); return H4D_ECAPACITY; }
    if (2.0 * (rmax_of(*params) + params->skin) >= sys->L[r]) { h4d_destroy(c); return H4D_EINVAL; }
    R.atom_off = off;
    off += R.cap_atoms;
    R.key = sys->replica_key ? sys->replica_key[r] : (uint64_t)r;
    set_rep_geometry(*params, R, sys->L[r]);
    R.tpa = choose_tpa(*params, R.cap_atoms);
    R.rec_cap = 1024;
    R.rec_off = r * R.rec_cap;
  }
  c->total_atoms = off;
  // rows are packed 4 per lane and tpa-interleaved: capacity is a multiple of 4 * 32
  c->max_nbr = ((c->max_nbr + 127) / 128) * 128;
  c->max_out = std::max(c->max_nbr, derive_max_rows(*params, rmax_of(*params) + outer_skin(*params)));
  rc = make_plan(c);
  if (rc) { h4d_destroy(c); return rc; }
  rc = alloc_all(c);
  if (rc) { h4d_destroy(c); return rc; }
  fill_eng(c);
  size_t xo = 0;
  for (int r = 0; r < c->R; ++r) {
    Rep& R = c->rep_h[r];
    rc = upload_replica(c, r, R.n_pairs, sys->host_x + xo, sys->host_v ? sys->host_v + xo : nullptr);
    if (rc) { h4d_destroy(c); return rc; }
    xo += 3 * (size_t)(R.nw3 + unit_of(*params) * R.n_pairs);
  }
  rc = push_plan(c);
  if (rc) { h4d_destroy(c); return rc; }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) { h4d_destroy(c); return H4D_ECUDA; }
  *out = c;
  return H4D_OK;
}

void h4d_destroy(h4d_ctx* c) {
  if (!c) return;
  void* ptrs[] = {c->d_rep, c->d_groups, c->d_cta_groups, c->d_pos, c->d_vhi, c->d_vlo, c->d_force,
                  c->d_pos_save, c->d_vhi_save, c->d_vlo_save, c->d_ref, c->d_nbr, c->d_ncnt, c->d_rec,
                  c->d_scratch, c->d_count, c->d_nbr_out, c->d_ncnt_out, c->d_ref_out, c->d_red,
                  c->d_lrank, c->d_lord};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  prop_free(c->prop);
  invalidate_graphs(c);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

int h4d_set_mu(h4d_ctx* c, double beta_mu) {
  if (!c || !std::isfinite(beta_mu)) return H4D_EINVAL;
  c->prm.beta_mu = beta_mu;
  c->eng.proto.beta_mu = beta_mu;
  invalidate_graphs(c);
  return H4D_OK;
}

int h4d_set_protocol(h4d_ctx* c, int32_t n_f, double w_max, double dt, double kappa_sr, int32_t schedule) {
  if (!c || n_f < 1 || !(w_max >= 0) || !(dt > 0) || !(kappa_sr >= 0) || schedule < 0 || schedule > 2)
    return H4D_EINVAL;
  c->prm.n_f = n_f;
  c->prm.w_max = w_max;
  c->prm.dt = dt;
  c->prm.kappa_sr = kappa_sr;
  c->prm.schedule = schedule;
  int rc = pull_reps(c);
  if (rc) return rc;
  for (auto& r : c->rep_h) r.c_drift = (float)(dt * kTwo32 / r.L);
  const Proto keep = c->eng.proto;
  fill_pot(c->prm, c->eng.pot, c->eng.proto);
  c->eng.proto.no_accept = keep.no_accept;
  c->eng.proto.prop_mode = keep.prop_mode;
  c->eng.proto.prop_record = keep.prop_record;
  c->eng.proto.prop_eps = keep.prop_eps;
  c->eng.proto.bias_on = keep.bias_on;
  c->eng.proto.bias_alpha = keep.bias_alpha;
  c->eng.proto.bias_xb = keep.bias_xb;
  c->eng.proto.fw = keep.fw;
  c->eng.proto.rw = species_rw(c->prm, keep.fw);
  c->eng.proto.vex_edge = keep.vex_edge;
  invalidate_graphs(c);
  return push_plan(c);
}

int h4d_set_species_wmax(h4d_ctx* c, double f_w) {
  if (c && (c->eng.proto.single || c->eng.proto.water) && f_w != 0.0) return H4D_EINVAL;  // a pair move
  if (!c || !std::isfinite(f_w) || f_w < 0 || (f_w > 0 && !(c->prm.w_max > 0))) return H4D_EINVAL;
  c->eng.proto.fw = f_w;
  c->eng.proto.rw = species_rw(c->prm, f_w);
  invalidate_graphs(c);
  return H4D_OK;
}

int h4d_set_bias(h4d_ctx* c, double alpha_b, double x_b) {
  if (c && (c->eng.proto.single || c->eng.proto.water) && alpha_b != 0.0) return H4D_EINVAL;  // a pair move
  if (!c || !std::isfinite(alpha_b) || !std::isfinite(x_b) || alpha_b < 0 || x_b < 0) return H4D_EINVAL;
  if (alpha_b > 0 && c->eng.proto.prop_mode) return H4D_EINVAL;  // one placement rule at a time
  c->eng.proto.bias_on = alpha_b > 0 ? 1 : 0;
  c->eng.proto.bias_alpha = alpha_b;
  c->eng.proto.bias_xb = x_b;
  invalidate_graphs(c);
  return H4D_OK;
}

int h4d_set_early_rejection(h4d_ctx* c, double v_ex) {
  if (c && (c->eng.proto.single || c->eng.proto.water) && v_ex != 0.0) return H4D_EINVAL;  // a pair move
  if (!c || !std::isfinite(v_ex) || v_ex < 0) return H4D_EINVAL;
  c->eng.proto.vex_edge = v_ex > 0 ? std::cbrt(v_ex) : 0.0;
  invalidate_graphs(c);
  return H4D_OK;
}

int h4d_set_no_accept(h4d_ctx* c, int32_t on) {
  if (!c) return H4D_EINVAL;
  c->eng.proto.no_accept = on ? 1 : 0;
  invalidate_graphs(c);
  return H4D_OK;
}

static int check_errors(h4d_ctx* c) {
  int rc = pull_reps(c);
  if (rc) return rc;
  for (auto& r : c->rep_h) {
    if (r.err & 1) return H4D_ECAPACITY;
    if (r.err & 4) return H4D_ETIMEOUT;  // the cause when a constraint solver gave up first
    if (r.err & 2) return H4D_ENAN;
  }
  return H4D_OK;
}

// persistent launch through a cached CUDA graph (captured on first use of a key)
static int run_cached(h4d_ctx* c, long long k, int n_eq, int do_trial) {
  const auto key = std::make_tuple(k, n_eq, do_trial);
  auto it = c->graphs.find(key);
  if (it == c->graphs.end()) {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int rc = launch_cycles(c->eng, c->n_ctas, c->cta_threads, c->smem, k, n_eq, do_trial, c->stream);
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
    if (rc || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return rc ? rc : H4D_ECUDA;
    }
    cudaError_t e3 = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) return H4D_ECUDA;
    it = c->graphs.emplace(key, ge).first;
  }
  CK(cudaGraphLaunch(it->second, c->stream));
  return H4D_OK;
}

int h4d_run_md(h4d_ctx* c, int64_t n_steps) {
  if (!c || n_steps < 0 || n_steps > (int64_t)1 << 30) return H4D_EINVAL;
  if (n_steps == 0) return H4D_OK;
  return run_cached(c, 1, (int)n_steps, 0);
}

int h4d_run_trials(h4d_ctx* c, int64_t k_cycles, int32_t n_eq) {
  if (!c || k_cycles < 0 || n_eq < 0) return H4D_EINVAL;
  if (k_cycles == 0) return H4D_OK;
  return run_cached(c, k_cycles, n_eq, 1);
}

int32_t h4d_num_replicas(h4d_ctx* c) { return c ? c->R : 0; }

int h4d_autotune(h4d_ctx* c, int32_t n_iter, double* pass_ns, double* build_ns) {
  if (!c || n_iter < 1 || n_iter > 100000) return H4D_EINVAL;
  int rc = pull_reps(c);
  if (rc) return rc;
  const std::vector<Rep> saved = c->rep_h;
  const int cand[5] = {1, 2, 4, 8, 16};
  std::vector<double> best_t(c->R, 1e300);
  std::vector<int> best(c->R, saved.empty() ? 4 : saved[0].tpa);
  for (int k = 0; k < 5; ++k) {
    for (int r = 0; r < c->R; ++r) {
      c->rep_h[r] = saved[r];
      c->rep_h[r].tpa = cand[k];
      c->rep_h[r].t_force_ns = 0.0;
      c->rep_h[r].t_build_ns = 0.0;
    }
    rc = push_plan(c);
    if (rc) return rc;
    rc = launch_forces(c->eng, c->n_ctas, c->cta_threads, c->smem, n_iter, c->stream);
    if (rc) return rc;
    rc = pull_reps(c);
    if (rc) return rc;
    double fsum = 0.0, bsum = 0.0;
    for (int r = 0; r < c->R; ++r) {
      if (c->rep_h[r].t_force_ns < best_t[r]) { best_t[r] = c->rep_h[r].t_force_ns; best[r] = cand[k]; }
      fsum += c->rep_h[r].t_force_ns;
      bsum += c->rep_h[r].t_build_ns;
    }
    if (pass_ns) pass_ns[k] = fsum / c->R / n_iter;
    if (build_ns) build_ns[k] = bsum / c->R;
  }
  for (int r = 0; r < c->R; ++r) {
    c->rep_h[r] = saved[r];
    c->rep_h[r].tpa = best[r];
  }
  // re-plan: a replica's weight is the work it measured (time x warps it had), so the
  // new warp counts equalise the time per step across replicas
  std::vector<double> weight(c->R);
  std::vector<int> nw_of(c->R, 1);
  for (const Group& g : c->groups_h) nw_of[g.rep] = g.nwarps;
  for (int r = 0; r < c->R; ++r) weight[r] = best_t[r] * nw_of[r];
  rc = make_plan(c, &weight);
  if (rc) return rc;
  rc = push_plan(c);
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->stream));
  return H4D_OK;
}

int h4d_get_counts(h4d_ctx* c, int32_t r, h4d_counts* out) {
  if (!c || !out || r < 0 || r >= c->R) return H4D_EINVAL;
  int rc = pull_reps(c);
  if (rc) return rc;
  const Rep& R = c->rep_h[r];
  out->n_pairs = R.n_pairs;
  out->cycles = R.cycles;
  out->trials_ins = R.trials_ins;
  out->trials_del = R.trials_del;
  out->accepted_ins = R.acc_ins;
  out->accepted_del = R.acc_del;
  out->rejected_status = R.rej_status;
  out->md_steps = R.md_steps;
  out->sum_n = R.sum_n;
  out->sum_n2 = R.sum_n2;
  out->nbr_builds = R.builds;
  out->error_flags = R.err;
  out->t_nemd_ns = R.t_nemd_ns;
  out->t_md_ns = R.t_md_ns;
  out->t_build_ns = R.t_build_ns;
  out->t_force_ns = R.t_force_ns;
  out->t_energy_ns = R.t_energy_ns;
  out->threads_per_atom = R.tpa;
  out->nbr_refreshes = R.refreshes;
  out->t_filter_ns = R.t_filter_ns;
  out->last_smid = R.smid;
  out->t_last_begin_ns = (double)R.t_begin;
  out->t_last_end_ns = (double)R.t_end;
  out->n_water = R.n_water;
  out->plan_warps = 0;
  out->plan_cta_groups = 0;
  for (size_t k = 0; k + 1 < c->cta_groups_h.size(); ++k)
    for (int g = c->cta_groups_h[k]; g < c->cta_groups_h[k + 1]; ++g)
      if (c->groups_h[g].rep == r) {
        out->plan_warps = c->groups_h[g].nwarps;
        out->plan_cta_groups = c->cta_groups_h[k + 1] - c->cta_groups_h[k];
      }
  return H4D_OK;
}

int h4d_get_energies(h4d_ctx* c, int32_t r, double* U, double* K) {
  if (!c || r < 0 || r >= c->R) return H4D_EINVAL;
  int rc = launch_energy(c->eng, c->n_ctas, c->cta_threads, c->smem, c->d_scratch, c->d_scratch + c->R, c->stream);
  if (rc) return rc;
  double u = 0, k = 0;
  CK(cudaMemcpyAsync(&u, c->d_scratch + r, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&k, c->d_scratch + c->R + r, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (U) *U = u;
  if (K) *K = k;
  return check_errors(c);
}

int h4d_get_work(h4d_ctx* c, int32_t r, h4d_record* out, int64_t cap, int64_t* n) {
  if (!c || r < 0 || r >= c->R || (cap > 0 && !out)) return H4D_EINVAL;
  int rc = pull_reps(c);
  if (rc) return rc;
  const Rep& R = c->rep_h[r];
  std::vector<h4d_record> buf(R.rec_cap);
  CK(cudaMemcpyAsync(buf.data(), c->d_rec + R.rec_off, R.rec_cap * sizeof(h4d_record), cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  int64_t have = std::min<int64_t>(R.rec_count, R.rec_cap);
  int64_t take = std::min<int64_t>(have, cap);
  for (int64_t k = 0; k < take; ++k) {
    int64_t idx = R.rec_count - take + k;
    out[k] = buf[idx % R.rec_cap];
  }
  if (n) *n = take;
  return H4D_OK;
}

int h4d_get_state(h4d_ctx* c, int32_t r, double* x, double* v, int64_t cap_atoms, int64_t* n_atoms) {
  if (!c || r < 0 || r >= c->R) return H4D_EINVAL;
  int rc = pull_reps(c);
  if (rc) return rc;
  const Rep& R = c->rep_h[r];
  int n = R.nw3 + unit_of(c->prm) * R.n_pairs;
  if (n_atoms) *n_atoms = n;
  if (n > cap_atoms) return H4D_ECAPACITY;
  std::vector<uint4> pos(n);
  std::vector<float4> vh(n), vl(n);
  if (n > 0) {
    CK(cudaMemcpyAsync(pos.data(), c->d_pos + R.atom_off, n * sizeof(uint4), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(vh.data(), c->d_vhi + R.atom_off, n * sizeof(float4), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(vl.data(), c->d_vlo + R.atom_off, n * sizeof(float4), cudaMemcpyDeviceToHost, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  const double h = R.L / kTwo32;
  for (int a = 0; a < n; ++a) {
    if (x) {
      x[3 * a] = (double)pos[a].x * h;
      x[3 * a + 1] = (double)pos[a].y * h;
      x[3 * a + 2] = (double)pos[a].z * h;
    }
    if (v) {
      v[3 * a] = (double)vh[a].x + (double)vl[a].x;
      v[3 * a + 1] = (double)vh[a].y + (double)vl[a].y;
      v[3 * a + 2] = (double)vh[a].z + (double)vl[a].z;
    }
  }
  return H4D_OK;
}

int h4d_set_state(h4d_ctx* c, int32_t r, int32_t n_pairs, const double* x, const double* v) {
  if (!c || r < 0 || r >= c->R || !x) return H4D_EINVAL;
  int rc = pull_reps(c);
  if (rc) return rc;
  rc = upload_replica(c, r, n_pairs, x, v);
  if (rc) return rc;
  return push_plan(c);
}

int h4d_set_water_state(h4d_ctx* c, int32_t r, int32_t n_water, int32_t n_pairs, const double* x, const double* v) {
  if (!c || r < 0 || r >= c->R || !x) return H4D_EINVAL;
  int rc = pull_reps(c);
  if (rc) return rc;
  Rep& R = c->rep_h[r];
  if (n_water < 0 || n_water > R.cap_water) return H4D_ECAPACITY;
  if (!c->eng.proto.water && n_water != R.n_water) return H4D_EINVAL;
  const int nw = R.n_water;
  R.n_water = n_water;
  R.nw3 = 3 * n_water;
  rc = upload_replica(c, r, n_pairs, x, v);
  if (rc) {
    R.n_water = nw;
    R.nw3 = 3 * nw;
    return rc;
  }
  return push_plan(c);
}

int h4d_count_pairs(h4d_ctx* c, int64_t* n) {
  if (!c || !n) return H4D_EINVAL;
  CK(cudaMemsetAsync(c->d_count, 0, sizeof(unsigned long long), c->stream));
  int rc = launch_count_pairs(c->eng, c->n_ctas, c->cta_threads, c->smem, c->d_count, c->stream);
  if (rc) return rc;
  unsigned long long v = 0;
  CK(cudaMemcpyAsync(&v, c->d_count, sizeof(v), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *n = (int64_t)v;
  return check_errors(c);
}

int h4d_coulomb_poly(double alpha, double rc_coul, float* coef, int32_t* used) {
  if (!coef || !used) return H4D_EINVAL;
  *used = fit_coul_poly(alpha, rc_coul, coef);
  return H4D_OK;
}

int h4d_device_info(int32_t* sm_count, int32_t* binary_version, int32_t* ptx_version) {
  if (!sm_count || !binary_version || !ptx_version) return H4D_EINVAL;
  int rc = check_device();
  if (rc) return rc;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(sm_count, cudaDevAttrMultiProcessorCount, dev));
  int b = 0, p = 0;
  rc = h4d::engine_binary_version(&b, &p);
  if (rc) return rc;
  *binary_version = b;
  *ptx_version = p;
  return H4D_OK;
}

// FP32 throughput probe: every thread runs 8 independent FMA chains (no memory traffic in
// the loop); the result is stored only when it equals a value it cannot reach, so the
// chains are kept but nothing is written
static __global__ void __launch_bounds__(256) fma_chain_kernel(int iters, float seed, float* sink) {
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = seed + 0.001f * (float)(threadIdx.x + k);
  const float m = 0.9999999f, d = 1e-7f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], m, d);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == -1.0f) sink[blockIdx.x] = s;
}

int h4d_measure_fp32_peak(double* tflops, double* seconds) {
  if (!tflops) return H4D_EINVAL;
  int rc = check_device();
  if (rc) return rc;
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  float* sink = nullptr;
  CK(cudaMalloc(&sink, sizeof(float) * (size_t)sms * 8));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = sms * 8, iters = 4096;  // 8 resident CTAs of 256 threads per SM
  fma_chain_kernel<<<blocks, 256>>>(16, 1.0f, sink);  // warm-up
  cudaEventRecord(e0);
  fma_chain_kernel<<<blocks, 256>>>(iters, 1.0f, sink);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (err != cudaSuccess || !(ms > 0.f)) return H4D_ECUDA;
  const double flops = 2.0 * 8.0 * 16.0 * (double)iters * 256.0 * (double)blocks;
  *tflops = flops / (ms * 1e-3) / 1e12;
  if (seconds) *seconds = ms * 1e-3;
  return H4D_OK;
}

// ---- checkpoint: a flat binary image of the replica table and per-atom state ----
static const uint64_t kMagic = 0x3530303044344848ULL;  // "HH4D0005"

int h4d_save(h4d_ctx* c, const char* path) {
  if (!c || !path) return H4D_EINVAL;
  int rc = pull_reps(c);
  if (rc) return rc;
  size_t na = (size_t)c->total_atoms;
  std::vector<uint4> pos(na);
  std::vector<float4> vh(na), vl(na);
  size_t nrec = (size_t)c->R * 1024;
  std::vector<h4d_record> rec(nrec);
  CK(cudaMemcpyAsync(pos.data(), c->d_pos, na * sizeof(uint4), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(vh.data(), c->d_vhi, na * sizeof(float4), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(vl.data(), c->d_vlo, na * sizeof(float4), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(rec.data(), c->d_rec, nrec * sizeof(h4d_record), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  FILE* f = std::fopen(path, "wb");
  if (!f) return H4D_EINVAL;
  uint64_t hdr[4] = {kMagic, (uint64_t)c->R, (uint64_t)na, c->seed};
  bool ok = std::fwrite(hdr, sizeof(hdr), 1, f) == 1;
  ok = ok && std::fwrite(c->rep_h.data(), sizeof(Rep), c->R, f) == (size_t)c->R;
  ok = ok && std::fwrite(pos.data(), sizeof(uint4), na, f) == na;
  ok = ok && std::fwrite(vh.data(), sizeof(float4), na, f) == na;
  ok = ok && std::fwrite(vl.data(), sizeof(float4), na, f) == na;
  ok = ok && std::fwrite(rec.data(), sizeof(h4d_record), nrec, f) == nrec;
  ok = (std::fclose(f) == 0) && ok;
  return ok ? H4D_OK : H4D_EINVAL;
}

int h4d_load(h4d_ctx* c, const char* path) {
  if (!c || !path) return H4D_EINVAL;
  FILE* f = std::fopen(path, "rb");
  if (!f) return H4D_EINVAL;
  uint64_t hdr[4];
  size_t na = (size_t)c->total_atoms;
  size_t nrec = (size_t)c->R * 1024;
  std::vector<Rep> reps(c->R);
  std::vector<uint4> pos(na);
  std::vector<float4> vh(na), vl(na);
  std::vector<h4d_record> rec(nrec);
  bool ok = std::fread(hdr, sizeof(hdr), 1, f) == 1 && hdr[0] == kMagic && hdr[1] == (uint64_t)c->R &&
            hdr[2] == (uint64_t)na;
  ok = ok && std::fread(reps.data(), sizeof(Rep), c->R, f) == (size_t)c->R;
  ok = ok && std::fread(pos.data(), sizeof(uint4), na, f) == na;
  ok = ok && std::fread(vh.data(), sizeof(float4), na, f) == na;
  ok = ok && std::fread(vl.data(), sizeof(float4), na, f) == na;
  ok = ok && std::fread(rec.data(), sizeof(h4d_record), nrec, f) == nrec;
  std::fclose(f);
  if (!ok) return H4D_EINVAL;
  for (int r = 0; r < c->R; ++r) {
    const Rep& cur = c->rep_h[r];
    const Rep& f = reps[r];
    // a checkpoint of the same system: its layout must be this context's, and the fields
    // the kernels index with must be in range
    if (f.atom_off != cur.atom_off || f.cap_atoms != cur.cap_atoms || f.cap_pairs != cur.cap_pairs ||
        f.cap_water != cur.cap_water || f.L != cur.L)
      return H4D_EINVAL;
    if (!c->eng.proto.water && f.n_water != cur.n_water) return H4D_EINVAL;
    if (f.n_water < 0 || f.n_water > cur.cap_water || f.nw3 != 3 * f.n_water) return H4D_EINVAL;
    if (f.n_pairs < 0 || f.n_pairs > cur.cap_pairs || f.rec_count < 0) return H4D_EINVAL;
    if (f.tpa < 1 || f.tpa > 32 || (f.tpa & (f.tpa - 1))) return H4D_EINVAL;  // lanes per row: 1..32, a power of two
    // only the chain's state and statistics come from the file; geometry, thresholds,
    // offsets, the proposal grid and the record rings stay this context's
    Rep m = cur;
    m.n_pairs = f.n_pairs;
    m.n_water = f.n_water;
    m.nw3 = f.nw3;
    m.tpa = f.tpa;
    m.rec_count = f.rec_count;
    m.trial_ctr = f.trial_ctr;
    m.step_ctr = f.step_ctr;
    m.key = f.key;
    m.cycles = f.cycles;
    m.trials_ins = f.trials_ins;
    m.trials_del = f.trials_del;
    m.acc_ins = f.acc_ins;
    m.acc_del = f.acc_del;
    m.rej_status = f.rej_status;
    m.md_steps = f.md_steps;
    m.builds = f.builds;
    m.refreshes = f.refreshes;
    m.err = f.err;
    m.sum_n = f.sum_n;
    m.sum_n2 = f.sum_n2;
    m.t_nemd_ns = f.t_nemd_ns;
    m.t_md_ns = f.t_md_ns;
    m.t_build_ns = f.t_build_ns;
    m.t_force_ns = f.t_force_ns;
    m.t_energy_ns = f.t_energy_ns;
    m.t_filter_ns = f.t_filter_ns;
    reps[r] = m;
  }
  c->seed = hdr[3];
  c->eng.seed = hdr[3];
  c->rep_h = reps;
  CK(cudaMemcpyAsync(c->d_pos, pos.data(), na * sizeof(uint4), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->d_vhi, vh.data(), na * sizeof(float4), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->d_vlo, vl.data(), na * sizeof(float4), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->d_rec, rec.data(), nrec * sizeof(h4d_record), cudaMemcpyHostToDevice, c->stream));
  int rc = push_plan(c);
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->stream));
  return H4D_OK;
}

// ---- stateless entry points ----
int h4d_eval_forces(const h4d_params* params, double L, int32_t n_water, int32_t n, const double* x,
                    const double* w, double* F, double* U) {
  int rc = check_params(params);
  if (rc) return rc;
  if (((!x || !F) && n > 0) || n < 0 || n_water < 0 || 3 * n_water > n || !(L > 0)) return H4D_EINVAL;
  if (unit_of(*params) == 2 && ((n - 3 * n_water) & 1) != 0) return H4D_EINVAL;
  if (2.0 * (rmax_of(*params) + params->skin) >= L) return H4D_EINVAL;
  if (n > 65535) return H4D_ECAPACITY;
  rc = check_device();
  if (rc) return rc;
  h4d_ctx* c = new (std::nothrow) h4d_ctx();
  if (!c) return H4D_ECUDA;
  c->prm = *params;
  c->seed = 0;
  c->stream = 0;
  c->R = 1;
  c->max_nbr = params->max_nbr > 0 ? params->max_nbr : derive_max_nbr(*params);
  c->max_nbr = ((c->max_nbr + 127) / 128) * 128;
  c->max_out = std::max(c->max_nbr, derive_max_rows(*params, rmax_of(*params) + outer_skin(*params)));
  c->rep_h.resize(1);
  Rep& R = c->rep_h[0];
  std::memset(&R, 0, sizeof(Rep));
  R.n_water = n_water;
  R.nw3 = 3 * n_water;
  R.cap_water = n_water;
  R.n_pairs = (n - 3 * n_water) / unit_of(*params);
  R.cap_pairs = R.n_pairs;
  R.cap_atoms = std::max(n, 1);
  R.atom_off = 0;
  set_rep_geometry(*params, R, L);
  R.tpa = choose_tpa(*params, n);
  R.rec_cap = 1;
  c->total_atoms = R.cap_atoms;
  rc = make_plan(c);
  if (rc) { delete c; return rc; }
  rc = alloc_all(c);
  if (rc) { h4d_destroy(c); return rc; }
  fill_eng(c);
  std::vector<uint4> pos(n);
  double wsum = 0.0;
  int wcnt = 0;
  for (int a = 0; a < n; ++a) {
    float wa = w ? (float)w[a] : 0.0f;
    if (wa != 0.0f) { wsum += w[a]; ++wcnt; }
    pos[a] = make_uint4(to_fixed(x[3 * a], L), to_fixed(x[3 * a + 1], L), to_fixed(x[3 * a + 2], L),
                        __float_as_uint_host(wa));
  }
  rc = H4D_OK;
  if (n > 0 && cudaMemcpy(c->d_pos, pos.data(), n * sizeof(uint4), cudaMemcpyHostToDevice) != cudaSuccess) rc = H4D_ECUDA;
  if (!rc) rc = push_plan(c);
  if (!rc) rc = launch_eval(c->eng, c->cta_threads, c->smem, (float)(wcnt ? wsum / wcnt : 0.0), c->d_scratch, 0);
  std::vector<float4> f(n);
  double u = 0.0;
  if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = H4D_ECUDA;
  if (!rc && n > 0 && cudaMemcpy(f.data(), c->d_force, n * sizeof(float4), cudaMemcpyDeviceToHost) != cudaSuccess) rc = H4D_ECUDA;
  if (!rc && cudaMemcpy(&u, c->d_scratch, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) rc = H4D_ECUDA;
  if (!rc) rc = check_errors(c);
  if (!rc) {
    for (int a = 0; a < n; ++a) {
      F[3 * a] = f[a].x;
      F[3 * a + 1] = f[a].y;
      F[3 * a + 2] = f[a].z;
    }
    if (U) *U = u;
  }
  h4d_destroy(c);
  return rc;
}

int h4d_neighbor_pairs(double L, int32_t n, const double* x, double r_list, int32_t* oi, int32_t* oj, int64_t cap,
                       int64_t* n_out) {
  if (!x || n < 0 || !(L > 0) || !(r_list > 0) || 2.0 * r_list >= L || (cap > 0 && (!oi || !oj))) return H4D_EINVAL;
  if (n > 65535) return H4D_ECAPACITY;
  int rc = check_device();
  if (rc) return rc;
  h4d_ctx* c = new (std::nothrow) h4d_ctx();
  if (!c) return H4D_ECUDA;
  std::memset(&c->prm, 0, sizeof(c->prm));
  c->prm.system = H4D_SYS_LJ;
  c->prm.ntypes = 2;
  c->prm.rc_lj = c->prm.rc_coul = r_list;
  c->prm.dt = 1.0;
  c->prm.beta = 1.0;
  c->prm.mvv2e = 1.0;
  c->prm.mass[0] = c->prm.mass[1] = 1.0;
  c->seed = 0;
  c->stream = 0;
  c->R = 1;
  c->max_nbr = ((std::min(std::max(n, 1), 4096) + 127) / 128) * 128;
  c->max_out = c->max_nbr;
  c->rep_h.resize(1);
  Rep& R = c->rep_h[0];
  std::memset(&R, 0, sizeof(Rep));
  int np = (n + 1) / 2;
  R.n_pairs = np;
  R.cap_pairs = np;
  R.cap_atoms = std::max(2 * np, 1);
  set_rep_geometry(c->prm, R, L);
  R.tpa = 1;
  R.rec_cap = 1;
  c->total_atoms = R.cap_atoms;
  rc = make_plan(c);
  if (rc) { delete c; return rc; }
  rc = alloc_all(c);
  if (rc) { h4d_destroy(c); return rc; }
  fill_eng(c);
  c->eng.rows_by_index = 1;  // rows read back below by atom index
  // atoms beyond n (odd n) are parked far away from every pair: they are dropped below
  std::vector<uint4> pos(R.cap_atoms);
  for (int a = 0; a < n; ++a)
    pos[a] = make_uint4(to_fixed(x[3 * a], L), to_fixed(x[3 * a + 1], L), to_fixed(x[3 * a + 2], L), 0u);
  for (int a = n; a < R.cap_atoms; ++a) pos[a] = pos[0];
  rc = H4D_OK;
  if (cudaMemcpy(c->d_pos, pos.data(), R.cap_atoms * sizeof(uint4), cudaMemcpyHostToDevice) != cudaSuccess) rc = H4D_ECUDA;
  if (!rc) rc = push_plan(c);
  if (!rc) rc = launch_list(c->eng, 1, c->cta_threads, c->smem, 0);
  if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = H4D_ECUDA;
  std::vector<int> cnt(R.cap_atoms);
  std::vector<uint16_t> nb((size_t)R.cap_atoms * c->max_nbr);
  if (!rc && cudaMemcpy(cnt.data(), c->d_ncnt, R.cap_atoms * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = H4D_ECUDA;
  if (!rc && cudaMemcpy(nb.data(), c->d_nbr, nb.size() * sizeof(uint16_t), cudaMemcpyDeviceToHost) != cudaSuccess) rc = H4D_ECUDA;
  if (!rc) rc = check_errors(c);
  if (!rc) {
    int64_t m = 0;
    for (int i = 0; i < n; ++i) {
      std::vector<int> row;
      for (int s = 0; s < cnt[i]; ++s) {
        int j = nb[((size_t)(s >> 2) * R.cap_atoms + i) * 4 + (s & 3)];  // tpa = 1 packet layout
        if (j > i && j < n) row.push_back(j);
      }
      std::sort(row.begin(), row.end());
      for (int j : row) {
        if (m < cap) { oi[m] = i; oj[m] = j; }
        ++m;
      }
    }
    if (n_out) *n_out = m;
  }
  h4d_destroy(c);
  return rc;
}

}  // extern "C"

// ------------------------------------------------------------------------------------
// h4d_eval_forces_static: the same computation as h4d_eval_forces for callers that must
// not allocate device memory (for example code running where cudaMalloc is forbidden or
// would break a memory budget they do not own).  Every device buffer it needs lives in
// one file-scope array of kStaticScratchBytes, which each GPU that loads the library
// holds until the process exits.
// ------------------------------------------------------------------------------------
static constexpr size_t kStaticScratchBytes = 16u << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_h4d_static_scratch[kStaticScratchBytes];

// The array's name in host code is only a host-side stand-in: its device address comes
// from cudaGetSymbolAddress, once per device, with that device current.
static std::mutex g_static_mu;
static void* g_static_addr[64];

static int static_scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return H4D_ECUDA;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_h4d_static_scratch) != cudaSuccess || !p) return H4D_ECUDA;
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return H4D_OK;
}

// doubles in, fixed-point box fractions out (same rule as to_fixed: wrap into [0, L),
// round x/L 2^32 to nearest, keep 32 bits); altitudes as FP32 bits
__global__ void static_convert_in(const double* x, const double* w, int n, double L, uint4* pos) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  unsigned f[3];
  for (int k = 0; k < 3; ++k) {
    double y = x[3 * a + k] - L * floor(x[3 * a + k] / L);
    if (y >= L) y -= L;
    const double sc = nearbyint(y / L * 4294967296.0);
    f[k] = (unsigned)((unsigned long long)sc & 0xffffffffULL);
  }
  const float wa = w ? (float)w[a] : 0.0f;
  pos[a] = make_uint4(f[0], f[1], f[2], __float_as_uint(wa));
}

__global__ void static_convert_out(const float4* f, int n, double* F) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  const float4 v = f[a];
  F[3 * a] = v.x;
  F[3 * a + 1] = v.y;
  F[3 * a + 2] = v.z;
}

static size_t carve_bytes(size_t& off, size_t bytes) {
  const size_t at = (off + 255) & ~(size_t)255;
  off = at + bytes;
  return at;
}

extern "C" int h4d_eval_forces_static(const h4d_params* params, double L, int32_t n_water, int32_t n,
                                      const double* x, const double* w, double* F, double* U) {
  int rc = check_params(params);
  if (rc) return rc;
  if (((!x || !F) && n > 0) || n < 0 || n_water < 0 || 3 * n_water > n || !(L > 0)) return H4D_EINVAL;
  if (unit_of(*params) == 2 && ((n - 3 * n_water) & 1) != 0) return H4D_EINVAL;
  if (2.0 * (rmax_of(*params) + params->skin) >= L) return H4D_EINVAL;
  rc = check_device();
  if (rc) return rc;
  if (n == 0) {  // no atoms: zero energy, nothing to write (as h4d_eval_forces)
    if (U) *U = 0.0;
    return H4D_OK;
  }
  void* base = nullptr;
  rc = static_scratch_address(&base);
  if (rc) return rc;

  // plan, geometry and the device layout inside the static array (host stack only)
  h4d_ctx c;
  c.prm = *params;
  c.seed = 0;
  c.stream = 0;
  c.R = 1;
  c.max_nbr = params->max_nbr > 0 ? params->max_nbr : derive_max_nbr(*params);
  c.max_nbr = ((c.max_nbr + 127) / 128) * 128;
  c.max_out = std::max(c.max_nbr, derive_max_rows(*params, rmax_of(*params) + outer_skin(*params)));
  Rep R;
  std::memset(&R, 0, sizeof(Rep));
  R.n_water = n_water;
  R.nw3 = 3 * n_water;
  R.cap_water = n_water;
  R.n_pairs = (n - 3 * n_water) / unit_of(*params);
  R.cap_pairs = R.n_pairs;
  R.cap_atoms = n;
  set_rep_geometry(*params, R, L);
  R.tpa = choose_tpa(*params, n);
  R.rec_cap = 1;
  Group G;
  std::memset(&G, 0, sizeof(Group));
  const int threads = choose_threads(n);
  G.nwarps = threads / 32;
  const size_t smem = group_smem_bytes(n, R.nc, threads);
  if (smem > 227 * 1024) return H4D_ECAPACITY;
  int cta_groups[2] = {0, 1};

  const size_t na = (size_t)n;
  size_t off = 0;
  const size_t o_rep = carve_bytes(off, sizeof(Rep));
  const size_t o_grp = carve_bytes(off, sizeof(Group));
  const size_t o_cg = carve_bytes(off, sizeof(cta_groups));
  const size_t o_u = carve_bytes(off, sizeof(double));
  const size_t o_rec = carve_bytes(off, sizeof(h4d_record));
  const size_t o_x = carve_bytes(off, na * 3 * sizeof(double));
  const size_t o_w = carve_bytes(off, w ? na * sizeof(double) : 0);
  const size_t o_pos = carve_bytes(off, na * sizeof(uint4));
  const size_t o_f = carve_bytes(off, na * sizeof(float4));
  const size_t o_fd = carve_bytes(off, na * 3 * sizeof(double));
  const size_t o_nbr = carve_bytes(off, na * (size_t)c.max_nbr * sizeof(uint16_t));
  const size_t o_cnt = carve_bytes(off, na * sizeof(int));
  const size_t o_ref = carve_bytes(off, na * sizeof(uint4));
  const size_t o_nbo = carve_bytes(off, na * (size_t)c.max_out * sizeof(uint16_t));
  const size_t o_cno = carve_bytes(off, na * sizeof(int));
  const size_t o_rfo = carve_bytes(off, na * sizeof(uint4));
  const size_t o_red = carve_bytes(off, na * sizeof(double));
  if (off > kStaticScratchBytes) return H4D_ECAPACITY;  // too many atoms for 16 MiB

  unsigned char* b = static_cast<unsigned char*>(base);
  Eng& e = c.eng;
  std::memset(&e, 0, sizeof(Eng));
  fill_pot(c.prm, e.pot, e.proto);
  e.rep = reinterpret_cast<Rep*>(b + o_rep);
  e.groups = reinterpret_cast<Group*>(b + o_grp);
  e.cta_groups = reinterpret_cast<int*>(b + o_cg);
  e.pos = reinterpret_cast<uint4*>(b + o_pos);
  e.force = reinterpret_cast<float4*>(b + o_f);
  // the evaluation never touches velocities or saved states; point them at valid memory
  e.vhi = e.vlo = e.vhi_save = e.vlo_save = e.force;
  e.pos_save = e.pos;
  e.ref = reinterpret_cast<uint4*>(b + o_ref);
  e.nbr = reinterpret_cast<uint16_t*>(b + o_nbr);
  e.ncnt = reinterpret_cast<int*>(b + o_cnt);
  e.nbr_out = reinterpret_cast<uint16_t*>(b + o_nbo);
  e.ncnt_out = reinterpret_cast<int*>(b + o_cno);
  e.ref_out = reinterpret_cast<uint4*>(b + o_rfo);
  e.rec = reinterpret_cast<h4d_record*>(b + o_rec);
  e.red = reinterpret_cast<double*>(b + o_red);
  e.max_nbr = c.max_nbr;
  e.max_out = c.max_out;
  e.seed = 0;

  // mean altitude of the flying particles (the nonzero altitudes), as in h4d_eval_forces
  double wsum = 0.0;
  int wcnt = 0;
  if (w)
    for (int a = 0; a < n; ++a)
      if ((float)w[a] != 0.0f) { wsum += w[a]; ++wcnt; }

  // the array keeps the previous call's contents: every region this call reads is
  // written first (the replica record with zeroed counters and flags, the inputs)
  if (cudaMemcpy(b + o_rep, &R, sizeof(Rep), cudaMemcpyHostToDevice) != cudaSuccess) return H4D_ECUDA;
  if (cudaMemcpy(b + o_grp, &G, sizeof(Group), cudaMemcpyHostToDevice) != cudaSuccess) return H4D_ECUDA;
  if (cudaMemcpy(b + o_cg, cta_groups, sizeof(cta_groups), cudaMemcpyHostToDevice) != cudaSuccess) return H4D_ECUDA;
  if (cudaMemcpy(b + o_x, x, na * 3 * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) return H4D_ECUDA;
  if (w && cudaMemcpy(b + o_w, w, na * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) return H4D_ECUDA;
  static_convert_in<<<(n + 255) / 256, 256>>>(reinterpret_cast<const double*>(b + o_x),
                                               w ? reinterpret_cast<const double*>(b + o_w) : nullptr, n, L, e.pos);
  if (cudaGetLastError() != cudaSuccess) return H4D_ECUDA;
  rc = launch_eval(e, threads, smem, (float)(wcnt ? wsum / wcnt : 0.0), reinterpret_cast<double*>(b + o_u), 0);
  if (rc) return rc;
  static_convert_out<<<(n + 255) / 256, 256>>>(e.force, n, reinterpret_cast<double*>(b + o_fd));
  if (cudaGetLastError() != cudaSuccess) return H4D_ECUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return H4D_ECUDA;
  Rep Rout;
  double u = 0.0;
  if (cudaMemcpy(&Rout, b + o_rep, sizeof(Rep), cudaMemcpyDeviceToHost) != cudaSuccess) return H4D_ECUDA;
  if (Rout.err & 1) return H4D_ECAPACITY;
  if (cudaMemcpy(&u, b + o_u, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return H4D_ECUDA;
  if (cudaMemcpy(F, b + o_fd, na * 3 * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return H4D_ECUDA;
  if (U) *U = u;
  return H4D_OK;
}

// ------------------------------------------------------------------------------------
// Learned insertion-site proposal
// ------------------------------------------------------------------------------------
static void prop_bind(h4d_ctx* c) {
  Eng& e = c->eng;
  PropDev* P = c->prop;
  e.net = prop_net(P);
  e.pg_cnt = P->cnt;
  e.pg_fld = P->fld;
  e.pg_logit = P->logit;
  e.pg_chunk = P->chunk;
  e.prec_feat = P->rfeat;
  e.prec_y = P->ry;
  e.prec_meta = P->rmeta;
}

static int prop_pack(PropDev* P, cudaStream_t s) {
  return launch_prop_pack(P->w, P->w1, P->w2, P->w3, P->w2t, P->w3r, P->b, s);
}

extern "C" {

int h4d_proposal(h4d_ctx* c, int32_t mode, double cell_len, double eps, int32_t records_per_replica) {
  if (c && (c->eng.proto.single || c->eng.proto.water)) return H4D_EINVAL;  // the proposal places ion pairs
  if (!c || (mode != H4D_PROPOSAL_UNIFORM && mode != H4D_PROPOSAL_LEARNED) || !(cell_len > 0) || !(eps > 0) ||
      !(eps <= 1) || records_per_replica < 0 || records_per_replica > (1 << 20))
    return H4D_EINVAL;
  if (mode == H4D_PROPOSAL_LEARNED && c->eng.proto.bias_on) return H4D_EINVAL;  // one placement rule
  int rc = pull_reps(c);
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->stream));
  if (!c->prop) {
    c->prop = new (std::nothrow) PropDev();
    if (!c->prop) return H4D_ECUDA;
    rc = prop_alloc_net(c->prop);
    if (rc) return rc;
    rc = prop_pack(c->prop, c->stream);
    if (rc) return rc;
  }
  PropDev* P = c->prop;
  // grid: G = max(3, floor(L / cell_len)) per replica, capped at kPropMaxG
  int cells = 0;
  for (auto& R : c->rep_h) {
    int G = (int)std::floor(R.L / cell_len);
    G = std::max(3, std::min(kPropMaxG, G));
    R.prop_G = G;
    R.prop_off = cells;
    cells += ((G * G * G + 31) / 32) * 32;
  }
  if (cells > P->cells) {
    void* old[] = {P->cnt, P->fld, P->logit, P->chunk, P->fout};
    for (void* q : old)
      if (q) cudaFree(q);
    P->cnt = nullptr; P->fld = nullptr; P->logit = nullptr; P->chunk = nullptr; P->fout = nullptr;
    CK(cudaMalloc(&P->cnt, (size_t)cells * sizeof(int4)));
    CK(cudaMalloc(&P->fld, (size_t)cells * 4 * sizeof(long long)));
    CK(cudaMalloc(&P->logit, (size_t)cells * sizeof(float2)));
    CK(cudaMalloc(&P->chunk, (size_t)(cells / 32) * sizeof(double2)));
    P->cells = cells;
  }
  // training-record rings
  const int n_rec = c->R * records_per_replica;
  if (n_rec != P->n_rec) {
    void* old[] = {P->rfeat, P->ry, P->rmeta, P->valid, P->n_valid};
    for (void* q : old)
      if (q) cudaFree(q);
    P->rfeat = nullptr; P->ry = nullptr; P->rmeta = nullptr; P->valid = nullptr; P->n_valid = nullptr;
    if (n_rec > 0) {
      CK(cudaMalloc(&P->rfeat, (size_t)n_rec * 192 * sizeof(float)));
      CK(cudaMalloc(&P->ry, (size_t)n_rec * sizeof(double)));
      CK(cudaMalloc(&P->rmeta, (size_t)n_rec * sizeof(int2)));
      CK(cudaMalloc(&P->valid, (size_t)n_rec * sizeof(int)));
      CK(cudaMalloc(&P->n_valid, sizeof(int)));
    }
    P->n_rec = n_rec;
  }
  if (n_rec > 0) CK(cudaMemsetAsync(P->rmeta, 0xff, (size_t)n_rec * sizeof(int2), c->stream));  // empty slots
  for (int r = 0; r < c->R; ++r) {
    Rep& R = c->rep_h[r];
    R.prec_off = r * records_per_replica;
    R.prec_cap = records_per_replica;
    R.prec_count = 0;
  }
  c->eng.proto.prop_mode = mode;
  c->eng.proto.prop_record = records_per_replica > 0 ? 1 : 0;
  c->eng.proto.prop_eps = eps;
  prop_bind(c);
  invalidate_graphs(c);
  rc = push_plan(c);
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->stream));
  return H4D_OK;
}

int h4d_proposal_set_weights(h4d_ctx* c, const double* w, int64_t n) {
  if (!c || !c->prop || !w || n != kPropNW) return H4D_EINVAL;
  std::vector<float> f(kPropNW);
  for (int i = 0; i < kPropNW; ++i) {
    if (!std::isfinite(w[i])) return H4D_EINVAL;
    f[i] = (float)w[i];
  }
  PropDev* P = c->prop;
  CK(cudaMemcpyAsync(P->w, f.data(), kPropNW * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemsetAsync(P->m, 0, kPropNW * sizeof(float), c->stream));
  CK(cudaMemsetAsync(P->v, 0, kPropNW * sizeof(float), c->stream));
  P->adam_t = 0;
  int rc = prop_pack(P, c->stream);
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->stream));
  return H4D_OK;
}

int h4d_proposal_get_weights(h4d_ctx* c, double* w, int64_t n) {
  if (!c || !c->prop || !w || n != kPropNW) return H4D_EINVAL;
  std::vector<float> f(kPropNW);
  CK(cudaMemcpyAsync(f.data(), c->prop->w, kPropNW * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int i = 0; i < kPropNW; ++i) w[i] = (double)f[i];
  return H4D_OK;
}

int h4d_proposal_records(h4d_ctx* c, int32_t r, float* feat, double* y, int32_t* move, int32_t* status, int64_t cap,
                         int64_t* n) {
  if (!c || !c->prop || r < 0 || r >= c->R || cap < 0) return H4D_EINVAL;
  int rc = pull_reps(c);
  if (rc) return rc;
  const Rep& R = c->rep_h[r];
  PropDev* P = c->prop;
  const int64_t have = std::min<int64_t>(R.prec_count, R.prec_cap);
  const int64_t take = std::min<int64_t>(have, cap);
  if (n) *n = take;
  if (take == 0) return H4D_OK;
  std::vector<float> fb((size_t)R.prec_cap * 192);
  std::vector<double> yb(R.prec_cap);
  std::vector<int2> mb(R.prec_cap);
  CK(cudaMemcpyAsync(fb.data(), P->rfeat + (size_t)R.prec_off * 192, fb.size() * sizeof(float),
                     cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(yb.data(), P->ry + R.prec_off, yb.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(mb.data(), P->rmeta + R.prec_off, mb.size() * sizeof(int2), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int64_t k = 0; k < take; ++k) {
    const int64_t idx = (R.prec_count - take + k) % R.prec_cap;
    if (feat) std::memcpy(feat + k * 192, fb.data() + idx * 192, 192 * sizeof(float));
    if (y) y[k] = yb[idx];
    if (move) move[k] = mb[idx].x;
    if (status) status[k] = mb[idx].y;
  }
  return H4D_OK;
}

int h4d_proposal_logits(h4d_ctx* c, int32_t r, float* logits, float* feat, int64_t cap_cells, int64_t* n_cells) {
  if (!c || !c->prop || r < 0 || r >= c->R) return H4D_EINVAL;
  int rc = pull_reps(c);
  if (rc) return rc;
  const Rep& R = c->rep_h[r];
  const int nc = R.prop_G * R.prop_G * R.prop_G;
  if (n_cells) *n_cells = nc;
  if (nc == 0) return H4D_EINVAL;
  if (nc > cap_cells) return H4D_ECAPACITY;
  PropDev* P = c->prop;
  float* fo = nullptr;
  if (feat) {
    if (P->fout) cudaFree(P->fout);
    P->fout = nullptr;
    CK(cudaMalloc(&P->fout, (size_t)nc * kPropNFeat * sizeof(float)));
    fo = P->fout;
  }
  rc = launch_prop_eval(c->eng, c->n_ctas, c->cta_threads, c->smem, r, fo, c->stream);
  if (rc) return rc;
  std::vector<float2> lg(nc);
  CK(cudaMemcpyAsync(lg.data(), P->logit + R.prop_off, nc * sizeof(float2), cudaMemcpyDeviceToHost, c->stream));
  if (feat) CK(cudaMemcpyAsync(feat, fo, (size_t)nc * kPropNFeat * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (logits)
    for (int i = 0; i < nc; ++i) {
      logits[2 * i] = lg[i].x;
      logits[2 * i + 1] = lg[i].y;
    }
  return H4D_OK;
}

int h4d_train_proposal(h4d_ctx* c, int64_t steps, int32_t batch, double lr, double y0, uint64_t seed,
                       double* loss_out) {
  if (!c || !c->prop || steps < 0 || batch < 1 || batch > (1 << 22) || !(lr >= 0) || !std::isfinite(y0))
    return H4D_EINVAL;
  PropDev* P = c->prop;
  if (P->n_rec == 0) return H4D_EINVAL;
  int rc = launch_prop_compact(P->rmeta, P->ry, P->n_rec, P->valid, P->n_valid, c->stream);
  if (rc) return rc;
  int n_valid = 0;
  CK(cudaMemcpyAsync(&n_valid, P->n_valid, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (n_valid == 0) return H4D_EINVAL;
  const int nb = std::min(batch, n_valid);
  const int rows_pad = ((2 * nb + 15) / 16) * 16;
  rc = prop_ensure_rows(P, rows_pad);
  if (rc) return rc;
  for (int64_t s = 0; s < steps; ++s) {
    rc = launch_prop_gather(P->rfeat, P->ry, P->valid, n_valid, nb, seed, (long long)P->adam_t, (float)y0, P->bfeat,
                            P->btgt, c->stream);
    if (rc) return rc;
    rc = prop_loss_grad(P, nb, rows_pad, c->stream);
    if (rc) return rc;
    P->adam_t++;
    rc = launch_prop_adam(P->w, P->m, P->v, P->grad, (int)std::min<long long>(P->adam_t, 1 << 30), (float)lr,
                          c->stream);
    if (rc) return rc;
    rc = prop_pack(P, c->stream);
    if (rc) return rc;
  }
  if (loss_out) {
    double l = 0.0;
    if (steps > 0) {
      CK(cudaMemcpyAsync(&l, P->loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
    }
    *loss_out = l / nb;
  }
  CK(cudaStreamSynchronize(c->stream));
  return H4D_OK;
}

int h4d_proposal_grad(const double* w, int64_t n_rec, const float* feat, const float* tgt, double* loss,
                      double* grad) {
  if (!w || !feat || !tgt || n_rec < 1 || n_rec > (1 << 22)) return H4D_EINVAL;
  int rc = check_device();
  if (rc) return rc;
  PropDev* P = new (std::nothrow) PropDev();
  if (!P) return H4D_ECUDA;
  cudaStream_t s = 0;
  const int n = (int)n_rec;
  const int rows_pad = ((2 * n + 15) / 16) * 16;
  std::vector<float> f(kPropNW);
  for (int i = 0; i < kPropNW; ++i) f[i] = (float)w[i];
  rc = prop_alloc_net(P);
  if (!rc) rc = prop_ensure_rows(P, rows_pad);
  if (!rc && cudaMemcpy(P->w, f.data(), kPropNW * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) rc = H4D_ECUDA;
  if (!rc && cudaMemcpy(P->bfeat, feat, (size_t)n * 192 * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    rc = H4D_ECUDA;
  if (!rc && cudaMemcpy(P->btgt, tgt, (size_t)n * 2 * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    rc = H4D_ECUDA;
  if (!rc) rc = prop_pack(P, s);
  if (!rc) rc = prop_loss_grad(P, n, rows_pad, s);
  double l = 0.0;
  if (!rc && cudaMemcpy(&l, P->loss, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) rc = H4D_ECUDA;
  if (!rc && cudaMemcpy(f.data(), P->grad, kPropNW * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = H4D_ECUDA;
  if (!rc) {
    if (loss) *loss = l / n;
    if (grad)
      for (int i = 0; i < kPropNW; ++i) grad[i] = (double)f[i];
  }
  prop_free(P);
  return rc;
}

}  // extern "C"
