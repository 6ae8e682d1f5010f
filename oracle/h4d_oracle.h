/*
 * h4d_oracle.h -- FP64 CPU oracle for the hybrid 4D NEMD/MC (H4D) grand-canonical
 * method of Kim, Belloni and Rotenberg, "Grand-canonical molecular dynamics
 * simulations powered by a hybrid 4D nonequilibrium MD/MC method" (arXiv:2307.11447).
 *
 * TEST INFRASTRUCTURE ONLY.  This header and h4d_oracle.c are the slow, plain,
 * double-precision statement of what the GPU library computes.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant generator with the CUDA library, and the CUDA
 * library never calls it.
 *
 * Conventions (each reading of the paper is stated where it is used):
 *   - atoms [0, 3*n_water) are rigid waters stored O,H,H; ions follow, stored as
 *     interleaved pairs: ion 2k is cation k (type 0), ion 2k+1 is anion k (type 1);
 *     water O is type 2 and H is type 3.
 *   - positions are kept wrapped into [0, L); every displacement uses the minimum image.
 *   - the random stream is Philox4x64-10 keyed by (seed, replica); every draw has a
 *     fixed (counter, purpose) address so that any implementation of the same method
 *     draws the same numbers independent of evaluation order.
 */
#ifndef H4D_ORACLE_H
#define H4D_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAXT 4

/* Philox purposes (counter word 2) */
#define ORC_PUR_TRIAL 1u
#define ORC_PUR_GAMMA 2u
#define ORC_PUR_THERMO 3u
#define ORC_PUR_VINIT 4u

/* altitude schedules: constant velocity (Eq. 2), w_v (Eq. S6), w_x (Eq. S7) */
#define ORC_SCHED_LINEAR 0
#define ORC_SCHED_WV 1
#define ORC_SCHED_WX 2

typedef struct {
  double L;        /* cubic box edge */
  double beta;     /* 1/kT */
  double beta_mu;  /* beta * mu of the ion pair (Lambda_s = 1) */
  /* pair potential: truncated-shifted LJ (Eq. 19, Lorentz-Berthelot), erfc Coulomb (Eq. 9, 20) */
  double rc_lj, rc_coul, alpha, kcoul, kappa_sr;
  int32_t ntypes, pad0;
  double q[ORC_MAXT], sig[ORC_MAXT], eps[ORC_MAXT], mass[ORC_MAXT];
  double mvv2e;    /* converts mass*velocity^2 into energy units */
  /* protocol */
  double dt, w_max, tau_t;
  int32_t n_f, schedule;
  double sched_n;  /* exponent n of Eqs. S6-S7 */
  /* rigid water geometry (SPC/E-like) */
  double d_oh, d_hh;
  int32_t n_water, use_cells;
  uint64_t seed, replica;
  /* bimodal flyer-distance bias (Sec. II.B.3, Eqs. 14-18): the anion is placed at an
   * offset from the cation drawn per axis from b (Eq. 16) with sharpness bias_alpha and
   * mean separation bias_xb; bias_alpha <= 0 switches it off */
  double bias_alpha, bias_xb;
  /* different w_max per species (SI, "Different w_max for different ion species"): the
   * anion starts (insertion) or ends (deletion) at w_max + 0.5 (sig_c + sig_a) fw and
   * moves proportionally faster, so both flyers reach w = 0 together; fw = 0: one w_max */
  double fw;
  /* early rejection (SI, "Simple, early rejection scheme"): a cube of volume v_ex
   * centred on the flying cation.  A pair whose anion lies inside it -- every axis of
   * the anion's minimum-image fixed-point offset from the cation within
   * round(0.5 cbrt(v_ex) / L 2^32) -- is exchanged by an instantaneous MC move (no NEMD:
   * Delta H = Delta U at unchanged velocities); any other pair by NEMD.  The same rule
   * classifies insertions and deletions, so each pair geometry has one kind of move in
   * both directions.  v_ex = 0 switches it off. */
  double v_ex;
  /* fixed-N work sampling (Sec. II.E, SI Sec. S1): trials run and are recorded but none
   * is accepted, so the work distributions are sampled at fixed particle numbers */
  int32_t no_accept;
  /* single-particle exchange (Sec. II.A: the pair rule translated to one flying
   * particle): every atom after the waters is one species of type 0, and a trial inserts
   * or deletes one of them; n_pairs and cap_pairs of the state count particles */
  int32_t single;
  /* rigid-water exchange (Sec. II.A for one flyer; Sec. II.C on flying rigid waters): a
   * trial inserts or deletes one rigid water, which flies frozen in 3D (position and
   * orientation) while the others move.  The number of waters then lives in the state
   * (orc_state.n_water, at most cap_water) and p->n_water is ignored by the functions
   * that take a state; ions keep their pairs and follow the waters in the layout. */
  int32_t water_ex, pad_w;
} orc_params;

typedef struct {
  int32_t n_pairs, cap_pairs;
  double *x, *v;       /* [(3*n_water + 2*cap_pairs) * 3]; 3*cap_water with water exchange */
  uint64_t trial_ctr;  /* trials done by this chain (Philox counter of trial draws) */
  uint64_t step_ctr;   /* equilibrium MD steps done (Philox counter of thermostat draws) */
  int32_t n_water, cap_water; /* water exchange only: current and largest number of waters */
} orc_state;

typedef struct {
  int32_t move;       /* 1 insertion, 0 deletion */
  int32_t accepted;
  int32_t n_before, n_after;
  int32_t status;     /* 0 ok, 1 deletion from empty system, 2 capacity, 3 non-finite energy */
  int32_t cation, anion;  /* chosen pair (deletion) or -1 */
  int32_t cell_c, cell_a; /* proposal-grid cells of the exchanged cation and anion, or -1 */
  int32_t instant;    /* 1: instantaneous move of the early-rejection scheme (no NEMD) */
  double dH;          /* H_end - H_start in energy units */
  double beta_dM;     /* beta * Delta M, insertion-direction convention (Eqs. 6, 8) */
  double w_prot;      /* protocol work sum_k [U(w_{k+1}) - U(w_k)] at fixed positions */
  double ln_u;        /* log of the uniform acceptance draw */
  double x_acc;       /* exponent compared with ln_u */
  double ln_q;        /* log proposal-density factor included in x_acc (0 for uniform) */
} orc_record;

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);

/* Ewald sum of the Coulomb energy of the periodic system (Sec. II.B.2, Eqs. 9-10: the
 * Coulomb energy split into a screened real-space part and a long-range part; the
 * long-range part U_lr = U_recip + U_self is what g^lr(w) = exp(-kappa_lr w) scales).
 * Charges p->q[type], prefactor p->kcoul, box p->L.  U_real: erfc(alpha r)/r over pairs
 * closer than rcut (minimum image, unshifted, intramolecular water pairs left out);
 * U_recip = (2 pi K / V) sum_{k != 0, |n_d| <= kmax} exp(-k^2 / 4 alpha^2) / k^2 |S(k)|^2 with
 * S(k) = sum_j q_j exp(i k.r_j), k = 2 pi n / L; U_self = -K alpha/sqrt(pi) sum q_j^2;
 * U_excl = -K sum over intramolecular water pairs q_i q_j erf(alpha r)/r (the reciprocal
 * sum includes them).  F_recip (may be NULL) receives -dU_recip/dx per atom.  Returns
 * U_real + U_recip + U_self + U_excl. */
double orc_ewald(const orc_params* p, int n, const double* x, double alpha, int kmax, double rcut,
                 double* U_real, double* U_recip, double* U_self, double* U_excl, double* F_recip);

/* pair energy and derivative at 4D distance r4 between types ti, tj with
 * short-range screening factor g (Eq. 11) applied to the Coulomb part */
void orc_pair(const orc_params* p, int ti, int tj, double r4, double g, double* u, double* dudr);

int orc_atom_type(const orc_params* p, int a);

/* total potential energy and 3D forces of n atoms at altitudes w (NULL = all zero),
 * flyers marked in fly (NULL = none); F may be NULL. Brute force O(n^2) unless
 * p->use_cells, in which case a plain cell list produces the same sum. */
double orc_energy_forces(const orc_params* p, int n, const double* x, const double* w,
                         const uint8_t* fly, double* F);

/* number of list pairs (i<j) under the fixed-point neighbour criterion; writes up to
 * cap pairs, sorted by (i, j) */
int64_t orc_neighbor_pairs(int n, const double* x, double L, double r_list,
                           int32_t* out_i, int32_t* out_j, int64_t cap);

/* altitude of a flyer at NEMD step k of n_f */
double orc_altitude(const orc_params* p, int insertion, int k);

/* kinetic energy of atoms (optionally skipping flyers) */
double orc_kinetic(const orc_params* p, int n, const double* v, const uint8_t* fly);

/* plain NVE velocity-Verlet steps (w = 0); returns final potential energy */
double orc_nve(const orc_params* p, orc_state* s, int64_t n_steps, double* e_trace);

/* equilibrium MD steps with the CSVR thermostat */
void orc_md(const orc_params* p, orc_state* s, int64_t n_steps);

/* one NEMD path with the flyers given, forward schedule (insertion or deletion);
 * used for the reversibility pin; returns the protocol work */
double orc_nemd_path(const orc_params* p, orc_state* s, const int32_t* flyers, int n_flyers,
                     int insertion, double* U_end);

/* one H4D pair-exchange trial (Sec. II.A) */
int orc_trial(const orc_params* p, orc_state* s, orc_record* rec);

/* early rejection: 1 if the anion at xa lies in the excluded cube (volume p->v_ex) centred
 * on the cation at xc, judged on fixed-point coordinates as in a trial; 0 otherwise */
int orc_in_excluded_volume(const orc_params* p, const double* xc, const double* xa);

/* n_cycles GCMD cycles: n_eq equilibrium MD steps then one trial (Fig. 1) */
int orc_run_cycles(const orc_params* p, orc_state* s, int64_t n_cycles, int64_t n_eq,
                   orc_record* recs);

/* draw initial Maxwell-Boltzmann velocities for all atoms */
void orc_init_velocities(const orc_params* p, orc_state* s);

/* Bimodal bias.  Density of the anion-cation offset x on one axis, x in [-L/2, L/2)
 * (Eq. 16, normalised on the box); the inverse error function used to draw from it
 * (Winitzki's approximation refined by Newton steps on erf); one draw of the offset from
 * two 64-bit random words (the top bit of r_mode picks the mode at +x_b or -x_b, which
 * carry equal mass; r_u drives the inverse CDF of that truncated Gaussian). */
double orc_bias_density(double alpha, double xb, double L, double x);
double orc_erfinv(double y);
double orc_bias_offset(double alpha, double xb, double L, uint64_t r_mode, uint64_t r_u);

/* ------------------------------------------------------------------------------------ */
/* Learned insertion-site proposal.  The box is cut into G^3 cells (cell index           */
/* (gx*G + gy)*G + gz, an atom with fixed-point coordinate X is in gx = floor(X G / 2^32)). */
/* Each cell has 96 features: for species s (cation, anion, water O) and each of the 27  */
/* cells of its 3x3x3 neighbourhood (slot (ex+1)*9 + (ey+1)*3 + (ez+1) for offset e),     */
/* 0.25 x the number of atoms (81); 0.1 x sum_j q_j d_j / max(|d_j|, 0.5)^3 over the      */
/* charges of those 27 cells, d_j = minimum image of (cell centre - x_j) (3); 12 zeros.  */
/* An MLP 96-64-64-2 (ReLU) maps them to a cation and an anion logit; the proposal of    */
/* species s is q_s = (1 - eps) softmax_cells(logit_s) + eps / G^3, and an ion is placed */
/* uniformly inside the drawn cell.  The ratio of this density to the uniform 1/V enters */
/* the acceptance exponent (the role of B^ins / B^del in Eqs. 15-16): insertion adds     */
/* -ln(q_c G^3) - ln(q_a G^3) with q from the start state, deletion adds                 */
/* +ln(q_c G^3) + ln(q_a G^3) with q from the end state (flyers removed).                */
/* ------------------------------------------------------------------------------------ */
#define ORC_NFEAT 96
#define ORC_HID 64
#define ORC_PROP_NW (ORC_NFEAT * ORC_HID + ORC_HID + ORC_HID * ORC_HID + ORC_HID + ORC_HID * 2 + 2)

typedef struct {
  int32_t mode;     /* 0 uniform placement, 1 learned density */
  int32_t G;        /* cells per box edge (>= 3) */
  int32_t bf16;     /* 1: round features, weights and hidden activations to bfloat16 and
                       sum each layer in binary32, the precision in which the GPU kernel
                       takes the cell decision; 0: plain FP64 */
  int32_t pad;
  double eps;       /* weight of the uniform component */
  const double* w;  /* ORC_PROP_NW weights, flat: W1[96][64], b1[64], W2[64][64], b2[64],
                       W3[64][2], b3[2] (row index = input unit) */
} orc_proposal;

/* features of every cell of n atoms (ex0/ex1 = atoms to leave out, or -1) */
int orc_proposal_features(const orc_params* p, int G, int n, const double* x, int ex0, int ex1,
                          double* feat);
/* logits [G^3][2] of every cell */
int orc_proposal_logits(const orc_params* p, const orc_proposal* q, int n, const double* x,
                        int ex0, int ex1, double* logits);
/* one trial with the given proposal (q NULL: uniform, no cells).  If site_feat is given
 * (and q is), it receives the features of the cation's and the anion's cell [2][96] in the
 * N-pair state of the move (start state of an insertion, end state of a deletion) and
 * site_y the insertion-direction exponent without the proposal factor (x_acc of an
 * insertion, -x_acc of a deletion) -- the training record of the move. */
int orc_trial_prop(const orc_params* p, const orc_proposal* q, orc_state* s, orc_record* rec,
                   double* site_feat, double* site_y);
int orc_run_cycles_prop(const orc_params* p, const orc_proposal* q, orc_state* s, int64_t n_cycles,
                        int64_t n_eq, orc_record* recs);

#ifdef __cplusplus
}
#endif
#endif
