/*
 * h4d.h -- C ABI of libh4d, a single-GPU (GB300, sm_103a) implementation of the hybrid 4D
 * nonequilibrium MD/MC ("H4D") grand-canonical method of Kim, Belloni and Rotenberg,
 * arXiv:2307.11447, "Grand-canonical molecular dynamics simulations powered by a hybrid
 * 4D nonequilibrium MD/MC method".
 *
 * What the library computes (paper sections and equations):
 *   - the short-range pair force and energy in the 4D metric r4^2 = r^2 + (w_i - w_j)^2:
 *     truncated-shifted Lennard-Jones (Eq. 19, Lorentz-Berthelot mixing, Sec. II.D) plus
 *     the real-space Coulomb term K q_i q_j erfc(alpha r4)/r4 shifted to zero at its
 *     cut-off (Eqs. 9, 20), multiplied by the altitude screening exp(-kappa_sr w) for
 *     pairs of one flying and one non-flying particle (Eqs. 10-11);
 *   - NEMD trajectories that carry an ion pair along the auxiliary axis w with the
 *     constant-velocity schedule of Eq. 2 (or w_v / w_x of Eqs. S6-S7), flying ions held
 *     at their 3D positions (Sec. II.B.1), everything else integrated by velocity Verlet
 *     in the NVE ensemble (Sec. II.A), rigid waters by RATTLE;
 *   - the FP64 nonequilibrium work Delta M and the pair-exchange Metropolis rule of
 *     Eqs. 3-8 with symmetric two-end momentum reversal (Sec. II.A), committed on the
 *     device with no host round trip;
 *   - equilibrium MD between trials (Fig. 1) with a CSVR thermostat;
 *   - the same rule with one flyer (Sec. II.A): single particles of a neutral species, or
 *     one rigid water frozen in 3D with molecular-frame velocities (Sec. II.C);
 *   - the long-range Coulomb part of one configuration as a reciprocal-space Ewald sum
 *     scaled by exp(-kappa_lr wbar) (Eqs. 9-10), as an evaluation entry point.
 *
 * Conventions shared by every entry point:
 *   - Return value: H4D_OK (0) on success, a negative H4D_E* code on error; no C++
 *     exception crosses the ABI.  h4d_strerror() names each code.
 *   - Pointers named host_* are host memory; the library copies from or into them and
 *     never keeps them.  Pointers named dev_* are device memory owned by the caller.
 *     All other device memory is owned by the context and freed by h4d_destroy().
 *   - Each context issues its work on the CUDA stream given at creation; with NULL the
 *     context creates a non-blocking stream of its own (CUDA-graph capture cannot use
 *     the legacy default stream) and destroys it in h4d_destroy().  Launching entry
 *     points return when the work is queued; getters synchronise the stream before they
 *     return.
 *   - Atom layout inside a replica: atoms [0, 3*n_water) are rigid waters stored as
 *     O,H,H; ions follow as interleaved pairs, ion 2k = cation k (type 0) and ion 2k+1 =
 *     anion k (type 1).  Water O is type 2 and H is type 3.  Positions are Cartesian in
 *     [0, L)^3 per replica (other values are wrapped); arrays are row-major [atom][xyz].
 *   - Random numbers: Philox4x64-10 keyed by (seed, replica key); draw addresses are fixed
 *     (trial counter, block, purpose) so results do not depend on thread scheduling.
 */
#ifndef H4D_H
#define H4D_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque context: owns the device state of all replicas, the stream and the launch plan. */
typedef struct h4d_ctx h4d_ctx;

/* ---- error codes ---- */
#define H4D_OK 0
#define H4D_EINVAL (-1)    /* bad argument (NULL pointer, size out of range, unknown mode) */
#define H4D_ECAPACITY (-2) /* a neighbour row, cell or replica capacity would be exceeded */
#define H4D_ETIMEOUT (-3)  /* a bounded device loop gave up (reported, never a hang) */
#define H4D_ENAN (-4)      /* non-finite force or energy in equilibrium MD */
#define H4D_ECUDA (-5)     /* a CUDA runtime call failed */
#define H4D_ENODEV (-6)    /* no CUDA device or the device is not sm_103 class */

/* ---- systems and schedules ---- */
#define H4D_SYS_LJ 0    /* LJ electrolyte: two ion types of equal size (Sec. II.D.1) */
#define H4D_SYS_AQ 1    /* rigid 3-site water + Na+/Cl- (Sec. II.D.2) */
#define H4D_SCHED_LINEAR 0 /* Eq. 2 */
#define H4D_SCHED_WV 1     /* Eq. S6 insertion form; deletion is its time reverse */
#define H4D_SCHED_WX 2     /* Eq. S7 insertion form; deletion is its time reverse */
#define H4D_EXCHANGE_PAIR 0   /* cation-anion pairs (Eqs. 3-8) */
#define H4D_EXCHANGE_SINGLE 1 /* single particles of one neutral species (Sec. II.A: the
                                 pair rule with one flyer, V/(N+1) to the first power) */
#define H4D_EXCHANGE_WATER 2  /* one rigid water per trial (Sec. II.A with one flyer; Sec.
                                 II.C: molecular-frame velocities), frozen in 3D while it flies */

/* Physics, protocol and engine settings common to all replicas of a context. */
typedef struct h4d_params {
  int32_t system;         /* H4D_SYS_LJ or H4D_SYS_AQ */
  int32_t ntypes;         /* 2 (LJ) or 4 (AQ) */
  double beta;            /* 1/kT in inverse energy units */
  double beta_mu;         /* beta * mu of the ion pair, Lambda_s = 1 (Eqs. 6, 8) */
  double rc_lj;           /* LJ cut-off (Eq. 19) */
  double rc_coul;         /* cut-off of the real-space Coulomb term */
  double alpha;           /* splitting parameter of erfc(alpha r) (Eq. 9) */
  double kcoul;           /* Coulomb prefactor: energy x length / e^2 */
  double kappa_sr;        /* kappa_w^sr of Eq. 11 */
  double q[4], sig[4], eps[4], mass[4]; /* per type */
  double mvv2e;           /* converts mass x velocity^2 into energy units */
  double dt;              /* time step (NEMD and equilibrium) */
  double w_max;           /* maximum altitude (Eq. 2) */
  double tau_t;           /* CSVR relaxation time of equilibrium MD; <= 0 disables it */
  double sched_n;         /* exponent n of Eqs. S6-S7 */
  int32_t n_f;            /* NEMD steps per trial */
  int32_t schedule;       /* H4D_SCHED_* */
  double d_oh, d_hh;      /* rigid water bond lengths (O-H, H-H) */
  double skin;            /* Verlet-list skin: rebuilt when the two largest displacements sum to it */
  double skin_outer;      /* skin of the outer list the Verlet list is filtered from (0 = 4 skin);
                             a Verlet refresh rebuilds both lists once the two largest
                             displacements since the outer build exceed skin_outer - skin */
  int32_t max_nbr;        /* neighbour-row capacity per atom; 0 = derived from density */
  int32_t threads_per_atom; /* 1,2,4,8,16 or 32; 0 = chosen per replica size (h4d_autotune measures) */
  int32_t exchange;       /* H4D_EXCHANGE_PAIR, or H4D_EXCHANGE_SINGLE: LJ system only, charges 0,
                             every ion-block atom is one species with the parameters of
                             type 0, and the "pair" counts of h4d_system, h4d_counts and the
                             records count particles; bias, learned proposal, species w_max
                             and early rejection are pair moves (H4D_EINVAL); or
                             H4D_EXCHANGE_WATER: aqueous system, one w_max (species w_max
                             off), the ion pairs stay, the "pair" counts of h4d_counts.sum_n
                             and of the records count waters, and a deletion record's
                             cation field holds the deleted water's index */
  int32_t pad_exchange;
} h4d_params;

/* Initial replicas.  Replica r holds 3*n_water[r] + 2*n_pairs[r] atoms; host_x (and
 * host_v when not NULL) concatenate the replicas in order, 3 doubles per atom.  With
 * host_v == NULL velocities are drawn from Maxwell-Boltzmann at 1/beta.
 * replica_key (may be NULL = the replica index r) gives each replica the second word of
 * its Philox key (seed, key): a replica keeps its key, and with it every random draw and
 * -- for the same threads_per_atom -- every result bit, whether it runs alone or packed
 * with other replicas, since all of the engine's sums are independent of the launch plan. */
typedef struct h4d_system {
  int32_t n_replicas;
  const double* L;          /* [R] cubic box edges */
  const int32_t* n_water;   /* [R] rigid waters (0 for the LJ electrolyte) */
  const int32_t* n_pairs;   /* [R] ion pairs at start */
  const int32_t* cap_pairs; /* [R] maximum ion pairs the replica may reach */
  const double* host_x;
  const double* host_v;
  const uint64_t* replica_key; /* [R] or NULL */
  const int32_t* cap_water;    /* [R] or NULL (= n_water): the most waters a replica may hold
                                  under water exchange; atoms [0, 3 n_water) are the waters and
                                  the ions follow them, so a water insertion moves every ion up
                                  by three atoms and a deletion moves them down */
} h4d_system;

/* Per-replica counters. */
typedef struct h4d_counts {
  int64_t n_pairs;          /* current ion pairs */
  int64_t cycles;           /* trials done */
  int64_t trials_ins, trials_del;
  int64_t accepted_ins, accepted_del;
  int64_t rejected_status;  /* deletion from an empty box, full capacity, non-finite work */
  int64_t md_steps;         /* equilibrium MD steps done */
  double sum_n, sum_n2;     /* running sums of N after each trial (for <N> and chi) */
  int64_t nbr_builds;       /* neighbour-list builds */
  int64_t error_flags;      /* bit 0 row overflow, bit 1 non-finite MD state, bit 2 timeout */
  double t_nemd_ns, t_md_ns; /* device time spent in NEMD trials and equilibrium MD */
  double t_build_ns;        /* of which: neighbour-list builds */
  double t_force_ns;        /* of which: FP32 force passes */
  double t_energy_ns;       /* of which: FP64 end-point energies */
  int64_t threads_per_atom; /* lanes that share one neighbour row in the force pass */
  int64_t nbr_refreshes;    /* Verlet-row refreshes filtered from the outer rows (between builds) */
  double t_filter_ns;       /* part of t_build_ns spent filtering Verlet rows from outer rows */
  int64_t last_smid;        /* SM that ran this replica's warps in the most recent launch */
  double t_last_begin_ns;   /* device global timer when this replica's warps started and */
  double t_last_end_ns;     /* finished the most recent launch (ns; compare across replicas) */
  int64_t plan_warps;       /* warps of this replica's group in the launch plan */
  int64_t plan_cta_groups;  /* replicas (groups) sharing its CTA, itself included */
  int64_t n_water;          /* current rigid waters (varies under water exchange) */
} h4d_counts;

/* One trial record; Delta M follows the insertion direction (Eqs. 6, 8). */
typedef struct h4d_record {
  int32_t move;       /* 1 insertion, 0 deletion */
  int32_t accepted;
  int32_t n_before, n_after;
  int32_t status;     /* 0 ok, 1 deletion from empty system, 2 capacity, 3 non-finite work */
  int32_t cation, anion; /* chosen pair index (deletion), else -1; water exchange: the
                            deleted water in cation, anion -1 */
  int32_t cell_c, cell_a; /* proposal-grid cells of the exchanged cation and anion, or -1
                             when no proposal grid is enabled */
  int32_t instant;    /* 1: instantaneous move of the early-rejection scheme (no NEMD) */
  double dH;          /* H_end - H_start (energy units, FP64) */
  double beta_dM;     /* beta Delta M */
  double w_prot;      /* protocol work sum_k [U(w_{k+1}) - U(w_k)] (FP32 pairs, FP64 sum) */
  double ln_u;        /* log of the acceptance uniform */
  double x_acc;       /* exponent compared with ln_u (includes the proposal factor) */
  double ln_q;        /* log proposal factor ln(q_c G^3) + ln(q_a G^3) of the learned
                         proposal (subtracted for an insertion, added for a deletion; 0
                         with uniform placement) */
} h4d_record;

/* ---- context lifetime ---- */

/* Create a context: copies params and the initial replicas to the device, sizes every
 * buffer for cap_pairs, picks the lanes per neighbour row by replica size when
 * threads_per_atom == 0 (h4d_autotune then measures and keeps the fastest).
 * seed keys the random stream.  cuda_stream is a cudaStream_t (NULL = a stream the context
 * creates and owns). */
int h4d_create(const h4d_params* params, const h4d_system* sys, uint64_t seed, void* cuda_stream,
               h4d_ctx** out);
void h4d_destroy(h4d_ctx* ctx);
const char* h4d_strerror(int code);

/* ---- settings (each applies from the next launch) ---- */
/* beta mu of the ion pair in the acceptance exponents of Eqs. 6 and 8 (Lambda_s = 1);
 * H4D_EINVAL when not finite. */
int h4d_set_mu(h4d_ctx* ctx, double beta_mu);
/* NEMD protocol (Sec. II.A): n_f >= 1 steps of length dt > 0 between w_max >= 0 and 0 on
 * the schedule H4D_SCHED_* (Eq. 2, Eqs. S6-S7), screening kappa_sr >= 0 (Eq. 11);
 * H4D_EINVAL otherwise.  The bias, proposal, species w_max, early-rejection and no-accept
 * settings are kept; synchronises the stream. */
int h4d_set_protocol(h4d_ctx* ctx, int32_t n_f, double w_max, double dt, double kappa_sr,
                     int32_t schedule);
/* Bimodal flyer-distance bias (Sec. II.B.3, Eqs. 14-18), off by default (alpha_b = 0).
 * Insertion: the cation is placed uniformly, the anion at an offset drawn per axis from
 * b(x) = sqrt(alpha_b/pi) [e^{-alpha_b (x - x_b)^2} + e^{-alpha_b (x + x_b)^2}] /
 * [erf(sqrt(alpha_b)(x_b + L/2)) - erf(sqrt(alpha_b)(x_b - L/2))] on [-L/2, L/2) (Eq. 16;
 * alpha_b in 1/length^2, x_b a length).  Deletion: the cation uniformly, the anion with
 * probability B^ins(r_a | r_c) / sum_n B^ins, B^ins = V prod_axes b.  The exponent gains
 * -ln q for an insertion (q over the end state) and +ln q for a deletion (start state),
 * q = mean of B^ins over the anions with the pair present relative to its cation
 * (Eqs. 17-18; record field ln_q).  Random draws: block 6 of the trial, words 0-2, pick
 * the mode (top bit) on x, y, z; the anion's position words of blocks 1-2 drive the
 * inverse CDF.  Cannot be combined with the learned proposal (H4D_EINVAL). */
int h4d_set_bias(h4d_ctx* ctx, double alpha_b, double x_b);
/* Early rejection (SI, "Simple, early rejection scheme"), off by default (v_ex = 0).  A
 * cube of volume v_ex (length^3) centred on the flying cation: a pair whose anion lies in
 * it -- every axis of the minimum-image fixed-point offset within
 * rint(0.5 cbrt(v_ex) / L 2^32) -- is exchanged by an instantaneous MC move (no NEMD
 * steps: Delta H = Delta U at unchanged velocities, protocol work 0, record field
 * instant = 1); any other pair by NEMD.  The pair's geometry decides the move type for
 * insertions (after placement, biased or learned) and deletions alike, so the
 * acceptance rule is unchanged.  H4D_EINVAL for a negative or non-finite v_ex. */
int h4d_set_early_rejection(h4d_ctx* ctx, double v_ex);
/* Different w_max for the two ion species (SI, "Different w_max for different ion
 * species"): the anion flies at w_max + 0.5 (sig_c + sig_a) f_w (sigmas of types 0 and 1)
 * and moves proportionally faster, so both flyers reach (insertion) or leave (deletion)
 * w = 0 together; the flyers' mutual pair then changes with the step and enters the
 * protocol work, and the screening of Eq. 11 uses the mean flyer altitude.  The
 * acceptance rule is unchanged.  f_w = 0 (default): one w_max for both. */
int h4d_set_species_wmax(h4d_ctx* ctx, double f_w);
/* fixed-N work sampling (SI Sec. S1, Eq. 21): trials are run and recorded but never
 * accepted when on != 0 */
int h4d_set_no_accept(h4d_ctx* ctx, int32_t on);

/* ---- running ---- */

/* n_steps of equilibrium MD (all w = 0, CSVR thermostat) on every replica. */
int h4d_run_md(h4d_ctx* ctx, int64_t n_steps);
/* k_cycles grand-canonical cycles on every replica (Fig. 1): n_eq equilibrium MD steps,
 * then one insertion or deletion trial (NEMD + Metropolis + commit).  One persistent
 * launch runs all cycles of all replicas. */
int h4d_run_trials(h4d_ctx* ctx, int64_t k_cycles, int32_t n_eq);

/* Autotuner: for every replica, time n_iter equilibrium force passes (device timers) for
 * each threads-per-atom value in {1, 2, 4, 8, 16} and keep the fastest.  State and
 * counters are left as they were; synchronises the stream.  When not NULL, host_pass_ns
 * and host_build_ns (5 entries each, one per candidate) receive the mean device time of
 * one force pass and of one neighbour build per replica. */
int h4d_autotune(h4d_ctx* ctx, int32_t n_iter, double* host_pass_ns, double* host_build_ns);

/* ---- getters (synchronise the context stream) ---- */
int h4d_get_counts(h4d_ctx* ctx, int32_t replica, h4d_counts* out);
/* current FP64 potential and kinetic energy of a replica */
int h4d_get_energies(h4d_ctx* ctx, int32_t replica, double* U, double* K);
/* the most recent trial records of a replica (up to cap, oldest first); *n receives
 * how many were written */
int h4d_get_work(h4d_ctx* ctx, int32_t replica, h4d_record* host_rec, int64_t cap, int64_t* n);
/* positions (in [0,L)) and velocities of a replica; *n_atoms receives the atom count;
 * fails with H4D_ECAPACITY when cap_atoms is too small */
int h4d_get_state(h4d_ctx* ctx, int32_t replica, double* host_x, double* host_v,
                  int64_t cap_atoms, int64_t* n_atoms);
/* overwrite a replica's state: n_pairs ion pairs, host_x [3*n_water + 2*n_pairs][3]
 * (wrapped into [0, L)), host_v of the same shape or NULL (Maxwell-Boltzmann draw);
 * H4D_EINVAL for a bad replica or NULL host_x, H4D_ECAPACITY when n_pairs is negative or
 * above the replica's cap_pairs.  Neighbour rows are rebuilt at the next launch. */
int h4d_set_state(h4d_ctx* ctx, int32_t replica, int32_t n_pairs, const double* host_x,
                  const double* host_v);
/* the same with the number of waters (water exchange: up to the replica's cap_water;
 * otherwise it must equal the replica's n_water): host_x [3*n_water + 2*n_pairs][3];
 * H4D_ECAPACITY when n_water is negative or above the capacity */
int h4d_set_water_state(h4d_ctx* ctx, int32_t replica, int32_t n_water, int32_t n_pairs,
                        const double* host_x, const double* host_v);
int32_t h4d_num_replicas(h4d_ctx* ctx);

/* ---- screened-Coulomb force term of the LJ electrolyte (Eqs. 9-11, host only) ----
 * The force pass of the LJ electrolyte evaluates -du/dr / r of K q_i q_j erfc(alpha r)/r
 * as K q_i q_j (r^-3 + C(r^2)), C(s) = alpha^3 H(alpha^2 s) with
 * H(v) = (erfc(x) + 2x/sqrt(pi) e^{-v} - 1)/x^3 (x^2 = v), an entire function of v.  This
 * returns the degree-7 interpolant of C in s = r^2 that the engine uses for this alpha and
 * Coulomb cut-off (coef[0..7], lowest power first; 8 floats written by the callee) and
 * *used = 1, or zeros and *used = 0 when alpha rc_coul > 1.3 (the cancellation of r^-3 + C
 * at the cut-off would cost accuracy; the engine then keeps the erfc form).  No GPU
 * needed; H4D_EINVAL for NULL pointers. */
int h4d_coulomb_poly(double alpha, double rc_coul, float* coef, int32_t* used);

/* ---- device facts (no paper counterpart; measurement support) ---- */
/* SM count of the current device, and the compute capability (major*10 + minor, 103 for
 * sm_103a) and PTX version the engine kernel of this build was compiled for, from the
 * CUDA runtime's kernel attributes.  H4D_ENODEV without a suitable device. */
int h4d_device_info(int32_t* sm_count, int32_t* binary_version, int32_t* ptx_version);
/* Measured FP32 throughput of the current device: a kernel of independent FMA chains on
 * every SM (8 CTAs of 256 threads per SM, no memory traffic), timed with CUDA events on
 * the legacy default stream; *tflops = 2 x FMAs / time (and *seconds the time when not
 * NULL).  Allocates a small device buffer; synchronises. */
int h4d_measure_fp32_peak(double* tflops, double* seconds);
/* total pairs inside the larger cut-off over all replicas at the current state (each
 * unordered pair once); the algorithmic work unit of the pair kernel */
int h4d_count_pairs(h4d_ctx* ctx, int64_t* n_pairs_in_cutoff);

/* ---- learned insertion-site proposal ----
 * A proposal density over a grid of G^3 cells per replica (G = max(3, floor(L/cell_len)),
 * at most 32) replaces the uniform placement of an inserted ion (Eq. 4).  Each cell has 96
 * features: for the cation, the anion and the water O, 0.25 x the atom count of each of
 * the 27 cells of its 3x3x3 neighbourhood (81); 0.1 x the field sum_j q_j d_j /
 * max(|d_j|, 0.5)^3 at the cell centre from the charges of those cells (3); zeros (12).
 * An MLP 96-64-64-2 (ReLU; BF16 operands, FP32 accumulation on the tensor cores) gives a
 * cation and an anion logit per cell; species s draws its cell from
 * q_s = (1 - eps) softmax(logit_s) + eps / G^3 and is placed uniformly inside it.  The
 * density ratio to uniform placement enters the acceptance exponent as the bias factors
 * B^ins / B^del do in Eqs. 15-16, so detailed balance holds for any weights: an insertion
 * subtracts ln(q_c G^3) + ln(q_a G^3) evaluated on the start state, a deletion adds it
 * evaluated on the end state with the flyers removed (record field ln_q).
 * Random draws: block 5 of the trial (counter {trial, 5, 1, 0}): words 0 and 1 choose the
 * uniform component (u < eps) for the cation and the anion, words 2 and 3 the cell; the
 * 32-bit position draws of blocks 1-2 place the ion inside the cell.  Cannot be combined
 * with the bimodal bias (H4D_EINVAL).
 * Flat weight layout (row index = input unit, doubles on the host, FP32 masters on the
 * device): W1[96][64], b1[64], W2[64][64], b2[64], W3[64][2], b3[2]. */
#define H4D_PROPOSAL_UNIFORM 0
#define H4D_PROPOSAL_LEARNED 1
#define H4D_PROP_NFEAT 96
#define H4D_PROP_NW (96 * 64 + 64 + 64 * 64 + 64 + 64 * 2 + 2) /* 10498 */

/* Enable the proposal grid on every replica.  mode UNIFORM keeps uniform placement (for
 * collecting training records), LEARNED draws cells from q (weights start at zero, i.e.
 * uniform, until set or trained).  eps in (0, 1].  records_per_replica > 0 allocates a
 * ring of training records per replica: every trial with status 0 or 3 stores the
 * features of the cation's and the anion's cell in the N-pair state of the move (start
 * state of an insertion, end state of a deletion) and the insertion-direction exponent y
 * (x_acc of an insertion, -x_acc of a deletion, both without the proposal factor).
 * Calling it again re-sizes the grid and empties the rings; the network is kept.
 * Allocates device memory; synchronises the stream. */
int h4d_proposal(h4d_ctx* ctx, int32_t mode, double cell_len, double eps, int32_t records_per_replica);
/* set / read the H4D_PROP_NW weights; setting resets the optimiser state */
int h4d_proposal_set_weights(h4d_ctx* ctx, const double* host_w, int64_t n);
int h4d_proposal_get_weights(h4d_ctx* ctx, double* host_w, int64_t n);
/* the most recent training records of a replica, oldest first: host_feat [n][2][96]
 * (cation cell, anion cell), host_y [n], host_move [n], host_status [n]; any output may be
 * NULL */
int h4d_proposal_records(h4d_ctx* ctx, int32_t replica, float* host_feat, double* host_y,
                         int32_t* host_move, int32_t* host_status, int64_t cap, int64_t* n);
/* logits [G^3][2] (and features [G^3][96] when host_feat is not NULL) of every cell of a
 * replica's current state; H4D_ECAPACITY when cap_cells < G^3 */
int h4d_proposal_logits(h4d_ctx* ctx, int32_t replica, float* host_logits, float* host_feat,
                        int64_t cap_cells, int64_t* n_cells);
/* steps of Adam (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on the recorded
 * trials of all replicas (status 0, finite y).  Loss of n records: (1/n) sum [BCE(cation
 * logit of the cation cell, t) + BCE(anion logit of the anion cell, t)] with
 * t = min(1, exp(y - y0)).  Each step draws batch records uniformly (Philox counter
 * {step, k/4, 5, 0}, key {seed, 2^63}); batch >= the number of valid records uses all of
 * them in ring order.  *host_loss receives the loss of the last step.  Synchronises. */
int h4d_train_proposal(h4d_ctx* ctx, int64_t steps, int32_t batch, double lr, double y0, uint64_t seed,
                       double* host_loss);
/* stateless: loss (as above) and its gradient [H4D_PROP_NW] for weights host_w on
 * n_rec records host_feat [n][2][96] with targets host_t [n][2] (cation row, anion row),
 * computed by the same BF16 forward and backward kernels as training.  Allocates device
 * scratch per call; synchronises the default stream. */
int h4d_proposal_grad(const double* host_w, int64_t n_rec, const float* host_feat, const float* host_t,
                      double* loss, double* host_grad);

/* ---- checkpoint ----
 * h4d_save writes a flat binary image (magic "HH4D0004", seed, replica table, positions,
 * velocities, trial records) of a context; it synchronises.  h4d_load restores it into a
 * context created with the same system (replica count, atom capacities, waters, box edges
 * and ion capacities must match, else H4D_EINVAL and nothing is changed): each chain's
 * ion count, counters, random-number keys and counters, statistics and records come from the file,
 * the context keeps its own geometry, thresholds, launch plan, proposal grid and record
 * rings.  Out-of-range fields (ion count above capacity, negative record count, an
 * lane count that is not a power of two up to 32) are rejected.  A resumed chain continues bit-identically. */
int h4d_save(h4d_ctx* ctx, const char* path);
int h4d_load(h4d_ctx* ctx, const char* path);

/* ---- stateless kernels (one system, host buffers) ---- */

/* 4D pair forces and energy of one configuration (Sec. II.A 4D distance; Eqs. 9-11, 19-20):
 * host_x [n][3] positions, host_w [n] altitudes (NULL = all 0); atom types follow the
 * layout above with n_water waters.  Writes host_F [n][3] (FP32 math, returned as
 * double) and *U (FP64).  Altitude-screening applies to pairs with exactly one nonzero
 * altitude.  Allocates device scratch per call. */
int h4d_eval_forces(const h4d_params* params, double L, int32_t n_water, int32_t n,
                    const double* host_x, const double* host_w, double* host_F, double* U);

/* The computation of h4d_eval_forces for callers that cannot allocate device memory
 * (for example a host that forbids cudaMalloc inside its own callbacks, or code that
 * runs under a device-memory budget it does not control).  The paper has no counterpart;
 * this entry point exists for such embedders only.
 * Same arguments, units and results as h4d_eval_forces (host buffers in and out; n = 0
 * gives *U = 0 and touches no device memory).  It
 * calls no cudaMalloc, cudaFree or other allocating routine: every device buffer lives in
 * one file-scope array of 16 MiB that each GPU loading the library holds until the
 * process exits.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current; make that first call before any stream
 * capture.  Sizes that do not fit (about 6000 LJ atoms with default capacities) return
 * H4D_ECAPACITY.  All calls share the array and it keeps the last call's contents (each
 * call writes everything it reads); calls that overlap on the GPU -- from several host
 * threads or processes sharing a context -- race on it and must be serialised by the
 * caller.  Works on the legacy default stream and returns after synchronising it. */
int h4d_eval_forces_static(const h4d_params* params, double L, int32_t n_water, int32_t n,
                           const double* host_x, const double* host_w, double* host_F, double* U);

/* Long-range Coulomb term of one configuration (Sec. II.B.2, Eqs. 9-10): the paper splits
 * the 4D Coulomb energy into the screened short-range part (the pair term of
 * h4d_eval_forces) and the 3D long-range part U_lr = U_recip + U_self, which NEMD scales
 * by g^lr(wbar) = exp(-kappa_lr wbar) (wbar = mean altitude of the flying particles).
 *   U_recip = g (2 pi K / V) sum_{k != 0} exp(-k^2 / 4 alpha^2) / k^2 |S(k)|^2,
 *   S(k) = sum_j q_j exp(i k.r_j), k = 2 pi n / L over 0 < max_d |n_d| <= kmax;
 *   U_self = -g K alpha / sqrt(pi) sum_j q_j^2;
 *   host_F (may be NULL) [n][3] = -dU_recip/dx (FP32 sums of k-vector tiles, FP64 totals).
 * Charges follow the atom layout of h4d_eval_forces (params->q by type, K = params->kcoul);
 * host_x [n][3] in [0, L) (wrapped otherwise).  Intramolecular exclusion corrections of
 * rigid waters are not included (they do not depend on the positions of other molecules).
 * t_kernel_ms (may be NULL) receives the device time of the two kernels (structure factors,
 * forces), from CUDA events recorded around each launch.
 * H4D_EINVAL for alpha <= 0, kmax outside 1..64, negative wbar or kappa_lr.  Allocates
 * device scratch per call; runs on the legacy default stream and synchronises it. */
int h4d_ewald_lr(const h4d_params* params, double L, int32_t n_water, int32_t n, const double* host_x,
                 double alpha, int32_t kmax, double wbar, double kappa_lr, double* U_recip,
                 double* U_self, double* host_F, double* t_kernel_ms);

/* Neighbour pairs (i < j) under the fixed-point criterion: X = round(x/L 2^32) mod 2^32
 * per coordinate, pair iff sum ((int32)(X_i - X_j))^2 <= floor((r_list/L 2^32)^2).
 * Writes up to cap pairs sorted by (i, j) and the total count to *n_out. */
int h4d_neighbor_pairs(double L, int32_t n, const double* host_x, double r_list, int32_t* host_i,
                       int32_t* host_j, int64_t cap, int64_t* n_out);

#ifdef __cplusplus
}
#endif
#endif /* H4D_H */
