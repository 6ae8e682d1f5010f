// h4d_engine.cuh -- device-side data layout of libh4d (shared by h4d_engine.cu and
// h4d_api.cu only).
//
// Layout in HBM (all replicas packed back to back, replica r at atom offset atom_off[r]):
//   pos   uint4  [atoms]  x,y,z as 32-bit fixed-point fractions of the box edge (exact
//                         periodic wrap and exact minimum-image differences), .w = altitude
//                         as float bits (nonzero only for flying ions)
//   vhi/vlo float4 [atoms] velocity as an unevaluated float-float sum (about 48 bits)
//   force float4  [atoms] FP32 force of the last evaluation
//   nbr   uint16  [atoms * max_nbr] full neighbour rows, tpa-interleaved (see nbr_index)
// Each replica is simulated by one group of warps (a whole CTA or a slice of one) that
// keeps the replica's positions in shared memory for the whole launch.
#pragma once
#include <cstdint>

#include "../../include/h4d.h"
#include "h4d_prop.cuh"

namespace h4d {

constexpr int kMaxT = 4;
constexpr int kMaxGroupsPerCta = 15;  // named barriers 1..15

struct Pot {
  int sys, ntypes;
  float sig2[16], eps4[16], ljshift[16], kq[16];  // per (ti*4 + tj)
  float rc2_lj, rc2_c, rc2_max, alpha, shift_c, two_alpha_sqrtpi, kappa_sr;
  float inv_m[kMaxT];  // 1 / (m mvv2e)
  float m_f[kMaxT];    // m mvv2e
  double dsig2[16], deps4[16], dljshift[16], dkq[16];
  double drc2_lj, drc2_c, dalpha, dshift_c, dkappa_sr;
  double dm[kMaxT];    // m mvv2e
  double d_oh2, d_hh2;  // squared water bond lengths
  double inv_m_d[kMaxT];
  float q[kMaxT];       // charges per type (proposal field feature)
  int erfcx_fit;        // alpha rc_coul within the range of the fitted erfcx (aqueous pair term)
  // LJ electrolyte: the screened-Coulomb force term -du/dr / r = kq g (r^-3 + C(r^2)), with
  // C a degree-7 polynomial in r^2 (coefficients cpoly[0..7], lowest first) when coul_poly
  int coul_poly;
  float cpoly[8];
  float lj12, lj6;      // 12 eps4 and 6 eps4 of the LJ electrolyte (one sigma, one epsilon)
};

struct Proto {
  int n_f, schedule;
  double w_max, sched_n, dt, tau_t;
  double beta, beta_mu;
  int no_accept;
  int prop_mode;    // 0 uniform placement, 1 learned proposal density
  int prop_record;  // write a training record for every trial
  int bias_on;      // bimodal flyer-distance bias (Sec. II.B.3)
  double prop_eps;  // weight of the uniform component of the learned proposal
  double bias_alpha, bias_xb;  // sharpness and mean separation of the bias (Eq. 16)
  double fw;  // species w_max: the anion's w_max is w_max + 0.5 (sig_c + sig_a) fw
  double rw;  // its ratio to the cation's (1 = one w_max); the anion's altitude is rw w
  double vex_edge;  // early rejection: edge of the excluded cube around the flying cation (0 = off)
  int single;       // single-particle exchange: one flyer, one atom per exchange unit
  int unit;         // atoms per exchange unit (2 for ion pairs, 1 for single particles)
  int water;        // rigid-water exchange: one flying water per trial, frozen in 3D
  int pad_w;
  // the water in its body frame (O at the origin, H atoms in the xy plane symmetric about
  // y): H offsets, centre of mass on y, total mass and principal moments about the centre
  // of mass, both times mvv2e, for the molecular-frame velocity draw of an insertion
  double wh[2][3], wcom_y, wM, wI[3];
};

struct Rep {
  double L;
  float scale;    // L / 2^32 (fixed-point unit in length)
  float c_drift;  // dt * 2^32 / L
  int n_water, nw3;
  int n_pairs, cap_pairs;
  int atom_off, cap_atoms;
  int cap_water, pad_cw;  // most waters the replica may hold (water exchange)
  int nc;         // cells per dimension (0 = all pairs)
  int reach;      // stencil half-width: cells are at least r_list / reach wide
  int tpa;
  int pad_r;
  unsigned long long T_list;   // neighbour criterion threshold (fixed-point units^2)
  unsigned long long T_move;   // (skin/2)^2 in fixed-point units^2
  float skin_fx;               // skin in fixed-point units
  float skin_out_fx;           // outer-list skin in fixed-point units
  unsigned long long T_out;    // outer-list threshold (fixed-point units^2)
  unsigned T16_out;            // conservative outer threshold on 16-bit coordinates
  unsigned T8_out;             // conservative outer threshold on 8-bit coordinates
  int rec_off, rec_cap;
  long long rec_count;
  unsigned long long trial_ctr, step_ctr;
  // statistics
  long long cycles, trials_ins, trials_del, acc_ins, acc_del, rej_status, md_steps, builds, err;
  double sum_n, sum_n2;
  double t_nemd_ns, t_md_ns;
  double t_build_ns, t_force_ns, t_energy_ns;  // phase timers (thread 0 of the group)
  long long refreshes;  // Verlet-row refreshes from the outer rows (outside full builds)
  double t_filter_ns;   // part of t_build_ns spent filtering Verlet rows from outer rows
  int dirty;      // state changed on the host: rebuild list and forces
  int prop_G;     // proposal grid cells per edge (0 = no grid)
  int prop_off;   // first cell of this replica in the grid arrays (a multiple of 32)
  int prec_off, prec_cap;  // training-record ring of this replica
  long long prec_count;
  unsigned long long key; // second Philox key word of this replica's random stream
  int smid, pad_s;        // SM of the group in the most recent launch
  unsigned long long t_begin, t_end;  // global timer at that launch's start and end
};

struct Group {
  int rep, warp0, nwarps, bar, smem_off, pad;
};

struct Eng {
  Pot pot;
  Proto proto;
  Rep* rep;
  const Group* groups;
  const int* cta_groups;  // groups of CTA c are [cta_groups[c], cta_groups[c+1])
  uint4* pos;
  float4* vhi;
  float4* vlo;
  float4* force;
  uint4* pos_save;
  float4* vhi_save;
  float4* vlo_save;
  uint4* ref;
  uint16_t* nbr;      // inner (Verlet) rows, tpa-interleaved packets
  int* ncnt;
  uint16_t* nbr_out;  // outer rows (larger skin, one lane per atom), rebuilt from cells
  int* ncnt_out;
  uint4* ref_out;     // positions at the last outer build
  h4d_record* rec;
  double* red;        // per-atom partial sums of the fixed-order FP64 reductions
  // learned proposal: packed network, per-cell grid of every replica, training records
  PropNet net;
  int4* pg_cnt;         // [cells] cation, anion, water-O counts of the cell itself
  long long* pg_fld;    // [cells][4] field at the cell centre, fixed point 2^-40
  float2* pg_logit;     // [cells] cation and anion logits
  double2* pg_chunk;    // [cells / 32] softmax partial sums per 32-cell chunk
  float* prec_feat;     // [records][2][96] features of the cation and the anion cell
  double* prec_y;       // [records] insertion-direction exponent without proposal factor
  int2* prec_meta;      // [records] move, status (-1 = empty slot)
  int max_nbr;
  int max_out;
  unsigned long long seed;
  int rows_by_index;  // 1: Verlet rows stored by atom index (the neighbour-pair export)
  int pad_e;
  // row layout (per replica, at atom_off): lrank[i] = row position of atom i at the next
  // outer build (from the row lengths of the last filter), lord[k] = atom whose rows are at
  // position k since the last outer build; NULL where the caller keeps rows by index
  uint16_t* lrank;
  uint16_t* lord;
};

// shared-memory bytes a group needs for a replica
__host__ __device__ inline size_t smem_align16(size_t b) { return (b + 15) & ~(size_t)15; }
// Per-group shared memory: positions (plus one sentinel slot after the last atom, which
// neighbour-row padding points at), cell starts, cell fill counters / work-item prefix,
// cell-sorted atom list (each cell padded to a multiple of 4 entries), the same list as
// packed 8-bit coordinates, scalars.  Every region starts on a 16-byte boundary.
__host__ __device__ inline size_t group_smem_bytes(int cap_atoms, int nc, int nthreads) {
  (void)nthreads;
  size_t ncell = nc > 0 ? (size_t)nc * nc * nc : 0;
  size_t slots = (size_t)cap_atoms + 3 * ncell;
  size_t b = smem_align16(16 * ((size_t)cap_atoms + 1));
  b += smem_align16(4 * (ncell + 1));
  b += smem_align16(4 * (ncell + 1));
  b += smem_align16(2 * slots);
  b += smem_align16(4 * slots);
  b += 1536;
  return (b + 127) & ~(size_t)127;
}

// Launches (h4d_engine.cu)
int launch_cycles(const Eng& e, int n_ctas, int cta_threads, size_t smem, long long k_cycles,
                  int n_eq, int do_trial, void* stream);
int launch_energy(const Eng& e, int n_ctas, int cta_threads, size_t smem, double* U, double* K,
                  void* stream);
int launch_eval(const Eng& e, int threads, size_t smem, float wbar, double* U, void* stream);
int launch_forces(const Eng& e, int n_ctas, int cta_threads, size_t smem, int n_iter, void* stream);
int launch_list(const Eng& e, int n_ctas, int cta_threads, size_t smem, void* stream);
int launch_count_pairs(const Eng& e, int n_ctas, int cta_threads, size_t smem,
                       unsigned long long* out, void* stream);
// compute capability the engine kernel was compiled for and its PTX version (x10 + minor)
int engine_binary_version(int* binary_version, int* ptx_version);
int launch_prop_eval(const Eng& e, int n_ctas, int cta_threads, size_t smem, int replica, float* feat_out,
                     void* stream);

}  // namespace h4d
