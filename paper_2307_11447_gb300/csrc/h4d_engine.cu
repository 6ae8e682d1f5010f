// h4d_engine.cu -- sm_103a kernels of libh4d: neighbour build, 4D pair force/energy,
// velocity Verlet with the altitude protocol, FP64 work/energy sums, Metropolis and
// commit, CSVR equilibrium MD.  One group of warps owns one replica for a whole launch
// and keeps its positions in shared memory; all steps of all cycles run inside the
// launch (persistent), synchronised by the group's named barrier.
//
// Paper references: Sec. II.A (Eq. 2 protocol, NVE evolution, two-end momentum reversal,
// Eqs. 3-8 Metropolis), Sec. II.B.1 (flyers fixed in 3D), Sec. II.B.2 (Eqs. 9-11
// screened 4D Coulomb), Sec. II.D (Eqs. 19-20 potentials), SI Sec. S5 (Eqs. S6-S7).
#include <cuda_runtime.h>

#include <cstdint>

#include "h4d_engine.cuh"
#include "h4d_philox.cuh"
#include "h4d_prop.cuh"

// Engine launch bounds: threads per CTA and CTAs per SM the register allocation targets
// launch bounds of the engine kernels: CTAs of up to 32 warps, 64 registers per thread
#ifndef H4D_MAXTHREADS
#define H4D_MAXTHREADS 1024
#endif
#ifndef H4D_MINBLOCKS
#define H4D_MINBLOCKS 1
#endif

// Attribute of the phase functions (list build, filter, force pass, kick/drift, FP64
// energy, the MD and NEMD step loops).  Empty: the compiler inlines them into the
// persistent kernel (measured faster on GB300 than __noinline__, where each phase would
// get a register budget of its own at the cost of a call and a context copy).
#ifndef H4D_PHASE
#define H4D_PHASE
#endif

namespace h4d {

// ------------------------------------------------------------------------------------
// small helpers
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void gsync(int bar, int nthreads) {
  if (bar == 0) __syncthreads();
  else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nthreads) : "memory");
}

__device__ __forceinline__ int type_of(int a, int nw3) {
  return a < nw3 ? ((a % 3 == 0) ? 2 : 3) : ((a - nw3) & 1);
}
template <int SYS>
__device__ __forceinline__ int type_t(int a, int nw3) {
  if (SYS == H4D_SYS_LJ) return a & 1;  // no waters: ions alternate cation/anion
  return type_of(a, nw3);
}

// float-float accumulate: (hi, lo) += d
__device__ __forceinline__ void ff_add(float& hi, float& lo, float d) {
  float s = hi + d;
  float bp = s - hi;
  float err = (hi - (s - bp)) + (d - bp);
  lo += err;
  float t = s + lo;
  lo = lo - (t - s);
  hi = t;
}
// (hi, lo) *= a
__device__ __forceinline__ void ff_scale(float& hi, float& lo, float a) {
  float p = hi * a;
  float e = fmaf(hi, a, -p);
  float l = fmaf(lo, a, e);
  float t = p + l;
  lo = l - (t - p);
  hi = t;
}

__device__ __forceinline__ float wbits(const uint4& p) { return __uint_as_float(p.w); }

// Abramowitz & Stegun 7.1.26: erfc(x) = t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) e^{-x^2},
// t = 1/(1 + p x), |error| <= 1.5e-7 for x >= 0.  Returns the polynomial factor; the
// caller multiplies by e^{-x^2}, which it also needs for the force.
__device__ __forceinline__ float as_erfc_poly(float x) {
  float t;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(fmaf(0.3275911f, x, 1.0f)));
  float p = fmaf(t, 1.061405429f, -1.453152027f);
  p = fmaf(t, p, 1.421413741f);
  p = fmaf(t, p, -0.284496736f);
  p = fmaf(t, p, 0.254829592f);
  return p * t;
}
// erfcx(x) = e^{x^2} erfc(x) on [0, 3.2] as t sum_k c_k t^k, t = 1/(1 + x/2), with the
// coefficients printed by fit_erfcx.py (a least-squares fit in relative error, reweighted
// toward minimax: 1.3e-10 in exact arithmetic, 3.3e-7 in this float32 evaluation)
__device__ __forceinline__ float erfcx_poly(float x) {
  const float t = __frcp_rn(fmaf(0.5f, x, 1.0f));
  float p = 3.845890611e-02f;
  p = fmaf(p, t, -2.708916664e-01f);
  p = fmaf(p, t, 7.915914059e-01f);
  p = fmaf(p, t, -1.178810358e+00f);
  p = fmaf(p, t, 8.702221513e-01f);
  p = fmaf(p, t, -3.565987349e-01f);
  p = fmaf(p, t, 3.224146068e-01f);
  p = fmaf(p, t, 2.157940567e-01f);
  p = fmaf(p, t, 2.859359086e-01f);
  p = fmaf(p, t, 2.818836868e-01f);
  return p * t;
}
__device__ __forceinline__ float exp_neg_sq(float x) {
  // e^{-x^2} = 2^{-x^2 log2 e}
  float y = -x * x * 1.4426950408889634f;
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
  return r;
}

// pair-table entry of (ti, tj)
template <int SYS>
struct PairCoef {
  float sig2, eps4, ljshift, kq;
};

template <int SYS>
__device__ __forceinline__ PairCoef<SYS> coef(const Pot& P, int ti, int tj) {
  PairCoef<SYS> c;
  if (SYS == H4D_SYS_LJ) {
    // equal sizes and energies; charges +1/-1 by type parity
    c.sig2 = P.sig2[0];
    c.eps4 = P.eps4[0];
    c.ljshift = P.ljshift[0];
    c.kq = (ti == tj) ? P.kq[0] : P.kq[1];
  } else {
    int k = ti * 4 + tj;
    c.sig2 = P.sig2[k];
    c.eps4 = P.eps4[k];
    c.ljshift = P.ljshift[k];
    c.kq = P.kq[k];
  }
  return c;
}

// -du/dr / r of the 4D pair term (FP32): LJ (Eq. 19) + screened erfc Coulomb (Eqs. 9-11, 20)
template <int SYS>
__device__ __forceinline__ float pair_fr(const Pot& P, const PairCoef<SYS>& c, float r2, float g) {
  float rinv = rsqrtf(r2);
  float rinv2 = rinv * rinv;
  float s2 = c.sig2 * rinv2;
  float s6 = s2 * s2 * s2;
  float fr_lj = c.eps4 * s6 * fmaf(12.0f, s6, -6.0f) * rinv2;
  fr_lj = (r2 < P.rc2_lj) ? fr_lj : 0.0f;
  float r = r2 * rinv;
  float x = P.alpha * r;
  float ex = exp_neg_sq(x);
  // LJ electrolyte: alpha r <= 1.2, where the A&S form (absolute error 1.5e-7) is ~1e-6
  // relative; aqueous: alpha r reaches 2.5, where only a relatively accurate erfc keeps
  // the cancelling water Coulomb sums at 1e-5: e^{-x^2} times the fitted erfcx (relative
  // error as small as the library erfcf's, and it shares e^{-x^2} with the force term),
  // or the library erfcf when the cut-off reaches beyond the fit
  float erfcx;
  if (SYS == H4D_SYS_LJ) {
    erfcx = as_erfc_poly(x) * ex;
  } else if (P.erfcx_fit) {
    erfcx = ex * erfcx_poly(x);
  } else {
    erfcx = erfcf(x);
  }
  float fr_c = c.kq * g * fmaf(erfcx, rinv, P.two_alpha_sqrtpi * ex) * rinv2;
  fr_c = (r2 < P.rc2_c) ? fr_c : 0.0f;
  return fr_lj + fr_c;
}

// Two LJ-electrolyte pair terms at once on the packed FP32x2 pipe (FFMA2 / FMUL2 / FADD2):
// every operation of pair_fr<H4D_SYS_LJ> in the same order and association, each lane
// rounded as the scalar operation is, so each result is bit-identical to pair_fr; the
// special functions (rsqrt, ex2, rcp) and the cut-off selects stay per lane.  kqg is the
// pair's charge prefactor times its screening factor.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float ex2_approx(float y) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
  return r;
}
__device__ __forceinline__ float rcp_approx(float y) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
  return r;
}
__device__ __forceinline__ float2 pair_fr_lj2(const Pot& P, float2 r2, float2 kqg) {
  const float2 rinv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
  const float2 rinv2 = __fmul2_rn(rinv, rinv);
  const float2 s2 = __fmul2_rn(f2(P.sig2[0]), rinv2);
  const float2 s6 = __fmul2_rn(__fmul2_rn(s2, s2), s2);
  float2 fr_lj = __fmul2_rn(__fmul2_rn(__fmul2_rn(f2(P.eps4[0]), s6), __ffma2_rn(f2(12.0f), s6, f2(-6.0f))), rinv2);
  fr_lj.x = (r2.x < P.rc2_lj) ? fr_lj.x : 0.0f;
  fr_lj.y = (r2.y < P.rc2_lj) ? fr_lj.y : 0.0f;
  const float2 x = __fmul2_rn(f2(P.alpha), __fmul2_rn(r2, rinv));
  const float2 y = __fmul2_rn(__fmul2_rn(make_float2(-x.x, -x.y), x), f2(1.4426950408889634f));
  const float2 ex = make_float2(ex2_approx(y.x), ex2_approx(y.y));
  const float2 d = __ffma2_rn(f2(0.3275911f), x, f2(1.0f));
  const float2 t = make_float2(rcp_approx(d.x), rcp_approx(d.y));
  float2 p = __ffma2_rn(t, f2(1.061405429f), f2(-1.453152027f));
  p = __ffma2_rn(t, p, f2(1.421413741f));
  p = __ffma2_rn(t, p, f2(-0.284496736f));
  p = __ffma2_rn(t, p, f2(0.254829592f));
  const float2 erfcx = __fmul2_rn(__fmul2_rn(p, t), ex);
  float2 fr_c = __fmul2_rn(__fmul2_rn(kqg, __ffma2_rn(erfcx, rinv, __fmul2_rn(f2(P.two_alpha_sqrtpi), ex))), rinv2);
  fr_c.x = (r2.x < P.rc2_c) ? fr_c.x : 0.0f;
  fr_c.y = (r2.y < P.rc2_c) ? fr_c.y : 0.0f;
  return __fadd2_rn(fr_lj, fr_c);
}

// The same two pair terms with the screened-Coulomb force as r^-3 + C(r^2) (C the degree-7
// polynomial the host interpolates for this alpha and cut-off, Pot::cpoly): Eqs. 9-11 with
// the erfc and Gaussian terms folded into C, so one rsqrt is the only special function of
// a pair.  The LJ term of Eq. 19 takes 12 eps4 and 6 eps4 as constants.  Pairs beyond a
// cut-off (skin entries, the sentinel at infinite altitude) are dropped by selects, so the
// polynomial's value there does not matter.
__device__ __forceinline__ float2 pair_fr_lj2_poly(const Pot& P, float2 r2, float2 kqg) {
  const float2 rinv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
  const float2 rinv2 = __fmul2_rn(rinv, rinv);
  const float2 s2 = __fmul2_rn(f2(P.sig2[0]), rinv2);
  const float2 s6 = __fmul2_rn(__fmul2_rn(s2, s2), s2);
  float2 fr_lj = __fmul2_rn(__fmul2_rn(s6, __ffma2_rn(f2(P.lj12), s6, f2(-P.lj6))), rinv2);
  fr_lj.x = (r2.x < P.rc2_lj) ? fr_lj.x : 0.0f;
  fr_lj.y = (r2.y < P.rc2_lj) ? fr_lj.y : 0.0f;
  float2 cp = __ffma2_rn(f2(P.cpoly[7]), r2, f2(P.cpoly[6]));
#pragma unroll
  for (int k = 5; k >= 0; --k) cp = __ffma2_rn(cp, r2, f2(P.cpoly[k]));
  float2 fr_c = __fmul2_rn(kqg, __ffma2_rn(rinv2, rinv, cp));
  fr_c.x = (r2.x < P.rc2_c) ? fr_c.x : 0.0f;
  fr_c.y = (r2.y < P.rc2_c) ? fr_c.y : 0.0f;
  return __fadd2_rn(fr_lj, fr_c);
}

// FP32 pair energy (protocol-work diagnostic only)
template <int SYS>
__device__ __forceinline__ float pair_u32(const Pot& P, const PairCoef<SYS>& c, float r2, float g) {
  float u = 0.0f;
  float rinv = rsqrtf(r2);
  if (r2 < P.rc2_lj) {
    float s2 = c.sig2 * rinv * rinv;
    float s6 = s2 * s2 * s2;
    u += c.eps4 * (s6 * s6 - s6) - c.ljshift;
  }
  if (r2 < P.rc2_c) {
    float x = P.alpha * r2 * rinv;
    float erfcx = (SYS == H4D_SYS_LJ) ? as_erfc_poly(x) * exp_neg_sq(x) : erfcf(x);
    u += c.kq * g * (erfcx * rinv - P.shift_c);
  }
  return u;
}

// FP64 pair energy for the end-point Hamiltonians of each trial
__device__ __forceinline__ double pair_u64(const Pot& P, int ti, int tj, double r2, double g) {
  int k = ti * 4 + tj;
  double u = 0.0;
  if (r2 < P.drc2_lj && P.deps4[k] != 0.0) {
    double s2 = P.dsig2[k] / r2;
    double s6 = s2 * s2 * s2;
    u += P.deps4[k] * (s6 * s6 - s6) - P.dljshift[k];
  }
  if (r2 < P.drc2_c && P.dkq[k] != 0.0) {
    double r = sqrt(r2);
    u += P.dkq[k] * g * (erfc(P.dalpha * r) / r - P.dshift_c);
  }
  return u;
}

// ------------------------------------------------------------------------------------
// Per-group shared memory
// ------------------------------------------------------------------------------------
struct GScal {
  int flag_rebuild, flag_overflow, flag_nan, n_tot;
  int fly0, fly1, ins, status;
  int flip_s, flip_e, cat, ani;
  int n_before, accept, inst;  // inst: instantaneous move (early rejection)
  int flag_timeout;            // a bounded iteration (SHAKE, RATTLE, gamma draw) gave up
  int fly2, flyw;              // water exchange: third flying atom, flying water (-1 = none)
  int nw_trial;                // waters in the layout of the running trial
  int n_ord;                   // atoms of the current Verlet-row layout (sorted[0, n_ord)); 0 = by index
  float w_cur, g_scr, pad2, pad3;
  double alpha_th, dW[3], wprot, wprot_c, red_out;
  double ln_u, ustart, kstart, uend, kend;
  double vfly[6];
  unsigned int xfly[6];
  double vw[9];            // velocities of an inserted water (O, H, H)
  unsigned int xw[9];      // its fixed-point coordinates
  double kw[32];
  float d1w[32], d2w[32];  // per-warp largest and second-largest displacement since the build
  float o1w[32], o2w[32];  // the same since the outer-list build
  int next_item, n_items;  // dynamic work items of the outer build
  // learned proposal of the current trial
  float pm[2];             // largest cation / anion logit
  float pmw[2][32];        // per-warp maxima
  double pZ[2];            // softmax normalisers sum_k exp(l_k - max)
  double lnq;              // log proposal factor of the trial
  int cell_c, cell_a;      // grid cells of the exchanged cation and anion
  int prec_slot;           // training-record slot of the trial (-1 = none)
  int n_rank;              // atoms ranked in lrank for the next outer build (0 = none)
  int n_lay;               // atoms of the outer-row layout in lord (0 = rows by index)
  int pad_l;
};
static_assert(sizeof(GScal) <= 1536, "per-group scalars exceed their shared-memory slot");

struct GView {
  uint4* pos;
  int* cstart;
  int* cfill;
  uint16_t* sorted;
  unsigned* sorted8;  // packed 8-bit box coordinates of the sorted list (x | y<<8 | z<<16)
  GScal* s;
};

__device__ __forceinline__ GView carve(char* base, int cap_atoms, int nc, int nthreads) {
  (void)nthreads;
  GView v;
  size_t ncell = nc > 0 ? (size_t)nc * nc * nc : 0;
  size_t slots = (size_t)cap_atoms + 3 * ncell;
  char* p = base;
  v.pos = (uint4*)p; p += smem_align16(16 * ((size_t)cap_atoms + 1));
  v.cstart = (int*)p; p += smem_align16(4 * (ncell + 1));
  v.cfill = (int*)p; p += smem_align16(4 * (ncell + 1));
  v.sorted = (uint16_t*)p; p += smem_align16(2 * slots);
  v.sorted8 = (unsigned*)p; p += smem_align16(4 * slots);
  v.s = (GScal*)p;
  return v;
}

// The sentinel slot after a replica's last possible atom: row padding (kNoAtom) is read
// as min(index, cap_atoms), i.e. as this slot, whose infinite altitude puts it beyond every
// cut-off, so padding needs neither a branch nor a mask in the pair loop.
__device__ __forceinline__ void write_sentinel(const GView& v, int cap_atoms) {
  v.pos[cap_atoms] = make_uint4(0u, 0u, 0u, 0x7F800000u);
}

__device__ __forceinline__ unsigned pack8(const uint4& p) {
  return (p.x >> 24) | ((p.y >> 24) << 8) | ((p.z >> 24) << 16);
}

// read-only geometry of the group's replica, held in registers for the whole launch so
// inner loops never reload it from global memory
struct RepC {
  double L;
  float scale, c_drift;
  int n_water, nw3, atom_off, cap_atoms, nc, cap_pairs;
  unsigned long long T_list, T_move;
  float skin_fx;      // Verlet-list skin in fixed-point units
  float skin_out_fx;  // outer-list skin in fixed-point units
  unsigned long long T_out;
  unsigned T16_out;   // conservative outer threshold on 16-bit coordinates
  unsigned T8_out;    // conservative outer threshold on 8-bit coordinates
};

__device__ __forceinline__ RepC repc_of(const Rep& R) {
  RepC r;
  r.L = R.L; r.scale = R.scale; r.c_drift = R.c_drift;
  r.n_water = R.n_water; r.nw3 = R.nw3; r.atom_off = R.atom_off; r.cap_atoms = R.cap_atoms;
  r.nc = R.nc; r.cap_pairs = R.cap_pairs; r.T_list = R.T_list; r.T_move = R.T_move;
  r.skin_fx = R.skin_fx;
  r.skin_out_fx = R.skin_out_fx;
  r.T_out = R.T_out;
  r.T16_out = R.T16_out;
  r.T8_out = R.T8_out;
  return r;
}

struct Ctx {
  GView v;
  RepC r;
  Rep* R;
  const Eng* e;
  int tid, T, bar, tpa, ltpa;
  __device__ void sync() const { gsync(bar, T); }
};

// Row slot s of atom i lives in packet P = s/4 (element s%4).  Packets are dealt to the
// atom's tpa lanes round-robin (lane P % tpa, its (P / tpa)-th packet), and the packets of
// consecutive atoms are adjacent, so one 8-byte load per lane gives four neighbours and a
// warp reads 256 contiguous bytes.  Builders fill a row packet by packet and store whole
// packets; the last packet of a row is padded with kNoAtom.
constexpr uint16_t kNoAtom = 0xFFFF;
__device__ __forceinline__ size_t packet_index(const Eng& e, const RepC& R, int i, int P, int ltpa) {
  return (size_t)R.atom_off * e.max_nbr / 4 + ((((size_t)(P >> ltpa) * R.cap_atoms + i) << ltpa) + (P & ((1 << ltpa) - 1)));
}
__device__ __forceinline__ size_t nbr_index(const Eng& e, const RepC& R, int i, int s, int ltpa) {
  return packet_index(e, R, i, s >> 2, ltpa) * 4 + (s & 3);
}
// outer rows: one lane per atom (packets of four indices, consecutive atoms adjacent)
__device__ __forceinline__ size_t out_packet_index(const Eng& e, const RepC& R, int i, int P) {
  return (size_t)R.atom_off * e.max_out / 4 + (size_t)P * R.cap_atoms + i;
}
__device__ __forceinline__ const uint2* out_packets(const Eng& e, const RepC& R) {
  return reinterpret_cast<const uint2*>(e.nbr_out + (size_t)R.atom_off * e.max_out);
}
__device__ __forceinline__ const uint2* nbr_packets(const Eng& e, const RepC& R) {
  return reinterpret_cast<const uint2*>(e.nbr + (size_t)R.atom_off * e.max_nbr);
}

// Exact group-wide sum of 64-bit fixed-point partials: integer addition is associative,
// so the result does not depend on how atoms are spread over threads or on the order of
// the warp slots (a replica gives the same sums in a CTA of its own and packed with others)
__device__ long long group_sum_fx(const Ctx& c, long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int warp = c.tid >> 5, lane = c.tid & 31;
  long long* slot = reinterpret_cast<long long*>(c.v.s->kw);
  c.sync();
  if (lane == 0) slot[warp] = x;
  c.sync();
  if (c.tid == 0) {
    long long s = 0;
    for (int w = 0; w < (c.T >> 5); ++w) s += slot[w];
    reinterpret_cast<long long*>(&c.v.s->red_out)[0] = s;
  }
  c.sync();
  return reinterpret_cast<const long long*>(&c.v.s->red_out)[0];
}

// kinetic-energy units of the fixed-point sums: 2^-32 per unit, per-atom values clamped
// at 2^16 so that 9160 atoms stay far inside int64 (a clamped atom also flags the state)
constexpr float kFxScale = 4294967296.0f;
constexpr float kFxClamp = 65536.0f;
__device__ __forceinline__ long long to_fx(float v, int& bad) {
  if (!(v <= kFxClamp)) { bad = 1; v = kFxClamp; }
  return __float2ll_rn(v * kFxScale);
}

// Sum of buf[0, n) (this replica's per-atom partials in global memory, written before the
// call) in an order fixed by n alone: thread k adds the 32 values of chunk k, then the
// lanes of warp 0 add every 32nd chunk sum and a fixed butterfly combines the lanes
__device__ double fixed_order_sum(const Ctx& c, double* buf, int n) {
  c.sync();
  const int nch = (n + 31) >> 5;
  for (int k = c.tid; k < nch; k += c.T) {
    double s = 0.0;
    const int q1 = min(n, 32 * k + 32);
    for (int q = 32 * k; q < q1; ++q) s += buf[q];
    buf[32 * k] = s;
  }
  c.sync();
  if (c.tid < 32) {
    double s = 0.0;
    for (int k = c.tid; k < nch; k += 32) s += buf[32 * k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (c.tid == 0) c.v.s->red_out = s;
  }
  c.sync();
  return c.v.s->red_out;
}

// L2 prefetch of a row packet a few packets ahead of the one being loaded: the rows stream
// from HBM and each lane walks its own, so the next packet alone does not cover the latency
// (distances in packets, build options; 0 = none)
#ifndef H4D_PF_FILTER
#define H4D_PF_FILTER 8
#endif
#ifndef H4D_PF_FORCE
#define H4D_PF_FORCE 4
#endif
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
__device__ __forceinline__ void prefetch_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

__device__ __forceinline__ u64 gtimer() {
  u64 t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// four row entries collected in a 64-bit shift register and stored as one 8-byte packet
// (first entry in the low 16 bits); a partial packet is completed with kNoAtom
struct RowBuf {
  unsigned long long b;
  int n;
  __device__ __forceinline__ void init() { b = ~0ull; n = 0; }
  __device__ __forceinline__ void put(int j) {
    b = (b >> 16) | ((unsigned long long)(unsigned)j << 48);
    ++n;
  }
  // put(j) when ok, with selects instead of a branch
  __device__ __forceinline__ void put_if(bool ok, int j) {
    const unsigned long long nb = (b >> 16) | ((unsigned long long)(unsigned)j << 48);
    b = ok ? nb : b;
    n += ok ? 1 : 0;
  }
  __device__ __forceinline__ uint2 packet() const {
    const unsigned long long x = b >> (16 * (4 - n));  // shift in kNoAtom for missing entries
    const unsigned long long y = x | (n == 4 ? 0ull : (~0ull << (16 * n)));
    return make_uint2((unsigned)y, (unsigned)(y >> 32));
  }
};

// ------------------------------------------------------------------------------------
// Neighbour list: fixed-point cells, deterministic stable counting sort, full rows
// ------------------------------------------------------------------------------------
__device__ __forceinline__ int cell_of_pos(const uint4& p, int nc) {
  int cx = (int)__umulhi(p.x, (unsigned)nc);
  int cy = (int)__umulhi(p.y, (unsigned)nc);
  int cz = (int)__umulhi(p.z, (unsigned)nc);
  return (cx * nc + cy) * nc + cz;
}

__device__ __forceinline__ u64 fixed_d2(const uint4& a, const uint4& b) {
  long long dx = (int)(a.x - b.x), dy = (int)(a.y - b.y), dz = (int)(a.z - b.z);
  return (u64)(dx * dx) + (u64)(dy * dy) + (u64)(dz * dz);
}

// Conservative squared distance on the top 16 bits of the fixed-point coordinates (32-bit
// arithmetic, about 3 ALU ops per axis).  With T16 = ceil(r/q + 1)^2 (q = L/2^16), every
// pair closer than r passes; a few pairs slightly farther may pass too, which is harmless
// for the outer list because the Verlet rows apply the exact criterion.
__device__ __forceinline__ unsigned d2_16(const uint4& a, const uint4& b) {
  const int dx = (int)(a.x - b.x) >> 16, dy = (int)(a.y - b.y) >> 16, dz = (int)(a.z - b.z) >> 16;
  return (unsigned)(dx * dx) + (unsigned)(dy * dy) + (unsigned)(dz * dz);
}

__device__ __forceinline__ bool excluded_pair(int i, int j, int nw3) {
  return i < nw3 && j < nw3 && (i / 3) == (j / 3);
}

// Verlet-row layout by row length (see next_rank): 64 length buckets; replicas of fewer
// atoms keep rows by index (the bucket histogram uses sorted8, 4 bytes per atom slot)
constexpr int kOrderBuckets = 64;
constexpr int kOrderMin = 128;
#ifndef H4D_LANE_ORDER
#define H4D_LANE_ORDER 1
#endif
__device__ H4D_PHASE void build_list_impl(const Ctx& cref);
__device__ H4D_PHASE void filter_list_impl(const Ctx& cref);
// full build: outer rows from the cell grid, then the Verlet rows filtered from them
__device__ void build_list(const Ctx& c) {
  const u64 t0 = (c.tid == 0) ? gtimer() : 0;
  build_list_impl(c);
  const u64 t1 = (c.tid == 0) ? gtimer() : 0;
  filter_list_impl(c);
  if (c.tid == 0) {
    const u64 t2 = gtimer();
    c.R->t_build_ns += (double)(t2 - t0);
    c.R->t_filter_ns += (double)(t2 - t1);
  }
}
// Verlet rows only, filtered from the outer rows (valid while the outer list is)
__device__ void refresh_list(const Ctx& c) {
  const u64 t0 = (c.tid == 0) ? gtimer() : 0;
  filter_list_impl(c);
  if (c.tid == 0) {
    const double dt = (double)(gtimer() - t0);
    c.R->t_build_ns += dt;
    c.R->t_filter_ns += dt;
    c.R->refreshes++;
  }
}
// Each phase of the engine is a function of its own (not inlined), with the context copied
// to locals at entry: its loops get the whole register budget instead of sharing it with
// whatever the caller keeps live across the call.
__device__ H4D_PHASE void build_list_impl(const Ctx& cref) {
  const Ctx c = cref;
  const Eng& e = *c.e;
  const RepC& R = c.r;
  GView& v = const_cast<GView&>(c.v);
  const int n = v.s->n_tot;
  const int nc = R.nc;
  // rows of home atom i go to position lrank[i] when the last filter ranked these n atoms
  const bool use_rank = H4D_LANE_ORDER && e.lrank && !e.rows_by_index && n >= kOrderMin && v.s->n_rank == n;
  if (c.tid == 0) v.s->n_ord = 0;  // the cell sort below overwrites the shared copy of lord
  if (nc > 0) {
    const int ncell = nc * nc * nc;
    for (int k = c.tid; k < ncell; k += c.T) v.cfill[k] = 0;
    c.sync();
    for (int a = c.tid; a < n; a += c.T) atomicAdd(&v.cfill[cell_of_pos(v.pos[a], nc)], 1);
    c.sync();
    if (c.tid < 32) {  // exclusive scan over cells by warp 0
      int lane = c.tid;
      int carry = 0;
      for (int b = 0; b < ncell; b += 32) {
        int k = b + lane;
        int x = (k < ncell) ? ((v.cfill[k] + 3) & ~3) : 0;  // cells padded to 4 entries
        int incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          int y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        if (k < ncell) { v.cstart[k] = carry + incl - x; v.cfill[k] = carry + incl - x; }
        carry += __shfl_sync(0xffffffffu, incl, 31);
      }
      if (lane == 0) v.cstart[ncell] = carry;
      __syncwarp();
      for (int q = lane; q < carry; q += 32) v.sorted[q] = kNoAtom;
      __syncwarp();
      // stable scatter: atoms of a cell end up in ascending index order
      unsigned lt = (1u << lane) - 1u;
      for (int b = 0; b < n; b += 32) {
        int a = b + lane;
        int cc = (a < n) ? cell_of_pos(v.pos[a], nc) : -1 - lane;
        unsigned peers = __match_any_sync(0xffffffffu, cc);
        int rank = __popc(peers & lt);
        int base = (a < n) ? v.cfill[cc] : 0;
        __syncwarp();
        if (a < n) {
          v.sorted[base + rank] = (uint16_t)a;
          v.sorted8[base + rank] = pack8(v.pos[a]);
          if (rank == 0) v.cfill[cc] = base + __popc(peers);
        }
        __syncwarp();
      }
      // work items = (cell, 32-atom home pass); cfill becomes their exclusive prefix
      int carry2 = 0;
      for (int b = 0; b < ncell; b += 32) {
        int k = b + lane;
        int x = (k < ncell) ? (v.cstart[k + 1] - v.cstart[k] + 31) >> 5 : 0;
        int incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          int y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        if (k < ncell) v.cfill[k] = carry2 + incl - x;
        carry2 += __shfl_sync(0xffffffffu, incl, 31);
      }
      if (lane == 0) { v.s->n_items = carry2; v.s->next_item = 0; }
    }
    c.sync();
  }
  // Rows: one warp per cell, its lanes holding up to 32 home atoms of the cell at a time.
  // The candidates of the 27 stencil cells stream through the warp one at a time, so
  // every lane reads the same shared-memory word (broadcast, no bank conflicts); each lane
  // appends the accepted candidates to its own row.  Cells are visited in a fixed order
  // and hold their atoms in ascending index order, so a row does not depend on the thread
  // mapping.  Without cells (small boxes) every atom is a candidate of every atom.
  const int nwarps = c.T >> 5, warp = c.tid >> 5, lane = c.tid & 31;
  // without cells, "cell" k is the k-th chunk of 32 home atoms and every atom is a candidate
  const int ncell_rows = (nc > 0) ? nc * nc * nc : (n + 31) / 32;
  const int maxo = e.max_out;
  const bool has_water = R.nw3 > 0;  // uniform: the exclusion test only where waters exist
  int overflow = 0;
  // Work items are (cell, home pass of up to 32 atoms), handed out through a shared
  // counter so clustered (dense) cells do not leave one warp with all the work.  Without
  // cells, item k is the k-th chunk of 32 home atoms, assigned round-robin.
  for (int it = 0;; ++it) {
    int item;
    if (nc > 0) {
      if (lane == 0) item = atomicAdd(&v.s->next_item, 1);
      item = __shfl_sync(0xffffffffu, item, 0);
      if (item >= v.s->n_items) break;
    } else {
      item = warp + it * nwarps;
      if (item >= ncell_rows) break;
    }
    int cell = 0, pass = item;
    if (nc > 0) {  // last cell whose first item is <= item (binary search on the prefix)
      int lo = 0, hi = ncell_rows - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (v.cfill[mid] <= item) lo = mid; else hi = mid - 1;
      }
      cell = lo;
      pass = item - v.cfill[lo];
    }
    const int h0 = (nc > 0) ? v.cstart[cell] + 32 * pass : 32 * item;
    const int h1 = (nc > 0) ? min(h0 + 32, v.cstart[cell + 1]) : min(32 * item + 32, n);
    if (nc == 0) cell = 0;
    const int cx = (nc > 0) ? cell / (nc * nc) : 0;
    const int cy = (nc > 0) ? (cell / nc) % nc : 0;
    const int cz = (nc > 0) ? cell % nc : 0;
    for (int hb = h0; hb < h1; hb += 32) {
      const int hq = hb + lane;
      const int ih = (hq < h1) ? ((nc > 0) ? (int)v.sorted[hq] : hq) : (int)kNoAtom;
      const bool act = ih != (int)kNoAtom;
      const int i = act ? ih : 0;
      const int pos = use_rank ? (int)e.lrank[R.atom_off + i] : i;  // where this atom's rows go
      const uint4 pi = v.pos[i];
      const unsigned pi8 = pack8(pi);
      int cnt = 0;
      RowBuf rb;
      rb.init();
      const int nst = (nc > 0) ? 27 : 1;
      for (int d = 0; d < nst; ++d) {
        int s0 = 0, s1 = n;
        if (nc > 0) {
          int ex = cx + d / 9 - 1, ey = cy + (d / 3) % 3 - 1, ez = cz + d % 3 - 1;
          ex += (ex < 0) ? nc : 0; ex -= (ex >= nc) ? nc : 0;
          ey += (ey < 0) ? nc : 0; ey -= (ey >= nc) ? nc : 0;
          ez += (ez < 0) ? nc : 0; ez -= (ez >= nc) ? nc : 0;
          const int cc = (ex * nc + ey) * nc + ez;
          s0 = v.cstart[cc];
          s1 = v.cstart[cc + 1];
        }
        // Four candidates per iteration.  With cells: one 8-byte index load and one 16-byte
        // load of their packed 8-bit coordinates; the per-byte wrapping difference is the
        // minimum image at 8-bit resolution and __dp4a squares it (a conservative test:
        // the Verlet filter applies the exact criterion).  Without cells: 16-bit test.
        for (int q = s0; q < s1; q += 4) {
          int jj[4];
          bool near[4];
          if (nc > 0) {
            const uint2 w4 = *reinterpret_cast<const uint2*>(v.sorted + q);
            const uint4 c8 = *reinterpret_cast<const uint4*>(v.sorted8 + q);
            jj[0] = (int)(w4.x & 0xFFFFu); jj[1] = (int)(w4.x >> 16);
            jj[2] = (int)(w4.y & 0xFFFFu); jj[3] = (int)(w4.y >> 16);
            const unsigned cu[4] = {c8.x, c8.y, c8.z, c8.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int d = (int)__vsub4(pi8, cu[u]);
              near[u] = __dp4a(d, d, 0) <= (int)R.T8_out;
            }
          } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              jj[u] = (q + u < s1) ? q + u : (int)kNoAtom;
              near[u] = d2_16(pi, v.pos[jj[u] == kNoAtom ? i : jj[u]]) <= R.T16_out;
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = jj[u];
            const bool ok = act && near[u] && (j != (int)kNoAtom) && (j != i) &&
                            !(has_water && excluded_pair(i, j, R.nw3));
            rb.put_if(ok, j);
            cnt += ok ? 1 : 0;
            if (rb.n == 4) {
              if (cnt <= maxo)
                reinterpret_cast<uint2*>(e.nbr_out)[out_packet_index(e, R, pos, (cnt - 1) >> 2)] = rb.packet();
              rb.init();
            }
          }
        }
      }
      if (act) {
        if (rb.n > 0 && cnt <= maxo)  // last partial packet, padded with kNoAtom
          reinterpret_cast<uint2*>(e.nbr_out)[out_packet_index(e, R, pos, (cnt - 1) >> 2)] = rb.packet();
        if (cnt > maxo) { overflow = 1; cnt = maxo & ~3; }
        e.ncnt_out[R.atom_off + pos] = cnt;
        e.ref_out[R.atom_off + i] = pi;
        if (use_rank) e.lord[R.atom_off + pos] = (uint16_t)i;
      }
    }
  }
  if (overflow) atomicOr(&v.s->flag_overflow, 1);
  c.sync();
  if (c.tid == 0) {
    c.R->builds++;
    v.s->flag_rebuild = 0;
    v.s->n_lay = use_rank ? n : 0;
  }
  c.sync();
}

// Row layout.  An outer build stores atom i's outer row at position lrank[i] (ranks by
// descending Verlet-row length at the last filter) and records lord[k], the atom at
// position k; the filter reads outer rows and writes Verlet rows at the same positions, and
// the passes that walk the Verlet rows (forces, FP64 energies, pair counts) take positions
// k in order with atom ord[k] (lord copied to shared memory).  The lanes of a warp then
// read adjacent packets (coalesced) and hold rows of about the same length.  No result
// depends on the layout: each row is summed in its own slot order, per-atom results are
// stored by atom, and the kinetic sums are exact integers, so positions within a length
// bucket are taken with atomics.  The ranks live in global memory (the cell sort of the
// outer build reuses the shared buffers); replicas below kOrderMin atoms, callers without
// rank arrays and the neighbour-pair export keep rows by atom index.
__device__ __forceinline__ int order_bucket(int cnt) { return kOrderBuckets - 1 - min((cnt + 3) >> 2, kOrderBuckets - 1); }

// lrank for the next outer build from the Verlet-row lengths at positions k (atom lord[k]
// when lay, else k); the histogram uses sorted8, free outside the outer build
__device__ void next_rank(const Ctx& c, int n, bool lay) {
  const Eng& e = *c.e;
  const GView& v = c.v;
  const int off = c.r.atom_off;
  int* hist = reinterpret_cast<int*>(v.sorted8);
  for (int b = c.tid; b < kOrderBuckets; b += c.T) hist[b] = 0;
  c.sync();
  for (int k = c.tid; k < n; k += c.T) atomicAdd(&hist[order_bucket(e.ncnt[off + k])], 1);
  c.sync();
  if (c.tid < 32) {  // exclusive prefix over the buckets
    const int lane = c.tid;
    const int a = hist[lane], b = hist[lane + 32];
    int ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int ya = __shfl_up_sync(0xffffffffu, ia, o), yb = __shfl_up_sync(0xffffffffu, ib, o);
      if (lane >= o) { ia += ya; ib += yb; }
    }
    const int tot_a = __shfl_sync(0xffffffffu, ia, 31);
    hist[lane] = ia - a;
    hist[lane + 32] = tot_a + ib - b;
  }
  c.sync();
  for (int k = c.tid; k < n; k += c.T) {
    const int i = lay ? (int)e.lord[off + k] : k;
    e.lrank[off + i] = (uint16_t)atomicAdd(&hist[order_bucket(e.ncnt[off + k])], 1);
  }
  if (c.tid == 0) v.s->n_rank = n;
  c.sync();
}

// Verlet rows filtered from the outer rows: one thread per atom streams its outer row
// (one 8-byte packet load per four candidates) and keeps the candidates inside r_list, in
// outer-row order, so the Verlet rows are as deterministic as the outer ones.
__device__ H4D_PHASE void filter_list_impl(const Ctx& cref) {
  const Ctx c = cref;
  const Eng& e = *c.e;
  const RepC& R = c.r;
  const GView& v = c.v;
  const int n = v.s->n_tot;
  const int ltpa = c.ltpa;
  const int maxn = e.max_nbr;
  const uint2* pko = out_packets(e, R);
  const size_t ostride = (size_t)R.cap_atoms;
  int overflow = 0;
  // positions k of the outer rows' layout (atom lord[k], or k when rows are by index): the
  // outer rows are read and the Verlet rows written at the same position, both coalesced
  const bool lay = v.s->n_lay == n;
  for (int k = c.tid; k < n; k += c.T) {
    const int i = lay ? (int)e.lord[R.atom_off + k] : k;
    if (lay) v.sorted[k] = (uint16_t)i;
    const int pos = k;
    const uint4 pi = v.pos[i];
    const int cnt_out = e.ncnt_out[R.atom_off + pos];
    const int npk = (cnt_out + 3) >> 2;
    int cnt = 0;
    RowBuf rb;
    rb.init();
    uint2* nbr2 = reinterpret_cast<uint2*>(e.nbr);
    uint2 q = (npk > 0) ? pko[pos] : make_uint2(0xFFFFFFFFu, 0xFFFFFFFFu);
    for (int p = 0; p < npk; ++p) {
      const uint2 qn = (p + 1 < npk) ? pko[(size_t)(p + 1) * ostride + pos] : make_uint2(0xFFFFFFFFu, 0xFFFFFFFFu);
      if (H4D_PF_FILTER > 0 && p + H4D_PF_FILTER < npk) prefetch_l2(pko + (size_t)(p + H4D_PF_FILTER) * ostride + pos);
      const int jj[4] = {(int)(q.x & 0xFFFFu), (int)(q.x >> 16), (int)(q.y & 0xFFFFu), (int)(q.y >> 16)};
      uint4 pj[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) pj[u] = v.pos[jj[u] == kNoAtom ? i : jj[u]];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const bool ok = jj[u] != kNoAtom && fixed_d2(pi, pj[u]) <= R.T_list;
        rb.put_if(ok, jj[u]);
        cnt += ok ? 1 : 0;
        if (rb.n == 4) {
          if (cnt <= maxn) nbr2[packet_index(e, R, pos, (cnt - 1) >> 2, ltpa)] = rb.packet();
          rb.init();
        }
      }
      q = qn;
    }
    if (rb.n > 0 && cnt <= maxn) nbr2[packet_index(e, R, pos, (cnt - 1) >> 2, ltpa)] = rb.packet();
    if (cnt > maxn) { overflow = 1; cnt = maxn & ~3; }
    e.ncnt[R.atom_off + pos] = cnt;
    e.ref[R.atom_off + i] = pi;
  }
  if (overflow) atomicOr(&v.s->flag_overflow, 1);
  c.sync();
  if (c.tid == 0) v.s->n_ord = lay ? n : 0;
  // ranks for the next outer build from the row lengths just found
  if (H4D_LANE_ORDER && e.lrank && !e.rows_by_index && n >= kOrderMin) next_rank(c, n, lay);
  else c.sync();
}

// One atom's LJ-electrolyte row on this lane (packets p = 0, 1, ... of its share), four
// slots per packet, pair terms two at a time on the packed FP32x2 pipe.  Padding slots read
// the sentinel (its infinite altitude puts it beyond every cut-off), and the charge sign of
// a pair is the parity of i + j (cations even, anions odd): the same values as the generic
// loop, with neither a branch nor a table load per slot.  POLY selects the polynomial
// Coulomb form (pair_fr_lj2_poly) over the erfc form (pair_fr_lj2).
template <bool NEMD, bool POLY>
__device__ __forceinline__ void lj_row(const Pot& P, const uint4* __restrict__ pos, const uint2* pk, size_t pstride,
                                       int npk, uint2 q, unsigned capa, int i, const uint4& pi, float scale, float wi,
                                       bool wnz_i, float gscr, float& fx, float& fy, float& fz) {
  const unsigned kq_i = __float_as_uint(P.kq[0]) ^ ((unsigned)i << 31);
  for (int p = 0; p < npk; ++p) {
    const uint2 qn = (p + 1 < npk) ? pk[(size_t)(p + 1) * pstride] : make_uint2(0xFFFFFFFFu, 0xFFFFFFFFu);
    if (H4D_PF_FORCE > 0 && p + H4D_PF_FORCE < npk) prefetch_l2(pk + (size_t)(p + H4D_PF_FORCE) * pstride);
    const unsigned jw[4] = {q.x & 0xFFFFu, q.x >> 16, q.y & 0xFFFFu, q.y >> 16};
    uint4 pj[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) pj[u] = pos[min(jw[u], capa)];
#pragma unroll
    for (int h = 0; h < 4; h += 2) {  // slots h and h+1 on the packed FP32x2 pipe
      const float2 dx = __fmul2_rn(make_float2((float)(int)(pj[h].x - pi.x), (float)(int)(pj[h + 1].x - pi.x)), f2(scale));
      const float2 dy = __fmul2_rn(make_float2((float)(int)(pj[h].y - pi.y), (float)(int)(pj[h + 1].y - pi.y)), f2(scale));
      const float2 dz = __fmul2_rn(make_float2((float)(int)(pj[h].z - pi.z), (float)(int)(pj[h + 1].z - pi.z)), f2(scale));
      float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
      const float2 wj = make_float2(wbits(pj[h]), wbits(pj[h + 1]));  // 0, a flyer's altitude, or +inf
      float2 kqg = make_float2(__uint_as_float(kq_i ^ (jw[h] << 31)), __uint_as_float(kq_i ^ (jw[h + 1] << 31)));
      if (NEMD) {
        const float2 dw = __fadd2_rn(f2(wi), make_float2(-wj.x, -wj.y));
        r2 = __ffma2_rn(dw, dw, r2);
        // charge prefactor times the screening g of the generic loop (exact when g = 1)
        kqg.x = (wnz_i != (wj.x != 0.0f)) ? kqg.x * gscr : kqg.x;
        kqg.y = (wnz_i != (wj.y != 0.0f)) ? kqg.y * gscr : kqg.y;
      } else {
        r2 = __ffma2_rn(wj, wj, r2);  // + 0 for every atom, +inf for the sentinel
      }
      const float2 fr = POLY ? pair_fr_lj2_poly(P, r2, kqg) : pair_fr_lj2(P, r2, kqg);
      // the force sums in slot order, as in the generic loop
      fx = fmaf(-fr.x, dx.x, fx);
      fy = fmaf(-fr.x, dy.x, fy);
      fz = fmaf(-fr.x, dz.x, fz);
      fx = fmaf(-fr.y, dx.y, fx);
      fy = fmaf(-fr.y, dy.y, fy);
      fz = fmaf(-fr.y, dz.y, fz);
    }
    q = qn;
  }
}

// ------------------------------------------------------------------------------------
// Force pass (FP32): tpa lanes per atom over its full row, butterfly reduction.
// mode bits: 1 = apply the second half kick, 2 = accumulate kinetic partials,
//            4 = flyer rows compute protocol work with previous altitude w_prev
// ------------------------------------------------------------------------------------
template <int SYS, bool NEMD>
__device__ H4D_PHASE void force_pass_impl(const Ctx& cref, int mode, float w_prev, double* kin_out);
// mode bits: 1 = apply the second half kick, 2 = return the kinetic energy after it,
//            4 = flyer rows accumulate the protocol work between w_prev and the current w.
// NEMD = false assumes every altitude is zero (equilibrium MD).
template <int SYS, bool NEMD = true>
__device__ void force_pass(const Ctx& c, int mode, float w_prev, double* kin_out) {
  const u64 t0 = (c.tid == 0) ? gtimer() : 0;
  force_pass_impl<SYS, NEMD>(c, mode, w_prev, kin_out);
  if (c.tid == 0) c.R->t_force_ns += (double)(gtimer() - t0);
}

template <int SYS, bool NEMD>
__device__ H4D_PHASE void force_pass_impl(const Ctx& cref, int mode, float w_prev, double* kin_out) {
  const Ctx c = cref;
  const Eng& e = *c.e;
  const RepC& R = c.r;
  const Pot& P = e.pot;
  const GView& v = c.v;
  const int n = v.s->n_tot;
  const int tpa = c.tpa, ltpa = c.ltpa;
  const int nsub = c.T >> ltpa;
  const int sub = c.tid >> ltpa, lin = c.tid & (tpa - 1);
  const int fly0 = NEMD ? v.s->fly0 : -1, fly1 = NEMD ? v.s->fly1 : -1, fly2 = NEMD ? v.s->fly2 : -1;
  const float gscr = NEMD ? v.s->g_scr : 1.0f;
  const float scale = R.scale;
  const float half_dt = 0.5f * (float)e.proto.dt;
  const uint2* packets = nbr_packets(e, R);
  const size_t pstride = (size_t)R.cap_atoms << ltpa;
  long long kin = 0;  // m v^2 of this thread's atoms, fixed point (exact, order-free sum)
  int kbad = 0;
  // row positions k in order, atom ord[k] (the layout of the last list pass)
  const bool use_ord = v.s->n_ord == n;
  for (int a0 = 0; a0 < n; a0 += nsub) {
    const int k = a0 + sub;
    const bool active = k < n;
    const int i = (use_ord && active) ? (int)v.sorted[k] : k;
    float fx = 0.f, fy = 0.f, fz = 0.f, dwk = 0.f;
    // aqueous: the per-atom force is a sum of hundreds of large, cancelling Coulomb
    // terms, so it is accumulated with Kahan compensation (cx, cy, cz)
    float cx = 0.f, cy = 0.f, cz = 0.f;
    const bool iflyer = NEMD && active && (i == fly0 || i == fly1 || i == fly2);
    if (active) {
      if ((mode & 1) && lin == 0) {  // the half kick after the row reads this atom's velocity
        prefetch_l1(e.vhi + R.atom_off + i);
        prefetch_l1(e.vlo + R.atom_off + i);
      }
      const uint4 pi = v.pos[i];
      const int ti = type_t<SYS>(i, R.nw3);
      const float wi = NEMD ? wbits(pi) : 0.0f;
      const bool wnz_i = wi != 0.0f;
      const int cnt = e.ncnt[R.atom_off + k];
      const uint2* pk = packets + ((size_t)k << ltpa) + lin;
      const int nP = (cnt + 3) >> 2;  // packets of the row; this lane owns lin, lin+tpa, ...
      const int npk = (nP > lin) ? (nP - lin + tpa - 1) >> ltpa : 0;
      uint2 q = (npk > 0) ? pk[0] : make_uint2(0xFFFFFFFFu, 0xFFFFFFFFu);
      if (SYS == H4D_SYS_LJ) {
        if (P.coul_poly)
          lj_row<NEMD, true>(P, v.pos, pk, pstride, npk, q, (unsigned)R.cap_atoms, i, pi, scale, wi, wnz_i, gscr, fx, fy, fz);
        else
          lj_row<NEMD, false>(P, v.pos, pk, pstride, npk, q, (unsigned)R.cap_atoms, i, pi, scale, wi, wnz_i, gscr, fx, fy, fz);
      } else
      for (int p = 0; p < npk; ++p) {
        const uint2 qn = (p + 1 < npk) ? pk[(size_t)(p + 1) * pstride] : make_uint2(0xFFFFFFFFu, 0xFFFFFFFFu);
        const int jj[4] = {(int)(q.x & 0xFFFFu), (int)(q.x >> 16), (int)(q.y & 0xFFFFu), (int)(q.y >> 16)};
        // branch-free over the four slots: a padding slot reads atom i and gets r^2 = 1e30,
        // for which every term of the pair function is exactly zero
        uint4 pj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) pj[u] = v.pos[jj[u] == kNoAtom ? i : jj[u]];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const bool valid = jj[u] != kNoAtom;
          const float dx = (float)(int)(pj[u].x - pi.x) * scale;
          const float dy = (float)(int)(pj[u].y - pi.y) * scale;
          const float dz = (float)(int)(pj[u].z - pi.z) * scale;
          float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          float g = 1.0f;
          if (NEMD) {
            const float wj = wbits(pj[u]);
            const float dw = wi - wj;
            r2 = fmaf(dw, dw, r2);
            g = (wnz_i != (wj != 0.0f)) ? gscr : 1.0f;
          }
          r2 = valid ? r2 : 1.0e30f;
          const PairCoef<SYS> cf = coef<SYS>(P, ti, type_t<SYS>(jj[u] & 0x7FFF, R.nw3));
          const float fr = pair_fr<SYS>(P, cf, r2, g);
          if (SYS == H4D_SYS_AQ) {
            const float tx = -fr * dx - cx, ty = -fr * dy - cy, tz = -fr * dz - cz;
            const float sx = fx + tx, sy = fy + ty, sz = fz + tz;
            cx = (sx - fx) - tx;
            cy = (sy - fy) - ty;
            cz = (sz - fz) - tz;
            fx = sx;
            fy = sy;
            fz = sz;
          } else {
            fx = fmaf(-fr, dx, fx);
            fy = fmaf(-fr, dy, fy);
            fz = fmaf(-fr, dz, fz);
          }
        }
        q = qn;
      }
      if (NEMD && (mode & 4) && iflyer) {
        // protocol work of a flying row: U(w_now) - U(w_prev) against every non-flyer
        // the anion flies rw times higher; screening uses the mean flyer altitude
        const float rw = (float)e.proto.rw;
        const float wp_i = (i == fly1) ? rw * w_prev : w_prev;
        const float go = __expf(-P.kappa_sr * (0.5f * (1.0f + rw) * w_prev));
        for (int s2 = lin; s2 < cnt; s2 += tpa) {
          const int j = e.nbr[nbr_index(e, R, k, s2, ltpa)];
          if (j == fly0 || j == fly1 || j == fly2) continue;
          const uint4 pj = v.pos[j];
          const float dx = (float)(int)(pj.x - pi.x) * scale;
          const float dy = (float)(int)(pj.y - pi.y) * scale;
          const float dz = (float)(int)(pj.z - pi.z) * scale;
          const float r3 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          const float r2n = fmaf(wi, wi, r3);
          const float r2o = fmaf(wp_i, wp_i, r3);
          const PairCoef<SYS> cf = coef<SYS>(P, ti, type_t<SYS>(j, R.nw3));
          const float un = (r2n < P.rc2_max) ? pair_u32<SYS>(P, cf, r2n, gscr) : 0.0f;
          const float uo = (r2o < P.rc2_max) ? pair_u32<SYS>(P, cf, r2o, go) : 0.0f;
          dwk += un - uo;
        }
      }
    }
    if (SYS == H4D_SYS_AQ) {
      fx -= cx;
      fy -= cy;
      fz -= cz;
    }
    for (int o = tpa >> 1; o > 0; o >>= 1) {
      fx += __shfl_xor_sync(0xffffffffu, fx, o, tpa);
      fy += __shfl_xor_sync(0xffffffffu, fy, o, tpa);
      fz += __shfl_xor_sync(0xffffffffu, fz, o, tpa);
      if (NEMD) dwk += __shfl_xor_sync(0xffffffffu, dwk, o, tpa);
    }
    if (active && lin == 0) {
      const int ga = R.atom_off + i;
      e.force[ga] = make_float4(fx, fy, fz, 0.f);
      if (NEMD && (mode & 4) && iflyer) v.s->dW[i == fly0 ? 0 : (i == fly1 ? 1 : 2)] = (double)dwk;
      if (!iflyer && (mode & 3)) {
        float4 h = e.vhi[ga], l = e.vlo[ga];
        const int ti = type_t<SYS>(i, R.nw3);
        if (mode & 1) {
          const float cm = half_dt * P.inv_m[ti];
          ff_add(h.x, l.x, fx * cm);
          ff_add(h.y, l.y, fy * cm);
          ff_add(h.z, l.z, fz * cm);
          e.vhi[ga] = h;
          e.vlo[ga] = l;
        }
        if (mode & 2) {
          const float vx = h.x + l.x, vy = h.y + l.y, vz = h.z + l.z;
          kin += to_fx(P.m_f[ti] * fmaf(vx, vx, fmaf(vy, vy, vz * vz)), kbad);
        }
      }
    }
  }
  if (mode & 2) {
    if (kbad) v.s->flag_nan = 1;
    *kin_out = 0.5 * (double)group_sum_fx(c, kin) / (double)kFxScale;
  }
}

// ------------------------------------------------------------------------------------
// Kick + drift pass: optional thermostat scale, half kick, fixed-point drift, move check
// ------------------------------------------------------------------------------------
// Rigid water, position stage of RATTLE (SHAKE): half kick of the three atoms, an
// unconstrained drift, then pairwise corrections along the previous bond vectors until
// O-H, O-H and H-H hold (the same impulses correct the half-step velocities).  Works in
// FP32 coordinates relative to the old O position, taken from exact fixed-point
// differences; the constrained displacements are added back in fixed point.
__device__ __forceinline__ void top2(float d, float& a, float& b) {
  if (d > a) { b = a; a = d; } else if (d > b) { b = d; }
}
__device__ void water_kick_drift(const Ctx& c, int m, float alpha, float& d1, float& d2, float& o1, float& o2,
                                 int& bad) {
  const Eng& e = *c.e;
  const RepC& R = c.r;
  const Pot& P = e.pot;
  const GView& v = c.v;
  const float h = (float)e.proto.dt;
  const float imv[3] = {P.inv_m[2], P.inv_m[3], P.inv_m[3]};  // 1/(m mvv2e): O, H, H
  const float mw[3] = {1.0f / P.inv_m[2], 1.0f / P.inv_m[3], 1.0f / P.inv_m[3]};
  float4 vh[3], vl[3];
  uint4 po[3];
  float x[3][3], ro[3][3];
  const int a0 = 3 * m;
  for (int k = 0; k < 3; ++k) {
    const int ga = R.atom_off + a0 + k;
    vh[k] = e.vhi[ga];
    vl[k] = e.vlo[ga];
    if (alpha != 1.0f) {
      ff_scale(vh[k].x, vl[k].x, alpha);
      ff_scale(vh[k].y, vl[k].y, alpha);
      ff_scale(vh[k].z, vl[k].z, alpha);
    }
    const float4 f = e.force[ga];
    const float cm = 0.5f * h * imv[k];
    ff_add(vh[k].x, vl[k].x, f.x * cm);
    ff_add(vh[k].y, vl[k].y, f.y * cm);
    ff_add(vh[k].z, vl[k].z, f.z * cm);
    po[k] = v.pos[a0 + k];
  }
  // old positions relative to the old O; unconstrained new positions
  for (int k = 0; k < 3; ++k) {
    ro[k][0] = (float)(int)(po[k].x - po[0].x) * R.scale;
    ro[k][1] = (float)(int)(po[k].y - po[0].y) * R.scale;
    ro[k][2] = (float)(int)(po[k].z - po[0].z) * R.scale;
    x[k][0] = ro[k][0] + (vh[k].x + vl[k].x) * h;
    x[k][1] = ro[k][1] + (vh[k].y + vl[k].y) * h;
    x[k][2] = ro[k][2] + (vh[k].z + vl[k].z) * h;
  }
  const int ca[3] = {0, 0, 1}, cb[3] = {1, 2, 2};
  const float dd[3] = {(float)P.d_oh2, (float)P.d_oh2, (float)P.d_hh2};
  float dv[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  // iterate to the tolerance (2e-7, near the FP32 floor); 100 iterations that end with a
  // violation above 1e-3 (or a non-finite one) mean the bonds could not be restored
  bool converged = false;
  float worst = 0.f;
  for (int it = 0; it < 100 && !converged; ++it) {
    worst = 0.f;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int a = ca[q], b = cb[q];
      float rn[3], rr[3], rn2 = 0.f, dot = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        rn[k] = x[a][k] - x[b][k];
        rr[k] = ro[a][k] - ro[b][k];
        rn2 = fmaf(rn[k], rn[k], rn2);
        dot = fmaf(rn[k], rr[k], dot);
      }
      const float diff = rn2 - dd[q];
      worst = fmaxf(worst, fabsf(diff) / dd[q]);
      const float g = diff / (2.0f * dot * (1.0f / mw[a] + 1.0f / mw[b]));
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float da = -g * rr[k] / mw[a], db = g * rr[k] / mw[b];
        x[a][k] += da;
        x[b][k] += db;
        dv[a][k] += da;
        dv[b][k] += db;
      }
    }
    converged = worst < 2e-7f;
  }
  if (!(worst < 1e-3f)) v.s->flag_timeout = 1;
  for (int k = 0; k < 3; ++k) {
    const int ga = R.atom_off + a0 + k;
    ff_add(vh[k].x, vl[k].x, dv[k][0] / h);
    ff_add(vh[k].y, vl[k].y, dv[k][1] / h);
    ff_add(vh[k].z, vl[k].z, dv[k][2] / h);
    e.vhi[ga] = vh[k];
    e.vlo[ga] = vl[k];
    const float sx = (x[k][0] - ro[k][0]) / R.scale, sy = (x[k][1] - ro[k][1]) / R.scale,
                sz = (x[k][2] - ro[k][2]) / R.scale;
    if (!(fabsf(sx) < 1.0e9f && fabsf(sy) < 1.0e9f && fabsf(sz) < 1.0e9f)) { bad = 1; continue; }
    uint4 p = po[k];
    p.x += (unsigned)__float2int_rn(sx);
    p.y += (unsigned)__float2int_rn(sy);
    p.z += (unsigned)__float2int_rn(sz);
    v.pos[a0 + k] = p;
    top2(sqrtf((float)fixed_d2(p, e.ref[ga])), d1, d2);
    top2(sqrtf((float)fixed_d2(p, e.ref_out[ga])), o1, o2);
  }
}

// Rigid water, velocity stage of RATTLE: remove the bond-parallel relative velocities;
// returns the kinetic energy of all atoms when want_k (after the projection)
__device__ double rattle_pass(const Ctx& c, bool want_k) {
  const Eng& e = *c.e;
  const RepC& R = c.r;
  const Pot& P = e.pot;
  const GView& v = c.v;
  const int n = v.s->n_tot;
  const int fly0 = v.s->fly0, fly1 = v.s->fly1;
  const float imv[3] = {P.inv_m[2], P.inv_m[3], P.inv_m[3]};
  const int ca[3] = {0, 0, 1}, cb[3] = {1, 2, 2};
  const float dd[3] = {(float)P.d_oh2, (float)P.d_oh2, (float)P.d_hh2};
  long long kin = 0;  // kinetic energy, fixed point (exact, order-free sum)
  int kbad = 0;
  const int flyw = v.s->flyw;
  for (int m = c.tid; m < R.n_water; m += c.T) {
    if (m == flyw) continue;  // frozen: its held velocities stay as drawn
    const int a0 = 3 * m;
    float4 vh[3], vl[3];
    uint4 po[3];
    float r[3][3], vv[3][3], dv[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    for (int k = 0; k < 3; ++k) {
      const int ga = R.atom_off + a0 + k;
      vh[k] = e.vhi[ga];
      vl[k] = e.vlo[ga];
      po[k] = v.pos[a0 + k];
      vv[k][0] = vh[k].x + vl[k].x;
      vv[k][1] = vh[k].y + vl[k].y;
      vv[k][2] = vh[k].z + vl[k].z;
    }
    for (int k = 0; k < 3; ++k) {
      r[k][0] = (float)(int)(po[k].x - po[0].x) * R.scale;
      r[k][1] = (float)(int)(po[k].y - po[0].y) * R.scale;
      r[k][2] = (float)(int)(po[k].z - po[0].z) * R.scale;
    }
    float worst = 0.f;
    for (int it = 0; it < 100; ++it) {
      worst = 0.f;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int a = ca[q], b = cb[q];
        float rab[3], dvv = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          rab[k] = r[a][k] - r[b][k];
          dvv = fmaf(rab[k], (vv[a][k] + dv[a][k]) - (vv[b][k] + dv[b][k]), dvv);
        }
        worst = fmaxf(worst, fabsf(dvv) / dd[q]);
        const float kk = dvv / (dd[q] * (imv[a] + imv[b]));
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          dv[a][k] -= kk * imv[a] * rab[k];
          dv[b][k] += kk * imv[b] * rab[k];
        }
      }
      if (worst < 1e-7f) break;
    }
    // the tolerance sits near the FP32 floor; a violation still above 1e-3 (or a non-finite
    // one) after 100 iterations means the velocities could not be made consistent
    if (!(worst < 1e-3f)) v.s->flag_timeout = 1;
    for (int k = 0; k < 3; ++k) {
      const int ga = R.atom_off + a0 + k;
      ff_add(vh[k].x, vl[k].x, dv[k][0]);
      ff_add(vh[k].y, vl[k].y, dv[k][1]);
      ff_add(vh[k].z, vl[k].z, dv[k][2]);
      e.vhi[ga] = vh[k];
      e.vlo[ga] = vl[k];
      if (want_k) {
        const float x = vh[k].x + vl[k].x, y = vh[k].y + vl[k].y, z = vh[k].z + vl[k].z;
        kin += to_fx(0.5f * (1.0f / imv[k]) * fmaf(x, x, fmaf(y, y, z * z)), kbad);
      }
    }
  }
  if (!want_k) return 0.0;
  for (int a = R.nw3 + c.tid; a < n; a += c.T) {
    if (a == fly0 || a == fly1) continue;
    const int ga = R.atom_off + a;
    const float4 h = e.vhi[ga], l = e.vlo[ga];
    const float x = h.x + l.x, y = h.y + l.y, z = h.z + l.z;
    kin += to_fx(0.5f * P.m_f[type_of(a, R.nw3)] * fmaf(x, x, fmaf(y, y, z * z)), kbad);
  }
  if (kbad) v.s->flag_nan = 1;
  return (double)group_sum_fx(c, kin) / (double)kFxScale;
}

template <int SYS>
__device__ H4D_PHASE void kick_drift(const Ctx& cref, float alpha) {
  const Ctx c = cref;
  const Eng& e = *c.e;
  const RepC& R = c.r;
  const Pot& P = e.pot;
  const GView& v = c.v;
  const int n = v.s->n_tot;
  const int fly0 = v.s->fly0, fly1 = v.s->fly1;
  const float half_dt = 0.5f * (float)e.proto.dt;
  int bad = 0;
  float d1 = 0.f, d2 = 0.f;  // this thread's two largest displacements (Verlet list)
  float o1 = 0.f, o2 = 0.f;  // the same against the outer-list reference
  const int n_units = R.n_water + (n - R.nw3);  // rigid waters first, then ions
  const int flyw = v.s->flyw;  // a flying water is frozen in 3D like a flying ion
  for (int u = c.tid; u < n_units; u += c.T) {
    if (SYS == H4D_SYS_AQ && u < R.n_water) {
      if (u != flyw) water_kick_drift(c, u, alpha, d1, d2, o1, o2, bad);
      continue;
    }
    const int a = R.nw3 + (u - R.n_water);
    if (a == fly0 || a == fly1) continue;  // flyers keep their 3D state (Sec. II.B.1)
    const int ga = R.atom_off + a;
    float4 h = e.vhi[ga], l = e.vlo[ga];
    if (alpha != 1.0f) {
      ff_scale(h.x, l.x, alpha);
      ff_scale(h.y, l.y, alpha);
      ff_scale(h.z, l.z, alpha);
    }
    const float4 f = e.force[ga];
    const float cm = half_dt * P.inv_m[type_of(a, R.nw3)];
    ff_add(h.x, l.x, f.x * cm);
    ff_add(h.y, l.y, f.y * cm);
    ff_add(h.z, l.z, f.z * cm);
    e.vhi[ga] = h;
    e.vlo[ga] = l;
    const float sx = fmaf(h.x, R.c_drift, l.x * R.c_drift);
    const float sy = fmaf(h.y, R.c_drift, l.y * R.c_drift);
    const float sz = fmaf(h.z, R.c_drift, l.z * R.c_drift);
    const float lim = 1.0e9f;
    if (!(fabsf(sx) < lim && fabsf(sy) < lim && fabsf(sz) < lim)) { bad = 1; continue; }
    uint4 p = v.pos[a];
    p.x += (unsigned)__float2int_rn(sx);
    p.y += (unsigned)__float2int_rn(sy);
    p.z += (unsigned)__float2int_rn(sz);
    v.pos[a] = p;
    top2(sqrtf((float)fixed_d2(p, e.ref[ga])), d1, d2);
    top2(sqrtf((float)fixed_d2(p, e.ref_out[ga])), o1, o2);
  }
  // A list stays valid while the two largest displacements since its build sum to less
  // than its skin (no pair distance can have shrunk by more).  Warp-level top-2 merges;
  // every thread folds the warp slots after the next barrier (maybe_rebuild).
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float b1 = __shfl_xor_sync(0xffffffffu, d1, o), b2 = __shfl_xor_sync(0xffffffffu, d2, o);
    const float hi = fmaxf(d1, b1);
    d2 = fmaxf(fminf(d1, b1), fmaxf(d2, b2));
    d1 = hi;
    const float c1 = __shfl_xor_sync(0xffffffffu, o1, o), c2 = __shfl_xor_sync(0xffffffffu, o2, o);
    const float hj = fmaxf(o1, c1);
    o2 = fmaxf(fminf(o1, c1), fmaxf(o2, c2));
    o1 = hj;
  }
  if ((c.tid & 31) == 0) {
    v.s->d1w[c.tid >> 5] = d1;
    v.s->d2w[c.tid >> 5] = d2;
    v.s->o1w[c.tid >> 5] = o1;
    v.s->o2w[c.tid >> 5] = o2;
  }
  if (bad) v.s->flag_nan = 1;
}

// after the barrier that follows kick_drift: fold the warp slots (same answer in every
// thread) and, when the Verlet rows are stale, refresh them from the outer rows or, when
// those cannot cover the Verlet radius any more, rebuild both
__device__ __forceinline__ void fold_top2(const float* a1, const float* a2, int nw, float& d1, float& d2) {
  d1 = 0.f;
  d2 = 0.f;
  for (int w = 0; w < nw; ++w) {
    const float hi = fmaxf(d1, a1[w]);
    d2 = fmaxf(fminf(d1, a1[w]), fmaxf(d2, a2[w]));
    d1 = hi;
  }
}
__device__ void build_list(const Ctx& c);
__device__ void refresh_list(const Ctx& c);
__device__ void maybe_rebuild(const Ctx& c) {
  float d1, d2, o1, o2;
  fold_top2(c.v.s->d1w, c.v.s->d2w, c.T >> 5, d1, d2);
  fold_top2(c.v.s->o1w, c.v.s->o2w, c.T >> 5, o1, o2);
  // The Verlet rows are refreshed from the outer rows, which hold every pair within the
  // outer radius at the outer build.  A pair now within the Verlet radius was then within
  // it plus o1 + o2, so the outer rows are complete only while o1 + o2 <= skin_out - skin;
  // past that the refresh rebuilds everything.
  if (d1 + d2 > c.r.skin_fx) {
    if (o1 + o2 > c.r.skin_out_fx - c.r.skin_fx) build_list(c);
    else refresh_list(c);
  }
}

__device__ void scale_velocities(const Ctx& c, float alpha) {
  const Eng& e = *c.e;
  const RepC& R = c.r;
  const int n = c.v.s->n_tot;
  for (int a = c.tid; a < n; a += c.T) {
    const int ga = R.atom_off + a;
    float4 h = e.vhi[ga], l = e.vlo[ga];
    ff_scale(h.x, l.x, alpha);
    ff_scale(h.y, l.y, alpha);
    ff_scale(h.z, l.z, alpha);
    e.vhi[ga] = h;
    e.vlo[ga] = l;
  }
}

__device__ void negate_velocities(const Ctx& c, int n) {
  const Eng& e = *c.e;
  const RepC& R = c.r;
  for (int a = c.tid; a < n; a += c.T) {
    const int ga = R.atom_off + a;
    float4 h = e.vhi[ga], l = e.vlo[ga];
    h.x = -h.x; h.y = -h.y; h.z = -h.z;
    l.x = -l.x; l.y = -l.y; l.z = -l.z;
    e.vhi[ga] = h;
    e.vlo[ga] = l;
  }
}

// ------------------------------------------------------------------------------------
// FP64 end-point energies
// ------------------------------------------------------------------------------------
// U over atoms [0, n_tot) leaving out ex0/ex1/ex2 (-1 = none); each unordered pair once
__device__ H4D_PHASE double energy64_impl(const Ctx& cref, int ex0, int ex1, int ex2);
__device__ double energy64(const Ctx& c, int ex0, int ex1, int ex2 = -1) {
  const u64 t0 = (c.tid == 0) ? gtimer() : 0;
  const double u = energy64_impl(c, ex0, ex1, ex2);
  if (c.tid == 0) c.R->t_energy_ns += (double)(gtimer() - t0);
  return u;
}
__device__ H4D_PHASE double energy64_impl(const Ctx& cref, int ex0, int ex1, int ex2) {
  const Ctx c = cref;
  const Eng& e = *c.e;
  const RepC& R = c.r;
  const Pot& P = e.pot;
  const GView& v = c.v;
  const int n = v.s->n_tot;
  const double scale = R.L * 0x1.0p-32;
  const double gscr = exp(-P.dkappa_sr * (double)v.s->w_cur);
  const double rc2max = P.drc2_lj > P.drc2_c ? P.drc2_lj : P.drc2_c;
  // per-atom Kahan sums over the row (j > i), then a sum over atoms in a fixed order;
  // rows are taken by position k (atom ord[k])
  const bool use_ord = v.s->n_ord == n;
  for (int k = c.tid; k < n; k += c.T) {
    const int i = use_ord ? (int)v.sorted[k] : k;
    double acc = 0.0, comp = 0.0;
    if (i == ex0 || i == ex1 || i == ex2) {
      e.red[R.atom_off + i] = 0.0;
      continue;
    }
    const uint4 pi = v.pos[i];
    const int ti = type_of(i, R.nw3);
    const double wi = (double)wbits(pi);
    const int cnt = e.ncnt[R.atom_off + k];
    for (int s = 0; s < cnt; ++s) {
      const int j = e.nbr[nbr_index(e, R, k, s, c.ltpa)];
      if (j <= i || j == ex0 || j == ex1 || j == ex2) continue;
      const uint4 pj = v.pos[j];
      const double dx = (double)(int)(pj.x - pi.x) * scale;
      const double dy = (double)(int)(pj.y - pi.y) * scale;
      const double dz = (double)(int)(pj.z - pi.z) * scale;
      const double wj = (double)wbits(pj);
      const double dw = wi - wj;
      const double r2 = dx * dx + dy * dy + dz * dz + dw * dw;
      if (r2 >= rc2max) continue;
      const double g = ((wi != 0.0) != (wj != 0.0)) ? gscr : 1.0;
      const double y = pair_u64(P, ti, type_of(j, R.nw3), r2, g) - comp;
      const double t = acc + y;
      comp = (t - acc) - y;
      acc = t;
    }
    e.red[R.atom_off + i] = acc;
  }
  return fixed_order_sum(c, e.red + R.atom_off, n);
}

__device__ double kinetic64(const Ctx& c) {
  const Eng& e = *c.e;
  const RepC& R = c.r;
  const int n = c.v.s->n_tot;
  const int fly0 = c.v.s->fly0, fly1 = c.v.s->fly1, fly2 = c.v.s->fly2;
  for (int a = c.tid; a < n; a += c.T) {
    const int ga = R.atom_off + a;
    if (a == fly0 || a == fly1 || a == fly2) {
      e.red[ga] = 0.0;
      continue;
    }
    const float4 h = e.vhi[ga], l = e.vlo[ga];
    const double vx = (double)h.x + (double)l.x, vy = (double)h.y + (double)l.y,
                 vz = (double)h.z + (double)l.z;
    e.red[ga] = 0.5 * e.pot.dm[type_of(a, R.nw3)] * (vx * vx + vy * vy + vz * vz);
  }
  return fixed_order_sum(c, e.red + R.atom_off, n);
}

// ------------------------------------------------------------------------------------
// Thermostat (equilibrium MD only): CSVR (Bussi, Donadio, Parrinello 2007, Eq. A7) with
// the chi-square variate from the Marsaglia-Tsang gamma sampler (ACM TOMS 2000).
// ------------------------------------------------------------------------------------
__device__ double chi2_variate(const Eng& e, const Rep& R, u64 rep_id, u64 step, double dof, int* timed_out) {
  double k = 0.5 * dof;
  if (k <= 0.0) return 0.0;
  const double k0 = k;
  if (k < 1.0) k += 1.0;
  const double d = k - 1.0 / 3.0, cc = 1.0 / sqrt(9.0 * d);
  double g = d, boost = 1.0;
  bool done = false;
  for (u64 attempt = 0; attempt < 4096 && !done; ++attempt) {
    u64 r[4];
    draw4(e.seed, rep_id, step, attempt, kPurGamma, r);
    const double z = gauss_c(r[0], r[1]);
    double t = 1.0 + cc * z;
    if (t <= 0.0) continue;
    t = t * t * t;
    const double u = u01_open(r[2]);
    if (log(u) < 0.5 * z * z + d - d * t + d * log(t)) {
      g = d * t;
      if (k0 < 1.0) boost = pow(u01_open(r[3]), 1.0 / k0);
      done = true;
    }
  }
  if (!done) *timed_out = 1;  // 4096 rejections in a row: reported, the mean is used
  return 2.0 * g * boost;
}

__device__ double csvr_alpha(const Eng& e, const Rep& R, u64 rep_id, u64 step, double K, int n, int* timed_out) {
  const double dof = 3.0 * n - 3.0 * R.n_water;
  if (dof < 1.0 || e.proto.tau_t <= 0.0 || K <= 0.0) return 1.0;
  const double Kbar = 0.5 * dof / e.proto.beta;
  const double cdec = exp(-e.proto.dt / e.proto.tau_t);
  u64 r[4];
  draw4(e.seed, rep_id, step, 0, kPurThermo, r);
  const double R1 = gauss_c(r[0], r[1]);
  const double S = chi2_variate(e, R, rep_id, step, dof - 1.0, timed_out);
  const double Knew = K + (1.0 - cdec) * (Kbar * (S + R1 * R1) / dof - K) +
                      2.0 * R1 * sqrt(Kbar * K * (1.0 - cdec) * cdec / dof);
  double a = sqrt(Knew / K);
  if (R1 + sqrt(dof * K * cdec / (Kbar * (1.0 - cdec))) < 0.0) a = -a;
  return a;
}

// ------------------------------------------------------------------------------------
// Protocol: altitude at NEMD step k (Eq. 2; Eqs. S6-S7 insertion forms; deletion is the
// time reverse of insertion)
// ------------------------------------------------------------------------------------
__device__ double altitude(const Proto& pr, int insertion, int k) {
  const int kk = insertion ? k : pr.n_f - k;
  const double xi = (double)kk / (double)pr.n_f;
  double s;
  if (pr.schedule == H4D_SCHED_WV) s = 1.0 - pow(xi, pr.sched_n);
  else if (pr.schedule == H4D_SCHED_WX) s = pow(1.0 - xi, pr.sched_n);
  else s = 1.0 - xi;
  return pr.w_max * s;
}

// ------------------------------------------------------------------------------------
// Phases
// ------------------------------------------------------------------------------------
template <int SYS>
__device__ void initial_forces(const Ctx& c) {
  build_list(c);
  force_pass<SYS, false>(c, 0, 0.f, nullptr);
  c.sync();
}

// equilibrium MD: n_steps velocity-Verlet steps at w = 0 with the CSVR thermostat
template <int SYS>
__device__ H4D_PHASE float md_steps(const Ctx& cref, int n_steps);

template <int SYS>
__device__ void md_phase(const Ctx& c, int n_steps) {
  const Eng& e = *c.e;
  Rep& R = *c.R;
  GScal* S = c.v.s;
  if (c.tid == 0) { S->flag_nan = 0; S->flag_timeout = 0; }
  initial_forces<SYS>(c);
  const float alpha = md_steps<SYS>(c, n_steps);
  if (alpha != 1.0f) scale_velocities(c, alpha);
  c.sync();
  if (c.tid == 0 && S->flag_nan) R.err |= 2;
  if (c.tid == 0 && S->flag_overflow) R.err |= 1;
  if (c.tid == 0 && S->flag_timeout) R.err |= 4;
}

// equilibrium MD steps with the CSVR thermostat, out of line like the NEMD loop; returns
// the last thermostat factor (applied by the caller)
template <int SYS>
__device__ H4D_PHASE float md_steps(const Ctx& cref, int n_steps) {
  const Ctx c = cref;
  const Eng& e = *c.e;
  Rep& R = *c.R;
  GScal* S = c.v.s;
  float alpha = 1.0f;
  for (int st = 0; st < n_steps; ++st) {
    kick_drift<SYS>(c, alpha);
    c.sync();
    maybe_rebuild(c);
    double K = 0.0;
    if (SYS == H4D_SYS_AQ && c.r.n_water > 0) {
      force_pass<SYS, false>(c, 1, 0.f, nullptr);
      c.sync();
      K = rattle_pass(c, true);  // ends with group syncs
    } else {
      force_pass<SYS, false>(c, 1 | 2, 0.f, &K);  // ends with group syncs
    }
    if (c.tid == 0) {
      const int n = S->n_tot;
      double a = csvr_alpha(e, R, R.key, R.step_ctr, K, n, &S->flag_timeout);
      if (!isfinite(a) || !isfinite(K)) { a = 1.0; S->flag_nan = 1; }
      S->alpha_th = a;
      R.step_ctr++;
      R.md_steps++;
    }
    c.sync();
    alpha = (float)S->alpha_th;
  }
  return alpha;
}

// The NEMD trajectory of a trial (Sec. II.A, Eq. 2 protocol), out of line: its step loop
// (force passes, list refreshes) gets the whole register budget of the engine instead of
// sharing it with the trial's scalars, which the caller keeps across the call.
template <int SYS>
__device__ H4D_PHASE void nemd_steps(const Ctx& cref, int n_steps) {
  const Ctx c = cref;
  const Eng& e = *c.e;
  Rep& R = *c.R;
  GScal* S = c.v.s;
  const int ins = S->ins;
  const bool single = e.proto.single != 0;
  const int f0 = S->fly0, f1 = S->fly1, f2 = S->fly2;
  if (n_steps > 0) {
    force_pass<SYS>(c, 0, 0.f, nullptr);
    c.sync();
  }
  for (int k = 0; k < n_steps; ++k) {
    kick_drift<SYS>(c, 1.0f);
    c.sync();
    maybe_rebuild(c);
    // the altitude before this step, from the schedule (S->w_cur holds the same value, but
    // thread 0 overwrites it below with no barrier in between when no rebuild happens)
    const float w_prev = (float)altitude(e.proto, ins, k);
    const float w_next = (float)altitude(e.proto, ins, k + 1);
    const float w_next_a = (float)(e.proto.rw * altitude(e.proto, ins, k + 1));
    if (c.tid == 0) {
      uint4 p0 = c.v.pos[f0];
      p0.w = __float_as_uint(w_next);
      c.v.pos[f0] = p0;
      if (!single) {
        uint4 p1 = c.v.pos[f1];
        p1.w = __float_as_uint(w_next_a);
        c.v.pos[f1] = p1;
      }
      if (f2 >= 0) {  // the third atom of a flying water (one w_max: w_next_a = w_next)
        uint4 p2 = c.v.pos[f2];
        p2.w = __float_as_uint(w_next);
        c.v.pos[f2] = p2;
      }
      S->w_cur = w_next;
      S->g_scr = expf(-e.pot.kappa_sr * (single ? w_next : 0.5f * (w_next + w_next_a)));
    }
    c.sync();
    force_pass<SYS>(c, 1 | 4, w_prev, nullptr);
    c.sync();
    if (SYS == H4D_SYS_AQ && c.r.n_water > 0) {
      rattle_pass(c, false);
      c.sync();
    }
    if (c.tid == 0) {
      double dff = 0.0;
      if (e.proto.rw != 1.0) {
        // the flyers' own pair: unscreened, its altitude gap changes with the step
        const uint4 a = c.v.pos[f0], b = c.v.pos[f1];
        const double s = R.L * 0x1.0p-32;
        const double dx = (double)(int)(b.x - a.x) * s, dy = (double)(int)(b.y - a.y) * s,
                     dz = (double)(int)(b.z - a.z) * s;
        const double r3 = dx * dx + dy * dy + dz * dz;
        const double dn = (double)w_next - (double)w_next_a;
        const double dp = (double)w_prev - (double)(float)(e.proto.rw * altitude(e.proto, ins, k));
        const int ta = type_of(f0, c.r.nw3), tb = type_of(f1, c.r.nw3);
        dff = pair_u64(e.pot, ta, tb, r3 + dn * dn, 1.0) - pair_u64(e.pot, ta, tb, r3 + dp * dp, 1.0);
      }
      const double y = (S->dW[0] + S->dW[1] + S->dW[2] + dff) - S->wprot_c;
      const double t = S->wprot + y;
      S->wprot_c = (t - S->wprot) - y;
      S->wprot = t;
    }
  }
}

// one pair-exchange trial (Sec. II.A); readings as in the oracle:
//  - insertion / deletion with probability 1/2, cation and anion chosen independently;
//  - all velocities reversed with probability 1/2 before NEMD and after the decision;
//    a rejection restores the state saved after the first reversal;
//  - Delta H = H_{N+1}(end, all in 3D) - H_N(start, flyers absent) for insertion and the
//    reverse for deletion, flyers' kinetic energy left out (it cancels against Eqs. 3-4).

// ------------------------------------------------------------------------------------
// Learned insertion-site proposal (grid features, BF16 MLP, softmax, cell draw).
// Cells: G per edge, cell (gx*G + gy)*G + gz with gx = floor(X G / 2^32) of the 32-bit
// coordinate.  Features of a cell: 0.25 x the cation, anion and water-O counts of the 27
// cells of its 3x3x3 neighbourhood (slot (ex+1)*9 + (ey+1)*3 + (ez+1) for offset e), then
// 0.1 sum_j q_j d_j / max(|d_j|, 0.5)^3 over the charges of those cells, d_j the minimum
// image of (cell centre - x_j), then zeros up to 96.  The proposal of species s draws a
// cell from q_s = (1 - eps) softmax(logit_s) + eps / G^3 and places the ion uniformly
// inside it; the density ratio to uniform placement, q_s G^3 per ion, enters the
// acceptance exponent (the role of B^ins / B^del in Eqs. 15-16): insertion uses q of the
// start state, deletion q of the end state without the flyers.
// ------------------------------------------------------------------------------------
struct PropView {
  int G, nc;
  int4* cnt;
  long long* fld;
  float2* logit;
  double2* chunk;
};

__device__ __forceinline__ PropView prop_view(const Eng& e, const Rep& R) {
  PropView v;
  v.G = R.prop_G;
  v.nc = R.prop_G * R.prop_G * R.prop_G;
  v.cnt = e.pg_cnt + R.prop_off;
  v.fld = e.pg_fld + 4 * (size_t)R.prop_off;
  v.logit = e.pg_logit + R.prop_off;
  v.chunk = e.pg_chunk + R.prop_off / 32;
  return v;
}

__device__ __forceinline__ int prop_cell_of(unsigned X, unsigned Y, unsigned Z, int G) {
  return ((int)__umulhi(X, (unsigned)G) * G + (int)__umulhi(Y, (unsigned)G)) * G + (int)__umulhi(Z, (unsigned)G);
}

__device__ __forceinline__ int wrap_g(int x, int G) { return x < 0 ? x + G : (x >= G ? x - G : x); }

// cell at neighbour slot n of cell c
__device__ __forceinline__ int prop_nb(int c, int n, int G) {
  const int gx = c / (G * G), gy = (c / G) % G, gz = c % G;
  return (wrap_g(gx + n / 9 - 1, G) * G + wrap_g(gy + (n / 3) % 3 - 1, G)) * G + wrap_g(gz + n % 3 - 1, G);
}

// feature k of cell c (grid counts and field must be complete).  The grid is written with
// atomics in L2, so it is read past L1.
__device__ __forceinline__ float prop_feature(const PropView& pv, int c, int k) {
  if (k < 81) {
    const int s = k / 27;
    const int4 q = __ldcg(pv.cnt + prop_nb(c, k - 27 * s, pv.G));
    return 0.25f * (float)(s == 0 ? q.x : (s == 1 ? q.y : q.z));
  }
  if (k < 84) return (float)((double)__ldcg(pv.fld + 4 * (size_t)c + (k - 81)) * 0x1.0p-40);
  return 0.f;
}

// coordinate of the centre of cell coordinate g (rounded down to the 32-bit grid)
__device__ __forceinline__ unsigned prop_centre(int g, int G) {
  return (unsigned)((((u64)(2 * g + 1)) << 31) / (u64)G);
}

// counts and field of the atoms [0, n_tot) other than ex0, ex1; integer atomics (the
// field in fixed point), so the sums do not depend on the order of the additions
__device__ void prop_grid(const Ctx& c, const PropView& pv, int ex0, int ex1) {
  const Eng& e = *c.e;
  for (int i = c.tid; i < pv.nc; i += c.T) {
    pv.cnt[i] = make_int4(0, 0, 0, 0);
    reinterpret_cast<longlong2*>(pv.fld)[2 * i] = make_longlong2(0, 0);
    reinterpret_cast<longlong2*>(pv.fld)[2 * i + 1] = make_longlong2(0, 0);
  }
  c.sync();
  const int n = c.v.s->n_tot, G = pv.G;
  for (int a = c.tid; a < n; a += c.T) {
    if (a == ex0 || a == ex1) continue;
    const uint4 p = c.v.pos[a];
    const int ty = type_of(a, c.r.nw3);
    const int gx = (int)__umulhi(p.x, (unsigned)G), gy = (int)__umulhi(p.y, (unsigned)G),
              gz = (int)__umulhi(p.z, (unsigned)G);
    if (ty <= 2) atomicAdd(reinterpret_cast<int*>(pv.cnt + (gx * G + gy) * G + gz) + ty, 1);
    const float q = e.pot.q[ty];
    if (q == 0.f) continue;
    for (int d = 0; d < 27; ++d) {
      const int cx = wrap_g(gx + d / 9 - 1, G), cy = wrap_g(gy + (d / 3) % 3 - 1, G), cz = wrap_g(gz + d % 3 - 1, G);
      const float dx = (float)(int)(prop_centre(cx, G) - p.x) * c.r.scale;
      const float dy = (float)(int)(prop_centre(cy, G) - p.y) * c.r.scale;
      const float dz = (float)(int)(prop_centre(cz, G) - p.z) * c.r.scale;
      const float r = fmaxf(sqrtf(dx * dx + dy * dy + dz * dz), 0.5f);
      const float f = 0.1f * q / (r * r * r);
      unsigned long long* dst = reinterpret_cast<unsigned long long*>(pv.fld + 4 * (size_t)((cx * G + cy) * G + cz));
      atomicAdd(dst + 0, (unsigned long long)__double2ll_rn((double)(f * dx) * 0x1.0p40));
      atomicAdd(dst + 1, (unsigned long long)__double2ll_rn((double)(f * dy) * 0x1.0p40));
      atomicAdd(dst + 2, (unsigned long long)__double2ll_rn((double)(f * dz) * 0x1.0p40));
    }
  }
  c.sync();
}

// logits of every cell: warps of the group take 16-cell tiles in turn
__device__ void prop_mlp_all(const Ctx& c, const PropView& pv) {
  const Eng& e = *c.e;
  const int lane = c.tid & 31, warp = c.tid >> 5, nw = c.T >> 5, g = lane >> 2, t = lane & 3;
  const int ntiles = (pv.nc + 15) >> 4;
  for (int tile = warp; tile < ntiles; tile += nw) {
    const int r0 = 16 * tile + g, r1 = r0 + 8;
    auto loadA = [&](int ks, unsigned (&a)[4]) {
      const int k = 16 * ks + 2 * t;
      const bool v0 = r0 < pv.nc, v1 = r1 < pv.nc;
      a[0] = v0 ? pack_bf16(prop_feature(pv, r0, k), prop_feature(pv, r0, k + 1)) : 0u;
      a[1] = v1 ? pack_bf16(prop_feature(pv, r1, k), prop_feature(pv, r1, k + 1)) : 0u;
      a[2] = v0 ? pack_bf16(prop_feature(pv, r0, k + 8), prop_feature(pv, r0, k + 9)) : 0u;
      a[3] = v1 ? pack_bf16(prop_feature(pv, r1, k + 8), prop_feature(pv, r1, k + 9)) : 0u;
    };
    float out[4];
    mlp_tile_forward(e.net, loadA, out);
    if (t == 0) {
      if (r0 < pv.nc) pv.logit[r0] = make_float2(out[0], out[1]);
      if (r1 < pv.nc) pv.logit[r1] = make_float2(out[2], out[3]);
    }
  }
  c.sync();
}

// largest logits and softmax normalisers; partial sums per 32-cell chunk in a fixed order
__device__ void prop_stats(const Ctx& c, const PropView& pv) {
  GScal* S = c.v.s;
  float m0 = -INFINITY, m1 = -INFINITY;
  for (int i = c.tid; i < pv.nc; i += c.T) {
    const float2 l = __ldcg(pv.logit + i);
    m0 = fmaxf(m0, l.x);
    m1 = fmaxf(m1, l.y);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, o));
    m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
  }
  if ((c.tid & 31) == 0) {
    S->pmw[0][c.tid >> 5] = m0;
    S->pmw[1][c.tid >> 5] = m1;
  }
  c.sync();
  if (c.tid == 0) {
    float a = -INFINITY, b = -INFINITY;
    for (int w = 0; w < (c.T >> 5); ++w) {
      a = fmaxf(a, S->pmw[0][w]);
      b = fmaxf(b, S->pmw[1][w]);
    }
    S->pm[0] = a;
    S->pm[1] = b;
  }
  c.sync();
  const double M0 = (double)S->pm[0], M1 = (double)S->pm[1];
  const int nch = (pv.nc + 31) >> 5;
  for (int j = c.tid; j < nch; j += c.T) {
    double s0 = 0.0, s1 = 0.0;
    const int end = min(32 * j + 32, pv.nc);
    for (int i = 32 * j; i < end; ++i) {
      const float2 l = __ldcg(pv.logit + i);
      s0 += exp((double)l.x - M0);
      s1 += exp((double)l.y - M1);
    }
    pv.chunk[j] = make_double2(s0, s1);
  }
  c.sync();
  if (c.tid == 0) {
    double z0 = 0.0, z1 = 0.0;
    for (int j = 0; j < nch; ++j) {
      const double2 z = __ldcg(pv.chunk + j);
      z0 += z.x;
      z1 += z.y;
    }
    S->pZ[0] = z0;
    S->pZ[1] = z1;
  }
  c.sync();
}

__device__ __forceinline__ double prop_weight(const PropView& pv, const GScal* S, int s, int k) {
  const float2 l = __ldcg(pv.logit + k);
  return exp((double)(s ? l.y : l.x) - (double)S->pm[s]);
}

// log of the proposal density relative to uniform, ln(q_s(k) G^3)
__device__ __forceinline__ double prop_lnq(const PropView& pv, const GScal* S, int s, int k, double eps) {
  return log(((1.0 - eps) * prop_weight(pv, S, s, k) / S->pZ[s] + eps / pv.nc) * pv.nc);
}

// cell of species s: with probability eps a uniform cell, else the first cell whose running
// softmax sum exceeds u Z (thread 0 only)
__device__ __noinline__ int prop_draw(const PropView& pv, const GScal* S, int s, u64 r_mix, u64 r_cell, double eps) {
  if (u01(r_mix) < eps) return pick_index(r_cell, pv.nc);
  const double target = u01(r_cell) * S->pZ[s];
  const int nch = (pv.nc + 31) >> 5;
  double cum = 0.0;
  for (int j = 0; j < nch; ++j) {
    const double2 z = __ldcg(pv.chunk + j);
    const double cs = s ? z.y : z.x;
    if (cum + cs > target) {  // the cell lies in this chunk (a rounding miss moves on)
      const double tt = target - cum;
      double part = 0.0;
      const int end = min(32 * j + 32, pv.nc);
      for (int i = 32 * j; i < end; ++i) {
        part += prop_weight(pv, S, s, i);
        if (part > tt) return i;
      }
    }
    cum += cs;
  }
  for (int i = pv.nc - 1; i > 0; --i)  // target not reached through rounding: last live cell
    if (prop_weight(pv, S, s, i) > 0.0) return i;
  return 0;
}

// a 32-bit coordinate uniform over cell coordinate g: [ceil(g 2^32/G), ceil((g+1) 2^32/G))
__device__ __forceinline__ unsigned prop_place(int g, int G, unsigned r32) {
  const u64 lo = ((((u64)g) << 32) + (u64)G - 1) / (u64)G;
  const u64 hi = ((((u64)(g + 1)) << 32) + (u64)G - 1) / (u64)G;
  return (unsigned)(lo + (((u64)r32 * (hi - lo)) >> 32));
}

// training record of the trial: features of the cation and the anion cell
__device__ __noinline__ void prop_record_features(const Ctx& c, const PropView& pv, int slot, int cell_c, int cell_a) {
  const Eng& e = *c.e;
  float* dst = e.prec_feat + (size_t)(c.R->prec_off + slot) * 192;
  for (int i = c.tid; i < 192; i += c.T) dst[i] = prop_feature(pv, i < 96 ? cell_c : cell_a, i % 96);
}

// grid (and, with the learned proposal, logits and normalisers) of the current state
// without ex0, ex1 (kept out of line: it runs once per trial)
__device__ __noinline__ void prop_prepare(const Ctx& c, const PropView& pv, int ex0, int ex1) {
  prop_grid(c, pv, ex0, ex1);
  if (c.e->proto.prop_mode) {
    prop_mlp_all(c, pv);
    prop_stats(c, pv);
  }
}


// ------------------------------------------------------------------------------------
// Bimodal flyer-distance bias (Sec. II.B.3, Eqs. 14-18).  The anion of an insertion sits
// at an offset from the (uniform) cation drawn per axis from b (Eq. 16): two Gaussians
// at +-x_b of sharpness alpha, truncated to [-L/2, L/2) and normalised there.  A deletion
// picks its anion with probability B^ins(r_a | r_c) / sum_n B^ins, B^ins = V prod_i b.
// The Metropolis exponent gains -ln q (insertion) or +ln q (deletion) with
// q = mean of B^ins over the anions of the state with the pair present.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ double bias_density(double alpha, double xb, double L, double x) {
  const double sa = sqrt(alpha);
  const double num = exp(-alpha * (x - xb) * (x - xb)) + exp(-alpha * (x + xb) * (x + xb));
  const double den = erf(sa * (xb + 0.5 * L)) - erf(sa * (xb - 0.5 * L));
  return sqrt(alpha / 3.141592653589793) * num / den;
}

// inverse error function: Winitzki's approximation (a = 0.147), then Newton steps on erf
__device__ double bias_erfinv(double y) {
  const double a = 0.147;
  const double w = log((1.0 - y) * (1.0 + y));
  const double t = 2.0 / (3.141592653589793 * a) + 0.5 * w;
  double x = copysign(sqrt(sqrt(t * t - w / a) - t), y);
  for (int k = 0; k < 6; ++k) {
    const double d = 1.1283791670955126 * exp(-x * x);  // 2/sqrt(pi) e^{-x^2}
    if (!(d > 0.0)) break;
    x -= (erf(x) - y) / d;
  }
  return x;
}

// one offset from b: the top bit of r_mode picks the mode (equal masses), r_u drives the
// inverse CDF of that truncated Gaussian
__device__ __noinline__ double bias_offset(double alpha, double xb, double L, u64 r_mode, u64 r_u) {
  const double c = (r_mode >> 63) ? xb : -xb;
  const double sa = sqrt(alpha);
  const double lo = erf(sa * (-0.5 * L - c)), hi = erf(sa * (0.5 * L - c));
  const double u = ((double)(r_u >> 11) + 0.5) * 0x1.0p-53;
  return c + bias_erfinv(lo + u * (hi - lo)) / sa;
}

// B^ins of the atom at pa relative to the one at pc (minimum-image offsets, exact)
__device__ __noinline__ double bias_B(const Proto& pr, double L, const uint4& pa, const uint4& pc) {
  const double s = L * 0x1.0p-32;
  double B = L * L * L;
  B *= bias_density(pr.bias_alpha, pr.bias_xb, L, (double)(int)(pa.x - pc.x) * s);
  B *= bias_density(pr.bias_alpha, pr.bias_xb, L, (double)(int)(pa.y - pc.y) * s);
  B *= bias_density(pr.bias_alpha, pr.bias_xb, L, (double)(int)(pa.z - pc.z) * s);
  return B;
}

// sum of B^ins over the anions 0..n_anions-1 relative to the cation at pc; with
// target >= 0 also the first anion whose running sum exceeds target (thread 0 only)
__device__ __noinline__ double bias_sum(const Proto& pr, double L, const uint4* pos, int nw3, int n_anions,
                                        const uint4 pc, double target, int* pick) {
  double sum = 0.0;
  int a = n_anions - 1;
  bool found = target < 0.0;
  for (int k = 0; k < n_anions; ++k) {
    sum += bias_B(pr, L, pos[nw3 + 2 * k + 1], pc);
    if (!found && sum > target) { a = k; found = true; }
  }
  if (pick) *pick = a;
  return sum;
}

// ------------------------------------------------------------------------------------
// Rigid-water exchange (Sec. II.A with one flyer; Sec. II.C: molecular-frame velocities).
// Readings as in the oracle: the flying water is frozen in 3D (position and orientation;
// no drift, kick or constraint step) while its altitude follows the schedule; Delta H and
// the momentum reversals as for pairs; V/(N_w+1) once.  Layout: waters first, ions
// after them, so an insertion moves the ions up by three atoms and places the new water
// last, and an accepted deletion moves the last water into the deleted slot and the ions
// down by three.
// ------------------------------------------------------------------------------------

// The inserted water from its trial draws: the O at the 32-bit box fractions of block 1
// words 0-2; the H atoms at the O's fixed-point coordinate plus the rotated body offsets
// rounded to the grid; a uniform orientation from the three uniforms of block 2 (unit
// quaternion (sqrt(1-u1) sin 2 pi u2, sqrt(1-u1) cos 2 pi u2, sqrt(u1) sin 2 pi u3,
// sqrt(u1) cos 2 pi u3), Shoemake 1992); velocities drawn in the molecular frame: centre of
// mass N(0, 1/(beta M)) per axis, angular velocity N(0, 1/(beta I_k)) about body axis k
// (six normals of blocks 3-4), atom a moving with V + R (omega x (a_body - com)).
__device__ __noinline__ void water_placement(const Proto& pr, double L, const u64* b1, const u64* b2,
                                             const u64* b3, const u64* b4, unsigned* xw, double* vw) {
  const double u1 = u01(b2[0]), u2 = u01(b2[1]), u3 = u01(b2[2]);
  const double a = sqrt(1.0 - u1), b = sqrt(u1);
  double s2, c2, s3, c3;
  sincospi(2.0 * u2, &s2, &c2);
  sincospi(2.0 * u3, &s3, &c3);
  const double qx = a * s2, qy = a * c2, qz = b * s3, qw = b * c3;
  const double Rm[3][3] = {{1.0 - 2.0 * (qy * qy + qz * qz), 2.0 * (qx * qy - qw * qz), 2.0 * (qx * qz + qw * qy)},
                           {2.0 * (qx * qy + qw * qz), 1.0 - 2.0 * (qx * qx + qz * qz), 2.0 * (qy * qz - qw * qx)},
                           {2.0 * (qx * qz - qw * qy), 2.0 * (qy * qz + qw * qx), 1.0 - 2.0 * (qx * qx + qy * qy)}};
  for (int d = 0; d < 3; ++d) xw[d] = (unsigned)(b1[d] >> 32);
  for (int k = 0; k < 2; ++k)
    for (int d = 0; d < 3; ++d) {
      const double off = Rm[d][0] * pr.wh[k][0] + Rm[d][1] * pr.wh[k][1] + Rm[d][2] * pr.wh[k][2];
      const long long dk = __double2ll_rn(off / L * 4294967296.0);
      xw[3 * (k + 1) + d] = xw[d] + (unsigned)(unsigned long long)dk;
    }
  const double sv = sqrt(1.0 / (pr.beta * pr.wM));
  const double V[3] = {sv * gauss_c(b3[0], b3[1]), sv * gauss_s(b3[0], b3[1]), sv * gauss_c(b3[2], b3[3])};
  const double om[3] = {sqrt(1.0 / (pr.beta * pr.wI[0])) * gauss_s(b3[2], b3[3]),
                        sqrt(1.0 / (pr.beta * pr.wI[1])) * gauss_c(b4[0], b4[1]),
                        sqrt(1.0 / (pr.beta * pr.wI[2])) * gauss_s(b4[0], b4[1])};
  for (int at = 0; at < 3; ++at) {
    double r[3];
    for (int d = 0; d < 3; ++d) r[d] = (at == 0 ? 0.0 : pr.wh[at - 1][d]) - (d == 1 ? pr.wcom_y : 0.0);
    const double u[3] = {om[1] * r[2] - om[2] * r[1], om[2] * r[0] - om[0] * r[2], om[0] * r[1] - om[1] * r[0]};
    for (int d = 0; d < 3; ++d) vw[3 * at + d] = V[d] + Rm[d][0] * u[0] + Rm[d][1] * u[1] + Rm[d][2] * u[2];
  }
}

// NEMD, decision and commit of a water trial whose flyer is in place (N waters before it,
// n atoms in the start layout)
template <int SYS>
__device__ void trial_water_run(const Ctx& c, int N, int n) {
  const Eng& e = *c.e;
  Rep& R = *c.R;
  GScal* S = c.v.s;
  const int ins = S->ins;
  Ctx cw = c;  // the trial's layout: an inserted water counts among the waters
  cw.r.n_water = S->nw_trial;
  cw.r.nw3 = 3 * S->nw_trial;
  build_list(cw);
  const int f0 = S->fly0, f1 = S->fly1, f2 = S->fly2;
  // H_start: insertion leaves the flyer out, deletion has everyone in 3D
  const double Us = ins ? energy64(cw, f0, f1, f2) : energy64(cw, -1, -1, -1);
  const double Ks = kinetic64(cw);
  if (e.proto.n_f > 0) nemd_steps<SYS>(cw, e.proto.n_f);
  c.sync();
  const double Ue = ins ? energy64(cw, -1, -1, -1) : energy64(cw, f0, f1, f2);
  const double Ke = kinetic64(cw);
  if (c.tid == 0) {
    const double dH = (Ue + Ke) - (Us + Ks);
    const double V = R.L * R.L * R.L;
    double bdm, xacc;
    if (ins) {
      bdm = e.proto.beta * dH - log(V / (double)(N + 1));
      xacc = -bdm + e.proto.beta_mu;
    } else {
      bdm = -e.proto.beta * dH - log(V / (double)N);
      xacc = bdm - e.proto.beta_mu;
    }
    const int status = (isfinite(dH) && !S->flag_nan && !S->flag_overflow && !S->flag_timeout) ? 0 : 3;
    S->flag_nan = 0;
    S->flag_overflow = 0;
    S->flag_timeout = 0;
    const int acc = (status == 0) && (S->ln_u < xacc) && !e.proto.no_accept;
    S->accept = acc;
    h4d_record rr;
    rr.move = ins; rr.accepted = acc; rr.n_before = N;
    rr.n_after = N + (acc ? (ins ? 1 : -1) : 0);
    rr.status = status;
    rr.cation = ins ? -1 : S->flyw; rr.anion = -1;
    rr.cell_c = -1; rr.cell_a = -1; rr.instant = 0;
    rr.dH = dH; rr.beta_dM = bdm; rr.w_prot = S->wprot; rr.ln_u = S->ln_u; rr.x_acc = xacc; rr.ln_q = 0.0;
    e.rec[R.rec_off + (int)(R.rec_count % R.rec_cap)] = rr;
    R.rec_count++;
    R.cycles++;
    if (ins) { R.trials_ins++; R.acc_ins += acc; } else { R.trials_del++; R.acc_del += acc; }
    if (status) R.rej_status++;
    S->ustart = Us; S->uend = Ue; S->kstart = Ks; S->kend = Ke;
  }
  c.sync();
  if (S->accept) {
    if (ins) {
      if (c.tid == 0) {
        for (int k = 0; k < 3; ++k) {
          uint4 p = c.v.pos[f0 + k];
          p.w = 0u;  // altitude(n_f) of an insertion is 0
          c.v.pos[f0 + k] = p;
        }
        R.n_water = N + 1;
        R.nw3 = 3 * (N + 1);
      }
    } else {
      const int m = S->flyw, last = N - 1;
      if (c.tid == 0 && m != last) {  // swap-with-last
        for (int k = 0; k < 3; ++k) {
          c.v.pos[3 * m + k] = c.v.pos[3 * last + k];
          e.vhi[R.atom_off + 3 * m + k] = e.vhi[R.atom_off + 3 * last + k];
          e.vlo[R.atom_off + 3 * m + k] = e.vlo[R.atom_off + 3 * last + k];
        }
      }
      // the ions move down by three atoms, staged through the (no longer needed) copy
      for (int a = 3 * N + c.tid; a < n; a += c.T) {
        const int ga = R.atom_off + a;
        e.pos_save[ga] = c.v.pos[a];
        e.vhi_save[ga] = e.vhi[ga];
        e.vlo_save[ga] = e.vlo[ga];
      }
      c.sync();
      for (int a = 3 * N + c.tid; a < n; a += c.T) {
        const int ga = R.atom_off + a;
        c.v.pos[a - 3] = e.pos_save[ga];
        e.vhi[ga - 3] = e.vhi_save[ga];
        e.vlo[ga - 3] = e.vlo_save[ga];
      }
      if (c.tid == 0) {
        R.n_water = N - 1;
        R.nw3 = 3 * (N - 1);
      }
    }
  } else {
    for (int a = c.tid; a < n; a += c.T) {
      const int ga = R.atom_off + a;
      c.v.pos[a] = e.pos_save[ga];
      e.vhi[ga] = e.vhi_save[ga];
      e.vlo[ga] = e.vlo_save[ga];
    }
  }
  c.sync();
  if (c.tid == 0) {
    S->n_tot = R.nw3 + e.proto.unit * R.n_pairs;
    S->fly0 = S->fly1 = S->fly2 = S->flyw = -1;
    S->w_cur = 0.f;
    S->g_scr = 1.f;
    const double Nn = (double)R.n_water;
    R.sum_n += Nn;
    R.sum_n2 += Nn * Nn;
  }
  c.sync();
  if (S->flip_e) negate_velocities(c, S->n_tot);
  c.sync();
}

template <int SYS>
__device__ __noinline__ void trial_water(const Ctx& c) {
  const Eng& e = *c.e;
  Rep& R = *c.R;
  GScal* S = c.v.s;
  const u64 rep_id = R.key;
  if (c.tid == 0) {
    const u64 t = R.trial_ctr++;
    u64 b0[4], b1[4], b2[4], b3[4], b4[4];
    draw4(e.seed, rep_id, t, 0, kPurTrial, b0);
    draw4(e.seed, rep_id, t, 1, kPurTrial, b1);
    draw4(e.seed, rep_id, t, 2, kPurTrial, b2);
    draw4(e.seed, rep_id, t, 3, kPurTrial, b3);
    draw4(e.seed, rep_id, t, 4, kPurTrial, b4);
    S->ins = (int)(b0[0] >> 63);
    S->flip_s = (int)(b0[1] >> 63);
    S->flip_e = (int)(b0[2] >> 63);
    S->ln_u = log(u01_open(b0[3]));
    const int N = R.n_water;
    S->n_before = N;
    S->status = 0;
    if (!S->ins && N == 0) S->status = 1;
    if (S->ins && N >= R.cap_water) S->status = 2;
    S->cat = -1;
    S->ani = -1;
    S->inst = 0;
    if (S->status == 0) {
      if (S->ins) water_placement(e.proto, R.L, b1, b2, b3, b4, S->xw, S->vw);
      else S->cat = pick_index(b1[0], N);
    }
  }
  c.sync();
  const int N = S->n_before;
  const int n_ion = e.proto.unit * R.n_pairs;
  const int n = 3 * N + n_ion;
  const int ins = S->ins;
  if (S->flip_s) negate_velocities(c, n);
  if (S->status != 0) {
    c.sync();
    if (S->flip_e) negate_velocities(c, n);
    if (c.tid == 0) {
      h4d_record rr;
      rr.move = ins; rr.accepted = 0; rr.n_before = N; rr.n_after = N; rr.status = S->status;
      rr.cation = -1; rr.anion = -1; rr.cell_c = -1; rr.cell_a = -1; rr.instant = 0;
      rr.dH = 0.0; rr.beta_dM = 0.0; rr.w_prot = 0.0; rr.ln_u = S->ln_u; rr.x_acc = 0.0; rr.ln_q = 0.0;
      e.rec[R.rec_off + (int)(R.rec_count % R.rec_cap)] = rr;
      R.rec_count++;
      R.cycles++;
      if (ins) R.trials_ins++; else R.trials_del++;
      R.rej_status++;
      R.sum_n += (double)N;
      R.sum_n2 += (double)N * (double)N;
    }
    c.sync();
    return;
  }
  // save the state for a rejection (positions from shared memory, velocities)
  for (int a = c.tid; a < n; a += c.T) {
    const int ga = R.atom_off + a;
    e.pos_save[ga] = c.v.pos[a];
    e.vhi_save[ga] = e.vhi[ga];
    e.vlo_save[ga] = e.vlo[ga];
  }
  c.sync();
  if (ins) {
    // room for the new water: every ion moves up by three atoms (read from the copy)
    for (int a = 3 * N + c.tid; a < n; a += c.T) {
      const int ga = R.atom_off + a;
      c.v.pos[a + 3] = e.pos_save[ga];
      e.vhi[ga + 3] = e.vhi_save[ga];
      e.vlo[ga + 3] = e.vlo_save[ga];
    }
  }
  const float w0 = (float)altitude(e.proto, ins, 0);
  if (c.tid == 0) {
    const int m = ins ? N : S->cat;
    if (ins) {
      for (int k = 0; k < 3; ++k) {
        const int a = 3 * N + k, ga = R.atom_off + a;
        c.v.pos[a] = make_uint4(S->xw[3 * k], S->xw[3 * k + 1], S->xw[3 * k + 2], __float_as_uint(w0));
        float4 h, l;
        h.x = (float)S->vw[3 * k]; l.x = (float)(S->vw[3 * k] - (double)h.x);
        h.y = (float)S->vw[3 * k + 1]; l.y = (float)(S->vw[3 * k + 1] - (double)h.y);
        h.z = (float)S->vw[3 * k + 2]; l.z = (float)(S->vw[3 * k + 2] - (double)h.z);
        h.w = 0.f; l.w = 0.f;
        e.vhi[ga] = h;
        e.vlo[ga] = l;
      }
    }
    S->fly0 = 3 * m;
    S->fly1 = 3 * m + 1;
    S->fly2 = 3 * m + 2;
    S->flyw = m;
    S->nw_trial = ins ? N + 1 : N;
    S->n_tot = ins ? n + 3 : n;
    S->w_cur = w0;
    S->g_scr = expf(-e.pot.kappa_sr * w0);  // screening at the flyer's altitude (Sec. II.B.2)
    S->wprot = 0.0;
    S->wprot_c = 0.0;
    S->dW[0] = S->dW[1] = S->dW[2] = 0.0;
    S->flag_nan = 0;
    S->flag_overflow = 0;
    S->flag_timeout = 0;
  }
  c.sync();
  trial_water_run<SYS>(c, N, n);
}

template <int SYS>
__device__ void trial_phase(const Ctx& c) {
  if (SYS == H4D_SYS_AQ && c.e->proto.water) {
    trial_water<SYS>(c);
    return;
  }
  const Eng& e = *c.e;
  Rep& R = *c.R;
  GScal* S = c.v.s;
  const u64 rep_id = R.key;
  if (c.tid == 0) {
    const u64 t = R.trial_ctr++;
    u64 b0[4], b1[4], b2[4], b3[4], b4[4];
    draw4(e.seed, rep_id, t, 0, kPurTrial, b0);
    draw4(e.seed, rep_id, t, 1, kPurTrial, b1);
    draw4(e.seed, rep_id, t, 2, kPurTrial, b2);
    draw4(e.seed, rep_id, t, 3, kPurTrial, b3);
    draw4(e.seed, rep_id, t, 4, kPurTrial, b4);
    S->ins = (int)(b0[0] >> 63);
    S->flip_s = (int)(b0[1] >> 63);
    S->flip_e = (int)(b0[2] >> 63);
    S->ln_u = log(u01_open(b0[3]));
    const int N = R.n_pairs;
    S->n_before = N;
    S->status = 0;
    if (!S->ins && N == 0) S->status = 1;
    if (S->ins && N >= R.cap_pairs) S->status = 2;
    S->cat = -1;
    S->ani = -1;
    S->lnq = 0.0;
    S->cell_c = S->cell_a = -1;
    S->prec_slot = -1;
    if (S->ins) {
      S->xfly[0] = (unsigned)(b1[0] >> 32); S->xfly[1] = (unsigned)(b1[1] >> 32);
      S->xfly[2] = (unsigned)(b1[2] >> 32); S->xfly[3] = (unsigned)(b1[3] >> 32);
      S->xfly[4] = (unsigned)(b2[0] >> 32); S->xfly[5] = (unsigned)(b2[1] >> 32);
      if (e.proto.bias_on) {
        // draw block 6: [0..2] the mode of the anion offset on x, y, z; the anion's
        // position words of blocks 1-2 drive the inverse CDF
        u64 b6[4];
        draw4(e.seed, rep_id, t, 6, kPurTrial, b6);
        const u64 ru[3] = {b1[3], b2[0], b2[1]};
        for (int d = 0; d < 3; ++d) {
          const double off = bias_offset(e.proto.bias_alpha, e.proto.bias_xb, R.L, b6[d], ru[d]);
          const long long k = __double2ll_rn(off / R.L * 4294967296.0);
          S->xfly[3 + d] = S->xfly[d] + (unsigned)(unsigned long long)k;
        }
      }
      const double sdc = sqrt(1.0 / (e.proto.beta * e.pot.dm[0]));
      const double sda = sqrt(1.0 / (e.proto.beta * e.pot.dm[1]));
      S->vfly[0] = sdc * gauss_c(b3[0], b3[1]);
      S->vfly[1] = sdc * gauss_s(b3[0], b3[1]);
      S->vfly[2] = sdc * gauss_c(b3[2], b3[3]);
      S->vfly[3] = sda * gauss_s(b3[2], b3[3]);
      S->vfly[4] = sda * gauss_c(b4[0], b4[1]);
      S->vfly[5] = sda * gauss_s(b4[0], b4[1]);
    } else if (N > 0) {
      S->cat = pick_index(b1[0], N);
      S->ani = pick_index(b1[1], N);
      if (e.proto.bias_on) {
        // the anion with probability B^ins(r_a,n | r_c) / sum_n B^ins (Eq. 15), in index
        // order; the factor B^ins / B^del is the mean of B^ins over the N anions
        const uint4 pc = c.v.pos[R.nw3 + 2 * S->cat];
        const double sum = bias_sum(e.proto, R.L, c.v.pos, R.nw3, N, pc, -1.0, nullptr);
        int a = N - 1;
        bias_sum(e.proto, R.L, c.v.pos, R.nw3, N, pc, u01(b1[1]) * sum, &a);
        S->ani = a;
        S->lnq = log(sum / (double)N);
      }
    }
  }
  c.sync();
  const int N = S->n_before;
  const bool single = e.proto.single != 0;  // one flyer (the draws of the anion are unused)
  const int n = R.nw3 + e.proto.unit * N;
  const int ins = S->ins;
  if (S->flip_s) negate_velocities(c, n);
  if (S->status != 0) {
    c.sync();
    if (S->flip_e) negate_velocities(c, n);
    if (c.tid == 0) {
      h4d_record rr;
      rr.move = ins; rr.accepted = 0; rr.n_before = N; rr.n_after = N; rr.status = S->status;
      rr.cation = -1; rr.anion = -1; rr.cell_c = -1; rr.cell_a = -1; rr.instant = 0;
      rr.dH = 0.0; rr.beta_dM = 0.0; rr.w_prot = 0.0; rr.ln_u = S->ln_u; rr.x_acc = 0.0; rr.ln_q = 0.0;
      e.rec[R.rec_off + (int)(R.rec_count % R.rec_cap)] = rr;
      R.rec_count++;
      R.cycles++;
      if (ins) R.trials_ins++; else R.trials_del++;
      R.rej_status++;
      R.sum_n += (double)N;
      R.sum_n2 += (double)N * (double)N;
    }
    c.sync();
    return;
  }
  // proposal grid: an insertion draws its cells from the start state (flyers absent)
  const bool grid = R.prop_G > 0 && (e.proto.prop_mode || e.proto.prop_record);
  if (grid && ins) {
    const PropView pv = prop_view(e, R);
    prop_prepare(c, pv, -1, -1);
    if (c.tid == 0) {
      if (e.proto.prop_mode) {
        // draw block 5: [0], [1] uniform-component choice, [2], [3] cell of the cation, anion;
        // the 32-bit position draws then place each ion inside its cell
        u64 b5[4];
        draw4(e.seed, rep_id, R.trial_ctr - 1, 5, kPurTrial, b5);
        const int G = pv.G;
        double lnq = 0.0;
        for (int sp = 0; sp < 2; ++sp) {
          const int k = prop_draw(pv, S, sp, b5[sp], b5[2 + sp], e.proto.prop_eps);
          lnq += prop_lnq(pv, S, sp, k, e.proto.prop_eps);
          S->xfly[3 * sp + 0] = prop_place(k / (G * G), G, S->xfly[3 * sp + 0]);
          S->xfly[3 * sp + 1] = prop_place((k / G) % G, G, S->xfly[3 * sp + 1]);
          S->xfly[3 * sp + 2] = prop_place(k % G, G, S->xfly[3 * sp + 2]);
        }
        S->lnq = lnq;
      }
      S->cell_c = prop_cell_of(S->xfly[0], S->xfly[1], S->xfly[2], pv.G);
      S->cell_a = prop_cell_of(S->xfly[3], S->xfly[4], S->xfly[5], pv.G);
      S->prec_slot = (e.proto.prop_record && R.prec_cap > 0) ? (int)(R.prec_count % R.prec_cap) : -1;
    }
    c.sync();
    if (S->prec_slot >= 0) prop_record_features(c, pv, S->prec_slot, S->cell_c, S->cell_a);
  }
  // early rejection (SI): a pair whose anion lies in the cube of edge vex_edge around the
  // cation, per axis on the minimum-image fixed-point offset, is exchanged by an
  // instantaneous move (no NEMD steps); the same rule classifies both directions
  if (c.tid == 0) {
    int inst = 0;
    if (e.proto.vex_edge > 0.0) {
      uint4 pc, pa;
      if (ins) {
        pc = make_uint4(S->xfly[0], S->xfly[1], S->xfly[2], 0u);
        pa = make_uint4(S->xfly[3], S->xfly[4], S->xfly[5], 0u);
      } else {
        pc = c.v.pos[R.nw3 + 2 * S->cat];
        pa = c.v.pos[R.nw3 + 2 * S->ani + 1];
      }
      const double half = rint(0.5 * e.proto.vex_edge / R.L * 4294967296.0);
      inst = fabs((double)(int)(pa.x - pc.x)) <= half && fabs((double)(int)(pa.y - pc.y)) <= half &&
             fabs((double)(int)(pa.z - pc.z)) <= half;
    }
    S->inst = inst;
  }
  c.sync();
  const bool inst = S->inst != 0;
  // save the state for a rejection (positions from shared memory, velocities)
  for (int a = c.tid; a < n; a += c.T) {
    const int ga = R.atom_off + a;
    e.pos_save[ga] = c.v.pos[a];
    e.vhi_save[ga] = e.vhi[ga];
    e.vlo_save[ga] = e.vlo[ga];
  }
  c.sync();
  // an instantaneous move keeps the flyers in 3D throughout
  const float w0 = inst ? 0.f : (float)altitude(e.proto, ins, 0);
  const float w0a = inst ? 0.f : (float)(e.proto.rw * altitude(e.proto, ins, 0));  // the anion's altitude
  if (c.tid == 0) {
    if (ins) {
      const int ci = n, ai = n + 1;
      c.v.pos[ci] = make_uint4(S->xfly[0], S->xfly[1], S->xfly[2], __float_as_uint(w0));
      e.vhi[R.atom_off + ci] = make_float4((float)S->vfly[0], (float)S->vfly[1], (float)S->vfly[2], 0.f);
      e.vlo[R.atom_off + ci] = make_float4((float)(S->vfly[0] - (double)(float)S->vfly[0]),
                                           (float)(S->vfly[1] - (double)(float)S->vfly[1]),
                                           (float)(S->vfly[2] - (double)(float)S->vfly[2]), 0.f);
      if (!single) {
        c.v.pos[ai] = make_uint4(S->xfly[3], S->xfly[4], S->xfly[5], __float_as_uint(w0a));
        e.vhi[R.atom_off + ai] = make_float4((float)S->vfly[3], (float)S->vfly[4], (float)S->vfly[5], 0.f);
        e.vlo[R.atom_off + ai] = make_float4((float)(S->vfly[3] - (double)(float)S->vfly[3]),
                                             (float)(S->vfly[4] - (double)(float)S->vfly[4]),
                                             (float)(S->vfly[5] - (double)(float)S->vfly[5]), 0.f);
      }
      S->fly0 = ci;
      S->fly1 = single ? -1 : ai;
      S->n_tot = n + e.proto.unit;
    } else {
      S->fly0 = R.nw3 + e.proto.unit * S->cat;
      S->fly1 = single ? -1 : R.nw3 + 2 * S->ani + 1;
      S->n_tot = n;
    }
    S->w_cur = w0;
    // screening at the mean altitude of the flyers (Sec. II.B.2)
    S->g_scr = expf(-e.pot.kappa_sr * (single ? w0 : 0.5f * (w0 + w0a)));
    S->wprot = 0.0;
    S->wprot_c = 0.0;
    S->dW[0] = S->dW[1] = S->dW[2] = 0.0;
    S->flag_nan = 0;       // a blow-up inside NEMD only rejects this trial
    S->flag_overflow = 0;  // so does a neighbour row that overflowed during it
    S->flag_timeout = 0;   // and a rigid-water constraint that did not converge
  }
  c.sync();
  build_list(c);
  const int f0 = S->fly0, f1 = S->fly1;
  // H_start: insertion leaves the flyers out, deletion has everyone in 3D
  const double Us = ins ? energy64(c, f0, f1) : energy64(c, -1, -1);
  const double Ks = kinetic64(c);
  const int n_steps = inst ? 0 : e.proto.n_f;
  if (n_steps > 0) nemd_steps<SYS>(c, n_steps);
  c.sync();
  // H_end: insertion has everyone in 3D, deletion leaves the flyers out
  const double Ue = ins ? energy64(c, -1, -1) : energy64(c, f0, f1);
  const double Ke = kinetic64(c);
  // proposal grid: the reverse insertion of a deletion draws from the end state, flyers
  // removed, the cells the flyers occupy
  if (grid && !ins) {
    const PropView pv = prop_view(e, R);
    prop_prepare(c, pv, f0, f1);
    if (c.tid == 0) {
      const uint4 pc = c.v.pos[f0], pa = c.v.pos[f1];
      S->cell_c = prop_cell_of(pc.x, pc.y, pc.z, pv.G);
      S->cell_a = prop_cell_of(pa.x, pa.y, pa.z, pv.G);
      if (e.proto.prop_mode)
        S->lnq = prop_lnq(pv, S, 0, S->cell_c, e.proto.prop_eps) + prop_lnq(pv, S, 1, S->cell_a, e.proto.prop_eps);
      S->prec_slot = (e.proto.prop_record && R.prec_cap > 0) ? (int)(R.prec_count % R.prec_cap) : -1;
    }
    c.sync();
    if (S->prec_slot >= 0) prop_record_features(c, pv, S->prec_slot, S->cell_c, S->cell_a);
  }
  if (c.tid == 0) {
    const double dH = (Ue + Ke) - (Us + Ks);
    const double V = R.L * R.L * R.L;
    double bdm, xacc;
    // the phase-space factor V/(N+1) once per flyer: squared for a pair (Eqs. 6, 8), once
    // for a single particle (Sec. II.A, the pair rule translated to one flyer)
    const double nfly = single ? 1.0 : 2.0;
    if (ins) {
      bdm = e.proto.beta * dH - nfly * log(V / (double)(N + 1));  // Eq. 6
      xacc = -bdm + e.proto.beta_mu;
    } else {
      bdm = -e.proto.beta * dH - nfly * log(V / (double)N);       // Eq. 8
      xacc = bdm - e.proto.beta_mu;
    }
    const double x_phys = xacc;
    if (ins && e.proto.bias_on) {
      // B^ins / B^del of the reverse deletion, in the end state: the mean of B^ins over the
      // N+1 anions relative to the inserted cation
      const double sum = bias_sum(e.proto, R.L, c.v.pos, R.nw3, N + 1, c.v.pos[f0], -1.0, nullptr);
      S->lnq = log(sum / (double)(N + 1));
    }
    xacc += ins ? -S->lnq : S->lnq;  // proposal density relative to uniform placement
    int status = (isfinite(dH) && !S->flag_nan && !S->flag_overflow && !S->flag_timeout) ? 0 : 3;
    S->flag_nan = 0;
    S->flag_overflow = 0;
    S->flag_timeout = 0;
    int acc = (status == 0) && (S->ln_u < xacc) && !e.proto.no_accept;
    S->accept = acc;
    h4d_record rr;
    rr.move = ins; rr.accepted = acc; rr.n_before = N;
    rr.n_after = N + (acc ? (ins ? 1 : -1) : 0);
    rr.status = status;
    rr.cation = ins ? -1 : S->cat; rr.anion = (ins || single) ? -1 : S->ani;
    rr.cell_c = S->cell_c; rr.cell_a = S->cell_a; rr.instant = S->inst;
    rr.dH = dH; rr.beta_dM = bdm; rr.w_prot = S->wprot; rr.ln_u = S->ln_u; rr.x_acc = xacc; rr.ln_q = S->lnq;
    if (S->prec_slot >= 0) {
      const int gi = R.prec_off + S->prec_slot;
      e.prec_y[gi] = ins ? x_phys : -x_phys;
      e.prec_meta[gi] = make_int2(ins, status);
      R.prec_count++;
    }
    e.rec[R.rec_off + (int)(R.rec_count % R.rec_cap)] = rr;
    R.rec_count++;
    R.cycles++;
    if (ins) { R.trials_ins++; R.acc_ins += acc; } else { R.trials_del++; R.acc_del += acc; }
    if (status) R.rej_status++;
    S->ustart = Us; S->uend = Ue; S->kstart = Ks; S->kend = Ke;
  }
  c.sync();
  const int acc = S->accept;
  if (acc) {
    if (c.tid == 0) {
      if (ins) {
        uint4 p0 = c.v.pos[f0];
        p0.w = 0u;  // altitude(n_f) of an insertion is 0
        c.v.pos[f0] = p0;
        if (!single) {
          uint4 p1 = c.v.pos[f1];
          p1.w = 0u;
          c.v.pos[f1] = p1;
        }
        R.n_pairs = N + 1;
      } else if (single) {
        const int last = R.nw3 + (N - 1);  // swap-with-last
        c.v.pos[f0] = c.v.pos[last];
        e.vhi[R.atom_off + f0] = e.vhi[R.atom_off + last];
        e.vlo[R.atom_off + f0] = e.vlo[R.atom_off + last];
        R.n_pairs = N - 1;
      } else {
        // swap-with-last keeps the interleaved cation/anion layout
        const int lc = R.nw3 + 2 * (N - 1), la = lc + 1;
        uint4 pc = c.v.pos[lc], pa = c.v.pos[la];
        c.v.pos[f0] = pc;
        c.v.pos[f1] = pa;
        e.vhi[R.atom_off + f0] = e.vhi[R.atom_off + lc];
        e.vlo[R.atom_off + f0] = e.vlo[R.atom_off + lc];
        e.vhi[R.atom_off + f1] = e.vhi[R.atom_off + la];
        e.vlo[R.atom_off + f1] = e.vlo[R.atom_off + la];
        R.n_pairs = N - 1;
      }
    }
  } else {
    for (int a = c.tid; a < n; a += c.T) {
      const int ga = R.atom_off + a;
      c.v.pos[a] = e.pos_save[ga];
      e.vhi[ga] = e.vhi_save[ga];
      e.vlo[ga] = e.vlo_save[ga];
    }
  }
  c.sync();
  if (c.tid == 0) {
    S->n_tot = R.nw3 + e.proto.unit * R.n_pairs;
    S->fly0 = S->fly1 = S->fly2 = S->flyw = -1;
    S->w_cur = 0.f;
    S->g_scr = 1.f;
    const double Nn = (double)R.n_pairs;
    R.sum_n += Nn;
    R.sum_n2 += Nn * Nn;
  }
  c.sync();
  if (S->flip_e) negate_velocities(c, S->n_tot);
  c.sync();
}

// ------------------------------------------------------------------------------------
// Kernels
// ------------------------------------------------------------------------------------

// bind this thread to its group's replica; false for warps outside every group
__device__ bool setup_ctx(const Eng& e, char* smem, Ctx& c) {
  const int warp = threadIdx.x >> 5;
  const int g0 = e.cta_groups[blockIdx.x], g1 = e.cta_groups[blockIdx.x + 1];
  int gi = -1;
  for (int g = g0; g < g1; ++g)
    if (warp >= e.groups[g].warp0 && warp < e.groups[g].warp0 + e.groups[g].nwarps) gi = g;
  if (gi < 0) return false;
  const Group G = e.groups[gi];
  Rep* R = &e.rep[G.rep];
  c.R = R;
  c.e = &e;
  c.tid = threadIdx.x - 32 * G.warp0;
  c.T = 32 * G.nwarps;
  c.bar = G.bar;
  c.tpa = R->tpa;
  c.ltpa = __ffs(R->tpa) - 1;
  c.r = repc_of(*R);
  c.v = carve(smem + G.smem_off, R->cap_atoms, R->nc, c.T);
  GScal* S = c.v.s;
  if (c.tid == 0) {
    S->flag_rebuild = 1; S->flag_overflow = 0; S->flag_nan = 0; S->flag_timeout = 0; S->n_ord = 0; S->n_rank = 0; S->n_lay = 0;
    S->n_tot = R->nw3 + e.proto.unit * R->n_pairs;
    S->fly0 = S->fly1 = S->fly2 = S->flyw = -1;
    S->w_cur = 0.f; S->g_scr = 1.f;
    write_sentinel(c.v, R->cap_atoms);
  }
  c.sync();
  for (int a = c.tid; a < S->n_tot; a += c.T) c.v.pos[a] = e.pos[R->atom_off + a];
  c.sync();
  return true;
}

template <int SYS>
__global__ void __launch_bounds__(H4D_MAXTHREADS, H4D_MINBLOCKS) cycles_kernel(const __grid_constant__ Eng e, long long k_cycles, int n_eq, int do_trial) {
  extern __shared__ __align__(16) char smem[];
  Ctx c;
  if (!setup_ctx(e, smem, c)) return;
  Rep* R = c.R;
  GScal* S = c.v.s;
  if (c.tid == 0) {
    unsigned sm;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
    R->smid = (int)sm;
    R->t_begin = gtimer();
  }
  for (long long cyc = 0; cyc < k_cycles; ++cyc) {
    u64 t0 = gtimer();
    if (n_eq > 0) md_phase<SYS>(c, n_eq);
    u64 t1 = gtimer();
    if (do_trial) {
      trial_phase<SYS>(c);
      // a water exchange changes where the ions start (every thread saw R after the sync)
      c.r.n_water = R->n_water;
      c.r.nw3 = R->nw3;
    }
    u64 t2 = gtimer();
    if (c.tid == 0) {
      R->t_md_ns += (double)(t1 - t0);
      R->t_nemd_ns += (double)(t2 - t1);
    }
  }
  c.sync();
  for (int a = c.tid; a < S->n_tot; a += c.T) e.pos[R->atom_off + a] = c.v.pos[a];
  if (c.tid == 0 && S->flag_overflow) R->err |= 1;
  if (c.tid == 0) R->t_end = gtimer();
}

// current U (FP64) and K of each replica
// proposal logits (and optionally every feature) of one replica's current state
__global__ void __launch_bounds__(1024) prop_eval_kernel(const __grid_constant__ Eng e, int replica, float* feat_out) {
  extern __shared__ __align__(16) char smem[];
  Ctx c;
  if (!setup_ctx(e, smem, c)) return;
  if ((int)(c.R - e.rep) != replica) return;
  const PropView pv = prop_view(e, *c.R);
  prop_grid(c, pv, -1, -1);
  prop_mlp_all(c, pv);
  if (feat_out)
    for (int i = c.tid; i < pv.nc * kPropNFeat; i += c.T) feat_out[i] = prop_feature(pv, i / kPropNFeat, i % kPropNFeat);
}

int launch_prop_eval(const Eng& e, int n_ctas, int cta_threads, size_t smem, int replica, float* feat_out,
                     void* stream) {
  cudaFuncSetAttribute(prop_eval_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  prop_eval_kernel<<<n_ctas, cta_threads, smem, (cudaStream_t)stream>>>(e, replica, feat_out);
  return cudaGetLastError() == cudaSuccess ? H4D_OK : H4D_ECUDA;
}

__global__ void __launch_bounds__(1024) energy_kernel(const __grid_constant__ Eng e, double* U, double* K) {
  extern __shared__ __align__(16) char smem[];
  Ctx c;
  if (!setup_ctx(e, smem, c)) return;
  build_list(c);
  const double u = energy64(c, -1, -1);
  const double k = kinetic64(c);
  const int r = (int)(c.R - e.rep);
  if (c.tid == 0) {
    U[r] = u; K[r] = k;
    if (c.v.s->flag_overflow) c.R->err |= 1;
  }
}

// pairs within the larger cut-off (each unordered pair once), summed over replicas
__global__ void __launch_bounds__(1024) count_kernel(const __grid_constant__ Eng e, unsigned long long* out) {
  extern __shared__ __align__(16) char smem[];
  Ctx c;
  if (!setup_ctx(e, smem, c)) return;
  Rep* R = c.R;
  GScal* S = c.v.s;
  build_list(c);
  unsigned long long cnt = 0;
  const float scale = R->scale;
  const bool use_ord = S->n_ord == S->n_tot;
  for (int k = c.tid; k < S->n_tot; k += c.T) {
    const int i = use_ord ? (int)c.v.sorted[k] : k;
    const uint4 pi = c.v.pos[i];
    const int m = e.ncnt[R->atom_off + k];
    for (int s = 0; s < m; ++s) {
      const int j = e.nbr[nbr_index(e, c.r, k, s, c.ltpa)];
      if (j <= i) continue;
      const uint4 pj = c.v.pos[j];
      const float dx = (float)(int)(pj.x - pi.x) * scale;
      const float dy = (float)(int)(pj.y - pi.y) * scale;
      const float dz = (float)(int)(pj.z - pi.z) * scale;
      if (dx * dx + dy * dy + dz * dz < e.pot.rc2_max) ++cnt;
    }
  }
  atomicAdd(out, cnt);
  if (c.tid == 0 && S->flag_overflow) R->err |= 1;
}

// one configuration as given: list, FP32 forces (written to e.force), FP64 energy;
// wbar is the mean altitude of the flying particles (Sec. II.B.2)
template <int SYS>
__global__ void __launch_bounds__(1024) eval_kernel(const __grid_constant__ Eng e, float wbar, double* U) {
  extern __shared__ __align__(16) char smem[];
  const Group G = e.groups[0];
  Rep* R = &e.rep[0];
  Ctx c;
  c.R = R; c.e = &e;
  c.tid = threadIdx.x;
  c.T = blockDim.x;
  c.bar = 0;
  c.tpa = R->tpa;
  c.ltpa = __ffs(R->tpa) - 1;
  c.r = repc_of(*R);
  c.v = carve(smem + G.smem_off, R->cap_atoms, R->nc, c.T);
  GScal* S = c.v.s;
  if (c.tid == 0) {
    S->flag_rebuild = 1; S->flag_overflow = 0; S->flag_nan = 0; S->flag_timeout = 0; S->n_ord = 0; S->n_rank = 0; S->n_lay = 0;
    S->n_tot = R->nw3 + e.proto.unit * R->n_pairs;
    S->fly0 = S->fly1 = S->fly2 = S->flyw = -1;
    S->w_cur = wbar;
    S->g_scr = expf(-e.pot.kappa_sr * wbar);
    write_sentinel(c.v, R->cap_atoms);
  }
  c.sync();
  for (int a = c.tid; a < S->n_tot; a += c.T) c.v.pos[a] = e.pos[R->atom_off + a];
  c.sync();
  build_list(c);
  force_pass<SYS>(c, 0, 0.f, nullptr);
  c.sync();
  const double u = energy64(c, -1, -1);
  if (c.tid == 0) {
    *U = u;
    if (S->flag_overflow) R->err |= 1;
  }
}

int launch_eval(const Eng& e, int threads, size_t smem, float wbar, double* U, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (e.pot.sys == H4D_SYS_LJ) {
    cudaFuncSetAttribute(eval_kernel<H4D_SYS_LJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    eval_kernel<H4D_SYS_LJ><<<1, threads, smem, st>>>(e, wbar, U);
  } else {
    cudaFuncSetAttribute(eval_kernel<H4D_SYS_AQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    eval_kernel<H4D_SYS_AQ><<<1, threads, smem, st>>>(e, wbar, U);
  }
  return cudaGetLastError() == cudaSuccess ? H4D_OK : H4D_ECUDA;
}

// n_iter equilibrium force passes on the current state (autotuning and profiling of the
// pair term in isolation); leaves positions and velocities untouched
template <int SYS>
__global__ void __launch_bounds__(H4D_MAXTHREADS, H4D_MINBLOCKS) forces_kernel(const __grid_constant__ Eng e, int n_iter) {
  extern __shared__ __align__(16) char smem[];
  Ctx c;
  if (!setup_ctx(e, smem, c)) return;
  build_list(c);
  for (int it = 0; it < n_iter; ++it) {
    force_pass<SYS, false>(c, 0, 0.f, nullptr);
    c.sync();
  }
}

int launch_forces(const Eng& e, int n_ctas, int cta_threads, size_t smem, int n_iter, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (e.pot.sys == H4D_SYS_LJ) {
    cudaFuncSetAttribute(forces_kernel<H4D_SYS_LJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    forces_kernel<H4D_SYS_LJ><<<n_ctas, cta_threads, smem, st>>>(e, n_iter);
  } else {
    cudaFuncSetAttribute(forces_kernel<H4D_SYS_AQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    forces_kernel<H4D_SYS_AQ><<<n_ctas, cta_threads, smem, st>>>(e, n_iter);
  }
  return cudaGetLastError() == cudaSuccess ? H4D_OK : H4D_ECUDA;
}

// neighbour rows only (for the bit-exact neighbour-set check)
__global__ void __launch_bounds__(1024) list_kernel(const __grid_constant__ Eng e) {
  extern __shared__ __align__(16) char smem[];
  Ctx c;
  if (!setup_ctx(e, smem, c)) return;
  build_list(c);
  if (c.tid == 0 && c.v.s->flag_overflow) c.R->err |= 1;
}

int launch_list(const Eng& e, int n_ctas, int cta_threads, size_t smem, void* stream) {
  cudaFuncSetAttribute(list_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  list_kernel<<<n_ctas, cta_threads, smem, (cudaStream_t)stream>>>(e);
  return cudaGetLastError() == cudaSuccess ? H4D_OK : H4D_ECUDA;
}

static int check(cudaError_t err) { return err == cudaSuccess ? H4D_OK : H4D_ECUDA; }

int engine_binary_version(int* binary_version, int* ptx_version) {
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, cycles_kernel<H4D_SYS_LJ>) != cudaSuccess) return H4D_ECUDA;
  *binary_version = a.binaryVersion;
  *ptx_version = a.ptxVersion;
  return H4D_OK;
}

int launch_cycles(const Eng& e, int n_ctas, int cta_threads, size_t smem, long long k_cycles, int n_eq,
                  int do_trial, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (e.pot.sys == H4D_SYS_LJ) {
    cudaFuncSetAttribute(cycles_kernel<H4D_SYS_LJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cycles_kernel<H4D_SYS_LJ><<<n_ctas, cta_threads, smem, st>>>(e, k_cycles, n_eq, do_trial);
  } else {
    cudaFuncSetAttribute(cycles_kernel<H4D_SYS_AQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cycles_kernel<H4D_SYS_AQ><<<n_ctas, cta_threads, smem, st>>>(e, k_cycles, n_eq, do_trial);
  }
  return check(cudaGetLastError());
}

int launch_energy(const Eng& e, int n_ctas, int cta_threads, size_t smem, double* U, double* K, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  cudaFuncSetAttribute(energy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  energy_kernel<<<n_ctas, cta_threads, smem, st>>>(e, U, K);
  return check(cudaGetLastError());
}

int launch_count_pairs(const Eng& e, int n_ctas, int cta_threads, size_t smem, unsigned long long* out,
                       void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  cudaFuncSetAttribute(count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  count_kernel<<<n_ctas, cta_threads, smem, st>>>(e, out);
  return check(cudaGetLastError());
}

}  // namespace h4d
