// h4d_prop.cuh -- the learned insertion-site proposal network on the tensor cores: BF16
// operands, FP32 accumulation, warp-level mma.sync m16n8k16 tiles of 16 rows (shared by
// the inference path inside the cycles kernel and by the training kernels).
//
// Network: 96 features -> 64 (ReLU) -> 64 (ReLU) -> 2 logits (cation site, anion site).
// Flat FP32 master layout (row index = input unit): W1[96][64], b1[64], W2[64][64], b2[64],
// W3[64][2], b3[2].
//
// Fragment layout of mma.m16n8k16 (g = lane / 4, t = lane % 4):
//   A (16 x 16, row major): reg0 = (row g, k 2t..2t+1), reg1 = (row g+8, k 2t..2t+1),
//                           reg2 = (row g, k 2t+8..2t+9), reg3 = (row g+8, k 2t+8..2t+9)
//   B (16 x 8):             reg0 = (k 2t..2t+1, col g), reg1 = (k 2t+8..2t+9, col g)
//   C (16 x 8, FP32):       c0,c1 = (row g, cols 2t, 2t+1), c2,c3 = (row g+8, same cols)
// Two bf16 values share a register, the lower k (or column) in the low half.  The
// weights are stored pre-packed as B fragments, [k-step][n-tile][lane] -> uint2, so a warp
// reads each fragment with one coalesced 8-byte load per lane.
#pragma once
#include <cstdint>

namespace h4d {

constexpr int kPropNFeat = 96;
constexpr int kPropHid = 64;
constexpr int kPropNW = kPropNFeat * kPropHid + kPropHid + kPropHid * kPropHid + kPropHid + kPropHid * 2 + 2;
constexpr int kPropOffB1 = kPropNFeat * kPropHid;
constexpr int kPropOffW2 = kPropOffB1 + kPropHid;
constexpr int kPropOffB2 = kPropOffW2 + kPropHid * kPropHid;
constexpr int kPropOffW3 = kPropOffB2 + kPropHid;
constexpr int kPropOffB3 = kPropOffW3 + kPropHid * 2;
constexpr int kPropMaxG = 32;

// packed network (device pointers)
struct PropNet {
  const uint2* w1;   // [6][8][32]   B fragments of W1
  const uint2* w2;   // [4][8][32]   B fragments of W2
  const uint2* w3;   // [4][1][32]   B fragments of W3, columns 2..7 zero
  const uint2* w2t;  // [4][8][32]   B fragments of W2^T (backward)
  const float* w3r;  // [64][2]      W3 rounded to bf16 (backward)
  const float* b;    // b1[64], b2[64], b3[2] (FP32)
};

// two floats -> bf16x2 (round to nearest even), lo in the low half
__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  unsigned r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
__device__ __forceinline__ float bf16_lo(unsigned v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(unsigned v) { return __uint_as_float(v & 0xffff0000u); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], uint2 b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

// C fragments of n-tiles 2j, 2j+1 (after bias and ReLU) -> A fragment of k-step j of the
// next layer
__device__ __forceinline__ void c_to_a(const float (&c0)[4], const float (&c1)[4], unsigned (&a)[4]) {
  a[0] = pack_bf16(c0[0], c0[1]);
  a[1] = pack_bf16(c0[2], c0[3]);
  a[2] = pack_bf16(c1[0], c1[1]);
  a[3] = pack_bf16(c1[2], c1[3]);
}

// bias + ReLU on a C fragment of n-tile nt
__device__ __forceinline__ void bias_relu(float (&c)[4], const float* b, int nt, int t) {
  const float b0 = b[8 * nt + 2 * t], b1 = b[8 * nt + 2 * t + 1];
  c[0] = fmaxf(c[0] + b0, 0.f);
  c[1] = fmaxf(c[1] + b1, 0.f);
  c[2] = fmaxf(c[2] + b0, 0.f);
  c[3] = fmaxf(c[3] + b1, 0.f);
}

// Forward of one 16-row tile for inference, in halves of 32 hidden units to keep few
// registers live.  loadA(ks, a) fills the layer-1 A fragment of k-step ks (6 k-steps).
// Returns the logit C fragment: out[0..1] = row g (cation, anion) on lanes with t == 0,
// out[2..3] = row g+8.
template <class LoadA>
__device__ __forceinline__ void mlp_tile_forward(const PropNet& net, LoadA loadA, float (&out)[4]) {
  const int lane = threadIdx.x & 31, t = lane & 3;
  unsigned h1[4][4];  // layer-2 A fragments (4 k-steps)
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
#pragma unroll 1
    for (int ks = 0; ks < 6; ++ks) {
      unsigned a[4];
      loadA(ks, a);
#pragma unroll
      for (int i = 0; i < 4; ++i) mma_bf16(acc[i], a, net.w1[(ks * 8 + 4 * half + i) * 32 + lane]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) bias_relu(acc[i], net.b, 4 * half + i, t);
    c_to_a(acc[0], acc[1], h1[2 * half]);
    c_to_a(acc[2], acc[3], h1[2 * half + 1]);
  }
  out[0] = out[1] = out[2] = out[3] = 0.f;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
#pragma unroll
    for (int ks = 0; ks < 4; ++ks)
#pragma unroll
      for (int i = 0; i < 4; ++i) mma_bf16(acc[i], h1[ks], net.w2[(ks * 8 + 4 * half + i) * 32 + lane]);
#pragma unroll
    for (int i = 0; i < 4; ++i) bias_relu(acc[i], net.b + kPropHid, 4 * half + i, t);
    unsigned a3[4];
    c_to_a(acc[0], acc[1], a3);
    mma_bf16(out, a3, net.w3[(2 * half) * 32 + lane]);
    c_to_a(acc[2], acc[3], a3);
    mma_bf16(out, a3, net.w3[(2 * half + 1) * 32 + lane]);
  }
  const float* b3 = net.b + 2 * kPropHid;
  out[0] += b3[0];
  out[1] += b3[1];
  out[2] += b3[0];
  out[3] += b3[1];
}

// Launches of the proposal kernels (h4d_train.cu)
int launch_prop_pack(const float* w, uint2* w1, uint2* w2, uint2* w3, uint2* w2t, float* w3r, float* b,
                     void* stream);
// rows = 2 * n_rec (cation row then anion row of each record); targets t[n_rec][2]
int launch_prop_fwd_bwd(const PropNet& net, const float* feat, const float* tgt, int n_rec, float inv_n,
                        uint16_t* xT, uint16_t* h1T, uint16_t* dz1T, uint16_t* h2T, uint16_t* dz2T,
                        uint16_t* dlT, float* loss_rows, int rows_pad, void* stream);
int launch_prop_wgrad(const uint16_t* xT, const uint16_t* h1T, const uint16_t* dz1T, const uint16_t* h2T,
                      const uint16_t* dz2T, const uint16_t* dlT, const float* loss_rows, int rows_pad,
                      float* grad, double* loss, void* stream);
int launch_prop_adam(float* w, float* m, float* v, const float* grad, int step, float lr, void* stream);
// minibatch of n_batch records (uniform draws keyed by (seed, step)), or all valid records
// in order when n_batch >= n_valid
int launch_prop_gather(const float* rec_feat, const double* rec_y, const int* valid, int n_valid, int n_batch,
                       unsigned long long seed, long long step, float y0, float* feat, float* tgt,
                       void* stream);
int launch_prop_compact(const int2* meta, const double* y, int n_rec, int* valid, int* n_valid, void* stream);

}  // namespace h4d
