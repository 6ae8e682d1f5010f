// h4d_train.cu -- training of the learned insertion-site proposal on the GPU: minibatch
// gather from the trial records, BF16 forward and backward through the 96-64-64-2 network
// on mma.sync tiles (FP32 accumulation), weight-gradient GEMMs over the batch, Adam.
//
// Loss of a batch of n records (each a cation row and an anion row):
//   L = (1/n) sum_records [BCE(logit_cation(f_c), t) + BCE(logit_anion(f_a), t)]
// with the soft target t = min(1, exp(y - y0)) of the record's insertion-direction
// Metropolis exponent y.  Every reduction runs in a fixed order, so a step is
// bit-reproducible.
#include <cuda_runtime.h>

#include <cstdint>

#include "h4d_engine.cuh"
#include "h4d_philox.cuh"
#include "h4d_prop.cuh"

namespace h4d {

// ---- weight packing: FP32 masters -> bf16 B fragments --------------------------------
// item ranges: w1 [0,1536), w2 [1536,2560), w3 [2560,2688), w2t [2688,3712),
// w3r [3712,3840), b [3840,3970)
__global__ void prop_pack_kernel(const float* __restrict__ w, uint2* w1, uint2* w2, uint2* w3, uint2* w2t,
                                 float* w3r, float* b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const float* W1 = w;
  const float* W2 = w + kPropOffW2;
  const float* W3 = w + kPropOffW3;
  if (i < 1536) {  // W1: K = 96 (6 k-steps), N = 64 (8 n-tiles)
    const int lane = i & 31, nt = (i >> 5) & 7, ks = i >> 8, g = lane >> 2, t = lane & 3;
    const int n = 8 * nt + g, k = 16 * ks + 2 * t;
    w1[i] = make_uint2(pack_bf16(W1[k * 64 + n], W1[(k + 1) * 64 + n]),
                       pack_bf16(W1[(k + 8) * 64 + n], W1[(k + 9) * 64 + n]));
  } else if (i < 2560) {  // W2: K = 64, N = 64
    const int j = i - 1536, lane = j & 31, nt = (j >> 5) & 7, ks = j >> 8, g = lane >> 2, t = lane & 3;
    const int n = 8 * nt + g, k = 16 * ks + 2 * t;
    w2[j] = make_uint2(pack_bf16(W2[k * 64 + n], W2[(k + 1) * 64 + n]),
                       pack_bf16(W2[(k + 8) * 64 + n], W2[(k + 9) * 64 + n]));
  } else if (i < 2688) {  // W3: K = 64, N = 8 (columns 2..7 zero)
    const int j = i - 2560, lane = j & 31, ks = j >> 5, g = lane >> 2, t = lane & 3;
    const int k = 16 * ks + 2 * t;
    float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f;
    if (g < 2) {
      v0 = W3[k * 2 + g]; v1 = W3[(k + 1) * 2 + g]; v2 = W3[(k + 8) * 2 + g]; v3 = W3[(k + 9) * 2 + g];
    }
    w3[j] = make_uint2(pack_bf16(v0, v1), pack_bf16(v2, v3));
  } else if (i < 3712) {  // W2^T: B[k][n] = W2[n][k]
    const int j = i - 2688, lane = j & 31, nt = (j >> 5) & 7, ks = j >> 8, g = lane >> 2, t = lane & 3;
    const int n = 8 * nt + g, k = 16 * ks + 2 * t;
    w2t[j] = make_uint2(pack_bf16(W2[n * 64 + k], W2[n * 64 + k + 1]),
                        pack_bf16(W2[n * 64 + k + 8], W2[n * 64 + k + 9]));
  } else if (i < 3840) {
    const int j = i - 3712;
    w3r[j] = bf16_lo(pack_bf16(W3[j], 0.f));
  } else if (i < 3970) {
    const int j = i - 3840;
    b[j] = j < 64 ? w[kPropOffB1 + j] : (j < 128 ? w[kPropOffB2 + j - 64] : w[kPropOffB3 + j - 128]);
  }
}

int launch_prop_pack(const float* w, uint2* w1, uint2* w2, uint2* w3, uint2* w2t, float* w3r, float* b,
                     void* stream) {
  prop_pack_kernel<<<(3970 + 255) / 256, 256, 0, (cudaStream_t)stream>>>(w, w1, w2, w3, w2t, w3r, b);
  return cudaGetLastError() == cudaSuccess ? H4D_OK : H4D_ECUDA;
}

// ---- forward + backward of 16-row tiles -------------------------------------------------
// Row r is record r/2, species r%2 (0 = cation row, 1 = anion row); feat is [rows][96],
// tgt [rows].  Outputs (bf16, transposed [unit][rows_pad] so the weight-gradient GEMMs
// read contiguous k pairs): xT, h1T, h2T, dz1T, dz2T, dlT (rows 0..1 of 8), and the
// per-row loss.
__device__ __forceinline__ void st_bf16(uint16_t* p, float v) { *p = (uint16_t)(pack_bf16(v, 0.f) & 0xffffu); }

// store the bf16 pairs of an A fragment (rows r0, r1; columns c, c+1) transposed
__device__ __forceinline__ void st_pairT(uint16_t* T, int rows_pad, int c, int r0, int r1, unsigned lo, unsigned hi) {
  T[(size_t)c * rows_pad + r0] = (uint16_t)(lo & 0xffffu);
  T[(size_t)(c + 1) * rows_pad + r0] = (uint16_t)(lo >> 16);
  T[(size_t)c * rows_pad + r1] = (uint16_t)(hi & 0xffffu);
  T[(size_t)(c + 1) * rows_pad + r1] = (uint16_t)(hi >> 16);
}

__global__ void __launch_bounds__(128) prop_fwd_bwd_kernel(PropNet net, const float* __restrict__ feat,
                                                          const float* __restrict__ tgt, int rows, float inv_n,
                                                          uint16_t* xT, uint16_t* h1T, uint16_t* dz1T,
                                                          uint16_t* h2T, uint16_t* dz2T, uint16_t* dlT,
                                                          float* loss_rows, int rows_pad) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int tile = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int r0 = 16 * tile + g, r1 = r0 + 8;
  if (16 * tile >= rows_pad) return;
  const bool v0 = r0 < rows, v1 = r1 < rows;
  // ---- layer 1 ----
  float acc1[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc1[i][0] = acc1[i][1] = acc1[i][2] = acc1[i][3] = 0.f;
#pragma unroll
  for (int ks = 0; ks < 6; ++ks) {
    const int k = 16 * ks + 2 * t;
    const float2 z2 = make_float2(0.f, 0.f);
    const float2 f00 = v0 ? *reinterpret_cast<const float2*>(feat + (size_t)r0 * 96 + k) : z2;
    const float2 f10 = v1 ? *reinterpret_cast<const float2*>(feat + (size_t)r1 * 96 + k) : z2;
    const float2 f01 = v0 ? *reinterpret_cast<const float2*>(feat + (size_t)r0 * 96 + k + 8) : z2;
    const float2 f11 = v1 ? *reinterpret_cast<const float2*>(feat + (size_t)r1 * 96 + k + 8) : z2;
    unsigned a[4] = {pack_bf16(f00.x, f00.y), pack_bf16(f10.x, f10.y), pack_bf16(f01.x, f01.y),
                     pack_bf16(f11.x, f11.y)};
    st_pairT(xT, rows_pad, k, r0, r1, a[0], a[1]);
    st_pairT(xT, rows_pad, k + 8, r0, r1, a[2], a[3]);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) mma_bf16(acc1[nt], a, net.w1[(ks * 8 + nt) * 32 + lane]);
  }
  unsigned mask1 = 0;  // bit 4*nt + e: pre-activation > 0
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float b0 = net.b[8 * nt + 2 * t], b1 = net.b[8 * nt + 2 * t + 1];
    acc1[nt][0] += b0; acc1[nt][1] += b1; acc1[nt][2] += b0; acc1[nt][3] += b1;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (acc1[nt][e] > 0.f) mask1 |= 1u << (4 * nt + e);
      else acc1[nt][e] = 0.f;
    }
  }
  unsigned a2[4][4];
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) c_to_a(acc1[2 * ks], acc1[2 * ks + 1], a2[ks]);
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
    st_pairT(h1T, rows_pad, 8 * nt + 2 * t, r0, r1, a2[nt >> 1][(nt & 1) * 2], a2[nt >> 1][(nt & 1) * 2 + 1]);
  // ---- layer 2 ----
  float acc2[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc2[i][0] = acc2[i][1] = acc2[i][2] = acc2[i][3] = 0.f;
#pragma unroll
  for (int ks = 0; ks < 4; ++ks)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) mma_bf16(acc2[nt], a2[ks], net.w2[(ks * 8 + nt) * 32 + lane]);
  unsigned mask2 = 0;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float b0 = net.b[64 + 8 * nt + 2 * t], b1 = net.b[64 + 8 * nt + 2 * t + 1];
    acc2[nt][0] += b0; acc2[nt][1] += b1; acc2[nt][2] += b0; acc2[nt][3] += b1;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (acc2[nt][e] > 0.f) mask2 |= 1u << (4 * nt + e);
      else acc2[nt][e] = 0.f;
    }
  }
  unsigned a3[4][4];
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) c_to_a(acc2[2 * ks], acc2[2 * ks + 1], a3[ks]);
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
    st_pairT(h2T, rows_pad, 8 * nt + 2 * t, r0, r1, a3[nt >> 1][(nt & 1) * 2], a3[nt >> 1][(nt & 1) * 2 + 1]);
  // ---- layer 3, loss and dL/dlogit ----
  float lg[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) mma_bf16(lg, a3[ks], net.w3[ks * 32 + lane]);
  const int s = r0 & 1;  // rows g and g+8 have the same species
  float dl0 = 0.f, dl1 = 0.f;
  if (t == 0) {
    const float b3 = net.b[128 + s];
    const float l0 = (s ? lg[1] : lg[0]) + b3, l1 = (s ? lg[3] : lg[2]) + b3;
    const float t0 = v0 ? tgt[r0] : 0.f, t1 = v1 ? tgt[r1] : 0.f;
    dl0 = v0 ? (1.f / (1.f + expf(-l0)) - t0) * inv_n : 0.f;
    dl1 = v1 ? (1.f / (1.f + expf(-l1)) - t1) * inv_n : 0.f;
    loss_rows[r0] = v0 ? fmaxf(l0, 0.f) - l0 * t0 + log1pf(expf(-fabsf(l0))) : 0.f;
    loss_rows[r1] = v1 ? fmaxf(l1, 0.f) - l1 * t1 + log1pf(expf(-fabsf(l1))) : 0.f;
    st_bf16(dlT + (size_t)s * rows_pad + r0, dl0);
    st_bf16(dlT + (size_t)s * rows_pad + r1, dl1);
    st_bf16(dlT + (size_t)(1 - s) * rows_pad + r0, 0.f);
    st_bf16(dlT + (size_t)(1 - s) * rows_pad + r1, 0.f);
  }
  dl0 = __shfl_sync(0xffffffffu, dl0, lane & ~3);
  dl1 = __shfl_sync(0xffffffffu, dl1, lane & ~3);
  // the backward pass uses dL/dlogit rounded to bf16, as the weight-gradient GEMM does
  dl0 = bf16_lo(pack_bf16(dl0, 0.f));
  dl1 = bf16_lo(pack_bf16(dl1, 0.f));
  // ---- dz2 = (dl W3^T) * [z2 > 0] ----
  float dz2[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int c = 8 * nt + 2 * t;
    const float w0 = net.w3r[c * 2 + s], w1 = net.w3r[(c + 1) * 2 + s];
    dz2[nt][0] = (mask2 >> (4 * nt + 0) & 1) ? dl0 * w0 : 0.f;
    dz2[nt][1] = (mask2 >> (4 * nt + 1) & 1) ? dl0 * w1 : 0.f;
    dz2[nt][2] = (mask2 >> (4 * nt + 2) & 1) ? dl1 * w0 : 0.f;
    dz2[nt][3] = (mask2 >> (4 * nt + 3) & 1) ? dl1 * w1 : 0.f;
  }
  unsigned ad[4][4];
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) c_to_a(dz2[2 * ks], dz2[2 * ks + 1], ad[ks]);
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
    st_pairT(dz2T, rows_pad, 8 * nt + 2 * t, r0, r1, ad[nt >> 1][(nt & 1) * 2], ad[nt >> 1][(nt & 1) * 2 + 1]);
  // ---- dz1 = (dz2 W2^T) * [z1 > 0] ----
  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
#pragma unroll
  for (int ks = 0; ks < 4; ++ks)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) mma_bf16(acc[nt], ad[ks], net.w2t[(ks * 8 + nt) * 32 + lane]);
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (!(mask1 >> (4 * nt + e) & 1)) acc[nt][e] = 0.f;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
    st_pairT(dz1T, rows_pad, 8 * nt + 2 * t, r0, r1, pack_bf16(acc[nt][0], acc[nt][1]),
             pack_bf16(acc[nt][2], acc[nt][3]));
}

int launch_prop_fwd_bwd(const PropNet& net, const float* feat, const float* tgt, int n_rec, float inv_n,
                        uint16_t* xT, uint16_t* h1T, uint16_t* dz1T, uint16_t* h2T, uint16_t* dz2T,
                        uint16_t* dlT, float* loss_rows, int rows_pad, void* stream) {
  const int tiles = rows_pad / 16;
  prop_fwd_bwd_kernel<<<(tiles + 3) / 4, 128, 0, (cudaStream_t)stream>>>(
      net, feat, tgt, 2 * n_rec, inv_n, xT, h1T, dz1T, h2T, dz2T, dlT, loss_rows, rows_pad);
  return cudaGetLastError() == cudaSuccess ? H4D_OK : H4D_ECUDA;
}

// ---- weight gradients: dW = A^T B over the batch rows ------------------------------------
// Warp tasks: 0..47 dW1 = X^T dz1 (6 x 8 tiles), 48..79 dW2 = h1^T dz2 (4 x 8), 80..83
// dW3 = h2^T dl (4 x 1), 84 db1, 85 db2, 86 db3 and the loss.  Each task sums its rows in
// order.
__device__ __forceinline__ unsigned ld_pair(const uint16_t* base, size_t row, int rows_pad, int k) {
  return *reinterpret_cast<const unsigned*>(base + row * rows_pad + k);
}

__global__ void __launch_bounds__(128) prop_wgrad_kernel(const uint16_t* __restrict__ xT,
                                                        const uint16_t* __restrict__ h1T,
                                                        const uint16_t* __restrict__ dz1T,
                                                        const uint16_t* __restrict__ h2T,
                                                        const uint16_t* __restrict__ dz2T,
                                                        const uint16_t* __restrict__ dlT,
                                                        const float* __restrict__ loss_rows, int rows_pad,
                                                        float* grad, double* loss) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int task = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (task < 84) {
    const uint16_t *A, *B;
    int mt, nt, ldo, off, ncols;
    if (task < 48) { A = xT; B = dz1T; mt = task >> 3; nt = task & 7; ldo = 64; off = 0; ncols = 64; }
    else if (task < 80) { A = h1T; B = dz2T; mt = (task - 48) >> 3; nt = (task - 48) & 7; ldo = 64; off = kPropOffW2; ncols = 64; }
    else { A = h2T; B = dlT; mt = task - 80; nt = 0; ldo = 2; off = kPropOffW3; ncols = 2; }
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const size_t ra = 16 * mt + g, rb = 8 * nt + g;
    for (int k0 = 0; k0 < rows_pad; k0 += 16) {
      const int k = k0 + 2 * t;
      unsigned a[4] = {ld_pair(A, ra, rows_pad, k), ld_pair(A, ra + 8, rows_pad, k), ld_pair(A, ra, rows_pad, k + 8),
                       ld_pair(A, ra + 8, rows_pad, k + 8)};
      const uint2 b = make_uint2(ld_pair(B, rb, rows_pad, k), ld_pair(B, rb, rows_pad, k + 8));
      mma_bf16(acc, a, b);
    }
    const int c = 8 * nt + 2 * t;
    if (c < ncols) {
      grad[off + (16 * mt + g) * ldo + c] = acc[0];
      grad[off + (16 * mt + g + 8) * ldo + c] = acc[2];
    }
    if (c + 1 < ncols) {
      grad[off + (16 * mt + g) * ldo + c + 1] = acc[1];
      grad[off + (16 * mt + g + 8) * ldo + c + 1] = acc[3];
    }
  } else if (task < 86) {
    const uint16_t* D = task == 84 ? dz1T : dz2T;
    const int off = task == 84 ? kPropOffB1 : kPropOffB2;
    for (int j = lane; j < 64; j += 32) {
      float s = 0.f;
      for (int r = 0; r < rows_pad; ++r) s += __uint_as_float((unsigned)D[(size_t)j * rows_pad + r] << 16);
      grad[off + j] = s;
    }
  } else if (task == 86) {
    if (lane < 2) {
      float s = 0.f;
      for (int r = 0; r < rows_pad; ++r) s += __uint_as_float((unsigned)dlT[(size_t)lane * rows_pad + r] << 16);
      grad[kPropOffB3 + lane] = s;
    } else if (lane == 2) {
      double s = 0.0;
      for (int r = 0; r < rows_pad; ++r) s += (double)loss_rows[r];
      *loss = s;
    }
  }
}

int launch_prop_wgrad(const uint16_t* xT, const uint16_t* h1T, const uint16_t* dz1T, const uint16_t* h2T,
                      const uint16_t* dz2T, const uint16_t* dlT, const float* loss_rows, int rows_pad,
                      float* grad, double* loss, void* stream) {
  prop_wgrad_kernel<<<(87 + 3) / 4, 128, 0, (cudaStream_t)stream>>>(xT, h1T, dz1T, h2T, dz2T, dlT, loss_rows,
                                                                   rows_pad, grad, loss);
  return cudaGetLastError() == cudaSuccess ? H4D_OK : H4D_ECUDA;
}

// ---- Adam (Kingma and Ba, 2015) on the FP32 masters ---------------------------------------
__global__ void prop_adam_kernel(float* w, float* m, float* v, const float* __restrict__ grad, float c1, float c2,
                                 float lr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kPropNW) return;
  const float gi = grad[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
}

int launch_prop_adam(float* w, float* m, float* v, const float* grad, int step, float lr, void* stream) {
  const float c1 = (float)(1.0 / (1.0 - pow(0.9, step)));
  const float c2 = (float)(1.0 / (1.0 - pow(0.999, step)));
  prop_adam_kernel<<<(kPropNW + 255) / 256, 256, 0, (cudaStream_t)stream>>>(w, m, v, grad, c1, c2, lr);
  return cudaGetLastError() == cudaSuccess ? H4D_OK : H4D_ECUDA;
}

// ---- valid records, in ring order: status 0 and a finite exponent -------------------------
__global__ void __launch_bounds__(1024) prop_compact_kernel(const int2* __restrict__ meta,
                                                           const double* __restrict__ y, int n_rec, int* valid,
                                                           int* n_valid) {
  __shared__ int warp_tot[32];
  __shared__ int base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c0 = 0; c0 < n_rec; c0 += 1024) {
    const int i = c0 + threadIdx.x;
    const bool ok = i < n_rec && meta[i].y == 0 && isfinite(y[i]);
    const unsigned bal = __ballot_sync(0xffffffffu, ok);
    if (lane == 0) warp_tot[warp] = __popc(bal);
    __syncthreads();
    int off = base;
    for (int w = 0; w < warp; ++w) off += warp_tot[w];
    off += __popc(bal & ((1u << lane) - 1u));
    if (ok) valid[off] = i;
    __syncthreads();
    if (threadIdx.x == 0) {
      int s = 0;
      for (int w = 0; w < 32; ++w) s += warp_tot[w];
      base += s;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *n_valid = base;
}

int launch_prop_compact(const int2* meta, const double* y, int n_rec, int* valid, int* n_valid, void* stream) {
  prop_compact_kernel<<<1, 1024, 0, (cudaStream_t)stream>>>(meta, y, n_rec, valid, n_valid);
  return cudaGetLastError() == cudaSuccess ? H4D_OK : H4D_ECUDA;
}

// ---- minibatch gather ---------------------------------------------------------------------
// Record b of the batch is valid[pick(draw)] with draw word b%4 of Philox counter
// {step, b/4, kPurTrain, 0} under key {seed, kTrainKey}; with n_batch >= n_valid the batch
// is every valid record in order.  feat [n][2][96], tgt [n][2] = min(1, exp(y - y0)).
__global__ void prop_gather_kernel(const float* __restrict__ rec_feat, const double* __restrict__ rec_y,
                                   const int* __restrict__ valid, int n_valid, int n_batch, u64 seed,
                                   long long step, float y0, float* feat, float* tgt) {
  const int b = blockIdx.x;
  if (b >= n_batch || n_valid <= 0) return;
  int idx;
  if (n_batch >= n_valid) {
    if (b >= n_valid) return;
    idx = valid[b];
  } else {
    u64 r[4];
    draw4(seed, kTrainKey, (u64)step, (u64)(b >> 2), kPurTrain, r);
    idx = valid[pick_index(r[b & 3], n_valid)];
  }
  for (int k = threadIdx.x; k < 192; k += blockDim.x) feat[(size_t)b * 192 + k] = rec_feat[(size_t)idx * 192 + k];
  if (threadIdx.x < 2) tgt[2 * b + threadIdx.x] = (float)exp(fmin(rec_y[idx] - (double)y0, 0.0));
}

int launch_prop_gather(const float* rec_feat, const double* rec_y, const int* valid, int n_valid, int n_batch,
                       unsigned long long seed, long long step, float y0, float* feat, float* tgt, void* stream) {
  if (n_batch <= 0) return H4D_OK;
  prop_gather_kernel<<<n_batch, 64, 0, (cudaStream_t)stream>>>(rec_feat, rec_y, valid, n_valid, n_batch, seed, step,
                                                               y0, feat, tgt);
  return cudaGetLastError() == cudaSuccess ? H4D_OK : H4D_ECUDA;
}

}  // namespace h4d
