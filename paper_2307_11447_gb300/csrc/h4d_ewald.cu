// h4d_ewald.cu -- long-range Coulomb term of Sec. II.B.2 (Eqs. 9-10): the reciprocal-space
// Ewald sum and the self energy of one configuration, scaled by the altitude screening
// g^lr(wbar) = exp(-kappa_lr wbar).  Two passes, both O(k-vectors x atoms), each a kernel
// over (k-vectors or atoms) x chunks of the other axis sized to fill the GPU, and an
// ordered reduction of the chunk partials:
//   - structure factor: S(k) = sum_j q_j exp(i k.r_j) for every k of one half space;
//   - forces: F_j = g (8 pi K q_j / V) sum_half A_k k [Re S sin(k.r_j) - Im S cos(k.r_j)].
// The phase k.r_j / 2 pi = (n_x X_j + n_y Y_j + n_z Z_j) / 2^32 is formed exactly in 32-bit
// integer arithmetic from the fixed-point coordinates X = round(x/L 2^32) (wrap-around is
// the periodicity); its conversion to a float in [-1, 1) half turns is the only rounding
// of the argument (at most 2^-24 of a half turn), whatever the size of k.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/h4d.h"

namespace {

constexpr int kTile = 256;  // atoms (or k-vectors) staged in shared memory per step

struct KVec {
  int nx, ny, nz;
  float pad;
};

// The grids cover the GPU: the k-vectors (or atoms) of a block times chunks of the other
// axis, each chunk a whole number of 256-wide tiles; every block writes its chunk's partial
// sums, and a second kernel adds the chunks in chunk order (a fixed order: the result does
// not depend on scheduling).  Within a chunk each tile's terms are summed in FP32 and added
// to FP64 partials.
constexpr int kBlocksTarget = 152 * 8;  // 8 resident 256-thread blocks on each of 152 SMs

// S(k) partials: thread t of block (bx, c) owns k-vector bx*256 + t and the atoms of chunk c
__global__ void __launch_bounds__(256) ewald_sk_kernel(const uint4* __restrict__ xq, int n, const KVec* __restrict__ kv,
                                                       int nk, int chunk_atoms, double2* __restrict__ part) {
  __shared__ uint4 tile[kTile];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const KVec kk = (k < nk) ? kv[k] : KVec{0, 0, 0, 0.f};
  const int a0 = blockIdx.y * chunk_atoms, a1 = min(n, a0 + chunk_atoms);
  double re = 0.0, im = 0.0;
  for (int t0 = a0; t0 < a1; t0 += kTile) {
    const int m = min(kTile, a1 - t0);
    __syncthreads();
    for (int a = threadIdx.x; a < m; a += blockDim.x) tile[a] = xq[t0 + a];
    __syncthreads();
    float fr = 0.f, fi = 0.f;
    for (int a = 0; a < m; ++a) {
      const uint4 p = tile[a];
      const unsigned ph = (unsigned)kk.nx * p.x + (unsigned)kk.ny * p.y + (unsigned)kk.nz * p.z;
      float s, c;
      sincospif((float)(int)ph * 4.656612873077393e-10f, &s, &c);  // 2 pi ph / 2^32 = pi (int)ph / 2^31
      const float q = __uint_as_float(p.w);
      fr = fmaf(q, c, fr);
      fi = fmaf(q, s, fi);
    }
    re += (double)fr;
    im += (double)fi;
  }
  if (k < nk) part[(size_t)blockIdx.y * nk + k] = make_double2(re, im);
}

__global__ void ewald_sk_reduce(const double2* __restrict__ part, int nk, int n_chunks, double2* __restrict__ sk) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nk) return;
  double re = 0.0, im = 0.0;
  for (int c = 0; c < n_chunks; ++c) {
    const double2 v = part[(size_t)c * nk + k];
    re += v.x;
    im += v.y;
  }
  sk[k] = make_double2(re, im);
}

// forces: thread t of block (bx, c) owns atom bx*256 + t and the k-vectors of chunk c; the
// k-vectors and their weighted structure factors (A_k Re S, A_k Im S) are staged in tiles
struct KW {
  int nx, ny, nz;
  float pad;
  float ar, ai;  // A_k Re S(k), A_k Im S(k)
  float pad2, pad3;
};

__global__ void __launch_bounds__(256) ewald_force_kernel(const uint4* __restrict__ xq, int n, const KW* __restrict__ kw,
                                                          int nk, int chunk_k, double* __restrict__ part) {
  __shared__ KW tile[kTile];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const uint4 p = (j < n) ? xq[j] : make_uint4(0u, 0u, 0u, 0u);
  const int k0 = blockIdx.y * chunk_k, k1 = min(nk, k0 + chunk_k);
  double gx = 0.0, gy = 0.0, gz = 0.0;
  for (int t0 = k0; t0 < k1; t0 += kTile) {
    const int m = min(kTile, k1 - t0);
    __syncthreads();
    for (int a = threadIdx.x; a < m; a += blockDim.x) tile[a] = kw[t0 + a];
    __syncthreads();
    float fx = 0.f, fy = 0.f, fz = 0.f;
    for (int a = 0; a < m; ++a) {
      const KW w = tile[a];
      const unsigned ph = (unsigned)w.nx * p.x + (unsigned)w.ny * p.y + (unsigned)w.nz * p.z;
      float s, c;
      sincospif((float)(int)ph * 4.656612873077393e-10f, &s, &c);
      const float f = fmaf(w.ar, s, -w.ai * c);  // A_k [Re S sin - Im S cos]
      fx = fmaf(f, (float)w.nx, fx);
      fy = fmaf(f, (float)w.ny, fy);
      fz = fmaf(f, (float)w.nz, fz);
    }
    gx += (double)fx;
    gy += (double)fy;
    gz += (double)fz;
  }
  if (j < n) {
    double* o = part + ((size_t)blockIdx.y * n + j) * 3;
    o[0] = gx;
    o[1] = gy;
    o[2] = gz;
  }
}

__global__ void ewald_force_reduce(const uint4* __restrict__ xq, const double* __restrict__ part, int n,
                                   int n_chunks, float two_pi_over_L, double pref, double* __restrict__ F) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double gx = 0.0, gy = 0.0, gz = 0.0;
  for (int c = 0; c < n_chunks; ++c) {
    const double* o = part + ((size_t)c * n + j) * 3;
    gx += o[0];
    gy += o[1];
    gz += o[2];
  }
  const double qj = (double)__uint_as_float(xq[j].w);
  const double cc = pref * qj * (double)two_pi_over_L;  // k = (2 pi / L) n
  F[3 * j] = cc * gx;
  F[3 * j + 1] = cc * gy;
  F[3 * j + 2] = cc * gz;
}

// chunks of the second axis (whole 256-wide tiles) so that blocks x chunks covers the GPU
__host__ inline void chunking(int n_first, int n_second, int* chunk, int* n_chunks) {
  const int blocks = (n_first + 255) / 256;
  const int tiles = (n_second + 255) / 256;
  int want = (kBlocksTarget + blocks - 1) / blocks;
  if (want < 1) want = 1;
  if (want > tiles) want = tiles > 0 ? tiles : 1;
  const int tiles_per_chunk = (tiles + want - 1) / want;
  *chunk = tiles_per_chunk * 256;
  *n_chunks = (n_second + *chunk - 1) / *chunk;
  if (*n_chunks < 1) *n_chunks = 1;
}

int type_of_host(int a, int nw3) { return a < nw3 ? ((a % 3 == 0) ? 2 : 3) : ((a - nw3) & 1); }

}  // namespace

#define CKE(x)                       \
  do {                               \
    if ((x) != cudaSuccess) {        \
      rc = H4D_ECUDA;                \
      goto done;                     \
    }                                \
  } while (0)

extern "C" int h4d_ewald_lr(const h4d_params* params, double L, int32_t n_water, int32_t n, const double* x,
                            double alpha, int32_t kmax, double wbar, double kappa_lr, double* U_recip,
                            double* U_self, double* F, double* t_kernel_ms) {
  if (!params || !x || n < 0 || n_water < 0 || 3 * n_water > n || !(L > 0) || !(alpha > 0) || kmax < 1 ||
      kmax > 64 || !(wbar >= 0) || !(kappa_lr >= 0))
    return H4D_EINVAL;
  const int single = params->exchange == H4D_EXCHANGE_SINGLE;
  const int nw3 = 3 * n_water;
  const double K = params->kcoul, V = L * L * L;
  const double g = std::exp(-kappa_lr * wbar);  // Eq. 10
  // atoms: fixed-point coordinates and charges
  std::vector<uint4> xq(n > 0 ? n : 1);
  double qq = 0.0;
  for (int a = 0; a < n; ++a) {
    const int t = single && a >= nw3 ? 0 : type_of_host(a, nw3);
    const float q = (float)params->q[t];
    qq += (double)params->q[t] * params->q[t];
    uint32_t X[3];
    for (int d = 0; d < 3; ++d) {
      double y = x[3 * a + d] - L * std::floor(x[3 * a + d] / L);
      double s = std::nearbyint(y / L * 4294967296.0);
      X[d] = (uint32_t)((uint64_t)s & 0xffffffffULL);
    }
    uint32_t qb;
    std::memcpy(&qb, &q, 4);
    xq[a] = make_uint4(X[0], X[1], X[2], qb);
  }
  // half space of k-vectors: n_x > 0, or n_x = 0 and n_y > 0, or n_x = n_y = 0 and n_z > 0
  std::vector<KVec> kv;
  std::vector<double> A;
  for (int nx = 0; nx <= kmax; ++nx)
    for (int ny = -kmax; ny <= kmax; ++ny)
      for (int nz = -kmax; nz <= kmax; ++nz) {
        if (nx == 0 && (ny < 0 || (ny == 0 && nz <= 0))) continue;
        const double kx = 2.0 * M_PI * nx / L, ky = 2.0 * M_PI * ny / L, kz = 2.0 * M_PI * nz / L;
        const double k2 = kx * kx + ky * ky + kz * kz;
        kv.push_back(KVec{nx, ny, nz, 0.f});
        A.push_back(std::exp(-k2 / (4.0 * alpha * alpha)) / k2);
      }
  const int nk = (int)kv.size();
  int rc = H4D_OK;
  uint4* d_xq = nullptr;
  KVec* d_kv = nullptr;
  double2* d_sk = nullptr;
  KW* d_kw = nullptr;
  double* d_F = nullptr;
  double2* d_psk = nullptr;  // S(k) partials per atom chunk
  double* d_pF = nullptr;    // force partials per k-vector chunk
  int chunk_a = 0, nch_a = 0, chunk_k = 0, nch_k = 0;
  chunking(nk, n, &chunk_a, &nch_a);
  chunking(n, nk, &chunk_k, &nch_k);
  std::vector<double2> sk(nk);
  std::vector<KW> kw(nk);
  double u = 0.0;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  float ms_sk = 0.f, ms_f = 0.f;
  if (t_kernel_ms) *t_kernel_ms = 0.0;
  if (n == 0) {
    if (U_recip) *U_recip = 0.0;
    if (U_self) *U_self = 0.0;
    return H4D_OK;
  }
  for (auto& x_ev : ev) CKE(cudaEventCreate(&x_ev));
  CKE(cudaMalloc(&d_xq, sizeof(uint4) * n));
  CKE(cudaMalloc(&d_kv, sizeof(KVec) * nk));
  CKE(cudaMalloc(&d_sk, sizeof(double2) * nk));
  CKE(cudaMalloc(&d_psk, sizeof(double2) * nk * (size_t)nch_a));
  CKE(cudaMemcpy(d_xq, xq.data(), sizeof(uint4) * n, cudaMemcpyHostToDevice));
  CKE(cudaMemcpy(d_kv, kv.data(), sizeof(KVec) * nk, cudaMemcpyHostToDevice));
  CKE(cudaEventRecord(ev[0]));
  ewald_sk_kernel<<<dim3((nk + 255) / 256, nch_a), 256>>>(d_xq, n, d_kv, nk, chunk_a, d_psk);
  CKE(cudaGetLastError());
  ewald_sk_reduce<<<(nk + 255) / 256, 256>>>(d_psk, nk, nch_a, d_sk);
  CKE(cudaGetLastError());
  CKE(cudaEventRecord(ev[1]));
  CKE(cudaMemcpy(sk.data(), d_sk, sizeof(double2) * nk, cudaMemcpyDeviceToHost));
  // U_recip = (2 pi K / V) sum_{all k != 0} A_k |S_k|^2 = (4 pi K / V) sum_half A_k |S_k|^2
  for (int k = 0; k < nk; ++k) {
    u += A[k] * (sk[k].x * sk[k].x + sk[k].y * sk[k].y);
    kw[k] = KW{kv[k].nx, kv[k].ny, kv[k].nz, 0.f, (float)(A[k] * sk[k].x), (float)(A[k] * sk[k].y), 0.f, 0.f};
  }
  if (U_recip) *U_recip = g * 4.0 * M_PI * K / V * u;
  if (U_self) *U_self = -g * K * alpha / std::sqrt(M_PI) * qq;
  if (F) {
    CKE(cudaMalloc(&d_kw, sizeof(KW) * nk));
    CKE(cudaMalloc(&d_F, sizeof(double) * 3 * n));
    CKE(cudaMalloc(&d_pF, sizeof(double) * 3 * n * (size_t)nch_k));
    CKE(cudaMemcpy(d_kw, kw.data(), sizeof(KW) * nk, cudaMemcpyHostToDevice));
    // F_j = g (4 pi K q_j / V) sum_{all k} A_k k [Re S sin - Im S cos]: twice the half space
    CKE(cudaEventRecord(ev[2]));
    ewald_force_kernel<<<dim3((n + 255) / 256, nch_k), 256>>>(d_xq, n, d_kw, nk, chunk_k, d_pF);
    CKE(cudaGetLastError());
    ewald_force_reduce<<<(n + 255) / 256, 256>>>(d_xq, d_pF, n, nch_k, (float)(2.0 * M_PI / L),
                                                 g * 8.0 * M_PI * K / V, d_F);
    CKE(cudaGetLastError());
    CKE(cudaEventRecord(ev[3]));
    CKE(cudaMemcpy(F, d_F, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost));
    CKE(cudaEventElapsedTime(&ms_f, ev[2], ev[3]));
  }
  CKE(cudaEventElapsedTime(&ms_sk, ev[0], ev[1]));
  if (t_kernel_ms) *t_kernel_ms = (double)ms_sk + (double)ms_f;
done:
  for (auto& x_ev : ev)
    if (x_ev) cudaEventDestroy(x_ev);
  cudaFree(d_xq);
  cudaFree(d_kv);
  cudaFree(d_sk);
  cudaFree(d_kw);
  cudaFree(d_F);
  cudaFree(d_psk);
  cudaFree(d_pF);
  return rc;
}
