// FP32 plain form of the dense step (3-mode tensors): Step (I) of Algorithm 1 with L^(k)
// materialised by the literal chain of Eq. (L=CUR),
//   L = R x_3 A_3 x_2 A_2 x_1 A_1,   A_i = C_i U_i^+ = B_i Q_i^T  (d_i x m_i),
// in FP32 FMA (three GEMM stages, about 2 d^3 m flops at d = 800, m = 101), then a separate
// thresholding pass over X and L. It is the unfused, unfactored reference the fused forms are
// measured against; it runs on the same graph branch as the fused pass would.
//
// The chain uses the Fiber CUR pieces of the previous iteration (R^(k), A_i^(k)), snapshot at
// the end of each iteration into copy (k+1) & 1 so the concurrent sampled chain can overwrite
// the live buffers.
#include "rtcur_internal.cuh"

namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16;

// C[b] (M x N, row-major, ldc) = A[b] (M x K, row-major, lda) * Bm[b] where Bm(k, n) is read at
// B[b] + k * sbk + n * sbn (so a transposed operand needs no copy). 256 threads, 4x4 outputs
// per thread, 64x64 tiles staged in shared memory. A and B come in two copies (A0/A1, B0/B1);
// the copy used is the parity of the iteration counter read on the device (pass the same
// pointer twice for an operand that has one copy).
__global__ void __launch_bounds__(256) k_sgemm(const float* A0, const float* A1, const float* B0,
                                               const float* B1, const State* st,
                                               float* __restrict__ C, int M, int N, int K,
                                               long long lda, long long sbk, long long sbn,
                                               long long ldc, long long sA, long long sB,
                                               long long sC) {
  __shared__ float As[kBK][kBM + 4];
  __shared__ float Bs[kBK][kBN + 4];
  const int cp = st->k & 1;
  const float* __restrict__ A = cp ? A1 : A0;
  const float* __restrict__ B = cp ? B1 : B0;
  const int bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += kBK) {
    for (int e = threadIdx.x; e < kBM * kBK; e += 256) {
      int r = e / kBK, kk = e % kBK;
      int gm = m0 + r, gk = k0 + kk;
      As[kk][r] = (gm < M && gk < K) ? A[(long long)gm * lda + gk] : 0.f;
    }
    for (int e = threadIdx.x; e < kBK * kBN; e += 256) {
      int kk = e / kBN, c = e % kBN;
      int gk = k0 + kk, gn = n0 + c;
      Bs[kk][c] = (gk < K && gn < N) ? B[(long long)gk * sbk + (long long)gn * sbn] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      float a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gm = m0 + ty * 4 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gn = n0 + tx * 4 + j;
      if (gn < N) C[(long long)gm * ldc + gn] = acc[i][j];
    }
  }
}

// Snapshot for the next iteration: A_i = B_i Q_i^T (FP32 product, FP32 result) and R.
__global__ void k_plain_prep(Geom g, Bufs b) {
  const int nxt = (b.st->k + 1) & 1;
  const long long tot = g.sumDM + g.nR;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += stride) {
    if (e < g.sumDM) {
      int i = 0;
      while (i + 1 < g.n && e >= g.offDM[i + 1]) ++i;
      const long long local = e - g.offDM[i];
      const int m = g.m[i], r = g.r[i];
      const long long t = local / m;
      const int a = (int)(local - t * m);
      const float* Bi = b.B[nxt] + g.offB[i] + t * r;
      const double* Q = b.Qr + g.offQ[i] + (long long)a * r;
      float acc = 0.f;
      for (int c = 0; c < r; ++c) acc = fmaf(Bi[c], (float)Q[c], acc);
      b.Ap[nxt][e] = acc;
    } else {
      const long long j = e - g.sumDM;
      b.Rp[nxt][j] = b.XS[j];
    }
  }
}

__device__ __forceinline__ double block_sum_p(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
  return t;
}

// S = HT_{zeta^(k+1)}(X - L) from the materialised L, with the residual/nnz/band sums.
__global__ void __launch_bounds__(256) k_plain_ht(Geom g, Bufs b) {
  __shared__ double sh[8];
  const State* st = b.st;
  const double zeta = g.gamma * st->zeta;
  const float zf = (float)zeta;
  const float band = (float)(g.inband * zeta);
  const float4* X4 = reinterpret_cast<const float4*>(b.sp->X);
  const float4* L4 = reinterpret_cast<const float4*>(b.Lplain);
  float4* S4 = reinterpret_cast<float4*>(b.sp->S);
  const long long n4 = g.N >> 2;
  float res = 0.f;
  unsigned nnz = 0u, inb = 0u;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n4; e += stride) {
    float4 x = __ldcs(X4 + e), l = __ldcs(L4 + e), sv;
    float xs[4] = {x.x, x.y, x.z, x.w}, ls[4] = {l.x, l.y, l.z, l.w}, ss[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      float dl = xs[u] - ls[u];
      float ad = fabsf(dl);
      bool keep = ad > zf;
      ss[u] = keep ? dl : 0.f;
      res = keep ? res : fmaf(dl, dl, res);
      nnz += keep ? 1u : 0u;
      inb += (fabsf(ad - zf) <= band) ? 1u : 0u;
    }
    sv = make_float4(ss[0], ss[1], ss[2], ss[3]);
    __stcs(S4 + e, sv);
  }
  double* part = b.red + (size_t)TK_DENSE * 1024 * RT_RED_SLOTS;
  double t0 = block_sum_p((double)res, sh);
  if (threadIdx.x == 0) part[blockIdx.x * RT_RED_SLOTS + 0] = t0;
  t0 = block_sum_p((double)nnz, sh);
  if (threadIdx.x == 0) part[blockIdx.x * RT_RED_SLOTS + 1] = t0;
  t0 = block_sum_p((double)inb, sh);
  if (threadIdx.x == 0) part[blockIdx.x * RT_RED_SLOTS + 2] = t0;
  if (last_block_arrive(b.ticket + TK_DENSE)) {
    State* w = b.st;
    for (int slot = 0; slot < 3; ++slot) {
      double acc = 0.0;
      for (unsigned i2 = threadIdx.x; i2 < gridDim.x; i2 += blockDim.x) acc += part[i2 * RT_RED_SLOTS + slot];
      acc = block_sum_p(acc, sh);
      if (threadIdx.x == 0) {
        if (slot == 0) w->resid_f = acc;
        if (slot == 1) w->nnz_f = (long long)acc;
        if (slot == 2) w->inband_f = (long long)acc;
      }
    }
    if (threadIdx.x == 0) b.ticket[TK_DENSE] = 0u;
  }
}

inline dim3 gemm_grid(int M, int N, int batch) {
  return dim3((unsigned)((N + kBN - 1) / kBN), (unsigned)((M + kBM - 1) / kBM), (unsigned)batch);
}

}  // namespace

cudaError_t launch_plain_prep(const Geom& g, const Bufs& b, cudaStream_t s) {
  long long tot = g.sumDM + g.nR;
  int blocks = (int)((tot + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  k_plain_prep<<<blocks, 256, 0, s>>>(g, b);
  return cudaGetLastError();
}

// Dense plain pass of iteration k (copy k & 1 of the chain inputs): Z1 = R x_3 A_3,
// Z2 = Z1 x_2 A_2, L = Z2 x_1 A_1 (three FP32 GEMM stages), then the HT pass.
cudaError_t launch_plain_dense(const Geom& g, const Bufs& b, cudaStream_t s) {
  const int d1 = (int)g.d[0], d2 = (int)g.d[1], d3 = (int)g.d[2];
  const int m1 = g.m[0], m2 = g.m[1], m3 = g.m[2];
  const float* A1[2] = {b.Ap[0] + g.offDM[0], b.Ap[1] + g.offDM[0]};
  const float* A2[2] = {b.Ap[0] + g.offDM[1], b.Ap[1] + g.offDM[1]};
  const float* A3[2] = {b.Ap[0] + g.offDM[2], b.Ap[1] + g.offDM[2]};
  // stage 1: Z1 (m1 m2 x d3) = R (m1 m2 x m3) * A3^T; A3^T(k, n) = A3[n * m3 + k]
  k_sgemm<<<gemm_grid(m1 * m2, d3, 1), 256, 0, s>>>(b.Rp[0], b.Rp[1], A3[0], A3[1], b.st, b.Z1p,
                                                     m1 * m2, d3, m3, m3, 1, m3, d3, 0, 0, 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // stage 2: for each a1, Z2[a1] (d2 x d3) = A2 (d2 x m2) * Z1[a1] (m2 x d3)
  k_sgemm<<<gemm_grid(d2, d3, m1), 256, 0, s>>>(A2[0], A2[1], b.Z1p, b.Z1p, b.st, b.Z2p, d2, d3, m2,
                                                  m2, d3, 1, d3, 0, (long long)m2 * d3,
                                                  (long long)d2 * d3);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // stage 3: L (d1 x d2 d3) = A1 (d1 x m1) * Z2 (m1 x d2 d3)
  const long long nn = (long long)d2 * d3;
  k_sgemm<<<gemm_grid(d1, (int)nn, 1), 256, 0, s>>>(A1[0], A1[1], b.Z2p, b.Z2p, b.st, b.Lplain, d1,
                                                     (int)nn, m1, m1, nn, 1, nn, 0, 0, 0);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_plain_ht<<<1024, 256, 0, s>>>(g, b);
  return cudaGetLastError();
}
