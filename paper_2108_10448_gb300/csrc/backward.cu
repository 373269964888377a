// Adjoint of K unrolled RTCUR iterations (rtcur_backward; 3-mode tensors).
//
// Forward (Algorithm 1, sampled S update of Eq. (partial S update), Fiber CUR update of
// Eq. (L=CUR)): at iteration k the sampled values are V = X - S on the subtensor and fiber slots,
// V_p = L^(k)(p) where the HT mask is set and X_p elsewhere; R = V(I_1, I_2, I_3),
// C_i = V_(i)(:, J_i), A_i = C_i P_i with P_i = U_i^+ = (SVD_r(W_i))^+, W_i = C_i(I_i, :), and
// L^(k+1) = R x_1 A_1 x_2 A_2 x_3 A_3. The forward records V and the masks of every iteration
// (the checkpoint); everything else is recomputed here in FP64.
//
// Reverse sweep, from the seed dL on L^(K):
//   R_bar = dL x_i A_i^T,  A_bar_i = dL_(i) (R x_{j != i} A_j)_(i)^T                (Tucker adjoint)
//   C_bar_i = A_bar_i P_i^T,  P_bar_i = C_i^T A_bar_i                                 (A_i = C_i P_i)
//   W_bar_i = Z P_bar^T + 2 M_bar W,  M_bar = U (F o (U^T sym(W P_bar) U)) U^T         (P = W^T Z)
//     with M = W W^T = U diag(lambda) U^T, Z = U_r diag(1/lambda_r) U_r^T and the
//     Daleckii-Krein divided differences F of f(lambda) = 1/lambda on the top r, 0 elsewhere;
//   C_bar_i(I_i, :) += W_bar_i;  the slot adjoint V_bar = (R_bar, C_bar_1..3);
//   dX += V_bar on unmasked slots; L^(k)_bar = V_bar on masked slots, and its adjoint through
//   the slot evaluations of L^(k) = R' x_i A'_i (subtensor: a Tucker adjoint with the rows
//   A'_i(I_i, :); fibers: A'_i z_j with z_j = R' x_{l != i} A'_l(p_l(j), :)) gives the
//   previous iteration's R_bar, A_bar.
// The FP64 eigenpairs of each M come from a parallel cyclic Jacobi (one CTA per matrix).
#include "rtcur_internal.cuh"

namespace {

constexpr int kT = 256;

// ------------------------------------------------------------------ generic contraction
struct Opnd {
  const void* p;
  int f64;                   // 1: double data, 0: float data
  long long sb, sx, sk1, sk2;  // strides: batch, own free index (i for A, j for B), k1, k2
};

__device__ __forceinline__ double ldv(const Opnd& o, long long off) {
  return o.f64 ? static_cast<const double*>(o.p)[off] : (double)static_cast<const float*>(o.p)[off];
}

// C[b, i, j] = alpha * sum_{k1, k2} A[b, i, k1, k2] B[b, k1, k2, j] + beta * C[b, i, j], FP64
// accumulation. blockIdx.y splits k1; with nsplit > 1 each split writes a partial sum instead.
__global__ void __launch_bounds__(kT) k_contract(Opnd A, Opnd B, double* C, long long csb,
                                                 long long csi, long long csj, int nb, int ni,
                                                 int nj, long long nk1, long long nk2, double alpha,
                                                 double beta, int nsplit, double* part) {
  const long long nout = (long long)nb * ni * nj;
  const long long o = (long long)blockIdx.x * kT + threadIdx.x;
  if (o >= nout) return;
  const int j = (int)(o % nj);
  const long long t = o / nj;
  const int i = (int)(t % ni);
  const int b = (int)(t / ni);
  const long long k1lo = nk1 * blockIdx.y / nsplit, k1hi = nk1 * (blockIdx.y + 1) / nsplit;
  const long long ab = b * A.sb + i * A.sx, bb = b * B.sb + j * B.sx;
  double acc = 0.0;
  for (long long k1 = k1lo; k1 < k1hi; ++k1)
    for (long long k2 = 0; k2 < nk2; ++k2)
      acc = fma(ldv(A, ab + k1 * A.sk1 + k2 * A.sk2), ldv(B, bb + k1 * B.sk1 + k2 * B.sk2), acc);
  if (nsplit > 1) {
    part[(long long)blockIdx.y * nout + o] = acc;
    return;
  }
  double* c = C + b * csb + i * csi + j * csj;
  *c = alpha * acc + (beta != 0.0 ? beta * *c : 0.0);
}

__global__ void k_contract_reduce(const double* part, int nsplit, double* C, long long csb,
                                  long long csi, long long csj, int nb, int ni, int nj,
                                  double alpha, double beta) {
  const long long nout = (long long)nb * ni * nj;
  const long long o = (long long)blockIdx.x * kT + threadIdx.x;
  if (o >= nout) return;
  double acc = 0.0;
  for (int s = 0; s < nsplit; ++s) acc += part[(long long)s * nout + o];  // fixed order
  const int j = (int)(o % nj);
  const long long t = o / nj;
  const int i = (int)(t % ni);
  const int b = (int)(t / ni);
  double* c = C + b * csb + i * csi + j * csj;
  *c = alpha * acc + (beta != 0.0 ? beta * *c : 0.0);
}

// One warp per output: the lanes split the contracted indices, then a fixed shuffle tree sums
// them (deterministic, one launch; for the many small products of the pinv adjoint).
__global__ void __launch_bounds__(256) k_contract_warp(Opnd A, Opnd B, double* C, long long csb,
                                                       long long csi, long long csj, int nb, int ni, int nj,
                                                       long long nk1, long long nk2, double alpha, double beta) {
  const long long nout = (long long)nb * ni * nj;
  const long long o = ((long long)blockIdx.x * 256 + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (o >= nout) return;  // uniform per warp
  const int j = (int)(o % nj);
  const long long t = o / nj;
  const int i = (int)(t % ni);
  const int b = (int)(t / ni);
  const long long ab = b * A.sb + i * A.sx, bb = b * B.sb + j * B.sx;
  const long long K = nk1 * nk2;
  double acc = 0.0;
  if (nk2 == 1) {
    for (long long k = lane; k < K; k += 32) acc = fma(ldv(A, ab + k * A.sk1), ldv(B, bb + k * B.sk1), acc);
  } else {
    for (long long k = lane; k < K; k += 32) {
      const long long k1 = k / nk2, k2 = k - k1 * nk2;
      acc = fma(ldv(A, ab + k1 * A.sk1 + k2 * A.sk2), ldv(B, bb + k1 * B.sk1 + k2 * B.sk2), acc);
    }
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) {
    double* c = C + b * csb + i * csi + j * csj;
    *c = alpha * acc + (beta != 0.0 ? beta * *c : 0.0);
  }
}

struct Ctx {
  double* part;
  long long partsz;
  cudaStream_t s;
};

cudaError_t contract(const Ctx& cx, const Opnd& A, const Opnd& B, double* C, long long csb,
                     long long csi, long long csj, int nb, int ni, int nj, long long nk1,
                     long long nk2, double alpha = 1.0, double beta = 0.0) {
  const long long nout = (long long)nb * ni * nj;
  if (nout == 0) return cudaSuccess;
  if (nk1 * nk2 >= 64 && nout <= (4LL << 20)) {
    k_contract_warp<<<(unsigned)((nout * 32 + 255) / 256), 256, 0, cx.s>>>(A, B, C, csb, csi, csj, nb, ni, nj,
                                                                          nk1, nk2, alpha, beta);
    return cudaGetLastError();
  }
  // few outputs: split the first contracted index so that enough threads run (each output is
  // an FP64 dot product; unsplit, a few thousand threads would run long serial chains)
  long long want = (2LL * 152 * 1024) / nout;
  int nsplit = (int)(want < 1 ? 1 : (want > nk1 ? nk1 : want));
  if (nsplit > 256) nsplit = 256;
  while (nsplit > 1 && (long long)nsplit * nout > cx.partsz) --nsplit;
  if (nsplit < 1) nsplit = 1;
  dim3 grid((unsigned)((nout + kT - 1) / kT), (unsigned)nsplit);
  k_contract<<<grid, kT, 0, cx.s>>>(A, B, C, csb, csi, csj, nb, ni, nj, nk1, nk2, alpha, beta,
                                     nsplit, cx.part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || nsplit == 1) return e;
  k_contract_reduce<<<(unsigned)((nout + kT - 1) / kT), kT, 0, cx.s>>>(cx.part, nsplit, C, csb, csi,
                                                                      csj, nb, ni, nj, alpha, beta);
  return cudaGetLastError();
}

inline Opnd opd(const void* p, int f64, long long sb, long long sx, long long sk1, long long sk2 = 0) {
  Opnd o;
  o.p = p;
  o.f64 = f64;
  o.sb = sb;
  o.sx = sx;
  o.sk1 = sk1;
  o.sk2 = sk2;
  return o;
}

// Tiled batched product for the large contractions: the same operand description as
// k_contract (one or two contracted indices), 64 x 64 output tiles, 16-deep K tiles staged in
// shared memory as FP32. Inner products run in FP32 within a K tile and are accumulated across
// K tiles in FP64 (relative error ~1e-6 however long K is). blockIdx.z = batch * nsplit + split.
constexpr int kGM = 64, kGN = 64, kGK = 16;

template <typename TA, typename TB, bool K2>
__global__ void __launch_bounds__(256) k_gemm_t(Opnd A, Opnd B, double* C, long long csb, long long csi,
                                                long long csj, int nb, int ni, int nj, long long nk1,
                                                long long nk2, double alpha, double beta, int nsplit,
                                                double* part) {
  const TA* __restrict__ Ap = static_cast<const TA*>(A.p);
  const TB* __restrict__ Bp = static_cast<const TB*>(B.p);
  __shared__ float As[kGK][kGM + 4];
  __shared__ float Bs[kGK][kGN + 4];
  const int b = blockIdx.z / nsplit, sp = blockIdx.z % nsplit;
  const int i0 = blockIdx.y * kGM, j0 = blockIdx.x * kGN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const long long K = nk1 * nk2;
  const long long ktiles = (K + kGK - 1) / kGK;
  const long long kt0 = ktiles * sp / nsplit, kt1 = ktiles * (sp + 1) / nsplit;
  const long long ab = (long long)b * A.sb, bb = (long long)b * B.sb;
  double acc64[4][4] = {};
  for (long long kt = kt0; kt < kt1; ++kt) {
    const long long k0 = kt * kGK;
    const bool a_rows = (A.sx == 1);  // stage along the contiguous index
    for (int e = threadIdx.x; e < kGM * kGK; e += 256) {
      const int r = a_rows ? e % kGM : e / kGK, kk = a_rows ? e / kGM : e % kGK;
      const int gi = i0 + r;
      const long long gk = k0 + kk;
      float v = 0.f;
      if (gi < ni && gk < K) {
        if (K2) {
          const long long k1 = gk / nk2, k2 = gk - k1 * nk2;
          v = (float)Ap[ab + gi * A.sx + k1 * A.sk1 + k2 * A.sk2];
        } else {
          v = (float)Ap[ab + gi * A.sx + gk * A.sk1];
        }
      }
      As[kk][r] = v;
    }
    const bool b_k = (B.sk1 == 1 && B.sx != 1);
    for (int e = threadIdx.x; e < kGK * kGN; e += 256) {
      const int kk = b_k ? e % kGK : e / kGN, c = b_k ? e / kGK : e % kGN;
      const int gj = j0 + c;
      const long long gk = k0 + kk;
      float v = 0.f;
      if (gj < nj && gk < K) {
        if (K2) {
          const long long k1 = gk / nk2, k2 = gk - k1 * nk2;
          v = (float)Bp[bb + gj * B.sx + k1 * B.sk1 + k2 * B.sk2];
        } else {
          v = (float)Bp[bb + gj * B.sx + gk * B.sk1];
        }
      }
      Bs[kk][c] = v;
    }
    __syncthreads();
    float acc[4][4] = {};
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      float a[4], w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = As[kk][ty * 4 + u];
#pragma unroll
      for (int v = 0; v < 4; ++v) w[v] = Bs[kk][tx * 4 + v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], w[v], acc[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc64[u][v] += (double)acc[u][v];
    __syncthreads();
  }
  const long long nout = (long long)nb * ni * nj;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int gi = i0 + ty * 4 + u;
    if (gi >= ni) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int gj = j0 + tx * 4 + v;
      if (gj >= nj) continue;
      if (nsplit > 1) {
        part[(long long)sp * nout + ((long long)b * ni + gi) * nj + gj] = acc64[u][v];
      } else {
        double* c = C + b * csb + gi * csi + gj * csj;
        *c = alpha * acc64[u][v] + (beta != 0.0 ? beta * *c : 0.0);
      }
    }
  }
}

cudaError_t gemm(const Ctx& cx, const Opnd& A, const Opnd& B, double* C, long long csb, long long csi,
                 long long csj, int nb, int ni, int nj, long long nk1, long long nk2, double alpha = 1.0,
                 double beta = 0.0) {
  const long long nout = (long long)nb * ni * nj;
  if (nout == 0) return cudaSuccess;
  const long long tiles = (long long)nb * ((ni + kGM - 1) / kGM) * ((nj + kGN - 1) / kGN);
  const long long ktiles = (nk1 * nk2 + kGK - 1) / kGK;
  long long want = (4LL * 152) / tiles;  // about four blocks per SM
  int nsplit = (int)(want < 1 ? 1 : (want > ktiles ? ktiles : want));
  if (nsplit > 64) nsplit = 64;
  while (nsplit > 1 && (long long)nsplit * nout > cx.partsz) --nsplit;
  if (nsplit < 1) nsplit = 1;
  if ((long long)nb * nsplit > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)((nj + kGN - 1) / kGN), (unsigned)((ni + kGM - 1) / kGM), (unsigned)(nb * nsplit));
  const bool k2 = nk2 > 1;
#define GEMM_LAUNCH(TA, TB, K2V) \
  k_gemm_t<TA, TB, K2V><<<grid, 256, 0, cx.s>>>(A, B, C, csb, csi, csj, nb, ni, nj, nk1, nk2, alpha, beta, nsplit, cx.part)
  if (A.f64 && B.f64) { if (k2) GEMM_LAUNCH(double, double, true); else GEMM_LAUNCH(double, double, false); }
  else if (A.f64) { if (k2) GEMM_LAUNCH(double, float, true); else GEMM_LAUNCH(double, float, false); }
  else if (B.f64) { if (k2) GEMM_LAUNCH(float, double, true); else GEMM_LAUNCH(float, double, false); }
  else { if (k2) GEMM_LAUNCH(float, float, true); else GEMM_LAUNCH(float, float, false); }
#undef GEMM_LAUNCH
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || nsplit == 1) return e;
  k_contract_reduce<<<(unsigned)((nout + kT - 1) / kT), kT, 0, cx.s>>>(cx.part, nsplit, C, csb, csi, csj, nb,
                                                                      ni, nj, alpha, beta);
  return cudaGetLastError();
}

// Y = X x_mode M for a 3-mode tensor X (dims n, float or double), M[j][k] at M + j*mr + k*mc
// (J rows, n[mode] columns); Y (double) has n[mode] replaced by J.
cudaError_t ttm3(const Ctx& cx, const void* X, int xf64, const long long n[3], int mode,
                 const double* M, long long mr, long long mc, int J, double* Y, double beta = 0.0) {
  if (mode == 0) {
    return gemm(cx, opd(M, 1, 0, mr, mc), opd(X, xf64, 0, 1, n[1] * n[2]), Y, 0, n[1] * n[2], 1,
                    1, J, (int)(n[1] * n[2]), n[0], 1, 1.0, beta);
  } else if (mode == 1) {
    return gemm(cx, opd(M, 1, 0, mr, mc), opd(X, xf64, n[1] * n[2], 1, n[2]), Y, (long long)J * n[2],
                    n[2], 1, (int)n[0], J, (int)n[2], n[1], 1, 1.0, beta);
  }
  return gemm(cx, opd(X, xf64, 0, n[2], 1), opd(M, 1, 0, mr, mc), Y, 0, J, 1, 1,
                  (int)(n[0] * n[1]), J, n[2], 1, 1.0, beta);
}

// out (n[mode] x m, row-major) = X_(mode) Y_(mode)^T, X dims n, Y dims n with n[mode] -> m.
cudaError_t contract_but3(const Ctx& cx, const void* X, int xf64, const long long n[3],
                          const double* Y, int m, int mode, double* out, double beta = 0.0) {
  if (mode == 0) {
    return gemm(cx, opd(X, xf64, 0, n[1] * n[2], 1), opd(Y, 1, 0, n[1] * n[2], 1), out, 0, m, 1, 1,
                    (int)n[0], m, n[1] * n[2], 1, 1.0, beta);
  } else if (mode == 1) {
    return gemm(cx, opd(X, xf64, 0, n[2], n[1] * n[2], 1), opd(Y, 1, 0, n[2], (long long)m * n[2], 1),
                    out, 0, m, 1, 1, (int)n[1], m, n[0], n[2], 1.0, beta);
  }
  return gemm(cx, opd(X, xf64, 0, 1, n[2]), opd(Y, 1, 0, 1, m), out, 0, m, 1, 1, (int)n[2], m,
                  n[0] * n[1], 1, 1.0, beta);
}

// ------------------------------------------------------------------ small kernels
// W_i (m x q, double) = C_i(I_i, :) from the slot values (C_i stored fiber-major: q x d).
__global__ void k_bw_gather_W(const float* C, const long long* I, int m, int q, long long d, double* W) {
  const long long e = (long long)blockIdx.x * kT + threadIdx.x;
  if (e >= (long long)m * q) return;
  const int a = (int)(e / q), c = (int)(e % q);
  W[e] = (double)C[(long long)c * d + I[a]];
}

// Z = U_r diag(1 / lambda_r) U_r^T (m x m)
__global__ void k_bw_Z(const double* U, const double* lam, int m, int r, double* Z) {
  const long long e = (long long)blockIdx.x * kT + threadIdx.x;
  if (e >= (long long)m * m) return;
  const int a = (int)(e / m), c = (int)(e % m);
  double acc = 0.0;
  for (int j = 0; j < r; ++j) acc += U[(long long)a * m + j] * U[(long long)c * m + j] / lam[j];
  Z[e] = acc;
}

// T <- F o sym(T) with the Daleckii-Krein divided differences of f = 1/lambda (top r), 0 (rest)
__global__ void k_bw_dk(double* T, const double* lam, int m, int r) {
  const long long e = (long long)blockIdx.x * kT + threadIdx.x;
  if (e >= (long long)m * m) return;
  const int j = (int)(e / m), k = (int)(e % m);
  if (k < j) return;  // each symmetric pair once
  const double v = 0.5 * (T[e] + T[(long long)k * m + j]);
  double f;
  if (j < r && k < r) f = -1.0 / (lam[j] * lam[k]);
  else if (j < r) f = 1.0 / (lam[j] * (lam[j] - lam[k]));
  else if (k < r) f = 1.0 / (lam[k] * (lam[k] - lam[j]));
  else f = 0.0;
  T[e] = f * v;
  T[(long long)k * m + j] = f * v;
}

// symmetric part in place
__global__ void k_bw_sym(double* T, int m) {
  const long long e = (long long)blockIdx.x * kT + threadIdx.x;
  if (e >= (long long)m * m) return;
  const int j = (int)(e / m), k = (int)(e % m);
  if (k <= j) return;
  const double v = 0.5 * (T[e] + T[(long long)k * m + j]);
  T[e] = v;
  T[(long long)k * m + j] = v;
}

// C_bar(I_i, :) += W_bar in slot layout: Cb[c * d + I[a]] += Wb[a * q + c]
__global__ void k_bw_scatter_W(double* Cb, const double* Wb, const long long* I, int m, int q, long long d) {
  const long long e = (long long)blockIdx.x * kT + threadIdx.x;
  if (e >= (long long)m * q) return;
  const int a = (int)(e / q), c = (int)(e % q);
  Cb[(long long)c * d + I[a]] += Wb[e];
}

// rows: P[a, :] = A[I[a], :] (A is d x m, P is m x m)
__global__ void k_bw_gather_rows(const double* A, const long long* I, int m, double* P) {
  const long long e = (long long)blockIdx.x * kT + threadIdx.x;
  if (e >= (long long)m * m) return;
  const int a = (int)(e / m), c = (int)(e % m);
  P[e] = A[I[a] * m + c];
}

// A_bar[I[a], :] = Pb[a, :] (I distinct), after A_bar was zeroed
__global__ void k_bw_scatter_rows(double* Ab, const double* Pb, const long long* I, int m) {
  const long long e = (long long)blockIdx.x * kT + threadIdx.x;
  if (e >= (long long)m * m) return;
  const int a = (int)(e / m), c = (int)(e % m);
  Ab[I[a] * m + c] += Pb[e];
}

// Slots [e0, e1) of one segment (R, or the fibers of one mode): X receives the unmasked adjoint,
// L^(k) the masked one. Positions are distinct within a segment, so segments launched one after
// another add into dX without atomics, in a fixed order.
__global__ void k_bw_slots(Geom g, const long long* set, const unsigned char* mask, const double* Vb,
                           double* Lb, double* dX, long long e0, long long e1) {
  long long p[RT_MAXN];
  const long long stride = (long long)gridDim.x * kT;
  for (long long e = e0 + (long long)blockIdx.x * kT + threadIdx.x; e < e1; e += stride) {
    const double v = Vb[e];
    if (mask[e]) {
      Lb[e] = v;
    } else {
      Lb[e] = 0.0;
      sample_coords(g, set, e, p);
      long long lin = 0;
      for (int l = 0; l < g.n; ++l) lin = lin * g.d[l] + p[l];
      dX[lin] += v;
    }
  }
}

// Other-mode coordinates of fiber c of mode i (column J[c] of X_(i), row-major over the others).
__device__ __forceinline__ void fiber_other(const Geom& g, int i, long long j, long long* p) {
  for (int l = g.n - 1; l >= 0; --l) {
    if (l == i) continue;
    p[l] = j % g.d[l];
    j /= g.d[l];
  }
}

// A_bar_l(t, :) += sum over the fibers c with p_l(c) = t, in ascending c, of G(c, :) (q x m_l):
// the row scatter of the per-fiber contributions without atomics.
__global__ void k_bw_rows_ordered(Geom g, const int* pl, int q, const double* Gc, int ml, double* Ab,
                                  long long dl) {
  const long long e = (long long)blockIdx.x * kT + threadIdx.x;
  if (e >= dl * ml) return;
  const int t = (int)(e / ml);
  const int x = (int)(e % ml);
  double acc = 0.0;
  for (int c = 0; c < q; ++c)
    if (pl[c] == t) acc += Gc[(long long)c * ml + x];
  Ab[e] += acc;
}

// Coordinate on mode l of each fiber of mode i.
__global__ void k_bw_fiber_coord(Geom g, const long long* J, int i, int l, int q, int* pl) {
  const int c = blockIdx.x * kT + threadIdx.x;
  if (c >= q) return;
  long long p[RT_MAXN];
  fiber_other(g, i, J[c], p);
  pl[c] = (int)p[l];
}

__global__ void k_bw_to_f32(const double* src, float* dst, long long n) {
  const long long stride = (long long)gridDim.x * kT;
  for (long long e = (long long)blockIdx.x * kT + threadIdx.x; e < n; e += stride) dst[e] = (float)src[e];
}

// ------------------------------------------------------------------ fiber contractions

// Rows of A'_l at the other-mode coordinates of each fiber of mode i: V[y q + c] = A'_l(p_l(c), y).
__global__ void k_bw_fiber_rows(Geom g, const long long* J, int i, int l, int q, const double* Al, int ml,
                                float* V) {
  const long long e = (long long)blockIdx.x * kT + threadIdx.x;
  if (e >= (long long)ml * q) return;
  const int y = (int)(e / q), c = (int)(e % q);
  long long p[RT_MAXN];
  fiber_other(g, i, J[c], p);
  V[e] = (float)Al[p[l] * ml + y];
}

// out[x q + c] = sum_y T[(x my + y) q + c] V[y q + c]
__global__ void k_bw_mid(const double* T, const float* V, int mx, int my, int q, double* out) {
  const long long e = (long long)blockIdx.x * kT + threadIdx.x;
  if (e >= (long long)mx * q) return;
  const int x = (int)(e / q), c = (int)(e % q);
  double acc = 0.0;
  for (int y = 0; y < my; ++y) acc = fma(T[((long long)x * my + y) * q + c], (double)V[(long long)y * q + c], acc);
  out[e] = acc;
}

// out[c my + y] = sum_x Zb[x q + c] T[(x my + y) q + c]
__global__ void k_bw_outer_mid(const double* T, const double* Zb, int mx, int my, int q, double* out) {
  const long long e = (long long)blockIdx.x * kT + threadIdx.x;
  if (e >= (long long)my * q) return;
  const int y = (int)(e / q), c = (int)(e % q);
  double acc = 0.0;
  for (int x = 0; x < mx; ++x) acc = fma(Zb[(long long)x * q + c], T[((long long)x * my + y) * q + c], acc);
  out[(long long)c * my + y] = acc;
}

// Khatri-Rao columns: KR[(y q + c) mz + z] = VA[y q + c] VB[z q + c]
__global__ void k_bw_kr(const float* VA, const float* VB, int my, int mz, int q, float* KR) {
  const long long e = (long long)blockIdx.x * kT + threadIdx.x;
  if (e >= (long long)my * q * mz) return;
  const int z = (int)(e % mz);
  const long long t = e / mz;
  const int c = (int)(t % q), y = (int)(t / q);
  KR[e] = VA[(long long)y * q + c] * VB[(long long)z * q + c];
}

// ------------------------------------------------------------------ FP64 Jacobi eigensolver
// One CTA per symmetric PSD m x m matrix (m <= kEigMax), all recorded iterations and modes in one
// launch: parallel cyclic Jacobi with the round-robin ordering (m/2 disjoint rotations per round,
// m-1 rounds per sweep), A in shared memory, U in global memory. A pair is rotated only when
// |a_pq| > 1e-15 sqrt(a_pp a_qq) (the relative test that gives PSD matrices eigenvalues to high
// relative accuracy); the sweeps stop when one rotates nothing. Output: lambda descending, the
// columns of U in the same order.
constexpr int kEigMax = 160;

struct EigArgs {
  const double* M;  // per slot and mode: the symmetric matrix
  double* U;        // eigenvectors on exit (FP64 polish: the starting basis on entry)
  double* W;        // FP64 polish scratch (M U)
  double* lam;
  long long offMM[RT_MAXN], offM[RT_MAXN];
  long long slotMM, slotM;
  int m[RT_MAXN];
  int nmodes;
};

__global__ void __launch_bounds__(kT) k_bw_eig(EigArgs ea, int max_sweeps, int polish) {
  extern __shared__ double sA[];
  __shared__ double cs[kEigMax / 2], sn[kEigMax / 2];
  __shared__ int pp[kEigMax / 2], qq[kEigMax / 2];
  __shared__ int perm[kEigMax];
  __shared__ int nrot;
  const int slot = blockIdx.x / ea.nmodes, mode = blockIdx.x % ea.nmodes;
  const int m = ea.m[mode];
  const long long off = slot * ea.slotMM + ea.offMM[mode];
  const double* M = ea.M + off;
  double* U = ea.U + off;
  double* lam = ea.lam + slot * ea.slotM + ea.offM[mode];
  const int mp = (m + 1) & ~1;  // padded to even; index m (if m odd) is a dummy
  const int ld = mp + 1;        // odd row stride: column sweeps hit distinct banks
  const int tid = threadIdx.x;
  if (!polish) {
    for (int e = tid; e < mp * mp; e += kT) {
      int r = e / mp, c = e % mp;
      sA[r * ld + c] = (r < m && c < m) ? M[(long long)r * m + c] : 0.0;
    }
    for (int e = tid; e < m * m; e += kT) U[e] = ((e / m) == (e % m)) ? 1.0 : 0.0;
  } else {
    // start from the FP32 basis: A = U^T M U (nearly diagonal), U kept as the accumulated basis
    double* W = ea.W + off;
    for (int e = tid; e < m * m; e += kT) {
      const int r = e / m, c = e % m;
      double acc = 0.0;
      for (int a = 0; a < m; ++a) acc = fma(M[(long long)r * m + a], U[(long long)a * m + c], acc);
      W[e] = acc;
    }
    __syncthreads();
    for (int e = tid; e < mp * mp; e += kT) {
      const int r = e / mp, c = e % mp;
      double acc = 0.0;
      if (r < m && c < m)
        for (int a = 0; a < m; ++a) acc = fma(U[(long long)a * m + r], W[(long long)a * m + c], acc);
      sA[r * ld + c] = acc;
    }
  }
  __syncthreads();
  // entries below 1e-17 of the largest diagonal entry are rounding noise of the FP64 Gram
  // matrix; rotating them would keep a rank-deficient matrix sweeping forever
  __shared__ double floor_abs;
  if (tid == 0) {
    double mxd = 0.0;
    for (int j = 0; j < m; ++j) mxd = fmax(mxd, fabs(sA[j * ld + j]));
    floor_abs = 1e-17 * mxd;
  }
  __syncthreads();
  for (int sw = 0; sw < max_sweeps; ++sw) {
    if (tid == 0) nrot = 0;
    __syncthreads();
    for (int rd = 0; rd < mp - 1; ++rd) {
      if (tid < mp / 2) {
        const int t = tid;
        const int k1 = t, k2 = mp - 1 - t;
        const int p = (k1 == 0) ? 0 : ((k1 - 1 + rd) % (mp - 1)) + 1;
        const int q = (k2 == 0) ? 0 : ((k2 - 1 + rd) % (mp - 1)) + 1;
        double c = 1.0, s = 0.0;
        if (p < m && q < m) {
          const double apq = sA[p * ld + q];
          const double app = sA[p * ld + p], aqq = sA[q * ld + q];
          if (fabs(apq) > 1e-15 * sqrt(fabs(app * aqq)) && fabs(apq) > floor_abs) {
            const double th = (aqq - app) / (2.0 * apq);
            double tt;
            if (fabs(th) > 1e150) tt = 0.5 / th;
            else tt = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            c = 1.0 / sqrt(tt * tt + 1.0);
            s = tt * c;
            atomicAdd(&nrot, 1);
          }
        }
        pp[t] = p;
        qq[t] = q;
        cs[t] = c;
        sn[t] = s;
      }
      __syncthreads();
      // rows: A <- G^T A
      for (int e = tid; e < (mp / 2) * mp; e += kT) {
        const int t = e / mp, col = e % mp;
        const double s = sn[t];
        if (s == 0.0) continue;
        const int p = pp[t], q = qq[t];
        const double c = cs[t];
        const double ap = sA[p * ld + col], aq = sA[q * ld + col];
        sA[p * ld + col] = c * ap - s * aq;
        sA[q * ld + col] = s * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A G, U <- U G
      for (int e = tid; e < (mp / 2) * mp; e += kT) {
        const int t = e / mp, row = e % mp;
        const double s = sn[t];
        if (s == 0.0) continue;
        const int p = pp[t], q = qq[t];
        const double c = cs[t];
        const double ap = sA[row * ld + p], aq = sA[row * ld + q];
        sA[row * ld + p] = c * ap - s * aq;
        sA[row * ld + q] = s * ap + c * aq;
        if (row < m && p < m && q < m) {
          const double up = U[(long long)row * m + p], uq = U[(long long)row * m + q];
          U[(long long)row * m + p] = c * up - s * uq;
          U[(long long)row * m + q] = s * up + c * uq;
        }
      }
      __syncthreads();
    }
    if (nrot == 0) break;  // uniform: read after the last barrier of the sweep
    __syncthreads();       // nobody resets nrot before everyone has read it
  }
  // sort descending (selection on one thread; m <= kEigMax)
  if (tid == 0) {
    for (int j = 0; j < m; ++j) perm[j] = j;
    for (int j = 0; j < m; ++j) {
      int best = j;
      for (int l = j + 1; l < m; ++l)
        if (sA[perm[l] * ld + perm[l]] > sA[perm[best] * ld + perm[best]]) best = l;
      int t = perm[j]; perm[j] = perm[best]; perm[best] = t;
    }
    for (int j = 0; j < m; ++j) lam[j] = sA[perm[j] * ld + perm[j]];
  }
  __syncthreads();
  for (int e = tid; e < m * m; e += kT) sA[e] = U[(long long)(e / m) * m + perm[e % m]];
  __syncthreads();
  for (int e = tid; e < m * m; e += kT) U[e] = sA[e];
}


// FP32 cyclic Jacobi, A and U in shared memory (the same round-robin ordering): the starting
// basis of the FP64 polish. A pair is rotated when |a_pq| > 1e-7 sqrt(a_pp a_qq) and above a
// noise floor of 1e-8 of the largest diagonal entry; output lambda descending, U as FP64.
__global__ void __launch_bounds__(kT) k_bw_eig32(EigArgs ea, int max_sweeps) {
  extern __shared__ float sF[];
  __shared__ float cs[kEigMax / 2], sn[kEigMax / 2];
  __shared__ int pp[kEigMax / 2], qq[kEigMax / 2];
  __shared__ int perm[kEigMax];
  __shared__ int nrot;
  __shared__ float floor_abs;
  const int slot = blockIdx.x / ea.nmodes, mode = blockIdx.x % ea.nmodes;
  const int m = ea.m[mode];
  const long long off = slot * ea.slotMM + ea.offMM[mode];
  const double* M = ea.M + off;
  double* Uout = ea.U + off;
  double* lam = ea.lam + slot * ea.slotM + ea.offM[mode];
  const int mp = (m + 1) & ~1;
  const int ld = mp + 1;  // odd row stride: column sweeps hit distinct banks
  float* sA = sF;
  float* sU = sF + mp * ld;
  const int tid = threadIdx.x;
  for (int e = tid; e < mp * mp; e += kT) {
    int r = e / mp, c = e % mp;
    sA[r * ld + c] = (r < m && c < m) ? (float)M[(long long)r * m + c] : 0.f;
    sU[r * ld + c] = (r == c) ? 1.f : 0.f;
  }
  __syncthreads();
  if (tid == 0) {
    float mxd = 0.f;
    for (int j = 0; j < m; ++j) mxd = fmaxf(mxd, fabsf(sA[j * ld + j]));
    floor_abs = 1e-8f * mxd;
  }
  __syncthreads();
  for (int sw = 0; sw < max_sweeps; ++sw) {
    if (tid == 0) nrot = 0;
    __syncthreads();
    for (int rd = 0; rd < mp - 1; ++rd) {
      if (tid < mp / 2) {
        const int t = tid;
        const int k1 = t, k2 = mp - 1 - t;
        const int p = (k1 == 0) ? 0 : ((k1 - 1 + rd) % (mp - 1)) + 1;
        const int q = (k2 == 0) ? 0 : ((k2 - 1 + rd) % (mp - 1)) + 1;
        float c = 1.f, s = 0.f;
        if (p < m && q < m) {
          const float apq = sA[p * ld + q];
          const float app = sA[p * ld + p], aqq = sA[q * ld + q];
          if (fabsf(apq) > 1e-7f * sqrtf(fabsf(app * aqq)) && fabsf(apq) > floor_abs) {
            const float th = (aqq - app) / (2.f * apq);
            float tt;
            if (fabsf(th) > 1e18f) tt = 0.5f / th;
            else tt = (th >= 0.f ? 1.f : -1.f) / (fabsf(th) + sqrtf(th * th + 1.f));
            c = 1.f / sqrtf(tt * tt + 1.f);
            s = tt * c;
            atomicAdd(&nrot, 1);
          }
        }
        pp[t] = p;
        qq[t] = q;
        cs[t] = c;
        sn[t] = s;
      }
      __syncthreads();
      for (int e = tid; e < (mp / 2) * mp; e += kT) {
        const int t = e / mp, col = e % mp;
        const float s = sn[t];
        if (s == 0.f) continue;
        const int p = pp[t], q = qq[t];
        const float c = cs[t];
        const float ap = sA[p * ld + col], aq = sA[q * ld + col];
        sA[p * ld + col] = c * ap - s * aq;
        sA[q * ld + col] = s * ap + c * aq;
      }
      __syncthreads();
      for (int e = tid; e < (mp / 2) * mp; e += kT) {
        const int t = e / mp, row = e % mp;
        const float s = sn[t];
        if (s == 0.f) continue;
        const int p = pp[t], q = qq[t];
        const float c = cs[t];
        const float ap = sA[row * ld + p], aq = sA[row * ld + q];
        sA[row * ld + p] = c * ap - s * aq;
        sA[row * ld + q] = s * ap + c * aq;
        const float up = sU[row * ld + p], uq = sU[row * ld + q];
        sU[row * ld + p] = c * up - s * uq;
        sU[row * ld + q] = s * up + c * uq;
      }
      __syncthreads();
    }
    if (nrot == 0) break;
    __syncthreads();
  }
  if (tid == 0) {
    for (int j = 0; j < m; ++j) perm[j] = j;
    for (int j = 0; j < m; ++j) {
      int best = j;
      for (int l = j + 1; l < m; ++l)
        if (sA[perm[l] * ld + perm[l]] > sA[perm[best] * ld + perm[best]]) best = l;
      int t = perm[j]; perm[j] = perm[best]; perm[best] = t;
    }
    for (int j = 0; j < m; ++j) lam[j] = (double)sA[perm[j] * ld + perm[j]];
  }
  __syncthreads();
  for (int e = tid; e < m * m; e += kT) Uout[e] = (double)sU[(e / m) * ld + perm[e % m]];
}

inline unsigned nblk(long long n) { return (unsigned)((n + kT - 1) / kT); }

#define BW_CK(x)                          \
  do {                                    \
    cudaError_t e_ = (x);                 \
    if (e_ != cudaSuccess) return e_;     \
  } while (0)

}  // namespace

size_t backward_eig_smem(int m) {
  const int mp = (m + 1) & ~1;
  return sizeof(double) * (size_t)mp * (mp + 1);  // FP64: one padded panel; FP32: two
}

cudaError_t prepare_backward(int max_m) {
  if (max_m > kEigMax) return cudaErrorInvalidValue;
  cudaError_t e = raise_smem_limit((const void*)k_bw_eig, (size_t)(backward_eig_smem(max_m)));
  if (e != cudaSuccess) return e;
  return raise_smem_limit((const void*)k_bw_eig32, (size_t)(backward_eig_smem(max_m)));  // 2 float panels
}

void backward_layout(const Geom& g, BwWork& w) {
  long long oW = 0, oMM = 0, oM = 0, oQM = 0, oDM = 0;
  for (int i = 0; i < g.n; ++i) {
    w.offW[i] = oW; oW += (long long)g.m[i] * g.q[i];
    w.offMM[i] = oMM; oMM += (long long)g.m[i] * g.m[i];
    w.offM[i] = oM; oM += g.m[i];
    w.offQM[i] = oQM; oQM += (long long)g.q[i] * g.m[i];
    w.offDM[i] = oDM; oDM += g.d[i] * g.m[i];
  }
  w.slotW = oW;
  w.slotMM = oMM;
  w.slotM = oM;
  w.slotQM = oQM;
  w.slotDM = oDM;
  // dense temporaries: the largest tensor with two original dims and one sampled dim
  long long t = g.nR;
  for (int i = 0; i < 3; ++i) {
    long long v = g.m[i];
    for (int l = 0; l < 3; ++l)
      if (l != i) v *= g.d[l];
    if (v > t) t = v;
    long long u = g.d[i];
    for (int l = 0; l < 3; ++l)
      if (l != i) u *= g.m[l];
    if (u > t) t = u;
  }
  // fiber products: T1, T2 (m_i x m_l x q) in tmp0/tmp1, the Khatri-Rao columns in kr
  long long kr = 0;
  for (int i = 0; i < 3; ++i) {
    long long v = g.q[i];
    for (int l = 0; l < 3; ++l)
      if (l != i) v *= g.m[l];
    if (v > kr) kr = v;
    if (v / g.m[(i + 1) % 3] * g.m[i] > t) t = v / g.m[(i + 1) % 3] * g.m[i];
    if (v / g.m[(i + 2) % 3] * g.m[i] > t) t = v / g.m[(i + 2) % 3] * g.m[i];
  }
  w.tmpsz = t;
  w.krsz = kr;
  w.partsz = 1LL << 22;
}

cudaError_t launch_backward(const Geom& g, const Bufs& b, const BwWork& w, int K, const float* dL,
                            float* dX, cudaStream_t s) {
  Ctx cx{w.part, w.partsz, s};
  const long long n3[3] = {g.d[0], g.d[1], g.d[2]};
  const long long mR[3] = {g.m[0], g.m[1], g.m[2]};
  auto set_of = [&](int k) { return b.idx + (long long)((g.variant == 1) ? (k % g.n_sets) : 0) * g.set_len; };
  auto V = [&](int k) { return b.ckV + (long long)k * g.nS; };
  auto Aof = [&](int k, int i) { return w.A + (long long)k * w.slotDM + w.offDM[i]; };
  auto Pof = [&](int k, int i) { return w.P + (long long)k * w.slotQM + w.offQM[i]; };
  auto Wof = [&](int k, int i) { return w.W + (long long)k * w.slotW + w.offW[i]; };
  auto Uof = [&](int k, int i) { return w.U + (long long)k * w.slotMM + w.offMM[i]; };
  auto Lof = [&](int k, int i) { return w.lam + (long long)k * w.slotM + w.offM[i]; };
  auto Zof = [&](int k, int i) { return w.Z + (long long)k * w.slotMM + w.offMM[i]; };

  // ---- forward pieces of every recorded iteration: W, M = W W^T, eigenpairs, Z, P, A
  for (int k = 0; k < K; ++k) {
    const long long* set = set_of(k);
    for (int i = 0; i < 3; ++i) {
      const int m = g.m[i], q = g.q[i];
      const float* C = V(k) + g.seg[i + 1];
      k_bw_gather_W<<<nblk((long long)m * q), kT, 0, s>>>(C, set + g.ioff[i], m, q, g.d[i], Wof(k, i));
      BW_CK(cudaGetLastError());
      // M = W W^T (in Z's slot until Z is formed)
      BW_CK(contract(cx, opd(Wof(k, i), 1, 0, q, 1), opd(Wof(k, i), 1, 0, q, 1), Zof(k, i), 0, m, 1, 1, m, m,
                     q, 1));
    }
  }
  {
    // every (iteration, mode) matrix at once: FP32 Jacobi, then the FP64 polish from its basis
    EigArgs ea;
    ea.M = w.Z;
    ea.U = w.U;
    ea.W = w.Ub;
    ea.lam = w.lam;
    ea.slotMM = w.slotMM;
    ea.slotM = w.slotM;
    ea.nmodes = 3;
    int mx = 0;
    for (int i = 0; i < 3; ++i) {
      ea.offMM[i] = w.offMM[i];
      ea.offM[i] = w.offM[i];
      ea.m[i] = g.m[i];
      mx = g.m[i] > mx ? g.m[i] : mx;
    }
    k_bw_eig32<<<K * 3, kT, backward_eig_smem(mx), s>>>(ea, 60);
    BW_CK(cudaGetLastError());
    k_bw_eig<<<K * 3, kT, backward_eig_smem(mx), s>>>(ea, 20, 1);
    BW_CK(cudaGetLastError());
  }
  for (int k = 0; k < K; ++k) {
    for (int i = 0; i < 3; ++i) {
      const int m = g.m[i], q = g.q[i], r = g.r[i];
      k_bw_Z<<<nblk((long long)m * m), kT, 0, s>>>(Uof(k, i), Lof(k, i), m, r, Zof(k, i));
      BW_CK(cudaGetLastError());
      // P = W^T Z (q x m)
      BW_CK(contract(cx, opd(Wof(k, i), 1, 0, 1, q), opd(Zof(k, i), 1, 0, 1, m), Pof(k, i), 0, m, 1, 1, q, m,
                     m, 1));
      // A = C P (d x m); C(t, c) = slot value c * d + t
      const float* C = V(k) + g.seg[i + 1];
      BW_CK(contract(cx, opd(C, 0, 0, 1, g.d[i]), opd(Pof(k, i), 1, 0, 1, m), Aof(k, i), 0, m, 1, 1,
                     (int)g.d[i], m, q, 1));
    }
  }

  // ---- seed: L^(K) = R x_i A_i with dL
  BW_CK(cudaMemsetAsync(w.dX64, 0, sizeof(double) * g.N, s));
  double* Rb = w.Vb;  // the R segment of the slot adjoint
  {
    const int k = K - 1;
    const float* R = V(k);
    long long sh[3];
    // R_bar = dL x_0 A_0^T x_1 A_1^T x_2 A_2^T
    BW_CK(ttm3(cx, dL, 0, n3, 0, Aof(k, 0), 1, g.m[0], g.m[0], w.tmp0));
    sh[0] = g.m[0]; sh[1] = n3[1]; sh[2] = n3[2];
    BW_CK(ttm3(cx, w.tmp0, 1, sh, 1, Aof(k, 1), 1, g.m[1], g.m[1], w.tmp1));
    sh[1] = g.m[1];
    BW_CK(ttm3(cx, w.tmp1, 1, sh, 2, Aof(k, 2), 1, g.m[2], g.m[2], Rb));
    // A_bar_i = dL_(i) (R x_{j != i} A_j)_(i)^T
    for (int i = 0; i < 3; ++i) {
      long long cur[3] = {mR[0], mR[1], mR[2]};
      const void* src = R;
      int sf64 = 0;
      double* bufs[2] = {w.tmp0, w.tmp1};
      int nb = 0;
      for (int l = 0; l < 3; ++l) {
        if (l == i) continue;
        BW_CK(ttm3(cx, src, sf64, cur, l, Aof(k, l), g.m[l], 1, (int)g.d[l], bufs[nb]));
        cur[l] = g.d[l];
        src = bufs[nb];
        sf64 = 1;
        nb ^= 1;
      }
      BW_CK(contract_but3(cx, dL, 0, n3, static_cast<const double*>(src), g.m[i], i, w.Ab + w.offDM[i]));
    }
  }

  // ---- reverse sweep over the recorded iterations
  for (int k = K - 1; k >= 0; --k) {
    const long long* set = set_of(k);
    for (int i = 0; i < 3; ++i) {
      const int m = g.m[i], q = g.q[i];
      const long long d = g.d[i];
      const float* C = V(k) + g.seg[i + 1];
      double* Ab = w.Ab + w.offDM[i];
      double* Cb = w.Vb + g.seg[i + 1];
      // C_bar (slot layout q x d) = A_bar P^T
      BW_CK(contract(cx, opd(Pof(k, i), 1, 0, m, 1), opd(Ab, 1, 0, m, 1), Cb, 0, d, 1, 1, q, (int)d, m, 1));
      // P_bar (q x m) = C^T A_bar
      BW_CK(contract(cx, opd(C, 0, 0, d, 1), opd(Ab, 1, 0, 1, m), w.Pb, 0, m, 1, 1, q, m, d, 1));
      // W_bar = Z P_bar^T + 2 M_bar W
      BW_CK(contract(cx, opd(Wof(k, i), 1, 0, q, 1), opd(w.Pb, 1, 0, 1, m), w.T0, 0, m, 1, 1, m, m, q, 1));
      k_bw_sym<<<nblk((long long)m * m), kT, 0, s>>>(w.T0, m);
      BW_CK(cudaGetLastError());
      BW_CK(contract(cx, opd(w.T0, 1, 0, m, 1), opd(Uof(k, i), 1, 0, 1, m), w.T1, 0, m, 1, 1, m, m, m, 1));
      BW_CK(contract(cx, opd(Uof(k, i), 1, 0, 1, m), opd(w.T1, 1, 0, 1, m), w.T0, 0, m, 1, 1, m, m, m, 1));
      k_bw_dk<<<nblk((long long)m * m), kT, 0, s>>>(w.T0, Lof(k, i), m, g.r[i]);
      BW_CK(cudaGetLastError());
      BW_CK(contract(cx, opd(Uof(k, i), 1, 0, m, 1), opd(w.T0, 1, 0, 1, m), w.T1, 0, m, 1, 1, m, m, m, 1));
      BW_CK(contract(cx, opd(w.T1, 1, 0, m, 1), opd(Uof(k, i), 1, 0, m, 1), w.T0, 0, m, 1, 1, m, m, m, 1));
      BW_CK(contract(cx, opd(Zof(k, i), 1, 0, m, 1), opd(w.Pb, 1, 0, m, 1), w.Wb, 0, q, 1, 1, m, q, m, 1));
      BW_CK(contract(cx, opd(w.T0, 1, 0, m, 1), opd(Wof(k, i), 1, 0, 1, q), w.Wb, 0, q, 1, 1, m, q, m, 1,
                     2.0, 1.0));
      k_bw_scatter_W<<<nblk((long long)m * q), kT, 0, s>>>(Cb, w.Wb, set + g.ioff[i], m, q, d);
      BW_CK(cudaGetLastError());
    }
    for (int sg = 0; sg <= 3; ++sg) {
      const long long e0 = g.seg[sg], e1 = g.seg[sg + 1];
      long long blocks = (e1 - e0 + kT - 1) / kT;
      if (blocks > 4096) blocks = 4096;
      k_bw_slots<<<(unsigned)blocks, kT, 0, s>>>(g, set, b.ckM + (long long)k * g.nS, w.Vb, w.Lb, w.dX64,
                                                 e0, e1);
      BW_CK(cudaGetLastError());
    }
    if (k == 0) break;
    // adjoint of the slot evaluations of L^(k) = R' x_i A'_i (iteration k-1's factors)
    const float* Rp = V(k - 1);
    const double* Ap[3] = {Aof(k - 1, 0), Aof(k - 1, 1), Aof(k - 1, 2)};
    for (int i = 0; i < 3; ++i) {
      k_bw_gather_rows<<<nblk((long long)g.m[i] * g.m[i]), kT, 0, s>>>(Ap[i], set + g.ioff[i], g.m[i],
                                                                       w.Pi + w.offMM[i]);
      BW_CK(cudaGetLastError());
    }
    const double* LbR = w.Lb;
    // R_bar = LbR x_i Pi_i^T
    BW_CK(ttm3(cx, LbR, 1, mR, 0, w.Pi + w.offMM[0], 1, g.m[0], g.m[0], w.tmp0));
    BW_CK(ttm3(cx, w.tmp0, 1, mR, 1, w.Pi + w.offMM[1], 1, g.m[1], g.m[1], w.tmp1));
    BW_CK(ttm3(cx, w.tmp1, 1, mR, 2, w.Pi + w.offMM[2], 1, g.m[2], g.m[2], Rb));
    // A_bar_i(I_i, :) = LbR_(i) (R' x_{j != i} Pi_j)_(i)^T
    BW_CK(cudaMemsetAsync(w.Ab, 0, sizeof(double) * w.slotDM, s));
    for (int i = 0; i < 3; ++i) {
      const void* src = Rp;
      int sf64 = 0;
      double* bufs[2] = {w.tmp0, w.tmp1};
      int nb = 0;
      for (int l = 0; l < 3; ++l) {
        if (l == i) continue;
        BW_CK(ttm3(cx, src, sf64, mR, l, w.Pi + w.offMM[l], g.m[l], 1, g.m[l], bufs[nb]));
        src = bufs[nb];
        sf64 = 1;
        nb ^= 1;
      }
      BW_CK(contract_but3(cx, LbR, 1, mR, static_cast<const double*>(src), g.m[i], i, w.T0));
      k_bw_scatter_rows<<<nblk((long long)g.m[i] * g.m[i]), kT, 0, s>>>(w.Ab + w.offDM[i], w.T0,
                                                                        set + g.ioff[i], g.m[i]);
      BW_CK(cudaGetLastError());
    }
    // fibers of each mode i: the fiber values are A'_i z_c, z_c = R' contracted on the other two
    // modes (l1 < l2) with the rows A'_l1(p_l1(c), :), A'_l2(p_l2(c), :). As products:
    //   T1[x][y][c] = sum_z R'[x, y, z] VB[z][c]  -> z_c = sum_y T1 VA, A_bar_l1 rows = sum_x Zb T1
    //   T2[x][z][c] = sum_y R'[x, y, z] VA[y][c]  -> A_bar_l2 rows = sum_x Zb T2
    //   R_bar[x, y, z] += sum_c Zb[x][c] VA[y][c] VB[z][c]
    // (x on mode i, y on l1, z on l2).
    const long long rs[3] = {(long long)g.m[1] * g.m[2], g.m[2], 1};
    for (int i = 0; i < 3; ++i) {
      const int m = g.m[i], q = g.q[i];
      const long long d = g.d[i];
      const double* LbC = w.Lb + g.seg[i + 1];
      const long long* J = set + g.joff[i];
      int l1 = -1, l2 = -1;
      for (int l = 0; l < 3; ++l)
        if (l != i) { if (l1 < 0) l1 = l; else l2 = l; }
      const int m1 = g.m[l1], m2 = g.m[l2];
      k_bw_fiber_rows<<<nblk((long long)m1 * q), kT, 0, s>>>(g, J, i, l1, q, Ap[l1], m1, w.va);
      BW_CK(cudaGetLastError());
      k_bw_fiber_rows<<<nblk((long long)m2 * q), kT, 0, s>>>(g, J, i, l2, q, Ap[l2], m2, w.vb);
      BW_CK(cudaGetLastError());
      BW_CK(gemm(cx, opd(Rp, 0, rs[i], rs[l1], rs[l2]), opd(w.vb, 0, 0, 1, q), w.tmp0, (long long)m1 * q, q, 1,
                 m, m1, q, m2, 1));
      k_bw_mid<<<nblk((long long)m * q), kT, 0, s>>>(w.tmp0, w.va, m, m1, q, w.Zf);
      BW_CK(cudaGetLastError());
      // A_bar_i += LbC Z^T; Z_bar = A'_i^T LbC
      BW_CK(contract(cx, opd(LbC, 1, 0, 1, d), opd(w.Zf, 1, 0, q, 1), w.Ab + w.offDM[i], 0, m, 1, 1, (int)d, m,
                     q, 1, 1.0, 1.0));
      BW_CK(contract(cx, opd(Ap[i], 1, 0, 1, m), opd(LbC, 1, 0, d, 1), w.Zfb, 0, q, 1, 1, m, q, d, 1));
      // A_bar_l1 rows
      k_bw_outer_mid<<<nblk((long long)m1 * q), kT, 0, s>>>(w.tmp0, w.Zfb, m, m1, q, w.Wb);
      BW_CK(cudaGetLastError());
      k_bw_fiber_coord<<<nblk(q), kT, 0, s>>>(g, J, i, l1, q, w.pc);
      BW_CK(cudaGetLastError());
      k_bw_rows_ordered<<<nblk(g.d[l1] * m1), kT, 0, s>>>(g, w.pc, q, w.Wb, m1, w.Ab + w.offDM[l1], g.d[l1]);
      BW_CK(cudaGetLastError());
      // A_bar_l2 rows
      BW_CK(gemm(cx, opd(Rp, 0, rs[i], rs[l2], rs[l1]), opd(w.va, 0, 0, 1, q), w.tmp1, (long long)m2 * q, q, 1,
                 m, m2, q, m1, 1));
      k_bw_outer_mid<<<nblk((long long)m2 * q), kT, 0, s>>>(w.tmp1, w.Zfb, m, m2, q, w.Wb);
      BW_CK(cudaGetLastError());
      k_bw_fiber_coord<<<nblk(q), kT, 0, s>>>(g, J, i, l2, q, w.pc);
      BW_CK(cudaGetLastError());
      k_bw_rows_ordered<<<nblk(g.d[l2] * m2), kT, 0, s>>>(g, w.pc, q, w.Wb, m2, w.Ab + w.offDM[l2], g.d[l2]);
      BW_CK(cudaGetLastError());
      // R_bar
      k_bw_kr<<<nblk((long long)m1 * q * m2), kT, 0, s>>>(w.va, w.vb, m1, m2, q, w.kr);
      BW_CK(cudaGetLastError());
      BW_CK(gemm(cx, opd(w.Zfb, 1, 0, q, 1), opd(w.kr, 0, (long long)q * m2, 1, m2), Rb, rs[l1], rs[i], rs[l2], m1,
                 m, m2, q, 1, 1.0, 1.0));
    }
  }
  int blocks = (int)((g.N + kT - 1) / kT);
  if (blocks > 8192) blocks = 8192;
  k_bw_to_f32<<<blocks, kT, 0, s>>>(w.dX64, dX, g.N);
  return cudaGetLastError();
}
