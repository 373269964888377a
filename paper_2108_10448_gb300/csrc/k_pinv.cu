// Truncated pseudoinverse of U_i = C_i(I_i, :) (Eq. (R, C_i, U_i): U_i = SVD_{r_i}(W_i),
// W_i = C_i(I_i, :), an m_i x q_i matrix), computed in FP64 as the top-r_i eigenpairs of the
// Gram matrix M_i = W_i W_i^T:  W_r^+ = V_r Sigma_r^-1 Q_r^T with V_r Sigma_r = W^T Q_r.
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so the FP64 work is kept to dot
// products spread over many lanes and SMs, and the sequential eigensolver runs in FP32:
//   1. k_gram    M_i in FP64 (FP32 products are exact in FP64), 8x8 output tiles over the grid,
//                each dot product split over a quad of lanes.
//   2. k_refine, mode 0 (warm attempt, iterations k >= 1): FP64 subspace iteration with Cholesky
//                QR from the previous iteration's basis (RTCUR-F) or the current factor's rows on
//                the new index set (RTCUR-R), accepted only with a certificate that separates the
//                top-r eigenvalues from the rest and bounds the basis error (below); then the
//                fast finish. When it succeeds for a mode, steps 3 and 4 do nothing for it.
//   3. k_eig_tri FP32 eigenbasis of fl32(M_i): Householder tridiagonalisation, multisection on
//                Sturm counts, twisted-factorisation eigenvectors, back-transformation; one CTA
//                per mode (k_jacobi, a round-robin parallel Jacobi, is the alternative option).
//   4. k_refine, mode 1 (cold path): FP64 refinement of the top-r subspace by the Ogita-Aishima
//                iteration (Ogita and Aishima 2018, "Iterative refinement for symmetric
//                eigenvalue decomposition"), restricted to the top block against the tail (pairs
//                inside the top block or inside the tail are not rotated; their first-order term
//                is the orthogonality correction only). Each step roughly squares the subspace
//                error; two steps take the FP32 basis to FP64 accuracy. Then the fast finish
//                (L needs only the top-r invariant subspace: one r x r Cholesky) or, near the
//                SVD_r cutoff, an FP64 Rayleigh-Ritz on the r x r block with the cutoff, and
//                Y_i = V_r Sigma_r^-1 = W^T Q_r Sigma_r^-2.
// k_refine runs one thread-block cluster of 16 (or 8, 4, 2) CTAs per mode; each CTA owns rows of
// the m x r panels and reads the others' rows from their shared memory (distributed shared
// memory) after a cluster barrier.
#include <cooperative_groups.h>

#include "rtcur_internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kGramTile = 8;
constexpr int kGramChunk = 512;
constexpr int kJacThreads = 1024;
constexpr int kRefThreads = 256;

__device__ __forceinline__ float w_entry(const Geom& g, const Bufs& b, const long long* set, int i,
                                         int a, int bcol) {
  // W_i[a, b] = C_i[I_i[a], b], kept compact (m_i x q_i, row-major) by the sampled threshold
  (void)set;
  return b.W[g.offW[i] + (long long)a * g.q[i] + bcol];
}

__device__ __forceinline__ const long long* set_of(const Geom& g, const Bufs& b) {
  long long s = (g.variant == 1) ? (long long)(b.st->k % g.n_sets) : 0;
  return b.idx + s * g.set_len;
}

// ------------------------------------------------------------------ 1. FP64 Gram matrix
// One 8 x 8 tile of M_i = W_i W_i^T per block; each entry's FP64 dot product is split over a quad
// of lanes (columns c = ql mod 4), so a block runs 8 warps and each FP64 chain is a quarter as long.
constexpr int kGramThreads = 4 * kGramTile * kGramTile;
__global__ void __launch_bounds__(kGramThreads) k_gram(Geom g, Bufs b) {
  TL_BEGIN();
  __shared__ float wa[kGramTile][kGramChunk + 1];
  __shared__ float wb[kGramTile][kGramChunk + 1];
  // locate (mode, tile) for this block: per mode nt(nt+1)/2 lower-triangle tiles
  int blk = blockIdx.x, i = 0, nt = 0;
  for (; i < g.n; ++i) {
    nt = (g.m[i] + kGramTile - 1) / kGramTile;
    int cnt = nt * (nt + 1) / 2;
    if (blk < cnt) break;
    blk -= cnt;
  }
  if (i >= g.n) return;
  int ta = 0;
  while ((ta + 1) * (ta + 2) / 2 <= blk) ++ta;
  int tb = blk - ta * (ta + 1) / 2;  // tb <= ta
  const long long* set = set_of(g, b);
  const int m = g.m[i], q = g.q[i];
  const int o = threadIdx.x >> 2, ql = threadIdx.x & 3;  // entry of the tile, lane of its quad
  const int ty = o / kGramTile, tx = o % kGramTile;
  const int a0 = ta * kGramTile, b0 = tb * kGramTile;
  double acc = 0.0;
  for (int c0 = 0; c0 < q; c0 += kGramChunk) {
    int cn = min(kGramChunk, q - c0);
    for (int e = threadIdx.x; e < kGramTile * cn; e += blockDim.x) {
      int rr = e / cn, cc = e % cn;
      wa[rr][cc] = (a0 + rr < m) ? w_entry(g, b, set, i, a0 + rr, c0 + cc) : 0.f;
      wb[rr][cc] = (b0 + rr < m) ? w_entry(g, b, set, i, b0 + rr, c0 + cc) : 0.f;
    }
    __syncthreads();
    for (int cc = ql; cc < cn; cc += 4) acc = fma((double)wa[ty][cc], (double)wb[tx][cc], acc);
    __syncthreads();
  }
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  acc += __shfl_xor_sync(0xffffffffu, acc, 2);
  int ra = a0 + ty, rb = b0 + tx;
  if (ql == 0 && ra < m && rb < m) {
    double* M = b.gram + g.offM[i];
    M[(long long)ra * m + rb] = acc;
    M[(long long)rb * m + ra] = acc;
  }
  TL_END(3);
}

// ------------------------------------------------------------------ 2. FP32 Jacobi
__device__ __forceinline__ int pk(int r, int c, int N) {
  if (r > c) { int t = r; r = c; c = t; }
  return r * N - (r * (r - 1)) / 2 + (c - r);
}

__device__ __forceinline__ void tri_decode(int w, int P, int& a, int& bb) {
  float tp = 2.f * P + 1.f;
  float fa = (tp - sqrtf(fmaxf(tp * tp - 8.f * (float)w, 0.f))) * 0.5f;
  int aa = max(0, min(P - 1, (int)fa));
  while (aa > 0 && aa * P - (aa * (aa - 1)) / 2 > w) --aa;
  while (aa + 1 < P && (aa + 1) * P - ((aa + 1) * aa) / 2 <= w) ++aa;
  a = aa;
  bb = aa + (w - (aa * P - (aa * (aa - 1)) / 2));
}

__global__ void __launch_bounds__(kJacThreads) k_jacobi(Geom g, Bufs b) {
  extern __shared__ float smem[];
  if (b.warm[blockIdx.x]) return;
  __shared__ int nrot;
  __shared__ float tabs;
  const int i = blockIdx.x;
  const int m = g.m[i];
  const int N = m + (m & 1);
  const int P = N / 2;
  const int Vs = N + 1;
  float* Mp = smem;                              // packed upper triangle, N(N+1)/2
  float* V = Mp + (N * (N + 1)) / 2;             // m x Vs
  int* pp = reinterpret_cast<int*>(V + m * Vs);  // P
  int* pq = pp + P;
  float* pc = reinterpret_cast<float*>(pq + P);
  float* ps = pc + P;
  float* pt = ps + P;
  const int tid = threadIdx.x;
  const double* M64 = b.gram + g.offM[i];
  for (int t = tid; t < N * N; t += blockDim.x) {
    int r = t / N, c = t % N;
    if (r <= c) Mp[pk(r, c, N)] = (c < m) ? (float)M64[(long long)r * m + c] : 0.f;
  }
  for (int t = tid; t < m * Vs; t += blockDim.x) {
    int r = t / Vs, c = t % Vs;
    V[t] = (r == c) ? 1.f : 0.f;
  }
  __syncthreads();
  const float tol = 4.f * 5.9604645e-8f;  // 4 * 2^-24
  const int nblk = (P * (P + 1)) / 2;
  for (int sw = 0; sw < g.max_sweeps; ++sw) {
    if (tid == 0) {
      nrot = 0;
      float mx = 0.f;
      for (int j = 0; j < m; ++j) mx = fmaxf(mx, Mp[pk(j, j, N)]);
      tabs = 5.9604645e-8f * mx;
    }
    __syncthreads();
    for (int rd = 0; rd < N - 1; ++rd) {
      if (tid < P) {
        int k = tid;
        int x = (k == 0) ? 0 : ((k - 1 + rd) % (N - 1)) + 1;
        int y = ((N - 1 - k - 1 + rd) % (N - 1)) + 1;
        int p = min(x, y), q = max(x, y);
        float c = 1.f, s = 0.f, tt = 0.f;
        if (q < m) {
          float app = Mp[pk(p, p, N)], aqq = Mp[pk(q, q, N)], apq = Mp[pk(p, q, N)];
          if (fabsf(apq) > tol * sqrtf(fabsf(app * aqq)) && fabsf(apq) > tabs) {
            float theta = (aqq - app) / (2.f * apq);
            tt = (theta >= 0.f ? 1.f : -1.f) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
            c = 1.f / sqrtf(tt * tt + 1.f);
            s = tt * c;
            atomicAdd(&nrot, 1);
          }
        }
        pp[k] = p; pq[k] = q; pc[k] = c; ps[k] = s; pt[k] = tt;
      }
      __syncthreads();
      for (int w = tid; w < nblk + m * P; w += blockDim.x) {
        if (w < nblk) {
          int a, bb;
          tri_decode(w, P, a, bb);
          float s1 = ps[a], s2 = ps[bb];
          if (s1 == 0.f && s2 == 0.f) continue;
          if (a == bb) {
            int p = pp[a], q = pq[a];
            float apq = Mp[pk(p, q, N)];
            float tt = pt[a];
            Mp[pk(p, p, N)] -= tt * apq;
            Mp[pk(q, q, N)] += tt * apq;
            Mp[pk(p, q, N)] = 0.f;
          } else {
            int p1 = pp[a], q1 = pq[a], p2 = pp[bb], q2 = pq[bb];
            float c1 = pc[a], c2 = pc[bb];
            int i00 = pk(p1, p2, N), i01 = pk(p1, q2, N), i10 = pk(q1, p2, N), i11 = pk(q1, q2, N);
            float x00 = Mp[i00], x01 = Mp[i01], x10 = Mp[i10], x11 = Mp[i11];
            float r00 = c1 * x00 - s1 * x10, r01 = c1 * x01 - s1 * x11;
            float r10 = s1 * x00 + c1 * x10, r11 = s1 * x01 + c1 * x11;
            Mp[i00] = c2 * r00 - s2 * r01;
            Mp[i01] = s2 * r00 + c2 * r01;
            Mp[i10] = c2 * r10 - s2 * r11;
            Mp[i11] = s2 * r10 + c2 * r11;
          }
        } else {
          int item = w - nblk;
          int k = item / m, a = item - k * m;
          float s = ps[k];
          if (s == 0.f) continue;
          float c = pc[k];
          float* row = V + a * Vs;
          float vp = row[pp[k]], vq = row[pq[k]];
          row[pp[k]] = c * vp - s * vq;
          row[pq[k]] = s * vp + c * vq;
        }
      }
      __syncthreads();
    }
    int done = (nrot == 0);
    __syncthreads();
    if (done) break;
  }
  float* outV = b.jV + g.offM[i];
  for (int t = tid; t < m * m; t += blockDim.x) {
    int r = t / m, c = t % m;
    outV[t] = V[r * Vs + c];
  }
  for (int j = tid; j < m; j += blockDim.x) b.jL[g.offL[i] + j] = Mp[pk(j, j, N)];
}

// Fast path for m <= 128: full (both triangles) storage so every 2x2 block (pair a, pair b) is
// updated by its own thread with plain row/column addressing, and block/vector-row ownership is
// fixed for the whole launch. With `warm` set (k >= 1) the basis of the previous iteration
// starts the sweep: M <- V0^T M V0 and V <- V0, so the rotations only have to follow the change
// of M between iterations.
constexpr int kFullMaxN = 128;
constexpr int kFullLd = kFullMaxN + 1;

__global__ void __launch_bounds__(kJacThreads, 1) k_jacobi_full(Geom g, Bufs b, int warm_ok) {
  extern __shared__ float smem[];
  if (b.warm[blockIdx.x]) return;
  __shared__ int nrot;
  __shared__ float tabs;
  __shared__ int pp[kFullMaxN / 2], pq[kFullMaxN / 2];
  __shared__ float pc[kFullMaxN / 2], ps[kFullMaxN / 2], pt[kFullMaxN / 2];
  const int i = blockIdx.x;
  const int m = g.m[i];
  const int N = m + (m & 1);
  const int P = N / 2;
  float* M = smem;                        // N x kFullLd
  float* V = M + kFullMaxN * kFullLd;     // m x kFullLd (row a, column j = vector j)
  float* Tm = V + kFullMaxN * kFullLd;    // scratch for the warm start
  const int tid = threadIdx.x;
  const double* M64 = b.gram + g.offM[i];
  float* outV = b.jV + g.offM[i];
  const bool warm = warm_ok && (b.st->k >= 1);
  for (int t = tid; t < N * N; t += blockDim.x) {
    int r = t / N, c = t - r * N;
    M[r * kFullLd + c] = (r < m && c < m) ? (float)M64[(long long)r * m + c] : 0.f;
  }
  for (int t = tid; t < m * N; t += blockDim.x) {
    int r = t / N, c = t - r * N;
    V[r * kFullLd + c] = warm ? ((c < m) ? outV[(long long)r * m + c] : 0.f) : ((r == c) ? 1.f : 0.f);
  }
  __syncthreads();
  if (warm) {  // M <- V^T M V in FP32 (two passes through the scratch panel)
    for (int t = tid; t < m * m; t += blockDim.x) {
      int r = t / m, c = t - r * m;
      float acc = 0.f;
      for (int u = 0; u < m; ++u) acc = fmaf(M[r * kFullLd + u], V[u * kFullLd + c], acc);
      Tm[r * kFullLd + c] = acc;
    }
    __syncthreads();
    for (int t = tid; t < m * m; t += blockDim.x) {
      int r = t / m, c = t - r * m;
      if (c < r) continue;
      float acc = 0.f;
      for (int u = 0; u < m; ++u) acc = fmaf(V[u * kFullLd + r], Tm[u * kFullLd + c], acc);
      M[r * kFullLd + c] = acc;
      M[c * kFullLd + r] = acc;
    }
    __syncthreads();
  }
  // fixed ownership: up to 4 blocks (P*P <= 4096) and 8 vector items (m*P <= 8192) per thread
  int ba[4], bb[4], nb = 0;
  for (int w = tid; w < P * P && nb < 4; w += blockDim.x, ++nb) { ba[nb] = w / P; bb[nb] = w - ba[nb] * P; }
  int vk[8], vr[8], nv = 0;
  for (int w = tid; w < m * P && nv < 8; w += blockDim.x, ++nv) { vk[nv] = w / m; vr[nv] = w - vk[nv] * m; }
  const float tol = 4.f * 5.9604645e-8f;  // 4 * 2^-24
  for (int sw = 0; sw < g.max_sweeps; ++sw) {
    if (tid == 0) {
      nrot = 0;
      float mx = 0.f;
      for (int j = 0; j < m; ++j) mx = fmaxf(mx, M[j * kFullLd + j]);
      tabs = 5.9604645e-8f * mx;
    }
    __syncthreads();
    for (int rd = 0; rd < N - 1; ++rd) {
      if (tid < P) {
        int k = tid;
        int x = (k == 0) ? 0 : ((k - 1 + rd) % (N - 1)) + 1;
        int y = ((N - 2 - k + rd) % (N - 1)) + 1;
        int p = min(x, y), q = max(x, y);
        float c = 1.f, s2 = 0.f, tt = 0.f;
        if (q < m) {
          float app = M[p * kFullLd + p], aqq = M[q * kFullLd + q], apq = M[p * kFullLd + q];
          if (fabsf(apq) > tol * sqrtf(fabsf(app * aqq)) && fabsf(apq) > tabs) {
            float theta = (aqq - app) / (2.f * apq);
            tt = (theta >= 0.f ? 1.f : -1.f) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
            c = 1.f / sqrtf(tt * tt + 1.f);
            s2 = tt * c;
            atomicAdd(&nrot, 1);
          }
        }
        pp[k] = p; pq[k] = q; pc[k] = c; ps[k] = s2; pt[k] = tt;
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (u >= nb) break;
        const int a = ba[u], c2i = bb[u];
        const float s1 = ps[a], s2 = ps[c2i];
        if (s1 == 0.f && s2 == 0.f) continue;
        const int p1 = pp[a], q1 = pq[a];
        if (a == c2i) {
          float apq = M[p1 * kFullLd + q1];
          float tt = pt[a];
          M[p1 * kFullLd + p1] -= tt * apq;
          M[q1 * kFullLd + q1] += tt * apq;
          M[p1 * kFullLd + q1] = 0.f;
          M[q1 * kFullLd + p1] = 0.f;
        } else {
          const int p2 = pp[c2i], q2 = pq[c2i];
          const float c1 = pc[a], c2 = pc[c2i];
          float* rp = M + p1 * kFullLd;
          float* rq = M + q1 * kFullLd;
          float x00 = rp[p2], x01 = rp[q2], x10 = rq[p2], x11 = rq[q2];
          float r00 = c1 * x00 - s1 * x10, r01 = c1 * x01 - s1 * x11;
          float r10 = s1 * x00 + c1 * x10, r11 = s1 * x01 + c1 * x11;
          rp[p2] = c2 * r00 - s2 * r01;
          rp[q2] = s2 * r00 + c2 * r01;
          rq[p2] = c2 * r10 - s2 * r11;
          rq[q2] = s2 * r10 + c2 * r11;
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (u >= nv) break;
        const int k = vk[u];
        const float s2 = ps[k];
        if (s2 == 0.f) continue;
        const float c = pc[k];
        float* row = V + vr[u] * kFullLd;
        const int p = pp[k], q = pq[k];
        float vp = row[p], vq = row[q];
        row[p] = c * vp - s2 * vq;
        row[q] = s2 * vp + c * vq;
      }
      __syncthreads();
    }
    int done = (nrot == 0);
    __syncthreads();
    if (tid == 0) atomicMax(&b.st->jsweeps, sw + 1);
    if (done) break;
  }
  for (int t = tid; t < m * m; t += blockDim.x) {
    int r = t / m, c = t - r * m;
    outV[t] = V[r * kFullLd + c];
  }
  for (int j = tid; j < m; j += blockDim.x) b.jL[g.offL[i] + j] = M[j * kFullLd + j];
}

// ------------------------------------------------------------------ 2b. FP32 tridiagonal eigensolver
// For m <= 128 the FP32 eigenbasis comes from a tridiagonal reduction instead of Jacobi sweeps
// (about m sequential steps instead of ~9 sweeps of m rounds):
//   a. Householder tridiagonalisation Q^T M Q = T (Golub and Van Loan, Alg. 8.3.1), one warp per
//      row, the reflector and the update vector cached in registers;
//   b. all eigenvalues of T by multisection on Sturm counts (8 shifts per eigenvalue per round,
//      pivots kept away from zero by pivmin as in LAPACK's bisection);
//   c. eigenvectors of T from twisted factorisations (Fernando 1997; Parlett and Dhillon 2000):
//      one stationary and one progressive qd recurrence, the twist index where |gamma_k| is
//      smallest, then two triangular sweeps -- no iteration and no per-thread work arrays.
//      The largest group of eigenvalues closer than 1e-5 ||T|| (in practice the near-zero tail
//      late in the solve) gets the orthogonal complement of all other vectors (Householder QR)
//      as its basis; any other small group is orthogonalised by Gram-Schmidt;
//   d. back-transformation by the stored reflectors, eight threads per column, each holding 16
//      consecutive entries of its column in registers.
// The result only has to be FP32-accurate: the FP64 refinement that follows fixes the top-r
// subspace to FP64 accuracy.
constexpr int kTriMax = 128;
constexpr int kTriLd = kTriMax + 1;

__device__ __forceinline__ float warp_sum_f(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Number of eigenvalues of T below x (Sturm count), pivots bounded away from zero by pivmin.
__device__ int sturm_count(const float* d, const float* e2, int m, float x, float pivmin) {
  int cnt = 0;
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  if (q < 0.f) ++cnt;
  for (int k = 1; k < m; ++k) {
    q = (d[k] - x) - __fdividef(e2[k - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    if (q < 0.f) ++cnt;
  }
  return cnt;
}

// Eigenvector of the tridiagonal T (d, e) for the eigenvalue lam by a twisted factorisation.
// z: output column (stride ld), also used for D-; w: scratch column (stride ld) for L+.
__device__ void twisted_vector(const float* d, const float* e, int m, float lam, float pivmin,
                               float* z, float* w, int ld) {
  float dm = d[m - 1] - lam;
  if (fabsf(dm) < pivmin) dm = pivmin;
  z[(m - 1) * ld] = dm;
  for (int j = m - 2; j >= 0; --j) {
    float u = e[j] / dm;
    dm = (d[j] - lam) - u * e[j];
    if (fabsf(dm) < pivmin) dm = pivmin;
    z[j * ld] = dm;
  }
  float dp = d[0] - lam;
  if (fabsf(dp) < pivmin) dp = pivmin;
  float best = fabsf(dp + z[0] - (d[0] - lam));
  int kb = 0;
  for (int j = 0; j < m - 1; ++j) {
    float l = e[j] / dp;
    w[j * ld] = l;
    dp = (d[j + 1] - lam) - l * e[j];
    if (fabsf(dp) < pivmin) dp = pivmin;
    float gk = fabsf(dp + z[(j + 1) * ld] - (d[j + 1] - lam));
    if (gk < best) { best = gk; kb = j + 1; }
  }
  float zj = 1.f;
  float nn = 1.f;
  for (int j = kb; j < m - 1; ++j) {  // z_{j+1} = -(e_j / D-_{j+1}) z_j
    float zn = -(e[j] / z[(j + 1) * ld]) * zj;
    z[(j + 1) * ld] = zn;
    nn = fmaf(zn, zn, nn);
    zj = zn;
  }
  z[kb * ld] = 1.f;
  zj = 1.f;
  for (int j = kb - 1; j >= 0; --j) {  // z_j = -L+_j z_{j+1}
    float zn = -w[j * ld] * zj;
    z[j * ld] = zn;
    nn = fmaf(zn, zn, nn);
    zj = zn;
  }
  float inv = 1.f / sqrtf(nn);
  for (int j = 0; j < m; ++j) z[j * ld] *= inv;
}

__global__ void __launch_bounds__(kJacThreads, 1) k_eig_tri(Geom g, Bufs b) {
  TL_BEGIN();
  extern __shared__ float smem[];
  if (b.warm[blockIdx.x]) {  // warm attempt certified for this mode
    TL_END(16);
    return;
  }
  __shared__ float dv[kTriMax], ev[kTriMax], e2[kTriMax], tauv[kTriMax], pv[kTriMax];
  __shared__ float lam[kTriMax], qt[kTriMax];
  __shared__ int cid[kTriMax], inbig[kTriMax], known[kTriMax];
  __shared__ float sh_lo, sh_hi, sh_nrm, sh_pivmin;
  __shared__ int sh_big, sh_nknown;
  const int i = blockIdx.x;
  const int m = g.m[i];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  float* A = smem;                       // m x kTriLd: matrix, then reflectors below the diagonal
  float* Z = A + kTriMax * kTriLd;       // m x kTriLd: eigenvectors of T (columns)
  float* Y = Z + kTriMax * kTriLd;       // m x kTriLd: per-vector scratch, then QR work
  const double* M64 = b.gram + g.offM[i];
  long long tph = clock64();
  for (int r = wid; r < m; r += nw)
    for (int c = lane; c < m; c += 32) A[r * kTriLd + c] = (float)M64[(long long)r * m + c];
  __syncthreads();
  PHASE_MARK(tph, "tri.load");
  // ---- a. tridiagonalisation. Two block barriers a step: every warp forms the reflector of
  //         column j itself (the same reduction in the same order, so the same tau and scale in
  //         every warp) instead of waiting for one warp to broadcast it, and reads the reflector
  //         straight from column j; after p = tau A22 v each row's owner stores the reflector's
  //         entry in column j (kept for the back-transformation) as it updates the row.
  for (int j = 0; j + 2 < m; ++j) {
    const int sN = m - j - 1;
    const float x0 = A[(j + 1) * kTriLd + j];
    float nacc = 0.f;
    for (int k = 1 + lane; k < sN; k += 32) {
      const float x = A[(j + 1 + k) * kTriLd + j];
      nacc = fmaf(x, x, nacc);
    }
    nacc = warp_sum_f(nacc);
    float tau = 0.f, scale = 0.f, beta = x0;
    if (nacc != 0.f) {
      const float nrm = sqrtf(x0 * x0 + nacc);
      beta = (x0 >= 0.f) ? -nrm : nrm;
      tau = (beta - x0) / beta;
      scale = 1.f / (x0 - beta);
    }
    if (tid == 0) {
      ev[j] = beta;
      dv[j] = A[j * kTriLd + j];
      tauv[j] = tau;
    }
    if (tau != 0.f) {
      float vreg[4], preg[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = lane + 32 * q;
        vreg[q] = (c < sN) ? ((c == 0) ? 1.f : A[(j + 1 + c) * kTriLd + j] * scale) : 0.f;
      }
      // p = tau * A22 v, one warp per row, four rows per warp reduced together
      for (int rb = wid; rb < sN; rb += 4 * nw) {
        float acc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int rr = rb + u * nw;
          acc[u] = 0.f;
          if (rr < sN) {
            const float* row = A + (j + 1 + rr) * kTriLd + (j + 1);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              int c = lane + 32 * q;
              if (c < sN) acc[u] = fmaf(row[c], vreg[q], acc[u]);
            }
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], o);
        if (lane == 0) {
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (rb + u * nw < sN) pv[rb + u * nw] = tau * acc[u];
        }
      }
      __syncthreads();  // pv complete; every warp has read column j
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int c = lane + 32 * q;
        preg[q] = (c < sN) ? pv[c] : 0.f;
        acc = fmaf(preg[q], vreg[q], acc);
      }
      const float K = 0.5f * tau * warp_sum_f(acc);
      float wreg[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) wreg[q] = preg[q] - K * vreg[q];
      // A22 -= v w^T + w v^T; the reflector entry of the row goes to column j
      for (int r = wid; r < sN; r += nw) {
        float* cj = A + (j + 1 + r) * kTriLd + j;
        const float vr = (r == 0) ? 1.f : cj[0] * scale, wr = pv[r] - K * vr;
        float* arow = cj + 1;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int c = lane + 32 * q;
          if (c < sN) arow[c] = arow[c] - vr * wreg[q] - wr * vreg[q];
        }
        __syncwarp();
        if (lane == 0) cj[0] = vr;
      }
    } else {
      for (int k = tid; k < sN; k += blockDim.x) A[(j + 1 + k) * kTriLd + j] = (k == 0) ? 1.f : 0.f;
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (m >= 2) {
      dv[m - 2] = A[(m - 2) * kTriLd + (m - 2)];
      ev[m - 2] = A[(m - 1) * kTriLd + (m - 2)];
    }
    dv[m - 1] = A[(m - 1) * kTriLd + (m - 1)];
    float lo = 3.4e38f, hi = -3.4e38f, nrm = 0.f;
    for (int k = 0; k < m; ++k) {
      float rad = ((k > 0) ? fabsf(ev[k - 1]) : 0.f) + ((k + 1 < m) ? fabsf(ev[k]) : 0.f);
      lo = fminf(lo, dv[k] - rad);
      hi = fmaxf(hi, dv[k] + rad);
      nrm = fmaxf(nrm, fabsf(dv[k]));
      if (k + 1 < m) nrm = fmaxf(nrm, fabsf(ev[k]));
      e2[k] = (k + 1 < m) ? ev[k] * ev[k] : 0.f;
    }
    float span = fmaxf(fabsf(lo), fabsf(hi));
    sh_lo = lo - 1e-6f * span - 1e-30f;
    sh_hi = hi + 1e-6f * span + 1e-30f;
    sh_nrm = nrm + 1e-30f;
    sh_pivmin = 7.8886091e-31f * fmaxf(1.f, sh_nrm * sh_nrm);  // 2^-100 max(1, ||T||^2)
  }
  __syncthreads();
  PHASE_MARK(tph, "tri.reduce");
  // ---- b. multisection: group of 8 lanes per eigenvalue (ascending index ei)
  {
    const int G = 8;
    const int ei = tid / G, gl = tid % G;
    const unsigned gmask = 0xffu << ((lane / G) * G);
    const float pivmin = sh_pivmin;
    float a = sh_lo, bnd = sh_hi;
    if (ei < m) {
      for (int rd = 0; rd < 40; ++rd) {
        // eigenvalues of the FP32 matrix are only determined to about eps ||T||
        if (bnd - a <= 2.f * 5.9604645e-8f * (fmaxf(fabsf(a), fabsf(bnd)) + sh_nrm)) break;
        float x = a + (bnd - a) * (float)(gl + 1) / (float)(G + 1);
        int cnt = sturm_count(dv, e2, m, x, pivmin);
        float na = a, nb = bnd;
        bool found = false;
        for (int t = 0; t < G; ++t) {
          float xt = __shfl_sync(gmask, x, (lane / G) * G + t);
          int ct = __shfl_sync(gmask, cnt, (lane / G) * G + t);
          if (!found) {
            if (ct <= ei) na = xt;
            else { nb = xt; found = true; }
          }
        }
        a = na;
        bnd = nb;
      }
      if (gl == 0) lam[ei] = 0.5f * (a + bnd);
    }
  }
  __syncthreads();
  PHASE_MARK(tph, "tri.bisect");
  // ---- c. groups, eigenvectors, complement
  if (tid == 0) {
    const float tol = 1e-5f * sh_nrm;
    int c = 0, best = 0, bestsz = 1, cur = 1;
    cid[0] = 0;
    for (int k = 1; k < m; ++k) {
      if (lam[k] - lam[k - 1] > tol) { ++c; cur = 1; }
      else if (++cur > bestsz) { bestsz = cur; best = c; }
      cid[k] = c;
    }
    sh_big = (bestsz >= 2) ? best : -1;
    int nk = 0;
    for (int k = 0; k < m; ++k) {
      inbig[k] = (cid[k] == sh_big) ? 1 : 0;
      if (!inbig[k]) known[nk++] = k;
    }
    sh_nknown = nk;
  }
  __syncthreads();
  if (tid < m && !inbig[tid] && (tid == 0 || cid[tid] != cid[tid - 1])) {
    // this thread owns its whole (non-big) group: members tid .. next group start
    const int c0 = tid;
    int c1 = c0 + 1;
    while (c1 < m && cid[c1] == cid[c0]) ++c1;
    for (int k = c0; k < c1; ++k) {
      float* y = Z + k;  // column k, stride kTriLd
      twisted_vector(dv, ev, m, lam[k], sh_pivmin, y, Y + k, kTriLd);
      if (k > c0) {
        for (int jj = c0; jj < k; ++jj) {  // Gram-Schmidt inside the group
          float dot = 0.f;
          for (int r = 0; r < m; ++r) dot = fmaf(Z[r * kTriLd + jj], y[r * kTriLd], dot);
          for (int r = 0; r < m; ++r) y[r * kTriLd] -= dot * Z[r * kTriLd + jj];
        }
        float nn = 0.f;
        for (int r = 0; r < m; ++r) nn = fmaf(y[r * kTriLd], y[r * kTriLd], nn);
        float inv = (nn > 0.f) ? 1.f / sqrtf(nn) : 0.f;
        for (int r = 0; r < m; ++r) y[r * kTriLd] *= inv;
      }
    }
  }
  __syncthreads();
  PHASE_MARK(tph, "tri.vectors");
  if (sh_big >= 0) {
    // Householder QR of the known vectors (m x nk), then the complement H_1..H_nk [0; I]
    const int nk = sh_nknown;
    for (int r = wid; r < m; r += nw)
      for (int c = lane; c < nk; c += 32) Y[r * kTriLd + c] = Z[r * kTriLd + known[c]];
    __syncthreads();
    for (int j = 0; j < nk; ++j) {
      if (wid == 0) {
        float acc = 0.f;
        for (int r = j + lane; r < m; r += 32) acc = fmaf(Y[r * kTriLd + j], Y[r * kTriLd + j], acc);
        acc = warp_sum_f(acc);
        if (lane == 0) {
          float x0 = Y[j * kTriLd + j];
          float nx = sqrtf(acc);
          float beta = (x0 >= 0.f) ? -nx : nx;
          float v0 = x0 - beta;
          float vn = acc - x0 * x0 + v0 * v0;
          qt[j] = (vn > 0.f) ? 2.f / vn : 0.f;
          Y[j * kTriLd + j] = v0;  // v = [v0, x(j+1:)] kept in column j
        }
      }
      __syncthreads();
      const float t2 = qt[j];
      for (int c = j + 1 + wid; c < nk; c += nw) {
        float acc = 0.f;
        for (int r = j + lane; r < m; r += 32) acc = fmaf(Y[r * kTriLd + j], Y[r * kTriLd + c], acc);
        acc = warp_sum_f(acc) * t2;
        for (int r = j + lane; r < m; r += 32) Y[r * kTriLd + c] -= acc * Y[r * kTriLd + j];
      }
      __syncthreads();
    }
    // complement columns: unit vectors e_{nk + cc}, then H_nk .. H_1 applied in reverse order
    int cc = 0;
    for (int k = 0; k < m; ++k) {
      if (!inbig[k]) continue;
      for (int r = tid; r < m; r += blockDim.x) Z[r * kTriLd + k] = (r == nk + cc) ? 1.f : 0.f;
      ++cc;
    }
    __syncthreads();
    for (int j = nk - 1; j >= 0; --j) {
      const float t2 = qt[j];
      for (int k = wid; k < m; k += nw) {
        if (!inbig[k]) continue;
        float acc = 0.f;
        for (int r = j + lane; r < m; r += 32) acc = fmaf(Y[r * kTriLd + j], Z[r * kTriLd + k], acc);
        acc = warp_sum_f(acc) * t2;
        for (int r = j + lane; r < m; r += 32) Z[r * kTriLd + k] -= acc * Y[r * kTriLd + j];
      }
      __syncthreads();
    }
  }
  __syncthreads();
  PHASE_MARK(tph, "tri.complement");
  // ---- d. back-transformation Z <- H_0 ... H_{m-3} Z: eight threads per column, thread gl of
  //         a column holding rows gl, gl + 8, ..., gl + 120 of it in registers. With this
  //         interleaving the eight threads read eight consecutive rows of a reflector (stored in
  //         column j of A, row stride kTriLd = 1 mod 32 banks) in one conflict-free access; with
  //         16 consecutive rows per thread the same reads hit 4-way bank conflicts.
  {
    const int G = 8;
    const int col = tid / G, gl = tid % G;
    const unsigned gmask = 0xffu << ((lane / G) * G);
    float z[16];
    if (col < m) {
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int r = gl + G * k;
        z[k] = (r < m) ? Z[r * kTriLd + col] : 0.f;
      }
    }
    for (int j = m - 3; j >= 0; --j) {
      const float tau = tauv[j];
      if (tau == 0.f) continue;
      float a[16];
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int r = gl + G * k;
        a[k] = (r > j && r < m) ? A[r * kTriLd + j] : 0.f;
        acc = fmaf(a[k], z[k], acc);
      }
      for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(gmask, acc, o);
      acc *= tau;
#pragma unroll
      for (int k = 0; k < 16; ++k) z[k] -= acc * a[k];
    }
    if (col < m) {
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int r = gl + G * k;
        if (r < m) Z[r * kTriLd + col] = z[k];
      }
    }
  }
  __syncthreads();
  PHASE_MARK(tph, "tri.backtransform");
  float* outV = b.jV + g.offM[i];
  for (int r = wid; r < m; r += nw)
    for (int c = lane; c < m; c += 32) outV[(long long)r * m + c] = Z[r * kTriLd + c];
  for (int j = tid; j < m; j += blockDim.x) b.jL[g.offL[i] + j] = lam[j];
  PHASE_MARK(tph, "tri.store");
  TL_END(5);
}

// ------------------------------------------------------------------ 3. FP64 refinement
// Cluster-wide barrier that also publishes this CTA's global-memory writes to the cluster: the
// arrive has release and the wait acquire semantics at cluster scope, so writes before it are
// visible to every thread of the cluster after it (no GPU-scope fence, whose write
// acknowledgements are slow while the concurrent dense pass saturates the memory system).
__device__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// Shared-memory layout of k_refine (doubles first): own rows of M, the full m x r panels X1, Yw
// and E (each CTA computes its own rows and gathers the others' from their shared memory after a
// cluster barrier), the FP32 basis restricted to this CTA's columns and rows, and a chunk of W
// columns for Y = W^T Q_r Sigma^-2.
constexpr int kWChunk = 32;
constexpr int kWarmMaxSteps = 12;  // subspace-iteration steps a warm attempt may take
// Cold path: when the FP32 eigenvalues put lambda_r below kLowLambda lambda_1 (sigma_r / sigma_1
// below 1e-2, where the FP32 eigenbasis stops resolving eigenvector r), kLowSteps FP64
// subspace-iteration steps replace the Ogita-Aishima refinement.
constexpr float kLowLambda = 1e-4f;
constexpr int kLowSteps = 4;
constexpr double kWarmGate = 1.5;  // attempt only if ||C||_F / lambda_r was below this last time

// 1 / sqrt(d) for d > 0 by Newton's iteration for the inverse square root,
// y <- y + y (1 - d y^2) / 2, from an FP32 seed: the error e of y becomes ~1.5 e^2 per step, so
// two steps take the seed's ~2^-22 to FP64 rounding level. Eight dependent FP64 operations,
// against the two much longer sequences of a correctly rounded sqrt and a division; outside the
// range where the FP32 seed is a normal number it falls back to those.
__device__ __forceinline__ double rsqrt_newton(double d) {
  if (!(d > 1e-35 && d < 1e35)) return 1.0 / sqrt(d);
  double y = (double)rsqrtf((float)d);
  double e = fma(-(d * y), y, 1.0);
  y = fma(0.5 * y, e, y);
  e = fma(-(d * y), y, 1.0);
  return fma(0.5 * y, e, y);
}

// In-place Cholesky of the r x r SPD matrix G (row-major; the lower triangle is read and
// overwritten with L, G = L L^T); inv[j] = 1 / L_jj so triangular solves multiply instead of
// divide (FP64 division is a long dependent sequence on this part). Returns false when a pivot
// is not positive. One thread.
__device__ bool chol_small(double* G, int r, double* inv) {
  for (int j = 0; j < r; ++j) {
    double d = G[j * r + j];
    for (int l = 0; l < j; ++l) d -= G[j * r + l] * G[j * r + l];
    if (!(d > 0.0)) return false;
    const double id = rsqrt_newton(d);
    d *= id;
    G[j * r + j] = d;
    inv[j] = id;
    for (int ii = j + 1; ii < r; ++ii) {
      double v = G[ii * r + j];
      for (int l = 0; l < j; ++l) v -= G[ii * r + l] * G[j * r + l];
      G[ii * r + j] = v * id;
    }
  }
  return true;
}

__host__ __device__ inline size_t refine_smem_bytes(int m, int r, int ncl) {
  int own = (m + ncl - 1) / ncl;
  return sizeof(double) * ((size_t)own * m + 3 * (size_t)m * r) +
         sizeof(float) * (2 * (size_t)own * m + (size_t)m * kWChunk);
}

// 4-byte asynchronous global -> shared copies (no register staging; the copies complete while
// the thread runs on), committed as one group and awaited before the data is read
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the 4 lanes of a quad (lanes 4k..4k+3). GB300 issues a warp-wide FP64 FMA about
// every 64 cycles per sub-partition, so each FP64 dot product of the refinement is split over
// a quad (4 lanes): enough warps to keep all four sub-partitions' FP64 pipes busy, and only
// two shuffle-adds per dot.
__device__ __forceinline__ double quad_sum_d(double v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  return v;
}

// C = A^T B for the m x r panels A, B (row-major, row stride r, shared memory), FP64: entry
// (j, l) is one dot product over a half warp (terms a = lane mod 16), so each warp forms two
// entries at a time and the chain of an entry is m / 16 FMAs and four shuffle-adds. The loop is
// uniform over the block (every lane takes part in every shuffle). sym (A = B): only l <= j is
// formed, and mirrored. The caller synchronises before C is read.
__device__ __forceinline__ void panel_atb(const double* A, const double* B, int m, int r, bool sym,
                                          double* C) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int h = lane >> 4, hl = lane & 15;
  const int ne = sym ? r * (r + 1) / 2 : r * r;
  for (int base = 0; base < ne; base += 2 * nw) {
    const int t = base + 2 * wid + h;
    const bool act = t < ne;
    int j = 0, l = 0;
    if (act) {
      if (sym) {
        while ((j + 1) * (j + 2) / 2 <= t) ++j;
        l = t - j * (j + 1) / 2;
      } else {
        j = t / r;
        l = t - j * r;
      }
    }
    double acc = 0.0;
    if (act)
      for (int a = hl; a < m; a += 16) acc = fma(A[a * r + j], B[a * r + l], acc);
    acc += __shfl_xor_sync(0xffffffffu, acc, 8);
    acc += __shfl_xor_sync(0xffffffffu, acc, 4);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    if (act && hl == 0) {
      C[j * r + l] = acc;
      if (sym) C[l * r + j] = acc;
    }
  }
}

__device__ __forceinline__ void load_panel(double* dst, const double* src, int n) {
  for (int t = threadIdx.x; t < n; t += blockDim.x) dst[t] = src[t];
}

// Panel exchange through distributed shared memory. The rows of an m-row panel are split over
// the cluster's CTAs as [m c / NCL, m (c + 1) / NCL) (row a belongs to rank owner[a]); every CTA
// has written its own rows of the m x r panel sP (same offset in every CTA's shared memory).
// After the cluster barrier (release / acquire at cluster scope, which orders the shared-memory
// writes) each CTA copies the other CTAs' rows from their shared memory. A CTA may overwrite its
// own rows again only after the next cluster barrier, and may exit only after a cluster barrier
// that follows the last exchange.
__device__ __forceinline__ void exchange_panel(double* sP, int m, int r, int crank,
                                            const unsigned char* owner) {
  cluster_barrier();
  cg::cluster_group cl = cg::this_cluster();
  for (int t = threadIdx.x; t < m * r; t += blockDim.x) {
    const int c = owner[t / r];
    if (c != crank) sP[t] = cl.map_shared_rank(sP, (unsigned)c)[t];
  }
  __syncthreads();
}

// mode 1: full refinement after the FP32 eigensolver (skipped for a mode whose warm attempt
//         succeeded). mode 0: warm attempt (k >= 1): three FP64 subspace-iteration steps (more
//         while converging) from the previous iteration's basis (RTCUR-F) or from the current
//         factor's rows on the new index set (RTCUR-R), accepted only when certified (see below).
__global__ void __launch_bounds__(kRefThreads) k_refine(Geom g, Bufs b, int mode) {
  TL_BEGIN();
  extern __shared__ double rsm[];
  cg::cluster_group cl = cg::this_cluster();
  const int crank = (int)cl.block_rank();
  const int NCL = g.ncl;
  const int i = blockIdx.x / NCL;
  const int m = g.m[i], r = g.r[i], q = g.q[i];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int ql = tid & 3, nq = blockDim.x >> 2;  // quad lane, number of quads
  __shared__ int top[RT_MAXR];
  __shared__ int pos_of[RT_MAXM];      // -1 for tail indices, else position in top
  __shared__ double lamT[RT_MAXR];
  __shared__ double Gq[RT_MAXR * RT_MAXR];
  __shared__ double Hs[RT_MAXR * RT_MAXR];
  __shared__ double Yh[RT_MAXR * RT_MAXR];
  __shared__ double wv[RT_MAXR];
  __shared__ double invd[RT_MAXR];
  __shared__ int order[RT_MAXR];
  __shared__ int tie;
  __shared__ float lam[RT_MAXM];
  __shared__ unsigned char rown[RT_MAXM];  // cluster rank that owns each panel row
  for (int a = tid; a < m; a += blockDim.x) {
    if (mode == 1) lam[a] = b.jL[g.offL[i] + a];  // the FP32 spectrum (not yet formed in mode 0)
    int c = (a * NCL) / m;
    while (c + 1 < NCL && (m * (c + 1)) / NCL <= a) ++c;
    while (c > 0 && (m * c) / NCL > a) --c;
    rown[a] = (unsigned char)c;
  }
  __syncthreads();
  const float* Xh = b.jV + g.offM[i];               // m x m, column j = vector j
  const double* M = b.gram + g.offM[i];
  double* Qr = b.Qr + g.offQ[i];
  double* sig = b.sig + g.offR[i];
  double* Yout = b.Y + g.offY[i];
  const long long* set = set_of(g, b);
  const int lo = (m * crank) / NCL, hi = (m * (crank + 1)) / NCL;
  const int own = hi - lo;
  const int ownmax = (m + NCL - 1) / NCL;
  double* sM = rsm;                         // own x m
  double* sX1 = sM + (size_t)ownmax * m;     // m x r
  double* sYw = sX1 + (size_t)m * r;         // m x r
  double* sE = sYw + (size_t)m * r;          // m x r
  float* sXc = reinterpret_cast<float*>(sE + (size_t)m * r);  // m x own: Xh[a][lo + j]
  float* sXr = sXc + (size_t)ownmax * m;     // own x m: Xh[lo + j][ii]
  float* sW = sXr + (size_t)ownmax * m;      // m x kWChunk

  long long tph = clock64();
  int wsteps = 3, wtotal = 0;  // warm attempt: steps of the next round, steps taken so far
  __shared__ int warm_retry;
  int* warm_flag = b.warm + i;
  if (mode == 1 && *warm_flag) {  // the warm attempt already produced this mode's factors
    TL_END(15);
    return;
  }
  if (mode == 0) {
    if (tid == 0 && crank == 0) *warm_flag = 0;
    if (b.st->k < 1) return;
    // skip the attempt when the last iteration's spectrum had no usable gap: its complement
    // block was at least kWarmGate times lambda_r, and the block moves slowly between iterations
    if (b.wratio[i] > kWarmGate) return;
  }
  // the first chunk of W's columns for Y = W^T P, fetched while the refinement runs
  const int blo = (q * crank) / NCL, bhi = (q * (crank + 1)) / NCL;
  {
    const int cn = min(kWChunk, bhi - blo);
    const float* Wi = b.W + g.offW[i];
    for (int t = tid; t < m * cn; t += blockDim.x) {
      int cc = t / m, a = t - cc * m;
      cp_async4(&sW[a * kWChunk + cc], Wi + (long long)a * q + blo + cc);
    }
    cp_async_commit();
  }
  if (tid == 0) tie = 0;
  // the FP32 eigenbasis and its top-r columns: the cold path only (the warm attempt runs before
  // the eigensolver of this iteration)
  if (mode == 1 && wid == 0) {
    // the r largest eigenvalues, descending, ties broken by the lower index: each round takes
    // the warp's (largest value, lowest index) among the indices not yet taken
    for (int a = lane; a < m; a += 32) pos_of[a] = -1;
    __syncwarp();
    for (int j = 0; j < r; ++j) {
      float bv = 0.f;
      int bi = -1;
      for (int a = lane; a < m; a += 32)
        if (pos_of[a] < 0 && (bi < 0 || lam[a] > bv)) { bv = lam[a]; bi = a; }
      for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi >= 0 && (bi < 0 || ov > bv || (ov == bv && oi < bi))) { bv = ov; bi = oi; }
      }
      if (lane == 0) {
        top[j] = bi;
        pos_of[bi] = j;
      }
      __syncwarp();
    }
    if (crank == 0) {  // the gate for the next warm attempt, from this spectrum
      double t2 = 0.0;
      for (int a = lane; a < m; a += 32)
        if (pos_of[a] < 0) t2 += (double)lam[a] * (double)lam[a];
      t2 = warp_sum_d(t2);
      const double lr = (double)lam[top[r - 1]];
      if (lane == 0) b.wratio[i] = (lr > 0.0) ? sqrt(t2) / lr : 1e30;
    }
  }
  for (int t = tid; t < own * m; t += blockDim.x) {
    int a = t / m, c = t - a * m;
    sM[t] = M[(long long)(lo + a) * m + c];
  }
  if (mode == 1) {
    for (int t = tid; t < own * m; t += blockDim.x) {
      int a = t / m, c = t - a * m;
      sXr[t] = Xh[(long long)(lo + a) * m + c];
    }
    for (int t = tid; t < m * own; t += blockDim.x) {
      int a = t / own, j = t - a * own;
      sXc[t] = Xh[(long long)a * m + lo + j];
    }
  }
  __syncthreads();
  __shared__ int chol_ok;
  // One FP64 subspace-iteration step with a Cholesky QR: X1 <- (M X1) L^-T, L L^T = (M X1)^T (M X1).
  // Each CTA forms its own rows of Y = M X1, the panel Y is exchanged, and every CTA then forms the
  // whole new X1 = Y L^-T itself (the same data and order in every CTA, so the copies agree bit
  // for bit): one cluster exchange per step. Y alternates between the panels sYw and sE, so a CTA
  // writes a panel again only after the next step's barrier, by which every CTA has finished
  // reading it; after a run of steps the caller passes one more cluster barrier before sYw or sE
  // is written again.
  // False when the Cholesky fails, or when a pivot of L falls below min_pivot L_00 (a column of
  // M X1 with no resolvable part outside the others); the same data in every CTA of the cluster
  // gives a uniform outcome.
  int sstep = 0;
  auto subspace_step = [&](double min_pivot) -> bool {
    double* sYb = (sstep & 1) ? sE : sYw;
    ++sstep;
    for (int t0 = tid >> 2; t0 < ((own * r + nq - 1) / nq) * nq; t0 += nq) {
      const int t = t0;
      const bool act = t < own * r;
      int a = act ? t / r : 0, j = act ? t - a * r : 0;
      double acc = 0.0;
      if (act) {
        const double* Ma = sM + (size_t)a * m;
        for (int c = ql; c < m; c += 4) acc = fma(Ma[c], sX1[c * r + j], acc);
      }
      acc = quad_sum_d(acc);
      if (act && ql == 0) sYb[(lo + a) * r + j] = acc;
    }
    exchange_panel(sYb, m, r, crank, rown);
    panel_atb(sYb, sYb, m, r, true, Gq);
    __syncthreads();
    if (tid == 0) {
      chol_ok = chol_small(Gq, r, invd) ? 1 : 0;
      for (int j = 1; j < r && chol_ok; ++j)
        if (Gq[j * r + j] <= min_pivot * Gq[0]) chol_ok = 0;
    }
    __syncthreads();
    if (!chol_ok) {
      cluster_barrier();  // the other CTAs may still be reading this CTA's rows of sYb
      return false;
    }
    for (int a = tid; a < m; a += blockDim.x) {
      double y[RT_MAXR];
#pragma unroll
      for (int j = 0; j < RT_MAXR; ++j) {
        if (j < r) {
          double v = sYb[a * r + j];
          for (int l = 0; l < j; ++l) v -= Gq[j * r + l] * y[l];
          y[j] = v * invd[j];
        }
      }
#pragma unroll
      for (int j = 0; j < RT_MAXR; ++j)
        if (j < r) sX1[a * r + j] = y[j];  // all rows: no thread reads sX1 in this phase
    }
    __syncthreads();
    return true;
  };
  int oa_steps = g.refine_steps;  // Ogita-Aishima steps of the cold path
  if (mode == 0) {
    // warm start, then FP64 subspace iteration. RTCUR-F keeps its index sets, so the previous
    // iteration's top-r basis of W_i (complete in global memory) starts it. RTCUR-R draws new sets
    // each iteration, so the start is the current iterate's factor restricted to the new rows,
    // B_i(I_i, :) of L^(k): W_i = C_i(I_i, :) takes its columns from X - S, which L^(k) approximates,
    // so its top-r left singular subspace is close to span B_i(I_i, :) (the first step
    // orthonormalises it).
    if (g.variant == 0) {
      load_panel(sX1, Qr, m * r);
    } else {
      const float* Bk = b.B[b.st->k & 1] + g.offB[i];
      for (int t = tid; t < m * r; t += blockDim.x) {
        const int a = t / r, j = t - a * r;
        sX1[t] = (double)Bk[set[g.ioff[i] + a] * r + j];
      }
    }
    __syncthreads();
  warm_steps:
    for (int it = 0; it < wsteps; ++it)
      if (!subspace_step(0.0)) {  // not certified: the full path runs
        cp_async_wait_all();
        return;
      }
    cluster_barrier();  // every CTA has read the last step's panel
    wtotal += wsteps;
    oa_steps = 0;
  } else {
  for (int t = tid; t < m * r; t += blockDim.x) {
    int a = t / r, j = t % r;
    sX1[t] = (double)Xh[(long long)a * m + top[j]];
  }
  __syncthreads();
  // lambda_r below the resolution of the FP32 eigenbasis (its eigenvalues carry an absolute
  // error of about m 2^-24 lambda_1): the FP32 basis does not resolve eigenvector r from the
  // complement, and the refinement below, which divides by FP32 eigenvalue gaps, cannot repair
  // it. FP64 subspace iteration from that basis can: each step shrinks the complement's share by
  // lambda_{r+1} / lambda_r. When eigenvalue r itself is at FP64's noise level (a rank-deficient
  // W, whose direction r the SVD_r cutoff drops anyway) a step finds no resolvable column and the
  // refinement runs as before, from the last good basis.
  if (lam[top[r - 1]] < kLowLambda * lam[top[0]]) {
    int done = 0;
    for (int it = 0; it < kLowSteps; ++it) {
      if (!subspace_step(1e-12)) break;
      ++done;
    }
    if (done == kLowSteps) {
      cluster_barrier();  // every CTA has read the last step's panel
      oa_steps = 0;
    }
  }
  }
  PHASE_MARK(tph, "ref.init");
  for (int step = 0; step < oa_steps; ++step) {
    // S1: Yw = M X1 on own rows (one quad per output)
    for (int t0 = tid >> 2; t0 < ((own * r + nq - 1) / nq) * nq; t0 += nq) {
      const int t = t0;
      double acc = 0.0;
      int a = 0, j = 0;
      if (t < own * r) {
        a = t / r; j = t - a * r;
        const double* Ma = sM + (size_t)a * m;
        for (int c = ql; c < m; c += 4) acc = fma(Ma[c], sX1[c * r + j], acc);
      }
      acc = quad_sum_d(acc);
      if (t < own * r && ql == 0) sYw[(lo + a) * r + j] = acc;
    }
    exchange_panel(sYw, m, r, crank, rown);
    // Rayleigh quotients of the current top columns (every CTA, redundantly)
    for (int j = wid; j < r; j += nw) {
      double s1 = 0.0, nn = 0.0;
      for (int a = lane; a < m; a += 32) {
        double x = sX1[a * r + j];
        s1 = fma(x, sYw[a * r + j], s1);
        nn = fma(x, x, nn);
      }
      s1 = warp_sum_d(s1);
      nn = warp_sum_d(nn);
      if (lane == 0) lamT[j] = s1 / nn;
    }
    __syncthreads();
    double lmax = lamT[0];
    for (int j = 1; j < r; ++j) lmax = fmax(lmax, lamT[j]);
    // S2: E for own basis indices ii; the basis is Xh with its top columns replaced by X1
    for (int t0 = tid >> 2; t0 < ((own * r + nq - 1) / nq) * nq; t0 += nq) {
      const int t = t0;
      const bool act = t < own * r;
      int jj = act ? t / r : 0, j = act ? t - jj * r : 0;
      int ii = lo + jj;
      int pi = act ? pos_of[ii] : 0;
      double s1 = 0.0, dot = 0.0;
      if (act) {
        if (pi >= 0) {
          for (int a = ql; a < m; a += 4) {
            double xf = sX1[a * r + pi];
            s1 = fma(xf, sYw[a * r + j], s1);
            dot = fma(xf, sX1[a * r + j], dot);
          }
        } else {
          for (int a = ql; a < m; a += 4) {
            double xf = (double)sXc[a * own + jj];
            s1 = fma(xf, sYw[a * r + j], s1);
            dot = fma(xf, sX1[a * r + j], dot);
          }
        }
      }
      s1 = quad_sum_d(s1);
      dot = quad_sum_d(dot);
      if (!act || ql != 0) continue;
      double Rij = ((pi == j) ? 1.0 : 0.0) - dot;
      double Eij;
      if (pi >= 0) {
        Eij = 0.5 * Rij;
      } else {
        double den = lamT[j] - (double)lam[ii];
        if (fabs(den) > 1e-6 * fabs(lmax)) {
          Eij = (s1 + lamT[j] * Rij) / den;
        } else {
          Eij = 0.5 * Rij;
          tie = 1;
        }
      }
      sE[ii * r + j] = Eij;  // own basis indices (no thread reads sE in this phase)
    }
    exchange_panel(sE, m, r, crank, rown);
    // S3: X1 <- X1 + Xf E on own rows (one quad per output)
    for (int t0 = tid >> 2; t0 < ((own * r + nq - 1) / nq) * nq; t0 += nq) {
      const int t = t0;
      const bool act = t < own * r;
      int a = act ? t / r : 0, j = act ? t - a * r : 0;
      double upd = 0.0;
      if (act) {
        const float* xr = sXr + (size_t)a * m;
        for (int ii = ql; ii < m; ii += 4) {
          int pi = pos_of[ii];
          double xf = (pi >= 0) ? sX1[(lo + a) * r + pi] : (double)xr[ii];
          upd = fma(xf, sE[ii * r + j], upd);
        }
      }
      upd = quad_sum_d(upd);
      // staged in sYw (not read in this phase; the other CTAs finished reading it before the last
      // exchange), because other threads still read sX1's own rows
      if (act && ql == 0) sYw[(lo + a) * r + j] = sX1[(lo + a) * r + j] + upd;
    }
    __syncthreads();
    for (int t = tid; t < own * r; t += blockDim.x) sX1[lo * r + t] = sYw[lo * r + t];
    exchange_panel(sX1, m, r, crank, rown);
    PHASE_MARK(tph, "ref.step");
  }
  // Fast finish. L needs only the top-r invariant subspace: for any basis X1 of it,
  // (M_r)^+ = X1 H^-1 X1^T with H = X1^T M X1, so U_i^+ = W^T X1 H^-1 X1^T, B_i = C_i W^T X1 H^-1
  // and G = R x_i X1^T give the same L as the singular-vector form. This needs one r x r FP64
  // Cholesky and no eigenvectors. It is taken when H is far from the SVD_r cutoff (its FP32
  // eigenvalues satisfy lambda_min > 1e-6 lambda_max, so every sigma_j exceeds the cutoff
  // max(m, q) 2^-24 sigma_1 by orders of magnitude); otherwise the exact path below runs.
  for (int t0 = tid >> 2; t0 < ((own * r + nq - 1) / nq) * nq; t0 += nq) {
    const int t = t0;
    const bool act = t < own * r;
    int a = act ? t / r : 0, j = act ? t - a * r : 0;
    double acc = 0.0;
    if (act) {
      const double* Ma = sM + (size_t)a * m;
      for (int c = ql; c < m; c += 4) acc = fma(Ma[c], sX1[c * r + j], acc);
    }
    acc = quad_sum_d(acc);
    if (act && ql == 0) sYw[(lo + a) * r + j] = acc;
  }
  exchange_panel(sYw, m, r, crank, rown);
  panel_atb(sX1, sYw, m, r, false, Hs);
  __syncthreads();
  __shared__ int fast_ok;
  __shared__ double cert[3];
  if (mode == 0) {
    // certificate, summed over the cluster (own rows): ||M||_F^2, ||R||_F^2 with
    // R = M X - X H, and ||M X||_F^2
    double fmp = 0.0, rsp = 0.0, mxp = 0.0;
    for (int t = tid; t < own * m; t += blockDim.x) fmp = fma(sM[t], sM[t], fmp);
    for (int t = tid; t < own * r; t += blockDim.x) {
      int a = t / r, j = t - a * r;
      double mx = sYw[(lo + a) * r + j];
      double v = mx;
      for (int l = 0; l < r; ++l) v -= sX1[(lo + a) * r + l] * Hs[l * r + j];
      rsp = fma(v, v, rsp);
      mxp = fma(mx, mx, mxp);
    }
    fmp = warp_sum_d(fmp);
    rsp = warp_sum_d(rsp);
    mxp = warp_sum_d(mxp);
    __shared__ double wpart[3][32];
    if (lane == 0) { wpart[0][wid] = fmp; wpart[1][wid] = rsp; wpart[2][wid] = mxp; }
    __syncthreads();
    __shared__ double cslot[3];  // this CTA's partials, read by the cluster's CTAs in rank order
    if (tid == 0) {
      double a0 = 0.0, a1 = 0.0, a2 = 0.0;
      for (int w = 0; w < nw; ++w) { a0 += wpart[0][w]; a1 += wpart[1][w]; a2 += wpart[2][w]; }
      cslot[0] = a0;
      cslot[1] = a1;
      cslot[2] = a2;
    }
    cluster_barrier();
    if (wid == 0) {  // the cluster's partials read in parallel, summed in rank order
      double v0 = 0.0, v1 = 0.0, v2 = 0.0;
      if (lane < NCL) {
        const double* slot = cl.map_shared_rank(cslot, (unsigned)lane);
        v0 = slot[0];
        v1 = slot[1];
        v2 = slot[2];
      }
      double a0 = 0.0, a1 = 0.0, a2 = 0.0;
      for (int c2 = 0; c2 < NCL; ++c2) {
        a0 += __shfl_sync(0xffffffffu, v0, c2);
        a1 += __shfl_sync(0xffffffffu, v1, c2);
        a2 += __shfl_sync(0xffffffffu, v2, c2);
      }
      if (lane == 0) {
        cert[0] = a0;
        cert[1] = a1;
        cert[2] = a2;
      }
    }
    __syncthreads();
  }
  // FP32 eigenvalues of H for the conditioning test: cyclic Jacobi on an r x r copy by warp 0
  // (each rotation's row and column updates spread over the lanes, its angle computed by every
  // lane from the same shared values); meanwhile thread 32 forms the FP64 Cholesky factor of H
  // that the fast finish uses
  __shared__ float hf[RT_MAXR * RT_MAXR];
  __shared__ int hchol_ok;
  if (wid == 0) {
    for (int t = lane; t < r * r; t += 32) {
      int j = t / r, l = t % r;
      hf[t] = (float)(0.5 * (Hs[j * r + l] + Hs[l * r + j]));
    }
    __syncwarp();
    for (int sw = 0; sw < 30; ++sw) {
      int nrot = 0;
      for (int p = 0; p < r - 1; ++p)
        for (int qq = p + 1; qq < r; ++qq) {
          const float apq = hf[p * r + qq], app = hf[p * r + p], aqq = hf[qq * r + qq];
          if (apq == 0.f || fabsf(apq) <= 1e-7f * sqrtf(fabsf(app * aqq))) continue;
          ++nrot;
          const float th = (aqq - app) / (2.f * apq);
          const float tt = (th >= 0.f ? 1.f : -1.f) / (fabsf(th) + sqrtf(th * th + 1.f));
          const float c = 1.f / sqrtf(tt * tt + 1.f), sn = tt * c;
          __syncwarp();  // every lane has read the pivot entries
          for (int l = lane; l < r; l += 32) {
            const float hp = hf[p * r + l], hq = hf[qq * r + l];
            hf[p * r + l] = c * hp - sn * hq;
            hf[qq * r + l] = sn * hp + c * hq;
          }
          __syncwarp();
          for (int l = lane; l < r; l += 32) {
            const float hp = hf[l * r + p], hq = hf[l * r + qq];
            hf[l * r + p] = c * hp - sn * hq;
            hf[l * r + qq] = sn * hp + c * hq;
          }
          __syncwarp();
        }
      if (nrot == 0) break;
    }
  } else if (tid == 32) {
    for (int t = 0; t < r * r; ++t) Gq[t] = 0.5 * (Hs[t] + Hs[(t % r) * r + t / r]);
    hchol_ok = chol_small(Gq, r, invd) ? 1 : 0;
  }
  __syncthreads();
  if (tid == 0) {
    float lmx = 0.f, lmn = 3.4e38f;
    for (int j = 0; j < r; ++j) { lmx = fmaxf(lmx, hf[j * r + j]); lmn = fminf(lmn, hf[j * r + j]); }
    fast_ok = (lmx > 0.f && lmn > 1e-6f * lmx) ? 1 : 0;
    warm_retry = 0;
    if (mode == 0 && fast_ok) {
      // In the basis [X, X_perp] (X orthonormal), M = [[H, B^T], [B, C]] with ||B||_F = ||R||_F
      // and ||C||_F^2 = ||M||_F^2 - ||M X||_F^2 - ||R||_F^2. ||C||_F bounds the largest eigenvalue
      // outside span(X). If it is below lambda_min(H) / 2 and ||R|| is tiny, Weyl's inequality
      // separates the top r eigenvalues of M from the rest by about lambda_min(H) / 2 and the
      // sin-theta theorem bounds the error of span(X) by ~2 ||R|| / lambda_min(H).
      const double c2 = cert[0] - cert[2] - cert[1];
      const double lmin = (double)lmn;
      const bool tail_ok = sqrt(fmax(c2, 0.0)) < 0.5 * lmin;
      const bool res_ok = sqrt(fmax(cert[1], 0.0)) <= 1e-11 * lmin;
      if (!(tail_ok && res_ok)) fast_ok = 0;
      if (crank == 0) b.wratio[i] = sqrt(fmax(c2, 0.0)) / lmin;
      // separated but not yet converged: more subspace steps (each shrinks the error by the
      // ratio lambda_{r+1} / lambda_r, about 1/2 or less once the tail test passes)
      if (tail_ok && !res_ok && wtotal + 2 <= kWarmMaxSteps) warm_retry = 1;
    }
    if (fast_ok) {
      // singular values (diagnostic), descending
      for (int j = 0; j < r; ++j) wv[j] = sqrt((double)fmaxf(hf[j * r + j], 0.f));
      for (int j = 0; j < r; ++j)
        for (int l = j + 1; l < r; ++l)
          if (wv[l] > wv[j]) { double t = wv[j]; wv[j] = wv[l]; wv[l] = t; }
      // FP64 Cholesky H = L L^T (in Gq, formed above)
      if (!hchol_ok) fast_ok = 0;
    }
    if (tie && crank == 0) atomicOr(&b.st->flags, 2);
    else if (tie) atomicOr(&b.st->flags, 2);
  }
  __syncthreads();
  if (mode == 0 && warm_retry) {  // uniform: every CTA of the cluster sums the same slots
    wsteps = 2;
    goto warm_steps;
  }
  if (fast_ok) {
    // P = X1 H^-1 on own rows (solve L L^T p = x1_a), Qr = X1
    for (int a = lo + tid; a < hi; a += blockDim.x) {
      double y[RT_MAXR];
#pragma unroll
      for (int j = 0; j < RT_MAXR; ++j) {
        if (j < r) {
          double v = sX1[a * r + j];
          for (int l = 0; l < j; ++l) v -= Gq[j * r + l] * y[l];
          y[j] = v * invd[j];
        }
      }
#pragma unroll
      for (int j = RT_MAXR - 1; j >= 0; --j) {
        if (j < r) {
          double v = y[j];
          for (int l = j + 1; l < r; ++l) v -= Gq[l * r + j] * y[l];
          y[j] = v * invd[j];
        }
      }
#pragma unroll
      for (int j = 0; j < RT_MAXR; ++j)
        if (j < r) {
          sE[a * r + j] = y[j];  // own rows (sE is not read in this phase)
          Qr[(long long)a * r + j] = sX1[a * r + j];
        }
    }
    if (crank == 0 && tid < r) sig[tid] = wv[tid];
    exchange_panel(sE, m, r, crank, rown);  // sE holds P = X1 H^-1
    // Y = W^T P (q x r) on own columns of W (the first chunk was prefetched at entry)
    for (int c0 = blo; c0 < bhi; c0 += kWChunk) {
      const int cn = min(kWChunk, bhi - c0);
      if (c0 == blo) {
        cp_async_wait_all();
      } else {
        for (int t = tid; t < m * cn; t += blockDim.x) {
          int cc = t / m, a = t - cc * m;
          sW[a * kWChunk + cc] = w_entry(g, b, set, i, a, c0 + cc);
        }
      }
      __syncthreads();
      for (int t0 = tid >> 2; t0 < ((cn * r + nq - 1) / nq) * nq; t0 += nq) {
        const int t = t0;
        const bool act = t < cn * r;
        int cc = act ? t / r : 0, j = act ? t - cc * r : 0;
        double acc = 0.0;
        if (act)
          for (int a = ql; a < m; a += 4) acc = fma((double)sW[a * kWChunk + cc], sE[a * r + j], acc);
        acc = quad_sum_d(acc);
        if (act && ql == 0) Yout[(long long)(c0 + cc) * r + j] = acc;
      }
      __syncthreads();
    }
    if (mode == 0 && crank == 0 && tid == 0) {
      *warm_flag = 1;
      atomicAdd((unsigned long long*)&b.st->warm_hits, 1ull);
    }
    PHASE_MARK(tph, "ref.fast");
    TL_END(4 + 10 * mode);
    cluster_barrier();  // no CTA leaves while another still reads its shared memory
    return;
  }
  if (mode == 0) {  // not certified: the eigensolver and the full refinement run
    cp_async_wait_all();
    cluster_barrier();  // no CTA leaves while another still reads its shared memory
    return;
  }
  // ---- exact path (H close to the SVD_r cutoff): singular vectors and the cutoff
  // F1: orthonormalise X1 (Cholesky QR in FP64)
  panel_atb(sX1, sX1, m, r, true, Gq);
  __syncthreads();
  if (tid == 0) {  // Gq <- L (lower Cholesky factor), in place
    for (int j = 0; j < r; ++j) {
      double d = Gq[j * r + j];
      for (int l = 0; l < j; ++l) d -= Gq[j * r + l] * Gq[j * r + l];
      d = (d > 0.0) ? sqrt(d) : 0.0;
      Gq[j * r + j] = d;
      for (int ii = j + 1; ii < r; ++ii) {
        double v = Gq[ii * r + j];
        for (int l = 0; l < j; ++l) v -= Gq[ii * r + l] * Gq[j * r + l];
        Gq[ii * r + j] = (d > 0.0) ? v / d : 0.0;
      }
    }
  }
  __syncthreads();
  // Q = X1 L^-T on own rows: row a solves L y = x (forward substitution)
  for (int a = lo + tid; a < hi; a += blockDim.x) {
    double y[RT_MAXR];
#pragma unroll
    for (int j = 0; j < RT_MAXR; ++j) {
      if (j < r) {
        double v = sX1[a * r + j];
        for (int l = 0; l < j; ++l) v -= Gq[j * r + l] * y[l];
        double d = Gq[j * r + j];
        y[j] = (d > 0.0) ? v / d : 0.0;
      }
    }
#pragma unroll
    for (int j = 0; j < RT_MAXR; ++j)
      if (j < r) sX1[a * r + j] = y[j];  // in place: this thread alone reads and writes row a
  }
  exchange_panel(sX1, m, r, crank, rown);  // sX1 now holds Q
  // F2: Yw = M Q on own rows (one quad per output)
  for (int t0 = tid >> 2; t0 < ((own * r + nq - 1) / nq) * nq; t0 += nq) {
    const int t = t0;
    const bool act = t < own * r;
    int a = act ? t / r : 0, j = act ? t - a * r : 0;
    double acc = 0.0;
    if (act) {
      const double* Ma = sM + (size_t)a * m;
      for (int c = ql; c < m; c += 4) acc = fma(Ma[c], sX1[c * r + j], acc);
    }
    acc = quad_sum_d(acc);
    if (act && ql == 0) sYw[(lo + a) * r + j] = acc;
  }
  exchange_panel(sYw, m, r, crank, rown);
  PHASE_MARK(tph, "ref.qr+MQ");
  // F3: H = Q^T M Q (r x r), its eigenpairs by FP64 cyclic Jacobi, cutoff of SVD_r
  panel_atb(sX1, sYw, m, r, false, Hs);
  __syncthreads();
  if (tid == 0) {
    for (int j = 0; j < r; ++j) {  // symmetrise, identity start
      for (int l = j + 1; l < r; ++l) {
        double v = 0.5 * (Hs[j * r + l] + Hs[l * r + j]);
        Hs[j * r + l] = Hs[l * r + j] = v;
      }
      for (int l = 0; l < r; ++l) Yh[j * r + l] = (j == l) ? 1.0 : 0.0;
    }
    for (int sw = 0; sw < 30; ++sw) {
      int nrot = 0;
      for (int p = 0; p < r - 1; ++p)
        for (int qq = p + 1; qq < r; ++qq) {
          double apq = Hs[p * r + qq];
          double app = Hs[p * r + p], aqq = Hs[qq * r + qq];
          // skip pairs already diagonal to working precision (no square root needed)
          if (apq * apq <= 1e-32 * fabs(app * aqq) || apq == 0.0) continue;
          ++nrot;
          // rotation angle from FP32 (an inexact angle only leaves a smaller off-diagonal for
          // the next sweep); the rotation itself is orthogonal to FP64 accuracy
          float thf = (float)((aqq - app) / 2.0) / (float)apq;
          float tf = (thf >= 0.f ? 1.f : -1.f) / (fabsf(thf) + sqrtf(thf * thf + 1.f));
          double tt = (double)tf;
          double x = 1.0 + tt * tt;
          double y = (double)rsqrtf((float)x);
          y = y * (1.5 - 0.5 * x * y * y);
          y = y * (1.5 - 0.5 * x * y * y);
          double c = y, s1 = tt * c;
          for (int l = 0; l < r; ++l) {  // rows p, q
            double hp = Hs[p * r + l], hq = Hs[qq * r + l];
            Hs[p * r + l] = c * hp - s1 * hq;
            Hs[qq * r + l] = s1 * hp + c * hq;
          }
          for (int l = 0; l < r; ++l) {  // columns p, q
            double hp = Hs[l * r + p], hq = Hs[l * r + qq];
            Hs[l * r + p] = c * hp - s1 * hq;
            Hs[l * r + qq] = s1 * hp + c * hq;
          }
          for (int l = 0; l < r; ++l) {
            double yp = Yh[l * r + p], yq = Yh[l * r + qq];
            Yh[l * r + p] = c * yp - s1 * yq;
            Yh[l * r + qq] = s1 * yp + c * yq;
          }
        }
      if (nrot == 0) break;
    }
    for (int j = 0; j < r; ++j) order[j] = j;
    for (int j = 0; j < r; ++j)  // sort eigenvalues descending (selection)
      for (int l = j + 1; l < r; ++l)
        if (Hs[order[l] * r + order[l]] > Hs[order[j] * r + order[j]]) {
          int t = order[j]; order[j] = order[l]; order[l] = t;
        }
    double s1 = sqrt(fmax(Hs[order[0] * r + order[0]], 0.0));
    double tau = (double)max(m, q) * 5.9604644775390625e-08 * s1;  // max(m,q) * 2^-24 * s_1
    int kept = 0;
    for (int j = 0; j < r; ++j) {
      double sj = sqrt(fmax(Hs[order[j] * r + order[j]], 0.0));
      bool keep = (sj > tau) && (s1 > 0.0);
      wv[j] = keep ? sj : 0.0;
      kept += keep ? 1 : 0;
    }
    int fl = 0;
    if (kept < r) fl |= 1;   // RTCUR_FLAG_RANK_DEFICIENT
    if (tie) fl |= 2;        // RTCUR_FLAG_TIE
    if (crank != 0) fl &= 2;
    if (fl) atomicOr(&b.st->flags, fl);
  }
  __syncthreads();
  // Q_r = Q Yh(:, order) on own rows, singular values
  for (int t = tid; t < own * r; t += blockDim.x) {
    int a = lo + t / r, j = t % r;
    double acc = 0.0;
    for (int l = 0; l < r; ++l) acc = fma(sX1[a * r + l], Yh[l * r + order[j]], acc);
    const double qv = (wv[j] > 0.0) ? acc : 0.0;
    Qr[(long long)a * r + j] = qv;
    sE[a * r + j] = qv;  // own rows (sE is not read in this phase)
  }
  if (crank == 0 && tid < r) sig[tid] = wv[tid];
  PHASE_MARK(tph, "ref.rr");
  exchange_panel(sE, m, r, crank, rown);  // sE now holds Q_r
  // F4: Y = W^T Q_r Sigma^-2 (q x r) on own columns of W, staged kWChunk columns at a time (the
  // first chunk was prefetched at entry)
  for (int c0 = blo; c0 < bhi; c0 += kWChunk) {
    const int cn = min(kWChunk, bhi - c0);
    if (c0 == blo) {
      cp_async_wait_all();
    } else {
      for (int t = tid; t < m * cn; t += blockDim.x) {
        int cc = t / m, a = t - cc * m;
        sW[a * kWChunk + cc] = w_entry(g, b, set, i, a, c0 + cc);
      }
    }
    __syncthreads();
    for (int t = wid; t < cn * r; t += nw) {
      int cc = t / r, j = t - cc * r;
      double acc = 0.0;
      if (wv[j] > 0.0) {
        for (int a = lane; a < m; a += 32) acc = fma((double)sW[a * kWChunk + cc], sE[a * r + j], acc);
        acc = warp_sum_d(acc) / (wv[j] * wv[j]);
      }
      if (lane == 0) Yout[(long long)(c0 + cc) * r + j] = acc;
    }
    __syncthreads();
  }
  PHASE_MARK(tph, "ref.Y");
  TL_END(4 + 10 * mode);
  cluster_barrier();  // no CTA leaves while another still reads its shared memory
}

}  // namespace

size_t jacobi_smem_bytes(int m) {
  int N = m + (m & 1);
  int P = N / 2;
  return sizeof(float) * ((size_t)(N * (N + 1)) / 2 + (size_t)m * (N + 1)) +
         (size_t)P * (2 * sizeof(int) + 3 * sizeof(float));
}

cudaError_t launch_gram(const Geom& g, const Bufs& b, cudaStream_t s) {
  int blocks = 0;
  for (int i = 0; i < g.n; ++i) {
    int nt = (g.m[i] + kGramTile - 1) / kGramTile;
    blocks += nt * (nt + 1) / 2;
  }
  k_gram<<<blocks, kGramThreads, 0, s>>>(g, b);
  return cudaGetLastError();
}

constexpr size_t kFullSmem = sizeof(float) * 3 * kFullMaxN * kFullLd;
constexpr size_t kTriSmem = sizeof(float) * 3 * kTriMax * kTriLd;

cudaError_t prepare_jacobi(size_t smem) {
  // same shared-memory carveout as the dense pass these kernels run beside
  const void* fns[] = {(const void*)k_gram, (const void*)k_jacobi, (const void*)k_jacobi_full,
                       (const void*)k_eig_tri, (const void*)k_refine};
  for (const void* f : fns) {
    cudaError_t e0 = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          cudaSharedmemCarveoutMaxShared);
    if (e0 != cudaSuccess) return e0;
  }
  cudaError_t e = raise_smem_limit((const void*)k_jacobi, (size_t)(smem));
  if (e != cudaSuccess) return e;
  e = raise_smem_limit((const void*)k_eig_tri, (size_t)(kTriSmem));
  if (e != cudaSuccess) return e;
  return raise_smem_limit((const void*)k_jacobi_full, (size_t)(kFullSmem));
}

cudaError_t launch_jacobi(const Geom& g, const Bufs& b, cudaStream_t s) {
  int mx = 0;
  for (int i = 0; i < g.n; ++i) mx = g.m[i] > mx ? g.m[i] : mx;
  if (mx <= kTriMax && g.eig_method == 0) {
    k_eig_tri<<<g.n, kJacThreads, kTriSmem, s>>>(g, b);
    return cudaGetLastError();
  }
  if (mx <= kFullMaxN) {
    k_jacobi_full<<<g.n, kJacThreads, kFullSmem, s>>>(g, b, g.warm_start);
    return cudaGetLastError();
  }
  size_t sm = jacobi_smem_bytes(mx);
  k_jacobi<<<g.n, kJacThreads, sm, s>>>(g, b);
  return cudaGetLastError();
}

size_t refine_smem_max(const Geom& g) {
  size_t mx = 0;
  for (int i = 0; i < g.n; ++i) {
    size_t v = refine_smem_bytes(g.m[i], g.r[i], g.ncl);
    mx = v > mx ? v : mx;
  }
  return mx;
}

// Chooses the cluster size of the refinement (`want` CTAs per mode when given, else 16 when the
// device can schedule such clusters, else 8) and sets the kernel's attributes. Updates g.ncl.
// Returns cudaErrorInvalidValue when the requested size cannot run (shared memory or occupancy).
cudaError_t prepare_refine(Geom& g, int want) {
  cudaError_t e = cudaFuncSetAttribute(k_refine, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  if (want > 0) {
    g.ncl = want;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (refine_smem_max(g) > (size_t)optin) return cudaErrorInvalidValue;
    e = raise_smem_limit((const void*)k_refine, (size_t)(refine_smem_max(g)));
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g.ncl * g.n);
    cfg.blockDim = dim3(kRefThreads);
    cfg.dynamicSmemBytes = refine_smem_max(g);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = g.ncl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_refine, &cfg) != cudaSuccess || nclusters < 1) {
      cudaGetLastError();
      return cudaErrorInvalidValue;
    }
    return cudaSuccess;
  }
  g.ncl = 16;
  e = raise_smem_limit((const void*)k_refine, (size_t)(refine_smem_max(g)));
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(g.ncl * g.n);
  cfg.blockDim = dim3(kRefThreads);
  cfg.dynamicSmemBytes = refine_smem_max(g);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = g.ncl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, k_refine, &cfg) != cudaSuccess || nclusters < 1) {
    cudaGetLastError();
    g.ncl = 8;
    e = raise_smem_limit((const void*)k_refine, (size_t)(refine_smem_max(g)));
  }
  return e;
}

cudaError_t launch_refine(const Geom& g, const Bufs& b, int mode, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(g.ncl * g.n);
  cfg.blockDim = dim3(kRefThreads);
  cfg.dynamicSmemBytes = refine_smem_max(g);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = g.ncl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_refine, g, b, mode);
}
