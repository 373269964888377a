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
  long long want = (2LL * 152 * 1024) / nout;  // enough threads to fill the GPU
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

// Y = X x_mode M for a 3-mode tensor X (dims n, float or double), M[j][k] at M + j*mr + k*mc
// (J rows, n[mode] columns); Y (double) has n[mode] replaced by J.
cudaError_t ttm3(const Ctx& cx, const void* X, int xf64, const long long n[3], int mode,
                 const double* M, long long mr, long long mc, int J, double* Y, double beta = 0.0) {
  if (mode == 0) {
    return contract(cx, opd(M, 1, 0, mr, mc), opd(X, xf64, 0, 1, n[1] * n[2]), Y, 0, n[1] * n[2], 1,
                    1, J, (int)(n[1] * n[2]), n[0], 1, 1.0, beta);
  } else if (mode == 1) {
    return contract(cx, opd(M, 1, 0, mr, mc), opd(X, xf64, n[1] * n[2], 1, n[2]), Y, (long long)J * n[2],
                    n[2], 1, (int)n[0], J, (int)n[2], n[1], 1, 1.0, beta);
  }
  return contract(cx, opd(X, xf64, 0, n[2], 1), opd(M, 1, 0, mr, mc), Y, 0, J, 1, 1,
                  (int)(n[0] * n[1]), J, n[2], 1, 1.0, beta);
}

// out (n[mode] x m, row-major) = X_(mode) Y_(mode)^T, X dims n, Y dims n with n[mode] -> m.
cudaError_t contract_but3(const Ctx& cx, const void* X, int xf64, const long long n[3],
                          const double* Y, int m, int mode, double* out, double beta = 0.0) {
  if (mode == 0) {
    return contract(cx, opd(X, xf64, 0, n[1] * n[2], 1), opd(Y, 1, 0, n[1] * n[2], 1), out, 0, m, 1, 1,
                    (int)n[0], m, n[1] * n[2], 1, 1.0, beta);
  } else if (mode == 1) {
    return contract(cx, opd(X, xf64, 0, n[2], n[1] * n[2], 1), opd(Y, 1, 0, n[2], (long long)m * n[2], 1),
                    out, 0, m, 1, 1, (int)n[1], m, n[0], n[2], 1.0, beta);
  }
  return contract(cx, opd(X, xf64, 0, 1, n[2]), opd(Y, 1, 0, 1, m), out, 0, m, 1, 1, (int)n[2], m,
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

// A_bar_l(t, :) += sum over the fibers c with p_l(c) = t, in ascending c, of G(c, :) (q x m_l):
// the row scatter of the per-fiber contributions without atomics.
__global__ void k_bw_rows_ordered(Geom g, const long long* J, int i, int l, int q, const double* Gc,
                                  int ml, double* Ab) {
  const long long e = (long long)blockIdx.x * kT + threadIdx.x;
  if (e >= g.d[l] * ml) return;
  const long long t = e / ml;
  const int x = (int)(e % ml);
  double acc = 0.0;
  long long p[RT_MAXN];
  for (int c = 0; c < q; ++c) {
    long long j = J[c];
    for (int l2 = g.n - 1; l2 >= 0; --l2) {
      if (l2 == i) continue;
      p[l2] = j % g.d[l2];
      j /= g.d[l2];
    }
    if (p[l] == t) acc += Gc[(long long)c * ml + x];
  }
  Ab[e] += acc;
}

__global__ void k_bw_to_f32(const double* src, float* dst, long long n) {
  const long long stride = (long long)gridDim.x * kT;
  for (long long e = (long long)blockIdx.x * kT + threadIdx.x; e < n; e += stride) dst[e] = (float)src[e];
}

// ------------------------------------------------------------------ fiber contractions
// Other-mode coordinates of fiber c of mode i (column J[c] of X_(i), row-major over the others).
__device__ __forceinline__ void fiber_other(const Geom& g, int i, long long j, long long* p) {
  for (int l = g.n - 1; l >= 0; --l) {
    if (l == i) continue;
    p[l] = j % g.d[l];
    j /= g.d[l];
  }
}

struct FiberArgs {
  const float* R;        // m0 x m1 x m2 (row-major)
  long long rs[3];       // strides of R
  int m[3];
  const double* A[3];    // A'_l (d_l x m_l)
  const long long* J;    // fibers of mode i
  int i;                 // fiber mode
  int q;
  // contraction: output mode go; vector modes ga (source sa), gb (source sb)
  int go, ga, gb;
  int sa, sb;            // 0: row p_mode of A'_mode; 1: column c of Zfb (m_i x q)
  const double* Zfb;
  int out_kind;          // 0: out[x * q + c] (m_go x q); 1: out[c * m_go + x] (q x m_go)
  double* out;
};

// out_go[x] = sum_{y, z} R[x @ go, y @ ga, z @ gb] va[y] vb[z] for fiber c = blockIdx.x.
// One warp per output x; lanes over y; the z sum in FP32, the y sum in FP64.
__global__ void __launch_bounds__(kT) k_bw_fiber(Geom g, FiberArgs f) {
  __shared__ float va[RT_MAXM], vb[RT_MAXM];
  const int c = blockIdx.x;
  long long p[RT_MAXN];
  fiber_other(g, f.i, f.J[c], p);
  const int ma = f.m[f.ga], mb = f.m[f.gb], mo = f.m[f.go];
  for (int t = threadIdx.x; t < ma; t += kT)
    va[t] = (float)(f.sa == 0 ? f.A[f.ga][p[f.ga] * ma + t] : f.Zfb[(long long)t * f.q + c]);
  for (int t = threadIdx.x; t < mb; t += kT)
    vb[t] = (float)(f.sb == 0 ? f.A[f.gb][p[f.gb] * mb + t] : f.Zfb[(long long)t * f.q + c]);
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long so = f.rs[f.go], sa = f.rs[f.ga], sbb = f.rs[f.gb];
  for (int x = wid; x < mo; x += kT / 32) {
    double acc = 0.0;
    for (int y = lane; y < ma; y += 32) {
      const float* row = f.R + x * so + y * sa;
      float t = 0.f;
      for (int z = 0; z < mb; ++z) t = fmaf(row[z * sbb], vb[z], t);
      acc = fma((double)t, (double)va[y], acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      if (f.out_kind == 0) f.out[(long long)x * f.q + c] = acc;
      else f.out[(long long)c * mo + x] = acc;
    }
  }
}

// R_bar[a] += sum_c Zfb[a_i, c] A'_l1(p_l1(c), a_l1) A'_l2(p_l2(c), a_l2) over the fibers of mode i
__global__ void __launch_bounds__(kT) k_bw_fiber_rbar(Geom g, FiberArgs f, double* Rb) {
  extern __shared__ int pc[];  // 2 x q other-mode coordinates
  int l1 = -1, l2 = -1;
  for (int l = 0; l < 3; ++l)
    if (l != f.i) { if (l1 < 0) l1 = l; else l2 = l; }
  for (int c = threadIdx.x; c < f.q; c += kT) {
    long long p[RT_MAXN];
    fiber_other(g, f.i, f.J[c], p);
    pc[c] = (int)p[l1];
    pc[f.q + c] = (int)p[l2];
  }
  __syncthreads();
  const long long nR = (long long)f.m[0] * f.m[1] * f.m[2];
  const long long e = (long long)blockIdx.x * kT + threadIdx.x;
  if (e >= nR) return;
  int a[3];
  a[2] = (int)(e % f.m[2]);
  a[1] = (int)((e / f.m[2]) % f.m[1]);
  a[0] = (int)(e / ((long long)f.m[1] * f.m[2]));
  const double* zr = f.Zfb + (long long)a[f.i] * f.q;
  const double* A1 = f.A[l1] + a[l1];
  const double* A2 = f.A[l2] + a[l2];
  const int m1 = f.m[l1], m2 = f.m[l2];
  double acc = 0.0;
  for (int c = 0; c < f.q; ++c)
    acc = fma(zr[c], A1[(long long)pc[c] * m1] * A2[(long long)pc[f.q + c] * m2], acc);
  Rb[e] += acc;
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
  double* U;        // per slot and mode: M on entry, eigenvectors on exit
  double* lam;
  long long offMM[RT_MAXN], offM[RT_MAXN];
  long long slotMM, slotM;
  int m[RT_MAXN];
  int nmodes;
};

__global__ void __launch_bounds__(kT) k_bw_eig(EigArgs ea, int max_sweeps) {
  extern __shared__ double sA[];
  __shared__ double cs[kEigMax / 2], sn[kEigMax / 2];
  __shared__ int pp[kEigMax / 2], qq[kEigMax / 2];
  __shared__ int perm[kEigMax];
  __shared__ int nrot;
  const int slot = blockIdx.x / ea.nmodes, mode = blockIdx.x % ea.nmodes;
  const int m = ea.m[mode];
  double* M = ea.U + slot * ea.slotMM + ea.offMM[mode];
  double* U = M;
  double* lam = ea.lam + slot * ea.slotM + ea.offM[mode];
  const int mp = (m + 1) & ~1;  // padded to even; index m (if m odd) is a dummy
  const int tid = threadIdx.x;
  for (int e = tid; e < mp * mp; e += kT) {
    int r = e / mp, c = e % mp;
    sA[e] = (r < m && c < m) ? M[(long long)r * m + c] : 0.0;
  }
  __syncthreads();  // M and U share storage: every read of M precedes the first write of U
  for (int e = tid; e < m * m; e += kT) U[e] = ((e / m) == (e % m)) ? 1.0 : 0.0;
  __syncthreads();
  // entries below 1e-17 of the largest diagonal entry are rounding noise of the FP64 Gram
  // matrix; rotating them would keep a rank-deficient matrix sweeping forever
  __shared__ double floor_abs;
  if (tid == 0) {
    double mxd = 0.0;
    for (int j = 0; j < m; ++j) mxd = fmax(mxd, fabs(sA[j * mp + j]));
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
          const double apq = sA[p * mp + q];
          const double app = sA[p * mp + p], aqq = sA[q * mp + q];
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
        const double ap = sA[p * mp + col], aq = sA[q * mp + col];
        sA[p * mp + col] = c * ap - s * aq;
        sA[q * mp + col] = s * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A G, U <- U G
      for (int e = tid; e < (mp / 2) * mp; e += kT) {
        const int t = e / mp, row = e % mp;
        const double s = sn[t];
        if (s == 0.0) continue;
        const int p = pp[t], q = qq[t];
        const double c = cs[t];
        const double ap = sA[row * mp + p], aq = sA[row * mp + q];
        sA[row * mp + p] = c * ap - s * aq;
        sA[row * mp + q] = s * ap + c * aq;
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
        if (sA[perm[l] * mp + perm[l]] > sA[perm[best] * mp + perm[best]]) best = l;
      int t = perm[j]; perm[j] = perm[best]; perm[best] = t;
    }
    for (int j = 0; j < m; ++j) lam[j] = sA[perm[j] * mp + perm[j]];
  }
  __syncthreads();
  for (int e = tid; e < m * m; e += kT) sA[e] = U[(long long)(e / m) * m + perm[e % m]];
  __syncthreads();
  for (int e = tid; e < m * m; e += kT) U[e] = sA[e];
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
  return sizeof(double) * (size_t)mp * mp;
}

cudaError_t prepare_backward(int max_m) {
  if (max_m > kEigMax) return cudaErrorInvalidValue;
  return raise_smem_limit((const void*)k_bw_eig, (size_t)(backward_eig_smem(max_m)));
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
  w.tmpsz = t;
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
      // M (stored in U's slot, the eigensolver works in place from it)
      BW_CK(contract(cx, opd(Wof(k, i), 1, 0, q, 1), opd(Wof(k, i), 1, 0, q, 1), Uof(k, i), 0, m, 1, 1, m, m,
                     q, 1));
    }
  }
  {
    // every (iteration, mode) matrix at once; M is read from U's slot, U overwritten in place
    EigArgs ea;
    ea.U = w.U;
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
    k_bw_eig<<<K * 3, kT, backward_eig_smem(mx), s>>>(ea, 60);
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
    // fibers of each mode i
    for (int i = 0; i < 3; ++i) {
      const int m = g.m[i], q = g.q[i];
      const long long d = g.d[i];
      const double* LbC = w.Lb + g.seg[i + 1];
      FiberArgs f;
      f.R = Rp;
      f.rs[0] = (long long)g.m[1] * g.m[2];
      f.rs[1] = g.m[2];
      f.rs[2] = 1;
      for (int l = 0; l < 3; ++l) {
        f.m[l] = g.m[l];
        f.A[l] = Ap[l];
      }
      f.J = set + g.joff[i];
      f.i = i;
      f.q = q;
      int l1 = -1, l2 = -1;
      for (int l = 0; l < 3; ++l)
        if (l != i) { if (l1 < 0) l1 = l; else l2 = l; }
      // z (m x q) = R' contracted with the rows of A'_l1, A'_l2
      f.go = i; f.ga = l1; f.gb = l2; f.sa = 0; f.sb = 0; f.Zfb = nullptr; f.out_kind = 0; f.out = w.Zf;
      k_bw_fiber<<<q, kT, 0, s>>>(g, f);
      BW_CK(cudaGetLastError());
      // A_bar_i += LbC Z^T; Z_bar = A'_i^T LbC
      BW_CK(contract(cx, opd(LbC, 1, 0, 1, d), opd(w.Zf, 1, 0, q, 1), w.Ab + w.offDM[i], 0, m, 1, 1, (int)d, m,
                     q, 1, 1.0, 1.0));
      BW_CK(contract(cx, opd(Ap[i], 1, 0, 1, m), opd(LbC, 1, 0, d, 1), w.Zfb, 0, q, 1, 1, m, q, d, 1));
      f.Zfb = w.Zfb;
      // R_bar += sum_c zbar_c x A'_l1 row x A'_l2 row
      k_bw_fiber_rbar<<<nblk(g.nR), kT, sizeof(int) * 2 * q, s>>>(g, f, Rb);
      BW_CK(cudaGetLastError());
      // A_bar_l1 rows += R' contracted with zbar (mode i) and the A'_l2 row; same for l2
      for (int side = 0; side < 2; ++side) {
        const int lo = side ? l2 : l1, lother = side ? l1 : l2;
        f.go = lo; f.ga = i; f.gb = lother; f.sa = 1; f.sb = 0; f.out_kind = 1; f.out = w.Zf;
        k_bw_fiber<<<q, kT, 0, s>>>(g, f);
        BW_CK(cudaGetLastError());
        k_bw_rows_ordered<<<nblk(g.d[lo] * g.m[lo]), kT, 0, s>>>(g, set + g.joff[i], i, lo, q, w.Zf, g.m[lo],
                                                                 w.Ab + w.offDM[lo]);
        BW_CK(cudaGetLastError());
      }
    }
  }
  int blocks = (int)((g.N + kT - 1) / kT);
  if (blocks > 8192) blocks = 8192;
  k_bw_to_f32<<<blocks, kT, 0, s>>>(w.dX64, dX, g.N);
  return cudaGetLastError();
}
