// Factor formation: the new L^(k+1) of Eq. (L=CUR) in Tucker form G x_i B_i.
//
// With W_i = C_i(I_i,:) = Q Sigma V^T and its rank-r truncation, C_i U_i^+ = C_i V_r Sigma_r^-1
// Q_r^T = B_i Q_r^T, so
//   L = R x_i (C_i U_i^+) = (R x_i Q_{r,i}^T) x_i B_i = G x_i B_i,
//   B_i = C_i Y_i with Y_i = V_r Sigma_r^-1 (d_i x r_i),   G = R x_1 Q_1^T ... x_n Q_n^T.
// The evaluation table T = G x_1 B_1 ... x_{n-1} B_{n-1} (prod_{i<n} d_i rows, r_n columns) is
// what every later L evaluation reads (see rtcur_internal.cuh).
#include "rtcur_internal.cuh"

namespace {

constexpr int kThreads = 128;
constexpr int kChunk = RT_BCHUNK;  // b-columns per split-K partial of B_i = C_i Y_i

// B partials: block -> (mode, t-block, chunk); thread -> row t.
__global__ void __launch_bounds__(kThreads) k_factor_B_partial(Geom g, Bufs b) {
  TL_BEGIN();
  int blk = blockIdx.x, i = 0;
  int tblocks = 0, chunks = 0;
  for (; i < g.n; ++i) {
    tblocks = (int)((g.d[i] + kThreads - 1) / kThreads);
    chunks = (g.q[i] + kChunk - 1) / kChunk;
    if (blk < tblocks * chunks) break;
    blk -= tblocks * chunks;
  }
  if (i >= g.n) return;
  const int ch = blk / tblocks;
  const long long t = (long long)(blk % tblocks) * kThreads + threadIdx.x;
  if (t >= g.d[i]) return;
  const int r = g.r[i];
  const int b0 = ch * kChunk, b1 = min(g.q[i], b0 + kChunk);
  const float* C = b.XS + g.seg[i + 1];
  const double* Y = b.Y + g.offY[i];
  double acc[RT_MAXR];
#pragma unroll
  for (int c = 0; c < RT_MAXR; ++c) acc[c] = 0.0;
  for (int bc = b0; bc < b1; ++bc) {
    double x = (double)C[(long long)bc * g.d[i] + t];
#pragma unroll
    for (int c = 0; c < RT_MAXR; ++c)
      if (c < r) acc[c] = fma(x, Y[(long long)bc * r + c], acc[c]);
  }
  double* out = b.Bpart + (long long)ch * g.sumB + g.offB[i] + t * r;
#pragma unroll
  for (int c = 0; c < RT_MAXR; ++c)
    if (c < r) out[c] = acc[c];
  TL_END(6);
}

// B_next = sum of the partials in chunk order (deterministic), rounded to FP32.
__global__ void __launch_bounds__(kThreads) k_factor_B_reduce(Geom g, Bufs b) {
  TL_BEGIN();
  long long e = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (e >= g.sumB) return;
  int i = 0;
  while (i + 1 < g.n && e >= g.offB[i + 1]) ++i;
  const int chunks = (g.q[i] + kChunk - 1) / kChunk;
  double acc = 0.0;
  for (int ch = 0; ch < chunks; ++ch) acc += b.Bpart[(long long)ch * g.sumB + e];
  b.B[(b.st->k + 1) & 1][e] = (float)acc;
  TL_END(7);
}

// One stage of G = R x_{n-1} Q^T ... x_0 Q^T (modes contracted from last to first).
// Before stage s the modes j' > j = n-1-s already have size r, the others m. Q_j (m_j x r_j,
// FP64) is staged in shared memory; each output is an FP64 dot product of length m_j split over a
// quad of lanes (terms a = ql mod 4), which quarters its dependent chain and quadruples the warps
// of the small later stages.
constexpr int kCoreOut = kThreads / 4;  // outputs per block
__global__ void __launch_bounds__(kThreads) k_core_stage(Geom g, Bufs b, int s, long long nout) {
  TL_BEGIN();
  __shared__ double Qs[RT_MAXM * RT_MAXR];
  const int n = g.n;
  const int j = n - 1 - s;
  const int r = g.r[j];
  const int mj = g.m[j];
  const double* Q = b.Qr + g.offQ[j];
  for (int t = threadIdx.x; t < mj * r; t += blockDim.x) Qs[t] = Q[t];
  __syncthreads();
  const int ql = threadIdx.x & 3;
  long long o = (long long)blockIdx.x * kCoreOut + (threadIdx.x >> 2);
  const bool act = o < nout;  // whole quads are active or not
  if (!act) o = 0;
  int shp_in[RT_MAXN], shp_out[RT_MAXN];
  for (int l = 0; l < n; ++l) {
    shp_in[l] = (l > j) ? g.r[l] : g.m[l];
    shp_out[l] = (l >= j) ? g.r[l] : g.m[l];
  }
  int co[RT_MAXN];
  long long rem = o;
  for (int l = n - 1; l >= 0; --l) {
    co[l] = (int)(rem % shp_out[l]);
    rem /= shp_out[l];
  }
  long long base = 0, strj = 1;
  {
    long long st = 1;
    for (int l = n - 1; l >= 0; --l) {
      if (l == j) strj = st;
      else base += (long long)co[l] * st;
      st *= shp_in[l];
    }
  }
  const int cj = co[j];
  double acc = 0.0;
  if (act) {
    if (s == 0) {
      const float* R = b.XS;  // segment 0
      for (int a = ql; a < mj; a += 4) acc = fma((double)R[base + a * strj], Qs[a * r + cj], acc);
    } else {
      const double* Zin = b.Z[(s - 1) & 1];
      for (int a = ql; a < mj; a += 4) acc = fma(Zin[base + a * strj], Qs[a * r + cj], acc);
    }
  }
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  acc += __shfl_xor_sync(0xffffffffu, acc, 2);
  if (act && ql == 0) {
    if (s == n - 1) {
      b.G[(b.st->k + 1) & 1][o] = (float)acc;
    } else {
      b.Z[s & 1][o] = acc;
    }
  }
  TL_END(8);
}

// Table stage A: H[c_0, p_1..p_{n-2}, c_{n-1}] = sum over c_1..c_{n-2} of
// G[c_0, c_1, .., c_{n-1}] prod_l B_l[p_l, c_l]   (H = G when n = 2).
__global__ void __launch_bounds__(kThreads) k_table_A(Geom g, Bufs b, int next) {
  TL_BEGIN();
  long long o = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (o >= g.nH) return;
  const int n = g.n;
  const int cp = next ? ((b.st->k + 1) & 1) : (b.st->k & 1);
  const float* G = b.G[cp];
  const float* B = b.B[cp];
  // decode o over (r_0, d_1, ..., d_{n-2}, r_{n-1})
  long long rem = o;
  const int cl = (int)(rem % g.r[n - 1]);
  rem /= g.r[n - 1];
  long long p[RT_MAXN];
  for (int l = n - 2; l >= 1; --l) {
    p[l] = rem % g.d[l];
    rem /= g.d[l];
  }
  const int c0 = (int)rem;
  // iterate over the middle core indices c_1..c_{n-2}
  int ncomb = 1;
  for (int l = 1; l <= n - 2; ++l) ncomb *= g.r[l];
  double acc = 0.0;
  for (int t = 0; t < ncomb; ++t) {
    int tr = t;
    double prod = 1.0;
    long long gidx = 0;
    int cmid[RT_MAXN];
    for (int l = n - 2; l >= 1; --l) {
      cmid[l] = tr % g.r[l];
      tr /= g.r[l];
    }
    gidx = c0;
    for (int l = 1; l <= n - 2; ++l) {
      gidx = gidx * g.r[l] + cmid[l];
      prod *= (double)B[g.offB[l] + p[l] * g.r[l] + cmid[l]];
    }
    gidx = gidx * g.r[n - 1] + cl;
    acc = fma((double)G[gidx], prod, acc);
  }
  b.H[o] = (float)acc;
  TL_END(9);
}

// Table stage B: T[p_0, rest] = sum_{c_0} B_0[p_0, c_0] H[c_0, rest], FP32 FMA in ascending c_0.
__global__ void __launch_bounds__(kThreads) k_table_B(Geom g, Bufs b, int next) {
  TL_BEGIN();
  const long long rest = g.nH / g.r[0];
  long long o = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (o >= g.d[0] * rest) return;
  const int cp = next ? ((b.st->k + 1) & 1) : (b.st->k & 1);
  const float* B0 = b.B[cp];
  const long long p0 = o / rest, w = o - p0 * rest;
  float acc = 0.f;
  for (int c = 0; c < g.r[0]; ++c) acc = fmaf(B0[p0 * g.r[0] + c], b.H[c * rest + w], acc);
  b.T[cp][o] = acc;
  TL_END(10);
}

// Algorithm 1's output (R, C_i, U_i^+) of the current L^(k), staged for the host:
//   curF[0, nR)             R = (X - S^(k))(I_1..I_n), the sample buffer's segment 0 as it is
//   curF[seg[1+i] + t q_i + j]  C_i(t, j), row-major d_i x q_i (the sample buffer holds it
//                           fiber-major: entry j d_i + t)
//   curU[sum_{l<i} q_l m_l + j m_i + a]  U_i^+(j, a) = sum_c Y_i(j, c) Q_{r,i}(a, c), FP64: the
//                           truncated pseudoinverse V_r Sigma_r^-1 Q_r^T of Eq. (R, C_i, U_i), from
//                           the factors the pinv stage left (Y_i = W_i^T Q_r Sigma_r^-2, or
//                           W_i^T X_1 H^-1 with Q_r = X_1 on the certified path: the same product)
__global__ void __launch_bounds__(kThreads) k_export_cur(Geom g, Bufs b) {
  long long e = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (e < g.nS) {
    if (e < g.nR) {
      b.curF[e] = b.XS[e];
      return;
    }
    int i = 0;
    while (i + 1 < g.n && e >= g.seg[i + 2]) ++i;
    const long long local = e - g.seg[i + 1];
    const long long t = local / g.q[i], j = local - t * g.q[i];
    b.curF[e] = b.XS[g.seg[i + 1] + j * g.d[i] + t];
    return;
  }
  e -= g.nS;
  long long off = 0;
  for (int i = 0; i < g.n; ++i) {
    const long long sz = (long long)g.q[i] * g.m[i];
    if (e < off + sz) {
      const long long local = e - off;
      const int j = (int)(local / g.m[i]), a = (int)(local - (long long)j * g.m[i]);
      const int r = g.r[i];
      const double* Y = b.Y + g.offY[i] + (long long)j * r;
      const double* Q = b.Qr + g.offQ[i] + (long long)a * r;
      double acc = 0.0;
      for (int c = 0; c < r; ++c) acc = fma(Y[c], Q[c], acc);
      b.curU[e] = acc;
      return;
    }
    off += sz;
  }
}

inline int nblocks(long long work) { return (int)((work + kThreads - 1) / kThreads); }

}  // namespace

// Same shared-memory carveout as the dense pass they run beside (see prepare_sample_kernels).
cudaError_t prepare_factor_kernels() {
  const void* fns[] = {(const void*)k_factor_B_partial, (const void*)k_factor_B_reduce,
                       (const void*)k_core_stage, (const void*)k_table_A, (const void*)k_table_B,
                       (const void*)k_export_cur};
  for (const void* f : fns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_factor_B(const Geom& g, const Bufs& b, cudaStream_t s) {
  int blocks = 0;
  for (int i = 0; i < g.n; ++i)
    blocks += (int)((g.d[i] + kThreads - 1) / kThreads) * ((g.q[i] + kChunk - 1) / kChunk);
  k_factor_B_partial<<<blocks, kThreads, 0, s>>>(g, b);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_factor_B_reduce<<<nblocks(g.sumB), kThreads, 0, s>>>(g, b);
  return cudaGetLastError();
}

cudaError_t launch_core(const Geom& g, const Bufs& b, cudaStream_t s) {
  for (int st = 0; st < g.n; ++st) {
    int j = g.n - 1 - st;
    long long nout = 1;
    for (int l = 0; l < g.n; ++l) nout *= (l >= j) ? g.r[l] : g.m[l];
    k_core_stage<<<(int)((nout + kCoreOut - 1) / kCoreOut), kThreads, 0, s>>>(g, b, st, nout);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_table(const Geom& g, const Bufs& b, int next, cudaStream_t s) {
  k_table_A<<<nblocks(g.nH), kThreads, 0, s>>>(g, b, next);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_table_B<<<nblocks(g.rowsT * g.rlast), kThreads, 0, s>>>(g, b, next);
  return cudaGetLastError();
}

cudaError_t launch_export_cur(const Geom& g, const Bufs& b, cudaStream_t s) {
  long long nU = 0;
  for (int i = 0; i < g.n; ++i) nU += (long long)g.q[i] * g.m[i];
  k_export_cur<<<nblocks(g.nS + nU), kThreads, 0, s>>>(g, b);
  return cudaGetLastError();
}
