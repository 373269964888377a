// Sampled-entry kernels of one RTCUR iteration.
//
//  sample_ht   Step (I) on the sample: S^(k+1) = HT_{zeta^(k+1)}(X - L^(k)) on R's entries and on
//              the fibers of C_i (Eq. partial S update), writing (X - S) into the sample buffer,
//              which then holds R^(k+1) and C_i^(k+1) of Eq. (R, C_i, U_i).
//  sample_err  e^(k+1) of Eq. (rel_err): per-segment Frobenius norms of E = X - L^(k+1) - S^(k+1)
//              over this iteration's sets, divided by those of X.
//  commit      k <- k+1, zeta <- gamma zeta (Sec. 3.2 decay), histories, loop condition.
//
// Reductions are deterministic: per-block partials in a fixed slot, then the last block to
// finish sums them in block order.
#include <cuda_bf16.h>

#include "../../include/rtcur.h"
#include "rtcur_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kHtBlocksFull = 2 * 152;
// Alone (SAMPLED scope) the threshold and error kernels run one wave of three blocks per SM, each
// thread looping over more entries: 1024 blocks (two waves of the four that fit an SM) took
// 5.6% longer per solve at 800^3, 608 blocks 1%.
constexpr int kHtBlocksSampled = 3 * 152;
constexpr int kMaxRedBlocks = 1024;

// X at flat index `idx` as the sampled step reads it: the caller's FP32 tensor, or its BF16 copy
// (sample_x BF16) widened back to FP32.
__device__ __forceinline__ float sample_x_at(const Bufs& b, const float* X, long long idx) {
  if (b.Xb) return __uint_as_float((unsigned)__ldg(b.Xb + idx) << 16);
  return __ldg(X + idx);
}

__device__ __forceinline__ const long long* current_set(const Geom& g, const Bufs& b, int k) {
  long long s = (g.variant == 1) ? (long long)(k % g.n_sets) : 0;
  return b.idx + s * g.set_len;
}

// Block-wide sums of N values at once (kThreads threads): each value is summed by a shuffle-down
// tree within every warp, then over the warps in order, all N sums sharing one barrier (instead
// of two per sum when summed one at a time; the order of every sum is the same). Sum j is
// returned in thread j (j < N).
template <int N>
__device__ __forceinline__ double block_sum_n(const double (&v)[N], double* sh) {
  double r[N];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    double x = v[j];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    r[j] = x;
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
#pragma unroll
    for (int j = 0; j < N; ++j) sh[j * (kThreads / 32) + w] = r[j];
  }
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < N)
    for (int i = 0; i < kThreads / 32; ++i) t += sh[threadIdx.x * (kThreads / 32) + i];
  return t;
}

// Sums of slots 0..N-1 over the first `nb` block partials (fixed order per thread, then the block
// sums), sum j in thread j.
template <int N>
__device__ __forceinline__ double sum_partials_n(const double* part, int nb, double* sh) {
  double acc[N];
#pragma unroll
  for (int j = 0; j < N; ++j) acc[j] = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x)
#pragma unroll
    for (int j = 0; j < N; ++j) acc[j] += part[i * RT_RED_SLOTS + j];
  return block_sum_n<N>(acc, sh);
}

__global__ void k_setup(Geom g, Bufs b, double zeta0) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  State* st = b.st;
  st->k = 0;
  st->err = 0;
  st->flags = 0;
  st->zeta = zeta0;
  st->zeta0 = zeta0;
  st->e = 1.0;  // L^(0) = S^(0) = 0 gives E = X
  st->e_stage = 1.0;
  st->cont = (g.max_iter > 0 && 1.0 > g.tol) ? 1 : 0;
  st->nnz_s = st->inband_s = 0;
  st->jsweeps = 0;
  st->warm_hits = 0;
  st->nnz_f = st->inband_f = -1;
  st->resid_f = -1.0;
  for (int i = 0; i < RT_MAXN + 1; ++i) st->den[i] = st->num[i] = 0.0;
  for (int i = 0; i < TK_COUNT; ++i) b.ticket[i] = 0u;
}

__global__ void __launch_bounds__(kThreads) k_maxabs(Geom g, Bufs b) {
  __shared__ double sh[kThreads / 32];
  const float* X = b.sp->X;
  float mx = 0.f;
  long long stride = (long long)gridDim.x * kThreads;
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < g.N; i += stride)
    mx = fmaxf(mx, fabsf(__ldg(X + i)));
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
  __syncthreads();
  double* part = b.red + (size_t)TK_MAXABS * kMaxRedBlocks * RT_RED_SLOTS;
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < kThreads / 32; ++i) m = fmax(m, sh[i]);
    part[blockIdx.x] = m;
  }
  if (last_block_arrive(b.ticket + TK_MAXABS)) {
    double m = 0.0;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) m = fmax(m, part[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int i = 0; i < kThreads / 32; ++i) m = fmax(m, sh[i]);
      b.st->zeta = m;
      b.st->zeta0 = m;
      b.ticket[TK_MAXABS] = 0u;
    }
  }
}

// Xs[e] = X at sampled entry e and rc[e] = (row of T, column of B_n) for the fixed sets
// (gathered once per solve).
__global__ void __launch_bounds__(kThreads) k_gather_x(Geom g, Bufs b) {
  const long long* set = current_set(g, b, 0);
  const float* X = b.sp->X;
  long long p[RT_MAXN];
  long long stride = (long long)gridDim.x * kThreads;
  for (long long e = (long long)blockIdx.x * kThreads + threadIdx.x; e < g.nS; e += stride) {
    sample_coords(g, set, e, p);
    long long row = table_row(g, p), col = p[g.n - 1];
    b.rc[e] = make_uint2((unsigned)row, (unsigned)col);
    b.Xs[e] = sample_x_at(b, X, row * g.d[g.n - 1] + col);
  }
}

// The BF16 copy of X for the sampled step (sample_x BF16): round to nearest even, four values per
// thread from one float4 (the tensor is 16-byte aligned; a tail of N % 4 values is done singly).
__device__ __forceinline__ unsigned short bf16_rne(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__global__ void __launch_bounds__(kThreads) k_x_bf16(long long N, const float* __restrict__ X,
                                                     unsigned short* __restrict__ Xb) {
  const long long n4 = N >> 2;
  const long long stride = (long long)gridDim.x * kThreads;
  for (long long v = (long long)blockIdx.x * kThreads + threadIdx.x; v < n4; v += stride) {
    const float4 x = __ldcs(reinterpret_cast<const float4*>(X) + v);
    ushort4 o;
    o.x = bf16_rne(x.x);
    o.y = bf16_rne(x.y);
    o.z = bf16_rne(x.z);
    o.w = bf16_rne(x.w);
    reinterpret_cast<ushort4*>(Xb)[v] = o;
  }
  for (long long e = (n4 << 2) + (long long)blockIdx.x * kThreads + threadIdx.x; e < N; e += stride)
    Xb[e] = bf16_rne(X[e]);
}

// Segment of entry e (0 = R, 1 + i = C_i).
__device__ __forceinline__ int segment_of(const Geom& g, long long e) {
  int s = 0;
  while (s < g.n && e >= g.seg[s + 1]) ++s;
  return s;
}

__global__ void __launch_bounds__(kThreads) k_sample_ht(Geom g, Bufs b) {
  TL_BEGIN();
  __shared__ double sh[8 * (kThreads / 32) + 16];  // block_sum_n<8> and the segment sums
  const State* st = b.st;
  const int k = st->k;
  const int cur = k & 1;
  const double zeta = g.gamma * st->zeta;  // zeta^(k+1)
  const float zf = (float)zeta;
  const float band = (float)(g.inband * zeta);
  const long long* set = current_set(g, b, k);
  const int* pos = b.pos + ((g.variant == 1) ? (long long)(k % g.n_sets) : 0LL) * g.sumD;
  const float* X = b.sp->X;
  const float* T = b.T[cur];
  const float* Bn = b.B[cur] + g.offB[g.n - 1];
  const int rn = g.rlast;
  const long long dn = g.d[g.n - 1];
  float den[RT_MAXN + 1];
#pragma unroll
  for (int s = 0; s < RT_MAXN + 1; ++s) den[s] = 0.f;
  float nnz = 0.f, inb = 0.f, bad = 0.f;
  long long p[RT_MAXN];
  long long stride = (long long)gridDim.x * kThreads;
  for (long long e = (long long)blockIdx.x * kThreads + threadIdx.x; e < g.nS; e += stride) {
    long long row, col;
    float x;
    int seg;
    if (g.variant == 1) {
      seg = sample_coords(g, set, e, p);
      row = table_row(g, p);
      col = p[g.n - 1];
      b.rc[e] = make_uint2((unsigned)row, (unsigned)col);
      x = sample_x_at(b, X, row * dn + col);
    } else {
      uint2 rc = b.rc[e];
      row = rc.x;
      col = rc.y;
      x = b.Xs[e];
      seg = segment_of(g, e);
    }
    float L = eval_L(T, Bn, rn, row, col);
    float dlt = x - L;
    float ad = fabsf(dlt);
    bool keep = ad > zf;                 // HT_zeta keeps |x| > zeta (strict)
    const float xs = keep ? L : x;       // (X - S) = X - (X - L) = L where S is nonzero
    b.XS[e] = xs;
    if (k < g.ck_iters) {                // checkpoint for the adjoint
      b.ckV[(long long)k * g.nS + e] = xs;
      b.ckM[(long long)k * g.nS + e] = keep ? 1 : 0;
    }
    if (seg > 0) {                       // fiber entry: also W_i = C_i(I_i, :) when t is in I_i
      const int i = seg - 1;
      const unsigned local = (unsigned)(e - g.seg[seg]);
      const unsigned bcol = local / (unsigned)g.d[i];
      const unsigned t = local - bcol * (unsigned)g.d[i];
      const int a = pos[g.offD[i] + t];
      if (a >= 0) b.W[g.offW[i] + (long long)a * g.q[i] + bcol] = xs;
    }
    nnz += keep ? 1.f : 0.f;
    inb += (fabsf(ad - zf) <= band) ? 1.f : 0.f;
    if (!isfinite(x)) bad += 1.f;
    float xx = x * x;
#pragma unroll
    for (int s = 0; s < RT_MAXN + 1; ++s)
      if (s == seg) den[s] += xx;
  }
  double* part = b.red + (size_t)TK_SAMPLE * kMaxRedBlocks * RT_RED_SLOTS;
  {
    double v[8];
#pragma unroll
    for (int s = 0; s < RT_MAXN + 1; ++s) v[s] = (double)den[s];
    v[5] = (double)nnz;
    v[6] = (double)inb;
    v[7] = (double)bad;
    const double tot = block_sum_n<8>(v, sh);
    if (threadIdx.x < 8) part[blockIdx.x * RT_RED_SLOTS + threadIdx.x] = tot;
  }
  if (last_block_arrive(b.ticket + TK_SAMPLE)) {
    State* w = b.st;
    const double acc = sum_partials_n<8>(part, gridDim.x, sh);  // slot j in thread j
    const int slot = threadIdx.x;
    if (slot < RT_MAXN + 1) w->den[slot] = acc;
    if (slot == 5) w->nnz_s = (long long)acc;
    if (slot == 6) w->inband_s = (long long)acc;
    if (slot == 7 && acc > 0.0) w->err = -4;  // RTCUR_ENONFINITE
    if (threadIdx.x == 0) {
      w->jsweeps = 0;
      b.ticket[TK_SAMPLE] = 0u;
    }
  }
  TL_END(2);
}

__global__ void __launch_bounds__(kThreads) k_sample_err(Geom g, Bufs b) {
  TL_BEGIN();
  __shared__ double sh[8 * (kThreads / 32) + 16];  // block_sum_n<8> and the segment sums
  const State* st = b.st;
  const int k = st->k;
  const int nxt = (k + 1) & 1;
  const float* T = b.T[nxt];
  const float* Bn = b.B[nxt] + g.offB[g.n - 1];
  const int rn = g.rlast;
  float num[RT_MAXN + 1];
#pragma unroll
  for (int s = 0; s < RT_MAXN + 1; ++s) num[s] = 0.f;
  long long stride = (long long)gridDim.x * kThreads;
  for (long long e = (long long)blockIdx.x * kThreads + threadIdx.x; e < g.nS; e += stride) {
    uint2 rc = b.rc[e];
    int seg = segment_of(g, e);
    float L = eval_L(T, Bn, rn, rc.x, rc.y);
    float E = b.XS[e] - L;   // X - S^(k+1) - L^(k+1)
    float ee = E * E;
#pragma unroll
    for (int s = 0; s < RT_MAXN + 1; ++s)
      if (s == seg) num[s] += ee;
  }
  double* part = b.red + (size_t)TK_ERR * kMaxRedBlocks * RT_RED_SLOTS;
  {
    double v[RT_MAXN + 1];
#pragma unroll
    for (int s = 0; s < RT_MAXN + 1; ++s) v[s] = (double)num[s];
    const double tot = block_sum_n<RT_MAXN + 1>(v, sh);
    if (threadIdx.x < RT_MAXN + 1) part[blockIdx.x * RT_RED_SLOTS + threadIdx.x] = tot;
  }
  if (last_block_arrive(b.ticket + TK_ERR)) {
    State* w = b.st;
    const double acc = sum_partials_n<RT_MAXN + 1>(part, gridDim.x, sh);  // segment j in thread j
    if (threadIdx.x <= g.n) sh[64 + threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sn = 0.0, sd = 0.0;
      for (int s = 0; s <= g.n; ++s) {
        const double a = sh[64 + s];
        w->num[s] = a;
        sn += sqrt(a);
        sd += sqrt(w->den[s]);
      }
      w->e_stage = (sd > 0.0) ? sn / sd : 0.0;
      b.ticket[TK_ERR] = 0u;
    }
  }
  TL_END(11);
}

__global__ void k_commit(Geom g, Bufs b, unsigned long long handle, int use_handle) {
  TL_BEGIN();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  State* st = b.st;
  int k = st->k;
  double zeta = g.gamma * st->zeta;
  double e = st->e_stage;
  if (k < g.max_iter) {
    b.e_hist[k] = e;
    b.z_hist[k] = zeta;
    b.nnz_hist[k] = st->nnz_s;
  }
  st->zeta = zeta;
  st->e = e;
  st->k = k + 1;
  int cont = (e > g.tol) && (k + 1 < g.max_iter) && (st->err == 0);
  st->cont = cont;
  if (use_handle) cudaGraphSetConditional((cudaGraphConditionalHandle)handle, cont ? 1u : 0u);
  TL_END(12);
}

// Batched solve: the loop continues while any problem of the batch continues.
__global__ void k_batch_any(State* const* sts, int count, unsigned long long handle) {
  int any = 0;
  for (int i = threadIdx.x; i < count; i += 32) any |= sts[i]->cont;
  any = __any_sync(0xffffffffu, any);
  if (threadIdx.x == 0) cudaGraphSetConditional((cudaGraphConditionalHandle)handle, any ? 1u : 0u);
}

int grid_for(long long work) {
  long long g = (work + kThreads - 1) / kThreads;
  if (g < 1) g = 1;
  if (g > kMaxRedBlocks) g = kMaxRedBlocks;
  return (int)g;
}

}  // namespace

cudaError_t launch_setup(const Geom& g, const Bufs& b, double zeta0, int use_maxabs, cudaStream_t s) {
  k_setup<<<1, 32, 0, s>>>(g, b, zeta0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !use_maxabs) return e;
  return launch_maxabs(g, b, s);
}

cudaError_t launch_maxabs(const Geom& g, const Bufs& b, cudaStream_t s) {
  k_maxabs<<<grid_for(g.N), kThreads, 0, s>>>(g, b);
  return cudaGetLastError();
}

// The sampled chain's kernels run beside the dense pass, whose persistent CTAs need the SM's
// maximum shared-memory carveout. A block of another carveout on an SM keeps a dense CTA off it
// until the block drains (the SM's L1/shared split changes only when it is idle), so the chain's
// kernels ask for the same carveout.
cudaError_t prepare_sample_kernels() {
  const void* fns[] = {(const void*)k_setup, (const void*)k_maxabs, (const void*)k_gather_x,
                       (const void*)k_x_bf16, (const void*)k_sample_ht, (const void*)k_sample_err,
                       (const void*)k_commit};
  for (const void* f : fns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_gather_x(const Geom& g, const Bufs& b, cudaStream_t s) {
  k_gather_x<<<grid_for(g.nS), kThreads, 0, s>>>(g, b);
  return cudaGetLastError();
}

cudaError_t launch_x_bf16(const Geom& g, const Bufs& b, const float* X, cudaStream_t s) {
  long long blocks = (g.N / 4 + kThreads - 1) / kThreads;
  if (blocks > 8 * 152) blocks = 8 * 152;  // grid-stride: a few waves of resident blocks
  if (blocks < 1) blocks = 1;
  k_x_bf16<<<(int)blocks, kThreads, 0, s>>>(g.N, X, b.Xb);
  return cudaGetLastError();
}

cudaError_t launch_sample_ht(const Geom& g, const Bufs& b, cudaStream_t s) {
  // In the FULL scope the dense pass starts beside this kernel: at most kHtBlocksFull blocks (two
  // per SM of 256 threads x 64 registers) leave every SM room for one of its persistent CTAs,
  // which would otherwise wait for this kernel's blocks to drain (~30 us per iteration).
  int grid = grid_for(g.nS);
  const int cap = (g.scope == RTCUR_SCOPE_FULL) ? kHtBlocksFull : kHtBlocksSampled;
  if (grid > cap) grid = cap;
  k_sample_ht<<<grid, kThreads, 0, s>>>(g, b);
  return cudaGetLastError();
}

cudaError_t launch_sample_err(const Geom& g, const Bufs& b, cudaStream_t s) {
  // In the FULL scope this kernel runs beside the dense pass: two blocks per SM, as for the
  // threshold kernel, take fewer of the pass's issue slots (measured 1.5% faster iterations at
  // 800^3 than 1024 blocks; one block per SM for both kernels lengthens the chain instead).
  int grid = grid_for(g.nS);
  const int cap = (g.scope == RTCUR_SCOPE_FULL) ? kHtBlocksFull : kHtBlocksSampled;
  if (grid > cap) grid = cap;
  k_sample_err<<<grid, kThreads, 0, s>>>(g, b);
  return cudaGetLastError();
}

cudaError_t launch_commit(const Geom& g, const Bufs& b, unsigned long long handle, int use_handle,
                          cudaStream_t s) {
  k_commit<<<1, 32, 0, s>>>(g, b, handle, use_handle);
  return cudaGetLastError();
}

cudaError_t launch_batch_any(State* const* sts, int count, unsigned long long handle, cudaStream_t s) {
  k_batch_any<<<1, 32, 0, s>>>(sts, count, handle);
  return cudaGetLastError();
}
