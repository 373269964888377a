// Dense fused pass (FULL scope): Step (I) of Algorithm 1 over the whole tensor,
//   S^(k+1) = HT_{zeta^(k+1)}(X - L^(k))          (Eq. S=HT(X-L), HT of Sec. 3.2)
// with L^(k) evaluated on the fly as the last-mode product of the table T and B_n, and the
// reductions ||X - L - S||_F^2, nnz(S) and the threshold-band count fused in. X is read once
// and S written once: 8 bytes of HBM traffic per element, so the kernel is bandwidth-bound.
//
// Mapping: the tensor is viewed as rowsT rows of d_n contiguous floats. A block owns a chunk of
// float4 columns and strides over rows; each thread keeps its four columns of B_n in registers
// for the whole launch, so the inner loop reads only X, one broadcast row of T, and writes S.
// Blocks use few threads per SM so that the latency-bound sampled chain, which runs
// concurrently on its own graph branch, finds room.
#include "../../include/rtcur.h"
#include "rtcur_internal.cuh"

namespace {

constexpr int kMaxRedBlocks = 1024;
constexpr int kRowUnroll = 4;

__device__ __forceinline__ double block_sum_d(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)((blockDim.x + 31) >> 5); ++i) t += sh[i];
  return t;
}

__device__ __forceinline__ void ht_acc(float x, float L, float zf, float band, float& s,
                                       float& res, unsigned& nnz, unsigned& inb) {
  float dl = x - L;
  float ad = fabsf(dl);
  bool keep = ad > zf;
  s = keep ? dl : 0.f;
  res = keep ? res : fmaf(dl, dl, res);
  nnz += keep ? 1u : 0u;
  inb += (fabsf(ad - zf) <= band) ? 1u : 0u;
}

template <bool VEC>
__global__ void __launch_bounds__(512) k_dense_fp32(Geom g, Bufs b) {
  __shared__ double sh[32];
  const State* st = b.st;
  const int cur = st->k & 1;
  const double zeta = g.gamma * st->zeta;
  const float zf = (float)zeta;
  const float band = (float)(g.inband * zeta);
  const float* __restrict__ X = b.sp->X;
  float* __restrict__ S = b.sp->S;
  const float* __restrict__ T = b.T[cur];
  const float* __restrict__ Bn = b.B[cur] + g.offB[g.n - 1];
  const int rn = g.rlast;
  const long long dn = g.d[g.n - 1];
  const long long rows = g.rowsT;
  float res = 0.f;
  unsigned nnz = 0u, inb = 0u;
  if (VEC) {
    const long long n4 = dn >> 2;
    const long long c4 = (long long)blockIdx.y * blockDim.x + threadIdx.x;
    if (c4 < n4) {
      float br[4][RT_MAXR];
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int c = 0; c < RT_MAXR; ++c) br[j][c] = (c < rn) ? __ldg(Bn + (c4 * 4 + j) * rn + c) : 0.f;
      const float4* X4 = reinterpret_cast<const float4*>(X);
      float4* S4 = reinterpret_cast<float4*>(S);
      for (long long r0 = blockIdx.x; r0 < rows; r0 += (long long)gridDim.x * kRowUnroll) {
        float4 xv[kRowUnroll];
#pragma unroll
        for (int u = 0; u < kRowUnroll; ++u) {
          long long r = r0 + (long long)u * gridDim.x;
          if (r < rows) xv[u] = __ldcs(X4 + r * n4 + c4);
        }
#pragma unroll
        for (int u = 0; u < kRowUnroll; ++u) {
          long long r = r0 + (long long)u * gridDim.x;
          if (r < rows) {
            const float* tr = T + r * rn;
            float L0 = 0.f, L1 = 0.f, L2 = 0.f, L3 = 0.f;
#pragma unroll
            for (int c = 0; c < RT_MAXR; ++c) {
              if (c < rn) {
                float t = __ldg(tr + c);
                L0 = fmaf(t, br[0][c], L0);
                L1 = fmaf(t, br[1][c], L1);
                L2 = fmaf(t, br[2][c], L2);
                L3 = fmaf(t, br[3][c], L3);
              }
            }
            float4 sv;
            ht_acc(xv[u].x, L0, zf, band, sv.x, res, nnz, inb);
            ht_acc(xv[u].y, L1, zf, band, sv.y, res, nnz, inb);
            ht_acc(xv[u].z, L2, zf, band, sv.z, res, nnz, inb);
            ht_acc(xv[u].w, L3, zf, band, sv.w, res, nnz, inb);
            __stcs(S4 + r * n4 + c4, sv);
          }
        }
      }
    }
  } else {
    const long long col = (long long)blockIdx.y * blockDim.x + threadIdx.x;
    if (col < dn) {
      float br[RT_MAXR];
#pragma unroll
      for (int c = 0; c < RT_MAXR; ++c) br[c] = (c < rn) ? __ldg(Bn + col * rn + c) : 0.f;
      for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
        float x = __ldcs(X + r * dn + col);
        const float* tr = T + r * rn;
        float L = 0.f;
#pragma unroll
        for (int c = 0; c < RT_MAXR; ++c)
          if (c < rn) L = fmaf(__ldg(tr + c), br[c], L);
        float s;
        ht_acc(x, L, zf, band, s, res, nnz, inb);
        __stcs(S + r * dn + col, s);
      }
    }
  }
  double* part = b.red + (size_t)TK_DENSE * kMaxRedBlocks * RT_RED_SLOTS;
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
  double t0 = block_sum_d((double)res, sh);
  if (threadIdx.x == 0) part[bid * RT_RED_SLOTS + 0] = t0;
  t0 = block_sum_d((double)nnz, sh);
  if (threadIdx.x == 0) part[bid * RT_RED_SLOTS + 1] = t0;
  t0 = block_sum_d((double)inb, sh);
  if (threadIdx.x == 0) part[bid * RT_RED_SLOTS + 2] = t0;
  if (last_block_arrive(b.ticket + TK_DENSE)) {
    State* w = b.st;
    const int nb = gridDim.x * gridDim.y;
    for (int slot = 0; slot < 3; ++slot) {
      double acc = 0.0;
      for (int i2 = threadIdx.x; i2 < nb; i2 += blockDim.x) acc += part[i2 * RT_RED_SLOTS + slot];
      acc = block_sum_d(acc, sh);
      if (threadIdx.x == 0) {
        if (slot == 0) w->resid_f = acc;
        if (slot == 1) w->nnz_f = (long long)acc;
        if (slot == 2) w->inband_f = (long long)acc;
      }
    }
    if (threadIdx.x == 0) b.ticket[TK_DENSE] = 0u;
  }
}

// ---------------------------------------------------------------- TMA-fed fused pass
// Persistent CTAs (148 of the 152 SMs, one CTA per SM by shared-memory footprint, so a few SMs
// stay free for the concurrent sampled chain). Each CTA streams tiles of `tr` whole rows of X
// (tr * d_n floats, ~32 KB) into a kStages-deep shared-memory ring with 1-D cp.async.bulk
// copies completed on mbarriers; one thread per float4 column computes L from its register
// copy of B_n and the tile's rows of T, thresholds, writes S over X in the stage, and the tile
// leaves in one 1-D bulk store. A stage is refilled once its store has read it (one tile
// later), so the stores overlap the next tile.
// Every mbarrier wait is bounded: on expiry the kernel records RTCUR_ETIMEOUT, drains its own
// copies (again bounded) and returns.
constexpr int kStages = 4;
constexpr long long kSpinLimit = 1LL << 26;
constexpr int kRowGroupsCompressed = 2;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
  for (long long i = 0; i < kSpinLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// 1-D bulk copy of streamed data with an L2 evict-first policy: the tensor passes through L2
// once, so it should not push out the small working set of the concurrent sampled chain.
__device__ __forceinline__ void bulk_g2s_stream(void* dst, const void* src, unsigned bytes,
                                                unsigned long long* bar) {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Compressed output of one row of S held by a warp: thread c4 (lane of warp w) owns columns
// 4 c4 .. 4 c4 + 3, so the warp owns the row's 128-column block w. Each lane's 4-bit keep nibble,
// shifted to its place and OR-reduced over groups of 8 lanes, gives the block's four mask words
// (word k from lanes 8k .. 8k + 7); four ballots give each kept value's rank in the block, and the
// values go, in order, from the block's first element on (vblk). Called by all 32 lanes of the
// warp (inactive lanes pass 0).
__device__ __forceinline__ void emit_row(unsigned* mrow, float* vblk, float4 sv, int wpr, int wid, int lane) {
  const bool k0 = sv.x != 0.f, k1 = sv.y != 0.f, k2 = sv.z != 0.f, k3 = sv.w != 0.f;
  unsigned w = ((unsigned)k0 | ((unsigned)k1 << 1) | ((unsigned)k2 << 2) | ((unsigned)k3 << 3)) << (4 * (lane & 7));
  w |= __shfl_xor_sync(0xffffffffu, w, 1);
  w |= __shfl_xor_sync(0xffffffffu, w, 2);
  w |= __shfl_xor_sync(0xffffffffu, w, 4);
  const int wk = 4 * wid + (lane >> 3);
  if ((lane & 7) == 0 && wk < wpr) mrow[wk] = w;
  const unsigned lt = (1u << lane) - 1u;
  unsigned rk = __popc(__ballot_sync(0xffffffffu, k0) & lt) + __popc(__ballot_sync(0xffffffffu, k1) & lt) +
                __popc(__ballot_sync(0xffffffffu, k2) & lt) + __popc(__ballot_sync(0xffffffffu, k3) & lt);
  if (k0) vblk[rk++] = sv.x;
  if (k1) vblk[rk++] = sv.y;
  if (k2) vblk[rk++] = sv.z;
  if (k3) vblk[rk] = sv.w;
}

// MODE 0: the fused threshold pass of an iteration (L^(k), zeta^(k+1), S into the solve's S
//         buffer, reductions). MODE 1: write L of copy `copy_sel` (0 = current, 1 = previous)
//         into `out` (no X read). MODE 2: write HT_{zeta^(k)}(X - L) of copy `copy_sel` into
//         `out` (zero when k = 0). Modes 1 and 2 materialise the solve's outputs.
// MODE 3: MODE 0 with S written compressed instead of dense: the support as bitmask words (bit
//         b of word w of row r is S(r, 32 w + b) != 0) and, for each 128-column block of a row,
//         its nonzero values in order from the block's first element index on. At 30% density
//         that is 4 + 1/8 + 1.2 bytes per element instead of 8.
// PAIR (MODE 0 only, blocks of at most 512 threads, i.e. d_n <= 2048): the row loop takes two
// rows per step, which needs more than the 64 registers a thread that a 1024-thread block allows.
template <int RN, int MODE, bool PAIR = false>
__global__ void __launch_bounds__(PAIR ? 512 : 1024, 1) k_dense_tma(Geom g, Bufs b, int tr, int copy_sel, float* out) {
  TL_BEGIN();
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ unsigned long long full[kStages];
  __shared__ double sh[32];
  __shared__ int abort_flag;
  __shared__ long long tile_of[kStages];     // tile held by each stage, -1: no more tiles
  const State* st = b.st;
  const int kk = st->k;
  const long long polls = st->wait_polls;
  constexpr bool kFused = (MODE == 0 || MODE == 3);  // the iteration's threshold pass
  const int cur = kFused ? (kk & 1) : ((kk + copy_sel) & 1);
  const double zeta = kFused ? g.gamma * st->zeta : st->zeta;
  const float zf = (float)zeta;
  const float band = (float)(g.inband * zeta);
  const bool zero_out = (MODE == 2) && (kk == 0);
  const float* __restrict__ X = b.sp->X;
  float* __restrict__ S = (MODE == 0) ? b.sp->S : out;  // unused by MODE 3
  const float* __restrict__ T = b.T[cur];
  const float* __restrict__ Bn = b.B[cur] + g.offB[g.n - 1];
  const long long dn = g.d[g.n - 1];
  const int n4 = (int)(dn >> 2);
  const long long rows = g.rowsT;
  const long long ntiles = (rows + tr - 1) / tr;
  const unsigned tile_bytes_full = (unsigned)(tr * dn * 4);
  float4* ring = reinterpret_cast<float4*>(dsm);
  const int stage_f4 = tr * n4;
  // T rows of a tile: floats [r0*RN rounded down to 4, (r0+nr)*RN rounded up to 4)
  const int tstage = ((tr * RN + 3) & ~3) + 4;
  float* tring = reinterpret_cast<float*>(ring + (size_t)kStages * stage_f4);
  // blockDim.x = G row groups of rowT threads: thread c4 of group grp owns float4 column c4 of
  // rows grp, grp + G, ... of each tile (G > 1 gives the latency-bound row loop more warps)
  const int rowT = ((n4 + 31) / 32) * 32;
  const int G = (int)blockDim.x / rowT;
  const int grp = (int)threadIdx.x / rowT;
  const int c4 = (int)threadIdx.x - grp * rowT;
  const int wpr = (int)((dn + 31) >> 5);  // MODE 3: mask words per row
  float br[4][RN];
  if (c4 < n4) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int c = 0; c < RN; ++c) br[j][c] = __ldg(Bn + ((long long)c4 * 4 + j) * RN + c);
  }
  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int i = 0; i < kStages; ++i) mbar_init(&full[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // Tiles: the first kStages x grid go out statically (stage s of CTA c holds tile c + s grid).
  // The compressed pass (MODE 3, ~3.7 us a tile) then hands out the rest from a counter, so CTAs
  // that share their SM with the sampled chain's blocks take fewer tiles (1.73 -> 1.67 ms at
  // 800^3). The other modes keep the static stride in a counted loop: the dense pass with tiles
  // from the counter ran at 0.84-0.85 ms against 0.67 ms, with one tile per atomic and equally
  // with 8 or 16, so the cost is the uncounted loop, not the atomics.
  // Thread 0 alone issues copies and counts, per stage, the copies issued and the completions it
  // has observed (for the bounded drain). In MODE 3 a stage past the last tile gets tile -1 and a
  // plain arrive instead of a copy.
  int issued[kStages], seen[kStages];
#pragma unroll
  for (int s = 0; s < kStages; ++s) issued[s] = seen[s] = 0;
  auto issue_tile = [&](int s, long long t) {  // MODE 3, thread 0 only
    if (t < ntiles) {
      long long r0 = t * tr;
      long long nr = (r0 + tr <= rows ? tr : rows - r0);
      unsigned bytes = (MODE == 1) ? 0u : (unsigned)(nr * dn * 4);
      long long a0 = (r0 * RN) & ~3LL, a1 = ((r0 + nr) * RN + 3) & ~3LL;
      unsigned tbytes = (unsigned)((a1 - a0) * 4);
      tile_of[s] = t;
      mbar_expect_tx(&full[s], bytes + tbytes);
      if (bytes) bulk_g2s_stream(ring + (size_t)s * stage_f4, X + r0 * dn, bytes, &full[s]);
      bulk_g2s(tring + (size_t)s * tstage, T + a0, tbytes, &full[s]);
    } else {
      tile_of[s] = -1;
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full[s])) : "memory");
    }
#pragma unroll
    for (int s2 = 0; s2 < kStages; ++s2) issued[s2] += (s2 == s) ? 1 : 0;
  };
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < kStages; ++s) {
      const long long t = (long long)blockIdx.x + (long long)s * gridDim.x;
      if (MODE == 3) {
        issue_tile(s, t);
      } else if (t < ntiles) {
        long long r0 = t * tr;
        long long nr = (r0 + tr <= rows ? tr : rows - r0);
        unsigned bytes = (MODE == 1) ? 0u : (unsigned)(nr * dn * 4);
        long long a0 = (r0 * RN) & ~3LL, a1 = ((r0 + nr) * RN + 3) & ~3LL;
        unsigned tbytes = (unsigned)((a1 - a0) * 4);
        mbar_expect_tx(&full[s], bytes + tbytes);
        if (bytes) bulk_g2s_stream(ring + (size_t)s * stage_f4, X + r0 * dn, bytes, &full[s]);
        bulk_g2s(tring + (size_t)s * tstage, T + a0, tbytes, &full[s]);
        issued[s] = 1;
      }
    }
  }
  float res = 0.f;
  unsigned nnz = 0u, inb = 0u;
  const long long stride = (long long)kStages * gridDim.x;
  // MODE 3: thread 0 keeps the next two tiles of the counter in hand, fetched two refills ahead
  // (the atomic's round trip under full HBM load). Tiles are issued in the order they were
  // fetched, so any left over at the end lie past the last tile.
  constexpr bool kDyn = (MODE == 3);
  long long tq0 = -1, tq1 = -1;
  if (kDyn && threadIdx.x == 0) {
    tq0 = stride + (long long)atomicAdd(b.ticket + TK_DTILE, 1u);
    tq1 = stride + (long long)atomicAdd(b.ticket + TK_DTILE, 1u);
  }
  if (polls > 0) {
    // a caller-set bound (rtcur_set_wait_limit): the launch's first wait makes `polls`
    // non-blocking tests and gives up if its copy has not landed by then. The tile loop below
    // then waits for that copy with the default bound and stops, and the drain completes the rest.
    // Kept out of the loop, whose code stays that of the default bound.
    bool ok = (blockIdx.x >= ntiles);
    for (long long i = 0; i < polls && !ok; ++i) ok = mbar_test(&full[0], 0u);
    if (!ok) abort_flag = 1;
    __syncthreads();
  }
  int it = 0;
  // static modes: tile t = CTA + it grid, known before the wait; MODE 3 reads it from the stage
  for (long long t = blockIdx.x; kDyn || t < ntiles; t += gridDim.x, ++it) {
    const int s = it % kStages;
    const unsigned par = (unsigned)((it / kStages) & 1);
    long long tnext = -1;
    if (kDyn && threadIdx.x == 0) {  // every iteration of MODE 3 refills a stage
      tnext = tq0;
      tq0 = tq1;
      tq1 = stride + (long long)atomicAdd(b.ticket + TK_DTILE, 1u);
    }
    if (!mbar_wait_bounded(&full[s], par)) {
      abort_flag = 1;
    } else if (threadIdx.x == 0) {
#pragma unroll
      for (int s2 = 0; s2 < kStages; ++s2) seen[s2] += (s2 == s) ? 1 : 0;
    }
    __syncthreads();
    if (abort_flag) break;
    if (kDyn) {
      t = tile_of[s];
      if (t < 0) break;  // the same value for every thread
    }
    const long long r0 = t * tr;
    const int nr = (int)(r0 + tr <= rows ? tr : rows - r0);
    if (MODE == 3 || c4 < n4) {  // MODE 3: whole warps, for the ballots of the compressed rows
      const bool act = c4 < n4;
      const float4* tile = ring + (size_t)s * stage_f4;
      const float* ttile = tring + (size_t)s * tstage + (r0 * RN - ((r0 * RN) & ~3LL));
      if (PAIR) {
        // two rows per step: both rows' T and X values are read before either S row is written
        // (row by row, each read waits for the previous row's store, whose address lies a runtime
        // stride away and so cannot be told apart by the compiler)
        for (int rr = grp; rr < nr && act; rr += 2 * G) {
          const int rb = rr + G;
          const bool two = rb < nr;
          float ta[RN], tb[RN];
#pragma unroll
          for (int c = 0; c < RN; ++c) {
            ta[c] = ttile[rr * RN + c];
            tb[c] = two ? ttile[rb * RN + c] : 0.f;
          }
          float4 xa = make_float4(0.f, 0.f, 0.f, 0.f), xb = xa;
          if (MODE != 1) {
            xa = tile[rr * n4 + c4];
            if (two) xb = tile[rb * n4 + c4];
          }
          float La[4] = {0.f, 0.f, 0.f, 0.f}, Lb[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int c = 0; c < RN; ++c)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              La[j] = fmaf(ta[c], br[j][c], La[j]);
              Lb[j] = fmaf(tb[c], br[j][c], Lb[j]);
            }
          float4 sa, sb;
          if (MODE == 1) {
            sa = make_float4(La[0], La[1], La[2], La[3]);
            sb = make_float4(Lb[0], Lb[1], Lb[2], Lb[3]);
          } else {
            sa = sb = make_float4(0.f, 0.f, 0.f, 0.f);
            ht_acc(xa.x, La[0], zf, band, sa.x, res, nnz, inb);
            ht_acc(xa.y, La[1], zf, band, sa.y, res, nnz, inb);
            ht_acc(xa.z, La[2], zf, band, sa.z, res, nnz, inb);
            ht_acc(xa.w, La[3], zf, band, sa.w, res, nnz, inb);
            if (two) {
              ht_acc(xb.x, Lb[0], zf, band, sb.x, res, nnz, inb);
              ht_acc(xb.y, Lb[1], zf, band, sb.y, res, nnz, inb);
              ht_acc(xb.z, Lb[2], zf, band, sb.z, res, nnz, inb);
              ht_acc(xb.w, Lb[3], zf, band, sb.w, res, nnz, inb);
            }
            if (zero_out) sa = sb = make_float4(0.f, 0.f, 0.f, 0.f);
          }
          const_cast<float4*>(tile)[rr * n4 + c4] = sa;  // in place: one copy out
          if (two) const_cast<float4*>(tile)[rb * n4 + c4] = sb;
        }
      } else
      for (int rr = grp; rr < nr; rr += G) {
        float4 sv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (act) {
          float tv[RN];
#pragma unroll
          for (int c = 0; c < RN; ++c) tv[c] = ttile[rr * RN + c];
          float L0 = 0.f, L1 = 0.f, L2 = 0.f, L3 = 0.f;
#pragma unroll
          for (int c = 0; c < RN; ++c) {
            L0 = fmaf(tv[c], br[0][c], L0);
            L1 = fmaf(tv[c], br[1][c], L1);
            L2 = fmaf(tv[c], br[2][c], L2);
            L3 = fmaf(tv[c], br[3][c], L3);
          }
          if (MODE == 1) {
            sv = make_float4(L0, L1, L2, L3);
          } else {
            float4 xv = tile[rr * n4 + c4];
            ht_acc(xv.x, L0, zf, band, sv.x, res, nnz, inb);
            ht_acc(xv.y, L1, zf, band, sv.y, res, nnz, inb);
            ht_acc(xv.z, L2, zf, band, sv.z, res, nnz, inb);
            ht_acc(xv.w, L3, zf, band, sv.w, res, nnz, inb);
            if (zero_out) sv = make_float4(0.f, 0.f, 0.f, 0.f);
          }
          if (MODE != 3) const_cast<float4*>(tile)[rr * n4 + c4] = sv;  // in place: one copy out
        }
        if (MODE == 3)
          emit_row(b.smask + (r0 + rr) * wpr, b.svals + (r0 + rr) * dn + (c4 & ~31) * 4, sv, wpr, c4 >> 5,
                   (int)(threadIdx.x & 31));
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // stage writes -> bulk store
    __syncthreads();  // stage s fully consumed and holding the output rows
    if (MODE == 3) {  // the stage is read: refill it
      if (threadIdx.x == 0) issue_tile(s, kDyn ? tnext : t + stride);
    } else if (threadIdx.x == 0) {
      // the tile's output rows leave in one bulk copy; the stage of the previous tile, whose
      // store has now read it, is refilled with the tile kStages ahead of that one
      asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(S + r0 * dn),
                   "r"(smem_u32(ring + (size_t)s * stage_f4)), "r"((unsigned)(nr * dn * 4))
                   : "memory");
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      if (it >= 1) {
        asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        const int sp = (it - 1) % kStages;
        const long long tn = t + (long long)(kStages - 1) * gridDim.x;
        if (tn < ntiles) {
          long long rn0 = tn * tr;
          long long nr2 = (rn0 + tr <= rows ? tr : rows - rn0);
          unsigned bytes = (MODE == 1) ? 0u : (unsigned)(nr2 * dn * 4);
          long long a0 = (rn0 * RN) & ~3LL, a1 = ((rn0 + nr2) * RN + 3) & ~3LL;
          unsigned tbytes = (unsigned)((a1 - a0) * 4);
          mbar_expect_tx(&full[sp], bytes + tbytes);
          if (bytes) bulk_g2s_stream(ring + (size_t)sp * stage_f4, X + rn0 * dn, bytes, &full[sp]);
          bulk_g2s(tring + (size_t)sp * tstage, T + a0, tbytes, &full[sp]);
#pragma unroll
          for (int s2 = 0; s2 < kStages; ++s2) issued[s2] += (s2 == sp) ? 1 : 0;
        }
      }
    }
  }
  if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // output written
  if (abort_flag) {
    // drain: wait (bounded) for every copy this CTA may still have in flight
    if (threadIdx.x == 0) {
      atomicExch(&b.st->err, -5);  // RTCUR_ETIMEOUT
#pragma unroll
      for (int s2 = 0; s2 < kStages; ++s2) {
        // the newest copy on stage s2 completes phase number issued-1 (parity (issued-1) & 1)
        if (issued[s2] > seen[s2]) mbar_wait_bounded(&full[s2], (unsigned)((issued[s2] - 1) & 1));
      }
    }
    __syncthreads();
  }
  (void)tile_bytes_full;
  if (!kFused) return;
  double* part = b.red + (size_t)TK_DENSE * kMaxRedBlocks * RT_RED_SLOTS;
  const int bid = blockIdx.x;
  double t0 = block_sum_d((double)res, sh);
  if (threadIdx.x == 0) part[bid * RT_RED_SLOTS + 0] = t0;
  t0 = block_sum_d((double)nnz, sh);
  if (threadIdx.x == 0) part[bid * RT_RED_SLOTS + 1] = t0;
  t0 = block_sum_d((double)inb, sh);
  if (threadIdx.x == 0) part[bid * RT_RED_SLOTS + 2] = t0;
  if (last_block_arrive(b.ticket + TK_DENSE)) {
    State* w = b.st;
    for (int slot = 0; slot < 3; ++slot) {
      double acc = 0.0;
      for (unsigned i2 = threadIdx.x; i2 < gridDim.x; i2 += blockDim.x) acc += part[i2 * RT_RED_SLOTS + slot];
      acc = block_sum_d(acc, sh);
      if (threadIdx.x == 0) {
        if (slot == 0) w->resid_f = acc;
        if (slot == 1) w->nnz_f = (long long)acc;
        if (slot == 2) w->inband_f = (long long)acc;
      }
    }
    if (threadIdx.x == 0) {
      if (MODE == 3) b.ticket[TK_DTILE] = 0u;  // every CTA has taken its last tile
      b.ticket[TK_DENSE] = 0u;
    }
  }
  TL_END(MODE == 3 ? 1 : 1 + 20 * MODE);
}

template <int RN>
cudaError_t launch_tma_rn(const Geom& g, const Bufs& b, int tr, size_t smem, int grid, int threads,
                          cudaStream_t s, int mode = 0, int copy_sel = 0, float* out = nullptr) {
  if (mode == 0 && threads <= 512)
    k_dense_tma<RN, 0, true><<<grid, threads, smem, s>>>(g, b, tr, copy_sel, out);
  else if (mode == 0)
    k_dense_tma<RN, 0><<<grid, threads, smem, s>>>(g, b, tr, copy_sel, out);
  else if (mode == 3)
    k_dense_tma<RN, 3><<<grid, threads, smem, s>>>(g, b, tr, copy_sel, out);
  else if (mode == 1)
    k_dense_tma<RN, 1><<<grid, threads, smem, s>>>(g, b, tr, copy_sel, out);
  else
    k_dense_tma<RN, 2><<<grid, threads, smem, s>>>(g, b, tr, copy_sel, out);
  return cudaGetLastError();
}

// The pass streams its data, so it gives L1 away: the SMs it runs on are configured with the
// maximum shared-memory carveout, which leaves room beside its ring for the concurrent sampled
// chain's blocks (a smaller carveout would make them wait for the pass to finish).
template <int RN>
cudaError_t prepare_tma_rn(size_t smem) {
  cudaError_t e = cudaSuccess;
  void* fns[5] = {(void*)k_dense_tma<RN, 0>, (void*)k_dense_tma<RN, 1>, (void*)k_dense_tma<RN, 2>,
                  (void*)k_dense_tma<RN, 3>, (void*)k_dense_tma<RN, 0, true>};
  for (void* f : fns) {
    if (e == cudaSuccess) e = raise_smem_limit((const void*)f, (size_t)(smem));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  }
  return e;
}

template <int RN>
cudaError_t tma_materialize_rn(const Geom& g, const Bufs& b, int tr, size_t smem, int grid,
                               int threads, float* L_out, float* S_out, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (L_out) e = launch_tma_rn<RN>(g, b, tr, smem, grid, threads, s, 1, 0, L_out);
  if (e == cudaSuccess && S_out) e = launch_tma_rn<RN>(g, b, tr, smem, grid, threads, s, 2, 1, S_out);
  return e;
}

// Tile geometry of the TMA pass; returns false when the pass does not apply (d_n % 4 != 0,
// d_n > 4096, r_n > 8).
bool tma_geometry(const Geom& g, int& tr, size_t& smem, int& threads) {
  const long long dn = g.d[g.n - 1];
  if (dn % 4 != 0 || dn > 4096 || g.rlast > 8) return false;
  long long t = 32768 / (dn * 4);  // ~32 KB tiles, kStages deep
  if (t < 1) t = 1;
  if (t > g.rowsT) t = g.rowsT;
  tr = (int)t;
  smem = (size_t)kStages * (tr * dn * 4 + (((tr * g.rlast + 3) & ~3) + 4) * 4);
  threads = (int)(((dn / 4 + 31) / 32) * 32);
  return true;
}

// L_out = L^(k) (copy k & 1); S_out = HT_{zeta^(k)}(X - L^(k-1)) (copy (k-1) & 1), zero if k = 0.
// Rows of d_n floats; a block strides over rows, each thread owns one column.
__global__ void __launch_bounds__(256) k_materialize(Geom g, Bufs b, float* L_out, float* S_out) {
  const State* st = b.st;
  const int k = st->k;
  const int cur = k & 1, prv = (k + 1) & 1;
  const float zf = (float)st->zeta;
  const float* X = b.sp->X;
  const int rn = g.rlast;
  const long long dn = g.d[g.n - 1];
  const long long col = (long long)blockIdx.y * blockDim.x + threadIdx.x;
  if (col >= dn) return;
  const float* Tc = b.T[cur];
  const float* Tp = b.T[prv];
  float bc[RT_MAXR], bp[RT_MAXR];
#pragma unroll
  for (int c = 0; c < RT_MAXR; ++c) {
    bc[c] = (c < rn) ? b.B[cur][g.offB[g.n - 1] + col * rn + c] : 0.f;
    bp[c] = (c < rn) ? b.B[prv][g.offB[g.n - 1] + col * rn + c] : 0.f;
  }
#pragma unroll 8
  for (long long r = blockIdx.x; r < g.rowsT; r += gridDim.x) {
    const long long e = r * dn + col;
    if (L_out) {
      float L = 0.f;
#pragma unroll
      for (int c = 0; c < RT_MAXR; ++c)
        if (c < rn) L = fmaf(__ldg(Tc + r * rn + c), bc[c], L);
      __stcs(L_out + e, (k == 0) ? 0.f : L);
    }
    if (S_out) {
      float sv = 0.f;
      if (k > 0) {
        float L = 0.f;
#pragma unroll
        for (int c = 0; c < RT_MAXR; ++c)
          if (c < rn) L = fmaf(__ldg(Tp + r * rn + c), bp[c], L);
        float dl = __ldcs(X + e) - L;
        sv = (fabsf(dl) > zf) ? dl : 0.f;
      }
      __stcs(S_out + e, sv);
    }
  }
}

// Expansion of the compressed S (MODE 3) into a dense tensor: one warp per row, one mask word
// (32 columns) per step; a value's rank in its 128-column block is the bits before it in the
// block's words.
__global__ void __launch_bounds__(256) k_decode_s(Geom g, Bufs b, float* S_out) {
  const long long row = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = (int)(threadIdx.x & 31);
  if (row >= g.rowsT) return;
  const long long dn = g.d[g.n - 1];
  const int wpr = (int)((dn + 31) >> 5);
  const unsigned* mrow = b.smask + row * wpr;
  const float* vrow = b.svals + row * dn;
  const unsigned lt = (1u << lane) - 1u;
  unsigned before = 0u;  // bits in the earlier words of the current block
  for (int w = 0; w < wpr; ++w) {
    if ((w & 3) == 0) before = 0u;
    const unsigned m = mrow[w];
    const long long c = 32LL * w + lane;
    if (c < dn) S_out[row * dn + c] = ((m >> lane) & 1u) ? vrow[128 * (w >> 2) + before + __popc(m & lt)] : 0.f;
    before += (unsigned)__popc(m);
  }
}

// Nonzeros per row: cnt[row] = popcount of the row's mask words (one warp per row).
__global__ void __launch_bounds__(256) k_row_counts(Geom g, Bufs b, long long* cnt) {
  const long long row = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = (int)(threadIdx.x & 31);
  if (row >= g.rowsT) return;
  const int wpr = (int)((g.d[g.n - 1] + 31) >> 5);
  unsigned c = 0u;
  for (int w = lane; w < wpr; w += 32) c += (unsigned)__popc(b.smask[row * wpr + w]);
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) cnt[row] = c;
}

// Exclusive scan, in place, of v[0 .. n) in chunks of 1024 (one block per chunk); the chunk's
// total goes to tot[chunk]. With add = 1 instead, each element gets tot[chunk] added.
__global__ void __launch_bounds__(1024) k_scan_chunks(long long* v, long long n, long long* tot, int add) {
  __shared__ long long wsum[32];
  const long long i = (long long)blockIdx.x * 1024 + threadIdx.x;
  if (add) {
    if (i < n) v[i] += tot[blockIdx.x];
    return;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long c = i < n ? v[i] : 0;
  long long x = c;
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    long long w = wsum[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    wsum[lane] = w;  // inclusive over the warps
  }
  __syncthreads();
  const long long before = wid > 0 ? wsum[wid - 1] : 0;
  if (i < n) v[i] = before + x - c;
  if (threadIdx.x == 1023) tot[blockIdx.x] = before + x;
}

// Every row's values, block after block, to out[off[row] ...]: the nonzeros in element order
// (one warp per row).
__global__ void __launch_bounds__(256) k_compact_s(Geom g, Bufs b, const long long* off, float* out) {
  const long long row = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = (int)(threadIdx.x & 31);
  if (row >= g.rowsT) return;
  const long long dn = g.d[g.n - 1];
  const int wpr = (int)((dn + 31) >> 5);
  const unsigned* mrow = b.smask + row * wpr;
  const float* vrow = b.svals + row * dn;
  long long o = off[row];
  for (int blk = 0; 4 * blk < wpr; ++blk) {
    unsigned n = 0u;
    for (int w = 4 * blk; w < 4 * blk + 4 && w < wpr; ++w) n += (unsigned)__popc(mrow[w]);
    for (unsigned i = lane; i < n; i += 32) out[o + i] = vrow[128 * blk + i];
    o += n;
  }
}

}  // namespace

bool compressed_geometry(const Geom& g, int& tile_rows) {
  int threads;
  size_t smem;
  int tr = 0;
  if (!tma_geometry(g, tr, smem, threads)) return false;
  tile_rows = tr;
  return true;
}

cudaError_t launch_decode_s(const Geom& g, const Bufs& b, float* S_out, cudaStream_t s) {
  k_decode_s<<<(unsigned)((g.rowsT + 7) / 8), 256, 0, s>>>(g, b, S_out);
  return cudaGetLastError();
}

// Exclusive scan of v[0 .. n) in place; scratch holds n / 1023 + 64 entries (the chunk totals of
// every level).
cudaError_t scan_exclusive(long long* v, long long n, long long* scratch, cudaStream_t s) {
  const long long nch = (n + 1023) / 1024;
  k_scan_chunks<<<(unsigned)nch, 1024, 0, s>>>(v, n, scratch, 0);
  if (nch == 1) return cudaGetLastError();
  cudaError_t e = scan_exclusive(scratch, nch, scratch + nch, s);
  if (e != cudaSuccess) return e;
  k_scan_chunks<<<(unsigned)nch, 1024, 0, s>>>(v, n, scratch, 1);
  return cudaGetLastError();
}

cudaError_t launch_compact_s(const Geom& g, const Bufs& b, long long* off, float* out, cudaStream_t s) {
  const long long rows = g.rowsT;
  const unsigned blocks = (unsigned)((rows + 7) / 8);
  cudaError_t e = cudaMemsetAsync(off + rows, 0, sizeof(long long), s);
  if (e != cudaSuccess) return e;
  k_row_counts<<<blocks, 256, 0, s>>>(g, b, off);
  if ((e = scan_exclusive(off, rows + 1, b.soff, s)) != cudaSuccess || !out) return e;
  k_compact_s<<<blocks, 256, 0, s>>>(g, b, off, out);
  return cudaGetLastError();
}

bool dense_form_supported(const Geom& g, int form) {
  if (form == 0) return true;
  if (form == 1) return g.n == 3 && (g.N % 4) == 0;
  if (form == 2) return umma_smem(g, 0) > 0;
  if (form == 3) return umma_smem(g, 1) > 0;
  return false;
}

cudaError_t prepare_dense(const Geom& g) {
  int tr, threads;
  size_t smem;
  if (g.dense_form == 2 || g.dense_form == 3) {
    cudaError_t e = prepare_umma(g, g.dense_form == 2 ? 0 : 1);
    if (e != cudaSuccess) return e;
  }
  if (!tma_geometry(g, tr, smem, threads)) return cudaSuccess;
  switch (g.rlast) {
    case 1: return prepare_tma_rn<1>(smem);
    case 2: return prepare_tma_rn<2>(smem);
    case 3: return prepare_tma_rn<3>(smem);
    case 4: return prepare_tma_rn<4>(smem);
    case 5: return prepare_tma_rn<5>(smem);
    case 6: return prepare_tma_rn<6>(smem);
    case 7: return prepare_tma_rn<7>(smem);
    default: return prepare_tma_rn<8>(smem);
  }
}

cudaError_t launch_dense(const Geom& g, const Bufs& b, int form, cudaStream_t s) {
  if (form == 1) return launch_plain_dense(g, b, s);
  if (form == 2) return launch_umma(g, b, 0, s);
  if (form == 3) return launch_umma(g, b, 1, s);
  if (form != 0) return cudaErrorNotSupported;
  if (g.s_format == RTCUR_S_COMPRESSED && g.tile_rows < 1) return cudaErrorNotSupported;
  {
    int tr, threads;
    size_t smem;
    if (tma_geometry(g, tr, smem, threads)) {
      long long ntiles = (g.rowsT + tr - 1) / tr;
      // 148 persistent CTAs: measured best for the iteration at 800^3 (the pass alone keeps
      // gaining up to 152, but the concurrent sampled chain then finds no room on any SM)
      int ctas = g.dense_ctas > 0 ? g.dense_ctas : 148;
      int grid = (int)(ntiles < ctas ? ntiles : ctas);
      const int mode = (g.s_format == RTCUR_S_COMPRESSED) ? 3 : 0;
      // the compressed pass runs two row groups: twice the warps for its longer row loop, and
      // still room beside it for a CTA of the sampled chain's refinement cluster
      if (mode == 3 && 2 * threads <= 1024) threads *= kRowGroupsCompressed;
      switch (g.rlast) {
        case 1: return launch_tma_rn<1>(g, b, tr, smem, grid, threads, s, mode);
        case 2: return launch_tma_rn<2>(g, b, tr, smem, grid, threads, s, mode);
        case 3: return launch_tma_rn<3>(g, b, tr, smem, grid, threads, s, mode);
        case 4: return launch_tma_rn<4>(g, b, tr, smem, grid, threads, s, mode);
        case 5: return launch_tma_rn<5>(g, b, tr, smem, grid, threads, s, mode);
        case 6: return launch_tma_rn<6>(g, b, tr, smem, grid, threads, s, mode);
        case 7: return launch_tma_rn<7>(g, b, tr, smem, grid, threads, s, mode);
        default: return launch_tma_rn<8>(g, b, tr, smem, grid, threads, s, mode);
      }
    }
  }
  const long long dn = g.d[g.n - 1];
  const bool vec = (dn % 4) == 0;
  const long long cols = vec ? dn / 4 : dn;
  int bx = (int)(((cols + 31) / 32) * 32);
  if (bx > 512) bx = 512;
  int gy = (int)((cols + bx - 1) / bx);
  // about four blocks of bx threads per SM, capped by the reduction slots
  long long gx = (152LL * 4 * 256) / bx;
  if (gx * gy > kMaxRedBlocks) gx = kMaxRedBlocks / gy;
  if (gx < 1) gx = 1;
  if (gx > g.rowsT) gx = g.rowsT;
  dim3 grid((unsigned)gx, (unsigned)gy);
  if (vec)
    k_dense_fp32<true><<<grid, bx, 0, s>>>(g, b);
  else
    k_dense_fp32<false><<<grid, bx, 0, s>>>(g, b);
  return cudaGetLastError();
}

cudaError_t launch_materialize(const Geom& g, const Bufs& b, float* L_out, float* S_out,
                               cudaStream_t s) {
  if (!L_out && !S_out) return cudaSuccess;
  {
    int tr, threads;
    size_t smem;
    if (tma_geometry(g, tr, smem, threads)) {
      long long ntiles = (g.rowsT + tr - 1) / tr;
      // the outputs are written after the loop, with nothing beside them: every SM
      int grid = (int)(ntiles < 152 ? ntiles : 152);
      switch (g.rlast) {
        case 1: return tma_materialize_rn<1>(g, b, tr, smem, grid, threads, L_out, S_out, s);
        case 2: return tma_materialize_rn<2>(g, b, tr, smem, grid, threads, L_out, S_out, s);
        case 3: return tma_materialize_rn<3>(g, b, tr, smem, grid, threads, L_out, S_out, s);
        case 4: return tma_materialize_rn<4>(g, b, tr, smem, grid, threads, L_out, S_out, s);
        case 5: return tma_materialize_rn<5>(g, b, tr, smem, grid, threads, L_out, S_out, s);
        case 6: return tma_materialize_rn<6>(g, b, tr, smem, grid, threads, L_out, S_out, s);
        case 7: return tma_materialize_rn<7>(g, b, tr, smem, grid, threads, L_out, S_out, s);
        default: return tma_materialize_rn<8>(g, b, tr, smem, grid, threads, L_out, S_out, s);
      }
    }
  }
  const long long dn = g.d[g.n - 1];
  int bx = (int)(dn < 256 ? ((dn + 31) / 32) * 32 : 256);
  unsigned gy = (unsigned)((dn + bx - 1) / bx);
  long long gx = (152LL * 8 * 256) / (bx * (long long)gy);
  if (gx < 1) gx = 1;
  if (gx > g.rowsT) gx = g.rowsT;
  k_materialize<<<dim3((unsigned)gx, gy), bx, 0, s>>>(g, b, L_out, S_out);
  return cudaGetLastError();
}
