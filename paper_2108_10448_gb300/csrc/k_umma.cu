// Tensor-core forms of the dense fused pass on the 5th-generation tensor cores (tcgen05):
// S^(k+1) = HT_{zeta^(k+1)}(X - L^(k)) over the whole tensor (Step (I) of Algorithm 1, Eq. (HT)),
// with the last mode product L = T B_n^T (T = G x_1 B_1 ... x_{n-1} B_{n-1}, Eq. (L=CUR) in
// Tucker form) computed by tcgen05.mma into tensor memory.
//
// The product is taken transposed: for a tile of 16 whole rows of X and a block of 128 columns,
// D = B_n(block, :) T(tile rows, :)^T is one MMA with M = 128 (columns of X: TMEM lanes) and
// N = 16 (rows of X: TMEM columns). X therefore moves in whole rows, as contiguous 1-D bulk copies
// in both directions, and the epilogue reads it with one column per thread: consecutive threads
// touch consecutive floats of shared memory, conflict-free without a swizzle.
// One persistent CTA per SM; its footprint (80 registers a thread, at most 184 KB of shared
// memory) leaves each SM room for a CTA of the sampled chain's refinement cluster, which runs
// beside this pass in the same iteration. Warp roles (a contiguous range of tiles per CTA):
//   * producer warp: 1-D bulk loads of half tiles (8 rows) into a shared-memory ring (mbarriers);
//   * MMA warp: the tile's 16 rows of T as the B operand (K-major, double-buffered) and one
//     tcgen05.mma per 128-column block into a per-tile TMEM accumulator (two tiles in flight);
//     B_n is the A operand, staged once per launch, one 128-row block per column block;
//   * two epilogue warpgroups, warpgroup h on rows 8h..8h+7 of every tile: tcgen05.ld of its 8
//     accumulator columns per block (warp w reads TMEM lanes 32(w%4)..: 32 columns of X), X from
//     its half stage, threshold, S written in place, then an arrive on the stage's done barrier
//     (each warp on its own: no barrier inside the warpgroup). The residual / nnz / band sums are
//     fused;
//   * store warp: once the four warps of a half tile have arrived, one 1-D bulk store of it; a
//     stage goes back to the producer once its store has read it (checked at the next store).
// Forms (FP32 accumulation in both):
//   BF16: kind::f16 with BF16 operands split x = hi + lo, the three significant products
//         B_hi T_hi + B_hi T_lo + B_lo T_hi packed along K = 16 (3 r_n <= 15); the dropped lo*lo
//         term is ~2^-16 relative.
//   TF32: kind::tf32, K = 8 >= r_n, operands rounded to TF32 (10-bit mantissa).
// Every mbarrier wait is bounded; on expiry the kernel records RTCUR_ETIMEOUT, waits (bounded) for
// its own copies and MMAs in flight, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include "rtcur_internal.cuh"

namespace {

constexpr int kUEpiWarps = 8;                      // warps 0-7: epilogue (two warpgroups)
// + warp 8: bulk-copy producer, warp 9: MMA, warp 10: bulk stores of S
constexpr int kUThreads = 32 * (kUEpiWarps + 3);
constexpr int kURows = 16;                         // rows per tile (N of the MMA)
constexpr int kUHalf = kURows / 2;                 // rows per ring stage (one warpgroup's half)
constexpr int kUCols = 128;                        // columns per block (M of the MMA)
constexpr int kUMaxStages = 8;
constexpr int kUOpBytesA = kUCols * 32;            // A: 128 rows (columns of X) x 32 bytes of K
constexpr int kUOpBytesB = kURows * 32;            // B: 16 rows of T x 32 bytes of K
constexpr int kUMaxCb = 8;                         // column blocks (d_n <= 1024)
constexpr int kUGroup = 2;                         // blocks read from TMEM per wait
constexpr int kUTmemCols = 2 * kUMaxCb * kURows;   // two tiles of up to 8 blocks x 16 columns
constexpr long long kUSpin = 1LL << 26;
constexpr int kUMaxRed = 1024;
// Room left on the SM for one CTA of the sampled chain's cluster kernel (256 threads x 128
// registers, ~40 KB of shared memory), which runs beside this pass: registers are split among the
// SM's four schedulers, three of this kernel's eleven warps share one, so 80 registers a thread.
constexpr int kUMaxRegs = 80;
constexpr int kUSmemLimit = 184 * 1024;            // dynamic shared memory of this pass

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mb_try(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mb_wait(unsigned bar, unsigned parity) {
  for (long long i = 0; i < kUSpin; ++i)
    if (mb_try(bar, parity)) return true;
  return false;
}
// K-major, no-swizzle operand block: row m (0..127), byte b (0..31) of its K slice.
__device__ __forceinline__ unsigned op_off(int m, int b) {
  return (unsigned)((m >> 3) * 256 + (b >> 4) * 128 + (m & 7) * 16 + (b & 15));
}
// tcgen05 shared-memory matrix descriptor: start address, LBO = 128 B between the two K halves of
// a core-matrix row, SBO = 256 B between 8-row groups, version 1, no swizzle.
__device__ __forceinline__ unsigned long long op_desc(unsigned addr) {
  return (unsigned long long)((addr & 0x3FFFF) >> 4) | ((unsigned long long)(128 >> 4) << 16) |
         ((unsigned long long)(256 >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ unsigned bf16x2(float lo_elem, float hi_elem) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo_elem, hi_elem);
  return *reinterpret_cast<unsigned*>(&v);
}
__device__ __forceinline__ float bf_hi(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ unsigned tf32_bits(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// The 32-byte K slice of one operand row from its R values v[0..R-1] (R a compile-time rank, so
// the slot arithmetic folds away and nothing spills to local memory).
//   BF16 (16 elements): A side [hi, hi, lo, 0], B side [hi, lo, hi, 0] (R each, zero padded)
//   TF32 (8 elements):  v[0..R-1], zero padded
template <int KIND, int R>
__device__ __forceinline__ void op_row_r(const float* v, bool a_side, unsigned w[8]) {
  if (KIND == 1) {
#pragma unroll
    for (int k = 0; k < 8; ++k) w[k] = (k < R) ? tf32_bits(v[k]) : 0u;
  } else {
    float hi[R], lo[R];
#pragma unroll
    for (int c = 0; c < R; ++c) {
      hi[c] = bf_hi(v[c]);
      lo[c] = v[c] - hi[c];
    }
    float e[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      float x = 0.f;
      if (k < R) x = hi[k];
      else if (k < 2 * R) x = a_side ? hi[k - R] : lo[k - R];
      else if (k < 3 * R) x = a_side ? lo[k - 2 * R] : hi[k - 2 * R];
      e[k] = x;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) w[k] = bf16x2(e[2 * k], e[2 * k + 1]);
  }
}
template <int KIND>
__device__ __forceinline__ void op_row(const float* v, int r, bool a_side, unsigned w[8]) {
  switch (r) {
    case 1: op_row_r<KIND, 1>(v, a_side, w); break;
    case 2: op_row_r<KIND, 2>(v, a_side, w); break;
    case 3: op_row_r<KIND, 3>(v, a_side, w); break;
    case 4: op_row_r<KIND, 4>(v, a_side, w); break;
    case 5: op_row_r<KIND, 5>(v, a_side, w); break;
    case 6: op_row_r<KIND, 6>(v, a_side, w); break;
    case 7: op_row_r<KIND, 7>(v, a_side, w); break;
    default: op_row_r<KIND, 8>(v, a_side, w); break;
  }
}

// One element of the epilogue: D = X - L in place of X (the stage), kept when |D| > zeta, with
// the residual, kept-count and band-count sums.
__device__ __forceinline__ float ht1v(float x, unsigned lbits, float zf, float band, float& res, unsigned& nnz,
                                     unsigned& inb) {
  const float dl = x - __uint_as_float(lbits);
  const float ad = fabsf(dl);
  const bool keep = ad > zf;
  res = keep ? res : fmaf(dl, dl, res);
  nnz += keep ? 1u : 0u;
  inb += (fabsf(ad - zf) <= band) ? 1u : 0u;
  return keep ? dl : 0.f;
}
__device__ __forceinline__ void ht1(float* p, unsigned lbits, float zf, float band, float& res, unsigned& nnz,
                                    unsigned& inb) {
  *p = ht1v(*p, lbits, zf, band, res, nnz, inb);
}
// A warp is done reading a TMEM accumulator: order its loads before the arrive on `bar`.
__device__ __forceinline__ void release_acc(unsigned long long* bar, int lane) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncwarp();
  if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}

// Starts the TMEM loads of blocks cb0 .. cb0 + kUGroup - 1 (those below nq): 8 accumulator columns
// (rows of X) of this warp's 32 lanes (columns of X) each. Completed by tcgen05.wait::ld.
__device__ __forceinline__ void tmem_group(unsigned tq, int cb0, int nq, unsigned (&l)[kUGroup][kUHalf]) {
#pragma unroll
  for (int c = 0; c < kUGroup; ++c)
    if (cb0 + c < nq)
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(l[c][0]), "=r"(l[c][1]), "=r"(l[c][2]), "=r"(l[c][3]), "=r"(l[c][4]), "=r"(l[c][5]),
                     "=r"(l[c][6]), "=r"(l[c][7])
                   : "r"(tq + (unsigned)((cb0 + c) * kURows)));
}

// The repeated last block (index cb): its 8 accumulator columns of this warp are loaded as for a
// full block (completed by tcgen05.wait::ld); tail_pick then keeps the rows of the half tile
// that lane quarter tk's copy handles, 2 tk, 2 tk + 1 (4 copies) or 4 tk .. 4 tk + 3 (2 copies).
__device__ __forceinline__ void tail_load8(unsigned tq, int cb, unsigned (&w)[kUHalf]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
               : "r"(tq + (unsigned)(cb * kURows)));
}
__device__ __forceinline__ void tail_pick(const unsigned (&w)[kUHalf], int trep, int tk, unsigned (&v)[4]) {
  if (trep == 4) {
    v[0] = tk == 0 ? w[0] : (tk == 1 ? w[2] : (tk == 2 ? w[4] : w[6]));
    v[1] = tk == 0 ? w[1] : (tk == 1 ? w[3] : (tk == 2 ? w[5] : w[7]));
    v[2] = v[3] = 0u;
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = tk == 0 ? w[e] : w[4 + e];
  }
}

__device__ __forceinline__ double block_sum_u(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
  return t;
}

template <int KIND>
__global__ void __maxnreg__(kUMaxRegs) k_dense_umma(Geom g, Bufs b, int nstages) {
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ unsigned long long xfull[kUMaxStages], xempty[kUMaxStages], sdone[kUMaxStages], tfull[2], tempty[2];
  __shared__ unsigned tbase;
  __shared__ volatile int ep_abort, prod_abort, mma_abort, st_abort;  // set to 1 only
  __shared__ int n_issued[kUMaxStages], n_mma[2];
  __shared__ double sh[kUThreads / 32];
  TL_BEGIN();
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
  const int dn = (int)g.d[g.n - 1];
  const long long rows = g.rowsT;
  const int ncb = (dn + kUCols - 1) / kUCols;
  const int stage_f = kUHalf * dn;                              // floats per ring stage
  float* ring = reinterpret_cast<float*>(dsm);
  unsigned char* aop = dsm + (size_t)nstages * stage_f * 4;     // ncb x 4 KB (B_n blocks)
  unsigned char* bop = aop + ncb * kUOpBytesA;                  // 2 x 512 B (T rows of a tile)
  const long long ntiles = (rows + kURows - 1) / kURows;
  const long long u0 = ntiles * blockIdx.x / gridDim.x, u1 = ntiles * (blockIdx.x + 1) / gridDim.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // Last column block: its w = d_n - 128 (ncb - 1) columns are repeated trep = 4 (w <= 32) or
  // 2 (w <= 64) times down the 128 TMEM lanes, so every lane quarter holds a copy and the four
  // quarters' warps split its rows (trep = 1: one copy, as the other blocks). Without the copies
  // the warps of lane quarter 0 alone would hold a narrow last block (at d_n = 800, 7 blocks
  // against 6 for the others).
  const int wtail = dn - (ncb - 1) * kUCols;
  const int trep = wtail <= 32 ? 4 : (wtail <= 64 ? 2 : 1);
  const int tspan = kUCols / trep;  // lanes per copy
  // A operand: row m of column block cb is B_n(cb * 128 + m, :), of the last block
  // B_n(cb * 128 + m mod tspan, :) (zero beyond d_n)
  for (int e = tid; e < ncb * kUCols; e += kUThreads) {
    const int cb = e / kUCols, m = e % kUCols;
    const int col = cb * kUCols + (cb == ncb - 1 ? m % tspan : m);
    float v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = (col < dn && c < rn) ? __ldg(Bn + (size_t)col * rn + c) : 0.f;
    unsigned w[8];
    op_row<KIND>(v, rn, true, w);
    unsigned char* blk = aop + cb * kUOpBytesA;
    *reinterpret_cast<uint4*>(blk + op_off(m, 0)) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4*>(blk + op_off(m, 16)) = make_uint4(w[4], w[5], w[6], w[7]);
  }
  if (tid == 0) {
    ep_abort = prod_abort = mma_abort = st_abort = 0;
    for (int s = 0; s < kUMaxStages; ++s) {
      n_issued[s] = 0;
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&xfull[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&xempty[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&sdone[s])), "r"(kUEpiWarps / 2) : "memory");
    }
    for (int a = 0; a < 2; ++a) {
      n_mma[a] = 0;
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&tfull[a])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&tempty[a])), "r"(kUEpiWarps) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tbase)),
                 "r"(kUTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // A operand -> async proxy
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tbase;

  float res = 0.f;
  unsigned nnz = 0u, inb = 0u;

  if (warp == kUEpiWarps) {
    // ---------------- producer: 1-D bulk loads of half tiles j = 2 (u - u0) + h, in order
    if (lane == 0) {
      const long long nj = 2 * (u1 - u0);
      for (long long j = 0; j < nj; ++j) {
        const int s = (int)(j % nstages);
        if (ep_abort || mma_abort || st_abort) break;
        if (j >= nstages && !mb_wait(su32(&xempty[s]), (unsigned)(((j / nstages) - 1) & 1))) {
          prod_abort = 1;
          break;
        }
        const long long r0 = (u0 + (j >> 1)) * kURows + (j & 1) * kUHalf;
        const long long nr = r0 >= rows ? 0 : (r0 + kUHalf <= rows ? kUHalf : rows - r0);
        const unsigned bar = su32(&xfull[s]);
        if (nr == 0) {  // empty second half of a ragged last tile: complete the phase
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
        } else {
          const unsigned bytes = (unsigned)(nr * dn * 4);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  su32(ring + (size_t)s * stage_f)),
              "l"(X + r0 * dn), "r"(bytes), "r"(bar)
              : "memory");
        }
        ++n_issued[s];
      }
    }
  } else if (warp == kUEpiWarps + 1) {
    // ---------------- MMA warp: B operand (the tile's 16 rows of T), one MMA per column block
    const unsigned idesc = (1u << 4) | ((KIND == 1 ? 2u : 1u) << 7) | ((KIND == 1 ? 2u : 1u) << 10) |
                           ((unsigned)(kURows >> 3) << 17) | ((unsigned)(kUCols >> 4) << 24);
    for (long long u = u0; u < u1; ++u) {
      const int i = (int)(u - u0), a = i & 1;
      // this tile's rows of T, loaded before the wait so their latency overlaps it
      const long long grow = u * kURows + (lane & (kURows - 1));
      float v[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) v[c] = (grow < rows && c < rn) ? __ldg(T + grow * rn + c) : 0.f;
      int stop = 0;  // decided by lane 0, broadcast: the warp leaves the loop together
      if (lane == 0) {
        const bool ok = (i < 2) || mb_wait(su32(&tempty[a]), (unsigned)(((i >> 1) - 1) & 1));
        if (!ok) mma_abort = 1;
        stop = (!ok || ep_abort) ? 1 : 0;
      }
      if (__shfl_sync(0xffffffffu, stop, 0)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      unsigned char* bb = bop + a * kUOpBytesB;
      if (lane < kURows) {  // the MMAs that read this buffer (two tiles ago) have completed
        unsigned w[8];
        op_row<KIND>(v, rn, false, w);
        *reinterpret_cast<uint4*>(bb + op_off(lane, 0)) = make_uint4(w[0], w[1], w[2], w[3]);
        *reinterpret_cast<uint4*>(bb + op_off(lane, 16)) = make_uint4(w[4], w[5], w[6], w[7]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        const unsigned long long bd = op_desc(su32(bb));
        for (int cb = 0; cb < ncb; ++cb) {
          const unsigned long long ad = op_desc(su32(aop + cb * kUOpBytesA));
          const unsigned dt = tmem + (unsigned)(a * (kUTmemCols / 2) + cb * kURows);
          if (KIND == 1)
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
                "l"(ad), "l"(bd), "r"(idesc), "r"(0)
                : "memory");
          else
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
                "l"(ad), "l"(bd), "r"(idesc), "r"(0)
                : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         su32(&tfull[a]))
                     : "memory");
        ++n_mma[a];
      }
      __syncwarp();
    }
  } else if (warp == kUEpiWarps + 2) {
    // ---------------- store warp: half tiles in order, each once its four epilogue warps are done
    if (lane == 0) {
      const long long nj = 2 * (u1 - u0);
      for (long long j = 0; j < nj; ++j) {
        const int s = (int)(j % nstages);
        if (!mb_wait(su32(&sdone[s]), (unsigned)((j / nstages) & 1))) {
          st_abort = 1;
          break;
        }
        const long long r0 = (u0 + (j >> 1)) * kURows + (j & 1) * kUHalf;
        const long long nr = r0 >= rows ? 0 : (r0 + kUHalf <= rows ? kUHalf : rows - r0);
        if (nr > 0)
          asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(S + r0 * dn),
                       "r"(su32(ring + (size_t)s * stage_f)), "r"((unsigned)(nr * dn * 4))
                       : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        if (j >= 1) {  // the previous half tile's store has read its stage: release it
          asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&xempty[(j - 1) % nstages]))
                       : "memory");
        }
      }
      asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // S is in memory
    }
  } else {
    // ---------------- epilogue: warpgroup h on rows 8h..8h+7 of each tile (its half stage)
    const int q = warp & 3;  // TMEM lane quarter: columns 32q.. of every block
    const int h = warp >> 2;
    // blocks handled in the group loop: those with columns in this quarter, less the repeated
    // last block
    const int nfull = trep > 1 ? ncb - 1 : (dn - q * 32 + kUCols - 1) / kUCols;
    // in the repeated last block: this lane's column and the rows (of the half tile) of its copy
    const int tcol = (ncb - 1) * kUCols + ((q * 32 + lane) % tspan);
    const int tk = (q * 32) / tspan;
    for (long long u = u0; u < u1; ++u) {
      const int i = (int)(u - u0), a = i & 1;
      const long long j = 2 * (long long)i + h;
      const int s = (int)(j % nstages);
      const long long r0 = u * kURows + h * kUHalf;
      const int nr = (int)(r0 >= rows ? 0 : (r0 + kUHalf <= rows ? kUHalf : rows - r0));
      const bool ok_t = mb_wait(su32(&tfull[a]), (unsigned)((i >> 1) & 1));
      const bool ok_x = ok_t && mb_wait(su32(&xfull[s]), (unsigned)((j / nstages) & 1));
      if (!__all_sync(0xffffffffu, ok_t && ok_x)) {  // the warp leaves together
        if (lane == 0) ep_abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // this warp's 8 accumulator columns of each block, kUGroup blocks per wait; the accumulator
      // goes back to the MMA warp after the last loads. The repeated last block is loaded and
      // handled after the loop, so its code exists once.
      const unsigned tq = tmem + ((unsigned)(q * 32) << 16) + (unsigned)(a * (kUTmemCols / 2) + h * kUHalf);
      float* stg = ring + (size_t)s * stage_f;
      bool freed = false;
#pragma unroll
      for (int g0 = 0; g0 < kUMaxCb; g0 += kUGroup) {
        if (g0 >= nfull) break;  // warp-uniform
        unsigned l[kUGroup][kUHalf];
        tmem_group(tq, g0, nfull, l);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (trep == 1 && g0 + kUGroup >= nfull) {
          release_acc(&tempty[a], lane);
          freed = true;
        }
        if (nr == kUHalf) {
          // the group's X values first, then S: written this way the loads are not ordered after
          // the stores (whose addresses, a runtime stride apart, the compiler cannot tell apart)
          float xv[kUGroup][kUHalf];
#pragma unroll
          for (int c = 0; c < kUGroup; ++c) {
            const int col = (g0 + c) * kUCols + q * 32 + lane;
            if (g0 + c < nfull && col < dn) {
#pragma unroll
              for (int r = 0; r < kUHalf; ++r) xv[c][r] = stg[col + r * dn];
            }
          }
#pragma unroll
          for (int c = 0; c < kUGroup; ++c) {
            const int col = (g0 + c) * kUCols + q * 32 + lane;
            if (g0 + c < nfull && col < dn) {
#pragma unroll
              for (int r = 0; r < kUHalf; ++r)
                stg[col + r * dn] = ht1v(xv[c][r], l[c][r], zf, band, res, nnz, inb);
            }
          }
        } else {
#pragma unroll
          for (int c = 0; c < kUGroup; ++c) {
            const int col = (g0 + c) * kUCols + q * 32 + lane;
            if (g0 + c < nfull && col < dn) {
              float* p = stg + col;
#pragma unroll
              for (int r = 0; r < kUHalf; ++r)
                if (r < nr) ht1(p + r * dn, l[c][r], zf, band, res, nnz, inb);
            }
          }
        }
      }
      if (trep > 1) {
        unsigned tw[kUHalf], tv[4];  // the repeated last block: loaded, and this quarter's rows
        tail_load8(tq, ncb - 1, tw);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        tail_pick(tw, trep, tk, tv);
        release_acc(&tempty[a], lane);
        freed = true;
        if (tcol < dn) {
          float* p = stg + tcol;
          const int rb = (trep == 4 ? 2 : 4) * tk, cnt = trep == 4 ? 2 : 4;
          float xt[4];
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (e < cnt && rb + e < nr) xt[e] = p[(rb + e) * dn];
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (e < cnt && rb + e < nr) p[(rb + e) * dn] = ht1v(xt[e], tv[e], zf, band, res, nnz, inb);
        }
      }
      if (!freed) release_acc(&tempty[a], lane);  // no column of this quarter
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // S half tile -> bulk store
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&sdone[s])) : "memory");
    }
  }
  __syncthreads();
  if ((ep_abort || prod_abort || mma_abort || st_abort) && tid == 0) {
    // drain: every bulk load and MMA this CTA issued completes before its shared and tensor
    // memory are released (at most one outstanding per stage and per accumulator; waiting on a
    // completed phase returns at once)
    for (int s = 0; s < nstages; ++s)
      if (n_issued[s] > 0) mb_wait(su32(&xfull[s]), (unsigned)((n_issued[s] - 1) & 1));
    for (int a = 0; a < 2; ++a)
      if (n_mma[a] > 0) mb_wait(su32(&tfull[a]), (unsigned)((n_mma[a] - 1) & 1));
    atomicExch(&b.st->err, -5);  // RTCUR_ETIMEOUT
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kUTmemCols) : "memory");
  }
  // reductions: residual, nnz, band count (the producer and MMA warps add zeros)
  double* part = b.red + (size_t)TK_DENSE * kUMaxRed * RT_RED_SLOTS;
  double t0 = block_sum_u((double)res, sh);
  if (tid == 0) part[blockIdx.x * RT_RED_SLOTS + 0] = t0;
  t0 = block_sum_u((double)nnz, sh);
  if (tid == 0) part[blockIdx.x * RT_RED_SLOTS + 1] = t0;
  t0 = block_sum_u((double)inb, sh);
  if (tid == 0) part[blockIdx.x * RT_RED_SLOTS + 2] = t0;
  if (last_block_arrive(b.ticket + TK_DENSE)) {
    State* w = b.st;
    for (int slot = 0; slot < 3; ++slot) {
      double acc = 0.0;
      for (unsigned i2 = threadIdx.x; i2 < gridDim.x; i2 += blockDim.x) acc += part[i2 * RT_RED_SLOTS + slot];
      acc = block_sum_u(acc, sh);
      if (threadIdx.x == 0) {
        if (slot == 0) w->resid_f = acc;
        if (slot == 1) w->nnz_f = (long long)acc;
        if (slot == 2) w->inband_f = (long long)acc;
      }
    }
    if (threadIdx.x == 0) b.ticket[TK_DENSE] = 0u;
  }
  TL_END(1);
}

// Ring stages (8-row halves) that fit beside the operands; 0: the form does not apply.
int umma_stages(const Geom& g, int kind) {
  const long long dn = g.d[g.n - 1];
  if (dn % 4 != 0 || dn > (long long)kUMaxCb * kUCols) return 0;
  if (kind == 0 ? (3 * g.rlast > 16) : (g.rlast > 8)) return 0;
  if (g.rowsT >= (1LL << 31)) return 0;
  const int ncb = (int)((dn + kUCols - 1) / kUCols);
  const long long fixed = (long long)ncb * kUOpBytesA + 2 * kUOpBytesB;
  const long long stage = (long long)kUHalf * dn * 4;
  long long n = (kUSmemLimit - fixed) / stage;
  if (n > kUMaxStages) n = kUMaxStages;
  // four stages at least: with three, one warpgroup can reach a stage whose previous load (a half
  // tile of the other warpgroup) has not completed, and the parity wait on it would pass early
  return n >= 4 ? (int)n : 0;
}

}  // namespace

size_t umma_smem(const Geom& g, int kind) {
  const int ns = umma_stages(g, kind);
  if (!ns) return 0;
  const long long dn = g.d[g.n - 1];
  const int ncb = (int)((dn + kUCols - 1) / kUCols);
  return (size_t)ns * kUHalf * dn * 4 + (size_t)ncb * kUOpBytesA + 2 * kUOpBytesB;
}

cudaError_t prepare_umma(const Geom& g, int kind) {
  const size_t smem = umma_smem(g, kind);
  if (!smem) return cudaSuccess;
  const void* f = kind == 0 ? (const void*)k_dense_umma<0> : (const void*)k_dense_umma<1>;
  cudaError_t e = raise_smem_limit(f, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                                 cudaSharedmemCarveoutMaxShared);
  return e;
}

cudaError_t launch_umma(const Geom& g, const Bufs& b, int kind, cudaStream_t s) {
  const size_t smem = umma_smem(g, kind);
  if (!smem) return cudaErrorNotSupported;
  const int ns = umma_stages(g, kind);
  const long long ntiles = (g.rowsT + kURows - 1) / kURows;
  const int ctas = g.dense_ctas > 0 ? g.dense_ctas : 148;
  const int grid = (int)(ntiles < ctas ? ntiles : ctas);
  if (kind == 0)
    k_dense_umma<0><<<grid, kUThreads, smem, s>>>(g, b, ns);
  else
    k_dense_umma<1><<<grid, kUThreads, smem, s>>>(g, b, ns);
  return cudaGetLastError();
}
