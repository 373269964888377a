// Tensor-core forms of the dense fused pass on the 5th-generation tensor cores (tcgen05):
// S^(k+1) = HT_{zeta^(k+1)}(X - L^(k)) over the whole tensor (Step (I) of Algorithm 1, Eq. (HT)),
// with the last mode product L = T B_n^T (T = G x_1 B_1 ... x_{n-1} B_{n-1}, Eq. (L=CUR) in
// Tucker form) computed by tcgen05.mma into tensor memory.
//
// Work unit: a tile of 128 rows of X (rows of d_n contiguous floats) by 64 columns. Each CTA
// (one per SM, persistent) takes a contiguous range of tiles, row tile outer, and runs three
// warp roles:
//   * producer warp: streams X tiles into a 5-stage shared-memory ring with 2-D TMA loads (two
//     128 x 32 boxes per tile, 128-byte swizzle) completed on mbarriers;
//   * MMA warp: writes the A operand (the tile's 128 rows of T, K-major, rebuilt when the row tile
//     changes, double-buffered) and issues one tcgen05.mma (M = 128, N = 64) per tile into one of
//     two 64-column TMEM accumulators, committed to an mbarrier; B (all of B_n, K-major, one
//     64-row block per column block) is built once per launch;
//   * two epilogue warpgroups on alternating tiles, each with its own accumulator: tcgen05.ld
//     (warp w owns TMEM lanes 32(w%4).., i.e. tile rows, one row per thread), X from the
//     swizzled stage (the 128-byte swizzle makes one row per thread conflict-free), threshold, S
//     written in place and stored back with 2-D TMA stores; a stage is released when its store
//     has read it, one tile of the warpgroup later, so stores overlap the next tiles. The
//     residual / nnz / band sums are fused in.
// Forms (FP32 accumulation in both):
//   BF16: kind::f16 with BF16 operands split x = hi + lo, the three significant products
//         T_hi B_hi + T_hi B_lo + T_lo B_hi packed along K = 16 (3 r_n <= 15); the dropped
//         T_lo B_lo term is ~2^-16 relative.
//   TF32: kind::tf32, K = 8 >= r_n, operands rounded to TF32 (10-bit mantissa).
// Every mbarrier wait is bounded; on expiry the kernel records RTCUR_ETIMEOUT, waits (bounded) for
// its own copies and MMA in flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "rtcur_internal.cuh"

namespace {

constexpr int kUEpiWarps = 8;        // warps 0-7: epilogue (two warpgroups on alternating tiles)
constexpr int kUThreads = 32 * (kUEpiWarps + 2);  // + warp 8: TMA producer, warp 9: MMA
constexpr int kURows = 128;          // M of the MMA, rows per tile
constexpr int kUCols = 64;           // N of the MMA, columns per tile
constexpr int kUBox = 32;            // columns per TMA box (128 bytes: the swizzle span)
constexpr int kUStages = 5;
constexpr int kUStageBytes = kURows * kUCols * 4;  // 32 KB
constexpr int kUBoxBytes = kURows * kUBox * 4;     // 16 KB
constexpr int kUOpBytes = kURows * 32;             // A: 128 rows x 32 bytes of K
constexpr int kUOpBytesB = kUCols * 32;            // B: 64 rows x 32 bytes of K per column block
constexpr int kUMaxCb = 16;                        // column blocks held in shared memory (d_n <= 1024)
constexpr long long kUSpin = 1LL << 26;
constexpr int kUMaxRed = 1024;

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
// AND of a predicate over the 128 threads of an epilogue warpgroup (named barrier `id`): a
// decision every thread of the warpgroup takes together.
__device__ __forceinline__ bool wg_all(bool v, int id) {
  unsigned out;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\tbar.red.and.pred po, %2, 128, pi;\n\t"
      "selp.u32 %0, 1, 0, po;\n\t}"
      : "=r"(out)
      : "r"(v ? 1u : 0u), "r"(id)
      : "memory");
  return out != 0;
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

__device__ __forceinline__ void ht4(float4 x, const unsigned* l, float zf, float band, bool valid_row,
                                    int col0, long long dn, float4& s, float& res, unsigned& nnz,
                                    unsigned& inb) {
  const float xs[4] = {x.x, x.y, x.z, x.w};
  float ss[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float dl = xs[e] - __uint_as_float(l[e]);
    const float ad = fabsf(dl);
    const bool keep = ad > zf;
    ss[e] = keep ? dl : 0.f;
    if (valid_row && col0 + e < dn) {
      res = keep ? res : fmaf(dl, dl, res);
      nnz += keep ? 1u : 0u;
      inb += (fabsf(ad - zf) <= band) ? 1u : 0u;
    }
  }
  s = make_float4(ss[0], ss[1], ss[2], ss[3]);
}

// Same without the bounds test: every element of an interior tile is in the tensor.
__device__ __forceinline__ void ht4_full(float4 x, const unsigned* l, float zf, float band, float4& s,
                                         float& res, unsigned& nnz, unsigned& inb) {
  const float xs[4] = {x.x, x.y, x.z, x.w};
  float ss[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float dl = xs[e] - __uint_as_float(l[e]);
    const float ad = fabsf(dl);
    const bool keep = ad > zf;
    ss[e] = keep ? dl : 0.f;
    res = keep ? res : fmaf(dl, dl, res);
    nnz += keep ? 1u : 0u;
    inb += (fabsf(ad - zf) <= band) ? 1u : 0u;
  }
  s = make_float4(ss[0], ss[1], ss[2], ss[3]);
}

// 32 consecutive accumulator columns of this thread's TMEM lane (32x32b shape, x32)
__device__ __forceinline__ void tmem_ld32(unsigned taddr, unsigned* l) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(l[0]), "=r"(l[1]), "=r"(l[2]), "=r"(l[3]), "=r"(l[4]), "=r"(l[5]), "=r"(l[6]), "=r"(l[7]),
        "=r"(l[8]), "=r"(l[9]), "=r"(l[10]), "=r"(l[11]), "=r"(l[12]), "=r"(l[13]), "=r"(l[14]), "=r"(l[15]),
        "=r"(l[16]), "=r"(l[17]), "=r"(l[18]), "=r"(l[19]), "=r"(l[20]), "=r"(l[21]), "=r"(l[22]), "=r"(l[23]),
        "=r"(l[24]), "=r"(l[25]), "=r"(l[26]), "=r"(l[27]), "=r"(l[28]), "=r"(l[29]), "=r"(l[30]), "=r"(l[31])
      : "r"(taddr));
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
__global__ void __launch_bounds__(kUThreads, 1) k_dense_umma(Geom g, Bufs b) {
  extern __shared__ unsigned char dsm_raw[];
  __shared__ unsigned long long xfull[kUStages], xempty[kUStages], tfull[2], tempty[2];
  __shared__ unsigned tbase;
  __shared__ volatile int ep_abort, prod_abort, mma_abort;  // each written by one thread only
  __shared__ int n_issued[kUStages], n_seen[kUStages], n_mma[2], n_mma_seen[2];
  __shared__ double sh[kUThreads / 32];
  TL_BEGIN();
  // 1024-byte aligned base (the 128-byte swizzle atoms of TMA need it)
  const unsigned raw = su32(dsm_raw);
  unsigned char* dsm = dsm_raw + (((raw + 1023u) & ~1023u) - raw);
  unsigned char* stage0 = dsm;                               // kUStages x 32 KB
  unsigned char* bop = dsm + kUStages * kUStageBytes;        // ncb x 2 KB
  const State* st = b.st;
  const int cur = st->k & 1;
  const double zeta = g.gamma * st->zeta;
  const float zf = (float)zeta;
  const float band = (float)(g.inband * zeta);
  const float* __restrict__ T = b.T[cur];
  const float* __restrict__ Bn = b.B[cur] + g.offB[g.n - 1];
  const int rn = g.rlast;
  const long long dn = g.d[g.n - 1];
  const long long rows = g.rowsT;
  const int ncb = (int)((dn + kUCols - 1) / kUCols);
  unsigned char* aop = bop + ncb * kUOpBytesB;               // 2 x 4 KB
  const long long nrt = (rows + kURows - 1) / kURows;
  const long long U = nrt * ncb;
  const long long u0 = U * blockIdx.x / gridDim.x, u1 = U * (blockIdx.x + 1) / gridDim.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const unsigned long long mapX = reinterpret_cast<unsigned long long>(b.tmap);
  const unsigned long long mapS = mapX + 128;

  // B operand: row n of column block cb is B_n(cb*64 + n, :) (zero beyond d_n)
  for (int e = tid; e < ncb * kUCols; e += kUThreads) {
    const int cb = e / kUCols, n = e % kUCols;
    const long long col = (long long)cb * kUCols + n;
    float v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = (col < dn && c < rn) ? __ldg(Bn + col * rn + c) : 0.f;
    unsigned w[8];
    op_row<KIND>(v, rn, false, w);
    unsigned char* blk = bop + cb * kUOpBytesB;
    *reinterpret_cast<uint4*>(blk + op_off(n, 0)) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4*>(blk + op_off(n, 16)) = make_uint4(w[4], w[5], w[6], w[7]);
  }
  if (tid == 0) {
    ep_abort = prod_abort = mma_abort = 0;
    for (int s = 0; s < kUStages; ++s) {
      n_issued[s] = n_seen[s] = 0;
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&xfull[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&xempty[s])) : "memory");
    }
    for (int a = 0; a < 2; ++a) {
      n_mma[a] = n_mma_seen[a] = 0;
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&tfull[a])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&tempty[a])), "r"(kUEpiWarps / 2) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // the maps were written by host copies: order them before the TMA proxy reads them
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(mapX) : "memory");
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(mapS) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(su32(&tbase))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // B operand -> async proxy
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tbase;

  float res = 0.f;
  unsigned nnz = 0u, inb = 0u;

  if (warp == kUEpiWarps) {
    // ---------------- producer: TMA loads of X tiles into the stage ring
    if (lane == 0) {
      for (long long u = u0; u < u1; ++u) {
        const int i = (int)(u - u0), s = i % kUStages;
        if (ep_abort || mma_abort) break;
        if (i >= kUStages && !mb_wait(su32(&xempty[s]), (unsigned)(((i / kUStages) - 1) & 1))) {
          prod_abort = 1;
          break;
        }
        const long long rt = u / ncb;
        const int cb = (int)(u % ncb);
        const int c0 = cb * kUCols;
        int nbox = (int)((dn - c0 + kUBox - 1) / kUBox);
        if (nbox > kUCols / kUBox) nbox = kUCols / kUBox;
        const unsigned bar = su32(&xfull[s]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"((unsigned)(nbox * kUBoxBytes))
                     : "memory");
        for (int j = 0; j < nbox; ++j) {
          const unsigned dst = su32(stage0 + s * kUStageBytes + j * kUBoxBytes);
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
                  dst),
              "l"(mapX), "r"(c0 + j * kUBox), "r"((int)(rt * kURows)), "r"(bar)
              : "memory");
        }
        ++n_issued[s];
      }
    }
  } else if (warp == kUEpiWarps + 1) {
    // ---------------- MMA warp: A operand (the tile's rows of T) and one MMA per tile
    long long prev_rt = -1;
    int abuf = 1;
    for (long long u = u0; u < u1; ++u) {
      const int i = (int)(u - u0), a = i & 1;
      int stop = 0;  // decided by lane 0, broadcast: the warp leaves the loop together
      if (lane == 0) {
        const bool ok = (i < 2) || mb_wait(su32(&tempty[a]), (unsigned)(((i >> 1) - 1) & 1));
        if (!ok) mma_abort = 1;
        stop = (!ok || ep_abort) ? 1 : 0;
      }
      if (__shfl_sync(0xffffffffu, stop, 0)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const long long rt = u / ncb;
      const int cb = (int)(u % ncb);
      if (rt != prev_rt) {  // every MMA that read this A buffer has completed (see tempty)
        abuf ^= 1;
        unsigned char* ab = aop + abuf * kUOpBytes;
        for (int r = lane; r < kURows; r += 32) {
          const long long grow = rt * kURows + r;
          float v[8];
#pragma unroll
          for (int c = 0; c < 8; ++c) v[c] = (grow < rows && c < rn) ? __ldg(T + grow * rn + c) : 0.f;
          unsigned w[8];
          op_row<KIND>(v, rn, true, w);
          *reinterpret_cast<uint4*>(ab + op_off(r, 0)) = make_uint4(w[0], w[1], w[2], w[3]);
          *reinterpret_cast<uint4*>(ab + op_off(r, 16)) = make_uint4(w[4], w[5], w[6], w[7]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        prev_rt = rt;
      }
      if (lane == 0) {
        const unsigned long long ad = op_desc(su32(aop + abuf * kUOpBytes));
        const unsigned long long bd = op_desc(su32(bop + cb * kUOpBytesB));
        const unsigned idesc = (1u << 4) | ((KIND == 1 ? 2u : 1u) << 7) | ((KIND == 1 ? 2u : 1u) << 10) |
                               ((unsigned)(kUCols >> 3) << 17) | ((unsigned)(kURows >> 4) << 24);
        const unsigned dt = tmem + (unsigned)(a * kUCols);
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
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         su32(&tfull[a]))
                     : "memory");
        ++n_mma[a];
      }
      __syncwarp();
    }
  } else {
    // ---------------- epilogue: two warpgroups on alternating tiles (warpgroup h takes the
    // tiles i = h, h + 2, ... and accumulator h)
    const int q = warp & 3;                // TMEM lane quarter of this warp
    const int h = warp >> 2;               // warpgroup
    const int r = q * 32 + lane;           // tile row == TMEM lane
    const int et = tid & 127;              // thread within the warpgroup
    const int bar_id = 1 + h;
    for (long long u = u0 + h; u < u1; u += 2) {
      const int i = (int)(u - u0), s = i % kUStages, a = h;
      const long long rt = u / ncb;
      const int cb = (int)(u % ncb);
      const int c0 = cb * kUCols;
      int nbox = (int)((dn - c0 + kUBox - 1) / kUBox);
      if (nbox > kUCols / kUBox) nbox = kUCols / kUBox;
      const long long grow = rt * kURows + r;
      const bool vrow = grow < rows;
      const bool ok_t = mb_wait(su32(&tfull[a]), (unsigned)((i >> 1) & 1));
      const bool ok_x = ok_t && mb_wait(su32(&xfull[s]), (unsigned)((i / kUStages) & 1));
      if (!wg_all(ok_t && ok_x, bar_id)) {  // uniform within the warpgroup
        if (et == 0) {
          if (ok_t) ++n_mma_seen[a];
          if (ok_x) ++n_seen[s];
          ep_abort = 1;
        }
        break;
      }
      if (et == 0) {
        ++n_mma_seen[a];
        ++n_seen[s];
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      unsigned char* stg = stage0 + s * kUStageBytes;
      // both 32-column halves of the accumulator, one wait
      unsigned l[64];
      const unsigned taddr = tmem + ((unsigned)(q * 32) << 16) + (unsigned)(a * kUCols);
      tmem_ld32(taddr, l);
      tmem_ld32(taddr + kUBox, l + 32);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      const bool interior = (rt + 1) * kURows <= rows && c0 + kUCols <= dn;
#pragma unroll
      for (int j = 0; j < kUCols / kUBox; ++j) {
        if (j >= nbox) break;
        unsigned char* rowp = stg + j * kUBoxBytes + r * 128;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          float4* p = reinterpret_cast<float4*>(rowp + ((c ^ (r & 7)) << 4));
          float4 sv;
          if (interior)
            ht4_full(*p, l + 32 * j + 4 * c, zf, band, sv, res, nnz, inb);
          else
            ht4(*p, l + 32 * j + 4 * c, zf, band, vrow, c0 + j * kUBox + 4 * c, dn, sv, res, nnz, inb);
          *p = sv;
        }
      }
      // this warp is done with accumulator a
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&tempty[a])) : "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // S tile -> TMA store
      asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
      if (et == 0) {
        for (int j = 0; j < nbox; ++j) {
          const unsigned src = su32(stg + j * kUBoxBytes);
          asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(mapS),
                       "r"(c0 + j * kUBox), "r"((int)(rt * kURows)), "r"(src)
                       : "memory");
        }
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        if (i >= 2) {  // this warpgroup's previous tile has been read by its store: release its stage
          asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&xempty[(i - 2) % kUStages]))
                       : "memory");
        }
      }
    }
    if (et == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // S is in memory
  }
  __syncthreads();
  if ((ep_abort || prod_abort || mma_abort) && tid == 0) {
    // drain: every TMA load and MMA this CTA issued completes before its shared and tensor
    // memory are released (at most one unconsumed load per stage and one MMA per accumulator)
    for (int s = 0; s < kUStages; ++s)
      if (n_issued[s] > n_seen[s]) mb_wait(su32(&xfull[s]), (unsigned)((n_issued[s] - 1) & 1));
    for (int a = 0; a < 2; ++a)
      if (n_mma[a] > n_mma_seen[a]) mb_wait(su32(&tfull[a]), (unsigned)((n_mma[a] - 1) & 1));
    atomicExch(&b.st->err, -5);  // RTCUR_ETIMEOUT
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
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

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

}  // namespace

size_t umma_smem(const Geom& g, int kind) {
  const long long dn = g.d[g.n - 1];
  if (dn % 4 != 0 || dn > (long long)kUMaxCb * kUCols) return 0;
  if (kind == 0 ? (3 * g.rlast > 16) : (g.rlast > 8)) return 0;
  if (g.rowsT >= (1LL << 31)) return 0;
  const int ncb = (int)((dn + kUCols - 1) / kUCols);
  return 1024 + (size_t)kUStages * kUStageBytes + (size_t)ncb * kUOpBytesB + 2 * (size_t)kUOpBytes;
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
  const long long dn = g.d[g.n - 1];
  const long long units = ((g.rowsT + kURows - 1) / kURows) * ((dn + kUCols - 1) / kUCols);
  const int ctas = g.dense_ctas > 0 ? g.dense_ctas : 144;
  const int grid = (int)(units < ctas ? units : ctas);
  if (kind == 0)
    k_dense_umma<0><<<grid, kUThreads, smem, s>>>(g, b);
  else
    k_dense_umma<1><<<grid, kUThreads, smem, s>>>(g, b);
  return cudaGetLastError();
}

// Host-encoded TMA maps of X (read) and S (written), each the 2-D view rows x d_n of FP32 with
// 128 x 32 boxes and the 128-byte swizzle, written into the 256 bytes at `dst_host` (copied to the
// plan's device buffer by the caller).
cudaError_t encode_umma_maps(const Geom& g, const float* X, float* S, void* dst_host) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  const long long dn = g.d[g.n - 1];
  cuuint64_t gdim[2] = {(cuuint64_t)dn, (cuuint64_t)g.rowsT};
  cuuint64_t gstride[1] = {(cuuint64_t)(dn * 4)};
  cuuint32_t box[2] = {(cuuint32_t)kUBox, (cuuint32_t)kURows};
  cuuint32_t estr[2] = {1, 1};
  CUtensorMap* maps = static_cast<CUtensorMap*>(dst_host);
  const float* ptrs[2] = {X, S};
  for (int k = 0; k < 2; ++k) {
    CUresult r = enc(&maps[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(ptrs[k]), gdim, gstride, box,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}
