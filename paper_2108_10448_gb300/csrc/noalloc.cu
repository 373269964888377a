// rtcur_threshold_dense_noalloc: the dense fused threshold pass for callers that cannot
// allocate device memory.
//
// Some callers must not call cudaMalloc: a serving process whose device memory is owned by a
// pre-reserved pool with a hard budget (a stray allocation either fails or breaks the pool's
// accounting), or a latency-critical caller for which cudaMalloc's possible implicit device
// synchronisation is unacceptable. For them this entry point takes all its scratch (the
// evaluation table T = G x_1 B_1 ... x_{n-1} B_{n-1}, the reduction partials and counters and
// the small device state) from one file-scope device array of kScratchBytes. Every GPU that
// loads the library holds that array until the process exits. The caller passes the inputs
// (X, G, B) and the output S; nothing else is allocated: no cudaMalloc, no cudaFree, no
// allocating library routine.
//
// The array is shared by every call on a device and keeps the last call's contents; the parts
// that must start at zero (the reduction tickets) are cleared at each call, by a one-thread-block
// kernel that also writes the call's state from its arguments (no host staging buffer). Calls
// whose work overlaps on the GPU (different streams, or different host threads) race on the
// array. Device-side errors (a bounded wait of the pass that gave up) are read back only when the
// caller asks for the counts.
//
// Host code cannot use the array's name as a device address (in host code the name is a
// host-side stand-in; a kernel given it would fault or, where the GPU can reach host memory,
// silently use the wrong memory). So the first call on each device, with that device current,
// looks up the array's device address with cudaGetSymbolAddress and caches it; that first call
// on a device should come before any stream capture. Device code may name the array directly.
#include <cstring>
#include <mutex>

#include "../../include/rtcur.h"
#include "rtcur_internal.cuh"

namespace {

constexpr size_t kScratchBytes = 32ull << 20;  // 32 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Resets the call's device state in the scratch: the loop state (k = 0 so that copy 0 holds the
// caller's G and B; zeta as given; the dense counters), the pointers to X and S, and the
// reduction tickets. Everything arrives as kernel arguments, so no host buffer has to outlive the
// call.
__global__ void k_noalloc_init(State* st, SolvePtrs* sp, unsigned* ticket, double zeta,
                               const float* X, float* S) {
  if (threadIdx.x == 0) {
    State h;
    memset(&h, 0, sizeof h);
    h.zeta = zeta;
    h.e = 1.0;
    h.nnz_f = h.inband_f = -1;
    h.resid_f = -1.0;
    *st = h;
    sp->X = X;
    sp->S = S;
  }
  if (threadIdx.x < TK_COUNT) ticket[threadIdx.x] = 0u;
}

}  // namespace

extern "C" RTCUR_API rtcur_status rtcur_threshold_dense_noalloc(
    int32_t n_modes, const int64_t* dims, const int32_t* ranks, const float* G, const float* B,
    const float* X, double zeta, float* S, double* counts, void* stream) {
  if (n_modes < 2 || n_modes > RT_MAXN || !dims || !ranks || !G || !B || !X || !S)
    return RTCUR_EINVAL;
  if (!(zeta >= 0.0) || zeta > 3.0e38) return RTCUR_EINVAL;
  if ((reinterpret_cast<uintptr_t>(X) & 15u) || (reinterpret_cast<uintptr_t>(S) & 15u)) return RTCUR_EINVAL;
  Geom g;
  memset(&g, 0, sizeof g);
  g.n = n_modes;
  g.N = 1;
  long long oB = 0;
  for (int i = 0; i < n_modes; ++i) {
    if (dims[i] < 1 || ranks[i] < 1 || ranks[i] > RT_MAXR) return RTCUR_EINVAL;
    if (g.N > (1LL << 40) / dims[i]) return RTCUR_EINVAL;
    g.d[i] = dims[i];
    g.r[i] = ranks[i];
    g.N *= dims[i];
    g.offB[i] = oB;
    oB += dims[i] * ranks[i];
  }
  g.sumB = oB;
  g.rlast = ranks[n_modes - 1];
  g.rowsT = g.N / dims[n_modes - 1];
  g.nH = (long long)ranks[0] * ranks[n_modes - 1];
  for (int l = 1; l <= n_modes - 2; ++l) g.nH *= dims[l];
  g.gamma = 1.0;  // the pass thresholds at zeta^(k+1) = gamma * zeta: gamma = 1 uses `zeta` as given
  g.inband = 1e-6;
  g.max_iter = 1;
  if (g.rowsT >= (1LL << 32) || dims[n_modes - 1] >= (1LL << 32)) return RTCUR_EINVAL;
  // scratch layout (each piece 256-byte aligned)
  const size_t oState = 0;
  const size_t oPtrs = align256(oState + sizeof(State));
  const size_t oTick = align256(oPtrs + sizeof(SolvePtrs));
  const size_t oRed = align256(oTick + sizeof(unsigned) * TK_COUNT);
  const size_t oH = align256(oRed + sizeof(double) * TK_COUNT * 1024 * RT_RED_SLOTS);
  const size_t oT = align256(oH + sizeof(float) * (size_t)g.nH);
  const size_t need = align256(oT + sizeof(float) * ((size_t)g.rowsT * g.rlast + 4));
  if (need > kScratchBytes) return RTCUR_EINVAL;  // problem larger than the fixed scratch

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RTCUR_ECUDA;
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return RTCUR_ECUDA;
      if (prepare_dense(g) != cudaSuccess) return RTCUR_ECUDA;
      g_scratch_ptr[dev] = ptr;
    } else if (prepare_dense(g) != cudaSuccess) {
      return RTCUR_ECUDA;
    }
    base = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Bufs b;
  memset(&b, 0, sizeof b);
  b.st = reinterpret_cast<State*>(base + oState);
  b.sp = reinterpret_cast<SolvePtrs*>(base + oPtrs);
  b.ticket = reinterpret_cast<unsigned*>(base + oTick);
  b.red = reinterpret_cast<double*>(base + oRed);
  b.H = reinterpret_cast<float*>(base + oH);
  b.T[0] = b.T[1] = reinterpret_cast<float*>(base + oT);
  b.G[0] = b.G[1] = const_cast<float*>(G);
  b.B[0] = b.B[1] = const_cast<float*>(B);
  k_noalloc_init<<<1, 32, 0, s>>>(b.st, b.sp, b.ticket, zeta, X, S);
  if (cudaGetLastError() != cudaSuccess) return RTCUR_ECUDA;
  if (launch_table(g, b, 0, s) != cudaSuccess) return RTCUR_ECUDA;
  if (launch_dense(g, b, RTCUR_FORM_FP32, s) != cudaSuccess) return RTCUR_ECUDA;
  if (counts) {
    State o;
    if (cudaMemcpyAsync(&o, b.st, sizeof o, cudaMemcpyDeviceToHost, s) != cudaSuccess) return RTCUR_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return RTCUR_ECUDA;
    counts[0] = o.resid_f;
    counts[1] = (double)o.nnz_f;
    counts[2] = (double)o.inband_f;
    if (o.err != 0) return (rtcur_status)o.err;
  }
  return RTCUR_OK;
}
