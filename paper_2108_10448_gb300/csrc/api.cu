// Host side of librtcur.so: argument validation, plan workspace, CUDA-graph construction and
// the extern "C" entry points declared in include/rtcur.h.
//
// One RTCUR iteration (Algorithm 1's loop body) is one captured graph with two branches that
// depend only on L^(k):
//   branch A (FULL scope only): the dense fused threshold pass over the whole tensor;
//   branch B: sampled threshold -> Gram -> FP32 Jacobi -> FP64 refinement -> B_i -> core G ->
//             table T -> sampled error e^(k+1).
// They join before the commit kernel, which advances k and zeta and sets the loop condition.
// rtcur_solve launches a graph whose single node is a conditional WHILE over that body, so the
// whole solve runs on the device with one host synchronisation at the end.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rtcur.h"
#include "rtcur_internal.cuh"

struct rtcur_plan;

// Cached graph of a batched solve (kept by the batch's first plan): a WHILE node whose body holds
// one IF node per problem (the problem's iteration, skipped once it has stopped) and a kernel
// that keeps the loop going while any problem continues.
struct BatchGraph {
  std::vector<rtcur_plan*> plans;
  std::vector<unsigned long long> serials;
  cudaGraph_t G = nullptr;
  cudaGraphExec_t X = nullptr;
  State** d_sts = nullptr;
};

struct rtcur_plan {
  unsigned long long serial = 0;  // unique per plan (a batch cache is keyed by these)
  BatchGraph* batch = nullptr;
  Geom g;
  Bufs b;
  rtcur_options opt;
  double zeta0;
  float* S_internal = nullptr;
  float* S_work = nullptr;
  const float* X = nullptr;
  cudaStream_t cap = nullptr, side = nullptr, side2 = nullptr;
  cudaEvent_t evFork = nullptr, evJoin = nullptr, evFork2 = nullptr, evJoin2 = nullptr;
  cudaGraph_t loopG = nullptr, iterG = nullptr;
  cudaGraphExec_t loopX = nullptr, iterX = nullptr;
  BwWork bw;             // adjoint workspace (options.checkpoint > 0)
  std::vector<void*> allocs;
  std::vector<int> pos_host;
  std::string err;
  bool begun = false;
};

namespace {

thread_local std::string g_create_err = "no error";
std::atomic<unsigned long long> g_serial{1};

rtcur_status fail(rtcur_plan* p, rtcur_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (p) p->err = buf; else g_create_err = buf;
  return st;
}

#define CKC(p, call)                                                                     \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(p, RTCUR_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));       \
  } while (0)

template <typename T>
cudaError_t dalloc(rtcur_plan* p, T** ptr, size_t count) {
  void* v = nullptr;
  size_t bytes = count * sizeof(T);
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&v, bytes);
  if (e != cudaSuccess) return e;
  p->allocs.push_back(v);
  *ptr = static_cast<T*>(v);
  return cudaSuccess;
}

cudaError_t capture_body(rtcur_plan* p, cudaStream_t s, unsigned long long handle, int use_handle) {
  const Geom& g = p->g;
  const Bufs& b = p->b;
  cudaError_t e;
  const bool full = (g.scope == RTCUR_SCOPE_FULL);
  if (full) {
    if ((e = cudaEventRecord(p->evFork, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(p->side, p->evFork, 0)) != cudaSuccess) return e;
    if ((e = launch_dense(g, b, p->opt.dense_form, p->side)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(p->evJoin, p->side)) != cudaSuccess) return e;
  }
  if ((e = launch_sample_ht(g, b, s)) != cudaSuccess) return e;
  if ((e = launch_gram(g, b, s)) != cudaSuccess) return e;
  if ((e = launch_refine(g, b, 0, s)) != cudaSuccess) return e;  // warm attempt
  if ((e = launch_jacobi(g, b, s)) != cudaSuccess) return e;
  if ((e = launch_refine(g, b, 1, s)) != cudaSuccess) return e;
  // B_i = C_i Y_i and the core G = R x_i Q_i^T read disjoint inputs and write disjoint buffers:
  // two branches of the graph, joined before the table that needs both
  if ((e = cudaEventRecord(p->evFork2, s)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(p->side2, p->evFork2, 0)) != cudaSuccess) return e;
  if ((e = launch_factor_B(g, b, p->side2)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(p->evJoin2, p->side2)) != cudaSuccess) return e;
  if ((e = launch_core(g, b, s)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(s, p->evJoin2, 0)) != cudaSuccess) return e;
  if ((e = launch_table(g, b, 1, s)) != cudaSuccess) return e;
  if (full && p->opt.dense_form == RTCUR_FORM_FP32_PLAIN && (e = launch_plain_prep(g, b, s)) != cudaSuccess) return e;
  if ((e = launch_sample_err(g, b, s)) != cudaSuccess) return e;
  if (full && (e = cudaStreamWaitEvent(s, p->evJoin, 0)) != cudaSuccess) return e;
  return launch_commit(g, b, handle, use_handle, s);
}

rtcur_status build_graphs(rtcur_plan* p) {
  if (p->iterX) return RTCUR_OK;
  // single-iteration graph (rtcur_iterate)
  CKC(p, cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = capture_body(p, p->cap, 0ull, 0);
  cudaGraph_t gr = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(p->cap, &gr);
  if (e != cudaSuccess) return fail(p, RTCUR_ECUDA, "capturing the iteration: %s", cudaGetErrorString(e));
  if (e2 != cudaSuccess) return fail(p, RTCUR_ECUDA, "ending capture: %s", cudaGetErrorString(e2));
  p->iterG = gr;
  CKC(p, cudaGraphInstantiate(&p->iterX, p->iterG, 0));
  // WHILE-loop graph (rtcur_solve): body = the same iteration, condition set by the commit kernel
  CKC(p, cudaGraphCreate(&p->loopG, 0));
  cudaGraphConditionalHandle h;
  CKC(p, cudaGraphConditionalHandleCreate(&h, p->loopG, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  CKC(p, cudaGraphAddNode(&node, p->loopG, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  CKC(p, cudaStreamBeginCaptureToGraph(p->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  e = capture_body(p, p->cap, (unsigned long long)h, 1);
  e2 = cudaStreamEndCapture(p->cap, &gr);
  if (e != cudaSuccess) return fail(p, RTCUR_ECUDA, "capturing the loop body: %s", cudaGetErrorString(e));
  if (e2 != cudaSuccess) return fail(p, RTCUR_ECUDA, "ending body capture: %s", cudaGetErrorString(e2));
  CKC(p, cudaGraphInstantiate(&p->loopX, p->loopG, 0));
  return RTCUR_OK;
}

void free_batch(BatchGraph* bg) {
  if (!bg) return;
  if (bg->X) cudaGraphExecDestroy(bg->X);
  if (bg->G) cudaGraphDestroy(bg->G);
  if (bg->d_sts) cudaFree(bg->d_sts);
  delete bg;
}

rtcur_status build_batch(rtcur_plan* const* plans, int count, BatchGraph** out) {
  rtcur_plan* p0 = plans[0];
  BatchGraph* bg = new BatchGraph();
  auto bail = [&](cudaError_t e, const char* what) {
    free_batch(bg);
    return fail(p0, RTCUR_ECUDA, "batched graph: %s: %s", what, cudaGetErrorString(e));
  };
  cudaError_t e;
  std::vector<State*> sts(count);
  for (int i = 0; i < count; ++i) {
    bg->plans.push_back(plans[i]);
    bg->serials.push_back(plans[i]->serial);
    sts[i] = plans[i]->b.st;
  }
  if ((e = cudaMalloc(&bg->d_sts, sizeof(State*) * count)) != cudaSuccess) return bail(e, "cudaMalloc");
  if ((e = cudaMemcpy(bg->d_sts, sts.data(), sizeof(State*) * count, cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail(e, "cudaMemcpy");
  if ((e = cudaGraphCreate(&bg->G, 0)) != cudaSuccess) return bail(e, "cudaGraphCreate");
  cudaGraphConditionalHandle hw;
  if ((e = cudaGraphConditionalHandleCreate(&hw, bg->G, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
    return bail(e, "WHILE handle");
  cudaGraphNodeParams wp = {cudaGraphNodeTypeConditional};
  wp.conditional.handle = hw;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wnode;
  if ((e = cudaGraphAddNode(&wnode, bg->G, nullptr, nullptr, 0, &wp)) != cudaSuccess) return bail(e, "WHILE node");
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  std::vector<cudaGraphNode_t> ifs(count);
  for (int i = 0; i < count; ++i) {
    rtcur_plan* p = plans[i];
    cudaGraphConditionalHandle hp;
    if ((e = cudaGraphConditionalHandleCreate(&hp, body, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
      return bail(e, "IF handle");
    cudaGraphNodeParams ip = {cudaGraphNodeTypeConditional};
    ip.conditional.handle = hp;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    if ((e = cudaGraphAddNode(&ifs[i], body, nullptr, nullptr, 0, &ip)) != cudaSuccess) return bail(e, "IF node");
    cudaGraph_t pb = ip.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(p->cap, pb, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return bail(e, "capture begin");
    cudaError_t ec = capture_body(p, p->cap, (unsigned long long)hp, 1);
    cudaGraph_t tmp = nullptr;
    e = cudaStreamEndCapture(p->cap, &tmp);
    if (ec != cudaSuccess) return bail(ec, "capturing a problem's iteration");
    if (e != cudaSuccess) return bail(e, "capture end");
  }
  if ((e = cudaStreamBeginCaptureToGraph(p0->cap, body, ifs.data(), nullptr, count, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
    return bail(e, "capture begin (join)");
  cudaError_t ec = launch_batch_any(bg->d_sts, count, (unsigned long long)hw, p0->cap);
  cudaGraph_t tmp = nullptr;
  e = cudaStreamEndCapture(p0->cap, &tmp);
  if (ec != cudaSuccess) return bail(ec, "join kernel");
  if (e != cudaSuccess) return bail(e, "capture end (join)");
  if ((e = cudaGraphInstantiate(&bg->X, bg->G, 0)) != cudaSuccess) return bail(e, "instantiate");
  *out = bg;
  return RTCUR_OK;
}

rtcur_status check_sets(rtcur_plan* p, const int64_t* idx) {
  const Geom& g = p->g;
  for (int s = 0; s < g.n_sets; ++s) {
    const int64_t* set = idx + (size_t)s * g.set_len;
    for (int i = 0; i < g.n; ++i) {
      long long other = g.N / g.d[i];
      const int64_t* I = set + g.ioff[i];
      const int64_t* J = set + g.joff[i];
      for (int a = 0; a < g.m[i]; ++a) {
        if (I[a] < 0 || I[a] >= g.d[i] || (a > 0 && I[a] <= I[a - 1]))
          return fail(p, RTCUR_EINVAL, "set %d: I_%d must be strictly increasing in [0, %lld)", s, i + 1, g.d[i]);
      }
      for (int a = 0; a < g.q[i]; ++a) {
        if (J[a] < 0 || J[a] >= other || (a > 0 && J[a] <= J[a - 1]))
          return fail(p, RTCUR_EINVAL, "set %d: J_%d must be strictly increasing in [0, %lld)", s, i + 1, other);
      }
    }
  }
  return RTCUR_OK;
}

bool aligned16(const void* ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15u) == 0; }

}  // namespace

extern "C" {

rtcur_status rtcur_create(rtcur_plan** out, int32_t n_modes, const int64_t* dims,
                          const int32_t* ranks, const int32_t* nI, const int32_t* nJ,
                          double zeta0, double gamma, double tol, int32_t max_iter,
                          int32_t variant, const rtcur_options* opt) {
  if (!out) return fail(nullptr, RTCUR_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_modes < 2 || n_modes > RT_MAXN) return fail(nullptr, RTCUR_EINVAL, "n_modes must be in [2, %d]", RT_MAXN);
  if (!dims || !ranks || !nI || !nJ) return fail(nullptr, RTCUR_EINVAL, "dims, ranks, nI and nJ must not be NULL");
  if (!(gamma > 0.0 && gamma < 1.0)) return fail(nullptr, RTCUR_EINVAL, "gamma must be in (0, 1)");
  if (!(tol >= 0.0) || std::isinf(tol)) return fail(nullptr, RTCUR_EINVAL, "tol must be finite and >= 0");
  if (std::isnan(zeta0) || std::isinf(zeta0)) return fail(nullptr, RTCUR_EINVAL, "zeta0 must be finite");
  if (max_iter < 1 || max_iter > 100000) return fail(nullptr, RTCUR_EINVAL, "max_iter must be in [1, 100000]");
  if (variant != RTCUR_VARIANT_F && variant != RTCUR_VARIANT_R) return fail(nullptr, RTCUR_EINVAL, "variant must be F (0) or R (1)");
  rtcur_options o;
  memset(&o, 0, sizeof o);
  o.scope = RTCUR_SCOPE_SAMPLED;
  o.dense_form = RTCUR_FORM_FP32;
  o.refine_steps = 2;
  o.jacobi_max_sweeps = 30;
  o.inband_rel = 1e-6;
  if (opt) {
    o = *opt;
    for (int i = 0; i < 2; ++i)
      if (o.reserved[i] != 0) return fail(nullptr, RTCUR_EINVAL, "options.reserved must be zero");
    if (o.refine_steps == 0 && o.jacobi_max_sweeps == 0 && o.inband_rel == 0.0) {
      o.refine_steps = 2; o.jacobi_max_sweeps = 30; o.inband_rel = 1e-6;
    }
  }
  if (o.scope != RTCUR_SCOPE_SAMPLED && o.scope != RTCUR_SCOPE_FULL) return fail(nullptr, RTCUR_EINVAL, "scope must be SAMPLED or FULL");
  if (o.dense_form < RTCUR_FORM_FP32 || o.dense_form > RTCUR_FORM_TF32) return fail(nullptr, RTCUR_EINVAL, "dense_form must be 0..3");
  if (o.refine_steps < 0 || o.refine_steps > 8) return fail(nullptr, RTCUR_EINVAL, "refine_steps must be in [0, 8]");
  if (o.jacobi_max_sweeps < 1 || o.jacobi_max_sweeps > 100) return fail(nullptr, RTCUR_EINVAL, "jacobi_max_sweeps must be in [1, 100]");
  if (!(o.inband_rel >= 0.0 && o.inband_rel < 1.0)) return fail(nullptr, RTCUR_EINVAL, "inband_rel must be in [0, 1)");
  if (o.eig_method != 0 && o.eig_method != 1) return fail(nullptr, RTCUR_EINVAL, "eig_method must be 0 (tridiagonal) or 1 (Jacobi)");
  if (o.refine_cluster != 0 && o.refine_cluster != 2 && o.refine_cluster != 4 && o.refine_cluster != 8 &&
      o.refine_cluster != 16)
    return fail(nullptr, RTCUR_EINVAL, "refine_cluster must be 0 (auto), 2, 4, 8 or 16");
  if (o.checkpoint < 0 || o.checkpoint > max_iter) return fail(nullptr, RTCUR_EINVAL, "checkpoint must be in [0, max_iter]");
  if (o.checkpoint > 0 && n_modes != 3) return fail(nullptr, RTCUR_EINVAL, "checkpoint (the adjoint) needs n_modes == 3");
  if (o.s_format != RTCUR_S_DENSE && o.s_format != RTCUR_S_COMPRESSED)
    return fail(nullptr, RTCUR_EINVAL, "s_format must be DENSE (0) or COMPRESSED (1)");
  if (o.s_format == RTCUR_S_COMPRESSED && (o.scope != RTCUR_SCOPE_FULL || o.dense_form != RTCUR_FORM_FP32))
    return fail(nullptr, RTCUR_EINVAL, "s_format COMPRESSED needs the FULL scope and dense_form FP32");
  if (o.dense_ctas < 0 || o.dense_ctas > 1024) return fail(nullptr, RTCUR_EINVAL, "dense_ctas must be in [0, 1024]");
  if (o.sample_x != RTCUR_SAMPLE_X_FP32 && o.sample_x != RTCUR_SAMPLE_X_BF16)
    return fail(nullptr, RTCUR_EINVAL, "sample_x must be FP32 (0) or BF16 (1)");
  if (o.sample_x == RTCUR_SAMPLE_X_BF16 && o.checkpoint > 0)
    return fail(nullptr, RTCUR_EINVAL, "sample_x BF16 cannot be combined with checkpoint (the adjoint is taken w.r.t. the FP32 X)");

  Geom g;
  memset(&g, 0, sizeof g);
  g.n = n_modes;
  g.N = 1;
  for (int i = 0; i < n_modes; ++i) {
    if (dims[i] < 1) return fail(nullptr, RTCUR_EINVAL, "dims[%d] must be >= 1", i);
    g.d[i] = dims[i];
    if (g.N > (1LL << 40) / dims[i]) return fail(nullptr, RTCUR_EINVAL, "prod(dims) must be < 2^40");
    g.N *= dims[i];
  }
  for (int i = 0; i < n_modes; ++i) {
    long long other = g.N / g.d[i];
    if (ranks[i] < 1 || ranks[i] > RT_MAXR) return fail(nullptr, RTCUR_EINVAL, "ranks[%d] must be in [1, %d]", i, RT_MAXR);
    if (nI[i] < ranks[i] || nI[i] > g.d[i] || nI[i] > RT_MAXM)
      return fail(nullptr, RTCUR_EINVAL, "nI[%d] must be in [ranks[%d], min(dims[%d], %d)]", i, i, i, RT_MAXM);
    if (nJ[i] < ranks[i] || nJ[i] > other || nJ[i] > RT_MAXQ)
      return fail(nullptr, RTCUR_EINVAL, "nJ[%d] must be in [ranks[%d], min(prod of other dims, %d)]", i, i, RT_MAXQ);
    g.r[i] = ranks[i];
    g.m[i] = nI[i];
    g.q[i] = nJ[i];
  }
  g.variant = variant;
  g.n_sets = (variant == RTCUR_VARIANT_R) ? max_iter : 1;
  g.max_iter = max_iter;
  g.scope = o.scope;
  g.refine_steps = o.refine_steps;
  g.max_sweeps = o.jacobi_max_sweeps;
  g.warm_start = 0;
  g.eig_method = o.eig_method;
  g.dense_ctas = o.dense_ctas;
  g.gamma = gamma;
  g.tol = tol;
  g.inband = o.inband_rel;
  g.ck_iters = o.checkpoint;
  g.nR = 1;
  g.nG = 1;
  for (int i = 0; i < n_modes; ++i) {
    g.nR *= g.m[i];
    g.nG *= g.r[i];
  }
  g.rlast = g.r[n_modes - 1];
  g.seg[0] = 0;
  g.seg[1] = g.nR;
  for (int i = 0; i < n_modes; ++i) g.seg[i + 2] = g.seg[i + 1] + g.d[i] * g.q[i];
  g.nS = g.seg[n_modes + 1];
  g.rowsT = g.N / g.d[n_modes - 1];
  long long off = 0;
  for (int i = 0; i < n_modes; ++i) { g.ioff[i] = off; off += g.m[i]; }
  for (int i = 0; i < n_modes; ++i) { g.joff[i] = off; off += g.q[i]; }
  g.set_len = off;
  long long oB = 0, oQ = 0, oM = 0, oY = 0, oR = 0, oL = 0, nch = 1;
  for (int i = 0; i < n_modes; ++i) {
    g.offB[i] = oB; oB += g.d[i] * g.r[i];
    g.offQ[i] = oQ; oQ += (long long)g.m[i] * g.r[i];
    g.offM[i] = oM; oM += (long long)g.m[i] * g.m[i];
    g.offY[i] = oY; oY += (long long)g.q[i] * g.r[i];
    g.offR[i] = oR; oR += g.r[i];
    g.offL[i] = oL; oL += g.m[i];
    long long c = (g.q[i] + RT_BCHUNK - 1) / RT_BCHUNK;
    if (c > nch) nch = c;
  }
  g.sumB = oB;
  g.sumMR = oQ;
  g.dense_form = o.dense_form;
  g.s_format = o.s_format;
  g.sample_x = o.sample_x;
  {
    long long oDM = 0;
    for (int i = 0; i < n_modes; ++i) { g.offDM[i] = oDM; oDM += g.d[i] * g.m[i]; }
    g.sumDM = oDM;
  }
  if (o.scope == RTCUR_SCOPE_FULL && !dense_form_supported(g, o.dense_form))
    return fail(nullptr, RTCUR_EINVAL, "dense_form %d does not support these dims/ranks (plain: 3 modes; BF16/TF32: d_n %% 4 == 0, d_n <= 1024; BF16: r_n <= 5; TF32: r_n <= 8)", o.dense_form);
  {
    long long oD = 0, oW = 0;
    for (int i = 0; i < n_modes; ++i) {
      g.offD[i] = oD; oD += g.d[i];
      g.offW[i] = oW; oW += (long long)g.m[i] * g.q[i];
      if (g.d[i] * (long long)g.q[i] >= (1LL << 31))
        return fail(nullptr, RTCUR_EINVAL, "dims[%d] * nJ[%d] must be < 2^31", i, i);
    }
    g.sumD = oD;
    g.sumW = oW;
  }
  g.nchunk = nch;
  g.nH = (long long)g.r[0] * g.r[n_modes - 1];
  for (int l = 1; l <= n_modes - 2; ++l) g.nH *= g.d[l];
  long long zs = 1;
  for (int st = 0; st < n_modes - 1; ++st) {
    int j = n_modes - 1 - st;
    long long sz = 1;
    for (int l = 0; l < n_modes; ++l) sz *= (l >= j) ? g.r[l] : g.m[l];
    if (sz > zs) zs = sz;
  }
  g.zsize = zs;

  if (g.rowsT >= (1LL << 32) || g.d[n_modes - 1] >= (1LL << 32))
    return fail(nullptr, RTCUR_EINVAL, "prod of the first n-1 dims and the last dim must be < 2^32");
  if (g.s_format == RTCUR_S_COMPRESSED && !compressed_geometry(g, g.tile_rows))
    return fail(nullptr, RTCUR_EINVAL, "s_format COMPRESSED needs d_n %% 4 == 0, d_n <= 4096 and r_n <= 8");
  int dev = 0, optin = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return fail(nullptr, RTCUR_ECUDA, "no CUDA device: %s", cudaGetErrorString(ce));
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  int mx = 0;
  for (int i = 0; i < n_modes; ++i) mx = g.m[i] > mx ? g.m[i] : mx;
  if (o.checkpoint > 0 && mx > 160)
    return fail(nullptr, RTCUR_EINVAL, "checkpoint (the adjoint) needs every |I_i| <= 160");
  if (jacobi_smem_bytes(mx) > (size_t)optin)
    return fail(nullptr, RTCUR_EINVAL, "|I_i| = %d needs %zu bytes of shared memory (device allows %d)", mx, jacobi_smem_bytes(mx), optin);

  rtcur_plan* p = new rtcur_plan();
  p->serial = g_serial.fetch_add(1);
  p->g = g;
  p->opt = o;
  p->zeta0 = zeta0;
  Bufs& b = p->b;
  memset(&b, 0, sizeof b);
  cudaError_t e = cudaSuccess;
#define AL(ptr, cnt) if (e == cudaSuccess) e = dalloc(p, &(ptr), (size_t)(cnt))
  AL(b.st, 1);
  AL(b.sp, 1);
  long long* idx = nullptr;
  AL(idx, (size_t)g.n_sets * g.set_len);
  b.idx = idx;
  AL(b.Xs, g.nS);
  AL(b.XS, g.nS);
  AL(b.rc, g.nS);
  AL(b.W, g.sumW);
  int* posd = nullptr;
  AL(posd, (size_t)g.n_sets * g.sumD);
  b.pos = posd;
  AL(b.gram, oM);
  AL(b.jV, oM);
  AL(b.jL, oL);
  AL(b.Qr, oQ);
  AL(b.sig, oR);
  AL(b.Y, oY);
  AL(b.warm, RT_MAXN);
  AL(b.wratio, RT_MAXN);
  AL(b.Bpart, g.nchunk * g.sumB);
  AL(b.B[0], g.sumB);
  AL(b.B[1], g.sumB);
  AL(b.G[0], g.nG);
  AL(b.G[1], g.nG);
  AL(b.Z[0], g.zsize);
  AL(b.Z[1], g.zsize);
  AL(b.H, g.nH);
  AL(b.T[0], g.rowsT * g.rlast + 4);  // +4: the dense pass copies 16-byte aligned windows
  AL(b.T[1], g.rowsT * g.rlast + 4);
  AL(b.red, (size_t)TK_COUNT * 1024 * RT_RED_SLOTS);
  AL(b.ticket, TK_COUNT);
  AL(b.e_hist, max_iter);
  AL(b.z_hist, max_iter);
  AL(b.nnz_hist, max_iter);
  {
    long long nU = 0;
    for (int i = 0; i < n_modes; ++i) nU += (long long)g.q[i] * g.m[i];
    AL(b.curF, g.nS);
    AL(b.curU, nU);
  }
#ifdef RTCUR_TIMELINE
  AL(b.tl, 4096);
  AL(b.tl_n, 1);
#endif
  if (o.scope == RTCUR_SCOPE_FULL && g.s_format == RTCUR_S_DENSE) AL(p->S_internal, g.N);
  if (g.sample_x == RTCUR_SAMPLE_X_BF16) AL(b.Xb, g.N);
  if (g.s_format == RTCUR_S_COMPRESSED) {
    const long long wpr = (g.d[n_modes - 1] + 31) / 32;
    AL(b.smask, g.rowsT * wpr);
    AL(b.svals, g.N);
    AL(b.srow, g.rowsT + 1);
    AL(b.soff, (g.rowsT + 1) / 1023 + 64);
  }
  if (o.scope == RTCUR_SCOPE_FULL && o.dense_form == RTCUR_FORM_FP32_PLAIN) {
    AL(b.Ap[0], g.sumDM);
    AL(b.Ap[1], g.sumDM);
    AL(b.Rp[0], g.nR);
    AL(b.Rp[1], g.nR);
    AL(b.Z1p, (long long)g.m[0] * g.m[1] * g.d[2]);
    AL(b.Z2p, (long long)g.m[0] * g.d[1] * g.d[2]);
    AL(b.Lplain, g.N);
  }
  if (o.checkpoint > 0) {
    AL(b.ckV, (long long)o.checkpoint * g.nS);
    AL(b.ckM, (long long)o.checkpoint * g.nS);
    BwWork& w = p->bw;
    memset(&w, 0, sizeof w);
    backward_layout(g, w);
    const long long K = o.checkpoint;
    long long mq = 0, mm = 0;
    for (int i = 0; i < n_modes; ++i) {
      mq = std::max(mq, (long long)g.m[i] * g.q[i]);
      mm = std::max(mm, (long long)g.m[i] * g.m[i]);
    }
    AL(w.W, K * w.slotW);
    AL(w.U, K * w.slotMM);
    AL(w.Ub, K * w.slotMM);
    AL(w.lam, K * w.slotM);
    AL(w.Z, K * w.slotMM);
    AL(w.P, K * w.slotQM);
    AL(w.A, K * w.slotDM);
    AL(w.Vb, g.nS);
    AL(w.Lb, g.nS);
    AL(w.Ab, w.slotDM);
    AL(w.Pb, mq);
    AL(w.Wb, mq);
    AL(w.T0, mm);
    AL(w.T1, mm);
    AL(w.Pi, w.slotMM);
    AL(w.Zf, mq);
    AL(w.Zfb, mq);
    AL(w.va, mq);
    AL(w.vb, mq);
    AL(w.kr, w.krsz);
    AL(w.pc, RT_MAXQ);
    AL(w.tmp0, w.tmpsz);
    AL(w.tmp1, w.tmpsz);
    AL(w.dX64, g.N);
    AL(w.part, w.partsz);
    if (e == cudaSuccess) e = prepare_backward(mx);
  }
#undef AL
  // the latency-bound sampled chain is captured from a high-priority stream, the bandwidth-bound
  // dense pass from a low-priority one (kernel nodes keep their stream's priority)
  int prio_lo = 0, prio_hi = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&p->cap, cudaStreamNonBlocking, prio_hi);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&p->side, cudaStreamNonBlocking, prio_lo);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&p->side2, cudaStreamNonBlocking, prio_hi);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->evFork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->evJoin, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->evFork2, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->evJoin2, cudaEventDisableTiming);
  if (e == cudaSuccess) {
    size_t sm = jacobi_smem_bytes(mx);
    e = prepare_jacobi(sm);
  }
  if (e == cudaSuccess) e = prepare_dense(g);
  if (e == cudaSuccess) e = prepare_sample_kernels();
  if (e == cudaSuccess) e = prepare_factor_kernels();
  if (e == cudaSuccess) {
    e = prepare_refine(p->g, o.refine_cluster);
    if (e == cudaErrorInvalidValue) {
      fail(nullptr, RTCUR_EINVAL, "refine_cluster %d cannot run for these sample sizes", o.refine_cluster);
      rtcur_destroy(p);
      return RTCUR_EINVAL;
    }
  }
  if (e == cudaSuccess) e = cudaMemset(b.ticket, 0, sizeof(unsigned) * TK_COUNT);
  if (e == cudaSuccess) e = cudaMemset(b.st, 0, sizeof(State));
  if (e != cudaSuccess) {
    rtcur_status st = (e == cudaErrorMemoryAllocation) ? RTCUR_ENOMEM : RTCUR_ECUDA;
    fail(nullptr, st, "allocating the plan: %s", cudaGetErrorString(e));
    rtcur_destroy(p);
    return st;
  }
  *out = p;
  return RTCUR_OK;
}

rtcur_status rtcur_begin(rtcur_plan* p, const float* X, const int64_t* idx, float* S_work,
                         void* stream) {
  if (!p) return fail(nullptr, RTCUR_EINVAL, "plan is NULL");
  if (!X || !idx) return fail(p, RTCUR_EINVAL, "X and idx must not be NULL");
  const Geom& g = p->g;
  const bool compressed = (g.s_format == RTCUR_S_COMPRESSED);
  float* S = compressed ? nullptr : (S_work ? S_work : p->S_internal);
  if (!aligned16(X) || (S && !aligned16(S))) return fail(p, RTCUR_EINVAL, "X and S must be 16-byte aligned");
  rtcur_status st = check_sets(p, idx);
  if (st != RTCUR_OK) return st;
  rtcur_status gb = build_graphs(p);
  if (gb != RTCUR_OK) return gb;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Bufs& b = p->b;
  CKC(p, cudaMemcpyAsync((void*)b.idx, idx, sizeof(int64_t) * g.n_sets * g.set_len, cudaMemcpyHostToDevice, s));
  // position tables: pos[t] = a if I_i[a] = t, else -1 (one table per set)
  p->pos_host.assign((size_t)g.n_sets * g.sumD, -1);
  for (int st2 = 0; st2 < g.n_sets; ++st2) {
    const int64_t* set = idx + (size_t)st2 * g.set_len;
    for (int i = 0; i < g.n; ++i)
      for (int a = 0; a < g.m[i]; ++a)
        p->pos_host[(size_t)st2 * g.sumD + g.offD[i] + set[g.ioff[i] + a]] = a;
  }
  CKC(p, cudaMemcpyAsync((void*)b.pos, p->pos_host.data(), sizeof(int) * p->pos_host.size(), cudaMemcpyHostToDevice, s));
  SolvePtrs sp;
  sp.X = X;
  sp.S = S;
  CKC(p, cudaMemcpyAsync(b.sp, &sp, sizeof sp, cudaMemcpyHostToDevice, s));

  CKC(p, cudaMemsetAsync(b.T[0], 0, sizeof(float) * g.rowsT * g.rlast, s));
  CKC(p, cudaMemsetAsync(b.B[0], 0, sizeof(float) * g.sumB, s));
  CKC(p, cudaMemsetAsync(b.G[0], 0, sizeof(float) * g.nG, s));
  CKC(p, cudaMemsetAsync(b.warm, 0, sizeof(int) * RT_MAXN, s));
  CKC(p, cudaMemsetAsync(b.wratio, 0, sizeof(double) * RT_MAXN, s));
  if (b.Ap[0]) {
    CKC(p, cudaMemsetAsync(b.Ap[0], 0, sizeof(float) * g.sumDM, s));
    CKC(p, cudaMemsetAsync(b.Rp[0], 0, sizeof(float) * g.nR, s));
  }
  CKC(p, launch_setup(g, b, p->zeta0, p->zeta0 <= 0.0 ? 1 : 0, s));
  if (b.Xb) CKC(p, launch_x_bf16(g, b, X, s));  // the sampled step's BF16 copy of this X
  if (g.variant == RTCUR_VARIANT_F) CKC(p, launch_gather_x(g, b, s));
  p->X = X;
  p->S_work = S;
  p->begun = true;
  return RTCUR_OK;
}

rtcur_status rtcur_iterate(rtcur_plan* p, int32_t n_iter, void* stream) {
  if (!p) return fail(nullptr, RTCUR_EINVAL, "plan is NULL");
  if (!p->begun) return fail(p, RTCUR_EINVAL, "rtcur_begin must come first");
  if (n_iter < 0) return fail(p, RTCUR_EINVAL, "n_iter must be >= 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < n_iter; ++i) CKC(p, cudaGraphLaunch(p->iterX, s));
  return RTCUR_OK;
}

rtcur_status rtcur_finish(rtcur_plan* p, float* L_out, float* S_out, rtcur_result* res,
                          void* stream) {
  if (!p) return fail(nullptr, RTCUR_EINVAL, "plan is NULL");
  if (!p->begun) return fail(p, RTCUR_EINVAL, "rtcur_begin must come first");
  if ((L_out && !aligned16(L_out)) || (S_out && !aligned16(S_out)))
    return fail(p, RTCUR_EINVAL, "L_out and S_out must be 16-byte aligned");
  const Geom& g = p->g;
  const Bufs& b = p->b;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool full = (g.scope == RTCUR_SCOPE_FULL);
  const bool compressed = (g.s_format == RTCUR_S_COMPRESSED);
  CKC(p, launch_materialize(g, b, L_out, full ? nullptr : S_out, s));
  if (full && !compressed && S_out && S_out != p->S_work)
    CKC(p, cudaMemcpyAsync(S_out, p->S_work, sizeof(float) * g.N, cudaMemcpyDeviceToDevice, s));
  State h;
  CKC(p, cudaMemcpyAsync(&h, b.st, sizeof h, cudaMemcpyDeviceToHost, s));
  CKC(p, cudaStreamSynchronize(s));
  if (full && S_out && h.k == 0) {  // no dense pass ran: S^(0) = 0
    CKC(p, cudaMemsetAsync(S_out, 0, sizeof(float) * g.N, s));
    CKC(p, cudaStreamSynchronize(s));
  } else if (full && S_out && compressed) {  // expand the last pass's compressed S
    CKC(p, launch_decode_s(g, b, S_out, s));
    CKC(p, cudaStreamSynchronize(s));
  }
  int nh = h.k < g.max_iter ? h.k : g.max_iter;
  if (res) {
    if (res->e_hist && nh) CKC(p, cudaMemcpy(res->e_hist, b.e_hist, sizeof(double) * nh, cudaMemcpyDeviceToHost));
    if (res->zeta_hist && nh) CKC(p, cudaMemcpy(res->zeta_hist, b.z_hist, sizeof(double) * nh, cudaMemcpyDeviceToHost));
    if (res->nnz_hist && nh) CKC(p, cudaMemcpy(res->nnz_hist, b.nnz_hist, sizeof(int64_t) * nh, cudaMemcpyDeviceToHost));
    res->iters = h.k;
    res->flags = h.flags;
    res->jacobi_sweeps = h.jsweeps;
    res->warm_hits = h.warm_hits;
    res->e = h.e;
    res->zeta = h.zeta;
    res->nnz_sample = h.nnz_s;
    res->inband_sample = h.inband_s;
    res->nnz_full = full ? h.nnz_f : -1;
    res->inband_full = full ? h.inband_f : -1;
    res->resid_full = full ? h.resid_f : -1.0;
    res->status = (h.e > g.tol) ? RTCUR_NOT_CONVERGED : RTCUR_OK;
  }
  if (h.err != 0) {
    if (h.err == RTCUR_ENONFINITE) return fail(p, RTCUR_ENONFINITE, "X holds NaN or Inf on the sampled entries");
    return fail(p, (rtcur_status)h.err, "device-side error %d", h.err);
  }
  return (h.e > g.tol) ? RTCUR_NOT_CONVERGED : RTCUR_OK;
}

rtcur_status rtcur_solve(rtcur_plan* p, const float* X, const int64_t* idx, float* L_out,
                         float* S_out, rtcur_result* res, void* stream) {
  rtcur_status st = rtcur_begin(p, X, idx, (p && p->g.scope == RTCUR_SCOPE_FULL) ? S_out : nullptr, stream);
  if (st != RTCUR_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (1.0 > p->g.tol) CKC(p, cudaGraphLaunch(p->loopX, s));
  return rtcur_finish(p, L_out, S_out, res, stream);
}

rtcur_status rtcur_solve_batched(rtcur_plan* const* plans, int32_t count, const float* const* X,
                                 const int64_t* const* idx, float* const* L_out, float* const* S_out,
                                 rtcur_result* res, void* stream) {
  if (!plans || count < 1 || count > 4096) return fail(nullptr, RTCUR_EINVAL, "plans must hold 1..4096 plans");
  if (!X || !idx) return fail(nullptr, RTCUR_EINVAL, "X and idx must not be NULL");
  for (int i = 0; i < count; ++i) {
    if (!plans[i]) return fail(nullptr, RTCUR_EINVAL, "plans[%d] is NULL", i);
    if (!(plans[i]->g.tol < 1.0)) return fail(plans[i], RTCUR_EINVAL, "a batched problem needs tol < 1 (e^(0) = 1)");
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) return fail(plans[i], RTCUR_EINVAL, "plans[%d] and plans[%d] are the same plan", j, i);
  }
  rtcur_plan* p0 = plans[0];
  for (int i = 0; i < count; ++i) {
    rtcur_plan* p = plans[i];
    rtcur_status st = rtcur_begin(p, X[i], idx[i],
                                  (p->g.scope == RTCUR_SCOPE_FULL && S_out) ? S_out[i] : nullptr, stream);
    if (st != RTCUR_OK) return fail(p0, st, "problem %d: %s", i, p->err.c_str());
  }
  BatchGraph* bg = p0->batch;
  bool hit = bg && (int)bg->plans.size() == count;
  for (int i = 0; hit && i < count; ++i) hit = bg->plans[i] == plans[i] && bg->serials[i] == plans[i]->serial;
  if (!hit) {
    free_batch(bg);
    p0->batch = nullptr;
    rtcur_status st = build_batch(plans, count, &p0->batch);
    if (st != RTCUR_OK) return st;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CKC(p0, cudaGraphLaunch(p0->batch->X, s));
  rtcur_status worst = RTCUR_OK;
  for (int i = 0; i < count; ++i) {
    rtcur_status st = rtcur_finish(plans[i], L_out ? L_out[i] : nullptr, S_out ? S_out[i] : nullptr,
                                   res ? &res[i] : nullptr, stream);
    if (st != RTCUR_OK && worst == RTCUR_OK) {
      worst = st;
      if (i > 0) fail(p0, st, "problem %d: %s", i, plans[i]->err.c_str());
    }
  }
  return worst;
}

rtcur_status rtcur_threshold_dense(rtcur_plan* p, int32_t n_launch, void* stream) {
  if (!p) return fail(nullptr, RTCUR_EINVAL, "plan is NULL");
  if (!p->begun) return fail(p, RTCUR_EINVAL, "rtcur_begin must come first");
  if (p->g.scope != RTCUR_SCOPE_FULL) return fail(p, RTCUR_EINVAL, "rtcur_threshold_dense needs a FULL-scope plan");
  if (n_launch < 0) return fail(p, RTCUR_EINVAL, "n_launch must be >= 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < n_launch; ++i) CKC(p, launch_dense(p->g, p->b, p->opt.dense_form, s));
  return RTCUR_OK;
}

rtcur_status rtcur_get_s_compressed(rtcur_plan* p, rtcur_s_compressed* out, void* stream) {
  if (!p) return fail(nullptr, RTCUR_EINVAL, "plan is NULL");
  if (!out) return fail(p, RTCUR_EINVAL, "out must not be NULL");
  const Geom& g = p->g;
  if (g.s_format != RTCUR_S_COMPRESSED) return fail(p, RTCUR_EINVAL, "the plan's s_format is not COMPRESSED");
  if (!p->begun) return fail(p, RTCUR_EINVAL, "rtcur_begin must come first");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  State h;
  CKC(p, cudaMemcpyAsync(&h, p->b.st, sizeof h, cudaMemcpyDeviceToHost, s));
  CKC(p, cudaStreamSynchronize(s));
  if (h.k == 0) return fail(p, RTCUR_EINVAL, "no dense pass has run (S^(0) = 0)");
  memset(out, 0, sizeof *out);
  out->mask = p->b.smask;
  out->vals = p->b.svals;
  out->nnz = h.nnz_f;
  out->rows = g.rowsT;
  out->cols = g.d[g.n - 1];
  out->words_per_row = (g.d[g.n - 1] + 31) / 32;
  out->block_cols = 128;
  return RTCUR_OK;
}

rtcur_status rtcur_compact_s(rtcur_plan* p, float* vals_out, int64_t* row_off, void* stream) {
  if (!p) return fail(nullptr, RTCUR_EINVAL, "plan is NULL");
  if (!vals_out && !row_off) return fail(p, RTCUR_EINVAL, "vals_out and row_off are both NULL");
  const Geom& g = p->g;
  if (g.s_format != RTCUR_S_COMPRESSED) return fail(p, RTCUR_EINVAL, "the plan's s_format is not COMPRESSED");
  if (!p->begun) return fail(p, RTCUR_EINVAL, "rtcur_begin must come first");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  State h;
  CKC(p, cudaMemcpyAsync(&h, p->b.st, sizeof h, cudaMemcpyDeviceToHost, s));
  CKC(p, cudaStreamSynchronize(s));
  if (h.k == 0) return fail(p, RTCUR_EINVAL, "no dense pass has run (S^(0) = 0)");
  long long* off = row_off ? reinterpret_cast<long long*>(row_off) : p->b.srow;
  CKC(p, launch_compact_s(g, p->b, off, vals_out, s));
  return RTCUR_OK;
}

rtcur_status rtcur_decode_s(rtcur_plan* p, float* S_out, void* stream) {
  if (!p) return fail(nullptr, RTCUR_EINVAL, "plan is NULL");
  if (!S_out) return fail(p, RTCUR_EINVAL, "S_out must not be NULL");
  const Geom& g = p->g;
  if (g.s_format != RTCUR_S_COMPRESSED) return fail(p, RTCUR_EINVAL, "the plan's s_format is not COMPRESSED");
  if (!p->begun) return fail(p, RTCUR_EINVAL, "rtcur_begin must come first");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  State h;
  CKC(p, cudaMemcpyAsync(&h, p->b.st, sizeof h, cudaMemcpyDeviceToHost, s));
  CKC(p, cudaStreamSynchronize(s));
  if (h.k == 0)
    CKC(p, cudaMemsetAsync(S_out, 0, sizeof(float) * g.N, s));
  else
    CKC(p, launch_decode_s(g, p->b, S_out, s));
  return RTCUR_OK;
}

rtcur_status rtcur_get_factors(rtcur_plan* p, float* G, float* B, int32_t* k, double* zeta,
                               void* stream) {
  if (!p) return fail(nullptr, RTCUR_EINVAL, "plan is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  State h;
  CKC(p, cudaMemcpyAsync(&h, p->b.st, sizeof h, cudaMemcpyDeviceToHost, s));
  CKC(p, cudaStreamSynchronize(s));
  int cp = h.k & 1;
  if (G) CKC(p, cudaMemcpy(G, p->b.G[cp], sizeof(float) * p->g.nG, cudaMemcpyDeviceToHost));
  if (B) CKC(p, cudaMemcpy(B, p->b.B[cp], sizeof(float) * p->g.sumB, cudaMemcpyDeviceToHost));
  if (k) *k = h.k;
  if (zeta) *zeta = h.zeta;
  return RTCUR_OK;
}

rtcur_status rtcur_get_cur(rtcur_plan* p, float* R, float* C, double* Upinv, int32_t* k,
                           void* stream) {
  if (!p) return fail(nullptr, RTCUR_EINVAL, "plan is NULL");
  if (!p->begun) return fail(p, RTCUR_EINVAL, "rtcur_begin must come first");
  const Geom& g = p->g;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  State h;
  CKC(p, cudaMemcpyAsync(&h, p->b.st, sizeof h, cudaMemcpyDeviceToHost, s));
  CKC(p, cudaStreamSynchronize(s));
  if (k) *k = h.k;
  if (h.k < 1) return fail(p, RTCUR_EINVAL, "no iteration has run (L^(0) = 0 has no CUR factors)");
  long long nU = 0;
  for (int i = 0; i < g.n; ++i) nU += (long long)g.q[i] * g.m[i];
  CKC(p, launch_export_cur(g, p->b, s));
  if (R) CKC(p, cudaMemcpyAsync(R, p->b.curF, sizeof(float) * g.nR, cudaMemcpyDeviceToHost, s));
  if (C) CKC(p, cudaMemcpyAsync(C, p->b.curF + g.nR, sizeof(float) * (g.nS - g.nR), cudaMemcpyDeviceToHost, s));
  if (Upinv) CKC(p, cudaMemcpyAsync(Upinv, p->b.curU, sizeof(double) * nU, cudaMemcpyDeviceToHost, s));
  CKC(p, cudaStreamSynchronize(s));
  return RTCUR_OK;
}

rtcur_status rtcur_backward(rtcur_plan* p, const float* dL, float* dX, void* stream) {
  if (!p) return fail(nullptr, RTCUR_EINVAL, "plan is NULL");
  if (!dL || !dX) return fail(p, RTCUR_EINVAL, "dL and dX must not be NULL");
  if (!aligned16(dX)) return fail(p, RTCUR_EINVAL, "dX must be 16-byte aligned");
  const Geom& g = p->g;
  if (g.ck_iters <= 0) return fail(p, RTCUR_EINVAL, "the plan records no iterations (options.checkpoint = 0)");
  if (!p->begun) return fail(p, RTCUR_EINVAL, "no solve to differentiate");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  State h;
  CKC(p, cudaMemcpyAsync(&h, p->b.st, sizeof h, cudaMemcpyDeviceToHost, s));
  CKC(p, cudaStreamSynchronize(s));
  if (h.k < 1) return fail(p, RTCUR_EINVAL, "the solve ran no iteration");
  if (h.k > g.ck_iters)
    return fail(p, RTCUR_EINVAL, "the solve ran %d iterations, more than the %d recorded", h.k, g.ck_iters);
  if (h.err != 0) return fail(p, (rtcur_status)h.err, "the forward pass latched device error %d", h.err);
  CKC(p, launch_backward(g, p->b, p->bw, h.k, dL, dX, s));
  return RTCUR_OK;
}

rtcur_status rtcur_set_wait_limit(rtcur_plan* p, int64_t polls, void* stream) {
  if (!p) return fail(nullptr, RTCUR_EINVAL, "plan is NULL");
  if (polls < 0) return fail(p, RTCUR_EINVAL, "polls must be >= 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  long long v = polls;
  CKC(p, cudaMemcpyAsync(&p->b.st->wait_polls, &v, sizeof v, cudaMemcpyHostToDevice, s));
  CKC(p, cudaStreamSynchronize(s));
  return RTCUR_OK;
}

int64_t rtcur_sample_count(const rtcur_plan* p) { return p ? p->g.nS : 0; }

#ifdef RTCUR_TIMELINE
// Diagnostic builds only: copy out the kernel timeline and reset it.
RTCUR_API int rtcur_debug_timeline(rtcur_plan* p, unsigned long long* out, int max_rec) {
  unsigned n = 0;
  cudaDeviceSynchronize();
  cudaMemcpy(&n, p->b.tl_n, sizeof n, cudaMemcpyDeviceToHost);
  if (n > 4096) n = 4096;
  if ((int)n > max_rec) n = (unsigned)max_rec;
  std::vector<TlRec> h(n);
  cudaMemcpy(h.data(), p->b.tl, sizeof(TlRec) * n, cudaMemcpyDeviceToHost);
  for (unsigned i = 0; i < n; ++i) { out[3 * i] = h[i].id; out[3 * i + 1] = h[i].t0; out[3 * i + 2] = h[i].t1; }
  cudaMemset(p->b.tl_n, 0, sizeof(unsigned));
  return (int)n;
}
#endif

const char* rtcur_last_error(const rtcur_plan* p) { return p ? p->err.c_str() : g_create_err.c_str(); }

void rtcur_destroy(rtcur_plan* p) {
  if (!p) return;
  cudaDeviceSynchronize();
  free_batch(p->batch);
  if (p->loopX) cudaGraphExecDestroy(p->loopX);
  if (p->iterX) cudaGraphExecDestroy(p->iterX);
  if (p->loopG) cudaGraphDestroy(p->loopG);
  if (p->iterG) cudaGraphDestroy(p->iterG);
  if (p->evFork) cudaEventDestroy(p->evFork);
  if (p->evJoin) cudaEventDestroy(p->evJoin);
  if (p->evFork2) cudaEventDestroy(p->evFork2);
  if (p->evJoin2) cudaEventDestroy(p->evJoin2);
  if (p->cap) cudaStreamDestroy(p->cap);
  if (p->side) cudaStreamDestroy(p->side);
  if (p->side2) cudaStreamDestroy(p->side2);
  for (void* v : p->allocs) cudaFree(v);
  delete p;
}

}  // extern "C"
