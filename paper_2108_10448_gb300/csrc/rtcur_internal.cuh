// Internal definitions shared by the RTCUR kernels and the C-ABI host code.
//
// Layout of the sampled entries ("sample list"), one float per entry, in this order:
//   segment 0      R = X(I_1, ..., I_n)           prod m_i entries, row-major over (a_1..a_n)
//   segment 1 + i  C_i = X_(i)(:, J_i)            d_i * q_i entries, fiber-major: entry
//                                                  b * d_i + t is row t of column b
// The same enumeration is used for X on the sample (Xs), for X - S on the sample (XS) and for
// the error terms of Eq. (rel_err).
//
// L^(k) is kept in Tucker form G x_1 B_1 ... x_n B_n (G: prod r_i, B_i: d_i x r_i). Its
// evaluation at any entry is the last-mode product L(p) = sum_c T[row(p), c] * B_n[p_n, c] with
// the table T = G x_1 B_1 ... x_{n-1} B_{n-1} (prod_{i<n} d_i rows, r_n columns). Every kernel
// that needs L (sampled threshold, sampled error, dense pass) evaluates it through T with the
// same FMA order, so all of them see the same FP32 value of L at a given entry.
//
// Two copies of (G, B, T) alternate between iterations: L^(k) lives in copy (k & 1).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <mutex>

#define RT_MAXN 4
#define RT_MAXR 16
#define RT_MAXM 192      // cap on |I_i| (the FP32 Jacobi keeps M and V in shared memory)
#define RT_MAXQ 4096     // cap on |J_i|
#define RT_RED_SLOTS 16  // doubles per block in reduction partials
#define RT_BCHUNK 8      // J_i columns per split-K partial of B_i = C_i Y_i

struct Geom {
  int n;
  int r[RT_MAXN];
  int m[RT_MAXN];
  int q[RT_MAXN];
  int variant;
  int n_sets;
  int max_iter;
  int scope;
  int refine_steps;
  int max_sweeps;
  int warm_start;                // start the Jacobi from the previous iteration's basis
  int eig_method;                // FP32 eigenbasis: 0 tridiagonal (m <= 128), 1 Jacobi
  int ncl;                       // CTAs per cluster in the FP64 refinement (16 or 8)
  int dense_ctas;                // persistent CTAs of the dense pass (0: default)
  int dense_form;                // RTCUR_FORM_* of the dense pass
  int ck_iters;                  // iterations recorded for the adjoint (0: none)
  int s_format;                  // RTCUR_S_* of the FULL scope's S output
  int tile_rows;                 // rows per tile of the FP32 bulk-copy pass (compressed S layout)
  int sample_x;                  // RTCUR_SAMPLE_X_*: the sampled step reads X (FP32) or its BF16 copy
  int nG;                       // prod r_i
  int rlast;                    // r_n
  long long d[RT_MAXN];
  long long N;                  // prod d_i
  long long nR;                 // prod m_i
  long long seg[RT_MAXN + 2];   // segment starts; seg[n + 1] = nS
  long long nS;
  long long rowsT;              // prod_{i < n-1} d_i
  long long set_len;            // sum m_i + sum q_i
  long long ioff[RT_MAXN];      // offset of I_i inside one set
  long long joff[RT_MAXN];      // offset of J_i inside one set
  long long offB[RT_MAXN];      // offsets of B_i inside a packed B (sum_{l<i} d_l r_l)
  long long offQ[RT_MAXN];      // offsets inside per-mode m_i x r_i arrays
  long long offM[RT_MAXN];      // offsets inside per-mode m_i x m_i arrays
  long long offY[RT_MAXN];      // offsets inside per-mode q_i x r_i arrays
  long long offR[RT_MAXN];      // offsets inside per-mode r_i arrays
  long long offL[RT_MAXN];      // offsets inside per-mode m_i arrays
  long long sumMR;              // sum m_i r_i
  long long sumD;               // sum d_i
  long long offD[RT_MAXN];      // offsets of per-mode d_i arrays (position tables)
  long long offW[RT_MAXN];      // offsets of the compact W_i = C_i(I_i, :) (m_i x q_i)
  long long sumW;               // sum m_i q_i
  long long offDM[RT_MAXN];     // offsets of A_i = B_i Q_i^T (d_i x m_i) in the plain form
  long long sumDM;              // sum d_i m_i
  long long nchunk;             // split-K chunks of the B_i product (max over modes)
  long long sumB;               // sum d_i r_i
  long long nH;                 // size of the T stage-A table
  long long zsize;              // scratch size of the core-formation stages
  double gamma;
  double tol;
  double inband;
};

// Device-resident loop state (one per plan).
struct State {
  int k;             // iterations done
  int cont;          // loop continues
  int err;           // latched device error (rtcur_status value, 0 = none)
  int flags;         // RTCUR_FLAG_* accumulated
  double zeta;       // zeta^(k)
  double e;          // e^(k)
  double e_stage;    // e^(k+1) from the error kernel, committed at the end of the iteration
  long long nnz_s;   // sampled nonzeros of S^(k+1) (this iteration)
  long long inband_s;
  long long nnz_f;   // dense pass: nonzeros of S^(k+1)
  long long inband_f;
  double resid_f;    // dense pass: ||X - L - S||_F^2
  double den[RT_MAXN + 1];  // sum of x^2 per segment (this iteration's sets)
  double num[RT_MAXN + 1];  // sum of E^2 per segment
  double zeta0;      // max|X| when requested
  int jsweeps;       // FP32 eigensolver sweeps/steps of the last iteration (max over modes)
  long long warm_hits;  // certified warm results, counted over the solve
  long long wait_polls; // polls of a bounded wait in the dense pass's tile loop (0: the default);
                        // set by rtcur_set_wait_limit, kept across solves
  int pad;
};

// Pointers that may change from solve to solve (read by kernels through one indirection so
// that captured graphs stay valid).
struct SolvePtrs {
  const float* X;
  float* S;          // dense S^(k+1) (FULL scope); may be null in SAMPLED scope
};

struct TlRec { int id; int pad; unsigned long long t0, t1; };  // diagnostic timeline record

struct Bufs {
  State* st;
  SolvePtrs* sp;
  const long long* idx;  // n_sets * set_len
  float* Xs;             // nS
  float* XS;             // nS
  uint2* rc;             // nS, (row of T, column of B_n) of each sampled entry
  const int* pos;        // n_sets * sum d_i: position of t in I_i, or -1
  float* W;              // sum m_i q_i: W_i = C_i(I_i, :), m_i x q_i row-major
  double* gram;          // sum m_i^2
  float* jV;             // sum m_i^2, FP32 eigenvectors (m x m, row-major, column j = vector j)
  float* jL;             // sum m_i, FP32 eigenvalues
  double* Qr;            // sum m_i r_i, final orthonormal top-r basis
  double* sig;           // sum r_i, singular values (0 where truncated)
  double* Y;             // sum q_i r_i, V_r Sigma_r^-1
  int* warm;             // n flags: the warm attempt produced mode i's factors this iteration
  double* wratio;        // n: ||C||_F / lambda_r of the last iteration (warm-attempt gate)
  double* Bpart;         // split-K partials of B (nchunk * sumB)
  float* B[2];           // sumB each
  float* G[2];           // nG each
  double* Z[2];          // zsize each (core-formation stages)
  float* H;              // nH
  float* T[2];           // rowsT * r_n each
  double* red;           // reduction partials
  unsigned* ticket;      // last-block tickets (one per reduction kind)
  double* e_hist;        // max_iter
  double* z_hist;        // max_iter
  long long* nnz_hist;   // max_iter
  float* Ap[2];          // plain form: A_i = B_i Q_i^T of L^(k), two copies
  float* Rp[2];          // plain form: R of L^(k), two copies
  float* Z1p;            // plain form: R x_3 A_3
  float* Z2p;            // plain form: R x_3 A_3 x_2 A_2
  float* Lplain;         // plain form: the materialised L^(k)
  TlRec* tl;             // diagnostic timeline (null unless built with -DRTCUR_TIMELINE)
  unsigned* tl_n;
  float* ckV;            // ck_iters * nS: sampled values X - S of each recorded iteration
  unsigned char* ckM;    // ck_iters * nS: their HT masks (1 = thresholded, the value is L^(k))
  // compressed S (FULL scope, s_format COMPRESSED): support bitmask of rowsT rows of
  // ceil(d_n / 32) words; the nonzero values of each 128-column block of a row, in order, from
  // the block's first element index on; row offsets and scan scratch for the compaction
  unsigned* smask;
  float* svals;
  long long* srow;   // rowsT + 1
  long long* soff;   // (rowsT + 1) / 1023 + 64
  // Algorithm 1's output staged for rtcur_get_cur: R and C_i (nS floats, C_i row-major) and
  // U_i^+ (sum q_i m_i doubles, q_i x m_i row-major)
  float* curF;
  double* curU;
  // sample_x BF16: the BF16 copy of X the sampled step reads (N values, round to nearest even)
  unsigned short* Xb;
};

// Workspace of the adjoint (rtcur_backward), 3-mode tensors. Per recorded iteration and mode:
// W_i (m x q), U (m x m; first M = W W^T, then its eigenvectors), lambda (m), Z (m x m),
// P_i = U_i^+ (q x m) and A_i = C_i P_i (d x m), all FP64; then one set of adjoint buffers.
struct BwWork {
  double *W, *U, *lam, *Z, *P, *A;
  double* Ub;  // per slot and mode, m x m: scratch of the FP64 eigen polish
  long long offW[RT_MAXN], offMM[RT_MAXN], offM[RT_MAXN], offQM[RT_MAXN], offDM[RT_MAXN];
  long long slotW, slotMM, slotM, slotQM, slotDM;
  double* Vb;    // nS: slot adjoint (R segment = R_bar, fiber segments = C_bar_i)
  double* Lb;    // nS: adjoint of L^(k) at the slots
  double* Ab;    // slotDM: A_bar_i
  double *Pb, *Wb, *T0, *T1, *Pi, *Zf, *Zfb;
  float *va, *vb, *kr;  // fiber rows of the two other modes (m x q) and their Khatri-Rao product
  int* pc;              // q: one coordinate of each fiber
  long long krsz;
  double *tmp0, *tmp1;  // tmpsz each
  double* dX64;  // N
  double* part;  // partsz: split-K partial sums
  long long tmpsz, partsz;
};

// compressed S: tile geometry of the FP32 bulk-copy pass (false: the format does not apply), and
// the expansion of the last pass's compressed S into a dense tensor
bool compressed_geometry(const Geom& g, int& tile_rows);
cudaError_t launch_decode_s(const Geom& g, const Bufs& b, float* S_out, cudaStream_t s);
// off (rowsT + 1) = exclusive prefix of the rows' nonzero counts; then, when out is given, every
// nonzero in element order into out
cudaError_t launch_compact_s(const Geom& g, const Bufs& b, long long* off, float* out, cudaStream_t s);

// tensor-core (tcgen05) forms of the dense pass: kind 0 = BF16 split, 1 = TF32
size_t umma_smem(const Geom& g, int kind);  // 0 when the form does not apply
cudaError_t prepare_umma(const Geom& g, int kind);
cudaError_t launch_umma(const Geom& g, const Bufs& b, int kind, cudaStream_t s);

void backward_layout(const Geom& g, BwWork& w);
cudaError_t prepare_backward(int max_m);
cudaError_t launch_backward(const Geom& g, const Bufs& b, const BwWork& w, int K, const float* dL,
                            float* dX, cudaStream_t s);

// Raises (never lowers) a kernel's dynamic shared-memory limit. The limit is a property of the
// function, shared by every plan in the process, so plans that coexist (a batch, say) must not
// shrink one another's.
inline cudaError_t raise_smem_limit(const void* f, size_t bytes) {
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, f);
  if (e != cudaSuccess) return e;
  if ((size_t)a.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

enum { TK_SAMPLE = 0, TK_ERR = 1, TK_DENSE = 2, TK_MAXABS = 3, TK_DTILE = 4, TK_COUNT = 8 };

// ---------------------------------------------------------------- host launch wrappers
// Every wrapper launches on `s` and returns the launch error.
cudaError_t launch_setup(const Geom& g, const Bufs& b, double zeta0, int use_maxabs, cudaStream_t s);
cudaError_t launch_maxabs(const Geom& g, const Bufs& b, cudaStream_t s);
cudaError_t launch_gather_x(const Geom& g, const Bufs& b, cudaStream_t s);
cudaError_t launch_x_bf16(const Geom& g, const Bufs& b, const float* X, cudaStream_t s);
cudaError_t launch_sample_ht(const Geom& g, const Bufs& b, cudaStream_t s);
cudaError_t launch_gram(const Geom& g, const Bufs& b, cudaStream_t s);
cudaError_t launch_jacobi(const Geom& g, const Bufs& b, cudaStream_t s);
cudaError_t launch_refine(const Geom& g, const Bufs& b, int mode, cudaStream_t s);
cudaError_t launch_factor_B(const Geom& g, const Bufs& b, cudaStream_t s);
cudaError_t launch_core(const Geom& g, const Bufs& b, cudaStream_t s);
cudaError_t launch_table(const Geom& g, const Bufs& b, int next, cudaStream_t s);
cudaError_t launch_export_cur(const Geom& g, const Bufs& b, cudaStream_t s);
cudaError_t launch_sample_err(const Geom& g, const Bufs& b, cudaStream_t s);
cudaError_t launch_commit(const Geom& g, const Bufs& b, unsigned long long handle, int use_handle,
                          cudaStream_t s);
cudaError_t launch_batch_any(State* const* sts, int count, unsigned long long handle, cudaStream_t s);
cudaError_t launch_dense(const Geom& g, const Bufs& b, int form, cudaStream_t s);
cudaError_t prepare_dense(const Geom& g);  // kernel attributes of the dense pass (call at create)
cudaError_t prepare_sample_kernels();      // shared-memory carveout of the sampled chain's kernels
cudaError_t prepare_factor_kernels();
bool dense_form_supported(const Geom& g, int form);
cudaError_t launch_plain_dense(const Geom& g, const Bufs& b, cudaStream_t s);
cudaError_t launch_plain_prep(const Geom& g, const Bufs& b, cudaStream_t s);
cudaError_t launch_materialize(const Geom& g, const Bufs& b, float* L_out, float* S_out,
                               cudaStream_t s);
size_t jacobi_smem_bytes(int m);
cudaError_t prepare_jacobi(size_t smem);
cudaError_t prepare_refine(Geom& g, int want);  // cluster size (g.ncl) and shared-memory limit of the refinement

// ---------------------------------------------------------------- device helpers
#ifdef __CUDACC__
// Diagnostic phase timer (compiled in only with -DRTCUR_PHASE_TIMING): block 0, thread 0
// prints the clock64() distance since the previous mark.
#ifdef RTCUR_PHASE_TIMING
#include <cstdio>
#define PHASE_MARK(t0, name)                                                               \
  do {                                                                                     \
    if (blockIdx.x == 0 && threadIdx.x == 0) {                                             \
      long long t1_ = clock64();                                                           \
      printf("[phase] %s %lld\n", name, t1_ - t0);                                         \
      t0 = t1_;                                                                            \
    }                                                                                      \
  } while (0)
#else
#define PHASE_MARK(t0, name) do { (void)t0; } while (0)
#endif
// Diagnostic timeline (compiled in only with -DRTCUR_TIMELINE): block 0, thread 0 of a kernel
// appends (id, globaltimer at entry, globaltimer at exit) to a device log.
#ifdef RTCUR_TIMELINE
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
#define TL_BEGIN() unsigned long long tl_t0_ = gtimer()
#define TL_END(kid_)                                                               \
  do {                                                                             \
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && b.tl) {          \
      unsigned i_ = atomicAdd(b.tl_n, 1u);                                         \
      if (i_ < 4096) { b.tl[i_].id = kid_; b.tl[i_].t0 = tl_t0_; b.tl[i_].t1 = gtimer(); } \
    }                                                                              \
  } while (0)
#else
#define TL_BEGIN() do { } while (0)
#define TL_END(kid_) do { } while (0)
#endif
__device__ __forceinline__ int cur_copy(const State* st) { return st->k & 1; }

// Coordinates of sampled entry e under index set `set` (pointer to the set's first int64).
// Writes p[0..n-1]; returns the segment (0 = R, 1 + i = C_i).
__device__ __forceinline__ int sample_coords(const Geom& g, const long long* set, long long e,
                                             long long* p) {
  if (e < g.nR) {
    long long rem = e;
    for (int l = g.n - 1; l >= 0; --l) {
      long long a = rem % g.m[l];
      rem /= g.m[l];
      p[l] = set[g.ioff[l] + a];
    }
    return 0;
  }
  int i = 0;
  while (i + 1 < g.n && e >= g.seg[i + 2]) ++i;
  long long local = e - g.seg[i + 1];
  long long b = local / g.d[i];
  long long t = local - b * g.d[i];
  long long j = set[g.joff[i] + b];
  for (int l = g.n - 1; l >= 0; --l) {
    if (l == i) continue;
    p[l] = j % g.d[l];
    j /= g.d[l];
  }
  p[i] = t;
  return 1 + i;
}

// Row of T (row-major over modes 0..n-2) for coordinates p.
__device__ __forceinline__ long long table_row(const Geom& g, const long long* p) {
  long long row = 0;
  for (int l = 0; l < g.n - 1; ++l) row = row * g.d[l] + p[l];
  return row;
}

// L(p) = sum_c T[row, c] * B_n[col, c], FP32 FMA in ascending c.
__device__ __forceinline__ float eval_L(const float* __restrict__ T, const float* __restrict__ Bn,
                                        int rn, long long row, long long col) {
  const float* t = T + row * rn;
  const float* bb = Bn + col * rn;
  float acc = 0.f;
  for (int c = 0; c < rn; ++c) acc = fmaf(__ldg(t + c), __ldg(bb + c), acc);
  return acc;
}

// Deterministic last-block reduction helper: every block stores its partials, the last block to
// arrive (ticket) gets true. Caller must __syncthreads() before and use the result uniformly.
__device__ __forceinline__ bool last_block_arrive(unsigned* ticket) {
  __shared__ bool amLast;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(ticket, 1u);
    amLast = (t == gridDim.x * gridDim.y - 1);
  }
  __syncthreads();
  return amLast;
}
#endif
