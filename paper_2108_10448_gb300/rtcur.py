"""Thin ctypes binding of librtcur.so (argument marshalling only; every step runs in the CUDA
library). Entry points keep the C names of include/rtcur.h. Device buffers are passed as
integer addresses (``tensor.data_ptr()`` of a CUDA tensor) and streams as ``cudaStream_t``
integers (``torch.cuda.current_stream().cuda_stream``)."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, os.environ.get("RTCUR_LIB", "librtcur.so"))

OK, NOT_CONVERGED, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, EDEVICE = 0, 1, -1, -2, -3, -4, -5, -6
VARIANT_F, VARIANT_R = 0, 1
SCOPE_SAMPLED, SCOPE_FULL = 0, 1
FORM_FP32, FORM_FP32_PLAIN, FORM_BF16, FORM_TF32 = 0, 1, 2, 3
FLAG_RANK_DEFICIENT, FLAG_TIE = 1, 2
S_DENSE, S_COMPRESSED = 0, 1
SAMPLE_X_FP32, SAMPLE_X_BF16 = 0, 1


class rtcur_options(C.Structure):
    _fields_ = [("scope", C.c_int32), ("dense_form", C.c_int32), ("refine_steps", C.c_int32),
                ("jacobi_max_sweeps", C.c_int32), ("inband_rel", C.c_double),
                ("eig_method", C.c_int32), ("checkpoint", C.c_int32), ("refine_cluster", C.c_int32), ("s_format", C.c_int32),
                ("sample_x", C.c_int32), ("dense_ctas", C.c_int32), ("reserved", C.c_int32 * 2)]


class rtcur_s_compressed(C.Structure):
    _fields_ = [("mask", C.c_void_p), ("vals", C.c_void_p), ("nnz", C.c_int64), ("rows", C.c_int64),
                ("cols", C.c_int64), ("words_per_row", C.c_int64), ("block_cols", C.c_int64)]


class rtcur_result(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("flags", C.c_int32),
                ("jacobi_sweeps", C.c_int32), ("e", C.c_double), ("zeta", C.c_double),
                ("nnz_sample", C.c_int64), ("inband_sample", C.c_int64),
                ("nnz_full", C.c_int64), ("inband_full", C.c_int64), ("resid_full", C.c_double),
                ("warm_hits", C.c_int64),
                ("e_hist", C.POINTER(C.c_double)), ("zeta_hist", C.POINTER(C.c_double)),
                ("nnz_hist", C.POINTER(C.c_int64))]


class RTCURError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"rtcur status {status}: {msg}")
        self.status = status


_lib = None


def load(path=LIB_PATH):
    """Load librtcur.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2108_10448_gb300/build.py")
    lib = C.CDLL(path)
    P = C.c_void_p
    lib.rtcur_create.argtypes = [C.POINTER(P), C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                 C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.c_double, C.c_double,
                                 C.c_double, C.c_int32, C.c_int32, C.POINTER(rtcur_options)]
    lib.rtcur_solve.argtypes = [P, P, C.POINTER(C.c_int64), P, P, C.POINTER(rtcur_result), P]
    lib.rtcur_begin.argtypes = [P, P, C.POINTER(C.c_int64), P, P]
    lib.rtcur_iterate.argtypes = [P, C.c_int32, P]
    lib.rtcur_finish.argtypes = [P, P, P, C.POINTER(rtcur_result), P]
    lib.rtcur_threshold_dense.argtypes = [P, C.c_int32, P]
    lib.rtcur_backward.argtypes = [P, P, P, P]
    lib.rtcur_solve_batched.argtypes = [C.POINTER(P), C.c_int32, C.POINTER(P), C.POINTER(P),
                                        C.POINTER(P), C.POINTER(P), P, P]
    lib.rtcur_threshold_dense_noalloc.argtypes = [C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                                  P, P, P, C.c_double, P, C.POINTER(C.c_double), P]
    lib.rtcur_threshold_dense_noalloc.restype = C.c_int
    lib.rtcur_get_factors.argtypes = [P, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                      C.POINTER(C.c_int32), C.POINTER(C.c_double), P]
    lib.rtcur_get_cur.argtypes = [P, C.POINTER(C.c_float), C.POINTER(C.c_float), C.POINTER(C.c_double),
                                  C.POINTER(C.c_int32), P]
    lib.rtcur_get_s_compressed.argtypes = [P, C.POINTER(rtcur_s_compressed), P]
    lib.rtcur_decode_s.argtypes = [P, P, P]
    lib.rtcur_compact_s.argtypes = [P, P, P, P]
    lib.rtcur_set_wait_limit.argtypes = [P, C.c_int64, P]
    lib.rtcur_sample_count.argtypes = [P]
    lib.rtcur_sample_count.restype = C.c_int64
    lib.rtcur_last_error.argtypes = [P]
    lib.rtcur_last_error.restype = C.c_char_p
    lib.rtcur_destroy.argtypes = [P]
    lib.rtcur_destroy.restype = None
    for f in ("rtcur_create", "rtcur_solve", "rtcur_begin", "rtcur_iterate", "rtcur_finish",
              "rtcur_get_factors", "rtcur_get_cur", "rtcur_threshold_dense", "rtcur_backward", "rtcur_solve_batched",
              "rtcur_get_s_compressed", "rtcur_decode_s", "rtcur_compact_s", "rtcur_set_wait_limit"):
        getattr(lib, f).restype = C.c_int
    _lib = lib
    return lib


def rtcur_last_error(plan=None):
    return load().rtcur_last_error(plan).decode()


def _check(status, plan=None, allow=(OK, NOT_CONVERGED)):
    if status not in allow:
        raise RTCURError(status, rtcur_last_error(plan))
    return status


def _i64(xs):
    return (C.c_int64 * len(xs))(*[int(x) for x in xs])


def _i32(xs):
    return (C.c_int32 * len(xs))(*[int(x) for x in xs])


EIG_TRIDIAGONAL, EIG_JACOBI = 0, 1


def make_options(scope=SCOPE_SAMPLED, dense_form=FORM_FP32, refine_steps=2, jacobi_max_sweeps=30,
                 inband_rel=1e-6, eig_method=EIG_TRIDIAGONAL, checkpoint=0, refine_cluster=0,
                 s_format=S_DENSE, sample_x=SAMPLE_X_FP32, dense_ctas=0):
    o = rtcur_options()
    o.scope, o.dense_form, o.refine_steps = scope, dense_form, refine_steps
    o.jacobi_max_sweeps, o.inband_rel, o.eig_method = jacobi_max_sweeps, inband_rel, eig_method
    o.checkpoint = checkpoint
    o.refine_cluster = refine_cluster
    o.s_format = s_format
    o.sample_x = sample_x
    o.dense_ctas = dense_ctas
    return o


def rtcur_create(dims, ranks, nI, nJ, zeta0, gamma, tol, max_iter, variant=VARIANT_F,
                 options=None):
    """Create a plan; returns its handle (an int). Raises RTCURError on failure."""
    lib = load()
    h = C.c_void_p()
    n = len(dims)
    st = lib.rtcur_create(C.byref(h), n, _i64(dims), _i32(ranks), _i32(nI), _i32(nJ),
                          float(zeta0), float(gamma), float(tol), int(max_iter), int(variant),
                          C.byref(options) if options is not None else None)
    _check(st, None, allow=(OK,))
    return h.value


def _idx_ptr(idx):
    arr = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    return arr, arr.ctypes.data_as(C.POINTER(C.c_int64))


class Result:
    def __init__(self, r, e_hist, z_hist, n_hist, status):
        k = r.iters
        self.status = status
        self.iters = k
        self.flags = r.flags
        self.jacobi_sweeps = r.jacobi_sweeps
        self.e = r.e
        self.zeta = r.zeta
        self.nnz_sample = r.nnz_sample
        self.inband_sample = r.inband_sample
        self.nnz_full = r.nnz_full
        self.inband_full = r.inband_full
        self.resid_full = r.resid_full
        self.warm_hits = r.warm_hits
        self.e_hist = e_hist[:min(k, e_hist.size)].copy()
        self.zeta_hist = z_hist[:min(k, z_hist.size)].copy()
        self.nnz_hist = n_hist[:min(k, n_hist.size)].copy()


def _result_struct(max_iter):
    e = np.zeros(max_iter, np.float64)
    z = np.zeros(max_iter, np.float64)
    nn = np.zeros(max_iter, np.int64)
    r = rtcur_result()
    r.e_hist = e.ctypes.data_as(C.POINTER(C.c_double))
    r.zeta_hist = z.ctypes.data_as(C.POINTER(C.c_double))
    r.nnz_hist = nn.ctypes.data_as(C.POINTER(C.c_int64))
    return r, e, z, nn


def rtcur_solve(plan, X_ptr, idx, L_ptr=0, S_ptr=0, stream=0, max_iter=1000):
    """Run Algorithm 1 to completion. Pointers are device addresses (0 = NULL)."""
    lib = load()
    arr, ip = _idx_ptr(idx)
    r, e, z, nn = _result_struct(max_iter)
    st = lib.rtcur_solve(plan, X_ptr, ip, L_ptr or None, S_ptr or None, C.byref(r), stream or None)
    _check(st, plan)
    return Result(r, e, z, nn, st)


def rtcur_begin(plan, X_ptr, idx, S_work_ptr=0, stream=0):
    arr, ip = _idx_ptr(idx)
    _check(load().rtcur_begin(plan, X_ptr, ip, S_work_ptr or None, stream or None), plan)


def rtcur_iterate(plan, n_iter, stream=0):
    _check(load().rtcur_iterate(plan, int(n_iter), stream or None), plan)


def rtcur_finish(plan, L_ptr=0, S_ptr=0, stream=0, max_iter=1000):
    r, e, z, nn = _result_struct(max_iter)
    st = load().rtcur_finish(plan, L_ptr or None, S_ptr or None, C.byref(r), stream or None)
    _check(st, plan)
    return Result(r, e, z, nn, st)


def rtcur_threshold_dense(plan, n_launch=1, stream=0):
    _check(load().rtcur_threshold_dense(plan, int(n_launch), stream or None), plan)


def rtcur_get_s_compressed(plan, stream=0):
    """The compressed S^(k) of a plan with s_format S_COMPRESSED: a dict of device addresses
    (mask, vals) and the layout fields of include/rtcur.h."""
    out = rtcur_s_compressed()
    _check(load().rtcur_get_s_compressed(plan, C.byref(out), stream or None), plan)
    return {f: getattr(out, f) for f, _ in rtcur_s_compressed._fields_}


def rtcur_compact_s(plan, vals_out=0, row_off=0, stream=0):
    """All nonzeros of the compressed S^(k) in element order into the device buffer vals_out
    (>= nnz floats) and/or the rows' exclusive prefix into row_off (rows + 1 int64)."""
    _check(load().rtcur_compact_s(plan, vals_out or None, row_off or None, stream or None), plan)


def rtcur_decode_s(plan, S_out, stream=0):
    """Expand the compressed S^(k) into the dense device buffer at address S_out."""
    _check(load().rtcur_decode_s(plan, S_out, stream or None), plan)


def rtcur_solve_batched(plans, X_ptrs, idxs, L_ptrs=None, S_ptrs=None, stream=0, max_iter=1000):
    """Solve len(plans) problems in one graph launch. Returns one Result per problem."""
    lib = load()
    n = len(plans)
    P = C.c_void_p
    pa = (P * n)(*plans)
    xa = (P * n)(*X_ptrs)
    keep = [_idx_ptr(ix) for ix in idxs]
    ia = (P * n)(*[C.cast(ip, P) for _, ip in keep])
    la = (P * n)(*(L_ptrs or [0] * n)) if L_ptrs else None
    sa = (P * n)(*(S_ptrs or [0] * n)) if S_ptrs else None
    structs = [_result_struct(max_iter) for _ in range(n)]
    ra = (rtcur_result * n)(*[s[0] for s in structs])
    st = lib.rtcur_solve_batched(pa, n, xa, ia, la, sa, C.cast(ra, P), stream or None)
    _check(st, plans[0])
    return [Result(ra[i], *structs[i][1:], ra[i].status) for i in range(n)]


def rtcur_backward(plan, dL_ptr, dX_ptr, stream=0):
    """dX = (dL^(K)/dX)^T dL for the last solve of a plan created with options.checkpoint >= K
    (device pointers; masks of the thresholding frozen at their forward values)."""
    _check(load().rtcur_backward(plan, dL_ptr, dX_ptr, stream or None), plan, allow=(OK,))


def rtcur_threshold_dense_noalloc(dims, ranks, G_ptr, B_ptr, X_ptr, zeta, S_ptr, stream=0,
                                  want_counts=True):
    """Allocation-free dense threshold pass S = HT_zeta(X - G x_i B_i) (device pointers). For
    callers that cannot allocate device memory; its scratch is a fixed array inside the library.
    Returns (resid, nnz, band) when want_counts, else None."""
    counts = (C.c_double * 3)()
    st = load().rtcur_threshold_dense_noalloc(len(dims), _i64(dims), _i32(ranks), G_ptr, B_ptr, X_ptr,
                                              float(zeta), S_ptr, counts if want_counts else None,
                                              stream or None)
    if st != OK:
        raise RTCURError(st, "rtcur_threshold_dense_noalloc failed")
    return (counts[0], int(counts[1]), int(counts[2])) if want_counts else None


def rtcur_get_factors(plan, dims, ranks, stream=0):
    """Return (G, [B_1..B_n], k, zeta) of the current L^(k) = G x_i B_i (FP32 host arrays)."""
    nG = int(np.prod(ranks))
    sumB = int(sum(int(d) * int(r) for d, r in zip(dims, ranks)))
    G = np.zeros(nG, np.float32)
    B = np.zeros(sumB, np.float32)
    k = C.c_int32()
    z = C.c_double()
    _check(load().rtcur_get_factors(plan, G.ctypes.data_as(C.POINTER(C.c_float)),
                                    B.ctypes.data_as(C.POINTER(C.c_float)), C.byref(k), C.byref(z),
                                    stream or None), plan)
    Bs, off = [], 0
    for d, r in zip(dims, ranks):
        Bs.append(B[off:off + d * r].reshape(d, r))
        off += d * r
    return G.reshape(tuple(ranks)), Bs, k.value, z.value


def rtcur_get_cur(plan, dims, nI, nJ, stream=0):
    """Algorithm 1's output for the current iterate: (R, [C_1..C_n], [U_1^+..U_n^+], k) with
    R (|I_1| x ... x |I_n|, FP32), C_i (d_i x |J_i|, FP32) and U_i^+ (|J_i| x |I_i|, FP64), host
    arrays, so that L^(k) = R x_i (C_i U_i^+)."""
    n = len(dims)
    R = np.zeros(int(np.prod(nI)), np.float32)
    Cf = np.zeros(int(sum(int(d) * int(q) for d, q in zip(dims, nJ))), np.float32)
    U = np.zeros(int(sum(int(q) * int(m) for q, m in zip(nJ, nI))), np.float64)
    k = C.c_int32()
    _check(load().rtcur_get_cur(plan, R.ctypes.data_as(C.POINTER(C.c_float)),
                                Cf.ctypes.data_as(C.POINTER(C.c_float)),
                                U.ctypes.data_as(C.POINTER(C.c_double)), C.byref(k), stream or None), plan)
    Cs, Us, oc, ou = [], [], 0, 0
    for i in range(n):
        d, q, m = int(dims[i]), int(nJ[i]), int(nI[i])
        Cs.append(Cf[oc:oc + d * q].reshape(d, q))
        Us.append(U[ou:ou + q * m].reshape(q, m))
        oc += d * q
        ou += q * m
    return R.reshape(tuple(int(m) for m in nI)), Cs, Us, k.value


def rtcur_set_wait_limit(plan, polls, stream=0):
    """Bound (in polls; 0 = default) on the waits of the plan's FP32 dense threshold pass."""
    _check(load().rtcur_set_wait_limit(plan, int(polls), stream or None), plan, allow=(OK,))


def rtcur_sample_count(plan):
    return load().rtcur_sample_count(plan)


def rtcur_destroy(plan):
    if plan:
        load().rtcur_destroy(plan)
