"""Compressed S output of the FULL scope (s_format COMPRESSED, GPU only).

The compressed pass runs the same iteration as the dense FP32 form, so the iterates, L and the
decoded S must equal the dense form's bit for bit. The layout of include/rtcur.h is checked by
an independent host decoder (numpy) of the exported mask and per-block value runs, and by the
compaction (all nonzeros in element order with the rows' exclusive prefix). One shape is
also compared with the FP64 oracle directly. Shapes cover d_n below, at and above a multiple of
32 (ragged mask words), a ragged last tile, a 4-mode tensor and an empty S."""
import numpy as np
import pytest

from oracle import rtcur_oracle as O
from paper_2108_10448_gb300 import rtcur as rt
from paper_2108_10448_gb300 import synth

from gpu_helpers import rel_fro, run_gpu, support_mismatch

pytestmark = pytest.mark.gpu

SHAPES = [
    # dims, ranks, alpha
    ((60, 52, 44), (3, 3, 3), 0.2),      # d_n = 44: two mask words per row, the second ragged
    ((30, 24, 128), (2, 3, 2), 0.3),     # d_n one 128-column block; rows 720 = 11.25 tiles of 64
    ((20, 18, 16, 20), (2, 2, 2, 2), 0.1),
    ((12, 10, 300), (2, 2, 3), 0.3),     # d_n = 300: blocks of 128, 128 and 44 columns
    ((40, 36, 8), (2, 2, 2), 0.1),       # one word per row, 8 of its 32 bits used
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as ge
    ge.build()


def _device_array(ptr, n, typestr):
    import torch

    class _Cai:
        __cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr), False),
                                    "version": 3, "strides": None}
    return torch.as_tensor(_Cai(), device="cuda:0").cpu().numpy().copy()


def host_decode(c):
    """Dense S from the compressed layout, written from the header's description alone."""
    rows, cols, wpr, bc = c["rows"], c["cols"], c["words_per_row"], c["block_cols"]
    assert bc == 128
    mask = _device_array(c["mask"], rows * wpr, "<u4").reshape(rows, wpr)
    vals = _device_array(c["vals"], rows * cols, "<f4").reshape(rows, cols)
    bits = ((mask[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(bool).reshape(rows, wpr * 32)
    assert not bits[:, cols:].any(), "bits set beyond d_n"
    bits = bits[:, :cols]
    S = np.zeros((rows, cols), np.float32)
    for k0 in range(0, cols, bc):
        blk = bits[:, k0:k0 + bc]
        cnt = blk.sum(axis=1)
        for r in np.nonzero(cnt)[0]:
            run = vals[r, k0:k0 + cnt[r]]
            assert np.all(run != 0)
            S[r, k0:k0 + bc][blk[r]] = run
    assert int(bits.sum()) == c["nnz"]
    return S


def _solve(p, sets, max_iter, s_format, keep_plan=False):
    import torch
    dev = torch.device("cuda:0")
    X = torch.from_numpy(np.ascontiguousarray(p.X)).to(dev)
    L = torch.empty_like(X)
    S = torch.full_like(X, np.nan)
    o = rt.make_options(scope=rt.SCOPE_FULL, s_format=s_format)
    plan = rt.rtcur_create(p.dims, p.ranks, p.m, p.q, p.zeta0, p.gamma, p.tol, max_iter, rt.VARIANT_F, o)
    stream = torch.cuda.current_stream().cuda_stream
    res = rt.rtcur_solve(plan, X.data_ptr(), synth.pack_index_sets(sets), L.data_ptr(), S.data_ptr(),
                         stream, max_iter=max_iter)
    out = (res, L.cpu().numpy(), S.cpu().numpy())
    if keep_plan:
        return out + (plan, X)
    rt.rtcur_destroy(plan)
    return out


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s[0])))
def test_compressed_equals_dense_form(shape):
    import torch
    dims, ranks, alpha = shape
    p = synth.make_tucker_problem(dims, ranks, alpha, 3.0, seed=41, max_iter=40)
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=41)
    rd, Ld, Sd = _solve(p, sets, 40, rt.S_DENSE)
    rc, Lc, Sc, plan, X = _solve(p, sets, 40, rt.S_COMPRESSED, keep_plan=True)
    try:
        assert rc.iters == rd.iters > 0
        np.testing.assert_array_equal(rc.e_hist[:rc.iters], rd.e_hist[:rd.iters])
        np.testing.assert_array_equal(Lc, Ld)
        np.testing.assert_array_equal(Sc, Sd)           # decoded by rtcur_finish
        assert rc.nnz_full == rd.nnz_full == int(np.count_nonzero(Sd))
        c = rt.rtcur_get_s_compressed(plan, torch.cuda.current_stream().cuda_stream)
        assert c["nnz"] == rc.nnz_full
        assert c["rows"] * c["cols"] == Sd.size and c["words_per_row"] == (dims[-1] + 31) // 32
        Sh = host_decode(c)
        np.testing.assert_array_equal(Sh.reshape(Sd.shape), Sd)
        S2 = torch.full_like(X, np.nan)
        rt.rtcur_decode_s(plan, S2.data_ptr(), torch.cuda.current_stream().cuda_stream)
        np.testing.assert_array_equal(S2.cpu().numpy(), Sd)
        # compaction: every nonzero in element order, and the rows' exclusive prefix (CSR)
        v = torch.full((max(c["nnz"], 1),), np.nan, dtype=torch.float32, device=X.device)
        off = torch.full((c["rows"] + 1,), -1, dtype=torch.int64, device=X.device)
        rt.rtcur_compact_s(plan, v.data_ptr(), off.data_ptr(), torch.cuda.current_stream().cuda_stream)
        flat = Sd.ravel()
        np.testing.assert_array_equal(v.cpu().numpy()[:c["nnz"]], flat[flat != 0])
        per_row = np.count_nonzero(Sd.reshape(c["rows"], c["cols"]), axis=1)
        np.testing.assert_array_equal(off.cpu().numpy(), np.concatenate([[0], np.cumsum(per_row)]))
    finally:
        rt.rtcur_destroy(plan)


def test_compressed_matches_oracle():
    p = synth.make_tucker_problem((48, 40, 36), (2, 2, 2), 0.2, 3.0, seed=43, max_iter=60)
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=43)
    ref = O.rtcur(p.X, p.ranks, sets, p.zeta0, p.gamma, p.tol, 60, "F", keep_full=True)
    res, L, S = run_gpu(p, sets, "F", scope=rt.SCOPE_FULL, max_iter=60, s_format=rt.S_COMPRESSED)
    assert res.iters == ref["iters"]
    np.testing.assert_allclose(res.e_hist[:res.iters], ref["hist"]["e"], rtol=1e-4, atol=2e-7)
    assert rel_fro(L, ref["L"]) <= 1e-5
    inb, outb = support_mismatch(S, ref, p.X)
    if outb:
        # only where the FP32 evaluation of L^(k-1) explains the flip (as in the dense-form tests)
        _, Lprev, _ = run_gpu(p, sets, "F", scope=rt.SCOPE_FULL, max_iter=ref["iters"] - 1, want_S=False,
                              s_format=rt.S_COMPRESSED)
        Lor = ref["prev_state"].full(p.dims)
        dist = np.abs(np.abs(p.X.astype(np.float64) - Lor) - ref["zeta"])
        diff = (S != 0) != (ref["S"] != 0)
        assert int(np.count_nonzero(diff & (dist > 1e-6 * ref["zeta"] + np.abs(Lprev - Lor)))) == 0


def test_no_pass_means_empty_s():
    import torch
    p = synth.make_tucker_problem((30, 28, 24), (2, 2, 2), 0.1, 3.0, seed=44, tol=1.0, max_iter=10)
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=44)
    res, L, S, plan, X = _solve(p, sets, 10, rt.S_COMPRESSED, keep_plan=True)
    try:
        assert res.iters == 0 and np.all(S == 0.0)
        with pytest.raises(rt.RTCURError) as ei:
            rt.rtcur_get_s_compressed(plan, torch.cuda.current_stream().cuda_stream)
        assert ei.value.status == rt.EINVAL
    finally:
        rt.rtcur_destroy(plan)
