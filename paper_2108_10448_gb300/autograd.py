"""torch.autograd.Function over the C ABI: L^(K) = RTCUR_K(X) with the hand-written adjoint.

Forward: K iterations of Algorithm 1 (sampled scope) through rtcur_begin / rtcur_iterate /
rtcur_finish on the current CUDA stream, recording each iteration's sampled values and HT masks
(the plan must be created with options.checkpoint >= K). Backward: rtcur_backward, the reverse
sweep through the Fiber CUR updates and the truncated pseudoinverses with the masks frozen.
Argument marshalling only: every step runs in librtcur.so."""
from __future__ import annotations

import torch

from . import rtcur as rt


class RTCURUnrolled(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, plan, idx, K):
        if not X.is_cuda or X.dtype != torch.float32:
            raise TypeError("X must be a float32 CUDA tensor")
        X = X.contiguous()
        L = torch.empty_like(X)
        s = torch.cuda.current_stream(X.device).cuda_stream
        rt.rtcur_begin(plan, X.data_ptr(), idx, 0, s)
        rt.rtcur_iterate(plan, int(K), s)
        rt.rtcur_finish(plan, L.data_ptr(), 0, s, max_iter=int(K))
        ctx.plan = plan
        ctx.save_for_backward(X)  # the plan's recorded pass refers to this X
        return L

    @staticmethod
    def backward(ctx, dL):
        dL = dL.contiguous().to(torch.float32)
        dX = torch.empty_like(dL)
        s = torch.cuda.current_stream(dL.device).cuda_stream
        rt.rtcur_backward(ctx.plan, dL.data_ptr(), dX.data_ptr(), s)
        return dX, None, None, None


def rtcur_unrolled(X, plan, idx, K):
    """L^(K) of K unrolled RTCUR iterations, differentiable with respect to X."""
    return RTCURUnrolled.apply(X, plan, idx, K)
