"""torch.autograd.Function over the library's travel-time kernel.

forward(src, rcv) returns T(src; rcv) for P pairs (FP32, T_hi + T_lo rounded);
backward(dL/dT) returns dL/dsrc = dL/dT * dT/dsrc, where dT/dsrc comes from
the same fused launch (reverse sweep through the MLP, Sec. 3.2).  The Jacobian
(16 B per pair) is kept for backward, or, when it would not fit in the free
device memory with headroom to spare, recomputed by a second launch."""
from __future__ import annotations

import torch

from .binding import FP32, Net, NetDevice


def _pack4(x: torch.Tensor) -> torch.Tensor:
    out = torch.zeros(x.shape[0], 4, device=x.device, dtype=torch.float32)
    out[:, :3] = x
    return out


class TravelTime(torch.autograd.Function):
    @staticmethod
    def forward(ctx, src, rcv, netdev: NetDevice, recompute: str = "auto"):
        assert src.is_cuda and rcv.is_cuda and src.shape == rcv.shape and src.shape[1] == 3
        P = src.shape[0]
        s4, r4 = _pack4(src.detach()), _pack4(rcv.detach())
        T = torch.empty(P, device=src.device, dtype=torch.float32)
        Tlo = torch.empty(P, device=src.device, dtype=torch.float32)
        need_grad = ctx.needs_input_grad[0]
        if recompute == "auto":
            free, _ = torch.cuda.mem_get_info(src.device)
            recompute_now = P * 16 > free // 4
        else:
            recompute_now = bool(recompute)
        J = None if (recompute_now or not need_grad) else torch.empty(P, 4, device=src.device)
        stream = torch.cuda.current_stream(src.device).cuda_stream
        netdev.spider_tt_pairs(P, s4.data_ptr(), r4.data_ptr(), T.data_ptr(), Tlo.data_ptr(),
                               J.data_ptr() if J is not None else 0, stream)
        ctx.netdev = netdev
        ctx.recompute = J is None and need_grad
        if J is not None:
            ctx.save_for_backward(J)
        else:
            ctx.save_for_backward(s4, r4)
        return T + Tlo

    @staticmethod
    def backward(ctx, gT):
        if ctx.recompute:
            s4, r4 = ctx.saved_tensors
            P = s4.shape[0]
            T = torch.empty(P, device=s4.device)
            J = torch.empty(P, 4, device=s4.device)
            stream = torch.cuda.current_stream(s4.device).cuda_stream
            ctx.netdev.spider_tt_pairs(P, s4.data_ptr(), r4.data_ptr(), T.data_ptr(), 0,
                                       J.data_ptr(), stream)
        else:
            (J,) = ctx.saved_tensors
        return gT[:, None] * J[:, :3], None, None, None


def travel_time(src, rcv, netdev: NetDevice, recompute: str = "auto"):
    return TravelTime.apply(src, rcv, netdev, recompute)
