"""torch.autograd.Function over the engine's hand-written amplitude-loss
adjoint (epie_amp_loss_grad in include/epie.h).

    L = sum_j || |F(S_dj P . O_j)| - sqrt(I_j) ||^2

The forward call runs the CUDA kernel once and returns the loss together with
the gradients for the object, the probe and the sub-pixel position offsets;
backward scales them by the incoming gradient.  Nothing is kept per position
(the far field is recomputed inside the kernel), so memory stays at the size
of the parameters.  PyTorch only provides the device tensors and the stream.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _binding as B

_DTYPES = {torch.int16: B.EPIE_U16, torch.uint16: B.EPIE_U16, torch.float16: B.EPIE_F16,
           torch.float32: B.EPIE_F32}


def frames_to_fft_order(frames: torch.Tensor) -> torch.Tensor:
    """DC-centred detector frames [n, N, N] on the device -> FFT order, by the
    engine's ingest kernel.  uint16 data may be passed as int16 (same bits)."""
    frames = frames.contiguous()
    out = torch.empty_like(frames)
    n, N = frames.shape[0], frames.shape[-1]
    B.epie_frames_to_fft_order(frames.data_ptr(), out.data_ptr(), n, N, _DTYPES[frames.dtype],
                               torch.cuda.current_stream(frames.device).cuda_stream)
    return out


class AmplitudeLoss(torch.autograd.Function):
    """loss = AmplitudeLoss.apply(obj, probe, shift, frames_fft, pos).

    obj [H, W] and probe [N, N] complex64, shift [n, 2] float32 (dy, dx) or
    None, frames_fft [n, N, N] in FFT order (int16-viewed uint16, float16 or
    float32), pos [n, 2] int32 patch top-left positions; all on one CUDA
    device.  Returns a float64 scalar tensor on that device."""

    @staticmethod
    def forward(ctx, obj, probe, shift, frames_fft, pos):
        dev = obj.device
        N, n = probe.shape[-1], pos.shape[0]
        obj_c, probe_c = obj.contiguous(), probe.contiguous()
        g_obj = torch.empty_like(obj_c)
        g_probe = torch.empty_like(probe_c)
        g_shift = None if shift is None else torch.empty(n, 2, dtype=torch.float32, device=dev)
        scratch = torch.empty(B.epie_amp_grad_scratch_bytes(N, n), dtype=torch.uint8, device=dev)
        a = B.epie_amp_grad_args()
        a.N, a.intensity_dtype = N, _DTYPES[frames_fft.dtype]
        a.obj_h, a.obj_w, a.n = obj_c.shape[0], obj_c.shape[1], n
        a.object, a.probe = obj_c.data_ptr(), probe_c.data_ptr()
        a.frames, a.pos = frames_fft.contiguous().data_ptr(), pos.contiguous().data_ptr()
        shift_c = None if shift is None else shift.contiguous()
        a.shift = None if shift_c is None else shift_c.data_ptr()
        a.grad_object, a.grad_probe = g_obj.data_ptr(), g_probe.data_ptr()
        a.grad_shift = None if g_shift is None else g_shift.data_ptr()
        a.scratch, a.scratch_bytes = scratch.data_ptr(), scratch.numel()
        a.stream = torch.cuda.current_stream(dev).cuda_stream
        loss = B.epie_amp_loss_grad(a)
        ctx.save_for_backward(g_obj, g_probe, g_shift if g_shift is not None else torch.empty(0))
        ctx.has_shift = shift is not None
        return torch.tensor(loss, dtype=torch.float64, device=dev)

    @staticmethod
    def backward(ctx, grad_out):
        g_obj, g_probe, g_shift = ctx.saved_tensors
        s = grad_out.to(torch.float32)
        gs = g_shift * s if ctx.has_shift else None
        return g_obj * s, g_probe * s, gs, None, None


def amplitude_loss(obj, probe, shift, frames_fft, pos):
    return AmplitudeLoss.apply(obj, probe, shift, frames_fft, pos)
