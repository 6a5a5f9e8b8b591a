"""torch.autograd.Function around the variable-diffusivity path.

    uT = VarcoefHeat.apply(u0, kappa, c, steps, every)

forward runs `steps` flux-form FTCS steps of u0 with diffusivity kappa on the
library's kernels and keeps a checkpoint tape (the state every `every` steps,
0 = ceil(sqrt(steps))); backward runs the library's discrete adjoint from that
tape (each segment recomputed from its checkpoint, no second forward pass)
seeded with the incoming gradient dL/du^T and returns dL/du0 and dL/dkappa.
c = dt/h^2 is a fixed parameter.  Tensors must be contiguous float64 CUDA
tensors of shape (ny, nx); PyTorch only provides their memory and the current
stream, every arithmetic step runs in libhxc.so.
"""
import ctypes

import torch

from . import hxc

_dev = None


def _device():
    global _dev
    if _dev is None:
        devs = hxc.get_all_devices(2, 0)
        if not devs:
            raise RuntimeError("no CUDA device for the heat-stencil library")
        _dev = devs[torch.cuda.current_device() % len(devs)]
    return _dev


def _wrap(dev, t):
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return dev.wrap(t.data_ptr(), t.numel() * 8)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _after_torch(dev):
    """A future for the work already queued on torch's current stream."""
    out = hxc.c_fut()
    hxc.check(hxc.lib().hxc_future_from_stream(dev.h, _stream(), ctypes.byref(out)))
    return hxc.Future(out.value)


def _torch_waits(fut):
    """Torch's current stream waits (on the device) for a library future."""
    hxc.check(hxc.lib().hxc_future_stream_wait(fut.h, _stream()))


class VarcoefHeat(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, kappa, c, steps, every=0):
        dev = _device()
        ny, nx = u0.shape
        uT = torch.empty_like(u0)
        tape = torch.empty((hxc.varcoef_tape_states(int(steps), int(every)), ny, nx),
                           dtype=torch.float64, device=u0.device)
        f, _ = hxc.varcoef_forward_tape(dev, _wrap(dev, u0), _wrap(dev, kappa), ny, nx, float(c),
                                        int(steps), _wrap(dev, uT), _wrap(dev, tape),
                                        every=int(every), deps=[_after_torch(dev)])
        _torch_waits(f)
        ctx.save_for_backward(tape, kappa)
        ctx.c, ctx.steps, ctx.every = float(c), int(steps), int(every)
        return uT

    @staticmethod
    def backward(ctx, grad_uT):
        tape, kappa = ctx.saved_tensors
        dev = _device()
        ny, nx = kappa.shape
        lamT = grad_uT.contiguous()
        gk = torch.empty_like(kappa)
        gu = torch.empty_like(kappa)
        f, _ = hxc.varcoef_adjoint_tape(dev, _wrap(dev, tape), _wrap(dev, kappa), _wrap(dev, lamT),
                                        ny, nx, ctx.c, ctx.steps, _wrap(dev, gk), _wrap(dev, gu),
                                        every=ctx.every, deps=[_after_torch(dev)])
        _torch_waits(f)
        return gu, gk, None, None, None
