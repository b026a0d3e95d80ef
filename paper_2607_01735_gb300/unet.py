"""Binding of the learned-initial-guess network (C ABI in include/rbgs_unet.h).

Argument marshalling only: the convolutions, pooling, upsampling, loss, backward pass
and Adam update all run in the library's CUDA kernels.  Tensors are torch CUDA
tensors; bf16 operands are passed as torch.bfloat16 tensors (their uint16 bit
patterns).  `network_input` assembles the four input channels (f, boundary mask,
boundary values, boundary interpolation) of one Poisson problem on an H x W grid padded
to a multiple of 8.
"""
from __future__ import annotations

import ctypes

import torch

from . import _check, load_library

_bound = False


def _lib():
    global _bound
    lib = load_library()
    if not _bound:
        vp, ci, cf = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
        lib.rbgs_conv_forward.argtypes = [vp, vp, vp, vp, ci, ci, ci, ci, ci, ci, ci, ci, vp]
        lib.rbgs_conv_forward.restype = ci
        lib.rbgs_conv_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp, ci, ci, ci, ci, ci, ci, ci, vp]
        lib.rbgs_conv_backward.restype = ci
        lib.rbgs_unet_create.argtypes = [ctypes.c_uint64, vp, ctypes.POINTER(vp)]
        lib.rbgs_unet_create.restype = ci
        lib.rbgs_unet_num_params.argtypes = [vp]
        lib.rbgs_unet_num_params.restype = ctypes.c_long
        lib.rbgs_unet_get_params.argtypes = [vp, vp]
        lib.rbgs_unet_get_params.restype = ci
        lib.rbgs_unet_set_params.argtypes = [vp, vp]
        lib.rbgs_unet_set_params.restype = ci
        lib.rbgs_unet_forward.argtypes = [vp, vp, vp, ci, ci, ci]
        lib.rbgs_unet_forward.restype = ci
        lib.rbgs_unet_train_step.argtypes = [vp, vp, vp, vp, ci, ci, ci, cf, ctypes.POINTER(cf), vp]
        lib.rbgs_unet_train_step.restype = ci
        lib.rbgs_unet_destroy.argtypes = [vp]
        lib.rbgs_unet_destroy.restype = None
        lib.rbgs_conv_set_engine.argtypes = [ci]
        lib.rbgs_conv_set_engine.restype = ci
        lib.rbgs_conv_get_engine.argtypes = []
        lib.rbgs_conv_get_engine.restype = ci
        lib.rbgs_conv_check.argtypes = [vp]
        lib.rbgs_conv_check.restype = ci
        _bound = True
    return lib


def _p(t):
    if t is None:
        return None
    if not t.is_contiguous():
        raise TypeError("tensors must be contiguous")
    return t.data_ptr()


def _stream(t):
    return torch.cuda.current_stream(t.device).cuda_stream


RBGS_CONV_TCGEN05 = 0
RBGS_CONV_MMA_SYNC = 1
RBGS_CONV_TCGEN05_GATHER = 2


def rbgs_conv_set_engine(engine: int) -> None:
    """Selects the convolution engine process-wide: RBGS_CONV_TCGEN05 (tensor memory
    accumulators, TMA-loaded operands where the channels allow; default),
    RBGS_CONV_TCGEN05_GATHER (the same with cp.async-gathered operands) or
    RBGS_CONV_MMA_SYNC (warp-level tiles)."""
    _check(_lib().rbgs_conv_set_engine(int(engine)))


def rbgs_conv_get_engine() -> int:
    return int(_lib().rbgs_conv_get_engine())


def rbgs_conv_check(device=None) -> None:
    """Synchronises the current stream; raises RbgsError(RBGS_ETIMEOUT) if a tcgen05
    convolution gave up a bounded wait since the last check."""
    dev = torch.device("cuda") if device is None else torch.device(device)
    _check(_lib().rbgs_conv_check(torch.cuda.current_stream(dev).cuda_stream))


def rbgs_conv_forward(x, w, bias, y, relu=True):
    """x: B,H,W,Cin bf16; w: Cout,k,k,Cin bf16; bias fp32 or None; y: B,H,W,Cout bf16 or fp32."""
    B, H, W, Cin = x.shape
    Cout, k = w.shape[0], w.shape[1]
    _check(_lib().rbgs_conv_forward(_p(x), _p(w), _p(bias), _p(y), B, H, W, Cin, Cout, k, int(relu),
                                    int(y.dtype == torch.float32), _stream(x)))


def rbgs_conv_backward(x, w, g, dx, dw, db, accumulate=False):
    """Gradients of rbgs_conv_forward (no activation): dx fp32 or None, dw/db fp32 (added to)."""
    B, H, W, Cin = x.shape
    Cout, k = w.shape[0], w.shape[1]
    scratch = torch.empty(w.numel(), dtype=torch.bfloat16, device=x.device)
    _check(_lib().rbgs_conv_backward(_p(x), _p(w), _p(g), _p(dx), _p(dw), _p(db), _p(scratch), B, H, W, Cin,
                                     Cout, k, int(accumulate), _stream(x)))


def boundary_blend(u_ring):
    """Transfinite (Coons) interpolation of the ring values of an (N+2)^2 grid into its
    interior: the bilinearly blended sum of the four edge interpolants minus the corner
    bilinear term.  It reproduces boundary data that is linear in x and y exactly."""
    g = u_ring.shape[0]
    t = torch.linspace(0.0, 1.0, g, dtype=torch.float64, device=u_ring.device)
    x, y = t[:, None], t[None, :]
    u = u_ring.to(torch.float64)
    north, south = u[0:1, :], u[g - 1:g, :]
    west, east = u[:, 0:1], u[:, g - 1:g]
    c00, c01, c10, c11 = u[0, 0], u[0, g - 1], u[g - 1, 0], u[g - 1, g - 1]
    return ((1 - x) * north + x * south + (1 - y) * west + y * east
            - ((1 - x) * (1 - y) * c00 + (1 - x) * y * c01 + x * (1 - y) * c10 + x * y * c11))


def network_input(f, u_ring, size=None):
    """4-channel input of one problem: f on the interior, mask 1 on the Dirichlet ring,
    ring values, and boundary_blend of the ring; the (N+2)^2 grid zero-padded to `size`
    (default: multiple of 8)."""
    n = f.shape[0]
    g = n + 2
    size = size or (g + 7) // 8 * 8
    x = torch.zeros((size, size, 4), dtype=torch.float32, device=f.device)
    x[1:n + 1, 1:n + 1, 0] = f.to(torch.float32)
    ring = torch.ones((g, g), dtype=torch.bool, device=f.device)
    ring[1:n + 1, 1:n + 1] = False
    x[:g, :g, 1] = ring.to(torch.float32)
    x[:g, :g, 2] = torch.where(ring, u_ring.to(torch.float32), torch.zeros_like(u_ring, dtype=torch.float32))
    x[:g, :g, 3] = boundary_blend(u_ring).to(torch.float32)
    return x


class UNet:
    """Owning wrapper around rbgs_unet_t."""

    def __init__(self, seed: int = 0, device="cuda"):
        self.device = torch.device(device)
        h = ctypes.c_void_p()
        s = torch.cuda.current_stream(self.device).cuda_stream
        _check(_lib().rbgs_unet_create(ctypes.c_uint64(seed), s, ctypes.byref(h)))
        self.handle = h.value
        self.num_params = int(_lib().rbgs_unet_num_params(self.handle))

    def get_params(self) -> torch.Tensor:
        out = torch.empty(self.num_params, dtype=torch.float32, device=self.device)
        _check(_lib().rbgs_unet_get_params(self.handle, _p(out)))
        return out

    def set_params(self, params: torch.Tensor) -> None:
        params = params.to(device=self.device, dtype=torch.float32).contiguous()
        _check(_lib().rbgs_unet_set_params(self.handle, _p(params)))

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        """x: B,H,W,4 fp32 -> B,H,W fp32."""
        B, H, W, _ = x.shape
        x = x.contiguous()
        y = torch.empty((B, H, W), dtype=torch.float32, device=x.device)
        _check(_lib().rbgs_unet_forward(self.handle, _p(x), _p(y), B, H, W))
        return y

    def train_step(self, x, target, mask, lr: float = 1e-3, grads: torch.Tensor | None = None) -> float:
        B, H, W, _ = x.shape
        loss = ctypes.c_float()
        _check(_lib().rbgs_unet_train_step(self.handle, _p(x.contiguous()), _p(target.contiguous()),
                                           _p(mask.contiguous()), B, H, W, float(lr), ctypes.byref(loss),
                                           _p(grads)))
        return float(loss.value)

    def close(self):
        if self.handle:
            _lib().rbgs_unet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
