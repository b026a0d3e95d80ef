"""Binding of the learned-initial-guess network (C ABI in include/rbgs_unet.h).

Argument marshalling only: the convolutions, pooling, upsampling, loss, backward pass
and Adam update all run in the library's CUDA kernels.  Tensors are torch CUDA
tensors; bf16 operands are passed as torch.bfloat16 tensors (their uint16 bit
patterns).  The grid operations around the network (the input channels, the boundary
interpolation, the training target, the guess, the coarse-grid transfer) are the
library's kernels too (rbgs_guess_*); torch only holds the memory.
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
        lib.rbgs_conv_set_wgrad_kernel.argtypes = [ci]
        lib.rbgs_conv_set_wgrad_kernel.restype = ci
        lib.rbgs_conv_get_wgrad_kernel.argtypes = []
        lib.rbgs_conv_get_wgrad_kernel.restype = ci
        lib.rbgs_conv_check.argtypes = [vp]
        lib.rbgs_conv_check.restype = ci
        lib.rbgs_guess_blend.argtypes = [vp, ci, vp, vp]
        lib.rbgs_guess_input.argtypes = [vp, vp, ci, ci, vp, vp]
        lib.rbgs_guess_target.argtypes = [vp, vp, ci, ci, vp, vp]
        lib.rbgs_guess_assemble.argtypes = [vp, vp, ci, ci, vp, vp]
        lib.rbgs_guess_coarsen.argtypes = [vp, vp, ci, ci, vp, vp, vp]
        lib.rbgs_guess_refine.argtypes = [vp, ci, vp, ci, vp, vp]
        for name in ("rbgs_guess_blend", "rbgs_guess_input", "rbgs_guess_target", "rbgs_guess_assemble",
                     "rbgs_guess_coarsen", "rbgs_guess_refine"):
            getattr(lib, name).restype = ci
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


RBGS_WGRAD_AUTO = 0
RBGS_WGRAD_RING = 1
RBGS_WGRAD_TAPROW = 2
RBGS_WGRAD_GATHER = 3


def rbgs_conv_set_wgrad_kernel(kind: int) -> None:
    """Selects the 3x3 weight-gradient kernel of the tcgen05 engine process-wide:
    RBGS_WGRAD_AUTO (per layer, the fastest measured), RBGS_WGRAD_RING, RBGS_WGRAD_TAPROW or
    RBGS_WGRAD_GATHER."""
    _check(_lib().rbgs_conv_set_wgrad_kernel(int(kind)))


def rbgs_conv_get_wgrad_kernel() -> int:
    return int(_lib().rbgs_conv_get_wgrad_kernel())


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


def _dev64(t):
    """A contiguous float64 CUDA tensor (the grid kernels read device memory)."""
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError("expected a CUDA tensor")
    return t.to(torch.float64).contiguous()


def boundary_blend(u_ring):
    """Transfinite (Coons) interpolation of the ring values of an (N+2)^2 grid into its
    interior (rbgs_guess_blend): the bilinearly blended edge interpolants minus the corner
    bilinear term; it reproduces boundary data that is linear in x and y exactly."""
    u = _dev64(u_ring)
    out = torch.empty_like(u)
    _check(_lib().rbgs_guess_blend(_p(u), u.shape[0] - 2, _p(out), _stream(u)))
    return out


def network_input(f, u_ring, size=None):
    """4-channel input of one problem (rbgs_guess_input): f on the interior, mask 1 on the
    Dirichlet ring, ring values, and boundary_blend of the ring; the (N+2)^2 grid
    zero-padded to `size` (default: multiple of 8)."""
    n = f.shape[0]
    size = size or (n + 2 + 7) // 8 * 8
    fd, u = _dev64(f), _dev64(u_ring)
    x = torch.empty((size, size, 4), dtype=torch.float32, device=fd.device)
    _check(_lib().rbgs_guess_input(_p(fd), _p(u), n, size, _p(x), _stream(fd)))
    return x


def guess_target(sol, u_ring, size):
    """Training target on the size^2 grid (rbgs_guess_target): sol - boundary_blend(u_ring)."""
    s_, u = _dev64(sol), _dev64(u_ring)
    t = torch.empty((size, size), dtype=torch.float32, device=u.device)
    _check(_lib().rbgs_guess_target(_p(s_), _p(u), u.shape[0] - 2, size, _p(t), _stream(u)))
    return t


def guess_assemble(u_ring, pred):
    """u0 (rbgs_guess_assemble): the ring of u_ring, interior blend + pred (size^2 floats)."""
    u = _dev64(u_ring)
    pred = pred.to(torch.float32).contiguous()
    u0 = torch.empty_like(u)
    _check(_lib().rbgs_guess_assemble(_p(u), _p(pred), u.shape[0] - 2, pred.shape[-1], _p(u0), _stream(u)))
    return u0


def guess_coarsen(f, u_ring, n_coarse):
    """(fc, uc_ring) on the n_coarse^2 grid (rbgs_guess_coarsen): f averaged over the
    (2r-1)^2 fine nodes around each coarse node, the ring sampled."""
    fd, u = _dev64(f), _dev64(u_ring)
    fc = torch.empty((n_coarse, n_coarse), dtype=torch.float64, device=fd.device)
    uc = torch.empty((n_coarse + 2, n_coarse + 2), dtype=torch.float64, device=fd.device)
    _check(_lib().rbgs_guess_coarsen(_p(fd), _p(u), fd.shape[0], n_coarse, _p(fc), _p(uc), _stream(fd)))
    return fc, uc


def guess_refine(uc, u_ring):
    """Fine u0 (rbgs_guess_refine): uc interpolated bilinearly, the fine ring kept."""
    c, u = _dev64(uc), _dev64(u_ring)
    u0 = torch.empty_like(u)
    _check(_lib().rbgs_guess_refine(_p(c), c.shape[0] - 2, _p(u), u.shape[0] - 2, _p(u0), _stream(u)))
    return u0


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
