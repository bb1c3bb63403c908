"""Torch-facing wrappers of the C ABI (argument marshalling only).

Every function takes CUDA tensors, passes their device pointers and the
current CUDA stream to ``libldbp.so`` and returns the outputs; no arithmetic
of the method runs here.
"""
from __future__ import annotations

import torch

from . import _lib


def _stream():
    return ctypes_void(torch.cuda.current_stream().cuda_stream)


def ctypes_void(v):
    import ctypes
    return ctypes.c_void_p(int(v))


def _ptr(t):
    return None if t is None else ctypes_void(t.data_ptr())


def _check_c64(name, t, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.complex64:
        raise ValueError(f"{name} must be complex64, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


def ldbp_apply(taps, T, c, x, ckpt=None, out=None):
    """Learned-DBP forward (Eq. (7), symmetric FIR steps).  x: complex64 [B, n] or [n]."""
    squeeze = x.dim() == 1
    x2 = x.unsqueeze(0) if squeeze else x
    _check_c64("x", x2)
    _check_c64("taps", taps)
    B, n = x2.shape
    M = len(T)
    if taps.dim() != 2 or taps.shape[0] != M:
        raise ValueError("taps must be [M, stride] with M = len(T)")
    y = torch.empty_like(x2) if out is None else out
    if ckpt is not None:
        _check_c64("ckpt", ckpt, (M, B, n))
    _lib.check(_lib.lib().ldbp_apply(_ptr(taps), taps.shape[1], _lib.i32_array(T), _lib.f32_array(c), M,
                                     _ptr(x2), _ptr(y), n, B, _ptr(ckpt), _stream()))
    return y[0] if squeeze else y


def ldbp_essm_apply(taps, T, c, eta, kappa, x, out=None, ckpt=None):
    """Learned enhanced SSM (filtered nonlinear steps, Sec. III-C): ldbp_apply whose
    Kerr phase uses sum_k eta_k |v_{j-k}|^2.  eta: device float32 [M, stride] with
    row i = (eta_{-kappa_i}, ..., eta_{kappa_i}); kappa: per-step half-widths;
    ckpt: optional complex64 [M, B, n] receiving the input of every step."""
    squeeze = x.dim() == 1
    x2 = x.unsqueeze(0) if squeeze else x
    _check_c64("x", x2)
    _check_c64("taps", taps)
    if eta.dtype != torch.float32 or not eta.is_cuda or not eta.is_contiguous() or eta.dim() != 2:
        raise ValueError("eta must be a contiguous CUDA float32 [M, stride] tensor")
    B, n = x2.shape
    M = len(T)
    if taps.shape[0] != M or eta.shape[0] != M or len(kappa) != M:
        raise ValueError("taps, eta and kappa need M = len(T) rows")
    if ckpt is not None:
        _check_c64("ckpt", ckpt, (M, B, n))
    y = torch.empty_like(x2) if out is None else out
    _lib.check(_lib.lib().ldbp_essm_apply(_ptr(taps), taps.shape[1], _lib.i32_array(T), _lib.f32_array(c), _ptr(eta),
                                          eta.shape[1], _lib.i32_array(kappa), M, _ptr(x2), _ptr(y), n, B,
                                          _ptr(ckpt), _stream()))
    return y[0] if squeeze else y


def ldbp_essm_backward(taps, T, c, eta, kappa, ckpt, gy, want_gx=True, workspace=None):
    """Adjoint of ldbp_essm_apply: returns (gx or None, gtaps [M, stride], geta [M, eta stride])."""
    import ctypes
    _check_c64("gy", gy)
    B, n = gy.shape
    M = len(T)
    _check_c64("ckpt", ckpt, (M, B, n))
    need = ctypes.c_size_t(0)
    _lib.check(_lib.lib().ldbp_essm_backward_workspace(n, B, _lib.i32_array(T), _lib.i32_array(kappa), M,
                                                       ctypes.byref(need)))
    if workspace is None or workspace.numel() < need.value:
        workspace = torch.empty(max(need.value, 8), dtype=torch.uint8, device=gy.device)
    gx = torch.empty_like(gy) if want_gx else None
    gt = torch.empty_like(taps)
    ge = torch.empty_like(eta)
    _lib.check(_lib.lib().ldbp_essm_backward(_ptr(taps), taps.shape[1], _lib.i32_array(T), _lib.f32_array(c),
                                             _ptr(eta), eta.shape[1], _lib.i32_array(kappa), M, _ptr(ckpt), _ptr(gy),
                                             _ptr(gx), _ptr(gt), _ptr(ge), n, B, _ptr(workspace), workspace.numel(),
                                             _stream()))
    return gx, gt, ge


def ldbp_apply_host_workspace(n, batch) -> int:
    """Device workspace bytes of ldbp_apply_host for [batch, n] waveforms."""
    return int(_lib.lib().ldbp_apply_host_workspace(n, batch))


def ldbp_apply_host(taps, T, c, x_host, y_host, chunks=8, workspace=None):
    """ldbp_apply on host (CPU) complex64 [B, n] tensors: chunked copy-in /
    compute / copy-out overlapped on the library's streams.  Ordered on the
    current stream; synchronise it before reading y_host.  workspace: a
    device uint8 tensor of ldbp_apply_host_workspace bytes (allocated if
    None)."""
    for name, t in (("x_host", x_host), ("y_host", y_host)):
        if t.device.type != "cpu" or t.dtype != torch.complex64 or not t.is_contiguous() or t.dim() != 2:
            raise ValueError(f"{name} must be a contiguous CPU complex64 [B, n] tensor")
    if x_host.shape != y_host.shape:
        raise ValueError("x_host and y_host must have the same shape")
    _check_c64("taps", taps)
    B, n = x_host.shape
    need = ldbp_apply_host_workspace(n, B)
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device="cuda")
    M = len(T)
    _lib.check(_lib.lib().ldbp_apply_host(_ptr(taps), taps.shape[1], _lib.i32_array(T), _lib.f32_array(c), M,
                                          x_host.data_ptr(), y_host.data_ptr(), n, B, int(chunks), _ptr(workspace),
                                          workspace.numel(), _stream()))
    return y_host


def ubench(kind: int) -> float:
    """Measured lane-operation throughput: 0 FP32 FMA, 1 FP32x2 FMA, 2 sine (ops/s)."""
    import ctypes
    out = ctypes.c_double(0.0)
    _lib.check(_lib.lib().ldbp_ubench(kind, ctypes.byref(out)))
    return out.value


def fiber_struct(fiber):
    """ldbp_fiber from an object with alpha_db_per_km, beta2_ps2_per_km, gamma_per_w_km."""
    return _lib.LdbpFiber(float(fiber.alpha_db_per_km), float(fiber.beta2_ps2_per_km), float(fiber.gamma_per_w_km))


def link_struct(link):
    return _lib.LdbpLink(int(link.n_spans), float(link.span_km), int(link.steps_per_span), int(bool(link.symmetric)),
                         int(bool(link.ase)), float(link.nf_db), float(link.carrier_hz), int(link.seed) & (2**64 - 1),
                         int(link.counter) & (2**64 - 1))


def _batched(x):
    squeeze = x.dim() == 1
    x2 = x.unsqueeze(0) if squeeze else x
    _check_c64("x", x2)
    return x2, squeeze


def ssm_forward(fiber, link, fs, x, out=None):
    """Split-step channel (Eqs. (6)/(8), Sec. IV-A).  x: complex64 [B, n] or [n] (n a power of two)."""
    import ctypes
    x2, squeeze = _batched(x)
    y = torch.empty_like(x2) if out is None else out
    f, l = fiber_struct(fiber), link_struct(link)
    _lib.check(_lib.lib().ssm_forward(ctypes.byref(f), ctypes.byref(l), float(fs), _ptr(x2), _ptr(y), x2.shape[1],
                                      x2.shape[0], _stream()))
    return y[0] if squeeze else y


def dbp_apply(fiber, link, fs, x, steps_per_span=1, symmetric=False, out=None):
    """Full-length frequency-domain DBP (the SSM run backwards)."""
    import ctypes
    x2, squeeze = _batched(x)
    y = torch.empty_like(x2) if out is None else out
    f, l = fiber_struct(fiber), link_struct(link)
    _lib.check(_lib.lib().dbp_apply(ctypes.byref(f), ctypes.byref(l), float(fs), int(steps_per_span),
                                    int(bool(symmetric)), _ptr(x2), _ptr(y), x2.shape[1], x2.shape[0], _stream()))
    return y[0] if squeeze else y


def ssm_cufft(fiber, link, fs, x, dbp_steps_per_span=0, dbp_symmetric=False, out=None):
    """The same split-step program run with cuFFT (comparison path only)."""
    import ctypes
    x2, squeeze = _batched(x)
    y = torch.empty_like(x2) if out is None else out
    f, l = fiber_struct(fiber), link_struct(link)
    _lib.check(_lib.lib().ssm_cufft(ctypes.byref(f), ctypes.byref(l), float(fs), int(dbp_steps_per_span),
                                    int(bool(dbp_symmetric)), _ptr(x2), _ptr(y), x2.shape[1], x2.shape[0], _stream()))
    return y[0] if squeeze else y


def resample(x, n_out, bandwidth=1.0, out=None):
    """Receiver front end of Sec. IV-A: brick-wall low-pass of bandwidth
    `bandwidth` x (the coarser grid's sample rate), sampled onto n_out points per
    waveform; with n_out > n_in, band-limited interpolation.  x: complex64 [B, n_in]."""
    x2, squeeze = _batched(x)
    B, n_in = x2.shape
    if out is None:
        y = torch.empty((B, int(n_out)), dtype=torch.complex64, device=x2.device)
    else:
        y = out.unsqueeze(0) if out.dim() == 1 else out
    _check_c64("out", y, (B, int(n_out)))
    _lib.check(_lib.lib().ldbp_resample(_ptr(x2), n_in, _ptr(y), int(n_out), float(bandwidth), B, _stream()))
    return y[0] if squeeze else y


def _power_tensor(power_w, B):
    if isinstance(power_w, torch.Tensor):
        p = power_w.to(device="cuda", dtype=torch.float32).reshape(-1)
    else:
        p = torch.as_tensor(power_w, dtype=torch.float32).reshape(-1).cuda()
    if p.numel() == 1 and B > 1:
        p = p.expand(B).contiguous()
    if p.numel() != B:
        raise ValueError("power_w must be a scalar or have one entry per waveform")
    return p.contiguous()


def tx(symbols, power_w, sps=2, rolloff=0.1, out=None):
    """Eq. (11): RRC-shaped waveform of 16-QAM (or any) symbols at power P (W)."""
    _check_c64("symbols", symbols)
    B, nsym = symbols.shape
    p = _power_tensor(power_w, B)
    x = torch.empty((B, nsym * sps), dtype=torch.complex64, device=symbols.device) if out is None else out
    _lib.check(_lib.lib().ldbp_tx(_ptr(symbols), _ptr(p), int(sps), float(rolloff), _ptr(x), nsym, B, _stream()))
    return x


def rx(y, symbols, power_w, sps=2, rolloff=0.1, grad=False, grad_scale=None, workspace=None):
    """Eq. (12) receiver: returns (stats[B, 2] float64 = (mse_b, mean |s_b|^2), phi[B] float32, grad or None)."""
    _check_c64("y", y)
    _check_c64("symbols", symbols)
    B, n = y.shape
    nsym = symbols.shape[1]
    p = _power_tensor(power_w, B)
    mse = torch.empty((B, 2), dtype=torch.float64, device=y.device)
    phi = torch.empty(B, dtype=torch.float32, device=y.device)
    ws = torch.empty_like(y) if workspace is None else workspace
    g = torch.empty_like(y) if grad else None
    gs = 2.0 / (nsym * B) if grad_scale is None else grad_scale
    _lib.check(_lib.lib().ldbp_rx(_ptr(y), _ptr(symbols), _ptr(p), int(sps), float(rolloff), nsym, B, _ptr(mse),
                                  _ptr(phi), _ptr(g), float(gs), _ptr(ws), _stream()))
    return mse, phi, g


def snr_db(stats):
    """Effective SNR (Eq. (14), read as sum_b ||s_b||^2 / sum_b ||s_hat_b - s_b||^2) in dB."""
    st = stats.double().cpu()
    return float(10.0 * torch.log10(st[:, 1].sum() / st[:, 0].sum()).item())


def ldbp_backward_workspace_bytes(n, batch, T):
    import ctypes
    out = ctypes.c_size_t(0)
    _lib.check(_lib.lib().ldbp_backward_workspace(int(n), int(batch), _lib.i32_array(T), len(T), ctypes.byref(out)))
    return out.value


def ldbp_backward(taps, T, c, ckpt, gy, want_gx=True, workspace=None, gtaps_out=None, want_gc=False):
    """Adjoint of ldbp_apply: returns (gx or None, gtaps [M, stride]) for the loss gradient gy,
    and with want_gc also gc (float32 [M], the gradients of the nonlinear coefficients)."""
    _check_c64("gy", gy)
    _check_c64("taps", taps)
    B, n = gy.shape
    M = len(T)
    _check_c64("ckpt", ckpt, (M, B, n))
    need = ldbp_backward_workspace_bytes(n, B, T)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 8), dtype=torch.uint8, device=gy.device)
    gx = torch.empty_like(gy) if want_gx else None
    gt = torch.empty_like(taps) if gtaps_out is None else gtaps_out
    gc = torch.empty(M, dtype=torch.float32, device=gy.device) if want_gc else None
    _lib.check(_lib.lib().ldbp_backward_c(_ptr(taps), taps.shape[1], _lib.i32_array(T), _lib.f32_array(c), M,
                                          _ptr(ckpt), _ptr(gy), _ptr(gx), _ptr(gt), _ptr(gc), n, B, _ptr(workspace),
                                          workspace.numel(), _stream()))
    return (gx, gt, gc) if want_gc else (gx, gt)


class LDBPFunction(torch.autograd.Function):
    """y = LDBP(x; taps) with the hand-written adjoint (checkpoints every step).

    forward(x, taps, T, c): x complex64 [B, n], taps complex64 [M, stride] (the
    trainable half-tap vectors), T list of filter lengths, c list of Kerr
    coefficients.  Gradients follow torch's complex convention
    (dl/dRe + j dl/dIm), which is the library's.
    """

    @staticmethod
    def forward(ctx, x, taps, T, c):
        M = len(T)
        B, n = x.shape
        ckpt = torch.empty((M, B, n), dtype=torch.complex64, device=x.device)
        y = ldbp_apply(taps.detach().contiguous(), list(T), list(c), x.detach().contiguous(), ckpt=ckpt)
        ctx.save_for_backward(taps.detach().contiguous(), ckpt)
        ctx.T, ctx.c = list(T), list(c)
        ctx.need_x = x.requires_grad
        return y

    @staticmethod
    def backward(ctx, gy):
        taps, ckpt = ctx.saved_tensors
        gx, gt = ldbp_backward(taps, ctx.T, ctx.c, ckpt, gy.contiguous(), want_gx=ctx.need_x)
        return gx, gt, None, None


def adam_step(taps, gtaps, m, v, T, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam update of taps [M, stride] with moments m, v (float32 [M, stride, 2])."""
    _check_c64("taps", taps)
    _check_c64("gtaps", gtaps, tuple(taps.shape))
    M, stride = taps.shape
    for name, t in (("m", m), ("v", v)):
        if t.dtype != torch.float32 or tuple(t.shape) != (M, stride, 2) or not t.is_contiguous():
            raise ValueError(f"{name} must be float32 [M, stride, 2]")
    _lib.check(_lib.lib().ldbp_adam_step(_ptr(taps), _ptr(gtaps), _ptr(m), _ptr(v), _lib.i32_array(T), M, stride,
                                         int(step), float(lr), float(beta1), float(beta2), float(eps), _stream()))


class RaggedPlan:
    """Persistent one-launch learned DBP over waveforms of uneven n, M and T.

    n: per-waveform lengths; T_steps: per-waveform lists of filter lengths.
    Device buffers: x/y packed complex64 [sum n], taps complex64
    [sum M, stride], c float32 [sum M].
    """

    def __init__(self, n, T_steps, taps_stride):
        import ctypes
        self.n = [int(v) for v in n]
        self.M = [len(t) for t in T_steps]
        self.T = [int(t) for ts in T_steps for t in ts]
        self.stride = int(taps_stride)
        h = ctypes.c_void_p()
        narr = (ctypes.c_int64 * len(self.n))(*self.n)
        _lib.check(_lib.lib().ldbp_ragged_plan_create(ctypes.byref(h), len(self.n), narr, _lib.i32_array(self.M),
                                                      _lib.i32_array(self.T), self.stride))
        self.handle = h
        self.offsets = [0]
        for v in self.n[:-1]:
            self.offsets.append(self.offsets[-1] + v)

    def info(self):
        import ctypes
        ts, st, it, cap, bps = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _lib.check(_lib.lib().ldbp_ragged_info(self.handle, ctypes.byref(ts), ctypes.byref(st), ctypes.byref(it),
                                               ctypes.byref(cap), ctypes.byref(bps)))
        return {"total_samples": ts.value, "total_steps": st.value, "items": it.value, "tile_cap": cap.value,
                "blocks_per_sm": bps.value}

    def autotune(self, taps, c, x, y):
        _lib.check(_lib.lib().ldbp_ragged_autotune(self.handle, _ptr(taps), _ptr(c), _ptr(x), _ptr(y), _stream()))

    def set_schedule(self, tile_cap, blocks_per_sm):
        """Pin the tile cap and blocks per SM (e.g. a configuration autotuned earlier)."""
        _lib.check(_lib.lib().ldbp_ragged_set_schedule(self.handle, int(tile_cap), int(blocks_per_sm)))

    def apply(self, taps, c, x, y, done_ns=None, start_ns=None):
        _lib.check(_lib.lib().ldbp_apply_ragged(self.handle, _ptr(taps), _ptr(c), _ptr(x), _ptr(y), _ptr(done_ns),
                                                _ptr(start_ns), _stream()))
        return y

    def capture(self, taps, c, x, y):
        _lib.check(_lib.lib().ldbp_ragged_graph_capture(self.handle, _ptr(taps), _ptr(c), _ptr(x), _ptr(y)))

    def replay(self):
        _lib.check(_lib.lib().ldbp_ragged_graph_launch(self.handle, _stream()))

    def close(self):
        if getattr(self, "handle", None):
            _lib.check(_lib.lib().ldbp_ragged_plan_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
