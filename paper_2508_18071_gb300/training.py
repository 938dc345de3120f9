"""The learned form: EvSNet trained on the GPU by the library's own kernels.

Marshalling over the training calls of include/eventtracer.h
(et_evsnet_train_forward / et_emd_count_loss / et_evsnet_train_backward /
et_adam_step), two torch.autograd.Function wrappers so the pieces compose with
autograd, and a small trainer.  Every numerical step runs in the CUDA library.

Loss (paper Eq. 7-11): bidirectional 1-D EMD per polarity plus lambda times the
spike-count difference, averaged over pixels; surrogate gradient of Eq. 4 with
the arctangent surrogate (alpha = 2); backpropagation through time with the
membrane checkpointed every `ckpt_every` steps.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np
import torch

from . import _lib as L
from .api import EvsNetDev, _ptr, _stream


def _shape(B, K, H, W, ckpt_every):
    return L.et_train_shape(B, K, H, W, ckpt_every)


def _net_struct(meta: EvsNetDev, w: torch.Tensor, b: torch.Tensor):
    # weights stay FP32; meta.dtype = ET_BF16 runs the 3x3 C -> C convolutions
    # (forward and data gradient) on the tensor cores with BF16 operands
    return meta.c_struct(w, b)


class Workspace:
    """Caller-owned device workspace for the training calls (grown on demand)."""

    def __init__(self):
        self.buf = torch.empty(0, dtype=torch.uint8, device="cuda")

    def get(self, meta: EvsNetDev, w, b, sh) -> torch.Tensor:
        nbytes = C.c_size_t()
        L.check("et_train_workspace_bytes",
                L.load().et_train_workspace_bytes(C.byref(_net_struct(meta, w, b)), C.byref(sh),
                                                  C.byref(nbytes)))
        if self.buf.numel() < nbytes.value:
            self.buf = torch.empty(nbytes.value, dtype=torch.uint8, device="cuda")
        return self.buf


_WS = {}


def _workspace() -> Workspace:
    dev = torch.cuda.current_device()
    if dev not in _WS:
        _WS[dev] = Workspace()
    return _WS[dev]


def train_forward(logl: torch.Tensor, meta: EvsNetDev, w: torch.Tensor, b: torch.Tensor,
                  ckpt_every=16, want_S=True, want_I=False, stream=None):
    """et_evsnet_train_forward on logl [B, K+1, H, W]; returns dict of device tensors."""
    B, K1, H, W = logl.shape
    K = K1 - 1
    sh = _shape(B, K, H, W, ckpt_every)
    dev = logl.device
    spikes = torch.empty((B, K, H, W), dtype=torch.int8, device=dev)
    S_on = torch.empty((B, K, H, W), dtype=torch.float32, device=dev) if want_S else None
    S_off = torch.empty((B, K, H, W), dtype=torch.float32, device=dev) if want_S else None
    nck = (K + ckpt_every - 1) // ckpt_every
    V_ckpt = torch.empty((B, nck, H, W), dtype=torch.float32, device=dev)
    I = torch.empty((B, K, H, W), dtype=torch.float32, device=dev) if want_I else None
    ws = _workspace().get(meta, w, b, sh)
    st = L.load().et_evsnet_train_forward(_ptr(logl), C.byref(sh), C.byref(_net_struct(meta, w, b)),
                                          _ptr(spikes), _ptr(S_on), _ptr(S_off), _ptr(V_ckpt), _ptr(I),
                                          _ptr(ws), ws.numel(), _stream(stream))
    L.check("et_evsnet_train_forward", st)
    return {"spikes": spikes, "S_on": S_on, "S_off": S_off, "V_ckpt": V_ckpt, "I": I}


def emd_count_loss(spikes: torch.Tensor, E: torch.Tensor, lam=0.01, stream=None):
    """et_emd_count_loss: (loss [3] = total, emd, count), dS_on, dS_off."""
    B, K, H, W = spikes.shape
    sh = _shape(B, K, H, W, 1)
    loss = torch.empty(3, dtype=torch.float32, device=spikes.device)
    dSon = torch.empty((B, K, H, W), dtype=torch.float32, device=spikes.device)
    dSoff = torch.empty_like(dSon)
    st = L.load().et_emd_count_loss(_ptr(spikes), _ptr(E), C.byref(sh), float(lam), _ptr(loss),
                                    _ptr(dSon), _ptr(dSoff), _stream(stream))
    L.check("et_emd_count_loss", st)
    return loss, dSon, dSoff


def train_backward(logl, meta: EvsNetDev, w, b, V_ckpt, dS_on, dS_off, ckpt_every=16, alpha=2.0,
                   grad_w: Optional[torch.Tensor] = None, grad_b: Optional[torch.Tensor] = None,
                   stream=None):
    """et_evsnet_train_backward; returns (grad_w, grad_b) (added to the given buffers)."""
    B, K1, H, W = logl.shape
    sh = _shape(B, K1 - 1, H, W, ckpt_every)
    if grad_w is None:
        grad_w = torch.zeros_like(w)
    if grad_b is None:
        grad_b = torch.zeros_like(b)
    ws = _workspace().get(meta, w, b, sh)
    st = L.load().et_evsnet_train_backward(_ptr(logl), C.byref(sh), C.byref(_net_struct(meta, w, b)),
                                           _ptr(V_ckpt), _ptr(dS_on), _ptr(dS_off), float(alpha),
                                           _ptr(grad_w), _ptr(grad_b), _ptr(ws), ws.numel(),
                                           _stream(stream))
    L.check("et_evsnet_train_backward", st)
    return grad_w, grad_b


def adam_step(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8, stream=None):
    st = L.load().et_adam_step(_ptr(p), _ptr(g), _ptr(m), _ptr(v), p.numel(), float(lr), float(b1),
                               float(b2), float(eps), int(step), _stream(stream))
    L.check("et_adam_step", st)


# ------------------------------------------------------------ autograd glue
class EvSNetTrainFn(torch.autograd.Function):
    """(logl, w, b) -> (S_on, S_off, spikes); backward = the library's BPTT."""

    @staticmethod
    def forward(ctx, logl, w, b, meta, ckpt_every, alpha):
        out = train_forward(logl, meta, w, b, ckpt_every=ckpt_every, want_S=True)
        ctx.save_for_backward(logl, w, b, out["V_ckpt"])
        ctx.meta, ctx.ckpt_every, ctx.alpha = meta, ckpt_every, alpha
        ctx.mark_non_differentiable(out["spikes"])
        return out["S_on"], out["S_off"], out["spikes"]

    @staticmethod
    def backward(ctx, g_on, g_off, _g_spikes):
        logl, w, b, V_ckpt = ctx.saved_tensors
        g_on = torch.zeros_like(w.new_empty(logl.shape[0], logl.shape[1] - 1, *logl.shape[2:])) \
            if g_on is None else g_on.contiguous()
        g_off = torch.zeros_like(g_on) if g_off is None else g_off.contiguous()
        gw, gb = train_backward(logl, ctx.meta, w, b, V_ckpt, g_on, g_off, ctx.ckpt_every, ctx.alpha)
        return None, gw, gb, None, None, None


class EmdCountLossFn(torch.autograd.Function):
    """(S_on, S_off, spikes, E) -> total loss; the kernel returns its gradient too."""

    @staticmethod
    def forward(ctx, S_on, S_off, spikes, E, lam):
        loss, dSon, dSoff = emd_count_loss(spikes, E, lam)
        ctx.save_for_backward(dSon, dSoff)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        dSon, dSoff = ctx.saved_tensors
        # the upstream gradient of a scalar loss is 1 in a plain .backward(); a
        # scaled loss multiplies the kernel's gradient
        if not bool(torch.all(g == 1)):
            dSon, dSoff = dSon * g, dSoff * g
        return dSon, dSoff, None, None, None


# ----------------------------------------------------------------- trainer
class Trainer:
    """Adam on the packed FP32 weights of an EvSNet, on the GPU.  dtype ET_BF16
    (3x3 stacks only) computes the C -> C convolutions of the forward and of the
    data gradient with BF16 operands on the tensor cores, FP32 accumulation."""

    def __init__(self, net: dict, lr=3e-3, lam=0.01, alpha=2.0, ckpt_every=16, dtype=L.ET_F32):
        self.meta = EvsNetDev.from_dict(net, dtype)
        self.w = self.meta.w.clone()
        self.b = self.meta.b.clone()
        self.mw, self.vw = torch.zeros_like(self.w), torch.zeros_like(self.w)
        self.mb, self.vb = torch.zeros_like(self.b), torch.zeros_like(self.b)
        self.gw, self.gb = torch.zeros_like(self.w), torch.zeros_like(self.b)
        self.lr, self.lam, self.alpha, self.ckpt = lr, lam, alpha, ckpt_every
        self.t = 0

    def step(self, logl: torch.Tensor, E: torch.Tensor, group=None) -> torch.Tensor:
        """One update on a batch; returns the device loss [3] (before the update).
        With a process group (data parallelism over clips: every rank passes its
        own equal share of the batch), the gradients are averaged over the ranks
        by one all_reduce before Adam, so every rank applies the same update."""
        out = train_forward(logl, self.meta, self.w, self.b, ckpt_every=self.ckpt, want_S=False)
        loss, dSon, dSoff = emd_count_loss(out["spikes"], E, self.lam)
        self.gw.zero_()
        self.gb.zero_()
        train_backward(logl, self.meta, self.w, self.b, out["V_ckpt"], dSon, dSoff, self.ckpt,
                       self.alpha, self.gw, self.gb)
        if group is not None:
            from .sharding import allreduce_mean
            allreduce_mean([self.gw, self.gb], group)
        self.t += 1
        adam_step(self.w, self.gw, self.mw, self.vw, self.t, self.lr)
        adam_step(self.b, self.gb, self.mb, self.vb, self.t, self.lr)
        return loss

    def save(self, path: str):
        """Checkpoint: FP32 weights, Adam moments, step count and hyper-parameters."""
        m = self.meta
        np.savez(path, w=self.w.cpu().numpy(), b=self.b.cpu().numpy(), mw=self.mw.cpu().numpy(),
                 vw=self.vw.cpu().numpy(), mb=self.mb.cpu().numpy(), vb=self.vb.cpu().numpy(),
                 t=self.t, lr=self.lr, lam=self.lam, alpha=self.alpha, ckpt=self.ckpt,
                 meta=np.array([m.kind, m.n_layers, m.C, m.kt, m.ks, m.ks0, m.delay]), dtype=m.dtype,
                 lif=np.array([m.beta, m.vth, m.reset], np.float64))

    @staticmethod
    def load(path: str) -> "Trainer":
        z = np.load(path)
        meta = [int(v) for v in z["meta"]] + [0, 0]
        kind, n_layers, C, kt, ks, ks0, delay = meta[:7]
        beta, vth, reset = (float(v) for v in z["lif"])
        net = {"kind": kind, "n_layers": n_layers, "C": C, "kt": kt, "ks": ks, "ks0": ks0,
               "delay": delay, "beta": beta,
               "vth": vth, "reset": reset, "w": z["w"], "b": z["b"]}
        T = Trainer(net, lr=float(z["lr"]), lam=float(z["lam"]), alpha=float(z["alpha"]),
                    ckpt_every=int(z["ckpt"]), dtype=int(z["dtype"]) if "dtype" in z else L.ET_F32)
        for k in ("mw", "vw", "mb", "vb"):
            getattr(T, k).copy_(torch.as_tensor(z[k]))
        T.t = int(z["t"])
        return T

    def net_dict(self) -> dict:
        m = self.meta
        return {"kind": m.kind, "n_layers": m.n_layers, "C": m.C, "kt": m.kt, "ks": m.ks,
                "ks0": m.ks0, "delay": m.delay, "beta": m.beta, "vth": m.vth, "reset": m.reset,
                "w": self.w.detach().cpu().numpy().astype(np.float32),
                "b": self.b.detach().cpu().numpy().astype(np.float32)}
