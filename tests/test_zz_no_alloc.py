"""The allocation-free training backward (et_evsnet_train_backward_static).

It serves callers that cannot allocate device memory themselves or through the
library -- a plugin living inside a framework whose allocator owns the device,
or a loop that must not call cudaMalloc / cudaFree because those calls can
synchronise the device.  Its scratch is an array compiled into the library.

Each test first makes one call with a different, larger shape and other
inputs, so that the shared array holds unrelated non-zero values; then it calls
the entry point through the C ABI twice in a row on the compared problem (the
second call sees the first call's leftovers) and compares both results with
the workspace-taking et_evsnet_train_backward, within the tolerance the other
gradient tests use (float atomics make the summation order vary):
max |difference| <= 1e-5 of the largest gradient component.  This file is
named to be collected last."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2508_18071_gb300 import inputs

pytestmark = pytest.mark.gpu


def _dirty_call(lib, _lib, training, api, d, B, K, H, W, ck, seed):
    """One static-workspace call on another problem (its own inputs and shape):
    leaves non-zero, unrelated values in the shared array."""
    meta = api.EvsNetDev.from_dict(d)
    lf = np.stack([inputs.random_logl_clip(seed + b, K + 1, H, W, step_std=0.5) for b in range(B)])
    E = np.random.default_rng(seed).choice([-2, -1, 0, 1, 2], (B, K, H, W)).astype(np.float32)
    lfd, Ed = torch.as_tensor(lf).cuda(), torch.as_tensor(E).cuda()
    out = training.train_forward(lfd, meta, meta.w, meta.b, ckpt_every=ck)
    _, dSon, dSoff = training.emd_count_loss(out["spikes"], Ed, 0.01)
    sh = _lib.et_train_shape(B, K, H, W, ck)
    net = meta.c_struct()
    need = C.c_size_t()
    assert lib.et_train_workspace_bytes(C.byref(net), C.byref(sh), C.byref(need)) == _lib.ET_OK
    assert need.value <= lib.et_train_static_workspace_capacity()
    gw, gb = torch.zeros_like(meta.w), torch.zeros_like(meta.b)
    st = lib.et_evsnet_train_backward_static(
        C.c_void_p(lfd.data_ptr()), C.byref(sh), C.byref(net), C.c_void_p(out["V_ckpt"].data_ptr()),
        C.c_void_p(dSon.data_ptr()), C.c_void_p(dSoff.data_ptr()), 2.0, C.c_void_p(gw.data_ptr()),
        C.c_void_p(gb.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == _lib.ET_OK, lib.et_status_str(st)
    torch.cuda.synchronize()
    assert float(torch.cat([gw, gb]).abs().max()) > 0
    return need.value


def test_static_workspace_backward_matches_workspace_backward():
    assert torch.cuda.is_available()
    from paper_2508_18071_gb300 import _lib, api, training
    lib = _lib.load()
    B, K, H, W, ck = 2, 24, 32, 32, 8
    d = inputs.random_evsnet(0, 4, 16, 1, 3, seed=7, vth=0.3, beta=0.9, std=0.3)
    lf = np.stack([inputs.random_logl_clip(40 + b, K + 1, H, W, step_std=0.3) for b in range(B)])
    E = np.random.default_rng(3).choice([-1, 0, 0, 0, 1], (B, K, H, W)).astype(np.float32)
    meta = api.EvsNetDev.from_dict(d)
    lfd, Ed = torch.as_tensor(lf).cuda(), torch.as_tensor(E).cuda()
    out = training.train_forward(lfd, meta, meta.w, meta.b, ckpt_every=ck)
    _, dSon, dSoff = training.emd_count_loss(out["spikes"], Ed, 0.01)
    ref_w, ref_b = training.train_backward(lfd, meta, meta.w, meta.b, out["V_ckpt"], dSon, dSoff,
                                           ckpt_every=ck)
    ref = torch.cat([ref_w, ref_b]).cpu().numpy()
    assert np.abs(ref).max() > 0

    sh = _lib.et_train_shape(B, K, H, W, ck)
    net = meta.c_struct()
    need = C.c_size_t()
    assert lib.et_train_workspace_bytes(C.byref(net), C.byref(sh), C.byref(need)) == _lib.ET_OK
    assert need.value <= lib.et_train_static_workspace_capacity()
    # leftovers of a larger problem with other weights and inputs
    d2 = inputs.random_evsnet(0, 4, 16, 1, 3, seed=17, vth=0.2, beta=0.95, std=0.5)
    assert _dirty_call(lib, _lib, training, api, d2, 3, 32, 48, 40, 8, 300) > need.value
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        gw = torch.zeros_like(meta.w)
        gb = torch.zeros_like(meta.b)
        st = lib.et_evsnet_train_backward_static(
            C.c_void_p(lfd.data_ptr()), C.byref(sh), C.byref(net), C.c_void_p(out["V_ckpt"].data_ptr()),
            C.c_void_p(dSon.data_ptr()), C.c_void_p(dSoff.data_ptr()), 2.0, C.c_void_p(gw.data_ptr()),
            C.c_void_p(gb.data_ptr()), stream)
        assert st == _lib.ET_OK, lib.et_status_str(st)
        torch.cuda.synchronize()
        got = torch.cat([gw, gb]).cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max(), (call, np.abs(got - ref).max())

    # a shape whose scratch exceeds the array is refused before anything runs
    big = _lib.et_train_shape(8, 64, 512, 512, 16)
    assert lib.et_evsnet_train_backward_static(
        C.c_void_p(lfd.data_ptr()), C.byref(big), C.byref(net), C.c_void_p(out["V_ckpt"].data_ptr()),
        C.c_void_p(dSon.data_ptr()), C.c_void_p(dSoff.data_ptr()), 2.0, C.c_void_p(gw.data_ptr()),
        C.c_void_p(gb.data_ptr()), stream) == _lib.ET_ERR_CAPACITY


def test_static_workspace_backward_temporal_form():
    """The same check for the paper's temporal form (kernel 7 along time, one
    residual block), whose scratch holds whole-clip activations; a clip too long
    for the array is refused with ET_ERR_CAPACITY."""
    assert torch.cuda.is_available()
    from paper_2508_18071_gb300 import _lib, api, training
    lib = _lib.load()
    B, K, H, W, ck = 1, 20, 16, 16, 8
    d = inputs.random_evsnet(1, 3, 8, 7, 1, seed=9, vth=0.3, beta=0.9, std=0.3)
    lf = np.stack([inputs.random_logl_clip(60 + b, K + 1, H, W, step_std=0.3) for b in range(B)])
    E = np.random.default_rng(5).choice([-1, 0, 0, 0, 1], (B, K, H, W)).astype(np.float32)
    meta = api.EvsNetDev.from_dict(d)
    lfd, Ed = torch.as_tensor(lf).cuda(), torch.as_tensor(E).cuda()
    out = training.train_forward(lfd, meta, meta.w, meta.b, ckpt_every=ck)
    _, dSon, dSoff = training.emd_count_loss(out["spikes"], Ed, 0.01)
    ref_w, ref_b = training.train_backward(lfd, meta, meta.w, meta.b, out["V_ckpt"], dSon, dSoff,
                                           ckpt_every=ck)
    ref = torch.cat([ref_w, ref_b]).cpu().numpy()
    assert np.abs(ref).max() > 0
    sh = _lib.et_train_shape(B, K, H, W, ck)
    net = meta.c_struct()
    need = C.c_size_t()
    assert lib.et_train_workspace_bytes(C.byref(net), C.byref(sh), C.byref(need)) == _lib.ET_OK
    d2 = inputs.random_evsnet(1, 3, 8, 7, 1, seed=19, vth=0.2, beta=0.95, std=0.5)
    assert _dirty_call(lib, _lib, training, api, d2, 2, 24, 20, 18, 8, 400) > need.value
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    args = lambda gw, gb, shape: (C.c_void_p(lfd.data_ptr()), C.byref(shape), C.byref(net),
                                  C.c_void_p(out["V_ckpt"].data_ptr()), C.c_void_p(dSon.data_ptr()),
                                  C.c_void_p(dSoff.data_ptr()), 2.0, C.c_void_p(gw.data_ptr()),
                                  C.c_void_p(gb.data_ptr()), stream)
    for call in range(2):
        gw = torch.zeros_like(meta.w)
        gb = torch.zeros_like(meta.b)
        st = lib.et_evsnet_train_backward_static(*args(gw, gb, sh))
        assert st == _lib.ET_OK, lib.et_status_str(st)
        torch.cuda.synchronize()
        got = torch.cat([gw, gb]).cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max(), (call, np.abs(got - ref).max())
    big = _lib.et_train_shape(8, 64, 128, 128, 16)
    assert lib.et_evsnet_train_backward_static(*args(gw, gb, big)) == _lib.ET_ERR_CAPACITY
