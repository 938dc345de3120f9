"""BF16 tensor-core training of the paper's temporal form (causal kernel kt
along time, plain stack or residual blocks, optionally a spatial stem as
layer 0) against the FP32 path and the oracle.

With net dtype ET_BF16 the C -> C temporal convolutions (forward, data
gradient and weight gradient) take BF16 operands (u = 2^-8) on the tensor
cores with FP32 accumulation; layer 0, the projection, BiLIF and the loss are
the FP32 path's.

* exact: with +-1/2 layer-0 weights, sparse +-1 weights in layers 1.., +-1
  projection, zero biases and log steps in {-2..2}/4, every activation is a
  short dyadic fraction (checked on the CPU first), so the BF16 forward's
  spikes, currents and checkpoints equal the FP32 path's bit for bit: this
  pins the operand layouts, the tap windows, the ring of past steps, residual
  sums, ragged tiles and both time directions;
* bounded: the backward rounds each layer's dL/dz (and, in the weight
  gradient, the activations) to BF16; with L - 1 tensor-core layers the weight
  gradients stay within (L + 1) u (relative L2) of the FP32 path's and of the
  oracle's -- a transposed, reversed or shifted operand gives O(1) errors;
* training: Adam steps with BF16 convolutions lower the loss of a denoising
  task as the FP32 ones do;
* a bounded MMA wait that runs out leaves NaN currents and a usable context;
  kernels longer than 7 are refused in BF16 (the FP32 path takes them)."""
import numpy as np
import pytest
import torch

from paper_2508_18071_gb300 import inputs

pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -8


@pytest.fixture(scope="module")
def tr():
    assert torch.cuda.is_available()
    from paper_2508_18071_gb300 import training
    return training


def _dyadic_net(kind, L, C, kt, ks0, seed, dens):
    rng = np.random.default_rng(seed)
    d = inputs.random_evsnet(kind, L, C, kt, 1, seed=seed, vth=0.0625, beta=1.0, ks0=ks0)
    d["reset"] = 0.0625
    w = rng.choice([-1.0, 0.0, 1.0], size=d["w"].shape, p=[dens / 2, 1 - dens, dens / 2])
    n0 = C * (ks0 * ks0 if ks0 else kt)
    w[:n0] = rng.choice([-0.5, 0.0, 0.5], size=n0, p=[0.2, 0.6, 0.2])
    w[-C:] = rng.choice([-1.0, 1.0], size=C)
    d["w"] = w.astype(np.float32)
    d["b"] = np.zeros_like(d["b"])
    return d


def _dyadic_clips(seed, B, K, H, W):
    rng = np.random.default_rng(seed)
    steps = rng.integers(-2, 3, (B, K + 1, H, W)) / 4.0
    steps[:, 0] = 0
    return np.cumsum(steps, 1).astype(np.float32)


def _tc_layer_inputs(orc, net, X):
    """Inputs of every tensor-core layer of the oracle's forward (float64)."""
    F_ = torch.nn.functional
    layers, _ = orc.torch_params(net)

    def conv(h, Wt, bt):
        kt, pad = Wt.shape[2], Wt.shape[3] // 2
        return F_.conv3d(F_.pad(h, (pad, pad, pad, pad, kt - 1, 0)), Wt, bt)

    outs = []
    h = torch.relu(conv(X.unsqueeze(1), *layers[0]))
    if net.kind == 0:
        for Wt, bt in layers[1:]:
            outs.append(h)
            h = torch.relu(conv(h, Wt, bt))
    else:
        for j in range(1, net.n_layers - 1, 2):
            outs.append(h)
            a = torch.relu(conv(h, *layers[j]))
            outs.append(a)
            h = torch.relu(h + conv(a, *layers[j + 1]))
    return outs


def _fwd_bwd(tr, d, lf, E, dtype, ck):
    from paper_2508_18071_gb300 import api
    meta = api.EvsNetDev.from_dict(d, dtype)
    lfd = torch.as_tensor(lf).cuda()
    out = tr.train_forward(lfd, meta, meta.w, meta.b, ckpt_every=ck, want_I=True)
    loss, dSon, dSoff = tr.emd_count_loss(out["spikes"], torch.as_tensor(E).cuda(), 0.01)
    gw, gb = tr.train_backward(lfd, meta, meta.w, meta.b, out["V_ckpt"], dSon, dSoff, ckpt_every=ck)
    return out, loss, np.concatenate([gw.cpu().numpy(), gb.cpu().numpy()]).astype(np.float64)


@pytest.mark.parametrize("kind,L,C,kt,ks0,B,K,H,W,ck,dens", [
    (1, 7, 16, 7, 0, 2, 40, 9, 23, 16, 0.04),     # the paper's form: k = 7, M = 3
    (1, 7, 16, 7, 3, 2, 33, 12, 17, 8, 0.04),     # 3 x 3 stem + the paper's blocks, odd K
    (0, 3, 8, 5, 0, 1, 26, 16, 16, 13, 0.1),      # plain stack, C = 8
    (1, 5, 12, 3, 5, 2, 21, 11, 13, 7, 0.06),     # 5 x 5 stem, M = 2, C = 12
])
def test_bf16_temporal_training_exact_forward_bounded_gradients(tr, orc, kind, L, C, kt, ks0, B, K, H,
                                                                W, ck, dens):
    from paper_2508_18071_gb300 import _lib
    d = _dyadic_net(kind, L, C, kt, ks0, seed=7 + L + C, dens=dens)
    lf = _dyadic_clips(8 + W, B, K, H, W)
    onet = orc.EvsNet.from_dict(d)
    X = np.diff(lf.astype(np.float64), axis=1)
    acts = _tc_layer_inputs(orc, onet, torch.tensor(X))
    assert all(torch.equal(a, a.to(torch.bfloat16).double()) for a in acts)   # precondition
    E = np.random.default_rng(9).choice([-1, 0, 0, 0, 1], (B, K, H, W)).astype(np.float32)
    o32, l32, g32 = _fwd_bwd(tr, d, lf, E, _lib.ET_F32, ck)
    o16, l16, g16 = _fwd_bwd(tr, d, lf, E, _lib.ET_BF16, ck)
    assert (o32["spikes"] != 0).sum().item() > 20
    for k in ("spikes", "V_ckpt", "I"):
        np.testing.assert_array_equal(o16[k].cpu().numpy(), o32[k].cpu().numpy())
    assert abs(l16[0].item() - l32[0].item()) <= 1e-6 * abs(l32[0].item())
    assert np.abs(g32).max() > 0
    rel = np.linalg.norm(g16 - g32) / np.linalg.norm(g32)
    assert rel <= (L + 1) * U_BF16, rel / U_BF16
    _, rgw, rgb = orc.torch_grads(X, E, onet, smooth=False, alpha=2.0, lam=0.01)
    r = np.concatenate([rgw, rgb])
    assert np.linalg.norm(g16 - r) <= (L + 1) * U_BF16 * np.linalg.norm(r)
    print("bf16 temporal training L=%d C=%d kt=%d: gradient relative L2 error %.2f u (FP32 path %.2e u)"
          % (L, C, kt, rel / U_BF16, np.linalg.norm(g32 - r) / np.linalg.norm(r) / U_BF16))


def test_bf16_temporal_training_reduces_the_loss(tr, orc):
    """Denoising: input = clean log clip + noise, target = contrast-threshold
    events of the clean clip.  40 Adam steps of the paper's form with BF16
    convolutions lower the loss as far as the FP32 ones (within 10 %), and by
    at least a fifth."""
    from paper_2508_18071_gb300 import _lib
    B, K, H, W = 4, 32, 24, 24
    rng = np.random.default_rng(5)
    clean = np.stack([inputs.random_logl_clip(10 + b, K + 1, H, W, step_std=0.05, jump_p=0.01)
                      for b in range(B)])
    noisy = (clean + rng.normal(0, 0.15, clean.shape)).astype(np.float32)
    E = np.zeros((B, K, H, W), np.float32)
    for b in range(B):
        ev = orc.threshold_events(clean[b], 0.2, orc.ThresholdState.new(H, W))
        E[b] = orc.events_to_dense(ev, K, H, W, t0=1)
    d = inputs.random_evsnet(1, 5, 8, 7, 1, seed=4, vth=0.2, beta=0.95, std=0.2)
    x, e = torch.as_tensor(noisy).cuda(), torch.as_tensor(E).cuda()
    res = {}
    for name, dt in (("f32", _lib.ET_F32), ("bf16", _lib.ET_BF16)):
        T = tr.Trainer(d, lr=1e-2, dtype=dt)
        res[name] = [T.step(x, e)[0].item() for _ in range(40)]
    l16, l32 = res["bf16"], res["f32"]
    assert np.isfinite(l16).all()
    assert min(l16[-5:]) < 0.8 * l16[0], (l16[0], l16[-5:])
    assert min(l16[-5:]) <= 1.1 * min(l32[-5:]), (l16[-5:], l32[-5:])


def test_bf16_temporal_training_wait_timeout_leaves_nan_and_recovers(tr):
    from paper_2508_18071_gb300 import _lib, api
    d = inputs.random_evsnet(1, 5, 16, 7, 1, seed=3, vth=0.2, beta=0.9, std=0.2, ks0=3)
    lf = torch.as_tensor(np.stack([inputs.random_logl_clip(3, 13, 20, 24, step_std=0.3)])).cuda()
    meta = api.EvsNetDev.from_dict(d, _lib.ET_BF16)
    ref = tr.train_forward(lf, meta, meta.w, meta.b, ckpt_every=8, want_I=True)["I"].clone()
    assert torch.isfinite(ref).all()
    lib = _lib.load()
    try:
        lib.et_set_wait_budget(0)
        bad = tr.train_forward(lf, meta, meta.w, meta.b, ckpt_every=8, want_I=True)["I"]
        torch.cuda.synchronize()
        assert torch.isnan(bad).all()
    finally:
        lib.et_set_wait_budget(-1)
    again = tr.train_forward(lf, meta, meta.w, meta.b, ckpt_every=8, want_I=True)["I"]
    assert torch.equal(again, ref)


def test_bf16_training_refuses_temporal_kernels_longer_than_7(tr):
    from paper_2508_18071_gb300 import _lib, api
    d = inputs.random_evsnet(1, 3, 8, 9, 1, seed=3)
    lf = torch.zeros((1, 5, 8, 8), device="cuda")
    meta = api.EvsNetDev.from_dict(d, _lib.ET_BF16)
    with pytest.raises(_lib.ETError) as e:
        tr.train_forward(lf, meta, meta.w, meta.b, ckpt_every=4)
    assert e.value.status == _lib.ET_ERR_UNIMPLEMENTED
    m32 = api.EvsNetDev.from_dict(d, _lib.ET_F32)
    tr.train_forward(lf, m32, m32.w, m32.b, ckpt_every=4)
