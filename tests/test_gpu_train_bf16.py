"""BF16 tensor-core training of the 3x3 form against the FP32 path and the oracle.

With net dtype ET_BF16 the C -> C convolutions (forward, data gradient and
weight gradient) take BF16 operands (unit roundoff u = 2^-8) on the tensor
cores with FP32 accumulation; layer 0, BiLIF and the loss are the FP32 path's.

* exact: on data whose weights and activations have few significant bits
  (+-1/2 weights, log steps in {-2..2}/4, zero biases, beta = 1) every rounding
  of the forward is exact, so the BF16 forward's spikes, currents and
  checkpoints equal the FP32 path's bit for bit: this pins the operand layout,
  the tap offsets, the tiles and the ragged image edges of the forward;
* bounded: on that same forward the backward rounds each layer's gradient dz
  (and, for the weight gradient, the activations) to BF16 (the +-1/2 weights
  are exact), so the weight gradients stay within 8 u (relative L2) of the
  FP32 path's and of the oracle's; a transposed, flipped or shifted operand
  gives O(1) errors;
* training: Adam steps with BF16 convolutions lower the loss of the denoising
  task as the FP32 ones do;
* a bounded MMA wait that runs out leaves NaN currents and a usable context."""
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


def _dyadic_net(seed, L, C):
    """Layer 0: one tap of +-1/2 per channel; layers 1..: one or two (input
    channel, tap) entries of +-1/2 per output channel; projection +-1; zero
    biases; beta = 1, Vth = reset = 1/16."""
    rng = np.random.default_rng(seed)
    d = inputs.random_evsnet(0, L, C, 1, 3, seed=seed, vth=0.0625, beta=1.0)
    w = np.zeros_like(d["w"])
    w0 = np.zeros((C, 9), np.float32)
    w0[np.arange(C), rng.integers(0, 9, C)] = rng.choice([-0.5, 0.5], C)
    w[:9 * C] = w0.ravel()
    off = 9 * C
    for _ in range(1, L):
        Wl = np.zeros((C, C * 9), np.float32)
        for co in range(C):
            k = rng.choice(C * 9, size=int(rng.integers(1, 3)), replace=False)
            Wl[co, k] = rng.choice([-0.5, 0.5], len(k))
        w[off:off + C * C * 9] = Wl.ravel()
        off += C * C * 9
    w[off:] = rng.choice([-1.0, 1.0], C)
    d["w"] = w
    d["b"] = np.zeros_like(d["b"])
    return d


def _dyadic_clips(seed, B, K, H, W):
    rng = np.random.default_rng(seed)
    steps = rng.integers(-2, 3, (B, K + 1, H, W)) / 4.0
    steps[:, 0] = 0
    return np.cumsum(steps, 1).astype(np.float32)


def _fwd_bwd(tr, d, lf, E, dtype, ck):
    from paper_2508_18071_gb300 import api
    meta = api.EvsNetDev.from_dict(d, dtype)
    lfd = torch.as_tensor(lf).cuda()
    out = tr.train_forward(lfd, meta, meta.w, meta.b, ckpt_every=ck, want_I=True)
    loss, dSon, dSoff = tr.emd_count_loss(out["spikes"], torch.as_tensor(E).cuda(), 0.01)
    gw, gb = tr.train_backward(lfd, meta, meta.w, meta.b, out["V_ckpt"], dSon, dSoff, ckpt_every=ck)
    return out, loss, np.concatenate([gw.cpu().numpy(), gb.cpu().numpy()]).astype(np.float64)


@pytest.mark.parametrize("B,K,H,W,L,C,ck", [(2, 20, 37, 45, 4, 16, 8), (1, 12, 64, 96, 3, 8, 12),
                                            (2, 16, 15, 32, 2, 16, 16), (1, 9, 31, 70, 4, 12, 4)])
def test_bf16_training_exact_forward_bounded_gradients(tr, orc, B, K, H, W, L, C, ck):
    from paper_2508_18071_gb300 import _lib
    d = _dyadic_net(5 + L + C, L, C)
    lf = _dyadic_clips(6 + W, B, K, H, W)
    E = np.random.default_rng(7).choice([-1, 0, 0, 0, 1], (B, K, H, W)).astype(np.float32)
    o32, l32, g32 = _fwd_bwd(tr, d, lf, E, _lib.ET_F32, ck)
    o16, l16, g16 = _fwd_bwd(tr, d, lf, E, _lib.ET_BF16, ck)
    assert (o32["spikes"] != 0).sum().item() > 10
    for k in ("spikes", "V_ckpt", "I"):
        np.testing.assert_array_equal(o16[k].cpu().numpy(), o32[k].cpu().numpy())
    # the loss sums per-block partials with atomics: equal up to their order
    assert abs(l16[0].item() - l32[0].item()) <= 1e-6 * abs(l32[0].item())
    assert np.abs(g32).max() > 0
    rel = np.linalg.norm(g16 - g32) / np.linalg.norm(g32)
    assert rel <= 8 * U_BF16, rel
    # and against the oracle (FP64 autograd of the same surrogate network)
    onet = orc.EvsNet(d["kind"], d["n_layers"], d["C"], d["kt"], d["ks"], d["beta"], d["vth"],
                      d["reset"], np.asarray(d["w"], np.float64), np.asarray(d["b"], np.float64))
    X = np.diff(lf.astype(np.float64), axis=1)
    _, rgw, rgb = orc.torch_grads(X, E, onet, smooth=False, alpha=2.0, lam=0.01)
    r = np.concatenate([rgw, rgb])
    assert np.linalg.norm(g16 - r) <= 8 * U_BF16 * np.linalg.norm(r)
    print("bf16 training L=%d C=%d: gradient relative L2 error %.2e u (FP32 path %.2e u)"
          % (L, C, rel / U_BF16, np.linalg.norm(g32 - r) / np.linalg.norm(r) / U_BF16))


def test_bf16_training_reduces_the_loss(tr, orc):
    """The denoising task of the FP32 trainer test: input = clean log clip +
    noise, target = contrast-threshold events of the clean clip; 40 Adam steps
    with BF16 convolutions cut the loss by a third, like the FP32 trainer."""
    from paper_2508_18071_gb300 import _lib
    B, K, H, W = 4, 32, 32, 32
    rng = np.random.default_rng(5)
    clean = np.stack([inputs.random_logl_clip(10 + b, K + 1, H, W, step_std=0.05, jump_p=0.01)
                      for b in range(B)])
    noisy = (clean + rng.normal(0, 0.15, clean.shape)).astype(np.float32)
    E = np.zeros((B, K, H, W), np.float32)
    for b in range(B):
        ev = orc.threshold_events(clean[b], 0.2, orc.ThresholdState.new(H, W))
        E[b] = orc.events_to_dense(ev, K, H, W, t0=1)
    d = inputs.random_evsnet(0, 3, 8, 1, 3, seed=4, vth=0.2, beta=0.95, std=0.2)
    x, e = torch.as_tensor(noisy).cuda(), torch.as_tensor(E).cuda()
    T16 = tr.Trainer(d, lr=1e-2, dtype=_lib.ET_BF16)
    losses = [T16.step(x, e)[0].item() for _ in range(40)]
    assert np.isfinite(losses).all()
    assert min(losses[-5:]) < 0.67 * losses[0], (losses[0], losses[-5:])


def test_bf16_training_wait_timeout_leaves_nan_and_recovers(tr):
    from paper_2508_18071_gb300 import _lib, api
    d = inputs.random_evsnet(0, 3, 16, 1, 3, seed=3, vth=0.2, beta=0.9, std=0.2)
    lf = torch.as_tensor(np.stack([inputs.random_logl_clip(3, 9, 24, 40, step_std=0.3)])).cuda()
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
