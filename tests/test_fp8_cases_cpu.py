"""CPU check of the FP8 temporal parity cases (tests/test_gpu_evsnet_tct_fp8.py):
on every exact case the oracle's tensor-core layer inputs are representable in
E4M3 after their power-of-two scales (the premise of the bit-exact GPU
comparison), the oracle's currents are not trivially small and its BiLIF emits
events, so that the GPU test compares something."""
import numpy as np
import torch

import test_gpu_evsnet_tct_fp8 as T


def _oracle_events(I, vth, reset, beta):
    V = np.zeros(I.shape[1:])
    n = 0
    for k in range(I.shape[0]):
        V = beta * V + I[k]
        S = (V >= vth).astype(int) - (V <= -vth).astype(int)
        V = V - reset * S
        n += int(np.abs(S).sum())
    return n


def test_fp8_exact_cases_are_exact_and_carry_signal(orc):
    for form, H, W, seed in T.EXACT_CASES:
        d, lf, scales = T._exact_case(orc, form, H, W, seed)      # asserts the E4M3 premise
        assert all(s > 0 and np.log2(s) == int(np.log2(s)) for s in scales)
        X = torch.tensor(np.diff(lf.astype(np.float64), axis=0)[None])
        _, _, oI, _ = orc.torch_forward(X, orc.EvsNet.from_dict(d))
        I = oI[0].numpy()
        assert np.abs(I).max() > 0.2, form
        assert _oracle_events(I, d["vth"], d["reset"], d["beta"]) > 20, form
