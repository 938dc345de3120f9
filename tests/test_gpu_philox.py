"""The device Philox4x32-10 (the renderer's and the sensor model's generator)
against the oracle's, written independently from the published definition and
pinned by the Random123 known-answer vectors (tests/test_oracle_philox.py):
bitwise on 10^6 counters -- random ones, the renderer's own (pixel, sample,
frame, word) counters with word = 0 and 4b + 1 / 4b + 2, and the extreme
values 0 and 2^32 - 1 in every word -- under random and extreme keys."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def test_gpu_philox_equals_oracle_on_a_million_counters(orc):
    from paper_2508_18071_gb300 import api
    rng = np.random.default_rng(13)
    n_rand = 600_000
    ctr = [rng.integers(0, 2 ** 32, (n_rand, 4), dtype=np.uint64)]
    # the renderer's counters: pixel of a 1280 x 720 frame, sample, frame, word
    m = 300_000
    pix = rng.integers(0, 1280 * 720, m)
    smp = rng.integers(0, 256, m)
    frame = rng.integers(0, 100_000, m)
    word = rng.choice([0, 1, 2, 5, 6, 9, 10, 17, 18], m)
    ctr.append(np.stack([pix, smp, frame, word], 1).astype(np.uint64))
    # extremes: every combination of 0 / 2^32 - 1 / 1 per word
    ext = np.array(np.meshgrid(*[[0, 1, 2 ** 32 - 1]] * 4)).reshape(4, -1).T
    ctr.append(np.repeat(ext, (100_000 - 0) // len(ext) + 1, 0)[:100_000].astype(np.uint64))
    ctr = np.concatenate(ctr).astype(np.uint32)
    n = len(ctr)
    assert n == 1_000_000
    key = rng.integers(0, 2 ** 32, (n, 2), dtype=np.uint64).astype(np.uint32)
    key[:1000] = 0
    key[1000:2000] = 0xFFFFFFFF
    key[-100_000:] = np.array([0x12345678, 0x9ABCDEF0], np.uint32)
    ref = orc.philox4x32_10(ctr, key)
    got = api.philox4x32_10(_dev(ctr), _dev(key)).cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(got, ref)


def test_gpu_philox_rejects_bad_arguments():
    from paper_2508_18071_gb300 import _lib
    lib = _lib.load()
    buf = torch.zeros(64, dtype=torch.int32, device="cuda")
    p = buf.data_ptr()
    assert lib.et_philox4x32_10(p, p, -1, p, None) == _lib.ET_ERR_ARG
    assert lib.et_philox4x32_10(p + 4, p, 1, p, None) == _lib.ET_ERR_ARG     # counters not 16-byte aligned
    assert lib.et_philox4x32_10(p, p, 0, p, None) == _lib.ET_OK
