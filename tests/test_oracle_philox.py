"""Pins for the oracle's Philox4x32-10 (Salmon et al., SC'11)."""
import numpy as np
from scipy import stats

# Known-answer vectors published with the Random123 library for philox4x32-10:
# (counter words, key words) -> output words.
KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


def test_known_answer_vectors(orc):
    ctr = np.array([k[0] for k in KAT], np.uint32)
    key = np.array([k[1] for k in KAT], np.uint32)
    out = orc.philox4x32_10(ctr, key)
    assert out.tolist() == [list(k[2]) for k in KAT]


def test_uniformity_chi2(orc):
    n = 1 << 18
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n)
    ctr[:, 2] = 7
    key = np.tile(np.array([[1234, 0]], np.uint32), (n, 1))
    u = orc.u01(orc.philox4x32_10(ctr, key).ravel())
    assert u.min() >= 0.0 and u.max() < 1.0
    counts, _ = np.histogram(u, bins=256, range=(0, 1))
    p = stats.chisquare(counts).pvalue
    assert p > 1e-4
    # neighbouring counters are uncorrelated
    assert abs(np.corrcoef(u[:-1], u[1:])[0, 1]) < 0.01


def test_u01_resolution(orc):
    assert orc.u01(np.array([0, 255, 256, 0xFFFFFFFF], np.uint32)).tolist() == \
        [0.0, 0.0, 2.0 ** -24, 1.0 - 2.0 ** -24]
