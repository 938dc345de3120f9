"""Helpers for the GPU parity tests."""
import numpy as np


def records_agree(rec_gpu, rec_orc):
    """Per pixel: True where every sample's path record (hit triangle per segment,
    light-sampling record) is identical on both sides.  [F,H,W,spp,D,2] -> [F,H,W]."""
    return (rec_gpu == rec_orc).all(axis=(-3, -2, -1))


def rel_close(a, b, rtol, atol):
    return np.abs(a - b) <= rtol * np.abs(b) + atol
