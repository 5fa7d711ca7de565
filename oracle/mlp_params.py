"""Flat parameter layout of the MLP shared by the tests (W1[64][8], b1[64],
W2[64][64], b2[64], W3[4][64], b3[4]) -- TEST INFRASTRUCTURE."""
import numpy as np

ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def flatten(p):
    return np.concatenate([np.asarray(p[k], np.float64).reshape(-1) for k in ORDER])


def unflatten(v):
    shapes = {"W1": (64, 8), "b1": (64,), "W2": (64, 64), "b2": (64,), "W3": (4, 64), "b3": (4,)}
    out, o = {}, 0
    for k in ORDER:
        n = int(np.prod(shapes[k]))
        out[k] = np.asarray(v[o:o + n], np.float64).reshape(shapes[k])
        o += n
    return out
