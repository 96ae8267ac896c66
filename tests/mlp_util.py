"""Seeded random classifier weights for the tests (an input generator: it holds
none of the method's arithmetic).  Parameter order: W1 (64x12), b1, W2 (64x64),
b2, w3, b3."""
import numpy as np

N_IN, N_H = 12, 64
SIZES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)), ("w3", (N_H,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)

# typical scale of each raw feature (cm, cm, cm, cm, cm, cm, -, -, -, -, -, -), used
# so that standardised inputs of real triplets are O(1)
FEATURE_MEAN = np.array([0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.66, 0.0, 0.0, 0.15, 0.15, 2.0], np.float32)
FEATURE_STD = np.array([0.5, 0.5, 1.0, 1.0, 0.2, 0.2, 0.2, 0.1, 0.2, 0.1, 0.1, 1.5], np.float32)


def zero_theta():
    return np.zeros(NPARAM, np.float32)


def theta_views(theta):
    out, off = {}, 0
    for name, shape in SIZES:
        size = int(np.prod(shape))
        out[name] = theta[off:off + size].reshape(shape)
        off += size
    return out


def random_net(seed, feature_scale=False):
    """(mean, inv_std, theta) with He-scaled weights and small biases."""
    rng = np.random.default_rng(seed)
    theta = zero_theta()
    v = theta_views(theta)
    v["W1"][:] = rng.standard_normal((N_H, N_IN)) * np.sqrt(2.0 / N_IN)
    v["b1"][:] = rng.standard_normal(N_H) * 0.1
    v["W2"][:] = rng.standard_normal((N_H, N_H)) * np.sqrt(2.0 / N_H)
    v["b2"][:] = rng.standard_normal(N_H) * 0.1
    v["w3"][:] = rng.standard_normal(N_H) * np.sqrt(1.0 / N_H)
    v["b3"][:] = rng.standard_normal(1) * 0.1
    if feature_scale:
        mean, inv_std = FEATURE_MEAN.copy(), (1.0 / FEATURE_STD).astype(np.float32)
    else:
        mean = rng.standard_normal(N_IN).astype(np.float32)
        inv_std = (0.5 + rng.random(N_IN)).astype(np.float32)
    return mean, inv_std, theta
