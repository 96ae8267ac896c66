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


def bf16(a):
    """Round float32 values to BF16 (nearest, ties to even), returned as float32."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def logit_flip_bound(mean, inv_std, theta, feat):
    """Per-row bound on how far an FP32 tensor-core logit may legitimately sit from
    the FP64 one.  The first hidden layer is rounded to BF16 after an FP32 sum: a
    unit whose FP64 pre-activation lies within the FP32 error of the sum (plus 2^-16
    of its bias, which a kernel may carry as two BF16 parts) of a BF16 rounding
    midpoint may round to the neighbouring BF16 value.  Each such unit moves the
    logit by that step times its path to the output (W2 through the active second
    layer units, times w3).  Returns (bound of the flips, scale of the FP32 sums)."""
    v = theta_views(theta)
    g = (np.asarray(feat, np.float32) - mean.astype(np.float32)).astype(np.float32)
    x = bf16((g * inv_std.astype(np.float32)).astype(np.float32)).astype(np.float64)
    w1, w2, w3 = (bf16(v[k].astype(np.float32)).astype(np.float64) for k in ("W1", "W2", "w3"))
    b1, b2 = v["b1"].astype(np.float64), v["b2"].astype(np.float64)
    z1 = x @ w1.T + b1
    eps = 2.0 ** -19 * (np.abs(x) @ np.abs(w1).T + np.abs(b1)) + 2.0 ** -16 * np.abs(b1)
    h = lambda z: bf16(np.maximum(z, 0.0).astype(np.float32)).astype(np.float64)
    h1 = h(z1)
    step = np.maximum(np.abs(h(z1 - eps) - h1), np.abs(h(z1 + eps) - h1))  # 0 away from a midpoint
    z2 = h1 @ w2.T + b2
    path = np.abs((w2 * w3[:, None]).T[None, :, :] * (z2 > 0)[:, None, :]).sum(axis=2)  # [row, unit]
    flips = (step * path).sum(axis=1)
    scale = np.abs(h1) @ np.abs(w2).T + np.abs(b2)
    return flips, np.abs(w3) @ scale.T + 1.0
