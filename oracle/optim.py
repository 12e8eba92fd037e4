"""FP64 CPU oracle of the splat optimiser step: Adam on the raw splat parameters with the
position noise of 3DGS-MCMC, and the 3DGS-MCMC relocation of dead splats with growth toward a
fixed splat budget.  SatSplat trains with Adam at the per-group learning rates of Supp. B and
relocates splats with the 3DGS-MCMC strategy under a bounded splat quota (Sec. 3.5, Sec. 4.4);
the update rules themselves are those of the cited works, restated here:

  - Adam (Kingma and Ba, Algorithm 1): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
    theta -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps);
  - 3DGS-MCMC position noise: mu += lr_means * noise_lr * sigmoid(-k (o - t)) * Sigma eta,
    eta ~ N(0, I), Sigma the splat's covariance;
  - 3DGS-MCMC relocation: every dead splat (opacity at or below a threshold) takes the
    parameters of a live one drawn with probability proportional to opacity; a live splat that
    is drawn N - 1 times shares its opacity and footprint among N copies:
      o' = 1 - (1 - o)^(1/N),
      s' = s * o / sum_{i=1}^{N} sum_{k=0}^{i-1} C(i-1, k) (-1)^k o'^(k+1) / sqrt(k+1)
    (the covariance rule of that work, per scale); the moments of every rewritten splat are
    reset.  Growth adds new splats the same way, up to the budget.

TEST INFRASTRUCTURE ONLY: only the test-suite may import this module.  It shares no code with
the CUDA path; the CUDA path never imports it.

Readings where the paper is silent:
  - raw parameters: means, log-scales (s = exp), quaternions (unnormalised), logit-opacity
    (o = 1 / (1 + exp(-x))) and rgb (identity); the rasterizer's gradients are with respect
    to the activated values, and the chain to the raw ones is part of the step;
  - the opacity learning rate (absent from Supp. B) defaults to 0.05; eps 1e-15;
  - a surfel's covariance is R diag(s_u^2, s_v^2, 0) R^T: the noise stays in its plane;
  - the noise is drawn after the Adam update, from the updated opacity, scales and rotation;
  - random numbers: Philox4x64-10 (Salmon et al., SC'11), key (seed, 0), counter
    (index, step, stream, 0); a uniform is ((x >> 40) + 0.5) 2^-24 and a normal pair comes from
    the Box-Muller transform of two uniforms;
  - opacity-proportional draws: integer weights floor(o * 2^24) of the live splats' stored
    opacities, r = floor(x W / 2^64) for the total W, and the source is the last splat whose
    exclusive prefix sum of weights is <= r (all in exact integer arithmetic);
  - the targets are the dead splats in index order, then the new slots; target j draws with
    counter (j, step, 1, 0); growth adds min(cap - n, floor(n * growth)) splats;
  - the copy count is capped at n_max (51); o' is clamped to [min_opacity, 1 - 2^-23].
"""
from __future__ import annotations

import math
from bisect import bisect_right

import numpy as np

# Philox4x64 constants (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as
# 1, 2, 3", SC'11): the two multipliers and the two Weyl key increments
PHILOX_M0 = 0xD2E7470EE14C6C93
PHILOX_M1 = 0xCA5A826395121157
PHILOX_W0 = 0x9E3779B97F4A7C15
PHILOX_W1 = 0xBB67AE8584CAA73B
MASK64 = (1 << 64) - 1

STREAM_NOISE = 0
STREAM_RELOCATE = 1

PARAM_ROWS = {"means": 3, "log_scales": 2, "quats": 4, "logit_opacity": 1, "rgb": 3}
GRAD_OF = {"means": "means", "log_scales": "scales", "quats": "quats", "logit_opacity": "opacity", "rgb": "rgb"}


def philox4x64(counter, key, rounds: int = 10):
    """One block of Philox4x64-R: four 64-bit outputs for a 4-word counter and a 2-word key."""
    c0, c1, c2, c3 = (int(v) & MASK64 for v in counter)
    k0, k1 = (int(v) & MASK64 for v in key)
    for r in range(rounds):
        if r > 0:
            k0 = (k0 + PHILOX_W0) & MASK64
            k1 = (k1 + PHILOX_W1) & MASK64
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        c0, c1, c2, c3 = ((p1 >> 64) ^ c1 ^ k0, p1 & MASK64, (p0 >> 64) ^ c3 ^ k1, p0 & MASK64)
    return c0, c1, c2, c3


def _mulhilo64(a, b):
    """(high, low) 64-bit words of the 128-bit products of uint64 arrays (32-bit limbs)."""
    m32 = np.uint64(0xFFFFFFFF)
    s32 = np.uint64(32)
    a_lo, a_hi = a & m32, a >> s32
    b_lo, b_hi = b & m32, b >> s32
    ll, hl, lh, hh = a_lo * b_lo, a_hi * b_lo, a_lo * b_hi, a_hi * b_hi
    cross = (ll >> s32) + (hl & m32) + (lh & m32)
    hi = hh + (hl >> s32) + (lh >> s32) + (cross >> s32)
    return hi, a * b


def philox4x64_vec(c0, c1, c2, c3, k0: int, k1: int, rounds: int = 10):
    """Philox4x64-R over uint64 counter arrays (the same generator as philox4x64, vectorised)."""
    with np.errstate(over="ignore"):
        c0, c1, c2, c3 = (np.asarray(c, np.uint64).copy() for c in (c0, c1, c2, c3))
        k0, k1 = np.uint64(k0 & MASK64), np.uint64(k1 & MASK64)
        m0, m1 = np.uint64(PHILOX_M0), np.uint64(PHILOX_M1)
        for r in range(rounds):
            if r > 0:
                k0 = np.uint64((int(k0) + PHILOX_W0) & MASK64)
                k1 = np.uint64((int(k1) + PHILOX_W1) & MASK64)
            hi0, lo0 = _mulhilo64(np.full_like(c0, m0), c0)
            hi1, lo1 = _mulhilo64(np.full_like(c2, m1), c2)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def mulhi64_vec(a, b):
    """floor(a b / 2^64) for uint64 arrays."""
    with np.errstate(over="ignore"):
        return _mulhilo64(np.asarray(a, np.uint64), np.asarray(b, np.uint64))[0]


def uniform24(x: int) -> float:
    """A uniform in (0, 1) from the top 24 bits of a 64-bit word (exact in float32)."""
    return ((x >> 40) + 0.5) / float(1 << 24)


def noise_normals(i: int, step: int, seed: int):
    """Three standard normals for splat i at Adam step `step` (Box-Muller on four uniforms)."""
    x = philox4x64((i, step, STREAM_NOISE, 0), (seed, 0))
    u = [uniform24(v) for v in x]
    r0 = math.sqrt(-2.0 * math.log(u[0]))
    r1 = math.sqrt(-2.0 * math.log(u[2]))
    return (r0 * math.cos(2.0 * math.pi * u[1]), r0 * math.sin(2.0 * math.pi * u[1]),
            r1 * math.cos(2.0 * math.pi * u[3]))


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def rotation(q):
    """R (3, 3, n) of unnormalised quaternions (w, x, y, z) [4, n]."""
    w, x, y, z = q / np.linalg.norm(q, axis=0)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def activated(raw: dict) -> dict:
    """The values the rasterizer reads: means, scales, quats, opacity, rgb."""
    return dict(means=raw["means"].copy(), scales=np.exp(raw["log_scales"]), quats=raw["quats"].copy(),
                opacity=sigmoid(raw["logit_opacity"]), rgb=raw["rgb"].copy())


def adam_update(x, m, v, g, lr: float, beta1: float, beta2: float, eps: float, step: int):
    """Adam with bias correction (Kingma and Ba, Algorithm 1) on arrays; returns (x, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** step)
    v_hat = v / (1.0 - beta2 ** step)
    return x - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def adam_step(raw: dict, m: dict, v: dict, grads: dict, lr: dict, beta1: float, beta2: float, eps: float,
              step: int, noise_lr: float = 0.0, noise_k: float = 100.0, noise_t: float = 0.005,
              seed: int = 0, index=None):
    """One optimiser step on copies of the raw parameters and moments ([C][n] float64 dicts).
    `grads` are with respect to the activated values (keys means, scales, quats, opacity, rgb);
    `lr` is keyed by raw parameter name.  `index` gives the splat index of each column (the
    counter of its noise draw; default 0..n-1).  Returns (raw, m, v, storage)."""
    raw = {k: np.array(a, np.float64) for k, a in raw.items()}
    m = {k: np.array(a, np.float64) for k, a in m.items()}
    v = {k: np.array(a, np.float64) for k, a in v.items()}
    # chain the gradients through the activations
    g = {k: np.array(grads[GRAD_OF[k]], np.float64).reshape(raw[k].shape) for k in raw}
    g["log_scales"] = g["log_scales"] * np.exp(raw["log_scales"])
    o = sigmoid(raw["logit_opacity"])
    g["logit_opacity"] = g["logit_opacity"] * o * (1.0 - o)
    for k in raw:
        raw[k], m[k], v[k] = adam_update(raw[k], m[k], v[k], g[k], lr[k], beta1, beta2, eps, step)
    if noise_lr != 0.0:
        raw["means"] = raw["means"] + position_noise(raw, lr["means"], noise_lr, noise_k, noise_t, step, seed,
                                                     index)
    return raw, m, v, activated(raw)


def position_noise(raw: dict, lr_means: float, noise_lr: float, k: float, t: float, step: int, seed: int,
                   index=None):
    """lr_means * noise_lr * sigmoid(-k (o - t)) * Sigma eta for every splat ([3, n]); column c
    draws with the counter of splat index[c] (default c)."""
    n = raw["means"].shape[1]
    idx = range(n) if index is None else [int(i) for i in index]
    o = sigmoid(raw["logit_opacity"][0])
    s = np.exp(raw["log_scales"])
    R = rotation(raw["quats"])
    eta = np.array([noise_normals(i, step, seed) for i in idx]).T  # [3, n]
    out = np.zeros((3, n))
    for i in range(n):
        Sigma = R[:, :, i] @ np.diag([s[0, i] ** 2, s[1, i] ** 2, 0.0]) @ R[:, :, i].T
        gate = 1.0 / (1.0 + math.exp(k * (o[i] - t)))
        out[:, i] = lr_means * noise_lr * gate * (Sigma @ eta[:, i])
    return out


def split_opacity(o: float, N: int, min_opacity: float) -> float:
    """o' with 1 - (1 - o')^N = o, clamped to [min_opacity, 1 - 2^-23]."""
    o_new = 1.0 - (1.0 - o) ** (1.0 / N)
    return min(max(o_new, min_opacity), 1.0 - 2.0 ** -23)


def split_scale_factor(o: float, o_new: float, N: int) -> float:
    """s' / s of the relocation rule: o over the double binomial sum."""
    den = 0.0
    for i in range(1, N + 1):
        for k in range(i):
            den += math.comb(i - 1, k) * (-1) ** k * o_new ** (k + 1) / math.sqrt(k + 1)
    return o / den


def grown_count(n_active: int, cap: int, growth: float) -> int:
    return min(cap, n_active + int(math.floor(n_active * float(np.float32(growth)))))


def relocate(raw: dict, m: dict, v: dict, stored_opacity, n_active: int, cap: int, min_opacity: float,
             growth: float, n_max: int, step: int, seed: int):
    """One relocation (and growth) on copies of the raw parameters and moments ([C][n_pad]).
    `stored_opacity` is the opacity the rasterizer reads (its float values).  Returns
    (raw, m, v, n_after, info) with info = dict(targets, sources, counts)."""
    raw = {k: np.array(a, np.float64) for k, a in raw.items()}
    m = {k: np.array(a, np.float64) for k, a in m.items()}
    v = {k: np.array(a, np.float64) for k, a in v.items()}
    thr = float(np.float32(min_opacity))
    o_st = [float(x) for x in np.asarray(stored_opacity, np.float64).reshape(-1)[:n_active]]
    dead = [x <= thr for x in o_st]
    w = [0 if d else int(math.floor(x * float(1 << 24))) for x, d in zip(o_st, dead)]
    W = sum(w)
    if W == 0:
        return raw, m, v, n_active, dict(targets=[], sources=[], counts={})
    n_after = grown_count(n_active, cap, growth)
    excl = [0] * n_active
    acc = 0
    for i in range(n_active):
        excl[i] = acc
        acc += w[i]
    targets = [i for i in range(n_active) if dead[i]] + list(range(n_active, n_after))
    sources, counts = [], {}
    for j in range(len(targets)):
        x = philox4x64((j, step, STREAM_RELOCATE, 0), (seed, 0))[0]
        r = (x * W) >> 64
        s = bisect_right(excl, r) - 1
        sources.append(s)
        counts[s] = counts.get(s, 0) + 1
    for s, c in counts.items():
        N = min(c + 1, n_max)
        o = float(sigmoid(raw["logit_opacity"][0, s]))
        o_new = split_opacity(o, N, thr)
        f = split_scale_factor(o, o_new, N)
        raw["logit_opacity"][0, s] = math.log(o_new / (1.0 - o_new))
        raw["log_scales"][:, s] = raw["log_scales"][:, s] + math.log(f)
        for k in raw:
            m[k][:, s] = 0.0
            v[k][:, s] = 0.0
    for t, s in zip(targets, sources):
        for k in raw:
            raw[k][:, t] = raw[k][:, s]
            m[k][:, t] = 0.0
            v[k][:, t] = 0.0
    return raw, m, v, n_after, dict(targets=targets, sources=sources, counts=counts)
