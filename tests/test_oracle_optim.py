"""Pins of the optimiser oracle (Adam with the 3DGS-MCMC position noise, and the 3DGS-MCMC
relocation with growth), on CPU: an independent Philox implementation, torch's Adam and
autograd, closed forms, numerical integration and sampling statistics."""
import math

import numpy as np
import pytest
import torch

from oracle import optim as O


def _params(rng, n):
    return dict(means=rng.normal(0, 0.3, (3, n)), log_scales=np.log(rng.uniform(0.005, 0.05, (2, n))),
                quats=rng.normal(size=(4, n)), logit_opacity=rng.normal(0, 2, (1, n)), rgb=rng.uniform(0, 1, (3, n)))


def _zeros_like(p):
    return {k: np.zeros_like(a) for k, a in p.items()}


LR = dict(means=0.075, log_scales=0.001, quats=0.001, logit_opacity=0.05, rgb=0.0025)


def test_philox_matches_numpy():
    """numpy's Philox bit generator (4x64, 10 rounds) advances its counter by one before each
    block; its first block for counter c is the block of c + 1."""
    for counter, key in [((0, 0, 0, 0), (0, 0)), ((7, 3, 1, 0), (12345, 0)),
                         ((2 ** 64 - 2, 5, 9, 11), (2 ** 63 + 17, 2 ** 40 + 3))]:
        bg = np.random.Philox(counter=np.array(counter, np.uint64), key=np.array(key, np.uint64))
        ref = [int(x) for x in bg.random_raw(4)]
        c1 = ((counter[0] + 1) & O.MASK64,) + tuple(counter[1:])
        assert list(O.philox4x64(c1, key)) == ref


def test_noise_normals_are_standard_normal():
    from scipy import stats
    z = np.array([O.noise_normals(i, 3, 99) for i in range(20000)])
    for c in range(3):
        assert abs(z[:, c].mean()) < 0.03 and abs(z[:, c].var() - 1.0) < 0.04
        assert stats.kstest(z[:, c], "norm").pvalue > 1e-3
    assert abs(np.corrcoef(z[:, 0], z[:, 1])[0, 1]) < 0.03


def test_adam_without_noise_equals_torch_adam_on_the_raw_parameters():
    """The chained gradient through the activations (torch autograd) and torch.optim.Adam."""
    rng = np.random.default_rng(1)
    n = 50
    raw = _params(rng, n)
    m, v = _zeros_like(raw), _zeros_like(raw)
    tp = {k: torch.tensor(a, dtype=torch.float64, requires_grad=True) for k, a in raw.items()}
    opt = torch.optim.Adam([dict(params=[tp[k]], lr=LR[k]) for k in tp], betas=(0.9, 0.999), eps=1e-15)
    for step in range(1, 4):
        ga = dict(means=rng.normal(size=(3, n)), scales=rng.normal(size=(2, n)), quats=rng.normal(size=(4, n)),
                  opacity=rng.normal(size=(1, n)), rgb=rng.normal(size=(3, n)))
        raw, m, v, store = O.adam_step(raw, m, v, ga, LR, 0.9, 0.999, 1e-15, step)
        opt.zero_grad()
        act = dict(means=tp["means"], scales=torch.exp(tp["log_scales"]), quats=tp["quats"],
                   opacity=torch.sigmoid(tp["logit_opacity"]), rgb=tp["rgb"])
        loss = sum((act[k] * torch.tensor(ga[k])).sum() for k in act)
        loss.backward()
        opt.step()
        for k in raw:
            np.testing.assert_allclose(raw[k], tp[k].detach().numpy(), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(store["opacity"], 1 / (1 + np.exp(-raw["logit_opacity"])), rtol=1e-15)


def test_first_adam_step_moves_by_lr():
    """m_hat = g and v_hat = g^2 after one step: every parameter moves by lr g / (|g| + eps)."""
    rng = np.random.default_rng(2)
    raw = _params(rng, 10)
    g = dict(means=rng.normal(size=(3, 10)), scales=np.zeros((2, 10)), quats=np.zeros((4, 10)),
             opacity=np.zeros((1, 10)), rgb=np.zeros((3, 10)))
    new, _, _, _ = O.adam_step(raw, _zeros_like(raw), _zeros_like(raw), g, LR, 0.9, 0.999, 1e-8, 1)
    np.testing.assert_allclose(new["means"] - raw["means"], -0.075 * g["means"] / (np.abs(g["means"]) + 1e-8),
                               rtol=1e-12)
    np.testing.assert_array_equal(new["rgb"], raw["rgb"])


def test_noise_lies_in_the_surfel_plane_and_is_gated_by_opacity():
    rng = np.random.default_rng(3)
    n = 40
    raw = _params(rng, n)
    raw["logit_opacity"][0, :] = math.log(0.005 / 0.995)  # o = t: gate = 1/2
    noise = O.position_noise(raw, 0.075, 5e5, 100.0, 0.005, step=2, seed=7)
    R = O.rotation(raw["quats"])
    normal = R[:, 2, :]
    assert np.abs(np.sum(noise * normal, axis=0)).max() <= 1e-12 * np.abs(noise).max()
    # a flat splat (identity rotation): (s_u^2 eta_0, s_v^2 eta_1, 0) times lr noise_lr / 2
    raw["quats"][:, 0] = [2.0, 0.0, 0.0, 0.0]
    noise = O.position_noise(raw, 0.075, 5e5, 100.0, 0.005, step=2, seed=7)
    s = np.exp(raw["log_scales"][:, 0])
    eta = O.noise_normals(0, 2, 7)
    expect = 0.075 * 5e5 * 0.5 * np.array([s[0] ** 2 * eta[0], s[1] ** 2 * eta[1], 0.0])
    np.testing.assert_allclose(noise[:, 0], expect, rtol=1e-12, atol=1e-18)
    # an opaque splat gets (almost) none: sigmoid(-100 (0.9 - 0.005)) < 1e-38
    raw["logit_opacity"][0, 0] = math.log(0.9 / 0.1)
    assert np.abs(O.position_noise(raw, 0.075, 5e5, 100.0, 0.005, 2, 7)[:, 0]).max() < 1e-30


@pytest.mark.parametrize("o", [0.05, 0.4, 0.9, 0.99])
def test_split_preserves_the_composited_opacity_and_footprint(o):
    """N copies of opacity o' composite to o at the centre, and the integral of the composited
    1-D profile 1 - (1 - o' G'(x))^N equals that of o G(x): the property the scale rule
    is built on."""
    from scipy import integrate
    sigma = 0.7
    for N in (1, 2, 3, 5, 8):
        o_new = O.split_opacity(o, N, 0.005)
        assert 1 - (1 - o_new) ** N == pytest.approx(o, rel=1e-12)
        s_new = sigma * O.split_scale_factor(o, o_new, N)
        lhs, _ = integrate.quad(lambda x: 1 - (1 - o_new * math.exp(-x * x / (2 * s_new ** 2))) ** N, -50, 50,
                                limit=200)
        assert lhs == pytest.approx(o * sigma * math.sqrt(2 * math.pi), rel=1e-9)
    assert O.split_scale_factor(o, o, 1) == pytest.approx(1.0, rel=1e-15)


def _relocation_case(seed, n_active, cap, dead_frac):
    rng = np.random.default_rng(seed)
    raw = _params(rng, cap)
    dead = rng.uniform(size=n_active) < dead_frac
    raw["logit_opacity"][0, :n_active][dead] = -8.0  # o = 3.4e-4 < 0.005
    m = {k: rng.normal(size=a.shape) for k, a in raw.items()}
    v = {k: rng.uniform(size=a.shape) for k, a in raw.items()}
    stored = O.sigmoid(raw["logit_opacity"][0]).astype(np.float32)
    # dead: the stored opacity at or below the threshold (a few of the random ones are too)
    dead = stored[:n_active] <= np.float32(0.005)
    return raw, m, v, stored, dead


def test_relocation_moves_dead_splats_onto_sampled_live_ones():
    raw, m, v, stored, dead = _relocation_case(4, 300, 340, 0.1)
    new, m2, v2, n_after, info = O.relocate(raw, m, v, stored, 300, 340, 0.005, 0.05, 51, step=5, seed=11)
    assert n_after == 300 + 15
    assert info["targets"] == list(np.nonzero(dead)[0]) + list(range(300, 315))
    touched = set(info["targets"]) | set(info["counts"])
    for s in info["sources"]:
        assert not dead[s]
    for t, s in zip(info["targets"], info["sources"]):
        for k in new:
            np.testing.assert_array_equal(new[k][:, t], new[k][:, s])
            assert np.all(m2[k][:, t] == 0) and np.all(v2[k][:, t] == 0)
    for s, c in info["counts"].items():
        o = O.sigmoid(raw["logit_opacity"][0, s])
        assert 1 - (1 - O.sigmoid(new["logit_opacity"][0, s])) ** (c + 1) == pytest.approx(o, rel=1e-12)
        assert np.all(new["log_scales"][:, s] < raw["log_scales"][:, s])
        assert np.all(new["means"][:, s] == raw["means"][:, s])
    for i in range(340):
        if i not in touched:
            for k in new:
                np.testing.assert_array_equal(new[k][:, i], raw[k][:, i])
                np.testing.assert_array_equal(m2[k][:, i], m[k][:, i])


def test_relocation_draws_in_proportion_to_opacity():
    """20000 targets over five live splats: frequencies within 5 binomial standard deviations of
    o_i / sum(o); the dead splats are never drawn."""
    n = 20005
    raw = dict(means=np.zeros((3, n)), log_scales=np.zeros((2, n)), quats=np.tile([[1.0], [0], [0], [0]], (1, n)),
               logit_opacity=np.full((1, n), -9.0), rgb=np.zeros((3, n)))
    ops = np.array([0.9, 0.5, 0.2, 0.05, 0.01])
    raw["logit_opacity"][0, :5] = np.log(ops / (1 - ops))
    stored = O.sigmoid(raw["logit_opacity"][0]).astype(np.float32)
    z = {k: np.zeros_like(a) for k, a in raw.items()}
    _, _, _, _, info = O.relocate(raw, z, z, stored, n, n, 0.005, 0.0, 51, step=1, seed=3)
    assert len(info["targets"]) == n - 5
    freq = np.bincount(info["sources"], minlength=5) / (n - 5)
    p = stored[:5].astype(np.float64) / stored[:5].astype(np.float64).sum()
    assert np.all(np.abs(freq - p) <= 5 * np.sqrt(p * (1 - p) / (n - 5)))


def test_no_live_splat_means_no_relocation():
    raw, m, v, stored, _ = _relocation_case(5, 20, 30, 1.1)
    new, _, _, n_after, info = O.relocate(raw, m, v, stored, 20, 30, 0.005, 0.05, 51, 1, 1)
    assert n_after == 20 and info["targets"] == []
    for k in new:
        np.testing.assert_array_equal(new[k], raw[k])


def test_growth_stops_at_the_budget():
    assert O.grown_count(1000, 1030, 0.05) == 1030
    assert O.grown_count(1000, 5000, 0.05) == 1050
    assert O.grown_count(7, 100, 0.05) == 7
