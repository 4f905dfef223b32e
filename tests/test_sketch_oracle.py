"""Pins of the learned-sketch oracle (oracle/sketch_mlp.py) against facts fixed outside it:
an independent BF16 cast, finite differences, conservation of leverage and diagonal mass,
and the plain method it must reduce to."""
import numpy as np
import pytest
import torch

from oracle import sketch_mlp as SM
from oracle import trg_oracle as O


def test_bf16_rounding_matches_torch():
    x = np.concatenate([np.random.default_rng(0).standard_normal(4000) * 10.0 ** np.arange(-8, 8, 4).repeat(1000),
                        [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -1.0 - 2 ** -8, 0.0, 65504.0]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(SM.bf16(x), ref)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    p = SM.init_params(3)
    X = rng.standard_normal((40, SM.NIN))
    t = rng.standard_normal(40)
    _, g = SM.loss_and_grads(p, X, t)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = SM.loss_and_grads(p, X, t)
            flat[idx] = old - h
            lm, _ = SM.loss_and_grads(p, X, t)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[name].reshape(-1)[idx]) <= 1e-6 * (1 + abs(fd)), (name, idx)


def test_bf16_inference_close_to_fp64_forward():
    p = SM.init_params(4)
    X = np.random.default_rng(2).standard_normal((64, SM.NIN))
    u64, _ = SM.forward(p, X)
    ub = SM.forward_bf16(p, X)
    assert np.abs(ub - u64).max() <= 0.03 * (1 + np.abs(u64).max())


def test_quantise_half_even_and_clamp():
    u = np.array([0.5, 1.5, 2.5, -0.5, 1e3, -1e3]) / SM.QSTEP
    assert np.array_equal(SM.quantise(u), [0.0, 2.0, 2.0, -0.0, 128.0, -128.0])


def test_features_and_leverage_conserve_mass():
    rng = np.random.default_rng(5)
    da, db, chi = 6, 4, 9
    A = rng.standard_normal((da * db, 30))
    rho = A @ A.T
    F1, F2 = SM.leg_features(rho, da, db, chi)
    for F, d in ((F1, da), (F2, db)):
        assert np.isclose((np.exp2(8 * F[:, 1]) / d).sum(), 1.0, rtol=1e-12)
        assert np.allclose(F[:, 4], chi / (da * db))
    Q = np.linalg.qr(rng.standard_normal((da * db, chi)))[0]
    t1, t2 = SM.leverage_targets(Q, da, db)
    assert np.isclose((np.exp2(2 * t1) / da).sum(), 1.0, rtol=1e-12)
    assert np.isclose((np.exp2(2 * t2) / db).sum(), 1.0, rtol=1e-12)


def test_zero_network_is_the_plain_method():
    """w = 1 everywhere: the learned form reduces to the paper's Gaussian sketch."""
    p = {k: v * 0.0 for k, v in SM.init_params(0).items()}
    a = O.run("ising", 4, 0.1497, 0.0, 6, 12, 4, mlp=p)
    b = O.run("ising", 4, 0.1497, 0.0, 6, 12, 4)
    assert O.free_energy(a) == O.free_energy(b)
    assert all(v["used"] in ("learned", "identity") for d in a.diag for v in d.get("sketch", {}).values())


def test_ideal_weights_reduce_one_pass_residual():
    """The reading's premise: with the exact leverages of the converged range as row
    weights, a one-pass range finder (q = 0) has a smaller probe residual than the plain
    Gaussian on a rho of the method (D = 8, step 4)."""
    caught = []
    orig = O.rsvd_range_sym

    def spy(rho, chi, q, key):
        f = __import__("sys")._getframe(1).f_locals
        if "chi_pair" in f:          # triad isometries only (not the squeezers)
            caught.append((rho.copy(), chi, key, f["d2"], f["d3"]))
        return orig(rho, chi, q, key)

    O.rsvd_range_sym = spy
    try:
        st = O.run("ising", 4, 0.1497, 0.0, 8, 16, 5)
    finally:
        O.rsvd_range_sym = orig
    ratios = []
    for rho, chi, key, da, db in caught[-4:]:
        n = rho.shape[0]
        if chi >= n:
            continue
        Q = orig(rho, chi, 6, key)
        t1, t2 = SM.leverage_targets(Q, da, db)
        w = (np.exp2(t1)[:, None] * np.exp2(t2)[None, :]).reshape(-1)
        G = O.gaussian(key, n, chi)
        kp = O.sketch_key(0x5EED, st.nsteps - 1, 13)
        rp = SM.probe_residual(rho, SM.range_finder(rho, G, chi, 0), kp)
        rl = SM.probe_residual(rho, SM.range_finder(rho, w[:, None] * G, chi, 0), kp)
        ratios.append(rl / rp)
    assert ratios and np.median(ratios) < 1.0, ratios
