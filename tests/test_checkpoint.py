"""Checkpoint/resume helpers (save_state / load_state): the .npz round trip, on stand-ins
for the device calls; and the scalar getter's error without a model (no GPU needed)."""
import ctypes

import numpy as np
import pytest


@pytest.fixture
def L():
    from paper_2507_21909_b300 import _lib
    return _lib


def test_get_scalars_without_model(L):
    lib = L.lib
    assert lib.trg_get_scalars(None, None, None) == -6


@pytest.mark.parametrize("with_imp", [True, False])
def test_save_load_round_trip(L, monkeypatch, tmp_path, with_imp):
    rng = np.random.default_rng(0)
    phi, psi, imp = (rng.standard_normal((3, 4, 5, 6, 7)) for _ in range(3))
    state = {0: phi, 1: psi, 2: imp if with_imp else None}

    def fake_get_state(which):
        if state[which] is None:
            raise L.TrgError(-1, "factor not present")
        return state[which], (2, 3, 0, 1)

    got = {}
    monkeypatch.setattr(L, "trg_get_state", fake_get_state)
    monkeypatch.setattr(L, "trg_get_scalars", lambda: (0.1497, 1.2345678901234567, 17))
    monkeypatch.setattr(L, "trg_set_state",
                        lambda *a: got.update(zip(("beta", "phi", "psi", "imp", "axes",
                                                   "nsteps", "logsum"), a)))
    path = str(tmp_path / "ck.npz")
    L.save_state(path)
    L.load_state(path)
    assert got["beta"] == 0.1497 and got["logsum"] == 1.2345678901234567
    assert got["nsteps"] == 17 and isinstance(got["nsteps"], int)
    assert got["axes"] == (2, 3, 0, 1)
    assert np.array_equal(got["phi"], phi) and np.array_equal(got["psi"], psi)
    assert (got["imp"] is None) != with_imp
    if with_imp:
        assert np.array_equal(got["imp"], imp)
