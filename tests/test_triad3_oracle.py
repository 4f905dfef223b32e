"""Pins of the oracle's three-dimensional triad step (the d = 3 case discussed at the end
of Sec. II B): exact when untruncated (free energy, one-site and pair impurities), and
equal to plain ATRG when the triad isometries keep the whole pair space (chi = D^2),
over truncating steps."""
import math

import pytest

from oracle import trg_oracle as O
from tests.test_oracle_pins import brute_force
from tests.test_two_impurity_oracle import brute_force_nn


@pytest.mark.parametrize("L,axes", [((2, 1, 1), [0]), ((2, 2, 1), [0, 1]),
                                    ((2, 1, 2), [2, 0]), ((4, 1, 1), [0, 0])])
@pytest.mark.parametrize("beta,h", [(0.3, 0.0), (0.25, 0.2)])
def test_triad3_brute_force_untruncated(L, axes, beta, h):
    lz_b, m_b = brute_force(L, beta, h)
    st = O.init_ising(3, beta, h)
    pair = O.init_ising(3, beta, h, impurity="pair")
    for ax in axes:
        O.step(st, ax, D=16, p=256, q_swap=2)
        O.step(pair, ax, D=16, p=256, q_swap=2)
    _, lz = O.free_energy(st)
    assert abs(lz - lz_b) < 1e-13 * abs(lz_b)
    assert abs(O.magnetisation(st) - m_b) < 1e-13
    assert abs(O.nn_correlation(pair) - brute_force_nn(L, axes[0], beta, h)) < 1e-13


def test_triad3_beta_zero_impurities():
    st = O.run("ising", 3, 0.0, 0.3, D=4, p=4, nsteps=6)
    assert abs(O.magnetisation(st) - math.tanh(0.3)) < 1e-14
    pair = O.run("ising", 3, 0.0, 0.3, D=4, p=4, nsteps=6, impurity="pair")
    assert abs(O.nn_correlation(pair) - math.tanh(0.3) ** 2) < 1e-14


@pytest.mark.parametrize("D", [3, 4, 5])
def test_triad3_with_full_chi_equals_atrg(D):
    a = O.run("ising", 3, 0.25, 0.05, D=D, p=D * D, nsteps=6, q_swap=6, method="triad")
    b = O.run("ising", 3, 0.25, 0.05, D=D, p=D * D, nsteps=6, q_swap=6, method="atrg")
    assert abs(O.free_energy(a)[1] - O.free_energy(b)[1]) < 1e-12 * abs(O.free_energy(b)[1])
    for da, db in zip(a.diag, b.diag):
        assert abs(da["log_c"] - db["log_c"]) < 1e-11


def test_triad3_truncates_the_pair_space():
    """chi < D^2 really cuts: the step differs from ATRG (guards the pin above against a
    triad step that silently keeps everything)."""
    a = O.run("ising", 3, 0.25, 0.05, D=5, p=5, nsteps=6, q_swap=6, method="triad")
    b = O.run("ising", 3, 0.25, 0.05, D=5, p=5, nsteps=6, q_swap=6, method="atrg")
    assert abs(O.free_energy(a)[1] - O.free_energy(b)[1]) > 1e-9


def test_triad_rejects_d2():
    st = O.init_ising(2, 0.3, 0.0)
    with pytest.raises(ValueError):
        O.step(st, 0, 4, 8, method="triad")
