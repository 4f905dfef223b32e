"""Pins of the oracle's two-impurity network (Sec. III D: the internal energy from two
impurity tensors): the nearest-neighbour product of the observable on the first step's
unit cell.

* Untruncated runs on lattices of at most 4 sites equal the brute-force correlation
  <s_x s_(x+e)> (e the first step's axis), with and without a field.
* beta = 0: independent sites, <s s'> = tanh(h)^2 at any D.
* The flag is consumed by the first step and the pair is rejected before it.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import trg_oracle as O


def brute_force_nn(L, axis, beta, h):
    """<s_0 s_(0+e_axis)> on the periodic Ising lattice L by enumeration."""
    d = len(L)
    sites = list(itertools.product(*[range(l) for l in L]))
    idx = {x: i for i, x in enumerate(sites)}
    bonds = []
    for x in sites:
        for mu in range(d):
            y = list(x)
            y[mu] = (y[mu] + 1) % L[mu]
            bonds.append((idx[x], idx[tuple(y)]))
    bonds = np.array(bonds)
    confs = np.array(list(itertools.product([1.0, -1.0], repeat=len(sites))))
    E = (confs[:, bonds[:, 0]] * confs[:, bonds[:, 1]]).sum(axis=1)
    w = np.exp(beta * E + h * confs.sum(axis=1))
    e = [0] * d
    e[axis] = 1 % L[axis]
    j = idx[tuple(e)]
    return float((confs[:, 0] * confs[:, j] * w).sum() / w.sum())


@pytest.mark.parametrize("L,axes", [((2, 1, 1, 1), [0]), ((2, 2, 1, 1), [0, 1]),
                                    ((2, 2, 1, 1), [1, 0]), ((4, 1, 1, 1), [0, 0]),
                                    ((1, 2, 1, 2), [3, 1])])
@pytest.mark.parametrize("beta,h", [(0.3, 0.0), (0.25, 0.2)])
def test_pair_equals_brute_force_untruncated(L, axes, beta, h):
    ref = brute_force_nn(L, axes[0], beta, h)
    st = O.init_ising(4, beta, h, impurity="pair")
    for ax in axes:
        O.step(st, ax, D=16, p=256, q_swap=2)
    assert abs(O.nn_correlation(st) - ref) < 1e-12, (O.nn_correlation(st), ref)


def test_pair_differs_from_site_impurity():
    """Guards the pin above against a pair that silently falls back to one impurity."""
    L, axes, beta, h = (2, 2, 1, 1), [0, 1], 0.25, 0.2
    st = O.init_ising(4, beta, h, impurity="site")
    for ax in axes:
        O.step(st, ax, D=16, p=256, q_swap=2)
    assert abs(O.magnetisation(st) - brute_force_nn(L, 0, beta, h)) > 1e-3


@pytest.mark.parametrize("h", [0.0, 0.3])
def test_beta_zero_is_independent_sites(h):
    st = O.run("ising", 4, 0.0, h, D=3, p=3, nsteps=6, impurity="pair")
    assert abs(O.nn_correlation(st) - math.tanh(h) ** 2) < 1e-13


def test_pair_flag_consumed_and_checked():
    st = O.init_ising(4, 0.2, 0.0, impurity="pair")
    with pytest.raises(ValueError):
        O.nn_correlation(st)
    O.step(st, 0, 4, 8)
    assert not st.imp_pair
    with pytest.raises(ValueError):
        O.init_ising(4, 0.2, 0.0, impurity="triple")
