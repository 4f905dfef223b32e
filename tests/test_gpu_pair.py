"""Two-impurity network (Sec. III D, internal energy) on the GPU, through the C ABI:
exhaustive enumeration on an untruncated lattice, and parity with the oracle's pair
(FP64 form, same sketches; beta = 0.16, h = 0.05, D = 6, p = 2D, q_swap = 5 has every
cut, range finders included, separated by a relative gap above 1e-2).  Tolerances: 1e-13 untruncated, 1e-9 absolute against the oracle.
"""
import math

import pytest

from oracle import trg_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trg(require_gpu):
    import paper_2507_21909_b300 as pkg
    return pkg


@pytest.mark.parametrize("axes", [(0, 1), (1, 0)])
def test_pair_brute_force_exact_on_gpu(trg, axes):
    """2x2x1x1 periodic lattice, untruncated: <s_x s_(x+e)> (e the first step's axis)
    equals exhaustive enumeration."""
    from tests.test_two_impurity_oracle import brute_force_nn
    ref = brute_force_nn((2, 2, 1, 1), axes[0], 0.25, 0.2)
    trg.trg_set_params(2, 4, 0x5EED, trg.TRG_PREC_FP64)
    trg.trg_init_ising(4, 0.25, 0.2)
    trg.trg_set_impurity_pair()
    for ax in axes:
        trg.trg_step(ax, 16, 256)
    assert abs(trg.trg_magnetisation_impurity() - ref) < 1e-13
    assert abs(trg.trg_internal_energy() + 4 * ref) < 4e-13


def test_pair_parity_with_oracle(trg):
    beta, h, D, p, nsteps = 0.16, 0.05, 6, 12, 8
    trg.trg_set_params(5, 4, 0x5EED, trg.TRG_PREC_FP64)
    trg.trg_init_ising(4, beta, h)
    trg.trg_set_impurity_pair()
    st = O.init_ising(4, beta, h, impurity="pair")
    for n in range(nsteps):
        trg.trg_step(n % 4, D, p)
        O.step(st, n % 4, D, p, 5, 4, 0x5EED)
        dg = st.diag[-1]
        assert min([dg["gap_swap"]] + list(dg["gap_sq"].values())) > 1e-3, n
    ref = O.nn_correlation(st)
    assert abs(trg.trg_magnetisation_impurity() - ref) < 1e-9
    assert abs(trg.trg_internal_energy() - O.internal_energy(st)) < 4e-9


def test_beta_zero_pair_is_tanh_squared(trg):
    trg.trg_set_params(4, 4, 1, trg.TRG_PREC_FP64)
    trg.trg_init_ising(4, 0.0, 0.3)
    trg.trg_set_impurity_pair()
    for ax in (0, 1, 2, 3):
        trg.trg_step(ax, 4, 4)
    assert abs(trg.trg_magnetisation_impurity() - math.tanh(0.3) ** 2) < 1e-14


def test_pair_errors_are_reported(trg):
    trg.trg_set_params(4, 4, 1, trg.TRG_PREC_FP64)
    trg.trg_init_ising(4, 0.2, 0.0)
    with pytest.raises(trg.TrgError):
        trg.trg_internal_energy()                 # no pair
    trg.trg_step(0, 4, 8)
    with pytest.raises(trg.TrgError):
        trg.trg_set_impurity_pair()               # after a step
    trg.trg_init_clock(4, 3, 0.2, 0.0)
    trg.trg_set_impurity_pair()
    trg.trg_step(0, 4, 8)
    with pytest.raises(trg.TrgError):
        trg.trg_internal_energy()                 # not the Ising model
    trg.trg_init_ising(4, 0.2, 0.0)               # a new model returns to one impurity
    trg.trg_step(0, 4, 8)
    with pytest.raises(trg.TrgError):
        trg.trg_internal_energy()
