"""The three-dimensional triad step on the GPU (the d = 3 case whose O(r^2 D^6) cost the
paper gives at the end of Sec. II B) against the oracle's 3D step, through the C ABI.

Same tolerances as the 4D parity tests: ln c_n per step to 1e-11, ln Z/V to 1e-10
relative, <s> and <s s'> to 1e-9 (FP64 form), the coarse tensor T = Phi Psi^T element by
element to 1e-10 of max|T| from a loaded oracle state; untruncated runs equal exhaustive
enumeration to 1e-13.  The configurations have every cut separated (asserted on the
oracle's gaps).
"""
import copy

import numpy as np
import pytest

from oracle import trg_oracle as O
from tests.test_oracle_pins import brute_force
from tests.test_two_impurity_oracle import brute_force_nn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trg(require_gpu):
    import paper_2507_21909_b300 as pkg
    return pkg


def _gap(dg):
    return min([dg["gap_swap"]] + list(dg["gap_sq"].values()))


@pytest.mark.parametrize("D,p,beta,h", [(4, 4, 0.2, 0.05), (6, 6, 0.2, 0.05),
                                        (6, 12, 0.22, 0.02)])
def test_triad3_parity_per_step(trg, D, p, beta, h):
    trg.trg_set_params(6, 4, 0x5EED, trg.TRG_PREC_FP64)
    trg.trg_init_ising(3, beta, h)
    st = O.init_ising(3, beta, h)
    for n in range(12):
        trg.trg_step(n % 3, D, p)
        O.step(st, n % 3, D, p, 6, 4, 0x5EED)
        assert _gap(st.diag[-1]) > 1e-3, n
        assert abs(trg.trg_diag()[0] - st.diag[-1]["log_c"]) < 1e-11, n
    _, lz = trg.trg_free_energy()
    _, lz_ref = O.free_energy(st)
    assert abs(lz - lz_ref) < 1e-10 * abs(lz_ref)
    assert abs(trg.trg_magnetisation_impurity() - O.magnetisation(st)) < 1e-9
    assert trg.trg_state_dims(0) == st.phi.shape


@pytest.mark.parametrize("L,axes", [((2, 2, 1), [0, 1]), ((2, 1, 2), [2, 0]),
                                    ((4, 1, 1), [0, 0])])
def test_triad3_untruncated_equals_enumeration(trg, L, axes):
    beta, h = 0.25, 0.2
    lz_b, m_b = brute_force(L, beta, h)
    trg.trg_set_params(2, 4, 0x5EED, trg.TRG_PREC_FP64)
    trg.trg_init_ising(3, beta, h)
    for ax in axes:
        trg.trg_step(ax, 16, 256)
    _, lz = trg.trg_free_energy()
    assert abs(lz - lz_b) < 1e-13 * lz_b
    assert abs(trg.trg_magnetisation_impurity() - m_b) < 1e-13
    # the nearest-neighbour pair along the first step's axis
    trg.trg_init_ising(3, beta, h)
    trg.trg_set_impurity_pair()
    for ax in axes:
        trg.trg_step(ax, 16, 256)
    assert abs(trg.trg_magnetisation_impurity() - brute_force_nn(L, axes[0], beta, h)) < 1e-13


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_triad3_coarse_tensor_elementwise(trg, axis):
    D, p = 6, 6
    st0 = O.run("ising", 3, 0.2, 0.05, D=D, p=p, nsteps=7, q_swap=6, q_rho=4)
    st = copy.deepcopy(st0)
    trg.trg_set_params(6, 4, 0x5EED, trg.TRG_PREC_FP64)
    trg.trg_set_state(st.beta, st.phi, st.psi, st.psi_imp, st.axes, st.nsteps, st.logsum)
    trg.trg_step(axis, D, p)
    O.step(st, axis, D, p, 6, 4, 0x5EED)
    assert _gap(st.diag[-1]) > 1e-3
    phi, axes = trg.trg_get_state(0)
    psi, _ = trg.trg_get_state(1)
    psi_imp, _ = trg.trg_get_state(2)
    assert axes == st.axes and phi.shape == st.phi.shape
    r = phi.shape[-1]
    T = phi.reshape(-1, r) @ psi.reshape(-1, r).T
    T_ref = st.phi.reshape(-1, r) @ st.psi.reshape(-1, r).T
    assert np.abs(T - T_ref).max() <= 1e-10 * np.abs(T_ref).max()
    Ti = phi.reshape(-1, r) @ psi_imp.reshape(-1, r).T
    Ti_ref = st.phi.reshape(-1, r) @ st.psi_imp.reshape(-1, r).T
    assert np.abs(Ti - Ti_ref).max() <= 1e-10 * np.abs(Ti_ref).max()


def test_triad3_pair_internal_energy(trg):
    """Two-impurity network in 3D: <s s'> and U = -3 <s s'> against the oracle."""
    beta, h, D, p = 0.2, 0.05, 6, 6
    trg.trg_set_params(6, 4, 0x5EED, trg.TRG_PREC_FP64)
    trg.trg_init_ising(3, beta, h)
    trg.trg_set_impurity_pair()
    st = O.init_ising(3, beta, h, impurity="pair")
    for n in range(9):
        trg.trg_step(n % 3, D, p)
        O.step(st, n % 3, D, p, 6, 4, 0x5EED)
    assert abs(trg.trg_magnetisation_impurity() - O.nn_correlation(st)) < 1e-9
    assert abs(trg.trg_internal_energy() - O.internal_energy(st)) < 3e-9


def test_triad3_mixed_form_oz5(trg):
    """The exact-digit mixed form in 3D (D = 12): f within 1e-8 relative of the oracle,
    with digit-GEMM launches on the tensor cores."""
    beta, h, D, N = 0.2, 0.01, 12, 12
    trg.trg_kernel_stats(reset=True)
    trg.trg_set_params(6, 4, 0x5EED, trg.TRG_PREC_OZ5)
    trg.trg_init_ising(3, beta, h)
    for n in range(N):
        trg.trg_step(n % 3, D, D)
    f, _ = trg.trg_free_energy()
    assert trg.trg_kernel_stats(reset=True)["oz_launches"] > 0
    trg.trg_set_params(6, 4, 0x5EED, trg.TRG_PREC_FP64)
    st = O.run("ising", 3, beta, h, D=D, p=D, nsteps=N, q_swap=6, q_rho=4)
    f_ref, _ = O.free_energy(st)
    assert abs(f - f_ref) < 1e-8 * abs(f_ref)


def test_triad3_rejects_axis_3(trg):
    trg.trg_init_ising(3, 0.2, 0.0)
    with pytest.raises(trg.TrgError) as e:
        trg.trg_step(3, 4, 4)
    assert e.value.code == -1
