"""GPU step against the oracle step, element by element, from the same loaded state.

The oracle's state after five steps (every leg at D, field h != 0) is loaded into the
library with trg_set_state; one GPU step and one oracle step follow along the same
axis, for each of the four axes.  The coarse tensor T = Phi Psi^T (forward legs x
backward legs) is independent of the gauge of the bond gamma, and its pair legs carry
the squeezer's sign gauge, so both implementations must produce the same matrix entry by
entry; likewise the impurity tensor T_imp = Phi Psi_imp^T.  Tolerance 1e-10 of max|T|
(FP64 form; the cuts of these configurations are separated by >= 8e-3, asserted).
A second test does the same in the exact-digit mixed form (OZ5) from a state at D = 14,
where the tensor-core GEMMs run at a tile-spanning size, to 1e-7 of max|T|.
"""
import copy

import numpy as np
import pytest

from oracle import trg_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trg(require_gpu):
    import paper_2507_21909_b300 as pkg
    return pkg


def _T(phi, psi):
    r = phi.shape[-1]
    return phi.reshape(-1, r) @ psi.reshape(-1, r).T


def _one_step_both(trg, st0, axis, D, p, q_swap, prec):
    st = copy.deepcopy(st0)
    trg.trg_set_params(q_swap, 4, 0x5EED, prec)
    trg.trg_set_state(st.beta, st.phi, st.psi, st.psi_imp, st.axes, st.nsteps, st.logsum)
    trg.trg_step(axis, D, p)
    O.step(st, axis, D, p, q_swap, 4, 0x5EED)
    dg = st.diag[-1]
    gap = min([dg["gap_swap"]] + list(dg["gap_sq"].values()))
    assert gap > 1e-3, f"near-degenerate cut (gap {gap:.1e}): pick another configuration"
    phi, axes = trg.trg_get_state(0)
    psi, _ = trg.trg_get_state(1)
    psi_imp, _ = trg.trg_get_state(2)
    assert axes == st.axes
    assert phi.shape == st.phi.shape
    return st, phi, psi, psi_imp


@pytest.mark.parametrize("D,p", [(5, 10), (6, 12)])
@pytest.mark.parametrize("axis", [0, 1, 2, 3])
def test_coarse_tensor_elementwise_fp64(trg, D, p, axis):
    st0 = O.run("ising", 4, 0.16, 0.05, D=D, p=p, nsteps=5, q_swap=6, q_rho=4)
    st, phi, psi, psi_imp = _one_step_both(trg, st0, axis, D, p, 6, trg.TRG_PREC_FP64)
    T_ref, T = _T(st.phi, st.psi), _T(phi, psi)
    assert np.abs(T - T_ref).max() <= 1e-10 * np.abs(T_ref).max()
    Ti_ref, Ti = _T(st.phi, st.psi_imp), _T(phi, psi_imp)
    assert np.abs(Ti - Ti_ref).max() <= 1e-10 * np.abs(Ti_ref).max()
    assert abs(trg.trg_diag()[0] - st.diag[-1]["log_c"]) < 1e-12


def test_coarse_tensor_elementwise_mixed_form(trg):
    """Exact-digit form from a D = 14 state after 6 steps (the mixed form runs its bulk
    GEMMs on the tensor cores from the fourth step on, so this step does): T within 1e-7
    of max|T| (measured 2.5e-8 with the decompositions' products on the FP64 CUDA cores:
    the 35-bit digits' error, amplified by the cuts' sensitivity ~ 1 / gap)."""
    D, p = 14, 28
    st0 = O.run("ising", 4, 0.1497, 0.01, D=D, p=p, nsteps=6, q_swap=4, q_rho=4)
    st, phi, psi, psi_imp = _one_step_both(trg, st0, 2, D, p, 4, trg.TRG_PREC_OZ5)
    T_ref, T = _T(st.phi, st.psi), _T(phi, psi)
    assert np.abs(T - T_ref).max() <= 1e-7 * np.abs(T_ref).max()
    Ti_ref, Ti = _T(st.phi, st.psi_imp), _T(phi, psi_imp)
    # the impurity-only products run as 6-product BF16 splits (FP32 accumulation, 24-bit
    # slices): measured 1.0e-5 of max|T_imp|
    assert np.abs(Ti - Ti_ref).max() <= 1e-4 * np.abs(Ti_ref).max()
