"""Pins of the oracle's ILO form (internal-line overspanning of the bond swap, Sec. II C
and Appendix A, r_bond > 1): the re-split and the swapped bond keep r_bond D values.

* r_bond = 1 is the plain method, bit for bit.
* Inside a step, the kept swap spectrum is the top r_bond D singular values of the
  bond-swap matrix M = sum_x C B formed directly from a re-split of width r_bond D.
* With untruncated triads (chi = D^2) the ILO triad step equals ILO ATRG over several
  truncating steps: the triad environments handle bond lines wider than D.
"""
import numpy as np
import pytest

from oracle import trg_oracle as O


def test_r_bond_one_is_the_plain_method():
    a = O.run("ising", 4, 0.16, 0.05, D=5, p=10, nsteps=4)
    b = O.run("ising", 4, 0.16, 0.05, D=5, p=10, nsteps=4, r_bond=1)
    assert O.free_energy(a) == O.free_energy(b)
    assert np.array_equal(a.phi, b.phi) and np.array_equal(a.psi, b.psi)


def test_rejects_r_bond_below_one():
    st = O.init_ising(4, 0.2, 0.0)
    with pytest.raises(ValueError):
        O.step(st, 0, 4, 8, r_bond=0)


@pytest.mark.parametrize("r_bond", [2, 3])
def test_step_keeps_top_r_bond_D_of_the_swap_spectrum(r_bond):
    D = 3
    st = O.run("ising", 4, 0.16, 0.05, D=D, p=2 * D, nsteps=2, r_bond=r_bond)
    ax = 2                                   # the third step of the axis cycle
    # the same rotation and re-split the step performs, then M formed directly
    sidx = st.axes.index(ax)
    order = [(sidx + i) % 4 for i in range(4)] + [4]
    phi = np.ascontiguousarray(st.phi.transpose(order))
    psi = np.ascontiguousarray(st.psi.transpose(order))
    A, Dm, s = O.resplit(phi, psi, r_bond * D)
    assert A.shape[-1] == min(r_bond * D, st.phi.shape[-1])
    C, B = A * s, Dm * s
    k, I = A.shape[-1], int(np.prod(A.shape[1:4]))
    M = np.einsum("xIJKb,xPQRa->aIJKbPQR", C, B).reshape(k * I, -1)
    ref = np.linalg.svd(M, compute_uv=False)
    O.step(st, ax, D, 2 * D, q_swap=12, r_bond=r_bond)
    sig = st.diag[-1]["sigma"]
    Db = min(r_bond * D, k * I)
    assert sig.size == Db
    live = ref[:Db] > 1e-12 * ref[0]
    assert np.allclose(sig[live], ref[:Db][live], rtol=1e-9)
    assert np.all(sig[~live] == 0.0)


@pytest.mark.parametrize("r_bond", [2])
def test_untruncated_ilo_triad_equals_ilo_atrg(r_bond):
    """chi = D^2 (no triad truncation): the ILO triad step and the ILO ATRG step share
    the re-split, the bond swap and the squeezer rule, so they agree over truncating
    steps (the plain form's identity, with bond lines of width r_bond D)."""
    D = 4
    a = O.run("ising", 4, 0.16, 0.05, D=D, p=D * D, nsteps=5, q_swap=6, method="triad",
              r_bond=r_bond)
    b = O.run("ising", 4, 0.16, 0.05, D=D, p=D * D, nsteps=5, q_swap=6, method="atrg",
              r_bond=r_bond)
    assert max(a.phi.shape[-1], b.phi.shape[-1]) > D          # the bond really is wider
    fa, fb = O.free_energy(a)[1], O.free_energy(b)[1]
    assert abs(fa - fb) < 1e-12 * abs(fb)
    for da, db in zip(a.diag, b.diag):
        assert abs(da["log_c"] - db["log_c"]) < 1e-11
