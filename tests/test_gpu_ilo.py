"""ILO form (internal-line overspanning of the bond swap, Sec. II C and Appendix A) on
the GPU against the oracle's ILO form: the re-split and swapped bonds keep r_bond D
values.  FP64 form, same sketches on both sides.  Tolerances as the plain parity tests:
ln c_n per step 1e-11, lnZ/V 1e-10 relative, <s> 1e-9.

Rounding-level parity needs every truncation to be well separated, including the
range finders of the triad isometries and squeezers: where chi exceeds the numerical
rank of rho, the extra columns are arbitrary directions of rounding-level weight (an
amplitude near sqrt(eps) of the largest), and the two sides keep different ones.  The
oracle run below records the relative eigen-gap at every range-finder cut and the
configurations have all gaps above 1e-3.
"""
import numpy as np
import pytest

from oracle import trg_oracle as O

pytestmark = pytest.mark.gpu


def _oracle_with_gap_check(beta, h, D, r_bond, nsteps, q_swap=4):
    """The oracle's ILO run, asserting a relative gap > 1e-3 at every cut (bond swap,
    squeezers and every range finder); yields the state after each step."""
    orig = O.rsvd_range_sym
    cuts = []

    def spy(rho, chi, q, key):
        if chi < rho.shape[0]:
            ev = np.sort(np.linalg.eigvalsh(rho))[::-1]
            cuts.append((ev[chi - 1] - ev[chi]) / ev[chi - 1] if ev[chi - 1] > 0 else -1.0)
        return orig(rho, chi, q, key)

    st = O.init_ising(4, beta, h)
    O.rsvd_range_sym = spy
    try:
        for n in range(nsteps):
            cuts.clear()
            O.step(st, n % 4, D, 2 * D, q_swap, 4, 0x5EED, r_bond=r_bond)
            dg = st.diag[-1]
            gap = min([dg["gap_swap"]] + list(dg["gap_sq"].values()) + cuts)
            assert gap > 1e-3, f"near-degenerate cut at step {n} ({gap:.1e})"
            yield st
    finally:
        O.rsvd_range_sym = orig


@pytest.fixture(scope="module")
def trg(require_gpu):
    import paper_2507_21909_b300 as pkg
    yield pkg
    pkg.trg_set_bond_overspan(1)


@pytest.mark.parametrize("D,r_bond", [(6, 2), (3, 3), (3, 2)])
def test_ilo_parity(trg, D, r_bond):
    beta, h, nsteps = 0.16, 0.05, 8
    trg.trg_set_params(4, 4, 0x5EED, trg.TRG_PREC_FP64)
    trg.trg_set_bond_overspan(r_bond)
    try:
        trg.trg_init_ising(4, beta, h)
        for n, st in enumerate(_oracle_with_gap_check(beta, h, D, r_bond, nsteps)):
            trg.trg_step(n % 4, D, 2 * D)
            assert abs(trg.trg_diag()[0] - st.diag[-1]["log_c"]) < 1e-11, n
        dims = trg.trg_state_dims()
        assert dims[4] == st.phi.shape[-1] == r_bond * D     # the bond really is wider
        _, lz = trg.trg_free_energy()
        _, lz_ref = O.free_energy(st)
        assert abs(lz - lz_ref) < 1e-10 * abs(lz_ref)
        assert abs(trg.trg_magnetisation_impurity() - O.magnetisation(st)) < 1e-9
    finally:
        trg.trg_set_bond_overspan(1)


def test_ilo_mixed_form_oz5_within_1e8_of_oracle(trg):
    """The exact-digit mixed form with r_bond = 2 (tensor cores from the fourth step):
    f within 1e-8 relative of the oracle's ILO form (D = 7, bond 14, 12 steps)."""
    beta, h, D, r_bond, N = 0.16, 0.05, 7, 2, 12
    trg.trg_set_params(4, 4, 0x5EED, trg.TRG_PREC_OZ5)
    trg.trg_set_bond_overspan(r_bond)
    try:
        trg.trg_kernel_stats(reset=True)
        trg.trg_init_ising(4, beta, h)
        for n in range(N):
            trg.trg_step(n % 4, D, 2 * D)
        f_gpu, _ = trg.trg_free_energy()
        assert trg.trg_kernel_stats(reset=True)["oz_launches"] > 0
    finally:
        trg.trg_set_bond_overspan(1)
        trg.trg_set_params(4, 4, 0x5EED, trg.TRG_PREC_FP64)
    for st in _oracle_with_gap_check(beta, h, D, r_bond, N):
        pass
    f_ref, _ = O.free_energy(st)
    assert abs(f_gpu - f_ref) < 1e-8 * abs(f_ref)
