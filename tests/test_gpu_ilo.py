"""ILO form (internal-line overspanning of the bond swap, Sec. II E and Appendix A) on
the GPU against the oracle's ILO form: the re-split and swapped bonds keep r_bond D
values.  FP64 form, same sketches on both sides; the configurations below have relative
gaps above 1e-3 at every cut (re-checked in the oracle).  Tolerances as the plain
parity tests: ln c_n per step 1e-11, lnZ/V 1e-10 relative, <s> 1e-9.
"""
import pytest

from oracle import trg_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trg(require_gpu):
    import paper_2507_21909_b300 as pkg
    yield pkg
    pkg.trg_set_bond_overspan(1)


@pytest.mark.parametrize("D,r_bond", [(5, 2), (3, 3), (6, 2)])
def test_ilo_parity(trg, D, r_bond):
    beta, h, p, nsteps = 0.16, 0.05, 2 * D, 8
    trg.trg_set_params(4, 4, 0x5EED, trg.TRG_PREC_FP64)
    trg.trg_set_bond_overspan(r_bond)
    try:
        trg.trg_init_ising(4, beta, h)
        st = O.init_ising(4, beta, h)
        for n in range(nsteps):
            trg.trg_step(n % 4, D, p)
            O.step(st, n % 4, D, p, 4, 4, 0x5EED, r_bond=r_bond)
            dg = st.diag[-1]
            assert min([dg["gap_swap"]] + list(dg["gap_sq"].values())) > 1e-3, n
            assert abs(trg.trg_diag()[0] - dg["log_c"]) < 1e-11, n
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
    f within 1e-8 relative of the oracle's ILO form (D = 7, bond 14, 12 steps; every cut
    has a relative gap above 3e-3)."""
    beta, D, r_bond, N = 0.1497, 7, 2, 12
    trg.trg_set_params(4, 4, 0x5EED, trg.TRG_PREC_OZ5)
    trg.trg_set_bond_overspan(r_bond)
    try:
        trg.trg_kernel_stats(reset=True)
        trg.trg_init_ising(4, beta, 0.0)
        for n in range(N):
            trg.trg_step(n % 4, D, 2 * D)
        f_gpu, _ = trg.trg_free_energy()
        assert trg.trg_kernel_stats(reset=True)["tc_launches"] > 0
    finally:
        trg.trg_set_bond_overspan(1)
        trg.trg_set_params(4, 4, 0x5EED, trg.TRG_PREC_FP64)
    st = O.run("ising", 4, beta, 0.0, D=D, p=2 * D, nsteps=N, r_bond=r_bond)
    f_ref, _ = O.free_energy(st)
    assert abs(f_gpu - f_ref) < 1e-8 * abs(f_ref)
