"""Plain ATRG on the GPU (the paper's comparison method, eqs. makeG / makeH) through the
C ABI: parity with the oracle's ATRG in d = 2, 3, 4 (FP64 form, same sketches; every
cut, range finders included, separated by a relative gap above 1e-2 in these
configurations), and the d = 2 free energy against Onsager's solution.
Tolerances: ln c_n per step 1e-11, lnZ/V 1e-10 relative; Onsager as the oracle's pin.
"""
import pytest

from oracle import trg_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trg(require_gpu):
    import paper_2507_21909_b300 as pkg
    return pkg


@pytest.mark.parametrize("d,D,nsteps,beta,h", [(2, 8, 12, 0.4, 0.01), (2, 12, 20, 0.35, 0.0),
                                               (3, 4, 6, 0.2, 0.02), (4, 4, 4, 0.16, 0.05)])
def test_atrg_parity(trg, d, D, nsteps, beta, h):
    trg.trg_set_params(4, 4, 0x5EED, trg.TRG_PREC_FP64)
    trg.trg_atrg_init_ising(d, beta, h)
    st = O.init_ising(d, beta, h)
    for n in range(nsteps):
        trg.trg_atrg_step(n % d, D, 2 * D)
        O.step(st, n % d, D, 2 * D, 4, 4, 0x5EED, method="atrg")
        assert abs(trg.trg_atrg_diag()[0] - st.diag[-1]["log_c"]) < 1e-11, n
    _, lz = trg.trg_atrg_free_energy()
    _, lz_ref = O.free_energy(st)
    assert abs(lz - lz_ref) < 1e-10 * abs(lz_ref)
    assert trg.trg_atrg_diag()[2] == nsteps


@pytest.mark.parametrize("beta", [0.3, 0.5])
def test_atrg_2d_onsager(trg, beta):
    """40 steps (L = 2^20) at D = 24: within 6e-8 of Onsager's lnZ/V, the oracle's bound."""
    from tests.test_oracle_pins import onsager_lnZ
    trg.trg_set_params(4, 4, 0x5EED, trg.TRG_PREC_FP64)
    trg.trg_atrg_init_ising(2, beta, 0.0)
    for n in range(40):
        trg.trg_atrg_step(n % 2, 24, 48)
    _, lz = trg.trg_atrg_free_energy()
    ex = onsager_lnZ(beta)
    assert abs(lz - ex) / ex < 6e-8


def test_atrg_errors(trg):
    with pytest.raises(trg.TrgError):
        trg.trg_atrg_init_ising(5, 0.2, 0.0)
    trg.trg_atrg_init_ising(2, 0.2, 0.0)
    with pytest.raises(trg.TrgError):
        trg.trg_atrg_step(2, 4, 8)                  # axis >= d
