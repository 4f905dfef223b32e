"""Conditioning of the step sequence, on the oracle (CPU).

The free energy after n steps is a function of beta; a relative change of 1e-14 in beta
changes f directly by about 1e-14 (f is smooth in beta).  Whether the coarse-graining
steps keep it there depends on the cuts: where a truncation falls between (nearly)
degenerate singular values, the kept subspace is decided by rounding and the change is
amplified by many orders of magnitude.  This fixes what any two implementations of the
method (the oracle and the GPU, or two precision forms) can be expected to agree to:
  * D = 12 (the parity configuration): no amplification over six steps;
  * D = 8: the bond swap of the second step cuts an exactly degenerate pair (lattice
    symmetry), and f moves by more than 1e-6 for the 1e-14 change;
  * D = 16: a near-degenerate bond-swap cut at the third step amplifies it by more than
    1e4 there and more again at the fifth step.
"""
import pytest

from oracle import trg_oracle as O


def _run(D, n, beta):
    st = O.init_ising(4, beta, 0.0)
    fs = []
    for k in range(n):
        O.step(st, k % 4, D, 2 * D, 4, 4, 0x5EED)
        fs.append(O.free_energy(st)[0])
    return fs, st


def test_parity_configuration_is_well_conditioned():
    f0, _ = _run(12, 6, 0.1497)
    f1, _ = _run(12, 6, 0.1497 * (1 + 1e-14))
    for a, b in zip(f0, f1):
        assert abs(a - b) / abs(a) < 1e-13


def test_degenerate_cut_amplifies_rounding_level_changes():
    f0, st = _run(8, 2, 0.1497)
    f1, _ = _run(8, 2, 0.1497 * (1 + 1e-14))
    assert st.diag[1]["gap_swap"] < 1e-12          # an exactly degenerate pair at the cut
    assert abs(f0[1] - f1[1]) / abs(f0[1]) > 1e-6  # ... decided by rounding


def test_near_degenerate_cut_amplifies():
    """D = 16: the bond swap of the third step cuts between singular values 4e-7 apart
    (relative), and the 1e-14 change of beta comes out at the 1e-8 level there and grows
    further at the next full-size step."""
    f0, st = _run(16, 5, 0.1497)
    f1, _ = _run(16, 5, 0.1497 * (1 + 1e-14))
    assert st.diag[2]["gap_swap"] < 1e-5
    assert abs(f0[2] - f1[2]) / abs(f0[2]) > 1e-10
    assert abs(f0[4] - f1[4]) / abs(f0[4]) > 1e-8
