"""Batched coupling sweep (S14): many instances on concurrent lanes against the oracle.

Each instance must give exactly what the single-instance path gives (the same kernels
in the same order), whatever the lane count, and match the FP64 oracle to 1e-10 in
ln Z/V (the instances below have relative gaps above 1e-3 at every cut; the test
re-checks that in the oracle).
"""
import numpy as np
import pytest

from oracle import trg_oracle as O

pytestmark = pytest.mark.gpu

# (model, beta, h, D): Ising (0) and Z3 clock (3) mixed
INST = [(0, 0.16, 0.05, 6), (3, 0.3, 0.05, 5), (0, 0.1497, 0.0, 5), (3, 0.25, 0.1, 6),
        (0, 0.14, 0.01, 6), (3, 0.3, 0.1, 7), (0, 0.145, 0.05, 5)]
NSTEPS = 5


@pytest.fixture(scope="module")
def trg(require_gpu):
    import paper_2507_21909_b300 as pkg
    return pkg


def _batch(trg, lanes, nsteps=NSTEPS, precision=0):
    model, beta, h, D = (list(x) for x in zip(*INST))
    n = trg.trg_batch_create(model, beta, h, D, lanes=lanes, q_swap=4, q_rho=4,
                             precision=precision)
    trg.trg_batch_step(2)
    trg.trg_batch_step(nsteps - 2)
    out = trg.trg_batch_results(n)
    trg.trg_batch_free()
    return out


def test_batch_matches_oracle(trg):
    out = _batch(trg, lanes=3)
    assert list(out["nsteps"]) == [NSTEPS] * len(INST)
    for i, (model, beta, h, D) in enumerate(INST):
        st = O.init_ising(4, beta, h) if model == 0 else O.init_clock(4, model, beta, h)
        for n in range(NSTEPS):
            O.step(st, n % 4, D, 2 * D, 4, 4, 0x5EED)
            dg = st.diag[-1]
            assert min([dg["gap_swap"]] + list(dg["gap_sq"].values())) > 1e-3, (i, n)
        f_ref, lz_ref = O.free_energy(st)
        assert abs(out["lnz"][i] - lz_ref) < 1e-10 * abs(lz_ref), (i, out["lnz"][i], lz_ref)
        assert abs(out["m"][i] - O.magnetisation(st)) < 1e-9, i


def test_lane_count_does_not_change_results(trg):
    a = _batch(trg, lanes=1)
    b = _batch(trg, lanes=4)
    for k in ("f", "lnz", "m"):
        assert np.array_equal(a[k], b[k]), k


def test_batch_equals_single_instance_path(trg):
    out = _batch(trg, lanes=2)
    trg.trg_set_params(4, 4, 0x5EED, trg.TRG_PREC_FP64)
    for i in (0, 3):
        model, beta, h, D = INST[i]
        if model == 0:
            trg.trg_init_ising(4, beta, h)
        else:
            trg.trg_init_clock(4, model, beta, h)
        for n in range(NSTEPS):
            trg.trg_step(n % 4, D, 2 * D)
        f, lz = trg.trg_free_energy()
        assert lz == out["lnz"][i] and f == out["f"][i]
        assert trg.trg_magnetisation_impurity() == out["m"][i]


def test_batch_mixed_precision_runs(trg):
    """The digit form on a batch (tensor-core GEMMs from the fourth step on): within the
    mixed form's error of the FP64 batch."""
    a = _batch(trg, lanes=3, nsteps=6, precision=0)
    b = _batch(trg, lanes=3, nsteps=6, precision=trg.TRG_PREC_OZ5)
    assert np.all(np.abs(a["lnz"] - b["lnz"]) < 1e-8 * np.abs(a["lnz"]))


def test_batch_rejects_bad_arguments(trg):
    with pytest.raises(trg.TrgError):
        trg.trg_batch_create([1], [0.1], [0.0], [4])      # q = 1 is not a model
    with pytest.raises(trg.TrgError):
        trg.trg_batch_step(1)                              # no batch


def test_batch_gu_wen_matches_single_instance(trg):
    model, beta, h, D = (list(x) for x in zip(*INST))
    n = trg.trg_batch_create(model, beta, h, D, lanes=3, precision=0)
    trg.trg_batch_step(NSTEPS)
    X = trg.trg_batch_gu_wen(n)
    trg.trg_batch_free()
    for i in (0, 1):
        m, b, hh, d = INST[i]
        st = O.init_ising(4, b, hh) if m == 0 else O.init_clock(4, m, b, hh)
        for k in range(NSTEPS):
            O.step(st, k % 4, d, 2 * d, 4, 4, 0x5EED)
        assert abs(X[i] - O.gu_wen_ratio(st)) < 1e-10
