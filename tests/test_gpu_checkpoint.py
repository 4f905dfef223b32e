"""Checkpoint / resume on the GPU: a run saved after n steps (save_state: factors, axis
order, beta, running ln-norm sum, step count) and loaded into a fresh context
(load_state) continues exactly as the uninterrupted run, bit for bit (every kernel of
the step is deterministic: fixed reduction orders, split-K partials summed in a fixed
order, the sketches keyed by the step count)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trg(require_gpu):
    import paper_2507_21909_b300 as pkg
    return pkg


@pytest.mark.parametrize("prec_name,d", [("FP64", 4), ("OZ5", 4), ("FP64", 3)])
def test_resume_is_bit_identical(trg, tmp_path, prec_name, d):
    prec = getattr(trg, "TRG_PREC_" + prec_name)
    D, p, n_save, n_total = (10, 20, 5, 9) if d == 4 else (6, 6, 4, 8)

    def run(n0, n1):
        out = []
        for n in range(n0, n1):
            trg.trg_step(n % d, D, p)
            out.append((trg.trg_free_energy(), trg.trg_magnetisation_impurity()))
        return out

    trg.trg_set_params(4, 4, 0x5EED, prec)
    trg.trg_init_ising(d, 0.1497, 0.02)
    whole = run(0, n_total)

    trg.trg_init_ising(d, 0.1497, 0.02)
    first = run(0, n_save)
    path = str(tmp_path / "state.npz")
    trg.save_state(path)
    trg.trg_finalize()                       # the resumed run starts from a fresh context
    trg.trg_set_params(4, 4, 0x5EED, prec)
    trg.load_state(path)
    rest = run(n_save, n_total)
    assert first + rest == whole              # exact equality of every float
