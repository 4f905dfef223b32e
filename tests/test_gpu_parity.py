"""GPU (CUDA, FP64 form) against the FP64 CPU oracle, through the C ABI.

The oracle is the plain NumPy restatement of the paper's step; both sides draw the same
counter-based Gaussian sketches, so parity is at rounding level wherever the spectra at
the truncations are not degenerate.  Tolerance: f (and lnZ/V) to 1e-10 relative, ln c_n
per step to 1e-11 absolute, <s> to 1e-9 absolute.
"""
import math

import numpy as np
import pytest

from oracle import trg_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trg(require_gpu):
    import paper_2507_21909_b300 as pkg
    return pkg


def run_both(trg, beta, h, D, p, nsteps, q_swap=4, q_rho=4, seed=0x5EED, axes=None, model="ising"):
    trg.trg_set_params(q_swap, q_rho, seed, trg.TRG_PREC_FP64)
    if model == "ising":
        trg.trg_init_ising(4, beta, h)
        st = O.init_ising(4, beta, h)
    else:
        trg.trg_init_clock(4, 3, beta, h)
        st = O.init_clock(4, 3, beta, h)
    logc = []
    for n in range(nsteps):
        ax = n % 4 if axes is None else axes[n]
        trg.trg_step(ax, D, p)
        O.step(st, ax, D, p, q_swap, q_rho, seed)
        logc.append((trg.trg_diag()[0], st.diag[-1]["log_c"]))
        dg = st.diag[-1]
        gap = min([dg["gap_swap"]] + list(dg["gap_sq"].values()))
        # parity at rounding level needs a non-degenerate spectrum at every truncation
        assert gap > 1e-8, f"degenerate cut at step {n} (gap {gap:.1e}): pick another config"
    return st, logc


def test_config1_parity_d12_40_steps(trg):
    """Ising beta=0.1497, h=0, D=12, p=2D, q_swap=20, 40 steps (L = 2^10): f to 1e-10."""
    st, logc = run_both(trg, 0.1497, 0.0, 12, 24, 40, q_swap=20, q_rho=4)
    f_gpu, lz_gpu = trg.trg_free_energy()
    f_ref, lz_ref = O.free_energy(st)
    assert abs(f_gpu - f_ref) < 1e-10 * abs(f_ref)
    assert abs(lz_gpu - lz_ref) < 1e-10 * abs(lz_ref)
    for n, (a, b) in enumerate(logc[:12]):
        assert abs(a - b) < 1e-11, (n, a, b)


@pytest.mark.parametrize("D,p,nsteps", [(5, 3, 8), (7, 0, 6), (6, 12, 8)])
def test_ragged_and_small_parity(trg, D, p, nsteps):
    """Odd bond dimensions, p = 0 (no oversampling), tiles with ragged tails."""
    st, logc = run_both(trg, 0.16, 0.01, D, p, nsteps, q_swap=5)
    _, lz_gpu = trg.trg_free_energy()
    _, lz_ref = O.free_energy(st)
    assert abs(lz_gpu - lz_ref) < 1e-10 * abs(lz_ref)
    assert abs(trg.trg_magnetisation_impurity() - O.magnetisation(st)) < 1e-9


def test_impurity_parity_field(trg):
    st, _ = run_both(trg, 0.1497, 1e-4, 10, 20, 8, q_swap=10)
    assert abs(trg.trg_magnetisation_impurity() - O.magnetisation(st)) < 1e-9


def test_brute_force_exact_on_gpu(trg):
    """2x2x1x1 periodic lattice, untruncated: GPU equals exhaustive enumeration."""
    from tests.test_oracle_pins import brute_force
    lz_b, m_b = brute_force((2, 2, 1, 1), 0.25, 0.2)
    trg.trg_set_params(2, 4, 0x5EED, trg.TRG_PREC_FP64)
    trg.trg_init_ising(4, 0.25, 0.2)
    for ax in (0, 1):
        trg.trg_step(ax, 16, 256)
    _, lz = trg.trg_free_energy()
    assert abs(lz - lz_b) < 1e-13 * lz_b
    assert abs(trg.trg_magnetisation_impurity() - m_b) < 1e-13


def test_beta_zero_and_axis_order(trg):
    """beta = 0 product state; arbitrary axis order (two steps along the same axis)."""
    trg.trg_set_params(4, 4, 1, trg.TRG_PREC_FP64)
    trg.trg_init_ising(4, 0.0, 0.3)
    for ax in (2, 2, 0, 3):
        trg.trg_step(ax, 6, 6)
    f, lz = trg.trg_free_energy()
    assert math.isnan(f)
    assert abs(lz - math.log(2 * math.cosh(0.3))) < 1e-14
    assert abs(trg.trg_magnetisation_impurity() - math.tanh(0.3)) < 1e-14


def test_clock_model_parity(trg):
    st, _ = run_both(trg, 0.3, 0.02, 6, 6, 5, q_swap=5, model="clock")
    _, lz_gpu = trg.trg_free_energy()
    _, lz_ref = O.free_energy(st)
    assert abs(lz_gpu - lz_ref) < 1e-10 * abs(lz_ref)


def test_per_step_parity_from_oracle_state(trg):
    """Load the oracle state after 5 steps, run one GPU step and one oracle step from it:
    ln c_n, Tr T and the singular values of T (gauge invariants) agree."""
    st = O.run("ising", 4, 0.1497, 0.0, D=10, p=20, nsteps=5, q_swap=10)
    trg.trg_set_params(10, 4, 0x5EED, trg.TRG_PREC_FP64)
    trg.trg_set_state(st.beta, st.phi, st.psi, st.psi_imp, st.axes, st.nsteps, st.logsum)
    trg.trg_step(1, 10, 20)
    O.step(st, 1, 10, 20, 10, 4, 0x5EED)
    assert abs(trg.trg_diag()[0] - st.diag[-1]["log_c"]) < 1e-11
    phi, axes = trg.trg_get_state(0)
    psi, _ = trg.trg_get_state(1)
    assert axes == st.axes
    assert abs(O.trace_T(phi, psi) - O.trace_T(st.phi, st.psi)) < 1e-11 * abs(O.trace_T(st.phi, st.psi))

    def spectrum(a, b):
        r = a.shape[-1]
        _, Ra = np.linalg.qr(a.reshape(-1, r))
        _, Rb = np.linalg.qr(b.reshape(-1, r))
        return np.linalg.svd(Ra @ Rb.T, compute_uv=False)
    s_gpu, s_ref = spectrum(phi, psi), spectrum(st.phi, st.psi)
    assert np.allclose(s_gpu, s_ref, rtol=1e-10, atol=1e-13 * s_ref[0])


def test_mixed_form_oz5_within_1e8_of_oracle(trg):
    """The exact-accumulation mixed form (5 digits, tensor cores from the fourth step) keeps
    the free energy within 1e-8 relative of the FP64 oracle (16 steps, D=14, p=2D; at
    D=16 the bond swap of step 2 has a 4e-7 relative gap, too close to degenerate for a
    comparison across implementations)."""
    beta, D, N = 0.1497, 14, 16
    trg.trg_set_params(4, 4, 0x5EED, trg.TRG_PREC_OZ5)
    trg.trg_init_ising(4, beta, 0.0)
    for n in range(N):
        trg.trg_step(n % 4, D, 2 * D)
    f_gpu, _ = trg.trg_free_energy()
    trg.trg_set_params(4, 4, 0x5EED, trg.TRG_PREC_FP64)
    st = O.run("ising", 4, beta, 0.0, D=D, p=2 * D, nsteps=N, q_swap=4, q_rho=4)
    f_ref, _ = O.free_energy(st)
    assert abs(f_gpu - f_ref) < 1e-8 * abs(f_ref)


def test_errors_are_reported(trg):
    with pytest.raises(trg.TrgError) as e:
        trg.trg_init_ising(2, 0.1, 0.0)          # the triad step is defined for d = 3, 4
    assert e.value.code == -1
    with pytest.raises(trg.TrgError):
        trg.trg_init_ising(4, -0.1, 0.0)
    trg.trg_init_ising(4, 0.1, 0.0)
    with pytest.raises(trg.TrgError) as e:
        trg.trg_step(4, 6, 6)
    assert e.value.code == -1
    with pytest.raises(trg.TrgError):
        trg.trg_step(0, 0, 6)


def test_sliced_contraction_parity(trg, monkeypatch):
    """The coarse contraction sliced over its first leg (one row of t per slice here)
    gives the oracle's result; the slices are independent GEMM chains."""
    monkeypatch.setenv("TRG_STUDY", "slice_mb=1")
    st, _ = run_both(trg, 0.16, 0.05, 6, 12, 6)
    _, lz_gpu = trg.trg_free_energy()
    _, lz_ref = O.free_energy(st)
    assert abs(lz_gpu - lz_ref) < 1e-10 * abs(lz_ref)
    assert abs(trg.trg_magnetisation_impurity() - O.magnetisation(st)) < 1e-9


def test_gu_wen_ratio_parity(trg):
    """Gu-Wen X of the GPU state against the oracle's at every step, plus the initial
    tensor's closed form 2 / (1 + e^{-4 beta})."""
    trg.trg_set_params(4, 4, 0x5EED, trg.TRG_PREC_FP64)
    trg.trg_init_ising(4, 0.3, 0.0)
    assert abs(trg.trg_gu_wen_ratio() - 2.0 / (1.0 + math.exp(-1.2))) < 1e-13
    st, _ = run_both(trg, 0.16, 0.05, 6, 12, 6)
    assert abs(trg.trg_gu_wen_ratio() - O.gu_wen_ratio(st)) < 1e-10


def test_bench_configuration_full_size(trg):
    """The bench's launch configuration (D = 48, p = 2D, OZ5 form, beta = 0.1497): the
    first three steps (FP64 by the mixed forms' policy; still small enough for the oracle)
    match the oracle, and the steps that follow at full size keep every leg at D with a
    finite free energy and impurity observable (properties that hold at any size).  The
    early bond-swap cuts here are exactly degenerate (Z2), but both sides keep the span
    their common Gaussian sketch selects, so ln Z/V agrees (measured: <= 3e-12)."""
    trg.trg_set_params(4, 4, 0x5EED, trg.TRG_PREC_OZ5)
    trg.trg_init_ising(4, 0.1497, 0.0)
    st = O.init_ising(4, 0.1497, 0.0)
    for n in range(3):
        trg.trg_step(n % 4, 48, 96)
        O.step(st, n % 4, 48, 96, 4, 4, 0x5EED)
        f, lz = trg.trg_free_energy()
        f_ref, lz_ref = O.free_energy(st)
        assert abs(lz - lz_ref) < 1e-10 * abs(lz_ref), (n, lz, lz_ref)
    for n in range(3, 5):
        trg.trg_step(n % 4, 48, 96)
        f, lz = trg.trg_free_energy()
        assert math.isfinite(f) and math.isfinite(trg.trg_magnetisation_impurity())
    assert list(trg.trg_state_dims(0)) == [48] * 5


def test_mixed_form_oz5_at_size_vs_fp64_form(trg):
    """The exact-digit mixed form at a size where the tensor-core GEMMs run at scale
    (D = 32, p = 2D: split-K digit products with millions of rows, the int64 drain of
    every 512-deep chunk) against the library's FP64 form (itself pinned to the oracle
    at 1e-10): the bench's coupling (beta = 0.1497, h = 0), 8 steps, of which steps 3..7
    run on the tensor cores.  Per step: dF/F <= 1e-8 (the headline's tolerance) and
    ln c_n within 1e-6.  Both forms draw the same sketches."""
    D, N = 32, 8
    res = {}
    for prec in (trg.TRG_PREC_FP64, trg.TRG_PREC_OZ5):
        trg.trg_set_params(4, 4, 0x5EED, prec)
        trg.trg_init_ising(4, 0.1497, 0.0)
        f, lc, gap = [], [], []
        for n in range(N):
            trg.trg_step(n % 4, D, 2 * D)
            f.append(trg.trg_free_energy()[0])
            d = trg.trg_diag()
            lc.append(d[0])
            gap.append(d[1])
        res[prec] = (f, lc, gap)
    f64, lc64, gap64 = res[trg.TRG_PREC_FP64]
    fmx, lcmx, _ = res[trg.TRG_PREC_OZ5]
    for n in range(N):
        rel = abs(fmx[n] - f64[n]) / abs(f64[n])
        assert rel <= 1e-8, (n, rel, gap64[n])
        assert abs(lcmx[n] - lc64[n]) <= 1e-6, (n, lcmx[n], lc64[n], gap64[n])
    assert list(trg.trg_state_dims(0)) == [D] * 5


_F14 = {}


def _oracle_f_d14():
    if "f" not in _F14:
        st = O.run("ising", 4, 0.1497, 0.0, D=14, p=28, nsteps=16, q_swap=4, q_rho=4)
        _F14["f"] = O.free_energy(st)[0]
    return _F14["f"]


@pytest.mark.parametrize("name,bound", [("BF16X6", 1e-5), ("TF32X3", 1e-4)])
def test_split_forms_error_vs_oracle(trg, name, bound):
    """The FP32-accumulating split forms (6-product BF16 and 3xTF32, tensor cores from the
    fourth step): their free-energy error against the oracle at D = 14 (16 steps) stays
    at the FP32 level, far from the 1e-8 the exact-digit forms reach."""
    prec = getattr(trg, "TRG_PREC_" + name)
    trg.trg_kernel_stats(reset=True)
    trg.trg_set_params(4, 4, 0x5EED, prec)
    trg.trg_init_ising(4, 0.1497, 0.0)
    for n in range(16):
        trg.trg_step(n % 4, 14, 28)
    f, _ = trg.trg_free_energy()
    assert trg.trg_kernel_stats(reset=True)["tc_launches"] > 0
    trg.trg_set_params(4, 4, 0x5EED, trg.TRG_PREC_FP64)
    f_ref = _oracle_f_d14()
    assert abs(f - f_ref) < bound * abs(f_ref)
