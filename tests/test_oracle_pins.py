"""Pins of the FP64 oracle to results that do not come from the oracle itself.

Each test fixes a quantity by the mathematics (closed forms, brute-force enumeration,
published generator outputs, exact algebraic identities) so that a dropped term, a
wrong sign, a swapped index or a transposed operand in the oracle fails one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import trg_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------- generator
def test_splitmix64_published_outputs():
    """mix64(k * golden) for k = 1..3 is SplitMix64 seeded with 0 (published values)."""
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as f:
        ref = [int(l, 16) for l in f if l.strip() and not l.startswith("#")]
    with np.errstate(over="ignore"):
        got = [int(O._mix64(O._GOLDEN * np.uint64(k))) for k in (1, 2, 3)]
    assert got == ref


def test_gaussian_sketch_moments_and_determinism():
    key = O.sketch_key(0x5EED, 3, 7)
    g = O.gaussian(key, 400, 250)
    assert np.array_equal(g, O.gaussian(key, 400, 250))
    assert abs(g.mean()) < 0.01 and abs(g.var() - 1.0) < 0.02
    assert abs(np.mean(g ** 4) - 3.0) < 0.1            # kurtosis of a normal
    assert not np.array_equal(g, O.gaussian(O.sketch_key(0x5EED, 3, 8), 400, 250))


# ------------------------------------------------------------------ exact limits
@pytest.mark.parametrize("h", [0.0, 0.3, -0.7])
def test_beta_zero_ising(h):
    """beta = 0: product state, lnZ/V = ln(2 cosh h) and <s> = tanh h."""
    st = O.run("ising", 4, 0.0, h, D=6, p=12, nsteps=5)
    _, lz = O.free_energy(st)
    assert abs(lz - math.log(2 * math.cosh(h))) < 1e-14
    assert abs(O.magnetisation(st) - math.tanh(h)) < 1e-14


def test_beta_zero_clock():
    """beta = 0, Z3 clock: lnZ/V = ln sum_k e^{h cos th_k}, <cos th> its h-derivative."""
    h = 0.4
    th = 2 * math.pi * np.arange(3) / 3
    z = np.exp(h * np.cos(th))
    st = O.run("clock", 4, 0.0, h, D=6, p=12, nsteps=4)
    _, lz = O.free_energy(st)
    assert abs(lz - math.log(z.sum())) < 1e-14
    assert abs(O.magnetisation(st) - (np.cos(th) * z).sum() / z.sum()) < 1e-14


def test_initial_tensor_is_the_boltzmann_weight():
    """Contracting two Ising W's over the bond gives e^{beta s s'} (Sec. III)."""
    beta = 0.37
    W, s = O.ising_factor(beta)
    assert np.allclose(W @ W.T, np.exp(beta * np.outer(s, s)), rtol=1e-15, atol=0)
    Wc, c = O.clock_factor(3, beta)
    th = 2 * math.pi * np.arange(3) / 3
    assert np.allclose(Wc @ Wc.T, np.exp(beta * np.cos(th[:, None] - th[None, :])), rtol=1e-14)


def test_step1_resplit_is_exact_rank_of_cp_form():
    """Step 1 of ATRG is exact for the CP initial tensor (eq. ABCD footnote): rank 2
    for Ising, 3 for the Z3 clock, and A s D^T reproduces T."""
    for st, rank in ((O.init_ising(4, 0.2, 0.1), 2), (O.init_clock(4, 3, 0.2, 0.1), 3)):
        A, Dm, s = O.resplit(st.phi, st.psi, 12)
        assert np.count_nonzero(s > 1e-12 * s[0]) == rank
        T = st.phi.reshape(-1, rank) @ st.psi.reshape(-1, rank).T
        Am, Dmm = A.reshape(-1, A.shape[-1]), Dm.reshape(-1, Dm.shape[-1])
        assert np.allclose(Am * s @ Dmm.T, T, atol=1e-15 * np.abs(T).max())
        assert np.allclose(Am[:, :rank].T @ Am[:, :rank], np.eye(rank), atol=1e-14)


# --------------------------------------------------------------- brute force
def brute_force(L, beta, h):
    """ln Z / V and <s_0> of the periodic Ising lattice L by enumerating all spins."""
    d = len(L)
    sites = list(itertools.product(*[range(l) for l in L]))
    idx = {x: i for i, x in enumerate(sites)}
    bonds = []
    for x in sites:
        for mu in range(d):
            y = list(x)
            y[mu] = (y[mu] + 1) % L[mu]
            bonds.append((idx[x], idx[tuple(y)]))
    bonds = np.array(bonds)
    confs = np.array(list(itertools.product([1.0, -1.0], repeat=len(sites))))
    E = (confs[:, bonds[:, 0]] * confs[:, bonds[:, 1]]).sum(axis=1)
    w = np.exp(beta * E + h * confs.sum(axis=1))
    return math.log(w.sum()) / len(sites), float((confs[:, 0] * w).sum() / w.sum())


@pytest.mark.parametrize("L,axes", [((2, 1, 1, 1), [0]), ((2, 2, 1, 1), [0, 1]),
                                    ((4, 1, 1, 1), [0, 0]), ((1, 2, 1, 2), [1, 3])])
@pytest.mark.parametrize("beta,h", [(0.3, 0.0), (0.25, 0.2)])
def test_brute_force_untruncated(L, axes, beta, h):
    """Every step untruncated (D = 16 >= every rank of a <= 4-site block): exact."""
    lz_b, m_b = brute_force(L, beta, h)
    st = O.init_ising(4, beta, h)
    for ax in axes:
        O.step(st, ax, D=16, p=256, q_swap=2)
    _, lz = O.free_energy(st)
    assert abs(lz - lz_b) < 1e-13 * abs(lz_b)
    assert abs(O.magnetisation(st) - m_b) < 1e-13


@pytest.mark.parametrize("d,L,axes", [(2, (2, 2), [0, 1]), (2, (4, 1), [0, 0]),
                                      (3, (2, 2, 1), [0, 1]), (3, (2, 1, 2), [2, 0]),
                                      (4, (2, 2, 1, 1), [1, 0])])
@pytest.mark.parametrize("beta,h", [(0.3, 0.0), (0.25, 0.2)])
def test_atrg_brute_force_untruncated(d, L, axes, beta, h):
    """Plain ATRG (eqs. makeG / makeH) in d = 2, 3, 4, every cut untruncated: exact."""
    lz_b, _ = brute_force(L, beta, h)
    st = O.init_ising(d, beta, h)
    for ax in axes:
        O.step(st, ax, D=16, p=256, q_swap=2, method="atrg")
    _, lz = O.free_energy(st)
    assert abs(lz - lz_b) < 1e-13 * abs(lz_b)


def test_2x2x2x2_lattice_against_enumeration():
    """The 2^4 periodic lattice (16 sites, 65536 configurations).  It cannot be contracted
    untruncated by the triad step: after three steps a leg carries the 8 spins of a face,
    rank 2^8, so D = 256 and D^5 ~ 1e12 values.  Truncated, the oracle's lnZ/V error
    falls at least fivefold from D = 8 to 16, to <= 3e-4, and the Z2 invariant m = 0 at h = 0 holds
    exactly under truncation."""
    L = (2, 2, 2, 2)
    for beta, h, bound16 in ((0.02, 0.0, 1e-4), (0.3, 0.1, 3e-4)):
        lz_b, m_b = brute_force(L, beta, h)
        errs = []
        for D in (8, 16):
            st = O.init_ising(4, beta, h)
            for ax in range(4):
                O.step(st, ax, D, 4 * D, 6, 4)
            errs.append(abs(O.free_energy(st)[1] - lz_b) / lz_b)
            if h == 0.0:
                assert abs(O.magnetisation(st)) < 1e-12
        assert errs[1] < bound16 and errs[1] < 0.2 * errs[0], errs


# ------------------------------------------------ triad with full chi == ATRG
@pytest.mark.parametrize("D", [4, 5])
def test_untruncated_triad_equals_atrg(D):
    """chi = D^2 (no triad truncation) recovers plain ATRG (Sec. II B, r = D remark):
    the triad environments (E F I J / G H K L with O, P) must equal the environments of
    the explicit ATRG blocks, over several truncating steps."""
    p = D * D
    a = O.run("ising", 4, 0.16, 0.05, D=D, p=p, nsteps=5, q_swap=6, method="triad")
    b = O.run("ising", 4, 0.16, 0.05, D=D, p=p, nsteps=5, q_swap=6, method="atrg")
    fa, fb = O.free_energy(a)[1], O.free_energy(b)[1]
    assert abs(fa - fb) < 1e-12 * abs(fb)
    for da, db in zip(a.diag, b.diag):
        assert abs(da["log_c"] - db["log_c"]) < 1e-11


# -------------------------------------------------------------- Onsager (d = 2)
def onsager_lnZ(beta, n=1500):
    """-beta f of the 2D Ising model (Onsager), by Gauss-Legendre quadrature."""
    x, w = np.polynomial.legendre.leggauss(n)
    th = (x + 1) * math.pi / 2
    w = w * math.pi / 2
    c = np.cos(th)
    a, b = math.cosh(2 * beta) ** 2, math.sinh(2 * beta)
    I = np.sum(w[:, None] * w[None, :] * np.log(a - b * (c[:, None] + c[None, :])))
    return math.log(2) + 4 * I / (8 * math.pi ** 2)


def test_onsager_quadrature_against_high_t_series():
    b = 0.05
    t = math.tanh(b)
    ser = math.log(2) + 2 * math.log(math.cosh(b)) + t ** 4 + 2 * t ** 6 + 4.5 * t ** 8
    assert abs(onsager_lnZ(b) - ser) < 20 * t ** 10


@pytest.mark.parametrize("beta", [0.3, 0.5])
def test_onsager_2d(beta):
    """d = 2: triad-ATRG is ATRG (Sec. II B); 40 steps, L = 2^20, converge to Onsager."""
    ex = onsager_lnZ(beta)
    errs = []
    for D in (8, 16, 24):
        st = O.run("ising", 2, beta, 0.0, D=D, p=2 * D, nsteps=40, q_swap=4, method="atrg")
        errs.append(abs(O.free_energy(st)[1] - ex) / ex)
    assert errs[-1] < 6e-8
    assert errs[0] > errs[-1]


@pytest.mark.parametrize("beta", [0.1, 0.15])
def test_high_t_series_2d(beta):
    """ln2 + 2 ln cosh b + t^4 + 2 t^6 + 9/2 t^8 + O(t^10) on the square lattice."""
    st = O.run("ising", 2, beta, 0.0, D=16, p=32, nsteps=30, method="atrg")
    t = math.tanh(beta)
    ser = math.log(2) + 2 * math.log(math.cosh(beta)) + t ** 4 + 2 * t ** 6 + 4.5 * t ** 8
    assert abs(O.free_energy(st)[1] - ser) < 20 * t ** 10


def test_high_t_4d_window():
    """4D: lnZ/V - ln 2 - 4 ln cosh b is the plaquette sum 6 t^4 (+ O(t^6)); at D = 8 the
    truncation keeps most of it, so it must sit in [3 t^4, 7 t^4]."""
    b = 0.05
    st = O.run("ising", 4, b, 0.0, D=8, p=16, nsteps=12)
    t = math.tanh(b)
    r = (O.free_energy(st)[1] - math.log(2) - 4 * math.log(math.cosh(b))) / t ** 4
    assert 3.0 < r < 7.0


# -------------------------------------------------------------------- Z2, impurity
def test_z2_magnetisation_zero_when_exact():
    """h = 0 and every randomized step exact (chi >= all dims): <s> = 0 by Z2."""
    st = O.run("ising", 4, 0.16, 0.0, D=4, p=12, nsteps=4, q_swap=6)
    assert abs(O.magnetisation(st)) < 1e-13


def test_z2_antisymmetry_when_exact():
    a = O.run("ising", 4, 0.16, 0.03, D=4, p=12, nsteps=4, q_swap=6)
    b = O.run("ising", 4, 0.16, -0.03, D=4, p=12, nsteps=4, q_swap=6)
    assert abs(O.magnetisation(a) + O.magnetisation(b)) < 1e-12
    assert abs(O.free_energy(a)[1] - O.free_energy(b)[1]) < 1e-13


def test_impurity_is_field_derivative_of_lnZ_brute():
    """On an exactly contracted lattice <s> = d(lnZ/V)/dh (finite difference)."""
    L, axes, beta, h, dh = (2, 2, 1, 1), [0, 1], 0.2, 0.1, 1e-4
    def lz(hh):
        st = O.init_ising(4, beta, hh)
        for ax in axes:
            O.step(st, ax, D=16, p=256, q_swap=2)
        return O.free_energy(st)[1], O.magnetisation(st)
    (lp, _), (lm, _), (_, m) = lz(h + dh), lz(h - dh), lz(h)
    assert abs((lp - lm) / (2 * dh) - m) < 1e-7


# ----------------------------------------------------- decomposition building blocks
def test_squeezer_is_truncated_svd_of_environment_overlap():
    """R1 M N^T R2^T equals the rank-D truncated SVD of R1 R2^T (Eckart-Young); with
    rank <= D it is R1 R2^T itself.  Swapping M and N or a transpose breaks this."""
    rng = np.random.default_rng(1)
    n, D = 36, 6
    for rank in (4, 12):
        R1 = rng.standard_normal((rank, n))
        R2 = rng.standard_normal((rank, n)) @ rng.standard_normal((n, n))
        M, N, _ = O.squeezer(R1.T @ R1, R2.T @ R2, D, n, 4, O.sketch_key(1, 0, 7),
                             O.sketch_key(1, 0, 10))
        U, S, Vt = np.linalg.svd(R1 @ R2.T)
        k = min(D, rank)
        best = (U[:, :k] * S[:k]) @ Vt[:k]
        got = R1 @ M @ N.T @ R2.T
        assert np.allclose(got, best, atol=1e-10 * S[0])


def test_bond_swap_matches_direct_svd_of_BC():
    """With q large and a full sketch the RSVD is the exact truncated SVD of
    M[(alpha I),(beta J)] = sum_x B[x J alpha] C[x I beta] (eq. bond-swapping)."""
    rng = np.random.default_rng(2)
    dx, d, da = 3, 3, 3
    B = rng.standard_normal((dx, d, d, d, da))
    C = rng.standard_normal((dx, d, d, d, da))
    D = 7
    X, sig, Y, _ = O.bond_swap(B, C, D, 200, 12, 3, 0)
    M = np.einsum("xJa,xIb->aIbJ", B.reshape(dx, -1, da), C.reshape(dx, -1, da))
    M = M.reshape(da * d ** 3, da * d ** 3)
    s_ex = np.linalg.svd(M, compute_uv=False)
    assert np.allclose(sig, s_ex[:D], rtol=1e-10)
    Xm = X.reshape(-1, D)
    Ym = Y.reshape(-1, D)
    assert np.allclose(Xm.T @ Xm, np.eye(D), atol=1e-12)
    assert np.allclose(Ym.T @ Ym, np.eye(D), atol=1e-12)
    assert np.allclose(Xm.T @ M @ Ym, np.diag(sig), atol=1e-10 * sig[0])


def test_gu_wen_ratio_closed_form_and_limits():
    """X of the initial Ising tensor at h = 0: A = e^{3 beta} sum_a W_a W_a^T gives
    X = 2 / (1 + e^{-4 beta}); the flow goes to 1 at beta = 0 and to 2 deep in the
    ordered phase (two ground states)."""
    for beta in (0.0, 0.1, 0.3, 1.0):
        st = O.init_ising(4, beta, 0.0)
        assert abs(O.gu_wen_ratio(st) - 2.0 / (1.0 + math.exp(-4.0 * beta))) < 1e-13
    st = O.init_ising(4, 0.0, 0.0)
    for n in range(4):
        O.step(st, n % 4, 4, 8, 4, 4)
        assert abs(O.gu_wen_ratio(st) - 1.0) < 1e-14
    st = O.init_ising(4, 1.0, 0.0)
    for n in range(6):
        O.step(st, n % 4, 4, 8, 4, 4)
    assert abs(O.gu_wen_ratio(st) - 2.0) < 1e-9
