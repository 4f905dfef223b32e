"""Pin of the oracle's canonical-form triad Grams (Sec. II B, eq. HOSVD).

The isometries U^A, U^X, U^Y, U^D are ranges of the Grams of Gamma^ATRG = A X sigma Y D
on one leg pair each.  The oracle forms them in canonical form (A W A^T, X sigma^2 X^T,
...), which relies on A, X, Y and D being isometries.  Here Gamma is formed explicitly,
leg by leg, from a truncating step of a real run, and its Gram on each pair is taken by
the definition (every other leg of Gamma summed); the oracle's reduced Grams must equal
it.  The untruncated pins cannot catch a mistake in these Grams (with chi >= the pair
dimension the range finder returns the identity and never reads rho), so this test is
their only exact check.
"""
import numpy as np
import pytest

from oracle import trg_oracle as O


def _step_factors(d, D, p, nsteps, beta=0.16, h=0.05, q_swap=4, seed=0x5EED):
    """A, Dm, s, X, sigma, Y of the step that follows `nsteps` steps of a triad run."""
    st = O.run("ising", d, beta, h, D=D, p=p, nsteps=nsteps, q_swap=q_swap, seed=seed)
    axis = nsteps % d
    O._rotate(st, axis)
    A, Dm, s = O.resplit(st.phi, st.psi, D)
    X, sig, Y, _ = O.bond_swap(Dm * s, A * s, D, p, q_swap, seed, st.nsteps)
    return A, Dm, s, X, sig, Y


def _gram_on(gamma, pair):
    """Gram of `gamma` with the legs `pair` open (rows) and every other leg summed."""
    rest = [i for i in range(gamma.ndim) if i not in pair]
    g = np.transpose(gamma, list(pair) + rest)
    n = g.shape[0] * g.shape[1]
    g = g.reshape(n, -1)
    return g @ g.T


def _gamma4(A, X, sig, Y, Dm):
    # A (t p2 p3 p4 al), X (al q2 q3 q4 g), Y (be P2 P3 P4 g), Dm (w Q2 Q3 Q4 be)
    return np.einsum("tabcA,AdefG,G,BghiG,wjklB->tabcdefghiwjkl", A, X, sig, Y, Dm,
                     optimize=True)


def _gamma3(A, X, sig, Y, Dm):
    # A (t p2 p3 al), X (al q2 q3 g), Y (be P2 P3 g), Dm (w Q2 Q3 be)
    return np.einsum("tabA,AcdG,G,BefG,wghB->tabcdefwgh", A, X, sig, Y, Dm, optimize=True)


# open pairs of each factor inside Gamma (positions of its legs i2, i3)
PAIRS4 = {"A": (1, 2), "X": (4, 5), "Y": (7, 8), "D": (11, 12)}
PAIRS3 = {"A": (1, 2), "X": (3, 4), "Y": (5, 6), "D": (8, 9)}


@pytest.mark.parametrize("d,D,p,nsteps", [(4, 3, 3, 4), (4, 3, 2, 5), (3, 4, 4, 3)])
def test_canonical_grams_equal_gram_of_explicit_gamma(d, D, p, nsteps):
    A, Dm, s, X, sig, Y = _step_factors(d, D, p, nsteps)
    # a truncating step: the bond swap keeps D of more singular values
    assert sig.size == D and A.shape[-1] == D
    gamma = (_gamma4 if d == 4 else _gamma3)(A, X, sig, Y, Dm)
    rho = O.triad_grams(A, Dm, X, sig, Y)
    pairs = PAIRS4 if d == 4 else PAIRS3
    for name, pair in pairs.items():
        ref = _gram_on(gamma, pair)
        got = rho[name].reshape(ref.shape)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), name
        # the four Grams differ from one another (a swapped factor would be seen)
    assert not np.allclose(rho["A"], rho["X"], rtol=1e-3)
    assert not np.allclose(rho["A"], rho["D"], rtol=1e-3)


def test_explicit_gram_sees_a_wrong_weight():
    """Self-check of the pin: with W_be in place of W_al in rho^A (a plausible slip), the
    explicit Gram disagrees far beyond the tolerance."""
    A, Dm, s, X, sig, Y = _step_factors(4, 3, 3, 4)
    gamma = _gamma4(A, X, sig, Y, Dm)
    ref = _gram_on(gamma, PAIRS4["A"])
    Ys = Y * sig
    W_be = np.tensordot(Ys, Ys, axes=([1, 2, 3, 4], [1, 2, 3, 4]))
    wrong = np.tensordot(np.tensordot(A, W_be, axes=([4], [0])), A, axes=([0, 3, 4], [0, 3, 4]))
    assert np.abs(wrong.reshape(ref.shape) - ref).max() > 1e-6 * np.abs(ref).max()
    # sigma in place of sigma^2 in rho^X
    Xs1 = X * np.sqrt(sig)
    wrongX = np.tensordot(Xs1, Xs1, axes=([0, 3, 4], [0, 3, 4]))
    refX = _gram_on(gamma, PAIRS4["X"])
    assert np.abs(wrongX.reshape(refX.shape) - refX).max() > 1e-6 * np.abs(refX).max()
