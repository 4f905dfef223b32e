"""CPU checks of two readings the CUDA path relies on, against the oracle's own method.

* Factor form of the triad range finders: range((F F^T)^(q+1) Omega) computed as
  F (F^T F)^q F^T Omega (no rho formed) equals the oracle's range finder on rho = F F^T.
* Bond swap in Gram coordinates: the subspace iteration run on coordinates Y' (Y = C Y')
  and W (V = B W) with G^C = C^T C and G^B = B^T B gives the oracle's QR-compressed
  (Appendix A) singular values and subspaces.
Both are NumPy restatements of the algorithm the library runs, written here only to pin
the equivalence; they are not used by the library.
"""
import numpy as np

from oracle import trg_oracle as O


def _proj(Q):
    return Q @ Q.T


def test_factor_form_range_equals_range_of_rho():
    rng = np.random.default_rng(3)
    n, m, chi, q = 36, 80, 10, 3
    # a factor with a decaying spectrum, as the canonical-form factors have
    U, _ = np.linalg.qr(rng.standard_normal((n, n)))
    V, _ = np.linalg.qr(rng.standard_normal((m, n)))
    F = (U * np.logspace(0, -6, n)) @ V.T
    key = O.sketch_key(0x5EED, 4, 3)
    Q_rho = O.rsvd_range_sym(F @ F.T, chi, q, key)
    Om = O.gaussian(key, n, chi)
    Q = O.orth(F @ (F.T @ Om), chi)
    for _ in range(q):
        Q = O.orth(F @ (F.T @ Q), chi)
    assert np.abs(_proj(Q) - _proj(Q_rho)).max() < 1e-10


def _gram_coordinate_swap(B, C, D, p, q_swap, seed, step):
    """The CUDA path's bond swap (reading 4), restated with NumPy."""
    x, I, k = C.shape[0], int(np.prod(C.shape[1:-1])), C.shape[-1]
    Cm = C.reshape(x, I, k)
    Bm = B.reshape(x, I, k)
    w = min(D + p, k * I)
    Cq = Cm.transpose(0, 2, 1).reshape(x * k, I)           # (x be) x I
    Bq = Bm.transpose(0, 2, 1).reshape(x * k, I)           # (x al) x J
    GC, GB = Cq @ Cq.T, Bq @ Bq.T
    g1 = O.gaussian(O.sketch_key(seed, step, O.TAG_SWAP_G1), k, w)
    g2 = O.gaussian(O.sketch_key(seed, step, O.TAG_SWAP_G2), I, w)
    h = (Bq @ g2).reshape(x, k, w)                         # (x al) m
    Yc = np.einsum("xam,bm->xbam", h, g1).reshape(x * k, k * w)   # (x be), (al m)

    def apply_gp(G, Z):                                    # P (G (x) 1) Z
        Y = (G @ Z).reshape(x, k, k, w)
        return Y.transpose(0, 2, 1, 3).reshape(x * k, k * w)

    def orth_g(G, Z):                                      # orthonormal in metric G (x) 1
        Zr = Z.reshape(x * k * k, w)
        S = Zr.T @ (G @ Z).reshape(x * k * k, w)
        lam, V = np.linalg.eigh((S + S.T) / 2)
        keep = lam > 1e-13 * lam.max()
        T = np.zeros((w, w))
        T[:, keep] = V[:, keep] / np.sqrt(lam[keep])
        return (Zr @ T).reshape(x * k, k * w)

    Qc = orth_g(GC, Yc)
    Yt = apply_gp(GC, Qc)
    for _ in range(q_swap - 1):
        W = orth_g(GB, Yt)
        Qc = orth_g(GC, apply_gp(GB, W))
        Yt = apply_gp(GC, Qc)
    # M^T Q in B-coordinates -> its singular values (= those of Q^T M)
    S = Yt.reshape(-1, w).T @ (GB @ Yt).reshape(-1, w)
    return np.sqrt(np.clip(np.sort(np.linalg.eigvalsh((S + S.T) / 2))[::-1], 0, None))


import pytest


@pytest.mark.parametrize("q", [1, 2, 6])
def test_gram_coordinate_bond_swap_equals_qr_compressed(q):
    """With one or two rounds the randomized SVD is far from converged, so its singular
    values depend on the sketch and on every step of the iteration: equality then pins
    the whole Gram-coordinate loop, not only its fixed point."""
    rng = np.random.default_rng(7)
    x, d, k = 3, 3, 3                        # C: (x, d, d, d, k), I = d^3
    s = np.logspace(0, -2, k)
    C = rng.standard_normal((x, d, d, d, k)) * s
    B = rng.standard_normal((x, d, d, d, k)) * s
    D, p = 4, 2
    _, sig_ref, _, _ = O.bond_swap(B, C, D, p, q, 0x5EED, 5)
    sig = _gram_coordinate_swap(B, C, D, p, q, 0x5EED, 5)
    assert np.allclose(sig[:D], sig_ref[:D], rtol=1e-10, atol=1e-13 * sig_ref[0])
