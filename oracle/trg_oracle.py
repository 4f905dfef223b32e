"""Plain FP64 CPU oracle of ATRG and triad-ATRG (arXiv 2507.21909) — TEST INFRASTRUCTURE.

This module is the parity reference for the CUDA path.  It is written for a reader who
checks it against the paper by eye: every tensor is an explicit NumPy array, every
contraction a single ``einsum``/``tensordot`` of the network the paper draws, and every
decomposition a LAPACK call (``qr``, ``svd``, ``eigh``).  It is slow on purpose and
shares no code with the GPU library.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference legs may import it.

Method (one coarse-graining step along axis "1", Sec. II and Appendix A):
  (a) re-split T = A B = C D by an SVD of T                       (Sec. II A, eq. ABCD)
  (b) bond swap  sum_{i1(n)} B C ~ X sigma Y by a QR-compressed randomized SVD
                                                       (eq. bond-swapping, eqs. bond1/bond2)
  (c) triad isometries U^A, U^X, U^Y, U^D from the Grams of the canonical form
      Gamma^ATRG = A X sigma Y D                                   (Sec. II B, eq. HOSVD)
  (d) triads E, F, G, H and I, J, K, L                         (Sec. II B, eqs. E-L)
  (e) squeezers M^(mu), N^(mu) from the environments built with the Gram matrices O, P
                                                       (Sec. II A makeG/makeH text; Sec. II B)
  (f) coarse contraction Phi (eq. makeMG) and Psi (eq. makeMH)     (Sec. II B)
The coarse tensor is kept as T = sum_gamma Phi[i1,k2,k3,k4,gamma] Psi[j1,k2',k3',k4',gamma].

Readings where the paper is silent:
  * r = eta and the overspanned lines have width chi = min(D + p, natural dim)  (Sec. II B
    footnote on r); the triad isometries keep all chi columns of their range finder.
  * Sketches are Gaussian, drawn from a counter-based SplitMix64 / Box-Muller generator
    keyed by (seed, step, tag); the bond-swap sketch is the Khatri-Rao product
    g1[beta,m] * g2[(j2 j3 j4)(n+1), m] (Appendix A gives only "random tensor Omega").
  * Ranks are structural (min of target and dimension); singular values at or below
    RANK_TOL * max are exact zeros and their vectors are set to zero.
  * Sign gauge: each kept column of A (re-split) and of M (squeezer) is flipped so that
    its first entry within 1e-6 of the largest magnitude is positive; the paired factor
    (D, resp. N) flips with it.
  * Squeezers: oblique projector from R1 R2^T (R1, R2 = Gram roots of the forward /
    backward environments), identity when the pair dimension is <= D.
  * Normalisation c_n = ||T||_F; lnZ/V = sum_n ln(c_n)/2^n + 2^-N ln Tr(T_N).
  * Field h and the one-site impurity (magnetisation) with frozen pure projectors.
  * Two-impurity network (Sec. III D, internal energy): the observable sits on both sites
    of the first step's unit cell (neighbours along its axis); that step contracts them
    into one coarse impurity with the pure tensor's projectors, which is then carried
    like the one-site impurity.  U = -d <s s'> uses the equivalence of the axes.
  * Three dimensions (end of Sec. II B gives only the cost, O(r^2 D^6)): the pair (i2, i3)
    of each of A, X, Y, D is compressed by a triad isometry; two squeezers; the coarse
    tensor is (E F)(I J M2 M3).  d = 2 uses plain ATRG, which the paper says coincides.
  * ILO form (r_bond > 1, Sec. II C and Appendix A): the re-split bonds and the swapped
    bond keep r_bond D values; the bond-swap sketch has r_bond D + p columns, so that
    p = D gives the (r_bond + 1) D of the appendix's footnote; the triad isometries,
    squeezers and pair legs are as in the plain form.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

RANK_TOL = 1e-13          # singular values <= RANK_TOL * max are exact zeros
SIGN_TIE = 1e-6           # sign gauge: first entry with |a| >= (1 - SIGN_TIE) max|a|

# ----------------------------------------------------------------------------------
# Counter-based Gaussian sketches: SplitMix64 output function (Steele, Lea, Flood 2014)
# applied to key + counter * golden-gamma, then the Box-Muller transform.
# ----------------------------------------------------------------------------------
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)

# tags of the sketches drawn in one step
TAG_SWAP_G1, TAG_SWAP_G2 = 1, 2
TAG_RHO = {"A": 3, "X": 4, "Y": 5, "D": 6}
TAG_SQ_F = {2: 7, 3: 8, 4: 9}
TAG_SQ_B = {2: 10, 3: 11, 4: 12}


def _mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        return z ^ (z >> np.uint64(31))


def sketch_key(seed: int, step: int, tag: int) -> np.uint64:
    """key = mix64(seed + gamma * (64 * step + tag + 1))   (all arithmetic mod 2^64)."""
    with np.errstate(over="ignore"):
        ctr = np.uint64(64 * step + tag + 1)
        return _mix64(np.uint64(seed) + _GOLDEN * ctr)


def gaussian(key, rows: int, cols: int) -> np.ndarray:
    """Standard normal matrix; entry (r, c) uses counter n = r * cols + c."""
    n = np.arange(rows * cols, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x = _mix64(np.uint64(key) + _GOLDEN * (np.uint64(2) * n + np.uint64(1)))
        y = _mix64(np.uint64(key) + _GOLDEN * (np.uint64(2) * n + np.uint64(2)))
    u1 = ((x >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53   # (0, 1]
    u2 = (y >> np.uint64(11)).astype(np.float64) * 2.0 ** -53           # [0, 1)
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos((2.0 * math.pi) * u2)
    return z.reshape(rows, cols)


# ----------------------------------------------------------------------------------
# Small helpers
# ----------------------------------------------------------------------------------
def _prod(shape) -> int:
    return int(np.prod(shape, dtype=np.int64)) if len(shape) else 1


def orth(Y: np.ndarray, ncols: int | None = None) -> np.ndarray:
    """Orthonormal basis of range(Y) (the "QR decomposition" step of the RSVD loop).

    Returned with ``ncols`` columns (default: Y's); directions whose singular value is
    at or below RANK_TOL * max are exact zeros and their columns are zero.
    """
    if ncols is None:
        ncols = Y.shape[1]
    Q = np.zeros((Y.shape[0], ncols))
    if Y.size == 0:
        return Q
    U, s, _ = np.linalg.svd(Y, full_matrices=False)
    if s.size == 0 or s[0] == 0.0:
        return Q
    k = int(np.count_nonzero(s > RANK_TOL * s[0]))
    k = min(k, ncols)
    Q[:, :k] = U[:, :k]
    return Q


def sign_gauge(cols: np.ndarray) -> np.ndarray:
    """+-1 per column: sign of the first entry within SIGN_TIE of the largest magnitude."""
    a = np.abs(cols)
    mx = a.max(axis=0) if cols.shape[0] else np.zeros(cols.shape[1])
    out = np.ones(cols.shape[1])
    for j in range(cols.shape[1]):
        if mx[j] == 0.0:
            continue
        i = int(np.argmax(a[:, j] >= (1.0 - SIGN_TIE) * mx[j]))
        out[j] = 1.0 if cols[i, j] > 0 else -1.0
    return out


def _alive(s: np.ndarray) -> np.ndarray:
    if s.size == 0 or s.max() <= 0.0:
        return np.zeros(s.shape, dtype=bool)
    return s > RANK_TOL * s.max()


# ----------------------------------------------------------------------------------
# Initial tensors (Sec. III: CP form T = sum_a prod_legs W[a, leg])
# ----------------------------------------------------------------------------------
def ising_factor(beta: float):
    """W of Sec. III (rows: spin state a with s_a = +1, -1; columns: bond index)."""
    if beta < 0:
        raise ValueError("beta must be >= 0")
    c, s = math.sqrt(math.cosh(beta)), math.sqrt(math.sinh(beta))
    W = np.array([[c, s], [c, -s]])
    spins = np.array([1.0, -1.0])
    return W, spins


def clock_factor(q: int, beta: float):
    """Z_q clock model: w(theta, theta') = exp(beta cos(theta - theta')) = W W^T.

    The circulant bond matrix is diagonal in the real Fourier basis; W = F sqrt(lambda).
    Returns W (rows: state k, columns: bond index) and cos(theta_k).
    """
    if beta < 0:
        raise ValueError("beta must be >= 0")
    th = 2.0 * math.pi * np.arange(q) / q
    B = np.exp(beta * np.cos(th[:, None] - th[None, :]))
    cols = [np.ones(q) / math.sqrt(q)]
    for m in range(1, (q - 1) // 2 + 1):
        cols.append(np.cos(m * th) * math.sqrt(2.0 / q))
        cols.append(np.sin(m * th) * math.sqrt(2.0 / q))
    if q % 2 == 0:
        cols.append(np.cos(math.pi * np.arange(q)) / math.sqrt(q))
    F = np.stack(cols, axis=1)
    lam = np.einsum("ki,kl,lj->ij", F, B, F, optimize=True).diagonal().copy()
    if np.any(lam < -1e-12 * np.abs(lam).max()):
        raise ValueError("clock bond matrix not positive semidefinite")
    W = F * np.sqrt(np.clip(lam, 0.0, None))[None, :]
    return W, np.cos(th)


@dataclass
class State:
    """Coarse tensor T = Phi Psi^T (+ impurity T_imp = Phi Psi_imp^T) and bookkeeping."""
    d: int
    beta: float
    phi: np.ndarray                 # legs (slot 0..d-1, gamma)
    psi: np.ndarray
    psi_imp: np.ndarray | None
    axes: tuple                     # physical axis of each leg slot (a cyclic rotation)
    nsteps: int = 0
    logsum: float = 0.0             # sum_n ln(c_n) / 2^n
    diag: list = field(default_factory=list)
    imp_pair: bool = False          # the impurity is a nearest-neighbour pair, merged by
                                    # the next step (two-impurity network, Sec. III D)


def _init_from_factor(d: int, beta: float, W: np.ndarray, weight: np.ndarray,
                      observable: np.ndarray) -> State:
    """Phi0[i1..id, a] = prod_mu W[a, i_mu];  Psi0[j1..jd, a] = w_a prod_mu W[a, j_mu]."""
    nstate, nb = W.shape
    phi = np.ones((nstate,) + (nb,) * d)
    for mu in range(d):
        shape = [nstate] + [1] * d
        shape[1 + mu] = nb
        phi = phi * W.reshape(shape)
    phi = np.moveaxis(phi, 0, -1).copy()                 # (i1..id, a)
    psi = phi * weight                                    # weight broadcast over the last leg
    psi_imp = phi * (weight * observable)
    st = State(d=d, beta=beta, phi=phi, psi=psi, psi_imp=psi_imp, axes=tuple(range(d)))
    c0 = frob_norm(st.phi, st.psi)
    st.psi = st.psi / c0
    st.psi_imp = st.psi_imp / c0
    st.logsum = math.log(c0)
    return st


def init_ising(d: int, beta: float, h: float = 0.0, impurity: str = "site") -> State:
    """d-dim Ising: T = sum_a e^{h s_a} prod W[a, .]  (Sec. III, field h added).
    impurity "site": one spin s (magnetisation); "pair": s on both sites of the first
    step's unit cell, i.e. the nearest-neighbour product s_x s_(x+e) along the first
    step's axis (the two-impurity network of Sec. III D)."""
    W, spins = ising_factor(beta)
    st = _init_from_factor(d, beta, W, np.exp(h * spins), spins)
    return _set_impurity(st, impurity)


def init_clock(d: int, q: int, beta: float, h: float = 0.0, impurity: str = "site") -> State:
    """Z_q clock model, site weight e^{h cos theta}, observable cos theta (impurity as in
    init_ising)."""
    W, cth = clock_factor(q, beta)
    st = _init_from_factor(d, beta, W, np.exp(h * cth), cth)
    return _set_impurity(st, impurity)


def _set_impurity(st: State, impurity: str) -> State:
    if impurity not in ("site", "pair"):
        raise ValueError("impurity is 'site' or 'pair'")
    st.imp_pair = impurity == "pair"
    return st


def frob_norm(phi: np.ndarray, psi: np.ndarray) -> float:
    """||Phi Psi^T||_F = sqrt(Tr((Phi^T Phi)(Psi^T Psi)))."""
    r = phi.shape[-1]
    P = phi.reshape(-1, r)
    S = psi.reshape(-1, r)
    return math.sqrt(max(float(np.trace((P.T @ P) @ (S.T @ S))), 0.0))


def trace_T(phi: np.ndarray, psi: np.ndarray) -> float:
    """Tr T = sum over legs and gamma of Phi * Psi (forward leg mu paired with backward mu)."""
    return float(np.sum(phi * psi))


# ----------------------------------------------------------------------------------
# (a) re-split: truncated SVD of T = Phi Psi^T  (eq. ABCD and its footnote)
# ----------------------------------------------------------------------------------
def resplit(phi: np.ndarray, psi: np.ndarray, D: int):
    """T ~ A s D^T with A, D isometric; returns A, Dm, s (dead columns zeroed)."""
    r = phi.shape[-1]
    P = phi.reshape(-1, r)
    S = psi.reshape(-1, r)
    Qp, Rp = np.linalg.qr(P)
    Qs, Rs = np.linalg.qr(S)
    u, s, vt = np.linalg.svd(Rp @ Rs.T)
    k = min(D, s.size)
    A = Qp @ u[:, :k]
    Dm = Qs @ vt.T[:, :k]
    s = s[:k].copy()
    sg = sign_gauge(A)
    A *= sg
    Dm *= sg
    alive = _alive(s)
    A[:, ~alive] = 0.0
    Dm[:, ~alive] = 0.0
    s[~alive] = 0.0
    return A.reshape(phi.shape[:-1] + (k,)), Dm.reshape(psi.shape[:-1] + (k,)), s


# ----------------------------------------------------------------------------------
# (b) bond swap: sum_{i1(n)} B C ~ X sigma Y  (eq. bond-swapping; Appendix A)
# ----------------------------------------------------------------------------------
def bond_swap(B: np.ndarray, C: np.ndarray, D: int, p: int, q_swap: int, seed: int,
              step: int):
    """B legs (i1(n), j2..jd(n+1), alpha);  C legs (i1(n), i2..id(n), beta).

    QR of B over (j2..jd) and of C over (i2..id) (Appendix A), the randomized-SVD loop of
    eqs. bond1/bond2 on M'[(alpha q),(beta p)] = sum_i1 R^C[q,(i1 beta)] R^B[p,(i1 alpha)],
    then the SVD of the projection Q^T M'.  X = U^bond Q^C and Y = V^bond Q^B (eqs. XY).
    """
    dx, dal = B.shape[0], B.shape[-1]
    Pshape, qshape = B.shape[1:-1], C.shape[1:-1]
    dP, dq, dbe = _prod(Pshape), _prod(qshape), C.shape[-1]
    Bm = B.reshape(dx, dP, dal).transpose(1, 0, 2).reshape(dP, dx * dal)
    Cm = C.reshape(dx, dq, dbe).transpose(1, 0, 2).reshape(dq, dx * dbe)
    QB, RB = np.linalg.qr(Bm)
    QC, RC = np.linalg.qr(Cm)
    pB, pC = RB.shape[0], RC.shape[0]
    # M'[(alpha, qc), (beta, pb)]
    Mp = np.einsum("cxb,pxa->acbp", RC.reshape(pC, dx, dbe), RB.reshape(pB, dx, dal))
    Mp = Mp.reshape(dal * pC, dbe * pB)
    w = min(D + p, dal * dq, dbe * dP)
    g1 = gaussian(sketch_key(seed, step, TAG_SWAP_G1), dbe, w)
    g2 = gaussian(sketch_key(seed, step, TAG_SWAP_G2), dP, w)
    Om = (g1[:, None, :] * (QB.T @ g2)[None, :, :]).reshape(dbe * pB, w)
    Q = None
    for _ in range(max(q_swap, 1)):
        Q = orth(Mp @ Om, w)
        Om = orth(Mp.T @ Q, w)
    core = Q.T @ Mp                                   # Q^dagger M'
    Ut, sig, Vt = np.linalg.svd(core, full_matrices=False)
    Dg = min(D, w)
    spec = sig.copy()
    sig = np.concatenate([sig, np.zeros(max(0, Dg - sig.size))])[:Dg]
    Ut = np.pad(Ut, ((0, 0), (0, max(0, Dg - Ut.shape[1]))))[:, :Dg]
    V = np.pad(Vt.T, ((0, 0), (0, max(0, Dg - Vt.shape[0]))))[:, :Dg]
    alive = _alive(sig)
    sig[~alive] = 0.0
    Ubond = (Q @ Ut) * alive                          # [(alpha qc), gamma]
    Vbond = V * alive                                 # [(beta pb), gamma]
    X = np.einsum("aqg,Iq->aIg", Ubond.reshape(dal, pC, Dg), QC)
    Y = np.einsum("bpg,Jp->bJg", Vbond.reshape(dbe, pB, Dg), QB)
    return (X.reshape((dal,) + qshape + (Dg,)), sig, Y.reshape((dbe,) + Pshape + (Dg,)),
            _rel_gap(spec, Dg))


def _rel_gap(spec: np.ndarray, k: int) -> float:
    if spec.size <= k or spec[k - 1] <= 0:
        return float("inf")
    return float((spec[k - 1] - spec[k]) / spec[k - 1])


# ----------------------------------------------------------------------------------
# Randomized range finder of a symmetric PSD matrix (triad isometries, squeezers)
# ----------------------------------------------------------------------------------
def rsvd_range_sym(rho: np.ndarray, chi: int, q_rho: int, key) -> np.ndarray:
    """Orthonormal basis (n x chi) of range(rho^(q_rho+1) Omega); identity if chi >= n."""
    n = rho.shape[0]
    if chi >= n:
        return np.eye(n)
    Q = orth(rho @ gaussian(key, n, chi), chi)
    for _ in range(q_rho):
        Q = orth(rho @ Q, chi)
    return Q


def gram_root(rho: np.ndarray, chi: int, q_rho: int, key) -> np.ndarray:
    """R (chi' x n) with R^T R = Q Q^T rho Q Q^T, Q the rank-chi range of rho."""
    Q = rsvd_range_sym(rho, chi, q_rho, key)
    lam, V = np.linalg.eigh(Q.T @ rho @ Q)
    lam = np.clip(lam, 0.0, None)
    return (np.sqrt(lam)[:, None] * V.T) @ Q.T


def squeezer(rho_f: np.ndarray, rho_b: np.ndarray, D: int, chi: int, q_rho: int,
             key_f, key_b):
    """Oblique projector M N^T on one pair bond (reading of Sec. II A / Sec. II B).

    rho_f: Gram of the block whose forward pair is open; rho_b: of the backward pair.
    R1^T R1 ~ rho_f, R2^T R2 ~ rho_b,  R1 R2^T = U S V^T (keep D),
    M = R2^T V_D S_D^{-1/2},  N = R1^T U_D S_D^{-1/2}  so that R1 M N^T R2^T = U_D S_D V_D^T.
    The pair index is (upper-site leg, lower-site leg) on both M and N.
    """
    n = rho_f.shape[0]
    if n <= D:
        I = np.eye(n)
        return I, I.copy(), float("inf")
    R1 = gram_root(rho_f, chi, q_rho, key_f)
    R2 = gram_root(rho_b, chi, q_rho, key_b)
    U, S, Vt = np.linalg.svd(R1 @ R2.T)
    k = min(D, S.size)
    alive = _alive(S[:k])
    inv = np.zeros(k)
    inv[alive] = 1.0 / np.sqrt(S[:k][alive])
    M = (R2.T @ Vt.T[:, :k]) * inv
    N = (R1.T @ U[:, :k]) * inv
    sg = sign_gauge(M)
    return M * sg, N * sg, _rel_gap(S, k)


# ----------------------------------------------------------------------------------
# (c)-(f): the triad step in four dimensions
# ----------------------------------------------------------------------------------
def triad_grams(A, Dm, X, sig, Y) -> dict:
    """The four Grams of eq. HOSVD (Sec. II B) on the leg pair (i2, i3) of each factor of
    Gamma^ATRG = A X sigma Y D, reduced with the canonical form (d = 3 or 4).

    Legs: A (t, p2, p3, [p4,] al), X (al, q2, q3, [q4,] g), Y (be, P2, P3, [P4,] g),
    Dm (w, Q2, Q3, [Q4,] be).  A is isometric from (t, p..) to al, X from (al, q..) to g,
    Y from (be, P..) to g and Dm from (w, Q..) to be (columns orthonormal or zero, zero
    columns only where sigma or s vanishes), so tracing Gamma Gamma^T over every leg but
    one pair leaves
        rho^A = A W_al A^T,  W_al[a, a'] = sum_{q, g} X[a q g] sigma_g^2 X[a' q g],
        rho^X = sum_{al, q_rest, g} X sigma^2 X^T,   rho^Y likewise with Y,
        rho^D = Dm W_be Dm^T,  W_be from Y as W_al from X,
    with the open pair as rows and every other leg of the factor summed.  Returned with
    shape (d2, d3, d2, d3) each, keys "A", "X", "Y", "D"."""
    Xs = X * sig
    Ys = Y * sig
    inner = list(range(1, X.ndim))                 # (q.., g) of X, (P.., g) of Y
    W_al = np.tensordot(Xs, Xs, axes=(inner, inner))
    W_be = np.tensordot(Ys, Ys, axes=(inner, inner))
    rest = [0] + list(range(3, A.ndim))            # every leg but the pair (1, 2)
    last = A.ndim - 1
    AW = np.tensordot(A, W_al, axes=([last], [0]))  # bond leg still last
    DW = np.tensordot(Dm, W_be, axes=([last], [0]))
    return {"A": np.tensordot(AW, A, axes=(rest, rest)),
            "X": np.tensordot(Xs, Xs, axes=(rest, rest)),
            "Y": np.tensordot(Ys, Ys, axes=(rest, rest)),
            "D": np.tensordot(DW, Dm, axes=(rest, rest))}


def _triad_step(A, Dm, s, D, p, q_swap, q_rho, seed, step, psi_imp_pair=None, mlp=None,
                Db=None, imp_two=False):
    """One triad-ATRG step on the re-split factors.  Legs (per site):
    A (t=i1(n+1), p2,p3,p4, al)   C = A s  (x=i1(n), q2,q3,q4, be)
    B = Dm s (x=j1(n+1)=i1(n), P2,P3,P4, al)   Dm (w=j1(n), Q2,Q3,Q4, be)
    Db: width kept on the bond-swap line gamma (r_bond D for the ILO form, Sec. II C and
    Appendix A; D by default).  The pair legs are still cut to D by the squeezers.
    """
    C = A * s
    B = Dm * s
    X, sig, Y, gap_swap = bond_swap(B, C, D if Db is None else Db, p, q_swap, seed, step)
    d2, d3, d4 = A.shape[1:4]
    chi_pair = d2 * d3

    # (c) triad isometries from the canonical form (eq. HOSVD)
    rho_all = triad_grams(A, Dm, X, sig, Y)
    chi = min(D + p, chi_pair)
    U = {}
    sketch_info = {}
    for name, rho in rho_all.items():
        key = sketch_key(seed, step, TAG_RHO[name])
        if mlp is None:
            Q = rsvd_range_sym(rho.reshape(chi_pair, chi_pair), chi, q_rho, key)
        else:  # learned sketch with the plain range as fallback (oracle/sketch_mlp.py)
            from . import sketch_mlp as SM
            Q, sketch_info[name] = SM.rsvd_learned(
                mlp, rho.reshape(chi_pair, chi_pair), d2, d3, chi, q_rho, key,
                sketch_key(seed, step, SM.TAG_PROBE[name]))
        U[name] = Q.reshape(d2, d3, -1)

    # (d) triads, eqs. E-L
    E = np.einsum("tbcda,bck->tkda", A, U["A"])
    F = np.einsum("abcdg,bck,g->akdg", X, U["X"], sig, optimize=True)
    G = np.einsum("bPQRg,PQk->bkRg", Y, U["Y"])
    H = np.einsum("wPQRb,PQk->wkRb", Dm, U["D"])
    I_, J_, K_, L_ = U["A"], U["X"], U["Y"], U["D"]

    # (e) Gram matrices O (upper block E F I J) and P (lower block G H K L)
    Ig = np.einsum("bck,bcl->kl", I_, I_)
    Jg = np.einsum("bck,bcl->kl", J_, J_)
    Kg = np.einsum("bck,bcl->kl", K_, K_)
    Lg = np.einsum("bck,bcl->kl", L_, L_)
    EEI = np.einsum("tkda,tlde,kl->ae", E, E, Ig, optimize=True)
    O = np.einsum("ae,akdg,eldh,kl->gh", EEI, F, F, Jg, optimize=True)
    HHL = np.einsum("wkdb,wlde,kl->be", H, H, Lg, optimize=True)
    Pm = np.einsum("be,bkdg,eldh,kl->gh", HHL, G, G, Kg, optimize=True)

    # environments of each pair (forward: upper block with P on gamma; backward: lower
    # block with O on gamma), then the squeezers
    EE4 = np.einsum("tkda,tlDe,kl->daDe", E, E, Ig, optimize=True)                 # (p4 al, p4' al')
    FPF4 = np.einsum("akdg,gh,elDh,kl->adeD", F, Pm, F, Jg, optimize=True)         # (al q4, al' q4')
    rho_f = {4: np.einsum("paPe,aqeQ->pqPQ", EE4, FPF4)}           # (p4 q4, p4' q4')
    GOG4 = np.einsum("bkPg,gh,elQh,kl->bPeQ", G, O, G, Kg, optimize=True)           # (be P4, be' P4')
    HH4 = np.einsum("wkdb,wlDe,kl->bdeD", H, H, Lg, optimize=True)                  # (be Q4, be' Q4')
    rho_b = {4: np.einsum("bPeR,bQeS->PQRS", GOG4, HH4)}

    EE2 = np.einsum("tkda,tlde->kale", E, E)                         # (kA al, kA' al')
    FPF2 = np.einsum("akdg,gh,eldh->akel", F, Pm, F, optimize=True)                 # (al kX, al' kX')
    GOG2 = np.einsum("bkdg,gh,eldh->kble", G, O, G, optimize=True)                  # (kY be, kY' be')
    HH2 = np.einsum("wkdb,wlde->kble", H, H)                         # (kD be, kD' be')
    for mu, sub in ((2, "bck,Bcl->bkBl"), (3, "cbk,cBl->bkBl")):
        II = np.einsum(sub, I_, I_)                                   # (p kA, p' kA')
        JJ = np.einsum(sub, J_, J_)                                   # (q kX, q' kX')
        KK = np.einsum(sub, K_, K_)
        LL = np.einsum(sub, L_, L_)
        G1 = np.einsum("pkPl,kale->paPe", II, EE2)                    # (p al, p' al')
        G2 = np.einsum("qkQl,akel->aqeQ", JJ, FPF2)                   # (al q, al' q')
        rho_f[mu] = np.einsum("paPe,aqeQ->pqPQ", G1, G2)
        G1b = np.einsum("PkRl,kble->PbRe", KK, GOG2)                  # (P be, P' be')
        G2b = np.einsum("QkSl,kble->bQeS", LL, HH2)                   # (be Q, be' Q')
        rho_b[mu] = np.einsum("PbRe,bQeS->PQRS", G1b, G2b)

    dims = {2: d2, 3: d3, 4: d4}
    Msq, Nsq, gaps = {}, {}, {}
    for mu in (2, 3, 4):
        n = dims[mu] ** 2
        chi_s = min(D + p, n)
        M, N, gaps[mu] = squeezer(rho_f[mu].reshape(n, n), rho_b[mu].reshape(n, n), D, chi_s,
                                  q_rho, sketch_key(seed, step, TAG_SQ_F[mu]),
                                  sketch_key(seed, step, TAG_SQ_B[mu]))
        Msq[mu] = M.reshape(dims[mu], dims[mu], -1)
        Nsq[mu] = N.reshape(dims[mu], dims[mu], -1)

    # (f) coarse contraction, eqs. makeMG / makeMH
    phi = contract_upper(E, F, I_, J_, Msq)
    psi = contract_lower(G, H, K_, L_, Nsq)

    psi_imp = None
    if psi_imp_pair is not None:
        phi_old, psi_imp_old = psi_imp_pair
        # impurity at slot n+1: exact backward factor B_imp = T_imp^T A, frozen X projector
        r = phi_old.shape[-1]
        PA = phi_old.reshape(-1, r).T @ A.reshape(-1, A.shape[-1])
        B_imp = (psi_imp_old.reshape(-1, r) @ PA).reshape(B.shape)
        CX = np.tensordot(C, X, axes=([1, 2, 3], [1, 2, 3]))          # (x be al g)
        Ytil = np.einsum("xPQRa,xbag->bPQRg", B_imp, CX)              # M_imp^T X
        sinv = np.zeros_like(sig)
        sinv[sig > 0] = 1.0 / sig[sig > 0]
        G_imp = np.einsum("bPQRg,PQk->bkRg", Ytil * sinv, U["Y"])
        # impurity at slot n: backward factor D_imp = T_imp^T A s^+, frozen U^D
        sp = np.zeros_like(s)
        sp[s > 0] = 1.0 / s[s > 0]
        D_imp = B_imp * sp
        H_imp = np.einsum("wPQRb,PQk->wkRb", D_imp, U["D"])
        if imp_two:
            # both sites of the unit cell carry the impurity: one coarse impurity tensor
            psi_imp = contract_lower(G_imp, H_imp, K_, L_, Nsq)
        else:
            # one impurity, at slot n+1 or at slot n with equal weight
            psi_imp = 0.5 * (contract_lower(G_imp, H, K_, L_, Nsq) +
                             contract_lower(G, H_imp, K_, L_, Nsq))
    diag = {"gap_swap": gap_swap, "gap_sq": gaps, "sigma": sig, "s": s}
    if sketch_info:
        diag["sketch"] = sketch_info
    return phi, psi, psi_imp, diag


def _triad3_step(A, Dm, s, D, p, q_swap, q_rho, seed, step, Db=None, psi_imp_pair=None,
                 imp_two=False):
    """The triad step in three dimensions (the d = 3 case the paper discusses at the end
    of Sec. II B, cost O(r^2 D^6)).  Legs (per site):
    A (t, p2, p3, al), C = A s (x, q2, q3, be), B = Dm s (x, P2, P3, al), Dm (w, Q2, Q3, be).
    The pair (i2, i3) of each of A, X, Y, D is compressed by a triad isometry of width
    chi = D + p (ranges of the canonical-form Grams, as in d = 4); the triads are
    E (t, kA, al), F (al, kX, g), G (be, kY, g), H (w, kD, be); two squeezers (mu = 2, 3)
    come from the environments of the upper block E F I J and the lower block G H K L;
    Phi = (E F)(I J M2 M3), Psi = (H G)(K L N2 N3)."""
    C = A * s
    B = Dm * s
    X, sig, Y, gap_swap = bond_swap(B, C, D if Db is None else Db, p, q_swap, seed, step)
    d2, d3 = A.shape[1:3]
    chi_pair = d2 * d3
    rho = triad_grams(A, Dm, X, sig, Y)
    chi = min(D + p, chi_pair)
    U = {name: rsvd_range_sym(r_.reshape(chi_pair, chi_pair), chi, q_rho,
                              sketch_key(seed, step, TAG_RHO[name])).reshape(d2, d3, -1)
         for name, r_ in rho.items()}
    E = np.einsum("tbca,bck->tka", A, U["A"])
    F = np.einsum("abcg,bck,g->akg", X, U["X"], sig, optimize=True)
    G = np.einsum("bPQg,PQk->bkg", Y, U["Y"])
    H = np.einsum("wPQb,PQk->wkb", Dm, U["D"])
    I_, J_, K_, L_ = U["A"], U["X"], U["Y"], U["D"]
    Ig, Jg = np.einsum("bck,bcl->kl", I_, I_), np.einsum("bck,bcl->kl", J_, J_)
    Kg, Lg = np.einsum("bck,bcl->kl", K_, K_), np.einsum("bck,bcl->kl", L_, L_)
    # Grams of the two blocks on the bond gamma
    EEI = np.einsum("tka,tle,kl->ae", E, E, Ig, optimize=True)
    O = np.einsum("ae,akg,elh,kl->gh", EEI, F, F, Jg, optimize=True)
    HHL = np.einsum("wkb,wle,kl->be", H, H, Lg, optimize=True)
    Pm = np.einsum("be,bkg,elh,kl->gh", HHL, G, G, Kg, optimize=True)
    # pair environments: forward = upper block with P on gamma, backward = lower with O
    EE2 = np.einsum("tka,tle->kale", E, E)
    FPF2 = np.einsum("akg,gh,elh->akel", F, Pm, F, optimize=True)
    GOG2 = np.einsum("bkg,gh,elh->kble", G, O, G, optimize=True)
    HH2 = np.einsum("wkb,wle->kble", H, H)
    Msq, Nsq, gaps = {}, {}, {}
    dims = {2: d2, 3: d3}
    for mu, sub in ((2, "bck,Bcl->bkBl"), (3, "cbk,cBl->bkBl")):
        II, JJ = np.einsum(sub, I_, I_), np.einsum(sub, J_, J_)
        KK, LL = np.einsum(sub, K_, K_), np.einsum(sub, L_, L_)
        rf = np.einsum("paPe,aqeQ->pqPQ", np.einsum("pkPl,kale->paPe", II, EE2),
                       np.einsum("qkQl,akel->aqeQ", JJ, FPF2))
        rb = np.einsum("PbRe,bQeS->PQRS", np.einsum("PkRl,kble->PbRe", KK, GOG2),
                       np.einsum("QkSl,kble->bQeS", LL, HH2))
        n = dims[mu] ** 2
        M, N, gaps[mu] = squeezer(rf.reshape(n, n), rb.reshape(n, n), D, min(D + p, n), q_rho,
                                  sketch_key(seed, step, TAG_SQ_F[mu]),
                                  sketch_key(seed, step, TAG_SQ_B[mu]))
        Msq[mu] = M.reshape(dims[mu], dims[mu], -1)
        Nsq[mu] = N.reshape(dims[mu], dims[mu], -1)
    ThU = np.einsum("bck,BCl,bBm,cCn->klmn", I_, J_, Msq[2], Msq[3], optimize=True)
    ThL = np.einsum("bck,BCl,bBm,cCn->klmn", K_, L_, Nsq[2], Nsq[3], optimize=True)
    phi = np.einsum("tka,alg,klmn->tmng", E, F, ThU, optimize=True)

    def lower(G_, H_):
        return np.ascontiguousarray(np.einsum("wlb,bkg,klmn->wmng", H_, G_, ThL, optimize=True))

    psi = lower(G, H)
    psi_imp = None
    if psi_imp_pair is not None:
        # impurity with the pure tensor's frozen projectors, as in the 4D step
        phi_old, psi_imp_old = psi_imp_pair
        r = phi_old.shape[-1]
        PA = phi_old.reshape(-1, r).T @ A.reshape(-1, A.shape[-1])
        B_imp = (psi_imp_old.reshape(-1, r) @ PA).reshape(B.shape)
        CX = np.tensordot(C, X, axes=([1, 2], [1, 2]))                 # (x be al g)
        Ytil = np.einsum("xPQa,xbag->bPQg", B_imp, CX)
        sinv = np.zeros_like(sig)
        sinv[sig > 0] = 1.0 / sig[sig > 0]
        G_imp = np.einsum("bPQg,PQk->bkg", Ytil * sinv, U["Y"])
        sp = np.zeros_like(s)
        sp[s > 0] = 1.0 / s[s > 0]
        H_imp = np.einsum("wPQb,PQk->wkb", B_imp * sp, U["D"])
        psi_imp = (lower(G_imp, H_imp) if imp_two
                   else 0.5 * (lower(G_imp, H) + lower(G, H_imp)))
    return (np.ascontiguousarray(phi), psi, psi_imp,
            {"gap_swap": gap_swap, "gap_sq": gaps, "sigma": sig, "s": s})


def contract_upper(E, F, I_, J_, Msq):
    """Phi[t,k2,k3,k4,g] = sum (E F M4)(I J M2 M3)   (eq. makeMG)."""
    Theta = np.einsum("bck,BCl,bBm,cCn->klmn", I_, J_, Msq[2], Msq[3], optimize=True)  # (kA kX k2 k3)
    EM = np.einsum("tkda,dDm->tkamD", E, Msq[4])                        # (t kA al k4 q4)
    Phi1 = np.tensordot(EM, F, axes=([2, 4], [0, 2]))                   # (t kA k4 kX g)
    Phi = np.tensordot(Phi1, Theta, axes=([1, 3], [0, 1]))              # (t k4 g k2 k3)
    return np.ascontiguousarray(Phi.transpose(0, 3, 4, 1, 2))


def contract_lower(G, H, K_, L_, Nsq):
    """Psi[w,k2',k3',k4',g] = sum (G H N4)(K L N2 N3)   (eq. makeMH), pairs (P, Q)."""
    Theta = np.einsum("bck,BCl,bBm,cCn->klmn", K_, L_, Nsq[2], Nsq[3], optimize=True)  # (kY kD k2 k3)
    HN = np.einsum("wkdb,Ddm->wkbmD", H, Nsq[4])                        # (w kD be k4 P4)
    Psi1 = np.tensordot(HN, G, axes=([2, 4], [0, 2]))                   # (w kD k4 kY g)
    Psi = np.tensordot(Psi1, Theta, axes=([3, 1], [0, 1]))              # (w k4 g k2 k3)
    return np.ascontiguousarray(Psi.transpose(0, 3, 4, 1, 2))


# ----------------------------------------------------------------------------------
# Plain ATRG coarse graining in d dimensions (eqs. makeG / makeH), same squeezer rule
# ----------------------------------------------------------------------------------
def _atrg_step(A, Dm, s, D, p, q_swap, q_rho, seed, step, Db=None):
    d = A.ndim - 1
    C = A * s
    B = Dm * s
    X, sig, Y, gap_swap = bond_swap(B, C, D if Db is None else Db, p, q_swap, seed, step)
    # Up[t, p2..pd, q2..qd, g] = sum_al A[t p al] X[al q g] sigma_g ;  Lo[w, P.., Q.., g]
    Up = np.tensordot(A, X * sig, axes=([d], [0]))
    Lo = np.moveaxis(np.tensordot(Y, Dm, axes=([0], [d])), d - 1, -1)   # (P.., w, Q.., g)
    Lo = np.moveaxis(Lo, d - 1, 0)                                      # (w, P.., Q.., g)
    nl = 2 * d - 1
    O = np.tensordot(Up, Up, axes=(list(range(nl)), list(range(nl))))
    Pm = np.tensordot(Lo, Lo, axes=(list(range(nl)), list(range(nl))))
    UpP = np.tensordot(Up, Pm, axes=([nl], [0]))
    LoO = np.tensordot(Lo, O, axes=([nl], [0]))
    Msq, Nsq, gaps = {}, {}, {}
    for mu in range(2, d + 1):
        pa, qa = mu - 1, mu - 1 + (d - 1)           # positions of p_mu, q_mu in Up/Lo
        other = [i for i in range(nl + 1) if i not in (pa, qa)]
        rf = np.tensordot(UpP, Up, axes=(other, other))   # (p, q, p', q')
        rb = np.tensordot(LoO, Lo, axes=(other, other))
        dm = A.shape[mu - 1]
        n = dm * dm
        chi_s = min(D + p, n)
        M, N, gaps[mu] = squeezer(rf.reshape(n, n), rb.reshape(n, n), D, chi_s, q_rho,
                                  sketch_key(seed, step, TAG_SQ_F.get(mu, 6 + mu)),
                                  sketch_key(seed, step, TAG_SQ_B.get(mu, 9 + mu)))
        Msq[mu] = M.reshape(dm, dm, -1)
        Nsq[mu] = N.reshape(dm, dm, -1)
    phi, psi = Up, Lo
    for mu in range(2, d + 1):
        # pair (p_mu, q_mu) sits at positions 1 and d - (mu - 2): earlier pairs are gone
        phi = np.tensordot(phi, Msq[mu], axes=([1, d - (mu - 2)], [0, 1]))
        psi = np.tensordot(psi, Nsq[mu], axes=([1, d - (mu - 2)], [0, 1]))
    # now (t, g, k2..kd)
    phi = np.ascontiguousarray(np.moveaxis(phi, 1, -1))
    psi = np.ascontiguousarray(np.moveaxis(psi, 1, -1))
    return phi, psi, None, {"gap_swap": gap_swap, "gap_sq": gaps, "sigma": sig, "s": s}


# ----------------------------------------------------------------------------------
# Driver: one step, free energy, magnetisation
# ----------------------------------------------------------------------------------
def _rotate(st: State, axis: int):
    """Bring the leg slot of physical `axis` to the front, keeping the cyclic order."""
    if axis not in st.axes:
        raise ValueError("axis out of range")
    sidx = st.axes.index(axis)
    d = st.d
    order = [(sidx + i) % d for i in range(d)] + [d]
    st.phi = np.ascontiguousarray(st.phi.transpose(order))
    st.psi = np.ascontiguousarray(st.psi.transpose(order))
    if st.psi_imp is not None:
        st.psi_imp = np.ascontiguousarray(st.psi_imp.transpose(order))
    st.axes = tuple(st.axes[(sidx + i) % d] for i in range(d))


def step(st: State, axis: int, D: int, p: int, q_swap: int = 4, q_rho: int = 4,
         seed: int = 0x5EED, method: str = "triad", mlp: dict | None = None,
         r_bond: int = 1) -> State:
    """One coarse-graining step along physical `axis` (in place; returns st).  `mlp`
    (parameters of oracle/sketch_mlp.py) selects the learned sketch of the triad
    isometries.  r_bond > 1 is the internal-line overspanning of the bond swap (ILO,
    Sec. II C, Appendix A): the re-split bonds alpha, beta and the swapped bond gamma
    keep r_bond D values instead of D; the sketch of the bond swap has r_bond D + p
    columns."""
    if D < 1 or p < 0 or r_bond < 1:
        raise ValueError("need D >= 1, p >= 0 and r_bond >= 1")
    Db = r_bond * D
    _rotate(st, axis)
    A, Dm, s = resplit(st.phi, st.psi, Db)
    if method == "triad" and st.d == 3:
        imp = (st.phi, st.psi_imp) if st.psi_imp is not None else None
        phi, psi, psi_imp, diag = _triad3_step(A, Dm, s, D, p, q_swap, q_rho, seed, st.nsteps,
                                               Db, imp, st.imp_pair)
    elif method == "triad":
        if st.d != 4:
            raise ValueError("triad-ATRG is defined for d = 3 and 4 (d = 2: method 'atrg')")
        imp = (st.phi, st.psi_imp) if st.psi_imp is not None else None
        phi, psi, psi_imp, diag = _triad_step(A, Dm, s, D, p, q_swap, q_rho, seed, st.nsteps, imp,
                                              mlp, Db, st.imp_pair)
    elif method == "atrg":
        phi, psi, psi_imp, diag = _atrg_step(A, Dm, s, D, p, q_swap, q_rho, seed, st.nsteps, Db)
    else:
        raise ValueError(method)
    c = frob_norm(phi, psi)
    st.imp_pair = False
    st.phi = phi
    st.psi = psi / c
    st.psi_imp = None if psi_imp is None else psi_imp / c
    st.nsteps += 1
    st.logsum += math.log(c) / 2.0 ** st.nsteps
    diag["log_c"] = math.log(c)
    st.diag.append(diag)
    return st


def lnZ_per_site(st: State) -> float:
    """lnZ/V = sum_n ln(c_n)/2^n + 2^-N ln Tr T_N on the 2^N-site periodic lattice."""
    tr = trace_T(st.phi, st.psi)
    return st.logsum + math.log(abs(tr)) / 2.0 ** st.nsteps


def free_energy(st: State):
    """(f, lnZ/V) with f = -(lnZ/V)/beta (Sec. III A); f is NaN at beta = 0."""
    lz = lnZ_per_site(st)
    f = -lz / st.beta if st.beta > 0 else float("nan")
    return f, lz


def magnetisation(st: State) -> float:
    """<observable> = Tr(Phi Psi_imp^T) / Tr(Phi Psi^T)."""
    return trace_T(st.phi, st.psi_imp) / trace_T(st.phi, st.psi)


def nn_correlation(st: State) -> float:
    """<o_x o_(x+e)> of a run started with impurity "pair": Tr(Phi Psi_imp^T) / Tr(Phi Psi^T)
    once the first step has merged the two impurities (Sec. III D, two impurity tensors)."""
    if st.imp_pair or st.nsteps < 1:
        raise ValueError("the pair impurity is merged by the first step")
    return trace_T(st.phi, st.psi_imp) / trace_T(st.phi, st.psi)


def internal_energy(st: State) -> float:
    """Ising coupling energy per site, U = -(1/V) d lnZ/d beta = -d <s_x s_(x+e)> on a
    lattice whose axes are equivalent (the pair lies along the first step's axis and
    stands for every axis; the field term -h<s> is not included)."""
    return -st.d * nn_correlation(st)


def run(model: str, d: int, beta: float, h: float, D: int, p: int, nsteps: int,
        q_swap: int = 4, q_rho: int = 4, seed: int = 0x5EED, method: str = "triad",
        axes=None, mlp: dict | None = None, r_bond: int = 1,
        impurity: str = "site") -> State:
    """Convenience driver: nsteps steps cycling the axes 0,1,..,d-1 (or `axes`)."""
    st = (init_ising(d, beta, h, impurity) if model == "ising"
          else init_clock(d, 3, beta, h, impurity))
    for n in range(nsteps):
        ax = (n % d) if axes is None else axes[n]
        step(st, ax, D, p, q_swap, q_rho, seed, method, mlp, r_bond)
    return st



def gu_wen_ratio(st: State) -> float:
    """X = (Tr A)^2 / Tr(A^2) with A_kl = sum T[i1 i2 i3 k, i1 i2 i3 l]  (Sec. III D, eq. X;
    the ratio of Gu and Wen, which counts the ground-state degeneracy: 1 disordered,
    2 in the Z2-ordered phase).  The open leg is the one of the last physical axis; the
    other legs are traced pairwise (forward index = backward index)."""
    d = st.d
    slot = st.axes.index(d - 1)
    legs = "abcdefgh"[:d]
    fa = "".join("k" if i == slot else legs[i] for i in range(d)) + "z"
    fb = "".join("l" if i == slot else legs[i] for i in range(d)) + "z"
    A = np.einsum(f"{fa},{fb}->kl", st.phi, st.psi)
    return float(np.trace(A) ** 2 / np.trace(A @ A))
