"""Learned sketch for the triad-isometry range finders — TEST INFRASTRUCTURE (oracle).

Plain FP64 NumPy statement of the learned-sketch variant of the randomized range finder
of the triad isometries (Sec. II B, eq. HOSVD: U^A, U^X, U^Y, U^D are ranges of the
Grams rho).  The paper draws a Gaussian sketch; this variant keeps the same Gaussian
draw G and rescales its rows by per-leg weights proposed by a small network:

    Omega[(a b), m] = w_1[a] w_2[b] G[(a b), m],     w_l[i] = 2^(q(u_l[i])),

with u_l[i] the network output for index i of leg l of the pair and q(u) = round(16 u)/16
clamped to [-8, 8] (a quantised code, so that the GPU and this oracle take the same
integer decision).  w = 1 is the paper's plain sketch.  Readings:

  * Inputs per leg index i (NIN = 5): (i + 0.5)/d_l, log2(m_i d_l)/8 with m_i the share
    of tr(rho) on the diagonal entries of index i (m_i d_l clipped at 2^-40, above the
    rounding level of entries that vanish by symmetry), log2(d_l)/8,
    log2(d_other)/8, chi/n.  The leg bases are re-chosen by the squeezers between steps,
    so the previous step's isometry has no index-wise meaning here; the diagonal share of
    rho carries the same information about where the range lives.
  * Network: 3 layers, NIN -> 256 -> 256 -> 1, ReLU, FP32 weights; inference runs with
    BF16 inputs, weights and hidden activations (FP32 biases, FP32 sums), emulated here
    by rounding to BF16 and summing exactly in FP64.
  * Training target: t_i = 0.5 log2(lev_i d_l), lev_i the leverage of index i in the
    converged plain range Q (sum over the other leg and the columns of Q^2, divided by
    the number of columns); loss = mean (u - t)^2.
  * Fallback: probe residual r(Q) = ||rho P - Q Q^T rho P||_F / ||rho P||_F with 8
    Gaussian probe columns (tag TAG_PROBE); the learned range is used unless
    r(learned) > 1.5 r(plain), in which case the plain range is returned.
"""
from __future__ import annotations

import numpy as np

from . import trg_oracle as O

NIN, NHID = 5, 256
TAG_PROBE = {"A": 13, "X": 14, "Y": 15, "D": 16}
NPROBE = 8
FALLBACK_RATIO = 1.5
QSTEP = 16.0            # u is quantised to 1/16 (in log2 units) ...
QMAX = 8.0              # ... and clamped to [-8, 8]


# ----------------------------------------------------------------------------------
# BF16 rounding (round to nearest even on the FP32 bit pattern), for the inference
# emulation
# ----------------------------------------------------------------------------------
def bf16(x) -> np.ndarray:
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    r = ((b + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


# ----------------------------------------------------------------------------------
# Network
# ----------------------------------------------------------------------------------
def init_params(seed: int = 0) -> dict:
    """He-style initial weights (FP32 values held in FP64 arrays)."""
    rng = np.random.default_rng(seed)
    p = {
        "W1": rng.standard_normal((NHID, NIN)) * np.sqrt(2.0 / NIN),
        "b1": np.zeros(NHID),
        "W2": rng.standard_normal((NHID, NHID)) * np.sqrt(2.0 / NHID),
        "b2": np.zeros(NHID),
        "W3": rng.standard_normal((1, NHID)) * np.sqrt(1.0 / NHID),
        "b3": np.zeros(1),
    }
    return {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}


def forward(p: dict, X: np.ndarray) -> tuple[np.ndarray, dict]:
    """FP64 forward pass; X rows x NIN -> u (rows,), plus the activations."""
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    u = (h2 @ p["W3"].T + p["b3"])[:, 0]
    return u, {"X": X, "z1": z1, "h1": h1, "z2": z2, "h2": h2}


def forward_bf16(p: dict, X: np.ndarray) -> np.ndarray:
    """Inference in the precision the method fixes for it: BF16 inputs, weights and
    hidden activations, FP32 biases and FP32 sums in a stated order, so that the
    quantised output code is a reproducible integer decision:
      layer 1: z = b1, then z += w1[i] x[i] for i = 0..4;
      layer 2: a = 0, then a += W2[j, k] h1[k] for k = 0..255; h2 = bf16(relu(a + b2));
      layer 3: products W3[j] h2[j] in 8 groups of 32 (j = 32 g + l), each group summed
               pairwise (halves added: 16, 8, 4, 2, 1), then u = b3 + group 0 + ... + 7.
    A product of two BF16 values is exact in FP32, so every step is one FP32 rounding."""
    f32 = np.float32
    Xb = bf16(X).astype(f32)
    W1, W2, W3 = (bf16(p[k]).astype(f32) for k in ("W1", "W2", "W3"))
    b1, b2, b3 = (p[k].astype(f32) for k in ("b1", "b2", "b3"))
    z = np.broadcast_to(b1, (X.shape[0], NHID)).copy()
    for i in range(NIN):
        z = (z + Xb[:, i:i + 1] * W1[None, :, i]).astype(f32)
    h1 = bf16(np.maximum(z, f32(0))).astype(f32)
    a = np.zeros((X.shape[0], NHID), dtype=f32)
    for k in range(NHID):
        a = (a + h1[:, k:k + 1] * W2[None, :, k]).astype(f32)
    h2 = bf16(np.maximum((a + b2).astype(f32), f32(0))).astype(f32)
    prod = (h2 * W3[0][None, :]).astype(f32).reshape(X.shape[0], 8, 32)
    half = 16
    while half >= 1:
        prod = (prod[:, :, :half] + prod[:, :, half:2 * half]).astype(f32)
        half //= 2
    u = np.broadcast_to(b3[0], (X.shape[0],)).astype(f32).copy()
    for g in range(8):
        u = (u + prod[:, g, 0]).astype(f32)
    return u.astype(np.float64)


def loss_and_grads(p: dict, X: np.ndarray, t: np.ndarray) -> tuple[float, dict]:
    """L = mean (u - t)^2 and its gradient with respect to every parameter (chain rule
    through the three affine maps and the two ReLUs)."""
    u, a = forward(p, X)
    n = X.shape[0]
    du = 2.0 * (u - t) / n                       # dL/du
    g = {}
    g["W3"] = du[None, :] @ a["h2"]
    g["b3"] = np.array([du.sum()])
    dh2 = du[:, None] * p["W3"]                  # rows x NHID
    dz2 = dh2 * (a["z2"] > 0)
    g["W2"] = dz2.T @ a["h1"]
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * (a["z1"] > 0)
    g["W1"] = dz1.T @ a["X"]
    g["b1"] = dz1.sum(axis=0)
    return float(np.mean((u - t) ** 2)), g


def quantise(u: np.ndarray) -> np.ndarray:
    """Integer code of u in steps of 1/16 (round half to even), clamped."""
    return np.clip(np.rint(u * QSTEP), -QMAX * QSTEP, QMAX * QSTEP)


# ----------------------------------------------------------------------------------
# Features, targets, learned range finder
# ----------------------------------------------------------------------------------
def leg_features(rho: np.ndarray, da: int, db: int, chi: int) -> tuple[np.ndarray, np.ndarray]:
    """Inputs (NIN columns, FP64) of every index of leg 1 (da rows) and leg 2 (db rows)."""
    n = da * db
    dg = np.diag(rho).reshape(da, db)
    tr = dg.sum()
    m1 = dg.sum(axis=1) / tr
    m2 = dg.sum(axis=0) / tr

    def feats(m, d, dother):
        F = np.empty((d, NIN))
        F[:, 0] = (np.arange(d) + 0.5) / d
        F[:, 1] = np.log2(np.maximum(m * d, 2.0 ** -40)) / 8.0
        F[:, 2] = np.log2(d) / 8.0
        F[:, 3] = np.log2(dother) / 8.0
        F[:, 4] = chi / n
        return F

    return feats(m1, da, db), feats(m2, db, da)


def leverage_targets(Q: np.ndarray, da: int, db: int) -> tuple[np.ndarray, np.ndarray]:
    """t_l[i] = 0.5 log2(lev_l[i] d_l) from an orthonormal range Q (n x c)."""
    c = max(int(np.count_nonzero(np.linalg.norm(Q, axis=0) > 0.5)), 1)
    sq = (Q ** 2).reshape(da, db, -1)
    lev1 = sq.sum(axis=(1, 2)) / c
    lev2 = sq.sum(axis=(0, 2)) / c
    t1 = 0.5 * np.log2(np.maximum(lev1 * da, 2.0 ** -40))
    t2 = 0.5 * np.log2(np.maximum(lev2 * db, 2.0 ** -40))
    return t1, t2


def sketch_weights(p: dict, rho: np.ndarray, da: int, db: int, chi: int) -> np.ndarray:
    """Row weights w_1[a] w_2[b] of Omega (length n), from the BF16 inference."""
    F1, F2 = leg_features(rho, da, db, chi)
    c1 = quantise(forward_bf16(p, F1))
    c2 = quantise(forward_bf16(p, F2))
    return (np.exp2(c1 / QSTEP)[:, None] * np.exp2(c2 / QSTEP)[None, :]).reshape(-1)


def probe_residual(rho: np.ndarray, Q: np.ndarray, key) -> float:
    P = rho @ O.gaussian(key, rho.shape[0], NPROBE)
    nrm = np.linalg.norm(P)
    return float(np.linalg.norm(P - Q @ (Q.T @ P)) / nrm) if nrm > 0 else 0.0


def range_finder(rho: np.ndarray, Omega: np.ndarray, chi: int, q_rho: int) -> np.ndarray:
    """Orthonormal basis of range(rho^(q_rho+1) Omega) (as in rsvd_range_sym)."""
    Q = O.orth(rho @ Omega, chi)
    for _ in range(q_rho):
        Q = O.orth(rho @ Q, chi)
    return Q


def rsvd_learned(p: dict, rho: np.ndarray, da: int, db: int, chi: int, q_rho: int, key,
                 key_probe) -> tuple[np.ndarray, dict]:
    """Learned-sketch range of rho with the plain range as fallback."""
    n = rho.shape[0]
    if chi >= n:
        return np.eye(n), {"used": "identity"}
    G = O.gaussian(key, n, chi)
    Qp = range_finder(rho, G, chi, q_rho)
    w = sketch_weights(p, rho, da, db, chi)
    Ql = range_finder(rho, w[:, None] * G, chi, q_rho)
    rl, rp = probe_residual(rho, Ql, key_probe), probe_residual(rho, Qp, key_probe)
    use = rl <= FALLBACK_RATIO * rp
    return (Ql if use else Qp), {"used": "learned" if use else "plain", "r_learned": rl,
                                 "r_plain": rp}
