"""FP64 reference of the learned support proposal for the generally K-sparse
path (not in the paper; the warm start of Algorithm 2's per-bin Subspace
Pursuit by a small network, judged by the paper's own residual).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU legs use it; the library never imports or calls it.  It shares no code
with the CUDA path.  Plain numpy in float64.

Per voted bin k (a_k > 0) of a signal with syndromes Y_l[k] for the shifts
sh_0..sh_{n-1} (the 2a_m consecutive shifts 0..2a_m-1, then the r random
shifts n_j):

  features   m~_l = Y_l[k] w^{-k sh_l} (w = e^{2 pi i/N}) removes the bin's
             own phase ramp, leaving m~_l = sum_j p_j e^{2 pi i t_j sh_l / d}
             for the aliases s_j = k + t_j M; then m~ is rotated so that m~_0
             is real and non-negative and scaled to unit 2-norm; the feature
             vector is (Re m~_0, Im m~_0, Re m~_1, ...), 2n values.
  network    z1 = f W1 + b1, a1 = relu(z1), z2 = a1 W2 + b2, a2 = relu(z2),
             z3 = a2 W3 + b3; W1..W3 are used rounded to FP16 ("FP16
             weights, FP32 accumulate" on the GPU), biases in full precision.
             z3[:d] are support logits over t = 0..d-1, z3[d:] count logits
             over 0..a_m+1 aliases (a_m+1 = "more than a_m").
  loss       per row: cross-entropy of the count logits plus the mean over
             t of the binary cross-entropy of the support logits; averaged
             over rows.
  proposal   the min(2 a_k, d) largest support logits (ties: lower t), in
             ascending t, replace the candidates of pruning Step 2; Subspace
             Pursuit with sparsity a_k runs on them as in Step 3.
  judge      both solutions' squared residuals over all 2a_m + r equations
             of Eq. (3); the network's replaces the plain one only when
             r_mlp^2 < (1 - 1e-6) r_plain^2; otherwise the plain solution
             stands (fallback).
"""
from __future__ import annotations

import numpy as np

JUDGE_MARGIN = 1e-6


# ------------------------------------------------------------------ layout
def param_layout(n_in: int, n_hidden: int, n_out: int):
    """(name, shape) of the flat FP32 parameter vector, in order."""
    return [("W1", (n_in, n_hidden)), ("b1", (n_hidden,)),
            ("W2", (n_hidden, n_hidden)), ("b2", (n_hidden,)),
            ("W3", (n_hidden, n_out)), ("b3", (n_out,))]


def unpack(flat, n_in, n_hidden, n_out):
    out, o = {}, 0
    for name, shape in param_layout(n_in, n_hidden, n_out):
        n = int(np.prod(shape))
        out[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def pack(params, n_in, n_hidden, n_out):
    return np.concatenate([np.asarray(params[name], np.float64).reshape(-1)
                           for name, _ in param_layout(n_in, n_hidden, n_out)])


def fp16(w):
    """The weights as the network uses them (rounded to FP16)."""
    return np.asarray(w, np.float64).astype(np.float16).astype(np.float64)


# ---------------------------------------------------------------- features
def features(Ybin, k: int, shifts, N: int):
    """Features of one bin from its syndromes Ybin[l] = Y_{sh_l}[k]."""
    sh = np.asarray(shifts, dtype=np.int64)
    ang = ((-(int(k) % N) * sh) % N).astype(np.float64) * (2.0 * np.pi / N)
    m = np.asarray(Ybin, np.complex128) * np.exp(1j * ang)
    a0 = abs(m[0])
    if a0 > 0:
        m = m * (np.conj(m[0]) / a0)
    nrm = np.sqrt(np.sum(np.abs(m) ** 2))
    if nrm > 0:
        m = m / nrm
    f = np.empty(2 * m.size)
    f[0::2] = m.real
    f[1::2] = m.imag
    return f


# ----------------------------------------------------------------- network
def forward(P, F, half=True):
    """Logits (rows x n_out) and the intermediate values; half=False skips
    the FP16 rounding of the weights (for finite-difference checks)."""
    q = fp16 if half else (lambda w: np.asarray(w, np.float64))
    F = np.asarray(F, np.float64)
    z1 = F @ q(P["W1"]) + P["b1"]
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ q(P["W2"]) + P["b2"]
    a2 = np.maximum(z2, 0.0)
    z3 = a2 @ q(P["W3"]) + P["b3"]
    return z3, (F, z1, a1, z2, a2)


def _softplus(z):
    return np.logaddexp(0.0, z)


def loss_and_grad(P, F, cls, sup, n_sup, half=True):
    """Mean loss over the rows and its gradient with respect to every
    parameter (the weights' gradient is taken at their FP16 values unless
    half=False).  cls: count labels (int, rows); sup: support labels
    (rows x n_sup, 0/1)."""
    q = fp16 if half else (lambda w: np.asarray(w, np.float64))
    z3, (F, z1, a1, z2, a2) = forward(P, F, half)
    R = F.shape[0]
    zs, zc = z3[:, :n_sup], z3[:, n_sup:]
    y = np.asarray(sup, np.float64)
    # BCE with logits: softplus(z) - y z
    bce = (_softplus(zs) - y * zs).mean(axis=1)
    zmax = zc.max(axis=1, keepdims=True)
    lse = zmax[:, 0] + np.log(np.exp(zc - zmax).sum(axis=1))
    ce = lse - zc[np.arange(R), np.asarray(cls)]
    loss = float((ce + bce).mean())
    d3 = np.empty_like(z3)
    d3[:, :n_sup] = (1.0 / (1.0 + np.exp(-zs)) - y) / (R * n_sup)
    p = np.exp(zc - lse[:, None])
    p[np.arange(R), np.asarray(cls)] -= 1.0
    d3[:, n_sup:] = p / R
    g = {"W3": a2.T @ d3, "b3": d3.sum(axis=0)}
    d2 = (d3 @ q(P["W3"]).T) * (z2 > 0)
    g["W2"], g["b2"] = a1.T @ d2, d2.sum(axis=0)
    d1 = (d2 @ q(P["W2"]).T) * (z1 > 0)
    g["W1"], g["b1"] = F.T @ d1, d1.sum(axis=0)
    return loss, g


def init_params(n_in, n_hidden, n_out, rng):
    """He-uniform weights, zero biases (for CPU-side training in tests)."""
    P = {}
    for name, shape in param_layout(n_in, n_hidden, n_out):
        if name.startswith("W"):
            lim = np.sqrt(6.0 / shape[0])
            P[name] = rng.uniform(-lim, lim, size=shape)
        else:
            P[name] = np.zeros(shape)
    return P


def train_adam(P, F, cls, sup, n_sup, epochs, batch, lr, seed):
    """Plain Adam on the FP64 loss (CPU; for small test networks)."""
    rng = np.random.default_rng(seed)
    m = {k: np.zeros_like(v) for k, v in P.items()}
    v = {k: np.zeros_like(x) for k, x in P.items()}
    b1, b2, eps, t = 0.9, 0.999, 1e-8, 0
    for _ in range(epochs):
        perm = rng.permutation(F.shape[0])
        for i in range(0, F.shape[0], batch):
            idx = perm[i:i + batch]
            _, g = loss_and_grad(P, F[idx], cls[idx], sup[idx], n_sup)
            t += 1
            for k in P:
                m[k] = b1 * m[k] + (1 - b1) * g[k]
                v[k] = b2 * v[k] + (1 - b2) * g[k] ** 2
                P[k] = P[k] - lr * (m[k] / (1 - b1 ** t)) / (np.sqrt(v[k] / (1 - b2 ** t)) + eps)
    return P


def proposal(logits_sup, a: int, d: int):
    """The min(2a, d) largest support logits (ties: lower t), ascending t."""
    n = min(2 * a, d)
    order = sorted(range(d), key=lambda t: (-logits_sup[t], t))
    return sorted(order[:n])


def boundary_gap(logits_sup, a: int, d: int):
    """Gap between the last kept and the first dropped support logit (how
    firmly the proposal is decided; infinite when nothing is dropped)."""
    n = min(2 * a, d)
    s = np.sort(np.asarray(logits_sup))[::-1]
    return float(s[n - 1] - s[n]) if n < d else float("inf")


# ------------------------------------------------------ judged Algorithm 2
def residual2(Ybin, shifts, k, M, N, ts, bs):
    """Squared residual of a bin's solution over all its equations (Eq. (3))."""
    sh = np.asarray(shifts, dtype=np.int64)
    r = np.asarray(Ybin, np.complex128).copy()
    for t, b in zip(ts, bs):
        e = ((int(k) + int(t) * M) * sh) % N
        r -= b * np.exp(2j * np.pi * e.astype(np.float64) / N)
    return float(np.sum(np.abs(r) ** 2))


def general_mlp(orc, x, M, K, logits_fn, a_max=3, r=None, seed=0, sp_iters=8, cap=None):
    """Algorithm 2 with the learned proposal judged per bin.

    orc: the oracle module (FP64 syndromes, plain Algorithm 2, Subspace
    Pursuit); logits_fn(F, bins): features (rows x 2n) of the voted bins
    `bins` -> logits (rows x n_out).
    Returns (idx, val, a_k, info) where info holds per voted bin the plain
    and network residuals, whether the network's solution was taken, and
    the proposal's boundary gap."""
    x = np.asarray(x).astype(np.complex128)
    N = x.size
    d = N // M
    r = 3 * a_max if r is None else r
    ns = orc.cs_shifts(seed, d, r)
    shifts = np.concatenate([np.arange(2 * a_max), ns]).astype(np.int64)
    idx, val, ak = orc.general(x, M, K, a_max=a_max, r=r, seed=seed, sp_iters=sp_iters,
                               cap=cap if cap is not None else 4 * K + 64)
    Y = np.stack([orc.syndrome(x, d, int(s)) for s in shifts])  # [n, M]
    plain = {}
    for s_, v_ in zip(idx.tolist(), val.tolist()):
        plain.setdefault(s_ % M, []).append((s_ // M, v_))
    ks = np.nonzero(ak)[0]
    out = {int(s_): v_ for s_, v_ in zip(idx.tolist(), val.tolist())}
    info = {}
    if ks.size:
        F = np.stack([features(Y[:, k], int(k), shifts, N) for k in ks])
        L = np.asarray(logits_fn(F, ks), np.float64)
        for j, k in enumerate(ks.tolist()):
            a = int(ak[k])
            cands = proposal(L[j, :d], a, d)
            gap = boundary_gap(L[j, :d], a, d)
            Phi = np.exp(2j * np.pi * (((k + np.asarray(cands, np.int64) * M)[None, :] *
                                        ns[:, None]) % N).astype(np.float64) / N)
            try:
                b = orc.subspace_pursuit(Phi, Y[2 * a_max:, k], a, iters=sp_iters)
            except ValueError:
                b = np.zeros(len(cands), np.complex128)
            nz = np.nonzero(b)[0]
            pl = plain.get(k, [])
            rp = residual2(Y[:, k], shifts, k, M, N, [t for t, _ in pl], [v for _, v in pl])
            rm = (residual2(Y[:, k], shifts, k, M, N, [cands[u] for u in nz], b[nz])
                  if nz.size else float("inf"))
            take = nz.size > 0 and rm < (1.0 - JUDGE_MARGIN) * rp
            info[k] = {"rp": rp, "rm": rm, "take": bool(take), "gap": gap}
            if take:
                for t, _ in pl:
                    out.pop(k + t * M, None)
                for u in nz:
                    out[int(k + cands[u] * M)] = complex(b[u])
    keys = np.array(sorted(out), dtype=np.int64)
    vals = np.array([out[i] for i in keys.tolist()], dtype=np.complex128)
    if cap is not None:
        keys, vals = keys[:cap], vals[:cap]
    return keys, vals, ak, info
