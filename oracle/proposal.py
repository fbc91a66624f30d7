"""Learned proposal: oracle (numpy, FP64) of the message-passing network.

THIS IS TEST INFRASTRUCTURE, NOT PRODUCT CODE (see oracle/__init__.py).

The paper names learned initial assignments as complementary to RbmSAT
(Sec. 2, related work on learned SAT heuristics). The network here is the
plain definition of the one the CUDA library trains, written with numpy and
scipy sparse products so that each step can be checked by eye:

    f_v = [pos_v / deg_v - 1/2, log(1 + deg_v) / 4, 1]     (0 for deg_v = 0)
    g_c = [log(w_c) / 8, len_c / 4, 1]
    h_v^0 = relu(Wf f_v),  h_c^0 = relu(Wg g_c)             (64 wide)
    for l = 1..L:
        m_c   = (1 / len_c) sum_{(v, s) in c} s h_v^{l-1}
        h_c^l = relu(Wc_l [m_c ; h_c^{l-1}] + bc_l)
        a_v   = (1 / deg_v) sum_{(c, s) : v in c} s h_c^l
        h_v^l = relu(Wv_l [a_v ; h_v^{l-1}] + bv_l)
    z_v = wo . h_v^L + bo,   p_v = sigmoid(z_v)
    loss = mean_v softplus(z_v) - y_v z_v                    (binary cross entropy)

s = +1 for a plain literal, -1 for a negated one; an empty clause has m_c = 0
and a variable in no clause a_v = 0. Weight matrices enter the forward pass
rounded to BF16 (round to nearest even) when bf16=True, as in the library;
biases and activations stay FP64 here.

Parameters are one flat vector; `layout(L, H)` gives the slices.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

H = 64


def layout(L: int = 3, Hd: int = H):
    """Ordered (name, shape) of the flat parameter vector."""
    out = [("Wf", (Hd, 3)), ("Wg", (Hd, 3))]
    for l in range(L):
        out += [(f"Wc{l}", (Hd, 2 * Hd)), (f"bc{l}", (Hd,)), (f"Wv{l}", (Hd, 2 * Hd)),
                (f"bv{l}", (Hd,))]
    out += [("wo", (Hd,)), ("bo", (1,))]
    return out


def n_params(L: int = 3, Hd: int = H) -> int:
    return int(sum(np.prod(s) for _, s in layout(L, Hd)))


def unpack(theta, L=3, Hd=H):
    P, o = {}, 0
    for name, shape in layout(L, Hd):
        k = int(np.prod(shape))
        P[name] = theta[o:o + k].reshape(shape)
        o += k
    return P


def bf16_round(a):
    """Round FP32 values to BF16 (nearest, ties to even), returned as float64."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def graph(n, off, lits, w):
    """Sparse incidence operators and input features of one formula (or of
    the disjoint union of a batch)."""
    off = np.asarray(off, np.int64)
    lits = np.asarray(lits, np.int64)
    m = len(off) - 1
    ln = np.diff(off)
    cl = np.repeat(np.arange(m), ln)
    var = np.abs(lits) - 1
    s = np.sign(lits).astype(np.float64)
    S = sp.csr_matrix((s, (cl, var)), shape=(m, n))  # signed clause x variable (duplicates add)
    deg = np.bincount(var, minlength=n).astype(np.float64)
    pos = np.bincount(var, weights=(s > 0).astype(np.float64), minlength=n)
    inv_len = np.where(ln > 0, 1.0 / np.maximum(ln, 1), 0.0)
    inv_deg = np.where(deg > 0, 1.0 / np.maximum(deg, 1), 0.0)
    f = np.stack([np.where(deg > 0, pos * inv_deg - 0.5, 0.0), np.log1p(deg) / 4, np.ones(n)], 1)
    wv = np.ones(m) if w is None else np.asarray(w, np.float64)
    g = np.stack([np.log(wv) / 8, ln / 4.0, np.ones(m)], 1)
    return dict(n=n, m=m, S=S, inv_len=inv_len, inv_deg=inv_deg, f=f, g=g)


def _relu(x):
    return np.maximum(x, 0.0)


def forward(G, theta, L=3, bf16=True):
    """Returns (z, cache)."""
    P = unpack(np.asarray(theta, np.float64), L)
    Wt = {k: (bf16_round(v) if bf16 and k[0] == "W" else v) for k, v in P.items()}
    S, il, idg = G["S"], G["inv_len"][:, None], G["inv_deg"][:, None]
    hv = _relu(G["f"] @ Wt["Wf"].T)
    hc = _relu(G["g"] @ Wt["Wg"].T)
    cache = dict(hv0=hv, hc0=hc, layers=[])
    for l in range(L):
        mc = il * (S @ hv)
        xc = np.concatenate([mc, hc], 1)
        hc = _relu(xc @ Wt[f"Wc{l}"].T + P[f"bc{l}"])
        av = idg * (S.T @ hc)
        xv = np.concatenate([av, hv], 1)
        hv = _relu(xv @ Wt[f"Wv{l}"].T + P[f"bv{l}"])
        cache["layers"].append(dict(xc=xc, hc=hc, xv=xv, hv=hv))
    z = hv @ P["wo"] + P["bo"][0]
    cache["W"] = Wt
    return z, cache


def loss(z, y):
    y = np.asarray(y, np.float64)
    return float(np.mean(np.logaddexp(0.0, z) - y * z))


def backward(G, theta, y, L=3, bf16=True):
    """(loss, gradient of the flat parameters). With bf16 the gradient is that
    of the network whose weights are the BF16-rounded values (the rounding
    itself is treated as the identity, as in mixed-precision training)."""
    z, C = forward(G, theta, L, bf16)
    P = unpack(np.asarray(theta, np.float64), L)
    W = C["W"]
    n = G["n"]
    y = np.asarray(y, np.float64)
    S, il, idg = G["S"], G["inv_len"][:, None], G["inv_deg"][:, None]
    grads = {k: np.zeros_like(v) for k, v in P.items()}
    dz = (1.0 / (1.0 + np.exp(-z)) - y) / n
    hvL = C["layers"][-1]["hv"] if L else C["hv0"]
    grads["wo"] = hvL.T @ dz
    grads["bo"] = np.array([dz.sum()])
    dhv = np.outer(dz, P["wo"])
    dhc = None
    for l in reversed(range(L)):
        Ly = C["layers"][l]
        # variable layer
        dv = dhv * (Ly["hv"] > 0)
        grads[f"Wv{l}"] = dv.T @ Ly["xv"]
        grads[f"bv{l}"] = dv.sum(0)
        dxv = dv @ W[f"Wv{l}"]
        dav, dhv_prev = dxv[:, :H], dxv[:, H:]
        dhc_l = S @ (idg * dav)
        if dhc is not None:
            dhc_l = dhc_l + dhc
        # clause layer
        dc = dhc_l * (Ly["hc"] > 0)
        grads[f"Wc{l}"] = dc.T @ Ly["xc"]
        grads[f"bc{l}"] = dc.sum(0)
        dxc = dc @ W[f"Wc{l}"]
        dmc, dhc = dxc[:, :H], dxc[:, H:]
        dhv = dhv_prev + S.T @ (il * dmc)
    dv0 = dhv * (C["hv0"] > 0)
    grads["Wf"] = dv0.T @ G["f"]
    dc0 = dhc * (C["hc0"] > 0)
    grads["Wg"] = dc0.T @ G["g"]
    flat = np.concatenate([grads[name].reshape(-1) for name, _ in layout(L)])
    return loss(z, y), flat


def init_params(seed=0, L=3):
    """He-style initial parameters (deterministic)."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in layout(L):
        if name[0] == "W":
            parts.append(rng.normal(0.0, np.sqrt(2.0 / shape[1]), size=shape).reshape(-1))
        elif name == "wo":
            parts.append(rng.normal(0.0, np.sqrt(1.0 / H), size=shape))
        else:
            parts.append(np.zeros(shape).reshape(-1))
    return np.concatenate(parts)
