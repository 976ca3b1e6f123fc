"""FP64 reference of the learned sampler (test infrastructure: only tests/, smoke() and the CPU legs of
bench.py use it).

The paper samples the emitted photon energy from the spin-resolved spectrum w(lambda; s_beta) with
inverse-CDF tables and rejects a direct three-dimensional table in (chi, r, s_beta) for its memory
(Sec. 5.1).  The learned sampler stands in for that table.  Since w is linear in s_beta, the exact
r-quantile of the mixture lies between the quantiles of the two spin branches; the network predicts
the correction to their rate-weighted blend:

  inputs   x = ((ln chi - m) / h, y / 10, s_beta),  y = logit(r) clamped to [-20, 20],
           m, h = centre and half-width of ln chi over [1e-3, 1e2];
  baseline ln u'_b = a ln u'_up(chi, r) + (1 - a) ln u'_down(chi, r),
           a = (1 + s) I_up / ((1 + s) I_up + (1 - s) I_down)  (branch ICDFs and rates from the tables),
           xi3_b = F3 / F0 at lambda(u'_b) (App. A.1, s_i = s beta_hat, s_f = 0);
  outputs  o = (100 (ln u' - ln u'_b), 100 xi1, 100 xi2, 100 (xi3 - xi3_b))
           (xi1 = xi2 = 0 for s_i along beta_hat with the final spin summed).

Network 3 -> 64 -> 64 -> 64 -> 4 with SiLU.  Numerics the CUDA kernels follow: the first layer in
FP32 arithmetic (here FP64) on unrounded inputs; layers 2-4 take BF16-rounded weights and activations
with higher-precision accumulation; biases are not rounded.  The backward pass is the exact derivative
of that forward with the rounding taken as the identity (straight-through).  Loss: the mean over the
batch of the squared error summed over the four outputs.
"""
from __future__ import annotations

import math

import numpy as np

LAYERS = (3, 64, 64, 64, 4)
LNCHI_LO, LNCHI_HI = math.log(1e-3), math.log(1e2)
LNCHI_MID, LNCHI_HALF = 0.5 * (LNCHI_LO + LNCHI_HI), 0.5 * (LNCHI_HI - LNCHI_LO)
Y_CLAMP = 20.0
OUT_SCALE = 100.0


def bf16(x):
    """Round to bfloat16 (round to nearest, ties to even), returned as float64."""
    x32 = np.asarray(x, dtype=np.float32)
    b = x32.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def features(chi, r, s):
    """Network inputs for arrays chi, r, s."""
    chi, r, s = (np.asarray(a, dtype=np.float64) for a in (chi, r, s))
    y = np.clip(np.log(r) - np.log1p(-r), -Y_CLAMP, Y_CLAMP)
    return np.stack([(np.log(chi) - LNCHI_MID) / LNCHI_HALF, y / 10.0, s], axis=1)


def init_params(seed: int = 0):
    """Deterministic FP32 initial weights (uniform +-sqrt(6/(fan_in+fan_out)) times 0.5, zero biases)."""
    rng = np.random.default_rng(seed)
    p = {}
    for l in range(4):
        fi, fo = LAYERS[l], LAYERS[l + 1]
        lim = 0.5 * math.sqrt(6.0 / (fi + fo))
        p[f"W{l + 1}"] = rng.uniform(-lim, lim, (fo, fi)).astype(np.float32).astype(np.float64)
        p[f"b{l + 1}"] = np.zeros(fo)
    return p


def forward(p, X, rounding: bool = True):
    """Outputs and the cache of pre-activations (B, 4)."""
    q = bf16 if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    z1 = X @ p["W1"].T + p["b1"]
    h1 = silu(z1)
    z2 = q(h1) @ q(p["W2"]).T + p["b2"]
    h2 = silu(z2)
    z3 = q(h2) @ q(p["W3"]).T + p["b3"]
    h3 = silu(z3)
    o = q(h3) @ q(p["W4"]).T + p["b4"]
    return o, {"X": X, "z1": z1, "h1": h1, "z2": z2, "h2": h2, "z3": z3, "h3": h3, "q": q}


def loss_and_grads(p, X, T, rounding: bool = True):
    """Loss L = mean_b sum_k (o_bk - t_bk)^2 and its gradients with respect to every parameter."""
    o, c = forward(p, X, rounding)
    q = c["q"]
    B = X.shape[0]
    L = float(np.sum((o - T) ** 2) / B)
    d = 2.0 * (o - T) / B
    g = {"W4": d.T @ q(c["h3"]), "b4": d.sum(0)}
    dh = d @ q(p["W4"])
    dz = dh * dsilu(c["z3"])
    g["W3"], g["b3"] = dz.T @ q(c["h2"]), dz.sum(0)
    dh = dz @ q(p["W3"])
    dz = dh * dsilu(c["z2"])
    g["W2"], g["b2"] = dz.T @ q(c["h1"]), dz.sum(0)
    dh = dz @ q(p["W2"])
    dz = dh * dsilu(c["z1"])
    g["W1"], g["b1"] = dz.T @ c["X"], dz.sum(0)
    return L, g


def adamw_step(p, g, state, lr, wd=1e-4, beta1=0.9, beta2=0.999, eps=1e-8):
    """One AdamW step (decoupled weight decay on the weights, not the biases); state holds m, v, t."""
    t = state.get("t", 0) + 1
    state["t"] = t
    for k in p:
        m = state.setdefault("m" + k, np.zeros_like(p[k]))
        v = state.setdefault("v" + k, np.zeros_like(p[k]))
        m[...] = beta1 * m + (1 - beta1) * g[k]
        v[...] = beta2 * v + (1 - beta2) * g[k] ** 2
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        p[k] = p[k] - lr * (mh / (np.sqrt(vh) + eps) + (wd * p[k] if k.startswith("W") else 0.0))
    return p


def baseline(tb, chi, r, s):
    """(ln u'_b, a): the rate-weighted blend of the two branch quantiles of the oracle's tables."""
    Iu, Id = tb.nlc_rate_lookup(0, chi), tb.nlc_rate_lookup(1, chi)
    a = (1.0 + s) * Iu / ((1.0 + s) * Iu + (1.0 - s) * Id)
    return a * tb.icdf(False, 0, chi, r) + (1.0 - a) * tb.icdf(False, 1, chi, r), a


def xi3_closed(chi, ln_up, s):
    """xi3 = F3/F0 at u' for s_i = s beta_hat, s_f = 0 (App. A.1, via the oracle's Stokes spectrum)."""
    import oracle as O
    up = math.exp(ln_up)
    lam = O.nlc_lambda(chi, up)
    F = O.nlc_stokes(lam, O.bessel(up), (0.0, s, 0.0), (0.0, 0.0, 0.0), (1, 0, 0), (0, 1, 0), (0, 0, 1))
    return F[3] / F[0]


def targets(tb, chi, r, s):
    """Scaled network targets for scalar inputs (exact quantile and Stokes vector minus the baseline)."""
    import oracle as O
    ex = O.mlp_target(chi, r, s)
    lb, _ = baseline(tb, chi, r, s)
    return np.array([OUT_SCALE * (ex[0] - lb), OUT_SCALE * ex[1], OUT_SCALE * ex[2],
                     OUT_SCALE * (ex[3] - xi3_closed(chi, lb, s))])


def decode(tb, chi, r, s, o):
    """Sampler outputs (ln u', xi1, xi2, xi3) from the network output o."""
    lb, _ = baseline(tb, chi, r, s)
    ln_up = lb + o[0] / OUT_SCALE
    return np.array([ln_up, o[1] / OUT_SCALE, o[2] / OUT_SCALE, xi3_closed(chi, lb, s) + o[3] / OUT_SCALE])
