"""Pins of the learned-sampler oracle (oracle/mlp.py and the exact target in oracle/qed_oracle.c), CPU only.

* BF16 rounding: against PyTorch's float32 -> bfloat16 conversion (an independent implementation).
* SiLU derivative and the whole backward pass: against central finite differences of the forward pass
  (rounding off, so the forward is differentiable).
* AdamW: the first step has the closed form lr (g / (|g| + eps) + wd w).
* Target: at s_beta = +-1 the mixture reduces to one spin branch, whose CDF the oracle also computes
  separately; the target is monotone in r; xi1 = xi2 = 0 and xi3 at s = 0 equals K23 / (-IntK13 +
  kappa K23) with the Bessel functions from scipy; the blended-branch baseline is within 0.05 of it.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import mlp as M


def test_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(size=20000) * 10.0 ** rng.integers(-20, 20, 20000),
                        np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -1.0 - 2.0 ** -8, 0.0, 2.0 ** -126])])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16(x), ref)


def test_dsilu_finite_difference():
    z = np.linspace(-12, 12, 97)
    h = 1e-6
    fd = (M.silu(z + h) - M.silu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - M.dsilu(z))) < 1e-8


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    p = M.init_params(3)
    for k in p:
        p[k] = p[k] + rng.normal(scale=0.1, size=p[k].shape)
    X = rng.normal(size=(5, 3))
    T = rng.normal(size=(5, 4))
    L, g = M.loss_and_grads(p, X, T, rounding=False)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            Lp, _ = M.loss_and_grads(p, X, T, rounding=False)
            flat[idx] = old - h
            Lm, _ = M.loss_and_grads(p, X, T, rounding=False)
            flat[idx] = old
            fd = (Lp - Lm) / (2 * h)
            an = g[k].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (k, idx, fd, an)


def test_adamw_first_step_closed_form():
    p = M.init_params(4)
    g = {k: np.full_like(v, 0.3) * np.sign(np.arange(v.size).reshape(v.shape) % 3 - 1) for k, v in p.items()}
    before = {k: v.copy() for k, v in p.items()}
    lr, wd, eps = 1e-3, 1e-2, 1e-8
    M.adamw_step(p, g, {}, lr, wd=wd, eps=eps)
    for k in p:
        step = g[k] / (np.abs(g[k]) + eps) + (wd * before[k] if k.startswith("W") else 0.0)
        assert np.allclose(p[k], before[k] - lr * step, rtol=0, atol=1e-15)


@pytest.mark.parametrize("chi", [2e-3, 0.3, 7.0, 80.0])
def test_target_reduces_to_one_branch_at_full_projection(chi):
    for s, sigma in ((1.0, 1), (-1.0, -1)):
        for r in (1e-7, 0.05, 0.5, 0.95, 1 - 1e-6):
            ln_up = O.mlp_target(chi, r, s)[0]
            c = O.cdf_t(False, chi, sigma, math.exp(ln_up / 3.0))  # the single branch's CDF
            assert abs(c - r) < 1e-10, (chi, s, r, c)


def test_target_monotone_in_r_and_stokes_closed_form():
    sp = pytest.importorskip("scipy.special")
    integrate = pytest.importorskip("scipy.integrate")
    chi = 1.5
    rs = np.linspace(0.01, 0.99, 25)
    ln_up = np.array([O.mlp_target(chi, r, 0.3)[0] for r in rs])
    assert np.all(np.diff(ln_up) > 0)
    for r in (0.1, 0.6):
        t = O.mlp_target(chi, r, 0.0)
        assert t[1] == 0.0 and t[2] == 0.0
        up = math.exp(t[0])
        lam = 3 * chi * up / (2 + 3 * chi * up)
        k13, k23 = sp.kv(1 / 3, up), sp.kv(2 / 3, up)
        ik13 = integrate.quad(lambda x: sp.kv(1 / 3, x), up, np.inf, epsabs=0, epsrel=1e-13, limit=200)[0]
        kappa = 1 / (1 - lam) + (1 - lam)
        assert abs(t[3] - k23 / (-ik13 + kappa * k23)) < 1e-9


def test_baseline_is_close_and_exact_at_full_projection():
    tb = O.tables(1e-4, 1e3, 64, 128)
    rng = np.random.default_rng(5)
    for _ in range(60):
        chi = math.exp(rng.uniform(M.LNCHI_LO, M.LNCHI_HI))
        r = 1 / (1 + math.exp(-rng.uniform(-10, 10)))
        s = rng.uniform(-1, 1)
        lb, a = M.baseline(tb, chi, r, s)
        assert 0.0 < a < 1.0
        assert abs(O.mlp_target(chi, r, s)[0] - lb) < 0.05
    # s = +1: the baseline is the up-branch table quantile, whose exact CDF is r within the interpolation
    # error of this coarse table (64 chi rows, linear in ln chi between them)
    for chi in (0.01, 1.0, 30.0):
        lb, a = M.baseline(tb, chi, 0.3, 1.0)
        assert a == 1.0
        assert abs(O.cdf_t(False, chi, 1, math.exp(lb / 3.0)) - 0.3) < 1e-4


def test_features_and_decode_round_trip():
    tb = O.tables(1e-4, 1e3, 64, 128)
    chi, r, s = 0.7, 0.42, -0.25
    X = M.features([chi], [r], [s])
    assert np.allclose(X[0], [(math.log(chi) - M.LNCHI_MID) / M.LNCHI_HALF, math.log(r / (1 - r)) / 10, s])
    t = M.targets(tb, chi, r, s)
    d = M.decode(tb, chi, r, s, t)
    ex = O.mlp_target(chi, r, s)
    assert np.allclose(d, ex, rtol=0, atol=1e-12)
