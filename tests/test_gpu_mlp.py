"""The learned sampler on the GPU (qed_mlp_*) against the FP64 oracle (oracle/mlp.py, orc_mlp_target).

* Training samples: the inputs are the oracle's own Philox draws for the same (index, seed); the
  table-based target quantile satisfies the exact mixture CDF to the tables' accuracy.
* Forward pass (tensor cores, BF16 weights and activations, FP32 accumulation) against the oracle's
  forward with the same roundings in FP64: the two differ by accumulation order, except for the rare
  activation that sits on a BF16 rounding boundary and rounds the other way (bar: median 1e-6, 99 % 1e-4,
  all 5e-2 of the output scale).
* Gradients (backward on tensor cores with BF16-rounded operands) against the oracle's exact backward:
  1e-2 relative in the norm of every parameter block; the loss 1e-5.
* AdamW: one step against the oracle's.
* Trained network: the loss falls; every sample the sampler returns from the network satisfies the
  exact CDF check and the Stokes closed form within the bound; every fallback sample is the table
  quantile; the network path is faster than the table path (the gain).
"""
import math
import time

import numpy as np
import pytest
import torch

import oracle as O
from oracle import mlp as OM
from paper_2511_08929_gb300 import binding as B
from paper_2511_08929_gb300 import buffers as Q
from paper_2511_08929_gb300 import mlp as GM

pytestmark = pytest.mark.gpu

# the production grid: its quantiles are within 1.4e-5 of the exact CDF (measured with the oracle over
# random chi and r on both spin branches; median 3e-8): linear interpolation in ln chi between rows
DESC = dict(chi_min=1e-4, chi_max=1e3, n_chi=256, n_r=256, y_lo=-20.0, y_hi=20.0)
TABLE_ERR = 4e-5
STEP = 0xFFFFFFFFFFFFFFFE


@pytest.fixture(scope="module")
def gpu_tables():
    from paper_2511_08929_gb300 import build as bld
    bld.build()
    t = Q.Tables(**DESC)
    yield t
    t.close()


@pytest.fixture(scope="module")
def ora_tables():
    return O.tables(*DESC.values())


def _oracle_params(flat):
    return GM.unflatten(np.asarray(flat, dtype=np.float32).astype(np.float64))


def test_targets_match_oracle(gpu_tables, ora_tables):
    n, seed, first = 300, 11, 1000
    x, y, raw = GM.targets(gpu_tables, n, seed, first)
    x, y, raw = x.cpu().numpy(), y.cpu().numpy(), raw.cpu().numpy()
    for i in range(n):
        u0, u1 = O.uniform_pair(first + i, seed, STEP, 0)
        u2, _ = O.uniform_pair(first + i, seed, STEP, 1)
        chi = math.exp(OM.LNCHI_LO + u0 * (OM.LNCHI_HI - OM.LNCHI_LO))
        assert raw[i, 0] == pytest.approx(chi, rel=1e-14) and raw[i, 1] == u1 and raw[i, 2] == 2 * u2 - 1
    X = OM.features(raw[:, 0], raw[:, 1], raw[:, 2])
    assert np.max(np.abs(x - X)) < 2e-7
    worst_cdf, worst_xi = 0.0, 0.0
    for i in range(0, n, 3):
        chi, r, s = raw[i]
        lb, _ = OM.baseline(ora_tables, chi, r, s)
        L = lb + y[i, 0] / OM.OUT_SCALE
        worst_cdf = max(worst_cdf, abs(O.mlp_cdf(chi, s, L) - r))
        ex = O.mlp_target(chi, r, s)
        xi3 = OM.xi3_closed(chi, lb, s) + y[i, 3] / OM.OUT_SCALE
        worst_xi = max(worst_xi, abs(xi3 - ex[3]))
        assert y[i, 1] == 0.0 and y[i, 2] == 0.0
    assert worst_cdf < TABLE_ERR, worst_cdf  # the tables' interpolation error of the quantile
    assert worst_xi < 5e-5, worst_xi


def test_forward_matches_oracle(gpu_tables):
    rng = np.random.default_rng(3)
    flat = GM.init_params(5) + rng.normal(scale=0.05, size=B.QED_MLP_PARAMS).astype(np.float32)
    smp = GM.Sampler(flat, max_batch=1024)
    X = rng.uniform(-1.2, 1.2, size=(3001, 3)).astype(np.float32)
    o = smp.forward(torch.from_numpy(X)).cpu().numpy()
    ref, _ = OM.forward(_oracle_params(smp.params()), X.astype(np.float64))
    err = np.abs(o - ref) / (1.0 + np.abs(ref))
    assert np.median(err) < 1e-6 and np.quantile(err, 0.99) < 1e-4 and err.max() < 5e-2, \
        (np.median(err), np.quantile(err, 0.99), err.max())
    smp.close()


def test_gradients_match_oracle(gpu_tables):
    flat = GM.init_params(6)
    smp = GM.Sampler(flat, max_batch=2048)
    x, y, _ = GM.targets(gpu_tables, 2048, 5, 0)
    g, loss = smp.grad(x, y)
    torch.cuda.synchronize()
    L, gr = OM.loss_and_grads(_oracle_params(smp.params()), x.cpu().numpy().astype(np.float64),
                              y.cpu().numpy().astype(np.float64))
    assert float(loss.item()) == pytest.approx(L, rel=1e-5)
    gg = GM.unflatten(g.cpu().numpy())
    for k in gr:
        rel = np.linalg.norm(gg[k] - gr[k]) / max(np.linalg.norm(gr[k]), 1e-30)
        assert rel < 1e-2, (k, rel)
    smp.close()


def test_adamw_matches_oracle(gpu_tables):
    flat = GM.init_params(7)
    smp = GM.Sampler(flat, max_batch=64)
    rng = np.random.default_rng(8)
    p = _oracle_params(smp.params())
    state = {}
    for step in range(3):
        gflat = rng.normal(size=B.QED_MLP_PARAMS).astype(np.float32)
        smp.adamw(torch.from_numpy(gflat).cuda(), 1e-3, 1e-2)
        OM.adamw_step(p, GM.unflatten(gflat), state, 1e-3, wd=1e-2)
    got = GM.unflatten(smp.params())
    for k in p:
        assert np.max(np.abs(got[k] - p[k])) < 2e-6, k
    smp.close()


@pytest.fixture(scope="module")
def trained(gpu_tables):
    """A network trained on 1200 x 4096 table samples (a shortened run of the full 5e7-sample training)."""
    smp = GM.Sampler(GM.init_params(1), max_batch=4096)
    losses = smp.train(gpu_tables, steps=1200, batch=4096, seed=21, lr=3e-3, lr_final=3e-5)
    yield smp, losses
    smp.close()


def _query(n, seed):
    rng = np.random.default_rng(seed)
    chi = np.exp(rng.uniform(OM.LNCHI_LO, OM.LNCHI_HI, n))
    r = rng.uniform(0, 1, n)
    s = rng.uniform(-1, 1, n)
    return [torch.from_numpy(a).cuda() for a in (chi, r, s)]


def test_training_reduces_loss(trained):
    _, losses = trained
    assert np.all(np.isfinite(losses))
    assert np.mean(losses[-50:]) < 0.05 * np.mean(losses[:10]), (losses[:10].mean(), losses[-50:].mean())


def test_sampler_output_meets_bound_or_falls_back(gpu_tables, ora_tables, trained):
    smp, _ = trained
    chi, r, s = _query(4096, 31)
    tol = 1e-4
    out, fell, nf = smp.sample(gpu_tables, chi, r, s, tol=tol)
    torch.cuda.synchronize()
    out, fell = out.cpu().numpy().astype(np.float64), fell.cpu().numpy()
    assert int(nf.item()) == int(fell.sum())
    chi, r, s = chi.cpu().numpy(), r.cpu().numpy(), s.cpu().numpy()
    frac = fell.mean()
    print(f"fallback fraction {frac:.4f}")
    assert frac < 0.5
    rng = np.random.default_rng(2)
    # the check and the fallback use the tables' mixture CDF: allow their interpolation error and the
    # float rounding of the returned ln u' on top of the bound
    for i in rng.choice(len(r), 160, replace=False):
        c = O.mlp_cdf(chi[i], s[i], out[i, 0])
        slack = TABLE_ERR + 1e-6 * abs(out[i, 0])
        if fell[i]:
            assert abs(c - r[i]) < slack, (i, c, r[i])
        else:
            assert abs(c - r[i]) < tol + slack, (i, c, r[i])
            assert abs(out[i, 3] - OM.xi3_closed(chi[i], out[i, 0], s[i])) < tol + 1e-6
        assert out[i, 1] == pytest.approx(0.0, abs=tol) and out[i, 2] == pytest.approx(0.0, abs=tol)


def test_network_gains_over_the_table_path(gpu_tables, trained):
    """What the network buys: the exact continuous-spin quantile without the root finding the two-branch
    tables need for it (the table path bisects the mixture CDF, each step inverting both branch rows)."""
    smp, _ = trained
    chi, r, s = _query(1 << 22, 41)

    def timed(table_only):
        smp.sample(gpu_tables, chi, r, s, table_only=table_only)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, nf = smp.sample(gpu_tables, chi, r, s, table_only=table_only)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, int(nf.item())

    t_net, nf = timed(False)
    t_tab, _ = timed(True)
    print(f"network {chi.shape[0] / t_net:.3e} samples/s ({nf} fallbacks), table path {chi.shape[0] / t_tab:.3e}")
    assert t_net < t_tab


@pytest.mark.parametrize("chi,s", [(0.01, 0.7), (1.0, -0.5), (30.0, 0.0)])
def test_branch_table_sampler_follows_the_mixture(gpu_tables, trained, chi, s):
    """The step's own sampler (spin branch, then one ICDF row), exposed for comparison: its ln u' for
    uniform r is distributed as the mixture w(lambda; s) (reading C4): the exact mixture CDF of the
    oracle at the samples is uniform (KS), and xi3 there matches its closed form."""
    st = pytest.importorskip("scipy.stats")
    smp, _ = trained
    n = 20000
    g = torch.Generator(device="cuda")
    g.manual_seed(7)
    r = torch.rand(n, dtype=torch.float64, device="cuda", generator=g) * (1 - 2.0 ** -40) + 2.0 ** -41
    cd = torch.full((n,), chi, dtype=torch.float64, device="cuda")
    sd = torch.full((n,), s, dtype=torch.float64, device="cuda")
    out, _, _ = smp.sample(gpu_tables, cd, r, sd, branch_table=True)
    torch.cuda.synchronize()
    out = out.cpu().numpy().astype(np.float64)
    c = np.array([O.mlp_cdf(chi, s, L) for L in out[:, 0]])
    assert st.kstest(c, "uniform").pvalue > 1e-3
    for i in range(0, n, 997):
        assert abs(out[i, 3] - OM.xi3_closed(chi, out[i, 0], s)) < 1e-5


def test_network_against_the_step_sampler(gpu_tables, trained):
    """The honest comparison: per sample, the step's sampler (branch + one float-float ICDF row, 2-D
    tables) is faster than the network with its check, which needs those same tables; the network's gain
    is only over the exact continuous-spin quantile by bisection.  Both relations are asserted, so the
    figures quoted for them stay true."""
    smp, _ = trained
    chi, r, s = _query(1 << 22, 43)

    def timed(**kw):
        smp.sample(gpu_tables, chi, r, s, **kw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        smp.sample(gpu_tables, chi, r, s, **kw)
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    t_net, t_bis, t_br = timed(), timed(table_only=True), timed(branch_table=True)
    n = chi.shape[0]
    print(f"network {n / t_net:.3e}/s, bisection {n / t_bis:.3e}/s, step sampler {n / t_br:.3e}/s")
    assert t_net < t_bis and t_br < t_net
