"""The learned sampler through the C ABI (qed_mlp_*): parameter layout, initial weights, training and
sampling.  Argument marshalling only; every step runs in libqedgb's kernels (see qed_mlp.cu)."""
from __future__ import annotations

import math

import numpy as np
import torch

from . import binding as B

LAYERS = (3, 64, 64, 64, 4)
# (name, shape) in the order of the flat FP32 parameter array
LAYOUT = (("W1", (64, 3)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (64, 64)), ("b3", (64,)),
          ("W4", (4, 64)), ("b4", (4,)))


def unflatten(flat) -> dict:
    out, o = {}, 0
    for name, shape in LAYOUT:
        n = int(np.prod(shape))
        out[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    assert o == B.QED_MLP_PARAMS
    return out


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float32).reshape(-1) for name, _ in LAYOUT])


def init_params(seed: int = 0) -> np.ndarray:
    """Initial weights uniform in +-0.5 sqrt(6 / (fan_in + fan_out)), zero biases (flat FP32)."""
    rng = np.random.default_rng(seed)
    p = {}
    for l in range(4):
        fi, fo = LAYERS[l], LAYERS[l + 1]
        lim = 0.5 * math.sqrt(6.0 / (fi + fo))
        p[f"W{l + 1}"] = rng.uniform(-lim, lim, (fo, fi))
        p[f"b{l + 1}"] = np.zeros(fo)
    return flatten(p)


class Sampler:
    """A network handle (parameters, optimiser state, training scratch for batches up to max_batch)."""

    def __init__(self, params=None, max_batch: int = 4096, device="cuda"):
        self.device = torch.device(device)
        self.max_batch = int(max_batch)
        self.handle = B.qed_mlp_create(self.max_batch, init_params() if params is None else params)

    def params(self) -> np.ndarray:
        return B.qed_mlp_get_params(self.handle)

    def set_params(self, flat):
        B.qed_mlp_set_params(self.handle, flat)

    def train(self, tables, steps: int, batch: int = 4096, seed: int = 7, first_index: int = 0, lr: float = 2e-3,
              lr_final: float = 2e-5, weight_decay: float = 1e-5, stream: int = 0) -> np.ndarray:
        """Train on steps x batch fresh table samples; returns the per-step losses."""
        loss = torch.zeros(max(1, steps), dtype=torch.float32, device=self.device)
        B.qed_mlp_train(self.handle, tables.handle, steps, batch, seed, first_index, lr, lr_final, weight_decay,
                        loss.data_ptr(), stream)
        return loss[:steps].cpu().numpy()

    def forward(self, x: torch.Tensor, stream: int = 0) -> torch.Tensor:
        x = x.to(device=self.device, dtype=torch.float32).contiguous()
        out = torch.empty((x.shape[0], 4), dtype=torch.float32, device=self.device)
        B.qed_mlp_forward(self.handle, x.data_ptr(), x.shape[0], out.data_ptr(), stream)
        return out

    def grad(self, x: torch.Tensor, y: torch.Tensor, stream: int = 0):
        g = torch.empty(B.QED_MLP_PARAMS, dtype=torch.float32, device=self.device)
        loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        B.qed_mlp_grad(self.handle, x.data_ptr(), y.data_ptr(), x.shape[0], g.data_ptr(), loss.data_ptr(), stream)
        return g, loss

    def adamw(self, g: torch.Tensor, lr: float, weight_decay: float, stream: int = 0):
        B.qed_mlp_adamw(self.handle, g.data_ptr(), lr, weight_decay, stream)

    def sample(self, tables, chi, r, s, tol: float = 1e-4, table_only: bool = False, stream: int = 0,
               with_error: bool = False, branch_table: bool = False):
        """(out4 = (ln u', xi1, xi2, xi3), fell_back mask, number of fallbacks[, network CDF errors]) for
        device double arrays chi, r, s.  table_only: the checked sampler's own fallback (the mixture
        quantile from the tables) for every sample; branch_table: the step's sampler (branch, then one ICDF
        row) instead of the network."""
        n = chi.shape[0]
        out = torch.empty((n, 4), dtype=torch.float32, device=self.device)
        fell = torch.zeros(n, dtype=torch.uint8, device=self.device)
        nf = torch.zeros(1, dtype=torch.int64, device=self.device)
        err = torch.empty(n, dtype=torch.float32, device=self.device) if with_error else None
        B.qed_mlp_sample(self.handle, tables.handle, chi.data_ptr(), r.data_ptr(), s.data_ptr(), n, tol,
                         (B.QED_MLP_ALWAYS_TABLE if table_only else 0) | (B.QED_MLP_BRANCH_TABLE if branch_table else 0),
                         out.data_ptr(), fell.data_ptr(), nf.data_ptr(),
                         stream, err.data_ptr() if with_error else 0)
        return (out, fell, nf, err) if with_error else (out, fell, nf)

    def close(self):
        if getattr(self, "handle", None):
            B.qed_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def targets(tables, n: int, seed: int, first_index: int = 0, device="cuda"):
    """(features n x 3, scaled targets n x 4, raw (chi, r, s) n x 3) drawn and computed on the device."""
    x = torch.empty((n, 3), dtype=torch.float32, device=device)
    y = torch.empty((n, 4), dtype=torch.float32, device=device)
    raw = torch.empty((n, 3), dtype=torch.float64, device=device)
    B.qed_mlp_targets(tables.handle, n, seed, first_index, x.data_ptr(), y.data_ptr(), raw.data_ptr())
    return x, y, raw
