"""Spectra versus polarization (the diagnostics of Sec. 8.6.3 and 8.6.4), computed on the device from an
FP32 particle buffer's own planes: the mean of a polarization component of the particles in each energy
bin.  Photons: the circular degree xi2 = P.k_hat against |k|; leptons: the longitudinal polarization
s.p_hat against gamma (energies in m c^2)."""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


def polarization_vs_energy(buf, edges) -> dict:
    """{"edges", "count", "mean"} for the buffer's particles [0, count): count and mean polarization
    component per energy bin [edges[i], edges[i+1]) (weights: the particles' macro-weights)."""
    n = buf.count()
    e_t = torch.as_tensor(np.asarray(edges, dtype=np.float64), device=buf.q.device)
    nb = len(edges) - 1
    if n == 0:
        return {"edges": list(map(float, edges)), "count": [0.0] * nb, "mean": [None] * nb}
    q = buf.q[:, :n].double()
    if buf.charge == B.QED_PHOTON:
        k = q[2, :, 0:3]
        P = torch.stack([q[0, :, 3], q[1, :, 0], q[1, :, 1]], 1)
        w = q[2, :, 3]
        en = torch.linalg.norm(k, dim=1)
        comp = (P * k).sum(1) / en.clamp_min(1e-300)
    else:
        p = torch.stack([q[0, :, 3], q[1, :, 0], q[1, :, 1]], 1)
        s = torch.stack([q[1, :, 2], q[1, :, 3], q[2, :, 0]], 1)
        w = q[2, :, 1]
        pn = torch.linalg.norm(p, dim=1)
        en = torch.sqrt(1.0 + pn * pn)
        comp = (s * p).sum(1) / pn.clamp_min(1e-300)
    idx = torch.bucketize(en, e_t, right=True) - 1
    ok = (idx >= 0) & (idx < nb)
    cnt = torch.zeros(nb, dtype=torch.float64, device=buf.q.device).index_add_(0, idx[ok], w[ok])
    sm = torch.zeros(nb, dtype=torch.float64, device=buf.q.device).index_add_(0, idx[ok], (w * comp)[ok])
    cnt, sm = cnt.cpu().numpy(), sm.cpu().numpy()
    return {"edges": [float(x) for x in edges], "count": cnt.tolist(),
            "mean": [float(a / c) if c > 0 else None for a, c in zip(sm, cnt)]}
