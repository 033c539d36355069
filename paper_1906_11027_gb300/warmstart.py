"""Training data and training of the warm-start network.

Steady droplets from the batched sweep become samples (G, tau, order, R_s, d) -> rho
for every cell within |d| <= 24 of the interface (the interface and the bulk
plateaus on both sides, whose densities set the mass balance of a start), where R_s is the steady
droplet's equimolar radius (the radius of a sharp droplet of the same excess
mass, R_s^2 pi = sum (rho - rho_g) / (rho_l - rho_g)) and d = r - R_s.  The same
radius is what lbm_init_droplet_learned bisects on, so training and inference
measure the distance from the same interface.  Whole domains (so whole (G, R)
pairs) are held out for validation.
"""
from __future__ import annotations

import numpy as np

from . import lbm

DMAX = 24.0
MAX_G = -4.65       # the library keeps the tanh start above this coupling
MIN_CONTRAST = 0.2  # rho_l - rho_g of a steady droplet (a dissolved one is not a sample)


def steady_samples(rho, G, tau, order, max_per_domain=4096, rng=None):
    """Samples of one steady 2-D droplet field rho [ny, nx] (centred on (nx/2, ny/2))."""
    ny, nx = rho.shape
    rl = float(rho[ny // 2, nx // 2])
    rg = float(rho[0, 0])
    if not (np.isfinite(rl) and np.isfinite(rg)) or rl - rg < MIN_CONTRAST:
        return None
    Rs = float(np.sqrt(max((rho - rg).sum() / (rl - rg), 0.0) / np.pi))
    yy, xx = np.meshgrid(np.arange(ny) - ny // 2, np.arange(nx) - nx // 2, indexing="ij")
    yy = np.where(yy > ny / 2, yy - ny, np.where(yy < -ny / 2, yy + ny, yy))
    xx = np.where(xx > nx / 2, xx - nx, np.where(xx < -nx / 2, xx + nx, xx))
    d = np.sqrt(xx * xx + yy * yy) - Rs
    sel = np.abs(d) <= DMAX
    dd, rr = d[sel], rho[sel]
    if rng is not None and len(dd) > max_per_domain:
        k = rng.choice(len(dd), size=max_per_domain, replace=False)
        dd, rr = dd[k], rr[k]
    raw = np.stack([np.full_like(dd, G), np.full_like(dd, tau), np.full_like(dd, float(order)),
                    np.full_like(dd, Rs), dd], axis=1)
    return raw, rr.astype(np.float32), Rs


def dataset_from_batch(batch, domains, obs, seed=11027, holdout=0.1, max_per_domain=4096):
    """(X_train, y_train, X_val, y_val, held-out domain indices) from a converged batch."""
    rng = np.random.default_rng(seed)
    good = [i for i, o in enumerate(obs) if np.isfinite(o["max_u"]) and domains[i]["G"] <= MAX_G]
    held = set(rng.choice(good, size=max(1, int(round(holdout * len(good)))), replace=False).tolist())
    parts = {True: ([], []), False: ([], [])}
    for i in good:
        d = domains[i]
        f = batch.get_f(i)
        rho = f.sum(axis=0)[0]
        s = steady_samples(rho, d["G"], d["tau"], d["stencil"], max_per_domain, rng)
        if s is None:
            continue
        raw, y, _ = s
        parts[i in held][0].append(raw)
        parts[i in held][1].append(y)
    def cat(key):
        if not parts[key][0]:
            return np.zeros((0, 5), np.float32), np.zeros(0, np.float32)
        return lbm.MLP.features(np.concatenate(parts[key][0])), np.concatenate(parts[key][1])
    Xt, yt = cat(False)
    Xv, yv = cat(True)
    return Xt, yt, Xv, yv, sorted(held)


def train(Xt, yt, epochs=40, lr=2e-3, batch=4096, seed=1906):
    """Train a fresh network; returns (mlp, final training loss)."""
    net = lbm.MLP(seed=seed)
    loss = net.train(Xt, yt, epochs=max(1, epochs // 2), lr=lr, batch=batch)
    loss = net.train(Xt, yt, epochs=max(1, epochs - epochs // 2), lr=lr / 4, batch=batch)
    return net, loss


def batch_warm_init(batch, domains, net):
    """Replace the tanh start of every batch domain by the learned warm start (mass
    matched to the tanh start; the tanh start stays where the library falls back).
    Returns the number of domains that kept the tanh start."""
    fallbacks = 0
    for i, d in enumerate(domains):
        # the caching allocator keeps the per-domain set-up free of cudaMalloc/cudaFree
        dom = lbm.Domain(d["nx"], d["ny"], G=d["G"], tau=d["tau"], stencil=d["stencil"], precision=lbm.LBM_FP64,
                         torch_alloc=True)
        fb, _ = dom.init_droplet_learned(net, d["R"], d["rho_l"], d["rho_g"], d["width"])
        if fb:
            fallbacks += 1
        else:
            batch.set_f(i, dom.get_f())
        dom.close()
    return fallbacks
