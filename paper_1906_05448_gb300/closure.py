"""Learned near-surface gradient closure for IBM (training data, training,
evaluation), driving the C ABI.

The paper finds that IBM underestimates the local dissipation inside its
diffused interface near particle surfaces, where IBB (sharp interface) does
not (Sec. 3.2, Sec. 4). The closure learns, from pairs that the method
itself produces, the IBB velocity gradients at near-surface nodes from the
IBM velocity stencil there:
  - the same seeded initial state is run with IBB and with IBM-B;
  - after `steps` steps, the IBM run's near-surface nodes give the features
    (lbm_closure_samples) and the IBB run the target gradients at the same
    cells (lbm_closure_targets); nodes solid in the IBB run are dropped.
Everything numerical runs in the CUDA library; this module only sequences
calls and shuffles samples (seeded numpy).
"""
from __future__ import annotations

import numpy as np

import workloads

from . import lbm


def hit_pair(n, n_particles, seed, radius=4.0, tau=0.51, density_ratio=5.0, k_peak=8.0, u_rms=0.03,
             storage=lbm.F32):
    """IBB and IBM-B contexts of the same seeded particle-laden box."""
    u = workloads.hit_velocity(n, seed=seed, k_peak=k_peak, u_rms=u_rms)
    X = workloads.place_spheres((n, n, n), n_particles, radius, 1.0, seed=seed)
    out = []
    for bc in (lbm.BC_IBB, lbm.BC_IBM_B):
        L = lbm.Lattice(n, n, n, tau, storage=storage, rates=lbm.RATES_DHUMIERES, max_particles=n_particles)
        L.init_velocity(u)
        L.add_spheres(X, radius, density_ratio=density_ratio)
        out.append((L, bc))
    return out


def paired_samples(n, n_particles, seeds, steps, u_scale, g_scale, radius=4.0, **kw):
    """(X, T) torch CUDA tensors of features and target gradients from the
    paired runs of every seed."""
    import torch
    Xs, Ts = [], []
    cap = 1500 * n_particles
    for seed in seeds:
        (ibb, bc_b), (ibm, bc_m) = hit_pair(n, n_particles, seed, radius=radius, **kw)
        ibb.step(steps, bc_b)
        ibm.step(steps, bc_m)
        X, cells = ibm.closure_samples(u_scale, cap)
        order = torch.argsort(cells)  # fixed row order
        X, cells = X[order], cells[order]
        T = ibb.closure_targets(cells, g_scale)
        ok = torch.isfinite(T).all(dim=1)
        Xs.append(X[ok])
        Ts.append(T[ok])
        ibb.close()
        ibm.close()
    return torch.cat(Xs), torch.cat(Ts)


def shuffle(X, T, seed, limit=None):
    import torch
    perm = np.random.default_rng(seed).permutation(X.shape[0])
    if limit is not None:
        perm = perm[:limit]
    idx = torch.as_tensor(perm, device=X.device)
    return X[idx].contiguous(), T[idx].contiguous()


def init_weights(seed):
    """He-normal weights, zero biases, seeded (layout of the C ABI)."""
    rng = np.random.default_rng(seed)
    sizes = [85, 64, 64, 64, 9]
    parts = []
    for i in range(4):
        a, b = sizes[i], sizes[i + 1]
        parts.append(rng.standard_normal(a * b) * np.sqrt(2.0 / a))
        parts.append(np.zeros(b))
    return np.concatenate(parts).astype(np.float32)


def near_surface_error(bins_model, bins_ref, radius, width=2.0):
    """Relative L1 error of the dissipation profile over the bins within
    `width` lattice units of the surface (r/r_p in (1, 1 + width/R])."""
    r = np.asarray(bins_ref["bin_r"])
    sel = (r > 1.0) & (r <= 1.0 + width / radius) & (np.asarray(bins_ref["bin_count"]) > 0)
    a = np.asarray(bins_model["bin_eps"])[sel] * bins_model["dissipation_fluid"]
    b = np.asarray(bins_ref["bin_eps"])[sel] * bins_ref["dissipation_fluid"]
    return float(np.sum(np.abs(a - b)) / np.sum(np.abs(b)))


def evaluate(n, n_particles, seeds, steps, weights, u_scale, g_scale, radius=4.0, **kw):
    """Near-surface dissipation-profile error against IBB, for plain IBM-B
    and for IBM-B with the closure, averaged over the seeds."""
    e_plain, e_closure = [], []
    for seed in seeds:
        (ibb, bc_b), (ibm, bc_m) = hit_pair(n, n_particles, seed, radius=radius, **kw)
        ibb.step(steps, bc_b)
        ibm.step(steps, bc_m)
        ref = ibb.stats(lbm.STATS_BINS)
        plain = ibm.stats(lbm.STATS_BINS)
        ibm.closure_set_weights(weights, u_scale, g_scale)
        learned = ibm.stats(lbm.STATS_BINS | lbm.STATS_CLOSURE)
        e_plain.append(near_surface_error(plain, ref, radius))
        e_closure.append(near_surface_error(learned, ref, radius))
        ibb.close()
        ibm.close()
    return float(np.mean(e_plain)), float(np.mean(e_closure))
