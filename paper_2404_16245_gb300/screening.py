"""Learned screening of (shell pair, nucleus) triples on top of the plain method.

The network (include/shgo_mlp.h) predicts log10 max|Z_C <a|1/r_C|b>| for one shell pair and one
nucleus from 16 features.  Triples predicted below threshold / margin are left out of the nucleus
sum; the exact method computes the labels it is trained on and judges a sampled audit of what was
skipped.  Everything numeric runs in the library's kernels; this module only samples indices,
moves arrays and drives the training loop.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import shgo, workloads


def _prim_index(nprim, poff, shells):
    """Indices of the primitives of `shells` (concatenated in order)."""
    counts = nprim[shells]
    starts = poff[shells]
    rep = np.repeat(starts - np.concatenate([[0], np.cumsum(counts)[:-1]]), counts)
    return rep + np.arange(int(counts.sum()))


def plain_labels(basis: dict, shell_a, shell_b, centers, charges, triples, chunk: int = 200_000, device="cuda"):
    """log10 max|block| of each triple (pair index, nucleus index) by the plain method: every
    triple is its own molecule (the pair's shells and that one nucleus) in batched calls."""
    import torch
    l = np.asarray(basis["l"], dtype=np.int32)
    nprim = np.asarray(basis["nprim"], dtype=np.int32)
    poff = np.concatenate([[0], np.cumsum(nprim)[:-1]]).astype(np.int64)
    out_all = np.empty(len(triples))
    for s0 in range(0, len(triples), chunk):
        tr = triples[s0:s0 + chunk]
        a = shell_a[tr[:, 0]]
        b = shell_b[tr[:, 0]]
        same = a == b
        nsh = np.where(same, 1, 2).astype(np.int32)
        shells = np.empty(int(nsh.sum()), dtype=np.int64)
        first = np.concatenate([[0], np.cumsum(nsh)[:-1]])
        shells[first] = a
        shells[first[~same] + 1] = b[~same]
        pidx = _prim_index(nprim, poff, shells)
        C = np.asarray(centers)[tr[:, 1]]
        Z = np.asarray(charges)[tr[:, 1]]
        mols = {"nshells": nsh, "l": l[shells], "nprim": nprim[shells], "exps": basis["exps"][pidx],
                "coefs": basis["coefs"][pidx], "xyz": basis["xyz"][shells]}
        batch = shgo.Batch.from_arrays(mols, np.ones(len(tr), dtype=np.int64))
        V = shgo.nuclear_attraction_batched(batch, torch.tensor(C, device=device), torch.tensor(Z, device=device))
        torch.cuda.synchronize()
        Vh = V.cpu().numpy()
        la = l[a]
        na = 2 * la + 1
        for t in range(len(tr)):
            blk = batch.block(Vh, t)
            m = blk if same[t] else blk[:na[t], na[t]:]
            out_all[s0 + t] = math.log10(float(np.max(np.abs(m))) + 1e-300)
        batch.close()
    return np.maximum(out_all, -40.0)


def sample_triples(rng, npairs, ncenters, n, pair_dist=None, near_fraction=0.5, near_cut=8.0):
    """n (pair, nucleus) indices: a near_fraction of them on pairs whose centres are closer than
    near_cut bohr (where blocks straddle the threshold), the rest uniform."""
    n_near = int(n * near_fraction) if pair_dist is not None else 0
    near_pairs = np.nonzero(pair_dist < near_cut)[0] if pair_dist is not None else np.arange(npairs)
    p = np.concatenate([rng.integers(0, npairs, n - n_near),
                        near_pairs[rng.integers(0, len(near_pairs), n_near)] if n_near else np.zeros(0, np.int64)])
    c = rng.integers(0, ncenters, n)
    return np.stack([p, c], axis=1).astype(np.int32)


def train(X, T, *, epochs=20, batch=4096, lr=2e-3, under_weight=4.0, seed=0, log=None):
    """Network fitted on features X [n, 16] and labels T [n] (torch CUDA tensors) with the library's
    training kernels; returns (MLP, per-epoch losses)."""
    import torch
    Xh = X.cpu().numpy()
    mean = Xh.mean(axis=0)
    sd = np.maximum(Xh.std(axis=0), 1e-3)
    net = shgo.MLP(workloads.mlp_init_params(seed), mean, sd)
    n = X.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    steps = max(1, n // batch)
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(X.device)
        rate = lr * (0.5 * (1 + math.cos(math.pi * ep / epochs)))
        tot = 0.0
        for s in range(steps):
            idx = perm[s * batch:(s + 1) * batch]
            xb = X.index_select(0, idx).contiguous()
            tb = T.index_select(0, idx).contiguous()
            want = s == steps - 1
            l = net.train_step(xb, tb, under_weight, rate, want_loss=want)
            if want:
                tot = l
        losses.append(tot)
        if log:
            log(f"epoch {ep}: loss {tot:.4f} lr {rate:.2e}")
    return net, losses


def calibrate_margin(net, X, T, log10_cut: float, safety: float = 1.0) -> float:
    """Margin (log10 units) for the rule "skip when prediction < log10_cut - margin" such that no
    held-out triple whose label is at or above the cut would be skipped: the largest
    under-prediction among those triples, plus `safety`.  X [n, 16] and T [n] are held-out
    features and labels (torch CUDA tensors / numpy)."""
    y = net.forward(X).cpu().numpy().astype(np.float64)
    t = np.asarray(T, dtype=np.float64)
    pos = t >= log10_cut
    if not np.any(pos):
        return safety
    return float(max(0.0, np.max(log10_cut - y[pos])) + safety)


def audit(basis: dict, shell_a, shell_b, centers, charges, mask, pair_nuc, fraction, rng, threshold,
          max_audit: int = 200_000):
    """Exact check of a random `fraction` of the skipped triples (at most max_audit of them).  mask is the
    screening mask over all triples in pair order (pair q owns pair_nuc[q] consecutive entries, nuclei in
    order).  Skipped triples are drawn by rejection from uniform triple indices, so no list of all skipped
    triples is formed."""
    n_skip = int(mask.size - np.count_nonzero(mask))
    if n_skip == 0:
        return {"audited": 0, "false_skips": 0, "false_skip_rate": 0.0, "max_skipped_block": 0.0}
    k = min(max(1, int(round(fraction * n_skip))), max_audit, n_skip)
    if k == n_skip:
        pick = np.nonzero(mask == 0)[0]
    else:
        chosen = set()
        while len(chosen) < k:
            cand = rng.integers(0, mask.size, size=4 * (k - len(chosen)) * max(1, mask.size // n_skip))
            for t in cand[mask[cand] == 0]:
                chosen.add(int(t))
                if len(chosen) == k:
                    break
        pick = np.sort(np.fromiter(chosen, dtype=np.int64))
    starts = np.concatenate([[0], np.cumsum(pair_nuc)[:-1]])
    q = np.searchsorted(starts, pick, side="right") - 1
    c = pick - starts[q]
    tr = np.stack([q, c], axis=1).astype(np.int32)
    lab = plain_labels(basis, shell_a, shell_b, centers, charges, tr)
    false = int(np.sum(lab > math.log10(threshold)))
    return {"audited": int(len(tr)), "false_skips": false, "false_skip_rate": false / len(tr),
            "max_skipped_block": float(10 ** lab.max())}
