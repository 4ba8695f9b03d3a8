"""Adaptive density control (paper App. F, Algorithm 2) in FP64 numpy --
TEST INFRASTRUCTURE ONLY (imported by tests/ alone; shares no code with the
CUDA path).

Readings taken where the algorithm is silent or ambiguous:
  * avg_grad of a Gaussian = the accumulated Euclidean norm of dL/dmu (world
    units) over the iterations since the last densification, divided by their
    number;
  * sigma of an anisotropic Gaussian = its largest axis scale (world units);
    theta = 0.005 x the grid's body diagonal; the pruning bound is 3 x size x h
    (size = box size in voxels, 17 by default);
  * top_k picks the largest avg_grad first, equal values by lower index;
  * the decisions (thresholds, order) are taken on FP32 values, as the
    kernel takes them;
  * clones and split children are new: pruning applies to the Gaussians that
    existed before this densification (a clone has zero gradient by
    construction and would otherwise be removed at once); a split original is
    replaced by its two children;
  * a child is mu + R(q) diag(s) z with z a standard normal 3-vector (the
    Gaussian's own density), scales s / 2^(1/3), the same rotation and
    intensity; the normals are inputs, two per Gaussian;
  * output order: surviving originals (index order), then clones (index order
    of their originals), then children (two per split original, index order);
  * optimiser state: survivors keep theta, m, v (a cloned original's intensity
    is halved, its theta entry recomputed); new entries start with m = v = 0.
"""
import numpy as np


def rotation(q):
    """R(q) of normalised quaternions (w, x, y, z): [n, 3, 3]."""
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], 1)


def top_k(avg, mask, k):
    """Boolean mask of the k entries of `mask` with the largest avg (ties by
    lower index)."""
    idx = np.flatnonzero(mask)
    order = idx[np.lexsort((idx, -avg[idx]))]
    sel = np.zeros(mask.shape, bool)
    sel[order[:k]] = True
    return sel


def densify(grid, mu, s, q, rho, grad_accum, iters, normals, tau=2e-4, n_max=500_000, size=17,
            theta_frac=0.005):
    """One application of Algorithm 2.  Returns (mu, s, q, rho, kind, src):
    kind 0 survivor, 1 clone, 2 child; src the original's index."""
    mu = np.asarray(mu, np.float64); s = np.asarray(s, np.float64)
    q = np.asarray(q, np.float64); rho = np.asarray(rho, np.float64)
    n = mu.shape[0]
    h = grid.h
    # the decisions are integer outcomes of FP32 comparisons: taken in FP32,
    # as the kernel takes them (avg = acc / iters rounded to FP32, thresholds
    # rounded to FP32)
    f32 = np.float32
    diag = float(np.sqrt(sum((float(d) * d) for d in grid.dims))) * h
    theta = f32(float(f32(theta_frac)) * diag)
    tau = f32(tau)
    avg = (np.asarray(grad_accum, f32) / f32(iters)).astype(f32)
    sig = np.asarray(s, f32).max(axis=1)
    prune_sig = f32(f32(3.0) * f32(size) * f32(h))
    # clone: under-reconstructed, small
    cand = (avg >= tau) & (sig <= theta)
    n_clone = min(max(n_max - n, 0), int(cand.sum()))
    clone = top_k(avg, cand, n_clone)
    rho_c = np.where(clone, rho / 2, rho)
    n1 = n + n_clone
    # split: under-reconstructed, large
    cand = (avg >= tau) & (sig > theta)
    n_split = min(max(n_max - n1, 0), int(cand.sum()))
    split = top_k(avg, cand, n_split)
    # prune among the originals that stay
    prune = ((avg <= tau) | (sig > prune_sig)) & ~split
    keep = ~split & ~prune
    out_mu = [mu[keep]]; out_s = [s[keep]]; out_q = [q[keep]]; out_rho = [rho_c[keep]]
    kind = [np.zeros(int(keep.sum()), int)]; src = [np.flatnonzero(keep)]
    ci = np.flatnonzero(clone)
    out_mu.append(mu[ci]); out_s.append(s[ci]); out_q.append(q[ci]); out_rho.append(rho_c[ci])
    kind.append(np.ones(ci.size, int)); src.append(ci)
    si = np.flatnonzero(split)
    R = rotation(q[si])
    z = np.asarray(normals, np.float64)[si]  # [k, 2, 3]
    ch_mu = mu[si][:, None, :] + np.einsum("kab,kcb->kca", R, s[si][:, None, :] * z)
    out_mu.append(ch_mu.reshape(-1, 3))
    out_s.append(np.repeat(s[si] / 2 ** (1 / 3), 2, axis=0))
    out_q.append(np.repeat(q[si], 2, axis=0))
    out_rho.append(np.repeat(rho[si], 2))
    kind.append(np.full(2 * si.size, 2)); src.append(np.repeat(si, 2))
    return (np.concatenate(out_mu), np.concatenate(out_s), np.concatenate(out_q),
            np.concatenate(out_rho), np.concatenate(kind), np.concatenate(src))
