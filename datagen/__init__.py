"""Seeded synthetic workloads (inputs only; none of the method's arithmetic).

The paper evaluates on seven real data sets (Audio, Deep, NUS, MNIST, GIST,
Cifar, Trevi) that are not available here.  These Gaussian mixtures stand in
for them at comparable n and d.  Both the CUDA path's tests and the oracle
draw their inputs from this module, and nothing else is shared between them.

Streams (numpy PCG64, identical on every platform):
    data points   default_rng(seed)      cluster centres, scales, members
    queries       default_rng(seed + 1)  same mixture, fresh members
    planted pairs default_rng(seed + 4)
The projection matrix, when drawn by the library, uses seed + 2; the r_min
pair sample uses seed + 3 (both inside the method, not here).
"""
import numpy as np

# name -> recipe.  sigma: per-cluster scale, a float or (lo, hi) for U[lo,hi].
WORKLOADS = {
    # plain c-ANN, FP32
    "c1": dict(n=10_000, d=128, clusters=50, sigma=1.0, nq=100, k=10, c=1.5),
    # batched c-ANN, the throughput workload
    "c2": dict(n=1_000_000, d=128, clusters=1000, sigma=(0.5, 2.0), nq=10_000,
               k=50, c=1.5),
    # high-dimensional, anisotropic covariance with eigenvalues i^-1
    "c3": dict(n=1_000_000, d=960, clusters=1000, sigma=1.0, aniso=True,
               nq=1000, k=10, c=1.5),
    # closest pairs with 20 planted near-duplicate pairs at distance 0.01
    "c4": dict(n=100_000, d=512, clusters=500, sigma=1.0, n_planted=20,
               planted_dist=0.01, k=10, c=1.5),
    # serving data set
    "c5": dict(n=2_000_000, d=256, clusters=2000, sigma=1.0, nq=4096, k=10,
               c=1.5),
}

CENTRE_SCALE = 10.0


def _mixture_params(rng, clusters, d, sigma):
    centres = rng.standard_normal((clusters, d), dtype=np.float64) * CENTRE_SCALE
    if isinstance(sigma, tuple):
        scales = rng.uniform(sigma[0], sigma[1], size=clusters)
    else:
        scales = np.full(clusters, float(sigma))
    return centres, scales


def _draw(rng, count, centres, scales, rot, chunk=1 << 16):
    clusters, d = centres.shape
    out = np.empty((count, d), dtype=np.float32)
    lab = rng.integers(0, clusters, size=count)
    if rot is not None:
        lam_sqrt = (1.0 / np.arange(1, d + 1, dtype=np.float64)) ** 0.5
    for s in range(0, count, chunk):
        e = min(count, s + chunk)
        z = rng.standard_normal((e - s, d), dtype=np.float64)
        if rot is not None:
            z = (z * lam_sqrt) @ rot.T
        out[s:e] = (centres[lab[s:e]] + scales[lab[s:e], None] * z).astype(np.float32)
    return out, lab


def mixture(n, d, clusters, sigma=1.0, seed=0, nq=0, aniso=False):
    """Gaussian mixture with uniform weights; centres ~ N(0, 10^2 I).

    aniso=True: x = mu_j + s_j * U (lambda^1/2 * z), lambda_i = i^-1, with one
    seeded global orthogonal U (QR of a Gaussian matrix).
    Returns (X [n,d] f32, Q [nq,d] f32, labels_X, labels_Q).
    """
    rng = np.random.default_rng(seed)
    centres, scales = _mixture_params(rng, clusters, d, sigma)
    rot = None
    if aniso:
        g = rng.standard_normal((d, d))
        qmat, rmat = np.linalg.qr(g)
        rot = qmat * np.sign(np.diag(rmat))[None, :]
    X, lx = _draw(rng, n, centres, scales, rot)
    Q = np.empty((0, d), dtype=np.float32)
    lq = np.empty(0, dtype=np.int64)
    if nq:
        Q, lq = _draw(np.random.default_rng(seed + 1), nq, centres, scales, rot)
    return X, Q, lx, lq


def plant_pairs(X, count, dist, seed=0):
    """Overwrite `count` points b with o_a + dist * u (u a random unit vector)
    for `count` other points a; all 2*count indices are distinct.
    Returns the planted (a, b) index pairs."""
    rng = np.random.default_rng(seed + 4)
    n, d = X.shape
    idx = rng.choice(n, size=2 * count, replace=False)
    a, b = idx[:count], idx[count:]
    u = rng.standard_normal((count, d))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    X[b] = (X[a].astype(np.float64) + dist * u).astype(np.float32)
    return np.stack([np.minimum(a, b), np.maximum(a, b)], axis=1)


def workload(name, seed=0, n=None, nq=None):
    """Materialise a named workload (optionally with smaller n / nq)."""
    w = dict(WORKLOADS[name])
    if n is not None:
        w["n"] = n
    if nq is not None:
        w["nq"] = nq
    X, Q, _, _ = mixture(w["n"], w["d"], w["clusters"], w.get("sigma", 1.0),
                         seed=seed, nq=w.get("nq", 0), aniso=w.get("aniso", False))
    planted = None
    if w.get("n_planted"):
        planted = plant_pairs(X, w["n_planted"], w["planted_dist"], seed=seed)
    return dict(X=X, Q=Q, planted=planted, **w)


def gaussian(n, d, seed=0, scale=1.0):
    """Plain i.i.d. N(0, scale^2) points (small unit tests)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((n, d)) * scale).astype(np.float32)
