"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module draws data only; it holds none of the selection method's arithmetic.
All arrays come from ``numpy.random.default_rng(seed)`` (PCG64) and are
deterministic given the seed.  They stand in for the paper's synthetic data sets
(Sec. 4.1) and the workloads of the library's benchmarks:

* ``uniform``                          i.i.d. U[0,1)
* ``paper_distribution``               the nine distributions of Sec. 4.1
* ``heavy_mixture``                    N(0,1) / lognormal(0,2) / Student-t(1) / their mix,
                                       with 5% exact duplicates of one value and 10 +-inf
* ``segment_sizes``, ``segmented``     thousands of normal arrays of log-uniform sizes
* ``regression``, ``elemental_thetas`` contaminated linear model and p-subset candidates
* ``training_array``                   arrays of the families the bracket MLP learns from
* ``knn_problem``                      labelled Gaussian clusters and queries for kNN
"""
from __future__ import annotations

import numpy as np


def uniform(n, seed=0, dtype=np.float32):
    """i.i.d. U[0,1) drawn directly in ``dtype`` (float32 or float64)."""
    return np.random.default_rng(seed).random(int(n), dtype=np.dtype(dtype).type)


PAPER_DISTRIBUTIONS = ("uniform", "normal", "halfnormal", "beta25", "mix1", "mix2",
                       "mix3", "mix4", "mix5")


def paper_distribution(name, n, seed, dtype=np.float32):
    """One of the nine synthetic distributions of Sec. 4.1.

    The garbled "50% of elements of x_i +1" of mixtures 2 and 5 is read as
    floor(n/2)+1 elements from the first component.
    """
    rng = np.random.default_rng(seed)
    n = int(n)
    if name == "uniform":
        x = rng.random(n)
    elif name == "normal":
        x = rng.standard_normal(n)
    elif name == "halfnormal":
        x = np.abs(rng.standard_normal(n))
    elif name == "beta25":
        x = rng.beta(2.0, 5.0, n)
    elif name in ("mix1", "mix2", "mix3", "mix4", "mix5"):
        n1 = {"mix1": (2 * n) // 3, "mix2": n // 2 + 1, "mix3": (9 * n) // 10,
              "mix4": (2 * n) // 3, "mix5": n // 2 + 1}[name]
        n1 = min(n1, n)
        half = name in ("mix3", "mix4", "mix5")
        first = rng.standard_normal(n1)
        if half:
            first = np.abs(first)
        if name == "mix3":
            second = np.full(n - n1, 10.0)
        else:
            second = rng.normal(100.0, 1.0, n - n1)
        x = np.concatenate([first, second])
        rng.shuffle(x)
    else:
        raise ValueError(name)
    return x.astype(dtype)


HEAVY_FAMILIES = ("normal", "lognormal", "cauchy", "mixture")


def heavy_mixture(family, n, seed, dtype=np.float32, dup_frac=0.05, n_inf=10):
    """Single-array workload: N(0,1), lognormal(0,2), Student-t nu=1 or an equal-weight
    mixture of the three, then ``dup_frac`` of the positions (without replacement) set
    to one value v (the base draw's [(n+1)/2]-th smallest, found with np.partition) and
    ``n_inf`` positions set to +-inf (half each)."""
    rng = np.random.default_rng(seed)
    n = int(n)
    if family == "normal":
        x = rng.standard_normal(n)
    elif family == "lognormal":
        x = rng.lognormal(0.0, 2.0, n)
    elif family == "cauchy":
        x = rng.standard_cauchy(n)          # Student-t with nu = 1
    elif family == "mixture":
        which = rng.integers(0, 3, n, dtype=np.int8)
        x = np.empty(n)
        for c, draw in enumerate((rng.standard_normal, lambda m: rng.lognormal(0.0, 2.0, m),
                                  rng.standard_cauchy)):
            sel = which == c
            x[sel] = draw(int(np.count_nonzero(sel)))
    else:
        raise ValueError(family)
    x = x.astype(dtype)
    n_dup = int(dup_frac * n)
    if n_dup > 0:
        v = np.partition(x, (n + 1) // 2 - 1)[(n + 1) // 2 - 1]
        pos = rng.choice(n, size=n_dup, replace=False)
        x[pos] = v
    if n_inf > 0 and n >= n_inf:
        pos = rng.choice(n, size=n_inf, replace=False)
        x[pos[: n_inf // 2]] = -np.inf
        x[pos[n_inf // 2:]] = np.inf
    return x


def segment_sizes(S, seed, lo=1e3, hi=1e6):
    """S sizes floor(10^U(log10 lo, log10 hi))."""
    rng = np.random.default_rng(seed)
    return np.floor(10.0 ** rng.uniform(np.log10(lo), np.log10(hi), int(S))).astype(np.int64)


def segmented(S, seed, lo=1e3, hi=1e6, dtype=np.float32):
    """(values, offsets[S+1]) for S normal arrays with mean ~U(-100,100) and
    std ~10^U(-3,3), sizes from :func:`segment_sizes`."""
    sizes = segment_sizes(S, seed, lo, hi)
    rng = np.random.default_rng(seed + 1)
    mu = rng.uniform(-100.0, 100.0, int(S))
    sd = 10.0 ** rng.uniform(-3.0, 3.0, int(S))
    offsets = np.zeros(int(S) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    x = np.empty(int(offsets[-1]), dtype=dtype)
    for s in range(int(S)):
        seg = rng.standard_normal(int(sizes[s]), dtype=np.float32) if dtype == np.float32 \
            else rng.standard_normal(int(sizes[s]))
        x[offsets[s]:offsets[s + 1]] = (seg * sd[s] + mu[s]).astype(dtype)
    return x, offsets


def regression(n, p, seed, contamination=0.3, dy=10.0, dx=5.0):
    """X ~ N(0,1) (n x p, float32), beta ~ N(0,1), y = X beta + N(0,1); a seeded
    ``contamination`` share of rows gets y += dy and X[:, 0] += dx."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((int(n), int(p)))
    beta = rng.standard_normal(int(p))
    y = X @ beta + rng.standard_normal(int(n))
    bad = rng.choice(int(n), size=int(contamination * n), replace=False)
    y[bad] += dy
    X[bad, 0] += dx
    return X.astype(np.float32), y.astype(np.float32), beta


def elemental_thetas(X, y, C, seed):
    """C candidates theta (p x C, float32) from random elemental p-subsets: each solves
    X_S theta = y_S exactly for a random set S of p rows (re-drawn while singular)."""
    rng = np.random.default_rng(seed)
    n, p = X.shape
    out = np.empty((p, int(C)), dtype=np.float64)
    Xd = X.astype(np.float64)
    yd = y.astype(np.float64)
    c = 0
    while c < C:
        rows = rng.choice(n, size=p, replace=False)
        A = Xd[rows]
        if abs(np.linalg.det(A)) < 1e-8:
            continue
        out[:, c] = np.linalg.solve(A, yd[rows])
        c += 1
    return out.astype(np.float32)


def knn_problem(n, p, m, n_classes, seed, lattice=False):
    """kNN workload: n training points in p dimensions from n_classes Gaussian clusters
    (centres ~ N(0, 4^2 I), unit spread), each point labelled with its cluster.  The
    ordinate is f = sum of sin(x_t) over the coordinates plus N(0, 0.1^2) noise.  The m
    queries are drawn the same way.  ``lattice`` rounds every coordinate to an integer,
    so float32 distances are exact and tied distances are common.  Returns X (n, p) and
    Q (m, p) float32, f (n,) float32 and labels (n,) int32."""
    rng = np.random.default_rng(seed)
    n, p, m, K = int(n), int(p), int(m), int(n_classes)
    centres = rng.normal(0.0, 4.0, (K, p))
    labels = rng.integers(0, K, n)
    X = centres[labels] + rng.standard_normal((n, p))
    Q = centres[rng.integers(0, K, m)] + rng.standard_normal((m, p))
    if lattice:
        X, Q = np.rint(X), np.rint(Q)
    f = np.sin(X).sum(axis=1) + 0.1 * rng.standard_normal(n)
    return X.astype(np.float32), Q.astype(np.float32), f.astype(np.float32), labels.astype(np.int32)


TRAIN_FAMILIES = ("normal", "student", "lognormal", "contaminated")


def training_array(seed, n=None, lo=2 ** 20, hi=2 ** 24):
    """One array of the bracket-proposal training distribution: n log-uniform in
    [lo, hi]; normal, Student-t with nu ~ U[1,5], lognormal, or a normal contaminated
    by 10-40% of a shifted, wider normal; random location and scale."""
    rng = np.random.default_rng(seed)
    if n is None:
        n = int(np.floor(2.0 ** rng.uniform(np.log2(lo), np.log2(hi))))
    fam = TRAIN_FAMILIES[rng.integers(0, len(TRAIN_FAMILIES))]
    loc = rng.uniform(-100.0, 100.0)
    scale = 10.0 ** rng.uniform(-2.0, 2.0)
    if fam == "normal":
        x = rng.standard_normal(n)
    elif fam == "student":
        x = rng.standard_t(rng.uniform(1.0, 5.0), n)
    elif fam == "lognormal":
        x = rng.lognormal(0.0, rng.uniform(0.25, 2.0), n)
    else:
        frac = rng.uniform(0.1, 0.4)
        x = rng.standard_normal(n)
        bad = rng.random(n) < frac
        x[bad] = rng.normal(rng.uniform(3.0, 20.0), rng.uniform(1.0, 10.0), int(bad.sum()))
    return (loc + scale * x).astype(np.float32)
