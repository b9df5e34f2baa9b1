"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and
the benchmark.

This module draws random numbers and nothing else: it holds none of the
correlation arithmetic (no means, norms, dot products or thresholds), so the
two sides that consume its arrays stay independent.

Workloads (stand-ins for the paper's data, Section IV):
  * ``modules_normal``  -- values 8 + N(0,1) with planted modules sharing a
    latent N(0,1) factor (the small FP64 parity workload).
  * ``counts_log``      -- log2(1 + count), count ~ NegBinomial(mean mu_g,
    dispersion alpha) with mu_g ~ LogNormal(3, 1.5), plus planted 40-gene
    modules (an RNA-seq-like expression matrix; the paper's SEEK GPL570 data
    is not available, this generator stands in for it).
  * ``uniform01``       -- U[0,1] values, the paper's own artificial data
    (Section IV-A).
  * ``fisher_yates_perms`` -- P seeded sample permutations (splitmix64 +
    Lemire's unbiased bounded draw), one row per permutation.
  * ``uneven_shapes``   -- the (n_b, l_b) list of a batch of uneven matrices.
  * ``counts_log_many`` -- many ``counts_log`` matrices drawn in parallel
    (spawned processes), identical to the serial calls.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "modules_normal",
    "counts_log",
    "uniform01",
    "fisher_yates_perms",
    "uneven_shapes",
    "counts_log_many",
    "module_assignment",
    "splitmix64",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def modules_normal(n: int = 2000, l: int = 128, seed: int = 1,
                   n_modules: int = 10, module_size: int = 50,
                   dtype=np.float64) -> np.ndarray:
    """Values 8 + N(0,1); genes 0 .. n_modules*module_size-1 form consecutive
    modules; gene g of module m gets + a_g * f_{m,s}, a_g ~ U(0.5, 2),
    f ~ N(0,1).  Draw order: noise (n x l), factors (n_modules x l),
    loadings (n_modules*module_size)."""
    rng = _rng(seed)
    x = 8.0 + rng.standard_normal((n, l))
    n_modules = min(n_modules, n // module_size)
    f = rng.standard_normal((n_modules, l))
    a = rng.uniform(0.5, 2.0, size=n_modules * module_size)
    for m in range(n_modules):
        g0 = m * module_size
        x[g0:g0 + module_size] += a[g0:g0 + module_size, None] * f[m][None, :]
    return np.ascontiguousarray(x.astype(dtype))


def module_assignment(n: int, n_modules: int, module_size: int,
                      rng: np.random.Generator) -> np.ndarray:
    """module id per gene (-1 = no module); module genes are a random subset
    so that planted pairs land in many tiles."""
    order = rng.permutation(n)
    mod = np.full(n, -1, dtype=np.int64)
    k = n_modules * module_size
    mod[order[:k]] = np.arange(k) // module_size
    return mod


def counts_log(n: int, l: int, seed: int, n_modules: int = 200,
               module_size: int = 40, dispersion: float = 0.2,
               meanlog: float = 3.0, sdlog: float = 1.5,
               dtype=np.float32, return_modules: bool = False):
    """log2(1 + count) + a_g * f_{m(g),s}.

    count_gs ~ NB with mean mu_g and variance mu + alpha*mu^2 (alpha =
    ``dispersion``, numpy's ``negative_binomial(1/alpha, p)`` with
    p = (1/alpha) / (1/alpha + mu)); mu_g ~ LogNormal(meanlog, sdlog).
    The module count is min(n_modules, n // 80).  All-zero count rows are
    kept: with no module they are constant rows (zero variance).
    Draw order: mu (n), counts (n x l), module assignment, loadings (n),
    factors (n_modules x l).  With return_modules, also returns the module
    id of every gene (-1 = none)."""
    rng = _rng(seed)
    mu = rng.lognormal(meanlog, sdlog, size=n)
    size = 1.0 / dispersion
    p = size / (size + mu)
    counts = rng.negative_binomial(size, p[:, None], size=(n, l))
    x = np.log2(1.0 + counts.astype(np.float64))
    n_mod = min(n_modules, n // 80)
    mod = module_assignment(n, n_mod, module_size, rng)
    a = rng.uniform(0.5, 2.0, size=n)
    f = rng.standard_normal((max(n_mod, 1), l))
    sel = mod >= 0
    if n_mod > 0:
        x[sel] += a[sel, None] * f[mod[sel]]
    x = np.ascontiguousarray(x.astype(dtype))
    return (x, mod) if return_modules else x


def _counts_log_job(job):
    n, l, seed, return_modules = job
    return counts_log(n, l, seed, return_modules=return_modules)


def counts_log_many(shapes, seeds, return_modules: bool = False,
                    workers: int | None = None):
    """``counts_log(n, l, seed)`` for every (n, l) of ``shapes`` with the
    matching seed, drawn in a pool of spawned processes (each matrix has its
    own generator, so the arrays equal the serial calls').  Spawned, not
    forked, so that it is safe after CUDA has been initialised."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    jobs = [(int(n), int(l), int(s), return_modules)
            for (n, l), s in zip(shapes, seeds)]
    if workers is None:
        workers = min(len(jobs), os.cpu_count() or 1, 16)
    if workers <= 1 or len(jobs) <= 1:
        return [_counts_log_job(j) for j in jobs]
    with cf.ProcessPoolExecutor(workers,
                                mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_counts_log_job, jobs))


def uniform01(n: int, l: int, seed: int, dtype=np.float32) -> np.ndarray:
    """U[0,1] expression values (the paper's artificial datasets)."""
    return np.ascontiguousarray(_rng(seed).random((n, l)).astype(dtype))


_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(state: np.ndarray):
    """One splitmix64 step on a uint64 array; returns (new_state, output).
    Published constants of Steele, Lea and Flood's SplitMix64."""
    with np.errstate(over="ignore"):
        state = state + np.uint64(0x9E3779B97F4A7C15)
        z = state.copy()
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return state, z


def fisher_yates_perms(P: int, l: int, seed: int = 4) -> np.ndarray:
    """P permutations of range(l), int32, shape (P, l).

    Permutation k starts from the identity and a splitmix64 stream seeded
    with (seed << 32) + k; for s = l-1 down to 1 it swaps position s with
    j drawn uniformly from [0, s] by Lemire's multiply-and-reject method on
    the high 32 bits of each splitmix64 output."""
    perms = np.tile(np.arange(l, dtype=np.int32), (P, 1))
    state = (np.uint64(seed) << np.uint64(32)) + np.arange(P, dtype=np.uint64)
    rows = np.arange(P)
    for s in range(l - 1, 0, -1):
        rng_range = np.uint64(s + 1)
        thresh = np.uint64((2**32 - (s + 1)) % (s + 1))
        j = np.zeros(P, dtype=np.uint64)
        todo = np.ones(P, dtype=bool)
        while todo.any():
            st, out = splitmix64(state[todo])
            state[todo] = st
            x32 = out >> np.uint64(32)
            m = x32 * rng_range
            low = m & np.uint64(0xFFFFFFFF)
            ok = low >= thresh
            idx = np.nonzero(todo)[0]
            j[idx[ok]] = m[ok] >> np.uint64(32)
            todo[idx[ok]] = False
        j = j.astype(np.int64)
        a = perms[rows, s].copy()
        perms[rows, s] = perms[rows, j]
        perms[rows, j] = a
    return perms


def uneven_shapes(B: int = 64, seed: int = 5, n_lo: int = 500,
                  n_hi: int = 20000, l_lo: int = 32, l_hi: int = 2048):
    """(n_b, l_b) for B matrices, independent inclusive uniform integers;
    matrix b's values come from ``counts_log(n_b, l_b, seed*1000 + b)``."""
    rng = _rng(seed)
    n = rng.integers(n_lo, n_hi + 1, size=B)
    l = rng.integers(l_lo, l_hi + 1, size=B)
    return [(int(a), int(b)) for a, b in zip(n, l)]
