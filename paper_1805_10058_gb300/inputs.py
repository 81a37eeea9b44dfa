"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

Only random numbers and workload lists live here (no arithmetic of the method):
right-hand sides with i.i.d. uniform[-1, 1] entries, parameter sweeps, serving-stream
arrival times.  Vectors use the library layout [nrhs][d][m]^d (x_d fastest).
"""
import numpy as np


def dofs(d, p, n):
    """d (n+p-2)^d, or d prod_l (n_l+p-2) for per-direction interval counts n = (n_1..n_d)."""
    if np.isscalar(n):
        return d * (n + p - 2) ** d
    return d * int(np.prod([v + p - 2 for v in n]))


def uniform_rhs(d, p, n, seed, nrhs=1):
    """nrhs right-hand sides with entries i.i.d. uniform[-1, 1] from default_rng(seed)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, (nrhs, dofs(d, p, n)))


def sine_rhs(d, p, n, seed, nrhs=1):
    """Smooth seeded right-hand sides: component c of each is prod_l sin(k_{c,l} pi x_l) sampled
    at the uniform interior points x = (i + 1) / (m + 1), i = 0..m-1 (m = n + p - 2), with the
    integers k_{c,l} drawn from default_rng(seed).integers(1, 5) per right-hand side (the
    manufactured sine fields of the 3D workload, as point samples)."""
    rng = np.random.default_rng(seed)
    m = n + p - 2
    x = (np.arange(m) + 1.0) / (m + 1.0)
    out = np.empty((nrhs, dofs(d, p, n)))
    for r in range(nrhs):
        ks = rng.integers(1, 5, (d, d))
        comps = []
        for c in range(d):
            f = np.ones([m] * d)
            for l in range(d):
                shape = [1] * d
                shape[l] = m
                f = f * np.sin(ks[c, l] * np.pi * x).reshape(shape)
            comps.append(f.ravel())
        out[r] = np.concatenate(comps)
    return out


def uniform_rhs_seeds(d, p, n, seeds):
    """One right-hand side per seed (uniform[-1, 1], default_rng(seed)), stacked."""
    return np.stack([uniform_rhs(d, p, n, s)[0] for s in seeds])


# The 2D sweep: p in {2, 3, 4}, n = 256, the parameter (beta, with alpha = 1) in
# {1e-6, 1e-3, 1, 1e3, 1e6}, 8 seeded uniform right-hand sides per case (seeds 0..7).
SWEEP_2D = dict(d=2, ps=(2, 3, 4), n=256, betas=(1e-6, 1e-3, 1.0, 1e3, 1e6), seeds=tuple(range(8)))


def sweep_cases(spec=SWEEP_2D):
    """[(d, p, n, alpha, beta, seed)] of a sweep specification."""
    out = []
    for p in spec["ps"]:
        for beta in spec["betas"]:
            for s in spec["seeds"]:
                out.append((spec["d"], p, spec["n"], 1.0, beta, s))
    return out


def loguniform_params(seed, count, lo=1e-6, hi=1e6):
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), count))


def serving_stream(seed=0, count=2000, rate=200.0):
    """Poisson arrivals (mean `rate`/s) of solve requests: 60% 2D (n in 32..256), 40% 3D
    (n in 16..96), p in 1..5, beta log-uniform in [1e-6, 1e6] (alpha = 1), 1-4 RHS each."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, count))
    reqs = []
    for i in range(count):
        is2d = rng.uniform() < 0.6
        d = 2 if is2d else 3
        n = int(rng.integers(32, 257)) if is2d else int(rng.integers(16, 97))
        p = int(rng.integers(1, 6))
        beta = float(np.exp(rng.uniform(np.log(1e-6), np.log(1e6))))
        nrhs = int(rng.integers(1, 5))
        reqs.append(dict(t=float(t[i]), d=d, p=p, n=n, alpha=1.0, beta=beta, nrhs=nrhs,
                         seed=int(rng.integers(0, 2 ** 31 - 1))))
    return reqs
