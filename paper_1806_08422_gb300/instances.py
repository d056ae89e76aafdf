"""Seeded synthetic Ising instances and annealing schedules.

These generators produce INPUT DATA only (couplings, fields, temperature arrays,
arrival streams); they contain none of the annealing arithmetic.  Both the CUDA
library and the CPU oracle consume their output.  Every generator draws from its own
numpy PCG64 stream keyed by `seed`, independent of the Philox noise stream of the
method.

Instance classes follow the paper's workloads (Sec. III):
  sk          -- Sherrington-Kirkpatrick, J_ij = +1 or -1 with probability 1/2
  gnp_maxcut  -- dense MAX-CUT, J_ij = 1 with probability p (p = 0.5 in the paper)
  regular3    -- degree-3 MAX-CUT, every spin coupled to three others with J = 1
  moebius     -- the Moebius ladder of Fig. 3 (ring plus antipodal chords, J = 1)
  ring, complete -- closed-form test graphs
All couplings are symmetric with zero diagonal; h = 0 unless asked.
"""
from __future__ import annotations

import math

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _symmetrize_upper(upper: np.ndarray) -> np.ndarray:
    u = np.triu(upper, 1)
    return u + u.T


def sk(n: int, seed: int = 0) -> np.ndarray:
    """SK instance: J_ij = +1 w.p. 1/2 and -1 otherwise (Sec. III, Fig. 4a)."""
    r = _rng(seed)
    upper = np.where(r.random((n, n)) < 0.5, 1.0, -1.0)
    return _symmetrize_upper(upper)


def gnp_maxcut(n: int, p: float = 0.5, seed: int = 0) -> np.ndarray:
    """Dense MAX-CUT: J_ij = 1 with probability p, else 0 (Sec. III, Fig. 4b)."""
    r = _rng(seed)
    upper = (r.random((n, n)) < p).astype(np.float64)
    return _symmetrize_upper(upper)


def ring(n: int) -> np.ndarray:
    J = np.zeros((n, n))
    for i in range(n):
        j = (i + 1) % n
        if j != i:
            J[i, j] = J[j, i] = 1.0
    return J


def complete(n: int) -> np.ndarray:
    J = np.ones((n, n))
    np.fill_diagonal(J, 0.0)
    return J


def moebius(n: int) -> np.ndarray:
    """Moebius ladder on n (even) spins: ring edges (i, i+1 mod n) and chords
    (i, i + n/2) for i < n/2, J = +1 per edge (the 16-spin example of Fig. 3)."""
    if n % 2 or n < 4:
        raise ValueError("Moebius ladder needs an even n >= 4")
    J = ring(n)
    for i in range(n // 2):
        j = i + n // 2
        J[i, j] = J[j, i] = 1.0
    return J


def regular3(n: int, seed: int = 0, max_tries: int = 10000) -> np.ndarray:
    """Random 3-regular graph by the configuration model with rejection of
    self-loops and multi-edges (Sec. III, Fig. 4c), J = +1 per edge."""
    if (3 * n) % 2 or n < 4:
        raise ValueError("3-regular graph needs even n >= 4")
    r = _rng(seed)
    for _ in range(max_tries):
        stubs = np.repeat(np.arange(n), 3)
        r.shuffle(stubs)
        a, b = stubs[0::2], stubs[1::2]
        if np.any(a == b):
            continue
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        keys = lo.astype(np.int64) * n + hi
        if np.unique(keys).size != keys.size:
            continue
        J = np.zeros((n, n))
        J[lo, hi] = 1.0
        J[hi, lo] = 1.0
        return J
    raise RuntimeError("configuration model did not produce a simple graph")


def random_fields(n: int, scale: float = 1.0, seed: int = 0) -> np.ndarray:
    """Real-valued local fields h_i ~ U(-scale, scale)."""
    return _rng(seed).uniform(-scale, scale, size=n)


def random_real_couplings(n: int, seed: int = 0, density: float = 1.0) -> np.ndarray:
    """Symmetric real-valued couplings J_ij ~ N(0,1) on a G(n, density) support."""
    r = _rng(seed)
    upper = r.standard_normal((n, n)) * (r.random((n, n)) < density)
    return _symmetrize_upper(upper)


def to_csr(J: np.ndarray):
    """Dense symmetric J -> (row_ptr int64[n+1], col int32[nnz], val float64[nnz]),
    columns ascending within each row."""
    n = J.shape[0]
    rows, cols = np.nonzero(J)
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return row_ptr, cols.astype(np.int32), J[rows, cols].astype(np.float64)


def moebius_csr(n: int):
    """The Moebius ladder of `moebius(n)` built directly in CSR form (no dense
    matrix, so it serves sizes whose n x n array would not fit in memory)."""
    if n % 2 or n < 4:
        raise ValueError("Moebius ladder needs an even n >= 4")
    i = np.arange(n)
    nbr = np.stack([(i - 1) % n, (i + 1) % n, (i + n // 2) % n], axis=1)
    nbr.sort(axis=1)
    if n == 4:  # K_4: the chords coincide with ring edges; keep each neighbour once
        rows = [np.unique(r) for r in nbr]
        row_ptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
        col = np.concatenate(rows).astype(np.int32)
        return row_ptr, col, np.ones(len(col), dtype=np.float64)
    row_ptr = np.arange(0, 3 * n + 1, 3, dtype=np.int64)
    return row_ptr, nbr.reshape(-1).astype(np.int32), np.ones(3 * n, dtype=np.float64)


# ----------------------------------------------------------------------------
# Annealing schedule.  The paper's Fig. 2 (a "three-segment piecewise
# exponential" schedule) survives only as its caption, so the default below is a
# reconstruction: log T is piecewise linear in t/t_f through the knots
#   (0, 10), (0.1, 2.0), (0.9, 0.5), (1.0, 0.05),
# i.e. a fast exponential cooling to just above the SK instability (T ~ 2 in the
# normalised units of Algorithm 1), a slow segment across it, and a final quench.
# The schedule is always an input array; nothing in the library hard-codes it.
# ----------------------------------------------------------------------------
DEFAULT_KNOTS = ((0.0, 10.0), (0.1, 2.0), (0.9, 0.5), (1.0, 0.05))


def schedule(t_f: int, knots=DEFAULT_KNOTS) -> np.ndarray:
    """T[0..t_f) with log T piecewise linear through `knots` (x in [0,1], T > 0),
    sampled at x = t / (t_f - 1)."""
    if t_f <= 0:
        return np.zeros(0)
    xs = np.array([k[0] for k in knots], dtype=np.float64)
    ls = np.log(np.array([k[1] for k in knots], dtype=np.float64))
    x = np.arange(t_f, dtype=np.float64) / max(t_f - 1, 1)
    return np.exp(np.interp(x, xs, ls))


# ----------------------------------------------------------------------------
# Workload recipes (the shapes of the paper's experiments, Sec. III).
# ----------------------------------------------------------------------------
def ragged_batch(count: int = 512, n_lo: int = 16, n_hi: int = 1000, seed: int = 0):
    """Ragged mix: N ~ U[n_lo, n_hi] integers; the first half SK +-1, the second
    half G(N, 0.5) MAX-CUT.  Returns a list of (kind, n, J)."""
    r = _rng(seed)
    ns = r.integers(n_lo, n_hi + 1, size=count)
    out = []
    for k, n in enumerate(ns):
        n = int(n)
        if k < count // 2:
            out.append(("sk", n, sk(n, seed=seed * 100003 + k)))
        else:
            out.append(("gnp", n, gnp_maxcut(n, 0.5, seed=seed * 100003 + k)))
    return out


def poisson_requests(count: int, rate_hz: float = 200.0, n_lo: int = 64, n_hi: int = 8192,
                     replica_choices=(64, 128, 256, 512, 1024), seed: int = 0):
    """Serving stream: exponential inter-arrival gaps (mean 1/rate), N log-uniform
    in [n_lo, n_hi], 50/50 SK or G(N, 0.5), replicas uniform over the choices.
    Returns a list of dicts with arrival time (s), kind, n, replicas, instance seed."""
    r = _rng(seed)
    t = 0.0
    reqs = []
    for k in range(count):
        t += r.exponential(1.0 / rate_hz)
        u = r.random()
        n = int(math.floor(n_lo * (n_hi / n_lo) ** u))
        n = max(n_lo, min(n_hi, n))
        kind = "sk" if r.random() < 0.5 else "gnp"
        reps = int(r.choice(replica_choices))
        reqs.append({"arrival": t, "kind": kind, "n": n, "replicas": reps,
                     "seed": seed * 1000003 + k})
    return reqs


def make_instance(kind: str, n: int, seed: int) -> np.ndarray:
    if kind == "sk":
        return sk(n, seed)
    if kind == "gnp":
        return gnp_maxcut(n, 0.5, seed)
    if kind == "moebius":
        return moebius(n)
    if kind == "regular3":
        return regular3(n, seed)
    raise ValueError(kind)


# ----------------------------------------------------------------------------
# Gset files (the format of the G22/G39 instances of Table I): a header line
# "n m" followed by m lines "i j w" with 1-based vertices; J_ij = w per edge, so the
# Ising energy H of Eq. (1) and the cut value relate by cut = (W - H) / 2 with
# W = sum_{i<j} J_ij (Table I reports cut values).  The files themselves are not
# shipped; a user who has them can reproduce Table I's setting.
# ----------------------------------------------------------------------------
def read_gset(path: str):
    """Returns (n, J) with J dense float64 symmetric, zero diagonal."""
    with open(path) as f:
        head = f.readline().split()
        n, m = int(head[0]), int(head[1])
        J = np.zeros((n, n))
        for _ in range(m):
            parts = f.readline().split()
            i, j, w = int(parts[0]) - 1, int(parts[1]) - 1, float(parts[2]) if len(parts) > 2 else 1.0
            if i == j:
                raise ValueError("self-loop in Gset file")
            J[i, j] += w
            J[j, i] += w
    return n, J


def write_gset(path: str, J: np.ndarray):
    n = J.shape[0]
    iu = np.argwhere(np.triu(J, 1) != 0)
    with open(path, "w") as f:
        f.write("%d %d\n" % (n, len(iu)))
        for i, j in iu:
            w = J[i, j]
            f.write("%d %d %s\n" % (i + 1, j + 1, repr(int(w)) if float(w).is_integer() else repr(float(w))))


def cut_value(J: np.ndarray, energy: float) -> float:
    """MAX-CUT value of a sign vector with Ising energy `energy` (h = 0)."""
    return 0.5 * (float(np.triu(J, 1).sum()) - energy)
