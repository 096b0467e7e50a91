"""Seeded synthetic inputs for the batched fermion-determinant path.

This module only *generates inputs*: the honeycomb hopping (adjacency) matrix ``A``, the hopping
exponential ``E = exp(delta*kappa*A)`` with its inverse, and Gaussian auxiliary fields ``phi``.
It holds none of the determinant arithmetic (no slice products, no QR, no assembly, no force);
the CPU oracle and the GPU library both consume the arrays made here and share nothing else.

The paper works with a generic ``M_t = exp(K_t)`` (Section 2).  The concrete model used by every
workload is a Hubbard-type model on a periodic L x L honeycomb lattice with time slices
``B_t = E diag(exp(i phi_t))``; ``phi_{t,x}`` are iid normal with variance ``delta*U``.

Seeds: workload ``k`` uses ``seed = 1000 + k``; configuration ``c`` of a batch draws its field
from ``numpy.random.default_rng([seed, c])``.  Proposals for local updates (``bss_proposals``):
step ``s`` of workload ``k`` draws one array for every configuration of the workload from
``numpy.random.default_rng([seed, 7, s])``.
"""
from __future__ import annotations

import dataclasses
from typing import List

import numpy as np

__all__ = [
    "honeycomb_adjacency",
    "honeycomb_spectrum",
    "hopping_exp",
    "field",
    "Problem",
    "make_problem",
    "workload",
    "WORKLOADS",
    "bss_proposals",
    "sparse_rows",
]


def honeycomb_adjacency(L: int) -> np.ndarray:
    """Adjacency matrix of the periodic L x L honeycomb lattice, Nx = 2 L^2 sites.

    Site (i, j, s) with s = 0 (A sublattice) or 1 (B sublattice) has index 2*(i*L + j) + s.
    A(i, j) is bonded to B(i, j), B(i-1, j) and B(i, j-1) (indices mod L), so every site has
    three neighbours and the lattice is bipartite.  Entries are 0 or 1.
    """
    if L < 2:
        raise ValueError("honeycomb lattice needs L >= 2 (L = 1 has multiple bonds)")
    nx = 2 * L * L
    A = np.zeros((nx, nx), dtype=np.float64)

    def idx(i: int, j: int, s: int) -> int:
        return 2 * ((i % L) * L + (j % L)) + s

    for i in range(L):
        for j in range(L):
            a = idx(i, j, 0)
            for (bi, bj) in ((i, j), (i - 1, j), (i, j - 1)):
                b = idx(bi, bj, 1)
                A[a, b] = 1.0
                A[b, a] = 1.0
    return A


def honeycomb_spectrum(L: int) -> np.ndarray:
    """Eigenvalues of :func:`honeycomb_adjacency` from momentum space (sorted ascending).

    For momentum k = 2 pi (m, n) / L the two bands are +-|1 + e^{i k1} + e^{i k2}|.
    Used to pin the lattice independently of a numerical eigen-solver.
    """
    ev = []
    for m in range(L):
        for n in range(L):
            f = 1.0 + np.exp(2j * np.pi * m / L) + np.exp(2j * np.pi * n / L)
            ev += [abs(f), -abs(f)]
    return np.sort(np.asarray(ev))


def hopping_exp(A: np.ndarray, delta: float, kappa: float = 1.0, sign: float = +1.0) -> np.ndarray:
    """``exp(sign*delta*kappa*A)`` for a real symmetric ``A`` via its eigen-decomposition.

    The result is symmetric; it is symmetrised explicitly so that row-major and column-major
    storage hold identical bytes.
    """
    lam, U = np.linalg.eigh(A)
    E = (U * np.exp(sign * delta * kappa * lam)[None, :]) @ U.T
    return 0.5 * (E + E.T)


def field(seed: int, c: int, nt: int, nx: int, delta: float, U: float) -> np.ndarray:
    """Auxiliary field phi[t, x] ~ N(0, delta*U) iid (variance delta*U), float64, shape (nt, nx).

    Row t-1 is the field of time slice t in the product B_Nt ... B_1.
    """
    rng = np.random.default_rng([int(seed), int(c)])
    return rng.normal(0.0, np.sqrt(delta * U), size=(nt, nx)).astype(np.float64)


@dataclasses.dataclass
class Problem:
    """One configuration: lattice size, time discretisation and the arrays the library takes."""

    L: int
    nt: int
    n_stab: int
    beta: float
    U: float
    kappa: float
    E: np.ndarray  # (nx, nx) float64, exp(delta*kappa*A)
    Einv: np.ndarray  # (nx, nx) float64, exp(-delta*kappa*A)
    phi: np.ndarray  # (nt, nx) float64
    A: np.ndarray  # (nx, nx) adjacency (for closed forms and invariants)

    @property
    def nx(self) -> int:
        return 2 * self.L * self.L

    @property
    def delta(self) -> float:
        return self.beta / self.nt


_CACHE: dict = {}


def _lattice(L: int, delta: float, kappa: float):
    key = (L, float(delta), float(kappa))
    if key not in _CACHE:
        A = honeycomb_adjacency(L)
        _CACHE[key] = (A, hopping_exp(A, delta, kappa, +1.0), hopping_exp(A, delta, kappa, -1.0))
    return _CACHE[key]


def make_problem(L: int, nt: int, beta: float, U: float, n_stab: int, seed: int, c: int,
                 kappa: float = 1.0, zero_field: bool = False) -> Problem:
    delta = beta / nt
    A, E, Einv = _lattice(L, delta, kappa)
    nx = 2 * L * L
    phi = np.zeros((nt, nx)) if zero_field else field(seed, c, nt, nx, delta, U)
    return Problem(L=L, nt=nt, n_stab=n_stab, beta=beta, U=U, kappa=kappa, E=E, Einv=Einv,
                   phi=phi, A=A)


# Named workloads.  Index k uses seed 1000 + k.
#   tiny8      : L=2 (Nx=8),  beta=2,  Nt=16,  U=2,   n_stab=4,  1 config
#   batch18    : L=3 (Nx=18), beta=8,  Nt=64,  U=3,   n_stab=8,  256 configs
#   cold72     : L=6 (Nx=72), beta=64, Nt=512, U=3.5, n_stab=16, 64 configs
#   force72    : L=6 (Nx=72), beta=32, Nt=256, U=3,   n_stab=8,  32 configs
#   sparse288  : L=12 (Nx=288), beta=8, Nt=64, U=3,  n_stab=16, 152 configs (intermediate volume)
#   uneven512  : Nx in {8,...,288} x Nt in {32,...,1024}, delta=1/16, U=3, 512 configs
WORKLOADS = {
    "tiny8": dict(index=0, L=2, nt=16, beta=2.0, U=2.0, n_stab=4, batch=1),
    "batch18": dict(index=1, L=3, nt=64, beta=8.0, U=3.0, n_stab=8, batch=256),
    "cold72": dict(index=2, L=6, nt=512, beta=64.0, U=3.5, n_stab=16, batch=64),
    "force72": dict(index=3, L=6, nt=256, beta=32.0, U=3.0, n_stab=8, batch=32),
    "sparse288": dict(index=5, L=12, nt=64, beta=8.0, U=3.0, n_stab=16, batch=152),
}

UNEVEN_L = (2, 3, 4, 5, 6, 7, 8, 12)
UNEVEN_NT = (32, 64, 128, 256, 512, 1024)


def uneven_sizes(batch: int = 512, first: int = 0) -> List[tuple]:
    """(L, Nt) of configurations first .. first+batch-1 of the uneven sequence (no fields drawn)."""
    pairs = [(L, nt) for L in UNEVEN_L for nt in UNEVEN_NT]
    order = [pairs[i % len(pairs)] for i in range(512)]
    perm = np.random.default_rng(1004).permutation(len(order))
    return [order[perm[c % 512]] for c in range(first, first + batch)]


def _uneven(batch: int = 512, n_stab: int = 16, first: int = 0) -> List[Problem]:
    """Configurations first .. first+batch-1 of the uneven sequence.  Every run of 512
    consecutive indices (k*512 .. k*512+511) holds the 48 (L, Nt) pairs round-robin -- the first
    32 pairs 11 times, the other 16 pairs 10 times -- in the order of one seeded shuffle; the field
    of index c is drawn from seed (1004, c), so later runs repeat the size mix with new fields."""
    seed = 1004
    probs = []
    for c, (L, nt) in zip(range(first, first + batch), uneven_sizes(batch, first)):
        beta = nt / 16.0
        probs.append(make_problem(L, nt, beta, 3.0, min(n_stab, nt), seed, c))
    return probs


def workload(name: str, batch: int | None = None, n_stab: int | None = None,
             zero_field: bool = False, first: int = 0) -> List[Problem]:
    """The configurations of a named workload (optionally ``batch`` of them, starting at
    configuration index ``first``; shards of a multi-GPU run use disjoint index ranges)."""
    if name == "uneven512":
        return _uneven(512 if batch is None else batch, n_stab or 16, first)
    w = WORKLOADS[name]
    b = w["batch"] if batch is None else batch
    ns = w["n_stab"] if n_stab is None else n_stab
    seed = 1000 + w["index"]
    return [make_problem(w["L"], w["nt"], w["beta"], w["U"], ns, seed, c, zero_field=zero_field)
            for c in range(first, first + b)]


def bss_proposals(name: str, step: int, first: int = 0, count: int | None = None):
    """Proposals for one local-update call on every site of one time slice, for configurations
    ``first .. first+count-1`` of a named workload: ``dphi ~ N(0, delta*U)`` (the field's own
    variance), ``u ~ U(0, 1)`` and ``w = 1`` (no weight factor besides the determinant ratio),
    each of shape (count, Nx).  The arrays are drawn for the whole workload, so a configuration
    gets the same proposals whichever shard asks for it."""
    w = WORKLOADS[name]
    nx = 2 * w["L"] * w["L"]
    total = w["batch"]
    count = total - first if count is None else count
    rng = np.random.default_rng([1000 + w["index"], 7, int(step)])
    dphi = rng.normal(0.0, np.sqrt(w["beta"] / w["nt"] * w["U"]), size=(total, nx))
    u = rng.uniform(size=(total, nx))
    sl = slice(first, first + count)
    return (np.ascontiguousarray(dphi[sl]), np.ascontiguousarray(u[sl]),
            np.ones((count, nx)))


def sparse_rows(A: np.ndarray, q: int | None = None):
    """The non-zero pattern of a (sparse) matrix as fixed-width rows: col (nx, q) int32 and
    val (nx, q) float64 with row i's entries at [i, 0..q-1]; rows with fewer than q entries are
    padded with (col = i, val = 0).  For the honeycomb adjacency q = 3."""
    nx = A.shape[0]
    rows = [np.flatnonzero(A[i]) for i in range(nx)]
    width = max(len(r) for r in rows) if q is None else q
    if any(len(r) > width for r in rows):
        raise ValueError("a row has more than q entries")
    col = np.empty((nx, width), dtype=np.int32)
    val = np.zeros((nx, width))
    for i, r in enumerate(rows):
        col[i, :len(r)] = r
        val[i, :len(r)] = A[i, r]
        col[i, len(r):] = i
    return col, val
