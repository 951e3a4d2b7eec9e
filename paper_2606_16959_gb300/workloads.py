"""Seeded synthetic inputs: Pauli-sum Hamiltonians and initial states.

The paper evaluates on HamLib instances (TFIM, Heisenberg, MaxCut, TSP;
Tab. 3, 6-16 qubits).  Those files are not available here, so every input is
generated from the closed-form family definitions with the same structure
(transverse-field Ising and Heisenberg chains, weighted MaxCut on a random
3-regular graph, one-hot TSP) and extended to the sizes of the benchmark
configurations.  This module holds no arithmetic of the method itself (no
rotations, grouping or diagonal layout): it only writes Hamiltonians as
labelled Pauli terms with real coefficients, plus initial states.  Both the
CUDA library and the FP64 oracle consume its outputs unchanged.

Label convention: the rightmost character of a label acts on qubit 0, which
is bit 0 of the basis index.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np


@dataclass
class Hamiltonian:
    family: str
    n_qubits: int
    labels: List[str]
    coeffs: np.ndarray                       # float64, one per label
    meta: Dict = field(default_factory=dict)  # graph / couplings / distances


def label_of(n: int, ops: Dict[int, str]) -> str:
    """Pauli label on n qubits with the given {qubit: 'X'|'Y'|'Z'} factors."""
    chars = ["I"] * n
    for q, p in ops.items():
        chars[n - 1 - q] = p
    return "".join(chars)


# ----------------------------------------------------------------------------
# Families
# ----------------------------------------------------------------------------

def tfim_chain(n: int, J: float = 1.0, h: float = 1.0, periodic: bool = False) -> Hamiltonian:
    """H = -J sum Z_i Z_{i+1} - h sum X_i.  Term order: ZZ bonds, then X_i."""
    bonds = [(i, i + 1) for i in range(n - 1)] + ([(n - 1, 0)] if periodic and n > 2 else [])
    labels = [label_of(n, {a: "Z", b: "Z"}) for a, b in bonds] + [label_of(n, {i: "X"}) for i in range(n)]
    coeffs = [-J] * len(bonds) + [-h] * n
    return Hamiltonian("tfim", n, labels, np.asarray(coeffs, dtype=np.float64),
                       {"J": J, "h": h, "periodic": periodic, "bonds": bonds})


def heisenberg_chain(n: int, J: Sequence[float], periodic: bool = True) -> Hamiltonian:
    """H = sum_i J_i (X_i X_{i+1} + Y_i Y_{i+1} + Z_i Z_{i+1}).  Bond-major term
    order (XX_i, YY_i, ZZ_i); the wrap-around bond (n-1, 0) comes last."""
    bonds = [(i, i + 1) for i in range(n - 1)] + ([(n - 1, 0)] if periodic and n > 2 else [])
    J = list(J)
    if len(J) != len(bonds):
        raise ValueError("one coupling per bond")
    labels, coeffs = [], []
    for (a, b), j in zip(bonds, J):
        for p in "XYZ":
            labels.append(label_of(n, {a: p, b: p}))
            coeffs.append(j)
    return Hamiltonian("heisenberg", n, labels, np.asarray(coeffs, dtype=np.float64),
                       {"J": J, "periodic": periodic, "bonds": bonds})


def random_regular_graph(n: int, degree: int, rng: np.random.Generator) -> List[Tuple[int, int]]:
    """Uniform random simple d-regular graph by the pairing model with rejection."""
    if (n * degree) % 2:
        raise ValueError("n * degree must be even")
    while True:
        stubs = np.repeat(np.arange(n), degree)
        rng.shuffle(stubs)
        pairs = stubs.reshape(-1, 2)
        edges = set()
        ok = True
        for a, b in pairs:
            a, b = int(min(a, b)), int(max(a, b))
            if a == b or (a, b) in edges:
                ok = False
                break
            edges.add((a, b))
        if ok:
            return sorted(edges)


def maxcut(n: int, edges: Sequence[Tuple[int, int]], weights: Sequence[float], mixer: float = 0.5) -> Hamiltonian:
    """H = sum_(i,j) w_ij (1 - Z_i Z_j) / 2 + mixer * sum X_i.
    Term order: identity (sum w / 2), then -w/2 Z_i Z_j per edge, then mixer X_i."""
    labels = [label_of(n, {})]
    coeffs = [0.5 * float(np.sum(weights))]
    for (a, b), w in zip(edges, weights):
        labels.append(label_of(n, {a: "Z", b: "Z"}))
        coeffs.append(-0.5 * float(w))
    if mixer:
        for i in range(n):
            labels.append(label_of(n, {i: "X"}))
            coeffs.append(float(mixer))
    return Hamiltonian("maxcut", n, labels, np.asarray(coeffs, dtype=np.float64),
                       {"edges": list(edges), "weights": [float(w) for w in weights], "mixer": mixer})


def maxcut_3regular(n: int, seed: int, mixer: float = 0.5) -> Hamiltonian:
    rng = np.random.default_rng(seed)
    edges = random_regular_graph(n, 3, rng)
    w = rng.uniform(0.0, 1.0, size=len(edges))
    return maxcut(n, edges, w, mixer)


def tsp_qubit(v: int, p: int, n_cities: int) -> int:
    """Qubit of the one-hot variable 'city v visited at position p'."""
    return v * n_cities + p


def tsp_onehot(n_cities: int, seed: int) -> Hamiltonian:
    """One-hot TSP cost as a diagonal Pauli-Z Hamiltonian on n_cities^2 qubits.

    With x_{v,p} = 1 iff city v is at tour position p,
      C(x) = A sum_v (1 - sum_p x_{v,p})^2 + A sum_p (1 - sum_v x_{v,p})^2
             + sum_{u != v} d_uv sum_p x_{u,p} x_{v,p+1 mod n},
    distances d ~ U[1,10] (symmetric), A = 2 max d.  Expanded with
    x = (1 - Z) / 2 into identity, Z_i (ascending) and Z_i Z_j (lexicographic
    i < j; pairs with a zero coefficient are left out)."""
    rng = np.random.default_rng(seed)
    nc = n_cities
    d = np.zeros((nc, nc))
    for u in range(nc):
        for v in range(u + 1, nc):
            d[u, v] = d[v, u] = rng.uniform(1.0, 10.0)
    A = 2.0 * d.max()
    nq = nc * nc
    # quadratic pseudo-boolean form: const + sum a_q x_q + sum_{q<r} b_qr x_q x_r
    const = 0.0
    a = np.zeros(nq)
    bq = np.zeros((nq, nq))

    def add_square_penalty(qs):
        # A (1 - sum x)^2 = A (1 - 2 sum x + sum x + 2 sum_{q<r} x_q x_r)   (x^2 = x)
        nonlocal const
        const += A
        for q in qs:
            a[q] += -A
        for i in range(len(qs)):
            for j in range(i + 1, len(qs)):
                q, r = sorted((qs[i], qs[j]))
                bq[q, r] += 2 * A

    for v in range(nc):
        add_square_penalty([tsp_qubit(v, p, nc) for p in range(nc)])
    for p in range(nc):
        add_square_penalty([tsp_qubit(v, p, nc) for v in range(nc)])
    for u in range(nc):
        for v in range(nc):
            if u == v:
                continue
            for p in range(nc):
                q, r = sorted((tsp_qubit(u, p, nc), tsp_qubit(v, (p + 1) % nc, nc)))
                bq[q, r] += d[u, v]
    # x_q = (1 - Z_q)/2 ;  x_q x_r = (1 - Z_q - Z_r + Z_q Z_r)/4
    c0 = const + 0.5 * a.sum()
    cz = -0.5 * a.copy()
    czz = {}
    for q in range(nq):
        for r in range(q + 1, nq):
            if bq[q, r] == 0.0:
                continue
            c0 += bq[q, r] / 4
            cz[q] -= bq[q, r] / 4
            cz[r] -= bq[q, r] / 4
            czz[(q, r)] = bq[q, r] / 4
    labels = [label_of(nq, {})]
    coeffs = [c0]
    for q in range(nq):
        labels.append(label_of(nq, {q: "Z"}))
        coeffs.append(cz[q])
    for (q, r), c in sorted(czz.items()):
        labels.append(label_of(nq, {q: "Z", r: "Z"}))
        coeffs.append(c)
    return Hamiltonian("tsp", nq, labels, np.asarray(coeffs, dtype=np.float64),
                       {"n_cities": nc, "dist": d, "A": A})


@dataclass
class DrivenHamiltonian:
    """H(t) = H0 + f(t) H1 on one term list: term j has coefficient a[j] in H0
    and b[j] in H1 (zero where it belongs to one of them only)."""
    family: str
    n_qubits: int
    labels: List[str]
    a: np.ndarray   # float64, H0 coefficient per label
    b: np.ndarray   # float64, H1 coefficient per label
    meta: Dict = field(default_factory=dict)


def anneal_maxcut(n: int, seed: int, mixer: float = 0.5) -> DrivenHamiltonian:
    """Annealing from the transverse mixer to weighted MaxCut on a random
    3-regular graph: H(s) = (1 - s) mixer sum X_i + s H_C with s = f(t) (a
    linear ramp s = t / T in the benchmark).  Term order: the mixer X_i, then the
    identity and the ZZ edges of H_C, so that the flip factors and the one
    diagonal factor of H_C group apart."""
    cost = maxcut_3regular(n, seed, mixer=0.0)
    labels = [label_of(n, {i: "X"}) for i in range(n)] + list(cost.labels)
    a = np.concatenate([np.full(n, float(mixer)), np.zeros(len(cost.labels))])
    b = np.concatenate([np.full(n, -float(mixer)), cost.coeffs])
    return DrivenHamiltonian("anneal_maxcut", n, labels, a, b, dict(cost.meta, mixer=mixer))


def driven_tfim(n: int, J: float = 1.0, h: float = 1.0, periodic: bool = False) -> DrivenHamiltonian:
    """Transverse-field Ising chain with a driven field: H0 = -J sum Z_i Z_{i+1},
    H1 = -h sum X_i (term order as tfim_chain)."""
    base = tfim_chain(n, J, h, periodic)
    n_b = len(base.meta["bonds"])
    a = np.concatenate([base.coeffs[:n_b], np.zeros(n)])
    b = np.concatenate([np.zeros(n_b), base.coeffs[n_b:]])
    return DrivenHamiltonian("driven_tfim", n, list(base.labels), a, b, dict(base.meta))


def midpoint_samples(fn, t: float, n_steps: int) -> np.ndarray:
    """f at the midpoints (s + 1/2) t / n_steps of the n_steps steps of [0, t]."""
    dt = float(t) / n_steps
    return np.array([float(fn((s + 0.5) * dt)) for s in range(n_steps)], dtype=np.float64)


# ----------------------------------------------------------------------------
# Initial states
# ----------------------------------------------------------------------------

def basis_state(n: int, b: int = 0) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[b] = 1.0
    return psi


def plus_state(n: int) -> np.ndarray:
    N = 1 << n
    return np.full(N, 1.0 / np.sqrt(N), dtype=np.complex128)


def gaussian_state(n: int, rng: np.random.Generator) -> np.ndarray:
    N = 1 << n
    v = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    return (v / np.linalg.norm(v)).astype(np.complex128)


# ----------------------------------------------------------------------------
# The five benchmark workloads
# ----------------------------------------------------------------------------

@dataclass
class Job:
    ham: Hamiltonian
    t: float
    n_steps: int
    budget: int
    psi0: Optional[np.ndarray]  # (N,) or (n_rhs, N) complex128; None: made from `seed` where it is used
    dtype: str = "c64"        # "c64" or "c128"
    arrival: float = 0.0      # seconds, serving only
    seed: int = 0             # seed of the initial state when psi0 is None
    drive: Optional[np.ndarray] = None  # time-dependent jobs (ham is a DrivenHamiltonian): f per step


def tfim10() -> Job:
    """1D open TFIM, n=10, J=h=1, |0...0>, t=1, 10 steps, budget 4, complex128."""
    return Job(tfim_chain(10, 1.0, 1.0, periodic=False), 1.0, 10, 4, basis_state(10), "c128")


def heis16(dtype: str = "c128", n: int = 16, seed: int = 1002, n_steps: int = 100) -> Job:
    """1D periodic Heisenberg XXX, n=16, J_i ~ U[0.5,1.5], Gaussian state, t=1,
    100 steps, budget 8."""
    rng = np.random.default_rng(seed)
    J = rng.uniform(0.5, 1.5, size=n)
    psi = gaussian_state(n, rng)
    return Job(heisenberg_chain(n, J, periodic=True), 1.0, n_steps, 8, psi, dtype)


def taylor_tfim(n: int = 16, h: float = 0.1, budget: int = 1024, seed: int = 1006, dtype: str = "c64") -> Job:
    """Single-factor Taylor-mode workload shaped like the largest TFIM row of
    the benchmark table (open chain, n=16, small transverse field h=0.1): J=1,
    Gaussian state, t=1, diagonal budget `budget` for the propagator; the step
    count is chosen by the budget search, so n_steps is 0 here."""
    rng = np.random.default_rng(seed)
    return Job(tfim_chain(n, 1.0, h, periodic=False), 1.0, 0, budget, gaussian_state(n, rng), dtype)


def maxcut24(n: int = 24, n_rhs: int = 16, seed: int = 1003, n_steps: int = 50) -> Job:
    """Weighted MaxCut on a random 3-regular graph plus 0.5 sum X_i; RHS 0 = |+>^n,
    RHS 1.. = Gaussian states; t=2, 50 steps, budget 4, complex64 bulk."""
    ham = maxcut_3regular(n, seed, 0.5)
    rng = np.random.default_rng(seed + 7919)
    rows = [plus_state(n)] + [gaussian_state(n, rng) for _ in range(n_rhs - 1)]
    return Job(ham, 2.0, n_steps, 4, np.stack(rows), "c64")


def anneal24(n: int = 24, n_rhs: int = 16, seed: int = 1003, n_steps: int = 50, T: float = 2.0) -> Job:
    """MaxCut annealing on the weighted 3-regular graph of maxcut24 (same seed):
    H(s) = (1 - s) 0.5 sum X_i + s H_C with the linear ramp s = t / T sampled at
    the step midpoints; RHS 0 = |+>^n (the mixer's ground state), RHS 1.. =
    Gaussian states; T = 2, 50 steps, budget 4, complex64 bulk."""
    ham = anneal_maxcut(n, seed, 0.5)
    rng = np.random.default_rng(seed + 7919)
    rows = [plus_state(n)] + [gaussian_state(n, rng) for _ in range(n_rhs - 1)]
    return Job(ham, T, n_steps, 4, np.stack(rows), "c64", drive=midpoint_samples(lambda u: u / T, T, n_steps))


def batch256(n_jobs: int = 256, seed: int = 1004, n_lo: int = 12, n_hi: int = 20, dtype: str = "c64") -> List[Job]:
    """Uneven batch: TFIM open chains and periodic Heisenberg chains (50/50),
    n ~ U{n_lo..n_hi}, J ~ U[0.5,1.5], h ~ U[0,2], steps ~ U{20..200},
    budget ~ U{4..16}, Gaussian states, t=1."""
    rng = np.random.default_rng(seed)
    jobs = []
    for _ in range(n_jobs):
        fam = "tfim" if rng.uniform() < 0.5 else "heisenberg"
        n = int(rng.integers(n_lo, n_hi + 1))
        steps = int(rng.integers(20, 201))
        budget = int(rng.integers(4, 17))
        if fam == "tfim":
            ham = tfim_chain(n, float(rng.uniform(0.5, 1.5)), float(rng.uniform(0.0, 2.0)), periodic=False)
        else:
            ham = heisenberg_chain(n, rng.uniform(0.5, 1.5, size=n), periodic=True)
        jobs.append(Job(ham, 1.0, steps, budget, gaussian_state(n, rng), dtype))
    return jobs


FAMILY_BUDGET = {"tfim": 4, "heisenberg": 8, "maxcut": 4, "tsp": 1}


def serve_stream(rate: float = 500.0, duration: float = 20.0, seed: int = 1005,
                 n_lo: int = 12, n_hi: int = 24, max_jobs: Optional[int] = None) -> List[Job]:
    """Poisson request stream mixing TFIM, Heisenberg, MaxCut and one-hot TSP
    (16 qubits).  n ~ U{n_lo..n_hi} (TSP fixed at 16), t ~ U[0.5,2],
    steps ~ U{10..100}, complex64, per-family default budgets."""
    rng = np.random.default_rng(seed)
    jobs = []
    tnow = 0.0
    while True:
        tnow += float(rng.exponential(1.0 / rate))
        if tnow >= duration or (max_jobs is not None and len(jobs) >= max_jobs):
            break
        fam = ["tfim", "heisenberg", "maxcut", "tsp"][int(rng.integers(0, 4))]
        n = int(rng.integers(n_lo, n_hi + 1))
        if fam == "tfim":
            ham = tfim_chain(n, float(rng.uniform(0.5, 1.5)), float(rng.uniform(0.0, 2.0)), periodic=False)
        elif fam == "heisenberg":
            ham = heisenberg_chain(n, rng.uniform(0.5, 1.5, size=n), periodic=True)
        elif fam == "maxcut":
            n = n + (n % 2) if n + (n % 2) <= n_hi else n - 1  # a 3-regular graph needs an even n
            ham = maxcut_3regular(n, int(rng.integers(0, 2**31)), 0.5)
        else:
            ham = tsp_onehot(4, int(rng.integers(0, 2**31)))
            n = ham.n_qubits
        t = float(rng.uniform(0.5, 2.0))
        steps = int(rng.integers(10, 101))
        # the initial state is a seeded Gaussian made on the device when served
        jobs.append(Job(ham, t, steps, FAMILY_BUDGET[fam], None, "c64", arrival=tnow,
                        seed=int(rng.integers(0, 2**31))))
    return jobs
