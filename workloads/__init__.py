"""Seeded synthetic inputs for the SP2 density / response / susceptibility path.

This module only draws numbers and lays them out as matrices. It holds none of
the method's arithmetic (no spectral bounds, no recursion, no traces), so the
oracle and the CUDA path can both consume its output without sharing any of
the computation they are checked on.

All generators use ``numpy.random.default_rng(seed)`` (PCG64) and draw in the
order documented in each function, so a (config, seed) pair always yields the
same matrices on every machine.

Workloads (the problem statement is the paper's Sec. II: a real symmetric
N x N Hamiltonian H with S = I and an occupation N_occ; perturbations H1 and
observables A are real symmetric N x N matrices, Sec. III and IV):

* ``random_spectrum``: H = Q diag(e) Q^T with Q Haar-orthogonal and a gapped
  two-band spectrum; A and H1_k symmetric Gaussian with sigma = 1/sqrt(N).
* ``tight_binding``: sites at random positions in a periodic cube of number
  density 0.1, 4 orbitals per site, hopping -exp(-r/1.5) for r < 6 between
  every orbital pair of two distinct sites, onsite U[-0.3, 0.3] plus an
  alternating +/-0.8 shift that opens a gap at half filling.
* ``metallic_spectrum``: H = Q diag(e) Q^T with e ~ U[-1, 1] (gapless), for
  the finite-temperature variant.
* ``nonorth_problem``: an overlap S = L L^T from a drawn unit lower-triangular
  L and H = L (Q diag(e) Q^T) L^T, so the generalized spectrum of (H, S) is the
  gapped e; observable and basis-set dependent perturbations (A_t, H_t, S_t).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "haar_orthogonal",
    "sym_gaussian",
    "RandomSpectrumProblem",
    "random_spectrum",
    "TightBinding",
    "tight_binding",
    "tb_dipole_observables",
    "tb_site_potentials",
    "metallic_spectrum",
    "NonOrthProblem",
    "nonorth_problem",
]


def haar_orthogonal(rng: np.random.Generator, n: int) -> np.ndarray:
    """Haar-distributed orthogonal n x n matrix: QR of an iid N(0,1) matrix,
    with the columns' signs fixed by sign(diag R) so the law is exactly Haar.
    Draws n*n normals (row-major)."""
    g = rng.standard_normal((n, n))
    q, r = np.linalg.qr(g)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s[None, :]


def sym_gaussian(rng: np.random.Generator, n: int, sigma: float) -> np.ndarray:
    """Symmetric matrix whose upper triangle (diagonal included) is iid
    N(0, sigma^2), mirrored. Draws n*n normals row-major and keeps the upper
    triangle, so the draw count does not depend on the layout."""
    g = rng.standard_normal((n, n)) * sigma
    u = np.triu(g)
    return u + np.triu(u, 1).T


@dataclasses.dataclass
class RandomSpectrumProblem:
    H: np.ndarray          # (N, N) float64, symmetric
    Q: np.ndarray          # (N, N) eigenvectors (columns)
    e: np.ndarray          # (N,) eigenvalues, H = Q diag(e) Q^T
    A: np.ndarray          # (N, N) observable
    H1: np.ndarray         # (K, N, N) perturbations
    nocc: int


def random_spectrum(n: int = 128, nocc: int | None = None, k: int = 8,
                    lo=(-1.0, -0.2), hi=(0.2, 1.0), seed: int = 0) -> RandomSpectrumProblem:
    """Gapped random-spectrum problem.

    Draw order: Q (n*n normals), then nocc eigenvalues U[lo], then n-nocc
    eigenvalues U[hi], then A (n*n normals), then H1_k for k = 0..K-1
    (n*n normals each). sigma = 1/sqrt(n) for A and H1_k."""
    if nocc is None:
        nocc = n // 2
    rng = np.random.default_rng(seed)
    q = haar_orthogonal(rng, n)
    e = np.concatenate([rng.uniform(lo[0], lo[1], nocc),
                        rng.uniform(hi[0], hi[1], n - nocc)])
    h = (q * e[None, :]) @ q.T
    h = 0.5 * (h + h.T)
    sig = 1.0 / math.sqrt(n)
    a = sym_gaussian(rng, n, sig)
    h1 = np.stack([sym_gaussian(rng, n, sig) for _ in range(k)]) if k else np.zeros((0, n, n))
    return RandomSpectrumProblem(H=h, Q=q, e=e, A=a, H1=h1, nocc=nocc)


@dataclasses.dataclass
class TightBinding:
    H: np.ndarray          # (N, N) float64
    pos: np.ndarray        # (n_sites, 3) site positions in [0, L)^3
    box: float             # cube edge L
    norb: int              # orbitals per site
    nocc: int

    @property
    def n(self) -> int:
        return self.H.shape[0]


def _tb_hopping(pos: np.ndarray, box: float, rcut: float, decay: float,
                norb: int, out: np.ndarray) -> None:
    """Adds -exp(-r/decay) to every orbital pair of every pair of distinct
    sites closer than rcut (minimum-image distance in the periodic box; box is
    the cube edge or the three box edges)."""
    ns = pos.shape[0]
    chunk = 512
    for s0 in range(0, ns, chunk):
        s1 = min(ns, s0 + chunk)
        d = pos[s0:s1, None, :] - pos[None, :, :]
        d -= box * np.round(d / box)
        r = np.sqrt(np.einsum("ijk,ijk->ij", d, d))
        for ia in range(s1 - s0):
            a = s0 + ia
            nb = np.nonzero((r[ia] < rcut))[0]
            nb = nb[nb != a]
            if nb.size == 0:
                continue
            t = -np.exp(-r[ia, nb] / decay)
            rows = slice(a * norb, (a + 1) * norb)
            blk = np.repeat(t, norb)[None, :]           # (1, nb*norb)
            cols = (nb[:, None] * norb + np.arange(norb)[None, :]).reshape(-1)
            out[rows, cols] += blk


def tight_binding(n: int, seed: int = 0, norb: int = 4, density: float = 0.1,
                  rcut: float = 6.0, decay: float = 1.5, onsite: float = 0.3,
                  stagger: float = 0.8, dtype=np.float64) -> TightBinding:
    """Dense-stored tight-binding Hamiltonian.

    n_sites = n / norb sites at positions U[0, L)^3 with L = (n_sites/density)^(1/3).
    Draw order: positions (n_sites*3 uniforms, row-major), then onsite energies
    (n uniforms, one per orbital). Orbital g (global index) gets
    U[-onsite, onsite] + stagger * (-1)^g on the diagonal. N_occ = n / 2."""
    assert n % norb == 0
    ns = n // norb
    rng = np.random.default_rng(seed)
    box = (ns / density) ** (1.0 / 3.0)
    pos = rng.uniform(0.0, box, (ns, 3))
    eps = rng.uniform(-onsite, onsite, n) + stagger * np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    h = np.zeros((n, n), dtype=dtype)
    _tb_hopping(pos, box, rcut, decay, norb, h)
    h[np.arange(n), np.arange(n)] += eps
    return TightBinding(H=h, pos=pos, box=box, norb=norb, nocc=n // 2)


def tight_binding_rod(n: int, seed: int = 0, norb: int = 4, density: float = 0.1,
                      width: float = 6.0, rcut: float = 6.0, decay: float = 1.5,
                      onsite: float = 0.3, stagger: float = 2.0,
                      dtype=np.float64) -> TightBinding:
    """Dense-stored tight-binding Hamiltonian of a long periodic rod: the stand-in
    for the large non-metallic systems where thresholded sparse algebra pays.

    n_sites = n / norb sites uniform in [0, L) x [0, width)^2 with
    L = n_sites / (density * width^2), periodic in all three directions, then
    sorted by their coordinate along the rod, so that orbital blocks are
    spatially local. Draw order: positions (n_sites*3 uniforms, row-major,
    scaled to the box), then onsite energies (n uniforms). Hopping and onsite
    terms as in tight_binding; the stagger (default 2.0) opens a gap of about
    0.95 at n = 4096. N_occ = n / 2."""
    assert n % norb == 0
    ns = n // norb
    rng = np.random.default_rng(seed)
    box = np.array([ns / (density * width * width), width, width])
    pos = rng.uniform(0.0, 1.0, (ns, 3)) * box
    pos = pos[np.argsort(pos[:, 0], kind="stable")]
    eps = rng.uniform(-onsite, onsite, n) + stagger * np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    h = np.zeros((n, n), dtype=dtype)
    _tb_hopping(pos, box, rcut, decay, norb, h)
    h[np.arange(n), np.arange(n)] += eps
    return TightBinding(H=h, pos=pos, box=float(box[0]), norb=norb, nocc=n // 2)


def tb_dipole_observables(tb: TightBinding) -> np.ndarray:
    """Four diagonal observables (returned as their diagonals, shape (4, N)):
    the x, y, z coordinates of each orbital's site relative to the box centre
    (dipole-like), and the population of site 0 (indicator of its orbitals)."""
    n = tb.n
    c = np.repeat(tb.pos - 0.5 * tb.box, tb.norb, axis=0)      # (N, 3)
    pop = np.zeros(n)
    pop[:tb.norb] = 1.0
    return np.stack([c[:, 0], c[:, 1], c[:, 2], pop])


def tb_site_potentials(tb: TightBinding, k: int, seed: int = 1) -> np.ndarray:
    """K random site-potential perturbations, returned as diagonals (K, N):
    each site's potential is U[-1, 1], shared by its orbitals. Draw order:
    K * n_sites uniforms, row-major."""
    rng = np.random.default_rng(seed)
    v = rng.uniform(-1.0, 1.0, (k, tb.n // tb.norb))
    return np.repeat(v, tb.norb, axis=1)


def metallic_spectrum(n: int = 8192, k: int = 256, seed: int = 0) -> RandomSpectrumProblem:
    """Gapless problem: e ~ U[-1, 1], Haar Q, A and H1_k symmetric
    N(0, 1/n). Draw order: Q, e (n uniforms), A, H1_k. nocc is n/2 (a
    nominal count; the finite-temperature variant fixes mu = 0)."""
    rng = np.random.default_rng(seed)
    q = haar_orthogonal(rng, n)
    e = rng.uniform(-1.0, 1.0, n)
    h = (q * e[None, :]) @ q.T
    h = 0.5 * (h + h.T)
    sig = 1.0 / math.sqrt(n)
    a = sym_gaussian(rng, n, sig)
    h1 = np.stack([sym_gaussian(rng, n, sig) for _ in range(k)]) if k else np.zeros((0, n, n))
    return RandomSpectrumProblem(H=h, Q=q, e=e, A=a, H1=h1, nocc=n // 2)


def site_kernel(tb: TightBinding, kind: str = "regularised") -> np.ndarray:
    """Site-site interaction kernel K (n_sites x n_sites) of the
    self-consistent response workload, from minimum-image distances r_ab:
    'literal':     K_ab = 1 on the diagonal, 1 / r_ab off it;
    'regularised': K_ab = 1 / sqrt(r_ab^2 + 1) (same diagonal, positive definite)."""
    p = tb.pos
    d = p[:, None, :] - p[None, :, :]
    d -= tb.box * np.round(d / tb.box)
    r = np.sqrt(np.einsum("ijk,ijk->ij", d, d))
    if kind == "literal":
        with np.errstate(divide="ignore"):
            K = np.where(np.eye(len(p), dtype=bool), 1.0, 1.0 / np.where(r > 0, r, 1.0))
        return K
    return 1.0 / np.sqrt(r * r + 1.0)


def site_fields(tb: TightBinding, f: int, sigma: float = 0.1, seed: int = 2) -> np.ndarray:
    """F external site potentials V_ext ~ N(0, sigma^2), shape (F, n_sites).
    Draw order: F * n_sites normals, row-major."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((f, tb.n // tb.norb)) * sigma


@dataclasses.dataclass
class NonOrthProblem:
    H: np.ndarray          # (N, N) symmetric, atomic-orbital representation
    S: np.ndarray          # (N, N) symmetric positive definite overlap
    A: np.ndarray          # (N, N) observable
    A_t: np.ndarray        # (K, N, N) derivatives of A along K perturbations
    H_t: np.ndarray        # (K, N, N) derivatives of H
    S_t: np.ndarray        # (K, N, N) derivatives of S
    e: np.ndarray          # (N,) generalized eigenvalues of (H, S)
    nocc: int


def nonorth_problem(n: int = 128, nocc: int | None = None, k: int = 3, overlap: float = 0.5,
                    seed: int = 0) -> NonOrthProblem:
    """Gapped generalized problem with a non-trivial overlap.

    Draw order: Q (n*n normals), nocc eigenvalues U[-1, -0.2], n - nocc
    eigenvalues U[0.2, 1], the lower triangle of L (n*n normals, strictly lower
    part scaled by overlap / sqrt(n), unit diagonal), A (n*n normals), then for
    each of the k perturbations A_t, H_t, S_t (n*n normals each). Symmetric
    draws use ``sym_gaussian`` with sigma = 1/sqrt(n)."""
    if nocc is None:
        nocc = n // 2
    rng = np.random.default_rng(seed)
    q = haar_orthogonal(rng, n)
    e = np.concatenate([rng.uniform(-1.0, -0.2, nocc), rng.uniform(0.2, 1.0, n - nocc)])
    lo = np.tril(rng.standard_normal((n, n)), -1) * (overlap / math.sqrt(n))
    L = lo + np.eye(n)
    hp = (q * e[None, :]) @ q.T
    h = L @ hp @ L.T
    h = 0.5 * (h + h.T)
    S = L @ L.T
    S = 0.5 * (S + S.T)
    sig = 1.0 / math.sqrt(n)
    a = sym_gaussian(rng, n, sig)
    at, ht, st = [], [], []
    for _ in range(k):
        at.append(sym_gaussian(rng, n, sig))
        ht.append(sym_gaussian(rng, n, sig))
        st.append(sym_gaussian(rng, n, sig))
    return NonOrthProblem(H=h, S=S, A=a, A_t=np.array(at), H_t=np.array(ht), S_t=np.array(st),
                          e=e, nocc=nocc)
