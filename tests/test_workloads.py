"""The seeded input generators follow the stated input recipe (CPU only): the
spectra, symmetry and scales of the random-spectrum problems, the form of the
tight-binding Hamiltonians (hopping -exp(-r/1.5) for r < 6 between distinct
sites, no intra-site hopping, onsite U[-0.3, 0.3] plus the alternating stagger),
the diagonal observables and perturbations, the site kernels, and
reproducibility by seed. Every parity test and the benchmark draw from these
generators, so a drift here would move every number downstream."""
import numpy as np
import pytest

import workloads


def test_haar_orthogonal_is_orthogonal():
    q = workloads.haar_orthogonal(np.random.default_rng(3), 64)
    assert np.allclose(q.T @ q, np.eye(64), atol=1e-12)


def test_sym_gaussian_is_symmetric_with_the_stated_scale():
    n = 256
    g = workloads.sym_gaussian(np.random.default_rng(4), n, 1.0 / np.sqrt(n))
    assert np.array_equal(g, g.T)
    iu = np.triu_indices(n)
    assert np.var(g[iu]) * n == pytest.approx(1.0, rel=0.05)


def test_random_spectrum_is_the_gapped_two_band_problem():
    p = workloads.random_spectrum(128, nocc=64, k=3, seed=0)
    assert np.allclose(p.H, (p.Q * p.e[None, :]) @ p.Q.T, atol=1e-12)
    assert np.array_equal(p.H, p.H.T)
    assert np.all((p.e[:64] >= -1.0) & (p.e[:64] <= -0.2))
    assert np.all((p.e[64:] >= 0.2) & (p.e[64:] <= 1.0))
    assert np.allclose(np.sort(np.linalg.eigvalsh(p.H)), np.sort(p.e), atol=1e-12)
    assert p.A.shape == (128, 128) and p.H1.shape == (3, 128, 128)
    assert np.array_equal(p.A, p.A.T) and all(np.array_equal(h, h.T) for h in p.H1)


def test_generators_are_reproducible_by_seed():
    a = workloads.random_spectrum(64, k=2, seed=5)
    b = workloads.random_spectrum(64, k=2, seed=5)
    c = workloads.random_spectrum(64, k=2, seed=6)
    assert np.array_equal(a.H, b.H) and np.array_equal(a.H1, b.H1)
    assert not np.array_equal(a.H, c.H)
    t1 = workloads.tight_binding(256, seed=1)
    t2 = workloads.tight_binding(256, seed=1)
    assert np.array_equal(t1.H, t2.H) and np.array_equal(t1.pos, t2.pos)


@pytest.mark.parametrize("rod", [False, True])
def test_tight_binding_has_the_stated_form(rod):
    n, norb = 512, 4
    tb = (workloads.tight_binding_rod(n, seed=0) if rod else workloads.tight_binding(n, seed=0))
    H = tb.H
    assert np.array_equal(H, H.T) and tb.nocc == n // 2 and tb.norb == norb
    stagger = 2.0 if rod else 0.8
    d = np.diag(H) - stagger * np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    assert np.all(np.abs(d) <= 0.3)
    # no hopping inside a site
    for s in range(n // norb):
        blk = H[s * norb:(s + 1) * norb, s * norb:(s + 1) * norb]
        assert np.count_nonzero(blk - np.diag(np.diag(blk))) == 0
    # between two sites, every orbital pair carries the same -exp(-r/1.5), r < 6
    box = np.array([tb.box, 6.0, 6.0]) if rod else tb.box
    rng = np.random.default_rng(9)
    for _ in range(200):
        a, b = rng.choice(n // norb, 2, replace=False)
        dv = tb.pos[a] - tb.pos[b]
        dv -= box * np.round(dv / box)
        r = float(np.sqrt(dv @ dv))
        blk = H[a * norb:(a + 1) * norb, b * norb:(b + 1) * norb]
        want = -np.exp(-r / 1.5) if r < 6.0 else 0.0
        assert np.allclose(blk, want, atol=1e-14)


def test_tight_binding_box_holds_the_stated_density():
    tb = workloads.tight_binding(4096, seed=0)
    ns = 4096 // 4
    assert tb.box ** 3 * 0.1 == pytest.approx(ns)
    assert np.all((tb.pos >= 0.0) & (tb.pos < tb.box))


def test_observables_and_site_potentials():
    tb = workloads.tight_binding(256, seed=0)
    A = workloads.tb_dipole_observables(tb)
    assert A.shape == (4, 256)
    # the dipole diagonals are each orbital's site coordinate about the box centre
    assert np.allclose(A[0], np.repeat(tb.pos[:, 0] - 0.5 * tb.box, 4))
    assert np.array_equal(A[3][:4], np.ones(4)) and np.count_nonzero(A[3]) == 4
    v = workloads.tb_site_potentials(tb, 5, seed=1)
    assert v.shape == (5, 256) and np.all(np.abs(v) <= 1.0)
    assert np.array_equal(v[:, 0::4], v[:, 3::4])   # one potential per site, shared by its orbitals


def test_site_kernels():
    tb = workloads.tight_binding(512, seed=0)
    K = workloads.site_kernel(tb, "regularised")
    assert np.allclose(np.diag(K), 1.0) and np.array_equal(K, K.T)
    assert np.linalg.eigvalsh(K).min() > 0.0          # positive definite (the reading taken)
    L = workloads.site_kernel(tb, "literal")
    assert np.allclose(np.diag(L), 1.0)
    off = ~np.eye(K.shape[0], dtype=bool)
    # literal 1/r and regularised 1/sqrt(r^2 + 1) describe the same distances
    assert np.allclose(1.0 / L[off] ** 2 + 1.0, 1.0 / K[off] ** 2)


def test_metallic_spectrum_is_gapless_uniform():
    p = workloads.metallic_spectrum(256, k=1, seed=0)
    assert np.all((p.e >= -1.0) & (p.e <= 1.0))
    assert np.allclose(np.sort(np.linalg.eigvalsh(p.H)), np.sort(p.e), atol=1e-12)
    # no gap: the largest spacing of 256 uniform draws is far below the band width
    assert np.max(np.diff(np.sort(p.e))) < 0.2
