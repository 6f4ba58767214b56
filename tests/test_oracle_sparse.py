"""Pins for the thresholded block-sparse SP2 oracle (oracle/sparse.py; CPU only).

Checked against things other than the function itself: the dense recursion
(tau = 0 must reproduce it), the exact projector from an eigendecomposition,
the exact block structure of decoupled subsystems, and the monotone approach
to the exact projector as tau falls on a gapped local chain.
"""
import numpy as np
import pytest

import workloads
from oracle import exact, sp2, sparse


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def chain(n, gap=1.0, t=1.0, seed=0):
    """Gapped 1D chain: staggered onsite +-gap/2 plus a small disorder, nearest-
    neighbour hopping -t. Its density matrix decays exponentially along the chain."""
    rng = np.random.default_rng(seed)
    H = np.diag(0.5 * gap * (-1.0) ** np.arange(n) + 0.05 * rng.standard_normal(n))
    i = np.arange(n - 1)
    H[i, i + 1] = H[i + 1, i] = -t
    return H


def test_block_norms_and_threshold_on_a_ragged_grid():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((21, 21))
    X = X + X.T
    nrm = sparse.block_norms(X, 8)                  # blocks of 8, 8, 5
    assert nrm.shape == (3, 3)
    assert np.isclose(nrm[2, 1], np.linalg.norm(X[16:21, 8:16]))
    assert np.isclose(nrm[0, 0], np.linalg.norm(X[:8, :8]))
    tau = float(np.median(nrm))
    Y, keep = sparse.threshold_blocks(X, tau, 8)
    for i in range(3):
        for j in range(3):
            blk = Y[i * 8:(i + 1) * 8, j * 8:(j + 1) * 8]
            if i == j or nrm[i, j] > tau:
                assert keep[i, j] and np.array_equal(blk, X[i * 8:(i + 1) * 8, j * 8:(j + 1) * 8])
            else:
                assert not keep[i, j] and not blk.any()
    # diagonal blocks stay even when they are the smallest
    Z = X.copy()
    Z[:8, :8] *= 1e-9
    Yz, kz = sparse.threshold_blocks(Z, 1.0, 8)
    assert kz[0, 0] and np.array_equal(Yz[:8, :8], Z[:8, :8])


def test_tau_zero_reproduces_the_dense_recursion():
    p = workloads.random_spectrum(96, nocc=40, k=1, seed=2)
    d = sp2.sp2_density(p.H, p.nocc)
    s = sparse.sp2_density_thresholded(p.H, p.nocc, 0.0, block=16)
    assert s.sigma == d.sigma and s.M == d.M
    assert rel(s.D, d.D) < 1e-12
    assert np.allclose(s.errors, d.errors, rtol=1e-9, atol=1e-12)
    assert all(m.all() for m in s.masks)           # a dense H keeps every block


def test_decoupled_subsystems_keep_exact_zero_blocks():
    """Two subsystems that do not couple: every iterate is block diagonal at
    the 2x2 block level, tau = 0 skips the coupling blocks exactly, and the
    result is the exact projector of the whole H."""
    rng = np.random.default_rng(4)
    A = workloads.sym_gaussian(rng, 32, 1.0)
    B = workloads.sym_gaussian(rng, 32, 1.0) + 0.3 * np.eye(32)
    H = np.zeros((64, 64))
    H[:32, :32] = A
    H[32:, 32:] = B
    s = sparse.sp2_density_thresholded(H, 30, 0.0, block=16)
    expect = np.kron(np.eye(2, dtype=bool), np.ones((2, 2), dtype=bool))
    for m in s.masks:
        assert np.array_equal(m, expect)
    assert not s.D[:32, 32:].any()
    e, V = exact.eigh(H)
    assert rel(s.D, exact.density_zero_T(e, V, 30)) < 1e-8
    assert sparse.block_fill(s.masks) == pytest.approx(6 / 10)


def test_threshold_floor_stops_where_the_dense_rules_do_not():
    """tau = 1e-2 on the chain: f settles near 1e-7 and creeps down, so neither a
    rise nor a four-step stall ever shows; without the ratio test the run takes
    all max_iter steps."""
    H = chain(256, gap=1.5)
    s = sparse.sp2_density_thresholded(H, 128, 1e-2, block=16)
    assert s.converged and s.M < 20
    saved = sparse.RATIO_GATE
    try:
        sparse.RATIO_GATE = 0.0        # disables the ratio test
        t = sparse.sp2_density_thresholded(H, 128, 1e-2, block=16, max_iter=60)
    finally:
        sparse.RATIO_GATE = saved
    assert not t.converged and t.M == 60
    # the ratio test returned an iterate as good as the long run's last one
    e, V = exact.eigh(H)
    D = exact.density_zero_T(e, V, 128)
    assert rel(s.D, D) < 1.5 * rel(t.D, D)


def test_thresholded_chain_approaches_the_exact_projector():
    n, nocc = 256, 128
    H = chain(n, gap=1.5)
    e, V = exact.eigh(H)
    D = exact.density_zero_T(e, V, nocc)
    errs, fills = [], []
    for tau in (1e-2, 1e-4, 1e-6, 1e-9):
        s = sparse.sp2_density_thresholded(H, nocc, tau, block=16)
        assert s.converged and s.M < 30
        if tau >= 1e-4:
            # on the threshold's floor f creeps down: only the ratio test stops the run
            d = sp2.sp2_density(H, nocc, max_iter=30)
            assert d.M < s.M + 3   # the dense run converges in a similar number of steps
            assert s.fro[-1] > 1e-12
        errs.append(rel(s.D, D))
        fills.append(sparse.block_fill(s.masks))
        # every off-diagonal block of the result is either above tau or zero
        nrm = sparse.block_norms(s.D, 16)
        off = ~np.eye(nrm.shape[0], dtype=bool)
        assert np.all((nrm[off] > tau) | (nrm[off] == 0.0))
        assert abs(np.trace(s.D) - nocc) < 1e-3 + 10 * tau * n
    assert errs == sorted(errs, reverse=True) and errs[-1] < 1e-7
    assert fills == sorted(fills) and fills[0] < 0.5
