"""Pins for the oracle's Eq. 4 (energy gradient): against a finite-difference derivative of
the variational energy <Psi|H|Psi>/<Psi|Psi> built from the dense Hamiltonian, and against
the invariants of the formula.  A dropped factor 2, a missing conjugate or a missing
centring (E_loc - <E>) breaks the first pin."""
import numpy as np

from paper_2506_23809_gb300 import inputs as I


def _log_linear_system(orc, seed=41, P=3):
    """N=8, 2+2 electrons, the whole 36-determinant sector.  Psi_n(theta) =
    Psi0_n exp(sum_p theta_p f_np) with complex features f, and |Psi0_n|^2 = k_n an integer,
    so the count-weighted sample average over the sector with counts k_n is the exact
    |Psi|^2-weighted expectation of Eq. 1 / Eq. 4 at theta = 0."""
    rng = np.random.default_rng(seed)
    ints = I.make_integrals(4, 8, seed)
    basis = orc.sector(8, 2, 2)
    n = basis.shape[0]
    k = rng.integers(1, 10, size=n)
    psi0 = np.sqrt(k) * np.exp(1j * rng.uniform(0, 2 * np.pi, n))
    f = rng.normal(size=(n, P)) + 1j * rng.normal(size=(n, P))
    H = orc.h_slater_condon(ints.h, ints.eri, 0.0, 8, basis)
    return ints, basis, k, psi0, f, H


def test_grad_matches_finite_difference_of_rayleigh_quotient(orc):
    ints, basis, k, psi0, f, H = _log_linear_system(orc)

    def energy(theta):
        psi = psi0 * np.exp(f @ theta)
        return float(np.real(np.vdot(psi, H @ psi)) / np.real(np.vdot(psi, psi)))

    eloc = orc.eloc(ints.h, ints.eri, 0.0, 8, basis, psi0)
    w, g = orc.grad(eloc, k, np.conj(f))       # d/d theta ln Psi* = conj(f)
    # the sample estimate of Eq. 1 at theta = 0 is the exact Rayleigh quotient here
    m, var, W, used = orc.reduce(eloc, k)
    assert abs(m.real - energy(np.zeros(f.shape[1]))) <= 1e-12 * abs(m.real) and abs(m.imag) <= 1e-12
    h = 1e-5
    for p in range(f.shape[1]):
        e = np.zeros(f.shape[1])
        e[p] = h
        fd = (energy(e) - energy(-e)) / (2 * h)
        assert abs(g[p] - fd) <= 1e-6 * max(1.0, abs(fd)), (p, g[p], fd)
    # the weights are centred: they sum to zero
    assert abs(w.sum()) <= 1e-14 * np.abs(w).sum()


def test_grad_of_constant_rows_is_zero_and_excluded_samples(orc):
    rng = np.random.default_rng(7)
    n, P = 50, 4
    e = rng.normal(size=n) + 1j * rng.normal(size=n)
    c = rng.integers(1, 20, size=n)
    row = rng.normal(size=P) + 1j * rng.normal(size=P)
    _, g = orc.grad(e, c, np.tile(row, (n, 1)))
    assert np.abs(g).max() <= 1e-12 * np.abs(row).max() * np.abs(e).max()
    # a non-finite E_loc gets weight 0 and leaves the mean and W of the others
    e2 = e.copy()
    e2[3] = np.nan
    w2, _ = orc.grad(e2, c)
    keep = np.arange(n) != 3
    W = c[keep].sum()
    mean = (c[keep] * e[keep]).sum() / W
    assert w2[3] == 0
    assert np.allclose(w2[keep], c[keep] * (e[keep] - mean) / W, rtol=0, atol=1e-15)
