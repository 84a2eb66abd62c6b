"""The seeded synthetic workloads (inputs.py): shapes, seeds and the statistics the
recipes state.  These hold no arithmetic of the method; they pin the inputs that the
oracle and the CUDA path both consume."""
import numpy as np

from paper_1703_06323_gb300 import inputs


def _rff_direct(cells, seed=0, sigma=1.0, ell=0.1, n_features=1024):
    """The random-Fourier-feature field summed feature by feature at every cell centre
    (the definition the separable evaluation must reproduce)."""
    rng = np.random.default_rng(seed + 7919)
    w = rng.normal(scale=1.0 / ell, size=(n_features, 3))
    b = rng.uniform(0.0, 2.0 * np.pi, n_features)
    a = rng.normal(size=n_features)
    X, Y, Z = inputs.cell_centres((0, 0, 0), (1, 1, 1), cells)
    g = np.cos(np.stack([X, Y, Z], axis=1) @ w.T + b) @ a
    return g * sigma * np.sqrt(2.0 / n_features)


def test_random_field_matches_the_feature_sum():
    for cells in [(8, 6, 4), (16, 16, 16), (5, 9, 7)]:
        k = inputs.random_field_kappa(cells, seed=3)
        assert k.shape == (np.prod(cells),)
        assert np.abs(np.log(k) - _rff_direct(cells, seed=3)).max() <= 1e-13


def test_random_field_statistics():
    """sigma = 1 log-normal field: log kappa has mean ~0 and standard deviation ~1
    over a grid much larger than the correlation length; neighbouring cells are
    strongly correlated (correlation length 0.1 = 6.4 cells at 64^3)."""
    g = np.log(inputs.random_field_kappa((64, 64, 64), seed=0)).reshape(64, 64, 64)
    assert abs(g.mean()) < 0.2 and 0.8 < g.std() < 1.2
    c = np.corrcoef(g[:, :, :-1].ravel(), g[:, :, 1:].ravel())[0, 1]
    assert 0.9 < c < 1.0


def test_coefficient_sphere_and_bumpy_sphere_are_seeded():
    p1 = inputs.coefficient_sphere(seed=1, n=16)
    p2 = inputs.coefficient_sphere(seed=1, n=16)
    p3 = inputs.coefficient_sphere(seed=2, n=16)
    assert np.array_equal(p1.kappa, p2.kappa) and not np.array_equal(p1.kappa, p3.kappa)
    assert p1.kappa.shape == (16 ** 3,) and p1.phi.shape == (17 ** 3,)
    b1, b2 = inputs.bumpy_sphere(0), inputs.bumpy_sphere(0)
    assert np.array_equal(b1.phi, b2.phi) and np.array_equal(b1.f, b2.f)
    assert b1.cells == (64, 64, 64) and b1.sub_cells == (8, 8, 8)
    assert np.abs(b1.f).max() <= 1.0
