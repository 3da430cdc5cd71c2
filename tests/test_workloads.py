"""The seeded synthetic inputs carry the structure their recipes state:
permittivity fields positive with the stated log statistics, charges where
and how many the recipe puts them, the batched set's sizes and ragged counts,
and the same numbers for the same seed.  CPU only."""
import numpy as np

from paper_1602_00001_gb300 import workloads as W


def test_eps_fourier_is_smooth_lognormal_unit_std():
    nx = ny = 100
    h = 1.0 / 99
    e = W.eps_fourier(nx, ny, h, seed=1)
    g = np.log(e) / 0.5
    assert np.all(e > 0)
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1.0) < 1e-12
    # smooth: neighbouring nodes differ by a small fraction of the field's spread
    assert np.max(np.abs(np.diff(g, axis=1))) < 0.5 and np.max(np.abs(np.diff(g, axis=0))) < 0.5
    assert np.array_equal(e, W.eps_fourier(nx, ny, h, seed=1))
    assert not np.array_equal(e, W.eps_fourier(nx, ny, h, seed=2))


def test_eps_lognormal_is_rough_with_sigma_half():
    e = W.eps_lognormal(200, 200, seed=4)
    z = np.log(e) / 0.5
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1.0) < 0.02
    # i.i.d.: neighbouring values uncorrelated
    assert abs(np.corrcoef(z[:, :-1].ravel(), z[:, 1:].ravel())[0, 1]) < 0.02


def test_gaussian_blobs_sit_inside_the_central_square():
    nx = ny = 81
    h = 1.0 / 80
    rho = W.gaussian_blobs(nx, ny, h, seed=0, batch=50)
    assert rho.shape == (50, 79 * 79)
    for col in rho:
        p = int(np.argmax(np.abs(col)))
        i, j = divmod(p, 79)
        x, y = h * (j + 1), h * (i + 1)
        # the largest |rho| lies within a blob width or two of [0.2, 0.8]^2
        assert 0.1 < x < 0.9 and 0.1 < y < 0.9


def test_moving_charges_are_continuous_in_time():
    nx = ny = 60
    h = 1.0 / 59
    rho = W.moving_charges(nx, ny, h, seed=5, steps=256)
    assert rho.shape == (256, 58 * 58)
    step = np.abs(np.diff(rho, axis=0)).max(axis=1)
    assert np.max(step) < 0.5 * np.abs(rho).max()        # small moves between steps
    assert np.array_equal(rho[:16], W.moving_charges(nx, ny, h, seed=5, steps=256)[:16])


def test_batched_problem_set_sizes_and_counts():
    probs = W.batched_problem_set(seed=3, nprob=64)
    assert len(probs) == 64
    sides = [p[0] for p in probs]
    assert set(sides) <= {32, 48, 64, 96, 128} and len(set(sides)) >= 4
    for side, eps, rho in probs:
        assert eps.shape == (side, side) and np.all(eps > 0)
        assert 1 <= rho.shape[0] <= 64 and rho.shape[1] == (side - 2) ** 2
    Bs = [p[2].shape[0] for p in probs]
    assert min(Bs) < 16 and max(Bs) > 48                 # ragged over 1..64
    again = W.batched_problem_set(seed=3, nprob=64)
    assert all(np.array_equal(a[2], b[2]) for a, b in zip(probs[:4], again[:4]))
