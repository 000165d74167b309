"""The seeded input generators follow the recipes they state: node positions, masks of closed balls,
sampled Gaussian sources, sine-mode fields, material-like coefficient maps and batch problem
lists. Each is checked against a direct NumPy evaluation on a small grid, or against the bounds
and counts the recipe fixes. Same seed, same draw."""
import numpy as np
import torch

from paper_1904_03057_gb300 import inputs


def _grid(nx, ny, nz, h):
    hs = (h, h, h) if np.isscalar(h) else h
    x = np.arange(1, nx + 1) * hs[0]
    y = np.arange(1, ny + 1) * hs[1]
    z = np.arange(1, nz + 1) * hs[2]
    return np.meshgrid(z, y, x, indexing="ij")


def test_node_coordinates():
    assert np.allclose(inputs.node_coords(4).numpy(), [0.2, 0.4, 0.6, 0.8], rtol=0, atol=1e-15)
    assert np.allclose(inputs.node_coords(3, h=0.1).numpy(), [0.1, 0.2, 0.3], rtol=0, atol=1e-15)


def test_sphere_masks_are_closed_balls():
    nx, ny, nz = 11, 9, 13
    Z, Y, X = _grid(nx, ny, nz, (1 / 12, 1 / 10, 1 / 14))
    ref = ((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2 <= 0.45 ** 2)
    assert np.array_equal(inputs.sphere_mask(nx, ny, nz).numpy().astype(bool), ref)
    centers, radii = inputs.random_spheres(5, count=6)
    ref = np.zeros_like(ref)
    for (cx, cy, cz), r in zip(centers, radii):
        ref |= (X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2 <= r * r
    assert np.array_equal(inputs.union_of_spheres_mask(nx, ny, nz, centers, radii).numpy().astype(bool), ref)


def test_random_spheres_recipe():
    centers, radii = inputs.random_spheres(5)
    assert len(centers) == len(radii) == 40
    for c, r in zip(centers, radii):
        assert 0.05 <= r <= 0.2
        assert all(r <= v <= 1 - r for v in c)
    assert inputs.random_spheres(5) == (centers, radii)
    assert inputs.random_spheres(6)[1] != radii


def test_gaussian_source_matches_direct_evaluation():
    nx, ny, nz, h = 10, 8, 12, 1 / 13
    cs = inputs.gaussian_centers(2, 5)
    assert all(0.2 <= v <= 0.8 for c in cs for v in c) and cs == inputs.gaussian_centers(2, 5)
    Z, Y, X = _grid(nx, ny, nz, h)
    ref = sum(np.exp(-((X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2) / (2 * 0.03 ** 2)) for cx, cy, cz in cs)
    g = inputs.gaussian_source(nx, ny, nz, cs, sigma=0.03, h=h).numpy()
    assert np.max(np.abs(g - ref)) <= 1e-14 * max(1.0, np.max(ref))
    mask = inputs.sphere_mask(nx, ny, nz, radius=0.3, h=h)
    gm = inputs.gaussian_source(nx, ny, nz, cs, sigma=0.03, h=h, mask=mask).numpy()
    assert np.array_equal(gm, np.where(mask.numpy() > 0, g, 0.0))


def test_sine_modes_recipe_and_field():
    modes = inputs.random_sine_modes(3)
    ks = [k for k, _ in modes]
    assert len(modes) == 64 and len(set(ks)) == 64
    assert all(1 <= v <= 16 for k in ks for v in k)
    assert modes == inputs.random_sine_modes(3)
    few = modes[:5]
    nx, ny, nz = 9, 7, 6
    Z, Y, X = _grid(nx, ny, nz, (1 / 10, 1 / 8, 1 / 7))
    ref = sum(a * np.sin(np.pi * k[0] * X) * np.sin(np.pi * k[1] * Y) * np.sin(np.pi * k[2] * Z) for k, a in few)
    f = inputs.sine_mode_field(nx, ny, nz, few).numpy()
    assert np.max(np.abs(f - ref)) <= 1e-14


def test_inclusion_coefficients_recipe():
    nx, ny, nz = 20, 18, 22
    d = inputs.inclusion_coefficients(nx, ny, nz, seed=7).numpy()
    assert d.shape == (nz + 2, ny + 2, nx + 2)
    vals = np.unique(d)
    inside = vals[vals != 1.0]
    assert inside.size >= 1 and np.all((inside >= 0.2) & (inside <= 5.0))
    assert np.max(d) / np.min(d) <= 25.0 + 1e-12
    assert np.array_equal(d, inputs.inclusion_coefficients(nx, ny, nz, seed=7).numpy())
    m = inputs.inclusion_coefficients(nx, ny, nz, seed=8, base=0.3).numpy()
    assert np.mean(m == 0.3) > 0.2                      # the background value
    assert np.all((m == 0.3) | ((m >= 0.2) & (m <= 5.0)))


def test_random_field_is_seeded_and_masked():
    mask = inputs.sphere_mask(6, 5, 4, radius=0.3)
    a = inputs.random_field((4, 5, 6), 9, mask=mask)
    assert torch.equal(a, inputs.random_field((4, 5, 6), 9, mask=mask))
    assert torch.all(a[mask == 0] == 0) and torch.any(a[mask > 0] != 0)


def test_batch_problem_recipe():
    probs = inputs.batch_problems()
    assert len(probs) == 64
    for p in probs:
        assert all(48 <= v <= 160 for v in (p.nx, p.ny, p.nz)) and p.degree in (2, 3, 4, 5)
        assert p.h == 1.0 / (max(p.nx, p.ny, p.nz) + 1) and len(p.centers) == 8
        ext = ((p.nx + 1) * p.h, (p.ny + 1) * p.h, (p.nz + 1) * p.h)
        assert all(0.2 * e <= c <= 0.8 * e for cc in p.centers for c, e in zip(cc, ext))
    assert {p.degree for p in probs} == {2, 3, 4, 5}
