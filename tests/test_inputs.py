"""The seeded input generators (meshgen) used by the benchmark's side legs: the Voronoi grains of
any mesh reduce, on the 3D-periodic cube, to the granular cell the local-term parity tests use."""
import numpy as np

import meshgen


def test_voronoi_grains_reduce_to_the_granular_cell_on_the_periodic_cube():
    mesh, gr = meshgen.granular_cell(n=8, grains=6, seed=2)
    v = meshgen.voronoi_grains(mesh, 6, 1e-9, seed=2)
    assert np.array_equal(v.tet_grain, gr.tet_grain)
    assert np.array_equal(v.A_tet, gr.A_tet)
    assert np.allclose(v.axes, gr.axes, rtol=0, atol=0) and np.allclose(v.u, gr.u, rtol=0, atol=0)


def test_voronoi_grains_see_seeds_through_the_period():
    # a 1D-periodic prism: a tetrahedron near the top face belongs to the seed nearest to it
    # across the period when that image is the nearest point of all
    mesh = meshgen.prism_cell(4, 4, 16, jitter=0.1, seed=1)
    v = meshgen.voronoi_grains(mesh, 5, 1e-9, seed=4)
    rng = np.random.default_rng(4 + 101)
    lo, hi = mesh.xyz.min(axis=0), mesh.xyz.max(axis=0)
    seeds = lo + rng.uniform(0, 1, size=(5, 3)) * (hi - lo)
    cen = mesh.xyz[mesh.tets].mean(axis=1)
    L = mesh.periods[2]
    d = cen[:, None, :] - seeds[None, :, :]
    d[:, :, 2] -= np.round(d[:, :, 2] / L) * L        # nearest image along z only
    want = np.argmin(np.linalg.norm(d, axis=2), axis=1)
    assert np.array_equal(v.tet_grain, want)
    counts = np.bincount(v.tet_grain, minlength=5)
    assert counts.sum() == mesh.n_tets
    # crystal axes are orthonormal frames (cubic anisotropy does not see their handedness)
    for R in v.axes:
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-12)
