"""FP64 set-up on the GPU (pmfem_set_setup_device(1)) against the host set-up.

The host set-up is pinned to the oracle (test_lib_host: spectrum, precorrection and near-element
matrices); here the GPU kernels that replace three of its stages -- the PGF spectrum (Eq. 15 by
Ewald-type sums on the grid of Eq. 16, and its transform), the exact near-element integrals of
Eq. 14c and the point precorrection of BAIM step 4 -- must give the same matrices (same sparsity,
values within 1e-13 of the largest) and the same field (1e-13, FP64 path).
"""
import numpy as np
import pytest

import meshgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _shifted_prism():
    p = meshgen.prism_cell(5, 5, 8, jitter=0.15, seed=5)
    xyz = p.xyz.copy()
    xyz[:, 2] += 0.37 * p.periods[2] + 0.2 * xyz[:, 0]
    return meshgen.Mesh(xyz, p.tets, p.periods)


CASES = {
    # name: (mesh factory, grid, p, near_boxes, near_elem_factor)
    "film_2d": (lambda: meshgen.film_cell(20, 20, 2), (32, 32, 8), 3, 3, 0.0),
    "cube_3d": (lambda: meshgen.cube_cell(6, jitter=0.2, seed=4), (16, 16, 16), 3, 2, 0.0),
    "prism_1d_protruding": (_shifted_prism, (16, 16, 32), 3, 3, 0.0),
    "sphere_3d_nt": (lambda: meshgen.sphere_lattice(target_nodes=2500, seed=7), (16, 16, 16), 3, 2, 0.0),
    "free_space": (lambda: meshgen.Mesh(*meshgen.kuhn_box(6, 5, 4, 1e-9, jitter=0.2, seed=6), (0.0, 0.0, 0.0)),
                   (16, 16, 16), 3, 2, 0.0),
    "film_p2_near_radius": (lambda: meshgen.film_cell(9, 7, 3, seed=8), (16, 16, 16), 2, 2, 1.0),
    "film_p5_nb4": (lambda: meshgen.film_cell(9, 7, 3, seed=9), (16, 16, 16), 5, 4, 0.0),
    "wire_20k": (lambda: meshgen.wire_cell(L=100e-9, R=20e-9, target_nodes=20_000, seed=0), (32, 32, 64), 3, 3, 0.0),
}


def _handle(mesh, grid, p, nb, f, gpu):
    from paper_2409_13958_gb300 import Pmfem
    h = Pmfem.create_mesh(mesh.xyz, mesh.tets, 8e5, 1.3e-11, 0.02)
    h.set_aim(*grid, p, nb, f)
    h.set_setup_device(gpu)
    h.set_periodicity(*mesh.periods)
    h.set_precision(0)
    return h


def _close(a, b, tol=1e-13):
    scale = max(np.abs(b).max(), 1e-300)
    return np.abs(a - b).max() <= tol * scale


@pytest.mark.parametrize("name", sorted(CASES))
def test_gpu_setup_equals_host_setup(name):
    from paper_2409_13958_gb300 import PMFEM_ALL
    mk, grid, p, nb, f = CASES[name]
    mesh = mk()
    hh = _handle(mesh, grid, p, nb, f, False)
    hg = _handle(mesh, grid, p, nb, f, True)
    assert _close(hg.export_spectrum(), hh.export_spectrum())
    for which in (2, 4, 5):                       # near-element E (pattern, extra), point precorrection C
        rh, ch, vh = hh.operator_export(which)
        rg, cg, vg = hg.operator_export(which)
        assert np.array_equal(rh, rg) and np.array_equal(ch, cg), which
        if vh.size:
            assert _close(vg, vh), which
    if f > 0:
        assert hh.operator_export(5)[1].size > 0          # the radius reaches beyond the pattern
    m = torch.tensor(meshgen.m_random(hh.num_unknowns(), seed=3), dtype=torch.float64, device="cuda")
    Hh, Hg = torch.empty_like(m), torch.empty_like(m)
    hh.field(m, Hh, PMFEM_ALL)
    hg.field(m, Hg, PMFEM_ALL)
    hh.sync()
    hg.sync()
    assert float((Hg - Hh).norm() / Hh.norm()) <= 1e-13
    t = hg.setup_times()
    assert all(v >= 0 for v in t.values())
    hh.destroy()
    hg.destroy()
