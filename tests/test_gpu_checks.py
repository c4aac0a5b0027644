"""The bounds-checked build and the out-of-memory paths, on the GPU.

* libpmfem_checks.so (PMFEM_CHECKS): every stored index of a device upload is checked against its
  bounds on the device before any kernel uses it; on correct data the checks pass and the fields
  equal the plain build's.
* pmfem_debug_fail_alloc: device allocations refused after a given count give ENOMEM from the
  call that builds the device data, leave the handle clean, and the next call (hook off) works.
"""
import numpy as np
import pytest

import meshgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def libs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2409_13958_gb300 import _build, binding
    checked = binding.load_variant(_build.build(variant="checks"))
    return binding.load_library(), checked


def _prism():
    p = meshgen.prism_cell(5, 5, 8, jitter=0.15, seed=5)
    xyz = p.xyz.copy()
    xyz[:, 2] += 0.37 * p.periods[2] + 0.2 * xyz[:, 0]
    return meshgen.Mesh(xyz, p.tets, p.periods), (16, 16, 32), 3


MESHES = {
    "film": (lambda: meshgen.film_cell(20, 20, 2), (32, 32, 8), 3),
    "prism_protruding": _prism,
    "cube": (lambda: meshgen.cube_cell(6, jitter=0.2, seed=4), (16, 16, 16), 2),
}


def _handle(lib, mesh, grid, nb, prec):
    from paper_2409_13958_gb300 import Pmfem
    h = Pmfem.create_mesh(mesh.xyz, mesh.tets, 8e5, 1.3e-11, 0.02, lib=lib)
    h.set_aim(*grid, 3, nb, 0.0)
    h.set_periodicity(*mesh.periods)
    h.set_precision(prec)
    h.set_applied_field(1e3, 0.0, -2e3)
    return h


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", sorted(MESHES))
def test_checked_build_passes_and_agrees(libs, name, prec):
    from paper_2409_13958_gb300 import PMFEM_ALL
    plain, checked = libs
    assert checked.pmfem_build_flags() == 1 and plain.pmfem_build_flags() == 0
    f = MESHES[name]
    mesh, grid, nb = f() if callable(f) else (f[0](), f[1], f[2])
    out = []
    for lib in (plain, checked):
        h = _handle(lib, mesh, grid, nb, prec)
        m = torch.tensor(meshgen.m_random(h.num_unknowns(), seed=2), dtype=torch.float64 if prec == 0 else torch.float32,
                         device="cuda")
        H = torch.empty_like(m)
        h.field(m, H, PMFEM_ALL)
        h.sync()                                # a failed layout check would raise EINVAL here
        h.set_m(m)
        h.llg_step(1e-15, 2)
        h.sync()
        out.append(H.double().cpu().numpy())
        h.destroy()
    err = np.linalg.norm(out[1] - out[0]) / np.linalg.norm(out[0])
    assert err <= (1e-13 if prec == 0 else 1e-6), err


def test_refused_allocations_give_enomem_and_leave_the_handle_usable(libs):
    from paper_2409_13958_gb300 import PMFEM_ALL, PmfemError
    plain, _ = libs
    mesh = meshgen.film_cell(10, 10, 2)
    h = _handle(plain, mesh, (16, 16, 8), 3, 0)
    m = torch.tensor(meshgen.m_random(h.num_unknowns(), seed=3), device="cuda")
    H = torch.empty_like(m)
    try:
        for after in (0, 1, 7, 25):
            assert plain.pmfem_debug_fail_alloc(after) == 0
            with pytest.raises(PmfemError) as e:
                h.field(m, H, PMFEM_ALL)
            assert e.value.code == -2, after
    finally:
        plain.pmfem_debug_fail_alloc(-1)
    h.field(m, H, PMFEM_ALL)
    h.sync()
    ref = _handle(plain, mesh, (16, 16, 8), 3, 0)
    H2 = torch.empty_like(m)
    ref.field(m, H2, PMFEM_ALL)
    ref.sync()
    assert float((H - H2).norm() / H2.norm()) <= 1e-14
    h.destroy()
    ref.destroy()
