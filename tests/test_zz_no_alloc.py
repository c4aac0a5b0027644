"""pmfem_field_noalloc: the field evaluation for callers that must not allocate device memory
(allocator-free loops, pooled device memory).  Its scratch is a fixed array
inside the library; it must give the same field as pmfem_field, also on a second call that
reuses the scratch the first one left behind.

Named to be collected last, so that a run stopping at its first failure has run every other
test before this one.
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


def _handle(mesh, grid, prec):
    from paper_2409_13958_gb300 import Pmfem
    h = Pmfem.create_mesh(mesh.xyz, mesh.tets, 8e5, 1.3e-11, 0.02)
    h.set_aim(*grid, 3, 3, 0.0)
    h.set_periodicity(*mesh.periods)
    h.set_precision(prec)
    h.set_applied_field(1e3, -2e3, 5e2)
    return h


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_noalloc_matches_field_on_two_calls(prec):
    from paper_2409_13958_gb300 import PMFEM_ALL, PMFEM_MS, PMFEM_EX
    mesh = meshgen.film_cell(20, 20, 2)
    h = _handle(mesh, (32, 32, 8), prec)
    n = h.num_unknowns()
    dt = torch.float64 if prec == 0 else torch.float32
    tol = 1e-12 if prec == 0 else 1e-6     # same kernels on the same operators: rounding order only
    for call, (seed, comps) in enumerate(((3, PMFEM_ALL), (4, PMFEM_MS | PMFEM_EX))):
        m = torch.tensor(meshgen.m_random(n, seed=seed), dtype=dt, device="cuda")
        ref = torch.empty_like(m)
        got = torch.full_like(m, float("nan"))
        h.field(m, ref, comps)           # the existing entry point (also uploads the operators)
        h.field_noalloc(m, got, comps)
        h.sync()
        err = float((got - ref).norm() / ref.norm())
        assert err <= tol, (call, err)
    h.destroy()


def test_noalloc_refuses_before_upload_and_beyond_its_size():
    from paper_2409_13958_gb300 import PmfemError
    mesh = meshgen.film_cell(10, 10, 2)
    h = _handle(mesh, (16, 16, 8), 0)
    m = torch.tensor(meshgen.m_random(h.num_unknowns(), seed=1), dtype=torch.float64, device="cuda")
    H = torch.empty_like(m)
    with pytest.raises(PmfemError) as e:
        h.field_noalloc(m, H)            # operators not on the device yet: no allocation here
    assert e.value.code == -7
    h.destroy()
    big = _handle(mesh, (1024, 1024, 8), 0)   # its FFT spectrum buffer alone is ~134 MB in FP64
    with pytest.raises(PmfemError) as e:
        big.field_noalloc(m, H)
    assert e.value.code == -1
    big.destroy()


def test_noalloc_after_set_m_upload():
    """The operators can reach the device through pmfem_set_m alone; the no-alloc call that
    follows then agrees with pmfem_field called afterwards."""
    from paper_2409_13958_gb300 import PMFEM_ALL
    mesh = meshgen.film_cell(12, 10, 2, seed=3)
    h = _handle(mesh, (16, 16, 8), 1)
    n = h.num_unknowns()
    m = torch.tensor(meshgen.m_random(n, seed=9), dtype=torch.float32, device="cuda")
    h.set_m(m)                           # uploads the operators; no field evaluated yet
    got = torch.full_like(m, float("nan"))
    h.field_noalloc(m, got, PMFEM_ALL)
    ref = torch.empty_like(m)
    h.field(m, ref, PMFEM_ALL)
    h.sync()
    assert float((got - ref).norm() / ref.norm()) <= 1e-6
    h.destroy()
