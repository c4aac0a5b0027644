"""CPU tests of libpmfem: exported symbols, error conventions, and the host set-up
(pairing, fold, operators, grid, spectrum, precorrection) against the oracle.

No test here launches a kernel: set-up runs on the host and the device is only touched
by calls that need it.
"""
import math
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

import meshgen
from oracle.problem import OracleProblem

pmf = pytest.importorskip("paper_2409_13958_gb300")
from paper_2409_13958_gb300 import binding as B  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2409_13958_gb300 import _build
    _build.build()
    B.load_library()


def test_every_declared_symbol_is_exported():
    hdr = open(os.path.join(ROOT, "include", "pmfem.h")).read()
    declared = set(re.findall(r"\b(pmfem_[a-z0-9_]+)\s*\(", hdr))
    assert declared == set(B.SYMBOLS)
    lib = B.load_library()
    for name in declared:
        assert hasattr(lib, name)
    assert b"sm_103a" in lib.pmfem_version()


def _mk(mesh, periods=None, grid=(0, 0, 0), p=3, nb=3, f=0.0, Ms=8e5, A=1.3e-11):
    h = B.Pmfem.create_mesh(mesh.xyz, mesh.tets, Ms, A, 0.02)
    h.set_aim(*grid, p, nb, f)
    h.set_periodicity(*(mesh.periods if periods is None else periods))
    return h


def test_error_conventions():
    m = meshgen.film_cell(4, 4, 2)
    for xyz, tets in ((np.zeros((0, 3)), np.zeros((0, 4), np.int32)), (m.xyz, np.zeros((0, 4), np.int32))):
        with pytest.raises(B.PmfemError) as e:      # empty mesh or no tetrahedra
            B.Pmfem.create_mesh(xyz, tets, 8e5, 1e-11, 0.02)
        assert e.value.code == -1
    bad = m.tets.copy()
    bad[0, 0] = m.n_nodes + 5
    with pytest.raises(B.PmfemError) as e:
        B.Pmfem.create_mesh(m.xyz, bad, 8e5, 1e-11, 0.02)
    assert e.value.code == -4
    deg = m.tets.copy()
    deg[0, 1] = deg[0, 0]
    with pytest.raises(B.PmfemError) as e:
        B.Pmfem.create_mesh(m.xyz, deg, 8e5, 1e-11, 0.02)
    assert e.value.code == -4
    with pytest.raises(B.PmfemError) as e:
        B.Pmfem.create_mesh(m.xyz, m.tets, -1.0, 1e-11, 0.02)
    assert e.value.code == -1
    h = B.Pmfem.create_mesh(m.xyz, m.tets, 8e5, 1e-11, 0.02)
    with pytest.raises(B.PmfemError) as e:
        h.num_unknowns()
    assert e.value.code == -7
    with pytest.raises(B.PmfemError) as e:
        h.field(1 << 20, 2 << 20)            # before set-up: refused without touching memory
    assert e.value.code == -7
    with pytest.raises(B.PmfemError) as e:
        h.set_aim(3, 8, 8, 3, 3, 0.0)
    assert e.value.code == -1
    with pytest.raises(B.PmfemError) as e:
        h.set_periodicity(-1.0, 0, 0)
    assert e.value.code == -1
    h.set_aim(8, 8, 8, 3, 2, 0.0)
    h.set_periodicity(*m.periods)
    with pytest.raises(B.PmfemError) as e:
        h.llg_step(-1e-13, 1)
    assert e.value.code == -1
    with pytest.raises(B.PmfemError) as e:
        h.field(1 << 20, 1 << 20)            # aliasing m and H
    assert e.value.code == -1
    with pytest.raises(B.PmfemError) as e:
        h.set_precision(7)
    assert e.value.code == -1
    h.set_precision(B.PMFEM_BF16SPLIT)
    h.set_bf16_operators(B.PMFEM_BF16_PRECORRECTION | B.PMFEM_BF16_EXCHANGE)
    with pytest.raises(B.PmfemError) as e:
        h.set_bf16_operators(32)
    assert e.value.code == -1
    # a node on a touching face without its partner
    xyz = m.xyz.copy()
    moved = np.nonzero(np.isclose(xyz[:, 0], m.periods[0]) & (xyz[:, 1] > 1e-9) & (xyz[:, 1] < 3e-9))[0][0]
    xyz[moved, 1] += 0.3e-9
    h2 = B.Pmfem.create_mesh(xyz, m.tets, 8e5, 1e-11, 0.02)
    with pytest.raises(B.PmfemError) as e:
        h2.set_periodicity(*m.periods)
    assert e.value.code == -4


def _csr(rp, col, vals, n):
    return sp.csr_matrix((vals, col, rp), shape=(n, n))


def _close(a, b, rtol):
    d = abs(a - b).max() if (a - b).nnz else 0.0
    scale = max(abs(b).max(), 1e-300)
    return d <= rtol * scale, d / scale


CASES = {
    "film": (lambda: meshgen.film_cell(10, 10, 2), None, (16, 16, 8), 3, 3, 0.0),
    "film_p2_f1": (lambda: meshgen.film_cell(8, 8, 2, seed=3), None, (16, 16, 8), 2, 2, 1.0),
    "cube": (lambda: meshgen.cube_cell(5, jitter=0.2, seed=4), None, (16, 16, 16), 3, 2, 0.0),
    "prism_shifted": (lambda: _shifted_prism(), None, (16, 16, 16), 3, 3, 0.0),
    "free": (lambda: meshgen.Mesh(*meshgen.kuhn_box(4, 3, 3, 1e-9, jitter=0.2, seed=6), (0.0, 0.0, 0.0)),
             None, (16, 16, 16), 3, 2, 0.5),
}


def _shifted_prism():
    p = meshgen.prism_cell(4, 4, 6, jitter=0.15, seed=5)
    xyz = p.xyz.copy()
    xyz[:, 2] += 0.37 * p.periods[2]
    xyz[:, 2] += 0.2 * xyz[:, 0]                # shear: the cell protrudes past its period
    return meshgen.Mesh(xyz, p.tets, p.periods)


@pytest.mark.parametrize("case", sorted(CASES))
def test_host_setup_matches_oracle(case):
    mk, per, grid, p, nb, f = CASES[case]
    mesh = mk()
    Ms, A = 8e5, 1.3e-11
    h = _mk(mesh, per, grid, p, nb, f, Ms, A)
    ob = OracleProblem(mesh.xyz, mesh.tets, mesh.periods, Ms=Ms, A=A, grid=grid, p=p, near_boxes=nb,
                       near_elem_factor=f)
    n = ob.Np
    assert h.num_unknowns() == n
    assert np.array_equal(h.lca_map(mesh.n_nodes), ob.lca)
    assert np.array_equal(h.folded_positions(), ob.pos_f)
    # exchange
    rp, col, v = h.operator_export(0)
    Kref = sp.csr_matrix(-(2 * A / (4e-7 * math.pi * Ms)) * sp.diags(1 / ob.V) @ ob.K)
    ok, err = _close(_csr(rp, col, v[:, 0], n), Kref, 1e-12)
    assert ok, err
    # charges, gradient, near elements
    rp, col, W = h.operator_export(1)
    _, _, G = h.operator_export(3)
    _, _, Ea = h.operator_export(2)
    rpx, colx, Ex = h.operator_export(5)
    for d in range(3):
        ok, err = _close(_csr(rp, col, W[:, d], n), Ms * ob.Wq[d], 1e-12)
        assert ok, ("Wq", d, err)
        Gref = sp.csr_matrix(-(sp.diags(1 / (4 * math.pi * ob.V)) @ ob.Wq[d].T))
        ok, err = _close(_csr(rp, col, G[:, d], n), Gref, 1e-12)
        assert ok, ("grad", d, err)
        Elib = _csr(rp, col, Ea[:, d], n) + _csr(rpx, colx, Ex[:, d], n)
        ok, err = _close(Elib, Ms * ob.E[d], 1e-11)
        assert ok, ("E", d, err)
    if f == 0.0:
        assert colx.size == 0              # touching elements stay on the adjacency pattern
    # grid and spectrum
    dims, fft, origin, delta = h.grid_info()
    assert tuple(dims) == ob.grid.dims and tuple(fft) == tuple(ob.grid.fft)
    assert np.array_equal(origin, ob.grid.origin) and np.array_equal(delta, ob.grid.delta)
    spec = h.export_spectrum()                                   # (z, y, x) reduced, unscaled
    ref = np.fft.fftn(ob.Ktab)[: fft[0] // 2 + 1, : fft[1] // 2 + 1, : fft[2] // 2 + 1]
    assert np.abs(ref.imag).max() < 1e-10 * np.abs(ref.real).max()
    assert np.abs(spec.transpose(2, 1, 0) - ref.real).max() < 1e-11 * np.abs(ref.real).max()
    # point precorrection
    rp, col, v = h.operator_export(4)
    ok, err = _close(_csr(rp, col, v[:, 0], n), ob.C, 1e-11)
    assert ok, ("C", err)


def test_set_aim_defaults_and_validation():
    m = meshgen.film_cell(10, 10, 2)
    h = B.Pmfem.create_mesh(m.xyz, m.tets, 8e5, 1.3e-11, 0.02)
    h.set_periodicity(*m.periods)
    dims, fft, origin, delta = h.grid_info()
    for a in range(3):
        assert fft[a] & (fft[a] - 1) == 0 and 4 <= fft[a] <= 1024
    h.set_aim(12, 16, 8, 3, 3, 0.0)             # 12 is not a power of two on a periodic axis
    with pytest.raises(B.PmfemError) as e:
        h.set_periodicity(*m.periods)
    assert e.value.code == -1


def test_batch_create_checks_its_cells_and_gives_offsets():
    """pmfem_batch_create is host-only: it checks that every cell is set up and that all
    share the stencil order, and reports where each cell's unknowns start."""
    from paper_2409_13958_gb300 import binding as B
    a = meshgen.film_cell(6, 5, 2, seed=1)
    c = meshgen.cube_cell(4, seed=2)
    ha = B.Pmfem.create_mesh(a.xyz, a.tets, 8e5, 1.3e-11, 0.02)
    ha.set_aim(8, 8, 8, 3, 2, 0.0)
    ha.set_periodicity(*a.periods)
    hc = B.Pmfem.create_mesh(c.xyz, c.tets, 8e5, 1.3e-11, 0.02)
    with pytest.raises(B.PmfemError) as e:
        B.PmfemBatch([ha, hc])                 # hc is not set up yet
    assert e.value.code == -7
    hc.set_aim(8, 8, 8, 2, 2, 0.0)
    hc.set_periodicity(*c.periods)
    with pytest.raises(B.PmfemError) as e:
        B.PmfemBatch([ha, hc])                 # stencil orders 3 and 2
    assert e.value.code == -1
    hc.set_aim(8, 8, 8, 3, 2, 0.0)
    hc.set_periodicity(*c.periods)
    b = B.PmfemBatch([ha, hc, ha])
    na, nc = ha.num_unknowns(), hc.num_unknowns()
    assert list(b.offsets()) == [0, na, na + nc, 2 * na + nc]
    with pytest.raises(B.PmfemError) as e:
        b.llg_step(-1.0, 1)
    assert e.value.code == -1
    with pytest.raises(B.PmfemError) as e:
        b.autotune(0)
    assert e.value.code == -1
    with pytest.raises(B.PmfemError) as e:
        b.set_applied_field(3, 1.0, 0.0, 0.0)
    assert e.value.code == -1
    b.destroy()


def test_setup_device_switch_rejects_bad_values():
    import meshgen
    from paper_2409_13958_gb300 import Pmfem, PmfemError
    m = meshgen.film_cell(4, 4, 2)
    h = Pmfem.create_mesh(m.xyz, m.tets, 8e5, 1.3e-11, 0.02)
    for bad in (2, -1):
        with pytest.raises(PmfemError) as e:
            h._ck(h._lib.pmfem_set_setup_device(h.h, bad))
        assert e.value.code == -1
    h.set_setup_device(False)
    h.set_periodicity(*m.periods)
    t = h.setup_times()
    assert set(t) == {"pairing", "operators", "grid", "spectrum", "near_elements", "precorrection", "device"}
    assert t["precorrection"] >= 0 and t["device"] == 0.0
    h.destroy()


def test_debug_hooks_without_a_gpu():
    from paper_2409_13958_gb300 import binding
    lib = binding.load_library()
    assert lib.pmfem_build_flags() == 0
    assert lib.pmfem_debug_fail_alloc(-2) == -1
    assert lib.pmfem_debug_fail_alloc(3) == 0
    assert lib.pmfem_debug_fail_alloc(-1) == 0


def test_local_terms_and_bloch_inputs_are_checked_without_a_gpu():
    """Invalid anisotropy, stiffness and Bloch inputs are refused on the host (EINVAL), and a Bloch
    call before the set-up with ESTATE, before any device work."""
    mesh, gr = meshgen.granular_cell(n=4, grains=3, seed=1)
    h = B.Pmfem.create_mesh(mesh.xyz, mesh.tets, 8e5, 1.3e-11, 0.02)
    h.set_aim(8, 8, 8, 3, 2, 0.0)
    k_lat = np.array([2 * np.pi / mesh.periods[0], 0.0, 0.0])      # on the reciprocal lattice
    with pytest.raises(B.PmfemError) as e:
        h.bloch_spectrum(0.3 * k_lat)
    assert e.value.code == -7
    for bad in (-1.0, np.nan):
        A = gr.A_tet.copy()
        A[3] = bad
        with pytest.raises(B.PmfemError) as e:
            h.set_exchange_per_tet(A)
        assert e.value.code == -1
    axes = gr.axes.reshape(-1, 9)
    tg = gr.tet_grain.copy()
    tg[0] = 3                                                       # only grains 0..2 exist
    cases = [dict(tet_grain=tg, axes=axes, K1=gr.K1),
             dict(tet_grain=gr.tet_grain, axes=2 * axes, K1=gr.K1),   # axes not unit rows
             dict(tet_grain=gr.tet_grain, axes=axes, Ku=np.ones(3)),  # Ku without u
             dict(tet_grain=gr.tet_grain, axes=axes)]                 # neither K1 nor Ku
    for kw in cases:
        with pytest.raises(B.PmfemError) as e:
            h.set_anisotropy(**kw)
        assert e.value.code == -1
    h.set_exchange_per_tet(gr.A_tet)
    h.set_periodicity(*mesh.periods)
    h.set_anisotropy(gr.tet_grain, axes, K1=gr.K1)
    with pytest.raises(B.PmfemError) as e:
        h.bloch_spectrum(k_lat)
    assert e.value.code == -1
    with pytest.raises(B.PmfemError) as e:
        h.bloch_convolve(k_lat, 1 << 20, 2 << 20)
    assert e.value.code == -1
    film = meshgen.film_cell(4, 4, 2)
    f = B.Pmfem.create_mesh(film.xyz, film.tets, 8e5, 1.3e-11, 0.02)
    f.set_aim(8, 8, 8, 3, 2, 0.0)
    f.set_periodicity(*film.periods)
    with pytest.raises(B.PmfemError) as e:                          # k0 along the open axis
        f.bloch_convolve(np.array([0.0, 0.0, 1e8]), 1 << 20, 2 << 20)
    assert e.value.code == -1


def test_host_exchange_with_a_stiffness_per_tet_matches_oracle():
    """The stored exchange operator with a grain-boundary stiffness layer (A inside the element
    sum) equals the oracle's K_A scaled by -2/(mu0 Ms V_n), on the granular 3D-periodic cell."""
    from oracle import local_terms as LT
    mesh, gr = meshgen.granular_cell(n=5, grains=4, seed=2)
    Ms = 8e5
    h = B.Pmfem.create_mesh(mesh.xyz, mesh.tets, Ms, 1.3e-11, 0.02)
    h.set_aim(8, 8, 8, 3, 2, 0.0)
    h.set_exchange_per_tet(gr.A_tet)
    h.set_periodicity(*mesh.periods)
    ob = OracleProblem(mesh.xyz, mesh.tets, mesh.periods, Ms=Ms, A=1.3e-11, grid=(8, 8, 8), p=3, near_boxes=2)
    KA = LT.exchange_matrix_per_tet(ob.xyz, ob.tets, ob.lca, ob.Np, gr.A_tet)
    ref = sp.csr_matrix(-(2.0 / (4e-7 * math.pi * Ms)) * sp.diags(1 / ob.V) @ KA)
    rp, col, v = h.operator_export(0)
    ok, err = _close(_csr(rp, col, v[:, 0], ob.Np), ref, 1e-12)
    assert ok, err
    assert 0 < (gr.A_tet < 1.3e-11).mean() < 1      # the layer is there and is not everything
