"""Anisotropy per grain and exchange stiffness per tetrahedron on the GPU against the oracle
(oracle/local_terms.py), through the C-ABI, on a seeded granular 3D-periodic cell.

Field tolerances are the path's (FP64 1e-10, FP32 1e-5, BF16-split 3e-3); an RK4 trajectory with
the anisotropy term is compared too (the term sits in the field kernel's epilogue, which also
does the RK4 stage update)."""
import numpy as np
import pytest

import meshgen
from oracle import local_terms as LT
from oracle.llg import rk4_step
from oracle.problem import OracleProblem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MS, A, ALPHA = 8e5, 1.3e-11, 0.05
TOL = {0: 1e-10, 1: 1e-5, 2: 3e-3}


@pytest.fixture(scope="module")
def cell():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    mesh, gr = meshgen.granular_cell(n=6, grains=5, K1=-4.5e4, seed=3)
    Ku = np.linspace(2e4, 6e4, gr.axes.shape[0])
    ob = OracleProblem(mesh.xyz, mesh.tets, mesh.periods, Ms=MS, A=A, alpha=ALPHA, H_ap=(1e3, 2e3, -1e3),
                       grid=(16, 16, 16), near_boxes=2)
    w = LT.grain_weights(ob.tets, ob.lca, ob.vol, gr.tet_grain, ob.Np, gr.axes.shape[0])
    KA = LT.exchange_matrix_per_tet(ob.xyz, ob.tets, ob.lca, ob.Np, gr.A_tet)

    def h_an(m):
        return LT.anisotropy_field(m, w, gr.axes, gr.K1, Ku, gr.u, MS)

    def h_ex(m):
        return LT.exchange_field_per_tet(KA, ob.V, m, MS)

    def h_eff(m):
        return h_ex(m) + ob.h_ms(m, "paim") + ob.H_ap[None, :] + h_an(m)

    return mesh, gr, Ku, ob, h_an, h_ex, h_eff


def _handle(cell, prec, with_aniso=True, per_tet=True):
    from paper_2409_13958_gb300 import Pmfem
    mesh, gr, Ku = cell[0], cell[1], cell[2]
    h = Pmfem.create_mesh(mesh.xyz, mesh.tets, MS, A, ALPHA)
    h.set_aim(16, 16, 16, 3, 2, 0.0)
    if per_tet:
        h.set_exchange_per_tet(gr.A_tet)
    h.set_periodicity(*mesh.periods)
    if with_aniso:
        h.set_anisotropy(gr.tet_grain, gr.axes.reshape(-1, 9), K1=gr.K1, Ku=Ku, u=gr.u)
    h.set_precision(prec)
    h.set_applied_field(1e3, 2e3, -1e3)
    return h


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_local_terms_match_the_oracle(cell, prec):
    from paper_2409_13958_gb300 import PMFEM_AN, PMFEM_EX, PMFEM_ALL
    mesh, gr, Ku, ob, h_an, h_ex, h_eff = cell
    h = _handle(cell, prec)
    m = meshgen.m_random(ob.Np, seed=5)
    if prec:
        m = m.astype(np.float32).astype(np.float64)
    dt = torch.float64 if prec == 0 else torch.float32
    mt = torch.tensor(m, dtype=dt, device="cuda")
    H = torch.empty_like(mt)
    for comps, ref in ((PMFEM_AN, h_an(m)), (PMFEM_EX, h_ex(m)), (PMFEM_ALL, h_eff(m))):
        H.fill_(float("nan"))
        h.field(mt, H, comps)
        h.sync()
        err = _rel(H.double().cpu().numpy(), ref)
        assert err <= TOL[prec], (prec, comps, err)
    h.destroy()


def test_anisotropy_is_absent_until_set_and_removable(cell):
    from paper_2409_13958_gb300 import PMFEM_AN
    mesh, gr, Ku, ob = cell[:4]
    h = _handle(cell, 0, with_aniso=False)
    m = torch.tensor(meshgen.m_random(ob.Np, seed=6), device="cuda")
    H = torch.full_like(m, 7.0)
    h.field(m, H, PMFEM_AN)
    h.sync()
    assert torch.count_nonzero(H) == 0
    h.set_anisotropy(gr.tet_grain, gr.axes.reshape(-1, 9), K1=gr.K1)
    h.field(m, H, PMFEM_AN)
    h.sync()
    assert torch.count_nonzero(H) > 0
    h.set_anisotropy(None)
    h.field(m, H, PMFEM_AN)
    h.sync()
    assert torch.count_nonzero(H) == 0
    h.destroy()


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-5)])
def test_rk4_with_local_terms_matches_the_oracle(cell, prec, tol):
    mesh, gr, Ku, ob, h_an, h_ex, h_eff = cell
    h = _handle(cell, prec)
    m0 = meshgen.m_random(ob.Np, seed=7)
    if prec:
        m0 = m0.astype(np.float32).astype(np.float64)
    dt_t = torch.float64 if prec == 0 else torch.float32
    h.set_m(torch.tensor(m0, dtype=dt_t, device="cuda"))
    dt = 5e-15
    h.llg_step(dt, 4)
    out = torch.empty((ob.Np, 3), dtype=dt_t, device="cuda")
    h.get_m(out)
    h.sync()
    m = m0
    for _ in range(4):
        m = rk4_step(m, dt, h_eff, ALPHA)
    assert _rel(out.double().cpu().numpy(), m) <= tol
    assert _rel(m, m0) > 1e-5
    h.destroy()
