"""Batches of cells (pmfem_batch_*): every pass is one launch over all cells and an RK4 step is
a replayed CUDA graph.  The batch must give each cell the field and the trajectory that the
cell gives alone (FP32, same operators), and the oracle's field within the FP32 tolerance.
"""
import numpy as np
import pytest

import meshgen
from oracle.problem import OracleProblem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5        # against the FP64 oracle, as for a single cell
TOL_SAME = 1e-6        # batch against the cell alone: the same FP32 operators and row code

HAP = [(2e3, -1e3, 5e2), (-4e4, 0.0, 1e3), (0.0, 3e4, -2e3), (8e4, 1e3, 0.0)]


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _cells():
    """Uneven cells: two films (2D-periodic), a 3D-periodic cube and a 1D-periodic prism,
    with different node counts and grid shapes (two share a grid shape)."""
    return [
        (meshgen.film_cell(12, 10, 2, seed=21), (16, 16, 8)),
        (meshgen.film_cell(14, 14, 3, seed=22), (16, 16, 8)),
        (meshgen.cube_cell(5, jitter=0.2, seed=23), (16, 16, 16)),
        (meshgen.prism_cell(4, 4, 7, jitter=0.15, seed=24), (16, 16, 32)),
    ]


def _handle(mesh, grid, hap):
    from paper_2409_13958_gb300 import Pmfem, PMFEM_FP32
    h = Pmfem.create_mesh(mesh.xyz, mesh.tets, 8e5, 1.3e-11, 0.02)
    h.set_aim(*grid, 3, 2, 0.0)
    h.set_periodicity(*mesh.periods)
    h.set_precision(PMFEM_FP32)
    h.set_applied_field(*hap)
    return h


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _setup():
    cells = _cells()
    hs = [_handle(m, g, hap) for (m, g), hap in zip(cells, HAP)]
    from paper_2409_13958_gb300 import PmfemBatch
    b = PmfemBatch(hs)
    return cells, hs, b


def test_batch_field_matches_each_cell_and_the_oracle():
    from paper_2409_13958_gb300 import PMFEM_ALL, PMFEM_MS, PMFEM_EX
    cells, hs, b = _setup()
    off = b.offsets()
    ms = [meshgen.m_random(h.num_unknowns(), seed=30 + k) for k, h in enumerate(hs)]
    m = torch.tensor(np.concatenate(ms), dtype=torch.float32, device="cuda")
    H = torch.full_like(m, float("nan"))
    for comps in (PMFEM_ALL, PMFEM_MS, PMFEM_EX):
        b.field(m, H, comps)
        b.sync()
        Hb = H.double().cpu().numpy()
        for k, h in enumerate(hs):
            mk = m[off[k]:off[k + 1]].contiguous()
            Hk = torch.empty_like(mk)
            h.field(mk, Hk, comps)
            h.sync()
            assert _rel(Hb[off[k]:off[k + 1]], Hk.double().cpu().numpy()) <= TOL_SAME, (k, comps)
    b.field(m, H, PMFEM_ALL)
    b.sync()
    Hb = H.double().cpu().numpy()
    for k, ((mesh, grid), hap) in enumerate(zip(cells, HAP)):
        ob = OracleProblem(mesh.xyz, mesh.tets, mesh.periods, Ms=8e5, A=1.3e-11, alpha=0.02, H_ap=hap,
                           grid=grid, p=3, near_boxes=2, near_elem_factor=0.0)
        assert _rel(Hb[off[k]:off[k + 1]], ob.h_eff(ms[k], "paim")) <= TOL_FP32, k
    b.destroy()


def test_batch_rk4_graph_matches_each_cell():
    cells, hs, b = _setup()
    off = b.offsets()
    ms = [meshgen.m_random(h.num_unknowns(), seed=40 + k) for k, h in enumerate(hs)]
    m = torch.tensor(np.concatenate(ms), dtype=torch.float32, device="cuda")
    dt = 2e-14
    b.set_m(m)
    b.llg_step(dt, 3)          # captures the step, replays it 3 times
    b.llg_step(dt, 2)          # replays the same graph
    out = torch.empty_like(m)
    b.get_m(out)
    b.sync()
    got = out.double().cpu().numpy()
    for k, h in enumerate(hs):
        mk = m[off[k]:off[k + 1]].contiguous()
        h.set_m(mk)
        h.llg_step(dt, 5)
        ref = torch.empty_like(mk)
        h.get_m(ref)
        h.sync()
        ref = ref.double().cpu().numpy()
        assert _rel(got[off[k]:off[k + 1]], ref) <= TOL_SAME, k
        assert np.abs(np.linalg.norm(got[off[k]:off[k + 1]], axis=1) - 1).max() < 1e-6
    b.destroy()


def test_batch_applied_field_update_reaches_the_graph():
    from paper_2409_13958_gb300 import PMFEM_AP
    cells, hs, b = _setup()
    n = int(b.offsets()[-1])
    m = torch.tensor(np.concatenate([meshgen.m_uniform(h.num_unknowns()) for h in hs]), dtype=torch.float32,
                     device="cuda")
    H = torch.empty_like(m)
    b.field(m, H, PMFEM_AP)
    b.set_applied_field(2, 1.0e5, -2.0e5, 3.0e5)
    b.field(m, H, PMFEM_AP)
    b.sync()
    off = b.offsets()
    Hn = H.cpu().numpy()
    assert np.allclose(Hn[off[2]:off[3]], [1.0e5, -2.0e5, 3.0e5])
    assert np.allclose(Hn[off[1]:off[2]], HAP[1])
    assert Hn.shape == (n, 3)
    b.destroy()


def test_batch_autotune_picks_listed_tiles_and_keeps_the_field():
    from paper_2409_13958_gb300 import PMFEM_ALL
    cells, hs, b = _setup()
    m = torch.tensor(np.concatenate([meshgen.m_random(h.num_unknowns(), seed=50 + k) for k, h in enumerate(hs)]),
                     dtype=torch.float32, device="cuda")
    H0 = torch.empty_like(m)
    b.field(m, H0, PMFEM_ALL)
    b.sync()
    b.autotune(reps=2)
    H1 = torch.empty_like(m)
    b.field(m, H1, PMFEM_ALL)
    b.sync()
    tiles = b.tiles()
    allowed = {(8, 4), (8, 2), (4, 4), (16, 2), (4, 2)}
    for k, (mesh, grid) in enumerate(cells):
        ty, tz = (int(x) for x in tiles[k])
        assert any(ty == min(a, grid[1]) and tz == min(c, grid[2]) for a, c in allowed), (k, ty, tz)
    assert _rel(H1.double().cpu().numpy(), H0.double().cpu().numpy()) <= TOL_FP32
    b.destroy()


def test_batch_profile_times_every_pass_and_keeps_the_trajectory():
    """With per-launch timing on, the batch steps kernel by kernel (no graph): the same
    trajectory as the replayed step, and a launch count per pass of every evaluation."""
    cells, hs, b = _setup()
    n = int(b.offsets()[-1])
    m0 = torch.tensor(meshgen.m_random(n, seed=77), dtype=torch.float32, device="cuda")
    dt = 2e-14
    b.set_m(m0)
    b.llg_step(dt, 2)          # replayed graph
    ref = torch.empty_like(m0)
    b.get_m(ref)
    b.set_m(m0)
    b.profile(True)
    b.llg_step(dt, 2)          # launch by launch, timed
    prof = b.profile_read()
    b.profile(False)
    got = torch.empty_like(m0)
    b.get_m(got)
    b.sync()
    # the same kernels in the same order (the few atomics of the projection's exception nodes may
    # sum in another order)
    assert _rel(got.double().cpu().numpy(), ref.double().cpu().numpy()) <= TOL_SAME
    evals = 2 * 4
    for name in ("charges", "projection", "interp_precorr", "gradient_exchange"):
        c, t = prof[name]
        assert c == evals and t > 0, name
    assert prof["fft_z_conv"][0] >= evals     # one per grid-shape group and evaluation
    assert prof["interp_stencil"][0] == 0     # the batch runs the fused interpolation
    b.destroy()
