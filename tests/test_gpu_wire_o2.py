"""The benchmark's wire against the oracle's P-AIM (O2) on sampled unknowns, where the device
layout takes the paths it takes only at scale: N' far above 2^16 (modular 16-bit column deltas
that wrap), many 1024-row length-sorted windows, ~216-entry precorrection rows.

The oracle builds the whole problem but its precorrection and near-element rows only for the
sampled unknowns and their adjacency neighbours (the gradient of Eq. 14d at a sampled unknown
reads the potential on its 1-ring); the magnetostatic and total fields at the sampled unknowns
are then compared element by element with the CUDA path's, at 1e-10 (FP64), 1e-5 (FP32) and
3e-3 (BF16-split), on the same input m (rounded to FP32 for the FP32 paths).

  * the full 1M-node wire in the launch configuration the benchmark times (grid 128 x 128 x 256,
    p = 3, near_boxes = 3, default layout);
  * a 120k-node wire with the benchmark's node-per-cell density (grid 64 x 64 x 128) under the
    default layout, 32-bit column deltas, and other box-order tiles and sort windows.
"""
import numpy as np
import pytest

import meshgen
from oracle.problem import OracleProblem
from oracle.topology import pair_nodes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WIRE_L, WIRE_R = 100e-9, 20e-9
MS, AEX, ALPHA = 8e5, 1.3e-11, 0.02
H_AP = (3e3, -1e3, 2e3)
TOL = {0: 1e-10, 1: 1e-5, 2: 3e-3}
SIZES = {"wire_1M": (1_000_000, (128, 128, 256)), "wire_120k": (125_000, (64, 64, 128))}


def _setup(key, samples):
    nodes, grid = SIZES[key]
    mesh = meshgen.wire_cell(L=WIRE_L, R=WIRE_R, target_nodes=nodes, seed=0)
    lca, roots = pair_nodes(mesh.xyz, mesh.periods)
    n_unk = int(roots.size)
    rng = np.random.default_rng(7)
    sample = np.sort(rng.choice(n_unk, size=samples, replace=False))
    touch = np.isin(lca[mesh.tets], sample).any(axis=1)
    obs = np.unique(lca[mesh.tets[touch]])
    ob = OracleProblem(mesh.xyz, mesh.tets, mesh.periods, Ms=MS, A=AEX, alpha=ALPHA, H_ap=H_AP, grid=grid,
                       p=3, near_boxes=3, near_elem_factor=0.0, observers=obs)
    return mesh, grid, ob, sample


@pytest.fixture(scope="module")
def build():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


_cache = {}


def _case(key, samples):
    if key not in _cache:
        _cache[key] = _setup(key, samples)
    return _cache[key]


def _handle(mesh, grid, prec, layout=None):
    from paper_2409_13958_gb300 import Pmfem
    h = Pmfem.create_mesh(mesh.xyz, mesh.tets, MS, AEX, ALPHA)
    h.set_aim(*grid, 3, 3, 0.0)
    h.set_periodicity(*mesh.periods)
    h.set_precision(prec)
    h.set_applied_field(*H_AP)
    if layout is not None:
        h.set_layout(*layout)
    return h


def _compare(h, ob, sample, prec, seed):
    from paper_2409_13958_gb300 import PMFEM_ALL, PMFEM_MS
    assert h.num_unknowns() == ob.Np
    m = meshgen.m_random(ob.Np, seed=seed)
    if prec:
        m = m.astype(np.float32).astype(np.float64)
    mt = torch.tensor(m, dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
    H = torch.empty_like(mt)
    h_ms = ob.h_ms(m, "paim")[sample]
    h_eff = h_ms + ob.h_ex(m)[sample] + ob.H_ap[None, :]
    for comps, ref in ((PMFEM_MS, h_ms), (PMFEM_ALL, h_eff)):
        H.fill_(float("nan"))
        h.field(mt, H, comps)
        h.sync()
        got = H.double().cpu().numpy()[sample]
        err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        assert err <= TOL[prec], (prec, comps, err)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_full_size_wire_matches_o2_on_sampled_unknowns(build, prec):
    mesh, grid, ob, sample = _case("wire_1M", 40)
    h = _handle(mesh, grid, prec)
    info = h.device_info()
    assert info["precorrection"]["col_bits"] == 16 and ob.Np > 1 << 16
    _compare(h, ob, sample, prec, seed=23)
    h.destroy()


LAYOUTS = [None, (0, 0, 0, 32), (4, 2, 256, 0), (16, 2, 4096, 32)]


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("layout", LAYOUTS, ids=["default", "int32_deltas", "tiles4x2_w256", "tiles16x2_w4096_int32"])
def test_wire_120k_layouts_match_o2_on_sampled_unknowns(build, layout, prec):
    mesh, grid, ob, sample = _case("wire_120k", 60)
    h = _handle(mesh, grid, prec, layout)
    if layout is not None and layout[3] == 32:
        assert h.device_info()["adjacency"]["col_bits"] == 32
    _compare(h, ob, sample, prec, seed=29)
    h.destroy()
