"""Full size: the 1M-node periodic wire of the benchmark, in the launch configuration bench.py
times (grid 128 x 128 x 256, p = 3, near_boxes = 3).  The oracle cannot build the whole
problem at this size, so the exchange field is checked on sampled unknowns, each computed by
the oracle from the tetrahedra around it, and the magnetostatic field by properties that hold at
any size (linearity, a negative magnetostatic energy, FP32 against FP64)."""
import numpy as np
import pytest

import meshgen
from oracle import operators as O
from oracle.topology import pair_nodes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WIRE_L, WIRE_R = 100e-9, 20e-9
MS, AEX = 8e5, 1.3e-11


@pytest.fixture(scope="module")
def wire():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2409_13958_gb300 import Pmfem
    mesh = meshgen.wire_cell(L=WIRE_L, R=WIRE_R, target_nodes=1_000_000, seed=0)
    h = Pmfem.create_mesh(mesh.xyz, mesh.tets, MS, AEX, 0.02)
    h.set_aim(128, 128, 256, 3, 3, 0.0)
    h.set_periodicity(0.0, 0.0, WIRE_L)
    yield mesh, h
    h.destroy()


def _field(h, prec, m, comps):
    dt = torch.float64 if prec == 0 else torch.float32
    h.set_precision(prec)
    mt = torch.tensor(m, dtype=dt, device="cuda")
    H = torch.empty_like(mt)
    h.field(mt, H, comps)
    h.sync()
    return H.double().cpu().numpy()


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-5)])
def test_exchange_on_sampled_unknowns_matches_the_oracle(wire, prec, tol):
    from paper_2409_13958_gb300 import PMFEM_EX
    mesh, h = wire
    lca, roots = pair_nodes(mesh.xyz, mesh.periods)          # the oracle's own pairing and numbering
    n_unk = roots.shape[0]
    assert n_unk == h.num_unknowns()
    rng = np.random.default_rng(5)
    sample = rng.choice(n_unk, size=48, replace=False)
    m = meshgen.m_random(n_unk, seed=17)
    H = _field(h, prec, m, PMFEM_EX)
    # the tetrahedra touching any node of each sampled unknown give its whole exchange row
    touch = np.isin(lca[mesh.tets], sample).any(axis=1)
    ops = O.assemble(mesh.xyz, mesh.tets[touch], lca, n_unk)
    Href = O.exchange_field(ops["K"], np.where(ops["V"] > 0, ops["V"], 1.0), m, AEX, MS)
    err = np.linalg.norm(H[sample] - Href[sample]) / np.linalg.norm(Href[sample])
    assert err <= tol, err


def test_magnetostatic_is_linear_at_full_size(wire):
    from paper_2409_13958_gb300 import PMFEM_MS
    mesh, h = wire
    n = h.num_unknowns()
    m1 = meshgen.m_random(n, seed=21)
    m2 = meshgen.m_vortex(h.folded_positions(), core=5e-9)
    a, b = 0.6, -1.7
    H1 = _field(h, 0, m1, PMFEM_MS)
    H2 = _field(h, 0, m2, PMFEM_MS)
    H12 = _field(h, 0, a * m1 + b * m2, PMFEM_MS)
    ref = a * H1 + b * H2
    assert np.linalg.norm(H12 - ref) <= 1e-11 * np.linalg.norm(ref)


def test_magnetostatic_energy_is_negative_at_full_size(wire):
    """sum_n V_n M_n . H_ms,n = -q^T G q < 0: the demagnetising field opposes M on average."""
    from paper_2409_13958_gb300 import PMFEM_MS
    mesh, h = wire
    n = h.num_unknowns()
    lca, roots = pair_nodes(mesh.xyz, mesh.periods)
    vol, _ = O.tet_geometry(mesh.xyz, mesh.tets)
    V = np.bincount(lca[mesh.tets].ravel(), weights=np.repeat(vol / 4.0, 4), minlength=n)
    for seed in (31, 32):
        m = meshgen.m_random(n, seed=seed)
        H = _field(h, 0, m, PMFEM_MS)
        assert np.sum(V[:, None] * m * H) < 0


def test_fp32_matches_fp64_at_full_size(wire):
    from paper_2409_13958_gb300 import PMFEM_EX, PMFEM_MS
    mesh, h = wire
    m = meshgen.m_vortex(h.folded_positions(), core=5e-9)
    m32 = m.astype(np.float32).astype(np.float64)             # the same input for both paths
    for comps, tol in ((PMFEM_MS, 1e-5), (PMFEM_EX, 1e-5)):
        H64 = _field(h, 0, m32, comps)
        H32 = _field(h, 1, m32, comps)
        assert np.linalg.norm(H32 - H64) <= tol * np.linalg.norm(H64), comps
