"""Implicit midpoint LLG steps with Newton-GMRES (pmfem_llg_step_implicit) against the oracle's
stepper of the same scheme (oracle/implicit.py), on the 2D-periodic film, through the C-ABI.

Both sides iterate Newton to a small relative correction, so the converged states agree to
about the tolerance of the iterations (FP64 1e-9; FP32 1e-4: its Newton stops at 1e-5 and its
field carries the FP32 rounding amplified by the large step).  The step, 1e-13 s, is about four
times the largest stable RK4 step on these 1 nm elements."""
import numpy as np
import pytest

import meshgen
from oracle.implicit import MidpointStepper
from oracle.operators import MU0
from oracle.problem import OracleProblem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

H_AP = (1e4, 0.0, 2e4)
DT = 1e-13


@pytest.fixture(scope="module")
def film():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    mesh = meshgen.film_cell(10, 10, 2, seed=3)
    pb = OracleProblem(mesh.xyz, mesh.tets, mesh.periods, grid=(16, 16, 8), near_boxes=3, H_ap=H_AP)
    c = -(2 * pb.A / (MU0 * pb.Ms)) * pb.K.diagonal() / pb.V
    return mesh, pb, c


def _handle(mesh, prec):
    from paper_2409_13958_gb300 import Pmfem
    h = Pmfem.create_mesh(mesh.xyz, mesh.tets, 8e5, 1.3e-11, 0.02)
    h.set_aim(16, 16, 8, 3, 3, 0.0)
    h.set_periodicity(*mesh.periods)
    h.set_precision(prec)
    h.set_applied_field(*H_AP)
    return h


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-4)])
@pytest.mark.parametrize("m0", ["tilted", "random"])
def test_implicit_steps_match_the_oracle(film, prec, tol, m0):
    mesh, pb, c = film
    m = meshgen.m_tilted(pb.Np, 5.0, seed=1) if m0 == "tilted" else meshgen.m_random(pb.Np, seed=8)
    if prec:
        m = m.astype(np.float32).astype(np.float64)
    st = MidpointStepper(lambda x: pb.h_eff(x, "paim"), lambda v: pb.h_eff(v, "paim", ap=False), c, pb.alpha,
                         newton_tol=1e-12, gmres_tol=1e-10)
    ref = m
    for _ in range(3):
        ref = st.step(ref, DT)
    h = _handle(mesh, prec)
    dt_t = torch.float64 if prec == 0 else torch.float32
    h.set_m(torch.tensor(m, dtype=dt_t, device="cuda"))
    nt, kt = (1e-12, 1e-10) if prec == 0 else (0.0, 0.0)
    stats = h.llg_step_implicit(DT, 3, newton_tol=nt, krylov_tol=kt)
    out = torch.empty((pb.Np, 3), dtype=dt_t, device="cuda")
    h.get_m(out)
    h.sync()
    got = out.double().cpu().numpy()
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref - m)
    assert err <= tol, (err, stats)
    assert np.abs(np.linalg.norm(got, axis=1) - 1).max() <= (1e-10 if prec == 0 else 1e-5)
    assert stats["steps"] == 3 and stats["newton"] >= 3 and stats["krylov"] > 0
    assert stats["field_evals"] >= stats["newton"] + stats["krylov"]      # one per residual and per J v
    h.destroy()


def test_implicit_reports_no_convergence_and_keeps_the_state(film):
    from paper_2409_13958_gb300 import PmfemError
    mesh, pb, c = film
    h = _handle(mesh, 0)
    m = torch.tensor(meshgen.m_random(pb.Np, seed=9), dtype=torch.float64, device="cuda")
    h.set_m(m)
    with pytest.raises(PmfemError) as e:
        h.llg_step_implicit(DT, 2, newton_tol=1e-14, max_newton=1)
    assert e.value.code == -8
    out = torch.empty_like(m)
    h.get_m(out)
    h.sync()
    assert torch.equal(out, m)
    h.destroy()
