"""The learned surrogate through the C-ABI: forward pass and gradients against the FP64
network oracle (oracle/surrogate.py), the Adam step, training on pairs the method itself
produces, and its use inside the RK4 step with the full P-AIM as judge."""
import numpy as np
import pytest

import meshgen
from oracle import surrogate as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _flat(params):
    return np.concatenate([p.ravel() for p in params]).astype(np.float32)


def _unflat(v, like):
    out, o = [], 0
    for p in like:
        out.append(v[o:o + p.size].reshape(p.shape).astype(np.float64))
        o += p.size
    return out


def _handle(kind):
    from paper_2409_13958_gb300 import Pmfem, PMFEM_FP32
    if kind == "cube":          # 3D periodic, grid 8 x 8 x 8 (circular padding on every axis)
        mesh, grid = meshgen.cube_cell(4, jitter=0.2, seed=61), (8, 8, 8)
    elif kind == "cube16":      # 3D periodic, grid 16^3: the tensor-core path with bfloat16 activations
        mesh, grid = meshgen.cube_cell(6, jitter=0.2, seed=63), (16, 16, 16)
    elif kind == "film16":      # 2D periodic film, grid 16 x 16 x 8 (tensor-core path, zero padding along z)
        mesh, grid = meshgen.film_cell(10, 10, 2, seed=64), (16, 16, 8)
    elif kind == "film64":      # grid 64 x 64 x 8: 128 tensor-core tiles, zero padding along z
        mesh, grid = meshgen.film_cell(10, 10, 2, seed=65), (64, 64, 8)
    elif kind == "cube64x32":   # grid 64 x 64 x 32, 3D periodic: 512 tensor-core tiles
        mesh, grid = meshgen.cube_cell(6, jitter=0.2, seed=66), (64, 64, 32)
    else:                       # 2D periodic film, grid 16 x 8 x 8 with zero padding along z
        mesh, grid = meshgen.film_cell(10, 6, 2, seed=62), (16, 8, 8)
    h = Pmfem.create_mesh(mesh.xyz, mesh.tets, 8e5, 1.3e-11, 0.02)
    h.set_aim(*grid, 3, 2, 0.0)
    h.set_periodicity(*mesh.periods)
    h.set_precision(PMFEM_FP32)
    dims = tuple(int(x) for x in h.grid_info()[0])
    return h, mesh, dims, tuple(p > 0 for p in mesh.periods)


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("kind,bf16,tol", [("cube", False, 1e-5), ("film", False, 1e-5), ("film", True, 2e-2),
                                          ("cube16", True, 2e-2), ("film16", True, 2e-2), ("film16", False, 1e-5),
                                          ("film64", True, 2e-2), ("cube64x32", True, 2e-2)])
def test_forward_matches_oracle(kind, bf16, tol):
    h, mesh, dims, per = _handle(kind)
    if kind == "cube64x32":
        # tensor-core tiles of 8 x 16 x 2 voxels, one persistent block per SM: at least three tiles
        # per block, so that the three halo stages and the two accumulator pairs are reused
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        assert (dims[0] // 8) * (dims[1] // 16) * (dims[2] // 2) >= 3 * sms
    params = S.init_params(C=32, seed=5)
    for k in range(1, 8, 2):
        params[k] = np.random.default_rng(10 + k).normal(0, 0.05, params[k].shape)
    sq, su = 2.5, 0.7
    h.surrogate_set_params(_flat(params), sq, su, act_bf16=bf16)
    Q = np.random.default_rng(3).standard_normal(dims[::-1])          # [Z, Y, X]
    Qd = torch.tensor(Q, dtype=torch.float32, device="cuda")
    Ud = torch.empty_like(Qd)
    h.surrogate_apply(Qd, Ud)
    h.sync()
    ref, _ = S.forward(params, Q, sq, su, per)
    assert _rel(Ud.double().cpu().numpy(), ref) <= tol
    back = h.surrogate_get_params()
    assert np.array_equal(back, _flat(params))
    h.destroy()


@pytest.mark.parametrize("kind,bf16,tol", [("cube", False, 1e-4), ("film", False, 1e-4), ("film16", True, 5e-2)])
def test_gradients_match_oracle(kind, bf16, tol):
    h, mesh, dims, per = _handle(kind)
    params = S.init_params(C=32, seed=6)
    for k in range(1, 8, 2):
        params[k] = np.random.default_rng(20 + k).normal(0, 0.05, params[k].shape)
    sq, su = 1.5, 0.4
    h.surrogate_set_params(_flat(params), sq, su, act_bf16=bf16)
    rng = np.random.default_rng(7)
    Q = rng.standard_normal(dims[::-1])
    U = rng.standard_normal(dims[::-1])
    loss, g = h.surrogate_grad(torch.tensor(Q, dtype=torch.float32, device="cuda"),
                               torch.tensor(U, dtype=torch.float32, device="cuda"))
    ref_loss, ref_g = S.loss_and_grad(params, Q, U, sq, su, per)
    assert abs(loss - ref_loss) <= 0.1 * tol * ref_loss
    for k, (a, b) in enumerate(zip(_unflat(g, params), ref_g)):
        assert _rel(a, b) <= tol, k
    h.destroy()


def test_one_adam_step_matches_oracle():
    h, mesh, dims, per = _handle("cube")
    params = S.init_params(C=32, seed=8)
    sq, su, lr = 1.0, 1.0, 1e-3
    h.surrogate_set_params(_flat(params), sq, su)
    rng = np.random.default_rng(9)
    Q = rng.standard_normal(dims[::-1])
    U = rng.standard_normal(dims[::-1])
    h.surrogate_train(torch.tensor(Q, dtype=torch.float32, device="cuda"),
                      torch.tensor(U, dtype=torch.float32, device="cuda"), 1, epochs=1, batch=1, lr=lr)
    after = _unflat(h.surrogate_get_params(), params)
    _, g = S.loss_and_grad(params, Q, U, sq, su, per)
    m = [np.zeros_like(p) for p in params]
    v = [np.zeros_like(p) for p in params]
    ref = [p.copy() for p in params]
    S.adam_step(ref, g, m, v, 1, lr=lr)
    for k in range(8):
        big = np.abs(g[k]) > 1e-3 * np.abs(g[k]).max()     # the first Adam step is lr * sign(g) there
        assert np.allclose((after[k] - params[k])[big], (ref[k] - params[k])[big], rtol=0, atol=1e-3 * lr), k
    h.destroy()


def _pairs(h, n, seed):
    """Grid pairs (Q, U) of the method for n seeded random magnetisations, and their increments."""
    Np = h.num_unknowns()
    dims = tuple(int(x) for x in h.grid_info()[0])
    V = dims[0] * dims[1] * dims[2]
    Q = torch.empty((n, V), dtype=torch.float32, device="cuda")
    U = torch.empty_like(Q)
    base = meshgen.m_tilted(Np, polar_deg=20.0, seed=seed)
    rng = np.random.default_rng(seed)
    for k in range(n):
        m = base + 0.05 * rng.standard_normal(base.shape)
        m /= np.linalg.norm(m, axis=1, keepdims=True)
        h.grid_pair(torch.tensor(m, dtype=torch.float32, device="cuda"), Q[k], U[k])
    h.sync()
    return Q, U


def test_training_on_method_pairs_lowers_the_loss():
    h, mesh, dims, per = _handle("film")
    Q, U = _pairs(h, 12, seed=70)
    dQ, dU = (Q[1:] - Q[:1]).contiguous(), (U[1:] - U[:1]).contiguous()   # increments, as used in RK stages
    sq = float(dQ.std()) or 1.0
    su = float(dU.std()) or 1.0
    h.surrogate_set_params(_flat(S.init_params(C=32, seed=11)), sq, su)
    losses = h.surrogate_train(dQ, dU, dQ.shape[0], epochs=40, batch=1, lr=2e-3)
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.25 * losses[0], losses
    h.destroy()


def test_rk4_with_surrogate_is_judged_and_stays_normalised():
    h, mesh, dims, per = _handle("film")
    h.surrogate_set_params(_flat(S.init_params(C=32, seed=12)), 1.0, 1.0)
    Np = h.num_unknowns()
    m = torch.tensor(meshgen.m_tilted(Np, polar_deg=10.0, seed=3), dtype=torch.float32, device="cuda")
    h.set_m(m)
    h.surrogate_enable(2)
    h.llg_step(1e-14, 4)
    out = torch.empty_like(m)
    h.get_m(out)
    h.sync()
    st = h.surrogate_stats()
    assert st["steps"] == 4 and st["judged_stages"] == 6 and st["net_stages"] == 6, st
    assert np.isfinite(st["judged_rel_l2"])
    nrm = np.linalg.norm(out.double().cpu().numpy(), axis=1)
    assert np.abs(nrm - 1).max() < 1e-6
    h.surrogate_enable(0)
    h.destroy()


def test_trained_network_beats_the_frozen_potential():
    """What the trained network gains: on RK stages 2-4 the step either freezes the potential
    of stage 1 (a network that outputs zero) or adds the trained network's increment.  The
    full P-AIM judges both on the same steps; the trained network must be closer to it."""
    h, mesh, dims, per = _handle("film")
    Np = h.num_unknowns()
    V = dims[0] * dims[1] * dims[2]
    # training increments from the method's own trajectory
    dt = 2e-14
    steps = 24
    Q = torch.empty((steps, V), dtype=torch.float32, device="cuda")
    U = torch.empty_like(Q)
    m = torch.tensor(meshgen.m_tilted(Np, polar_deg=30.0, seed=80), dtype=torch.float32, device="cuda")
    h.set_m(m)
    for k in range(steps):
        h.get_m(m)
        h.grid_pair(m, Q[k], U[k])
        h.llg_step(dt, 1)
    h.sync()
    dQ = (Q[1:] - Q[:-1]).contiguous()
    dU = (U[1:] - U[:-1]).contiguous()
    sq, su = float(dQ.std()), float(dU.std())

    def judged_error(params):
        h.surrogate_set_params(params, sq, su)
        h.set_m(torch.tensor(meshgen.m_tilted(Np, polar_deg=30.0, seed=81), dtype=torch.float32, device="cuda"))
        h.surrogate_enable(1)            # judge every step: the error of every network stage is measured
        h.llg_step(dt, 6)
        st = h.surrogate_stats()
        h.surrogate_enable(0)
        return st["judged_rel_l2"]

    frozen = judged_error(np.zeros(h.NET_PARAMS, dtype=np.float32))
    h.surrogate_set_params(_flat(S.init_params(C=32, seed=14)), sq, su)
    h.surrogate_train(dQ, dU, dQ.shape[0], epochs=60, batch=1, lr=2e-3)
    trained = judged_error(h.surrogate_get_params())
    assert trained < frozen, (trained, frozen)
    h.destroy()
