"""The hand-written adjoint (genga_adjoint_*) of kick-drift-kick steps with
frozen encounters, through the C ABI:
  * replaying the oracle's recorded rc and pairs reproduces the oracle's run;
  * the adjoint and the oracle's tangent-linear integration satisfy
    <lam_N, T delta> = <A lam_N, delta> (dot-product identity);
  * the adjoint matches central finite differences (h = 1e-7 in state units)
    taken on the GPU with the same frozen records;
  * gradients do not depend on the checkpoint interval;
  * torch.autograd reaches the same gradients.
"""
import numpy as np
import pytest

import oracle as O
from workloads import disk

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


@pytest.fixture(scope="module")
def case():
    wl = disk(160, 0.9, 1.1, 2.0, 31, name="dense")
    p = O.make_params(wl, nthreads=8)
    x, v = wl.x, wl.v
    rcs, pairs = [], []
    for _ in range(6):
        x, v, rc, pr, st = O.step_record(x, v, wl.m, p)
        assert st == 0
        rcs.append(rc)
        pairs.append(pr)
    assert sum(len(q) for q in pairs) > 0
    return wl, p, np.array(rcs), pairs, x, v


def _system(g, wl, x=None, v=None):
    torch = _torch()
    dev = torch.device("cuda:0")
    pos = torch.tensor(np.ascontiguousarray((wl.x if x is None else x).T), device=dev)
    vel = torch.tensor(np.ascontiguousarray((wl.v if v is None else v).T), device=dev)
    mass = torch.tensor(wl.m, device=dev)
    p = g.default_params(G=wl.G, m_star=wl.m_star, dt=wl.dt, n1=wl.n1, n2=wl.n2, f_pc=wl.f_pc)
    return g.System(pos, vel, mass, p), pos, vel, mass


def test_replay_of_oracle_records_matches_oracle(cuda_lib, case):
    wl, p, rcs, pairs, xN, vN = case
    s, pos, vel, mass = _system(cuda_lib, wl)
    s.adjoint_load(2, rcs, pairs)
    xg = pos.cpu().numpy().T
    assert np.abs(xg - xN).max() <= 1e-12 * np.abs(xN).max()


def _directions(wl, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(wl.x.shape), rng.standard_normal(wl.v.shape) * 0.017,
            rng.standard_normal(wl.m.shape) * wl.m)


def test_adjoint_dot_product_identity_with_oracle_tangent(cuda_lib, case):
    torch = _torch()
    wl, p, rcs, pairs, xN, vN = case
    dx0, dv0, dm0 = _directions(wl, 1)
    x, v, dx, dv = wl.x, wl.v, dx0, dv0
    for rc, pr in zip(rcs, pairs):
        x, v, dx, dv, st = O.step_frozen(x, v, wl.m, p, rc, pr, dx, dv, dm0)
        assert st == 0
    rng = np.random.default_rng(2)
    lx, lv = rng.standard_normal(wl.x.shape), rng.standard_normal(wl.v.shape)
    lhs = (lx * dx).sum() + (lv * dv).sum()
    s, pos, vel, mass = _system(cuda_lib, wl)
    s.adjoint_load(3, rcs, pairs)
    T = lambda a: torch.tensor(np.ascontiguousarray(a.T), device="cuda:0")
    gx, gv, gm = s.adjoint_backward(T(lx), T(lv))
    gx, gv, gm = gx.cpu().numpy().T, gv.cpu().numpy().T, gm.cpu().numpy()
    rhs = (gx * dx0).sum() + (gv * dv0).sum() + (gm * dm0).sum()
    scale = abs((gx * dx0).sum()) + abs((gv * dv0).sum()) + abs((gm * dm0).sum())
    assert abs(lhs - rhs) <= 1e-9 * scale, (lhs, rhs)


def test_adjoint_matches_gpu_finite_differences(cuda_lib, case):
    torch = _torch()
    g = cuda_lib
    wl, p, rcs, pairs, xN, vN = case
    dx0, dv0, dm0 = _directions(wl, 5)
    rng = np.random.default_rng(6)
    lx, lv = rng.standard_normal(wl.x.shape), rng.standard_normal(wl.v.shape)

    def final(eps):
        s, pos, vel, mass = _system(g, wl, wl.x + eps * dx0, wl.v + eps * dv0)
        mass.copy_(torch.tensor(wl.m + eps * dm0))
        s.adjoint_load(6, rcs, pairs)
        return pos.cpu().numpy().T, vel.cpu().numpy().T

    h = 1e-7
    xp, vp = final(h)
    xm, vm = final(-h)
    fd = ((lx * (xp - xm)).sum() + (lv * (vp - vm)).sum()) / (2 * h)
    s, pos, vel, mass = _system(g, wl)
    s.adjoint_load(6, rcs, pairs)
    T = lambda a: torch.tensor(np.ascontiguousarray(a.T), device="cuda:0")
    gx, gv, gm = s.adjoint_backward(T(lx), T(lv))
    ad = ((gx.cpu().numpy().T * dx0).sum() + (gv.cpu().numpy().T * dv0).sum()
          + (gm.cpu().numpy() * dm0).sum())
    assert abs(ad - fd) <= 1e-6 * abs(ad), (ad, fd)


def test_gradients_do_not_depend_on_checkpoint_interval(cuda_lib, case):
    torch = _torch()
    wl, p, rcs, pairs, xN, vN = case
    rng = np.random.default_rng(8)
    T = lambda a: torch.tensor(np.ascontiguousarray(a.T), device="cuda:0")
    lx, lv = T(rng.standard_normal(wl.x.shape)), T(rng.standard_normal(wl.v.shape))
    out = []
    for every in (1, 4, 6):
        s, pos, vel, mass = _system(cuda_lib, wl)
        s.adjoint_load(every, rcs, pairs)
        out.append([t.cpu().numpy() for t in s.adjoint_backward(lx, lv)])
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
    for a, b in zip(out[0], out[2]):
        assert np.array_equal(a, b)


def test_own_recording_and_autograd(cuda_lib, case):
    torch = _torch()
    from paper_2201_10058_gb300.autograd import integrate
    g = cuda_lib
    wl = disk(256, 0.5, 2.0, 2.0, 20110062, name="adjoint-disk")
    dev = torch.device("cuda:0")
    x0 = torch.tensor(np.ascontiguousarray(wl.x.T), device=dev, requires_grad=True)
    v0 = torch.tensor(np.ascontiguousarray(wl.v.T), device=dev, requires_grad=True)
    m = torch.tensor(wl.m, device=dev, requires_grad=True)
    p = g.default_params(G=wl.G, m_star=wl.m_star, dt=wl.dt)
    xN, vN = integrate(x0, v0, m, p, 12, 4)
    rng = np.random.default_rng(9)
    wx = torch.tensor(rng.standard_normal((3, wl.n)), device=dev)
    loss = (wx * xN).sum()
    loss.backward()
    assert x0.grad is not None and v0.grad is not None and m.grad is not None
    # directional check against finite differences of the same recorded run
    s, pos, vel, mass = _system(g, wl)
    s.adjoint_forward(12, 4)
    assert np.allclose(pos.cpu().numpy(), xN.detach().cpu().numpy(), rtol=0, atol=0)
    gx, gv, gm = s.adjoint_backward(wx, torch.zeros_like(wx))
    np.testing.assert_array_equal(gx.cpu().numpy(), x0.grad.cpu().numpy())
    np.testing.assert_array_equal(gm.cpu().numpy(), m.grad.cpu().numpy())


def test_exported_recording_replays_bit_exactly(cuda_lib):
    wl = disk(200, 0.9, 1.1, 2.0, 41, name="dense2")
    s, pos, vel, mass = _system(cuda_lib, wl)
    s.adjoint_forward(5, 2)
    rc, pairs = s.adjoint_export()
    assert rc.shape == (5, wl.n) and len(pairs) == 5 and sum(len(q) for q in pairs) > 0
    s2, pos2, vel2, _ = _system(cuda_lib, wl)
    s2.adjoint_load(2, rc, pairs)
    assert np.array_equal(pos.cpu().numpy(), pos2.cpu().numpy())
    assert np.array_equal(vel.cpu().numpy(), vel2.cpu().numpy())
