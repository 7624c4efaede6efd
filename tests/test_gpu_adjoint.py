"""Hand-written adjoint (lbve_adjoint_step) against finite differences of
the FP64 oracle.

Loss L = 1/2 sum |u(T) - u_t|^2 + 1/2 c sum (A_xy(T) - a_t)^2 over the fields
after T steps; gradient with respect to the per-node body force.  The oracle
gradient entries are fourth-order central differences
    (8 (L(+h) - L(-h)) - (L(+2h) - L(-2h))) / (12 h),
exact to O(h^4) plus round-off ~ eps L / h.  Tolerance 1e-6 relative to the
largest gradient entry (the stated target for the adjoint)."""
import numpy as np
import pytest

from oracle_helpers import oracle_sim
from paper_2508_16997_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbve():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_16997_gb300 import build, lbve as L
    build.build()
    return L


def loss_and_grad_fields(fields, ut, at, c):
    du = fields[1:3] - ut
    da = fields[4] - at
    L = 0.5 * np.sum(du * du) + 0.5 * c * np.sum(da * da)
    g = np.zeros_like(fields)
    g[1:3] = du
    g[4] = c * da
    return L, g


def oracle_loss(inst, F, T, init, ut, at, c):
    saved = inst.force_field
    inst.force_field = F
    try:
        s = oracle_sim(inst, init=init)
        s.step(T)
        return loss_and_grad_fields(s.fields(), ut, at, c)[0]
    finally:
        inst.force_field = saved


def fd_directional(inst, F, v, T, init, ut, at, c, h):
    Lp1 = oracle_loss(inst, F + h * v, T, init, ut, at, c)
    Lm1 = oracle_loss(inst, F - h * v, T, init, ut, at, c)
    Lp2 = oracle_loss(inst, F + 2 * h * v, T, init, ut, at, c)
    Lm2 = oracle_loss(inst, F - 2 * h * v, T, init, ut, at, c)
    return (8 * (Lp1 - Lm1) - (Lp2 - Lm2)) / (12 * h)


def gpu_gradient(L, inst, F, T, init, ut, at, c, precision=0):
    import torch
    inst.force_field = F
    sim = L.Simulation([inst], precision=precision, init_fields=[init])
    sim.step(T)
    fields = sim.fields(0)
    _, g = loss_and_grad_fields(fields, ut, at, c)
    d_g = torch.from_numpy(g).cuda()
    nbytes = L.lbve_adjoint_workspace_bytes(sim.h, 0, T)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    out = torch.empty((2, inst.ny, inst.nx), dtype=torch.float64, device="cuda")
    L.lbve_adjoint_step(sim.h, 0, init, d_g.data_ptr(), T, ws.data_ptr(), nbytes, out.data_ptr(),
                        inst.n_nodes)
    return out.cpu().numpy(), fields


CASES = {
    "frm_periodic": lambda: wl.frm(20, beta=0.5, Wi=0.7, Re=1.0, Ma=0.1, Sc=1e3),
    "channel_walls": lambda: wl.channel(12, nx=6, beta=0.5, Wi=2.0, Sc=1e3),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_adjoint_matches_oracle_fd(lbve, case):
    inst = CASES[case]()
    rng = np.random.default_rng(11)
    F = (inst.force_field if inst.force_field is not None else
         np.stack([np.full((inst.ny, inst.nx), inst.Fx), np.zeros((inst.ny, inst.nx))]))
    F = F + wl.random_force(inst.nx, inst.ny, seed=12, amp=2e-5)
    init = wl.random_fields(inst.nx, inst.ny, seed=13)
    T = 17
    ut = 1e-3 * rng.standard_normal((2, inst.ny, inst.nx))
    at = 0.05 * rng.standard_normal((inst.ny, inst.nx))
    c = 0.1
    g, _ = gpu_gradient(lbve, inst, F, T, init, ut, at, c)
    scale = np.abs(g).max()
    assert scale > 0
    h = 1e-6
    # individual entries
    idx = [(rng.integers(2), rng.integers(inst.ny), rng.integers(inst.nx)) for _ in range(8)]
    for comp, y, x in idx:
        v = np.zeros_like(F)
        v[comp, y, x] = 1.0
        fd = fd_directional(inst, F, v, T, init, ut, at, c, h)
        assert abs(g[comp, y, x] - fd) <= 1e-6 * scale, (case, comp, y, x, g[comp, y, x], fd)
    # random directions
    for _ in range(3):
        v = rng.standard_normal(F.shape)
        fd = fd_directional(inst, F, v, T, init, ut, at, c, h)
        ad = float(np.sum(g * v))
        assert abs(ad - fd) <= 1e-6 * np.abs(g).sum(), (ad, fd)


def test_adjoint_single_step_and_checkpoint_segments(lbve):
    """T = 1 (no full step between the initial collision and the loss) and a
    T whose checkpoint segments are ragged (T = 10: interval 4, segments 4+4+2)
    give the same gradients as the finite differences."""
    inst = wl.frm(12, beta=0.6, Wi=0.5, Re=1.0, Ma=0.1, Sc=1e2)
    F = inst.force_field + wl.random_force(12, 12, seed=3, amp=1e-5)
    init = wl.random_fields(12, 12, seed=4)
    rng = np.random.default_rng(5)
    ut = 1e-3 * rng.standard_normal((2, 12, 12))
    at = 0.05 * rng.standard_normal((12, 12))
    for T in (1, 10):
        g, _ = gpu_gradient(lbve, inst, F, T, init, ut, at, 0.1)
        v = rng.standard_normal(F.shape)
        fd = fd_directional(inst, F, v, T, init, ut, at, 0.1, 1e-6)
        assert abs(float(np.sum(g * v)) - fd) <= 1e-6 * np.abs(g).sum(), (T, np.sum(g * v), fd)


def test_autograd_function(lbve):
    """force_to_fields: torch autograd through the C ABI adjoint equals the
    direct lbve_adjoint_step gradient."""
    import torch
    inst = wl.frm(16, Wi=1.0, Re=1.0, Ma=0.1)
    init = wl.random_fields(16, 16, seed=21)
    sim = lbve.Simulation([inst], init_fields=[init])
    F = torch.tensor(inst.force_field, dtype=torch.float64, requires_grad=True)
    fields = lbve.force_to_fields(sim, 0, F, 9, init_fields=init)
    target = torch.zeros_like(fields)
    loss = 0.5 * ((fields[1:3] - target[1:3]) ** 2).sum()
    loss.backward()
    g_direct, _ = gpu_gradient(lbve, inst, inst.force_field.copy(), 9, init,
                               np.zeros((2, 16, 16)), np.zeros((16, 16)), 0.0)
    np.testing.assert_allclose(F.grad.cpu().numpy(), g_direct, rtol=1e-12, atol=1e-18)


def full_loss_and_grad(fields, tgt, wts):
    """L = 1/2 sum_k w_k sum (fields_k - tgt_k)^2 over all six fields."""
    d = fields - tgt
    L = 0.5 * float(np.sum(wts[:, None, None] * d * d))
    return L, wts[:, None, None] * d


@pytest.mark.parametrize("case", ["periodic", "walled"])
def test_adjoint_full_gradient_every_field(lbve, case):
    """Every entry of dL/dF against the oracle's finite differences, with a
    loss on all six fields (rho, u, Axx, Axy, Ayy), on tiny grids: relative L2
    error of the whole gradient <= 1e-7 (FP64)."""
    import torch
    if case == "periodic":
        inst = wl.frm(8, beta=0.4, Wi=0.6, Re=1.0, Ma=0.1, Sc=10.0)
    else:
        inst = wl.channel(6, nx=5, beta=0.7, Wi=1.5, Sc=10.0)
    ny, nx = inst.ny, inst.nx
    F = (inst.force_field if inst.force_field is not None else
         np.stack([np.full((ny, nx), inst.Fx), np.zeros((ny, nx))]))
    F = F + wl.random_force(nx, ny, seed=41, amp=5e-5)
    init = wl.random_fields(nx, ny, seed=42)
    rng = np.random.default_rng(43)
    T = 6
    tgt = init + 0.01 * rng.standard_normal(init.shape)
    wts = np.array([3.0, 1.0, 1.0, 0.2, 0.3, 0.4])
    inst.force_field = F
    sim = lbve.Simulation([inst], init_fields=[init])
    sim.step(T)
    _, gf = full_loss_and_grad(sim.fields(0), tgt, wts)
    d_g = torch.from_numpy(np.ascontiguousarray(gf)).cuda()
    nbytes = lbve.lbve_adjoint_workspace_bytes(sim.h, 0, T)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    out = torch.empty((2, ny, nx), dtype=torch.float64, device="cuda")
    lbve.lbve_adjoint_step(sim.h, 0, init, d_g.data_ptr(), T, ws.data_ptr(), nbytes,
                           out.data_ptr(), inst.n_nodes)
    g = out.cpu().numpy()

    def L_of(Fp):
        inst.force_field = Fp
        s = oracle_sim(inst, init=init)
        s.step(T)
        return full_loss_and_grad(s.fields(), tgt, wts)[0]

    h = 1e-6
    fd = np.zeros_like(F)
    for idx in np.ndindex(*F.shape):
        v = np.zeros_like(F)
        v[idx] = h
        fd[idx] = (8 * (L_of(F + v) - L_of(F - v)) - (L_of(F + 2 * v) - L_of(F - 2 * v))) / (12 * h)
    rel = np.linalg.norm(g - fd) / np.linalg.norm(fd)
    assert rel <= 1e-7, (case, rel)


def test_fp32_adjoint_matches_fp64(lbve):
    """The FP32-deviation adjoint on the four-roll mill (C1 parameters, 32^2,
    T = 50, 1% random force perturbation) agrees with the FP64 adjoint (which
    matches the oracle's finite differences) to 1e-6 relative L2; measured
    4.3e-7 (1.3e-6 after 200 steps)."""
    N, T = 32, 50
    inst = wl.frm(N, Wi=5.0)
    F = inst.force_field + wl.random_force(N, N, seed=1, amp=0.01 * np.abs(inst.force_field).max())
    init = np.zeros((6, N, N))
    init[0] = init[3] = init[5] = 1.0
    z2, z1 = np.zeros((2, N, N)), np.zeros((N, N))
    g64, _ = gpu_gradient(lbve, inst, F, T, init, z2, z1, 0.0, precision=0)
    g32, _ = gpu_gradient(lbve, inst, F, T, init, z2, z1, 0.0, precision=1)
    assert np.linalg.norm(g32 - g64) / np.linalg.norm(g64) <= 1e-6


@pytest.mark.parametrize("precision", [0, 1])
def test_adjoint_checkpoint_interval_does_not_change_gradient(lbve, precision):
    """The adjoint takes the shortest checkpoint interval whose workspace fits
    the bytes it is given.  With the square-root workspace (interval 6 for
    T = 30), an interval-4 workspace and an interval-1 workspace (every state
    stored, nothing recomputed) the gradients are bit-identical: each state
    is recomputed by the same step from the same predecessor.  A walled
    channel and a periodic mill with a disc mask cover the wall rows and the
    mask's scratch-copy path."""
    import torch
    T = 30
    insts = [wl.channel(10, nx=7, beta=0.5, Wi=2.0, Sc=1e3),
             wl.circle_box(16, 14, 3.2, 7.3, 6.6, Fx=2e-5, Sc=1e3)]
    for inst in insts:
        sim = lbve.Simulation([inst], precision=precision)
        sim.step(T)
        f = sim.fields(0)
        g = np.zeros_like(f)
        g[1:3] = f[1:3]
        g[4] = f[4]
        d_g = torch.from_numpy(g).cuda()
        sizes = [lbve.lbve_adjoint_workspace_bytes(sim.h, 0, T),
                 lbve.lbve_adjoint_workspace_bytes_interval(sim.h, 0, T, 4),
                 lbve.lbve_adjoint_workspace_bytes_interval(sim.h, 0, T, 1)]
        assert sizes[0] == lbve.lbve_adjoint_workspace_bytes_interval(sim.h, 0, T, 6)
        assert sizes[0] < sizes[1] < sizes[2]
        grads = []
        for nb in sizes:
            ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
            out = torch.empty((2, inst.ny, inst.nx), dtype=torch.float64, device="cuda")
            lbve.lbve_adjoint_step(sim.h, 0, None, d_g.data_ptr(), T, ws.data_ptr(), nb,
                                   out.data_ptr(), inst.n_nodes)
            grads.append(out.cpu().numpy())
        assert np.abs(grads[0]).max() > 0
        np.testing.assert_array_equal(grads[1], grads[0])
        np.testing.assert_array_equal(grads[2], grads[0])


def test_adjoint_workload_fd_gate_32(lbve):
    """The adjoint workload's finite-difference gate on a 32^2 oracle: the
    four-roll mill with the small configuration's parameters (beta 0.5,
    Wi 5, Re 0.01, Sc 1e5, Ma 1e-3), T = 2000 steps from rest (the adjoint
    workload's horizon; checkpoints every 45 steps), loss
    L = 1/2 sum |u(T) - u_t|^2 with u_t from the oracle run with the force
    F + 0.01 F0 xi (xi ~ N(0, 1) per node and component, seed 5).  The FP64
    adjoint against fourth-order central differences of the oracle with
    h = 1e-3 F0: the three largest and three random entries of dL/dF to 1e-6
    of the largest entry, and three random directions to 1e-6 relative.
    Calibration on the oracle: the directional difference at h = 1e-3 F0
    and at 1e-2 F0 agree to 5e-10 relative.  The 37 oracle runs (2 s each)
    go to a spawn pool over the host cores (this process holds a CUDA
    context)."""
    import copy
    import multiprocessing as mp
    import os
    import torch
    from oracle_helpers import oracle_fields_after
    N, T = 32, 2000
    inst = wl.frm(N)
    F = inst.force_field.copy()
    F0 = float(np.abs(F).max())
    xi = np.random.default_rng(5).standard_normal(F.shape)

    def with_force(Fp):
        i = copy.copy(inst)
        i.force_field = Fp
        return i

    workers = max(1, min(16, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(workers) as pool:
        ut = pool.map(oracle_fields_after, [(with_force(F + 0.01 * F0 * xi), T)])[0][1:3]
        sim = lbve.Simulation([inst], precision=0)
        sim.step(T)
        g_fields = np.zeros((6, N, N))
        g_fields[1:3] = sim.fields(0)[1:3] - ut
        d_g = torch.from_numpy(g_fields).cuda()
        nbytes = lbve.lbve_adjoint_workspace_bytes(sim.h, 0, T)
        ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        out = torch.empty((2, N, N), dtype=torch.float64, device="cuda")
        lbve.lbve_adjoint_step(sim.h, 0, None, d_g.data_ptr(), T, ws.data_ptr(), nbytes,
                               out.data_ptr(), inst.n_nodes)
        g = out.cpu().numpy()
        scale = np.abs(g).max()
        assert scale > 0

        rng = np.random.default_rng(6)
        dirs = []
        for flat in list(np.argsort(np.abs(g).ravel())[-3:]) + list(rng.integers(g.size, size=3)):
            v = np.zeros(g.size)
            v[flat] = 1.0
            dirs.append(("entry", v.reshape(g.shape)))
        for _ in range(3):
            dirs.append(("direction", rng.standard_normal(g.shape)))
        h = 1e-3 * F0
        jobs = [(with_force(F + s * h * v), T) for _, v in dirs for s in (1, -1, 2, -2)]
        us = [f[1:3] for f in pool.map(oracle_fields_after, jobs)]
    losses = np.array([0.5 * float(((u - ut) ** 2).sum()) for u in us]).reshape(len(dirs), 4)
    for (kind, v), (lp1, lm1, lp2, lm2) in zip(dirs, losses):
        fd = (8 * (lp1 - lm1) - (lp2 - lm2)) / (12 * h)
        ad = float(np.sum(g * v))
        if kind == "entry":
            assert abs(ad - fd) <= 1e-6 * scale, (kind, ad, fd, scale)
        else:
            assert abs(ad - fd) <= 1e-6 * abs(fd), (kind, ad, fd)
