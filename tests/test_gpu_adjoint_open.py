"""The adjoint of open channels (inlet and outlet columns completed from the
neighbouring column, Sec. 4.3 set-up) against fourth-order central
differences of the FP64 oracle.

Two cases, T = 20 steps from random initial fields with a random per-node
force: a walled Oldroyd-B channel open in x whose inlet profile does not
match its own flow (a transverse inlet velocity included), and the paper's
cylinder set-up at a small size (inlet profile, outlet at density 1, curved
cylinder walls).  Loss
    L = 1/2 sum |u(T) - u_t|^2 + 1/2 c sum (A_xy(T) - a_t)^2 [+ a F_x + b F_y],
the bracket the force on the cylinder over the final step (eq_F_x).
Checked: dL/dF along random directions and at single nodes of the inlet and
outlet columns and their neighbours (wall rows included), and for the
cylinder dL/dq of single wall links.  Tolerance 1e-6 relative to the largest
gradient entry, as for the closed-channel adjoint."""
import numpy as np
import pytest

from oracle_helpers import oracle_sim
from paper_2508_16997_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
T = 20
C_AXY = 2.0
DRAG_W = (1.0, 0.3)


@pytest.fixture(scope="module")
def lbve():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_16997_gb300 import build, lbve as L
    build.build()
    return L


def open_channel():
    H, nx = 9, 12
    inst = wl.channel(H, nx=nx, Wi=2.0, Sc=1e3, Ma=0.1)
    Uc = wl.velocity_scale(inst.Ma)
    prof = wl.poiseuille_inlet(H, 1.4 * Uc, 30.0)
    prof[1] = 0.1 * prof[0]
    inst.open_x = True
    inst.inlet = prof
    inst.force_field = wl.random_force(nx, H + 1, seed=91, amp=3e-4)
    inst.force_field[0] += inst.Fx
    return inst


def open_cylinder():
    inst = wl.cylinder_channel(2, L=16, H=10, Wi=0.8, Sc=1e3, Ma=0.1, open_x=True)
    inst.force_field = wl.random_force(inst.nx, inst.ny, seed=92, amp=3e-4)
    return inst


CASES = {"open_channel": open_channel, "open_cylinder": open_cylinder}


def targets(inst, seed):
    rng = np.random.default_rng(seed)
    ut = 0.01 * rng.standard_normal((2, inst.ny, inst.nx))
    at = 0.1 * rng.standard_normal((inst.ny, inst.nx))
    return ut, at


def field_loss(fields, ut, at):
    du = fields[1:3] - ut
    da = fields[4] - at
    g = np.zeros_like(fields)
    g[1:3] = du
    g[4] = C_AXY * da
    return 0.5 * np.sum(du * du) + 0.5 * C_AXY * np.sum(da * da), g


def oracle_loss(inst, init, ut, at, F, q=None):
    saved = inst.force_field
    inst.force_field = F
    try:
        s = oracle_sim(inst, init=init)
        masked = inst.solid is not None
        if masked:
            s.set_mask(inst.solid, inst.wall_q if q is None else q)
        s.step(T)
        loss = field_loss(s.fields(), ut, at)[0]
        if masked:
            tot = s.totals()
            loss += DRAG_W[0] * tot[12] + DRAG_W[1] * tot[13]
        return loss
    finally:
        inst.force_field = saved


def fd4(f, h):
    return (8 * (f(h) - f(-h)) - (f(2 * h) - f(-2 * h))) / (12 * h)


@pytest.fixture(scope="module", params=sorted(CASES))
def gpu(request, lbve):
    import torch
    L = lbve
    inst = CASES[request.param]()
    init = wl.random_fields(inst.nx, inst.ny, seed=93)
    ut, at = targets(inst, 94)
    sim = L.Simulation([inst], precision=0, init_fields=[init])
    sim.step(T)
    _, g = field_loss(sim.fields(0), ut, at)
    d_g = torch.from_numpy(g).cuda()
    nbytes = L.lbve_adjoint_workspace_bytes(sim.h, 0, T)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    dF = torch.empty((2, inst.ny, inst.nx), dtype=torch.float64, device="cuda")
    masked = inst.solid is not None
    dq = torch.empty((8, inst.ny, inst.nx), dtype=torch.float64, device="cuda") if masked else None
    L.lbve_adjoint_step_ex(sim.h, 0, init, d_g.data_ptr(), DRAG_W if masked else None, T,
                           ws.data_ptr(), nbytes, dF.data_ptr(),
                           None if dq is None else dq.data_ptr(), inst.n_nodes)
    return (request.param, inst, init, ut, at, dF.cpu().numpy(),
            None if dq is None else dq.cpu().numpy())


def test_open_adjoint_force_gradient(gpu):
    name, inst, init, ut, at, dF, _ = gpu
    F0 = inst.force_field.copy()
    fluid = np.ones((inst.ny, inst.nx)) if inst.solid is None else (inst.solid == 0)
    scale = np.abs(dF).max()
    assert scale > 0
    rng = np.random.default_rng(95)
    checks = []
    for _ in range(2):
        v = rng.standard_normal(F0.shape) * fluid
        fd = fd4(lambda h: oracle_loss(inst, init, ut, at, F0 + h * v), 1e-5)
        checks.append(("random", fd, float(np.sum(dF * v)), np.abs(v).sum()))
    # single entries on the inlet and outlet columns and their neighbours,
    # on wall rows and inside
    nx, ny = inst.nx, inst.ny
    for (c, y, x) in ((0, 0, 0), (1, ny // 2, 0), (0, ny - 1, 1), (1, 3, 1), (0, 4, 2),
                      (0, ny // 2, nx - 1), (1, 0, nx - 1), (0, ny - 1, nx - 2), (1, 2, nx - 3)):
        v = np.zeros_like(F0)
        v[c, y, x] = 1.0
        fd = fd4(lambda h: oracle_loss(inst, init, ut, at, F0 + h * v), 1e-5)
        checks.append(((c, y, x), fd, float(dF[c, y, x]), 1.0))
    for where, fd, ad, norm in checks:
        assert abs(fd - ad) <= 1e-6 * scale * norm, (name, where, fd, ad)


def test_open_adjoint_wall_fraction_gradient(gpu):
    """dL/dq of single cylinder wall links on both interpolation branches."""
    name, inst, init, ut, at, _, dq = gpu
    if dq is None:
        pytest.skip("no mask in this case")
    links = inst.wall_links()
    lo = [(k, i, q) for k, i, q in links if q < 0.45]
    hi = [(k, i, q) for k, i, q in links if 0.55 < q < 0.99]  # q + 2h stays in (0, 1]
    assert lo and hi
    scale = np.abs(dq).max()
    assert scale > 0
    for k, i, q in lo[:2] + hi[:2]:
        y, x = divmod(k, inst.nx)

        def f(h, y=y, x=x, i=i):
            qq = inst.wall_q.copy()
            qq[i, y, x] += h
            return oracle_loss(inst, init, ut, at, inst.force_field, qq)
        fd = fd4(f, 1e-5)
        ad = dq[i - 1, y, x]
        assert abs(fd - ad) <= 1e-6 * max(scale, abs(fd)), (k, i, q, fd, ad)
