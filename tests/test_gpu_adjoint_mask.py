"""The adjoint with a solid mask (lbve_adjoint_step_ex) against fourth-order
central differences of the FP64 oracle.

A disc with curved wall fractions in a periodic box, a random per-node force
and random initial fields, T = 20 steps.  Loss
    L = 1/2 sum |u(T) - u_t|^2 + 1/2 c sum (A_xy(T) - a_t)^2 + a F_x + b F_y,
the last two terms the force on the disc over the final step (eq_F_x).
Checked: dL/dF along random directions and at single nodes next to the
disc, and dL/dq of single wall links on both interpolation branches
(q < 1/2 with a second fluid node, q >= 1/2) -- the gradient with respect to
the wall geometry.  Tolerance 1e-6 relative to the largest gradient entry,
as for the mask-free adjoint."""
import numpy as np
import pytest

from oracle_helpers import oracle_sim
from paper_2508_16997_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
T = 20
DRAG_W = (1.0, 0.3)
C_AXY = 2.0


@pytest.fixture(scope="module")
def lbve():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_16997_gb300 import build, lbve as L
    build.build()
    return L


def make_case():
    inst = wl.circle_box(14, 12, R=2.7, cx=6.3, cy=5.6, Fx=0.0, Wi=0.8, Sc=1e3, Ma=0.1)
    inst.force_field = wl.random_force(14, 12, seed=81, amp=3e-4)
    init = wl.random_fields(14, 12, seed=82)
    rng = np.random.default_rng(83)
    ut = 0.01 * rng.standard_normal((2, 12, 14))
    at = 0.1 * rng.standard_normal((12, 14))
    return inst, init, ut, at


def field_loss(fields, ut, at):
    du = fields[1:3] - ut
    da = fields[4] - at
    g = np.zeros_like(fields)
    g[1:3] = du
    g[4] = C_AXY * da
    return 0.5 * np.sum(du * du) + 0.5 * C_AXY * np.sum(da * da), g


def oracle_loss(inst, init, ut, at, F, q):
    saved = inst.force_field
    inst.force_field = F
    try:
        s = oracle_sim(inst, init=init)
        s.set_mask(inst.solid, q)
        s.step(T)
        tot = s.totals()
        return field_loss(s.fields(), ut, at)[0] + DRAG_W[0] * tot[12] + DRAG_W[1] * tot[13]
    finally:
        inst.force_field = saved


def fd4(f, h):
    return (8 * (f(h) - f(-h)) - (f(2 * h) - f(-2 * h))) / (12 * h)


@pytest.fixture(scope="module")
def gpu(lbve):
    import torch
    L = lbve
    inst, init, ut, at = make_case()
    sim = L.Simulation([inst], precision=0, init_fields=[init])
    sim.step(T)
    _, g = field_loss(sim.fields(0), ut, at)
    d_g = torch.from_numpy(g).cuda()
    nbytes = L.lbve_adjoint_workspace_bytes(sim.h, 0, T)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    dF = torch.empty((2, 12, 14), dtype=torch.float64, device="cuda")
    dq = torch.empty((8, 12, 14), dtype=torch.float64, device="cuda")
    L.lbve_adjoint_step_ex(sim.h, 0, init, d_g.data_ptr(), DRAG_W, T, ws.data_ptr(), nbytes,
                           dF.data_ptr(), dq.data_ptr(), inst.n_nodes)
    return inst, init, ut, at, dF.cpu().numpy(), dq.cpu().numpy()


def test_mask_adjoint_force_gradient(gpu):
    inst, init, ut, at, dF, _ = gpu
    F0 = inst.force_field.copy()
    q0 = inst.wall_q
    scale = np.abs(dF).max()
    assert scale > 0
    rng = np.random.default_rng(84)
    checks = []
    for _ in range(2):
        v = rng.standard_normal(F0.shape) * (inst.solid == 0)
        fd = fd4(lambda h: oracle_loss(inst, init, ut, at, F0 + h * v, q0), 1e-5)
        checks.append((fd, float(np.sum(dF * v)), np.abs(v).sum()))
    # single entries next to the disc
    for (c, y, x) in ((0, 2, 6), (1, 5, 9), (0, 8, 4)):
        if inst.solid[y, x]:
            continue
        v = np.zeros_like(F0)
        v[c, y, x] = 1.0
        fd = fd4(lambda h: oracle_loss(inst, init, ut, at, F0 + h * v, q0), 1e-5)
        checks.append((fd, float(dF[c, y, x]), 1.0))
    for fd, ad, norm in checks:
        assert abs(fd - ad) <= 1e-6 * scale * norm, (fd, ad)


def test_mask_adjoint_wall_fraction_gradient(gpu):
    """dL/dq of single wall links on both interpolation branches."""
    inst, init, ut, at, _, dq = gpu
    links = inst.wall_links()
    lo = [(k, i, q) for k, i, q in links if q < 0.45]
    hi = [(k, i, q) for k, i, q in links if q > 0.55]
    assert lo and hi
    pick = lo[:2] + hi[:2]
    scale = np.abs(dq).max()
    assert scale > 0
    for k, i, q in pick:
        y, x = divmod(k, inst.nx)

        def f(h, y=y, x=x, i=i):
            qq = inst.wall_q.copy()
            qq[i, y, x] += h
            return oracle_loss(inst, init, ut, at, inst.force_field, qq)
        fd = fd4(f, 1e-5)
        ad = dq[i - 1, y, x]
        assert abs(fd - ad) <= 1e-6 * max(scale, abs(fd)), (k, i, q, fd, ad)
    # nothing outside the wall links
    mask = np.zeros_like(dq, dtype=bool)
    for k, i, _ in links:
        mask[i - 1, k // inst.nx, k % inst.nx] = True
    assert np.all(dq[~mask] == 0.0)


def test_mask_adjoint_drag_only(lbve):
    """A pure drag loss (no field term) through lbve_adjoint_step_ex."""
    import torch
    L = lbve
    inst, init, ut, at = make_case()
    sim = L.Simulation([inst], precision=0, init_fields=[init])
    sim.step(T)
    nbytes = L.lbve_adjoint_workspace_bytes(sim.h, 0, T)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    dF = torch.empty((2, 12, 14), dtype=torch.float64, device="cuda")
    L.lbve_adjoint_step_ex(sim.h, 0, init, None, (1.0, 0.0), T, ws.data_ptr(), nbytes,
                           dF.data_ptr(), None, inst.n_nodes)
    dF = dF.cpu().numpy()
    F0 = inst.force_field.copy()

    def drag(h, v):
        saved = inst.force_field
        inst.force_field = F0 + h * v
        try:
            s = oracle_sim(inst, init=init)
            s.set_mask(inst.solid, inst.wall_q)
            s.step(T)
            return s.totals()[12]
        finally:
            inst.force_field = saved
    v = np.random.default_rng(85).standard_normal(F0.shape) * (inst.solid == 0)
    fd = fd4(lambda h: drag(h, v), 1e-5)
    assert abs(fd - np.sum(dF * v)) <= 1e-6 * np.abs(dF).max() * np.abs(v).sum(), (fd, np.sum(dF * v))
