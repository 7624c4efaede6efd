"""Small helpers shared by the tests: turn a workload instance into oracle
parameters and run the oracle.  (Test infrastructure; no method arithmetic.)"""
from __future__ import annotations

from oracle import oracle as o


def oracle_params(inst, **override):
    d = dict(beta=inst.beta, Wi=inst.Wi, Re=inst.Re, Sc=inst.Sc, Ma=inst.Ma, Lc=inst.Lc,
             Lambda_s=inst.Lambda_s, Lambda_p=inst.Lambda_p, Fx=inst.Fx, Fy=inst.Fy,
             model=getattr(inst, "model", 0), gtilde=getattr(inst, "gtilde", 0),
             L2=getattr(inst, "L2", 0.0))
    d.update(override)
    return o.make_params(inst.nx, inst.ny, inst.periodic_y, open_x=getattr(inst, "open_x", False),
                         **d)


def oracle_sim(inst, init=None, **override):
    s = o.Sim(oracle_params(inst, **override), force=inst.force_field, init=init)
    if getattr(inst, "open_x", False) and getattr(inst, "inlet", None) is not None:
        s.set_inlet(inst.inlet)
    return s


def oracle_fields_after(job):
    """Process-pool worker: the oracle's fields after `steps` steps of `inst`
    from its default initial state.  job = (inst, steps)."""
    inst, steps = job
    o.build()
    s = oracle_sim(inst)
    s.step(steps)
    return s.fields()
