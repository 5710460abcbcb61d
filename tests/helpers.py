"""Test glue: build the oracle problem and the CUDA solver from one workload definition."""
import numpy as np

import oracle
from oracle import integrate, tables
from paper_2112_05946_gb300 import workloads


def oracle_problem(wl, **over):
    kw = dict(wl["solver"])
    kw.update(over)
    kw.pop("precision", None)
    prob = oracle.Problem(**kw)
    if "boundary" in wl:
        g = tables.gpc_tables(prob.N, prob.Q)
        dirichlet = {}
        for side, fn in wl["boundary"].items():
            vals = np.stack([np.asarray(fn(zq), dtype=np.float64) for zq in g["z"]], 0)   # [Q, S]
            dirichlet[side] = g["Pz"] @ vals                                               # [M, S]
        prob.dirichlet = dirichlet
    return prob


def solver(wl, **over):
    from paper_2112_05946_gb300 import frsg
    kw = dict(wl["solver"])
    kw.update(over)
    s = frsg.Solver(**kw)
    if "boundary" in wl:
        z = s.nodes()[-1]
        for side, fn in wl["boundary"].items():
            s.set_boundary_nodal(side, workloads.boundary_values(fn, z))
    return s


def oracle_initial(prob, wl):
    return integrate.project_initial(prob, wl["ic"])


def gpu_initial(s, wl):
    nodes = s.nodes()
    if len(nodes) == 2:
        vals = workloads.nodal_values(wl["ic"], nodes[0], nodes[1])
    else:
        vals = workloads.nodal_values(wl["ic"], nodes[0], nodes[2], nodes[1])
    s.set_initial_nodal(vals)


def rel_l2(a, b):
    den = np.sqrt(np.sum(b ** 2))
    return float(np.sqrt(np.sum((a - b) ** 2)) / (den if den > 0 else 1.0))
