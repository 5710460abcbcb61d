"""Oracle on a window of a large 2D mesh.

TEST INFRASTRUCTURE ONLY.  One stage of the scheme changes an element from its own
coefficients and those of its four face neighbours (the interface fluxes of §3.3-3.5);
the limiter (§4.3) and the detector and filter (§4.1-4.2) act element by element.  After n
SSP-RK3 steps (3n stages) an element's state therefore depends only on the elements within
3n face-to-face moves of it.  Run on a window of the mesh, with any boundary condition on
the sides that cut through the mesh, the oracle gives the full-mesh result on the window's
elements that lie at least 3n elements from every cut side: exactly when the element size is
a binary fraction, else up to the rounding of the window's element size.  Sides of the window
that lie on the domain boundary keep the problem's own boundary conditions.  This lets the
plain oracle check states of meshes too large for it to step whole.
"""
import dataclasses

import numpy as np

from . import integrate


def window_problem(prob, ex0, ex1, ey0, ey1):
    """The problem restricted to elements ex0 <= ex < ex1, ey0 <= ey < ey1 of a 2D mesh: the
    same element size, orders and physics; the domain's own boundary conditions where the
    window touches the domain boundary, outflow on the cut sides."""
    if prob.dim != 2:
        raise ValueError("windows are defined for 2D meshes")
    if not (0 <= ex0 < ex1 <= prob.nx and 0 <= ey0 < ey1 <= prob.ny):
        raise ValueError("window outside the mesh")
    bc = (prob.bc[0] if ex0 == 0 else "outflow",
          prob.bc[1] if ex1 == prob.nx else "outflow",
          prob.bc[2] if ey0 == 0 else "outflow",
          prob.bc[3] if ey1 == prob.ny else "outflow")
    if "periodic" in bc:
        raise ValueError("a window of a periodic direction must span it (not supported)")
    return dataclasses.replace(prob, nx=ex1 - ex0, ny=ey1 - ey0,
                               x0=prob.x0 + ex0 * prob.dx, x1=prob.x0 + ex1 * prob.dx,
                               y0=prob.y0 + ey0 * prob.dy, y1=prob.y0 + ey1 * prob.dy, bc=bc)


def window_state(prob, u, ex0, ex1, ey0, ey1):
    """The window's elements of a full-mesh state u [E, Np, M, S] (element e = ey nx + ex)."""
    U = u.reshape((prob.ny, prob.nx) + u.shape[1:])
    return np.ascontiguousarray(U[ey0:ey1, ex0:ex1]).reshape((-1,) + u.shape[1:])


def exact_elements(prob, ex0, ex1, ey0, ey1, nsteps):
    """Full-mesh element indices and window element indices of the elements whose state
    after nsteps steps the window reproduces exactly (at least 3 nsteps from every cut)."""
    r = 3 * nsteps
    lox = ex0 if ex0 == 0 else ex0 + r
    hix = ex1 if ex1 == prob.nx else ex1 - r
    loy = ey0 if ey0 == 0 else ey0 + r
    hiy = ey1 if ey1 == prob.ny else ey1 - r
    if lox >= hix or loy >= hiy:
        raise ValueError("window too small for this many steps")
    ey, ex = np.meshgrid(np.arange(loy, hiy), np.arange(lox, hix), indexing="ij")
    full = (ey * prob.nx + ex).ravel()
    local = ((ey - ey0) * (ex1 - ex0) + (ex - ex0)).ravel()
    return full, local


def run_window(prob, u, box, dt, nsteps, record=None):
    """nsteps SSP-RK3 steps of the oracle on window box = (ex0, ex1, ey0, ey1) of the full-mesh
    state u.  Returns (full-mesh indices, states [n, Np, M, S]) of the exactly reproduced
    elements; `record` (a list) receives per stage the filter flags of those elements."""
    ex0, ex1, ey0, ey1 = box
    pw = window_problem(prob, ex0, ex1, ey0, ey1)
    uw = window_state(prob, u, ex0, ex1, ey0, ey1)
    rec = [] if record is not None else None
    out = integrate.run(pw, uw, dt, nsteps, record=rec)
    full, local = exact_elements(prob, ex0, ex1, ey0, ey1, nsteps)
    if record is not None:
        record.extend(np.asarray(f)[local] for f in rec)
    return full, out[local]
