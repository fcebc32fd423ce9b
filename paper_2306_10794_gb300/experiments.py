"""Post-processing of the paper's experiments (no time-step arithmetic).

* ``molins_ravg`` -- average reaction rate of the reactive disc in a channel
  flow, Eq. avgReactionRateMolins: (1 / (pi D)) (integral over the outlet of
  C u_x dy - C_in u_in H), in lattice units and in the paper's unit.
* ``mean_abs_error`` -- Eq. avgAbsError over the fluid cells (the paper
  prints a sum and calls it a mean; both are returned).
"""
from __future__ import annotations

import math

import numpy as np


def molins_ravg(u, c, geom):
    """u: (nz, ny, nx, 3) velocities, c: (nz, ny, nx) concentrations of a
    ``workloads.case_molins`` run.  Returns (R_lattice, R_paper_units); a
    positive rate means the disc consumes solute."""
    ux = u[0, :, -1, 0]
    cc = c[0, :, -1]
    outflow = float((cc * ux).sum())
    inflow = geom["c_in"] * geom["U"] * geom["H"]
    r = (inflow - outflow) / (math.pi * geom["d_obj"])
    return r, r * geom["to_paper"]


def mean_abs_error(c, exact, fluid):
    e = np.abs(c - exact)[fluid]
    return float(e.mean()), float(e.sum())
