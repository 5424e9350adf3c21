"""Dirichlet node sets of a problem description (oracle).

Test infrastructure only (see oracle/__init__.py).

Velocity: every node on a face with a prescribed velocity is Dirichlet; where such
faces meet the face with the highest priority gives the value (ties: lowest face
index in the order x-, x+, y-, y+, z-, z+).  Nodes inside the optional prescribed
box (bounds inclusive, coordinates i*hx etc.) take the box velocity, overriding
faces.  Pressure: the pin node (if any) has p = 0.  Phase indicators and B have no
Dirichlet condition (natural zero flux).
"""
from __future__ import annotations

import numpy as np

from workloads import BC_DIRICHLET, MeshDesc


def dirichlet(desc: MeshDesc):
    """Returns (vmask (nn,) bool, vD (3, nn) float64, pmask (nn,) bool)."""
    nx, ny, nz = desc.nx, desc.ny, desc.nz
    nn = desc.nn
    n = np.arange(nn)
    i = n % (nx + 1)
    j = (n // (nx + 1)) % (ny + 1)
    k = n // ((nx + 1) * (ny + 1))
    on_face = [i == 0, i == nx, j == 0, j == ny, k == 0, k == nz]
    vmask = np.zeros(nn, dtype=bool)
    vD = np.zeros((3, nn))
    best = np.full(nn, -(10 ** 9))
    for f in range(6):
        bc = desc.faces[f]
        if bc.kind != BC_DIRICHLET:
            continue
        sel = on_face[f] & (bc.priority > best)
        vmask |= on_face[f]
        for c in range(3):
            vD[c, sel] = bc.vel[c]
        best = np.where(sel, bc.priority, best)
    if desc.prescribed_box is not None:
        lo, hi, vel = desc.prescribed_box
        hx, hy, hz = desc.h
        x, y, z = i * hx, j * hy, k * hz
        inside = (x >= lo[0]) & (x <= hi[0]) & (y >= lo[1]) & (y <= hi[1]) & (z >= lo[2]) & (z <= hi[2])
        vmask |= inside
        for c in range(3):
            vD[c, inside] = vel[c]
    pmask = np.zeros(nn, dtype=bool)
    if desc.pin_node >= 0:
        pmask[desc.pin_node] = True
    return vmask, vD, pmask
