"""Small problem builders shared by the tests (inputs only)."""
import numpy as np

from workloads import BC_DIRICHLET, BC_NATURAL, FaceBC, MeshDesc, Phase, random_state


def desc_small(n=(3, 3, 3), L=(1.0, 1.0, 1.0), dirichlet=True, n_fluid=1, n_solid=1,
               gravity=(0.0, 0.0, 0.0), pin=0, dt=0.01, rho_inf=0.0, eps=None, mu_L=0.3):
    phases = [Phase(rho=1.0 + 0.5 * f, mu=0.01 + 0.005 * f) for f in range(n_fluid)]
    phases += [Phase(rho=1.3 + 0.2 * s, mu=0.02, mu_L=mu_L * (1 + s), solid=True) for s in range(n_solid)]
    if dirichlet:
        faces = [FaceBC(BC_DIRICHLET, (0.0, 0.0, 0.0), 0) for _ in range(5)] + \
                [FaceBC(BC_DIRICHLET, (1.0, 0.0, 0.0), 1)]
    else:
        faces = [FaceBC(BC_NATURAL) for _ in range(6)]
        pin = -1
    h = min(L[0] / n[0], L[1] / n[1], L[2] / n[2])
    return MeshDesc(n[0], n[1], n[2], L[0], L[1], L[2], phases, gravity,
                    eps=1.5 * h if eps is None else eps, eta=0.2, dt=dt, rho_inf=rho_inf,
                    c_i=36.0, faces=faces, pin_node=pin)


def state_of(desc, seed, **kw):
    from oracle.fields import State
    x1, xn, xdn = random_state(desc, seed, **kw)
    return State(x1, xn, xdn)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
